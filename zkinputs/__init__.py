"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the method: it only draws random numbers
and encodes them as field elements.  Both sides (``oracle/`` and the CUDA
library) read the arrays produced here and nothing else.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  It is counter based, so the
k-th output of a stream is ``mix(seed + (k + 1) * 0x9E3779B97F4A7C15)`` and a
whole stream can be evaluated vectorised.

Field elements are (n, 4) arrays of uint64 limbs, little endian, canonical
(value < modulus).  Group elements are (n, 8) uint64 arrays: x limbs then y
limbs, canonical affine; the point at infinity is eight zero limbs.

Streams (seed assignment):
  * tau: seed 0, the first accepted non-zero element of F_r;
  * scalars / vector entries of a workload: the seed named by the workload;
  * fold challenges gamma for tree level l (1-based), fold j: seed 1000 + l,
    j-th accepted draw.
"""
from __future__ import annotations

import numpy as np

# BN254 scalar field modulus r (the group order "p" of the paper's Sec. 2) and
# base field modulus q, as 64-bit little-endian limbs.  Used here only to
# reject out-of-range draws and to encode negative fixed-point values as r - x.
R_MOD = 21888242871839275222246405745257275088548364400416034343698204186575808495617
Q_MOD = 21888242871839275222246405745257275088696311157297823662689037894645226208583
R_LIMBS = np.array([(R_MOD >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)], dtype=np.uint64)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK62 = np.uint64((1 << 62) - 1)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _less_than_r(l: np.ndarray) -> np.ndarray:
    """Row-wise ``value < r`` for (m, 4) little-endian limb arrays."""
    r0, r1, r2, r3 = (R_LIMBS[i] for i in range(4))
    return (l[:, 3] < r3) | ((l[:, 3] == r3) & (
        (l[:, 2] < r2) | ((l[:, 2] == r2) & (
            (l[:, 1] < r1) | ((l[:, 1] == r1) & (l[:, 0] < r0))))))


def fr_uniform(seed: int, n: int, nonzero: bool = False) -> np.ndarray:
    """n elements uniform in F_r by rejection: 4 outputs per candidate, top limb
    masked to 62 bits (254-bit candidates), candidates >= r rejected."""
    out = np.empty((n, 4), dtype=np.uint64)
    got = 0
    pos = 0
    while got < n:
        m = max(64, int((n - got) * 1.4) + 16)
        raw = splitmix64(seed, pos, 4 * m).reshape(m, 4)
        pos += 4 * m
        raw[:, 3] &= _MASK62
        ok = _less_than_r(raw)
        if nonzero:
            ok &= raw.any(axis=1)
        acc = raw[ok]
        take = min(n - got, acc.shape[0])
        out[got:got + take] = acc[:take]
        got += take
    return out


def tau(seed: int = 0) -> np.ndarray:
    """The SRS trapdoor: first accepted non-zero draw of stream ``seed``."""
    return fr_uniform(seed, 1, nonzero=True)[0]


def encode_signed(vals: np.ndarray, shift: int = 16) -> np.ndarray:
    """Fixed-point encoding of small signed integers: x * 2^shift mod r, with a
    negative x mapped to r - |x| * 2^shift (requires |x| * 2^shift < 2^62)."""
    v = np.asarray(vals, dtype=np.int64)
    mag = (np.abs(v).astype(np.uint64)) << np.uint64(shift)
    assert v.size == 0 or int(mag.max()) < (1 << 62)
    out = np.zeros((v.shape[0], 4), dtype=np.uint64)
    neg = v < 0
    pos = ~neg & (v != 0)
    out[pos, 0] = mag[pos]
    # r - m for m < 2^62 < r0 (= 0x43e1f593f0000001): limb 0 never borrows.
    out[neg, 0] = R_LIMBS[0] - mag[neg]
    out[neg, 1] = R_LIMBS[1]
    out[neg, 2] = R_LIMBS[2]
    out[neg, 3] = R_LIMBS[3]
    return out


def int8_uniform(seed: int, n: int) -> np.ndarray:
    """int8 values uniform in [-128, 127], one SplitMix64 output each."""
    return (splitmix64(seed, 0, n) & np.uint64(0xFF)).astype(np.int64) - 128


def int8_gauss(seed: int, n: int, sigma: float = 32.0) -> np.ndarray:
    """int8 values clamp(round(N(0, sigma^2))) by Box-Muller on SplitMix64."""
    raw = splitmix64(seed, 0, 2 * n).reshape(n, 2)
    u1 = ((raw[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (raw[:, 1] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2) * sigma
    return np.clip(np.rint(z), -128, 127).astype(np.int64)


def zkml_scalars(seed: int, n: int, dist: str = "uniform") -> np.ndarray:
    """Quantised ML values mapped into F_r: q * 2^16 with q an int8."""
    q = int8_uniform(seed, n) if dist == "uniform" else int8_gauss(seed, n)
    return encode_signed(q, 16)


def gammas(level: int, count: int) -> np.ndarray:
    """Fold challenges of one tree level (1-based): stream 1000 + level."""
    return fr_uniform(1000 + level, count)


def shuffle(seed: int, n: int) -> np.ndarray:
    """A Fisher-Yates permutation of range(n) driven by SplitMix64."""
    perm = np.arange(n)
    raw = splitmix64(seed, 0, n)
    for i in range(n - 1, 0, -1):
        j = int(raw[n - 1 - i] % np.uint64(i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def uniform01(seed: int, n: int) -> np.ndarray:
    """Doubles in (0, 1] from the top 53 bits of SplitMix64 outputs."""
    return ((splitmix64(seed, 0, n) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


# ---------------------------------------------------------------------------
# Workload shapes.
# ---------------------------------------------------------------------------

# Batched commitments of one synthetic CNN inference: 256 polynomial sizes
# (log2 -> count) totalling exactly 2^24 coefficients, standing in for the
# per-layer tensors of a 20-layer ResNet-like conv/matmul stack.
CNN_SIZE_HIST = {18: 19, 17: 40, 16: 59, 15: 60, 14: 29, 13: 21, 12: 12, 11: 8, 10: 8}


def cnn_poly_sizes(seed: int = 8) -> np.ndarray:
    sizes = []
    for lg, cnt in sorted(CNN_SIZE_HIST.items()):
        sizes += [1 << lg] * cnt
    sizes = np.array(sizes, dtype=np.int64)
    assert sizes.shape[0] == 256 and int(sizes.sum()) == 1 << 24
    return sizes[shuffle(seed, sizes.shape[0])]


def transformer_job_sizes() -> list:
    """log2 sizes of the basic-block jobs of one 12-layer, width-768,
    FFN-3072, sequence-128 transformer layer, padded to powers of two."""
    per_layer = ([17] * 5 + [19] + [18] * 2 + [19] * 2 + [13] + [14] + [12]
                 + [20, 21, 22, 22])
    return per_layer


def poisson_arrivals(seed: int, count: int, rate_hz: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    u = uniform01(seed, count)
    return np.cumsum(-np.log(u) / rate_hz)


def as_bytes_fr(a: np.ndarray) -> bytes:
    return np.ascontiguousarray(a, dtype=np.uint64).tobytes()


def fr_to_int(a) -> int:
    a = np.asarray(a, dtype=np.uint64)
    return sum(int(a[i]) << (64 * i) for i in range(4))


def int_to_fr(x: int) -> np.ndarray:
    return np.array([(x >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)], dtype=np.uint64)
