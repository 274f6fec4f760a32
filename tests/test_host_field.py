"""CPU checks of the library's field code that need no GPU.

1. The divstep inversion and the Montgomery constants are host-and-device
   code: `tests/host/field_host.cu` builds that same source for the host.
   Its inverses are compared with Python's pow(x, -1, p), and its constants
   with their definitions (R = 2^256), for both BN254 fields.
2. The product difference a b - c d with one Montgomery reduction is
   device-only (PTX carry chains).  A word-level model of its steps checks
   the bounds that its carry chains rely on: the 512-bit difference, lifted
   by p 2^256 when negative, stays below p 2^256; no carry leaves word 15
   during the reduction rows; the reduced value is below 2p.  The device
   routine itself is compared bit for bit with the oracle on the GPU
   (ZK_FOP_MULSUB).

The moduli are the published BN254 primes (EIP-196), written out here."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
Q = 21888242871839275222246405745257275088696311157297823662689037894645226208583
R = 21888242871839275222246405745257275088548364400416034343698204186575808495617
MODULI = {"q": Q, "r": R}
W32 = (1 << 32) - 1


@pytest.fixture(scope="module")
def field_host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("host") / "field_host")
    src = os.path.join(ROOT, "tests", "host", "field_host.cu")
    inc = os.path.join(ROOT, "paper_2507_07031_b300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                    "arch=compute_103a,code=sm_103a", "-I", inc, "-o", exe, src],
                   check=True, capture_output=True, timeout=300)
    return exe


def _run(exe, args, stdin=""):
    r = subprocess.run([exe] + args, input=stdin, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return [int(x, 16) for x in r.stdout.split()]


def _edge(p):
    vals = [0, 1, 2, 3, p - 1, p - 2, p - 3, (p - 1) // 2, (p + 1) // 2]
    for k in (29, 30, 31, 32, 33, 60, 64, 128, 200, 252, 253):
        vals += [(1 << k) - 1, 1 << k, p - (1 << k)]
    return sorted({v % p for v in vals})


@pytest.mark.parametrize("f", ["q", "r"])
def test_montgomery_constants_match_definitions(field_host, f):
    p = MODULI[f]
    got = _run(field_host, ["consts", f])
    R256 = 1 << 256
    assert got[0] == p
    assert got[1] == R256 % p
    assert got[2] == R256 ** 2 % p
    assert got[3] == R256 ** 3 % p
    assert got[4] == (p - 1) // 2
    assert got[5] == (-pow(p, -1, 1 << 32)) % (1 << 32)
    assert got[6] == (-pow(p, -1, R256)) % R256
    assert got[6] & W32 == got[5]
    assert got[7] == pow(2, -128, p)


@pytest.mark.parametrize("f", ["q", "r"])
def test_divstep_inverse_matches_pow(field_host, f):
    p = MODULI[f]
    rng = random.Random(53 if f == "q" else 59)
    xs = _edge(p) + [rng.randrange(p) for _ in range(20000)]
    got = _run(field_host, ["inv", f], "".join("%064x\n" % x for x in xs))
    assert len(got) == len(xs)
    for x, y in zip(xs, got):
        assert y == (pow(x, -1, p) if x else 0), hex(x)


def _words(x, n):
    return [(x >> (32 * i)) & W32 for i in range(n)]


def _val(w):
    return sum(v << (32 * i) for i, v in enumerate(w))


def _mul_sub_mul_model(a, b, c, d, p):
    """The device routine's steps on 32-bit words, with its bound checks."""
    n0 = (-pow(p, -1, 1 << 32)) % (1 << 32)
    diff = a * b - c * d
    t = _words(diff % (1 << 512), 16) + [0]  # 512-bit two's complement
    if diff < 0:  # lift: + p 2^256, the carry out of word 15 dropped
        t = t[:8] + _words((_val(t[8:16]) + p) % (1 << 256), 8) + [0]
    assert _val(t[:16]) < p << 256
    carry = 0
    for i in range(8):  # reduction row i: t += m p 2^(32 i), carry word kept
        m = (t[i] * n0) & W32
        seg = _val(t[i:i + 9]) + m * p + (carry << 256)
        carry = seg >> 288
        t[i:i + 9] = _words(seg, 9)
        assert t[i] == 0
    assert carry == 0  # nothing leaves word 15
    r = _val(t[8:16])
    assert r < 2 * p
    return r - p if r >= p else r


@pytest.mark.parametrize("f", ["q", "r"])
def test_product_difference_model_bounds(f):
    p = MODULI[f]
    rinv = pow(1 << 256, -1, p)
    edge = _edge(p)
    rng = random.Random(61 if f == "q" else 67)
    cases = [(a, b, c, d) for a in edge[::3] for b in edge[::3] for c in edge[::5] for d in edge[::5]]
    cases += [tuple(rng.randrange(p) for _ in range(4)) for _ in range(5000)]
    for a, b, c, d in cases:
        assert _mul_sub_mul_model(a, b, c, d, p) == (a * b - c * d) * rinv % p
