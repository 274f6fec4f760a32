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
3. The product by a constant with a precomputed quotient (NTT butterflies,
   fold RLC, products by a window-table point): a word-level model of its
   truncated quotient checks the error bound (at most two units), the
   carry windows and exactness for every first operand below 2^256; the
   closed form of the quotient from the Montgomery form is checked against
   floor division.  The device routine is compared with the oracle on the
   GPU (ZK_FOP_MULC).
4. The scaled bucket start of the MSM accumulation (lambda = 2^-128) is
   checked to represent the same affine point, with a model of the
   four-row reduction that forms y 2^-128.

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


def _shoup_model(a, w, p):
    """fe_mul_shoup's steps on 32-bit words, with the bounds its carry chains
    rely on.  The quotient takes only the partial products of a wq in columns
    >= 7 (lo(a_i wq_j) for i + j >= 7, hi for i + j >= 6), row by row into
    the window of words 7 .. i + 8; then a w + q (2^256 - p) mod 2^256 and
    two conditional subtractions (2p, then p)."""
    wq = (w << 256) // p
    A, WQ = _words(a, 8), _words(wq, 8)
    acc = 0
    for i in range(8):
        for j in range(8):
            prod = A[i] * WQ[j]
            if i + j >= 7:
                acc += (prod & W32) << (32 * (i + j))
            if i + j >= 6:
                acc += (prod >> 32) << (32 * (i + j + 1))
        assert acc % (1 << 224) == 0  # nothing below word 7
        assert acc >> 224 < 1 << (32 * (i + 2))  # the window t[7 .. i + 8] holds it
    q = acc >> 256
    Q = a * w // p
    assert 0 <= Q - q <= 2  # the dropped columns sum to below 2^228
    low = lambda x, y: sum(((X * Y) & W32) << (32 * (i + j)) for i, X in enumerate(_words(x, 8))
                           for j, Y in enumerate(_words(y, 8)) if i + j <= 7) + \
        sum(((X * Y) >> 32) << (32 * (i + j + 1)) for i, X in enumerate(_words(x, 8))
            for j, Y in enumerate(_words(y, 8)) if i + j <= 6)
    r = (low(q, (1 << 256) - p) + low(w, a)) % (1 << 256)  # lower triangles only
    assert r == a * w - q * p < 3 * p < 1 << 256
    if r >= 2 * p:
        r -= 2 * p
    if r >= p:
        r -= p
    return r


@pytest.mark.parametrize("f", ["q", "r"])
def test_precomputed_quotient_product_model(f):
    """The product by a constant with a precomputed quotient (the NTT's
    butterflies, the fold's RLC, the MSM's products by a table point): exact
    for every first operand below 2^256, the range the lazy butterflies feed
    it (values up to 4p), including its top 2^256 - 1."""
    p = MODULI[f]
    rng = random.Random(71 if f == "q" else 73)
    edge = _edge(p)
    firsts = edge + [(1 << 256) - 1, 4 * p - 1, 3 * p, 2 * p - 1] + [rng.randrange(1 << 256) for _ in range(300)]
    consts = edge + [rng.randrange(p) for _ in range(60)]
    for a in firsts[::2]:
        for w in consts[::3]:
            assert _shoup_model(a, w, p) == a * w % p, (hex(a), hex(w))
    for _ in range(3000):
        a, w = rng.randrange(1 << 256), rng.randrange(p)
        assert _shoup_model(a, w, p) == a * w % p


@pytest.mark.parametrize("f", ["q", "r"])
def test_quotient_from_montgomery_form(f):
    """floor(w 2^256 / p) = -(w R mod p) p^-1 mod 2^256 (R = 2^256): the
    closed form the device takes the quotient from, one lower-triangle
    product of w's Montgomery form with the constant -p^-1 mod 2^256."""
    p = MODULI[f]
    R = 1 << 256
    ninv = (-pow(p, -1, R)) % R
    rng = random.Random(79 if f == "q" else 83)
    for w in _edge(p) + [rng.randrange(p) for _ in range(5000)]:
        assert (w * R % p) * ninv % R == (w << 256) // p, hex(w)


def _mul_2m128_model(a, p):
    """fe_mul_2m128's steps: four word-level Montgomery reduction rows
    t += m p 2^(32 i), m = t_i n0 mod 2^32, then words 4 .. 11 and one
    conditional subtraction."""
    n0 = (-pow(p, -1, 1 << 32)) % (1 << 32)
    t = a
    for i in range(4):
        m = ((t >> (32 * i)) & W32) * n0 & W32
        t += (m * p) << (32 * i)
        assert (t >> (32 * i)) & W32 == 0
        assert t < 1 << (32 * (i + 9))  # the row's window t[i .. i + 8]
    r = t >> 128
    assert r < 2 * p
    return r - p if r >= p else r


def test_scaled_bucket_start():
    """A bucket's first table point enters the accumulator as the XYZZ point
    with Montgomery words (x, y 2^-128, 1, 2^-128 mod q), x and y the entry's
    canonical coordinates: the representation lambda = 2^-128 of the same
    affine point.  Checked on the field values the words stand for (word R^-1),
    with y 2^-128 from the four-row reduction model, on points of the curve."""
    q = MODULI["q"]
    R = 1 << 256
    rinv = pow(R, -1, q)
    rinvh = pow(2, -128, q)
    rng = random.Random(89)
    pts = []
    x, y = 1, 2  # the generator of y^2 = x^3 + 3
    for _ in range(40):
        pts.append((x, y))
        k = rng.randrange(1, 1 << 64)
        # k P by double-and-add in affine coordinates (Python integers)
        acc = None
        base = (x, y)
        while k:
            if k & 1:
                acc = base if acc is None else _affine_add(acc, base, q)
            base = _affine_add(base, base, q)
            k >>= 1
        x, y = acc
    for x, y in pts:
        assert (y * y - x ** 3 - 3) % q == 0
        words = (x, _mul_2m128_model(y, q), 1, rinvh)
        X, Y, ZZ, ZZZ = (v * rinv % q for v in words)
        assert ZZ ** 3 % q == ZZZ ** 2 % q
        assert X * pow(ZZ, -1, q) % q == x
        assert Y * pow(ZZZ, -1, q) % q == y
    for a in _edge(q) + [R - 1]:
        assert _mul_2m128_model(a, q) == a * rinvh % q


def _affine_add(P, Q, p):
    (x1, y1), (x2, y2) = P, Q
    if P == Q:
        lam = 3 * x1 * x1 * pow(2 * y1, -1, p) % p
    else:
        lam = (y2 - y1) * pow(x2 - x1, -1, p) % p
    x3 = (lam * lam - x1 - x2) % p
    return x3, (lam * (x1 - x3) - y1) % p
