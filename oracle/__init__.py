"""CPU oracle for the BN254 prover hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The arithmetic lives in ``zk_oracle.c`` (plain C,
schoolbook big integers, affine double-and-add, O(n^2) DFT, sequential fold);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Every function here is pinned by ``tests/test_oracle_*.py`` against values the
mathematics fixes (closed forms, group order, curve equation, transform
identities, brute force, Python's own integers); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zk_oracle.c")
_LIB = os.path.join(_HERE, "libzkoracle.so")

FQ, FR = 0, 1
INST_LIMBS = 44  # C_1..C_4 (4 x 8 limbs), E (8), mu (4)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_P = ctypes.POINTER(ctypes.c_uint64)
_PI = ctypes.POINTER(ctypes.c_int64)
_SZ = ctypes.c_size_t


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        sig = {
            "orc_set_threads": (None, [ctypes.c_int]),
            "orc_set_degree": (None, [ctypes.c_int]),
            "orc_get_degree": (ctypes.c_int, []),
            "orc_get_threads": (ctypes.c_int, []),
            "orc_has_openmp": (ctypes.c_int, []),
            "orc_fadd": (None, [ctypes.c_int, _P, _P, _P]),
            "orc_fsub": (None, [ctypes.c_int, _P, _P, _P]),
            "orc_fmul": (None, [ctypes.c_int, _P, _P, _P]),
            "orc_finv": (None, [ctypes.c_int, _P, _P]),
            "orc_fpow": (None, [ctypes.c_int, _P, _P, _P]),
            "orc_freduce512": (None, [ctypes.c_int, _P, _P]),
            "orc_on_curve": (ctypes.c_int, [_P]),
            "orc_g1_add": (None, [_P, _P, _P]),
            "orc_g1_dbl": (None, [_P, _P]),
            "orc_g1_neg": (None, [_P, _P]),
            "orc_g1_mul": (None, [_P, _P, _P]),
            "orc_g1_generator": (None, [_P]),
            "orc_count_off_curve": (_SZ, [_P, _SZ]),
            "orc_srs_gen": (None, [_P, _SZ, _P]),
            "orc_msm": (None, [_P, _P, _SZ, _P]),
            "orc_commit_coeffs_tau": (None, [_P, _SZ, _P, _P]),
            "orc_open": (None, [_P, _SZ, _P, _P, _P]),
            "orc_mul_quotient": (ctypes.c_int, [_P, _P, _SZ, _P]),
            "orc_commit_hiding": (None, [_P, _P, _SZ, _P, _P, _P]),
            "orc_open_batch": (None, [_P, ctypes.c_void_p, _SZ, _P, _P, _P, _P]),
            "orc_root_of_unity": (None, [_SZ, _P]),
            "orc_lagrange_at": (None, [_SZ, _P, _P]),
            "orc_commit_evals_tau": (None, [_P, _SZ, _P, _P]),
            "orc_dft": (None, [_P, _SZ, ctypes.c_int, _P]),
            "orc_dft_rows": (None, [_P, _SZ, ctypes.c_int, _PI, _SZ, _P]),
            "orc_poly_eval": (None, [_P, _SZ, _P, _P]),
            "orc_ntt_fingerprint": (ctypes.c_int, [_P, _SZ, _P, _P]),
            "orc_fold": (None, [_SZ, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P, _P,
                                _P, _P, _P, _P]),
            "orc_leaf_init": (None, [_SZ, _P, _P, _P, ctypes.c_int, _P, _P]),
            "orc_fold_tree": (None, [_SZ, _SZ, _P, _P, _P, _P, ctypes.c_int, _P, _P]),
            "orc_decide_relation": (_SZ, [_SZ, _P, _P, _P]),
            "orc_verify_fold": (ctypes.c_int, [_P, _P, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        set_threads(int(os.environ.get("ZK_ORACLE_THREADS", os.cpu_count() or 1)))
    return _lib


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def threads() -> int:
    return lib().orc_get_threads()


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_P)


def _u(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _none():
    return ctypes.cast(None, _P)


# ----------------------------------------------------------------------------
# Integer <-> limbs helpers (test convenience)
# ----------------------------------------------------------------------------

def to_int(a) -> int:
    a = np.asarray(a, dtype=np.uint64).reshape(-1)
    return sum(int(a[i]) << (64 * i) for i in range(a.shape[0]))


def from_int(x: int, limbs: int = 4) -> np.ndarray:
    return np.array([(x >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(limbs)], dtype=np.uint64)


def point_to_ints(p):
    p = np.asarray(p, dtype=np.uint64).reshape(8)
    return to_int(p[:4]), to_int(p[4:])


def point_from_ints(x: int, y: int) -> np.ndarray:
    return np.concatenate([from_int(x), from_int(y)])


# ----------------------------------------------------------------------------
# Field and group
# ----------------------------------------------------------------------------

def _f2(fn, f, a, b):
    out = np.zeros(4, dtype=np.uint64)
    fn(f, _p(_u(a)), _p(_u(b)), _p(out))
    return out


def fadd(f, a, b): return _f2(lib().orc_fadd, f, a, b)
def fsub(f, a, b): return _f2(lib().orc_fsub, f, a, b)
def fmul(f, a, b): return _f2(lib().orc_fmul, f, a, b)
def fpow(f, a, e): return _f2(lib().orc_fpow, f, a, e)


def finv(f, a):
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_finv(f, _p(_u(a)), _p(out))
    return out


def freduce512(f, a8):
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_freduce512(f, _p(_u(a8)), _p(out))
    return out


def on_curve(p) -> bool:
    return bool(lib().orc_on_curve(_p(_u(p))))


def count_off_curve(pts) -> int:
    pts = _u(pts).reshape(-1, 8)
    return int(lib().orc_count_off_curve(_p(pts), pts.shape[0]))


def g1_generator():
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_g1_generator(_p(out))
    return out


def g1_add(a, b):
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_g1_add(_p(_u(a)), _p(_u(b)), _p(out))
    return out


def g1_dbl(a):
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_g1_dbl(_p(_u(a)), _p(out))
    return out


def g1_neg(a):
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_g1_neg(_p(_u(a)), _p(out))
    return out


def g1_mul(a, k):
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_g1_mul(_p(_u(a)), _p(_u(k)), _p(out))
    return out


# ----------------------------------------------------------------------------
# SRS, commitments, transforms
# ----------------------------------------------------------------------------

def srs_gen(tau, n: int) -> np.ndarray:
    out = np.zeros((n, 8), dtype=np.uint64)
    lib().orc_srs_gen(_p(_u(tau)), n, _p(out))
    return out


def msm(points, scalars) -> np.ndarray:
    points = _u(points).reshape(-1, 8)
    scalars = _u(scalars).reshape(-1, 4)
    assert points.shape[0] >= scalars.shape[0]
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_msm(_p(points), _p(scalars), scalars.shape[0], _p(out))
    return out


def commit_coeffs_tau(coeffs, tau) -> np.ndarray:
    c = _u(coeffs).reshape(-1, 4)
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_commit_coeffs_tau(_p(c), c.shape[0], _p(_u(tau)), _p(out))
    return out


def open_poly(coeffs, x):
    """KZG opening by synthetic division: (y = f(x), quotient (f - y)/(X - x))."""
    c = _u(coeffs).reshape(-1, 4)
    n = c.shape[0]
    y = np.zeros(4, dtype=np.uint64)
    q = np.zeros((max(n - 1, 1), 4), dtype=np.uint64)
    lib().orc_open(_p(c), n, _p(_u(x)), _p(y), _p(q))
    return y, q[: max(n - 1, 0)]


def open_batch(polys, x, gamma):
    """Batch opening at x: ([f_i(x)], quotient of sum_i gamma^i f_i)."""
    polys = [_u(f).reshape(-1, 4) for f in polys]
    lens = (ctypes.c_size_t * len(polys))(*[f.shape[0] for f in polys])
    flat = np.ascontiguousarray(np.concatenate(polys)) if polys else np.zeros((1, 4), np.uint64)
    nmax = max(f.shape[0] for f in polys)
    ys = np.zeros((len(polys), 4), dtype=np.uint64)
    h = np.zeros((max(nmax - 1, 1), 4), dtype=np.uint64)
    lib().orc_open_batch(_p(flat), lens, len(polys), _p(_u(x)), _p(_u(gamma)), _p(ys), _p(h))
    return ys, h[: max(nmax - 1, 0)]


def mul_quotient(a, b):
    """t = (A B - L) / (X^n - 1) for evaluation vectors a, b over H (L
    interpolates a o b): (t with n - 1 coefficients, exact division flag)."""
    a = _u(a).reshape(-1, 4)
    b = _u(b).reshape(-1, 4)
    n = a.shape[0]
    t = np.zeros((max(n - 1, 1), 4), dtype=np.uint64)
    bad = lib().orc_mul_quotient(_p(a), _p(b), n, _p(t))
    return t[: max(n - 1, 0)], bad == 0


def commit_hiding(points, coeffs, H, s):
    """[f(tau)]_1 + s H: MSM over `points` plus s H."""
    points = _u(points).reshape(-1, 8)
    c = _u(coeffs).reshape(-1, 4)
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_commit_hiding(_p(points), _p(c), c.shape[0], _p(_u(H)), _p(_u(s)), _p(out))
    return out


def commit_evals_tau(v, tau) -> np.ndarray:
    v = _u(v).reshape(-1, 4)
    out = np.zeros(8, dtype=np.uint64)
    lib().orc_commit_evals_tau(_p(v), v.shape[0], _p(_u(tau)), _p(out))
    return out


def lagrange_at(n: int, tau) -> np.ndarray:
    out = np.zeros((n, 4), dtype=np.uint64)
    lib().orc_lagrange_at(n, _p(_u(tau)), _p(out))
    return out


def root_of_unity(n: int) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_root_of_unity(n, _p(out))
    return out


def ntt(c) -> np.ndarray:
    """NTT(c)_k = sum_j c_j omega^{jk} (O(n^2) DFT)."""
    c = _u(c).reshape(-1, 4)
    out = np.zeros_like(c)
    lib().orc_dft(_p(c), c.shape[0], 0, _p(out))
    return out


def intt(v) -> np.ndarray:
    """INTT(v)_j = n^{-1} sum_k v_k omega^{-jk} (O(n^2) DFT)."""
    v = _u(v).reshape(-1, 4)
    out = np.zeros_like(v)
    lib().orc_dft(_p(v), v.shape[0], 1, _p(out))
    return out


def dft_rows(x, rows, inverse: bool) -> np.ndarray:
    x = _u(x).reshape(-1, 4)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((rows.shape[0], 4), dtype=np.uint64)
    lib().orc_dft_rows(_p(x), x.shape[0], int(inverse), rows.ctypes.data_as(_PI), rows.shape[0], _p(out))
    return out


def poly_eval(v, z) -> np.ndarray:
    """sum_k v_k z^k (Horner)."""
    v = _u(v).reshape(-1, 4)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_poly_eval(_p(v), v.shape[0], _p(_u(z)), _p(out))
    return out


def ntt_fingerprint(c, z) -> np.ndarray:
    """sum_k z^k NTT(c)_k, computed as sum_j c_j (z^n - 1)/(z omega^j - 1)
    in O(n) (no transform).  Raises if z omega^j = 1 for some j."""
    c = _u(c).reshape(-1, 4)
    out = np.zeros(4, dtype=np.uint64)
    ok = lib().orc_ntt_fingerprint(_p(c), c.shape[0], _p(_u(z)), _p(out))
    if not ok:
        raise ValueError("z omega^j = 1: the fingerprint identity does not apply")
    return out


# ----------------------------------------------------------------------------
# Fold (generalised Mira, Sec. 4.2)
# ----------------------------------------------------------------------------

COMMIT_NONE, COMMIT_MSM, COMMIT_TAU = 0, 1, 2


class Acc:
    """Accumulator: m (4, n, 4), e (n, 4), inst (44,) = C_1..C_4, E, mu."""

    def __init__(self, m, e, inst):
        self.m = np.ascontiguousarray(m, dtype=np.uint64).reshape(4, -1, 4)
        self.e = np.ascontiguousarray(e, dtype=np.uint64).reshape(-1, 4)
        self.inst = np.ascontiguousarray(inst, dtype=np.uint64).reshape(INST_LIMBS)

    @property
    def n(self):
        return self.e.shape[0]

    @property
    def C(self):
        return self.inst[:32].reshape(4, 8)

    @property
    def E(self):
        return self.inst[32:40]

    @property
    def mu(self):
        return self.inst[40:44]

    def copy(self):
        return Acc(self.m.copy(), self.e.copy(), self.inst.copy())


def _commit_args(mode, srs, tau):
    s = _p(_u(srs).reshape(-1, 8)) if srs is not None else _none()
    t = _p(_u(tau)) if tau is not None else _none()
    return mode, s, t


def leaf_init(m1, m2, m4, mode=COMMIT_TAU, srs=None, tau=None) -> Acc:
    """Degree 2: inputs m1, m2, m4 (m3 = m1 o m2); degree 3: inputs m1, m2, m3
    in the three positional slots (m4 = m1 o m2 o m3)."""
    n = np.asarray(m1).reshape(-1, 4).shape[0]
    m = np.zeros((4, n, 4), dtype=np.uint64)
    third = 2 if get_degree() == 3 else 3
    m[0], m[1], m[third] = (np.asarray(x, dtype=np.uint64).reshape(n, 4) for x in (m1, m2, m4))
    e = np.zeros((n, 4), dtype=np.uint64)
    inst = np.zeros(INST_LIMBS, dtype=np.uint64)
    md, s, t = _commit_args(mode, srs, tau)
    lib().orc_leaf_init(n, _p(m), _p(e), _p(inst), md, s, t)
    return Acc(m, e, inst)


def set_degree(d: int) -> None:
    """Degree of the folded relation: 2 (m1 o m2 - mu m3 = e) or 3
    (m1 o m2 o m3 - mu^2 m4 = e)."""
    lib().orc_set_degree(int(d))


def get_degree() -> int:
    return int(lib().orc_get_degree())


def fold(L: Acc, R: Acc, gamma, mode=COMMIT_TAU, srs=None, tau=None):
    """Returns (acc'', E) with E = E_1 (degree 2) or (E_1, E_2) (degree 3)."""
    n = L.n
    Om = np.zeros_like(L.m)
    Oe = np.zeros_like(L.e)
    Oi = np.zeros(INST_LIMBS, dtype=np.uint64)
    E1 = np.zeros(8 * (get_degree() - 1), dtype=np.uint64)
    md, s, t = _commit_args(mode, srs, tau)
    lib().orc_fold(n, _p(L.m), _p(L.e), _p(L.inst), _p(R.m), _p(R.e), _p(R.inst), _p(_u(gamma)),
                   md, s, t, _p(Om), _p(Oe), _p(Oi), _p(E1))
    return Acc(Om, Oe, Oi), E1


def fold_tree(leaves, gammas, mode=COMMIT_TAU, srs=None, tau=None) -> Acc:
    """Sequential binary fold tree; gammas level-major (count - 1, 4)."""
    count = len(leaves)
    n = leaves[0].n
    m = np.ascontiguousarray(np.stack([a.m for a in leaves]))
    e = np.ascontiguousarray(np.stack([a.e for a in leaves]))
    inst = np.ascontiguousarray(np.stack([a.inst for a in leaves]))
    g = _u(gammas).reshape(-1, 4)
    assert g.shape[0] == count - 1
    md, s, t = _commit_args(mode, srs, tau)
    lib().orc_fold_tree(count, n, _p(m), _p(e), _p(inst), _p(g), md, s, t)
    return Acc(m[0], e[0], inst[0])


def fold_tree_stacked(m, e, inst, gammas, mode=COMMIT_NONE, srs=None, tau=None) -> None:
    """The sequential fold tree of fold_tree() on accumulators already stacked
    as m (count, 4, n, 4), e (count, n, 4), inst (count, 44), in place (the
    root ends in slot 0).  For trees too large to hold twice in host memory."""
    count, n = m.shape[0], m.shape[2]
    for a in (m, e, inst):
        assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    assert e.shape == (count, n, 4) and inst.shape == (count, INST_LIMBS)
    g = _u(gammas).reshape(-1, 4)
    assert g.shape[0] == count - 1
    md, s, t = _commit_args(mode, srs, tau)
    lib().orc_fold_tree(count, n, _p(m), _p(e), _p(inst), _p(g), md, s, t)


def leaf_init_into(m, e, inst, mode=COMMIT_NONE, srs=None, tau=None) -> None:
    """leaf_init() on caller-owned arrays m (4, n, 4), e (n, 4), inst (44,)
    (for example, one slot of the stacked arrays of fold_tree_stacked)."""
    n = m.shape[1]
    for a in (m, e, inst):
        assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    md, s, t = _commit_args(mode, srs, tau)
    lib().orc_leaf_init(n, _p(m), _p(e), _p(inst), md, s, t)


def decide_relation(acc: Acc) -> int:
    """Number of positions where m1 o m2 - mu m3 != e (0 = decider accepts)."""
    return int(lib().orc_decide_relation(acc.n, _p(acc.m), _p(acc.e), _p(_u(acc.mu))))


def verify_fold(L: Acc, R: Acc, O: Acc, E1, gamma) -> bool:
    return bool(lib().orc_verify_fold(_p(L.inst), _p(R.inst), _p(O.inst), _p(_u(E1)), _p(_u(gamma))))
