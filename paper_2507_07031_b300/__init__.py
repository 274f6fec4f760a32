"""Python binding of libzkb300 (the C ABI in include/zk_b300.h).

Argument marshalling only: every function below forwards to the C entry
point of the same name, passing raw device/host pointers and the current
torch CUDA stream.  Field elements travel as (n, 4) int64 tensors or uint64
numpy arrays (little-endian limbs, canonical); G1 points as (n, 8).  PyTorch
provides device memory and streams; all arithmetic runs in the library's
CUDA kernels.  Importing this module fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzkb300.so")

ZK_OK, ZK_EINVAL, ZK_ESRS, ZK_ENOMEM, ZK_ECUDA, ZK_ETIMEOUT, ZK_EBUSY = range(7)
ZK_EVALS = 1
ZK_LAGRANGE = 2
ZK_ROUTE_INTT, ZK_ROUTE_LAGRANGE = 0, 1


class ZkError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (code %d)" % (where, zk_strerror(code), code))


class ZkAcc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_size_t), ("m", ctypes.c_void_p * 4), ("e", ctypes.c_void_p),
                ("x", ctypes.c_void_p)]


class ZkJob(ctypes.Structure):
    _fields_ = [("n", ctypes.c_size_t), ("w", ctypes.c_void_p * 3), ("leaf", ctypes.c_void_p),
                ("acc_in", ctypes.c_void_p), ("acc_out", ctypes.c_void_p), ("gamma", ctypes.c_void_p)]


class ZkTicketInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("error", ctypes.c_int), ("lane", ctypes.c_int),
                ("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double)]


class ZkServerInfo(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_ulonglong), ("queued", ctypes.c_size_t),
                ("reserved_bytes", ctypes.c_size_t), ("peak_reserved_bytes", ctypes.c_size_t),
                ("busy_lanes", ctypes.c_int), ("cancelled", ctypes.c_ulonglong)]


ZK_JOB_QUEUED, ZK_JOB_RUNNING, ZK_JOB_DONE, ZK_JOB_FAILED, ZK_JOB_CANCELLED = range(5)


_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_SZP = ctypes.POINTER(ctypes.c_size_t)


def _load(path: str = LIB_PATH):
    """Loads the library at `path` (the in-tree build by default) and declares
    every entry point's argument types."""
    if not os.path.exists(path):
        raise ImportError("%s not built: run `python paper_2507_07031_b300/build.py` "
                          "(or __graft_entry__.build())" % os.path.basename(path))
    L = ctypes.CDLL(path)
    sig = {
        "zk_init": [ctypes.POINTER(_VP), ctypes.c_int, _SZ],
        "zk_destroy": [_VP],
        "zk_lane_create": [_VP, ctypes.POINTER(_VP)],
        "zk_srs_load": [_VP, _VP, _SZ],
        "zk_srs_generate": [_VP, _VP, _SZ],
        "zk_srs_size": [_VP, _SZP],
        "zk_srs_export": [_VP, _VP, _SZ, _SZ, _VP],
        "zk_commit": [_VP, _VP, _SZ, _VP, _VP],
        "zk_commit_noalloc": [_VP, _VP, _SZ, _VP, _VP],
        "zk_commit_batch": [_VP, _VP, _VP, _SZ, ctypes.c_uint, _VP, _VP],
        "zk_ntt": [_VP, _VP, _SZ, _VP],
        "zk_intt": [_VP, _VP, _SZ, _VP],
        "zk_ntt_batch": [_VP, _VP, _VP, _SZ, ctypes.c_int, _VP],
        "zk_leaf_init": [_VP, _VP, _SZ, _VP],
        "zk_fold": [_VP, _VP, _VP, _VP, _VP, _VP, _VP],
        "zk_fold_tree": [_VP, _VP, _SZ, _VP, _VP, _VP],
        "zk_fold_tree_levels": [_VP, _VP, _SZ, _VP, _SZ, _VP],
        "zk_timing_enable": [_VP, ctypes.c_int],
        "zk_set_commit_route": [_VP, ctypes.c_int],
        "zk_tune_set": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "zk_plan_commit_batch": [_VP, _VP, _VP, _SZ, ctypes.c_uint, _VP, ctypes.POINTER(_VP)],
        "zk_plan_fold_tree": [_VP, _VP, _SZ, _VP, _VP, ctypes.POINTER(_VP)],
        "zk_plan_launch": [_VP, _VP],
        "zk_plan_nodes": [_VP, _SZP],
        "zk_plan_destroy": [_VP],
        "zk_server_create": [_VP, ctypes.c_int, _SZ, ctypes.POINTER(_VP)],
        "zk_submit": [_VP, _VP, ctypes.POINTER(ctypes.c_uint64)],
        "zk_poll": [_VP, ctypes.c_uint64, _VP],
        "zk_wait": [_VP, ctypes.c_uint64, ctypes.c_int, _VP],
        "zk_server_stats": [_VP, _VP],
        "zk_server_destroy": [_VP],
        "zk_cancel": [_VP, ctypes.c_uint64],
        "zk_check_status": [_VP, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int)],
        "zk_tune_get": [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "zk_tune_measure": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_double)],
        "zk_timing_read": [_VP, _VP, _VP],
        "zk_field_op": [ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _SZ, _VP],
        "zk_open": [_VP, _VP, _SZ, _VP, _VP, _VP, _VP, _VP],
        "zk_open_batch": [_VP, _VP, _VP, _SZ, _VP, _VP, _VP, _VP, _VP],
        "zk_mul_quotient": [_VP, _VP, _VP, _SZ, _VP, _VP, _VP],
        "zk_set_hiding_base": [_VP, _VP],
        "zk_set_fold_degree": [_VP, ctypes.c_int],
        "zk_commit_hiding": [_VP, _VP, _SZ, _VP, _VP, _VP],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.zk_strerror.argtypes = [ctypes.c_int]
    L.zk_strerror.restype = ctypes.c_char_p
    L.zk_kernel_launches.argtypes = []
    L.zk_kernel_launches.restype = ctypes.c_ulonglong
    L.zk_probe_rates.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    L.zk_probe_rates.restype = ctypes.c_int
    L.zk_probe_pipes.argtypes = [ctypes.c_int, _VP]
    L.zk_probe_pipes.restype = ctypes.c_int
    return L


lib = _load()

EXPORTED = ["zk_init", "zk_destroy", "zk_lane_create", "zk_srs_load", "zk_srs_generate",
            "zk_srs_size", "zk_srs_export", "zk_commit", "zk_commit_noalloc", "zk_commit_batch", "zk_ntt", "zk_intt",
            "zk_ntt_batch", "zk_leaf_init", "zk_fold", "zk_fold_tree", "zk_fold_tree_levels", "zk_strerror",
            "zk_kernel_launches", "zk_probe_rates", "zk_probe_pipes", "zk_timing_enable", "zk_timing_read",
            "zk_tune_set", "zk_tune_get", "zk_tune_measure", "zk_plan_commit_batch",
            "zk_plan_fold_tree", "zk_plan_launch", "zk_plan_nodes", "zk_plan_destroy",
            "zk_server_create", "zk_submit", "zk_poll", "zk_wait", "zk_server_stats", "zk_cancel", "zk_check_status",
            "zk_server_destroy", "zk_set_commit_route", "zk_field_op", "zk_open", "zk_open_batch",
            "zk_mul_quotient", "zk_set_hiding_base", "zk_commit_hiding", "zk_set_fold_degree"]

ZK_TUNE_MSM_WINDOW, ZK_TUNE_NTT_RADIX = 0, 1
ZK_TUNE_MSM_CHUNK, ZK_TUNE_MSM_TAIL, ZK_TUNE_MSM_SEG, ZK_TUNE_MSM_SEGBIG = 2, 3, 4, 5
ZK_FIELD_Q, ZK_FIELD_R = 0, 1
ZK_FOP_MUL, ZK_FOP_SQR, ZK_FOP_INV, ZK_FOP_ADD, ZK_FOP_SUB, ZK_FOP_MULSUB, ZK_FOP_MULC = range(7)

PHASES = ["msm_sort", "msm_accum", "msm_reduce", "ntt", "fold_witness", "fold_instance"]


def zk_strerror(code: int) -> str:
    return lib.zk_strerror(int(code)).decode()


def zk_kernel_launches() -> int:
    return int(lib.zk_kernel_launches())


def zk_probe_rates(device: int = 0):
    """(IMAD/s, F_q Montgomery products/s) measured on `device`."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.zk_probe_rates(int(device), ctypes.byref(a), ctypes.byref(b)), "zk_probe_rates")
    return a.value, b.value


PROBES = ["mad_lo", "mad_hi", "mad_wide", "mad_pair", "add_pair", "fq_mul", "fr_mul"]


def zk_probe_pipes(device: int = 0) -> dict:
    """Measured issue rates (per second) of the integer instruction forms the
    product code is built from, and of the F_q / F_r products themselves."""
    r = (ctypes.c_double * len(PROBES))()
    _check(lib.zk_probe_pipes(int(device), r), "zk_probe_pipes")
    return {k: r[i] for i, k in enumerate(PROBES)}


def zk_field_op(field: int, op: int, a, b, out, n: int = None, stream=None) -> None:
    """Elementwise field arithmetic on device vectors of canonical elements
    (int64 tensors of shape (n, 4)); b is ignored by SQR and INV."""
    if n is None:
        n = a.numel() // 4
    _check(lib.zk_field_op(int(field), int(op), _ptr(a), _ptr(b), _ptr(out), int(n), _stream(stream)),
           "zk_field_op")


def zk_open(ctx: int, coeffs, x, y, proof, quotient=None, n: int = None, stream=None) -> None:
    """KZG opening at x: y = f(x), proof = [q(tau)]_1, q = (f - y)/(X - x)
    (optionally written to `quotient`, n - 1 scalars).  Buffers: torch tensors
    (device or host) or numpy arrays of canonical limbs."""
    if n is None:
        n = _nelem(coeffs, 4)
    _check(lib.zk_open(ctx, _ptr(coeffs), int(n), _ptr(x), _ptr(y), _ptr(proof), _ptr(quotient),
                       _stream(stream)), "zk_open")


def zk_open_batch(ctx: int, polys, x, gamma, ys, proof, stream=None) -> None:
    """Batch opening at x: ys[i] = f_i(x), one proof for sum_i gamma^i f_i."""
    ptrs = (ctypes.c_void_p * len(polys))(*[_ptr(p) for p in polys])
    lens = (ctypes.c_size_t * len(polys))(*[_nelem(p, 4) for p in polys])
    _check(lib.zk_open_batch(ctx, ptrs, lens, len(polys), _ptr(x), _ptr(gamma), _ptr(ys), _ptr(proof),
                             _stream(stream)), "zk_open_batch")


def zk_mul_quotient(ctx: int, a, b, com, t=None, n: int = None, stream=None) -> None:
    """Mul / MatMul quotient t = (A B - L)/(X^n - 1) of evaluation vectors a, b
    over H (L interpolates a o b); com = [t(tau)]_1, t optional."""
    if n is None:
        n = _nelem(a, 4)
    _check(lib.zk_mul_quotient(ctx, _ptr(a), _ptr(b), int(n), _ptr(t), _ptr(com), _stream(stream)),
           "zk_mul_quotient")


def zk_set_fold_degree(ctx: int, degree: int) -> None:
    """Folded relation: 2 (m1 o m2 - mu m3 = e) or 3 (m1 o m2 o m3 - mu^2 m4 = e)."""
    _check(lib.zk_set_fold_degree(ctx, int(degree)), "zk_set_fold_degree")


def zk_set_hiding_base(ctx: int, H) -> None:
    """Hiding base H (64-byte canonical affine point) for zk_commit_hiding."""
    _check(lib.zk_set_hiding_base(ctx, _ptr(H)), "zk_set_hiding_base")


def zk_commit_hiding(ctx: int, coeffs, s, out, n: int = None, stream=None) -> None:
    """out = [f(tau)]_1 + s H."""
    if n is None:
        n = _nelem(coeffs, 4)
    _check(lib.zk_commit_hiding(ctx, _ptr(coeffs), int(n), _ptr(s), _ptr(out), _stream(stream)),
           "zk_commit_hiding")


def zk_set_commit_route(ctx: int, route: int) -> None:
    _check(lib.zk_set_commit_route(ctx, int(route)), "zk_set_commit_route")


def zk_timing_enable(ctx: int, on: bool = True) -> None:
    _check(lib.zk_timing_enable(ctx, int(bool(on))), "zk_timing_enable")


def zk_timing_read(ctx: int) -> dict:
    """{phase: (device ms, intervals)} since the last read."""
    ms = (ctypes.c_double * len(PHASES))()
    cnt = (ctypes.c_ulonglong * len(PHASES))()
    _check(lib.zk_timing_read(ctx, ms, cnt), "zk_timing_read")
    return {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}


def zk_tune_set(ctx: int, op: int, log2n: int, value: int) -> None:
    _check(lib.zk_tune_set(ctx, int(op), int(log2n), int(value)), "zk_tune_set")


def zk_tune_get(ctx: int, op: int, log2n: int) -> int:
    v = ctypes.c_int()
    _check(lib.zk_tune_get(ctx, int(op), int(log2n), ctypes.byref(v)), "zk_tune_get")
    return v.value


def zk_tune_measure(ctx: int, op: int, log2n: int, value: int, reps: int = 3) -> float:
    ms = ctypes.c_double()
    _check(lib.zk_tune_measure(ctx, int(op), int(log2n), int(value), int(reps), ctypes.byref(ms)),
           "zk_tune_measure")
    return ms.value


def _check(rc: int, where: str):
    if rc != ZK_OK:
        raise ZkError(rc, where)


# ---------------------------------------------------------------------------
# Pointer / stream marshalling
# ---------------------------------------------------------------------------

def _ptr(buf) -> int:
    """Address of a torch tensor (device or host) or a numpy array (host)."""
    if buf is None:
        return 0
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"], "numpy buffers must be contiguous"
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        assert buf.is_contiguous(), "tensors must be contiguous"
        return buf.data_ptr()
    return int(buf)


def _stream(stream=None) -> int:
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return 0
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _nelem(buf, width: int) -> int:
    n = buf.numel() if hasattr(buf, "numel") else buf.size
    assert n % width == 0
    return n // width


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def zk_init(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = _VP()
    _check(lib.zk_init(ctypes.byref(h), int(device), int(hbm_budget_bytes)), "zk_init")
    return h.value


def zk_destroy(ctx: int) -> None:
    _check(lib.zk_destroy(ctx), "zk_destroy")


def zk_lane_create(ctx: int) -> int:
    h = _VP()
    _check(lib.zk_lane_create(ctx, ctypes.byref(h)), "zk_lane_create")
    return h.value


def zk_srs_load(ctx: int, pts, n: int | None = None) -> None:
    n = _nelem(pts, 8) if n is None else n
    _check(lib.zk_srs_load(ctx, _ptr(pts), n), "zk_srs_load")


def zk_srs_generate(ctx: int, tau, n: int) -> None:
    t = np.ascontiguousarray(np.asarray(tau, dtype=np.uint64).reshape(4))
    _check(lib.zk_srs_generate(ctx, t.ctypes.data, int(n)), "zk_srs_generate")


def zk_srs_size(ctx: int) -> int:
    n = ctypes.c_size_t()
    _check(lib.zk_srs_size(ctx, ctypes.byref(n)), "zk_srs_size")
    return n.value


def zk_srs_export(ctx: int, out, first: int, count: int, stream=None) -> None:
    _check(lib.zk_srs_export(ctx, _ptr(out), first, count, _stream(stream)), "zk_srs_export")


def zk_commit(ctx: int, coeffs, out, n: int | None = None, stream=None) -> None:
    n = _nelem(coeffs, 4) if n is None else n
    _check(lib.zk_commit(ctx, _ptr(coeffs), n, _ptr(out), _stream(stream)), "zk_commit")


def zk_commit_noalloc(ctx: int, coeffs, out, n: int | None = None, stream=None) -> None:
    """zk_commit without any device allocation (device buffers, n <= 4096)."""
    n = _nelem(coeffs, 4) if n is None else n
    _check(lib.zk_commit_noalloc(ctx, _ptr(coeffs), n, _ptr(out), _stream(stream)),
           "zk_commit_noalloc")


def zk_commit_batch(ctx: int, vecs, out, flags: int = 0, lens=None, stream=None) -> None:
    count = len(vecs)
    ptrs = (ctypes.c_void_p * max(count, 1))(*[_ptr(v) for v in vecs])
    lens = [(_nelem(v, 4)) for v in vecs] if lens is None else list(lens)
    ls = (ctypes.c_size_t * max(count, 1))(*lens)
    _check(lib.zk_commit_batch(ctx, ptrs, ls, count, int(flags), _ptr(out), _stream(stream)),
           "zk_commit_batch")


def zk_ntt(ctx: int, data, n: int | None = None, stream=None) -> None:
    n = _nelem(data, 4) if n is None else n
    _check(lib.zk_ntt(ctx, _ptr(data), n, _stream(stream)), "zk_ntt")


def zk_intt(ctx: int, data, n: int | None = None, stream=None) -> None:
    n = _nelem(data, 4) if n is None else n
    _check(lib.zk_intt(ctx, _ptr(data), n, _stream(stream)), "zk_intt")


def zk_ntt_batch(ctx: int, vecs, inverse: bool, stream=None) -> None:
    count = len(vecs)
    ptrs = (ctypes.c_void_p * max(count, 1))(*[_ptr(v) for v in vecs])
    ls = (ctypes.c_size_t * max(count, 1))(*[_nelem(v, 4) for v in vecs])
    _check(lib.zk_ntt_batch(ctx, ptrs, ls, count, int(bool(inverse)), _stream(stream)), "zk_ntt_batch")


def zk_plan_commit_batch(ctx: int, vecs, out, flags: int = 0, lens=None) -> int:
    count = len(vecs)
    ptrs = (ctypes.c_void_p * max(count, 1))(*[_ptr(v) for v in vecs])
    lens = [(_nelem(v, 4)) for v in vecs] if lens is None else list(lens)
    ls = (ctypes.c_size_t * max(count, 1))(*lens)
    h = _VP()
    _check(lib.zk_plan_commit_batch(ctx, ptrs, ls, count, int(flags), _ptr(out), ctypes.byref(h)),
           "zk_plan_commit_batch")
    return h.value


def zk_plan_fold_tree(ctx: int, leaves, gammas, root) -> int:
    arr = (ZkAcc * len(leaves))(*leaves)
    h = _VP()
    _check(lib.zk_plan_fold_tree(ctx, arr, len(leaves), _ptr(gammas), ctypes.byref(root), ctypes.byref(h)),
           "zk_plan_fold_tree")
    return h.value


def zk_plan_launch(plan: int, stream=None) -> None:
    _check(lib.zk_plan_launch(plan, _stream(stream)), "zk_plan_launch")


def zk_plan_nodes(plan: int) -> int:
    n = ctypes.c_size_t()
    _check(lib.zk_plan_nodes(plan, ctypes.byref(n)), "zk_plan_nodes")
    return n.value


def zk_plan_destroy(plan: int) -> None:
    _check(lib.zk_plan_destroy(plan), "zk_plan_destroy")


def zk_server_create(ctx: int, lanes: int = 4, hbm_budget_bytes: int = 0) -> int:
    h = _VP()
    _check(lib.zk_server_create(ctx, int(lanes), int(hbm_budget_bytes), ctypes.byref(h)),
           "zk_server_create")
    return h.value


def make_job(n: int, w, leaf: ZkAcc, acc_in: ZkAcc | None = None, acc_out: ZkAcc | None = None,
             gamma=None) -> ZkJob:
    j = ZkJob()
    j.n = n
    for i in range(3):
        j.w[i] = _ptr(w[i])
    j.leaf = ctypes.addressof(leaf)
    j.acc_in = ctypes.addressof(acc_in) if acc_in is not None else 0
    j.acc_out = ctypes.addressof(acc_out) if acc_out is not None else 0
    j.gamma = _ptr(gamma)
    return j


def zk_submit(srv: int, job: ZkJob) -> int:
    t = ctypes.c_uint64()
    _check(lib.zk_submit(srv, ctypes.byref(job), ctypes.byref(t)), "zk_submit")
    return t.value


def zk_poll(srv: int, ticket: int) -> ZkTicketInfo:
    info = ZkTicketInfo()
    _check(lib.zk_poll(srv, ticket, ctypes.byref(info)), "zk_poll")
    return info


def zk_wait(srv: int, ticket: int, timeout_ms: int = 60000) -> ZkTicketInfo:
    info = ZkTicketInfo()
    _check(lib.zk_wait(srv, ticket, int(timeout_ms), ctypes.byref(info)), "zk_wait")
    return info


def zk_server_stats(srv: int) -> ZkServerInfo:
    info = ZkServerInfo()
    _check(lib.zk_server_stats(srv, ctypes.byref(info)), "zk_server_stats")
    return info


ZK_CHECK_SCALAR, ZK_CHECK_BUCKET, ZK_CHECK_ENTRY, ZK_CHECK_NTT_IDX = 1, 2, 4, 8


def zk_check_status(ctx: int):
    """(flags raised since the last call, whether this is the checked build)."""
    f, c = ctypes.c_uint(), ctypes.c_int()
    _check(lib.zk_check_status(ctx, ctypes.byref(f), ctypes.byref(c)), "zk_check_status")
    return f.value, bool(c.value)


def load_checked():
    """The checked build (libzkb300_check.so, built by `build.py --check`) as
    a raw ctypes library with the same entry points: call it as `lib.zk_...`
    with the pointer arguments the functions above pass."""
    return _load(os.path.join(_HERE, "libzkb300_check.so"))


def zk_cancel(srv: int, ticket: int) -> None:
    """Takes a still-queued job out of the queue (ZK_EBUSY if it already ran)."""
    _check(lib.zk_cancel(srv, int(ticket)), "zk_cancel")


def zk_server_destroy(srv: int) -> None:
    _check(lib.zk_server_destroy(srv), "zk_server_destroy")


def make_acc(m, e, x) -> ZkAcc:
    """Accumulator descriptor from device tensors: m = four (n, 4) tensors (or
    one (4, n, 4) tensor), e (n, 4), x (44,) int64 (zk_acc_inst)."""
    a = ZkAcc()
    ms = [m[i] for i in range(4)]
    a.n = _nelem(e, 4)
    for i in range(4):
        a.m[i] = _ptr(ms[i])
    a.e = _ptr(e)
    a.x = _ptr(x)
    return a


def zk_leaf_init(ctx: int, accs, stream=None) -> None:
    arr = (ZkAcc * len(accs))(*accs)
    _check(lib.zk_leaf_init(ctx, arr, len(accs), _stream(stream)), "zk_leaf_init")


def zk_fold(ctx: int, L: ZkAcc, R: ZkAcc, gamma, out: ZkAcc, E1_out=None, stream=None) -> None:
    _check(lib.zk_fold(ctx, ctypes.byref(L), ctypes.byref(R), _ptr(gamma), ctypes.byref(out),
                       _ptr(E1_out), _stream(stream)), "zk_fold")


def zk_fold_tree(ctx: int, leaves, gammas, root: ZkAcc, stream=None) -> None:
    arr = (ZkAcc * len(leaves))(*leaves)
    _check(lib.zk_fold_tree(ctx, arr, len(leaves), _ptr(gammas), ctypes.byref(root), _stream(stream)),
           "zk_fold_tree")


def zk_fold_tree_levels(ctx: int, leaves, gammas, levels: int, stream=None) -> list:
    """The first `levels` levels of the fold tree; returns the indices of the
    leaves that now hold that level's accumulators (the checkpoint)."""
    arr = (ZkAcc * len(leaves))(*leaves)
    _check(lib.zk_fold_tree_levels(ctx, arr, len(leaves), _ptr(gammas), int(levels), _stream(stream)),
           "zk_fold_tree_levels")
    span = 1 << int(levels)
    return [j * span + span - 1 for j in range(len(leaves) // span)]
