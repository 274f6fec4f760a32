"""GPU parity of the SRS and the KZG commitment MSM against the oracle.

Bit-exact throughout (finite-field arithmetic is exact; points are compared
in canonical affine form).  Small sizes compare with the oracle's affine
double-and-add MSM; sizes the oracle cannot run in seconds (2^20, 2^22)
compare with the commitment's closed form [f(tau)]_1 for the known tau."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def _commit(zk, ctx, c):
    import torch
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    zk.zk_commit(ctx, to_dev(c), out)
    torch.cuda.synchronize()
    return to_host(out)


def test_generated_srs_matches_oracle(zk, ctx_small, srs_small):
    import torch
    n = srs_small.shape[0]
    out = torch.zeros((n, 8), dtype=torch.int64, device="cuda")
    zk.zk_srs_export(ctx_small, out, 0, n)
    torch.cuda.synchronize()
    assert pts_equal(to_host(out), srs_small)


def test_loaded_srs_validation_and_use(zk, orc, srs_small):
    ctx = zk.zk_init(0)
    try:
        pts = np.ascontiguousarray(srs_small[:256])
        zk.zk_srs_load(ctx, pts)            # host pointer
        assert zk.zk_srs_size(ctx) == 256
        c = Z.fr_uniform(41, 256)
        assert pts_equal(_commit(zk, ctx, c), orc.msm(pts, c))
        zk.zk_srs_load(ctx, to_dev(pts))    # device pointer
        assert pts_equal(_commit(zk, ctx, c), orc.msm(pts, c))
        for bad in ("off", "noncanon", "inf"):
            p = pts.copy()
            if bad == "off":
                p[7, 4] ^= np.uint64(1)
            elif bad == "noncanon":
                p[9, :4] = orc.from_int(Z.Q_MOD + 1)
            else:
                p[11] = 0
            with pytest.raises(zk.ZkError) as ei:
                zk.zk_srs_load(ctx, p)
            assert ei.value.code == zk.ZK_EINVAL
            assert zk.zk_srs_size(ctx) == 0
    finally:
        zk.zk_destroy(ctx)


def test_msm_full_oracle_2_12(zk, orc, ctx_small, srs_small, tau):
    n = 1 << 12
    c = Z.fr_uniform(1, n)
    got = _commit(zk, ctx_small, c)
    assert pts_equal(got, orc.msm(srs_small, c))
    assert pts_equal(got, orc.commit_coeffs_tau(c, tau))


@pytest.mark.parametrize("n", [1, 2, 3, 31, 1000, 4095])
def test_msm_ragged_lengths(zk, orc, ctx_small, tau, n):
    c = Z.fr_uniform(100 + n, n)
    assert pts_equal(_commit(zk, ctx_small, c), orc.commit_coeffs_tau(c, tau))


@pytest.mark.parametrize("dist", ["uniform", "gauss"])
def test_msm_quantised_scalars(zk, orc, ctx_small, srs_small, dist):
    n = 1 << 12
    c = Z.zkml_scalars(4, n, dist)
    assert pts_equal(_commit(zk, ctx_small, c), orc.msm(srs_small, c))


def test_msm_edge_cases(zk, orc, ctx_small, srs_small, tau):
    n = 512
    inf = np.zeros(8, dtype=np.uint64)
    assert pts_equal(_commit(zk, ctx_small, np.zeros((n, 4), np.uint64)), inf)
    c = np.zeros((n, 4), np.uint64)
    c[17] = Z.int_to_fr(R - 1)
    assert pts_equal(_commit(zk, ctx_small, c), orc.g1_neg(srs_small[17]))
    # Recentring boundary (r-1)/2 and (r+1)/2, the largest digits, powers of two.
    specials = [(R - 1) // 2, (R + 1) // 2, R - 2, 1, 2, (1 << 253) - 1, 1 << 252, (1 << 16) - 1,
                1 << 15, (1 << 15) + 1, 3 << 240]
    c = np.stack([Z.int_to_fr(v % R) for v in specials])
    assert pts_equal(_commit(zk, ctx_small, c), orc.commit_coeffs_tau(c, tau))
    # Every scalar equal: all points land in the same buckets (maximal skew).
    c = np.tile(Z.fr_uniform(7, 1)[0], (4096, 1))
    assert pts_equal(_commit(zk, ctx_small, c), orc.commit_coeffs_tau(c, tau))
    c = np.tile(Z.int_to_fr(5), (4096, 1))
    assert pts_equal(_commit(zk, ctx_small, c), orc.commit_coeffs_tau(c, tau))


def test_msm_host_buffers(zk, orc, ctx_small, tau):
    n = 777
    c = Z.fr_uniform(55, n)
    out = np.zeros(8, dtype=np.uint64)
    zk.zk_commit(ctx_small, np.ascontiguousarray(c), out)
    assert pts_equal(out, orc.commit_coeffs_tau(c, tau))


def test_commit_batch_ragged_and_evals(zk, orc, ctx_small, tau):
    import torch
    lens = [1, 5, 64, 100, 1024, 3000, 4096, 2]
    vecs = [Z.fr_uniform(200 + i, l) for i, l in enumerate(lens)]
    out = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_small, [to_dev(v) for v in vecs], out)
    torch.cuda.synchronize()
    got = to_host(out)
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), k
    # Evaluation form: INTT then MSM, padded to a power of two.
    evals = [Z.zkml_scalars(300 + i, l) for i, l in enumerate([4, 64, 1000, 4096])]
    out2 = np.zeros((len(evals), 8), dtype=np.uint64)
    zk.zk_commit_batch(ctx_small, [np.ascontiguousarray(v) for v in evals], out2, flags=zk.ZK_EVALS)
    for k, v in enumerate(evals):
        n2 = 1 << (len(v) - 1).bit_length()
        vp = np.zeros((n2, 4), np.uint64)
        vp[:len(v)] = v
        assert pts_equal(out2[k], orc.commit_evals_tau(vp, tau)), k


@pytest.mark.parametrize("dist", ["fr", "zkml", "zkml_gauss"])
def test_msm_at_scale_2_20(zk, orc, ctx_big, tau, dist):
    n = 1 << 20
    c = {"fr": lambda: Z.fr_uniform(3, n),
         "zkml": lambda: Z.zkml_scalars(4, n),
         "zkml_gauss": lambda: Z.zkml_scalars(4, n, "gauss")}[dist]()
    assert pts_equal(_commit(zk, ctx_big, c), orc.commit_coeffs_tau(c, tau))


def test_msm_at_scale_2_22(zk, orc, ctx_big, tau):
    n = 1 << 22
    c = Z.fr_uniform(12, n)
    assert pts_equal(_commit(zk, ctx_big, c), orc.commit_coeffs_tau(c, tau))


def test_big_srs_samples(zk, orc, ctx_big, tau):
    import torch
    n = 1 << 22
    out = torch.zeros((n, 8), dtype=torch.int64, device="cuda")
    zk.zk_srs_export(ctx_big, out, 0, n)
    torch.cuda.synchronize()
    pts = to_host(out)
    assert orc.count_off_curve(pts) == 0  # every point on the curve
    G = orc.g1_generator()
    t = Z.fr_to_int(tau)
    rng = np.random.default_rng(0)
    for i in [0, 1, 2, n - 1] + rng.integers(0, n, 64).tolist():
        assert pts_equal(pts[i], orc.g1_mul(G, Z.int_to_fr(pow(t, int(i), R)))), i


@pytest.fixture(scope="module")
def window_case(tau):
    c = Z.fr_uniform(77, 4096)
    return c


@pytest.mark.parametrize("c", list(range(9, 21)))
def test_msm_every_window_width(zk, orc, ctx_small, tau, window_case, c):
    try:
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_MSM_WINDOW, 12, c)
        got = _commit(zk, ctx_small, window_case)
    finally:
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_MSM_WINDOW, 12, 0)
    assert pts_equal(got, orc.commit_coeffs_tau(window_case, tau))


def test_autotune_table(zk, ctx_small, tmp_path):
    from paper_2507_07031_b300 import autotune
    path = str(tmp_path / "tune.json")
    table = autotune.tune(ctx_small, msm_logs=[10, 12], ntt_logs=[10, 12], reps=1,
                          windows=range(10, 14), radices=range(5, 12), path=path, layout_logs=[12])
    assert set(table["msm_window"]) == {"10", "12"} and set(table["ntt_radix"]) == {"10", "12"}
    for lg, e in table["msm_window"].items():
        assert zk.zk_tune_get(ctx_small, zk.ZK_TUNE_MSM_WINDOW, int(lg)) == e["best"]
    for name, (op, values) in autotune.MSM_LAYOUT.items():
        e = table["msm_layout"][name]["12"]
        assert set(e["ms"]) == {str(v) for v in values}
        assert zk.zk_tune_get(ctx_small, op, 12) == e["best"]
    autotune.apply(ctx_small, path)
    for lg in (10, 12):
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_MSM_WINDOW, lg, 0)
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_NTT_RADIX, lg, 0)
        for op, _ in autotune.MSM_LAYOUT.values():
            zk.zk_tune_set(ctx_small, op, lg, 0)
    assert zk.zk_tune_get(ctx_small, zk.ZK_TUNE_MSM_TAIL, 12) == 4  # built-in: eight items per lane


def test_large_mixed_batch(zk, orc, ctx_big, tau):
    """A batch of many small and some large MSMs (as a model's witness
    commitments): the bucket reduction then widens its segments to amortise
    each team's scans, down to levels whose items fit one segment."""
    import torch
    rng = np.random.default_rng(5)
    lens = [int(x) for x in (1 << rng.integers(6, 13, 600))] + [1 << 14] * 6 + [3000, 1 << 15]
    vecs = [Z.zkml_scalars(40_000 + i, l) if i % 3 else Z.fr_uniform(40_000 + i, l)
            for i, l in enumerate(lens)]
    out = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_big, [to_dev(v) for v in vecs], out)
    torch.cuda.synchronize()
    got = to_host(out)
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), (k, lens[k])


@pytest.mark.parametrize("g", [1, 2, 3, 4, 5])
def test_batch_sequential_reduction_level(zk, orc, ctx_big, tau, g):
    """A large batch runs the first level of its bucket reduction one thread
    per 2^g buckets (running sums), g the largest value up to 5 for which the
    batch's buckets give every resident thread (512 per SM) two segments.
    Batches of 2^12-point jobs (4096 buckets each) are sized here for each g.
    Every third job has quantised scalars, for which the device lowers the
    bucket count to 2^8 (the threads past it exit); one job is all zero."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 1 << 12
    count = (2 * sms * 512 << g) // 4096 + 1
    vecs = []
    for i in range(count):
        if i == 1:
            vecs.append(np.zeros((n, 4), dtype=np.uint64))
        elif i % 3 == 0:
            vecs.append(Z.zkml_scalars(50_000 + i, n))
        else:
            vecs.append(Z.fr_uniform(50_000 + i, n))
    out = torch.zeros((count, 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_big, [to_dev(v) for v in vecs], out)
    torch.cuda.synchronize()
    got = to_host(out)
    assert not got[1].any()  # the zero job commits to infinity
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), (g, k)


def test_batch_wide_recode(zk, orc, ctx_big, tau):
    """In a batch whose long jobs (2^14 points or more, window width <= 16)
    give every SM at least two chunks of 8192 scalars, those jobs are sorted
    through shared-memory histograms (one block per chunk).  Here: 2^16-point
    jobs at width 15 (uniform, and every fourth quantised), two ragged long
    jobs (2^14 + 3, 2^15 - 1), an all-zero long job, a shorter job of the same
    width (10000 points, on the per-scalar path) and one of another width."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nbig = (2 * sms + 7) // 8 + 2
    lens = [1 << 16] * nbig + [(1 << 14) + 3, (1 << 15) - 1, 1 << 16, 10000, 3000]
    vecs = []
    for i, n in enumerate(lens):
        if i == nbig + 2:
            vecs.append(np.zeros((n, 4), dtype=np.uint64))
        elif i % 4 == 3:
            vecs.append(Z.zkml_scalars(60_000 + i, n))
        else:
            vecs.append(Z.fr_uniform(60_000 + i, n))
    out = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_big, [to_dev(v) for v in vecs], out)
    torch.cuda.synchronize()
    got = to_host(out)
    assert not got[nbig + 2].any()
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), (k, lens[k])


def test_batch_window_rule(zk, orc, ctx_big, tau):
    """Calls of 64 jobs or more give 2^17- and 2^18-point jobs window width
    16 (single MSMs take 15): three such jobs, one ragged, among 67 short
    ones, against the closed form."""
    import torch
    lens = [1 << 17, 1 << 18, (1 << 17) + 5] + [1 << 10] * 67
    vecs = [Z.fr_uniform(70_000 + i, n) if i % 2 == 0 else Z.zkml_scalars(70_000 + i, n)
            for i, n in enumerate(lens)]
    out = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_big, [to_dev(v) for v in vecs], out)
    torch.cuda.synchronize()
    got = to_host(out)
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), (k, lens[k])


@pytest.fixture(scope="module")
def layout_case():
    n = 1 << 18
    return {"int8": Z.zkml_scalars(31, n), "uniform": Z.fr_uniform(32, n)}


@pytest.mark.parametrize("op,value", [("CHUNK", v) for v in range(1, 5)] + [("TAIL", v) for v in range(1, 5)]
                         + [("SEG", v) for v in range(3, 6)] + [("SEGBIG", v) for v in range(6, 9)])
def test_msm_every_bucket_layout(zk, orc, ctx_big, tau, layout_case, op, value):
    """Every value of every bucket-layout knob gives the closed form, on
    quantised scalars (2^18 entries in 128 buckets: round 0, the team tail,
    small reduction segments) and uniform ones (many buckets, large
    segments)."""
    code = getattr(zk, "ZK_TUNE_MSM_" + op)
    try:
        zk.zk_tune_set(ctx_big, code, 18, value)
        assert zk.zk_tune_get(ctx_big, code, 18) == value
        for name, c in layout_case.items():
            assert pts_equal(_commit(zk, ctx_big, c), orc.commit_coeffs_tau(c, tau)), name
    finally:
        zk.zk_tune_set(ctx_big, code, 18, 0)
    with pytest.raises(zk.ZkError):
        zk.zk_tune_set(ctx_big, code, 18, 99)


def test_msm_small_scalar_path(zk, orc, ctx_small, tau):
    """Short recentred scalars: common trailing zeros are shifted out and only
    the windows that can hold digits are used (one window, read from the SRS,
    when the rest fits).  Mixed in one batch with full-width and zero jobs."""
    import torch
    n = 4096
    rng = np.random.default_rng(11)
    small = rng.integers(-300, 300, n)
    cases = {
        "int8x2^16": Z.zkml_scalars(21, n),
        "pm1": Z.encode_signed(rng.integers(-1, 2, n), 0),
        "shift200": np.stack([Z.int_to_fr((int(v) << 200) % R) for v in small]),
        "shift37_wide": np.stack([Z.int_to_fr((int(v) << 37) % R) for v in rng.integers(0, 1 << 60, n)]),
        "uniform": Z.fr_uniform(22, n),
        "zero": np.zeros((n, 4), np.uint64),
    }
    names = list(cases)
    out = torch.zeros((len(names), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_small, [to_dev(cases[k]) for k in names], out)
    torch.cuda.synchronize()
    got = to_host(out)
    for i, k in enumerate(names):
        assert pts_equal(got[i], orc.commit_coeffs_tau(cases[k], tau)), k
        assert pts_equal(_commit(zk, ctx_small, cases[k]), got[i]), k


def test_msm_repeated_and_opposite_points(zk, orc):
    """An SRS of 2048 copies of G puts equal and opposite points into the same
    buckets, so the bucket sums meet a = b (doubling) and a = -b (infinity)
    throughout; the commitment must be (sum_i s_i) G."""
    n = 2048
    G = orc.g1_generator()
    ctx = zk.zk_init(0)
    try:
        zk.zk_srs_load(ctx, np.ascontiguousarray(np.tile(G, (n, 1))))
        rng = np.random.default_rng(5)
        cases = {
            "small": Z.encode_signed(rng.integers(-300, 300, n), 0),
            "pm1": Z.encode_signed(rng.integers(-1, 2, n), 0),
            "uniform": Z.fr_uniform(9, n),
            "equal": np.tile(Z.int_to_fr(7), (n, 1)),
            "cancel": np.concatenate([np.tile(Z.int_to_fr(5), (n // 2, 1)),
                                      np.tile(Z.int_to_fr(R - 5), (n // 2, 1))]),
        }
        for name, c in cases.items():
            total = sum(Z.fr_to_int(v) for v in c) % R
            want = orc.g1_mul(G, Z.int_to_fr(total)) if total else np.zeros(8, np.uint64)
            assert pts_equal(_commit(zk, ctx, c), want), name
    finally:
        zk.zk_destroy(ctx)


def test_host_buffer_commit_at_2_20(zk, orc, ctx_big, tau):
    """The end-to-end call: scalars and output in host memory (staged through
    the workspace inside the call), against the closed form."""
    n = (1 << 20) + 5
    c = np.ascontiguousarray(Z.fr_uniform(91, n))
    h_out = np.zeros(8, dtype=np.uint64)
    zk.zk_commit(ctx_big, c, h_out)
    assert pts_equal(h_out, orc.commit_coeffs_tau(c, tau))
