"""Benchmark of the BN254 prover hot path on B300.

One step = one pass of the whole hot path over its synthetic inputs, all
resident in HBM: KZG commitment MSMs of n = 2^20 points (scalars uniform in
F_r, and quantised int8 * 2^16 values), F_r NTT + INTT of lengths 2^20 and
2^22, the batched commitment of a CNN's 256 witness polynomials (2^24
evaluations: INTT + MSM each, one batch), and the parallel fold tree of 1024
accumulators of n = 2^16 (1023 generalised-Mira folds: cross terms, their
commitments, witness and instance combinations).  L2 is flushed before every
op.  The headline value is MSM throughput (Mpts/s) at 2^20 with uniform
scalars; the JSON line also carries every op's time and roofline (IMAD pipe
against the live mad.lo probe, HBM against the measured copy bandwidth), the
batched-vs-plain comparisons, the small-task regime of the graph plans, the
serving loop at its stated load, the end-to-end commitment through the C ABI
with host buffers, and the CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import zkinputs as Z  # noqa: E402

METRIC = "BN254 MSM Mpts/s & Fr NTT Melem/s at 2^20; batched folds/s vs plain; % roofline"
UNIT = "Mpts/s"
WORKLOAD = ("hot path at scale: MSM 2^20 (uniform F_r; int8*2^16), NTT/INTT 2^20 and 2^22, "
            "256-poly CNN commitment batch (2^24 evaluations), fold tree 1024 x 2^16")
L2_FLUSH_BYTES = 512 << 20
SRS_LOG = 22
# Per mixed addition (madd-2008-s): 8 multiplications + 2 squarings in F_q;
# per Montgomery product 264 32-bit IMADs (8 x (16 product + 16 reduction + 1)).
FQ_MUL_PER_MADD = 10
IMAD_PER_MUL = 264
IMAD_LO, IMAD_HI = 136, 128  # mad.lo (incl. the 8 m = t n0 products) and mad.hi per product
FOLD_MULS = 11               # F_r products per element of the degree-2 witness pass
FOLD_BYTES = 512             # bytes per element of the witness pass (10 vectors read, 6 written)
NTT_BYTES_PER_ELEM = 2 * 64  # two passes, each reading and writing 32 B per element
HBM_FALLBACK = 6400.0        # GB/s, used only when MEASURED_PEAKS.json is absent
# DRAM bytes (read + write) of one k_pieces_first launch, uniform 2^20, c = 17,
# from an ncu capture of that launch (dram__bytes_read.sum +
# dram__bytes_write.sum); None when the kernel has changed since.
ACCUM_TRAFFIC = 2.1457e9
CPU_SAMPLE_LOG = 15  # oracle MSM sample: 2^15 points, ~10-15 s on 16 cores


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the comparisons and the serving run")
    ap.add_argument("--serving-jobs", type=int, default=1200, help="jobs of the serving run (Poisson, 20/s)")
    ap.add_argument("--case", default=None, choices=["msm", "ntt", "fold", "open", "batch"],
                    help="profiling case: two calls of one op at --log2n (for ncu captures); batch: "
                         "two batched commitments of --count polynomials of 2^log2n (a fold-tree level)")
    ap.add_argument("--count", type=int, default=512, help="polynomials of the batch case")
    ap.add_argument("--log2n", type=int, default=18)
    ap.add_argument("--cpu-sample-log", type=int, default=CPU_SAMPLE_LOG,
                    help="log2 points of the oracle MSM sample (cpu_baseline; the reference arm "
                         "times 2^(this - 1) per step)")
    return ap.parse_args()


def run_case(args):
    """Small profiling case: set-up, then the same op twice (warm-up + the
    captured launch).  Inputs exceed L2 (table or data > 126 MB)."""
    import torch
    import paper_2507_07031_b300 as zk
    n = 1 << args.log2n

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()

    ctx = zk.zk_init(0)
    zk.zk_srs_generate(ctx, Z.tau(0), n if args.case != "ntt" else 2)
    if args.case == "msm":
        sc = dev(Z.fr_uniform(3, n))
        out = torch.zeros(8, dtype=torch.int64, device="cuda")
        for _ in range(2):
            zk.zk_commit(ctx, sc, out)
    elif args.case == "ntt":
        x = dev(Z.fr_uniform(5, n))
        for _ in range(2):
            zk.zk_ntt(ctx, x)
    elif args.case == "batch":
        sc = dev(Z.fr_uniform(13, args.count * n)).view(args.count, n, 4)
        vecs = [sc[i] for i in range(args.count)]
        out = torch.zeros((args.count, 8), dtype=torch.int64, device="cuda")
        for _ in range(2):
            zk.zk_commit_batch(ctx, vecs, out)
    elif args.case == "open":
        c = dev(Z.fr_uniform(11, n + 1))
        pt = dev(Z.fr_uniform(12, 1)[0])
        y = torch.zeros(4, dtype=torch.int64, device="cuda")
        proof = torch.zeros(8, dtype=torch.int64, device="cuda")
        for _ in range(2):
            zk.zk_open(ctx, c, pt, y, proof)
    else:
        L, R = [], []
        for j in range(2):
            m = torch.zeros((4, n, 4), dtype=torch.int64, device="cuda")
            for i in (0, 1, 3):
                m[i].copy_(dev(Z.zkml_scalars(100 + 4 * j + i, n)))
            e = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
            x = torch.zeros(44, dtype=torch.int64, device="cuda")
            (L if j == 0 else R).extend([m, e, x])
        dl, dr = zk.make_acc(*L), zk.make_acc(*R)
        zk.zk_leaf_init(ctx, [dl, dr])
        g = dev(Z.gammas(1, 1))
        for _ in range(2):
            zk.zk_fold(ctx, dl, dr, g, dr)
    torch.cuda.synchronize()
    zk.zk_destroy(ctx)
    print(json.dumps({"case": args.case, "log2n": args.log2n, "ok": True}))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist=None) -> float:
    """Largest value of x over the ranks (the slowest replica sets the job's
    time).  Uses a CUDA tensor under NCCL and a CPU tensor under gloo."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_per_rank: float, world: int, dist=None) -> float:
    """Weak-scaling throughput: the units all ranks processed divided by the
    slowest rank's time."""
    return units_per_rank * world / max_over_ranks(seconds_per_rank, dist)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

_ORACLE_SRS = {}


def oracle_msm_rate(sample_n: int):
    """The oracle's affine double-and-add MSM timed on sample_n points (its
    SRS is generated once per process, untimed)."""
    import oracle as orc
    orc.lib()
    if sample_n not in _ORACLE_SRS:
        _ORACLE_SRS[sample_n] = orc.srs_gen(Z.tau(0), sample_n)
    srs = _ORACLE_SRS[sample_n]
    c = Z.fr_uniform(3, sample_n)
    t0 = time.perf_counter()
    orc.msm(srs, c)
    dt = time.perf_counter() - t0
    return sample_n / dt / 1e6, dt, orc.threads()


def run_reference(args):
    """The oracle as it stands on the host cores: each step is an affine
    double-and-add MSM over a power-of-two sample sized so that the whole
    --steps K --warmup W run takes about a minute."""
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    import oracle as orc
    orc.lib()
    probe_rate, _, _ = oracle_msm_rate(1 << 10)  # Mpts/s of this host
    per_step_s = 60.0 / max(args.steps + args.warmup, 1)
    lg = int(np.clip(np.floor(np.log2(max(probe_rate * 1e6 * per_step_s, 1.0))), 8, args.cpu_sample_log))
    sample = 1 << lg
    rates, times = [], []
    for _ in range(args.warmup):
        oracle_msm_rate(sample)
    for _ in range(args.steps):
        r, dt, cores = oracle_msm_rate(sample)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "MSM of %d points" % sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "affine double-and-add MSM, %d points per step, SRS from seeded tau" % sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measured_peaks():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json copy benchmark)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK, "of fallback (6.4 TB/s, one earlier B300 measurement)"


def imad_roof(imads, ms, rates):
    """IMAD-pipe roofline entry: algorithmic IMADs per op over its time,
    against the live mad.lo issue rate; the product-mix ceiling (136 mad.lo +
    128 mad.hi per product at the measured lo and hi rates) as an extra."""
    achieved = imads / (ms * 1e-3) / 1e12
    lo, hi = rates["mad_lo"] / 1e12, rates["mad_hi"] / 1e12
    mix = IMAD_PER_MUL / (IMAD_LO / lo + IMAD_HI / hi)
    return {"bound": "alu", "achieved": achieved, "peak": lo, "unit": "TIMAD/s", "frac": achieved / lo,
            "peak_source": "of measured: live mad.lo.u32 issue rate (zk_probe_pipes)",
            "mix_ceiling": mix, "frac_of_mix_ceiling": achieved / mix, "algorithmic_imad": imads}


def hbm_roof(nbytes, ms, hbm, src):
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_source": src, "algorithmic_bytes": nbytes}


def ntt_imads(n):
    return (n // 2) * (n.bit_length() - 1) * IMAD_PER_MUL


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2507_07031_b300 as zk

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()

    ctx = zk.zk_init(local)
    zk.zk_srs_generate(ctx, Z.tau(0), 1 << SRS_LOG)
    n20, n22 = 1 << 20, 1 << 22
    sc_uni = dev(Z.fr_uniform(3, n20))
    sc_q = dev(Z.zkml_scalars(4, n20))
    x20 = dev(Z.fr_uniform(5, n20))
    x22 = dev(Z.fr_uniform(6, n22))
    out = torch.zeros((2, 8), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    # CNN batch: 256 evaluation vectors (int8 * 2^16), INTT + commit each.
    cnn_sizes = Z.cnn_poly_sizes(8)
    cnn = [dev(Z.zkml_scalars(7_000_000 + i, int(s))) for i, s in enumerate(cnn_sizes)]
    cnn_out = torch.zeros((len(cnn), 8), dtype=torch.int64, device="cuda")
    # Fold tree: 1024 leaves of 2^16 (matmul block, 4 witness vectors); the
    # tree overwrites its leaves, so every step restores them first.
    tree = FoldTree(zk, ctx, dev, torch)
    tree.init_leaves()

    ops = [
        ("msm_2^20_uniform", n20, lambda: zk.zk_commit(ctx, sc_uni, out[0])),
        ("msm_2^20_int8x2^16", n20, lambda: zk.zk_commit(ctx, sc_q, out[1])),
        ("ntt_2^20", n20, lambda: zk.zk_ntt(ctx, x20)),
        ("intt_2^20", n20, lambda: zk.zk_intt(ctx, x20)),
        ("ntt_2^22", n22, lambda: zk.zk_ntt(ctx, x22)),
        ("intt_2^22", n22, lambda: zk.zk_intt(ctx, x22)),
        ("cnn_batch_commit", int(cnn_sizes.sum()),
         lambda: zk.zk_commit_batch(ctx, cnn, cnn_out, flags=zk.ZK_EVALS)),
        ("fold_tree_1024x2^16", tree.count - 1, tree.run),
    ]
    ev = {name: [] for name, _, _ in ops}

    def step(record):
        for name, _, fn in ops:
            if name.startswith("fold_tree"):
                tree.restore()  # not part of the op's interval
            flush.fill_(1)  # evict L2 (512 MiB > 126 MB) between ops
            if record:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                # phase intervals of the headline MSM only (the roofline's)
                zk.zk_timing_enable(ctx, name == "msm_2^20_uniform")
                a.record(stream)
                fn()
                b.record(stream)
                ev[name].append((a, b))
            else:
                fn()
        zk.zk_timing_enable(ctx, False)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    zk.zk_timing_read(ctx)  # discard
    sampler = ClockSampler(local)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = zk.zk_kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = zk.zk_kernel_launches() - launches0
    sampler.stop()
    phases = zk.zk_timing_read(ctx)
    total_ms = max_over_ranks(t0.elapsed_time(t1), dist)
    same_tree = tree.root_matches_last()

    per_op = {}
    for name, n, _ in ops:
        ms = statistics.median([a.elapsed_time(b) for a, b in ev[name]])
        unit = ("Mpts/s" if name.startswith("msm") else "Mcoef/s" if name.startswith("cnn")
                else "folds/s" if name.startswith("fold") else "Melem/s")
        per_op[name] = {"ms": ms, unit: (n / (ms * 1e-3) / 1e6) if unit != "folds/s" else n / (ms * 1e-3)}
    msm_ms = per_op["msm_2^20_uniform"]["ms"]
    value = whole_job_rate(n20, msm_ms * 1e-3, world, dist) / 1e6

    # Per-op phase split, from one extra untimed pass with phase timing on.
    phase_split = {}
    for name, _, fn in ops:
        if name.startswith("fold_tree"):
            tree.restore()
        torch.cuda.synchronize()
        zk.zk_timing_read(ctx)
        zk.zk_timing_enable(ctx, True)
        fn()
        zk.zk_timing_enable(ctx, False)
        torch.cuda.synchronize()
        phase_split[name] = {k: round(v[0], 4) for k, v in zk.zk_timing_read(ctx).items() if v[1]}

    # Rooflines.  Denominators: the live probes of this run (IMAD) and the
    # measured copy bandwidth (HBM).
    rates = zk.zk_probe_pipes(local)
    hbm, hbm_src = measured_peaks()
    c20 = zk.zk_tune_get(ctx, zk.ZK_TUNE_MSM_WINDOW, 20)
    W = -(-254 // c20)
    madd = FQ_MUL_PER_MADD * IMAD_PER_MUL
    roofs = {}
    roofs["msm_2^20_uniform"] = imad_roof(n20 * W * madd, msm_ms, rates)
    # int8 * 2^16: one 9-bit window after the shift, one mixed addition per point
    roofs["msm_2^20_int8x2^16"] = imad_roof(n20 * madd, per_op["msm_2^20_int8x2^16"]["ms"], rates)
    for name, n in (("ntt_2^20", n20), ("intt_2^20", n20), ("ntt_2^22", n22), ("intt_2^22", n22)):
        ms = per_op[name]["ms"]
        roofs[name] = {"imad": imad_roof(ntt_imads(n), ms, rates),
                       "hbm": hbm_roof(n * NTT_BYTES_PER_ELEM, ms, hbm, hbm_src)}
    # CNN batch: INTT of every polynomial, then full-width MSMs of its
    # coefficients (ceil(254 / c) windows at each length's window width).
    cnn_imad = 0
    for s_ in cnn_sizes:
        lg = int(s_).bit_length() - 1
        cnn_imad += ntt_imads(int(s_)) + int(s_) * (-(-254 // zk.zk_tune_get(ctx, zk.ZK_TUNE_MSM_WINDOW, lg))) * madd
    roofs["cnn_batch_commit"] = imad_roof(cnn_imad, per_op["cnn_batch_commit"]["ms"], rates)
    # Fold tree: witness passes (11 F_r products, 512 B per element), the
    # cross terms' INTTs and full-width MSMs; instance combinations excluded.
    folds, nf = tree.count - 1, tree.n
    wit_ms = phase_split["fold_tree_1024x2^16"].get("fold_witness", 0.0)
    c16 = zk.zk_tune_get(ctx, zk.ZK_TUNE_MSM_WINDOW, 16)
    tree_imad = folds * (nf * FOLD_MULS * IMAD_PER_MUL + ntt_imads(nf) + nf * (-(-254 // c16)) * madd)
    roofs["fold_tree_1024x2^16"] = imad_roof(tree_imad, per_op["fold_tree_1024x2^16"]["ms"], rates)
    if wit_ms:
        roofs["fold_witness_pass"] = {"imad": imad_roof(folds * nf * FOLD_MULS * IMAD_PER_MUL, wit_ms, rates),
                                      "hbm": hbm_roof(folds * nf * FOLD_BYTES, wit_ms, hbm, hbm_src),
                                      "ms_per_tree": wit_ms}

    # Dominant kernel: bucket accumulation of the uniform 2^20 MSM
    # (round 0, k_pieces_first, and the bucket completion after it).
    acc_ms, acc_cnt = phases["msm_accum"]
    adds = n20 * W * args.steps  # one mixed addition per nonzero signed digit
    acc = imad_roof(adds * madd, acc_ms, rates)
    roofline = dict(acc)
    roofline.update({
        "kernel": "MSM bucket accumulation (k_pieces_first + bucket completion), uniform 2^20, c=%d" % c20,
        "algorithmic": "%d mixed additions x 10 F_q products x 264 IMADs per MSM" % (n20 * W),
        "traffic": ACCUM_TRAFFIC, "traffic_kernel": "k_pieces_first (ncu, bytes per launch)",
        "ms_per_launch": acc_ms / max(acc_cnt, 1),
        "phase_ms_per_msm": {k: v[0] / args.steps for k, v in phases.items() if v[1]},
        "probes_per_s": rates,
    })

    # End to end through the C ABI with host buffers (pinned): H2D of the
    # scalars and D2H of the commitment inside the timed region.
    h_sc = torch.from_numpy(Z.fr_uniform(3, n20).view(np.int64)).pin_memory()
    h_out = torch.zeros(8, dtype=torch.int64).pin_memory()
    for _ in range(2):
        zk.zk_commit(ctx, h_sc, h_out)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(args.steps, 5)):
        s0 = time.perf_counter()
        zk.zk_commit(ctx, h_sc, h_out)
        e2e_t.append(time.perf_counter() - s0)
    e2e = {"value": whole_job_rate(n20, statistics.median(e2e_t), world, dist) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": n20 * 32, "d2h_bytes_per_step": 64,
           "call": "zk_commit(host scalars, host out)"}

    extras = {}
    if not args.no_extras:
        extras = run_extras(zk, ctx, dev, torch, cnn, cnn_sizes, cnn_out, tree, args)
    del tree

    cpu = None
    if rank == 0:
        r, dt, cores = oracle_msm_rate(1 << args.cpu_sample_log)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "affine double-and-add MSM of %d uniform scalars (SRS from seeded tau), %.1f s"
                         % (1 << args.cpu_sample_log, dt)}

    zk.zk_destroy(ctx)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded SplitMix64; SRS from seeded tau)",
        "config": {"workload": WORKLOAD, "srs": "2^22 points, window tables c=16 and per-length widths",
                   "routes": "evaluation-form commitments by INTT + MSM (the paper's encoding)",
                   "l2": "flushed (512 MiB write) before every op",
                   "parallelism": "replicas" if world > 1 else "single"},
        "ops": per_op, "phases_ms": phase_split, "roofline": roofline, "rooflines": roofs,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": sampler.summary(),
        "fold_tree_root_repeatable": same_tree, **extras,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


class FoldTree:
    """The fold-tree workload: 1024 leaf accumulators of n = 2^16 (m1, m2, m4
    int8 * 2^16, stream 9 * 2^20 + 4 j + i), level-major gammas, and a saved
    copy of the initialised leaves that restores them before each run."""

    def __init__(self, zk, ctx, dev, torch, count=1024, n=1 << 16):
        self.zk, self.ctx, self.torch = zk, ctx, torch
        self.count, self.n = count, n
        self.m = torch.zeros((count, 4, n, 4), dtype=torch.int64, device="cuda")
        self.e = torch.zeros((count, n, 4), dtype=torch.int64, device="cuda")
        self.x = torch.zeros((count, 44), dtype=torch.int64, device="cuda")
        for j in range(count):
            base = (9 << 20) + 4 * j
            self.m[j, 0].copy_(dev(Z.zkml_scalars(base, n)))
            self.m[j, 1].copy_(dev(Z.zkml_scalars(base + 1, n)))
            self.m[j, 3].copy_(dev(Z.zkml_scalars(base + 3, n)))
        self.descs = [zk.make_acc(self.m[j], self.e[j], self.x[j]) for j in range(count)]
        self.gam = dev(np.concatenate([Z.gammas(l, count >> l) for l in range(1, count.bit_length())]))
        self.root = (torch.zeros((4, n, 4), dtype=torch.int64, device="cuda"),
                     torch.zeros((n, 4), dtype=torch.int64, device="cuda"),
                     torch.zeros(44, dtype=torch.int64, device="cuda"))
        self.rdesc = zk.make_acc(*self.root)
        self.saved = None
        self.first_root = None

    def init_leaves(self):
        self.zk.zk_leaf_init(self.ctx, self.descs)
        self.saved = (self.m.clone(), self.e.clone(), self.x.clone())

    def restore(self):
        self.m.copy_(self.saved[0])
        self.e.copy_(self.saved[1])
        self.x.copy_(self.saved[2])

    def run(self):
        self.zk.zk_fold_tree(self.ctx, self.descs, self.gam, self.rdesc)
        if self.first_root is None:
            self.first_root = [r.clone() for r in self.root]

    def root_matches_last(self):
        return bool(self.first_root is not None and
                    all(self.torch.equal(a, b) for a, b in zip(self.first_root, self.root)))

    def plain(self):
        width, goff, span = self.count, 0, 2
        while span <= self.count:
            for j in range(width // 2):
                L = self.descs[j * span + span // 2 - 1]
                R = self.descs[j * span + span - 1]
                self.zk.zk_fold(self.ctx, L, R, self.gam[goff + j], R)
            goff += width // 2
            width //= 2
            span *= 2

    def last_slot(self):
        return (self.m[self.count - 1], self.e[self.count - 1], self.x[self.count - 1])


def run_extras(zk, ctx, dev, torch, cnn, cnn_sizes, cnn_out, tree, args):
    """Batched vs plain vs graph vs Lagrange route for the CNN batch and the
    fold tree, the small-task regime, openings, and the serving loop."""
    res = {}
    ref = cnn_out.clone()
    outp = torch.zeros_like(cnn_out)

    def plain():
        for i, v in enumerate(cnn):
            zk.zk_commit_batch(ctx, [v], outp[i:i + 1], flags=zk.ZK_EVALS)

    plain()
    torch.cuda.synchronize()
    tp = _time(torch, plain, 3)
    outl = torch.zeros_like(cnn_out)
    zk.zk_commit_batch(ctx, cnn, outl, flags=zk.ZK_LAGRANGE)  # builds the bases
    tl = _time(torch, lambda: zk.zk_commit_batch(ctx, cnn, outl, flags=zk.ZK_LAGRANGE), 3)
    outg = torch.zeros_like(cnn_out)
    plan = zk.zk_plan_commit_batch(ctx, cnn, outg, flags=zk.ZK_EVALS)
    tg = _time(torch, lambda: zk.zk_plan_launch(plan), 3)
    nodes = zk.zk_plan_nodes(plan)
    zk.zk_plan_destroy(plan)
    outgl = torch.zeros_like(cnn_out)
    plan = zk.zk_plan_commit_batch(ctx, cnn, outgl, flags=zk.ZK_LAGRANGE)
    tgl = _time(torch, lambda: zk.zk_plan_launch(plan), 3)
    zk.zk_plan_destroy(plan)
    tb = _time(torch, lambda: zk.zk_commit_batch(ctx, cnn, cnn_out, flags=zk.ZK_EVALS), 3)
    res["cnn_batch_commit"] = {"polys": len(cnn), "coeffs": int(cnn_sizes.sum()), "batched_ms": tb,
                               "plain_ms": tp, "graph_ms": tg, "graph_nodes": nodes,
                               "lagrange_batched_ms": tl, "lagrange_graph_ms": tgl, "speedup": tp / tb,
                               "identical": bool(torch.equal(ref, outp) and torch.equal(outg, ref)
                                                 and torch.equal(outl, ref) and torch.equal(outgl, ref))}
    # Fold tree: batched (the step's op) vs per-fold calls vs one graph, and
    # the Lagrange route; degree 3 on the Lagrange route.
    tree.restore()
    tree.run()
    root_b = [r.clone() for r in tree.root]
    tree.restore()
    tree.plain()
    tree.restore()
    torch.cuda.synchronize()
    t_plain = _time(torch, tree.plain, 1)
    same = all(torch.equal(a, b) for a, b in zip(tree.last_slot(), root_b))
    tree.restore()
    torch.cuda.synchronize()
    plan = zk.zk_plan_fold_tree(ctx, tree.descs, tree.gam, tree.rdesc)  # its warm-up consumes the leaves
    tree.restore()
    torch.cuda.synchronize()
    t_graph = _time(torch, lambda: zk.zk_plan_launch(plan), 1)
    same = same and all(torch.equal(a, b) for a, b in zip(tree.root, root_b))
    zk.zk_plan_destroy(plan)
    tree.restore()
    t_batched = _time(torch, tree.run, 1)
    zk.zk_set_commit_route(ctx, zk.ZK_ROUTE_LAGRANGE)
    m0 = tree.saved[0]
    tree.m.copy_(m0)
    zk.zk_leaf_init(ctx, tree.descs)  # builds the 2^16 basis
    torch.cuda.synchronize()
    t_leaf_l = _time(torch, lambda: zk.zk_leaf_init(ctx, tree.descs), 1)
    leaf_same = torch.equal(tree.x, tree.saved[2])
    tree.restore()
    tree.run()
    tree.restore()
    torch.cuda.synchronize()
    t_lag = _time(torch, tree.run, 1)
    same = same and leaf_same and all(torch.equal(a, b) for a, b in zip(tree.root, root_b))
    # Degree 3 (m1 o m2 o m3 - mu^2 m4 = e, two cross terms), Lagrange route:
    # m3 := the degree-2 leaves' fourth int8 vector; leaf init computes m4.
    zk.zk_set_fold_degree(ctx, 3)
    tree.m.copy_(m0)
    tree.m[:, 2].copy_(m0[:, 3])
    tree.e.zero_()
    zk.zk_leaf_init(ctx, tree.descs)
    tree.saved = (tree.m.clone(), tree.e.clone(), tree.x.clone())
    tree.run()
    tree.restore()
    torch.cuda.synchronize()
    t3 = _time(torch, tree.run, 1)
    zk.zk_set_fold_degree(ctx, 2)
    zk.zk_set_commit_route(ctx, zk.ZK_ROUTE_INTT)
    folds = tree.count - 1
    res["fold_tree"] = {"leaves": tree.count, "n": tree.n, "folds": folds,
                        "batched_ms": t_batched, "plain_ms": t_plain, "graph_ms": t_graph,
                        "batched_folds_per_s": folds / (t_batched * 1e-3),
                        "plain_folds_per_s": folds / (t_plain * 1e-3),
                        "graph_folds_per_s": folds / (t_graph * 1e-3), "speedup": t_plain / t_batched,
                        "lagrange_ms": t_lag, "lagrange_folds_per_s": folds / (t_lag * 1e-3),
                        "lagrange_leaf_commit_ms": t_leaf_l,
                        "degree3_lagrange_ms": t3, "degree3_lagrange_folds_per_s": folds / (t3 * 1e-3),
                        "identical": bool(same)}
    tree.m = tree.e = tree.x = tree.saved = None
    torch.cuda.empty_cache()
    res["small_tasks"] = run_small_tasks(zk, ctx, dev, torch)
    res["kzg_open_and_quotient"] = run_openings(zk, ctx, dev, torch)
    if args.serving_jobs > 0:
        zk.zk_set_commit_route(ctx, zk.ZK_ROUTE_LAGRANGE)
        res["serving"] = run_serving(zk, ctx, dev, torch, jobs=args.serving_jobs)
        res["serving"]["route"] = "lagrange"
        zk.zk_set_commit_route(ctx, zk.ZK_ROUTE_INTT)
        res["serving_intt"] = run_serving(zk, ctx, dev, torch, jobs=args.serving_jobs)
        res["serving_intt"]["route"] = "intt"
    return res


def run_small_tasks(zk, ctx, dev, torch, count=4096, seed=12):
    """Many tiny uneven tasks: 4096 evaluation vectors of 2^8 .. 2^12 (INTT +
    commit each), as per-task calls, one batched call, and one graph."""
    rng = np.random.default_rng(seed)
    sizes = (1 << rng.integers(8, 13, count)).astype(np.int64)
    vecs = [dev(Z.zkml_scalars(8_000_000 + i, int(s))) for i, s in enumerate(sizes)]
    outb = torch.zeros((count, 8), dtype=torch.int64, device="cuda")
    outp = torch.zeros_like(outb)
    outg = torch.zeros_like(outb)

    def plain():
        for i, v in enumerate(vecs):
            zk.zk_commit_batch(ctx, [v], outp[i:i + 1], flags=zk.ZK_EVALS)

    def batched():
        zk.zk_commit_batch(ctx, vecs, outb, flags=zk.ZK_EVALS)

    plain()
    batched()
    tp = _time(torch, plain, 3)
    tb = _time(torch, batched, 3)
    torch.cuda.synchronize()
    zk.zk_timing_read(ctx)
    zk.zk_timing_enable(ctx, True)
    batched()
    zk.zk_timing_enable(ctx, False)
    torch.cuda.synchronize()
    ph = {k: round(v[0], 3) for k, v in zk.zk_timing_read(ctx).items() if v[1]}
    plan = zk.zk_plan_commit_batch(ctx, vecs, outg, flags=zk.ZK_EVALS)
    tg = _time(torch, lambda: zk.zk_plan_launch(plan), 3)
    zk.zk_plan_destroy(plan)
    return {"tasks": count, "sizes": "2^8 .. 2^12 (uniform log2)", "coeffs": int(sizes.sum()),
            "plain_ms": tp, "batched_ms": tb, "graph_ms": tg, "batched_speedup": tp / tb, "batched_phase_ms": ph,
            "graph_vs_batched": tb / tg,
            "identical": bool(torch.equal(outb, outp) and torch.equal(outg, outb))}

def run_openings(zk, ctx, dev, torch, reps=5):
    """KZG opening (Sec. 2.1) at 2^20: one polynomial (division + MSM of the
    quotient), and a gamma-batched opening of 16 polynomials of 2^16 at one
    point.  Device time with CUDA events, inputs resident, L2 flushed."""
    n = 1 << 20
    c = dev(Z.fr_uniform(13, n + 1))
    pt = dev(Z.fr_uniform(14, 1)[0])
    y = torch.zeros(4, dtype=torch.int64, device="cuda")
    proof = torch.zeros(8, dtype=torch.int64, device="cuda")
    polys = [dev(Z.fr_uniform(15 + i, 1 << 16)) for i in range(16)]
    gamma = dev(Z.fr_uniform(40, 1)[0])
    ys = torch.zeros((16, 4), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(2):
            fn()
        ms = []
        for _ in range(reps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    zk.zk_timing_read(ctx)
    one = timed(lambda: zk.zk_open(ctx, c, pt, y, proof))
    zk.zk_timing_enable(ctx, True)
    zk.zk_open(ctx, c, pt, y, proof)
    torch.cuda.synchronize()
    ph = zk.zk_timing_read(ctx)
    zk.zk_timing_enable(ctx, False)
    msm_ms = sum(ph[k][0] for k in ("msm_sort", "msm_accum", "msm_reduce"))
    batch = timed(lambda: zk.zk_open_batch(ctx, polys, pt, gamma, ys, proof))
    # Mul / MatMul quotient (Sec. 4.4.1) of two 2^20 evaluation vectors:
    # six transforms of length 2^20, three pointwise passes, one MSM.
    a = dev(Z.zkml_scalars(41, n))
    b = dev(Z.fr_uniform(42, n))
    com = torch.zeros(8, dtype=torch.int64, device="cuda")
    mq = timed(lambda: zk.zk_mul_quotient(ctx, a, b, com))
    return {"open_2^20_ms": one, "open_2^20_msm_ms": msm_ms, "open_2^20_division_ms": one - msm_ms,
            "open_batch_16x2^16_ms": batch, "mul_quotient_2^20_ms": mq}


def run_serving(zk, ctx, dev, torch, jobs=1200, lanes=4, rate_hz=20.0):
    """Poisson stream (20 jobs/s) of the basic-block jobs of a 12-layer,
    width-768 transformer (sequence 128), inference after inference: each job
    commits to its witness (three int8 * 2^16 vectors, as a leaf accumulator)
    and folds it into the resident accumulator of its size.  Jobs reuse a pool
    of output buffers per size.  Latency = end - arrival; it splits into the
    submission delay (the driver loop was late), the wait in the server's
    queue (submit -> start) and the run on a lane (start -> end)."""
    import time as _t
    per_inf = [1 << lg for lg in Z.transformer_job_sizes()] * 12
    sizes = [per_inf[i % len(per_inf)] for i in range(jobs)]
    arrivals = Z.poisson_arrivals(10, len(sizes), rate_hz)
    pool = {}

    def new_acc(n):
        m = torch.zeros((4, n, 4), dtype=torch.int64, device="cuda")
        e = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
        x = torch.zeros(44, dtype=torch.int64, device="cuda")
        return (m, e, x), zk.make_acc(m, e, x)

    for n in sorted(set(sizes)):
        w = [dev(Z.zkml_scalars((11 << 24) + 4 * n.bit_length() + i, n)) for i in range(3)]
        (rm, re_, rx), rd = new_acc(n)
        for i, k in ((0, 0), (1, 1), (3, 2)):
            rm[i].copy_(w[k])
        zk.zk_leaf_init(ctx, [rd])
        slots = [(new_acc(n), new_acc(n)) for _ in range(lanes + 1)]
        pool[n] = {"w": w, "res": ((rm, re_, rx), rd), "slots": slots, "last": [None] * len(slots), "k": 0}
    gam = dev(Z.gammas(12, 1))
    torch.cuda.synchronize()
    srv = zk.zk_server_create(ctx, lanes=lanes, hbm_budget_bytes=150 << 30)
    tickets, delays = [], []
    keep = []
    t0 = _t.perf_counter()
    for n, at in zip(sizes, arrivals):
        now = _t.perf_counter() - t0
        if at > now:
            _t.sleep(at - now)
        p = pool[n]
        k = p["k"] % len(p["slots"])
        p["k"] += 1
        if p["last"][k] is not None:
            zk.zk_wait(srv, p["last"][k], 600000)
        (_, leaf), (_, out) = p["slots"][k]
        job = zk.make_job(n, p["w"], leaf, p["res"][1], out, gam)
        keep.append(job)
        delay = max(0.0, _t.perf_counter() - t0 - at)
        tk = zk.zk_submit(srv, job)
        p["last"][k] = tk
        tickets.append(tk)
        delays.append(delay * 1e3)
    infos = [zk.zk_wait(srv, t, 600000) for t in tickets]
    st = zk.zk_server_stats(srv)
    zk.zk_server_destroy(srv)
    ok = all(i.status == zk.ZK_JOB_DONE for i in infos)
    delay = np.array(delays)
    queue = np.array([i.start_ms - i.submit_ms for i in infos])
    run = np.array([i.end_ms - i.start_ms for i in infos])
    lat = delay + queue + run
    span_s = (max(i.end_ms for i in infos) - min(i.submit_ms for i in infos)) / 1e3

    def pct(a):
        return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "mean": float(a.mean())}

    by_size = {}
    for lg in sorted(set(n.bit_length() - 1 for n in sizes)):
        sel = np.array([n.bit_length() - 1 == lg for n in sizes])
        by_size[str(lg)] = {"jobs": int(sel.sum()), "run_p50_ms": float(np.percentile(run[sel], 50)),
                            "latency_p99_ms": float(np.percentile(lat[sel], 99))}
    worst = int(np.argmax(lat))
    return {"jobs": len(sizes), "rate_hz": rate_hz, "lanes": lanes, "all_done": ok,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "jobs_per_s": len(sizes) / span_s,
            "latency_ms": pct(lat), "submit_delay_ms": pct(delay), "queue_ms": pct(queue), "run_ms": pct(run),
            "worst_job": {"log2n": sizes[worst].bit_length() - 1, "queue_ms": float(queue[worst]),
                          "run_ms": float(run[worst]), "delay_ms": float(delay[worst])},
            "by_log2n": by_size, "peak_reserved_gb": st.peak_reserved_bytes / 2 ** 30,
            "budget_gb": 150, "sizes_log2": sorted(set(Z.transformer_job_sizes()))}


def _time(torch, fn, reps):
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


if __name__ == "__main__":
    main()
