"""Autotuner: per length, the MSM window width, the MSM bucket layout and the
largest NTT pass radix.

Each candidate is timed on the device by zk_tune_measure (synthetic data,
median of a few runs); the fastest is installed with zk_tune_set and all
results are written to a JSON table that `apply` installs in a later context:

    {"msm_window": {"16": {"best": 16, "ms": {...}}, ...},
     "msm_layout": {"chunk": {"20": {"best": 2, "ms": {...}}, ...}, "tail": ...,
                    "seg": ..., "segbig": ...},
     "ntt_radix": {"20": {"best": 10, "ms": {...}}, ...}}

The layout knobs (ZK_TUNE_MSM_CHUNK, _TAIL, _SEG, _SEGBIG) are swept one at
a time in that order, each with the winners of the earlier ones installed;
the library times CHUNK, TAIL and SEG on quantised int8 x 2^16 scalars (few,
full buckets) and SEGBIG on uniform ones.
"""
from __future__ import annotations

import json

from . import (ZK_TUNE_MSM_CHUNK, ZK_TUNE_MSM_SEG, ZK_TUNE_MSM_SEGBIG, ZK_TUNE_MSM_TAIL,
               ZK_TUNE_MSM_WINDOW, ZK_TUNE_NTT_RADIX, zk_srs_size, zk_tune_measure, zk_tune_set)

MSM_WINDOWS = range(9, 21)
NTT_RADIX = range(6, 12)
# knob name -> (op, candidate values)
MSM_LAYOUT = {"chunk": (ZK_TUNE_MSM_CHUNK, range(1, 5)), "tail": (ZK_TUNE_MSM_TAIL, range(1, 5)),
              "seg": (ZK_TUNE_MSM_SEG, range(3, 6)), "segbig": (ZK_TUNE_MSM_SEGBIG, range(6, 9))}


def tune(ctx: int, msm_logs=range(10, 23), ntt_logs=range(10, 23), reps: int = 3,
         windows=MSM_WINDOWS, radices=NTT_RADIX, path: str | None = None, layout_logs=(),
         layout=MSM_LAYOUT) -> dict:
    table = {"msm_window": {}, "msm_layout": {k: {} for k in layout}, "ntt_radix": {}}
    srs = zk_srs_size(ctx)
    for lg in msm_logs:
        if (1 << lg) > srs:
            continue
        res = {}
        for c in windows:
            # window widths far from the length waste bucket memory and time
            if c > lg + 2 or c < lg - 10:
                continue
            res[c] = zk_tune_measure(ctx, ZK_TUNE_MSM_WINDOW, lg, c, reps)
        best = min(res, key=res.get)
        zk_tune_set(ctx, ZK_TUNE_MSM_WINDOW, lg, best)
        table["msm_window"][str(lg)] = {"best": best, "ms": {str(k): v for k, v in res.items()}}
    for lg in layout_logs:
        if (1 << lg) > srs:
            continue
        for name, (op, values) in layout.items():
            res = {v: zk_tune_measure(ctx, op, lg, v, reps) for v in values}
            best = min(res, key=res.get)
            zk_tune_set(ctx, op, lg, best)
            table["msm_layout"][name][str(lg)] = {"best": best, "ms": {str(k): v for k, v in res.items()}}
    for lg in ntt_logs:
        res = {}
        for r in radices:
            if r > lg or -(-lg // r) > 4:
                continue
            res[r] = zk_tune_measure(ctx, ZK_TUNE_NTT_RADIX, lg, r, reps)
        if not res:
            continue
        best = min(res, key=res.get)
        zk_tune_set(ctx, ZK_TUNE_NTT_RADIX, lg, best)
        table["ntt_radix"][str(lg)] = {"best": best, "ms": {str(k): v for k, v in res.items()}}
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    return table


def apply(ctx: int, table) -> None:
    """Installs a table produced by `tune` (a dict or a JSON file path)."""
    if isinstance(table, str):
        with open(table) as f:
            table = json.load(f)
    for lg, e in table.get("msm_window", {}).items():
        zk_tune_set(ctx, ZK_TUNE_MSM_WINDOW, int(lg), int(e["best"]))
    for lg, e in table.get("ntt_radix", {}).items():
        zk_tune_set(ctx, ZK_TUNE_NTT_RADIX, int(lg), int(e["best"]))
    for name, per in table.get("msm_layout", {}).items():
        for lg, e in per.items():
            zk_tune_set(ctx, MSM_LAYOUT[name][0], int(lg), int(e["best"]))
