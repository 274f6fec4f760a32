"""Autotuner: per length, the MSM window width and the largest NTT pass radix.

Each candidate is timed on the device by zk_tune_measure (synthetic data,
median of a few runs); the fastest is installed with zk_tune_set and all
results are written to a JSON table that `apply` installs in a later context:

    {"device": ..., "msm_window": {"16": {"best": 16, "ms": {...}}, ...},
     "ntt_radix": {"20": {"best": 10, "ms": {...}}, ...}}
"""
from __future__ import annotations

import json

from . import (ZK_TUNE_MSM_WINDOW, ZK_TUNE_NTT_RADIX, zk_srs_size, zk_tune_measure,
               zk_tune_set)

MSM_WINDOWS = range(9, 21)
NTT_RADIX = range(6, 12)


def tune(ctx: int, msm_logs=range(10, 23), ntt_logs=range(10, 23), reps: int = 3,
         windows=MSM_WINDOWS, radices=NTT_RADIX, path: str | None = None) -> dict:
    table = {"msm_window": {}, "ntt_radix": {}}
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
