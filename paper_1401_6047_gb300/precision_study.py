"""Per-result error of the FP32-mixed path against the FP64 path on the GPU.

Usage: python -m paper_1401_6047_gb300.precision_study [c1|c2|c3|table1 ...] [--periods P]

For each configuration both precisions run the same protocol through the
C ABI; the line printed per configuration gives the absorption, the
time-averaged drift velocity and the largest |norm - 1| of each precision
and the absolute differences.  The FP64 path is the reference here: it
matches the FP64 oracle to 1e-10 relative on the configurations the tests
can afford (tests/test_gpu_parity.py).
"""
from __future__ import annotations

import argparse
import json
import time

from . import bte
from . import workloads as W

CONFIGS = {"c1": W.c1_fp64, "c2": W.c2, "c3": W.c3, "table1": W.paper_table1}


def study(name: str, periods: float = 0.0) -> dict:
    p = CONFIGS[name]()
    if periods:
        if p.omega > 0:
            p = p.replace(periods=periods, avg_window=min(p.avg_window, periods))
        else:
            p = p.replace(t_max=periods, avg_window=min(p.avg_window, periods))
    out = {"config": name, "n_max": p.n_max, "m_points": p.m_points}
    res = {}
    for prec, tag in ((W.FP64, "fp64"), (W.FP32_MIXED, "fp32")):
        t0 = time.perf_counter()
        o = bte.solve(p.replace(precision=prec))
        res[tag] = o
        out[tag] = {"absorption": o.absorption, "v_dc": o.v_dc_avg,
                    "norm_max_abs_err": o.norm_max_abs_err, "steps": o.steps_total,
                    "seconds": time.perf_counter() - t0}
    out["abs_err_absorption"] = abs(res["fp32"].absorption - res["fp64"].absorption)
    out["abs_err_v_dc"] = abs(res["fp32"].v_dc_avg - res["fp64"].v_dc_avg)
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("configs", nargs="*", default=["c1", "c2"])
    ap.add_argument("--periods", type=float, default=0.0,
                    help="shorter runs (drive periods, or time units when omega = 0)")
    args = ap.parse_args()
    for name in args.configs:
        print(json.dumps(study(name, args.periods)), flush=True)


if __name__ == "__main__":
    main()
