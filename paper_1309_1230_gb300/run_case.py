"""Run one synthetic workload for a few steps through the C ABI.

Used for profiler captures and quick throughput checks, e.g.

    python -m paper_1309_1230_gb300.run_case --case river --n 4096 --steps 4
    python -m paper_1309_1230_gb300.run_case --case dambreak --n 2048 --precision fp64 --kernel plain
    python -m paper_1309_1230_gb300.run_case --case ensemble --count 64 --steps 100
    python -m paper_1309_1230_gb300.run_case --case adjoint --n 512 --steps 20 --precision fp32

(the ensemble case runs the batched FP32 form: --count dam breaks with sides
U{128..min(n, 1024)}, all --steps in one persistent launch; the adjoint case
runs swe_adjoint over --steps steps on the n x n adjoint workload, synthetic
gauge records, and prints its wall time)

Prints one line with the step time measured with CUDA events.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="river", choices=["river", "dambreak", "basin", "ensemble", "adjoint"])
    ap.add_argument("--count", type=int, default=256, help="ensemble: number of scenarios")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--kernel", default="fused",
                    choices=["fused", "plain", "paper", "paper_devdt", "paper_shared", "paper_shared_devdt"])
    ap.add_argument("--seg-rows", type=int, default=0, help="rows per work item (0: automatic)")
    ap.add_argument("--dry-skip", type=int, default=1, choices=[0, 1], help="skip all-dry work items")
    ap.add_argument("--kappa", type=float, default=None, help="S15 coefficient (default: the case's)")
    ap.add_argument("--friction", type=int, default=0, choices=[0, 1], help="1: explicit friction (ablation)")
    ap.add_argument("--dissipation", type=int, default=0, choices=[0, 1], help="1: the TVD term (ablation)")
    a = ap.parse_args(argv)

    import torch

    from . import inputs as I
    from . import swe

    if a.case == "ensemble":
        return run_ensemble(a)
    if a.case == "adjoint":
        return run_adjoint(a)
    if a.case == "river":
        case = I.river(a.n, a.n)
    elif a.case == "dambreak":
        case = I.dam_break(a.n, a.n)
    else:
        case = I.basin_hump(a.n, a.n, manning_n=0.03, kappa=0.25)
    prec = swe.SWE_FP32 if a.precision == "fp32" else swe.SWE_FP64
    kern = {"fused": swe.SWE_KERNEL_FUSED, "plain": swe.SWE_KERNEL_PLAIN, "paper": swe.SWE_KERNEL_PAPER,
            "paper_devdt": swe.SWE_KERNEL_PAPER_DEVDT, "paper_shared": swe.SWE_KERNEL_PAPER_SHARED,
            "paper_shared_devdt": swe.SWE_KERNEL_PAPER_SHARED_DEVDT}[a.kernel]
    kappa = case["kappa"] if a.kappa is None else a.kappa
    s = swe.Solver(case["nx"], case["ny"], manning_n=case["manning_n"], kappa=kappa, bc=case["bc"],
                   q_in=case["q_in"], precision=prec, kernel=kern, seg_rows=a.seg_rows, dry_skip=a.dry_skip,
                   friction=a.friction, dissipation=a.dissipation)
    s.set_bed(case["z"])
    s.set_state(case["eta"], case["u"], case["v"])
    s.step(a.warmup, want_info=False)
    stream = torch.cuda.ExternalStream(s.stream_handle())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(a.steps, want_info=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, a.steps)
    info = s.info()
    print(json.dumps({"case": a.case, "n": a.n, "precision": a.precision, "kernel": a.kernel, "steps": a.steps,
                      "seg_rows": a.seg_rows, "dry_skip": a.dry_skip, "kappa": kappa, "friction": a.friction,
                      "dissipation": a.dissipation,
                      "ms_per_step": ms, "cell_updates_per_s": case["nx"] * case["ny"] / (ms / 1e3),
                      "volume": info.volume, "t": info.t, "time": time.time()}))
    s.close()


def run_ensemble(a):
    import torch

    from . import inputs as I
    from . import swe

    cases = I.ensemble(a.count, side=(128, min(max(a.n, 128), 1024)))
    st = torch.cuda.Stream()
    b = swe.Batch([(c["nx"], c["ny"]) for c in cases], [c["manning_n"] for c in cases], kappa=cases[0]["kappa"],
                  seg_rows=a.seg_rows, dry_skip=a.dry_skip, stream=st.cuda_stream)
    for i, c in enumerate(cases):
        b.set_bed(i, c["z"])
        b.set_state(i, c["eta"], c["u"], c["v"])
    b.step(a.warmup, want_info=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    b.step(a.steps, want_info=False)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cells = sum(c["nx"] * c["ny"] for c in cases)
    print(json.dumps({"case": "ensemble", "count": a.count, "cells": cells, "steps": a.steps, "dry_skip": a.dry_skip,
                      "ms_per_call": ms, "cell_updates_per_s": cells * a.steps / (ms / 1e3), "time": time.time()}))
    b.close()


def run_adjoint(a):
    import numpy as np
    import torch

    from . import inputs as I
    from . import swe

    c = I.adjoint_case(a.n, a.n)
    prec = swe.SWE_FP32 if a.precision == "fp32" else swe.SWE_FP64
    rng = np.random.Generator(np.random.PCG64(5))
    obs = c["eta"].ravel()[c["gauges"]][None, :] + 0.01 * rng.standard_normal((a.steps, len(c["gauges"])))
    s = swe.Solver(a.n, a.n, manning_n=0.03, kappa=0.0, precision=prec)
    s.set_bed(c["z"], np.full((a.n, a.n), 0.03))
    s.set_state(c["eta"], c["u"], c["v"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, gn, ge, gz = s.adjoint(a.steps, c["gauges"], obs, with_bed=True)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    print(json.dumps({"case": "adjoint", "n": a.n, "precision": a.precision, "steps": a.steps, "seconds": secs,
                      "loss": loss, "time": time.time()}))
    s.close()


if __name__ == "__main__":
    main()
