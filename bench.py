"""Benchmark of the fused shallow-water MacCormack step on one GB300.

Workload (N=1): the 8192 x 8192 FP32 river reach (bed sloping 1e-3 along x
plus seeded smooth noise of amplitude 0.5 m, inflow 2 m^2/s west, free
outflow east, walls south/north, depth 1 m, n = 0.03, kappa = 0.25).  A bench
"step" is one full time step (all 16 sub-steps, the CFL reduction included)
over the whole grid.  The state read per step (1.07 GB) is larger than L2, so
no flush is needed between timed steps.

Printed: one JSON line with the driver contract's keys, plus the roofline of
the fused kernel against the measured HBM copy bandwidth, the FP64 CPU oracle
timed on the host cores on a bounded sample, an end-to-end number through
the C ABI with pinned host buffers, and SM clock samples taken during the
timed region.

The line's "forms" object measures the rest of the metric in the same
process (rank 0): the same river in FP64 (the fused sweep and the plain
two-kernel step), the 256-scenario batched ensemble (1000 steps in one
persistent graph-captured launch, with and without the dry-item skip) and
the discrete adjoint's cost against a forward run (512^2, 2000 steps, FP64
and FP32), with its own clock samples.

--impl reference times the FP64 CPU oracle on the host cores (bounded crop
of the same workload) and prints the same line with "impl": "reference".
Multi-GPU (torchrun, N ranks): N independent replicas, one per GPU
(the single-grid step has no data-path exchange to shard here), timed
between barriers, max over ranks.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX = NY = 8192
BYTES_PER_CELL_FP32 = 28  # read eta, u, v, z; write eta, u, v (4 B each)
WORKLOAD = "river reach 8192x8192 FP32, bed slope 1e-3 + seeded noise 0.5 m, inflow 2 m^2/s W, outflow E, walls S/N, n=0.03, kappa=0.25, CFL 0.5"
METRIC = "cell-updates/s"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "fused_step_river_fp32.md")
FUSED_SOURCES = ["paper_1309_1230_gb300/csrc/swe_fused.cuh", "paper_1309_1230_gb300/csrc/swe_cell.cuh",
                 "paper_1309_1230_gb300/csrc/swe_fused.cu"]


_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/', re.S)


def _code_only(src: str) -> str:
    """The source with comments removed and whitespace collapsed (string
    literals kept), so that a comment edit does not change the hash."""
    out = _TOKENS.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", src)
    return " ".join(out.split())


def sources_sha() -> str:
    """Hash of the fused kernel's code (comments and whitespace ignored)."""
    h = hashlib.sha256()
    for p in FUSED_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def recorded_traffic(rows_per_item: int):
    """DRAM bytes per launch of the fused step from the committed ncu summary,
    valid only while the kernel sources hash to the recorded value and for the
    rows per item the capture used."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    m = re.search(r"traffic_bytes_per_launch_8192_rows%d:\s*([0-9.eE+]+)" % rows_per_item, text)
    s = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != sources_sha():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        rows = [r for r in csv.reader(io.StringIO(getattr(self, "out", ""))) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_solver(case, precision, device=0):
    from paper_1309_1230_gb300 import swe
    s = swe.Solver(case["nx"], case["ny"], manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"],
                   q_in=case["q_in"], precision=precision, kernel=swe.SWE_KERNEL_FUSED, device=device)
    s.set_bed(case["z"])
    s.set_state(case["eta"], case["u"], case["v"])
    return s


def oracle_rate(case, nsteps: int, crop: int, threads: int):
    """FP64 oracle on a crop x crop window (west end, inflow boundary kept) for
    nsteps steps on `threads` host threads; returns cell-updates/s."""
    from oracle import oracle as O
    sl = (slice(0, crop), slice(0, crop))
    z = case["z"][sl].copy()
    p = O.Params(nx=crop, ny=crop, manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"], q_in=case["q_in"])
    e, u, v = O.prepare_state(p, z, case["eta"][sl], case["u"][sl], case["v"][sl])
    t = time.perf_counter()
    r = O.run(p, z, e, u, v, nsteps, nthreads=threads)
    dt = time.perf_counter() - t
    assert r.status == 0
    return crop * crop * nsteps / dt, dt


def slowest_rank_ms(local_ms: float, dist=None) -> float:
    """The largest per-rank duration (ms): the job takes as long as its slowest
    replica.  Single process when dist is None or not initialised."""
    if dist is None or not dist.is_initialized():
        return local_ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_rank: int, steps: int, local_ms: float, dist=None):
    """Whole-job cell-updates/s: the cells every rank advanced (weak scaling,
    one replica of the workload per rank) over the slowest rank's time;
    returns (rate, that time in ms)."""
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    ms = slowest_rank_ms(local_ms, dist)
    return world * cells_per_rank * steps / (ms / 1e3), ms


def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_fp64_steps(case, steps: int, device: int) -> dict:
    """The same river in FP64: the fused sweep and the plain one-thread-per-cell
    step (two kernels per step), each timed with CUDA events on its stream."""
    import torch
    from paper_1309_1230_gb300 import swe
    out = {}
    for name, kern in (("fused", swe.SWE_KERNEL_FUSED), ("plain", swe.SWE_KERNEL_PLAIN)):
        s = swe.Solver(case["nx"], case["ny"], manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"],
                       q_in=case["q_in"], precision=swe.SWE_FP64, kernel=kern, device=device)
        s.set_bed(case["z"])
        s.set_state(case["eta"], case["u"], case["v"])
        st = torch.cuda.ExternalStream(s.stream_handle(), device=device)
        s.step(2, want_info=False)
        e0, e1 = _events(st)
        torch.cuda.synchronize()
        e0.record(st)
        s.step(steps, want_info=False)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        cells = case["nx"] * case["ny"]
        out[name] = {"ms_per_step": ms, "value": cells / (ms / 1e3), "steps": steps}
        s.close()
    out["unit"] = METRIC
    out["workload"] = "the same river reach 8192x8192, FP64 state and arithmetic"
    out["roofline"] = {"bound": "fp64 alu", "note": "56 B/cell of state traffic; GB300's FP64 rate (~1.25 TFLOP/s) "
                       "bounds it, not HBM"}
    return out


def bench_batched(steps: int, device: int) -> dict:
    """The ensemble form: 256 dam breaks of uneven size (Nx, Ny ~ U{128..1024}),
    FP32, `steps` steps in one persistent cooperative launch captured in a CUDA
    graph; timed with CUDA events on the batch's stream, with the dry-item skip
    (default) and without it.  Every cell of every scenario counts."""
    import torch
    from paper_1309_1230_gb300 import inputs as I
    from paper_1309_1230_gb300 import swe
    cases = I.ensemble(256)
    cells = sum(c["nx"] * c["ny"] for c in cases)
    st = torch.cuda.Stream(device=device)
    peaks = measured_peaks()
    out = {"workload": "256 dam-break scenarios, Nx, Ny ~ U{128..1024}, n ~ U(0.01,0.05), H ~ U(2,10) m, "
                       "dry right half, FP32, one persistent graph-captured launch per call",
           "scenarios": len(cases), "cells": cells, "steps": steps, "unit": METRIC}
    for skip in (1, 0):
        b = swe.Batch([(c["nx"], c["ny"]) for c in cases], [c["manning_n"] for c in cases], kappa=cases[0]["kappa"],
                      dry_skip=skip, stream=st.cuda_stream, device=device)
        for i, c in enumerate(cases):
            b.set_bed(i, c["z"])
            b.set_state(i, c["eta"], c["u"], c["v"])
        b.step(steps, want_info=False)  # the first call of this length captures its graph
        for i, c in enumerate(cases):
            b.set_state(i, c["eta"], c["u"], c["v"])
        e0, e1 = _events(st)
        torch.cuda.synchronize()
        e0.record(st)
        b.step(steps, want_info=False)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rate = cells * steps / (ms / 1e3)
        achieved = BYTES_PER_CELL_FP32 * rate / 1e9
        key = "dry_skip" if skip else "no_dry_skip"
        out[key] = {"value": rate, "ms_per_call": ms, "rows_per_item": int(b.params.seg_rows) or 192,
                    "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": achieved / peaks["hbm_gbs"], "bytes_per_cell": BYTES_PER_CELL_FP32,
                                 "note": "algorithmic bytes of every cell, skipped dry cells included"
                                 if skip else "algorithmic bytes of every cell"}}
        b.close()
    out["value"] = out["dry_skip"]["value"]
    return out


def bench_adjoint(T: int, device: int) -> dict:
    """Cost of the discrete adjoint on the 512^2 adjoint workload: one
    swe_adjoint call over T steps (its own forward run with sqrt(T)
    checkpoints, the recomputation and the reverse sweep) against a plain
    T-step forward of the same context, wall clock with the device
    synchronised on both sides, FP64 and FP32.  The gauge records are
    synthetic (the cost does not depend on them)."""
    import numpy as np
    import torch
    from paper_1309_1230_gb300 import inputs as I
    from paper_1309_1230_gb300 import swe
    c = I.adjoint_case(512, 512)
    rng = np.random.Generator(np.random.PCG64(5))
    obs = c["eta"].ravel()[c["gauges"]][None, :] + 0.01 * rng.standard_normal((T, len(c["gauges"])))
    out = {"workload": f"adjoint: 512x512, {T} steps, 16 gauges, kappa 0, gradient w.r.t. n and eta0, "
                       f"ceil(sqrt(T)) = {int(np.ceil(np.sqrt(T)))} checkpoints", "steps": T}
    for name, prec in (("fp64", swe.SWE_FP64), ("fp32", swe.SWE_FP32)):
        def fresh():
            s = swe.Solver(512, 512, manning_n=0.03, kappa=0.0, precision=prec, device=device)
            s.set_bed(c["z"], np.full((512, 512), 0.03))
            s.set_state(c["eta"], c["u"], c["v"])
            return s
        s = fresh()
        s.step(T, want_info=False)  # warm-up: graphs captured, kernels loaded
        s.set_state(c["eta"], c["u"], c["v"])
        s.set_clock(0, 0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(T, want_info=False)
        torch.cuda.synchronize()
        fwd = time.perf_counter() - t0
        s.close()
        s = fresh()
        s.adjoint(T, c["gauges"], obs)  # warm-up
        s.set_state(c["eta"], c["u"], c["v"])
        s.set_clock(0, 0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.adjoint(T, c["gauges"], obs)
        torch.cuda.synchronize()
        adj = time.perf_counter() - t0
        s.close()
        out[name] = {"forward_s": fwd, "adjoint_s": adj, "cost_ratio": adj / fwd}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1309_1230_gb300 import inputs as I
    threads = os.cpu_count() or 1
    crop = 1024
    case = I.river(NX, NY)
    if args.warmup > 0:
        oracle_rate(case, min(args.warmup, 3), crop, threads)
    rate, secs = oracle_rate(case, args.steps, crop, threads)
    sample = f"FP64 oracle, {crop}x{crop} west-end window of the 8192^2 river, {args.steps} steps, OpenMP over rows"
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": f"{NX}x{NY}", "sample": sample},
            "cpu_baseline": {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP64, batched and adjoint measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1309_1230_gb300 import inputs as I
    from paper_1309_1230_gb300 import swe

    case = I.river(NX, NY)
    cells = NX * NY
    s = make_solver(case, swe.SWE_FP32, device=local)
    stream = torch.cuda.ExternalStream(s.stream_handle(), device=local)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- rows per work item from the autotuner (on the live state, which it restores)
    tuned_rows, tune_table = s.autotune(probe_steps=10)

    # ---- device-resident timing: W warm-up steps, then exactly K steps
    s.step(args.warmup, want_info=False)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        s.step(args.steps, want_info=False)
        ev1.record(stream)
        barrier()
    value, ms = job_rate(cells, args.steps, ev0.elapsed_time(ev1), dist)
    info = s.info()
    launch_ms = ms / args.steps  # one fused kernel per step (plus one tiny bookkeeping kernel per call)
    peaks = measured_peaks()
    achieved = BYTES_PER_CELL_FP32 * cells / (launch_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic(tuned_rows),
                "peak_source": peaks["source"], "bytes_per_cell": BYTES_PER_CELL_FP32,
                "kernel": "k_fused<float,2,...> (one launch per step)"}

    # ---- end to end through the C ABI: host (pinned) state in, K steps, state out
    e2e = None
    if not args.no_e2e:
        import ctypes
        import numpy as np
        pin = [torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in range(6)]
        for t_, a in zip(pin[:3], (case["eta"], case["u"], case["v"])):
            t_.numpy()[...] = a
        ptr = [ctypes.cast(t_.data_ptr(), ctypes.POINTER(ctypes.c_double)) for t_ in pin]
        lib = swe.load()
        barrier()
        t0 = time.perf_counter()
        st = lib.swe_set_state(s.ctx, ptr[0], ptr[1], ptr[2])
        st |= lib.swe_step(s.ctx, args.steps, None, None, None)
        st |= lib.swe_get_state(s.ctx, ptr[3], ptr[4], ptr[5])
        torch.cuda.synchronize()
        e2e_rate, _ = job_rate(cells, args.steps, (time.perf_counter() - t0) * 1e3, dist)
        assert st == 0, "e2e C-ABI calls failed"
        io_bytes = 3 * 8 * cells
        e2e = {"value": e2e_rate, "unit": METRIC,
               "h2d_bytes_per_step": io_bytes / args.steps, "d2h_bytes_per_step": io_bytes / args.steps,
               "calls": "swe_set_state(host f64) + swe_step(K) + swe_get_state(host f64), pinned buffers"}
        if not np.isfinite(pin[3].numpy()).all():
            raise RuntimeError("non-finite state after the e2e run")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, secs = oracle_rate(case, 60, 4096, threads)
        cpu = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle",
               "sample": f"FP64 oracle, 4096x4096 west-end window of the workload, 60 steps ({secs:.1f} s)"}

    forms = None
    if rank == 0 and not args.no_forms:
        with ClockSampler(local) as fclk:
            forms = {"fp32_step": {"value": value, "ms_per_step": ms / args.steps, "unit": METRIC},
                     "fp64_step": bench_fp64_steps(case, 5, local),
                     "batched": bench_batched(1000, local),
                     "adjoint": bench_adjoint(2000, local)}
        forms["fp64_step"]["fp32_over_fp64_fused"] = value / forms["fp64_step"]["fused"]["value"]
        forms["clocks"] = fclk.summary()

    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": f"{NX}x{NY}", "cells": cells, "precision": "FP32 state, FP64 dt and tallies",
                       "l2": "inputs larger than L2 (1.07 GB state read per step)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "rows_per_item": tuned_rows,
                       "autotune_ms_per_step": {str(k): round(v, 4) for k, v in tune_table.items()},
                       "t_end_s": info.t, "dt_last_s": info.dt_last},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "forms": forms,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"],
                       "samples": clocks["samples"]},
            "gpu_launches": args.steps + 1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
