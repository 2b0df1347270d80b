"""Times the FP64 oracle on the host cores for the small workloads: the 64^2
basin for its full 200 steps on one thread (the "oracle in seconds" case),
and the 2048^2 dam break and a 4096^2 window of the 8192^2 river for a few
steps on every core (OpenMP over rows).  Prints one JSON line per case.

This is test infrastructure: it runs the oracle only, to state what the CPU
reference costs on the machine at hand.

    python -m oracle.timing
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _time(O, case, steps, threads, crop=None):
    nx, ny = case["nx"], case["ny"]
    z, e, u, v = case["z"], case["eta"], case["u"], case["v"]
    if crop:
        sl = (slice(0, crop), slice(0, crop))
        nx = ny = crop
        z, e, u, v = z[sl].copy(), e[sl], u[sl], v[sl]
    p = O.Params(nx=nx, ny=ny, manning_n=case["manning_n"], kappa=case["kappa"], bc=case["bc"], q_in=case["q_in"])
    e0, u0, v0 = O.prepare_state(p, z, e, u, v)
    t = time.perf_counter()
    r = O.run(p, z, e0, u0, v0, steps, nthreads=threads)
    secs = time.perf_counter() - t
    assert r.status == 0
    return {"cells": nx * ny, "steps": steps, "threads": threads, "seconds": secs,
            "cell_updates_per_s": nx * ny * steps / secs}


def main():
    from oracle import oracle as O
    from paper_1309_1230_gb300 import inputs as I
    cores = os.cpu_count() or 1
    cases = [
        ("basin 64x64, 200 steps, one thread", I.basin_hump(64, 64, manning_n=0.03, kappa=0.25), 200, 1, None),
        ("dam break 2048x2048, 20 steps, all cores", I.dam_break(2048, 2048), 20, cores, None),
        ("river 8192x8192, 4096x4096 west window, 20 steps, all cores", I.river(8192, 8192), 20, cores, 4096),
    ]
    for name, case, steps, threads, crop in cases:
        print(json.dumps({"case": name, **_time(O, case, steps, threads, crop)}), flush=True)


if __name__ == "__main__":
    main()
