"""How far the FP64 oracle itself moves when its input is rounded to binary32.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): it calls the oracle
alone, never the CUDA package.

The FP32 form stores eta, u, v and z in binary32, so even with exact
arithmetic its run starts from an input that differs from the FP64 run's by
up to half an ulp of binary32 per cell (~5e-7 m at 10 m).  This script runs
the oracle (FP64 throughout) from three inputs of the same workload:

  base     the FP64 input;
  rounded  eta and z rounded to binary32 (the FP32 form's input, nothing else);
  ulp      eta moved by one binary32 ulp in every wet cell, with a seeded
           random sign (a dry cell keeps eta = z);
  stored32 z rounded to binary32 once, and eta, u, v rounded to binary32
           after every step (FP64 arithmetic within a step, binary32
           storage between steps: the FP32 form's storage without its
           arithmetic);

and reports max and L2 of the depth difference against the base run, each
relative to the base run's maximum depth, plus the share of cells beyond
1e-4.  If moving the input by binary32 rounding alone moves the FP64 result
by ~1e-3 at the moving bores, a max-norm tolerance of 1e-4 is not a property
the scheme has in any precision, and the FP32 form can only be held to norms
that average over the bore positions (L2, the share of cells beyond 1e-4).

    python -m oracle.perturbation --n 2048 --steps 1000 --threads 16
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import oracle as O  # noqa: E402
from paper_1309_1230_gb300 import inputs as I  # noqa: E402


def round32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def ulp_move(a, seed):
    """a moved by one binary32 ulp toward +inf or -inf (seeded random sign)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a32 = np.asarray(a, dtype=np.float32)
    up = rng.integers(0, 2, a32.shape).astype(bool)
    moved = np.where(up, np.nextafter(a32, np.float32(np.inf)), np.nextafter(a32, np.float32(-np.inf)))
    return moved.astype(np.float64)


def depth_diff(h, h_base):
    scale = float(np.max(h_base))
    d = np.abs(h - h_base)
    return dict(max=float(d.max()) / scale, l2=float(np.sqrt(np.mean(d * d))) / scale,
                share_above_1e4=float(np.mean(d > 1e-4 * scale)), cells_above_1e4=int(np.sum(d > 1e-4 * scale)))


def run(n: int, steps: int, threads: int, seed: int = 1310, stored32: bool = True) -> dict:
    case = I.dam_break(n, n, seed=seed)
    p = O.Params(nx=n, ny=n, dx=case["dx"], dy=case["dy"], manning_n=case["manning_n"], kappa=case["kappa"],
                 bc=case["bc"], q_in=case["q_in"])
    out = dict(workload=f"dam break {n}x{n}, {steps} steps, FP64 oracle", steps=steps)
    inputs = {
        "base": (case["z"], case["eta"]),
        "rounded": (round32(case["z"]), round32(case["eta"])),
        "ulp": (case["z"], np.where(case["eta"] - case["z"] > 1e-3, ulp_move(case["eta"], 7), case["eta"])),
    }
    res = {}
    for name, (z, eta) in inputs.items():
        t0 = time.time()
        e0, u0, v0 = O.prepare_state(p, z, eta, case["u"], case["v"])
        r = O.run(p, z, e0, u0, v0, steps, nthreads=threads)
        assert r.status == 0, name
        res[name] = (r.eta - z, r.dt)
        out[f"seconds_{name}"] = round(time.time() - t0, 1)
    if stored32:
        t0 = time.time()
        z = round32(case["z"])
        e, u, v = O.prepare_state(p, z, round32(case["eta"]), case["u"], case["v"])
        dts = []
        for k in range(steps):
            r = O.run(p, z, e, u, v, 1, step0=k, nthreads=threads)
            assert r.status == 0
            e, u, v = round32(r.eta), round32(r.u), round32(r.v)
            dts.append(r.dt[0])
        res["stored32"] = (e - z, np.array(dts))
        out["seconds_stored32"] = round(time.time() - t0, 1)
    hb = res["base"][0]
    for name in [k for k in ("rounded", "ulp", "stored32") if k in res]:
        out[name] = depth_diff(res[name][0], hb)
        out[name]["dt_max_rel"] = float(np.max(np.abs(res[name][1] - res["base"][1]) / res["base"][1]))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.n, a.steps, a.threads), indent=1))


if __name__ == "__main__":
    main()
