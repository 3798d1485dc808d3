"""Batched lockstep RHF over a seeded set of organic-like clouds.

    python -m paper_2510_24968_gb300.batched_scf --nmol 64 --nmin 3 --nmax 8

Draws `nmol` molecules with U{nmin..nmax} heavy atoms (fsim_synth.batched_set),
runs fsim_scf_batched on them (mixed precision by default) and prints one JSON
object: wall time, molecules/s, converged count, p50/p99 of the per-molecule
times, the mean iteration count, the set-up inside the call (one-electron
matrices, orthogonalisers, guesses, batch plans) and the length of each lockstep
iteration.  Every step runs in libfsim.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from fsim_synth import batched_set

from .fsim import FSIM_FP64, FSIM_MIXED, Basis, scf_batched


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nmol", type=int, default=64)
    ap.add_argument("--nmin", type=int, default=3)
    ap.add_argument("--nmax", type=int, default=8)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--tau", type=float, default=1e-11)
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-fp64-reset", action="store_true", help="mixed without the final FP64 builds")
    a = ap.parse_args(argv)

    mols = batched_set(a.nmol, seed=a.seed, nmin=a.nmin, nmax=a.nmax)
    t0 = time.perf_counter()
    bases = [Basis(m) for m in mols]
    for b in bases:
        b.schwarz()
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    prec = FSIM_MIXED if a.precision == "mixed" else FSIM_FP64
    t0 = time.perf_counter()
    res = scf_batched(bases, precision=prec, tau=a.tau, final_fp64=not a.no_fp64_reset, max_iter=a.max_iter)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ts = sorted(r["time_s"] for r in res)
    # lockstep: every molecule still iterating shares the iteration end times
    th = max((r["times"] for r in res), key=len)
    print(json.dumps({
        "nmol": a.nmol, "heavy_atoms": [a.nmin, a.nmax], "nbf_range": [min(b.nbf for b in bases),
                                                                     max(b.nbf for b in bases)],
        "precision": a.precision, "fp64_reset": not a.no_fp64_reset, "tau": a.tau, "setup_s": setup,
        "wall_s": wall, "molecules_per_s": a.nmol / wall, "converged": sum(r["converged"] for r in res),
        "p50_s": ts[len(ts) // 2], "p99_s": ts[min(len(ts) - 1, int(0.99 * len(ts)))],
        "mean_iters": float(np.mean([r["iters"] for r in res])),
        "fp64_builds": int(sum(r["fp64_builds"] for r in res)),
        "in_call_setup_s": wall - float(th[-1]) if len(th) else None,
        "iteration_s": [float(x) for x in np.diff(np.concatenate([[0.0], th]))],
    }))


if __name__ == "__main__":
    main()
