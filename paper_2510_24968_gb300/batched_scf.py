"""Batched lockstep RHF over a seeded set of organic-like clouds.

    python -m paper_2510_24968_gb300.batched_scf --nmol 64 --nmin 3 --nmax 8

Draws `nmol` molecules with U{nmin..nmax} heavy atoms (fsim_synth.batched_set),
runs fsim_scf_batched on them (mixed precision by default) and prints one JSON
object: wall time, molecules/s, converged count, p50/p99 of the per-molecule
times (all molecules, and the converged ones), the mean iteration count, how
many molecules ran FP64-accurate builds because their overlap's smallest
eigenvalue is below FSIM_MIXED_MIN_S_EIG, the set-up inside the call (one-electron
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


def partition(costs, world: int):
    """Molecules over ranks, heaviest first onto the least loaded rank (the
    molecules are independent: no exchange until the results are gathered)."""
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: -costs[k]):
        r = min(range(world), key=lambda q: load[q])
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def run_sharded(mols, solve, cost=lambda m: float(m.nbf) ** 4):
    """Batched SCF over the ranks of the default process group: rank r solves
    its share (solve(list of molecules) -> list of per-molecule results) and
    the results are gathered back into the input order on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank() if world > 1 else 0
    parts = partition([cost(m) for m in mols], world)
    mine = parts[rank]
    res = solve([mols[i] for i in mine]) if mine else []
    if world == 1:
        return res
    got = [None] * world
    dist.all_gather_object(got, list(zip(mine, res)))
    out = [None] * len(mols)
    for chunk in got:
        for i, r in chunk:
            out[i] = r
    return out


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
    ap.add_argument("--dw-screen", action="store_true", help="density-weighted screening of the increments")
    ap.add_argument("--indices", default=None,
                    help="comma-separated members of the set to run (per-molecule rows are printed)")
    a = ap.parse_args(argv)

    mols = batched_set(a.nmol, seed=a.seed, nmin=a.nmin, nmax=a.nmax)
    if a.indices:
        idx = [int(x) for x in a.indices.split(",")]
        prec = FSIM_MIXED if a.precision == "mixed" else FSIM_FP64
        bases = [Basis(mols[i]) for i in idx]
        res = scf_batched(bases, precision=prec, tau=a.tau, final_fp64=not a.no_fp64_reset, max_iter=a.max_iter,
                          dw_screen=a.dw_screen)
        for i, b, r in zip(idx, bases, res):
            print(json.dumps({"index": i, "nbf": b.nbf, "converged": r["converged"], "iters": r["iters"],
                              "e_total": r["e_total"], "last_de": float(np.abs(np.diff(r["energies"][-3:])).max())
                              if len(r["energies"]) > 2 else None, "min_s_eig": r["min_s_eig"],
                              "mixed_fallback": r["mixed_fallback"]}))
        return
    import os
    if int(os.environ.get("WORLD_SIZE", 1)) > 1:
        return main_sharded(a, mols)
    t0 = time.perf_counter()
    bases = [Basis(m) for m in mols]
    for b in bases:
        b.schwarz()
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    prec = FSIM_MIXED if a.precision == "mixed" else FSIM_FP64
    t0 = time.perf_counter()
    res = scf_batched(bases, precision=prec, tau=a.tau, final_fp64=not a.no_fp64_reset, max_iter=a.max_iter,
                      dw_screen=a.dw_screen)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ts = sorted(r["time_s"] for r in res)
    tc = sorted(r["time_s"] for r in res if r["converged"])
    # lockstep: every molecule still iterating shares the iteration end times
    th = max((r["times"] for r in res), key=len)
    print(json.dumps({
        "nmol": a.nmol, "heavy_atoms": [a.nmin, a.nmax], "nbf_range": [min(b.nbf for b in bases),
                                                                     max(b.nbf for b in bases)],
        "precision": a.precision, "fp64_reset": not a.no_fp64_reset, "dw_screen": a.dw_screen, "tau": a.tau,
        "setup_s": setup,
        "wall_s": wall, "molecules_per_s": a.nmol / wall, "converged": sum(r["converged"] for r in res),
        "p50_s": ts[len(ts) // 2], "p99_s": ts[min(len(ts) - 1, int(0.99 * len(ts)))],
        "p50_converged_s": tc[len(tc) // 2] if tc else None,
        "p99_converged_s": tc[min(len(tc) - 1, int(0.99 * len(tc)))] if tc else None,
        "mixed_fallback": int(sum(r["mixed_fallback"] for r in res)),
        "min_s_eig_p50": float(np.median([r["min_s_eig"] for r in res])),
        "mean_iters": float(np.mean([r["iters"] for r in res])),
        "fp64_builds": int(sum(r["fp64_builds"] for r in res)),
        "in_call_setup_s": wall - float(th[-1]) if len(th) else None,
        "iteration_s": [float(x) for x in np.diff(np.concatenate([[0.0], th]))],
    }))


def main_sharded(a, mols):
    """One rank per GPU (torch.distributed.run): each rank runs the batched SCF
    of its share of the molecules; rank 0 prints the gathered summary with the
    slowest rank's wall time."""
    import os

    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = FSIM_MIXED if a.precision == "mixed" else FSIM_FP64

    def solve(ms):
        bases = [Basis(m) for m in ms]
        return scf_batched(bases, precision=prec, tau=a.tau, final_fp64=not a.no_fp64_reset, max_iter=a.max_iter,
                           dw_screen=a.dw_screen)

    dist.barrier()
    t0 = time.perf_counter()
    res = run_sharded(mols, lambda ms: [{k: v for k, v in r.items() if k in ("e_total", "iters", "converged", "time_s")}
                                        for r in solve(ms)])
    wall = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
    dist.all_reduce(wall, op=dist.ReduceOp.MAX)
    if dist.get_rank() == 0:
        ok = [r for r in res if r["converged"]]
        ts = sorted(r["time_s"] for r in ok) or [float("nan")]
        print(json.dumps({"nmol": a.nmol, "ranks": dist.get_world_size(), "wall_s": wall.item(),
                          "molecules_per_s": a.nmol / wall.item(), "converged": len(ok),
                          "p50_s_converged": ts[len(ts) // 2],
                          "p99_s_converged": ts[min(len(ts) - 1, int(0.99 * len(ts)))]}))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
