"""The paper's two experiment shapes on the synthetic workloads, on one GPU.

    python -m paper_2510_24968_gb300.experiments diis --workload water
    python -m paper_2510_24968_gb300.experiments shards --workload cloud30 --nshards 1,2,4,8

diis: SCF energy error per iteration with DIIS (Algorithm 1, 8 stored pairs) and
without (plain Roothaan iteration), FP64 builds; the error is taken against
the DIIS run's converged energy (the shape of the paper's DIIS-vs-plain
convergence figure, Sec. 3.2.1).

shards: the Fock build split into bra-pair shards i % N (the partition a run on
N GPUs uses, Sec. 3.3.1), each shard timed on its own.  With one GPU per shard
the build takes the slowest shard plus one J/K all-reduce; the projected
strong-scaling speedup is T_1 / max_s T_s, so this measures the partition's
load balance, not an interconnect.

Every step runs in libfsim; this module draws the seeded density and prints
one JSON object.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from fsim_synth import workload

from .fsim import FSIM_FP64, FSIM_MIXED, Basis


def run_diis(a):
    gb = Basis(workload(a.workload))
    prec = FSIM_FP64 if a.precision == "fp64" else FSIM_MIXED
    runs = {}
    for name, m in (("diis", 8), ("plain", 0)):
        r = gb.scf(precision=prec, tau=a.tau, max_iter=a.max_iter, diis_size=m)
        runs[name] = r
    e_ref = runs["diis"]["e_total"]
    out = {"workload": a.workload, "nbf": gb.nbf, "precision": a.precision, "tau": a.tau, "e_ref": e_ref}
    for name, r in runs.items():
        err = np.abs(np.asarray(r["energies"]) - e_ref)
        out[name] = {"iters": r["iters"], "converged": bool(r["converged"]), "wall_s": r["time_s"],
                     "abs_error_per_iteration": [float(f"{x:.3e}") for x in err]}
    return out


def run_shards(a):
    import torch

    gb = Basis(workload(a.workload))
    gb.schwarz()
    N = gb.nbf
    Dn = np.random.default_rng(0).standard_normal((N, N)) * 0.02
    D = torch.from_numpy(Dn + Dn.T).cuda()
    J, K = torch.zeros_like(D), torch.zeros_like(D)
    out = {"workload": a.workload, "nbf": N, "tau": a.tau, "precision": "mixed", "runs": {}}
    t1 = None
    for ns in [int(x) for x in a.nshards.split(",")]:
        times, quartets = [], []
        for s in range(ns):
            kw = dict(tau=a.tau, precision=FSIM_MIXED, shard=s, nshards=ns)
            gb.fock_build(D, J, K, **kw)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(a.reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gb.fock_build(D, J, K, **kw)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            times.append(best)
            quartets.append(gb.last_quartet_count())
        if t1 is None:
            t1 = times[0] if ns == 1 else sum(times)
        tmax = max(times)
        out["runs"][ns] = {"shard_ms": [round(t, 3) for t in times], "shard_quartets": quartets,
                           "max_ms": tmax, "projected_speedup": t1 / tmax,
                           "projected_efficiency": t1 / tmax / ns,
                           "quartet_imbalance": max(quartets) / (sum(quartets) / ns)}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    d = sub.add_parser("diis")
    d.add_argument("--workload", default="water")
    d.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    d.add_argument("--tau", type=float, default=0.0)
    d.add_argument("--max-iter", type=int, default=100)
    s = sub.add_parser("shards")
    s.add_argument("--workload", default="water8")
    s.add_argument("--tau", type=float, default=1e-10)
    s.add_argument("--nshards", default="1,2,4,8")
    s.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    print(json.dumps(run_diis(a) if a.cmd == "diis" else run_shards(a)))


if __name__ == "__main__":
    main()
