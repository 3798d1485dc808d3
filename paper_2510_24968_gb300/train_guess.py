"""Train the learned initial density and measure what it gains.

    python -m paper_2510_24968_gb300.train_guess --train 400 --test 20 --steps 3000 --out result.json

Training set: seeded (H2O)_k clusters, k = 2..6 in turn (geometry seeds
10^6 + i, the (H2O)_8 workload's per-element basis), converged by the
library's SCF; test set: held-out (H2O)_8 clusters (seeds 2*10^6 + i).  For
each test molecule the SCF runs from the core-Hamiltonian guess and from the
network's guess inside fsim_scf (FSIM_GUESS_LEARNED; mixed precision with
the default double-float resets, tau 1e-10); reported:
iterations, time to an energy within 1e-8 Eh of the core-guess run's final
energy, the energy difference, and how often the guess failed its
trace/idempotency check (fallback to core-H).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from fsim_synth import water_cluster

from . import FSIM_MIXED, Basis
from .guess import GuessNet, train, train_data_parallel, training_data, training_data_batched


def time_to(res, e_ref, tol=1e-8):
    E, T = res["energies"], res["times"]
    for i in range(len(E)):
        if all(abs(e - e_ref) < tol for e in E[i:]):
            return float(T[i])
    return None


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained weights (fsim_mlp_save) here")
    ap.add_argument("--batched", action="store_true", help="converge the training clusters with fsim_scf_batched")
    a = ap.parse_args(argv)
    import os
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = 0
    if world > 1:
        # data parallel: one rank per GPU (torch.distributed.run), each with its
        # share of the training clusters; gradients combined every step
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", 0))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        rank = dist.get_rank()
    t0 = time.time()
    mols = [water_cluster(2 + i % 5, geom_seed=10**6 + i) for i in range(a.train) if i % world == rank]
    X, T, M, e_train = training_data_batched(mols) if a.batched else training_data(mols)
    t_data = time.time() - t0
    net = GuessNet(seed=3)
    t0 = time.time()
    if world > 1:
        ls = train_data_parallel(net, X, T, M, steps=a.steps, batch=a.batch, lr0=1e-3)
        losses = [(0, ls[0]), (a.steps - 1, ls[-1])]
    else:
        losses = train(net, X, T, M, steps=a.steps, batch=a.batch, lr0=1e-3, log_every=max(1, a.steps // 10))
    t_train = time.time() - t0
    if a.save and rank == 0:
        net.save(a.save)
    if rank != 0:
        return None
    import tempfile
    wpath = a.save or os.path.join(tempfile.mkdtemp(), "guess.fsimmlp")
    if not a.save:
        net.save(wpath)
    rows = []
    for i in range(a.test):
        b = Basis(water_cluster(8, geom_seed=2 * 10**6 + i))
        core = b.scf(precision=FSIM_MIXED, tau=1e-10)
        # the learned guess inside fsim_scf (features, network, assembly, check);
        # both times to energy include the guess (core-H: its diagonalisation)
        lrn = b.scf(precision=FSIM_MIXED, tau=1e-10, guess_model=wpath)
        ct, lt = time_to(core, core["e_total"]), time_to(lrn, core["e_total"])
        rows.append({"core_iters": core["iters"], "learned_iters": lrn["iters"], "fallback": lrn["guess_fallback"],
                     "de": lrn["e_total"] - core["e_total"],
                     "core_tte": None if ct is None else ct + core["guess_s"],
                     "learned_tte": None if lt is None else lt + lrn["guess_s"], "predict_s": lrn["guess_s"],
                     "converged": core["converged"] and lrn["converged"]})
    ok = [r for r in rows if r["converged"]]
    summary = {
        "train_clusters": a.train, "train_converged": len(e_train), "train_pairs": int(X.shape[0]), "steps": a.steps, "data_s": t_data,
        "train_s": t_train, "loss_first_last": [losses[0][1], losses[-1][1]], "test_molecules": a.test,
        "converged_both": len(ok),
        "mean_iters_core": float(np.mean([r["core_iters"] for r in ok])),
        "mean_iters_learned": float(np.mean([r["learned_iters"] for r in ok])),
        "mean_tte_core_s": float(np.mean([r["core_tte"] for r in ok if r["core_tte"]])),
        "mean_tte_learned_s": float(np.mean([r["learned_tte"] for r in ok if r["learned_tte"]])),
        "mean_guess_s_learned": float(np.mean([r["predict_s"] for r in rows])),
        "max_abs_de_eh": float(max(abs(r["de"]) for r in ok)),
        "fallback_rate": float(np.mean([r["fallback"] for r in rows])),
        "rows": rows,
    }
    print(json.dumps({k: v for k, v in summary.items() if k != "rows"}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(summary, f, indent=1)
    return summary


if __name__ == "__main__":
    main()
