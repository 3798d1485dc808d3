"""Writes config3_oracle.json: the oracle's RHF energies of sampled molecules of
the batched workload (512 organic-like clouds of 3..30 heavy atoms,
fsim_synth.batched_set(512)): the 4 smallest, and 4 drawn at random (seeded)
among those with at most 5 heavy atoms.  The plain CPU oracle builds J/K over
N^4 quartets, so larger members of the set take it hours per SCF; the bound
keeps this script to about an hour on a few cores.

    python -m tests.golden.make_config3_oracle [--threads N]

Only oracle/ and fsim_synth/ are used.  Same SCF settings as the library's
batched SCF: core-H guess, DIIS (8), |dE| < 1e-10 and rms(dD) < 1e-7, Schwarz
tau 1e-11, at most 150 iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from fsim_synth import SplitMix64, batched_set
from oracle import OracleBasis, rhf

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_oracle.json")
TAU = 1e-11


def sample(mols):
    sizes = [m.nbf for m in mols]
    smallest = [int(i) for i in np.argsort(sizes, kind="stable")[:4]]
    pool = [i for i, m in enumerate(mols) if sum(1 for z in m.Z if z > 1) <= 5 and i not in smallest]
    rng = SplitMix64(2024)
    rng.shuffle(pool)
    return smallest, sorted(pool[:4])


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args(argv)
    mols = batched_set(512)
    smallest, rand = sample(mols)
    rows = []
    for kind, idx in (("smallest", smallest), ("random_le5_heavy", rand)):
        for i in idx:
            m = mols[i]
            ob = OracleBasis(m)
            S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
            t0 = time.time()
            r = rhf(S, H, lambda D: ob.jk(D, tau=TAU, nthreads=a.threads)[:2], m.nelec, ob.enuc(), max_iter=150)
            rows.append({"index": i, "kind": kind, "nbf": m.nbf, "natom": m.natom, "converged": bool(r.converged),
                         "iters": r.iters, "e_total": r.e_total, "seconds": time.time() - t0})
            print(json.dumps(rows[-1]), flush=True)
    with open(OUT, "w") as f:
        json.dump({"workload": "fsim_synth.batched_set(512)", "tau": TAU, "max_iter": 150,
                   "source": "oracle/ (plain FP64 C J/K, numpy SCF)", "molecules": rows}, f, indent=1)


if __name__ == "__main__":
    main()
