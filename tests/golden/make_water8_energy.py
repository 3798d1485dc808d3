"""Writes water8_scf_oracle.json: the CPU oracle's RHF energy of the (H2O)_8
cluster workload (152 Cartesian functions, Schwarz tau = 1e-10), used as the
expected value of the full-size energy parity test.  Calls only oracle/ (and
the seeded input generator); takes ~15 min on 8 cores.

    python tests/golden/make_water8_energy.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from fsim_synth import workload  # noqa: E402
from oracle import OracleBasis, rhf  # noqa: E402


def main():
    m = workload("water8")
    B = OracleBasis(m)
    S, H = B.onee("S"), B.onee("T") + B.onee("V")
    t0 = time.time()
    tau = 1e-10
    r = rhf(S, H, lambda D: B.jk(D, tau=tau)[:2], m.nelec, B.enuc(), conv_dE=1e-10, conv_dD=1e-7)
    out = {"workload": "(H2O)_8, seeded cluster, 152 Cartesian functions", "schwarz_tau": tau,
           "e_total": r.e_total, "e_nuc": r.e_nuc, "iters": r.iters, "converged": r.converged,
           "energies": r.energies, "min_s_eig": r.min_s_eig, "oracle_seconds": time.time() - t0}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "water8_scf_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["e_total"], out["iters"], out["converged"])


if __name__ == "__main__":
    main()
