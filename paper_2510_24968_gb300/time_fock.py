"""Time Fock builds (and optionally the SCF) of one synthetic workload.

    python -m paper_2510_24968_gb300.time_fock --workload cloud60 --tau 1e-11 --precision mixed

Prints one JSON object: per precision the build time of each repetition
(CUDA events on the launching stream), the screened unique quartet count,
quartets/s and the per-class-pair kernel times and quartet counts of a separate
timed build.
Every step runs in libfsim; this module only draws the seeded density and
reads the results.  Also the fixed command line used for kernel profiles.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from fsim_synth import workload

from .fsim import FSIM_DFLOAT, FSIM_FP64, FSIM_MIXED, Basis

_NAMES = ["ss", "ps", "pp", "ds", "dp", "dd"]


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="water8")
    ap.add_argument("--tau", type=float, default=1e-10)
    ap.add_argument("--precision", choices=["mixed", "fp64", "dfloat", "both", "all"], default="mixed")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune", action="store_true", help="autotune launch shapes first")
    ap.add_argument("--boys-fp64-T", type=float, default=0.0)
    ap.add_argument("--scf", action="store_true", help="also run the SCF to convergence")
    ap.add_argument("--spherical", action="store_true", help="real solid-harmonic basis")
    ap.add_argument("--jengine", action="store_true", help="also time Coulomb-only J-engine builds")
    ap.add_argument("--dw-screen", action="store_true", help="SCF: density-weighted screening of the increments")
    ap.add_argument("--skip-builds", action="store_true", help="only the SCF (with --scf)")
    ap.add_argument("--shape-sweep", default="",
                    help="comma-separated class pairs (e.g. dd|dd,dd|dp): time each with every legal launch "
                         "shape (median of 5 per-class timings), after the build timings")
    a = ap.parse_args(argv)

    mol = workload(a.workload)
    t0 = time.perf_counter()
    gb = Basis(mol, spherical=a.spherical)
    gb.schwarz()
    torch.cuda.synchronize()
    out = {"workload": a.workload, "nbf": gb.nbf, "nbf_cart": gb.nbf_cart, "spherical": a.spherical,
           "nshell": mol.nshell, "tau": a.tau,
           "setup_s": time.perf_counter() - t0}
    N = gb.nbf
    Dn = np.random.default_rng(0).standard_normal((N, N)) * 0.02
    D = torch.from_numpy(Dn + Dn.T).cuda()
    J, K = torch.zeros_like(D), torch.zeros_like(D)
    precs = {"mixed": [FSIM_MIXED], "fp64": [FSIM_FP64], "dfloat": [FSIM_DFLOAT], "both": [FSIM_MIXED, FSIM_FP64],
             "all": [FSIM_MIXED, FSIM_FP64, FSIM_DFLOAT]}[a.precision]
    for prec in precs:
        name = {FSIM_MIXED: "mixed", FSIM_FP64: "fp64", FSIM_DFLOAT: "dfloat"}[prec]
        kw = dict(tau=a.tau, precision=prec, boys_fp64_T=a.boys_fp64_T)
        if a.skip_builds and a.scf:
            out[name] = {"scf": _scf(gb, prec, a)}
            continue
        if a.tune:
            tuned = gb.autotune(tau=a.tau, precision=prec)
            out[f"{name}_autotune"] = {f"{_NAMES[x]}|{_NAMES[y]}": c for (x, y), (c, _) in tuned.items()}
        gb.fock_build(D, J, K, **kw)
        torch.cuda.synchronize()
        ts = []
        torch.cuda.nvtx.range_push(f"time_fock_{name}")  # profilers can filter on this range
        for _ in range(a.reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            gb.fock_build(D, J, K, **kw)
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        torch.cuda.nvtx.range_pop()
        q = gb.last_quartet_count()
        gb.fock_build(D, J, K, timing=True, **kw)
        ms, qs, nl = gb.last_class_times()
        out[name] = {"build_ms": ts, "quartets": q, "quartets_per_s": q / (min(ts) * 1e-3),
                     "class_ms": {f"{_NAMES[x]}|{_NAMES[y]}": round(v, 4) for (x, y), v in ms.items()},
                     "class_quartets": {f"{_NAMES[x]}|{_NAMES[y]}": int(v) for (x, y), v in qs.items() if v},
                     "launches": nl}
        if a.jengine and prec != FSIM_DFLOAT:
            gb.j_build(D, J, tau=a.tau, precision=prec, boys_fp64_T=a.boys_fp64_T)
            tj = []
            for _ in range(a.reps):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                gb.j_build(D, J, tau=a.tau, precision=prec, boys_fp64_T=a.boys_fp64_T)
                e.record()
                torch.cuda.synchronize()
                tj.append(s.elapsed_time(e))
            out[name]["jengine_ms"] = tj
            out[name]["jengine_ordered_quartets"] = gb.last_quartet_count()
        if a.scf:
            out[name]["scf"] = _scf(gb, prec, a)
        if a.shape_sweep and prec != FSIM_DFLOAT:
            out[name]["shape_sweep_ms"] = _shape_sweep(gb, D, J, K, kw, a)
    print(json.dumps(out))


def _shape_sweep(gb, D, J, K, kw, a):
    """Per class pair: median per-class kernel time (ms) of each launch shape the
    library accepts, keyed by fsim_autotune's encoding (10 * psplit + csplit, -1 the
    cooperative kernel); the class pair is left at its fastest shape."""
    from .fsim import FsimError
    res = {}
    for lab in a.shape_sweep.split(","):
        xy = tuple(_NAMES.index(t) for t in lab.split("|"))
        times = {}
        for code in [-1] + [10 * ps + cs for ps in (1, 3, 9, 27) for cs in (1, 2, 4)]:
            try:
                gb.set_launch({xy: code}, tau=a.tau, precision=kw["precision"])
            except FsimError:
                continue
            t = []
            for _ in range(5):
                gb.fock_build(D, J, K, timing=True, **kw)
                t.append(gb.last_class_times()[0][xy])
            times[str(code)] = round(sorted(t)[2], 4)
        gb.set_launch({xy: int(min(times, key=times.get))}, tau=a.tau, precision=kw["precision"])
        res[lab] = times
    return res


def _scf(gb, prec, a):
    """SCF to convergence; time from the start of the call until the energy stays
    within 1e-8 Eh of the run's own converged energy (set-up and guess included)."""
    t0 = time.perf_counter()
    r = gb.scf(precision=prec, tau=a.tau, dw_screen=a.dw_screen, max_iter=150)
    wall = time.perf_counter() - t0
    E, T = r["energies"], r["times"]
    setup = wall - r["time_s"]
    tte = None
    for i in range(len(E)):
        if all(abs(e - r["e_total"]) < 1e-8 for e in E[i:]):
            tte = float(T[i]) + setup
            break
    return {"e_total": r["e_total"], "iters": r["iters"], "converged": bool(r["converged"]), "wall_s": wall,
            "setup_s": setup, "time_to_1e-8_of_final_s": tte, "fp64_accurate_builds": r["fp64_builds"],
            "mixed_builds": r["mixed_builds"], "quartets": r["quartets"], "dw_screen": a.dw_screen,
            "energies": [float(e) for e in E], "times": [float(t) for t in T]}


if __name__ == "__main__":
    main()
