#!/usr/bin/env python3
"""Benchmark of the McMurchie-Davidson RHF hot path on GB300.

A step is one Fock build J, K <- D (fsim_fock_build: Boys, Hermite Coulomb
recursion, Hermite-to-Cartesian contraction and J/K digestion of every unique
shell quartet that survives Schwarz screening) of the seeded (H2O)_8 cluster
(152 Cartesian functions, tau = 1e-10) in mixed precision (FP32 integrals,
FP64 J/K accumulation).  Basis, pair data, Schwarz bounds and quartet lists
are built once before timing.  value = ERI quartets/s; the FP64 and the
double-float (FP64-accurate, FP32 pipe) Fock builds, Fock builds/s and the
time to an RHF energy within 1e-8 Eh (FP64, double-float, mixed with
double-float or FP64 resets) are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (one rank per GPU; started through torch.distributed.run, or by
this script itself when --gpus N > 1 comes without a launcher) the bra pairs
are sharded over the ranks (fsim_fock_opts.shard) and J, K are summed with one
NCCL all-reduce per build: the same total work on N GPUs (strong scaling).
--impl reference times the CPU oracle (tests-only code) on a bounded sample of
the same workload.

At N = 1 the line also carries the 60-heavy-atom organic cloud (1140
functions, tau = 1e-11): mixed builds with the FP32 large-T Boys branch and
with FP64 Boys above T = 30, and an FP64-accurate (double-float / FP64 kernel
mix) build of one bra-pair shard, with quartets/s, Fock builds/s and the
roofline of its mixed build.

Roofline flop counts: "method" counts what Eq. twoe-final asks for per
primitive quartet -- the R recursion and the Hermite-to-Cartesian sums over
the non-zero E^{ab}_{tuv} only (t <= i_x + j_x etc.), the first of the two
transforms per primitive quartet and the second amortised over the other
side's primitive pairs, whichever order is cheaper -- plus 12 flops per
integral of J/K digestion; "dense" is the Hermite-dense count (every t, u, v
up to the pair's total angular momentum), reported only as an equivalent rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ERI quartets/s, Fock builds/s, time-to-RHF-energy at 1e-8 Eh: mixed vs FP64"
UNIT = "ERI quartets/s"
WORKLOAD = "water8"
WORKLOAD_DESC = "(H2O)_8 seeded cluster, 152 Cartesian s/p/d functions, Schwarz tau 1e-10"
NPRIM = 3  # primitives per shell in every synthetic basis
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock
FP64_PEAK_TFLOPS = 1.25                             # GB300 FP64 (non-tensor), nominal


def ncart(l):
    return (l + 1) * (l + 2) // 2


def nherm(L):
    return (L + 1) * (L + 2) * (L + 3) // 6


PAIR_L = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]


def flops_per_quartet(X, Y, nprim=NPRIM):
    """Hermite-dense flops of one contracted quartet of class pair (X|Y):
    per primitive quartet 2 sum_n n_h(L-n) (R recursion) +
    2 min(A H1 H2 + A C H2, C H1 H2 + A C H1) (Hermite contraction with every
    Hermite index of the pair), plus 12 A C per contracted quartet (J/K
    digestion, 6 FMA per integral).  An equivalent rate only: the method never
    touches the E^{ab}_{tuv} that vanish (t > i_x + j_x etc.)."""
    (la, lb), (lc, ld) = PAIR_L[X], PAIR_L[Y]
    L = la + lb + lc + ld
    A, Cc = ncart(la) * ncart(lb), ncart(lc) * ncart(ld)
    H1, H2 = nherm(la + lb), nherm(lc + ld)
    rec = 2 * sum(nherm(L - n) for n in range(L + 1))
    con = 2 * min(A * H1 * H2 + A * Cc * H2, Cc * H1 * H2 + A * Cc * H1)
    return nprim ** 4 * (rec + con) + 12 * A * Cc


def cart_components(l):
    return [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]


def pair_nnz(la, lb):
    """Non-zero E^{ab}_{tuv} over the Cartesian components of a pair class:
    sum over (a, b) of prod_axis (i_axis + j_axis + 1)."""
    n = 0
    for ca in cart_components(la):
        for cb in cart_components(lb):
            n += (ca[0] + cb[0] + 1) * (ca[1] + cb[1] + 1) * (ca[2] + cb[2] + 1)
    return n


def method_flops_per_quartet(X, Y, nprim=NPRIM):
    """Flops of one contracted quartet as Eq. twoe-final asks for them: per
    primitive quartet the R recursion (2 sum_n n_h(L-n)) and the first transform
    (2 H_other nnz_side), the second transform (2 nnz_other n_c(side)) once per
    primitive pair of its side, cheaper order of the two; plus 12 flops per
    integral of J/K digestion.  Boys evaluations are not counted."""
    (la, lb), (lc, ld) = PAIR_L[X], PAIR_L[Y]
    L = la + lb + lc + ld
    A, Cc = ncart(la) * ncart(lb), ncart(lc) * ncart(ld)
    H1, H2 = nherm(la + lb), nherm(lc + ld)
    nzb, nzk = pair_nnz(la, lb), pair_nnz(lc, ld)
    npp = nprim * nprim
    rec = 2 * sum(nherm(L - n) for n in range(L + 1))
    ket_first = 2 * H1 * nzk + 2 * nzb * Cc / npp   # W = E_cd R per primitive quartet, then E_ab W per bra pp
    bra_first = 2 * H2 * nzb + 2 * nzk * A / npp
    return npp * npp * (rec + min(ket_first, bra_first)) + 12 * A * Cc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.lines, self.proc = [], None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ["eri_core.cuh", "eri_launch.cuh", "boys.cuh", "md_tables.cuh", "fsim_internal.h", "dfloat.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")


def kernel_source_digest() -> str:
    """sha256 over the code of the sources that define the Fock-build kernels: line
    comments, trailing blanks and empty lines removed, so that an edited comment
    keeps a capture valid while any code change invalidates it."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2510_24968_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh.read().splitlines():
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def recorded_traffic(cls_label: str):
    """DRAM bytes per launch of the mixed kernel of a class pair from the last ncu
    capture, or None when no capture exists or the kernel sources changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256") != kernel_source_digest():
        return None
    k = rec.get("mixed", {}).get(cls_label)
    return k["dram_bytes_per_launch"] if k else None


def allreduce_sum(tensors):
    """Sum partial J/K (or counts) over the ranks in place (the exchange step of
    a sharded Fock build); no-op on one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        for t in tensors:
            dist.all_reduce(t)
    return tensors


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks (timings are reported as the slowest rank)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([value], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return value


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def cpu_sample(mol, seconds_target: float, tau: float, stride0: int = 64, ob=None):
    """The oracle's J/K over a bounded sample of bra pairs: (quartets/s, quartets, seconds, stride)."""
    import numpy as np
    from oracle import OracleBasis
    ob = ob or OracleBasis(mol)
    D = np.random.default_rng(0).standard_normal((ob.nbf, ob.nbf)) * 0.05
    D = D + D.T
    Q = ob.schwarz()  # noqa: F841  (warms the oracle's Schwarz path like a first build)
    stride = stride0
    t0 = time.perf_counter()
    _, _, nq = ob.jk_sample(D, tau, stride)
    dt = time.perf_counter() - t0
    # scale the sample toward the target duration (bounded below by every 4th bra pair)
    stride2 = max(4, int(stride * dt / max(seconds_target, 1e-3)))
    if stride2 < stride:
        t0 = time.perf_counter()
        _, _, nq = ob.jk_sample(D, tau, stride2)
        dt = time.perf_counter() - t0
        stride = stride2
    return nq / dt, nq, dt, stride


def screened_quartets(mol, tau: float) -> int:
    """Unique shell quartets of a full build (Q_ab Q_cd >= tau, pair-of-pairs order), from the oracle's Q."""
    import numpy as np
    from oracle import OracleBasis
    Q = OracleBasis(mol).schwarz()
    q = np.sort(Q[np.tril_indices(Q.shape[0])])[::-1]
    # pairs (i <= j) of sorted pair bounds with q_i q_j >= tau: for each i, kets j >= i up to the cutoff
    cut = np.searchsorted(-q, -tau / np.maximum(q, 1e-300), side="right")
    return int(np.maximum(cut - np.arange(q.size), 0).sum())


def bench_config(tau: float, world: int) -> dict:
    """The workload both arms measure (identical dict on both lines)."""
    return {"workload": WORKLOAD_DESC, "nbf": 152, "schwarz_tau": tau,
            "step": "one Fock build J,K <- D over the screened unique shell quartets",
            "l2": "GPU arm: 256 MiB device write before every timed step; CPU arm: no flush",
            "parallelism": f"bra-pair shards x{world}" if world > 1 else "1 device"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from fsim_synth import workload
    mol = workload(WORKLOAD)
    vals, secs, desc = [], [], ""
    # each step is a bounded sample of the same build, sized so that the whole
    # --steps/--warmup run stays within about 100 s of oracle time
    per_step = max(1.0, min(8.0, 100.0 / (args.warmup + args.steps)))
    for it in range(args.warmup + args.steps):
        v, nq, dt, stride = cpu_sample(mol, per_step, args.tau)
        if it >= args.warmup:
            vals.append(v)
            secs.append(dt)
        desc = f"oracle J/K over bra pairs ij with ij % {stride} == 0 ({nq} unique quartets per step)"
    v = statistics.mean(vals)
    cores = os.cpu_count()
    nq_full = screened_quartets(mol, args.tau)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args.tau, world),
            "precision": "FP64 oracle (plain C, OpenMP over bra pairs)",
            "full_build_ms_extrapolated": nq_full / v * 1e3,
            "full_build_note": f"one full build ({nq_full} quartets) at the sampled rate (extrapolated)",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_oracle_timings(args):
    """--oracle-timings: the oracle (plain FP64 C J/K with OpenMP over bra pairs,
    numpy SCF; test infrastructure) timed on this host's cores for the four
    configurations.  Whole SCFs where they end in seconds; otherwise one J/K
    build, or a bra-pair sample of one, scaled by the screened quartet count and
    by the oracle's own SCF iteration count (tests/golden), each labelled as an
    extrapolation.  One JSON line."""
    import platform

    import numpy as np
    from fsim_synth import batched_set, workload
    from oracle import OracleBasis, rhf
    gold = os.path.join(ROOT, "tests", "golden")
    out = {"impl": "oracle-timings", "cores": os.cpu_count(), "machine": platform.machine(),
           "oracle": "plain C FP64 J/K (OpenMP over bra pairs), numpy SCF"}
    # water, 13 functions: the whole RHF (one-electron matrices, J/K, DIIS)
    t0 = time.perf_counter()
    mol = workload("water")
    ob = OracleBasis(mol)
    S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
    r = rhf(S, H, lambda d: ob.jk(d)[:2], mol.nelec, ob.enuc())
    out["water"] = {"scf_s": time.perf_counter() - t0, "iters": r.iters, "e_total": r.e_total,
                    "kind": "measured: whole SCF, unscreened"}
    # (H2O)_8, tau 1e-10: a bra-pair sample of one build, scaled to the full
    # screened build and to the oracle SCF's 17 iterations
    mol = workload(WORKLOAD)
    v, nq, dt, stride = cpu_sample(mol, 15.0, 1e-10)
    nq_full = screened_quartets(mol, 1e-10)
    with open(os.path.join(gold, "water8_scf_oracle.json")) as f:
        it8 = json.load(f)["iters"]
    out["water8"] = {"quartets_per_s": v, "sample": f"bra pairs ij % {stride} == 0: {nq} quartets in {dt:.1f} s",
                     "build_s_extrapolated": nq_full / v, "scf_s_extrapolated": it8 * nq_full / v,
                     "scf_iters": it8, "kind": "extrapolated from the sample"}

    # 60-heavy-atom cloud, tau 1e-11: Schwarz bounds once, then bra-pair samples
    # of one build (each sample call recomputes the bounds: their time is taken off)
    mol = workload("cloud60")
    ob = OracleBasis(mol)
    D = np.random.default_rng(0).standard_normal((ob.nbf, ob.nbf)) * 0.05
    D = D + D.T
    t0 = time.perf_counter()
    ob.schwarz()
    t_q = time.perf_counter() - t0
    stride = 40000
    while True:
        t0 = time.perf_counter()
        _, _, nq = ob.jk_sample(D, 1e-11, stride)
        dt = max(time.perf_counter() - t0 - t_q, 1e-3)
        if dt >= 10.0 or stride <= 2000:
            break
        stride = max(2000, int(stride * max(dt, 0.5) / 20.0))
    nq_full = screened_quartets(mol, 1e-11)
    out["cloud60"] = {"schwarz_s": t_q, "quartets_per_s": nq / dt,
                      "sample": f"bra pairs ij % {stride} == 0: {nq} quartets in {dt:.1f} s (Schwarz excluded)",
                      "screened_quartets": nq_full, "build_s_extrapolated": nq_full * dt / nq,
                      "kind": "extrapolated from the sample; the sampled pairs' class mix sets the rate"}
    # 512-molecule set: one J/K build of each member whose oracle SCF converged
    # (tests/golden/config3_oracle.json), scaled by that SCF's iteration count
    with open(os.path.join(gold, "config3_oracle.json")) as f:
        g3 = json.load(f)
    mols = batched_set(512)
    rows = []
    for m in g3["molecules"]:
        if not m["converged"]:
            continue
        obm = OracleBasis(mols[m["index"]])
        Dm = np.eye(obm.nbf)
        t0 = time.perf_counter()
        _, _, nqm = obm.jk(Dm, tau=g3["tau"])
        dt = time.perf_counter() - t0
        rows.append({"index": m["index"], "nbf": obm.nbf, "build_s": dt, "quartets": nqm, "iters": m["iters"],
                     "scf_s_extrapolated": dt * m["iters"]})
    out["batched_set_sample"] = {"molecules": rows, "kind": "one measured build per molecule x its oracle SCF iterations"}
    print(json.dumps(out), flush=True)

def time_to_energy(res, e_ref, tol=1e-8):
    """Seconds until the energy stays within tol of e_ref for the rest of the run."""
    E, T = res["energies"], res["times"]
    ok = [abs(e - e_ref) < tol for e in E]
    for i in range(len(E)):
        if all(ok[i:]):
            return float(T[i])
    return None


CLOUD_TAU = 1e-11
CLOUD_SHARDS = 16


def cloud60_section(args, gb_dev, sptr, flush):
    """The 60-heavy-atom organic cloud (1140 functions, tau 1e-11): mixed builds
    (FP32 large-T Boys branch; FP64 Boys above T = 30) and an FP64-accurate build
    of one bra-pair shard (round-robin over the cost-sorted bra list), each timed
    with per-class CUDA events (class pairs serialised on the stream)."""
    import numpy as np
    import torch

    from fsim_synth import workload
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_MIXED, Basis
    names = ["ss", "ps", "pp", "ds", "dp", "dd"]
    mol = workload("cloud60")
    t0 = time.perf_counter()
    gb = Basis(mol)
    gb.schwarz()
    N = gb.nbf
    Dn = np.random.default_rng(1).standard_normal((N, N)) * 0.02
    D = torch.from_numpy(Dn + Dn.T).to(gb_dev)
    J, K = torch.zeros_like(D), torch.zeros_like(D)
    setup_s = time.perf_counter() - t0

    def one(prec, b64=0.0, shard=0, nshards=1, timing=True):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        gb.fock_build(D, J, K, tau=CLOUD_TAU, precision=prec, stream=sptr, boys_fp64_T=b64, shard=shard,
                      nshards=nshards, timing=timing)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t, q, _ = gb.last_class_times()
        return e0.elapsed_time(e1), t, q

    # first build: the plan is made on the host before the launches, the per-class
    # events time only the GPU work of each class pair (serialised)
    _, t_mx, q = one(FSIM_MIXED)
    ms_mx, _, _ = one(FSIM_MIXED, timing=False)   # concurrent class-pair launches, as in the headline
    _, t_b64, _ = one(FSIM_MIXED, b64=30.0)
    ms_mx_ser, ms_b64 = sum(t_mx.values()), sum(t_b64.values())
    nq = sum(q.values())
    fl = sum(q[k] * method_flops_per_quartet(*k) for k in q)
    dom = max(t_mx, key=t_mx.get)
    dom_fl = q[dom] * method_flops_per_quartet(*dom)
    J1 = torch.zeros_like(D)
    gb.j_build(D, J1, tau=CLOUD_TAU, precision=FSIM_MIXED, stream=sptr)
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream())
    gb.j_build(D, J1, tau=CLOUD_TAU, precision=FSIM_MIXED, stream=sptr)
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms_j = e0.elapsed_time(e1)
    nq_j = gb.last_quartet_count()
    _, t_df, q_df = one(FSIM_DFLOAT, shard=0, nshards=CLOUD_SHARDS)
    ms_df = sum(t_df.values())
    nq_df = sum(q_df.values())
    return {
        "workload": "organic cloud, 60 heavy atoms (C/N/O 70/15/15) on a jittered 2.8-bohr lattice, "
                    f"4s3p1d per heavy atom, H-capped; {N} Cartesian functions, tau {CLOUD_TAU:g}",
        "nbf": N, "unique_quartets": nq, "setup_s": setup_s,
        "mixed_fp32_boys": {"ms": ms_mx, "eri_quartets_per_s": nq / (ms_mx * 1e-3), "fock_builds_per_s": 1e3 / ms_mx,
                            "ms_serialised": ms_mx_ser},
        "mixed_fp64_boys_T30": {"ms_serialised": ms_b64, "eri_quartets_per_s_serialised": nq / (ms_b64 * 1e-3),
                                "fock_builds_per_s_serialised": 1e3 / ms_b64,
                                "vs_fp32_boys_serialised": ms_b64 / ms_mx_ser},
        "j_engine_mixed": {"ms": ms_j, "vs_fused_jk": ms_j / ms_mx, "ordered_quartets": nq_j},
        "fp64_accurate_shard": {"precision": "double-float kernels up to L = 4, FP64 kernels above",
                                "shard": f"0 of {CLOUD_SHARDS} (bra pairs i % {CLOUD_SHARDS} == 0)",
                                "ms": ms_df, "unique_quartets": nq_df,
                                "eri_quartets_per_s": nq_df / (ms_df * 1e-3),
                                "full_build_ms_extrapolated": ms_df * nq / max(nq_df, 1)},
        "build_roofline": {"flops": "method count", "achieved_tflops": fl / (ms_mx * 1e-3) / 1e12,
                           "frac_fp32": fl / (ms_mx * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                           "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "dominant_kernel": {"class": f"{names[dom[0]]}|{names[dom[1]]}", "ms": t_mx[dom], "quartets": q[dom],
                            "achieved_tflops": dom_fl / (t_mx[dom] * 1e-3) / 1e12,
                            "frac_fp32": dom_fl / (t_mx[dom] * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                            "share_of_build": t_mx[dom] / sum(t_mx.values())},
        "class_ms": {f"{names[k[0]]}|{names[k[1]]}": round(v, 3) for k, v in t_mx.items()},
        "class_quartets": {f"{names[k[0]]}|{names[k[1]]}": int(v) for k, v in q.items() if v},
        "class_frac_fp32": {f"{names[k[0]]}|{names[k[1]]}":
                            round(q[k] * method_flops_per_quartet(*k) / (v * 1e-3) / 1e12 / FP32_PEAK_TFLOPS, 4)
                            for k, v in t_mx.items() if v > 0},
        "class_ms_fp64_boys_T30": {f"{names[k[0]]}|{names[k[1]]}": round(v, 3) for k, v in t_b64.items()},
    }


def j_engine_times(gb, D, tau, sptr, flush, rank, world, reps=5):
    """Coulomb-only builds (fsim_j_build, Hermite-space J-engine) against the
    fused J/K build of the same screened quartets: CUDA events per build."""
    import torch

    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    out = {}
    Jo = torch.zeros_like(D)
    for name, prec in (("mixed", FSIM_MIXED), ("fp64", FSIM_FP64)):
        gb.j_build(D, Jo, tau=tau, precision=prec, stream=sptr, shard=rank, nshards=world)  # plan
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            gb.j_build(D, Jo, tau=tau, precision=prec, stream=sptr, shard=rank, nshards=world)
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = {"ms": statistics.median(ts), "ordered_quartets": gb.last_quartet_count()}
    return out


def run_ours(args):
    import numpy as np
    import torch

    from fsim_synth import workload
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_FP64, FSIM_MIXED, Basis

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    mol = workload(WORKLOAD)

    # CPU baseline first (rank 0, N = 1): the oracle as it stands on the host cores
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, nq, dt, stride = cpu_sample(mol, 15.0, args.tau)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle J/K of (H2O)_8 over bra pairs ij % {stride} == 0: {nq} unique quartets in {dt:.1f} s"}

    gb = Basis(mol)
    gb.schwarz()
    tuned = gb.autotune(tau=args.tau, precision=FSIM_MIXED, shard=rank, nshards=world) if not args.no_tune else {}
    # the FP64-accurate builds get the same treatment (their plans also serve the SCF runs)
    tuned_64 = {p: gb.autotune(tau=args.tau, precision=p, shard=rank, nshards=world)
                for p in (FSIM_FP64, FSIM_DFLOAT)} if not args.no_tune else {}
    N = gb.nbf
    Dn = np.random.default_rng(0).standard_normal((N, N)) * 0.05
    Dn = Dn + Dn.T
    D = torch.from_numpy(Dn).to(dev)
    J, K = torch.zeros_like(D), torch.zeros_like(D)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def build(prec, timing=False):
        gb.fock_build(D, J, K, tau=args.tau, precision=prec, stream=sptr, shard=rank, nshards=world,
                      timing=timing)
        if world > 1:
            allreduce_sum([J, K])

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            build(prec)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.nvtx.range_push(f"fock_timed_{prec}")
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            build(prec)
            ev[k][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev), dev)
        _, q, n = gb.last_class_times()
        launches, quartets = n * steps, sum(q.values())
        # per-class attribution: the same builds again, class pairs one after the
        # other on the stream, each bracketed by CUDA events
        per_class = {}
        for k in range(steps):
            flush.zero_()
            build(prec, timing=True)
            t, _, _ = gb.last_class_times()
            for key, v in t.items():
                per_class.setdefault(key, []).append(v)
        if world > 1:
            qq = torch.tensor([quartets], device=dev, dtype=torch.float64)
            allreduce_sum([qq])
            quartets = int(qq.item())
        return ms / steps, quartets, per_class, launches, q

    clocks = ClockSampler(local)
    ms_mixed, q_mixed, cls_mixed, launches, qcls = timed(FSIM_MIXED, args.steps, args.warmup)
    clk = clocks.stop()
    ms_fp64, q_fp64, cls_fp64, _, _ = timed(FSIM_FP64, max(2, min(args.steps, 3)), 1)
    ms_df, q_df, cls_df, _, _ = timed(FSIM_DFLOAT, max(2, min(args.steps, 3)), 1)
    jeng = j_engine_times(gb, D, args.tau, sptr, flush, rank, world) if not args.no_jengine else None

    # roofline of the dominant kernel (largest time share of the mixed build)
    tot = {k: sum(v) for k, v in cls_mixed.items()}
    dom = max(tot, key=tot.get)
    avg_ms = tot[dom] / len(cls_mixed[dom])
    fl = qcls[dom] * method_flops_per_quartet(*dom)
    achieved = fl / (avg_ms * 1e-3) / 1e12
    dense_dom = qcls[dom] * flops_per_quartet(*dom) / (avg_ms * 1e-3) / 1e12
    names = ["ss", "ps", "pp", "ds", "dp", "dd"]
    all_fl = sum(qcls[k] * method_flops_per_quartet(*k) for k in qcls)
    all_fl_dense = sum(qcls[k] * flops_per_quartet(*k) for k in qcls)
    # primitive quartets and Cartesian integrals per build (every shell of the
    # workload has NPRIM primitives, so a shell quartet holds NPRIM^4)
    assert all(len(sh.alpha) == NPRIM for sh in mol.shells)
    prim_q = sum(qcls.values()) * NPRIM ** 4
    cart_ints = sum(qcls[k] * ncart(PAIR_L[k[0]][0]) * ncart(PAIR_L[k[0]][1]) * ncart(PAIR_L[k[1]][0]) *
                    ncart(PAIR_L[k[1]][1]) for k in qcls)
    cloud = cloud60_section(args, gb_dev=dev, sptr=sptr, flush=flush) if rank == 0 and world == 1 \
        and not args.no_cloud60 else None

    # end to end through the C-ABI with pinned host buffers (copies inside the timed region)
    Dh = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
    Dh.copy_(torch.from_numpy(Dn))
    Jh = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
    Kh = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
    Dnp, Jnp, Knp = Dh.numpy(), Jh.numpy(), Kh.numpy()
    for _ in range(2):
        gb.fock_build(Dnp, Jnp, Knp, tau=args.tau, precision=FSIM_MIXED, stream=sptr, shard=rank, nshards=world)
    t0 = time.perf_counter()
    ne = max(3, args.steps)
    for _ in range(ne):
        gb.fock_build(Dnp, Jnp, Knp, tau=args.tau, precision=FSIM_MIXED, stream=sptr, shard=rank, nshards=world)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ne, dev)

    # time to a converged energy, mixed vs FP64 (rank 0, whole molecule on one GPU)
    tte = None
    if rank == 0 and not args.no_scf:
        r64 = gb.scf(precision=FSIM_FP64, tau=args.tau, stream=sptr)
        # mixed: FP32 builds, resets as double-float builds (the default), or as FP64 builds
        rmx = gb.scf(precision=FSIM_MIXED, tau=args.tau, stream=sptr, final_fp64=2)
        rfr = gb.scf(precision=FSIM_MIXED, tau=args.tau, stream=sptr, final_fp64=1)
        # every build FP64-accurate, in the autotuned double-float/FP64 kernel mix
        rdd = gb.scf(precision=FSIM_DFLOAT, tau=args.tau, stream=sptr)
        tte = {"fp64_s": time_to_energy(r64, r64["e_total"]), "mixed_s": time_to_energy(rmx, r64["e_total"]),
               "mixed_fp64_resets_s": time_to_energy(rfr, r64["e_total"]),
               "dfloat_s": time_to_energy(rdd, r64["e_total"]), "dfloat_iters": rdd["iters"],
               "dfloat_vs_fp64_eh": rdd["e_total"] - r64["e_total"],
               "fp64_iters": r64["iters"], "mixed_iters": rmx["iters"], "mixed_resets": rmx["fp64_builds"],
               "mixed_fp64_resets_iters": rfr["iters"], "mixed_fp64_resets_builds": rfr["fp64_builds"],
               "mixed_vs_fp64_eh": rmx["e_total"] - r64["e_total"], "mixed_fallback": rmx["mixed_fallback"],
               "min_s_eig": rmx["min_s_eig"],
               "mixed_fp64_resets_vs_fp64_eh": rfr["e_total"] - r64["e_total"], "e_total_fp64": r64["e_total"],
               "mixed_reset_builds": "double-float (mixed_fp64_resets_*: the same SCF with FP64 resets)"}
        gold = os.path.join(ROOT, "tests", "golden", "water8_scf_oracle.json")
        if os.path.exists(gold):
            with open(gold) as f:
                g = json.load(f)
            tte["fp64_vs_oracle_eh"] = r64["e_total"] - g["e_total"]
            tte["mixed_vs_oracle_eh"] = rmx["e_total"] - g["e_total"]
            tte["mixed_fp64_resets_vs_oracle_eh"] = rfr["e_total"] - g["e_total"]
            tte["dfloat_vs_oracle_eh"] = rdd["e_total"] - g["e_total"]
        if tte["fp64_s"] and tte["mixed_s"]:
            tte["speedup"] = tte["fp64_s"] / tte["mixed_s"]
        if tte["fp64_s"] and tte["mixed_fp64_resets_s"]:
            tte["speedup_fp64_resets"] = tte["fp64_s"] / tte["mixed_fp64_resets_s"]

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    value = q_mixed / (ms_mixed * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(args.tau, world),
        "precision": "mixed: FP32 Boys/R/contraction, FP64 J/K accumulation",
        "unique_quartets_per_build": q_mixed,
        "fock_builds_per_s": {"mixed": 1e3 / ms_mixed, "fp64": 1e3 / ms_fp64, "dfloat": 1e3 / ms_df},
        "eri_quartets_per_s": {"mixed": value, "fp64": q_fp64 / (ms_fp64 * 1e-3), "dfloat": q_df / (ms_df * 1e-3)},
        "primitive_quartets_per_s": {"mixed": prim_q / (ms_mixed * 1e-3), "fp64": prim_q / (ms_fp64 * 1e-3),
                                     "dfloat": prim_q / (ms_df * 1e-3)},
        "cartesian_integrals_per_s": {"mixed": cart_ints / (ms_mixed * 1e-3), "fp64": cart_ints / (ms_fp64 * 1e-3),
                                      "dfloat": cart_ints / (ms_df * 1e-3)},
        "per_build": {"unique_quartets": q_mixed, "primitive_quartets": prim_q, "cartesian_integrals": cart_ints},
        "class_ms_fp64_dfloat": {f"{names[k[0]]}|{names[k[1]]}": [round(sum(cls_fp64[k]) / len(cls_fp64[k]), 3),
                                                                  round(sum(cls_df[k]) / len(cls_df[k]), 3)]
                                 for k in cls_fp64 if k in cls_df},
        "time_to_energy_1e-8": tte,
        "roofline": {"kernel": f"jk_kernel<float> ({names[dom[0]]}|{names[dom[1]]})", "bound": "alu",
                     "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": recorded_traffic(f"{names[dom[0]]}|{names[dom[1]]}"),
                     "flops": "method count (E non-zeros only), per launch: quartets x "
                              f"{method_flops_per_quartet(*dom):.0f}",
                     "dense_equivalent_tflops": dense_dom,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (no measured FP32 peak)",
                     "share_of_build": tot[dom] / sum(tot.values()),
                     "timing": "per-launch CUDA events; class pairs serialised on the launching stream"},
        "build_roofline": {"flops": "method count, all class pairs", "unit": "TFLOP/s",
                           "achieved": all_fl / (ms_mixed * 1e-3) / 1e12,
                           "frac_fp32": all_fl / (ms_mixed * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                           "fp64_achieved": all_fl / (ms_fp64 * 1e-3) / 1e12,
                           "frac_fp64": all_fl / (ms_fp64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                           "fp64_peak_source": "nominal 1.25 TFLOP/s FP64 (non-tensor)",
                           "dense_equivalent_tflops": {"mixed": all_fl_dense / (ms_mixed * 1e-3) / 1e12,
                                                       "fp64": all_fl_dense / (ms_fp64 * 1e-3) / 1e12}},
        "cloud60": cloud,
        "j_engine": None if jeng is None else dict(jeng, **{
            "note": "J alone by the Hermite-space J-engine (both orders of every screened unique quartet)",
            "mixed_vs_fused_jk": jeng["mixed"]["ms"] / ms_mixed, "fp64_vs_fused_jk": jeng["fp64"]["ms"] / ms_fp64}),
        "class_ms": {f"{names[k[0]]}|{names[k[1]]}": round(tot[k] / len(cls_mixed[k]), 4) for k in tot},
        "autotune": {f"{names[k[0]]}|{names[k[1]]}": v[0] for k, v in tuned.items()},
        "autotune_fp64_dfloat": {f"{names[k[0]]}|{names[k[1]]}": [tuned_64[FSIM_FP64].get(k, (0,))[0],
                                                                  tuned_64[FSIM_DFLOAT].get(k, (0,))[0]]
                                 for k in tuned} if tuned_64 else {},
        "cpu_baseline": cpu,
        "e2e": {"value": q_mixed / e2e_s, "unit": UNIT, "h2d_bytes_per_step": N * N * 8,
                "d2h_bytes_per_step": 2 * N * N * 8},
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tau", type=float, default=1e-10)
    ap.add_argument("--no-scf", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-cloud60", action="store_true")
    ap.add_argument("--no-jengine", action="store_true")
    ap.add_argument("--oracle-timings", action="store_true",
                    help="time the CPU oracle on the host cores for all configurations (one JSON line), then exit")
    args = ap.parse_args()
    if args.oracle_timings:
        run_oracle_timings(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.gpus < 1:
        sys.exit("bench.py: --gpus must be >= 1")
    if "WORLD_SIZE" in os.environ:
        if int(os.environ["WORLD_SIZE"]) != args.gpus:
            sys.exit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={os.environ['WORLD_SIZE']}")
    elif args.gpus > 1:
        sys.exit(self_launch(args.gpus))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


def self_launch(n: int) -> int:
    """--gpus N > 1 without a launcher: start N ranks on this node through
    torch.distributed.run (rendezvous on 127.0.0.1) and return their exit code."""
    import socket
    import torch
    if torch.cuda.is_available() and torch.cuda.device_count() < n:
        print(f"bench.py: --gpus {n} but only {torch.cuda.device_count()} visible GPU(s)", file=sys.stderr)
        return 2
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


if __name__ == "__main__":
    main()
