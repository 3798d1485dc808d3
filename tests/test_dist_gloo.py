"""World-size-2 gloo run of the sharded Fock-build exchange on CPU: each rank
computes the J/K contribution of its bra-pair shard (oracle shards stand in for
the GPU shards, which run the same i % nshards partition), the partials are
summed with the helper bench.py uses for N > 1 ranks, and the sum must equal
the unsharded J/K.  Also checks the slowest-rank timing reduction."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from fsim_synth import workload
        from oracle import OracleBasis

        ob = OracleBasis(workload("water"))
        D = np.random.default_rng(0).standard_normal((ob.nbf, ob.nbf))
        D = D + D.T
        J, K, nq = ob.jk_shard(D, rank, world, tau=1e-10, nthreads=1)
        Jt, Kt = torch.from_numpy(J), torch.from_numpy(K)
        q = torch.tensor([float(nq)], dtype=torch.float64)
        bench.allreduce_sum([Jt, Kt, q])
        slow = bench.max_over_ranks(1.0 + rank)
        if rank == 0:
            Jf, Kf, nf = ob.jk(D, tau=1e-10, nthreads=1)
            out.put((float(np.abs(Jt.numpy() - Jf).max()), float(np.abs(Kt.numpy() - Kf).max()),
                     int(q.item()), nf, slow))
    finally:
        dist.destroy_process_group()


def test_two_rank_shard_sum_equals_full_build():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dj, dk, nq, nfull, slow = res
    assert dj < 1e-12 and dk < 1e-12
    assert nq == nfull
    assert slow == 2.0


def _oracle_scf_energies(mols):
    from oracle import OracleBasis, rhf
    out = []
    for m in mols:
        ob = OracleBasis(m)
        S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
        r = rhf(S, H, lambda d: ob.jk(d, nthreads=1)[:2], m.nelec, ob.enuc())
        out.append(r.e_total)
    return out


def _split_rank(rank, world, port, out):
    # the batched SCF's molecule split (paper_2510_24968_gb300.batched_scf.run_sharded)
    # with the oracle's SCF standing in for the GPU batch: results gathered in input order
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from fsim_synth import water
        from paper_2510_24968_gb300.batched_scf import run_sharded
        mols = [water(s) for s in range(5)]
        got = run_sharded(mols, _oracle_scf_energies)
        if rank == 0:
            out.put((got, _oracle_scf_energies(mols)))
    finally:
        dist.destroy_process_group()


def test_two_rank_molecule_split_gathers_every_molecule_once():
    from paper_2510_24968_gb300.batched_scf import partition
    parts = partition([5.0, 1.0, 4.0, 2.0, 3.0], 2)
    assert sorted(parts[0] + parts[1]) == [0, 1, 2, 3, 4]
    assert sum([5.0, 1.0, 4.0, 2.0, 3.0][i] for i in parts[0]) in (7.0, 8.0)
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got, ref = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert len(got) == len(ref) and all(abs(a - b) < 1e-12 for a, b in zip(got, ref))


def _dp_rank(rank, world, port, out):
    # data-parallel gradient: each rank's oracle gradient of its share, combined
    # by the helper the GPU training uses, must equal the whole batch's gradient
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import mlp
        from paper_2510_24968_gb300.guess import combine_gradients
        rng = np.random.default_rng(17)
        nin, w, nout, n = 6, 8, 5, 40
        p = rng.standard_normal(mlp.nparams(nin, w, nout)) * 0.3
        x, t = rng.standard_normal((n, nin)), rng.standard_normal((n, nout))
        m = (rng.random((n, nout)) < np.linspace(0.2, 0.9, n)[:, None]).astype(float)  # unequal mask sums
        sl = slice(0, 13) if rank == 0 else slice(13, n)
        g = mlp.grad(p, x[sl], t[sl], m[sl], nin, w, nout)
        comb = combine_gradients(g, float(m[sl].sum()))
        if rank == 0:
            full = mlp.grad(p, x, t, m, nin, w, nout)
            out.put((np.abs(comb - full).max() / np.abs(full).max(), float(np.abs(full).max())))
    finally:
        dist.destroy_process_group()


def test_two_rank_data_parallel_gradient_equals_full_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    rel, scale = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert scale > 0 and rel < 1e-6  # FP32 result of an FP64 combination
