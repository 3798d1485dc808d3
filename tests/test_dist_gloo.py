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
