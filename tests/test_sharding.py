"""Sharded builds: the host-side partition and all-reduce run on CPU ranks
(gloo, world size 2), each rank standing in for a GPU with its slice of the
oracle's unique-quartet loop; the GPU test sums sequential shards of the CUDA
build on one GPU."""
import os
import socket

import numpy as np
import pytest

from paper_2002_00322_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from oracle.oracle import Oracle
    from paper_2002_00322_gb300.sharding import allreduce_outputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.small_random(14, 3, 8, tol=1e-8, edge=6.0)
    o = Oracle(w.basis)
    npair = w.basis.n * (w.basis.n + 1) // 2
    b0, b1 = npair * rank // world, npair * (rank + 1) // world
    J, K, _ = o.jk_unique(w.D, w.tol, pair_range=(b0, b1))
    Jt, Kt = torch.from_numpy(J), torch.from_numpy(K)
    allreduce_outputs((Jt, Kt))
    if rank == 0:
        Jf, Kf, _ = o.jk_unique(w.D, w.tol)
        q.put((float(np.max(np.abs(Jt.numpy() - Jf))), float(np.max(np.abs(Kt.numpy() - Kf)))))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_allreduce_on_cpu_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    dj, dk = q.get(timeout=5)
    assert dj <= 1e-12 and dk <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol,case", [("fp64", 1e-12, "small"), ("fp16x2", 1e-6, "small"),
                                           ("fp16x2", 1e-6, "stored_n200_m16"),
                                           ("fp16x2", 1e-6, "direct_stored_n200_m16")])
def test_sequential_shards_sum_to_full_build(esmf, prec, tol, case):
    """Shards are cut at equal estimated cost on item boundaries, and on the
    tensor-core path each shard has its own cost-balanced CTA split: the
    shards still sum to the whole build.  The integral-direct tensor-core
    case (a 64 MB budget: many chunks) cuts shards across its chunks."""
    import torch
    w = W.small_random(45, 4, 9, tol=1e-10, edge=12.0) if case == "small" else W.stored()
    D = torch.from_numpy(w.D).cuda()
    direct = case.startswith("direct")
    with esmf.FockBuilder(w.basis, w.tol, "direct" if direct else "stored", prec,
                          budget_bytes=(64 << 20) if direct else 0) as fb:
        J, K, F, t = fb.build(D, want_F=True)
        acc = [torch.zeros_like(J), torch.zeros_like(K), torch.zeros_like(F), torch.zeros_like(t)]
        for s in range(4):
            parts = [torch.empty_like(J), torch.empty_like(K), torch.empty_like(F), torch.empty_like(t)]
            esmf.esmf_fock_build_shard(fb.h, s, 4, w.m, D, *parts)
            for a, p in zip(acc, parts):
                a += p
        torch.cuda.synchronize()
    for a, r in zip(acc, (J, K, F, t)):
        assert float((a - r).norm() / r.norm()) <= tol
