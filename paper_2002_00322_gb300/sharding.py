"""Builds sharded across processes (one GPU each): every rank builds its slice
of the kept brick list (esmf_fock_build_shard) and one SUM all-reduce per
output completes J, K, F and the traces, which are linear in the integrals.
"""
from __future__ import annotations


def allreduce_outputs(outputs, group=None):
    """SUM all-reduce of every tensor in `outputs` (in place); returns them."""
    import torch.distributed as dist
    for t in outputs:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return outputs


def build_sharded(builder, D, group=None, want_F=True, stream=None):
    """Sharded grouped build on this rank's GPU: `builder` is a FockBuilder for
    the same basis on every rank, D the full (m, N, N) densities on this
    rank's device.  Returns (J, K, F, traces), identical on all ranks."""
    import torch
    import torch.distributed as dist

    from . import fock
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    D = D.contiguous()
    m = D.shape[0]
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    F = torch.empty_like(D) if want_F else None
    t = torch.empty(m, dtype=torch.float64, device=D.device)
    fock.esmf_fock_build_shard(builder.h, rank, world, m, D, J, K, F, t, stream)
    return tuple(allreduce_outputs((J, K, F, t), group))
