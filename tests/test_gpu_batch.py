"""Batched builds (esmf_fock_build_batch): several molecules of uneven size and
density count in one persistent tensor-core launch per pass of 16 densities.
Each result equals the same handle built alone, and the smallest matches the
FP64 oracle; the call replays from a CUDA graph; bad batches are rejected."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (functions, densities, seed): 1, 2 and 3 passes of 16 densities
MOLS = [(40, 3, 31), (64, 8, 32), (96, 16, 33), (120, 20, 34), (150, 33, 35)]


def rel(x, r):
    return float(np.linalg.norm(x - r) / max(np.linalg.norm(r), 1e-300))


@pytest.fixture(scope="module")
def mols():
    return [W.small_random(n, m, seed, tol=1e-10, edge=7.0 * (n / 48) ** (1 / 3), min_dist=1.2)
            for (n, m, seed) in MOLS]


def builders(esmf, ws, precs):
    return [esmf.FockBuilder(w.basis, w.tol, "stored", p) for w, p in zip(ws, precs)]


@pytest.mark.parametrize("precs", [["fp16x2"] * 5, ["fp16x2", "bf16x2", "fp16x2", "bf16x2", "fp16x2"]])
def test_batch_equals_builds_alone(esmf, mols, precs):
    import torch
    fbs = builders(esmf, mols, precs)
    try:
        Ds = [torch.from_numpy(w.D).cuda() for w in mols]
        alone = [fb.build(D, want_traces=False)[:2] for fb, D in zip(fbs, Ds)]
        alone = [(J.cpu().numpy(), K.cpu().numpy()) for J, K in alone]
        for _ in range(2):                       # twice: the second reuses the work memory
            out = esmf.build_batch(fbs, Ds)
            torch.cuda.synchronize()
            for (J, K), (Ja, Ka), w in zip(out, alone, mols):
                assert rel(J.cpu().numpy(), Ja) < 1e-12 and rel(K.cpu().numpy(), Ka) < 1e-12, w.name
        assert all(fb.device_error() == 0 for fb in fbs)
    finally:
        for fb in fbs:
            fb.close()


def test_batch_matches_oracle(esmf, mols):
    import torch
    w = mols[0]
    Jr, Kr, _ = Oracle(w.basis).jk_unique(w.D, w.tol)
    fbs = builders(esmf, mols, ["fp16x2"] * len(mols))
    try:
        out = esmf.build_batch(fbs, [torch.from_numpy(x.D).cuda() for x in mols])
        J, K = out[0][0].cpu().numpy(), out[0][1].cpu().numpy()
    finally:
        for fb in fbs:
            fb.close()
    assert max(rel(J[k], Jr[k]) for k in range(w.m)) <= 2e-6
    assert max(rel(K[k], Kr[k]) for k in range(w.m)) <= 2e-6


def test_batch_replays_from_a_cuda_graph(esmf, mols):
    import torch
    fbs = builders(esmf, mols, ["fp16x2"] * len(mols))
    try:
        Ds = [torch.from_numpy(w.D).cuda() for w in mols]
        ref = [(J.cpu().numpy(), K.cpu().numpy()) for J, K in esmf.build_batch(fbs, Ds)]
        Js = [torch.zeros_like(D) for D in Ds]
        Ks = [torch.zeros_like(D) for D in Ds]
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            esmf.esmf_fock_build_batch([fb.h for fb in fbs], [w.m for w in mols], Ds, Js, Ks)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        for J, K, (Jr, Kr) in zip(Js, Ks, ref):
            assert rel(J.cpu().numpy(), Jr) < 1e-12 and rel(K.cpu().numpy(), Kr) < 1e-12
    finally:
        for fb in fbs:
            fb.close()


def test_bad_batches_are_rejected(esmf, mols):
    import torch
    w = mols[0]
    D = torch.from_numpy(w.D).cuda()
    J, K = torch.empty_like(D), torch.empty_like(D)
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp16x2") as a, \
            esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as b:
        for hs in ([], [a.h] * 17, [a.h, a.h]):
            with pytest.raises(esmf.EsmfError):
                esmf.esmf_fock_build_batch(hs, [w.m] * len(hs), [D] * len(hs), [J] * len(hs), [K] * len(hs))
        with pytest.raises(esmf.EsmfError) as ei:             # FP64 handle: not on the tensor path
            esmf.esmf_fock_build_batch([a.h, b.h], [w.m] * 2, [D] * 2, [J, J.clone()], [K, K.clone()])
        assert ei.value.code == esmf.ESMF_ERR_UNSUPPORTED
