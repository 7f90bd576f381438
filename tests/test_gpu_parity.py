"""GPU parity: the CUDA library (called through its C ABI) against the FP64
oracle on the same seeded inputs.

Tolerances (relative Frobenius error per J_k and K_k, and relative trace
error): FP64 path <= 1e-10, FP32 and FP16 hi+lo paths <= 2e-6.  The BF16
hi+lo ablation keeps 16 significand bits, so it is held to 3e-5.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "f32x2": 1e-10, "fp32": 2e-6, "fp16x2": 2e-6, "bf16x2": 3e-5}


def relerr(x, r):
    nr = np.linalg.norm(r)
    return np.linalg.norm(x - r) / (nr if nr > 0 else 1.0)


def trace_err(t, tr, D, F):
    scale = np.maximum(np.abs(tr), np.linalg.norm(D.reshape(D.shape[0], -1), axis=1) *
                       np.linalg.norm(F.reshape(F.shape[0], -1), axis=1))
    return np.max(np.abs(t - tr) / np.where(scale > 0, scale, 1.0))


def gpu_build(fock, w, mode, prec, D=None):
    import torch
    D = w.D if D is None else D
    with fock.FockBuilder(w.basis, w.tol, mode, prec) as fb:
        Dt = torch.from_numpy(np.ascontiguousarray(D)).cuda()
        J, K, F, t = fb.build(Dt, want_F=True)
        torch.cuda.synchronize()
        st = fb.stats()
        return J.cpu().numpy(), K.cpu().numpy(), F.cpu().numpy(), t.cpu().numpy(), st


def check(J, K, F, t, Jr, Kr, D, tol, label):
    Fr, tr = Oracle.fock_traces(D, Jr, Kr)
    for k in range(D.shape[0]):
        ej, ek = relerr(J[k], Jr[k]), relerr(K[k], Kr[k])
        assert ej <= tol and ek <= tol, (label, k, ej, ek)
    assert relerr(F, Fr) <= tol, label
    assert trace_err(t, tr, D, Fr) <= tol, (label, t, tr)


@pytest.fixture(scope="module")
def tiny_ref():
    w = W.tiny()
    o = Oracle(w.basis)
    E = o.eri_tensor()
    Jr, Kr = o.jk_brute(E, w.D, w.tol)
    return w, o, Jr, Kr


@pytest.mark.parametrize("mode,prec", [("stored", "fp64"), ("stored", "fp32"), ("direct", "fp64"),
                                       ("direct", "fp32"), ("stored", "fp16x2"), ("stored", "bf16x2"),
                                       ("stored", "f32x2"), ("direct", "fp16x2"), ("direct", "bf16x2")])
def test_tiny_all_paths(esmf, tiny_ref, mode, prec):
    w, o, Jr, Kr = tiny_ref
    J, K, F, t, st = gpu_build(esmf, w, mode, prec)
    check(J, K, F, t, Jr, Kr, w.D, TOL[prec], (mode, prec))
    P = w.basis.n * (w.basis.n + 1) // 2
    assert st["n_quartets_kept"] == P * (P + 1) // 2


def test_schwarz_table(esmf, tiny_ref):
    w, o, _, _ = tiny_ref
    with esmf.FockBuilder(w.basis, 0.0) as fb:
        Q = fb.schwarz()
    assert np.max(np.abs(Q - o.Q) / np.maximum(o.Q, 1e-300)) <= 1e-12


@pytest.mark.parametrize("n,m,tol,seed", [(1, 1, 0.0, 1), (8, 2, 0.0, 2), (9, 3, 1e-9, 3),
                                          (21, 5, 1e-7, 4), (37, 4, 1e-10, 5)])
@pytest.mark.parametrize("mode,prec", [("stored", "fp64"), ("direct", "fp32"), ("stored", "fp16x2"),
                                       ("direct", "fp64"), ("stored", "f32x2"), ("direct", "fp16x2")])
def test_ragged_sizes(esmf, n, m, tol, seed, mode, prec):
    w = W.small_random(n, m, seed, tol=tol, edge=4.0 + n / 4)
    rng = np.random.default_rng(seed)
    D = w.D + 0.3 * rng.standard_normal(w.D.shape)           # non-symmetric
    o = Oracle(w.basis)
    Jr, Kr, nk = o.jk_unique(D, tol)
    J, K, F, t, st = gpu_build(esmf, w, mode, prec, D)
    check(J, K, F, t, Jr, Kr, D, TOL[prec], (n, mode, prec))
    assert st["n_quartets_kept"] == nk == o.count_kept(tol)


def test_everything_screened_gives_zero(esmf):
    w = W.small_random(12, 2, 6)
    import torch
    with esmf.FockBuilder(w.basis, 1e6) as fb:
        J, K, F, t = fb.build(torch.from_numpy(w.D).cuda(), want_F=True)
        assert fb.stats()["n_bricks"] == 0
    assert float(J.abs().max()) == 0.0 and float(K.abs().max()) == 0.0 and float(t.abs().max()) == 0.0


def test_grouped_equals_separate_and_host_entry(esmf, tiny_ref):
    import torch
    w, _, _, _ = tiny_ref
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        J, K, _, t = fb.build(torch.from_numpy(w.D).cuda())
        for k in range(w.m):
            Jk, Kk, _, tk = fb.build(torch.from_numpy(w.D[k:k + 1].copy()).cuda())
            assert relerr(Jk[0].cpu().numpy(), J[k].cpu().numpy()) <= 1e-13
            assert relerr(Kk[0].cpu().numpy(), K[k].cpu().numpy()) <= 1e-13
        Jh, Kh, th = fb.build_host(np.ascontiguousarray(w.D), traces=np.zeros(w.m))
        assert relerr(Jh, J.cpu().numpy()) <= 1e-13 and relerr(Kh, K.cpu().numpy()) <= 1e-13
        assert np.allclose(th, t.cpu().numpy(), rtol=1e-12)


def test_fd_derivative_identity_on_gpu(esmf, tiny_ref):
    """d/dTheta_kp (F[Theta^T Theta] . Theta^T Theta) = 4 (Theta F)_kp
    (Appendix, Eq. eng2_der_theta_kp4) with every F from the GPU build."""
    import torch
    w, _, _, _ = tiny_ref
    rng = np.random.default_rng(12)
    n, no = w.basis.n, 3
    Th = rng.standard_normal((no, n)) / math.sqrt(n)
    with esmf.FockBuilder(w.basis, 0.0, "stored", "fp64") as fb:
        def fock_of(T):
            D = torch.from_numpy((T.T @ T)[None].copy()).cuda()
            _, _, F, t = fb.build(D, want_F=True)
            return F[0].cpu().numpy(), float(t[0])
        F0, _ = fock_of(Th)
        grad = 4 * Th @ F0
        h = 1e-4
        for (k, p) in [(0, 1), (1, 9), (2, 20)]:
            Tp, Tm = Th.copy(), Th.copy()
            Tp[k, p] += h
            Tm[k, p] -= h
            fd = (fock_of(Tp)[1] - fock_of(Tm)[1]) / (2 * h)
            assert abs(fd - grad[k, p]) <= 1e-7 * max(1.0, abs(grad[k, p]))


def test_invalid_build_arguments(esmf, tiny_ref):
    import torch
    w, _, _, _ = tiny_ref
    with esmf.FockBuilder(w.basis, 0.0) as fb:
        D = torch.from_numpy(w.D).cuda()
        J = torch.empty_like(D)
        with pytest.raises(esmf.EsmfError) as e:
            esmf.esmf_fock_build(fb.h, 0, D, J, J)
        assert e.value.code == esmf.ESMF_ERR_INVALID_ARG
        Dh = torch.from_numpy(w.D)        # host memory passed as device
        with pytest.raises(esmf.EsmfError) as e:
            esmf.esmf_fock_build(fb.h, w.m, Dh, J, J)
        assert e.value.code == esmf.ESMF_ERR_INVALID_ARG


# ------------------------------------------------------------- full sizes
# Whole-matrix parity at the full workload sizes lives in test_gpu_fullsize.py.
def test_direct_small_ribbon_full(esmf):
    w = W.direct(length=6, m=5)
    o = Oracle(w.basis)
    Jr, Kr, nk = o.jk_unique(w.D, w.tol)
    J, K, F, t, st = gpu_build(esmf, w, "direct", "fp32")
    check(J, K, F, t, Jr, Kr, w.D, TOL["fp32"], "direct ribbon")
    assert st["n_quartets_kept"] == nk


# ------------------------------------------------------------- tensor cores
@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
@pytest.mark.parametrize("case", ["ragged", "stored"])
def test_tensor_path_matches_cuda_core_path(esmf, prec, case):
    """The tcgen05 kernel and the CUDA-core kernel read the same split store;
    they must agree to the split precision, and the tensor kernel must report
    no expired wait."""
    import torch
    if case == "ragged":
        w = W.small_random(37, 5, 5, tol=1e-10, edge=13.25)
    else:
        w = W.stored()
    D = torch.from_numpy(np.ascontiguousarray(w.D)).cuda()
    with esmf.FockBuilder(w.basis, w.tol, "stored", prec) as fb:
        J1, K1, _, t1 = fb.build(D)
        torch.cuda.synchronize()
        assert fb.device_error() == 0
        fb.set_path("cuda_core")
        J2, K2, _, t2 = fb.build(D)
        torch.cuda.synchronize()
    tol = TOL[prec]
    for k in range(w.m):
        assert relerr(J1[k].cpu().numpy(), J2[k].cpu().numpy()) <= tol
        assert relerr(K1[k].cpu().numpy(), K2[k].cpu().numpy()) <= tol


@pytest.mark.parametrize("prec", ["fp16x2", "fp32", "fp64"])
def test_autotune_keeps_results(esmf, prec):
    """The autotuner may change how many densities each pass contracts; the
    results must not change beyond the precision's tolerance."""
    import torch
    w = W.small_random(37, 12, 5, tol=1e-10, edge=13.25)
    D = torch.from_numpy(w.D).cuda()
    with esmf.FockBuilder(w.basis, w.tol, "stored", prec) as fb:
        J0, K0, _, _ = fb.build(D)
        chosen = fb.autotune(D, reps=2)
        J1, K1, _, _ = fb.build(D)
        torch.cuda.synchronize()
    assert chosen in (4, 8, 16)
    for k in range(w.m):
        assert relerr(J1[k].cpu().numpy(), J0[k].cpu().numpy()) <= TOL[prec]
        assert relerr(K1[k].cpu().numpy(), K0[k].cpu().numpy()) <= TOL[prec]
