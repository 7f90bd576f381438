"""esmf_fock_build_noalloc: the build for callers that may not allocate device
memory while building (an application that owns all device memory through
its own pool, or a latency-critical loop where cudaMalloc would stall other
streams).  It must give the same J, K, F and traces as esmf_fock_build, call
after call, although every call reuses one static scratch array.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest

from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# tolerance of each handle's arithmetic: stored FP64 runs the same kernels on
# both entry points; a split FP16 hi+lo store runs the tensor-core kernel in
# esmf_fock_build and the CUDA-core kernel here, equal within the FP32-class
# tolerance of that precision; integral-direct FP32 runs the same kernel
TOL = {"fp64": 1e-10, "fp32": 2e-6, "fp16x2": 2e-6}


def relerr(x, r):
    nr = float(np.linalg.norm(r))
    return float(np.linalg.norm(x - r)) / (nr if nr > 0 else 1.0)


@pytest.mark.parametrize("case,mode,prec", [("tiny", "stored", "fp64"), ("ragged", "stored", "fp64"),
                                            ("ragged", "stored", "fp16x2"), ("ragged", "direct", "fp32"),
                                            ("ragged", "direct", "fp16x2")])
def test_noalloc_matches_build_twice(esmf, case, mode, prec):
    import torch
    if case == "tiny":
        w = W.tiny()
        D = w.D
    else:
        w = W.small_random(37, 5, 5, tol=1e-10, edge=13.25)
        D = w.D + 0.3 * np.random.default_rng(5).standard_normal(w.D.shape)
    tol = TOL[prec]
    with esmf.FockBuilder(w.basis, w.tol, mode, prec) as fb:
        Dt = torch.from_numpy(np.ascontiguousarray(D)).cuda()
        m = Dt.shape[0]
        J0, K0, F0, t0 = fb.build(Dt, want_F=True)
        torch.cuda.synchronize()
        for _ in range(2):                      # two calls in a row share the scratch
            J = torch.full_like(Dt, np.nan)
            K = torch.full_like(Dt, np.nan)
            F = torch.full_like(Dt, np.nan)
            t = torch.full((m,), np.nan, dtype=torch.float64, device=Dt.device)
            esmf.esmf_fock_build_noalloc(fb.h, m, Dt, J, K, F, t)
            torch.cuda.synchronize()
            for a, b in ((J, J0), (K, K0), (F, F0)):
                for k in range(m):
                    assert relerr(a[k].cpu().numpy(), b[k].cpu().numpy()) <= tol, (prec, k)
            tn, t0n = t.cpu().numpy(), t0.cpu().numpy()
            scale = np.linalg.norm(Dt.cpu().numpy().reshape(m, -1), axis=1) * \
                np.linalg.norm(F0.cpu().numpy().reshape(m, -1), axis=1)
            assert np.all(np.abs(tn - t0n) <= tol * np.maximum(np.abs(t0n), scale)), prec


def test_noalloc_rejects_sizes_beyond_the_static_scratch(esmf):
    import torch
    w = W.small_random(400, 1, 9, tol=1e-10, edge=20.0)
    with esmf.FockBuilder(w.basis, w.tol, "direct", "fp32") as fb:
        np_ = 400
        m = esmf.NOALLOC_MAX_SCRATCH_DOUBLES // (2 * np_ * np_) + 1
        D = torch.zeros((m, 400, 400), dtype=torch.float64, device="cuda")
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        with pytest.raises(esmf.EsmfError) as e:
            esmf.esmf_fock_build_noalloc(fb.h, m, D, J, K)
        assert e.value.code == esmf.ESMF_ERR_INVALID_ARG
        assert "static limit" in esmf.esmf_last_error()
