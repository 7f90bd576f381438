"""Precision of every build path against the FP64 oracle, per result.

Full comparison (every J_k, K_k and D_k.F_k) on a C4-like molecule small enough
for the oracle (80 s functions on 40 random centers at the C4 density, m = 64
densities); the full C4 size (400 functions, m = 64) is compared with stored
oracle rows in test_gpu_fullsize.py.
Prints one line per path: max / median relative Frobenius error over k for J
and K, and the max relative trace error.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PATHS = [("stored", "fp64", 1e-10), ("stored", "fp32", 2e-6), ("stored", "fp16x2", 2e-6),
         ("stored", "bf16x2", 3e-5), ("direct", "fp32", 2e-6), ("direct", "fp64", 1e-10)]


def rel(x, r):
    return np.linalg.norm(x - r) / max(np.linalg.norm(r), 1e-300)


@pytest.fixture(scope="module")
def c4_small():
    rng = W.rng_for(W.BASE_SEED + 3 + 500)
    cen = W.cube_centers(rng, 40, 12.6 * (40 / 200) ** (1 / 3), 1.4)
    b = W.s_basis(rng, cen, 2, 3)
    D = W.esmf_densities(rng, b.n, 16, 64)
    w = W.Workload("precision_small_n80_m64", b, D, 1e-10, 16)
    Jr, Kr, _ = Oracle(w.basis).jk_unique(w.D, w.tol)
    Fr, tr = Oracle.fock_traces(w.D, Jr, Kr)
    return w, Jr, Kr, Fr, tr


@pytest.mark.parametrize("mode,prec,tol", PATHS)
def test_per_result_errors_small(esmf, c4_small, mode, prec, tol):
    import torch
    w, Jr, Kr, Fr, tr = c4_small
    with esmf.FockBuilder(w.basis, w.tol, mode, prec) as fb:
        J, K, F, t = fb.build(torch.from_numpy(w.D).cuda(), want_F=True)
        J, K, t = J.cpu().numpy(), K.cpu().numpy(), t.cpu().numpy()
    ej = np.array([rel(J[k], Jr[k]) for k in range(w.m)])
    ek = np.array([rel(K[k], Kr[k]) for k in range(w.m)])
    scale = np.maximum(np.abs(tr), np.linalg.norm(w.D.reshape(w.m, -1), axis=1) *
                       np.linalg.norm(Fr.reshape(w.m, -1), axis=1))
    et = np.abs(t - tr) / scale
    print(f"\nPRECISION {w.name} {mode}/{prec}: J max {ej.max():.2e} median {np.median(ej):.2e} | "
          f"K max {ek.max():.2e} median {np.median(ek):.2e} | trace max {et.max():.2e}")
    assert ej.max() <= tol and ek.max() <= tol and et.max() <= tol


def test_full_c4_split_against_fp32(esmf):
    """Whole matrices at the full C4 size (400 functions, 50 function blocks,
    so the tensor-core path splits items at 16 R blocks): the split FP16 build
    against the FP32 CUDA-core build (itself within about 2e-7 of FP64),
    relative Frobenius error of every J_k and K_k."""
    import torch
    w = W.precision()
    D = torch.from_numpy(w.D).cuda()
    out = {}
    for prec in ("fp32", "fp16x2"):
        with esmf.FockBuilder(w.basis, w.tol, "stored", prec) as fb:
            J, K, _, _ = fb.build(D, want_traces=False)
            out[prec] = (J.cpu().numpy(), K.cpu().numpy())
    (J32, K32), (J16, K16) = out["fp32"], out["fp16x2"]
    ej = max(rel(J16[k], J32[k]) for k in range(w.m))
    ek = max(rel(K16[k], K32[k]) for k in range(w.m))
    print(f"\nPRECISION {w.name} stored/fp16x2 vs stored/fp32, whole matrices: J {ej:.2e} K {ek:.2e}")
    assert ej <= 2e-6 and ek <= 2e-6
