"""Bases with Cartesian p and d functions (esmf_fock_create_cart) on the GPU
against the oracle's Obara-Saika integrals: the Schwarz table, kept-quartet
counts and J, K, F, traces of every store precision, including the
tensor-core path, and integral-direct builds; the entries that take s
functions only (pair-max rule, density fitting) must refuse."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-6, "fp16x2": 2e-6, "bf16x2": 3e-5}


def rel(x, r):
    return float(np.linalg.norm(x - r)) / max(float(np.linalg.norm(r)), 1e-300)


@pytest.fixture(scope="module")
def sp_tiny():
    w = W.sp_random(3, 3, 7, tol=0.0, edge=3.0, min_dist=0.8)        # 12 functions
    o = Oracle(w.basis)
    D = w.D + 0.2 * np.random.default_rng(1).standard_normal(w.D.shape)
    Jr, Kr = o.jk_brute(o.eri_tensor(), D, 0.0)
    return w, o, D, Jr, Kr


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16x2", "bf16x2"])
def test_tiny_sp_all_precisions(esmf, sp_tiny, prec):
    import torch
    w, o, D, Jr, Kr = sp_tiny
    with esmf.FockBuilder(w.basis, 0.0, "stored", prec) as fb:
        J, K, F, t = fb.build(torch.from_numpy(D).cuda(), want_F=True)
        torch.cuda.synchronize()
        assert fb.device_error() == 0
        Q = fb.schwarz()
    J, K, F, t = J.cpu().numpy(), K.cpu().numpy(), F.cpu().numpy(), t.cpu().numpy()
    Fr, tr = Oracle.fock_traces(D, Jr, Kr)
    for k in range(D.shape[0]):
        assert rel(J[k], Jr[k]) <= TOL[prec] and rel(K[k], Kr[k]) <= TOL[prec], (prec, k)
    assert rel(F, Fr) <= TOL[prec]
    scale = np.maximum(np.abs(tr), np.linalg.norm(D.reshape(D.shape[0], -1), axis=1) *
                       np.linalg.norm(Fr.reshape(D.shape[0], -1), axis=1))
    assert np.all(np.abs(t - tr) <= TOL[prec] * scale)
    assert np.max(np.abs(Q - o.Q)) <= 1e-12 * np.max(o.Q)


@pytest.mark.parametrize("prec", ["fp64", "fp16x2"])
def test_screened_sp_molecule(esmf, prec):
    """32 functions (8 centers, s and p shells), 4 densities, tol 1e-8: kept
    quartets equal the oracle's exactly; J, K within the precision."""
    import torch
    w = W.sp_random(8, 4, 3, tol=1e-8)
    o = Oracle(w.basis)
    Jr, Kr, nk = o.jk_unique(w.D, w.tol)
    with esmf.FockBuilder(w.basis, w.tol, "stored", prec) as fb:
        J, K, _, _ = fb.build(torch.from_numpy(w.D).cuda())
        torch.cuda.synchronize()
        st = fb.stats()
    assert st["n_quartets_kept"] == nk
    J, K = J.cpu().numpy(), K.cpu().numpy()
    for k in range(w.m):
        assert rel(J[k], Jr[k]) <= TOL[prec] and rel(K[k], Kr[k]) <= TOL[prec], (prec, k, rel(K[k], Kr[k]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_integral_direct_sp(esmf, sp_tiny, prec):
    """Integral-direct builds evaluate the p integrals inside every build."""
    import torch
    w, o, D, Jr, Kr = sp_tiny
    with esmf.FockBuilder(w.basis, 0.0, "direct", prec) as fb:
        J, K, _, _ = fb.build(torch.from_numpy(D).cuda())
        torch.cuda.synchronize()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    for k in range(D.shape[0]):
        assert rel(J[k], Jr[k]) <= TOL[prec] and rel(K[k], Kr[k]) <= TOL[prec], (prec, k)


def test_paths_without_p_integrals_refuse(esmf):
    w = W.sp_random(2, 1, 5)
    with pytest.raises(ValueError):
        esmf.FockBuilder(w.basis, 1e-10, "stored", "fp64", screening="pair_max")
    with pytest.raises(ValueError):
        esmf.FockBuilder(w.basis, 0.0, "df", "fp64", aux=W.even_tempered_aux(w.basis))


@pytest.fixture(scope="module")
def spd_tiny():
    w = W.spd_random(2, 3, 11, tol=0.0, edge=2.6, min_dist=1.0, nprim=2)   # 20 functions: s, p, d per centre
    o = Oracle(w.basis)
    D = w.D + 0.2 * np.random.default_rng(2).standard_normal(w.D.shape)
    Jr, Kr = o.jk_brute(o.eri_tensor(), D, 0.0)
    return w, o, D, Jr, Kr


def check_all(J, K, F, t, D, Jr, Kr, tol):
    Fr, tr = Oracle.fock_traces(D, Jr, Kr)
    for k in range(D.shape[0]):
        assert rel(J[k], Jr[k]) <= tol and rel(K[k], Kr[k]) <= tol, (k, rel(J[k], Jr[k]), rel(K[k], Kr[k]))
    if F is not None:
        assert rel(F, Fr) <= tol
        scale = np.maximum(np.abs(tr), np.linalg.norm(D.reshape(D.shape[0], -1), axis=1) *
                           np.linalg.norm(Fr.reshape(D.shape[0], -1), axis=1))
        assert np.all(np.abs(t - tr) <= tol * scale)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16x2", "bf16x2"])
def test_tiny_spd_all_precisions(esmf, spd_tiny, prec):
    """d functions (McMurchie-Davidson on the device, Obara-Saika in the
    oracle): every store precision, the Schwarz table to 1e-12."""
    import torch
    w, o, D, Jr, Kr = spd_tiny
    with esmf.FockBuilder(w.basis, 0.0, "stored", prec) as fb:
        J, K, F, t = fb.build(torch.from_numpy(D).cuda(), want_F=True)
        torch.cuda.synchronize()
        assert fb.device_error() == 0
        Q = fb.schwarz()
    check_all(J.cpu().numpy(), K.cpu().numpy(), F.cpu().numpy(), t.cpu().numpy(), D, Jr, Kr, TOL[prec])
    assert np.max(np.abs(Q - o.Q)) <= 1e-12 * np.max(o.Q)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_integral_direct_spd(esmf, spd_tiny, prec):
    import torch
    w, o, D, Jr, Kr = spd_tiny
    with esmf.FockBuilder(w.basis, 0.0, "direct", prec) as fb:
        J, K, _, _ = fb.build(torch.from_numpy(D).cuda())
        torch.cuda.synchronize()
    check_all(J.cpu().numpy(), K.cpu().numpy(), None, None, D, Jr, Kr, TOL[prec])


@pytest.fixture(scope="module")
def spd_screened():
    w = W.spd_random(4, 3, 5, tol=1e-8, nprim=2)
    Jr, Kr, nk = Oracle(w.basis).jk_unique(w.D, w.tol)
    return w, Jr, Kr, nk


@pytest.mark.parametrize("prec", ["fp64", "fp16x2"])
def test_screened_spd_molecule(esmf, spd_screened, prec):
    """40 functions (4 centres of s, p and d shells), 3 densities, tol 1e-8:
    kept quartets equal the oracle's exactly; J, K within the precision."""
    import torch
    w, Jr, Kr, nk = spd_screened
    with esmf.FockBuilder(w.basis, w.tol, "stored", prec) as fb:
        J, K, _, _ = fb.build(torch.from_numpy(w.D).cuda())
        torch.cuda.synchronize()
        st = fb.stats()
    assert st["n_quartets_kept"] == nk
    check_all(J.cpu().numpy(), K.cpu().numpy(), None, None, w.D, Jr, Kr, TOL[prec])
