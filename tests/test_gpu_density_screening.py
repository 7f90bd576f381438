"""Density-weighted screening on the GPU against the oracle's rule.

A Schwarz-kept quartet is also dropped when Q_pq Q_rs times the largest
|D_k| of its six index pairs is below tol_d.  Every path must give the
oracle's J and K for that rule within the arithmetic's tolerance; tol_d = 0
must give the plain build; the handles that cannot apply it must say so.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-6, "fp16x2": 2e-6}


def rel(x, r):
    return float(np.linalg.norm(x - r)) / max(float(np.linalg.norm(r)), 1e-300)


@pytest.fixture(scope="module")
def case():
    w = W.small_random(37, 5, 5, tol=1e-10, edge=13.25)
    D = w.D + 0.02 * np.random.default_rng(9).standard_normal(w.D.shape)    # non-symmetric
    o = Oracle(w.basis)
    tol_d = 1e-5
    Jd, Kd, nkd = o.jk_unique_dw(D, w.tol, tol_d)
    _, _, nk = o.jk_unique(D, w.tol)
    assert 0 < nkd < nk                                                      # the rule bites
    return w, D, tol_d, Jd, Kd


@pytest.mark.parametrize("mode,prec", [("stored", "fp64"), ("stored", "fp32"), ("stored", "fp16x2"),
                                       ("direct", "fp64"), ("direct", "fp32")])
def test_density_screened_build_matches_oracle(esmf, case, mode, prec):
    import torch
    w, D, tol_d, Jd, Kd = case
    with esmf.FockBuilder(w.basis, w.tol, mode, prec) as fb:
        fb.set_density_screening(tol_d)
        J, K, _, _ = fb.build(torch.from_numpy(D).cuda())
        torch.cuda.synchronize()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    for k in range(D.shape[0]):
        assert rel(J[k], Jd[k]) <= TOL[prec], (k, rel(J[k], Jd[k]))
        assert rel(K[k], Kd[k]) <= TOL[prec], (k, rel(K[k], Kd[k]))


def test_zero_threshold_is_the_plain_build(esmf, case):
    import torch
    w, D, _, _, _ = case
    Dt = torch.from_numpy(D).cuda()
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        J0, K0, _, _ = fb.build(Dt)
        fb.set_density_screening(0.0)
        J1, K1, _, _ = fb.build(Dt)
        torch.cuda.synchronize()
    assert rel(J1.cpu().numpy(), J0.cpu().numpy()) <= 1e-13
    assert rel(K1.cpu().numpy(), K0.cpu().numpy()) <= 1e-13


def test_stored_n200_m16_within_the_screening_bound(esmf):
    """At the benchmark size: every dropped update is below tol_d, so the
    screened build differs from the plain one by at most tol_d times the N^2
    updates of an element; in practice far less."""
    import torch
    w = W.stored()
    n = w.basis.n
    D = torch.from_numpy(w.D).cuda()
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        J0, K0, _, _ = fb.build(D)
        for tol_d in (1e-9, 1e-6):
            fb.set_density_screening(tol_d)
            J1, K1, _, _ = fb.build(D)
            torch.cuda.synchronize()
            dj = float((J1 - J0).abs().max())
            dk = float((K1 - K0).abs().max())
            print(f"\nDENSITY-SCREENED stored_n200_m16 tol_d {tol_d:g}: max |dJ| {dj:.2e} max |dK| {dk:.2e}")
            assert dj <= tol_d * n * n and dk <= tol_d * n * n


def test_entries_that_cannot_apply_it_refuse(esmf, case):
    import torch
    w, D, tol_d, _, _ = case
    Dt = torch.from_numpy(D).cuda()
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp16x2") as fb:
        fb.set_density_screening(tol_d)
        J, K = torch.empty_like(Dt), torch.empty_like(Dt)
        with pytest.raises(esmf.EsmfError) as e:
            esmf.esmf_fock_build_batch([fb.h], [Dt.shape[0]], [Dt], [J], [K])
        assert e.value.code == esmf.ESMF_ERR_UNSUPPORTED
        with pytest.raises(esmf.EsmfError) as e:
            esmf.esmf_fock_build_noalloc(fb.h, Dt.shape[0], Dt, J, K)
        assert e.value.code == esmf.ESMF_ERR_UNSUPPORTED
        with pytest.raises(esmf.EsmfError) as e:
            fb.set_density_screening(-1.0)
        assert e.value.code == esmf.ESMF_ERR_INVALID_ARG
