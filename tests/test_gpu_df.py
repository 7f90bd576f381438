"""Density-fitted J and K on the GPU (esmf_fock_create_df) against the
oracle's fit, and against the exact integrals where the fit is exact.

FP64 GEMMs are held to the FP64 tolerance 1e-10.  FP32 GEMMs accumulate
inner products of length N x n_aux in FP32, so their error grows like
sqrt(N n_aux) x 2^-24; at these sizes it is held to 1e-5.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(x, r):
    return float(np.linalg.norm(x - r)) / max(float(np.linalg.norm(r)), 1e-300)


def gpu_df(esmf, basis, aux, D, prec):
    import torch
    with esmf.FockBuilder(basis, 0.0, "df", prec, aux=aux) as fb:
        J, K, F, t = fb.build(torch.from_numpy(np.ascontiguousarray(D)).cuda(), want_F=True)
        torch.cuda.synchronize()
        st = fb.stats()
    return J.cpu().numpy(), K.cpu().numpy(), F.cpu().numpy(), t.cpu().numpy(), st


def test_exact_fit_gives_the_exact_build(esmf):
    """Auxiliaries = every primitive product: the fitted integrals are the
    exact ones, so the GPU's density-fitted J and K equal the oracle's exact
    build."""
    cen = np.array([[0, 0, 0], [1.2, 0.3, -0.4], [-0.5, 1.7, 0.9]], float)
    ex = np.array([0.4, 1.3, 3.1])
    b = W.Basis(cen, np.ones(3, dtype=np.int32), ex, np.ones(3))
    ac = np.array([(ex[i] * cen[i] + ex[j] * cen[j]) / (ex[i] + ex[j]) for i in range(3) for j in range(i + 1)])
    ae = np.array([ex[i] + ex[j] for i in range(3) for j in range(i + 1)])
    D = np.random.default_rng(1).standard_normal((3, 3, 3))
    o = Oracle(b)
    Jr, Kr = o.jk_brute(o.eri_tensor(), D, 0.0)
    J, K, _, _, _ = gpu_df(esmf, b, (ac, ae), D, "fp64")
    assert rel(J, Jr) <= 1e-10 and rel(K, Kr) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_matches_the_oracle_fit(esmf, prec, tol):
    w = W.small_random(40, 6, 21, tol=0.0, edge=8.0)
    D = w.D + 0.05 * np.random.default_rng(3).standard_normal(w.D.shape)        # non-symmetric
    aux = W.even_tempered_aux(w.basis)
    o = Oracle(w.basis)
    Jr, Kr = o.jk_df(D, *aux)
    Fr, tr = Oracle.fock_traces(D, Jr, Kr)
    J, K, F, t, st = gpu_df(esmf, w.basis, aux, D, prec)
    assert st["mode"] == 3
    for k in range(D.shape[0]):
        assert rel(J[k], Jr[k]) <= tol and rel(K[k], Kr[k]) <= tol, (k, rel(J[k], Jr[k]), rel(K[k], Kr[k]))
    assert rel(F, Fr) <= tol
    scale = np.maximum(np.abs(tr), np.linalg.norm(D.reshape(D.shape[0], -1), axis=1) *
                       np.linalg.norm(Fr.reshape(D.shape[0], -1), axis=1))
    assert np.all(np.abs(t - tr) <= tol * scale)
    # and the fit's own error against the exact build, for the record
    Je, Ke, _ = o.jk_unique(D, 0.0)
    print(f"\nDF n={w.basis.n} n_aux={aux[1].size} {prec}: vs oracle fit J {max(rel(J[k], Jr[k]) for k in range(D.shape[0])):.2e} "
          f"K {max(rel(K[k], Kr[k]) for k in range(D.shape[0])):.2e}; fit vs exact J {rel(Jr, Je):.2e} K {rel(Kr, Ke):.2e}")


def test_entries_without_a_fitted_path_refuse(esmf):
    import torch
    w = W.small_random(12, 2, 22, edge=5.0)
    aux = W.even_tempered_aux(w.basis, count=4)
    Dt = torch.from_numpy(w.D).cuda()
    J, K = torch.empty_like(Dt), torch.empty_like(Dt)
    with esmf.FockBuilder(w.basis, 0.0, "df", "fp64", aux=aux) as fb:
        for call in (lambda: esmf.esmf_fock_build_noalloc(fb.h, 2, Dt, J, K),
                     lambda: esmf.esmf_fock_build_shard(fb.h, 0, 2, 2, Dt, J, K),
                     lambda: fb.autotune(Dt),
                     lambda: esmf.esmf_fock_build_batch([fb.h], [2], [Dt], [J], [K]),
                     lambda: fb.set_density_screening(1e-6)):
            with pytest.raises(esmf.EsmfError) as e:
                call()
            assert e.value.code == esmf.ESMF_ERR_UNSUPPORTED
    with pytest.raises(esmf.EsmfError) as e:
        esmf.FockBuilder(w.basis, 0.0, "df", "fp16x2", aux=aux)
    assert e.value.code == esmf.ESMF_ERR_UNSUPPORTED
    dup = (np.vstack([aux[0], aux[0][:1]]), np.concatenate([aux[1], aux[1][:1]]))   # singular metric
    with pytest.raises(esmf.EsmfError) as e:
        esmf.FockBuilder(w.basis, 0.0, "df", "fp64", aux=dup)
    assert e.value.code == esmf.ESMF_ERR_INVALID_ARG
