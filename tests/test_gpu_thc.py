"""Tensor-hypercontracted J and K on the GPU (esmf_fock_create_thc) against
the oracle's least-squares THC (same grid, Schwarz tolerance and ridge), and
against the exact build where the grid spans every orbital product.

The fit Z = (S + lam I)^-1 E (S + lam I)^-1 is conditioned to about 1/ridge,
so the rounding of E and S (different summation orders here and in the
oracle) moves J and K by about 2e-16 / ridge relative: FP64 builds are held
to 1e-9 at ridge 1e-6 and 2e-7 at ridge 1e-8.  FP32 GEMMs (inner products of
length N and n_grid against the cancelling entries of Z) add about 2e-6 and
are held to 2e-5.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(x, r):
    return float(np.linalg.norm(x - r)) / max(float(np.linalg.norm(r)), 1e-300)


def gpu_thc(esmf, basis, pts, tol, ridge, D, prec):
    import torch
    with esmf.FockBuilder(basis, tol, "thc", prec, grid=pts, ridge=ridge) as fb:
        J, K, F, t = fb.build(torch.from_numpy(np.ascontiguousarray(D)).cuda(), want_F=True)
        torch.cuda.synchronize()
        st = fb.stats()
    return J.cpu().numpy(), K.cpu().numpy(), F.cpu().numpy(), t.cpu().numpy(), st


def oracle_thc(o, fit, D):
    """J and K of Eq. (J_and_K) over the oracle's fitted tensor (fit = (X, Z))."""
    V = Oracle.thc_tensor(*fit)
    J = np.einsum("pqrs,krs->kpq", V, D, optimize=True)
    K = np.einsum("pqrs,kqs->kpr", V, D, optimize=True)
    return J, K


def check(J, K, F, t, D, Jr, Kr, tol):
    Fr, tr = Oracle.fock_traces(D, Jr, Kr)
    for k in range(D.shape[0]):
        assert rel(J[k], Jr[k]) <= tol and rel(K[k], Kr[k]) <= tol, (k, rel(J[k], Jr[k]), rel(K[k], Kr[k]))
    assert rel(F, Fr) <= tol
    scale = np.maximum(np.abs(tr), np.linalg.norm(D.reshape(D.shape[0], -1), axis=1) *
                       np.linalg.norm(Fr.reshape(D.shape[0], -1), axis=1))
    assert np.all(np.abs(t - tr) <= tol * scale)


@pytest.fixture(scope="module")
def mol40():
    """40 s functions on 20 random centers, tol 1e-10, the 21-point-per-center
    grid (420 points), 16 ESMF densities plus a non-symmetric perturbation."""
    w = W.small_random(40, 16, 1, tol=1e-10, min_dist=1.4)
    D = w.D + 0.05 * np.random.default_rng(5).standard_normal(w.D.shape)
    o = Oracle(w.basis)
    return w, D, o, W.thc_grid(w.basis), {}


@pytest.mark.parametrize("prec,ridge,tol", [("fp64", 1e-6, 1e-9), ("fp64", 1e-8, 2e-7), ("fp32", 1e-8, 2e-5)])
def test_matches_the_oracle_fit(esmf, mol40, prec, ridge, tol):
    w, D, o, pts, fits = mol40
    if ridge not in fits:
        fits[ridge] = o.thc_fit(pts, w.tol, ridge)
    Jr, Kr = oracle_thc(o, fits[ridge], D)
    J, K, F, t, st = gpu_thc(esmf, w.basis, pts, w.tol, ridge, D, prec)
    assert st["mode"] == 4
    assert st["n_quartets_kept"] == o.count_kept(w.tol)
    check(J, K, F, t, D, Jr, Kr, tol)
    Je, Ke, _ = o.jk_unique(D, w.tol)
    print(f"\nTHC n={w.basis.n} n_grid={pts.shape[0]} ridge={ridge} {prec}: vs oracle fit "
          f"J {max(rel(J[k], Jr[k]) for k in range(D.shape[0])):.2e} "
          f"K {max(rel(K[k], Kr[k]) for k in range(D.shape[0])):.2e}; "
          f"fit vs exact J {rel(Jr, Je):.2e} K {rel(Kr, Ke):.2e}")


def test_pair_space_grid_reproduces_the_exact_build(esmf):
    """21 generic points for 6 functions: the pair products span the pair
    space and the ridge-0 fit is exact, so the GPU's hypercontracted build
    equals the oracle's exact one (to the conditioning of the normal
    equations, S ~ 1e11 here: rounding of 3e-16 in E and S moves J and K by
    at most 4e-8 on this case)."""
    w = W.small_random(6, 3, 3, tol=0.0)
    rng = np.random.default_rng(1)
    pts = w.basis.center[rng.integers(0, 6, 21)] + rng.normal(0.0, 0.7, (21, 3))
    o = Oracle(w.basis)
    Je, Ke = o.jk_brute(o.eri_tensor(), w.D, 0.0)
    J, K, F, t, _ = gpu_thc(esmf, w.basis, pts, 0.0, 0.0, w.D, "fp64")
    check(J, K, F, t, w.D, Je, Ke, 1e-6)


def test_batches_of_densities(esmf, mol40):
    """700 densities exceed one batch of per-build work (about 1 GiB: 680
    densities here), so the build runs two batches; every density, F and
    trace still equals the oracle."""
    w, _, o, pts, fits = mol40
    if 1e-6 not in fits:
        fits[1e-6] = o.thc_fit(pts, w.tol, 1e-6)
    D = np.random.default_rng(9).standard_normal((700, 40, 40))
    Jr, Kr = oracle_thc(o, fits[1e-6], D)
    J, K, F, t, _ = gpu_thc(esmf, w.basis, pts, w.tol, 1e-6, D, "fp64")
    check(J, K, F, t, D, Jr, Kr, 1e-9)


def test_entries_without_a_fitted_path_refuse(esmf):
    import torch
    w = W.small_random(12, 2, 22, edge=5.0)
    pts = W.thc_grid(w.basis, radii=(0.8,), corner=0.0)
    Dt = torch.from_numpy(w.D).cuda()
    J, K = torch.empty_like(Dt), torch.empty_like(Dt)
    with esmf.FockBuilder(w.basis, 0.0, "thc", "fp64", grid=pts, ridge=1e-6) as fb:
        for call in (lambda: esmf.esmf_fock_build_noalloc(fb.h, 2, Dt, J, K),
                     lambda: esmf.esmf_fock_build_shard(fb.h, 0, 2, 2, Dt, J, K),
                     lambda: fb.autotune(Dt),
                     lambda: esmf.esmf_fock_build_batch([fb.h], [2], [Dt], [J], [K]),
                     lambda: fb.set_density_screening(1e-6)):
            with pytest.raises(esmf.EsmfError) as e:
                call()
            assert e.value.code == esmf.ESMF_ERR_UNSUPPORTED
    dup = np.vstack([pts, pts[:1]])            # a repeated point: S + 0 I is singular
    with pytest.raises(esmf.EsmfError) as e:
        esmf.FockBuilder(w.basis, 0.0, "thc", "fp64", grid=dup, ridge=0.0)
    assert e.value.code == esmf.ESMF_ERR_INVALID_ARG
