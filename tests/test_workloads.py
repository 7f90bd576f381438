"""The seeded input recipe (paper_2002_00322_gb300/workloads.py): the same
seed gives the same inputs, and the geometry, basis and density properties
the recipe states hold.  The generators hold no integral or contraction
arithmetic; these tests pin the inputs both the oracle and the CUDA path
read.  CPU only."""
import numpy as np

from paper_2002_00322_gb300 import workloads as W


def pairwise_min(x):
    d = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=-1)
    return d[np.triu_indices(len(x), 1)].min()


def test_same_seed_same_inputs():
    a, b = W.stored(), W.stored()
    for f in ("center", "nprim", "exps", "coefs"):
        assert np.array_equal(getattr(a.basis, f), getattr(b.basis, f))
    assert np.array_equal(a.D, b.D)
    c = W.stored(seed_offset=1)
    assert not np.array_equal(a.basis.center, c.basis.center)


def test_stored_workload_geometry_and_basis():
    """200 functions, two per center on 100 centers in a 10 bohr cube at least
    1.4 bohr apart; 3 primitives with exponents in [0.1, 10] and coefficients
    in (0.1, 1]; m = 16, tol 1e-10."""
    w = W.stored()
    b = w.basis
    cen = np.unique(b.center, axis=0)
    assert b.n == 200 and cen.shape == (100, 3) and w.m == 16 and w.tol == 1e-10 and w.nocc == 40
    assert np.all((cen >= 0.0) & (cen <= 10.0))
    assert pairwise_min(cen) >= 1.4
    assert np.all(b.nprim == 3)
    assert np.all((b.exps >= 0.1) & (b.exps <= 10.0))
    assert np.all((b.coefs > 0.1) & (b.coefs <= 1.0))


def test_ribbon_lattice():
    """The integral-direct ribbon: a 4 x L square lattice at 1.4 bohr in the
    xy plane, two functions per site."""
    w = W.direct(length=12, m=4)
    cen = np.unique(w.basis.center, axis=0)
    assert cen.shape == (48, 3) and w.basis.n == 96
    assert np.all(cen[:, 2] == 0.0)
    assert np.allclose(np.sort(np.unique(np.round(cen[:, 0] / 1.4, 9))), np.arange(12))
    assert np.allclose(np.sort(np.unique(np.round(cen[:, 1] / 1.4, 9))), np.arange(4))


def test_esmf_densities_follow_table_one():
    """With orthonormal orbital rows V = [Theta; Gamma]: Theta^T Theta is a
    symmetric projector of trace N_o; Theta^T sigma Gamma is traceless and of
    unit norm (sigma of unit norm) and not symmetric; A = Gamma^T sigma^T sigma
    Gamma - Theta^T sigma sigma^T Theta is symmetric and traceless; extra
    densities past the nine are transition densities of unit norm."""
    rng = W.rng_for(123)
    n, nocc = 30, 6
    D = W.esmf_densities(rng, n, nocc, 12)
    P, T, A = D[0], D[1], D[2]
    assert np.allclose(P, P.T, atol=1e-13) and np.allclose(P @ P, P, atol=1e-12)
    assert abs(np.trace(P) - nocc) < 1e-12
    assert abs(np.trace(T)) < 1e-12 and abs(np.linalg.norm(T) - 1.0) < 1e-12
    assert np.abs(T - T.T).max() > 1e-3
    assert np.allclose(A, A.T, atol=1e-13) and abs(np.trace(A)) < 1e-12
    for k in range(9, 12):
        assert abs(np.trace(D[k])) < 1e-12 and abs(np.linalg.norm(D[k]) - 1.0) < 1e-12


def test_tiny_densities_closed_open_transition():
    """The tiny configuration's first two densities: closed shell P and the
    open-shell HOMO -> LUMO alpha density (same trace, P with the HOMO
    replaced by the LUMO)."""
    w = W.tiny()
    P, O = w.D[0], w.D[1]
    assert abs(np.trace(P) - w.nocc) < 1e-12 and abs(np.trace(O) - w.nocc) < 1e-12
    assert np.allclose(O @ O, O, atol=1e-12)
    assert np.linalg.matrix_rank(P - O, tol=1e-8) == 2


def test_thc_grid_recipe():
    """21 points per distinct center with the defaults: the center, +-x, +-y,
    +-z at 0.6 and 1.4 bohr and the eight cube corners at 1 bohr."""
    w = W.small_random(8, 1, 3)
    cen = np.unique(w.basis.center, axis=0)
    pts = W.thc_grid(w.basis)
    assert pts.shape == (21 * len(cen), 3)
    for i, c in enumerate(cen):
        d = np.sort(np.linalg.norm(pts[21 * i:21 * (i + 1)] - c, axis=1))
        assert np.allclose(d, [0.0] + [0.6] * 6 + [1.0] * 8 + [1.4] * 6)
    assert W.thc_grid(w.basis, radii=(0.6, 1.4), corner=0.0).shape == (13 * len(cen), 3)


def test_serving_stream():
    """256 requests over a pool of 32 molecules, N even in [50, 600], m in
    [4, 32]; the same stream every time."""
    mols, reqs = W.serving_requests()
    assert len(mols) == 32 and len(reqs) == 256
    ns = [w.basis.n for w in mols]
    assert all(50 <= n <= 600 and n % 2 == 0 for n in ns)
    assert all(0 <= i < 32 and 4 <= m <= 32 for i, m, _ in reqs)
    _, again = W.serving_requests()
    assert reqs == again
    D = W.request_densities(mols[reqs[0][0]], reqs[0][1], reqs[0][2])
    assert D.shape == (reqs[0][1], ns[reqs[0][0]], ns[reqs[0][0]])
