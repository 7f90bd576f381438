"""Pins of the oracle's tensor-hypercontraction route (the other acceleration
the paper names as future work, Sec. I; LS-THC of Parrish et al. 2012):
the collocation against Gaussian overlap closed forms, the Coulomb matrix
E formed from rank-one density builds against the brute N^4 sum, the
least-squares Z against a generic least-squares solver, exactness when the
grid spans every orbital product, monotone fits over nested grids, and the
symmetries and positivity the fitted tensor keeps.  CPU only."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W


def gauss_legendre(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def kept_tensor(o, tol):
    V = o.eri_tensor()
    if tol > 0:
        V = V * (np.multiply.outer(o.Q, o.Q) >= tol)
    return V


def pair_products(X):
    n, G = X.shape
    return np.einsum("pP,qP->pqP", X, X).reshape(n * n, G)


def test_collocation_overlaps_by_quadrature():
    """int phi_p phi_q dV by a cylindrical quadrature over collocated values
    (both centers on the z axis) equals the Gaussian overlap closed form
    sum_kl w_k w_l (pi/(a+b))^{3/2} exp(-ab/(a+b) R^2); the diagonal is 1."""
    rng = np.random.default_rng(11)
    for R in (0.0, 0.9, 2.3):
        b = W.Basis(np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]]), np.array([3, 2], dtype=np.int32),
                    np.exp(rng.uniform(np.log(0.1), np.log(10.0), 5)), rng.uniform(0.1, 1.0, 5))
        o = Oracle(b)
        rho, wr = gauss_legendre(0.0, 14.0, 400)
        z, wz = gauss_legendre(-14.0, 14.0 + R, 800)
        rr, zz = np.meshgrid(rho, z, indexing="ij")
        pts = np.stack([rr.ravel(), np.zeros(rr.size), zz.ravel()], axis=1)
        X = o.collocation(pts)
        wt = (2.0 * math.pi * rr * np.outer(wr, wz)).ravel()
        S = (X * wt) @ X.T
        off = [0, 3, 5]
        ref = np.zeros((2, 2))
        for p in range(2):
            for q in range(2):
                d2 = float(np.sum((b.center[p] - b.center[q]) ** 2))
                for k in range(off[p], off[p + 1]):
                    for l in range(off[q], off[q + 1]):
                        a, c = b.exps[k], b.exps[l]
                        ref[p, q] += o.w[k] * o.w[l] * (math.pi / (a + c)) ** 1.5 * math.exp(-a * c / (a + c) * d2)
        assert np.allclose(np.diag(S), 1.0, atol=1e-9)
        assert np.allclose(S, ref, atol=1e-9)


def test_coulomb_matrix_from_rank_one_builds_equals_brute_sum():
    """thc_fit forms E_PQ = x_P^T J[x_Q x_Q^T] x_P through the grouped build;
    the brute sum X2^T V X2 over the Schwarz-kept integrals gives the same Z."""
    for tol in (0.0, 1e-4):
        w = W.small_random(8, 1, 5, tol=tol)
        o = Oracle(w.basis)
        pts = W.thc_grid(w.basis, radii=(0.8,), corner=0.0)
        X, Z = o.thc_fit(pts, tol, 1e-6)
        X2 = pair_products(X)
        V = kept_tensor(o, tol).reshape(64, 64)
        E = X2.T @ V @ X2
        S = (X.T @ X) ** 2
        Sr = S + 1e-6 * S.diagonal().max() * np.eye(S.shape[0])
        Zb = np.linalg.inv(Sr) @ E @ np.linalg.inv(Sr)
        assert np.abs(Z - Zb).max() <= 1e-8 * np.abs(Zb).max()
        if tol > 0:
            assert (np.multiply.outer(o.Q, o.Q) < tol).any()     # the screened case drops quartets


def test_least_squares_against_a_generic_solver():
    """With ridge 0, X2 Z X2^T is the least-squares fit of the integral
    tensor in the span of the pair products: a generic least-squares solve
    of vec(V) ~ (X2 kron X2) vec(Z) gives the same fitted tensor."""
    w = W.small_random(4, 1, 7, tol=0.0)
    o = Oracle(w.basis)
    rng = np.random.default_rng(2)
    pts = w.basis.center[rng.integers(0, 4, 6)] + rng.normal(0.0, 0.6, (6, 3))
    X, Z = o.thc_fit(pts, 0.0, 0.0)
    X2 = pair_products(X)
    V = o.eri_tensor().reshape(16, 16)
    Zls = np.linalg.lstsq(np.kron(X2, X2), V.ravel(), rcond=None)[0].reshape(6, 6)
    fit, fit_ls = X2 @ Z @ X2.T, X2 @ Zls @ X2.T
    assert np.abs(fit - fit_ls).max() <= 1e-9 * np.abs(V).max()
    assert np.abs(fit - V).max() > 1e-4 * np.abs(V).max()      # a real approximation


def test_grid_spanning_every_pair_product_is_exact():
    """N(N+1)/2 generic grid points make the pair products a basis of the
    symmetric pair space, so the fit reproduces the integrals and the build
    (up to the conditioning of S)."""
    w = W.small_random(6, 3, 3, tol=0.0)
    o = Oracle(w.basis)
    rng = np.random.default_rng(1)
    pts = w.basis.center[rng.integers(0, 6, 21)] + rng.normal(0.0, 0.7, (21, 3))
    X, Z = o.thc_fit(pts, 0.0, 0.0)
    V = o.eri_tensor()
    assert np.abs(o.thc_tensor(X, Z) - V).max() <= 1e-6 * np.abs(V).max()
    J, K = o.jk_thc(w.D, pts, 0.0, 0.0)
    Je, Ke = o.jk_brute(V, w.D, 0.0)
    for a, b in ((J, Je), (K, Ke)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_nested_grids_never_worsen_the_fit():
    """The ridge-0 fit is an orthogonal projection onto the span of the pair
    products; nested grids give nested spans, so the error cannot grow."""
    w = W.small_random(6, 1, 4, tol=0.0)
    o = Oracle(w.basis)
    rng = np.random.default_rng(8)
    pts = w.basis.center[rng.integers(0, 6, 18)] + rng.normal(0.0, 0.7, (18, 3))
    V = o.eri_tensor()
    errs = []
    for G in (4, 8, 12, 18):
        X, Z = o.thc_fit(pts[:G], 0.0, 0.0)
        errs.append(np.linalg.norm(o.thc_tensor(X, Z) - V))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.5 * errs[0]


def test_fitted_tensor_symmetries_and_positivity():
    """Z = (S + lam I)^-1 E (S + lam I)^-1 is symmetric positive semi-definite
    (in exact arithmetic; rounding leaves tiny negative eigenvalues in the
    directions S barely spans, which the pair products do not reach), so the
    fitted pair matrix is positive semi-definite, the fitted tensor keeps the
    8-fold symmetry, J is symmetric and depends
    on (D + D^T)/2, K[D^T] = K[D]^T, and D.J[D] >= 0 for any D, D.K[D] >= 0
    for a positive semi-definite D."""
    w = W.small_random(8, 3, 6, tol=0.0)
    o = Oracle(w.basis)
    pts = W.thc_grid(w.basis, radii=(0.7,), corner=1.0)
    X, Z = o.thc_fit(pts, 0.0, 1e-8)
    assert np.array_equal(Z, Z.T)
    V = o.thc_tensor(X, Z)
    ev = np.linalg.eigvalsh(V.reshape(64, 64))        # the fitted pair matrix (pq|rs)
    assert ev.min() >= -1e-10 * ev.max()
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)):
        assert np.abs(V - V.transpose(perm)).max() <= 1e-12 * np.abs(V).max()
    D = w.D
    J, K = o.jk_thc(D, pts, 0.0, 1e-8)
    Jt, Kt = o.jk_thc(np.transpose(D, (0, 2, 1)), pts, 0.0, 1e-8)
    Js, _ = o.jk_thc(0.5 * (D + np.transpose(D, (0, 2, 1))), pts, 0.0, 1e-8)
    scale = np.abs(K).max()
    assert np.abs(J - np.transpose(J, (0, 2, 1))).max() <= 1e-12 * scale
    assert np.abs(Kt - np.transpose(K, (0, 2, 1))).max() <= 1e-12 * scale
    assert np.abs(Js - J).max() <= 1e-12 * scale
    assert all(np.sum(D[k] * J[k]) >= 0 for k in range(3))
    C = np.random.default_rng(4).standard_normal((8, 3))
    P = (C @ C.T)[None]
    _, KP = o.jk_thc(P, pts, 0.0, 1e-8)
    assert np.sum(P[0] * KP[0]) >= 0


def _fit_with(o, points, tol, ridge, slip):
    """thc_fit with one plausible slip planted (the oracle itself is untouched)."""
    X = o.collocation(points)
    G = X.shape[1]
    DQ = np.einsum("pQ,qQ->Qpq", X, X)
    JQ, _, _ = o.jk_unique(DQ, tol)
    E = np.einsum("pP,qP,Qpq->PQ", X, X, JQ)
    if slip == "E_one_side":
        E = np.einsum("pP,qQ,Qpq->PQ", X, X, JQ)
    S = (X.T @ X) ** 2
    if slip == "S_unsquared":
        S = X.T @ X
    lam = ridge * S.diagonal().max()
    if slip == "ridge_absolute":
        lam = ridge
    Sr = S + lam * np.eye(G)
    Z = np.linalg.solve(Sr, np.linalg.solve(Sr, E).T).T
    if slip == "one_solve":
        Z = np.linalg.solve(Sr, E)
    return X, 0.5 * (Z + Z.T)


_THC_TENSOR = Oracle.thc_tensor


def _tensor_with(X, Z, slip):
    if slip == "tensor_pairing":
        return np.einsum("pP,qQ,PQ,rP,sQ->pqrs", X, X, Z, X, X)
    return _THC_TENSOR(X, Z)


@pytest.mark.parametrize("slip", ["S_unsquared", "E_one_side", "one_solve", "ridge_absolute",
                                  "tensor_pairing", "exchange_transposed"])
def test_pins_catch_planted_slips(monkeypatch, slip):
    """Each slip planted in a copy of the THC oracle fails at least one pin."""
    def fit(self, points, tol, ridge):
        return _fit_with(self, points, tol, ridge, slip)

    def tensor(X, Z):
        return _tensor_with(X, Z, slip)

    def jk(self, D, points, tol, ridge):
        D = np.ascontiguousarray(D, dtype=np.float64)
        X, Z = self.thc_fit(points, tol, ridge)
        V = self.thc_tensor(X, Z)
        J = np.einsum("pqrs,krs->kpq", V, D)
        K = np.einsum("pqrs,kqs->kpr", V, D)
        if slip == "exchange_transposed":
            K = np.einsum("pqrs,ksq->kpr", V, D)
        return J, K

    monkeypatch.setattr(Oracle, "thc_fit", fit)
    monkeypatch.setattr(Oracle, "thc_tensor", staticmethod(tensor))
    monkeypatch.setattr(Oracle, "jk_thc", jk)
    pins = [test_coulomb_matrix_from_rank_one_builds_equals_brute_sum, test_least_squares_against_a_generic_solver,
            test_grid_spanning_every_pair_product_is_exact, test_nested_grids_never_worsen_the_fit,
            test_fitted_tensor_symmetries_and_positivity]
    failed = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the slip {slip}"
