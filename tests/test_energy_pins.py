"""Pins of the ESMF energy / gradient / GVP oracle (oracle/esmf_energy.py)
against facts that do not come from the oracle itself: the HF special case of
Eq. (esmf_eng_hf), the Slater-Condon CIS energy in the MO basis, finite
differences of the energy, of its gradient (the Hessian-vector tangent) and
of the GVP objective of Eq. (esmf_gvb) through exact matrix exponentials, the
scale invariance of E in (c0, sigma) and the GVP objective's limits.  CPU only."""
import numpy as np
import pytest

from oracle import esmf_energy as EE
from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W


@pytest.fixture(scope="module")
def case():
    w = W.small_random(10, 1, 7)
    o = Oracle(w.basis)
    eri = o.eri_tensor()
    jk = lambda D: o.jk_brute(eri, D, 0.0)
    return w, eri, jk


def state(w, seed, nocc=3, sigma_norm=0.3):
    return W.esmf_state(W.rng_for(seed), w.basis, nocc, sigma_norm)


def test_hf_special_case(case):
    """sigma = 0, c0 = 1: E is the HF energy 2 Tr[P G] + F[P] . P (Eq.
    esmf_eng_hf), equal to the MO-basis E0 = 2 sum_i h_ii + sum_ij [2(ii|jj)
    - (ij|ji)], and dE/dc0 vanishes (E is stationary in c0 there)."""
    w, eri, jk = case
    st = state(w, 1)
    sig = np.zeros_like(st.sigma)
    E, dc0, dsig, dV = EE.energy_gradient(jk, st.G, st.V, sig, 1.0, st.nocc)
    Th = st.V[:st.nocc]
    P = Th.T @ Th
    FP = EE.fock(jk, P[None])[0]
    assert E == pytest.approx(2.0 * np.trace(P @ st.G) + np.sum(FP * P), rel=1e-13)
    assert E == pytest.approx(EE.cis_energy_mo(eri, st.G, st.V, sig, 1.0, st.nocc), rel=1e-12)
    assert abs(dc0) < 1e-12 * abs(E)
    # Brillouin-type coupling: dE/dsigma = 4 (Theta Fk Gamma^T) at sigma = 0
    Fk = st.G + FP
    np.testing.assert_allclose(dsig, 4.0 * Th @ Fk @ st.V[st.nocc:].T, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("seed,nocc", [(2, 3), (3, 4), (4, 1)])
def test_ao_energy_matches_slater_condon(case, seed, nocc):
    w, eri, jk = case
    st = state(w, seed, nocc, sigma_norm=0.5)
    E = EE.energy(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    Emo = EE.cis_energy_mo(eri, st.G, st.V, st.sigma, st.c0, st.nocc)
    assert E == pytest.approx(Emo, rel=1e-12, abs=1e-12)


def test_gradient_matches_finite_differences(case):
    w, eri, jk = case
    st = state(w, 5, 3, sigma_norm=0.4)
    E, dc0, dsig, dV = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    assert E == pytest.approx(EE.energy(jk, st.G, st.V, st.sigma, st.c0, st.nocc), rel=1e-14)
    h = 1e-5
    f = lambda c0=st.c0, s=st.sigma, V=st.V: EE.energy(jk, st.G, V, s, c0, st.nocc)
    assert dc0 == pytest.approx((f(c0=st.c0 + h) - f(c0=st.c0 - h)) / (2 * h), rel=1e-7, abs=1e-9)
    for i in range(st.sigma.shape[0]):
        for a in range(0, st.sigma.shape[1], 2):
            sp, sm = st.sigma.copy(), st.sigma.copy()
            sp[i, a] += h
            sm[i, a] -= h
            assert dsig[i, a] == pytest.approx((f(s=sp) - f(s=sm)) / (2 * h), rel=1e-6, abs=1e-8)
    for r in range(w.basis.n):                  # rows 0..2 Theta, 3..9 Gamma
        for p in range(0, w.basis.n, 3):
            Vp, Vm = st.V.copy(), st.V.copy()
            Vp[r, p] += h
            Vm[r, p] -= h
            assert dV[r, p] == pytest.approx((f(V=Vp) - f(V=Vm)) / (2 * h), rel=1e-6, abs=1e-8)


def test_scale_invariance(case):
    """E is a ratio of quadratic forms in (c0, sigma): E(l c0, l sigma) = E
    and c0 dE/dc0 + sigma . dE/dsigma = 0 (Euler)."""
    w, eri, jk = case
    st = state(w, 6, 3, sigma_norm=0.7)
    E, dc0, dsig, _ = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    E2 = EE.energy(jk, st.G, st.V, 2.5 * st.sigma, 2.5 * st.c0, st.nocc)
    assert E2 == pytest.approx(E, rel=1e-13)
    assert abs(st.c0 * dc0 + np.sum(st.sigma * dsig)) < 1e-12 * max(1.0, abs(E))


def test_printed_last_e2_term_fails_the_mo_pin(case, monkeypatch):
    """Planted in the oracle: the last term of Eq. (esmf_energy_2b) exactly as
    printed, 2 F[T] . (Theta^T Theta).  The Slater-Condon pin rejects it, which
    is what the reading 2 F[T] . T rests on."""
    w, eri, jk = case
    st = state(w, 2, 3, sigma_norm=0.5)
    orig = EE.energy_terms

    def printed(G, Th, Ga, sigma, c0, N2, FP, FT, P, T, A):
        E1, E2 = orig(G, Th, Ga, sigma, c0, N2, FP, FT, P, T, A)
        return E1, E2 - 2.0 * EE.dot(FT, T) + 2.0 * EE.dot(FT, P)

    monkeypatch.setattr(EE, "energy_terms", printed)
    E = EE.energy(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    Emo = EE.cis_energy_mo(eri, st.G, st.V, st.sigma, st.c0, st.nocc)
    assert abs(E - Emo) > 1e-3 * abs(Emo)


def test_printed_theta_derivative_disagrees_with_finite_differences(case):
    """Eq. (eng_der_ukp) as printed (F - F^T combinations, 4 c0 sigma Gamma F[T],
    4 sigma Gamma F[T] / N2) is not the derivative of E; the oracle's
    term-by-term form is (previous test)."""
    w, eri, jk = case
    st = state(w, 5, 3, sigma_norm=0.4)
    Th, Ga, N2, P, T, A = EE.pieces(st.G, st.V, st.sigma, st.c0, st.nocc)
    FP, FT, FA = EE.fock(jk, np.stack([P, T, A]))
    s, c0, G = st.sigma, st.c0, st.G
    printed = (4 * N2 * Th @ G + 4 * c0 * s @ Ga @ G - 4 * s @ s.T @ Th @ G + 4 * N2 * Th @ FP
               + 4 * c0 * s @ Ga @ FT + 4 * c0 * Th @ (FT - FT.T) + 2 * Th @ (FA - FA.T)
               - 4 * s @ s.T @ Th @ FP + 4 * s @ Ga @ FT / N2) / N2
    _, _, _, dV = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    assert np.max(np.abs(printed - dV[:st.nocc])) > 1e-2 * np.max(np.abs(dV[:st.nocc]))


def richardson(f, h):
    """Central difference at h and h/2, extrapolated (error O(h^4))."""
    c = lambda t: (np.asarray(f(t)) - np.asarray(f(-t))) / (2 * t)
    return (4.0 * c(h / 2) - c(h)) / 3.0


def test_gradient_tangent_matches_finite_differences(case):
    """energy_gradient_tangent (the product rule through every term of the
    gradient) equals the directional derivative of energy_gradient."""
    w, eri, jk = case
    st = state(w, 8, 3, sigma_norm=0.4)
    rng = np.random.default_rng(1)
    dV = rng.standard_normal(st.V.shape)
    ds = rng.standard_normal(st.sigma.shape)
    dc = 0.7
    prim, tan = EE.energy_gradient_tangent(jk, st.G, st.V, st.sigma, st.c0, st.nocc, dV, ds, dc)
    ref = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    assert prim[0] == pytest.approx(ref[0], rel=1e-14)
    g = lambda i: (lambda t: EE.energy_gradient(jk, st.G, st.V + t * dV, st.sigma + t * ds,
                                                 st.c0 + t * dc, st.nocc)[i])
    for i in range(4):
        fd = richardson(g(i), 1e-4)
        scale = max(1.0, float(np.max(np.abs(fd))))
        assert np.max(np.abs(np.asarray(tan[i]) - fd)) < 1e-8 * scale, i


def test_rotation_gradient_at_zero(case):
    """The exact exp-map rotation gradient at X = 0 is Gam - Gam^T."""
    w, eri, jk = case
    st = state(w, 9, 3)
    _, _, _, gV = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    a = EE.rotation_gradient(st.V, gV)
    b = EE.rotation_gradient_at(jk, st.G, st.V, st.sigma, st.c0, st.nocc, np.zeros_like(st.V))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def gvp_objective(jk, st, om, mu, chi, c0=None, s=None, X=None):
    """L_mu,chi of Eq. (esmf_gvb) at (c0, sigma, X), |grad E|^2 with the exact
    rotation gradient of V(X) = exp(X) V."""
    from scipy.linalg import expm
    c0 = st.c0 if c0 is None else c0
    s = st.sigma if s is None else s
    X = np.zeros_like(st.V) if X is None else X
    V = expm(X) @ st.V
    E, gc, gs, _ = EE.energy_gradient(jk, st.G, V, s, c0, st.nocc)
    Gx = EE.rotation_gradient_at(jk, st.G, st.V, s, c0, st.nocc, X)
    gn = gc * gc + np.sum(gs * gs) + 0.5 * np.sum(Gx * Gx)
    return chi * (mu * (om - E) ** 2 + (1 - mu) * gn) + (1 - chi) * E


@pytest.mark.parametrize("om,mu,chi", [(-2.5, 0.4, 0.8), (0.0, 0.0, 1.0)])
def test_gvp_gradient_matches_finite_differences(case, om, mu, chi):
    """dL/dc0, dL/dsigma and dL/dX of Eq. (esmf_l_gvp_der) (with the Hessian-
    vector product) against finite differences of L itself."""
    pytest.importorskip("scipy")
    w, eri, jk = case
    st = state(w, 5, 3, sigma_norm=0.4)
    L, E, gn2, dLc, dLs, dLX = EE.gvp_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc, om, mu, chi)
    assert L == pytest.approx(gvp_objective(jk, st, om, mu, chi), rel=1e-12)
    h = 1e-4
    assert dLc == pytest.approx(richardson(lambda t: gvp_objective(jk, st, om, mu, chi, c0=st.c0 + t), h),
                                rel=1e-6)
    for (i, a) in [(0, 0), (1, 2), (2, 5)]:
        d = np.zeros_like(st.sigma)
        d[i, a] = 1.0
        fd = richardson(lambda t: gvp_objective(jk, st, om, mu, chi, s=st.sigma + t * d), h)
        assert dLs[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    for (p, q) in [(5, 1), (8, 4), (2, 0), (9, 7)]:
        Z = np.zeros_like(st.V)
        Z[p, q], Z[q, p] = 1.0, -1.0
        fd = richardson(lambda t: gvp_objective(jk, st, om, mu, chi, X=t * Z), h)
        assert dLX[p, q] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    np.testing.assert_allclose(dLX, -dLX.T, atol=1e-12)


def test_gvp_limits(case):
    """chi = 0: L = E and dL = grad E.  chi = 1, mu = 1: dL = -2 (omega - E) grad E."""
    w, eri, jk = case
    st = state(w, 4, 3)
    E, gc, gs, gV = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    Gx = EE.rotation_gradient(st.V, gV)
    L, E0, _, dLc, dLs, dLX = EE.gvp_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc, 1.0, 0.3, 0.0)
    assert L == pytest.approx(E, rel=1e-14) and dLc == pytest.approx(gc, rel=1e-13)
    np.testing.assert_allclose(dLs, gs, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(dLX, Gx, rtol=1e-13, atol=1e-14)
    L, _, _, dLc, dLs, dLX = EE.gvp_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc, 1.0, 1.0, 1.0)
    f = -2.0 * (1.0 - E)
    assert L == pytest.approx((1.0 - E) ** 2, rel=1e-13) and dLc == pytest.approx(f * gc, rel=1e-12)
    np.testing.assert_allclose(dLX, f * Gx, rtol=1e-12, atol=1e-13)
