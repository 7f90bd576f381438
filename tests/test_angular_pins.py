"""Pins of the oracle's p-function integrals (Obara-Saika recurrences),
against facts outside the recurrences: the Boys functions' integral
definition; radial quadrature of the contracted p normalisation; p
primitives as centre derivatives of s primitives, (x - A_x) exp(-a r_A^2) =
(1/2a) d/dA_x exp(-a r_A^2), checked by finite differences of the s-type
closed form; invariance under a rotation of the molecule with the p
components turned as vectors; the 8-fold permutational symmetry; positivity
of the Coulomb pair matrix; brute == unique J/K.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

from oracle.oracle import Oracle, boys, boys0
from paper_2002_00322_gb300 import workloads as W


def test_boys_orders_against_quadrature():
    for m in range(5):
        for T in (0.0, 1e-9, 1e-4, 0.3, 2.0, 9.0, 27.0, 80.0):
            ref, _ = integrate.quad(lambda u: u ** (2 * m) * math.exp(-T * u * u), 0, 1,
                                    epsabs=1e-16, epsrel=1e-14)
            assert abs(boys(m, T) - ref) <= 2e-14 * max(ref, 1e-300), (m, T)
        assert abs(boys(0, 0.7) - boys0(0.7)) <= 1e-15


def p_basis(centers, exps, carts, coefs=None):
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    n = centers.shape[0]
    npr = np.ones(n, dtype=np.int32) if coefs is None else np.full(n, len(exps[0]), dtype=np.int32)
    ex = np.asarray(exps, dtype=np.float64).ravel()
    co = np.ones(ex.size) if coefs is None else np.asarray(coefs, dtype=np.float64).ravel()
    return W.Basis(centers, npr, ex, co, np.asarray(carts, dtype=np.int32))


def test_contracted_p_normalisation_by_radial_quadrature():
    w = W.sp_random(3, 1, 1)
    o = Oracle(w.basis)
    off = np.concatenate([[0], np.cumsum(w.basis.nprim)])
    for mu in range(w.basis.n):
        a = w.basis.exps[off[mu]:off[mu + 1]]
        c = o.w[off[mu]:off[mu + 1]]
        ang = 1.0 / 3.0 if w.basis.cart[mu] else 1.0           # <x^2> over the sphere is r^2 / 3
        f = lambda r: 4 * np.pi * r * r * (r * r if w.basis.cart[mu] else 1.0) * ang * \
            np.sum(c * np.exp(-a * r * r)) ** 2
        val, _ = integrate.quad(f, 0, np.inf, epsabs=1e-14, epsrel=1e-12)
        assert abs(val - 1.0) < 1e-10, mu


def raw_s(centers, exps):
    """[ab|cd] over raw s primitives, from the oracle's s-type closed form."""
    o = Oracle(W.Basis(np.asarray(centers, float), np.ones(4, dtype=np.int32), np.asarray(exps, float),
                       np.ones(4)))
    return o.eri(0, 1, 2, 3) / np.prod((2 * np.asarray(exps) / np.pi) ** 0.75)


def raw_l(centers, exps, carts):
    """[ab|cd] over raw primitives with Cartesian labels, from the recurrences."""
    o = Oracle(p_basis(centers, exps, carts))
    nrm = [(2 * a / np.pi) ** 0.75 * (2 * math.sqrt(a) if c else 1.0) for a, c in zip(exps, carts)]
    return o.eri(0, 1, 2, 3) / np.prod(nrm)


def fd(f, x0, h):
    """d f / dx at x0 by Richardson-extrapolated central differences."""
    d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
    d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p_primitives_are_centre_derivatives_of_s(seed):
    rng = np.random.default_rng(40 + seed)
    cen = rng.uniform(-1.2, 1.2, size=(4, 3))
    ex = np.exp(rng.uniform(np.log(0.2), np.log(5), size=4))
    for pos in range(4):                                   # one p function at position pos
        for i in range(3):
            carts = [0, 0, 0, 0]
            carts[pos] = i + 1

            def f(x):
                c = cen.copy()
                c[pos, i] = x
                return raw_s(c, ex)
            ref = fd(f, cen[pos, i], 1e-3) / (2 * ex[pos])
            val = raw_l(cen, ex, carts)
            assert abs(val - ref) <= 1e-8 * max(abs(ref), 1e-3 * abs(raw_s(cen, ex))), (pos, i, val, ref)
    # two p functions: a mixed second derivative (positions 0 and 2, and a
    # same-centre pair 0/1 with B moved onto A)
    for (pa, pb, same) in ((0, 2, False), (0, 1, True)):
        c0 = cen.copy()
        if same:
            c0[pb] = c0[pa]
        for i, j in ((0, 0), (1, 2)):
            carts = [0, 0, 0, 0]
            carts[pa], carts[pb] = i + 1, j + 1

            def g(x, y):
                c = c0.copy()
                c[pa, i] = x
                c[pb, j] = y
                return raw_s(c, ex)
            h = 2e-3
            x0, y0 = c0[pa, i], c0[pb, j]
            dxy = lambda hh: (g(x0 + hh, y0 + hh) - g(x0 + hh, y0 - hh) - g(x0 - hh, y0 + hh)
                              + g(x0 - hh, y0 - hh)) / (4 * hh * hh)
            ref = (4 * dxy(h / 2) - dxy(h)) / 3 / (4 * ex[pa] * ex[pb])
            val = raw_l(c0, ex, carts)
            scale = max(abs(ref), abs(raw_s(c0, ex)))
            assert abs(val - ref) <= 1e-6 * scale, (pa, pb, i, j, val, ref)


@pytest.fixture(scope="module")
def sp_small():
    w = W.sp_random(3, 2, 7, edge=3.0, min_dist=0.8)         # 12 functions: 3 s + 3 p shells
    o = Oracle(w.basis)
    return w, o, o.eri_tensor()


def test_rotation_invariance(sp_small):
    """Rotating the molecule and turning every p shell's components with the
    same rotation leaves the integrals a tensor: E'(abcd) = U_ai U_bj U_ck U_dl E(ijkl)."""
    w, o, E = sp_small
    b = w.basis
    R = Rotation.from_rotvec([0.3, -1.1, 0.7]).as_matrix()
    rb = W.Basis(b.center @ R.T, b.nprim, b.exps, b.coefs, b.cart)
    Er = Oracle(rb).eri_tensor()
    n = b.n
    U = np.zeros((n, n))
    for mu in range(n):
        if b.cart[mu] == 0:
            U[mu, mu] = 1.0
    for s in range(0, n, 4):                                   # s, px, py, pz per centre
        U[s + 1:s + 4, s + 1:s + 4] = R
    Et = np.einsum("ai,bj,ck,dl,ijkl->abcd", U, U, U, U, E, optimize=True)
    np.testing.assert_allclose(Er, Et, rtol=0, atol=1e-12 * np.abs(E).max())


def test_eightfold_symmetry_and_positivity(sp_small):
    w, o, E = sp_small
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)):
        np.testing.assert_allclose(E, E.transpose(perm), rtol=0, atol=1e-14 * np.abs(E).max())
    n = w.basis.n
    ev = np.linalg.eigvalsh(E.reshape(n * n, n * n))
    assert ev.min() >= -1e-12 * ev.max()
    Q = o.Q
    assert np.allclose(Q * Q, np.einsum("pqpq->pq", E), rtol=1e-13, atol=1e-15)


def test_brute_equals_unique_with_p_functions(sp_small):
    w, o, E = sp_small
    rng = np.random.default_rng(4)
    D = w.D + 0.2 * rng.standard_normal(w.D.shape)
    Jb, Kb = o.jk_brute(E, D, 0.0)
    Ju, Ku, _ = o.jk_unique(D, 0.0)
    np.testing.assert_allclose(Ju, Jb, rtol=0, atol=1e-13 * np.abs(Jb).max())
    np.testing.assert_allclose(Ku, Kb, rtol=0, atol=1e-13 * np.abs(Kb).max())
    # screening with Q from the p-aware Schwarz table: the kept count is the
    # number of unique quartets whose Schwarz product reaches tol
    n = w.basis.n
    Q = o.Q
    tol = float(np.median(Q) ** 2)
    Js, Ks, nk = o.jk_unique(D, tol)
    pairs = [(p, q) for p in range(n) for q in range(p + 1)]
    expect = sum(1 for i in range(len(pairs)) for j in range(i + 1)
                 if Q[pairs[i]] * Q[pairs[j]] >= tol)
    assert nk == expect < len(pairs) * (len(pairs) + 1) // 2
