"""Pins of the oracle's p- and d-function integrals (Obara-Saika
recurrences), against facts outside the recurrences: the Boys functions'
integral definition; radial quadrature of the contracted p and d
normalisations; p and d primitives as centre derivatives of s primitives,
(x - A_x) exp(-a r_A^2) = (1/2a) d/dA_x exp(-a r_A^2),
(x - A_x)^2 exp(-a r_A^2) = (1/4a^2) (d^2/dA_x^2 + 2a) exp(-a r_A^2) and
(x - A_x)(y - A_y) exp(-a r_A^2) = (1/4a^2) d^2/dA_x dA_y exp(-a r_A^2),
checked by finite differences of the s-type closed form; invariance under a
rotation of the molecule with the p components turned as vectors and the d
components as symmetric tensors; the 8-fold permutational symmetry;
positivity of the Coulomb pair matrix; brute == unique J/K.  CPU only."""
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


def test_boys_orders_against_incomplete_gamma():
    """F_m(T) = gamma(m + 1/2, T) / (2 T^(m + 1/2)) (substitute t = T u^2 in the
    integral definition), with the lower incomplete gamma function from scipy;
    orders 0..8, the range (dd|dd) needs."""
    from scipy.special import gamma, gammainc
    for m in range(9):
        a = m + 0.5
        assert abs(boys(m, 0.0) - 1.0 / (2 * m + 1)) <= 1e-15
        for T in (1e-9, 1e-4, 0.3, 1.0, 2.0, 9.0, 27.0, 80.0, 300.0):
            ref = gammainc(a, T) * gamma(a) / (2.0 * T ** a)
            assert abs(boys(m, T) - ref) <= 5e-14 * ref, (m, T, boys(m, T), ref)


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


# exponent triples of the Cartesian labels 0..9 (s; p_x, p_y, p_z; d_xx, d_yy,
# d_zz, d_xy, d_xz, d_yz)
LABELS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2),
          (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def raw_norm(a, c):
    """Norm of the raw primitive x^lx y^ly z^lz exp(-a r^2) from the Gaussian
    moments int x^{2n} exp(-2a x^2) dx = (2n-1)!!/(4a)^n sqrt(pi/2a)."""
    v = LABELS[c]
    mom = np.prod([(1.0 if k < 2 else 3.0) / (4 * a) ** k for k in v]) * (np.pi / (2 * a)) ** 1.5
    return 1.0 / math.sqrt(mom)


def raw_l(centers, exps, carts):
    """[ab|cd] over raw primitives with Cartesian labels, from the recurrences."""
    o = Oracle(p_basis(centers, exps, carts))
    nrm = [raw_norm(a, c) for a, c in zip(exps, carts)]
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


def test_contracted_d_normalisation_by_radial_quadrature():
    w = W.spd_random(1, 1, 2)
    o = Oracle(w.basis)
    off = np.concatenate([[0], np.cumsum(w.basis.nprim)])
    for mu in range(w.basis.n):
        lab = int(w.basis.cart[mu])
        if lab < 4:
            continue
        a = w.basis.exps[off[mu]:off[mu + 1]]
        c = o.w[off[mu]:off[mu + 1]]
        # sphere averages: <x^4> = r^4 / 5, <x^2 y^2> = r^4 / 15
        ang = 1.0 / 5.0 if lab <= 6 else 1.0 / 15.0
        f = lambda r: 4 * np.pi * r ** 6 * ang * np.sum(c * np.exp(-a * r * r)) ** 2
        val, _ = integrate.quad(f, 0, np.inf, epsabs=1e-14, epsrel=1e-12)
        assert abs(val - 1.0) < 1e-10, (mu, lab, val)


def fd2(f, x0, h):
    """d^2 f / dx^2 at x0 by Richardson-extrapolated central differences."""
    d = lambda hh: (f(x0 + hh) - 2 * f(x0) + f(x0 - hh)) / (hh * hh)
    return (4 * d(h / 2) - d(h)) / 3


def fd11(g, x0, y0, h):
    """d^2 g / dx dy at (x0, y0) by Richardson-extrapolated central differences."""
    d = lambda hh: (g(x0 + hh, y0 + hh) - g(x0 + hh, y0 - hh) - g(x0 - hh, y0 + hh)
                    + g(x0 - hh, y0 - hh)) / (4 * hh * hh)
    return (4 * d(h / 2) - d(h)) / 3


@pytest.mark.parametrize("seed", [0, 1])
def test_d_primitives_are_second_centre_derivatives_of_s(seed):
    rng = np.random.default_rng(60 + seed)
    cen = rng.uniform(-1.2, 1.2, size=(4, 3))
    ex = np.exp(rng.uniform(np.log(0.2), np.log(4), size=4))
    s0 = abs(raw_s(cen, ex))
    for pos in range(4):
        a = ex[pos]
        for lab in range(4, 10):
            carts = [0, 0, 0, 0]
            carts[pos] = lab
            v = LABELS[lab]
            dims = [i for i in range(3) for _ in range(v[i])]
            if dims[0] == dims[1]:
                i = dims[0]

                def f(x):
                    c = cen.copy()
                    c[pos, i] = x
                    return raw_s(c, ex)
                ref = (fd2(f, cen[pos, i], 4e-3) + 2 * a * raw_s(cen, ex)) / (4 * a * a)
            else:
                i, j = dims

                def g(x, y):
                    c = cen.copy()
                    c[pos, i] = x
                    c[pos, j] = y
                    return raw_s(c, ex)
                ref = fd11(g, cen[pos, i], cen[pos, j], 4e-3) / (4 * a * a)
            val = raw_l(cen, ex, carts)
            assert abs(val - ref) <= 1e-7 * max(abs(ref), s0), (pos, lab, val, ref)
    # a d and a p function on different centres: the third derivative is
    # checked as the first derivative (in the p centre) of the d integral
    for (pd, pp) in ((0, 2), (1, 3)):
        for lab, i in ((4, 0), (7, 2)):
            carts = [0, 0, 0, 0]
            carts[pd] = lab

            def fp(x):
                c = cen.copy()
                c[pp, i] = x
                return raw_l(c, ex, carts)
            ref = fd(fp, cen[pp, i], 1e-3) / (2 * ex[pp])
            carts2 = list(carts)
            carts2[pp] = i + 1
            val = raw_l(cen, ex, carts2)
            assert abs(val - ref) <= 1e-8 * max(abs(ref), s0), (pd, pp, lab, i, val, ref)


@pytest.fixture(scope="module")
def spd_small():
    w = W.spd_random(2, 2, 3, edge=2.6, min_dist=1.2, nprim=2)   # 20 functions: s, p, d per centre
    o = Oracle(w.basis)
    return w, o, o.eri_tensor()


def d_rotation(R):
    """Map of the six normalised Cartesian d functions of one shell under a
    rotation R: with T_kl = x_k x_l g(r), d_kk = T_kk and d_kl = sqrt(3) T_kl
    (k < l) for a shell normalised component by component, and
    T'_ij = sum_kl R_ik R_jl T_kl."""
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    scale = [1.0, 1.0, 1.0, math.sqrt(3.0), math.sqrt(3.0), math.sqrt(3.0)]
    U = np.zeros((6, 6))
    for a, (i, j) in enumerate(pairs):
        for b, (k, l) in enumerate(pairs):
            coef = R[i, k] * R[j, l] + (R[i, l] * R[j, k] if k != l else 0.0)
            U[a, b] = scale[a] / scale[b] * coef
    return U


def test_rotation_invariance_with_d_functions(spd_small):
    w, o, E = spd_small
    b = w.basis
    R = Rotation.from_rotvec([-0.9, 0.4, 1.3]).as_matrix()
    rb = W.Basis(b.center @ R.T, b.nprim, b.exps, b.coefs, b.cart)
    Er = Oracle(rb).eri_tensor()
    n = b.n
    U = np.zeros((n, n))
    for c0 in range(0, n, 10):                       # s, p_x..p_z, d_xx..d_yz per centre
        U[c0, c0] = 1.0
        U[c0 + 1:c0 + 4, c0 + 1:c0 + 4] = R
        U[c0 + 4:c0 + 10, c0 + 4:c0 + 10] = d_rotation(R)
    Et = np.einsum("ai,bj,ck,dl,ijkl->abcd", U, U, U, U, E, optimize=True)
    np.testing.assert_allclose(Er, Et, rtol=0, atol=1e-12 * np.abs(E).max())


def test_spd_symmetry_positivity_and_brute_equals_unique(spd_small):
    w, o, E = spd_small
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)):
        np.testing.assert_allclose(E, E.transpose(perm), rtol=0, atol=1e-14 * np.abs(E).max())
    n = w.basis.n
    ev = np.linalg.eigvalsh(E.reshape(n * n, n * n))
    assert ev.min() >= -1e-12 * ev.max()
    assert np.allclose(o.Q * o.Q, np.einsum("pqpq->pq", E), rtol=1e-13, atol=1e-15)
    rng = np.random.default_rng(5)
    D = w.D + 0.2 * rng.standard_normal(w.D.shape)
    Jb, Kb = o.jk_brute(E, D, 0.0)
    Ju, Ku, _ = o.jk_unique(D, 0.0)
    np.testing.assert_allclose(Ju, Jb, rtol=0, atol=1e-13 * np.abs(Jb).max())
    np.testing.assert_allclose(Ku, Kb, rtol=0, atol=1e-13 * np.abs(Kb).max())
