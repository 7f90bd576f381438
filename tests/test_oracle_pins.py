"""Pins for the FP64 oracle against facts that do not come from the oracle.

Each test names the closed form, invariant or brute-force relation it uses.
A plausible slip in the oracle (a dropped permutation, a transposed operand,
a wrong prefactor or exponent, the wrong exchange index order) fails at least
one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle.oracle import Oracle, boys0
from paper_2002_00322_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, val, _cite = line.split(None, 2)
        out[name] = float(val)
    return out


def one_prim_basis(centers, exps):
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    n = centers.shape[0]
    return W.Basis(centers, np.ones(n, dtype=np.int32),
                   np.asarray(exps, dtype=np.float64), np.ones(n))


@pytest.fixture(scope="module")
def tiny():
    w = W.tiny()
    o = Oracle(w.basis)
    return w, o, o.eri_tensor()


# ------------------------------------------------------------- integrals
def test_normalisation_radial_quadrature():
    """<phi|phi> = 1 by direct radial quadrature of the contracted function."""
    w = W.tiny()
    o = Oracle(w.basis)
    off = np.concatenate([[0], np.cumsum(w.basis.nprim)])
    for mu in (0, 5, 17):
        a = w.basis.exps[off[mu]:off[mu + 1]]
        c = o.w[off[mu]:off[mu + 1]]
        f = lambda r: 4 * np.pi * r * r * (np.sum(c * np.exp(-a * r * r))) ** 2
        val, _ = integrate.quad(f, 0, np.inf, epsabs=1e-13, epsrel=1e-12)
        assert abs(val - 1.0) < 1e-10


def test_boys_against_its_integral_definition():
    """F0(T) = int_0^1 exp(-T u^2) du, on both sides of the series switch."""
    g = golden()
    assert boys0(0.0) == g["boys0_at_zero"]
    for T in [1e-12, 1e-8, 9.99e-7, 1e-6, 1.01e-6, 1e-3, 0.1, 1.0, 7.5, 30.0, 300.0]:
        ref, _ = integrate.quad(lambda u: math.exp(-T * u * u), 0, 1, epsabs=1e-15, epsrel=1e-14)
        assert abs(boys0(T) - ref) <= 1e-14 * max(1.0, ref), T
    # large-T asymptote (1/2) sqrt(pi/T)
    assert abs(boys0(400.0) - 0.5 * math.sqrt(math.pi / 400.0)) < 1e-15


def test_self_repulsion_closed_form():
    """(ss|ss) of one normalised primitive = 2 sqrt(a/pi) (golden values)."""
    g = golden()
    o = Oracle(one_prim_basis([[0.3, -1.0, 2.0]], [1.0]))
    assert abs(o.eri(0, 0, 0, 0) - g["ss_self_repulsion_a1"]) < 1e-15
    o = Oracle(one_prim_basis([[0.0, 0.0, 0.0]], [0.5]))
    assert abs(o.eri(0, 0, 0, 0) - g["ss_self_repulsion_a0p5"]) < 1e-15


def test_two_center_gaussian_charges():
    """(aa|bb) for normalised primitives at distance R equals the interaction
    of two Gaussian charge clouds: erf(sqrt(2ab/(a+b)) R) / R."""
    rng = np.random.default_rng(7)
    for _ in range(12):
        a, b = np.exp(rng.uniform(np.log(0.1), np.log(10), size=2))
        R = rng.uniform(0.05, 12.0)
        o = Oracle(one_prim_basis([[0, 0, 0], [0, R * 0.6, R * 0.8]], [a, b]))
        ref = special.erf(math.sqrt(2 * a * b / (a + b)) * R) / R
        assert abs(o.eri(0, 0, 1, 1) - ref) <= 1e-13 * ref


def test_contracted_two_center_charge_clouds():
    """Contracted (mu mu|nu nu), mu on A and nu on B (three primitives each):
    the product of two s Gaussians on one center is a Gaussian charge of
    exponent p = a_i + a_j and charge (pi/p)^{3/2}, and two such clouds at
    distance R interact by erf(sqrt(pq/(p+q)) R) / R (2 sqrt(rho/pi) at R = 0),
    so (mu mu|nu nu) = sum_ijkl w_i w_j w_k w_l (pi/p)^{3/2} (pi/q)^{3/2}
    erf(sqrt(rho) R)/R.  The weights w come from a radial quadrature of the
    contraction's norm, not from the oracle.  This pins the contracted sum of
    the primitive quartets: a slip that counted the diagonal primitive pairs
    twice, or dropped the cross pairs, changes the value by far more than the
    tolerance (checked below)."""
    rng = np.random.default_rng(19)

    def weights(a, d):
        g = d * (2 * a / np.pi) ** 0.75
        f = lambda r: 4 * np.pi * r * r * np.sum(g * np.exp(-a * r * r)) ** 2
        nrm, _ = integrate.quad(f, 0, np.inf, epsabs=1e-14, epsrel=1e-13)
        return g / math.sqrt(nrm)

    def cloud_sum(wa, a, wb, b, R, diag=1.0, cross=1.0):
        tot = 0.0
        for i in range(3):
            for j in range(3):
                fij = diag if i == j else cross
                p = a[i] + a[j]
                for k in range(3):
                    for l in range(3):
                        fkl = diag if k == l else cross
                        q = b[k] + b[l]
                        rho = p * q / (p + q)
                        inter = (2 * math.sqrt(rho / math.pi) if R == 0.0
                                 else special.erf(math.sqrt(rho) * R) / R)
                        tot += fij * fkl * wa[i] * wa[j] * wb[k] * wb[l] * \
                            (math.pi / p) ** 1.5 * (math.pi / q) ** 1.5 * inter
        return tot

    for R in (0.0, 0.7, 2.5, 9.0):
        a = np.exp(rng.uniform(np.log(0.1), np.log(10), size=3))
        b = np.exp(rng.uniform(np.log(0.1), np.log(10), size=3))
        da, db = rng.uniform(0.1, 1.0, size=3), rng.uniform(0.1, 1.0, size=3)
        basis = W.Basis(np.array([[0.0, 0.0, 0.0], [0.0, R * 0.8, -R * 0.6]]),
                        np.array([3, 3], dtype=np.int32), np.concatenate([a, b]),
                        np.concatenate([da, db]))
        o = Oracle(basis)
        wa, wb = weights(a, da), weights(b, db)
        ref = cloud_sum(wa, a, wb, b, R)
        assert abs(o.eri(0, 0, 1, 1) - ref) <= 1e-12 * ref, R
        assert abs(o.eri(1, 1, 0, 0) - ref) <= 1e-12 * ref, R
        # the pin's sensitivity to the slips it is meant to catch
        assert abs(cloud_sum(wa, a, wb, b, R, diag=2.0) - ref) > 1e-3 * ref
        assert abs(cloud_sum(wa, a, wb, b, R, cross=0.0) - ref) > 1e-3 * ref


def test_four_center_integral_by_quadrature():
    """General (ab|cd) against 1/r = (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt,
    with the six-dimensional Gaussian integral done in closed form and the
    t integral done numerically (independent of F0 and its prefactor)."""
    rng = np.random.default_rng(11)
    for _ in range(6):
        cen = rng.uniform(-1.5, 1.5, size=(4, 3))
        ex = np.exp(rng.uniform(np.log(0.1), np.log(10), size=4))
        o = Oracle(one_prim_basis(cen, ex))
        a, b, c, d = ex
        A, B, Cc, Dd = cen
        nrm = np.prod((2 * ex / np.pi) ** 0.75)
        p, q = a + b, c + d
        P, Q = (a * A + b * B) / p, (c * Cc + d * Dd) / q
        Kab = math.exp(-a * b / p * np.sum((A - B) ** 2))
        Kcd = math.exp(-c * d / q * np.sum((Cc - Dd) ** 2))
        R2 = np.sum((P - Q) ** 2)

        def f(t):
            det = p * q + (p + q) * t * t
            return (np.pi ** 2 / det) ** 1.5 * math.exp(-p * q * t * t / det * R2)

        val, _ = integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)
        ref = nrm * Kab * Kcd * 2 / math.sqrt(math.pi) * val
        assert abs(o.eri(0, 1, 2, 3) - ref) <= 1e-11 * abs(ref)


def test_eightfold_symmetry(tiny):
    _, _, E = tiny
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.array_equal(E, E.transpose(perm)) or \
            np.max(np.abs(E - E.transpose(perm))) <= 1e-15 * np.max(np.abs(E))


def test_cauchy_schwarz_bound(tiny):
    _, o, E = tiny
    Q = o.Q
    bound = Q[:, :, None, None] * Q[None, None, :, :]
    assert np.all(np.abs(E) <= bound * (1 + 1e-12) + 1e-300)
    assert np.array_equal(Q, Q.T)
    assert np.allclose(np.diag(Q) ** 2, np.einsum('pppp->p', E), rtol=1e-13)
    i, j = 3, 17
    assert abs(Q[i, j] ** 2 - E[i, j, i, j]) <= 1e-13 * E[i, j, i, j]


# ------------------------------------------------------------- J / K
def test_exchange_index_order_two_far_centers():
    """K[D]_pq = sum_rs D_rs (pr|qs) (Eq. J_and_K).  With two far-apart
    functions only (pp|qq) survives, so for D with only D_01 = 1:
    K_01 = (00|11) = erf(sqrt(2ab/(a+b)) R)/R and K_10 = 0 -- the
    transposed convention sum_rs D_rs (ps|qr) would swap them."""
    a, b, R = 1.3, 0.7, 40.0
    o = Oracle(one_prim_basis([[0, 0, 0], [R, 0, 0]], [a, b]))
    D = np.zeros((1, 2, 2))
    D[0, 0, 1] = 1.0
    J, K, _ = o.jk_unique(D, 0.0)
    coul = special.erf(math.sqrt(2 * a * b / (a + b)) * R) / R
    assert abs(K[0, 0, 1] - coul) < 1e-14
    assert abs(K[0, 1, 0]) < 1e-200
    assert np.max(np.abs(J)) < 1e-200


def test_brute_equals_unique_tiny(tiny):
    w, o, E = tiny
    Jb, Kb = o.jk_brute(E, w.D, w.tol)
    Ju, Ku, nk = o.jk_unique(w.D, w.tol)
    P = w.basis.n * (w.basis.n + 1) // 2
    assert nk == P * (P + 1) // 2
    assert np.max(np.abs(Jb - Ju)) <= 1e-13 * np.max(np.abs(Jb))
    assert np.max(np.abs(Kb - Ku)) <= 1e-13 * np.max(np.abs(Kb))


@pytest.mark.parametrize("n,tol,seed", [(7, 0.0, 1), (10, 1e-3, 2), (13, 1e-6, 3)])
def test_brute_equals_unique_random(n, tol, seed):
    w = W.small_random(n, 3, seed, tol=tol, edge=5.0)
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((3, w.basis.n, w.basis.n))     # fully non-symmetric
    o = Oracle(w.basis)
    E = o.eri_tensor()
    Jb, Kb = o.jk_brute(E, D, tol)
    Ju, Ku, nk = o.jk_unique(D, tol)
    assert np.max(np.abs(Jb - Ju)) <= 1e-13 * np.max(np.abs(Jb))
    assert np.max(np.abs(Kb - Ku)) <= 1e-13 * np.max(np.abs(Kb))
    # kept count matches the rule applied to the unique quartets directly
    Q = o.Q
    cnt = 0
    for p in range(w.basis.n):
        for q in range(p + 1):
            for r in range(p + 1):
                for s in range(r + 1):
                    if r * (r + 1) // 2 + s <= p * (p + 1) // 2 + q and Q[p, q] * Q[r, s] >= tol:
                        cnt += 1
    assert nk == cnt == o.count_kept(tol)


def test_coulomb_einsum_and_hf_identity(tiny):
    """J[D]_pq = sum_rs D_rs (rs|pq) as a tensor contraction, and the HF
    reduction F[P].P = sum P_pq P_rs (2(pq|rs) - (pr|qs)) (Eq. esmf_eng_hf)."""
    w, o, E = tiny
    J, K, _ = o.jk_unique(w.D, 0.0)
    for k in range(w.m):
        Jt = np.einsum("rspq,rs->pq", E, w.D[k])
        assert np.max(np.abs(J[k] - Jt)) <= 1e-13 * np.max(np.abs(Jt))
    P = w.D[0]
    F, t = Oracle.fock_traces(w.D, J, K)
    ref = np.einsum("pq,rs,pqrs->", P, P, 2 * E) - np.einsum("pq,rs,prqs->", P, P, E)
    assert abs(t[0] - ref) <= 1e-12 * abs(ref)


def test_symmetry_relations(tiny):
    w, o, _ = tiny
    rng = np.random.default_rng(3)
    D = rng.standard_normal((1, w.basis.n, w.basis.n))
    J, K, _ = o.jk_unique(D, 0.0)
    Jt, Kt, _ = o.jk_unique(np.ascontiguousarray(D.transpose(0, 2, 1)), 0.0)
    Js, Ks, _ = o.jk_unique(0.5 * (D + D.transpose(0, 2, 1)), 0.0)
    sc = np.max(np.abs(K))
    assert np.max(np.abs(J - J.transpose(0, 2, 1))) <= 1e-13 * np.max(np.abs(J))   # J symmetric
    assert np.max(np.abs(Kt - K.transpose(0, 2, 1))) <= 1e-13 * sc                  # K[D^T] = K[D]^T
    assert np.max(np.abs(Js - J)) <= 1e-13 * np.max(np.abs(J))                      # J[D] = J[(D+D^T)/2]
    assert np.max(np.abs(Ks - Ks.transpose(0, 2, 1))) <= 1e-13 * sc                 # K symmetric for symmetric D
    assert np.max(np.abs(K - K.transpose(0, 2, 1))) > 1e-6 * sc                     # and not otherwise


def test_positivity(tiny):
    """D.J[D] >= 0 and D.K[D] >= 0 for any real D (1/r12 is a positive kernel)."""
    w, o, _ = tiny
    rng = np.random.default_rng(5)
    D = rng.standard_normal((4, w.basis.n, w.basis.n))
    J, K, _ = o.jk_unique(D, 0.0)
    assert np.all(np.einsum("kpq,kpq->k", D, J) > 0)
    assert np.all(np.einsum("kpq,kpq->k", D, K) > 0)


def test_grouped_equals_separate_and_linearity(tiny):
    w, o, _ = tiny
    J, K, _ = o.jk_unique(w.D, 0.0)
    for k in range(w.m):
        Jk, Kk, _ = o.jk_unique(w.D[k:k + 1], 0.0)
        assert np.array_equal(Jk[0], J[k]) and np.array_equal(Kk[0], K[k])
    a, b = 0.7, -1.9
    Jl, Kl, _ = o.jk_unique((a * w.D[1] + b * w.D[2])[None], 0.0)
    assert np.max(np.abs(Jl[0] - (a * J[1] + b * J[2]))) <= 1e-13 * np.max(np.abs(Jl))
    assert np.max(np.abs(Kl[0] - (a * K[1] + b * K[2]))) <= 1e-13 * np.max(np.abs(Kl))


def test_fd_derivative_identity(tiny):
    """d/dTheta_kp (F[Theta^T Theta] . Theta^T Theta) = 4 (Theta F[Theta^T Theta])_kp
    (Appendix, Eq. eng2_der_theta_kp4 with N2 = 1), by central differences."""
    w, o, E = tiny
    rng = np.random.default_rng(9)
    n, no = w.basis.n, 3
    Th = rng.standard_normal((no, n)) / math.sqrt(n)

    def energy(T):
        D = (T.T @ T)[None]
        J, K = o.jk_brute(E, D, 0.0)
        return float(np.sum(D[0] * (2 * J[0] - K[0])))

    D = (Th.T @ Th)[None]
    J, K = o.jk_brute(E, D, 0.0)
    grad = 4 * Th @ (2 * J[0] - K[0])
    h = 1e-4
    for (k, p) in [(0, 0), (1, 5), (2, 11), (0, 23), (2, 17)]:
        Tp, Tm = Th.copy(), Th.copy()
        Tp[k, p] += h
        Tm[k, p] -= h
        fd = (energy(Tp) - energy(Tm)) / (2 * h)
        assert abs(fd - grad[k, p]) <= 1e-7 * max(1.0, abs(grad[k, p])), (k, p, fd, grad[k, p])


def test_screening_bound():
    """Each dropped integral obeys |(pq|rs)| <= Q_pq Q_rs < tol, so
    |J_scr - J_full|_pq <= tol * sum_rs |D_rs| (likewise K)."""
    w = W.small_random(14, 2, 4, edge=9.0)
    o = Oracle(w.basis)
    tol = 1e-4
    Jf, Kf, nf = o.jk_unique(w.D, 0.0)
    Js, Ks, ns = o.jk_unique(w.D, tol)
    assert ns < nf
    for k in range(w.m):
        bound = tol * np.sum(np.abs(w.D[k]))
        assert np.max(np.abs(Js[k] - Jf[k])) <= bound
        assert np.max(np.abs(Ks[k] - Kf[k])) <= bound
    assert np.max(np.abs(Js - Jf)) > 0


def test_rows_equal_the_unique_loop():
    """Whole rows of J and K (each integral with first index p evaluated once)
    equal the rows of the unique-quartet build, with screening and a
    non-symmetric density."""
    w = W.small_random(21, 3, 4, tol=1e-7, edge=9.25)
    D = w.D + 0.3 * np.random.default_rng(1).standard_normal(w.D.shape)
    o = Oracle(w.basis)
    J, K, _ = o.jk_unique(D, w.tol)
    rows = [0, 5, 7, 8, w.basis.n - 1]
    Jr, Kr = o.jk_rows(D, w.tol, rows)
    assert np.max(np.abs(Jr - J[:, rows, :])) <= 1e-13 * np.max(np.abs(J))
    assert np.max(np.abs(Kr - K[:, rows, :])) <= 1e-13 * np.max(np.abs(K))


def test_elements_and_ranges_and_stored_list(tiny):
    w, o, _ = tiny
    J, K, nk = o.jk_unique(w.D, 0.0)
    idx = [(0, 0), (3, 17), (17, 3), (23, 9)]
    Je, Ke = o.jk_elements(w.D, 0.0, idx, idx)
    for e, (p, q) in enumerate(idx):
        assert np.allclose(Je[:, e], J[:, p, q], rtol=1e-13, atol=1e-15)
        assert np.allclose(Ke[:, e], K[:, p, q], rtol=1e-13, atol=1e-15)
    npair = w.basis.n * (w.basis.n + 1) // 2
    J1, K1, n1 = o.jk_unique(w.D, 0.0, pair_range=(0, 100))
    J2, K2, n2 = o.jk_unique(w.D, 0.0, pair_range=(100, npair))
    assert n1 + n2 == nk
    assert np.max(np.abs(J1 + J2 - J)) <= 1e-13 * np.max(np.abs(J))
    lst, cnt = o.unique_list(0.0, (100, 160), 10 ** 6)
    Ja, Ka, _ = o.jk_unique(w.D, 0.0, pair_range=(100, 160))
    Jb, Kb, _ = o.jk_unique(w.D, 0.0, pair_range=(100, 160), eri_list=lst)
    assert cnt == lst.size and np.array_equal(Ja, Jb) and np.array_equal(Ka, Kb)
