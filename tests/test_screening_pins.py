"""Pins of the oracle's pair rule (Sec. II.C: discard pair (p, q) when
max_rs |(pq|rs)| <= tol) against facts outside its loop: the closed-form
self-repulsion of one function, the Cauchy-Schwarz sandwich
Q_pq^2 <= max_rs |(pq|rs)| <= Q_pq max Q, the maximum over the full integral
tensor, and J/K of the surviving quartets written as masked tensor
contractions.  CPU only."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W
from test_oracle_pins import golden, one_prim_basis


def test_single_function_pair_max_is_self_repulsion():
    g = golden()
    o = Oracle(one_prim_basis([[0.3, -1.0, 2.0]], [1.0]))
    assert abs(o.pair_max()[0, 0] - g["ss_self_repulsion_a1"]) < 1e-15


@pytest.fixture(scope="module")
def small():
    w = W.small_random(10, 1, 7, edge=9.0)
    o = Oracle(w.basis)
    return w, o, o.eri_tensor()


def test_pair_max_is_the_tensor_maximum_and_is_bounded(small):
    w, o, eri = small
    n = w.basis.n
    pm = o.pair_max()
    np.testing.assert_allclose(pm, np.abs(eri).reshape(n, n, n * n).max(axis=2), rtol=0, atol=1e-15)
    np.testing.assert_allclose(pm, pm.T, rtol=0, atol=0)
    Q = o.Q
    assert np.all(pm >= Q * Q * (1 - 1e-13))
    assert np.all(pm <= Q * Q.max() * (1 + 1e-13))


@pytest.mark.parametrize("thr", [1e-6, 1e-3])
def test_pair_rule_jk_is_the_masked_contraction(small, thr):
    """jk_unique over the 0/1 pair table (tol 0.5) keeps exactly the quartets
    of two surviving pairs: J and K equal Eq. (J_and_K) over the tensor with
    every dropped pair zeroed."""
    w, o, eri = small
    n = w.basis.n
    S = o.pair_mask_table(thr)
    assert 0 < S.sum() < n * n                     # the rule bites on this geometry
    mask = S[:, :, None, None] * S[None, None, :, :]
    e = eri * mask
    D = W.esmf_densities(W.rng_for(3), n, 3, 3)
    J, K, nk = o.jk_unique(D, 0.5, Q=S)
    Jr = np.einsum("rspq,krs->kpq", e, D)
    Kr = np.einsum("prqs,krs->kpq", e, D)
    np.testing.assert_allclose(J, Jr, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(K, Kr, rtol=1e-12, atol=1e-13)
    iu = [(p, q) for p in range(n) for q in range(p + 1)]
    keep = [S[p, q] > 0.5 for (p, q) in iu]
    expect = sum(1 for i in range(len(iu)) for j in range(i + 1) if keep[i] and keep[j])
    assert nk == expect == o.count_kept(0.5, Q=S)


# ------------------------------------------------- density-weighted screening
@pytest.mark.parametrize("tol_d", [1e-5, 1e-3])
def test_density_weighted_jk_is_the_masked_contraction(small, tol_d):
    """The density-weighted rule keeps a Schwarz-kept quartet iff Q_pq Q_rs
    times the largest |D_k| over its six index pairs (both orders, all k)
    reaches tol_d.  J and K equal Eq. (J_and_K) over the tensor with every
    dropped quartet zeroed; the weight is formed here with numpy."""
    w, o, eri = small
    n = w.basis.n
    D = W.esmf_densities(W.rng_for(5), n, 3, 4)
    D = D + 0.05 * np.random.default_rng(2).standard_normal(D.shape)       # non-symmetric
    Wd = np.max(np.maximum(np.abs(D), np.abs(D.transpose(0, 2, 1))), axis=0)
    np.testing.assert_array_equal(o.density_weight(D), Wd)
    Q = o.Q
    QQ = Q[:, :, None, None] * Q[None, None, :, :]
    wt = np.maximum.reduce([Wd[None, None, :, :] + 0 * QQ,                 # r s
                            Wd[:, :, None, None] + 0 * QQ,                 # p q
                            Wd[None, :, None, :] + 0 * QQ,                 # q s
                            Wd[:, None, None, :] + 0 * QQ,                 # p s
                            Wd[None, :, :, None] + 0 * QQ,                 # q r
                            Wd[:, None, :, None] + 0 * QQ])                # p r
    mask = (QQ * wt >= tol_d).astype(float)
    assert 0 < mask.mean() < 1                                             # the rule bites
    e = eri * mask
    J, K, nk = o.jk_unique_dw(D, 0.0, tol_d)
    np.testing.assert_allclose(J, np.einsum("rspq,krs->kpq", e, D), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(K, np.einsum("prqs,krs->kpq", e, D), rtol=1e-12, atol=1e-13)
    # kept unique quartets: the mask is invariant under the 8 permutations
    iu = [(p, q) for p in range(n) for q in range(p + 1)]
    expect = sum(1 for i in range(len(iu)) for j in range(i + 1)
                 if mask[iu[i][0], iu[i][1], iu[j][0], iu[j][1]] > 0)
    assert nk == expect


def test_density_weighted_zero_tolerance_is_schwarz_alone(small):
    w, o, _ = small
    D = W.esmf_densities(W.rng_for(6), w.basis.n, 3, 2)
    J0, K0, n0 = o.jk_unique(D, 1e-9)
    J1, K1, n1 = o.jk_unique_dw(D, 1e-9, 0.0)
    assert n0 == n1
    np.testing.assert_array_equal(J0, J1)
    np.testing.assert_array_equal(K0, K1)


def test_density_weighted_error_bound(small):
    """Each dropped update is below tol_d, so |X_dw - X|_pq <= tol_d times the
    number of ordered quartets that update element pq (N^2 for J and K)."""
    w, o, _ = small
    n = w.basis.n
    D = W.esmf_densities(W.rng_for(8), n, 3, 3)
    tol_d = 1e-4
    J0, K0, _ = o.jk_unique(D, 0.0)
    J1, K1, nk = o.jk_unique_dw(D, 0.0, tol_d)
    assert nk < n * (n + 1) // 2 * (n * (n + 1) // 2 + 1) // 2
    assert np.max(np.abs(J1 - J0)) <= tol_d * n * n
    assert np.max(np.abs(K1 - K0)) <= tol_d * n * n
