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
