"""FP64 oracle of the ESMF energy and its first derivatives.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.  Plain NumPy in float64,
written term by term from the equations it cites; the Fock-like builds come
from a caller-supplied jk(D) -> (J, K) (the oracle's unique-quartet loop).

Notation (Table I): Theta = first N_o rows of V, Gamma = last N_v rows,
N2 = c0^2 + 2 sum_ia sigma_ia^2, A = Gamma^T sigma^T sigma Gamma -
Theta^T sigma sigma^T Theta, F[D] = 2 J[D] - K[D] (Eq. J_and_K) and
X . Y = sum_pq X_pq Y_pq.  Below P = Theta^T Theta and T = Theta^T sigma Gamma.

Readings of garbled or inconsistent printed equations (each pinned in
tests/test_energy_pins.py):
  * Eq. (esmf_energy_2b), last term.  Printed 2 F[Theta^T sigma Gamma] .
    (Theta^T Theta), which is linear in sigma although the purely excited
    block must be quadratic in sigma; the printed sigma derivative contains
    4 Theta F[T] Gamma^T, the derivative of 2 F[T] . T.  Read as 2 F[T] . T.
    Pinned against the Slater-Condon CIS energy in the MO basis.
  * Eq. (eng_der_sigma_jb).  The term printed 4 sum_pq (F[P] Theta^T Theta)_pq
    sigma_jb is read as 4 (F[P] . P) sigma_jb (the sigma derivative of the
    N2 F[P] . P term of E2).
  * Eq. (eng_der_ukp), dE/dTheta.  As printed it pairs F[A] - F[A]^T (zero for
    the symmetric A), has sign and transpose slips and a misplaced 1/N2; the
    derivative is written here from E directly (each line below names the
    energy term it differentiates) and pinned by finite differences.
  * Eq. (eng_der_ucp), dE/dGamma.  Printed without the overall 1/N2 that E
    carries (N2 does not depend on Gamma); read with it.
"""
from __future__ import annotations

import numpy as np


def fock(jk, D):
    """F[D_k] = 2 J[D_k] - K[D_k] for a batch D of shape (m, N, N) (Eq. J_and_K)."""
    J, K = jk(np.ascontiguousarray(D))[:2]
    return 2.0 * J - K


def dot(X, Y):
    """Matrix inner product X . Y = sum_pq X_pq Y_pq (Table I)."""
    return float(np.sum(X * Y))


def pieces(G, V, sigma, c0, nocc):
    """Table I quantities of one ESMF state."""
    Th = V[:nocc]
    Ga = V[nocc:]
    N2 = c0 * c0 + 2.0 * float(np.sum(sigma * sigma))
    P = Th.T @ Th
    T = Th.T @ sigma @ Ga
    A = Ga.T @ sigma.T @ sigma @ Ga - Th.T @ sigma @ sigma.T @ Th
    return Th, Ga, N2, P, T, A


def energy_terms(G, Th, Ga, sigma, c0, N2, FP, FT, P, T, A):
    """E1 (Eq. esmf_energy_1b) and E2 (Eq. esmf_energy_2b, last term read as
    2 F[T] . T)."""
    E1 = (2.0 * N2 * np.trace(Th @ G @ Th.T)
          + 4.0 * c0 * np.trace(Th @ G @ Ga.T @ sigma.T)
          + 2.0 * np.trace(sigma @ Ga @ G @ Ga.T @ sigma.T - Th @ G @ Th.T @ sigma @ sigma.T))
    E2 = (N2 * dot(FP, P) + 4.0 * c0 * dot(FP, T) + 2.0 * dot(FP, A)
          + 2.0 * dot(FT, T))
    return float(E1), float(E2)


def energy(jk, G, V, sigma, c0, nocc):
    """ESMF energy E = (E1 + E2) / N2 (Eq. esmf_eng); needs F[P] and F[T]."""
    Th, Ga, N2, P, T, A = pieces(G, V, sigma, c0, nocc)
    FP, FT = fock(jk, np.stack([P, T]))
    E1, E2 = energy_terms(G, Th, Ga, sigma, c0, N2, FP, FT, P, T, A)
    return (E1 + E2) / N2


def energy_gradient(jk, G, V, sigma, c0, nocc):
    """E and its derivatives with respect to c0, sigma and V (rows Theta then
    Gamma), from one grouped build of F[P], F[T], F[A] (the three builds the
    energy derivatives need, Sec. II.B.3)."""
    Th, Ga, N2, P, T, A = pieces(G, V, sigma, c0, nocc)
    FP, FT, FA = fock(jk, np.stack([P, T, A]))
    E1, E2 = energy_terms(G, Th, Ga, sigma, c0, N2, FP, FT, P, T, A)
    E = (E1 + E2) / N2
    s = sigma
    # Eq. (eng_der_c0)
    dc0 = (4.0 * c0 * np.trace(Th @ G @ Th.T) + 4.0 * np.trace(Th @ G @ Ga.T @ s.T)
           + 2.0 * c0 * dot(FP, P) + 4.0 * dot(FP, T)) / N2 - 2.0 * c0 * E / N2
    # Eq. (eng_der_sigma_jb)
    dsig = (4.0 * c0 * (Th @ G @ Ga.T) + 4.0 * (s @ Ga @ G @ Ga.T)
            - 4.0 * (Th @ G @ Th.T @ s) + 8.0 * np.trace(Th @ G @ Th.T) * s
            + 4.0 * c0 * (Th @ FP @ Ga.T) + 4.0 * (s @ Ga @ FP @ Ga.T)
            - 4.0 * (Th @ FP @ Th.T @ s) + 4.0 * (Th @ FT @ Ga.T)
            + 4.0 * dot(FP, P) * s) / N2 - 4.0 * E * s / N2
    # dE/dTheta, term by term from E (N2 does not depend on Theta):
    dth = (4.0 * N2 * (Th @ G)                       # 2 N2 Tr[Theta G Theta^T]
           + 4.0 * c0 * (s @ Ga @ G)                 # 4 c0 Tr[Theta G Gamma^T sigma^T]
           - 4.0 * (s @ s.T @ Th @ G)                # -2 Tr[Theta G Theta^T sigma sigma^T]
           + 4.0 * N2 * (Th @ FP)                    # N2 F[P] . P
           + 4.0 * c0 * (s @ Ga @ FP)                # 4 c0 F[P] . T, through T
           + 4.0 * c0 * (Th @ (FT + FT.T))           # 4 c0 F[P] . T, through F[P]
           + 2.0 * (Th @ (FA + FA.T))                # 2 F[P] . A, through F[P]
           - 4.0 * (s @ s.T @ Th @ FP)               # 2 F[P] . A, through A
           + 4.0 * (s @ Ga @ FT.T)) / N2             # 2 F[T] . T
    # Eq. (eng_der_ucp), with the 1/N2 of E
    dga = (4.0 * c0 * (s.T @ Th @ G) + 4.0 * (s.T @ s @ Ga @ G)
           + 4.0 * c0 * (s.T @ Th @ FP) + 4.0 * (s.T @ s @ Ga @ FP)
           + 4.0 * (s.T @ Th @ FT)) / N2
    dV = np.vstack([dth, dga])
    return float(E), float(dc0), dsig, dV


def cis_energy_mo(eri, G, V, sigma, c0, nocc):
    """The same energy from the MO basis by the Slater-Condon rules for a
    reference determinant plus spin-adapted single excitations (Szabo and
    Ostlund, Ch. 2 and 4): with the singles written sigma_ia (E_ai,alpha +
    E_ai,beta)|Phi>, the norm is N2 and
      <Psi|H|Psi> = c0^2 E0 + 4 c0 sum_ia sigma_ia f_ia
                  + 2 sum_ia,jb sigma_ia sigma_jb [delta_ij delta_ab E0
                      + delta_ij f_ab - delta_ab f_ij + 2 (ia|jb) - (ij|ab)],
    E0 = 2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)], f = h + sum_j [2 (..|jj)
    - (.j|j.)].  eri is the full AO tensor (pq|rs).  An independent check of
    the AO-basis expressions, not used by them."""
    no = nocc
    h = V @ G @ V.T
    g = np.einsum("pqrs,ip,jq,kr,ls->ijkl", eri, V, V, V, V, optimize=True)
    o, v = slice(0, no), slice(no, None)
    E0 = 2.0 * np.trace(h[o, o]) + sum(2.0 * g[i, i, j, j] - g[i, j, j, i]
                                       for i in range(no) for j in range(no))
    f = h + 2.0 * np.einsum("pqjj->pq", g[:, :, o, o]) - np.einsum("pjjq->pq", g[:, o, o, :])
    s = sigma
    N2 = c0 * c0 + 2.0 * float(np.sum(s * s))
    cross = 4.0 * c0 * float(np.sum(s * f[o, v]))
    blk = (E0 * float(np.sum(s * s))
           + float(np.einsum("ia,ab,ib->", s, f[v, v], s))
           - float(np.einsum("ia,ij,ja->", s, f[o, o], s))
           + float(np.einsum("ia,jb,iajb->", s, s, 2.0 * g[o, v, o, v]))
           - float(np.einsum("ia,jb,ijab->", s, s, g[o, o, v, v])))
    return (c0 * c0 * E0 + cross + 2.0 * blk) / N2


# ---------------------------------------------------------------------------
# GVP objective (Eq. esmf_gvb) and its derivatives (Eq. esmf_l_gvp_der)
#
# Variables x: c0, sigma_ia and the orbital rotation X (antisymmetric,
# independent entries X_pq, p > q), with V(X) = exp(X) V at the current
# orbitals (the paper's U -> U exp(-X) with X reset to zero after each step,
# Eq. redefine_U).  At X = 0 the rotation gradient is Gx = Gam - Gam^T with
# Gam = (dE/dV) V^T, and |grad E|^2 = (dE/dc0)^2 + |dE/dsigma|^2 + |Gx|_F^2 / 2.
# The sum over y of dE/dy d2E/dxdy is the Hessian-vector product H g, the
# directional derivative of the gradient along g; it is written out below by
# the product rule (energy_gradient_tangent), so its Fock builds are the
# three of the tangent densities (P', T', A') rather than the paper's six
# (those are pieces of the same three, Sec. II.B.3).
# ---------------------------------------------------------------------------


def energy_gradient_tangent(jk, G, V, sigma, c0, nocc, dV, dsig, dc0):
    """energy_gradient and its directional derivative along (dc0, dsigma, dV):
    returns (E, gc0, gsig, gV) and (E', gc0', gsig', gV'), each term of
    energy_gradient differentiated by the product rule."""
    Th, Ga, N2, P, T, A = pieces(G, V, sigma, c0, nocc)
    Tt, Gt = dV[:nocc], dV[nocc:]
    s, st = sigma, dsig
    FP, FT, FA = fock(jk, np.stack([P, T, A]))
    Pt = Tt.T @ Th + Th.T @ Tt
    Ttan = Tt.T @ s @ Ga + Th.T @ st @ Ga + Th.T @ s @ Gt
    At = (Gt.T @ s.T @ s @ Ga + Ga.T @ st.T @ s @ Ga + Ga.T @ s.T @ st @ Ga + Ga.T @ s.T @ s @ Gt
          - Tt.T @ s @ s.T @ Th - Th.T @ st @ s.T @ Th - Th.T @ s @ st.T @ Th - Th.T @ s @ s.T @ Tt)
    FPt, FTt, FAt = fock(jk, np.stack([Pt, Ttan, At]))
    Fk, Fkt = G + FP, FPt
    N2t = 2.0 * c0 * dc0 + 4.0 * dot(s, st)
    s0, s1, s2, s3 = dot(G + Fk, P), dot(Fk, T), dot(Fk, A), dot(FT, T)
    s0t = dot(Fkt, P) + dot(G + Fk, Pt)
    s1t = dot(Fkt, T) + dot(Fk, Ttan)
    s2t = dot(Fkt, A) + dot(Fk, At)
    s3t = dot(FTt, T) + dot(FT, Ttan)
    num = N2 * s0 + 4.0 * c0 * s1 + 2.0 * s2 + 2.0 * s3
    numt = N2t * s0 + N2 * s0t + 4.0 * dc0 * s1 + 4.0 * c0 * s1t + 2.0 * s2t + 2.0 * s3t
    E = num / N2
    Et = (numt - E * N2t) / N2
    # dE/dc0 = Yc / N2
    Yc = 2.0 * c0 * s0 + 4.0 * s1 - 2.0 * c0 * E
    Yct = 2.0 * dc0 * s0 + 2.0 * c0 * s0t + 4.0 * s1t - 2.0 * dc0 * E - 2.0 * c0 * Et
    gc0 = Yc / N2
    gc0t = (Yct - gc0 * N2t) / N2
    # dE/dsigma = Ys / N2
    Ys = (4.0 * c0 * Th @ Fk @ Ga.T + 4.0 * s @ Ga @ Fk @ Ga.T - 4.0 * Th @ Fk @ Th.T @ s
          + 4.0 * Th @ FT @ Ga.T + 4.0 * (s0 - E) * s)
    Yst = (4.0 * dc0 * Th @ Fk @ Ga.T
           + 4.0 * c0 * (Tt @ Fk @ Ga.T + Th @ Fkt @ Ga.T + Th @ Fk @ Gt.T)
           + 4.0 * (st @ Ga @ Fk @ Ga.T + s @ Gt @ Fk @ Ga.T + s @ Ga @ Fkt @ Ga.T + s @ Ga @ Fk @ Gt.T)
           - 4.0 * (Tt @ Fk @ Th.T @ s + Th @ Fkt @ Th.T @ s + Th @ Fk @ Tt.T @ s + Th @ Fk @ Th.T @ st)
           + 4.0 * (Tt @ FT @ Ga.T + Th @ FTt @ Ga.T + Th @ FT @ Gt.T)
           + 4.0 * (s0t - Et) * s + 4.0 * (s0 - E) * st)
    gs = Ys / N2
    gst = (Yst - gs * N2t) / N2
    # dE/dTheta = 4 Theta Fk + Yt / N2
    Yt = (4.0 * c0 * s @ Ga @ Fk + 4.0 * c0 * Th @ (FT + FT.T) + 2.0 * Th @ (FA + FA.T)
          - 4.0 * s @ s.T @ Th @ Fk + 4.0 * s @ Ga @ FT.T)
    Ytt = (4.0 * dc0 * s @ Ga @ Fk + 4.0 * c0 * (st @ Ga @ Fk + s @ Gt @ Fk + s @ Ga @ Fkt)
           + 4.0 * dc0 * Th @ (FT + FT.T) + 4.0 * c0 * (Tt @ (FT + FT.T) + Th @ (FTt + FTt.T))
           + 2.0 * Tt @ (FA + FA.T) + 2.0 * Th @ (FAt + FAt.T)
           - 4.0 * (st @ s.T @ Th @ Fk + s @ st.T @ Th @ Fk + s @ s.T @ Tt @ Fk + s @ s.T @ Th @ Fkt)
           + 4.0 * (st @ Ga @ FT.T + s @ Gt @ FT.T + s @ Ga @ FTt.T))
    gth = 4.0 * Th @ Fk + Yt / N2
    gtht = 4.0 * (Tt @ Fk + Th @ Fkt) + (Ytt - Yt / N2 * N2t) / N2
    # dE/dGamma = Yg / N2
    Yg = 4.0 * c0 * s.T @ Th @ Fk + 4.0 * s.T @ s @ Ga @ Fk + 4.0 * s.T @ Th @ FT
    Ygt = (4.0 * dc0 * s.T @ Th @ Fk + 4.0 * c0 * (st.T @ Th @ Fk + s.T @ Tt @ Fk + s.T @ Th @ Fkt)
           + 4.0 * (st.T @ s @ Ga @ Fk + s.T @ st @ Ga @ Fk + s.T @ s @ Gt @ Fk + s.T @ s @ Ga @ Fkt)
           + 4.0 * (st.T @ Th @ FT + s.T @ Tt @ FT + s.T @ Th @ FTt))
    gga = Yg / N2
    ggat = (Ygt - gga * N2t) / N2
    return ((float(E), float(gc0), gs, np.vstack([gth, gga])),
            (float(Et), float(gc0t), gst, np.vstack([gtht, ggat])))


def rotation_gradient(V, gV):
    """Gx = Gam - Gam^T, Gam = (dE/dV) V^T: the derivative with respect to
    the independent entries X_pq (p > q) of V(X) = exp(X) V at X = 0."""
    Gam = gV @ V.T
    return Gam - Gam.T


def gvp_gradient(jk, G, V, sigma, c0, nocc, omega, mu, chi):
    """L_mu,chi = chi (mu (omega - E)^2 + (1 - mu) |grad E|^2) + (1 - chi) E
    (Eq. esmf_gvb) and its derivatives (Eq. esmf_l_gvp_der):
      dL/dx = chi (-2 mu (omega - E) g_x + 2 (1 - mu) (H g)_x) + (1 - chi) g_x.
    Returns (L, E, |grad E|^2, dL/dc0, dL/dsigma, dL/dX) with dL/dX an
    antisymmetric N x N matrix (entry p > q is the derivative by X_pq)."""
    E, gc0, gs, gV = energy_gradient(jk, G, V, sigma, c0, nocc)
    Gam = gV @ V.T
    Gx = Gam - Gam.T
    gnorm2 = gc0 * gc0 + float(np.sum(gs * gs)) + 0.5 * float(np.sum(Gx * Gx))
    # H g: tangent of the gradient along (gc0, gs, Gx); V moves as Gx V
    Adir = Gx
    _, (_, Hc0, Hs, Mt) = energy_gradient_tangent(jk, G, V, sigma, c0, nocc, Adir @ V, gs, gc0)
    Dt = Mt @ V.T - 0.5 * (Adir @ Gam + Gam @ Adir)
    HX = Dt - Dt.T
    L = chi * (mu * (omega - E) ** 2 + (1.0 - mu) * gnorm2) + (1.0 - chi) * E
    a, b = chi * (-2.0 * mu * (omega - E)) + (1.0 - chi), chi * 2.0 * (1.0 - mu)
    return (float(L), float(E), float(gnorm2), a * gc0 + b * Hc0, a * gs + b * Hs, a * Gx + b * HX)


def rotation_gradient_at(jk, G, V0, sigma, c0, nocc, X):
    """Exact dE/dX_pq (p > q) at a nonzero X for V(X) = exp(X) V0, through
    the derivative of the matrix exponential from the block identity
    exp([[X, Z], [0, X]]) = [[e^X, dexp_X(Z)], [0, e^X]] (for tests: one
    2N x 2N exponential per entry, small N only)."""
    from scipy.linalg import expm
    n = X.shape[0]
    V = expm(X) @ V0
    _, _, _, gV = energy_gradient(jk, G, V, sigma, c0, nocc)
    out = np.zeros_like(X)
    for p in range(n):
        for q in range(p):
            Z = np.zeros_like(X)
            Z[p, q], Z[q, p] = 1.0, -1.0
            big = np.zeros((2 * n, 2 * n))
            big[:n, :n] = X
            big[n:, n:] = X
            big[:n, n:] = Z
            dV = expm(big)[:n, n:] @ V0
            out[p, q] = float(np.sum(gV * dV))
            out[q, p] = -out[p, q]
    return out
