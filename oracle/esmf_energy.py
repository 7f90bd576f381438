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
