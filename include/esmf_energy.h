/*
 * esmf_energy.h -- ESMF energy and its first derivatives on the device,
 * built on the grouped generalized-Fock builds of esmf_fock.h.
 *
 * Sec. II.B.2 ("ESMF Energy"): with orbital coefficients V = U^T C (rows are
 * orbitals; Theta = the first N_o rows, Gamma = the last N_v = N - N_o),
 * singles coefficients sigma (N_o x N_v), reference coefficient c0 and the
 * one-electron AO integrals G,
 *     E = (E1 + E2) / N2,  N2 = c0^2 + 2 sum_ia sigma_ia^2      (Eq. esmf_eng)
 *     E1 = 2 N2 Tr[Theta G Theta^T] + 4 c0 Tr[Theta G Gamma^T sigma^T]
 *          + 2 Tr[sigma Gamma G Gamma^T sigma^T - Theta G Theta^T sigma sigma^T]
 *                                                             (Eq. esmf_energy_1b)
 *     E2 = N2 F[P].P + 4 c0 F[P].T + 2 F[P].A + 2 F[T].T        (Eq. esmf_energy_2b)
 * where P = Theta^T Theta, T = Theta^T sigma Gamma, A = Gamma^T sigma^T sigma
 * Gamma - Theta^T sigma sigma^T Theta (Table I), F[D] = 2 J[D] - K[D] and
 * X.Y = sum_pq X_pq Y_pq.  The last E2 term is printed in the paper as
 * 2 F[T].(Theta^T Theta); it is used here as 2 F[T].T, the form that the
 * paper's own sigma derivative and the Slater-Condon CIS energy imply.
 * The derivatives with respect to c0, sigma, Theta and Gamma are those of the
 * appendix (Eqs. eng_der_c0, eng_der_sigma_jb, eng_der_ukp, eng_der_ucp),
 * with dE/dTheta and dE/dGamma written from E directly where the printed
 * equations are inconsistent; dE/dU follows as C (dE/dV)^T (Eq. der_v_to_u).
 *
 * All three Fock-like matrices the derivatives need, F[P], F[T] and F[A]
 * (Sec. II.B.3), come from ONE grouped build over the handle's integrals
 * (two, F[P] and F[T], for the energy alone).  Everything else is O(N^3)
 * FP64 matrix algebra on the device.  Conventions as in esmf_fock.h.
 */
#ifndef ESMF_ENERGY_H
#define ESMF_ENERGY_H

#include "esmf_fock.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * esmf_energy_gradient -- ESMF energy and, optionally, its gradient.
 *   h          handle from esmf_fock_create; N = its basis size
 *   n_occ      N_o, 1 <= n_occ < N
 *   c0         reference-determinant coefficient (finite)
 *   G          device, N x N, symmetric one-electron AO matrix
 *   V          device, N x N, orbitals in rows (Theta rows first)
 *   sigma      device, N_o x N_v
 *   scalars    device, 2 doubles, receives {E, dE/dc0}
 *   dE_dsigma  device, N_o x N_v, receives dE/dsigma; NULL for the energy only
 *   dE_dV      device, N x N, receives dE/dV (dE/dTheta rows, then dE/dGamma);
 *              NULL exactly when dE_dsigma is NULL
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 * Asynchronous like esmf_fock_build, and it shares the handle's work memory:
 * calls on one handle must not overlap on the GPU.  The handle keeps at most
 * 26 N^2 doubles of energy work memory, allocated on first use (and grown
 * when n_occ changes the layout) and freed by esmf_fock_destroy.
 * Precision: the products are FP64; the Fock builds run in the handle's
 * precision (FP64, FP32 or split FP16 with FP32 accumulation).
 * Errors: INVALID_ARG (sizes, NULL or host pointers, non-finite c0), OOM,
 * CUDA, and those of esmf_fock_build.
 */
int esmf_energy_gradient(esmf_fock_t *h, int n_occ, double c0, const double *G,
                         const double *V, const double *sigma, double *scalars,
                         double *dE_dsigma, double *dE_dV, void *stream);

/*
 * esmf_gvp_gradient -- the generalized-variational-principle objective of
 * Eq. (esmf_gvb),
 *     L = chi (mu (omega - E)^2 + (1 - mu) |grad E|^2) + (1 - chi) E,
 * and its derivatives (Eq. esmf_l_gvp_der)
 *     dL/dx = chi (-2 mu (omega - E) dE/dx + 2 (1 - mu) sum_y dE/dy d2E/dxdy)
 *             + (1 - chi) dE/dx
 * over the variables x = c0, sigma_ia and the orbital rotation X
 * (antisymmetric, independent entries X_pq with p > q) of V(X) = exp(X) V at
 * X = 0 (the paper's U -> U exp(-X), reset to zero after every step, Eq.
 * redefine_U).  |grad E|^2 = (dE/dc0)^2 + |dE/dsigma|^2 + |Gx|^2 / 2 with
 * Gx = (dE/dV) V^T - V (dE/dV)^T the rotation gradient.
 * Two passes, as Sec. II.B.3 describes: pass 1 is esmf_energy_gradient (one
 * grouped build of F[P], F[T], F[A]); pass 2 takes the gradient as the
 * direction and builds, in one grouped pass, the three Fock-like matrices of
 * the tangent densities P', T', A' (the paper's six pass-2 builds are pieces
 * of these three), then forms the Hessian-vector product by the product rule
 * and adds the second-order term of exp(X).
 *   h, n_occ, c0, G, V, sigma, stream  as for esmf_energy_gradient
 *   omega, mu, chi  the objective's target energy and weights (finite)
 *   scalars    device, 4 doubles, receives {L, E, |grad E|^2, dL/dc0}
 *   dL_dsigma  device, N_o x N_v
 *   dL_dX      device, N x N, antisymmetric; entry (p, q), p > q, is dL/dX_pq
 * Work memory: the energy's plus at most 31 N^2 doubles, owned by the handle.
 * Errors as for esmf_energy_gradient.
 */
int esmf_gvp_gradient(esmf_fock_t *h, int n_occ, double c0, const double *G,
                      const double *V, const double *sigma, double omega, double mu,
                      double chi, double *scalars, double *dL_dsigma, double *dL_dX,
                      void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ESMF_ENERGY_H */
