// Device integrals over contracted Cartesian p and d functions, in FP64.
// Labels: 0 s; 1-3 p_x, p_y, p_z; 4-6 d_xx, d_yy, d_zz; 7-9 d_xy, d_xz, d_yz.
// Quartets of s and p functions: the Obara-Saika vertical recurrence (Obara &
// Saika, J. Chem. Phys. 84, 3963 (1986)) written out for orders up to two per
// side, and the horizontal recurrence of Head-Gordon & Pople (J. Chem. Phys.
// 89, 5777 (1988)).  Quartets with a d function: the McMurchie-Davidson
// scheme (McMurchie & Davidson, J. Comput. Phys. 26, 218 (1978)) — Hermite
// expansion coefficients of each primitive pair and Hermite Coulomb integrals
// R_tuv by their recurrences.
#pragma once

#include "esmf_internal.cuh"
#include "integrals.cuh"

namespace esmf {
namespace angular {

// F_m(T), m = 0..4: below T = 1 the Taylor series sum_k (-T)^k / (k! (2m+2k+1))
// (30 terms, truncation < 1e-33); above, F_0 from erf and the upward
// recurrence F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), whose error grows by at
// most (1/2)(3/2)(5/2)(7/2) < 7 over the four steps at T = 1.
__device__ __forceinline__ void boys_upto4(double T, double *F) {
    if (T < 1.0) {
        for (int m = 0; m <= 4; ++m) {
            double term = 1.0, sum = 1.0 / (2 * m + 1);
            for (int k = 1; k < 30; ++k) {
                term *= -T / k;
                sum += term / (2 * m + 2 * k + 1);
            }
            F[m] = sum;
        }
        return;
    }
    const double e = exp(-T), x = sqrt(T);
    F[0] = T > 40.0 ? kHalfSqrtPi / x : kHalfSqrtPi * erf(x) / x;
    for (int m = 0; m < 4; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
}

// F_m(T), m = 0..M (M <= 8): below T = 3 the Taylor series of the top order
// (40 terms, truncation < 1e-28, alternating terms below 5 in size) and the
// downward recurrence F_{m-1} = (2T F_m + exp(-T)) / (2m-1), which damps
// errors; above, F_0 from erf and the upward recurrence, whose error grows by
// at most prod_m (2m+1)/(2T) < 1.3 over eight steps at T = 3.
__device__ inline void boys_upto8(int M, double T, double *F) {
    if (T < 3.0) {
        double term = 1.0, sum = 1.0 / (2 * M + 1);
        for (int k = 1; k < 40; ++k) {
            term *= -T / k;
            sum += term / (2 * M + 2 * k + 1);
        }
        F[M] = sum;
        const double e = exp(-T);
        for (int m = M; m > 0; --m) F[m - 1] = (2.0 * T * F[m] + e) / (2 * m - 1);
        return;
    }
    const double e = exp(-T), x = sqrt(T);
    F[0] = T > 40.0 ? kHalfSqrtPi / x : kHalfSqrtPi * erf(x) / x;
    for (int m = 0; m < M; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
}

// exponent triple (lx, ly, lz) of a Cartesian label
__device__ __forceinline__ void label_exps(int lab, int *v) {
    const int x = (lab == 1) + 2 * (lab == 4) + (lab == 7) + (lab == 8);
    const int y = (lab == 2) + 2 * (lab == 5) + (lab == 7) + (lab == 9);
    const int z = (lab == 3) + 2 * (lab == 6) + (lab == 8) + (lab == 9);
    v[0] = x; v[1] = y; v[2] = z;
}

// Hermite expansion of one Cartesian direction of a primitive pair:
// (x - A)^i (x - B)^j exp(-a (x-A)^2 - b (x-B)^2)
//   = exp(-ab/p (A-B)^2) sum_t E_t Lambda_t(x; p, P),
// with E^{00}_0 = 1 (the Gaussian factor is applied with the pair) and
//   E^{i+1,j}_t = E^{ij}_{t-1} / (2p) + (P - A) E^{ij}_t + (t+1) E^{ij}_{t+1},
// and the same with (P - B) for j.  i, j <= 2, so t <= 4.
__device__ inline void hermite_e(int i, int j, double PA, double PB, double p, double *E) {
    const double h = 0.5 / p;
    E[0] = 1.0; E[1] = E[2] = E[3] = E[4] = 0.0;
    int top = 0;                                  // E_t = 0 above t = top
    for (int s = 0; s < i + j; ++s) {
        const double X = s < i ? PA : PB;
        double nx[5];
        for (int t = 0; t <= top + 1 && t < 5; ++t)
            nx[t] = (t > 0 ? h * E[t - 1] : 0.0) + X * (t <= top ? E[t] : 0.0) + (t + 1 <= top ? (t + 1) * E[t + 1] : 0.0);
        ++top;
        for (int t = 0; t <= top && t < 5; ++t) E[t] = nx[t];
    }
}

// Hermite Coulomb integrals R_tuv = R^0_tuv(alpha, PQ) for t <= TX, u <= TY,
// v <= TZ (TX + TY + TZ = L <= 8, so at most 4 x 4 x 3 = 48 of them):
//   R^n_000 = (-2 alpha)^n F_n(alpha |PQ|^2),
//   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}   (and for u, v),
// level by level from n = L down to 0; entries above t+u+v = L - n at level n
// are never used and not formed.  R is indexed (t (TY+1) + u)(TZ+1) + v.
__device__ inline void hermite_r(int TX, int TY, int TZ, double alpha, double X, double Y, double Z,
                                 const double *F, double *R) {
    const int L = TX + TY + TZ, NY = TY + 1, NZ = TZ + 1, nbox = (TX + 1) * NY * NZ;
    double other[48];
    double *prev = other, *cur = R;
    for (int k = 0; k < nbox; ++k) prev[k] = 0.0;
    double f = 1.0;
    for (int n = 0; n < L; ++n) f *= -2.0 * alpha;   // (-2 alpha)^L
    for (int n = L; n >= 0; --n) {
        for (int t = 0; t <= TX; ++t)
            for (int u = 0; u <= TY; ++u)
                for (int v = 0; v <= TZ; ++v) {
                    if (t + u + v > L - n) break;
                    const int k = (t * NY + u) * NZ + v;
                    double r;
                    if (t > 0) r = (t > 1 ? (t - 1) * prev[k - 2 * NY * NZ] : 0.0) + X * prev[k - NY * NZ];
                    else if (u > 0) r = (u > 1 ? (u - 1) * prev[k - 2 * NZ] : 0.0) + Y * prev[k - NZ];
                    else if (v > 0) r = (v > 1 ? (v - 1) * prev[k - 2] : 0.0) + Z * prev[k - 1];
                    else r = f * F[n];
                    cur[k] = r;
                }
        f /= -2.0 * alpha;
        double *tmp = prev; prev = cur; cur = tmp;
    }
    // level 0 is in prev: after an odd number of levels that is R itself
    if (prev != R)
        for (int k = 0; k < nbox; ++k) R[k] = prev[k];
}

struct OS {
    double PA[3], WP[3], QC[3], WQ[3], AB[3], CD[3];
    double p, q, rho, K;
    double F[5];
};

// [e0|f0]^(m) for e, f of order <= 2, written out (see the vertical
// recurrence above): S order 0/0, s1 1/0, t1 0/1, s2 2/0, t2 0/2, u11 1/1,
// u21 2/1, u12 1/2, u22 2/2.  Indices are Cartesian directions 0..2.
__device__ __forceinline__ double S(const OS &o, int m) { return o.K * o.F[m]; }
__device__ inline double s1(const OS &o, int i, int m) { return o.PA[i] * S(o, m) + o.WP[i] * S(o, m + 1); }
__device__ inline double t1(const OS &o, int k, int m) { return o.QC[k] * S(o, m) + o.WQ[k] * S(o, m + 1); }
__device__ inline double s2(const OS &o, int i, int j, int m) {
    double v = o.PA[j] * s1(o, i, m) + o.WP[j] * s1(o, i, m + 1);
    if (i == j) v += (S(o, m) - o.rho / o.p * S(o, m + 1)) / (2.0 * o.p);
    return v;
}
__device__ inline double t2(const OS &o, int k, int l, int m) {
    double v = o.QC[l] * t1(o, k, m) + o.WQ[l] * t1(o, k, m + 1);
    if (k == l) v += (S(o, m) - o.rho / o.q * S(o, m + 1)) / (2.0 * o.q);
    return v;
}
__device__ inline double u11(const OS &o, int i, int k, int m) {
    double v = o.PA[i] * t1(o, k, m) + o.WP[i] * t1(o, k, m + 1);
    if (i == k) v += S(o, m + 1) / (2.0 * (o.p + o.q));
    return v;
}
__device__ inline double u21(const OS &o, int i, int j, int k, int m) {
    double v = o.PA[j] * u11(o, i, k, m) + o.WP[j] * u11(o, i, k, m + 1);
    if (i == j) v += (t1(o, k, m) - o.rho / o.p * t1(o, k, m + 1)) / (2.0 * o.p);
    if (j == k) v += s1(o, i, m + 1) / (2.0 * (o.p + o.q));
    return v;
}
__device__ inline double u12(const OS &o, int i, int k, int l, int m) {
    double v = o.PA[i] * t2(o, k, l, m) + o.WP[i] * t2(o, k, l, m + 1);
    double c = 0.0;
    if (i == k) c += t1(o, l, m + 1);
    if (i == l) c += t1(o, k, m + 1);
    return v + c / (2.0 * (o.p + o.q));
}
__device__ inline double u22(const OS &o, int i, int j, int k, int l, int m) {
    double v = o.PA[j] * u12(o, i, k, l, m) + o.WP[j] * u12(o, i, k, l, m + 1);
    if (i == j) v += (t2(o, k, l, m) - o.rho / o.p * t2(o, k, l, m + 1)) / (2.0 * o.p);
    double c = 0.0;
    if (j == k) c += u11(o, i, l, m + 1);
    if (j == l) c += u11(o, i, k, m + 1);
    return v + c / (2.0 * (o.p + o.q));
}

// [e0|f0]^(0), e = 1_e1 + 1_e2, f = 1_f1 + 1_f2 (an index of -1 is absent;
// e1 = -1 implies e2 = -1, likewise for f)
__device__ inline double vrr0(const OS &o, int e1, int e2, int f1, int f2) {
    const int ne = (e1 >= 0) + (e2 >= 0), nf = (f1 >= 0) + (f2 >= 0);
    if (ne == 0 && nf == 0) return S(o, 0);
    if (ne == 1 && nf == 0) return s1(o, e1, 0);
    if (ne == 0 && nf == 1) return t1(o, f1, 0);
    if (ne == 2 && nf == 0) return s2(o, e1, e2, 0);
    if (ne == 0 && nf == 2) return t2(o, f1, f2, 0);
    if (ne == 1 && nf == 1) return u11(o, e1, f1, 0);
    if (ne == 2 && nf == 1) return u21(o, e1, e2, f1, 0);
    if (ne == 1 && nf == 2) return u12(o, e1, f1, f2, 0);
    return u22(o, e1, e2, f1, f2, 0);
}

// [a b|c d] over raw primitives with labels la..ld (0 s, 1..3 p_x..p_z) by the
// horizontal recurrence [a, b+1_j| = [a+1_j, b| + AB_j [a, b| (and the ket)
__device__ inline double prim_l(const OS &o, int la, int lb, int lc, int ld) {
    const int a = la - 1, b = lb - 1, c = lc - 1, d = ld - 1;
    // bra: {a + 1_b, coefficient 1} and {a, coefficient AB_b} when b is a p
    int be1[2], be2[2], nb = 0;
    double bc[2];
    if (b >= 0) {
        if (a >= 0) { be1[nb] = a; be2[nb] = b; } else { be1[nb] = b; be2[nb] = -1; }
        bc[nb++] = 1.0;
        be1[nb] = a; be2[nb] = -1; bc[nb++] = o.AB[b];
    } else {
        be1[nb] = a; be2[nb] = -1; bc[nb++] = 1.0;
    }
    int kf1[2], kf2[2], nk = 0;
    double kc[2];
    if (d >= 0) {
        if (c >= 0) { kf1[nk] = c; kf2[nk] = d; } else { kf1[nk] = d; kf2[nk] = -1; }
        kc[nk++] = 1.0;
        kf1[nk] = c; kf2[nk] = -1; kc[nk++] = o.CD[d];
    } else {
        kf1[nk] = c; kf2[nk] = -1; kc[nk++] = 1.0;
    }
    double v = 0.0;
    for (int x = 0; x < nb; ++x)
        for (int y = 0; y < nk; ++y) {
            const double w = bc[x] * kc[y];
            if (w != 0.0) v += w * vrr0(o, be1[x], be2[x], kf1[y], kf2[y]);
        }
    return v;
}

// contracted (pq|rs) with a d function among the four, by the McMurchie-
// Davidson scheme: per primitive quartet
//   [ab|cd] = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD
//       sum_{tuv} E^{ab}_t E^{ab}_u E^{ab}_v
//       sum_{tau nu phi} (-1)^{tau+nu+phi} E^{cd}_tau E^{cd}_nu E^{cd}_phi R_{t+tau, u+nu, v+phi}.
// Kept out of line: it is a correctness path with a large frame.
static __device__ __noinline__ double contracted_md(const DevBasis &b, int p, int q, int r, int s) {
    const double *A = b.center + 3 * p, *B = b.center + 3 * q, *C = b.center + 3 * r, *D = b.center + 3 * s;
    int va[3], vb[3], vc[3], vd[3];
    label_exps(b.cart[p], va);
    label_exps(b.cart[q], vb);
    label_exps(b.cart[r], vc);
    label_exps(b.cart[s], vd);
    int T[3], Tab[3], Tcd[3];
    for (int x = 0; x < 3; ++x) {
        Tab[x] = va[x] + vb[x];
        Tcd[x] = vc[x] + vd[x];
        T[x] = Tab[x] + Tcd[x];
    }
    const int L = T[0] + T[1] + T[2];
    double ab2 = 0.0, cd2 = 0.0;
    for (int x = 0; x < 3; ++x) {
        ab2 += (A[x] - B[x]) * (A[x] - B[x]);
        cd2 += (C[x] - D[x]) * (C[x] - D[x]);
    }
    double acc = 0.0;
    for (int i = 0; i < b.nprim[p]; ++i)
        for (int j = 0; j < b.nprim[q]; ++j) {
            const double ea = b.exps[b.poff[p] + i], eb = b.exps[b.poff[q] + j];
            const double pe = ea + eb;
            const double wab = b.w[b.poff[p] + i] * b.w[b.poff[q] + j] * exp(-ea * eb / pe * ab2);
            double P[3], Eab[3][5];
            for (int x = 0; x < 3; ++x) {
                P[x] = (ea * A[x] + eb * B[x]) / pe;
                hermite_e(va[x], vb[x], P[x] - A[x], P[x] - B[x], pe, Eab[x]);
            }
            for (int k = 0; k < b.nprim[r]; ++k)
                for (int l = 0; l < b.nprim[s]; ++l) {
                    const double ec = b.exps[b.poff[r] + k], ed = b.exps[b.poff[s] + l];
                    const double qe = ec + ed;
                    double Q[3], Ecd[3][5], PQ[3], pq2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        Q[x] = (ec * C[x] + ed * D[x]) / qe;
                        hermite_e(vc[x], vd[x], Q[x] - C[x], Q[x] - D[x], qe, Ecd[x]);
                        PQ[x] = P[x] - Q[x];
                        pq2 += PQ[x] * PQ[x];
                    }
                    const double alpha = pe * qe / (pe + qe);
                    double F[9], R[48];
                    boys_upto8(L, alpha * pq2, F);
                    hermite_r(T[0], T[1], T[2], alpha, PQ[0], PQ[1], PQ[2], F, R);
                    const int NY = T[1] + 1, NZ = T[2] + 1;
                    double sum = 0.0;
                    for (int t = 0; t <= Tab[0]; ++t)
                        for (int u = 0; u <= Tab[1]; ++u)
                            for (int v = 0; v <= Tab[2]; ++v) {
                                const double eab = Eab[0][t] * Eab[1][u] * Eab[2][v];
                                double inner = 0.0;
                                for (int tau = 0; tau <= Tcd[0]; ++tau)
                                    for (int nu = 0; nu <= Tcd[1]; ++nu)
                                        for (int phi = 0; phi <= Tcd[2]; ++phi) {
                                            const double ecd = Ecd[0][tau] * Ecd[1][nu] * Ecd[2][phi];
                                            const double rv = R[((t + tau) * NY + (u + nu)) * NZ + (v + phi)];
                                            inner += ((tau + nu + phi) & 1) ? -ecd * rv : ecd * rv;
                                        }
                                sum += eab * inner;
                            }
                    const double K = kTwoPi52 / (pe * qe * sqrt(pe + qe)) * wab * b.w[b.poff[r] + k] *
                                     b.w[b.poff[s] + l] * exp(-ec * ed / qe * cd2);
                    acc += K * sum;
                }
        }
    return acc;
}

// contracted (pq|rs) for a basis with Cartesian labels, FP64
__device__ inline double contracted_l(const DevBasis &b, int p, int q, int r, int s) {
    if (b.cart[p] >= 4 || b.cart[q] >= 4 || b.cart[r] >= 4 || b.cart[s] >= 4) return contracted_md(b, p, q, r, s);
    const double *A = b.center + 3 * p, *B = b.center + 3 * q, *C = b.center + 3 * r, *D = b.center + 3 * s;
    const int la = b.cart[p], lb = b.cart[q], lc = b.cart[r], ld = b.cart[s];
    const int L = (la > 0) + (lb > 0) + (lc > 0) + (ld > 0);
    double AB[3], CD[3], ab2 = 0.0, cd2 = 0.0;
    for (int x = 0; x < 3; ++x) {
        AB[x] = A[x] - B[x];
        CD[x] = C[x] - D[x];
        ab2 += AB[x] * AB[x];
        cd2 += CD[x] * CD[x];
    }
    double acc = 0.0;
    for (int i = 0; i < b.nprim[p]; ++i)
        for (int j = 0; j < b.nprim[q]; ++j) {
            const double ea = b.exps[b.poff[p] + i], eb = b.exps[b.poff[q] + j];
            const double pe = ea + eb;
            const double wab = b.w[b.poff[p] + i] * b.w[b.poff[q] + j] * exp(-ea * eb / pe * ab2);
            double P[3];
            for (int x = 0; x < 3; ++x) P[x] = (ea * A[x] + eb * B[x]) / pe;
            for (int k = 0; k < b.nprim[r]; ++k)
                for (int l = 0; l < b.nprim[s]; ++l) {
                    const double ec = b.exps[b.poff[r] + k], ed = b.exps[b.poff[s] + l];
                    const double qe = ec + ed;
                    OS o;
                    double pq2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        const double Qx = (ec * C[x] + ed * D[x]) / qe;
                        const double Wx = (pe * P[x] + qe * Qx) / (pe + qe);
                        o.PA[x] = P[x] - A[x];
                        o.WP[x] = Wx - P[x];
                        o.QC[x] = Qx - C[x];
                        o.WQ[x] = Wx - Qx;
                        o.AB[x] = AB[x];
                        o.CD[x] = CD[x];
                        pq2 += (P[x] - Qx) * (P[x] - Qx);
                    }
                    o.p = pe; o.q = qe; o.rho = pe * qe / (pe + qe);
                    o.K = kTwoPi52 / (pe * qe * sqrt(pe + qe)) * wab * b.w[b.poff[r] + k] * b.w[b.poff[s] + l] *
                          exp(-ec * ed / qe * cd2);
                    if (L == 0) {
                        acc += o.K * boys0_d(o.rho * pq2);
                    } else {
                        boys_upto4(o.rho * pq2, o.F);
                        acc += prim_l(o, la, lb, lc, ld);
                    }
                }
        }
    return acc;
}

}  // namespace angular
}  // namespace esmf
