// Device integrals over contracted Cartesian p functions (angular momentum
// at most one per function, at most two per pair), in FP64: the Obara-Saika
// vertical recurrence (Obara & Saika, J. Chem. Phys. 84, 3963 (1986)) written
// out for orders up to two per side, and the horizontal recurrence of
// Head-Gordon & Pople (J. Chem. Phys. 89, 5777 (1988)).
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

// contracted (pq|rs) for a basis with Cartesian labels, FP64
__device__ inline double contracted_l(const DevBasis &b, int p, int q, int r, int s) {
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
