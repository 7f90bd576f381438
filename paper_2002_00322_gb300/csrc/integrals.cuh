// Device-side s-type integral arithmetic.
//
// Raw Gaussian primitives exp(-a |r - A|^2) with normalised weights w
// (contracted function = sum_k w_k exp(-a_k |r - A|^2)); the two-electron
// integral over four raw primitives is the textbook closed form (Boys 1950;
// Szabo & Ostlund App. A, which the paper cites for its integral theory):
//   p = a + b, P = (a A + b B)/p, q = c + d, Q = (c C + d D)/q,
//   [ab|cd] = 2 pi^{5/2} / (p q sqrt(p + q)) * exp(-ab/p |AB|^2)
//             * exp(-cd/q |CD|^2) * F0(pq/(p+q) |PQ|^2),
// F0(T) = int_0^1 exp(-T u^2) du = (1/2) sqrt(pi/T) erf(sqrt(T)).
// The pair factors (p, P, w_a w_b exp(-ab/p |AB|^2)) are formed once per
// primitive pair; the quartet loop only needs T, one erf and a reciprocal
// square root per primitive quartet.
#pragma once

#include <cuda_runtime.h>

namespace esmf {

constexpr double kTwoPi52 = 34.986836655249725;    // 2 pi^{5/2}
constexpr double kHalfSqrtPi = 0.88622692545275801; // sqrt(pi)/2

// F0 in double: Taylor series sum_k (-T)^k/(k!(2k+1)) below 1e-6 (four terms,
// truncation < 1e-25), erf form above; for T > 40 erf(sqrt T) = 1 to double.
__device__ __forceinline__ double boys0_d(double T) {
    if (T < 1e-6) return 1.0 - T * (1.0 / 3.0) + T * T * 0.1 - T * T * T * (1.0 / 42.0);
    double x = sqrt(T);
    if (T > 40.0) return kHalfSqrtPi / x;
    return kHalfSqrtPi * erf(x) / x;
}

// F0 for the FP32 paths: near the small-T limit (below 1e-3; truncation
// < 1e-14) the series is summed in FP64 and rounded once, so F0 there is
// correctly rounded to FP32; the erf form above; for T > 16 erff(sqrt T)
// rounds to 1.  Small T occurs only for nearly concentric primitive pairs, so
// the FP64 branch is rare.
__device__ __forceinline__ float boys0_f(float T) {
    if (T < 1e-3f) {
        const double t = (double)T;
        return (float)(1.0 - t * (1.0 / 3.0) + t * t * 0.1 - t * t * t * (1.0 / 42.0));
    }
    float r = rsqrtf(T);
    if (T > 16.0f) return (float)kHalfSqrtPi * r;
    return (float)kHalfSqrtPi * erff(T * r) * r;
}

template <typename T> struct Boys;
template <> struct Boys<double> {
    static __device__ __forceinline__ double f0(double t) { return boys0_d(t); }
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
};
template <> struct Boys<float> {
    static __device__ __forceinline__ float f0(float t) { return boys0_f(t); }
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
};

// Primitive-pair data of one function pair, structure of arrays in shared
// memory: exponent sum p, product center P (relative to a local origin),
// and weight K/p with K = w_a w_b exp(-ab/p |AB|^2).
// Indexed [primitive pair][function pair], so that the lanes of a warp reading
// primitive pair k of consecutive function pairs hit consecutive banks.
template <typename T, int NPAIR, int MAXPP_>
struct PairSmem {
    T pe[MAXPP_][NPAIR];
    T px[MAXPP_][NPAIR];
    T py[MAXPP_][NPAIR];
    T pz[MAXPP_][NPAIR];
    T kw[MAXPP_][NPAIR];
    int npp[NPAIR];
};

// contracted (bra pair ib | ket pair ik) from shared pair data.  Per primitive
// quartet one reciprocal square root r = (p+q)^{-1/2} gives both
// rho = p q r^2 and the prefactor 2 pi^{5/2} r / (p q) (the 1/p, 1/q factors
// are folded into the stored pair weights), so no division is needed.
template <typename T, int NPAIR, int MAXPP_>
__device__ __forceinline__ T contracted_eri(const PairSmem<T, NPAIR, MAXPP_> &bra, int ib,
                                            const PairSmem<T, NPAIR, MAXPP_> &ket, int ik) {
    T acc = T(0);
    const int nb = bra.npp[ib], nk = ket.npp[ik];
    for (int i = 0; i < nb; ++i) {
        const T p = bra.pe[i][ib];
        const T Px = bra.px[i][ib], Py = bra.py[i][ib], Pz = bra.pz[i][ib];
        const T kb = bra.kw[i][ib] * T(kTwoPi52);
        T part = T(0);
        for (int k = 0; k < nk; ++k) {
            const T q = ket.pe[k][ik];
            const T dx = Px - ket.px[k][ik], dy = Py - ket.py[k][ik], dz = Pz - ket.pz[k][ik];
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T r = Boys<T>::rsq(p + q);
            const T rho = p * q * r * r;
            part += ket.kw[k][ik] * r * Boys<T>::f0(rho * r2);
        }
        acc += kb * part;
    }
    return acc;
}

// Primitive pairs of the function pair (p, q), leaving out those too small
// to matter: calls out(c, p_ab, Px, Py, Pz, K_ab / p_ab) for c = 0, 1, ...
// with the absolute product center in FP64, and returns the count.
// Primitive-pair screening: a pair whose weight K/p times p^(-1/2) (its
// contribution to any integral, up to the ket factors) is below eps of the
// largest pair of this function pair is left out; the relative change of an
// integral stays below about 1e4 eps (the ratio of Boys-function and
// prefactor extremes), under the precision of T (FP32: 1e-12; FP64 drops
// only underflowing pairs).  Shared by the per-brick fill below and by the
// pair table of integral-direct handles, so both give the same integrals.
template <typename T, int MAXPP_, typename Out>
__device__ __forceinline__ int pair_prims(int p, int q, const double *center, const int *nprim, const int *poff,
                                          const double *exps, const double *w, Out &&out) {
    const int np_ = nprim[p], nq_ = nprim[q];
    const double ax = center[3 * p], ay = center[3 * p + 1], az = center[3 * p + 2];
    const double bx = center[3 * q], by = center[3 * q + 1], bz = center[3 * q + 2];
    const double ab2 = (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
    double kws[MAXPP_];
    float size[MAXPP_], smax = 0.0f;
    for (int i = 0; i < np_; ++i)
        for (int j = 0; j < nq_; ++j) {
            const int k = i * nq_ + j;
            const double a = exps[poff[p] + i], b = exps[poff[q] + j];
            const double pe = a + b;
            kws[k] = w[poff[p] + i] * w[poff[q] + j] * exp(-a * b / pe * ab2) / pe;
            size[k] = fabsf((float)kws[k]) * rsqrtf((float)pe);
            smax = fmaxf(smax, size[k]);
        }
    const float eps = sizeof(T) == 4 ? 1e-12f : 1e-30f;
    int cnt = 0;
    for (int i = 0; i < np_; ++i)
        for (int j = 0; j < nq_; ++j) {
            const int k = i * nq_ + j;
            if (!(size[k] >= eps * smax)) continue;
            const double a = exps[poff[p] + i], b = exps[poff[q] + j];
            const double pe = a + b;
            const double Px = (a * ax + b * bx) / pe, Py = (a * ay + b * by) / pe, Pz = (a * az + b * bz) / pe;
            out(cnt, pe, Px, Py, Pz, kws[k]);
            ++cnt;
        }
    return cnt;
}

// Fill pair data for the 64 ordered pairs (p, q) of function blocks (PB, QB)
// with local origin (ox, oy, oz).  Called by all threads of a block.
template <typename T, int MAXPP_>
__device__ __forceinline__ void fill_pairs(PairSmem<T, 128, MAXPP_> &ps, int base, int PB, int QB,
                                           const double *center, const int *nprim, const int *poff,
                                           const double *exps, const double *w, int np,
                                           double ox, double oy, double oz) {
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        const int p = PB * 8 + (t >> 3), q = QB * 8 + (t & 7);
        const int slot = base + t;
        int cnt = 0;
        if (p < np && q < np)
            cnt = pair_prims<T, MAXPP_>(p, q, center, nprim, poff, exps, w,
                                        [&](int c, double pe, double Px, double Py, double Pz, double kw) {
                                            ps.pe[c][slot] = (T)pe;
                                            ps.px[c][slot] = (T)(Px - ox);
                                            ps.py[c][slot] = (T)(Py - oy);
                                            ps.pz[c][slot] = (T)(Pz - oz);
                                            ps.kw[c][slot] = (T)kw;
                                        });
        ps.npp[slot] = cnt;
    }
}

// Primitive-pair data of one function-block pair (B1, B2), B1 >= B2, for
// integral-direct builds: the 64 ordered function pairs (B1*8 + t/8,
// B2*8 + t%8), entries c < npp[t] valid, product centers absolute in FP64
// (a brick subtracts its local origin when it loads them).
template <typename T, int MAXPP_>
struct PairTable {
    T pe[MAXPP_][64];
    double px[MAXPP_][64], py[MAXPP_][64], pz[MAXPP_][64];
    T kw[MAXPP_][64];
    int npp[64];
};

// Load the bra (slot base 0) and ket (slot base 64) pair data of a brick from
// two table entries, subtracting the local origin.  Called by all threads.
template <typename T, int MAXPP_>
__device__ __forceinline__ void load_pairs(PairSmem<T, 128, MAXPP_> &ps, const PairTable<T, MAXPP_> &bra,
                                           const PairTable<T, MAXPP_> &ket, double ox, double oy, double oz) {
    for (int t = threadIdx.x; t < 2 * 64 * MAXPP_; t += blockDim.x) {
        const int side = t >= 64 * MAXPP_;
        const int u = side ? t - 64 * MAXPP_ : t;
        const int c = u >> 6, s = u & 63;
        const PairTable<T, MAXPP_> &src = side ? ket : bra;
        const int slot = side * 64 + s;
        const int n = src.npp[s];
        if (c == 0) ps.npp[slot] = n;
        if (c < n) {
            ps.pe[c][slot] = src.pe[c][s];
            ps.px[c][slot] = (T)(src.px[c][s] - ox);
            ps.py[c][slot] = (T)(src.py[c][s] - oy);
            ps.pz[c][slot] = (T)(src.pz[c][s] - oz);
            ps.kw[c][slot] = src.kw[c][s];
        }
    }
}

}  // namespace esmf
