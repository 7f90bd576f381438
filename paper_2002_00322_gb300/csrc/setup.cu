// Screening set-up kernels run once per basis (Sec. II.C: the screening
// data are formed "at the beginning of an ESMF optimization"):
//   normalisation of the contracted s functions, the Schwarz table
//   Q_pq = sqrt((pq|pq)) in FP64, per-brick kept-element counts, and the
//   evaluation of every kept integral into the packed brick store.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "esmf_internal.cuh"
#include "integrals.cuh"

namespace esmf {

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                    \
            return ESMF_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

static inline int grid_for(int64_t work, int per_block, int cap = 152 * 32) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------- normalise
// <g_k|g_l> for normalised primitives on one center is
// (2 sqrt(a_k a_l)/(a_k + a_l))^{3/2}; phi = c sum_k d_k g_k, <phi|phi> = 1;
// w_k = c d_k (2 a_k / pi)^{3/4} multiplies the raw exp(-a_k r^2).
__global__ void k_normalize(int n, const int *nprim, const int *poff, const double *exps,
                            const double *coefs, double *w) {
    int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= n) return;
    const int o = poff[mu], np_ = nprim[mu];
    double s = 0.0;
    for (int k = 0; k < np_; ++k)
        for (int l = 0; l < np_; ++l) {
            const double ak = exps[o + k], al = exps[o + l];
            const double r = 2.0 * sqrt(ak * al) / (ak + al);
            s += coefs[o + k] * coefs[o + l] * r * sqrt(r);
        }
    const double c = rsqrt(s);
    for (int k = 0; k < np_; ++k) {
        const double t = 2.0 * exps[o + k] / 3.14159265358979323846;
        w[o + k] = c * coefs[o + k] * sqrt(t * sqrt(t));   // t^{3/4}
    }
}

int launch_normalize(const DevBasis &b, const double *coefs, double *w, cudaStream_t s) {
    k_normalize<<<grid_for(b.n, 128), 128, 0, s>>>(b.n, b.nprim, b.poff, b.exps, coefs, w);
    CK(cudaGetLastError());
    return ESMF_OK;
}

// ---------------------------------------------------------------- Schwarz
// One thread per pair p >= q: (pq|pq) over all primitive quartets in FP64,
// Q_pq = Q_qp = sqrt((pq|pq)).  Padded functions get Q = 0.
__global__ void k_schwarz(DevBasis b, double *Q) {
    const int64_t npair = (int64_t)b.np * (b.np + 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npair;
         t += (int64_t)gridDim.x * blockDim.x) {
        int p = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((int64_t)p * (p + 1) / 2 > t) --p;
        while ((int64_t)(p + 1) * (p + 2) / 2 <= t) ++p;
        const int q = (int)(t - (int64_t)p * (p + 1) / 2);
        double v = 0.0;
        if (p < b.n && q < b.n) {
            double pe[MAXPP], px[MAXPP], py[MAXPP], pz[MAXPP], kw[MAXPP];
            const double ax = b.center[3 * p], ay = b.center[3 * p + 1], az = b.center[3 * p + 2];
            const double bx = b.center[3 * q], by = b.center[3 * q + 1], bz = b.center[3 * q + 2];
            const double ab2 = (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
            int c = 0;
            for (int i = 0; i < b.nprim[p]; ++i)
                for (int j = 0; j < b.nprim[q]; ++j) {
                    const double a = b.exps[b.poff[p] + i], bb = b.exps[b.poff[q] + j];
                    const double e = a + bb;
                    pe[c] = e;
                    px[c] = (a * ax + bb * bx) / e - ax;
                    py[c] = (a * ay + bb * by) / e - ay;
                    pz[c] = (a * az + bb * bz) / e - az;
                    kw[c] = b.w[b.poff[p] + i] * b.w[b.poff[q] + j] * exp(-a * bb / e * ab2);
                    ++c;
                }
            for (int i = 0; i < c; ++i) {
                double part = 0.0;
                for (int k = 0; k < c; ++k) {
                    const double dx = px[i] - px[k], dy = py[i] - py[k], dz = pz[i] - pz[k];
                    const double pq = pe[i] * pe[k], sum = pe[i] + pe[k];
                    part += kw[k] * kTwoPi52 * rsqrt(sum) / pq *
                            boys0_d(pq / sum * (dx * dx + dy * dy + dz * dz));
                }
                v += kw[i] * part;
            }
        }
        const double qv = sqrt(v > 0.0 ? v : 0.0);
        Q[(int64_t)p * b.np + q] = qv;
        Q[(int64_t)q * b.np + p] = qv;
    }
}

// ---------------------------------------------------------------- pair rule
// Contracted (pq|rs) in FP64 from the basis arrays (all primitive products).
__device__ double eri_fp64(const DevBasis &b, int p, int q, int r, int s) {
    double v = 0.0;
    const double ax = b.center[3 * p], ay = b.center[3 * p + 1], az = b.center[3 * p + 2];
    const double bx = b.center[3 * q], by = b.center[3 * q + 1], bz = b.center[3 * q + 2];
    const double cx = b.center[3 * r], cy = b.center[3 * r + 1], cz = b.center[3 * r + 2];
    const double dx = b.center[3 * s], dy = b.center[3 * s + 1], dz = b.center[3 * s + 2];
    const double ab2 = (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
    const double cd2 = (cx - dx) * (cx - dx) + (cy - dy) * (cy - dy) + (cz - dz) * (cz - dz);
    for (int i = 0; i < b.nprim[p]; ++i)
        for (int j = 0; j < b.nprim[q]; ++j) {
            const double a1 = b.exps[b.poff[p] + i], a2 = b.exps[b.poff[q] + j], e1 = a1 + a2;
            const double k1 = b.w[b.poff[p] + i] * b.w[b.poff[q] + j] * exp(-a1 * a2 / e1 * ab2);
            const double Px = (a1 * ax + a2 * bx) / e1, Py = (a1 * ay + a2 * by) / e1, Pz = (a1 * az + a2 * bz) / e1;
            for (int k = 0; k < b.nprim[r]; ++k)
                for (int l = 0; l < b.nprim[s]; ++l) {
                    const double a3 = b.exps[b.poff[r] + k], a4 = b.exps[b.poff[s] + l], e2 = a3 + a4;
                    const double k2 = b.w[b.poff[r] + k] * b.w[b.poff[s] + l] * exp(-a3 * a4 / e2 * cd2);
                    const double Qx = (a3 * cx + a4 * dx) / e2, Qy = (a3 * cy + a4 * dy) / e2,
                                 Qz = (a3 * cz + a4 * dz) / e2;
                    const double R2 = (Px - Qx) * (Px - Qx) + (Py - Qy) * (Py - Qy) + (Pz - Qz) * (Pz - Qz);
                    v += k1 * k2 * kTwoPi52 / (e1 * e2 * sqrt(e1 + e2)) * boys0_d(e1 * e2 / (e1 + e2) * R2);
                }
        }
    return v;
}

// The pair rule of Sec. II.C: pair (p, q) survives iff some (r, s) has
// |(pq|rs)| > thr.  One warp per pair.  (pq|pq) = Q_pq^2 decides at once;
// otherwise the candidates (r, s) are visited in descending Q order, 32 at a
// time, and since |(pq|rs)| <= Q_pq Q_rs the search ends at the first
// candidate whose bound is <= thr (no later one can exceed thr) or at the
// first integral above thr.  S[p][q] = S[q][p] = 1 for survivors (S zeroed
// by the caller); FP64 throughout, like the oracle's decision.
__global__ void k_pair_rule(DevBasis b, const double *Q, double thr, const int2 *order, int64_t npairs,
                            double *S) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = wid; t < npairs; t += nw) {
        const int2 pq = order[t];
        const int p = pq.x, q = pq.y;
        const double qpq = Q[(int64_t)p * b.np + q];
        bool keep = qpq * qpq > thr;
        for (int64_t base = 0; !keep && base < npairs; base += 32) {
            const int64_t i = base + lane;
            double v = 0.0;
            bool live = false;
            if (i < npairs) {
                const int2 rs = order[i];
                live = qpq * Q[(int64_t)rs.x * b.np + rs.y] > thr;
                if (live) v = fabs(eri_fp64(b, p, q, rs.x, rs.y));
            }
            if (__any_sync(0xffffffffu, v > thr)) keep = true;
            else if (!__all_sync(0xffffffffu, live)) break;
        }
        if (lane == 0 && keep) {
            S[(int64_t)p * b.np + q] = 1.0;
            S[(int64_t)q * b.np + p] = 1.0;
        }
    }
}

int launch_pair_rule(const DevBasis &b, const double *Q, double thr, const int2 *order, int64_t npairs, double *S,
                     cudaStream_t s) {
    CK(cudaMemsetAsync(S, 0, sizeof(double) * (size_t)b.np * b.np, s));
    if (npairs == 0) return ESMF_OK;
    k_pair_rule<<<grid_for(npairs * 32, 256, 152 * 8), 256, 0, s>>>(b, Q, thr, order, npairs, S);
    CK(cudaGetLastError());
    return ESMF_OK;
}

int launch_schwarz(const DevBasis &b, double *Q, cudaStream_t s) {
    const int64_t npair = (int64_t)b.np * (b.np + 1) / 2;
    k_schwarz<<<grid_for(npair, 128), 128, 0, s>>>(b, Q);
    CK(cudaGetLastError());
    return ESMF_OK;
}

// ---------------------------------------------------------------- masks
// Element (p q | r s) of a brick is kept iff all four functions are real and
// Q_pq * Q_rs >= tol (the same FP64 product the oracle forms).
__device__ __forceinline__ bool elem_kept(const double *qb, const double *qk, int e, double tol,
                                          int n, int P, int Qb, int R, int S) {
    const int p = e >> 9, q = (e >> 6) & 7, r = (e >> 3) & 7, s = e & 7;
    if (P * 8 + p >= n || Qb * 8 + q >= n || R * 8 + r >= n || S * 8 + s >= n) return false;
    return qb[p * 8 + q] * qk[r * 8 + s] >= tol;
}

// An element counts once per unique quartet: among the members of its
// 8-fold permutation orbit that lie inside this brick, the one with the
// smallest local index is the representative.
__device__ __forceinline__ bool elem_canonical(int e, int P, int Qb, int R, int S) {
    const int g[4] = {P * 8 + (e >> 9), Qb * 8 + ((e >> 6) & 7), R * 8 + ((e >> 3) & 7), S * 8 + (e & 7)};
    const int perm[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                            {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};
    const int blk[4] = {P, Qb, R, S};
    for (int t = 1; t < 8; ++t) {
        int a[4];
        bool inside = true;
        for (int x = 0; x < 4; ++x) {
            a[x] = g[perm[t][x]];
            inside &= (a[x] >> 3) == blk[x];
        }
        if (!inside) continue;
        const int le = ((a[0] & 7) << 9) | ((a[1] & 7) << 6) | ((a[2] & 7) << 3) | (a[3] & 7);
        if (le < e) return false;
    }
    return true;
}

__global__ void k_brick_count(DevBasis b, const double *Q, double tol, const BrickDesc *bricks,
                              int64_t nbricks, int32_t *counts, int32_t *canon) {
    __shared__ double qb[64], qk[64];
    __shared__ int red[2][4];
    for (int64_t bi = blockIdx.x; bi < nbricks; bi += gridDim.x) {
        const BrickDesc d = bricks[bi];
        __syncthreads();
        if (threadIdx.x < 64) {
            const int t = threadIdx.x;
            qb[t] = Q[(int64_t)(d.P * 8 + (t >> 3)) * b.np + d.Q * 8 + (t & 7)];
            qk[t] = Q[(int64_t)(d.R * 8 + (t >> 3)) * b.np + d.S * 8 + (t & 7)];
        }
        __syncthreads();
        int c = 0, cc = 0;
        for (int e = threadIdx.x; e < BRICK; e += blockDim.x) {
            if (elem_kept(qb, qk, e, tol, b.n, d.P, d.Q, d.R, d.S)) {
                ++c;
                cc += elem_canonical(e, d.P, d.Q, d.R, d.S);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            cc += __shfl_xor_sync(0xffffffffu, cc, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = c;
            red[1][threadIdx.x >> 5] = cc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            counts[bi] = red[0][0] + red[0][1] + red[0][2] + red[0][3];
            canon[bi] = red[1][0] + red[1][1] + red[1][2] + red[1][3];
        }
    }
}

int launch_brick_count(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                       int64_t nbricks, int32_t *counts, cudaStream_t s) {
    // counts holds 2*nbricks: kept elements, then canonical kept elements
    k_brick_count<<<grid_for(nbricks, 1, 152 * 16), 128, 0, s>>>(b, Q, tol, bricks, nbricks, counts,
                                                                  counts + nbricks);
    CK(cudaGetLastError());
    return ESMF_OK;
}

// ---------------------------------------------------------------- generation
// 256 threads; thread t owns the 16 consecutive local indices [16t, 16t+16).
// A block-wide exclusive scan of the kept counts gives packed positions.
__device__ __forceinline__ int block_excl_scan256(int v, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = (lane < 8) ? wsum[lane] : 0;
        for (int o = 1; o < 8; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) wsum[8 + lane] = w;   // inclusive warp prefix
    }
    __syncthreads();
    const int before = (wid > 0) ? wsum[8 + wid - 1] : 0;
    total = wsum[15];
    return before + x - v;
}

template <typename T>
struct GenSmem {
    PairSmem<T, 128, MAXPP> pairs;
    double qb[64], qk[64];
    int wsum[16];
    unsigned short klist[BRICK];   // local indices of the kept elements, ascending
};

// precision: 0 FP64 store (T = double), 1 FP32 store, 2 FP16 hi+lo, 3 BF16 hi+lo,
// 4 double-FP32 hi+lo floats (T = double)
template <typename T, int PREC>
__global__ void __launch_bounds__(256) k_brick_generate(DevBasis b, const double *Q, double tol,
                                                        const BrickDesc *bricks, int64_t nbricks,
                                                        const int64_t *offsets, void *store,
                                                        float vscale, const void *ptab, const int *pslot) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GenSmem<T> &sm = *reinterpret_cast<GenSmem<T> *>(smraw);
    for (int64_t bi = blockIdx.x; bi < nbricks; bi += gridDim.x) {
        const BrickDesc d = bricks[bi];
        __syncthreads();
        // local origin: center of the first function of block P (keeps FP32
        // coordinate differences small)
        const int o = d.P * 8;
        const double ox = b.center[3 * o], oy = b.center[3 * o + 1], oz = b.center[3 * o + 2];
        if (ptab) {
            // primitive pairs of (P,Q) and (R,S) from the create-time table (formed
            // once per block pair, not once per brick)
            const PairTable<T, MAXPP> *tab = reinterpret_cast<const PairTable<T, MAXPP> *>(ptab);
            load_pairs<T, MAXPP>(sm.pairs, tab[pslot[d.P * b.nb + d.Q]], tab[pslot[d.R * b.nb + d.S]], ox, oy, oz);
        } else {
            fill_pairs<T, MAXPP>(sm.pairs, 0, d.P, d.Q, b.center, b.nprim, b.poff, b.exps, b.w, b.np,
                                 ox, oy, oz);
            fill_pairs<T, MAXPP>(sm.pairs, 64, d.R, d.S, b.center, b.nprim, b.poff, b.exps, b.w, b.np,
                                 ox, oy, oz);
        }
        if (threadIdx.x < 64) {
            const int t = threadIdx.x;
            sm.qb[t] = Q[(int64_t)(d.P * 8 + (t >> 3)) * b.np + d.Q * 8 + (t & 7)];
            sm.qk[t] = Q[(int64_t)(d.R * 8 + (t >> 3)) * b.np + d.S * 8 + (t & 7)];
        }
        __syncthreads();
        // Thread t tests the 16 local indices [16t, 16t+16); the kept ones are
        // listed in ascending order and then evaluated round-robin, so a warp
        // takes 32 consecutive kept elements (mostly one bra pair: broadcast
        // bra reads, distinct ket pairs) and the threads share the work evenly.
        const int e0 = threadIdx.x * 16;
        unsigned mask = 0;
        for (int j = 0; j < 16; ++j)
            if (elem_kept(sm.qb, sm.qk, e0 + j, tol, b.n, d.P, d.Q, d.R, d.S)) mask |= 1u << j;
        int total;
        int pos = block_excl_scan256(__popc(mask), sm.wsum, total);
        for (int j = 0; j < 16; ++j)
            if (mask & (1u << j)) sm.klist[pos++] = (unsigned short)(e0 + j);
        // record: 512-byte keep mask, then the kept values (FP64 / FP32, or
        // (hi | lo << 16) words of the value times the store's power-of-two
        // scale); offsets count store elements of sizeof(element) bytes
        constexpr int EB = (PREC == 0 || PREC == 4) ? 8 : 4;
        const int64_t base = offsets[bi];
        unsigned char *mk = reinterpret_cast<unsigned char *>(store) + base * EB;
        mk[2 * threadIdx.x] = (unsigned char)(mask & 0xffu);
        mk[2 * threadIdx.x + 1] = (unsigned char)(mask >> 8);
        const int64_t vbase = base + MASK_BYTES / EB;
        uint32_t *rec = reinterpret_cast<uint32_t *>(store) + (PREC >= 2 ? vbase : 0);
        __syncthreads();
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int e = sm.klist[i];
            const T v = contracted_eri<T, 128, MAXPP>(sm.pairs, e >> 6, sm.pairs, 64 + (e & 63));
            if (PREC == 0 || PREC == 1) {
                reinterpret_cast<T *>(store)[vbase + i] = v;
            } else if (PREC == 4) {
                // double-FP32 store: the FP64 value as hi + lo floats
                const float hi = __double2float_rn((double)v);
                reinterpret_cast<float2 *>(store)[vbase + i] = make_float2(hi, __double2float_rn((double)v - (double)hi));
            } else if constexpr (sizeof(T) == 4) {
                // FP32-evaluated value: the power-of-two scale is exact in FP32 and
                // the residual of the 16-bit rounding too (Sterbenz), so the FP32
                // split equals the FP64 one and keeps off GB300's narrow FP64 pipe
                const float xs = v * vscale;
                uint16_t hb, lb;
                if (PREC == 2) {
                    const __half h = __float2half_rn(xs);
                    hb = __half_as_ushort(h);
                    lb = __half_as_ushort(__float2half_rn(xs - __half2float(h)));
                } else {
                    const __nv_bfloat16 h = __float2bfloat16_rn(xs);
                    hb = __bfloat16_as_ushort(h);
                    lb = __bfloat16_as_ushort(__float2bfloat16_rn(xs - __bfloat162float(h)));
                }
                rec[i] = (uint32_t)hb | ((uint32_t)lb << 16);
            } else {
                const double xs = (double)v * (double)vscale;
                uint16_t hb, lb;
                if (PREC == 2) {
                    __half h = __double2half(xs);
                    __half l = __double2half(xs - (double)__half2float(h));
                    hb = __half_as_ushort(h);
                    lb = __half_as_ushort(l);
                } else {
                    __nv_bfloat16 h = __double2bfloat16(xs);
                    __nv_bfloat16 l = __double2bfloat16(xs - (double)__bfloat162float(h));
                    hb = __bfloat16_as_ushort(h);
                    lb = __bfloat16_as_ushort(l);
                }
                rec[i] = (uint32_t)hb | ((uint32_t)lb << 16);
            }
        }
    }
}

// ---------------------------------------------------------------- pair table
// Entry e holds the primitive pairs of function-block pair (blocks[2e],
// blocks[2e+1]) for integral-direct builds; one 64-thread block per entry.
template <typename T>
__global__ void __launch_bounds__(64) k_pair_table(DevBasis b, const int *blocks, int nentries,
                                                   PairTable<T, MAXPP> *tab) {
    const int e = blockIdx.x;
    if (e >= nentries) return;
    PairTable<T, MAXPP> &te = tab[e];
    const int t = threadIdx.x;
    const int p = blocks[2 * e] * 8 + (t >> 3), q = blocks[2 * e + 1] * 8 + (t & 7);
    int cnt = 0;
    if (p < b.np && q < b.np)
        cnt = pair_prims<T, MAXPP>(p, q, b.center, b.nprim, b.poff, b.exps, b.w,
                                   [&](int c, double pe, double Px, double Py, double Pz, double kw) {
                                       te.pe[c][t] = (T)pe;
                                       te.px[c][t] = Px;
                                       te.py[c][t] = Py;
                                       te.pz[c][t] = Pz;
                                       te.kw[c][t] = (T)kw;
                                   });
    te.npp[t] = cnt;
}

// FP64 and double-FP32 stores evaluate in FP64 (double tables), the others in FP32
static bool table_fp64(int precision) { return precision == ESMF_PREC_FP64 || precision == ESMF_PREC_F32X2; }

size_t pair_table_entry_bytes(int precision) {
    return table_fp64(precision) ? sizeof(PairTable<double, MAXPP>) : sizeof(PairTable<float, MAXPP>);
}

int launch_pair_table(const DevBasis &b, const int *blocks, int nentries, int precision, void *tab,
                      cudaStream_t s) {
    if (nentries < 1) return ESMF_OK;
    if (table_fp64(precision))
        k_pair_table<double><<<nentries, 64, 0, s>>>(b, blocks, nentries, (PairTable<double, MAXPP> *)tab);
    else
        k_pair_table<float><<<nentries, 64, 0, s>>>(b, blocks, nentries, (PairTable<float, MAXPP> *)tab);
    CK(cudaGetLastError());
    return ESMF_OK;
}

template <typename T, int PREC>
static int gen_launch(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                      int64_t nbricks, const int64_t *offsets, void *store, float vscale,
                      const void *ptab, const int *pslot, cudaStream_t s) {
    const size_t smem = sizeof(GenSmem<T>);
    CK(cudaFuncSetAttribute(k_brick_generate<T, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    k_brick_generate<T, PREC><<<grid_for(nbricks, 1, 152 * 4), 256, smem, s>>>(
        b, Q, tol, bricks, nbricks, offsets, store, vscale, ptab, pslot);
    CK(cudaGetLastError());
    return ESMF_OK;
}

int launch_brick_generate(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                          int64_t nbricks, const int64_t *offsets, int precision, void *store,
                          float vscale, cudaStream_t s, const void *ptab, const int *pslot) {
    switch (precision) {
        case ESMF_PREC_FP64: return gen_launch<double, 0>(b, Q, tol, bricks, nbricks, offsets, store, vscale, ptab, pslot, s);
        case ESMF_PREC_F32X2: return gen_launch<double, 4>(b, Q, tol, bricks, nbricks, offsets, store, vscale, ptab, pslot, s);
        case ESMF_PREC_FP32: return gen_launch<float, 1>(b, Q, tol, bricks, nbricks, offsets, store, vscale, ptab, pslot, s);
        case ESMF_PREC_FP16X2: return gen_launch<float, 2>(b, Q, tol, bricks, nbricks, offsets, store, vscale, ptab, pslot, s);
        case ESMF_PREC_BF16X2: return gen_launch<float, 3>(b, Q, tol, bricks, nbricks, offsets, store, vscale, ptab, pslot, s);
    }
    set_error("unknown precision %d", precision);
    return ESMF_ERR_INVALID_ARG;
}

}  // namespace esmf
