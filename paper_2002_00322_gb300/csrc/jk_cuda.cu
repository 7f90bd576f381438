// Grouped J/K contraction on CUDA cores (Eq. J_and_K, all m densities in one
// pass over the integrals, Sec. II.C).
//
// One CTA processes one brick (P Q | R S) at a time.  The brick's kept
// integrals are expanded into a dense 8^4 tile in shared memory (from the
// packed store, whose records carry their keep masks, or evaluated in place
// in direct mode), and every DISTINCT ordered block tuple of its permutation
// orbit
//   (P Q R S) (Q P R S) (P Q S R) (Q P S R) (R S P Q) (S R P Q) (R S Q P) (S R Q P)
// contributes, for every density k,
//   K[a][c] += sum_{b,d} (ab|cd) D_k[b][d]      (tuple (A,B,C,E), a in A ...)
//   J[a][b] += sum_{c,d} (ab|cd) D_k[c][d]      (tuples with A >= B)
// which is the ordered-tuple form of Eq. J_and_K.  The Coulomb updates of a
// tuple and of its (C,E)-swapped partner share the output block, so they are
// formed once against Dj[C,E] = D[C,E] + [C != E] D[E,C]^T: J[P,Q] from
// Dj[R,S] and J[R,S] from Dj[P,Q] (ten output blocks per brick, not twelve).
// Each output element is a 64-term dot product accumulated in registers (TA)
// and flushed to the FP64 accumulators with one atomic add per brick.  J is
// accumulated only on the lower block triangle and mirrored by the
// finalisation kernel.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <type_traits>

#include "angular.cuh"
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

__constant__ int c_tuple[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                                  {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};
__constant__ int c_stride[4] = {512, 64, 8, 1};
// Output slots of a brick: 0-7 exchange (tuple t), 8 Coulomb J[P,Q] (terms
// over R x S against Dj[R,S]), 9 Coulomb J[R,S] (terms over P x Q against
// Dj[P,Q]).  Per slot the brick index position of the output row index, the
// output column index, and the two summed indices.
__constant__ int c_slot[10][4] = {{0, 2, 1, 3}, {1, 2, 0, 3}, {0, 3, 1, 2}, {1, 3, 0, 2},
                                  {2, 0, 3, 1}, {3, 0, 2, 1}, {2, 1, 3, 0}, {3, 1, 2, 0},
                                  {0, 1, 2, 3}, {2, 3, 0, 1}};

// Double-FP32 arithmetic (ESMF_PREC_F32X2): a value is an unevaluated sum
// hi + lo of two floats (48 significand bits).  Products are formed without
// error in their leading part (p = fl(a.hi b.hi), e = fma(a.hi, b.hi, -p),
// the error-free product of Ogita, Rump and Oishi 2005) plus the two cross
// terms, and added to the running sum with Knuth's TwoSum, the rounding error
// of every addition kept in lo: about 2^-44 relative over a 64-term dot
// product, at the FP32 pipe's rate (12 FP32 operations per product-add).
struct f32x2 {
    float hi, lo;
    f32x2() = default;
    __device__ __forceinline__ f32x2(double v) {
        hi = __double2float_rn(v);
        lo = __double2float_rn(v - (double)hi);
    }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// FP32 -> FP64 widening by the IEEE-754 formats alone (sign, rebiased exponent,
// mantissa shifted into place), on the integer pipe instead of GB300's narrow
// FP64 pipe; exact for every normal float, zero for zero and subnormals
// (below 1.2e-38, far under every contribution here).
__device__ __forceinline__ double widen(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const uint64_t d = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                       ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// a brick's partial sum as the FP64 value its accumulator receives
__device__ __forceinline__ double flush_value(float v) { return widen(v); }
__device__ __forceinline__ double flush_value(double v) { return v; }

__device__ __forceinline__ f32x2 make_f32x2(float hi, float lo) {
    f32x2 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// sums of two density elements (the symmetrised Coulomb tiles), in the
// arithmetic type; the double-FP32 sum keeps TwoSum's error in lo
__device__ __forceinline__ float add_ta(float a, float b) { return a + b; }
__device__ __forceinline__ double add_ta(double a, double b) { return a + b; }
__device__ __forceinline__ f32x2 add_ta(const f32x2 &a, const f32x2 &b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return make_f32x2(s, __fadd_rn(__fadd_rn(a.lo, b.lo), err));
}

__device__ __forceinline__ double flush_value(const f32x2 &v) { return widen(v.hi) + widen(v.lo); }

__device__ __forceinline__ void macc(float &acc, float v, float d) { acc = fmaf(v, d, acc); }
__device__ __forceinline__ void macc(double &acc, double v, double d) { acc = fma(v, d, acc); }
__device__ __forceinline__ void macc(f32x2 &acc, const f32x2 &a, const f32x2 &b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

__device__ __forceinline__ bool kept_e(const double *qb, const double *qk, int e, double tol, int n,
                                       int P, int Q, int R, int S) {
    const int p = e >> 9, q = (e >> 6) & 7, r = (e >> 3) & 7, s = e & 7;
    if (P * 8 + p >= n || Q * 8 + q >= n || R * 8 + r >= n || S * 8 + s >= n) return false;
    return qb[p * 8 + q] * qk[r * 8 + s] >= tol;
}

// Bank-conflict-free placement of the dense 8^4 tile in shared memory: element
// (p q | r s), logical index ((p*8+q)*8+r)*8+s, is stored at
//   logical XOR H(logical >> 5),
// H linear over GF(2) (one 5-bit vector per index bit 5..11, found by search
// and checked exhaustively).  In the contraction the 32 lanes of a warp take
// 4 consecutive values of one index and all 8 of another, for every ordered
// pair of the four indices; with H these 32 elements fall into 32 different
// banks (FP32) or 16 different 8-byte slots twice (FP64).  H is linear and the
// four indices occupy disjoint bit fields, so the placement of a sum of
// per-index offsets is the XOR of their placements.
__device__ __forceinline__ int tile_swizzle(int x) {
    const int hi = x >> 5;
    int h = 0;
    if (hi & 1) h ^= 21;
    if (hi & 2) h ^= 20;
    if (hi & 4) h ^= 11;
    if (hi & 8) h ^= 18;
    if (hi & 16) h ^= 12;
    if (hi & 32) h ^= 27;
    if (hi & 64) h ^= 17;
    return x ^ h;
}

__device__ __forceinline__ int scan256(int v, int *wsum) {
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
        if (lane < 8) wsum[8 + lane] = w;
    }
    __syncthreads();
    return ((wid > 0) ? wsum[8 + wid - 1] : 0) + x - v;
}

// density tiles of one brick: 0-7 D[B][E] of exchange tuple t (its summed
// blocks), 8 Dj[R,S], 9 Dj[P,Q]
template <typename TA, int MC, bool DIRECT>
struct JKSmem {
    TA V[BRICK];
    TA Ds[10][64][MC];
    double qb[64], qk[64];
    int wsum[16];
    int slots[10];            // active output slots of the brick
    int nslots;
    int skip;                 // brick dropped by density-weighted screening
    double wblk;              // largest density weight of the brick's six block pairs
    double dwt[6][64];        // density weights of (R,S) (P,Q) (Q,S) (P,S) (Q,R) (P,R)
    int blk[4];
    int tsw[4][8];            // tile_swizzle(v * stride[dim]) for each index and value
};
template <typename TA, int MC>
struct JKSmemDirect : JKSmem<TA, MC, true> {
    PairSmem<TA, 128, MAXPP> pairs;
};

// CTAs of 256 threads that fit one SM by shared memory (at most 4): the
// register budget is capped so that as many fit by registers too.
template <typename TA, int MC, int SRC>
constexpr int jk_ctas_per_sm() {
    constexpr size_t bytes = SRC == 4 ? sizeof(JKSmemDirect<TA, MC>) : sizeof(JKSmem<TA, MC, false>);
    constexpr int k = (int)((227 * 1024) / (bytes + 1024));
    return k < 1 ? 1 : (k > 4 ? 4 : k);
}

// SRC: 0 fp64 store, 1 fp32 store, 2 fp16 hi+lo, 3 bf16 hi+lo, 4 direct (evaluated in TA),
// 5 fp64 store contracted in double-FP32 (TA = f32x2), 6 direct with p functions
// (Obara-Saika integrals evaluated in FP64, converted to TA)
template <typename TA, int MC, int SRC>
__global__ void __launch_bounds__(256, (jk_ctas_per_sm<TA, MC, SRC>())) k_jk_cuda(JKArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    using SM = typename std::conditional<SRC == 4, JKSmemDirect<TA, MC>, JKSmem<TA, MC, false>>::type;
    SM &sm = *reinterpret_cast<SM *>(smraw);
    const int n = a.b.n, np = a.b.np;
    const int64_t nn = (int64_t)n * n, npnp = (int64_t)np * np;
    if (threadIdx.x < 32) sm.tsw[threadIdx.x >> 3][threadIdx.x & 7] = tile_swizzle((threadIdx.x & 7) * c_stride[threadIdx.x >> 3]);

    for (int64_t bi = blockIdx.x; bi < a.nbricks; bi += gridDim.x) {
        const BrickDesc d = a.bricks[bi];
        __syncthreads();
        if (threadIdx.x == 0) {
            sm.blk[0] = d.P; sm.blk[1] = d.Q; sm.blk[2] = d.R; sm.blk[3] = d.S;
            const int bl[4] = {d.P, d.Q, d.R, d.S};
            int ns = 0, act4 = 0;
            for (int t = 0; t < 8; ++t) {
                int act = 1;
                for (int u = 0; u < t; ++u) {
                    bool same = true;
                    for (int x = 0; x < 4; ++x) same &= bl[c_tuple[t][x]] == bl[c_tuple[u][x]];
                    if (same) { act = 0; break; }
                }
                if (act) sm.slots[ns++] = t;
                if (t == 4) act4 = act;
            }
            // J[P,Q] always; J[R,S] unless (R,S) = (P,Q) (tuple 4 repeats tuple 0)
            sm.slots[ns++] = 8;
            if (act4) sm.slots[ns++] = 9;
            sm.nslots = ns;
        }
        const bool dens = a.dw != nullptr;
        if ((SRC == 4 || SRC == 6 || dens) && threadIdx.x < 64) {
            const int t = threadIdx.x;
            sm.qb[t] = a.Q[(int64_t)(d.P * 8 + (t >> 3)) * np + d.Q * 8 + (t & 7)];
            sm.qk[t] = a.Q[(int64_t)(d.R * 8 + (t >> 3)) * np + d.S * 8 + (t & 7)];
        }
        if (dens) {
            // weights of the six block pairs a quartet's updates multiply by
            const int bx[6] = {d.R, d.P, d.Q, d.P, d.Q, d.P}, by[6] = {d.S, d.Q, d.S, d.S, d.R, d.R};
            for (int t = threadIdx.x; t < 6 * 64; t += blockDim.x) {
                const int j = t >> 6, e = t & 63;
                sm.dwt[j][e] = a.dw[(int64_t)(bx[j] * 8 + (e >> 3)) * np + by[j] * 8 + (e & 7)];
            }
            if (threadIdx.x == 0) {
                double wm = 0.0;
                for (int j = 0; j < 6; ++j) wm = fmax(wm, a.dwb[bx[j] * a.b.nb + by[j]]);
                sm.wblk = wm;
            }
        }
        if constexpr (SRC == 4) {
            const int o = d.P * 8;
            const double ox = a.b.center[3 * o], oy = a.b.center[3 * o + 1], oz = a.b.center[3 * o + 2];
            // primitive pairs of (P,Q) and (R,S) from the handle's table
            const PairTable<TA, MAXPP> *tab = reinterpret_cast<const PairTable<TA, MAXPP> *>(a.ptab);
            load_pairs<TA, MAXPP>(sm.pairs, tab[a.pslot[d.P * a.b.nb + d.Q]], tab[a.pslot[d.R * a.b.nb + d.S]],
                                  ox, oy, oz);
        }
        __syncthreads();
        if (dens) {
            // brick-level bound of density-weighted screening: when the largest
            // Schwarz product times the largest weight is below tol_d, no
            // element of the brick survives
            if (threadIdx.x < 32) {
                double qm = fmax(fmax(sm.qb[threadIdx.x], sm.qb[threadIdx.x + 32]), 0.0);
                double km = fmax(sm.qk[threadIdx.x], sm.qk[threadIdx.x + 32]);
                for (int o = 16; o > 0; o >>= 1) {
                    qm = fmax(qm, __shfl_xor_sync(0xffffffffu, qm, o));
                    km = fmax(km, __shfl_xor_sync(0xffffffffu, km, o));
                }
                if (threadIdx.x == 0) sm.skip = qm * km * sm.wblk < a.tol_d;
            }
            __syncthreads();
            if (sm.skip) continue;
        }
        // ---- dense brick tile
        {
            const int e0 = threadIdx.x * 16;
            unsigned mask = 0, dmask = 0xffffu;
            constexpr int EB = (SRC == 0 || SRC == 5) ? 8 : 4;   // bytes per store element
            if (dens) {
                // element-level rule: Q_pq Q_rs times the largest weight of the
                // quartet's six index pairs must reach tol_d
                dmask = 0;
                for (int j = 0; j < 16; ++j) {
                    const int e = e0 + j;
                    const int p = e >> 9, q = (e >> 6) & 7, r = (e >> 3) & 7, s_ = e & 7;
                    double wt = fmax(fmax(sm.dwt[0][r * 8 + s_], sm.dwt[1][p * 8 + q]),
                                     fmax(sm.dwt[2][q * 8 + s_], sm.dwt[3][p * 8 + s_]));
                    wt = fmax(wt, fmax(sm.dwt[4][q * 8 + r], sm.dwt[5][p * 8 + r]));
                    if (sm.qb[p * 8 + q] * sm.qk[r * 8 + s_] * wt >= a.tol_d) dmask |= 1u << j;
                }
            }
            if constexpr (SRC == 4 || SRC == 6) {
                for (int j = 0; j < 16; ++j)
                    if (kept_e(sm.qb, sm.qk, e0 + j, a.tol, n, d.P, d.Q, d.R, d.S)) mask |= 1u << j;
                mask &= dmask;
            } else {
                // the record's keep mask: bytes 2t and 2t + 1 cover elements 16t .. 16t + 15
                const unsigned char *mk = reinterpret_cast<const unsigned char *>(a.store) + a.offsets[bi] * EB;
                mask = (unsigned)mk[2 * threadIdx.x] | ((unsigned)mk[2 * threadIdx.x + 1] << 8);
            }
            if constexpr (SRC == 4 || SRC == 6) {
                // kept local indices listed in ascending order (in the density
                // tiles' space, unused until the first chunk's barrier), then
                // evaluated round-robin: a warp takes 32 consecutive kept
                // elements, mostly of one bra pair, and the work is shared evenly
                static_assert(sizeof(sm.Ds) >= BRICK * sizeof(unsigned short), "list does not fit");
                unsigned short *klist = reinterpret_cast<unsigned short *>(&sm.Ds[0][0][0]);
                int pos = scan256(__popc(mask), sm.wsum);
                const int total = sm.wsum[15];
                for (int j = 0; j < 16; ++j) {
                    const int e = e0 + j;
                    if (mask & (1u << j)) klist[pos++] = (unsigned short)e;
                    else sm.V[tile_swizzle(e)] = TA(0);
                }
                __syncthreads();
                if constexpr (SRC == 6) {
                    // p functions: the Obara-Saika integral in FP64 from the basis arrays
                    for (int i = threadIdx.x; i < total; i += blockDim.x) {
                        const int e = klist[i];
                        sm.V[tile_swizzle(e)] = (TA)angular::contracted_l(
                            a.b, d.P * 8 + (e >> 9), d.Q * 8 + ((e >> 6) & 7), d.R * 8 + ((e >> 3) & 7),
                            d.S * 8 + (e & 7));
                    }
                } else {
                    for (int i = threadIdx.x; i < total; i += blockDim.x) {
                        const int e = klist[i];
                        sm.V[tile_swizzle(e)] = contracted_eri<TA, 128, MAXPP>(sm.pairs, e >> 6, sm.pairs, 64 + (e & 63));
                    }
                }
            } else {
                int pos = scan256(__popc(mask), sm.wsum);
                const int64_t base = a.offsets[bi] + MASK_BYTES / EB;
                const float inv = (SRC >= 2) ? 1.0f / a.vscale : 1.0f;
                for (int j = 0; j < 16; ++j) {
                    TA v = TA(0);
                    if (mask & (1u << j)) {
                        const int64_t i = base + pos++;
                        if (!(dmask & (1u << j))) {          // kept by Schwarz, dropped by the density rule
                            sm.V[tile_swizzle(e0 + j)] = TA(0);
                            continue;
                        }
                        if (SRC == 0) v = (TA)reinterpret_cast<const double *>(a.store)[i];
                        else if constexpr (SRC == 5) {
                            const float2 u = reinterpret_cast<const float2 *>(a.store)[i];
                            v = make_f32x2(u.x, u.y);
                        }
                        else if (SRC == 1) v = (TA)reinterpret_cast<const float *>(a.store)[i];
                        else {
                            const uint32_t u = reinterpret_cast<const uint32_t *>(a.store)[i];
                            float hi, lo;
                            if (SRC == 2) {
                                hi = __half2float(__ushort_as_half((unsigned short)(u & 0xffffu)));
                                lo = __half2float(__ushort_as_half((unsigned short)(u >> 16)));
                            } else {
                                hi = __bfloat162float(__ushort_as_bfloat16((unsigned short)(u & 0xffffu)));
                                lo = __bfloat162float(__ushort_as_bfloat16((unsigned short)(u >> 16)));
                            }
                            v = (TA)((hi + lo) * inv);
                        }
                    }
                    sm.V[tile_swizzle(e0 + j)] = v;
                }
            }
        }
        // ---- densities in chunks of MC
        for (int d0 = 0; d0 < a.m; d0 += MC) {
            __syncthreads();
            for (int t = threadIdx.x; t < 10 * 64 * MC; t += blockDim.x) {
                const int dd = t % MC, ij = (t / MC) & 63, tile = t / (MC * 64);
                const int x = ij >> 3, y = ij & 7;
                TA v = TA(0);
                if (d0 + dd < a.m) {
                    // the per-build copy of D in the arithmetic type when there is
                    // one (no conversion on the FP64 pipe here), else D itself
                    const TA *Dt = reinterpret_cast<const TA *>(a.Dt);
                    const int64_t kofs = (int64_t)(d0 + dd) * nn;
                    auto at = [&](int64_t idx) -> TA { return Dt ? Dt[kofs + idx] : (TA)a.D[kofs + idx]; };
                    if (tile < 8) {
                        const int ra = sm.blk[c_tuple[tile][1]] * 8 + x, cb = sm.blk[c_tuple[tile][3]] * 8 + y;
                        if (ra < n && cb < n) v = at((int64_t)ra * n + cb);
                    } else {
                        // Dj of the summed blocks (C, E): D[C,E] + [C != E] D[E,C]^T
                        const int C = sm.blk[tile == 8 ? 2 : 0], E = sm.blk[tile == 8 ? 3 : 1];
                        const int ra = C * 8 + x, cb = E * 8 + y;
                        if (ra < n && cb < n) {
                            if (C == E) v = at((int64_t)ra * n + cb);
                            else if (Dt) v = add_ta(Dt[kofs + (int64_t)ra * n + cb], Dt[kofs + (int64_t)cb * n + ra]);
                            else v = (TA)(a.D[kofs + (int64_t)ra * n + cb] + a.D[kofs + (int64_t)cb * n + ra]);
                        }
                    }
                }
                sm.Ds[tile][ij][dd] = v;
            }
            __syncthreads();
            const int ntask = sm.nslots * 64;
            for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
                const int slot = sm.slots[task >> 6], e = task & 63;
                const int A = c_slot[slot][0], C = c_slot[slot][1], X = c_slot[slot][2], Y = c_slot[slot][3];
                // output (a in block A, c in block C), terms (x in block X, y in block Y)
                const int ia = e >> 3, ic = e & 7;
                const int base = sm.tsw[A][ia] ^ sm.tsw[C][ic];
                const int orow = sm.blk[A] * 8 + ia, ocol = sm.blk[C] * 8 + ic;
                // placement of y * stride[Y] from its three bits (the swizzle is linear)
                const int t1 = sm.tsw[Y][1], t2 = sm.tsw[Y][2], t4 = sm.tsw[Y][4];
                TA acc[MC];
#pragma unroll
                for (int dd = 0; dd < MC; ++dd) acc[dd] = TA(0);
                for (int x = 0; x < 8; ++x) {
                    const int bx = base ^ sm.tsw[X][x];
#pragma unroll
                    for (int y = 0; y < 8; ++y) {
                        const TA v = sm.V[bx ^ ((y & 1) ? t1 : 0) ^ ((y & 2) ? t2 : 0) ^ ((y & 4) ? t4 : 0)];
                        const TA *dp = sm.Ds[slot][x * 8 + y];
#pragma unroll
                        for (int dd = 0; dd < MC; ++dd) macc(acc[dd], v, dp[dd]);
                    }
                }
                double *out = slot >= 8 ? a.Jacc : a.Kacc;
#pragma unroll
                for (int dd = 0; dd < MC; ++dd)
                    if (d0 + dd < a.m) atomicAdd(out + (int64_t)(d0 + dd) * npnp + (int64_t)orow * np + ocol, flush_value(acc[dd]));
            }
        }
    }
}

template <typename TA, int MC, int SRC>
static int jk_launch(const JKArgs &a, cudaStream_t s) {
    using SM = typename std::conditional<SRC == 4, JKSmemDirect<TA, MC>, JKSmem<TA, MC, false>>::type;
    const size_t smem = sizeof(SM);
    CK(cudaFuncSetAttribute(k_jk_cuda<TA, MC, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jk_cuda<TA, MC, SRC>, 256, smem));
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (grid > a.nbricks) grid = a.nbricks;
    if (grid < 1) return ESMF_OK;
    k_jk_cuda<TA, MC, SRC><<<(int)grid, 256, smem, s>>>(a);
    CK(cudaGetLastError());
    return ESMF_OK;
}

// MC (densities per pass over a brick's shared-memory tile) is a tuning
// parameter: 4/8/16 for float arithmetic, 4/8 for double (0 = default).  The
// defaults are the autotuner's choices on GB300 for the 200-function stored
// and 2000-function integral-direct workloads: 8 for stored FP64 and FP32,
// 16 for the split-store cross-check, 4 for integral-direct (its evaluation
// phase then fits two CTAs per SM: 1.74 s per 2000-function build against
// 2.22 s at 16).
template <typename TA, int SRC>
static int jk_launch_mc(const JKArgs &a, cudaStream_t s) {
    const int mc = a.mc ? a.mc : ((SRC == 4 || SRC == 6) ? 4 : ((SRC <= 1 || SRC == 5) ? 8 : 16));
    if (sizeof(TA) == 8) {
        if (mc == 4) return jk_launch<TA, 4, SRC>(a, s);
        return jk_launch<TA, 8, SRC>(a, s);
    }
    if (mc == 4) return jk_launch<TA, 4, SRC>(a, s);
    if (mc == 8) return jk_launch<TA, 8, SRC>(a, s);
    return jk_launch<TA, 16, SRC>(a, s);
}

int launch_jk_cuda(const JKArgs &a, cudaStream_t s) {
    if (a.mode == ESMF_MODE_DIRECT) {
        if (a.nbricks > 0 && (!a.ptab || !a.pslot)) {
            set_error("launch_jk_cuda: integral-direct build without a pair table");
            return ESMF_ERR_INVALID_ARG;
        }
        if (a.b.cart) {
            if (a.precision == ESMF_PREC_FP64) return jk_launch_mc<double, 6>(a, s);
            return jk_launch_mc<float, 6>(a, s);
        }
        if (a.precision == ESMF_PREC_FP64) return jk_launch_mc<double, 4>(a, s);
        return jk_launch_mc<float, 4>(a, s);
    }
    switch (a.precision) {
        case ESMF_PREC_FP64: return jk_launch_mc<double, 0>(a, s);
        case ESMF_PREC_FP32: return jk_launch_mc<float, 1>(a, s);
        case ESMF_PREC_F32X2: return jk_launch_mc<f32x2, 5>(a, s);
        default: break;
    }
    set_error("launch_jk_cuda: precision %d needs the split-precision path", a.precision);
    return ESMF_ERR_UNSUPPORTED;
}

// split-precision stores on CUDA cores (reference path for the tensor kernel)
int launch_jk_cuda_split(const JKArgs &a, cudaStream_t s) {
    if (a.precision == ESMF_PREC_FP16X2) return jk_launch_mc<float, 2>(a, s);
    if (a.precision == ESMF_PREC_BF16X2) return jk_launch_mc<float, 3>(a, s);
    set_error("launch_jk_cuda_split: bad precision %d", a.precision);
    return ESMF_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------- typed densities
// D (FP64, m x n x n) once per build in the contraction's arithmetic type.
template <typename T>
__global__ void k_density_typed(int64_t cnt, const double *D, T *Dt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        Dt[i] = T(D[i]);
}

size_t density_typed_bytes(int precision) {
    return precision == ESMF_PREC_F32X2 ? sizeof(f32x2) : (precision == ESMF_PREC_FP64 ? 0 : sizeof(float));
}

int launch_density_typed(int precision, int64_t cnt, const double *D, void *Dt, cudaStream_t s) {
    int64_t g = (cnt + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    if (precision == ESMF_PREC_F32X2)
        k_density_typed<f32x2><<<(int)g, 256, 0, s>>>(cnt, D, reinterpret_cast<f32x2 *>(Dt));
    else
        k_density_typed<float><<<(int)g, 256, 0, s>>>(cnt, D, reinterpret_cast<float *>(Dt));
    CK(cudaGetLastError());
    return ESMF_OK;
}

// ---------------------------------------------------------------- density weights
// dw[x][y] = max over k of max(|D_k[x][y]|, |D_k[y][x]|) on the padded grid
// (zero outside N), and dwb[X][Y] its 8 x 8 block maxima.  One block per row x.
// Non-negative doubles order like their bit patterns, so the block maxima are
// 64-bit integer atomic maxima.
__global__ void k_density_weight(int n, int np, int nb, int m, const double *D, double *dw,
                                 unsigned long long *dwb) {
    const int x = blockIdx.x;
    const int64_t nn = (int64_t)n * n;
    for (int y = threadIdx.x; y < np; y += blockDim.x) {
        double v = 0.0;
        if (x < n && y < n)
            for (int k = 0; k < m; ++k)
                v = fmax(v, fmax(fabs(D[k * nn + (int64_t)x * n + y]), fabs(D[k * nn + (int64_t)y * n + x])));
        dw[(int64_t)x * np + y] = v;
        atomicMax(dwb + (x >> 3) * nb + (y >> 3), (unsigned long long)__double_as_longlong(v));
    }
}

int launch_density_weight(const DevBasis &b, int m, const double *D, double *dw, double *dwb, cudaStream_t s) {
    CK(cudaMemsetAsync(dwb, 0, sizeof(double) * b.nb * b.nb, s));
    k_density_weight<<<b.np, 256, 0, s>>>(b.n, b.np, b.nb, m, D, dw, reinterpret_cast<unsigned long long *>(dwb));
    CK(cudaGetLastError());
    return ESMF_OK;
}

// ---------------------------------------------------------------- finalise
// J from the lower block triangle, F = 2J - K, t_k = sum_pq D_k[pq] F_k[pq].
__global__ void k_finalize(int n, int np, int m, const double *D, const double *Jacc,
                           const double *Kacc, double *J, double *K, double *F, double *tsum) {
    const int k = blockIdx.y;
    const int64_t nn = (int64_t)n * n, npnp = (int64_t)np * np;
    double part = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e / n), q = (int)(e % n);
        const double jv = ((p >> 3) >= (q >> 3)) ? Jacc[k * npnp + (int64_t)p * np + q]
                                                 : Jacc[k * npnp + (int64_t)q * np + p];
        const double kv = Kacc[k * npnp + (int64_t)p * np + q];
        const double fv = 2.0 * jv - kv;
        J[k * nn + e] = jv;
        K[k * nn + e] = kv;
        if (F) F[k * nn + e] = fv;
        part += D[k * nn + e] * fv;
    }
    if (tsum) {
        __shared__ double red[8];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            atomicAdd(tsum + k, s);
        }
    }
}

int launch_finalize(const DevBasis &b, int m, const double *D, const double *Jacc,
                    const double *Kacc, double *J, double *K, double *F, double *tsum,
                    cudaStream_t s) {
    const int64_t nn = (int64_t)b.n * b.n;
    int gx = (int)((nn + 255) / 256);
    if (gx > 512) gx = 512;
    dim3 grid(gx, m);
    k_finalize<<<grid, 256, 0, s>>>(b.n, b.np, m, D, Jacc, Kacc, J, K, F, tsum);
    CK(cudaGetLastError());
    return ESMF_OK;
}

}  // namespace esmf
