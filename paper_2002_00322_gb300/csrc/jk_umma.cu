// Grouped J/K contraction on the sm_103a tensor cores (tcgen05), for integral
// stores held as scaled 16-bit hi+lo pairs (FP16 or BF16 halves).
//
// Every kept brick (P Q | R S) of 8x8x8x8 integrals feeds, for all m densities,
// the ordered-tuple updates of Eq. (J_and_K) (see jk_cuda.cu).  Grouped by
// output block they are six small GEMMs with M = 64 output rows, K = 64:
//   exchange  V1 (pr|qs): K[P,R] += V D[Q,S],  K[R,P]^T += V D[S,Q]^T
//             V2 (qr|ps): K[Q,R] += V D[P,S],  K[R,Q]^T += V D[S,P]^T
//             V3 (ps|qr): K[P,S] += V D[Q,R],  K[S,P]^T += V D[R,Q]^T
//             V4 (qs|pr): K[Q,S] += V D[P,R],  K[S,Q]^T += V D[R,P]^T
//   Coulomb   J1 (pq|rs): J[P,Q] += V Dj[R,S],  J2 (rs|pq): J[R,S] += V^T Dj[P,Q]
// with Dj[X,Y] = D[X,Y] + [X != Y] D[Y,X]^T.  The brick tile V[p][q][r][s]
// (fp16, s fastest) is a canonical no-swizzle operand for all four exchange
// views (two K-major, two MN-major descriptors over the same bytes); the
// Coulomb views read a second copy W[p][r][q][s].  Products are formed as
//   V_hi D_hi + V_hi D_lo + V_lo D_hi   (FP32 accumulation in tensor memory),
// three MMAs into the same columns ([D | D^T] for exchange, N = 2m).
//
// Bricks come in items: a bra pair (P,Q) with a window of SWIN S blocks, all
// R; within an item, runs share R.  V3 and V4 accumulate K{P,S} and K{Q,S}
// for every S of the window over the whole item, V1 and V2 accumulate K{P,R}
// and K{Q,R} over a run (double-buffered by run), and the Coulomb views are
// flushed per brick (double-buffered; their FP32 sums over longer spans lose
// accuracy when transition densities cancel).  Flushes add into FP64
// accumulators with reductions straight from the registers that the
// tensor-memory loads fill: each epilogue warp reads its 16 accumulator rows
// in the 16x32bx2 shape (threads 0-15 the first half of the density columns,
// threads 16-31 the second), so every lane carries data and a warp's
// reduction covers 2 x 16 consecutive FP64 values of a block (the D^T parts,
// written transposed, 16 values in 8 pairs); no shared-memory staging.
//
// Warp roles (320 threads): warp 0 producer (bulk copies of the packed brick
// record and the six density tiles), warp 1 tensor-memory owner and MMA
// issuer, warps 2-5 expand packed records into the operand tiles, warps 6-9
// read accumulators and reduce them into the FP64 accumulators.  Every mbarrier wait is bounded; on
// timeout the kernel records an error and all roles leave.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "esmf_internal.cuh"
#include "umma.cuh"

namespace esmf {

using namespace umma;

namespace {

constexpr int NTHREADS = 320;
constexpr int MPMAX = 16;                         // densities per pass
constexpr int KB_BYTES_MAX = 512 * MPMAX;         // 4 mp rows x 64 k x 2 B
constexpr int JB_BYTES_MAX = 256 * MPMAX;         // 2 mp rows x 64 k x 2 B
constexpr int IN_BYTES = 512 + 4 * BRICK;         // mask + packed values
// per-stage layout
constexpr int OFF_VH = 0, OFF_VL = 8192, OFF_WH = 16384, OFF_WL = 24576;
constexpr int OFF_B1 = 32768;                     // four exchange tiles
constexpr int OFF_B5 = OFF_B1 + 4 * KB_BYTES_MAX; // two Coulomb tiles
constexpr int OFF_IN = OFF_B5 + 2 * JB_BYTES_MAX;
constexpr int STAGE_BYTES = ((OFF_IN + IN_BYTES + 1023) / 1024) * 1024;
constexpr int CTRL_BYTES = 4096;
constexpr int CQ = 16;                 // chunk queue slots
constexpr int MAX_ENTRIES_CTRL = 16;   // entries per launch (MAX_ENTRIES)
constexpr int CHUNKS_PER_CTA = 4;      // chunks of an entry without a part list, per CTA
constexpr int SMEM_TOTAL = 2 * STAGE_BYTES + CTRL_BYTES;

struct Ctrl {
    uint64_t full[2], conv[2], mmad[2], acce[2], runfree[2];
    // window region w has been read at the end of wstaged[w] / 4 items (each
    // epilogue warp adds one); monotonic, so a waiter can be any number of
    // items behind (an mbarrier phase parity could alias two completions)
    unsigned wstaged[SWIN];
    uint32_t tmem_base;
    int abort_flag;
    int cdecide, edecide;   // group-uniform copies of abort_flag (converters, epilogue)
    int scan[8];
    int vpos[512];
    // dynamic work: the producer takes chunk indices from the launch's counter
    // and publishes them in order (cq_pub counts published slots, cq_done four
    // per chunk the epilogue has finished); -1 ends the sequence
    int cq[CQ];
    unsigned cq_pub, cq_done;
    int cbase[MAX_ENTRIES_CTRL + 1];   // first global chunk index of each entry
};
static_assert(sizeof(Ctrl) <= CTRL_BYTES, "control block");

__device__ __forceinline__ float density_scale(const unsigned int *dmax_bits) {
    const float dm = __uint_as_float(*dmax_bits);
    if (!(dm > 0.f)) return 1.0f;
    int e;
    frexpf(2.0f * dm, &e);            // 2 max|D| in [2^(e-1), 2^e)
    return ldexpf(1.0f, 14 - e);
}

}  // namespace

// ---------------------------------------------------------------- density tiles
__global__ void k_dmax(const double *D, int64_t count, unsigned int *out) {
    float mx = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, __double2float_ru(fabs(D[i])));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

__device__ __forceinline__ uint16_t split16(float x, int part_lo, int bf16) {
    if (bf16) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        if (!part_lo) return __bfloat16_as_ushort(h);
        return __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    }
    __half h = __float2half_rn(x);
    if (!part_lo) return __half_as_ushort(h);
    return __half_as_ushort(__float2half_rn(x - __half2float(h)));
}

// canonical K-major operand tile: row n (density column of the MMA), k = b*8 + d
__device__ __forceinline__ int tile_off(int row, int k) {
    return (row & 7) * 16 + (k & 7) * 2 + (k >> 3) * 128 + (row >> 3) * 1024;
}

// Density tiles of one pass (densities d0 .. d0+mp-1; rows kk >= m are zero):
// K bank, tile (X,Y) of nb*nb, rows kk / mp+kk / 2mp+kk / 3mp+kk hold D_hi,
// D^T_hi, D_lo, D^T_lo at k = b*8 + d (D[X*8+b][Y*8+d], and for the
// transposed parts D[Y*8+d][X*8+b]); J bank, lower block triangle X >= Y,
// rows kk / mp+kk hold the hi / lo halves of D[X*8+b][Y*8+d] + D[Y*8+d][X*8+b]
// (the first term alone on the diagonal block).  One block per (row p of the
// padded matrix, kk): each thread converts one element (p, q) once and writes
// its four K-bank halves and, for X >= Y, its two J-bank halves, so every
// position of both banks is written exactly once per pass.
__global__ void k_dbank(const double *D, int n, int nb, int m, int d0, int mp, const unsigned int *dmax_bits,
                        int bf16, uint16_t *kbank, uint16_t *jbank) {
    const double sD = (double)density_scale(dmax_bits);
    const int np = nb * 8;
    const int p = blockIdx.x, kk = blockIdx.y;
    const int X = p >> 3, b = p & 7;
    const int F = 4 * mp, G = 2 * mp;
    const bool live = kk < m && p < n;
    const double *Dk = D + (int64_t)(d0 + kk) * n * n;
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const int Y = q >> 3, d = q & 7;
        const bool in = live && q < n;
        const double v = in ? Dk[(int64_t)p * n + q] : 0.0;
        const float x = (float)(v * sD);
        const uint16_t hi = split16(x, 0, bf16), lo = split16(x, 1, bf16);
        uint16_t *kt = kbank + ((int64_t)X * nb + Y) * (F * 64);
        const int o1 = tile_off(kk, b * 8 + d) >> 1, o3 = tile_off(2 * mp + kk, b * 8 + d) >> 1;
        kt[o1] = hi;
        kt[o3] = lo;
        uint16_t *kt2 = kbank + ((int64_t)Y * nb + X) * (F * 64);
        kt2[tile_off(mp + kk, d * 8 + b) >> 1] = hi;
        kt2[tile_off(3 * mp + kk, d * 8 + b) >> 1] = lo;
        if (X >= Y) {
            double vj = v;
            if (X != Y && in) vj += Dk[(int64_t)q * n + p];
            const float xj = (X != Y) ? (float)(vj * sD) : x;
            uint16_t *jt = jbank + ((int64_t)X * (X + 1) / 2 + Y) * (G * 64);
            jt[tile_off(kk, b * 8 + d) >> 1] = split16(xj, 0, bf16);
            jt[tile_off(mp + kk, b * 8 + d) >> 1] = split16(xj, 1, bf16);
        }
    }
}

// ---------------------------------------------------------------- main kernel
// One entry of a launch: the bricks of one handle contracted with one chunk of
// at most 16 of its densities.  A launch holds up to MAX_ENTRIES entries
// (several molecules, uneven basis sizes and density counts) and every CTA
// takes chunks of the entries from a launch-wide counter.
struct UmmaEntry {
    const BrickDesc *bricks;
    int64_t nbricks;
    const int64_t *offsets;        // record start, in 32-bit words
    const uint32_t *store;
    const uint16_t *kbank, *jbank;
    const int64_t *part;           // chunk brick ranges (nparts + 1), or null: even chunks by count
    int nparts, nb, m, d0, mtot, bf16;
    float vscale;
    const unsigned int *dmax_bits;
    double *Jacc, *Kacc;           // block-major: [X][Y][k][x][y], k < mtot
    int *error;                    // the entry's handle's device error flag
};
constexpr int MAX_ENTRIES = 16;
struct UmmaParams {
    UmmaEntry e[MAX_ENTRIES];
    int nentries, mp;              // mp: density columns per pass, the same for every entry
    unsigned *counter;             // chunks taken so far (zero at launch)
};
static_assert(MAX_ENTRIES == MAX_ENTRIES_CTRL, "entries per launch");

namespace {

// Chunks of entry E: its part list (cost-balanced brick ranges, several per
// CTA), or CHUNKS_PER_CTA even ranges per CTA.  CTAs take chunks dynamically,
// in the order of a launch-wide counter.
__device__ __forceinline__ int entry_chunks(const UmmaEntry &E) {
    if (E.part) return E.nparts;
    const int64_t k = (int64_t)CHUNKS_PER_CTA * gridDim.x;
    return (int)(E.nbricks < k ? E.nbricks : k);
}
__device__ __forceinline__ void chunk_range(const UmmaEntry &E, int j, int64_t &beg, int64_t &end) {
    if (E.part) {
        beg = E.part[j];
        end = E.part[j + 1];
    } else {
        const int nc = entry_chunks(E);
        beg = E.nbricks * j / nc;
        end = E.nbricks * (j + 1) / nc;
    }
}

}  // namespace

namespace {

// 16 lanes x 32-bit from the warp's lane quarter, two halves: threads 0-15
// take lane (base + t) at columns [0, N), threads 16-31 lane (base + t - 16) at
// columns [N, 2N) (split offset N), N = 8 or 4 registers.
__device__ __forceinline__ void tmem_ld_half8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.16x32bx2.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], 8;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_half4(uint32_t taddr, float *v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.16x32bx2.x4.b32 {%0,%1,%2,%3}, [%4], 4;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
#pragma unroll
    for (int i = 4; i < 8; ++i) v[i] = 0.f;
}

// Error-free sum (Knuth's TwoSum) of the running value hi and the term t:
// hi <- fl(hi + t), lo collects the rounding error, so hi + lo carries the
// sum of all terms to about twice single precision.  Written with explicit
// round-to-nearest intrinsics so that no step is contracted or reassociated.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float t) {
    const float s = __fadd_rn(hi, t);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

}  // namespace

__global__ void __launch_bounds__(NTHREADS, 1) k_jk_umma(const __grid_constant__ UmmaParams P) {
    extern __shared__ __align__(1024) unsigned char sm[];
    Ctrl &c = *reinterpret_cast<Ctrl *>(sm + 2 * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mp = P.mp;
    const uint32_t kbytes = 512u * mp, jbytes = 256u * mp;
    volatile int *abort_flag = &c.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&c.full[s], 1);
            mbar_init(&c.conv[s], 4);
            mbar_init(&c.mmad[s], 1);
            mbar_init(&c.acce[s], 4);
        }
        mbar_init(&c.runfree[0], 4);
        mbar_init(&c.runfree[1], 4);
        for (int w = 0; w < SWIN; ++w) c.wstaged[w] = 0;
        c.abort_flag = 0;
        c.cq_pub = 0;
        c.cq_done = 0;
        c.cbase[0] = 0;
        for (int e = 0; e < P.nentries; ++e) c.cbase[e + 1] = c.cbase[e] + entry_chunks(P.e[e]);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&c.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = c.tmem_base;
    // A CTA that gives up leaves the rest of its chunks of every entry
    // unprocessed, so every entry of the launch is marked incomplete.
    auto fail = [&](int code) {
        *abort_flag = 1;
        for (int e = 0; e < P.nentries; ++e)
            if (P.e[e].error) atomicExch(P.e[e].error, code);
    };
    const int nchunks = c.cbase[P.nentries];
    // global chunk ch -> entry e and its brick range
    auto resolve = [&](int ch, int &e, int64_t &beg, int64_t &end) {
        e = 0;
        while (e + 1 < P.nentries && ch >= c.cbase[e + 1]) ++e;
        chunk_range(P.e[e], ch - c.cbase[e], beg, end);
    };
    // the qr-th chunk of this CTA, as the producer published it; false at the
    // end of the sequence or when the wait gives up
    auto take_chunk = [&](int qr, int &e, int64_t &beg, int64_t &end) -> bool {
        if (!counter_wait(&c.cq_pub, (unsigned)qr + 1u, abort_flag)) {
            if (!*abort_flag) fail(11);
            return false;
        }
        const int ch = c.cq[qr % CQ];
        if (ch < 0) return false;
        resolve(ch, e, beg, end);
        return true;
    };

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ producer
        int issued = 0;
        // the next brick's descriptor and record offset are loaded one
        // iteration ahead, so their latency overlaps the wait for a free stage
        int i = 0;
        bool stop = false;
        for (int qr = 0; !stop; ++qr) {
            // take the next chunk of the launch and publish it to the other
            // roles (its queue slot is free once the epilogue finished chunk qr - CQ)
            if (qr >= CQ && !counter_wait(&c.cq_done, 4u * (unsigned)(qr - CQ + 1), abort_flag)) {
                if (!*abort_flag) fail(12);
                break;
            }
            int ch = (int)atomicAdd(P.counter, 1u);
            if (ch >= nchunks) ch = -1;
            c.cq[qr % CQ] = ch;
            counter_release_add(&c.cq_pub);
            if (ch < 0) break;
            int e;
            int64_t beg, end;
            resolve(ch, e, beg, end);
            if (beg >= end) continue;
            const UmmaEntry &E = P.e[e];
            const BrickDesc *bricks = E.bricks;
            const int64_t *offsets = E.offsets;
            const uint32_t *store = E.store;
            const uint16_t *kb = E.kbank, *jb = E.jbank;
            const int enb = E.nb;
            BrickDesc dnext = bricks[beg];
            int64_t onext = offsets[beg];
            for (int64_t ib = beg; ib < end; ++ib, ++i) {
                const int s = i & 1;
                const BrickDesc d = dnext;
                const int64_t off = onext;
                if (ib + 1 < end) {
                    dnext = bricks[ib + 1];
                    onext = offsets[ib + 1];
                }
                if (i >= 2 && !mbar_wait(&c.mmad[s], ((i - 2) >> 1) & 1, abort_flag)) { fail(2); stop = true; break; }
                unsigned char *st = sm + s * STAGE_BYTES;
                const uint32_t rec = ((512u + 4u * (uint32_t)d.nkept) + 15u) & ~15u;
                const size_t kw = kbytes / 2, jw = jbytes / 2;
                mbar_arrive_expect_tx(&c.full[s], rec + 4 * kbytes + 2 * jbytes);
                bulk_g2s(st + OFF_IN, store + off, rec, &c.full[s]);
                bulk_g2s(st + OFF_B1 + 0 * KB_BYTES_MAX, kb + ((size_t)d.Q * enb + d.S) * kw, kbytes, &c.full[s]);
                bulk_g2s(st + OFF_B1 + 1 * KB_BYTES_MAX, kb + ((size_t)d.P * enb + d.S) * kw, kbytes, &c.full[s]);
                bulk_g2s(st + OFF_B1 + 2 * KB_BYTES_MAX, kb + ((size_t)d.Q * enb + d.R) * kw, kbytes, &c.full[s]);
                bulk_g2s(st + OFF_B1 + 3 * KB_BYTES_MAX, kb + ((size_t)d.P * enb + d.R) * kw, kbytes, &c.full[s]);
                bulk_g2s(st + OFF_B5, jb + ((size_t)d.R * (d.R + 1) / 2 + d.S) * jw, jbytes, &c.full[s]);
                bulk_g2s(st + OFF_B5 + JB_BYTES_MAX, jb + ((size_t)d.P * (d.P + 1) / 2 + d.Q) * jw, jbytes, &c.full[s]);
                issued = i + 1;
            }
        }
        // no copy may still be landing when the CTA leaves
        for (int k = (issued > 2 ? issued - 2 : 0); k < issued; ++k)
            mbar_wait(&c.full[k & 1], (k >> 1) & 1, abort_flag);
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        // The whole warp runs the loop and takes every wait (decisions made
        // warp-uniform); one elected lane issues the MMAs and the commit.
        // Descriptors are formed once per view and advanced by adding the
        // byte offset / 16 to the start-address field (shared addresses stay
        // below 256 KB, so the 14-bit field never carries).
        // tensor memory: window regions V3[w] at RW*w and V4[w] at RW*(SWIN+w);
        // run regions V1, V2 at WV + rb*2RW (+RW); per-brick J2, J1 at
        // WJ + b*2mp (+mp).  At mp = 16: 320 + 128 + 64 = 512 columns.
        const uint32_t RW = 2 * mp, WV = 2 * SWIN * RW, WJ = WV + 4 * RW;
        const uint32_t klo = 256u * mp, jlo = 128u * mp;     // byte offset of the lo rows in B tiles
        int run = 0, item = 0, committed = 0;
        unsigned touched3 = 0, touched4 = 0;
        int i = 0;
        bool stop = false;
        for (int qr = 0; !stop; ++qr) {
            int e;
            int64_t beg, end;
            if (!take_chunk(qr, e, beg, end)) break;
            if (beg >= end) continue;
            const UmmaEntry &E = P.e[e];
            const BrickDesc *bricks = E.bricks;
            // instruction descriptors of the entry (FP16 or BF16 halves)
            const uint32_t id_k = idesc_f16(64, RW, 0, E.bf16), idm_k = idesc_f16(64, RW, 1, E.bf16);
            const uint32_t id_j = idesc_f16(64, mp, 0, E.bf16), idm_j = idesc_f16(64, mp, 1, E.bf16);
            BrickDesc dnext = bricks[beg];
            for (int64_t ib = beg; ib < end; ++ib, ++i) {
                const int s = i & 1, b = i & 1;
                const BrickDesc d = dnext;
                const bool sfirst = ib == beg, slast = ib == end - 1;
                if (ib + 1 < end) dnext = bricks[ib + 1];
                const bool frun = sfirst || (d.pad & BRICK_RUN_FIRST);
                const bool lrun = slast || (d.pad & BRICK_RUN_LAST);
                const bool fitem = sfirst || (d.pad & BRICK_ITEM_FIRST);
                const bool litem = slast || (d.pad & BRICK_ITEM_LAST);
                const int rb = run & 1;
                if (!__all_sync(~0u, mbar_wait(&c.conv[s], (i >> 1) & 1, abort_flag))) { fail(3); stop = true; break; }
                if (i >= 2 && !__all_sync(~0u, mbar_wait(&c.acce[b], ((i - 2) >> 1) & 1, abort_flag))) { fail(4); stop = true; break; }
                if (frun && run >= 2 && !__all_sync(~0u, mbar_wait(&c.runfree[rb], ((run - 2) >> 1) & 1, abort_flag))) { fail(5); stop = true; break; }
                if (fitem) { touched3 = 0; touched4 = 0; }
                // window region w (V3[w] and V4[w]) is free once the epilogue has
                // read it at the end of the previous item
                const int wreg = d.S % SWIN;
                if (d.R != d.S && item >= 1 && !((touched3 | touched4) & (1u << wreg)) &&
                    !__all_sync(~0u, counter_wait(&c.wstaged[wreg], 4u * (unsigned)item, abort_flag))) { fail(10); stop = true; break; }
                tc_fence_after();
                const bool pq_diff = d.P != d.Q, rs_diff = d.R != d.S;
                const int w = d.S % SWIN;
                const bool fresh3 = !(touched3 & (1u << w)), fresh4 = !(touched4 & (1u << w));
                if (rs_diff) touched3 |= 1u << w;
                if (rs_diff && pq_diff) touched4 |= 1u << w;
                if (elect_one()) {
                    const uint32_t st = smem_u32(sm + s * STAGE_BYTES);
                    const uint32_t VH = st + OFF_VH, VL = st + OFF_VL, WH = st + OFF_WH, WL = st + OFF_WL;
                    const uint32_t B1 = st + OFF_B1, B2 = B1 + KB_BYTES_MAX, B3 = B2 + KB_BYTES_MAX,
                                   B4 = B3 + KB_BYTES_MAX, B5 = st + OFF_B5, B6 = B5 + JB_BYTES_MAX;
                    // three passes into the same columns: hi x [D|D^T]_hi, hi x [D|D^T]_lo, lo x [D|D^T]_hi
                    auto view = [&](uint32_t col, uint32_t AH, uint32_t AL, uint32_t kstep, uint32_t lbo, uint32_t sbo,
                                    uint32_t id, uint32_t B, uint32_t blo, bool fresh) {
                        const uint64_t ah = sdesc(AH, lbo, sbo), al = ah + ((AL - AH) >> 4);
                        const uint64_t bh = sdesc(B, 128, 1024), bl = bh + (blo >> 4);
                        const uint32_t ks = kstep >> 4;
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            mma_f16(tmem + col, ah + j * ks, bh + 16 * j, id, (j > 0 || !fresh) ? 1u : 0u);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            mma_f16(tmem + col, ah + j * ks, bl + 16 * j, id, 1u);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            mma_f16(tmem + col, al + j * ks, bh + 16 * j, id, 1u);
                    };
                    // exchange: V1, V2 over the run; V3, V4 over the item (nothing when R == S,
                    // V2 and V4 nothing when P == Q: those permutations repeat others)
                    view(WV + rb * 2 * RW, VH, VL, 256, 128, 1024, id_k, B1, klo, frun);
                    if (pq_diff) view(WV + rb * 2 * RW + RW, VH, VL, 2048, 1024, 128, id_k, B2, klo, frun);
                    if (rs_diff) view(RW * w, VH, VL, 256, 128, 1024, idm_k, B3, klo, fresh3);
                    if (rs_diff && pq_diff) view(RW * (SWIN + w), VH, VL, 2048, 1024, 128, idm_k, B4, klo, fresh4);
                    // Coulomb views, per brick: J1 (K-major over W) and J2 (MN-major over W)
                    view(WJ + b * 2 * mp + mp, WH, WL, 256, 128, 1024, id_j, B5, jlo, true);
                    view(WJ + b * 2 * mp, WH, WL, 2048, 1024, 128, idm_j, B6, jlo, true);
                    mma_commit(&c.mmad[s]);
                }
                __syncwarp();
                committed = i + 1;
                if (lrun) ++run;
                if (litem) ++item;
            }
        }
        if (committed > 0) {
            const int i = committed - 1;
            mbar_wait(&c.mmad[i & 1], (i >> 1) & 1, abort_flag);
        }
    } else if (warp >= 2 && warp < 6) {
        // ------------------------------------------------ converters
        const int ct = threadIdx.x - 64;
        int i = 0;                     // bricks of this CTA so far
        int64_t left = 0;              // bricks left in the current chunk
        for (int qr = 0;; ++i, --left) {
            while (left == 0) {
                int e;
                int64_t beg, end;
                if (!take_chunk(qr++, e, beg, end)) break;
                left = end - beg;
            }
            if (left == 0) break;
            const int s = i & 1;
            if (!mbar_wait(&c.full[s], (i >> 1) & 1, abort_flag)) fail(6);
            // leave together: every converter thread must reach the same named barriers
            named_bar_sync(1, 128);
            if (ct == 0) c.cdecide = *abort_flag;
            named_bar_sync(1, 128);
            if (c.cdecide) break;
            unsigned char *st = sm + s * STAGE_BYTES;
            const unsigned char *mask = st + OFF_IN;
            const uint32_t *vals = reinterpret_cast<const uint32_t *>(st + OFF_IN + 512);
            // packed positions: exclusive scan of per-vector counts in local order
            int cnt[4], tot = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) { cnt[j] = __popc(mask[4 * ct + j]); tot += cnt[j]; }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) c.scan[ct >> 5] = incl;
            named_bar_sync(1, 128);
            int base = incl - tot;
            for (int w = 0; w < (ct >> 5); ++w) base += c.scan[w];
#pragma unroll
            for (int j = 0; j < 4; ++j) { c.vpos[4 * ct + j] = base; base += cnt[j]; }
            named_bar_sync(1, 128);
            // expand: 4 s-vectors per thread, mapped so that both the V and the
            // W tile stores of 8 neighbouring threads hit distinct bank groups
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int u = k * 128 + ct;
                const int jj = u & 7, cc = (u >> 3) & 7, p = u >> 6;
                const int q = jj, r = (jj + cc) & 7;
                const int v = p * 64 + q * 8 + r;
                const unsigned m8 = mask[v];
                int pos = c.vpos[v];
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    uint32_t x0 = 0, x1 = 0;
                    if (m8 & (1u << (2 * h))) x0 = vals[pos++];
                    if (m8 & (1u << (2 * h + 1))) x1 = vals[pos++];
                    hi[h] = (x0 & 0xffffu) | (x1 << 16);
                    lo[h] = (x0 >> 16) | (x1 & 0xffff0000u);
                }
                const uint4 H = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                const uint4 L = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<uint4 *>(st + OFF_VH + v * 16) = H;
                *reinterpret_cast<uint4 *>(st + OFF_VL + v * 16) = L;
                const int vw = p * 64 + r * 8 + q;
                *reinterpret_cast<uint4 *>(st + OFF_WH + vw * 16) = H;
                *reinterpret_cast<uint4 *>(st + OFF_WL + vw * 16) = L;
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&c.conv[s]);
            named_bar_sync(1, 128);   // vpos / scan reused by the next brick
        }
    } else if (warp >= 6) {
        // ------------------------------------------------ epilogue
        const int slice = warp & 3;
        const uint32_t tl = tmem + ((uint32_t)(slice * 32) << 16);
        const uint32_t RW = 2 * mp, WV = 2 * SWIN * RW, WJ = WV + 4 * RW;
        // compensated running sum of J1 -> J[P,Q] over the item (P, Q fixed)
        float j1h[MPMAX / 2], j1l[MPMAX / 2];
#pragma unroll
        for (int k = 0; k < MPMAX / 2; ++k) { j1h[k] = 0.f; j1l[k] = 0.f; }
        const int jrow = slice * 16 + (lane & 15);      // accumulator row of this thread (all lanes)
        // per-entry constants (refreshed when the stream enters a new entry)
        int m = 0, nb = 0, mtot = 0, d0 = 0;
        float inv = 1.0f;
        double *Jacc = nullptr, *Kacc = nullptr;
        auto blk = [&](double *base, int X, int Y) { return base + ((int64_t)(X * nb + Y) * mtot + d0) * 64; };
        const int trow = (jrow & 7) * 8 + (jrow >> 3);  // its place in a transposed block
        // an exchange region [D part | D^T part] read in the half layout: this
        // thread's densities cb .. cb + mp/2 - 1 of both parts
        auto ld_x = [&](uint32_t col, float *vd, float *vt) {
            if (mp == 16) { tmem_ld_half8(tl + col, vd); tmem_ld_half8(tl + col + mp, vt); }
            else { tmem_ld_half4(tl + col, vd); tmem_ld_half4(tl + col + mp, vt); }
        };
        // reductions of a loaded region into K[A,C] (D part) and K[C,A] (D^T part)
        auto red_x = [&](const float *vd, const float *vt, int A, int C, bool with_t) {
            const int half = mp / 2, cb = lane < 16 ? 0 : half;
            double *dd = blk(Kacc, A, C) + jrow, *dt = blk(Kacc, C, A) + trow;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < half && cb + j < m) {
                    atomicAdd(dd + (cb + j) * 64, (double)(vd[j] * inv));
                    if (with_t) atomicAdd(dt + (cb + j) * 64, (double)(vt[j] * inv));
                }
        };
        auto release = [&](uint64_t *bar) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar);
        };
        int run = 0;
        unsigned touched3 = 0, touched4 = 0;
        int i = 0;
        bool stop = false;
        for (int qr = 0; !stop; ++qr) {
            int e;
            int64_t beg, end;
            if (!take_chunk(qr, e, beg, end)) break;
            const UmmaEntry &E = P.e[e];
            const BrickDesc *bricks = E.bricks;
            m = E.m; nb = E.nb; mtot = E.mtot; d0 = E.d0; Jacc = E.Jacc; Kacc = E.Kacc;
            inv = 1.0f / (E.vscale * density_scale(E.dmax_bits));
            for (int64_t ib = beg; ib < end; ++ib, ++i) {
                const int s = i & 1, b = i & 1;
                const BrickDesc d = bricks[ib];
                const bool sfirst = ib == beg, slast = ib == end - 1;
                const bool lrun = slast || (d.pad & BRICK_RUN_LAST);
                const bool fitem = sfirst || (d.pad & BRICK_ITEM_FIRST);
                const bool litem = slast || (d.pad & BRICK_ITEM_LAST);
                const bool pq_diff = d.P != d.Q, rs_diff = d.R != d.S;
                const bool diag = d.R == d.P && d.S == d.Q;
                if (fitem) { touched3 = 0; touched4 = 0; }
                if (rs_diff) touched3 |= 1u << (d.S % SWIN);
                if (rs_diff && pq_diff) touched4 |= 1u << (d.S % SWIN);
                if (!mbar_wait(&c.mmad[s], (i >> 1) & 1, abort_flag)) fail(7);
                // leave together: every epilogue thread must reach the same named barriers
                named_bar_sync(2, 128);
                if (threadIdx.x == 192) c.edecide = *abort_flag;
                named_bar_sync(2, 128);
                if (c.edecide) { stop = true; break; }
                tc_fence_after();
                // per brick: Coulomb view J2 -> J[R,S] (not for the (PQ|PQ) brick) is
                // flushed; J1 -> J[P,Q] joins the item's compensated sum
                {
                    float vj2[8], vj1[8];
                    if (mp == 16) { tmem_ld_half8(tl + WJ + b * 2 * mp, vj2); tmem_ld_half8(tl + WJ + b * 2 * mp + mp, vj1); }
                    else { tmem_ld_half4(tl + WJ + b * 2 * mp, vj2); tmem_ld_half4(tl + WJ + b * 2 * mp + mp, vj1); }
                    tmem_wait_ld();
                    release(&c.acce[b]);
                    const int half = mp / 2, cb = lane < 16 ? 0 : half;
                    if (!diag) {
                        double *dst = blk(Jacc, d.R, d.S) + jrow;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < half && cb + j < m) atomicAdd(dst + (cb + j) * 64, (double)(vj2[j] * inv));
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < half) two_sum_acc(j1h[j], j1l[j], __fmul_rn(vj1[j], inv));
                }
                if (lrun) {
                    // V1 -> K[P,R] (and K[R,P] unless (PQ|PQ)), V2 -> K[Q,R], K[R,Q] (P != Q)
                    const int rb = run & 1;
                    float a1[8], a2[8], b1[8], b2[8];
                    ld_x(WV + rb * 2 * RW, a1, a2);
                    if (pq_diff) ld_x(WV + rb * 2 * RW + RW, b1, b2);
                    tmem_wait_ld();
                    release(&c.runfree[rb]);
                    red_x(a1, a2, d.P, d.R, !diag);
                    if (pq_diff) red_x(b1, b2, d.Q, d.R, !diag);
                    ++run;
                }
                if (litem) {
                    {
                        const int half = mp / 2, cb = lane < 16 ? 0 : half;
                        double *dst = blk(Jacc, d.P, d.Q) + jrow;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < half && cb + j < m) atomicAdd(dst + (cb + j) * 64, (double)j1h[j] + (double)j1l[j]);
#pragma unroll
                        for (int j = 0; j < 8; ++j) { j1h[j] = 0.f; j1l[j] = 0.f; }
                    }
                    // window regions: V3 -> K[P,S], K[S,P]; V4 -> K[Q,S], K[S,Q] (D^T parts
                    // not for the (PQ|PQ) item)
                    const int S0 = d.S - d.S % SWIN;
                    for (int w = 0; w < SWIN; ++w) {
                        const bool h3 = touched3 & (1u << w), h4 = touched4 & (1u << w);
                        float a1[8], a2[8], b1[8], b2[8];
                        if (h3) ld_x(RW * w, a1, a2);
                        if (h4) ld_x(RW * (SWIN + w), b1, b2);
                        if (h3 || h4) tmem_wait_ld();
                        tc_fence_before();                  // every region, once per item
                        __syncwarp();
                        if (lane == 0) counter_release_add(&c.wstaged[w]);
                        const int S = S0 + w;
                        if (h3) red_x(a1, a2, d.P, S, !diag);
                        if (h4) red_x(b1, b2, d.Q, S, !diag);
                    }
                }
            }
            // this chunk's queue slot may be reused
            __syncwarp();
            if (lane == 0) counter_release_add(&c.cq_done);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Several handles in one persistent launch per pass of 16 densities: pass c
// contracts density chunk c of every handle with more than 16c densities
// (one launch when every m <= 16).  Each handle keeps its own density bank
// and accumulators; the CTAs take cost-balanced chunks of every handle.
int launch_jk_umma_batch(const UmmaLaunch *Ls, int count, cudaStream_t s) {
    if (count < 1 || count > MAX_ENTRIES) {
        set_error("batch of %d handles outside [1, %d]", count, MAX_ENTRIES);
        return ESMF_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaFuncSetAttribute(k_jk_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL);
    if (e != cudaSuccess) { set_error("smem attribute: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    int mmax = 0, grid = 1;
    for (int i = 0; i < count; ++i) {
        const UmmaLaunch &L = Ls[i];
        const int64_t nn = (int64_t)L.n * L.n;
        e = cudaMemsetAsync(L.dmax_bits, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) { set_error("memset dmax: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
        k_dmax<<<256, 256, 0, s>>>(L.D, (int64_t)L.m * nn, L.dmax_bits);
        mmax = L.m > mmax ? L.m : mmax;
        const int g = L.nbricks < L.num_sms ? (int)L.nbricks : L.num_sms;
        grid = g > grid ? g : grid;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("k_dmax: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    for (int d0 = 0; d0 < mmax; d0 += MPMAX) {
        UmmaParams p;
        p.nentries = 0;
        p.mp = MPMAX;
        for (int i = 0; i < count; ++i) {
            const UmmaLaunch &L = Ls[i];
            if (d0 >= L.m) continue;
            const int mc = (L.m - d0) < MPMAX ? (L.m - d0) : MPMAX;
            k_dbank<<<dim3(L.nb * 8, MPMAX), 256, 0, s>>>(L.D, L.n, L.nb, mc, d0, MPMAX, L.dmax_bits, L.bf16,
                                                          L.kbank, L.jbank);
            if (L.nbricks == 0) continue;
            UmmaEntry &E = p.e[p.nentries++];
            E.bricks = L.bricks; E.nbricks = L.nbricks; E.offsets = L.offsets; E.store = L.store;
            E.kbank = L.kbank; E.jbank = L.jbank; E.part = L.part; E.nparts = L.nparts;
            E.nb = L.nb; E.m = mc; E.d0 = d0; E.mtot = L.m; E.bf16 = L.bf16;
            E.vscale = L.vscale; E.dmax_bits = L.dmax_bits; E.Jacc = L.Jacc; E.Kacc = L.Kacc;
            E.error = L.error;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) { set_error("k_dbank: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
        if (p.nentries == 0) continue;
        p.counter = Ls[0].counter;
        e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) { set_error("memset chunk counter: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
        k_jk_umma<<<grid, NTHREADS, SMEM_TOTAL, s>>>(p);
        e = cudaGetLastError();
        if (e != cudaSuccess) { set_error("k_jk_umma: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    }
    return ESMF_OK;
}

int umma_smem_bytes() { return SMEM_TOTAL; }
size_t umma_kbank_bytes(int nb) { return (size_t)nb * nb * KB_BYTES_MAX; }
size_t umma_jbank_bytes(int nb) { return (size_t)nb * (nb + 1) / 2 * JB_BYTES_MAX; }

int launch_jk_umma(const UmmaLaunch &L, cudaStream_t s) {
    // density tiles for chunks of at most 16 densities; one contraction pass per chunk
    const int64_t nn = (int64_t)L.n * L.n;
    cudaError_t e = cudaMemsetAsync(L.dmax_bits, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) { set_error("memset dmax: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    k_dmax<<<256, 256, 0, s>>>(L.D, (int64_t)L.m * nn, L.dmax_bits);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("k_dmax: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    e = cudaFuncSetAttribute(k_jk_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL);
    if (e != cudaSuccess) { set_error("smem attribute: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    const int chunk = (L.chunk == 8) ? 8 : MPMAX;
    for (int d0 = 0; d0 < L.m; d0 += chunk) {
        const int mc = (L.m - d0) < chunk ? (L.m - d0) : chunk;
        const int mp = mc <= 8 ? 8 : 16;
        k_dbank<<<dim3(L.nb * 8, mp), 256, 0, s>>>(L.D, L.n, L.nb, mc, d0, mp, L.dmax_bits, L.bf16, L.kbank, L.jbank);
        e = cudaGetLastError();
        if (e != cudaSuccess) { set_error("k_dbank: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
        if (L.nbricks == 0) continue;
        UmmaParams p;
        p.nentries = 1;
        p.mp = mp;
        UmmaEntry &E = p.e[0];
        E.bricks = L.bricks; E.nbricks = L.nbricks; E.offsets = L.offsets; E.store = L.store;
        E.kbank = L.kbank; E.jbank = L.jbank; E.part = L.part; E.nparts = L.nparts;
        E.nb = L.nb; E.m = mc; E.d0 = d0; E.mtot = L.m; E.bf16 = L.bf16;
        E.vscale = L.vscale; E.dmax_bits = L.dmax_bits; E.Jacc = L.Jacc; E.Kacc = L.Kacc;
        E.error = L.error;
        int grid = L.num_sms;
        if (grid > L.nbricks) grid = (int)L.nbricks;
        p.counter = L.counter;
        e = cudaMemsetAsync(L.counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) { set_error("memset chunk counter: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
        if (L.ev_start && d0 == 0) cudaEventRecord(L.ev_start, s);
        k_jk_umma<<<grid, NTHREADS, SMEM_TOTAL, s>>>(p);
        if (L.ev_stop && d0 + chunk >= L.m) cudaEventRecord(L.ev_stop, s);
        e = cudaGetLastError();
        if (e != cudaSuccess) { set_error("k_jk_umma: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    }
    return ESMF_OK;
}

// J from the lower block triangle of the block-major accumulators, F = 2J - K,
// t_k = sum_pq D_k[pq] F_k[pq]; outputs in the caller's [k][p][q] layout.  One
// block per (row p, density k), threads over the columns q.
__global__ void k_finalize_blocked(int n, int nb, int m, const double *D, const double *Jb,
                                   const double *Kb, double *J, double *K, double *F, double *tsum) {
    const int p = blockIdx.x, k = blockIdx.y;
    const int X = p >> 3, x = p & 7;
    const int64_t row = (int64_t)k * n * n + (int64_t)p * n;
    double part = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int Y = q >> 3, y = q & 7;
        const double jv = (X >= Y) ? Jb[(((int64_t)X * nb + Y) * m + k) * 64 + x * 8 + y]
                                   : Jb[(((int64_t)Y * nb + X) * m + k) * 64 + y * 8 + x];
        const double kv = Kb[(((int64_t)X * nb + Y) * m + k) * 64 + x * 8 + y];
        const double fv = 2.0 * jv - kv;
        J[row + q] = jv;
        K[row + q] = kv;
        if (F) F[row + q] = fv;
        part += D[row + q] * fv;
    }
    if (tsum) {
        __shared__ double red[8];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
            atomicAdd(tsum + k, sum);
        }
    }
}

int launch_finalize_blocked(const DevBasis &b, int m, const double *D, const double *Jb, const double *Kb,
                            double *J, double *K, double *F, double *tsum, cudaStream_t s) {
    if (b.n < 1 || m < 1) return ESMF_OK;
    const int threads = b.n <= 128 ? 128 : 256;
    k_finalize_blocked<<<dim3(b.n, m), threads, 0, s>>>(b.n, b.nb, m, D, Jb, Kb, J, K, F, tsum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("k_finalize_blocked: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    return ESMF_OK;
}

}  // namespace esmf
