// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "esmf_fock.h"

namespace esmf {

// Function blocks of 8: a "brick" is the 8x8x8x8 block of integrals
// (P Q | R S) between four function blocks.  Bricks are kept in canonical
// form P >= Q, R >= S, pair(P,Q) >= pair(R,S); a brick stores every element
// (p q | r s) with p in P, q in Q, r in R, s in S at local index
// ((p*8 + q)*8 + r)*8 + s, of which only the Schwarz-kept ones are stored
// (packed, in local-index order).
// Split 16-bit store precisions (FP16X2, BF16X2): the tensor-core path.
inline bool is_split16(int prec) { return prec == ESMF_PREC_FP16X2 || prec == ESMF_PREC_BF16X2; }

constexpr int BLK = 8;
constexpr int BRICK = BLK * BLK * BLK * BLK;   // 4096
constexpr int MAXP = ESMF_MAX_PRIM;
constexpr int MAXPP = MAXP * MAXP;

struct BrickDesc {          // 16 bytes
    int16_t P, Q, R, S;     // function-block indices
    int32_t nkept;          // kept elements
    int32_t pad;            // bits 0/1: first/last brick of a run, bits 2/3: first/last of an item
};

// Brick order of a store: by bra block pair (P,Q), then by window of SWIN
// consecutive S blocks (an "item"), then R (a "run": fixed P, Q, R), then S.
// The brick (P Q | P Q) forms an item of its own.
constexpr int SWIN = 5;
enum : int { BRICK_RUN_FIRST = 1, BRICK_RUN_LAST = 2, BRICK_ITEM_FIRST = 4, BRICK_ITEM_LAST = 8 };

// Every stored record starts with a 512-byte keep mask (byte v = p*64 + q*8 +
// r, bit s), followed by the kept values in local-index order: FP64 or FP32
// values, or, for split 16-bit stores (FP16X2 / BF16X2), 32-bit words (hi
// half in the low 16 bits, lo half in the high 16 bits) of the value times
// one power of two (the handle's vscale).  The mask spans MASK_BYTES / eb
// store elements of eb bytes.
constexpr int MASK_BYTES = 512;
constexpr int MASK_WORDS = MASK_BYTES / 4;

// device view of the basis: functions padded to a multiple of BLK; padded
// functions have nprim = 0 and Q = 0 and are never kept
struct DevBasis {
    int n;          // real functions
    int np;         // padded
    int nb;         // blocks
    const double *center;  // np x 3
    const int *nprim;      // np
    const int *poff;       // np
    const double *exps;    // primitives
    const double *w;       // normalised raw-Gaussian weights
    const int *cart = nullptr;  // np Cartesian labels (0 s, 1..3 p_x..p_z); null: all s
};

void set_error(const char *fmt, ...);

// ---- setup.cu
int launch_normalize(const DevBasis &b, const double *coefs, double *w, cudaStream_t s);
int launch_schwarz(const DevBasis &b, double *Q, cudaStream_t s);
// pair rule of Sec. II.C into a 0/1 screening table S (np x np)
int launch_pair_rule(const DevBasis &b, const double *Q, double thr, const int2 *order, int64_t npairs, double *S,
                     cudaStream_t s);
int launch_brick_count(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                       int64_t nbricks, int32_t *counts, cudaStream_t s);
// ptab / pslot: the create-time primitive-pair table of the block pairs the
// bricks use (as for integral-direct handles); null: pairs formed per brick
int launch_brick_generate(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                          int64_t nbricks, const int64_t *offsets, int precision, void *store,
                          float vscale, cudaStream_t s, const void *ptab = nullptr, const int *pslot = nullptr);

// ---- angular.cu (bases with Cartesian p functions)
int launch_normalize_l(const DevBasis &b, const double *coefs, double *w, cudaStream_t s);
int launch_schwarz_l(const DevBasis &b, double *Q, cudaStream_t s);
int launch_brick_generate_l(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                            int64_t nbricks, const int64_t *offsets, int precision, void *store, float vscale,
                            cudaStream_t s);

// ---- jk_cuda.cu (CUDA-core contraction)
// primitive-pair table of integral-direct handles: one entry per function-
// block pair (B1, B2), B1 >= B2, that some kept brick uses as bra or ket
size_t pair_table_entry_bytes(int precision);
int launch_pair_table(const DevBasis &b, const int *blocks, int nentries, int precision, void *tab,
                      cudaStream_t s);

struct JKArgs {
    DevBasis b;
    const double *Q;
    double tol;
    const BrickDesc *bricks;
    int64_t nbricks;
    const int64_t *offsets;   // packed-store element offsets (stored mode)
    const void *store;
    int precision;
    int mode;
    int m;
    const double *D;          // m x n x n (caller layout)
    double *Jacc, *Kacc;      // m x np x np accumulators (zeroed by caller)
    float vscale;             // store scale of the split 16-bit precisions
    int mc = 0;               // densities per pass (0: default for the precision)
    const void *ptab = nullptr;     // direct mode: pair table (PairTable<TA> entries)
    const int *pslot = nullptr;     // direct mode: entry of block pair (B1, B2) at B1 * nb + B2
    // density-weighted screening (off when dw is null): dw = np x np weights
    // max_k max(|D_k[x][y]|, |D_k[y][x]|), dwb = nb x nb block maxima of dw
    const double *dw = nullptr, *dwb = nullptr;
    double tol_d = 0.0;
    // D in the contraction's arithmetic type (FP32 or double-FP32), formed once
    // per build; null: the kernel converts FP64 D as it loads its tiles
    const void *Dt = nullptr;
};
// bytes per element of the typed density copy of a precision (0: none, FP64)
size_t density_typed_bytes(int precision);
int launch_density_typed(int precision, int64_t cnt, const double *D, void *Dt, cudaStream_t s);
int launch_jk_cuda(const JKArgs &a, cudaStream_t s);
// density weights of one build for density-weighted screening (dwb zeroed here)
int launch_density_weight(const DevBasis &b, int m, const double *D, double *dw, double *dwb, cudaStream_t s);
int launch_jk_cuda_split(const JKArgs &a, cudaStream_t s);

// ---- jk_umma.cu (tensor-core contraction for split 16-bit stores)
struct UmmaLaunch {
    const BrickDesc *bricks;
    int64_t nbricks;
    const int64_t *offsets;
    const uint32_t *store;
    uint16_t *kbank, *jbank;     // density operand tiles (work memory)
    unsigned int *dmax_bits;     // work scalar
    const double *D;
    int n, np, nb, m, bf16, num_sms;
    float vscale;
    double *Jacc, *Kacc;         // block-major accumulators [X][Y][k][x][y]
    int *error;                  // device flag, 0 = ok
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;   // optional timing
    int chunk = 16;              // densities per tensor-core pass (8 or 16)
    const int64_t *part = nullptr;   // optional brick ranges (nparts + 1 entries) that CTAs take
    int nparts = 0;                  // dynamically, several per CTA
    unsigned *counter = nullptr;     // device work counter of the launch (zeroed per launch)
};
int launch_jk_umma(const UmmaLaunch &L, cudaStream_t s);
int launch_jk_umma_batch(const UmmaLaunch *Ls, int count, cudaStream_t s);   // count <= 16
int launch_finalize_blocked(const DevBasis &b, int m, const double *D, const double *Jb, const double *Kb,
                            double *J, double *K, double *F, double *tsum, cudaStream_t s);
int umma_smem_bytes();
size_t umma_kbank_bytes(int nb);
size_t umma_jbank_bytes(int nb);
int launch_finalize(const DevBasis &b, int m, const double *D, const double *Jacc,
                    const double *Kacc, double *J, double *K, double *F, double *tsum,
                    cudaStream_t s);

// ---- df.cu (density-fitted J and K)
struct DfBuild {
    void *cublas;
    int n, naux, m, fp32;
    const void *B, *B2;          // B[P][p][q] and B''[p][P][q] in the arithmetic type
    const double *D;             // caller's densities (m x n x n)
    void *Dt, *Jt, *Kt, *g, *Y;  // work: arithmetic-type D (FP32 only), J, K, g, Y
    double *J, *K, *F, *traces;  // caller's outputs
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
};
int launch_df_integrals(const DevBasis &b, int naux, const double *acen, const double *aexp, double *T, double *V,
                        cudaStream_t s);
int launch_df_layouts(int naux, int n, const double *B, int fp32, void *Bout, void *B2, cudaStream_t s);
int df_gemm_fold(void *cublas, int naux, int64_t nn, const double *Linv, const double *T, double *B, cudaStream_t s);
int df_build(const DfBuild &a, cudaStream_t s);
int df_cublas_create(void **out);
void df_cublas_destroy(void *h);
// F = 2 J - K and t_k = D_k . F_k from the arithmetic-type Jt, Kt of a
// factored (density-fitted or hypercontracted) build of m densities; writes
// the caller's FP64 J, K (and F), zeroes and fills the traces
int launch_factored_finalize(int n, int m, int fp32, const double *D, const void *Jt, const void *Kt, double *J,
                             double *K, double *F, double *traces, cudaStream_t s);

// ---- thc.cu (tensor hypercontraction)
struct ThcBuild {
    void *cublas;
    int n, G, m, fp32;
    const void *X, *Z;           // X[p][P] (n x G) and Z[P][Q] (G x G) in the arithmetic type
    const double *D;             // caller's densities (m x n x n)
    void *Dt, *A, *M, *y, *z, *Jt, *Kt;   // work for m densities (see thc_build)
    double *J, *K, *F, *traces;  // caller's outputs
};
int launch_thc_collocate(const DevBasis &b, int G, const double *pts, double *X, cudaStream_t s);
int launch_thc_rank_one(int n, int G, int q0, int mq, const double *X, double *Dq, cudaStream_t s);
int thc_coulomb_columns(void *cublas, int n, int G, int q0, int mq, const double *X, const double *Jq, double *R,
                        double *E, cudaStream_t s);
int thc_gram(void *cublas, int n, int G, const double *X, double *C, cudaStream_t s);
int thc_solve_z(void *cublas, int G, const double *L, double *W, int fp32, void *Zout, cudaStream_t s);
int launch_thc_convert(int64_t cnt, const double *src, float *dst, cudaStream_t s);
int thc_build(const ThcBuild &a, cudaStream_t s);

// ---- energy.cu (ESMF energy and gradient around the grouped build)
struct EnergyWork {
    double *D, *J, *K, *F;               // 3 x N x N each: P, T, A and their J, K, F
    double *Fk, *M1, *Wc, *Wm;           // N x N
    double *X1, *X2, *X3, *R1, *R2, *R3; // N_o x N
    double *X4, *Rg1, *Rg2;              // N_v x N
    double *Z1a, *Z1b, *Z1c, *Z3, *Z2;   // N_o x N_v (four), N_o x N_o
    double *partial, *sc;                // reduction partials; {E_HF, E, N2}
};
// GVP objective (second pass): the gradient kept internally and the tangent
// (directional-derivative) copies of the energy intermediates
struct GvpWork {
    double *gs, *gV, *scE;               // dE/dsigma (N_o x N_v), dE/dV (N x N), {E, dE/dc0}
    double *Gam, *Gx, *Vt, *Wct, *Wmt;   // N x N
    double *Dt, *Jt, *Kt, *Ft;           // 3 x N x N each: P', T', A' and their J, K, F
    double *M1t, *Mt, *Dd;               // N x N
    double *X1, *X2, *X3, *R1, *R2, *R3; // tangents, N_o x N
    double *X4, *Rg1, *Rg2;              // tangents, N_v x N
    double *Z1a, *Z1b, *Z1c, *Z3, *Hs;   // N_o x N_v
    double *Z2;                          // N_o x N_o
    double *partial, *st;                // dot partials; tangent scalars
};
size_t gvp_work_doubles(int n, int no);
GvpWork gvp_work_layout(double *base, int n, int no);
int launch_gvp_tangent_densities(int n, int no, const double *V, const double *sigma, const EnergyWork &w,
                                 const GvpWork &v, cudaStream_t s);
int launch_gvp_finish(int n, int no, double c0, double omega, double mu, double chi, const double *G,
                      const double *V, const double *sigma, const EnergyWork &w, const GvpWork &v,
                      double *scalars, double *dLs, double *dLX, cudaStream_t s);
size_t energy_work_doubles(int n, int no);
EnergyWork energy_work_layout(double *base, int n, int no);
int launch_energy_densities(int n, int no, const double *V, const double *sigma, const EnergyWork &w,
                            cudaStream_t s);
int launch_energy_finish(int n, int no, double c0, const double *G, const double *V, const double *sigma,
                         const EnergyWork &w, double *scalars, double *dsig, double *dV, cudaStream_t s);

}  // namespace esmf
