/*
 * esmf_fock.h -- C ABI of the GB300 grouped generalized-Fock-build library.
 *
 * The library builds, for a batch of m generalized density matrices D_k
 * (closed-shell, open-shell or non-symmetric transition-like), the
 * generalized Coulomb and exchange matrices of Eq. (J_and_K), Sec. II.B.1:
 *
 *     J[D]_pq = sum_rs D_rs (rs|pq)
 *     K[D]_pq = sum_rs D_rs (pr|qs)
 *     F[D]_pq = 2 J[D]_pq - K[D]_pq
 *
 * with the two-electron integrals (pq|rs) in chemists' (1122) order over a
 * basis of contracted Gaussians (s functions; Cartesian p and d functions
 * through esmf_fock_create_cart), all m matrices in ONE pass over the
 * integrals ("grouping Fock builds", Sec. II.C), or over approximate
 * integrals by density fitting (esmf_fock_create_df) or tensor
 * hypercontraction (esmf_fock_create_thc), with Schwarz screening of
 * integral quartets (kept iff Q_pq * Q_rs >= tol, Q_pq = sqrt((pq|pq)); the
 * bound-based form of the shell-pair screening of Sec. II.C).  It also forms
 * the inner products t_k = D_k . F_k = sum_pq D_k,pq F_k,pq (Table I).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major N x N float64; a batch of m matrices is one
 *     contiguous array of m * N * N doubles, matrix k at offset k*N*N.
 *   - Pointers documented as "device" must be CUDA device (or managed)
 *     memory on the handle's device; "host" pointers are ordinary host
 *     memory (page-locked memory makes the host-buffer entry faster).
 *   - The caller owns every buffer it passes; the handle owns the integral,
 *     pair, Schwarz and work memory it allocates and frees it on destroy.
 *   - Functions return 0 (ESMF_OK) or a negative ESMF_ERR_* code; nothing
 *     throws.  esmf_strerror() names a code, esmf_last_error() gives the
 *     calling thread's most recent detailed message.
 *   - A handle may be used from one host thread at a time.
 */
#ifndef ESMF_FOCK_H
#define ESMF_FOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESMF_OK                 0
#define ESMF_ERR_INVALID_ARG   -1   /* bad size, pointer, exponent, NaN ...   */
#define ESMF_ERR_OOM           -2   /* device or host allocation failed       */
#define ESMF_ERR_CUDA          -3   /* a CUDA runtime call failed             */
#define ESMF_ERR_TIMEOUT       -4   /* a bounded wait expired                 */
#define ESMF_ERR_UNSUPPORTED   -5   /* mode/precision not available for input */

/* integral handling */
#define ESMF_MODE_STORED  0   /* screened unique integrals stored at create   */
#define ESMF_MODE_DIRECT  1   /* integrals recomputed inside every build      */
#define ESMF_MODE_AUTO    2   /* stored if it fits the device budget          */
#define ESMF_MODE_DF      3   /* density fitting (esmf_fock_create_df)        */
#define ESMF_MODE_THC     4   /* tensor hypercontraction (esmf_fock_create_thc) */

/* arithmetic of the integral x density products (accumulation is FP64) */
#define ESMF_PREC_FP64    0   /* FP64 integrals, FP64 products                */
#define ESMF_PREC_FP32    1   /* FP32 integrals and products, FP64 flushes    */
#define ESMF_PREC_FP16X2  2   /* integrals as scaled FP16 hi+lo pairs, tensor */
                              /* cores with FP32 accumulation (stored only)   */
#define ESMF_PREC_BF16X2  3   /* as FP16X2 with BF16 halves (ablation)        */
#define ESMF_PREC_F32X2   4   /* FP64 integrals contracted in double-FP32     */
                              /* (hi+lo) arithmetic on CUDA cores: error-free */
                              /* products (FMA) and compensated sums (TwoSum),*/
                              /* about 2^-44 relative, at FP32-pipe rates;    */
                              /* stored only                                   */

/*
 * Basis of N contracted s-type Gaussians.  All pointers are HOST memory,
 * read during esmf_fock_create only.
 *   n_basis  N > 0
 *   center   N x 3 Cartesian centers in bohr
 *   n_prim   N primitive counts, each in [1, ESMF_MAX_PRIM]
 *   exps     sum(n_prim) exponents in bohr^-2, finite and > 0, function by
 *            function in order
 *   coefs    sum(n_prim) unnormalised contraction coefficients (finite); the
 *            library normalises each primitive and each contraction to one.
 */
#define ESMF_MAX_PRIM 4
typedef struct {
    int32_t        n_basis;
    const double  *center;
    const int32_t *n_prim;
    const double  *exps;
    const double  *coefs;
} esmf_basis_t;

typedef struct esmf_fock esmf_fock_t;

typedef struct {
    int64_t n_basis;            /* N                                           */
    int64_t n_pairs;            /* N(N+1)/2                                    */
    int64_t n_quartets_unique;  /* P(P+1)/2, P = n_pairs                       */
    int64_t n_quartets_kept;    /* unique quartets with Q_pq Q_rs >= tol       */
    int64_t n_bricks;           /* kept 8x8x8x8 function-block quartets        */
    int64_t n_stored;           /* integrals held in the store (stored mode)   */
    int64_t store_bytes;        /* bytes of the integral store                 */
    int64_t device_bytes;       /* all device memory held by the handle        */
    int32_t mode;               /* ESMF_MODE_STORED, _DIRECT, _DF or _THC      */
    int32_t precision;          /* ESMF_PREC_*                                 */
    double  schwarz_tol;
    double  create_ms;          /* wall time of esmf_fock_create               */
    int32_t screening;          /* ESMF_SCREEN_*                               */
    int64_t n_pairs_kept;       /* pairs in at least one kept quartet          */
    int64_t n_chunks;           /* integral-direct FP16X2/BF16X2: chunks each  */
                                /* build regenerates (0 otherwise)             */
    int64_t scratch_bytes;      /* their scratch buffer (part of device_bytes) */
} esmf_stats_t;

/*
 * esmf_fock_create -- Sec. II.C screening set-up, run once per basis
 * ("at the beginning of an ESMF optimization"): normalises the basis,
 * builds primitive-pair data, the Schwarz table Q_pq = sqrt((pq|pq)) in
 * FP64, the list of kept 8x8x8x8 function-block quartets, and in stored
 * mode evaluates and stores every kept unique integral.
 *   basis        host description (above)
 *   schwarz_tol  >= 0; quartets with Q_pq Q_rs < tol are dropped, 0 keeps all
 *   mode         ESMF_MODE_*;   precision  ESMF_PREC_*
 *   device       CUDA device ordinal the handle lives on
 *   budget_bytes device-memory budget for AUTO mode (0 = no limit)
 *   out          receives the handle (NULL on failure)
 * Integral-direct handles in FP16X2 / BF16X2 (s bases) contract on the
 * tensor cores: every build evaluates the kept integrals in FP32 chunk by
 * chunk (whole items of the brick list, at most 2 GiB of split records per
 * chunk, or a quarter of budget_bytes when it is given) into a scratch buffer
 * the handle owns, and contracts each chunk with the tensor-core kernel of
 * the stored split precisions; the FP64 accumulators sum over the chunks.
 * Their CUDA-core path (ESMF_PATH_CUDA_CORE, density-weighted screening, the
 * no-allocation entry) is the FP32 integral-direct kernel.  ESMF_MODE_AUTO
 * keeps choosing FP32 integral-direct builds when a split store does not fit.
 * Runs on the device's legacy default stream and returns after it has
 * finished.  Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED (F32X2 requested in
 * direct mode, or stored mode beyond budget_bytes).
 */
int esmf_fock_create(const esmf_basis_t *basis, double schwarz_tol, int mode,
                     int precision, int device, int64_t budget_bytes,
                     esmf_fock_t **out);

/*
 * esmf_fock_create_screened -- esmf_fock_create with a choice of screening
 * rule (esmf_fock_create uses ESMF_SCREEN_SCHWARZ):
 *   ESMF_SCREEN_SCHWARZ   quartet (pq|rs) kept iff Q_pq Q_rs >= tol (the
 *                         Cauchy-Schwarz bound of the integral)
 *   ESMF_SCREEN_PAIR_MAX  the pair rule as Sec. II.C states it: pair (p, q)
 *                         is discarded when max_rs |(pq|rs)| <= tol (the
 *                         paper uses 1e-9), and every quartet of two
 *                         surviving pairs is kept.  The maximum is decided in
 *                         FP64 at create time (one warp per pair, searching
 *                         the pairs in descending Q order and stopping at
 *                         the first integral above tol or the first Schwarz
 *                         bound at or below it).
 * Other arguments, outputs and errors as esmf_fock_create (INVALID_ARG also
 * for an unknown screening value).  esmf_fock_schwarz still returns Q, and
 * the split-16-bit store scale is still chosen from max Q^2.
 */
#define ESMF_SCREEN_SCHWARZ   0
#define ESMF_SCREEN_PAIR_MAX  1
int esmf_fock_create_screened(const esmf_basis_t *basis, double tol, int screening,
                              int mode, int precision, int device,
                              int64_t budget_bytes, esmf_fock_t **out);

/*
 * esmf_fock_create_cart -- esmf_fock_create for a basis that mixes s, p and
 * d Cartesian functions, the angular momenta of polarised bases such as
 * cc-pVDZ (the paper's molecules use cc-pVDZ, Sec. III.A).  Function i has the
 * Cartesian label cart[i]: 0 for s, 1/2/3 for p_x/p_y/p_z, 4/5/6 for
 * d_xx/d_yy/d_zz and 7/8/9 for d_xy/d_xz/d_yz, i.e. primitives
 * (x - A_x)^lx (y - A_y)^ly (z - A_z)^lz exp(-a |r - A|^2), each component
 * normalised to one (each contraction to one); the functions of a shell are
 * listed separately with the same centre, exponents and coefficients.
 * Integrals come in FP64 from the Obara-Saika / Head-Gordon-Pople
 * recurrences (s and p quartets) and the McMurchie-Davidson scheme (quartets
 * with a d function), at create time for stored handles and inside every
 * build for integral-direct ones (a correctness path: the s-type direct
 * kernel is the fast one).  The Schwarz table, screening, store and every
 * build kernel are those of s bases (the contraction works on integral
 * values by function index), so all precisions and the tensor-core path
 * apply.
 *   cart     host array of n_basis labels in [0, 9] (all zero: an s basis)
 *   others   as esmf_fock_create, Schwarz screening
 * Errors: as esmf_fock_create; INVALID_ARG for a label outside [0, 9].
 * esmf_fock_create_df and the pair-max rule take s bases only.
 */
int esmf_fock_create_cart(const esmf_basis_t *basis, const int32_t *cart, double schwarz_tol,
                          int mode, int precision, int device, int64_t budget_bytes,
                          esmf_fock_t **out);

/*
 * esmf_fock_create_df -- a handle whose builds use density-fitted integrals,
 * the acceleration the paper names as future work (Sec. I), in the Coulomb-
 * metric form (pq|rs) ~ sum_PQ (pq|P) [V^-1]_PQ (Q|rs), V_PQ = (P|Q), over
 * auxiliary s Gaussians chi_P(r) = exp(-e_P |r - C_P|^2).  At create time the
 * three-centre integrals T_P,pq = (pq|P) and the metric V are evaluated on the
 * device in FP64, V = L L^T is factored on the host, and B = L^-1 T is formed
 * (one FP64 GEMM) and kept in the handle in the build arithmetic, in two
 * layouts ([P][p][q] and [p][P][q]).  Every build is then dense GEMMs:
 * J_k = B^T (B vec(D_k)) and K_k[p][q] = sum_{P,s} (B''_p D_k)[P][s] B''_q[P][s].
 * There is no integral screening; esmf_fock_build and esmf_fock_build_host
 * accept the handle (m densities per build as usual); the batched, shard,
 * no-alloc and autotune entries reject it (UNSUPPORTED).
 *   basis      as for esmf_fock_create
 *   aux        host description of the auxiliary set (read during this call)
 *   precision  ESMF_PREC_FP64 or ESMF_PREC_FP32 (GEMM arithmetic; the fit
 *              itself is always formed in FP64)
 *   device, out  as for esmf_fock_create
 * Device memory: about 2 n_aux N^2 elements for B and B'', plus n_aux N^2
 * elements of per-build work.  Errors: INVALID_ARG (bad basis or auxiliary
 * set, or a metric that is not positive definite), UNSUPPORTED (split 16-bit
 * precisions), OOM, CUDA.
 */
typedef struct {
    int32_t       n_aux;      /* number of auxiliary functions, > 0          */
    const double *center;     /* n_aux x 3 centres, bohr                      */
    const double *exps;       /* n_aux exponents, bohr^-2, finite and > 0     */
} esmf_aux_t;
int esmf_fock_create_df(const esmf_basis_t *basis, const esmf_aux_t *aux, int precision,
                        int device, esmf_fock_t **out);

/*
 * esmf_fock_create_thc -- a handle whose builds use least-squares tensor
 * hypercontraction (THC) of the integrals, the other acceleration the paper
 * names as future work (Sec. I), in the LS-THC form of Parrish, Hohenstein,
 * Martinez and Sherrill (J. Chem. Phys. 137, 224106, 2012):
 *   (pq|rs) ~ sum_PQ X_pP X_qP Z_PQ X_rQ X_sQ,   X_pP = phi_p(r_P),
 * over caller-chosen grid points r_P.  At create time, in FP64: the
 * collocation X on the device; the Coulomb matrix
 *   E_PQ = sum_pqrs X_pP X_qP (pq|rs) X_rQ X_sQ   (Schwarz-kept quartets)
 * from the library's own grouped builds over the rank-one densities
 * x_Q x_Q^T (an internal ESMF_MODE_AUTO FP64 handle with schwarz_tol and
 * budget_bytes, destroyed before return; 64 grid points per build);
 * S_PQ = (sum_p X_pP X_pQ)^2; and the regularised least-squares fit
 *   Z = (S + lam I)^-1 E (S + lam I)^-1,   lam = ridge * max_P S_PP,
 * through a host Cholesky factor of S + lam I and four device triangular
 * solves, symmetrised to the last bit.  Every build is then dense GEMMs and
 * elementwise kernels (Eq. J_and_K over the fitted integrals, any D):
 *   M_k = X^T D_k X,   J_k = X diag(Z diag(M_k)) X^T,   K_k = X (Z o M_k) X^T.
 * esmf_fock_build and esmf_fock_build_host accept the handle (m densities per
 * build as usual, in batches whose work fits about 1 GiB); the batched,
 * shard, no-alloc and autotune entries reject it (UNSUPPORTED).
 *   basis        as for esmf_fock_create (s functions)
 *   grid         host grid points (read during this call)
 *   schwarz_tol  >= 0: screening of the exact integrals behind E
 *   ridge        >= 0, finite: relative regularisation (0: the plain least-
 *                squares fit; 1e-8 keeps S + lam I conditioned to about 1e8,
 *                so that rounding in E and S moves J and K by ~1e-8 relative)
 *   precision    ESMF_PREC_FP64 or ESMF_PREC_FP32 (build GEMM arithmetic;
 *                the fit is always formed in FP64)
 *   device, budget_bytes, out   as for esmf_fock_create
 * esmf_fock_stats reports mode ESMF_MODE_THC, n_quartets_kept of the exact
 * integrals behind E, and store_bytes of X and Z.
 * Cost: the fit takes n_grid / 64 exact grouped builds and O(n_grid^3) host
 * work for the Cholesky factor.  Device memory: X (N n_grid) and Z
 * (n_grid^2) in the build arithmetic, plus per-build work of about
 * m (N n_grid + n_grid^2) elements (at most about 1 GiB); during create also
 * the internal handle and four n_grid^2 FP64 matrices.
 * Errors: INVALID_ARG (bad basis or grid, a negative or non-finite tol or
 * ridge, or S + lam I not numerically positive definite: grid points that
 * the others reproduce), UNSUPPORTED (split 16-bit precisions), OOM, CUDA,
 * TIMEOUT (a bounded wait of the fit's builds expired).
 */
#define ESMF_MAX_GRID 8192
typedef struct {
    int32_t       n_grid;     /* number of grid points, 1 .. ESMF_MAX_GRID   */
    const double *points;     /* n_grid x 3, bohr, finite                     */
} esmf_grid_t;
int esmf_fock_create_thc(const esmf_basis_t *basis, const esmf_grid_t *grid, double schwarz_tol,
                         double ridge, int precision, int device, int64_t budget_bytes,
                         esmf_fock_t **out);

/*
 * esmf_fock_build -- one grouped pass over the (stored or recomputed)
 * integrals building J_k and K_k for all k < m (Eq. J_and_K), then
 * optionally F_k = 2 J_k - K_k and t_k = D_k . F_k (Table I).
 *   h        handle from esmf_fock_create
 *   m        number of densities, 1 <= m <= ESMF_MAX_DENSITIES
 *   D        device, m x N x N, read only, any (non-symmetric) values
 *   J, K     device, m x N x N, overwritten (not accumulated)
 *   F        device, m x N x N or NULL
 *   traces   device, m doubles or NULL
 *   stream   cudaStream_t to run on (NULL = legacy default stream)
 * Asynchronous: returns once the work is queued; the results are ready
 * when the stream reaches that point.  The handle's work memory is reused
 * by the next build, so builds on one handle must not overlap on the GPU
 * (issue them on one stream, or synchronise in between).
 * Errors: INVALID_ARG, OOM (growing the work memory), CUDA.
 */
#define ESMF_MAX_DENSITIES 1024
int esmf_fock_build(esmf_fock_t *h, int m, const double *D, double *J,
                    double *K, double *F, double *traces, void *stream);

/*
 * esmf_fock_build_batch -- esmf_fock_build for several handles (molecules of
 * different sizes, each with its own density count) in ONE persistent
 * tensor-core launch per pass of 16 densities (a single launch when every
 * m <= 16): the CTAs take cost-balanced chunks of every handle's bricks
 * in turn, so small molecules share the GPU instead of each filling a launch
 * of its own.  The whole call allocates nothing once each handle has built
 * with at least its m before, and can then be captured in a CUDA graph.
 *   count   1 <= count <= ESMF_MAX_BATCH, distinct handles on one device, all
 *           created stored with ESMF_PREC_FP16X2 or ESMF_PREC_BF16X2 (the
 *           tensor-core path) and not switched to ESMF_PATH_CUDA_CORE
 *   h, m    count handles and their density counts (host arrays)
 *   D, J, K count device pointers each (host arrays of device pointers),
 *           laid out as for esmf_fock_build with that entry's N and m
 *   F, traces  NULL, or count device pointers each (entries may be NULL)
 *   stream  cudaStream_t (NULL = legacy default stream)
 * Asynchronous.  A device-side timeout (an expired bounded wait in the
 * launch) sets the error flag of EVERY handle of the batch, since a CTA that
 * gives up leaves its share of all of them unfinished; read each handle's flag
 * with esmf_fock_device_error.  Errors: INVALID_ARG, UNSUPPORTED (a
 * handle off the tensor-core path), OOM, CUDA.  The grouping of Sec. II.C
 * (all densities of one molecule in one pass over its integrals) is kept per
 * handle; batching across molecules has no counterpart in the paper.
 */
#define ESMF_MAX_BATCH 16
int esmf_fock_build_batch(int count, esmf_fock_t *const *h, const int *m,
                          const double *const *D, double *const *J, double *const *K,
                          double *const *F, double *const *traces, void *stream);

/*
 * esmf_fock_build_shard -- the part of esmf_fock_build contributed by shard
 * `shard` of `nshards` contiguous slices of the handle's kept brick list.
 * The slices hold equal shares of the estimated contraction cost (the
 * per-brick cost model of the tensor kernel's chunks), each cut moved to
 * the next item boundary of the brick order; on the tensor-core path each
 * shard gets its own cost-balanced chunks (formed on the first build of
 * that shard: that build allocates a few hundred bytes).  J, K, F and the
 * traces are linear in the integrals, so the element-wise sum of the outputs
 * of all shards (e.g. one all-reduce across GPUs, each holding a handle for
 * the same basis) equals the full build.  Same buffers, asynchrony and
 * errors as esmf_fock_build; INVALID_ARG for a bad shard; UNSUPPORTED for
 * density-fitted handles.
 */
int esmf_fock_build_shard(esmf_fock_t *h, int shard, int nshards, int m, const double *D,
                          double *J, double *K, double *F, double *traces, void *stream);

/*
 * esmf_fock_build_host -- the same build with HOST buffers: copies D to the
 * device, builds, copies J, K (and F, traces when non-NULL) back, and waits
 * for completion with a bounded wait of timeout_ms milliseconds (<= 0 means
 * 600000).  Host buffers: m x N x N doubles (traces: m doubles).
 * Errors: as esmf_fock_build, plus TIMEOUT if the wait expires (the work may
 * still be running; the handle must not be reused until it finishes).
 */
int esmf_fock_build_host(esmf_fock_t *h, int m, const double *D_host,
                         double *J_host, double *K_host, double *F_host,
                         double *traces_host, void *stream, int timeout_ms);

/*
 * esmf_fock_set_density_screening -- density-weighted screening for later
 * builds on this handle (0 turns it off; the default).  On top of the
 * create-time screening, a quartet is dropped from a build when
 *     Q_pq Q_rs max(W_rs, W_pq, W_qs, W_ps, W_qr, W_pr) < tol_d,
 *     W_xy = max over the build's densities k of max(|D_k[x][y]|, |D_k[y][x]|),
 * i.e. when every update of Eq. (J_and_K) it makes (each multiplies it by one
 * of those density elements, and |(pq|rs)| <= Q_pq Q_rs) is below tol_d in
 * magnitude.  The weights are formed on the device from each build's D; a
 * brick whose largest Schwarz product times largest weight is below tol_d is
 * skipped whole.  The paper screens by integral size only (Sec. II.C); this
 * is the density-weighted variant of the same Schwarz bound.  Builds with
 * screening on run the CUDA-core kernels (split 16-bit stores included) and
 * are not accepted by esmf_fock_build_batch (UNSUPPORTED) or
 * esmf_fock_build_noalloc (UNSUPPORTED: it needs per-build work memory).
 * Errors: INVALID_ARG (NULL handle, negative or non-finite tol_d),
 * UNSUPPORTED (density-fitted or hypercontracted handles: no quartets).
 */
int esmf_fock_set_density_screening(esmf_fock_t *h, double tol_d);

/*
 * Contraction kernel choice for split 16-bit stores (FP16X2 / BF16X2):
 * ESMF_PATH_AUTO uses the tensor-core kernel, ESMF_PATH_CUDA_CORE the
 * CUDA-core kernel (same results within rounding; kept as a cross-check).
 * Other precisions always use the CUDA-core kernels.  Errors: INVALID_ARG.
 */
#define ESMF_PATH_AUTO       0
#define ESMF_PATH_CUDA_CORE  1
int esmf_fock_set_path(esmf_fock_t *h, int path);

/*
 * esmf_fock_autotune -- pick the number of densities contracted per pass
 * over each brick tile for builds with m densities on this handle: times each
 * candidate (16 or 8 per tensor-core pass; 16/8/4 per CUDA-core pass for
 * FP32, 8/4 for FP64) as the median of `reps` builds (after one warm-up) on
 * the caller's device buffers D (read), J and K (overwritten), and records
 * the fastest; later builds with the same m use it.  *chosen (optional)
 * receives it.  Synchronises the stream.  Errors: as esmf_fock_build.
 */
int esmf_fock_autotune(esmf_fock_t *h, int m, const double *D, double *J, double *K, int reps,
                       void *stream, int *chosen);

/*
 * Device-side error flag of the handle: non-zero when a bounded wait inside
 * the tensor-core kernel expired (its results are then incomplete).  Read it
 * after the build has completed (stream synchronised); reset != 0 clears it.
 * esmf_fock_build_host checks it itself and returns ESMF_ERR_TIMEOUT.
 * Returns the flag (>= 0) or INVALID_ARG.
 */
int esmf_fock_device_error(esmf_fock_t *h, int reset);

/*
 * Kernel timing (measurement aid).  With timing enabled, each build records a
 * pair of CUDA events on its stream around its grouped contraction kernel
 * (the dominant kernel).  esmf_fock_kernel_time waits for the recorded
 * events, returns the summed milliseconds and the number of timed launches,
 * and clears the record when reset != 0.  At most 65536 launches are kept
 * between resets; later ones are not timed.  Errors: INVALID_ARG, CUDA.
 */
int esmf_fock_set_timing(esmf_fock_t *h, int enable);
int esmf_fock_kernel_time(esmf_fock_t *h, double *ms, int64_t *launches, int reset);

/*
 * esmf_fock_build_noalloc -- the build of esmf_fock_build for callers that
 * must not allocate device memory while they build: the host application
 * owns every device allocation through its own pool or fixed memory plan, or
 * the caller sits on a latency-critical path where cudaMalloc / cudaFree would
 * synchronise the device and stall unrelated streams.  The paper has no
 * counterpart; it is a property of this library's memory handling only.
 *
 * Same arguments and asynchrony as esmf_fock_build.  Stored FP64 and FP32
 * handles and integral-direct handles run the same CUDA-core kernels as
 * esmf_fock_build (with the handle's autotuned densities per pass), so the
 * results are the same.  Handles with split 16-bit stores (FP16X2 / BF16X2)
 * run the CUDA-core kernel over that store here, not the tensor-core kernel
 * (which needs per-handle density tiles in work memory): their results equal
 * esmf_fock_build's within the precision's tolerance (2e-6 relative for
 * FP16X2, 3e-5 for BF16X2), and the call is slower.  Integral-direct
 * FP16X2 / BF16X2 handles (which contract on the tensor cores in
 * esmf_fock_build) run the FP32 integral-direct CUDA-core kernel here: their
 * results equal esmf_fock_build's within the same tolerances.  The FP64 J/K
 * accumulators are taken from one static device array of
 * ESMF_NOALLOC_MAX_SCRATCH_DOUBLES doubles (32 MiB) that the library holds on
 * every device it is loaded on until the process exits; nothing is allocated
 * by this call.  It needs 2 * m * Np^2 doubles, Np = N rounded up to a
 * multiple of 8; larger requests are rejected with ESMF_ERR_INVALID_ARG.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current: make that first call
 * before any stream capture.  Every call clears and reuses the one array, so
 * calls through this entry point must not overlap on the GPU (one stream, or
 * synchronise in between); overlapping calls race and give wrong sums.
 * The handle itself comes from esmf_fock_create as usual.
 * Errors: INVALID_ARG (including the size limit), CUDA.
 */
#define ESMF_NOALLOC_MAX_SCRATCH_DOUBLES 4194304
int esmf_fock_build_noalloc(esmf_fock_t *h, int m, const double *D, double *J,
                            double *K, double *F, double *traces, void *stream);

/*
 * esmf_measure_fma_peak -- measured CUDA-core fused-multiply-add throughput of
 * a device, the denominator of the FP64 / FP32 ALU rooflines of the CUDA-core
 * contraction kernels (a measurement aid; the paper has no counterpart).
 * Runs independent FMA chains on every SM (grid a multiple of the SM count,
 * one warm-up launch, best of three timed with CUDA events on a private
 * stream) and writes the rate in TFLOP/s (2 flops per FMA) to *tflops.
 * Changes no clock, power or other device setting.  Takes about 0.5 s.
 *   precision  ESMF_PREC_FP64 or ESMF_PREC_FP32
 *   device     CUDA device ordinal
 * Errors: INVALID_ARG, CUDA.
 */
int esmf_measure_fma_peak(int precision, int device, double *tflops);

/* Statistics of a handle (host struct filled in).  Errors: INVALID_ARG. */
int esmf_fock_stats(const esmf_fock_t *h, esmf_stats_t *out);

/* Schwarz table: copies the N x N FP64 matrix Q_pq = sqrt((pq|pq)) into the
 * host array Q_host.  Errors: INVALID_ARG, CUDA. */
int esmf_fock_schwarz(const esmf_fock_t *h, double *Q_host);

/* Frees every device and host resource of the handle (NULL is a no-op).
 * Waits for the handle's outstanding work first. */
void esmf_fock_destroy(esmf_fock_t *h);

/* Static string naming a status code. */
const char *esmf_strerror(int status);

/* Most recent detailed error message of the calling host thread. */
const char *esmf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ESMF_FOCK_H */
