// C ABI of the grouped generalized-Fock-build library (declared in
// include/esmf_fock.h).  Host-side orchestration only: argument checks,
// device memory ownership, the kept-brick list, and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "esmf_energy.h"
#include "esmf_internal.cuh"

namespace esmf {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace esmf

using namespace esmf;

struct esmf_fock {
    int device = 0;
    int n = 0, np = 0, nb = 0;
    double tol = 0.0;
    int mode = ESMF_MODE_STORED, prec = ESMF_PREC_FP64;
    // basis (device)
    double *center = nullptr, *exps = nullptr, *w = nullptr, *coefs = nullptr;
    int *nprim = nullptr, *poff = nullptr;
    int *cart = nullptr;           // Cartesian labels (device, np), null when every function is s
    double *Q = nullptr;
    // screening table and threshold of the quartet rule S_pq S_rs >= tol_s:
    // the Schwarz table itself (S = Q, tol_s = tol), or the 0/1 table of the
    // paper's pair rule (tol_s = 0.5)
    double *S = nullptr;
    double tol_s = 0.0;
    int screening = ESMF_SCREEN_SCHWARZ;
    int64_t n_pairs_kept = 0;
    // bricks and store (device)
    BrickDesc *bricks = nullptr;
    int64_t nbricks = 0;
    int64_t *offsets = nullptr;
    void *store = nullptr;
    // integral-direct mode: primitive-pair table, one entry per block pair a
    // kept brick uses (entry of (B1, B2) at pslot[B1 * nb + B2])
    void *ptab = nullptr;
    int *pslot = nullptr, *pblocks = nullptr;
    int n_ptab = 0;
    float vscale = 1.0f;           // power-of-two scale of split 16-bit stores
    // integral-direct builds on the tensor cores (FP16X2 / BF16X2 direct
    // handles): the brick list cut at item boundaries into chunks whose packed
    // records fit the scratch buffer; chunk c is bricks [chunks[c], chunks[c+1]),
    // its records regenerated into `scratch` by every build (offsets above are
    // then relative to the chunk's first brick).  Generation and contraction
    // of a chunk are not overlapped with the next chunk's: both kernels fill
    // every SM, so on two streams they only interleave (measured no faster).
    std::vector<int64_t> chunks;
    void *scratch = nullptr;
    int64_t scratch_bytes = 0;
    int path = ESMF_PATH_AUTO;
    // density-weighted screening threshold (0: off) and its per-build weights
    double tol_d = 0.0;
    double *dw = nullptr, *dwb = nullptr;
    // density fitting (mode ESMF_MODE_DF): auxiliary set, fitted factor in two
    // layouts (arithmetic type), per-build work for up to df_m densities
    void *cublas = nullptr;
    int naux = 0;
    void *dfB = nullptr, *dfB2 = nullptr;
    void *dfDt = nullptr, *dfJt = nullptr, *dfKt = nullptr, *dfg = nullptr, *dfY = nullptr;
    int df_m = 0;
    // tensor hypercontraction (mode ESMF_MODE_THC): grid size, collocation X
    // and fitted Z (arithmetic type), per-build work for up to thc_m densities
    int thc_G = 0;
    void *thcX = nullptr, *thcZ = nullptr;
    void *thcDt = nullptr, *thcA = nullptr, *thcM = nullptr, *thcy = nullptr, *thcz = nullptr;
    void *thcJt = nullptr, *thcKt = nullptr;
    int thc_m = 0;
    std::vector<std::pair<int, int>> tuned;   // (m, densities per pass) picked by esmf_fock_autotune
    int force_chunk = 0;                      // set while the autotuner times a candidate
    int num_sms = 0;
    // cost-balanced chunks of the whole brick list for the tensor kernel:
    // chunk g is bricks [parts[g], parts[g+1]) (device, nparts + 1), and the
    // kernel's CTAs take chunks dynamically
    int64_t *parts = nullptr;
    int nparts = 0;
    // host copy of the brick list's estimated cost prefix (cost_prefix[i] =
    // cost of bricks [0, i)) and item starts, for cost-balanced shards; the
    // chunks of each shard's range are built on first use
    std::vector<double> cost_prefix;
    std::vector<BrickDesc> hbricks;
    std::map<std::pair<int64_t, int64_t>, std::pair<int64_t *, int>> shard_parts;
    // tensor-core path work memory
    uint16_t *kbank = nullptr, *jbank = nullptr;
    unsigned int *dmax = nullptr;
    unsigned *sched = nullptr;     // the tensor kernel's work counter
    int *err_host = nullptr, *err_dev = nullptr;   // mapped page-locked flag
    int64_t n_stored = 0, store_bytes = 0, n_kept_unique = 0;
    // work (device)
    double *Jacc = nullptr, *Kacc = nullptr;
    void *Dt = nullptr;            // D in the CUDA-core arithmetic type (FP32 / double-FP32), work_m densities
    double *ework = nullptr;       // ESMF energy / gradient work memory
    size_t ework_n = 0;
    int work_m = 0;
    // staging for the host-buffer entry (device)
    double *sD = nullptr, *sJ = nullptr, *sK = nullptr, *sF = nullptr, *st = nullptr;
    int stage_m = 0;
    cudaEvent_t done = nullptr;
    // optional kernel timing
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    size_t ev_used = 0;
    int64_t device_bytes = 0;
    double create_ms = 0.0;

    DevBasis dev() const {
        DevBasis b;
        b.n = n; b.np = np; b.nb = nb;
        b.center = center; b.nprim = nprim; b.poff = poff; b.exps = exps; b.w = w;
        b.cart = cart;
        return b;
    }
};

// Most runs (R blocks) per item of the tensor-core brick order (see below).
// Whole-row parity of the 400-function, 64-density build against the FP64
// oracle set it: the worst relative K error over the densities was 2.1e-6
// at 32 runs, 1.1e-6 at 16 (3.7 % slower there, 1 % at 200 functions) and
// 7.0e-7 at 8 (15 % slower).
#ifndef ESMF_ITEM_RUNS
#define ESMF_ITEM_RUNS 16
#endif

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CKR(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                    \
            return e_ == cudaErrorMemoryAllocation ? ESMF_ERR_OOM : ESMF_ERR_CUDA; \
        }                                                                          \
    } while (0)

#define RET(x)                                                                     \
    do {                                                                           \
        int r_ = (x);                                                              \
        if (r_ != ESMF_OK) return r_;                                              \
    } while (0)

template <typename T>
int dalloc(esmf_fock *h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? ESMF_ERR_OOM : ESMF_ERR_CUDA;
    }
    h->device_bytes += (int64_t)(count * sizeof(T));
    return ESMF_OK;
}

template <typename T>
void dfree(esmf_fock *h, T **p, size_t count) {
    if (*p) {
        cudaFree(*p);
        h->device_bytes -= (int64_t)((count ? count : 1) * sizeof(T));
    }
    *p = nullptr;
}

// Relative cost of each brick in the tensor-core contraction, for cutting the
// list into chunks: a base cost, one unit per issued exchange/Coulomb view and
// one per output block whose flush the brick triggers (its Coulomb J2 block;
// at a run end the run's V1/V2 blocks; at an item end the J1 block and the
// window's V3/V4 blocks).  The coefficients came from a least-squares fit of
// per-CTA cycle counts on GB300 (stored_n200_m16, 152 CTAs); the chunks are
// taken dynamically, so the model only has to keep them of similar size.
constexpr double kCostBrick = 1900.0, kCostView = 100.0, kCostBlock = 840.0;

std::vector<double> cost_prefix(const std::vector<BrickDesc> &kept) {
    const int64_t n = (int64_t)kept.size();
    std::vector<double> pre(n + 1, 0.0);
    unsigned t3 = 0, t4 = 0;
    for (int64_t i = 0; i < n; ++i) {
        const BrickDesc &d = kept[i];
        const bool pq = d.P != d.Q, rs = d.R != d.S, diag = d.R == d.P && d.S == d.Q;
        const int two = diag ? 1 : 2;
        if (d.pad & BRICK_ITEM_FIRST) t3 = t4 = 0;
        if (rs) t3 |= 1u << (d.S % SWIN);
        if (rs && pq) t4 |= 1u << (d.S % SWIN);
        double blocks = diag ? 0 : 1;
        if (d.pad & BRICK_RUN_LAST) blocks += two + (pq ? two : 0);
        if (d.pad & BRICK_ITEM_LAST) blocks += 1 + two * (__builtin_popcount(t3) + __builtin_popcount(t4));
        const int views = 2 + (pq ? 1 : 0) + (rs ? 1 : 0) + (pq && rs ? 1 : 0);
        pre[i + 1] = pre[i] + kCostBrick + kCostView * views + kCostBlock * blocks;
    }
    return pre;
}

// Brick ranges of equal estimated cost for the tensor kernel, kChunksPerSM
// per SM: its CTAs take them dynamically (a launch-wide counter), so a CTA
// that runs slow for reasons the cost model does not see takes fewer.
constexpr int kChunksPerSM = 4;

std::vector<int64_t> balance_parts(const std::vector<BrickDesc> &kept, int G) {
    const int64_t n = (int64_t)kept.size();
    if (G > n) G = (int)n;
    std::vector<int64_t> parts;
    if (G < 1) return parts;
    const std::vector<double> pre = cost_prefix(kept);
    parts.resize(G + 1);
    parts[0] = 0;
    int64_t j = 0;
    for (int g = 1; g < G; ++g) {
        const double target = pre[n] * g / G;
        while (j < n && pre[j] < target) ++j;
        // cuts need not fall on item starts: a chunk that splits an item
        // flushes the item's resident output blocks at its end, and cutting at
        // item starts instead leaves chunks too uneven where items are about
        // as long as chunks (measured slower)
        parts[g] = std::max(j, parts[g - 1] + 1);      // every chunk gets a brick
    }
    parts[G] = n;
    for (int g = G - 1; g >= 1; --g) parts[g] = std::min(parts[g], parts[g + 1] - 1);
    return parts;
}

void release(esmf_fock *h) {
    if (!h) return;
    cudaFree(h->center); cudaFree(h->exps); cudaFree(h->w); cudaFree(h->coefs);
    cudaFree(h->nprim); cudaFree(h->poff); cudaFree(h->cart);
    if (h->S != h->Q) cudaFree(h->S);
    cudaFree(h->Q);
    cudaFree(h->bricks); cudaFree(h->offsets); cudaFree(h->store); cudaFree(h->parts); cudaFree(h->scratch);
    for (auto &sp : h->shard_parts) cudaFree(sp.second.first);
    cudaFree(h->ptab); cudaFree(h->pslot); cudaFree(h->pblocks);
    cudaFree(h->kbank); cudaFree(h->jbank); cudaFree(h->dmax); cudaFree(h->sched);
    if (h->err_host) cudaFreeHost(h->err_host);
    cudaFree(h->Jacc); cudaFree(h->Kacc); cudaFree(h->ework); cudaFree(h->Dt);
    cudaFree(h->dw); cudaFree(h->dwb);
    cudaFree(h->dfB); cudaFree(h->dfB2); cudaFree(h->dfDt); cudaFree(h->dfJt); cudaFree(h->dfKt);
    cudaFree(h->dfg); cudaFree(h->dfY);
    cudaFree(h->thcX); cudaFree(h->thcZ); cudaFree(h->thcDt); cudaFree(h->thcA); cudaFree(h->thcM);
    cudaFree(h->thcy); cudaFree(h->thcz); cudaFree(h->thcJt); cudaFree(h->thcKt);
    df_cublas_destroy(h->cublas);
    cudaFree(h->sD); cudaFree(h->sJ); cudaFree(h->sK); cudaFree(h->sF); cudaFree(h->st);
    if (h->done) cudaEventDestroy(h->done);
    for (auto &e : h->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    delete h;
}

bool is_finite(double x) { return std::isfinite(x); }

int elem_bytes(int prec) {
    switch (prec) {
        case ESMF_PREC_FP64: return 8;
        case ESMF_PREC_FP32: return 4;
        case ESMF_PREC_F32X2: return 8;     // FP64 values as FP32 hi + lo pairs
        default: return 4;   // hi+lo 16-bit pair
    }
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// integral-direct handle whose builds regenerate split 16-bit records chunk by
// chunk and contract them on the tensor cores
bool tensor_direct(const esmf_fock *h) { return h->mode == ESMF_MODE_DIRECT && is_split16(h->prec) && h->scratch; }

int ensure_work(esmf_fock *h, int m) {
    if ((h->mode == ESMF_MODE_STORED || tensor_direct(h)) && is_split16(h->prec) && !h->kbank) {
        RET(dalloc(h, (unsigned char **)&h->kbank, umma_kbank_bytes(h->nb)));
        RET(dalloc(h, (unsigned char **)&h->jbank, umma_jbank_bytes(h->nb)));
        RET(dalloc(h, &h->dmax, 1));
        RET(dalloc(h, &h->sched, 1));
    }
    if (h->tol_d > 0.0 && !h->dw) {
        RET(dalloc(h, &h->dw, (size_t)h->np * h->np));
        RET(dalloc(h, &h->dwb, (size_t)h->nb * h->nb));
    }
    if (m <= h->work_m) return ESMF_OK;
    const size_t cnt = (size_t)m * h->np * h->np;
    const size_t tb = density_typed_bytes(h->prec);
    dfree(h, &h->Jacc, (size_t)h->work_m * h->np * h->np);
    dfree(h, &h->Kacc, (size_t)h->work_m * h->np * h->np);
    dfree(h, (unsigned char **)&h->Dt, (size_t)h->work_m * h->n * h->n * tb);
    h->work_m = 0;
    RET(dalloc(h, &h->Jacc, cnt));
    RET(dalloc(h, &h->Kacc, cnt));
    if (tb) RET(dalloc(h, (unsigned char **)&h->Dt, (size_t)m * h->n * h->n * tb));
    h->work_m = m;
    return ESMF_OK;
}

// Checks of a basis description (host memory); sets *nprim_tot.
int check_basis(const esmf_basis_t *basis, int64_t *nprim_tot_out) {
    if (!basis || basis->n_basis <= 0 || !basis->center || !basis->n_prim || !basis->exps ||
        !basis->coefs) {
        set_error("basis missing or empty");
        return ESMF_ERR_INVALID_ARG;
    }
    const int n = basis->n_basis;
    if (n > 8 * 32767) { set_error("n_basis %d too large", n); return ESMF_ERR_INVALID_ARG; }
    int64_t nprim_tot = 0;
    for (int i = 0; i < n; ++i) {
        const int k = basis->n_prim[i];
        if (k < 1 || k > ESMF_MAX_PRIM) { set_error("n_prim[%d] = %d outside [1, %d]", i, k, ESMF_MAX_PRIM); return ESMF_ERR_INVALID_ARG; }
        for (int x = 0; x < 3; ++x)
            if (!is_finite(basis->center[3 * i + x])) { set_error("center[%d] not finite", i); return ESMF_ERR_INVALID_ARG; }
        nprim_tot += k;
    }
    for (int64_t j = 0; j < nprim_tot; ++j) {
        if (!(basis->exps[j] > 0.0) || !is_finite(basis->exps[j])) { set_error("exps[%lld] must be finite and > 0", (long long)j); return ESMF_ERR_INVALID_ARG; }
        if (!is_finite(basis->coefs[j])) { set_error("coefs[%lld] not finite", (long long)j); return ESMF_ERR_INVALID_ARG; }
    }
    // every contraction must have a positive norm
    {
        int64_t o = 0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < basis->n_prim[i]; ++k)
                for (int l = 0; l < basis->n_prim[i]; ++l) {
                    const double ak = basis->exps[o + k], al = basis->exps[o + l];
                    s += basis->coefs[o + k] * basis->coefs[o + l] * std::pow(2.0 * std::sqrt(ak * al) / (ak + al), 1.5);
                }
            if (!(s > 0.0)) { set_error("contraction %d has zero norm", i); return ESMF_ERR_INVALID_ARG; }
            o += basis->n_prim[i];
        }
    }
    *nprim_tot_out = nprim_tot;
    return ESMF_OK;
}

// Device copies of the basis (padded to the block size), normalised weights
// and the Schwarz table, on stream cs.
int upload_basis(esmf_fock *h, const esmf_basis_t *basis, int64_t nprim_tot, cudaStream_t cs,
                 const int32_t *cart = nullptr) {
    const int n = h->n, np = h->np;
    int rc;
    std::vector<int> hcart;
    if (cart) {
        hcart.assign(np, 0);
        for (int i = 0; i < n; ++i) hcart[i] = cart[i];
        if ((rc = dalloc(h, &h->cart, np))) return rc;
        CKR(cudaMemcpyAsync(h->cart, hcart.data(), sizeof(int) * np, cudaMemcpyHostToDevice, cs));
    }
    std::vector<double> hc((size_t)np * 3, 0.0);
    std::vector<int> hn(np, 0), ho(np, 0);
    std::memcpy(hc.data(), basis->center, sizeof(double) * 3 * n);
    int64_t o = 0;
    for (int i = 0; i < np; ++i) {
        ho[i] = (int)o;
        if (i < n) { hn[i] = basis->n_prim[i]; o += hn[i]; }
    }
    if ((rc = dalloc(h, &h->center, (size_t)np * 3)) || (rc = dalloc(h, &h->nprim, np)) ||
        (rc = dalloc(h, &h->poff, np)) || (rc = dalloc(h, &h->exps, nprim_tot)) ||
        (rc = dalloc(h, &h->coefs, nprim_tot)) || (rc = dalloc(h, &h->w, nprim_tot)) ||
        (rc = dalloc(h, &h->Q, (size_t)np * np)))
        return rc;
    CKR(cudaMemcpyAsync(h->center, hc.data(), sizeof(double) * np * 3, cudaMemcpyHostToDevice, cs));
    CKR(cudaMemcpyAsync(h->nprim, hn.data(), sizeof(int) * np, cudaMemcpyHostToDevice, cs));
    CKR(cudaMemcpyAsync(h->poff, ho.data(), sizeof(int) * np, cudaMemcpyHostToDevice, cs));
    CKR(cudaMemcpyAsync(h->exps, basis->exps, sizeof(double) * nprim_tot, cudaMemcpyHostToDevice, cs));
    CKR(cudaMemcpyAsync(h->coefs, basis->coefs, sizeof(double) * nprim_tot, cudaMemcpyHostToDevice, cs));
    const DevBasis db = h->dev();
    if (h->cart) {
        RET(launch_normalize_l(db, h->coefs, h->w, cs));
        RET(launch_schwarz_l(db, h->Q, cs));
    } else {
        RET(launch_normalize(db, h->coefs, h->w, cs));
        RET(launch_schwarz(db, h->Q, cs));
    }
    // the host copies above must outlive the copies
    CKR(cudaStreamSynchronize(cs));
    return ESMF_OK;
}

}  // namespace

static int create_impl(const esmf_basis_t *basis, const int32_t *cart, double tol, int screening, int mode,
                       int precision, int device, int64_t budget_bytes, esmf_fock_t **out);

extern "C" {

const char *esmf_strerror(int status) {
    switch (status) {
        case ESMF_OK: return "ok";
        case ESMF_ERR_INVALID_ARG: return "invalid argument";
        case ESMF_ERR_OOM: return "out of memory";
        case ESMF_ERR_CUDA: return "CUDA error";
        case ESMF_ERR_TIMEOUT: return "timed out";
        case ESMF_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *esmf_last_error(void) { return g_err; }

int esmf_fock_create(const esmf_basis_t *basis, double tol, int mode, int precision, int device,
                     int64_t budget_bytes, esmf_fock_t **out) {
    return esmf_fock_create_screened(basis, tol, ESMF_SCREEN_SCHWARZ, mode, precision, device, budget_bytes, out);
}

int esmf_fock_create_screened(const esmf_basis_t *basis, double tol, int screening, int mode, int precision,
                              int device, int64_t budget_bytes, esmf_fock_t **out) {
    return create_impl(basis, nullptr, tol, screening, mode, precision, device, budget_bytes, out);
}

int esmf_fock_create_cart(const esmf_basis_t *basis, const int32_t *cart, double tol, int mode, int precision,
                          int device, int64_t budget_bytes, esmf_fock_t **out) {
    if (!basis || !cart || basis->n_basis <= 0) { set_error("basis and cart are required"); return ESMF_ERR_INVALID_ARG; }
    bool any_p = false;
    for (int i = 0; i < basis->n_basis; ++i) {
        if (cart[i] < 0 || cart[i] > 9) { set_error("cart[%d] = %d outside [0, 9]", i, cart[i]); return ESMF_ERR_INVALID_ARG; }
        any_p |= cart[i] != 0;
    }
    if (!any_p) cart = nullptr;          // all s: the s-type path
    return create_impl(basis, cart, tol, ESMF_SCREEN_SCHWARZ, mode, precision, device, budget_bytes, out);
}

}  // extern "C"

static int create_impl(const esmf_basis_t *basis, const int32_t *cart, double tol, int screening, int mode,
                       int precision, int device, int64_t budget_bytes, esmf_fock_t **out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) { set_error("out is NULL"); return ESMF_ERR_INVALID_ARG; }
    if (screening != ESMF_SCREEN_SCHWARZ && screening != ESMF_SCREEN_PAIR_MAX) {
        set_error("bad screening %d", screening);
        return ESMF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!basis) { set_error("basis missing or empty"); return ESMF_ERR_INVALID_ARG; }
    if (!(tol >= 0.0) || !is_finite(tol)) { set_error("schwarz_tol must be finite and >= 0"); return ESMF_ERR_INVALID_ARG; }
    if (mode < ESMF_MODE_STORED || mode > ESMF_MODE_AUTO) { set_error("bad mode %d", mode); return ESMF_ERR_INVALID_ARG; }
    if (precision < ESMF_PREC_FP64 || precision > ESMF_PREC_F32X2) { set_error("bad precision %d", precision); return ESMF_ERR_INVALID_ARG; }
    if (budget_bytes < 0) { set_error("budget_bytes < 0"); return ESMF_ERR_INVALID_ARG; }
    const int n = basis->n_basis;
    int64_t nprim_tot = 0;
    RET(check_basis(basis, &nprim_tot));
    if (mode == ESMF_MODE_DIRECT && (precision == ESMF_PREC_F32X2 || (is_split16(precision) && cart))) {
        set_error("double-FP32 needs stored integrals, and split 16-bit integral-direct builds take s bases");
        return ESMF_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("device %d not available (%d devices)", device, ndev);
        return ESMF_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    if (!g.ok) { set_error("cudaSetDevice(%d) failed", device); return ESMF_ERR_CUDA; }

    esmf_fock *h = new (std::nothrow) esmf_fock();
    if (!h) { set_error("host allocation failed"); return ESMF_ERR_OOM; }
    h->device = device; h->n = n; h->tol = tol; h->prec = precision; h->screening = screening;
    h->nb = (n + BLK - 1) / BLK;
    h->np = h->nb * BLK;
    const int np = h->np;
    // create runs on a private non-blocking stream so that it does not wait for
    // (or stall) builds of other handles running on other streams
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error("cudaStreamCreate failed");
        return ESMF_ERR_CUDA;
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } cs_guard{cs};
    auto fail = [&](int code) { cudaStreamSynchronize(cs); cudaGetLastError(); release(h); return code; };
    int rc;

    if ((rc = upload_basis(h, basis, nprim_tot, cs, cart))) return fail(rc);
    cudaStream_t s = cs;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess) { set_error("%s: %s", what, cudaGetErrorString(e)); return false; }
        return true;
    };
    const DevBasis db = h->dev();
    std::vector<double> hQ((size_t)np * np);
    if (!ck(cudaMemcpyAsync(hQ.data(), h->Q, sizeof(double) * np * np, cudaMemcpyDeviceToHost, cs), "copy Q") ||
        !ck(cudaStreamSynchronize(cs), "Schwarz table"))
        return fail(ESMF_ERR_CUDA);
    // the screening table: Schwarz (S = Q, keep Q_pq Q_rs >= tol), or the pair
    // rule (S_pq = 1 iff max_rs |(pq|rs)| > tol, keep S_pq S_rs >= 0.5)
    std::vector<double> hS;
    if (screening == ESMF_SCREEN_SCHWARZ) {
        h->S = h->Q;
        h->tol_s = tol;
        // pairs that take part in at least one kept quartet: Q_pq max Q >= tol
        double qmax = 0.0;
        for (double x : hQ) qmax = std::max(qmax, x);
        int64_t cnt = 0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q <= p; ++q) cnt += hQ[(size_t)p * np + q] * qmax >= tol ? 1 : 0;
        h->n_pairs_kept = cnt;
    } else {
        std::vector<int2> order;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q <= p; ++q) order.push_back(make_int2(p, q));
        std::stable_sort(order.begin(), order.end(), [&](const int2 &x, const int2 &y) {
            return hQ[(size_t)x.x * np + x.y] > hQ[(size_t)y.x * np + y.y];
        });
        int2 *dorder = nullptr;
        if ((rc = dalloc(h, &h->S, (size_t)np * np)) || (rc = dalloc(h, &dorder, order.size()))) {
            dfree(h, &dorder, order.size());
            return fail(rc);
        }
        bool ok = ck(cudaMemcpyAsync(dorder, order.data(), sizeof(int2) * order.size(), cudaMemcpyHostToDevice, cs),
                     "copy pair order");
        if (ok) ok = (rc = launch_pair_rule(db, h->Q, tol, dorder, (int64_t)order.size(), h->S, s)) == ESMF_OK;
        hS.resize((size_t)np * np);
        if (ok) ok = ck(cudaMemcpyAsync(hS.data(), h->S, sizeof(double) * np * np, cudaMemcpyDeviceToHost, cs), "copy S");
        if (ok) ok = ck(cudaStreamSynchronize(cs), "pair rule");
        dfree(h, &dorder, order.size());
        if (!ok) return fail(rc ? rc : ESMF_ERR_CUDA);
        h->tol_s = 0.5;
        int64_t cnt = 0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q <= p; ++q) cnt += hS[(size_t)p * np + q] > 0.5 ? 1 : 0;
        h->n_pairs_kept = cnt;
    }
    const std::vector<double> &hScr = screening == ESMF_SCREEN_SCHWARZ ? hQ : hS;
    const double tol_s = h->tol_s;

    // block-level screening: Qblk = max over the 8x8 block; brick kept iff
    // Qblk(PQ) * Qblk(RS) >= tol (element-level screening inside the brick)
    const int nb = h->nb;
    std::vector<double> qblk((size_t)nb * nb, 0.0);
    for (int p = 0; p < np; ++p)
        for (int q = 0; q < np; ++q) {
            double &m_ = qblk[(size_t)(p / BLK) * nb + q / BLK];
            m_ = std::max(m_, hScr[(size_t)p * np + q]);
        }
    std::vector<std::pair<int, int>> bp;
    std::vector<double> bq;
    for (int P = 0; P < nb; ++P)
        for (int Q = 0; Q <= P; ++Q) { bp.push_back({P, Q}); bq.push_back(qblk[(size_t)P * nb + Q]); }
    std::vector<BrickDesc> cand;
    for (size_t i = 0; i < bp.size(); ++i)
        for (size_t j = 0; j <= i; ++j)
            if (bq[i] * bq[j] >= tol_s) {
                BrickDesc d;
                d.P = (int16_t)bp[i].first; d.Q = (int16_t)bp[i].second;
                d.R = (int16_t)bp[j].first; d.S = (int16_t)bp[j].second;
                d.nkept = 0; d.pad = 0;
                cand.push_back(d);
            }
    int64_t ncand = (int64_t)cand.size();
    std::vector<int32_t> counts;
    if (ncand > 0) {
        BrickDesc *dc = nullptr;
        int32_t *dcount = nullptr;
        if ((rc = dalloc(h, &dc, ncand)) || (rc = dalloc(h, &dcount, 2 * ncand))) {
            dfree(h, &dc, ncand);
            return fail(rc);
        }
        counts.resize(2 * ncand);
        bool ok = ck(cudaMemcpyAsync(dc, cand.data(), sizeof(BrickDesc) * ncand, cudaMemcpyHostToDevice, cs), "copy bricks");
        if (ok) ok = (rc = launch_brick_count(db, h->S, tol_s, dc, ncand, dcount, s)) == ESMF_OK;
        if (ok) ok = ck(cudaMemcpyAsync(counts.data(), dcount, sizeof(int32_t) * 2 * ncand, cudaMemcpyDeviceToHost, cs), "copy counts");
        dfree(h, &dc, ncand);
        dfree(h, &dcount, 2 * ncand);
        if (!ok) return fail(rc ? rc : ESMF_ERR_CUDA);
    }
    std::vector<BrickDesc> kept;
    std::vector<int64_t> offs;
    const int eb = elem_bytes(precision);
    const int align_elems = 16 / eb;     // every brick's record starts on 16 bytes
    const bool split16 = is_split16(precision);
    const int head = MASK_BYTES / eb;            // keep mask ahead of the values
    int64_t unique = 0;
    std::vector<int64_t> order;
    for (int64_t i = 0; i < ncand; ++i) {
        if (counts[i] == 0) continue;
        order.push_back(i);
        unique += counts[ncand + i];
    }
    // bricks of one bra pair are consecutive in candidate order (R, S ascending);
    // reorder them by (S window, R, S)
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const BrickDesc &x = cand[a], &y = cand[b];
        if (x.P != y.P) return x.P < y.P;
        if (x.Q != y.Q) return x.Q < y.Q;
        if (x.S / SWIN != y.S / SWIN) return x.S / SWIN < y.S / SWIN;
        if (x.R != y.R) return x.R < y.R;
        return x.S < y.S;
    });
    int64_t off = 0;
    for (int64_t i : order) {
        BrickDesc d = cand[i];
        d.nkept = counts[i];
        kept.push_back(d);
        offs.push_back(off);
        off += (head + counts[i] + align_elems - 1) / align_elems * align_elems;
    }
    offs.push_back(off);
    // runs share (P, Q, R) inside an item; items share (P, Q, S window); the
    // brick (P Q | P Q) is a run and an item of its own.  An item holds at
    // most kItemRuns runs: its window regions sum every run's contributions in
    // FP32 tensor memory before their FP64 flush, so the cap bounds that
    // accumulation length (and its rounding error) for large molecules; up to
    // 8 * kItemRuns functions no item is split.
    {
        constexpr int kItemRuns = ESMF_ITEM_RUNS;
        auto diag = [&](size_t i) { return kept[i].R == kept[i].P && kept[i].S == kept[i].Q; };
        auto same_window = [&](size_t i, size_t j) {
            return kept[i].P == kept[j].P && kept[i].Q == kept[j].Q && kept[i].S / SWIN == kept[j].S / SWIN &&
                   !diag(i) && !diag(j);
        };
        const size_t nk = kept.size();
        std::vector<char> first_run(nk), first_item(nk);
        int runs = 0;
        for (size_t i = 0; i < nk; ++i) {
            bool fi = i == 0 || !same_window(i, i - 1);
            const bool fr = fi || kept[i].R != kept[i - 1].R;
            if (!fi && fr && runs == kItemRuns) fi = true;
            if (fi) runs = 0;
            if (fr) ++runs;
            first_run[i] = fr;
            first_item[i] = fi;
        }
        for (size_t i = 0; i < nk; ++i) {
            const bool lr = i + 1 == nk || first_run[i + 1];
            const bool li = i + 1 == nk || first_item[i + 1];
            kept[i].pad = (first_run[i] ? BRICK_RUN_FIRST : 0) | (lr ? BRICK_RUN_LAST : 0) |
                          (first_item[i] ? BRICK_ITEM_FIRST : 0) | (li ? BRICK_ITEM_LAST : 0);
        }
    }
    // split 16-bit stores: one power-of-two scale with |value * scale| < 2^14
    // (Cauchy-Schwarz: |(pq|rs)| <= Q_pq Q_rs <= max Q^2)
    if (split16) {
        double qmax = 0.0;
        for (double x : hQ) qmax = std::max(qmax, x);
        int e = 0;
        if (qmax > 0.0) std::frexp(qmax * qmax, &e);
        h->vscale = qmax > 0.0 ? (float)std::ldexp(1.0, 14 - e) : 1.0f;
    }
    if (!ck(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device), "SM count"))
        return fail(ESMF_ERR_CUDA);
    const std::vector<int64_t> parts = balance_parts(kept, kChunksPerSM * h->num_sms);
    h->cost_prefix = cost_prefix(kept);
    h->hbricks = kept;
    h->nbricks = (int64_t)kept.size();
    h->n_kept_unique = unique;
    h->n_stored = 0;
    for (auto &d : kept) h->n_stored += d.nkept;
    h->store_bytes = off * eb;

    int use_mode = mode;
    if (mode == ESMF_MODE_AUTO) {
        use_mode = (budget_bytes == 0 || h->device_bytes + h->store_bytes <= budget_bytes) ? ESMF_MODE_STORED
                                                                                          : ESMF_MODE_DIRECT;
        if (use_mode == ESMF_MODE_DIRECT && is_split16(precision)) h->prec = ESMF_PREC_FP32;
        if (use_mode == ESMF_MODE_DIRECT && precision == ESMF_PREC_F32X2) h->prec = ESMF_PREC_FP64;
    } else if (mode == ESMF_MODE_STORED && budget_bytes > 0 && h->device_bytes + h->store_bytes > budget_bytes) {
        set_error("stored integrals need %lld bytes, budget %lld", (long long)h->store_bytes, (long long)budget_bytes);
        return fail(ESMF_ERR_UNSUPPORTED);
    }
    h->mode = use_mode;
    if (use_mode != ESMF_MODE_STORED) h->store_bytes = 0;

    std::vector<int> pslot_h, pblocks_h;
    if (h->nbricks > 0) {
        if ((rc = dalloc(h, &h->bricks, h->nbricks))) return fail(rc);
        if (!ck(cudaMemcpyAsync(h->bricks, kept.data(), sizeof(BrickDesc) * h->nbricks, cudaMemcpyHostToDevice, cs), "copy kept bricks"))
            return fail(ESMF_ERR_CUDA);
        if (!parts.empty()) {
            if ((rc = dalloc(h, &h->parts, parts.size()))) return fail(rc);
            if (!ck(cudaMemcpyAsync(h->parts, parts.data(), sizeof(int64_t) * parts.size(), cudaMemcpyHostToDevice, cs), "copy parts"))
                return fail(ESMF_ERR_CUDA);
            h->nparts = (int)parts.size() - 1;
        }
        if (use_mode == ESMF_MODE_DIRECT && is_split16(h->prec) && !h->cart) {
            // integral-direct on the tensor cores: chunks of whole items whose
            // records fit the scratch buffer (2 GiB, or a quarter of the budget;
            // an item larger than that is a chunk of its own)
            int64_t cap = (int64_t)2 << 30;
            if (budget_bytes > 0) cap = std::min<int64_t>(cap, budget_bytes / 4);
            const int64_t nk = h->nbricks;
            std::vector<int64_t> ch{0};
            int64_t prev = 0;                        // the last item start seen
            for (int64_t i = 1; i <= nk; ++i) {
                if (i < nk && !(kept[i].pad & BRICK_ITEM_FIRST)) continue;
                if ((offs[i] - offs[ch.back()]) * eb > cap && prev > ch.back()) ch.push_back(prev);
                prev = i;
            }
            if (ch.back() != nk) ch.push_back(nk);
            std::vector<int64_t> roff(nk + 1, 0);
            int64_t most = 0;
            for (size_t c = 0; c + 1 < ch.size(); ++c) {
                for (int64_t i = ch[c]; i < ch[c + 1]; ++i) roff[i] = offs[i] - offs[ch[c]];
                most = std::max(most, (offs[ch[c + 1]] - offs[ch[c]]) * eb);
            }
            h->chunks = ch;
            h->scratch_bytes = most;
            if ((rc = dalloc(h, &h->offsets, nk + 1))) return fail(rc);
            if ((rc = dalloc(h, (unsigned char **)&h->scratch, (size_t)h->scratch_bytes))) return fail(rc);
            if (!ck(cudaMemcpyAsync(h->offsets, roff.data(), sizeof(int64_t) * (nk + 1), cudaMemcpyHostToDevice, cs), "copy chunk offsets") ||
                !ck(cudaMemsetAsync(h->scratch, 0, (size_t)h->scratch_bytes, cs), "clear scratch"))
                return fail(ESMF_ERR_CUDA);
            // each scratch chunk's cost-balanced chunks for the tensor kernel
            for (size_t c = 0; c + 1 < ch.size(); ++c) {
                std::vector<BrickDesc> sub(kept.begin() + ch[c], kept.begin() + ch[c + 1]);
                const std::vector<int64_t> sp = balance_parts(sub, kChunksPerSM * h->num_sms);
                int64_t *dp = nullptr;
                if ((rc = dalloc(h, &dp, sp.size()))) return fail(rc);
                h->shard_parts.emplace(std::make_pair(ch[c], ch[c + 1]), std::make_pair(dp, (int)sp.size() - 1));
                if (!ck(cudaMemcpyAsync(dp, sp.data(), sizeof(int64_t) * sp.size(), cudaMemcpyHostToDevice, cs), "copy chunk parts") ||
                    !ck(cudaStreamSynchronize(cs), "chunk parts"))
                    return fail(ESMF_ERR_CUDA);
            }
        }
        if (use_mode == ESMF_MODE_STORED) {
            if ((rc = dalloc(h, &h->offsets, h->nbricks + 1))) return fail(rc);
            if ((rc = dalloc(h, (unsigned char **)&h->store, (size_t)h->store_bytes))) return fail(rc);
            if (!ck(cudaMemcpyAsync(h->offsets, offs.data(), sizeof(int64_t) * (h->nbricks + 1), cudaMemcpyHostToDevice, cs), "copy offsets"))
                return fail(ESMF_ERR_CUDA);
            if (!ck(cudaMemsetAsync(h->store, 0, (size_t)h->store_bytes, cs), "clear store")) return fail(ESMF_ERR_CUDA);
        }
        if (use_mode != ESMF_MODE_STORED || !h->cart) {
            // the primitive pairs of every block pair that a kept brick uses as
            // bra or ket, formed once here instead of in every brick (of the store
            // generation, or of every integral-direct build)
            pslot_h.assign((size_t)h->nb * h->nb, -1);
            auto use = [&](int X, int Y) {
                int &e = pslot_h[(size_t)X * h->nb + Y];
                if (e < 0) {
                    e = (int)(pblocks_h.size() / 2);
                    pblocks_h.push_back(X);
                    pblocks_h.push_back(Y);
                }
            };
            for (const BrickDesc &d : kept) { use(d.P, d.Q); use(d.R, d.S); }
            h->n_ptab = (int)(pblocks_h.size() / 2);
            if ((rc = dalloc(h, &h->pslot, pslot_h.size())) || (rc = dalloc(h, &h->pblocks, pblocks_h.size())) ||
                (rc = dalloc(h, (unsigned char **)&h->ptab, (size_t)h->n_ptab * pair_table_entry_bytes(h->prec))))
                return fail(rc);
            if (!ck(cudaMemcpyAsync(h->pslot, pslot_h.data(), sizeof(int) * pslot_h.size(), cudaMemcpyHostToDevice, cs), "copy pair slots") ||
                !ck(cudaMemcpyAsync(h->pblocks, pblocks_h.data(), sizeof(int) * pblocks_h.size(), cudaMemcpyHostToDevice, cs), "copy pair blocks"))
                return fail(ESMF_ERR_CUDA);
            if ((rc = launch_pair_table(db, h->pblocks, h->n_ptab, h->prec, h->ptab, s))) return fail(rc);
        }
        if (use_mode == ESMF_MODE_STORED) {
            if (h->cart)
                rc = launch_brick_generate_l(db, h->S, tol_s, h->bricks, h->nbricks, h->offsets, h->prec, h->store,
                                             h->vscale, s);
            else
                rc = launch_brick_generate(db, h->S, tol_s, h->bricks, h->nbricks, h->offsets, h->prec, h->store,
                                           h->vscale, s, h->ptab, h->pslot);
            if (rc) return fail(rc);
            // a stored handle needs the pair table only for the generation
            if (h->ptab && !ck(cudaStreamSynchronize(cs), "store generation")) return fail(ESMF_ERR_CUDA);
            dfree(h, (unsigned char **)&h->ptab, (size_t)h->n_ptab * pair_table_entry_bytes(h->prec));
            dfree(h, &h->pslot, pslot_h.size());
            dfree(h, &h->pblocks, pblocks_h.size());
            h->n_ptab = 0;
        }
    }
    if (!ck(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming), "event")) return fail(ESMF_ERR_CUDA);
    if (!ck(cudaHostAlloc((void **)&h->err_host, sizeof(int), cudaHostAllocMapped), "error flag") ||
        !ck(cudaHostGetDevicePointer((void **)&h->err_dev, h->err_host, 0), "error flag address"))
        return fail(ESMF_ERR_CUDA);
    *h->err_host = 0;
    if (!ck(cudaStreamSynchronize(cs), "create kernels")) return fail(ESMF_ERR_CUDA);
    h->create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return ESMF_OK;
}

extern "C" {

// Cholesky factor V = L L^T in place (lower triangle, row-major, FP64; the
// entries above the diagonal keep V's), on the host; false when V is not
// numerically positive definite (a pivot at or below 1e-13 of its diagonal
// element: a function that the others reproduce).
static bool cholesky_factor(int n, std::vector<double> &V) {
    for (int j = 0; j < n; ++j) {
        const double vjj = V[(size_t)j * n + j];
        double d = vjj;
        for (int k = 0; k < j; ++k) d -= V[(size_t)j * n + k] * V[(size_t)j * n + k];
        if (!(d > 1e-13 * vjj)) return false;
        const double l = std::sqrt(d);
        V[(size_t)j * n + j] = l;
        for (int i = j + 1; i < n; ++i) {
            double x = V[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) x -= V[(size_t)i * n + k] * V[(size_t)j * n + k];
            V[(size_t)i * n + j] = x / l;
        }
    }
    return true;
}

// Cholesky factor V = L L^T (as cholesky_factor) and L^-1, on the host.
static bool cholesky_inverse(int n, std::vector<double> &V, std::vector<double> &Linv) {
    if (!cholesky_factor(n, V)) return false;
    // forward substitution for each column of the identity: L X = I
    Linv.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c)
        for (int i = c; i < n; ++i) {
            double x = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) x -= V[(size_t)i * n + k] * Linv[(size_t)k * n + c];
            Linv[(size_t)i * n + c] = x / V[(size_t)i * n + i];
        }
    return true;
}

int esmf_fock_create_df(const esmf_basis_t *basis, const esmf_aux_t *aux, int precision, int device,
                        esmf_fock_t **out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) { set_error("out is NULL"); return ESMF_ERR_INVALID_ARG; }
    *out = nullptr;
    int64_t nprim_tot = 0;
    RET(check_basis(basis, &nprim_tot));
    if (!aux || aux->n_aux <= 0 || aux->n_aux > 8192 || !aux->center || !aux->exps) {
        set_error("auxiliary set missing, empty or above 8192 functions");
        return ESMF_ERR_INVALID_ARG;
    }
    for (int P = 0; P < aux->n_aux; ++P) {
        if (!(aux->exps[P] > 0.0) || !is_finite(aux->exps[P])) { set_error("aux exps[%d] must be finite and > 0", P); return ESMF_ERR_INVALID_ARG; }
        for (int x = 0; x < 3; ++x)
            if (!is_finite(aux->center[3 * P + x])) { set_error("aux center[%d] not finite", P); return ESMF_ERR_INVALID_ARG; }
    }
    if (precision != ESMF_PREC_FP64 && precision != ESMF_PREC_FP32) {
        set_error("density fitting runs in FP64 or FP32");
        return precision >= ESMF_PREC_FP16X2 && precision <= ESMF_PREC_F32X2 ? ESMF_ERR_UNSUPPORTED : ESMF_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("device %d not available (%d devices)", device, ndev);
        return ESMF_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    if (!g.ok) { set_error("cudaSetDevice(%d) failed", device); return ESMF_ERR_CUDA; }
    esmf_fock *h = new (std::nothrow) esmf_fock();
    if (!h) { set_error("host allocation failed"); return ESMF_ERR_OOM; }
    const int n = basis->n_basis, naux = aux->n_aux;
    h->device = device; h->n = n; h->prec = precision; h->mode = ESMF_MODE_DF;
    h->nb = (n + BLK - 1) / BLK;
    h->np = h->nb * BLK;
    h->naux = naux;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error("cudaStreamCreate failed");
        return ESMF_ERR_CUDA;
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } cs_guard{cs};
    double *acen = nullptr, *aexp = nullptr, *T = nullptr, *V = nullptr, *Linv = nullptr, *B = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(cs);
        cudaFree(acen); cudaFree(aexp); cudaFree(T); cudaFree(V); cudaFree(Linv); cudaFree(B);
    };
    auto fail = [&](int code) { cleanup(); cudaGetLastError(); release(h); return code; };
    int rc;
    if ((rc = upload_basis(h, basis, nprim_tot, cs))) return fail(rc);
    if ((rc = df_cublas_create(&h->cublas))) return fail(rc);
    const size_t nn = (size_t)n * n, es = precision == ESMF_PREC_FP32 ? 4 : 8;
    if (cudaMalloc(&acen, sizeof(double) * 3 * naux) || cudaMalloc(&aexp, sizeof(double) * naux) ||
        cudaMalloc(&T, sizeof(double) * naux * nn) || cudaMalloc(&V, sizeof(double) * naux * naux) ||
        cudaMalloc(&Linv, sizeof(double) * naux * naux) || cudaMalloc(&B, sizeof(double) * naux * nn)) {
        cudaGetLastError();
        set_error("density-fitting set-up memory (%zu bytes of three-centre integrals)", sizeof(double) * naux * nn);
        return fail(ESMF_ERR_OOM);
    }
    if (cudaMemcpyAsync(acen, aux->center, sizeof(double) * 3 * naux, cudaMemcpyHostToDevice, cs) ||
        cudaMemcpyAsync(aexp, aux->exps, sizeof(double) * naux, cudaMemcpyHostToDevice, cs)) {
        set_error("copy auxiliary set failed");
        return fail(ESMF_ERR_CUDA);
    }
    if ((rc = launch_df_integrals(h->dev(), naux, acen, aexp, T, V, cs))) return fail(rc);
    std::vector<double> hV((size_t)naux * naux), hL;
    if (cudaMemcpyAsync(hV.data(), V, sizeof(double) * naux * naux, cudaMemcpyDeviceToHost, cs) ||
        cudaStreamSynchronize(cs)) {
        set_error("metric copy failed");
        return fail(ESMF_ERR_CUDA);
    }
    if (!cholesky_inverse(naux, hV, hL)) {
        set_error("the auxiliary Coulomb metric is not positive definite (near-duplicate auxiliaries?)");
        return fail(ESMF_ERR_INVALID_ARG);
    }
    if (cudaMemcpyAsync(Linv, hL.data(), sizeof(double) * naux * naux, cudaMemcpyHostToDevice, cs)) {
        set_error("copy L^-1 failed");
        return fail(ESMF_ERR_CUDA);
    }
    if ((rc = df_gemm_fold(h->cublas, naux, (int64_t)nn, Linv, T, B, cs))) return fail(rc);
    if ((rc = dalloc(h, (unsigned char **)&h->dfB2, naux * nn * es)) ||
        (rc = dalloc(h, (unsigned char **)&h->dfY, naux * nn * es)))
        return fail(rc);
    if (es == 4) {
        if ((rc = dalloc(h, (unsigned char **)&h->dfB, naux * nn * es))) return fail(rc);
        if ((rc = launch_df_layouts(naux, n, B, 1, h->dfB, h->dfB2, cs))) return fail(rc);
    } else {
        if ((rc = launch_df_layouts(naux, n, B, 0, nullptr, h->dfB2, cs))) return fail(rc);
        h->dfB = B;                       // the FP64 factor itself is the [P][p][q] layout
        h->device_bytes += (int64_t)(naux * nn * es);
        B = nullptr;
    }
    h->store_bytes = (int64_t)(2 * naux * nn * es);
    if (cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc((void **)&h->err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&h->err_dev, h->err_host, 0) != cudaSuccess) {
        set_error("event / error flag creation failed");
        return fail(ESMF_ERR_CUDA);
    }
    *h->err_host = 0;
    cleanup();
    if (cudaGetLastError() != cudaSuccess) { set_error("density-fitting set-up kernels failed"); release(h); return ESMF_ERR_CUDA; }
    h->create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return ESMF_OK;
}

int esmf_fock_create_thc(const esmf_basis_t *basis, const esmf_grid_t *grid, double schwarz_tol, double ridge,
                         int precision, int device, int64_t budget_bytes, esmf_fock_t **out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) { set_error("out is NULL"); return ESMF_ERR_INVALID_ARG; }
    *out = nullptr;
    int64_t nprim_tot = 0;
    RET(check_basis(basis, &nprim_tot));
    if (!grid || grid->n_grid <= 0 || grid->n_grid > ESMF_MAX_GRID || !grid->points) {
        set_error("grid missing, empty or above %d points", ESMF_MAX_GRID);
        return ESMF_ERR_INVALID_ARG;
    }
    for (int P = 0; P < 3 * grid->n_grid; ++P)
        if (!is_finite(grid->points[P])) { set_error("grid point %d not finite", P / 3); return ESMF_ERR_INVALID_ARG; }
    if (!(schwarz_tol >= 0.0) || !is_finite(schwarz_tol) || !(ridge >= 0.0) || !is_finite(ridge) || budget_bytes < 0) {
        set_error("schwarz_tol and ridge must be finite and >= 0, budget_bytes >= 0");
        return ESMF_ERR_INVALID_ARG;
    }
    if (precision != ESMF_PREC_FP64 && precision != ESMF_PREC_FP32) {
        set_error("tensor hypercontraction runs in FP64 or FP32");
        return precision >= ESMF_PREC_FP16X2 && precision <= ESMF_PREC_F32X2 ? ESMF_ERR_UNSUPPORTED : ESMF_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("device %d not available (%d devices)", device, ndev);
        return ESMF_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    if (!g.ok) { set_error("cudaSetDevice(%d) failed", device); return ESMF_ERR_CUDA; }
    esmf_fock *h = new (std::nothrow) esmf_fock();
    if (!h) { set_error("host allocation failed"); return ESMF_ERR_OOM; }
    const int n = basis->n_basis, G = grid->n_grid;
    h->device = device; h->n = n; h->prec = precision; h->mode = ESMF_MODE_THC; h->tol = schwarz_tol;
    h->nb = (n + BLK - 1) / BLK;
    h->np = h->nb * BLK;
    h->thc_G = G;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error("cudaStreamCreate failed");
        return ESMF_ERR_CUDA;
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } cs_guard{cs};
    // rank-one densities per grouped Coulomb build of the fit
    const int MQ = G < 64 ? G : 64;
    const size_t nn = (size_t)n * n, nG = (size_t)n * G, GG = (size_t)G * G;
    const size_t es = precision == ESMF_PREC_FP32 ? 4 : 8;
    double *pts = nullptr, *X = nullptr, *Dq = nullptr, *Jq = nullptr, *Kq = nullptr, *R = nullptr, *E = nullptr,
           *C = nullptr, *L = nullptr;
    esmf_fock_t *hx = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(cs);
        if (hx) esmf_fock_destroy(hx);
        hx = nullptr;
        cudaFree(pts); cudaFree(X); cudaFree(Dq); cudaFree(Jq); cudaFree(Kq); cudaFree(R); cudaFree(E);
        cudaFree(C); cudaFree(L);
    };
    auto fail = [&](int code) { cleanup(); cudaGetLastError(); release(h); return code; };
    int rc;
    if ((rc = upload_basis(h, basis, nprim_tot, cs))) return fail(rc);
    if ((rc = df_cublas_create(&h->cublas))) return fail(rc);
    if (cudaMalloc(&pts, sizeof(double) * 3 * G) || cudaMalloc(&X, sizeof(double) * nG) ||
        cudaMalloc(&Dq, sizeof(double) * MQ * nn) || cudaMalloc(&Jq, sizeof(double) * MQ * nn) ||
        cudaMalloc(&Kq, sizeof(double) * MQ * nn) || cudaMalloc(&R, sizeof(double) * MQ * nG) ||
        cudaMalloc(&E, sizeof(double) * GG) || cudaMalloc(&C, sizeof(double) * GG) ||
        cudaMalloc(&L, sizeof(double) * GG)) {
        cudaGetLastError();
        set_error("hypercontraction set-up memory (%zu bytes per grid matrix)", sizeof(double) * GG);
        return fail(ESMF_ERR_OOM);
    }
    if (cudaMemcpyAsync(pts, grid->points, sizeof(double) * 3 * G, cudaMemcpyHostToDevice, cs)) {
        set_error("copy grid failed");
        return fail(ESMF_ERR_CUDA);
    }
    if ((rc = launch_thc_collocate(h->dev(), G, pts, X, cs))) return fail(rc);
    // E from the exact screened integrals: grouped Coulomb builds over the
    // rank-one densities x_Q x_Q^T, MQ grid points per build
    if ((rc = esmf_fock_create(basis, schwarz_tol, ESMF_MODE_AUTO, ESMF_PREC_FP64, device, budget_bytes, &hx)))
        return fail(rc);
    for (int q0 = 0; q0 < G; q0 += MQ) {
        const int mq = G - q0 < MQ ? G - q0 : MQ;
        if ((rc = launch_thc_rank_one(n, G, q0, mq, X, Dq, cs))) return fail(rc);
        if ((rc = esmf_fock_build(hx, mq, Dq, Jq, Kq, nullptr, nullptr, cs))) return fail(rc);
        if ((rc = thc_coulomb_columns(h->cublas, n, G, q0, mq, X, Jq, R, E, cs))) return fail(rc);
    }
    h->n_kept_unique = hx->n_kept_unique;
    if ((rc = thc_gram(h->cublas, n, G, X, C, cs))) return fail(rc);
    std::vector<double> hS(GG), hE(GG);
    if (cudaMemcpyAsync(hS.data(), C, sizeof(double) * GG, cudaMemcpyDeviceToHost, cs) ||
        cudaMemcpyAsync(hE.data(), E, sizeof(double) * GG, cudaMemcpyDeviceToHost, cs) || cudaStreamSynchronize(cs)) {
        set_error("fit matrices copy failed");
        return fail(ESMF_ERR_CUDA);
    }
    if (*hx->err_host) {
        set_error("a bounded wait expired in the Coulomb builds of the fit");
        return fail(ESMF_ERR_TIMEOUT);
    }
    esmf_fock_destroy(hx);
    hx = nullptr;
    // S = (X^T X) o (X^T X) + lam I and E, both made exactly symmetric
    double smax = 0.0;
    for (int i = 0; i < G; ++i)
        for (int j = 0; j <= i; ++j) {
            const double c = 0.5 * (hS[(size_t)i * G + j] + hS[(size_t)j * G + i]);
            const double e = 0.5 * (hE[(size_t)i * G + j] + hE[(size_t)j * G + i]);
            hS[(size_t)i * G + j] = hS[(size_t)j * G + i] = c * c;
            hE[(size_t)i * G + j] = hE[(size_t)j * G + i] = e;
            if (i == j && c * c > smax) smax = c * c;
        }
    const double lam = ridge * smax;
    for (int i = 0; i < G; ++i) hS[(size_t)i * G + i] += lam;
    if (!cholesky_factor(G, hS)) {
        set_error("S + lam I is not positive definite (grid points that the others reproduce; raise ridge)");
        return fail(ESMF_ERR_INVALID_ARG);
    }
    if (cudaMemcpyAsync(L, hS.data(), sizeof(double) * GG, cudaMemcpyHostToDevice, cs) ||
        cudaMemcpyAsync(E, hE.data(), sizeof(double) * GG, cudaMemcpyHostToDevice, cs)) {
        set_error("copy of the fit matrices failed");
        return fail(ESMF_ERR_CUDA);
    }
    if ((rc = dalloc(h, (unsigned char **)&h->thcZ, GG * es))) return fail(rc);
    if ((rc = thc_solve_z(h->cublas, G, L, E, es == 4, h->thcZ, cs))) return fail(rc);
    if (es == 4) {
        if ((rc = dalloc(h, (unsigned char **)&h->thcX, nG * es))) return fail(rc);
        if ((rc = launch_thc_convert((int64_t)nG, X, (float *)h->thcX, cs))) return fail(rc);
    } else {
        h->thcX = X;                      // the FP64 collocation itself
        h->device_bytes += (int64_t)(nG * es);
        X = nullptr;
    }
    h->store_bytes = (int64_t)((nG + GG) * es);
    if (cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc((void **)&h->err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&h->err_dev, h->err_host, 0) != cudaSuccess) {
        set_error("event / error flag creation failed");
        return fail(ESMF_ERR_CUDA);
    }
    *h->err_host = 0;
    cleanup();
    if (cudaGetLastError() != cudaSuccess) { set_error("hypercontraction set-up kernels failed"); release(h); return ESMF_ERR_CUDA; }
    h->create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return ESMF_OK;
}

}  // extern "C"

namespace {

// One hypercontracted build: per-build work grown for up to m densities
// (batches of densities whose work stays within about 1 GiB), then the GEMM
// sequence of thc.cu per batch.
int build_thc(esmf_fock_t *h, int m, const double *D, double *J, double *K, double *F, double *traces,
              cudaStream_t s) {
    const size_t es = h->prec == ESMF_PREC_FP32 ? 4 : 8;
    const size_t n = (size_t)h->n, G = (size_t)h->thc_G, nn = n * n, nG = n * G, GG = G * G;
    const size_t per = nG + GG + 2 * G + 2 * nn + (es == 4 ? nn : 0);
    int mc = (int)std::max<size_t>(1, std::min<size_t>((size_t)m, ((size_t)1 << 30) / (es * per)));
    if (mc > h->thc_m) {
        const size_t o = (size_t)h->thc_m;
        dfree(h, (unsigned char **)&h->thcDt, es == 4 ? o * nn * es : 1);
        dfree(h, (unsigned char **)&h->thcA, o * nG * es);
        dfree(h, (unsigned char **)&h->thcM, o * GG * es);
        dfree(h, (unsigned char **)&h->thcy, o * G * es);
        dfree(h, (unsigned char **)&h->thcz, o * G * es);
        dfree(h, (unsigned char **)&h->thcJt, o * nn * es);
        dfree(h, (unsigned char **)&h->thcKt, o * nn * es);
        h->thc_m = 0;
        const size_t c = (size_t)mc;
        RET(dalloc(h, (unsigned char **)&h->thcDt, es == 4 ? c * nn * es : 1));
        RET(dalloc(h, (unsigned char **)&h->thcA, c * nG * es));
        RET(dalloc(h, (unsigned char **)&h->thcM, c * GG * es));
        RET(dalloc(h, (unsigned char **)&h->thcy, c * G * es));
        RET(dalloc(h, (unsigned char **)&h->thcz, c * G * es));
        RET(dalloc(h, (unsigned char **)&h->thcJt, c * nn * es));
        RET(dalloc(h, (unsigned char **)&h->thcKt, c * nn * es));
        h->thc_m = mc;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (h->timing && h->ev_used < 65536) {
        if (h->ev_used == h->ev_pool.size()) {
            cudaEvent_t x, y;
            CKR(cudaEventCreate(&x));
            CKR(cudaEventCreate(&y));
            h->ev_pool.push_back({x, y});
        }
        ev0 = h->ev_pool[h->ev_used].first;
        ev1 = h->ev_pool[h->ev_used].second;
        ++h->ev_used;
        CKR(cudaEventRecord(ev0, s));
    }
    for (int k0 = 0; k0 < m; k0 += mc) {
        const int kc = m - k0 < mc ? m - k0 : mc;
        const size_t off = (size_t)k0 * nn;
        ThcBuild a;
        a.cublas = h->cublas; a.n = h->n; a.G = h->thc_G; a.m = kc; a.fp32 = es == 4;
        a.X = h->thcX; a.Z = h->thcZ; a.D = D + off;
        a.Dt = h->thcDt; a.A = h->thcA; a.M = h->thcM; a.y = h->thcy; a.z = h->thcz; a.Jt = h->thcJt; a.Kt = h->thcKt;
        a.J = J + off; a.K = K + off; a.F = F ? F + off : nullptr; a.traces = traces ? traces + k0 : nullptr;
        RET(thc_build(a, s));
    }
    if (ev1) CKR(cudaEventRecord(ev1, s));
    return ESMF_OK;
}

// One density-fitted build: per-build work grown for m densities, then the
// GEMM sequence of df.cu.
int build_df(esmf_fock_t *h, int m, const double *D, double *J, double *K, double *F, double *traces,
             cudaStream_t s) {
    const size_t es = h->prec == ESMF_PREC_FP32 ? 4 : 8;
    const size_t nn = (size_t)h->n * h->n;
    if (m > h->df_m) {
        dfree(h, (unsigned char **)&h->dfDt, es == 4 ? h->df_m * nn * es : 1);
        dfree(h, (unsigned char **)&h->dfJt, h->df_m * nn * es);
        dfree(h, (unsigned char **)&h->dfKt, h->df_m * nn * es); dfree(h, (unsigned char **)&h->dfg, (size_t)h->df_m * h->naux * es);
        h->df_m = 0;
        RET(dalloc(h, (unsigned char **)&h->dfDt, es == 4 ? m * nn * es : 1));
        RET(dalloc(h, (unsigned char **)&h->dfJt, m * nn * es));
        RET(dalloc(h, (unsigned char **)&h->dfKt, m * nn * es));
        RET(dalloc(h, (unsigned char **)&h->dfg, (size_t)m * h->naux * es));
        h->df_m = m;
    }
    DfBuild a;
    a.cublas = h->cublas; a.n = h->n; a.naux = h->naux; a.m = m; a.fp32 = h->prec == ESMF_PREC_FP32;
    a.B = h->dfB; a.B2 = h->dfB2; a.D = D;
    a.Dt = h->dfDt; a.Jt = h->dfJt; a.Kt = h->dfKt; a.g = h->dfg; a.Y = h->dfY;
    a.J = J; a.K = K; a.F = F; a.traces = traces;
    if (h->timing && h->ev_used < 65536) {
        if (h->ev_used == h->ev_pool.size()) {
            cudaEvent_t x, y;
            CKR(cudaEventCreate(&x));
            CKR(cudaEventCreate(&y));
            h->ev_pool.push_back({x, y});
        }
        a.ev_start = h->ev_pool[h->ev_used].first;
        a.ev_stop = h->ev_pool[h->ev_used].second;
        ++h->ev_used;
    }
    return df_build(a, s);
}

// the build over kept bricks [b0, b1) of the handle's list; J, K, F and the
// traces are linear in the integrals, so builds over a partition of the list
// sum to the full build
int build_range(esmf_fock_t *h, int64_t b0, int64_t b1, int m, const double *D, double *J, double *K,
                double *F, double *traces, void *stream) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    if (m < 1 || m > ESMF_MAX_DENSITIES) { set_error("m = %d outside [1, %d]", m, ESMF_MAX_DENSITIES); return ESMF_ERR_INVALID_ARG; }
    if (!D || !J || !K) { set_error("D, J and K are required"); return ESMF_ERR_INVALID_ARG; }
    DeviceGuard g(h->device);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    if (!is_device_ptr(D) || !is_device_ptr(J) || !is_device_ptr(K) || (F && !is_device_ptr(F)) ||
        (traces && !is_device_ptr(traces))) {
        set_error("D, J, K, F and traces must be device memory");
        return ESMF_ERR_INVALID_ARG;
    }
    if (h->mode == ESMF_MODE_DF) {
        if (b0 != 0 || b1 != h->nbricks) { set_error("density-fitted handles build whole only"); return ESMF_ERR_UNSUPPORTED; }
        return build_df(h, m, D, J, K, F, traces, (cudaStream_t)stream);
    }
    if (h->mode == ESMF_MODE_THC) {
        if (b0 != 0 || b1 != h->nbricks) { set_error("hypercontracted handles build whole only"); return ESMF_ERR_UNSUPPORTED; }
        return build_thc(h, m, D, J, K, F, traces, (cudaStream_t)stream);
    }
    RET(ensure_work(h, m));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t acc = sizeof(double) * (size_t)m * h->np * h->np;
    CKR(cudaMemsetAsync(h->Jacc, 0, acc, s));
    CKR(cudaMemsetAsync(h->Kacc, 0, acc, s));
    if (traces) CKR(cudaMemsetAsync(traces, 0, sizeof(double) * m, s));
    if (b1 > b0) {
        JKArgs a;
        a.b = h->dev(); a.Q = h->S; a.tol = h->tol_s; a.bricks = h->bricks + b0; a.nbricks = b1 - b0;
        a.offsets = h->offsets ? h->offsets + b0 : nullptr; a.store = h->store; a.precision = h->prec;
        a.mode = h->mode;
        a.m = m; a.D = D; a.Jacc = h->Jacc; a.Kacc = h->Kacc;
        a.ptab = h->ptab; a.pslot = h->pslot;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing && h->ev_used < 65536) {
            if (h->ev_used == h->ev_pool.size()) {
                cudaEvent_t x, y;
                CKR(cudaEventCreate(&x));
                CKR(cudaEventCreate(&y));
                h->ev_pool.push_back({x, y});
            }
            e0 = h->ev_pool[h->ev_used].first;
            e1 = h->ev_pool[h->ev_used].second;
            ++h->ev_used;
        }
        a.vscale = h->vscale;
        int chunk = h->force_chunk;
        if (!chunk)
            for (auto &t : h->tuned)
                if (t.first == m) chunk = t.second;
        a.mc = chunk;
        const bool split16 = h->mode == ESMF_MODE_STORED && is_split16(h->prec);
        const bool tdirect = tensor_direct(h);
        if (h->tol_d > 0.0) {
            // density-weighted screening runs on the CUDA-core kernels
            RET(launch_density_weight(h->dev(), m, D, h->dw, h->dwb, s));
            a.dw = h->dw; a.dwb = h->dwb; a.tol_d = h->tol_d;
        }
        if ((split16 || tdirect) && h->path != ESMF_PATH_CUDA_CORE && h->tol_d == 0.0) {
            UmmaLaunch L;
            L.kbank = h->kbank; L.jbank = h->jbank;
            L.dmax_bits = h->dmax; L.D = D; L.n = h->n; L.np = h->np; L.nb = h->nb; L.m = m;
            L.bf16 = h->prec == ESMF_PREC_BF16X2; L.num_sms = h->num_sms; L.vscale = h->vscale;
            L.Jacc = h->Jacc; L.Kacc = h->Kacc; L.error = h->err_dev; L.counter = h->sched;
            L.chunk = chunk ? chunk : 16;
            // chunks of bricks [r0, r1) for the tensor kernel: the whole list's, or
            // the range's own cost-balanced ones (scratch chunks and shards), built once
            auto set_parts = [&](int64_t r0, int64_t r1) -> int {
                if (r0 == 0 && r1 == h->nbricks && h->parts && !tdirect) {
                    L.part = h->parts; L.nparts = h->nparts;
                } else if (r1 - r0 >= 1 && (int64_t)h->hbricks.size() == h->nbricks) {
                    auto key = std::make_pair(r0, r1);
                    auto it = h->shard_parts.find(key);
                    if (it == h->shard_parts.end()) {
                        std::vector<BrickDesc> sub(h->hbricks.begin() + r0, h->hbricks.begin() + r1);
                        const std::vector<int64_t> sp = balance_parts(sub, kChunksPerSM * h->num_sms);
                        int64_t *dp = nullptr;
                        RET(dalloc(h, &dp, sp.size()));
                        CKR(cudaMemcpy(dp, sp.data(), sizeof(int64_t) * sp.size(), cudaMemcpyHostToDevice));
                        it = h->shard_parts.emplace(key, std::make_pair(dp, (int)sp.size() - 1)).first;
                    }
                    L.part = it->second.first; L.nparts = it->second.second;
                }
                return ESMF_OK;
            };
            if (!tdirect) {
                L.bricks = h->bricks + b0; L.nbricks = b1 - b0; L.offsets = h->offsets + b0;
                L.store = (const uint32_t *)h->store;
                L.ev_start = e0; L.ev_stop = e1;
                RET(set_parts(b0, b1));
                RET(launch_jk_umma(L, s));
            } else {
                // integral-direct: per chunk, the packed split records of its bricks
                // into the scratch buffer, then the tensor-core contraction of them;
                // the FP64 accumulators sum over the chunks
                if (e0) CKR(cudaEventRecord(e0, s));
                const DevBasis db = h->dev();
                for (size_t c = 0; c + 1 < h->chunks.size(); ++c) {
                    const int64_t r0 = std::max(b0, h->chunks[c]), r1 = std::min(b1, h->chunks[c + 1]);
                    if (r1 <= r0) continue;
                    RET(launch_brick_generate(db, h->S, h->tol_s, h->bricks + r0, r1 - r0, h->offsets + r0, h->prec,
                                              h->scratch, h->vscale, s, h->ptab, h->pslot));
                    L.bricks = h->bricks + r0; L.nbricks = r1 - r0; L.offsets = h->offsets + r0;
                    L.store = (const uint32_t *)h->scratch;
                    L.part = nullptr; L.nparts = 0;
                    RET(set_parts(r0, r1));
                    RET(launch_jk_umma(L, s));
                }
                if (e1) CKR(cudaEventRecord(e1, s));
            }
            return launch_finalize_blocked(h->dev(), m, D, h->Jacc, h->Kacc, J, K, F, traces, s);
        }
        if (h->Dt) {
            RET(launch_density_typed(h->prec, (int64_t)m * h->n * h->n, D, h->Dt, s));
            a.Dt = h->Dt;
        }
        if (e0) CKR(cudaEventRecord(e0, s));
        if (split16) RET(launch_jk_cuda_split(a, s));
        else RET(launch_jk_cuda(a, s));
        if (e1) CKR(cudaEventRecord(e1, s));
    }
    RET(launch_finalize(h->dev(), m, D, h->Jacc, h->Kacc, J, K, F, traces, s));
    return ESMF_OK;
}

}  // namespace

extern "C" {

int esmf_fock_build(esmf_fock_t *h, int m, const double *D, double *J, double *K, double *F,
                    double *traces, void *stream) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    return build_range(h, 0, h->nbricks, m, D, J, K, F, traces, stream);
}

int esmf_fock_build_batch(int count, esmf_fock_t *const *hs, const int *ms, const double *const *Ds,
                          double *const *Js, double *const *Ks, double *const *Fs, double *const *traces,
                          void *stream) {
    if (count < 1 || count > ESMF_MAX_BATCH || !hs || !ms || !Ds || !Js || !Ks) {
        set_error("batch: count must be in [1, %d] and h, m, D, J, K given", ESMF_MAX_BATCH);
        return ESMF_ERR_INVALID_ARG;
    }
    const int dev = hs[0] ? hs[0]->device : 0;
    for (int i = 0; i < count; ++i) {
        esmf_fock_t *h = hs[i];
        if (!h) { set_error("batch: handle %d is NULL", i); return ESMF_ERR_INVALID_ARG; }
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) { set_error("batch: handle %d repeats handle %d", i, j); return ESMF_ERR_INVALID_ARG; }
        if (h->device != dev) { set_error("batch: handles on different devices"); return ESMF_ERR_INVALID_ARG; }
        if (ms[i] < 1 || ms[i] > ESMF_MAX_DENSITIES) { set_error("batch: m[%d] = %d", i, ms[i]); return ESMF_ERR_INVALID_ARG; }
        if (!Ds[i] || !Js[i] || !Ks[i]) { set_error("batch: D, J, K of entry %d are required", i); return ESMF_ERR_INVALID_ARG; }
        if (!(h->mode == ESMF_MODE_STORED && is_split16(h->prec)) || h->path == ESMF_PATH_CUDA_CORE ||
            h->tol_d > 0.0) {
            set_error("batch: handle %d is not on the tensor-core path (stored FP16X2/BF16X2, no density "
                      "screening)", i);
            return ESMF_ERR_UNSUPPORTED;
        }
    }
    DeviceGuard g(dev);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    UmmaLaunch L[ESMF_MAX_BATCH];
    for (int i = 0; i < count; ++i) {
        esmf_fock_t *h = hs[i];
        const int m = ms[i];
        double *F = Fs ? Fs[i] : nullptr, *tr = traces ? traces[i] : nullptr;
        if (!is_device_ptr(Ds[i]) || !is_device_ptr(Js[i]) || !is_device_ptr(Ks[i]) || (F && !is_device_ptr(F)) ||
            (tr && !is_device_ptr(tr))) {
            set_error("batch: entry %d buffers must be device memory", i);
            return ESMF_ERR_INVALID_ARG;
        }
        RET(ensure_work(h, m));
        const size_t acc = sizeof(double) * (size_t)m * h->np * h->np;
        CKR(cudaMemsetAsync(h->Jacc, 0, acc, s));
        CKR(cudaMemsetAsync(h->Kacc, 0, acc, s));
        if (tr) CKR(cudaMemsetAsync(tr, 0, sizeof(double) * m, s));
        UmmaLaunch &l = L[i];
        l.bricks = h->bricks; l.nbricks = h->nbricks; l.offsets = h->offsets;
        l.store = (const uint32_t *)h->store; l.kbank = h->kbank; l.jbank = h->jbank;
        l.dmax_bits = h->dmax; l.D = Ds[i]; l.n = h->n; l.np = h->np; l.nb = h->nb; l.m = m;
        l.bf16 = h->prec == ESMF_PREC_BF16X2; l.num_sms = h->num_sms; l.vscale = h->vscale;
        l.Jacc = h->Jacc; l.Kacc = h->Kacc; l.error = h->err_dev; l.counter = h->sched;
        l.chunk = 16;
        if (h->parts) { l.part = h->parts; l.nparts = h->nparts; }
    }
    RET(launch_jk_umma_batch(L, count, s));
    for (int i = 0; i < count; ++i) {
        esmf_fock_t *h = hs[i];
        RET(launch_finalize_blocked(h->dev(), ms[i], Ds[i], h->Jacc, h->Kacc, Js[i], Ks[i], Fs ? Fs[i] : nullptr,
                                    traces ? traces[i] : nullptr, s));
    }
    return ESMF_OK;
}

int esmf_energy_gradient(esmf_fock_t *h, int n_occ, double c0, const double *G, const double *V,
                         const double *sigma, double *scalars, double *dE_dsigma, double *dE_dV,
                         void *stream) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    const int n = h->n;
    if (n_occ < 1 || n_occ >= n) {
        set_error("n_occ = %d outside [1, %d)", n_occ, n);
        return ESMF_ERR_INVALID_ARG;
    }
    if (!is_finite(c0)) { set_error("c0 is not finite"); return ESMF_ERR_INVALID_ARG; }
    if (!G || !V || !sigma || !scalars) { set_error("G, V, sigma and scalars are required"); return ESMF_ERR_INVALID_ARG; }
    if ((dE_dsigma == nullptr) != (dE_dV == nullptr)) {
        set_error("dE_dsigma and dE_dV must both be given or both be NULL");
        return ESMF_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    if (!is_device_ptr(G) || !is_device_ptr(V) || !is_device_ptr(sigma) || !is_device_ptr(scalars) ||
        (dE_dsigma && (!is_device_ptr(dE_dsigma) || !is_device_ptr(dE_dV)))) {
        set_error("G, V, sigma, scalars and the gradient outputs must be device memory");
        return ESMF_ERR_INVALID_ARG;
    }
    const size_t need = energy_work_doubles(n, n_occ);
    if (need > h->ework_n) {
        dfree(h, &h->ework, h->ework_n);
        h->ework_n = 0;
        RET(dalloc(h, &h->ework, need));
        h->ework_n = need;
    }
    const EnergyWork w = energy_work_layout(h->ework, n, n_occ);
    if (w.sc + 8 > h->ework + need) { set_error("internal: energy work layout"); return ESMF_ERR_CUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    const bool grad = dE_dsigma != nullptr;
    RET(launch_energy_densities(n, n_occ, V, sigma, w, s));
    // one grouped build: F[P], F[T] (energy) and F[A] (gradient)
    RET(build_range(h, 0, h->nbricks, grad ? 3 : 2, w.D, w.J, w.K, w.F, nullptr, stream));
    return launch_energy_finish(n, n_occ, c0, G, V, sigma, w, scalars, dE_dsigma, dE_dV, s);
}

int esmf_gvp_gradient(esmf_fock_t *h, int n_occ, double c0, const double *G, const double *V,
                      const double *sigma, double omega, double mu, double chi, double *scalars,
                      double *dL_dsigma, double *dL_dX, void *stream) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    const int n = h->n;
    if (n_occ < 1 || n_occ >= n) {
        set_error("n_occ = %d outside [1, %d)", n_occ, n);
        return ESMF_ERR_INVALID_ARG;
    }
    if (!is_finite(c0) || !is_finite(omega) || !is_finite(mu) || !is_finite(chi)) {
        set_error("c0, omega, mu and chi must be finite");
        return ESMF_ERR_INVALID_ARG;
    }
    if (!G || !V || !sigma || !scalars || !dL_dsigma || !dL_dX) {
        set_error("G, V, sigma, scalars, dL_dsigma and dL_dX are required");
        return ESMF_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    if (!is_device_ptr(G) || !is_device_ptr(V) || !is_device_ptr(sigma) || !is_device_ptr(scalars) ||
        !is_device_ptr(dL_dsigma) || !is_device_ptr(dL_dX)) {
        set_error("G, V, sigma, scalars, dL_dsigma and dL_dX must be device memory");
        return ESMF_ERR_INVALID_ARG;
    }
    const size_t ne = energy_work_doubles(n, n_occ), need = ne + gvp_work_doubles(n, n_occ);
    if (need > h->ework_n) {
        dfree(h, &h->ework, h->ework_n);
        h->ework_n = 0;
        RET(dalloc(h, &h->ework, need));
        h->ework_n = need;
    }
    const EnergyWork w = energy_work_layout(h->ework, n, n_occ);
    const GvpWork v = gvp_work_layout(h->ework + ne, n, n_occ);
    if (w.sc + 8 > h->ework + ne || v.st + 8 > h->ework + need) {
        set_error("internal: GVP work layout");
        return ESMF_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // pass 1: E and its gradient from F[P], F[T], F[A]
    RET(launch_energy_densities(n, n_occ, V, sigma, w, s));
    RET(build_range(h, 0, h->nbricks, 3, w.D, w.J, w.K, w.F, nullptr, stream));
    RET(launch_energy_finish(n, n_occ, c0, G, V, sigma, w, v.scE, v.gs, v.gV, s));
    // pass 2: the tangent densities along the gradient, F[P'], F[T'], F[A']
    RET(launch_gvp_tangent_densities(n, n_occ, V, sigma, w, v, s));
    RET(build_range(h, 0, h->nbricks, 3, v.Dt, v.Jt, v.Kt, v.Ft, nullptr, stream));
    return launch_gvp_finish(n, n_occ, c0, omega, mu, chi, G, V, sigma, w, v, scalars, dL_dsigma, dL_dX, s);
}

int esmf_fock_build_shard(esmf_fock_t *h, int shard, int nshards, int m, const double *D, double *J,
                          double *K, double *F, double *traces, void *stream) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    if (nshards < 1 || shard < 0 || shard >= nshards) {
        set_error("shard %d of %d", shard, nshards);
        return ESMF_ERR_INVALID_ARG;
    }
    if (h->mode == ESMF_MODE_DF || h->mode == ESMF_MODE_THC) {
        set_error("density-fitted and hypercontracted handles are not sharded");
        return ESMF_ERR_UNSUPPORTED;
    }
    // shard s takes bricks [cut(s), cut(s + 1)): equal shares of the estimated
    // cost (the tensor-kernel cost model of the per-CTA split), each cut moved
    // forward to the next item start so that no item is divided between shards
    auto cut = [&](int k) -> int64_t {
        const int64_t n = h->nbricks;
        if (k <= 0) return 0;
        if (k >= nshards || (int64_t)h->cost_prefix.size() != n + 1) return k >= nshards ? n : n * k / nshards;
        const double target = h->cost_prefix[n] * k / nshards;
        int64_t j = std::lower_bound(h->cost_prefix.begin(), h->cost_prefix.end(), target) - h->cost_prefix.begin();
        if (j > n) j = n;
        while (j < n && !(h->hbricks[j].pad & BRICK_ITEM_FIRST)) ++j;
        return j;
    };
    const int64_t b0 = cut(shard), b1 = std::max(b0, cut(shard + 1));
    return build_range(h, b0, b1, m, D, J, K, F, traces, stream);
}

int esmf_fock_build_host(esmf_fock_t *h, int m, const double *D_host, double *J_host, double *K_host,
                         double *F_host, double *traces_host, void *stream, int timeout_ms) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    if (m < 1 || m > ESMF_MAX_DENSITIES) { set_error("m = %d outside [1, %d]", m, ESMF_MAX_DENSITIES); return ESMF_ERR_INVALID_ARG; }
    if (!D_host || !J_host || !K_host) { set_error("D, J and K are required"); return ESMF_ERR_INVALID_ARG; }
    DeviceGuard g(h->device);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    const size_t mat = (size_t)h->n * h->n;
    if (m > h->stage_m) {
        dfree(h, &h->sD, (size_t)h->stage_m * mat); dfree(h, &h->sJ, (size_t)h->stage_m * mat);
        dfree(h, &h->sK, (size_t)h->stage_m * mat); dfree(h, &h->sF, (size_t)h->stage_m * mat);
        dfree(h, &h->st, (size_t)h->stage_m);
        h->stage_m = 0;
        RET(dalloc(h, &h->sD, m * mat)); RET(dalloc(h, &h->sJ, m * mat)); RET(dalloc(h, &h->sK, m * mat));
        RET(dalloc(h, &h->sF, m * mat)); RET(dalloc(h, &h->st, (size_t)m));
        h->stage_m = m;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * m * mat;
    CKR(cudaMemcpyAsync(h->sD, D_host, bytes, cudaMemcpyHostToDevice, s));
    RET(esmf_fock_build(h, m, h->sD, h->sJ, h->sK, F_host ? h->sF : nullptr, traces_host ? h->st : nullptr, s));
    CKR(cudaMemcpyAsync(J_host, h->sJ, bytes, cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(K_host, h->sK, bytes, cudaMemcpyDeviceToHost, s));
    if (F_host) CKR(cudaMemcpyAsync(F_host, h->sF, bytes, cudaMemcpyDeviceToHost, s));
    if (traces_host) CKR(cudaMemcpyAsync(traces_host, h->st, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->done, s));
    // bounded wait: poll the event, give up after timeout_ms
    const int limit = timeout_ms > 0 ? timeout_ms : 600000;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(h->done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) { set_error("build: %s", cudaGetErrorString(q)); return ESMF_ERR_CUDA; }
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > limit) { set_error("build did not finish within %d ms", limit); return ESMF_ERR_TIMEOUT; }
        // spin (yielding) for the first 5 ms so that a sub-millisecond build is
        // picked up without sleep granularity, then poll every 20 us
        if (ms < 5.0) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (*(volatile int *)h->err_host) {
        set_error("a bounded wait inside the contraction kernel expired (code %d)", *(volatile int *)h->err_host);
        return ESMF_ERR_TIMEOUT;
    }
    return ESMF_OK;
}

int esmf_fock_set_density_screening(esmf_fock_t *h, double tol_d) {
    if (!h || !(tol_d >= 0.0) || !is_finite(tol_d)) {
        set_error("density screening needs a handle and a finite tol_d >= 0");
        return ESMF_ERR_INVALID_ARG;
    }
    if (h->mode == ESMF_MODE_DF || h->mode == ESMF_MODE_THC) {
        set_error("density-fitted and hypercontracted builds have no quartets to screen");
        return ESMF_ERR_UNSUPPORTED;
    }
    h->tol_d = tol_d;
    return ESMF_OK;
}

int esmf_fock_set_path(esmf_fock_t *h, int path) {
    if (!h || path < ESMF_PATH_AUTO || path > ESMF_PATH_CUDA_CORE) { set_error("bad handle or path"); return ESMF_ERR_INVALID_ARG; }
    h->path = path;
    return ESMF_OK;
}

int esmf_fock_autotune(esmf_fock_t *h, int m, const double *D, double *J, double *K, int reps,
                       void *stream, int *chosen) {
    if (!h || m < 1 || m > ESMF_MAX_DENSITIES || !D || !J || !K) { set_error("bad autotune arguments"); return ESMF_ERR_INVALID_ARG; }
    if (h->mode == ESMF_MODE_DF || h->mode == ESMF_MODE_THC) {
        set_error("density-fitted and hypercontracted handles have nothing to tune");
        return ESMF_ERR_UNSUPPORTED;
    }
    DeviceGuard g(h->device);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    const bool tensor = (h->mode == ESMF_MODE_STORED || tensor_direct(h)) && is_split16(h->prec) &&
                        h->path != ESMF_PATH_CUDA_CORE;
    std::vector<int> cand;
    if (tensor) { cand.push_back(16); if (m > 8) cand.push_back(8); }
    else if (h->prec == ESMF_PREC_FP64 || h->prec == ESMF_PREC_F32X2) { cand.push_back(8); cand.push_back(4); }
    else { cand.push_back(16); cand.push_back(8); cand.push_back(4); }
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CKR(cudaEventCreate(&e0));
    CKR(cudaEventCreate(&e1));
    int best = cand[0];
    float best_ms = 0.f;
    int rc = ESMF_OK;
    for (int c : cand) {
        h->force_chunk = c;
        if ((rc = esmf_fock_build(h, m, D, J, K, nullptr, nullptr, s)) != ESMF_OK) break;   // warm-up
        std::vector<float> t;
        for (int r = 0; r < reps && rc == ESMF_OK; ++r) {
            cudaEventRecord(e0, s);
            rc = esmf_fock_build(h, m, D, J, K, nullptr, nullptr, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = ESMF_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms);
        }
        if (rc != ESMF_OK) break;
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (c == cand[0] || med < best_ms) { best = c; best_ms = med; }
    }
    h->force_chunk = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ESMF_OK) return rc;
    bool found = false;
    for (auto &t : h->tuned)
        if (t.first == m) { t.second = best; found = true; }
    if (!found) h->tuned.push_back({m, best});
    if (chosen) *chosen = best;
    return ESMF_OK;
}

int esmf_fock_device_error(esmf_fock_t *h, int reset) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    const int v = *(volatile int *)h->err_host;
    if (reset) *(volatile int *)h->err_host = 0;
    return v;
}

int esmf_fock_set_timing(esmf_fock_t *h, int enable) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    h->timing = enable != 0;
    return ESMF_OK;
}

int esmf_fock_kernel_time(esmf_fock_t *h, double *ms, int64_t *launches, int reset) {
    if (!h || !ms || !launches) { set_error("NULL argument"); return ESMF_ERR_INVALID_ARG; }
    DeviceGuard g(h->device);
    double tot = 0.0;
    for (size_t i = 0; i < h->ev_used; ++i) {
        CKR(cudaEventSynchronize(h->ev_pool[i].second));
        float x = 0.f;
        CKR(cudaEventElapsedTime(&x, h->ev_pool[i].first, h->ev_pool[i].second));
        tot += x;
    }
    *ms = tot;
    *launches = (int64_t)h->ev_used;
    if (reset) h->ev_used = 0;
    return ESMF_OK;
}

int esmf_fock_stats(const esmf_fock_t *h, esmf_stats_t *out) {
    if (!h || !out) { set_error("NULL argument"); return ESMF_ERR_INVALID_ARG; }
    const int64_t P = (int64_t)h->n * (h->n + 1) / 2;
    out->n_basis = h->n;
    out->n_pairs = P;
    out->n_quartets_unique = P * (P + 1) / 2;
    out->n_quartets_kept = h->n_kept_unique;
    out->n_bricks = h->nbricks;
    out->n_stored = h->mode == ESMF_MODE_STORED ? h->n_stored : 0;
    out->store_bytes = h->store_bytes;
    out->device_bytes = h->device_bytes;
    out->mode = h->mode;
    out->precision = h->prec;
    out->schwarz_tol = h->tol;
    out->create_ms = h->create_ms;
    out->screening = h->screening;
    out->n_pairs_kept = h->n_pairs_kept;
    out->n_chunks = h->chunks.empty() ? 0 : (int64_t)h->chunks.size() - 1;
    out->scratch_bytes = h->scratch_bytes;
    return ESMF_OK;
}

int esmf_fock_schwarz(const esmf_fock_t *h, double *Q_host) {
    if (!h || !Q_host) { set_error("NULL argument"); return ESMF_ERR_INVALID_ARG; }
    DeviceGuard g(h->device);
    CKR(cudaMemcpy2D(Q_host, sizeof(double) * h->n, h->Q, sizeof(double) * h->np, sizeof(double) * h->n,
                     h->n, cudaMemcpyDeviceToHost));
    return ESMF_OK;
}

void esmf_fock_destroy(esmf_fock_t *h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    release(h);
}

}  // extern "C"

namespace esmf {

// Fills the contraction arguments of handle h for m densities D without
// touching its work memory (the caller supplies the accumulators).
int handle_prepare_noalloc(esmf_fock_t *h, int m, const double *D, JKArgs *a, int *device,
                           bool *split) {
    if (h->tol_d > 0.0) {
        set_error("density-weighted screening needs per-build work memory; the no-alloc entry does not apply it");
        return ESMF_ERR_UNSUPPORTED;
    }
    if (h->mode == ESMF_MODE_DF || h->mode == ESMF_MODE_THC) {
        set_error("density-fitted and hypercontracted builds need per-build GEMM work memory; the no-alloc "
                  "entry does not run them");
        return ESMF_ERR_UNSUPPORTED;
    }
    a->b = h->dev(); a->Q = h->S; a->tol = h->tol_s; a->bricks = h->bricks; a->nbricks = h->nbricks;
    a->offsets = h->offsets; a->store = h->store; a->precision = h->prec; a->mode = h->mode;
    a->m = m; a->D = D; a->Jacc = nullptr; a->Kacc = nullptr;
    a->vscale = h->vscale;
    a->ptab = h->ptab; a->pslot = h->pslot;
    // densities per pass as esmf_fock_build picks them (autotuned or forced);
    // a tensor-core choice of 16 has no CUDA-core meaning for FP64 and falls
    // back to that kernel's default
    int chunk = h->force_chunk;
    if (!chunk)
        for (auto &t : h->tuned)
            if (t.first == m) chunk = t.second;
    a->mc = chunk;
    *device = h->device;
    *split = h->mode == ESMF_MODE_STORED && is_split16(h->prec);
    return ESMF_OK;
}

}  // namespace esmf

namespace esmf {

// Grow the handle's work memory for builds with m densities now (so that a
// later build, e.g. one being captured into a CUDA graph, allocates nothing).
int handle_reserve(esmf_fock_t *h, int m) {
    if (!h || m < 1 || m > ESMF_MAX_DENSITIES) { set_error("bad reserve arguments"); return ESMF_ERR_INVALID_ARG; }
    DeviceGuard g(h->device);
    if (!g.ok) { set_error("cudaSetDevice failed"); return ESMF_ERR_CUDA; }
    return ensure_work(h, m);
}

}  // namespace esmf
