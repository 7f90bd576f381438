// Contracted Cartesian p and d functions on the device: normalisation, the
// Schwarz table and the integral store for bases that mix s, p and d shells.
// The integrals (angular.cuh) follow the Obara-Saika and Head-Gordon-Pople
// recurrences for s and p functions and the McMurchie-Davidson scheme for
// quartets with a d function, in FP64.  Every other step of a build
// (screening, the contraction kernels, finalisation) works on the integral
// values by function index and is the same as for s functions.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "angular.cuh"
#include "esmf_internal.cuh"
#include "integrals.cuh"

namespace esmf {

using namespace angular;

namespace {

#define CKA(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                    \
            return ESMF_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

int grid_a(int64_t work, int per_block, int cap = 152 * 32) {
    int64_t g = (work + per_block - 1) / per_block;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// normalisation: a primitive N x^lx y^ly z^lz exp(-a r^2) (l = lx + ly + lz,
// powers of the offsets from its centre) has unit norm for
// N = (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2lx-1)!! (2ly-1)!! (2lz-1)!!); two of
// one label on one centre overlap N_k N_l (pi/s)^{3/2} (2lx-1)!! (2ly-1)!!
// (2lz-1)!! / (2s)^l with s = a_k + a_l (the Gaussian moments
// int x^{2n} exp(-s x^2) dx = (2n-1)!! / (2s)^n sqrt(pi/s)).
__global__ void k_normalize_l(int n, const int *nprim, const int *poff, const int *cart, const double *exps,
                              const double *coefs, double *w) {
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= n) return;
    const int o = poff[mu], np_ = nprim[mu];
    int v[3];
    label_exps(cart[mu], v);
    const int l = v[0] + v[1] + v[2];
    const double df = (v[0] == 2 ? 3.0 : 1.0) * (v[1] == 2 ? 3.0 : 1.0) * (v[2] == 2 ? 3.0 : 1.0);
    const double pi = 3.14159265358979323846;
    auto nrm = [&](double a) { return pow(2.0 * a / pi, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(df); };
    double s = 0.0;
    for (int k = 0; k < np_; ++k)
        for (int j = 0; j < np_; ++j) {
            const double ak = exps[o + k], aj = exps[o + j], sum = ak + aj;
            const double ov = pow(pi / sum, 1.5) * df / pow(2.0 * sum, (double)l);
            s += coefs[o + k] * coefs[o + j] * nrm(ak) * nrm(aj) * ov;
        }
    const double c = rsqrt(s);
    for (int k = 0; k < np_; ++k) w[o + k] = c * coefs[o + k] * nrm(exps[o + k]);
}

__global__ void k_schwarz_l(DevBasis b, double *Q) {
    const int64_t npair = (int64_t)b.np * (b.np + 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npair; t += (int64_t)gridDim.x * blockDim.x) {
        int p = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((int64_t)p * (p + 1) / 2 > t) --p;
        while ((int64_t)(p + 1) * (p + 2) / 2 <= t) ++p;
        const int q = (int)(t - (int64_t)p * (p + 1) / 2);
        double v = 0.0;
        if (p < b.n && q < b.n) v = sqrt(fmax(contracted_l(b, p, q, p, q), 0.0));
        Q[(int64_t)p * b.np + q] = v;
        Q[(int64_t)q * b.np + p] = v;
    }
}

// The store of a basis with p functions: one CTA per brick at a time, kept
// elements from the Schwarz rule (as for s bases), each evaluated by one
// thread in FP64 and written in the store's format.
template <int PREC>
__global__ void __launch_bounds__(256) k_brick_generate_l(DevBasis b, const double *Q, double tol,
                                                          const BrickDesc *bricks, int64_t nbricks,
                                                          const int64_t *offsets, void *store, float vscale) {
    __shared__ int wsum[16];
    __shared__ unsigned short klist[BRICK];
    __shared__ double qb[64], qk[64];
    for (int64_t bi = blockIdx.x; bi < nbricks; bi += gridDim.x) {
        const BrickDesc d = bricks[bi];
        __syncthreads();
        if (threadIdx.x < 64) {
            const int t = threadIdx.x;
            qb[t] = Q[(int64_t)(d.P * 8 + (t >> 3)) * b.np + d.Q * 8 + (t & 7)];
            qk[t] = Q[(int64_t)(d.R * 8 + (t >> 3)) * b.np + d.S * 8 + (t & 7)];
        }
        __syncthreads();
        const int e0 = threadIdx.x * 16;
        unsigned mask = 0;
        for (int j = 0; j < 16; ++j) {
            const int e = e0 + j;
            const int p = e >> 9, q = (e >> 6) & 7, r = (e >> 3) & 7, s = e & 7;
            const bool in = d.P * 8 + p < b.n && d.Q * 8 + q < b.n && d.R * 8 + r < b.n && d.S * 8 + s < b.n;
            if (in && qb[p * 8 + q] * qk[r * 8 + s] >= tol) mask |= 1u << j;
        }
        // exclusive scan of the per-thread counts (256 threads, 8 warps)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, cnt = __popc(mask);
        int x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < 8; ++w) { const int t = wsum[w]; wsum[8 + w] = acc; acc += t; }
            wsum[0] = acc;   // total (wsum[0..7] are not needed any more)
        }
        __syncthreads();
        int pos = wsum[8 + wid] + x - cnt;
        const int total = wsum[0];
        for (int j = 0; j < 16; ++j)
            if (mask & (1u << j)) klist[pos++] = (unsigned short)(e0 + j);
        constexpr int EB = (PREC == 0 || PREC == 4) ? 8 : 4;
        const int64_t base = offsets[bi];
        unsigned char *mk = reinterpret_cast<unsigned char *>(store) + base * EB;
        mk[2 * threadIdx.x] = (unsigned char)(mask & 0xffu);
        mk[2 * threadIdx.x + 1] = (unsigned char)(mask >> 8);
        const int64_t vbase = base + MASK_BYTES / EB;
        __syncthreads();
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int e = klist[i];
            const int p = d.P * 8 + (e >> 9), q = d.Q * 8 + ((e >> 6) & 7), r = d.R * 8 + ((e >> 3) & 7),
                      s = d.S * 8 + (e & 7);
            const double v = contracted_l(b, p, q, r, s);
            if (PREC == 0) {
                reinterpret_cast<double *>(store)[vbase + i] = v;
            } else if (PREC == 1) {
                reinterpret_cast<float *>(store)[vbase + i] = (float)v;
            } else if (PREC == 4) {
                const float hi = __double2float_rn(v);
                reinterpret_cast<float2 *>(store)[vbase + i] = make_float2(hi, __double2float_rn(v - (double)hi));
            } else {
                const double xs = v * (double)vscale;
                uint16_t hb, lb;
                if (PREC == 2) {
                    const __half h = __double2half(xs);
                    hb = __half_as_ushort(h);
                    lb = __half_as_ushort(__double2half(xs - (double)__half2float(h)));
                } else {
                    const __nv_bfloat16 h = __double2bfloat16(xs);
                    hb = __bfloat16_as_ushort(h);
                    lb = __bfloat16_as_ushort(__double2bfloat16(xs - (double)__bfloat162float(h)));
                }
                reinterpret_cast<uint32_t *>(store)[vbase + i] = (uint32_t)hb | ((uint32_t)lb << 16);
            }
        }
    }
}

}  // namespace

int launch_normalize_l(const DevBasis &b, const double *coefs, double *w, cudaStream_t s) {
    k_normalize_l<<<grid_a(b.n, 128), 128, 0, s>>>(b.n, b.nprim, b.poff, b.cart, b.exps, coefs, w);
    CKA(cudaGetLastError());
    return ESMF_OK;
}

int launch_schwarz_l(const DevBasis &b, double *Q, cudaStream_t s) {
    const int64_t npair = (int64_t)b.np * (b.np + 1) / 2;
    k_schwarz_l<<<grid_a(npair, 128), 128, 0, s>>>(b, Q);
    CKA(cudaGetLastError());
    return ESMF_OK;
}

int launch_brick_generate_l(const DevBasis &b, const double *Q, double tol, const BrickDesc *bricks,
                            int64_t nbricks, const int64_t *offsets, int precision, void *store, float vscale,
                            cudaStream_t s) {
    const int grid = grid_a(nbricks, 1, 152 * 8);
    switch (precision) {
        case ESMF_PREC_FP64:
            k_brick_generate_l<0><<<grid, 256, 0, s>>>(b, Q, tol, bricks, nbricks, offsets, store, vscale);
            break;
        case ESMF_PREC_F32X2:
            k_brick_generate_l<4><<<grid, 256, 0, s>>>(b, Q, tol, bricks, nbricks, offsets, store, vscale);
            break;
        case ESMF_PREC_FP32:
            k_brick_generate_l<1><<<grid, 256, 0, s>>>(b, Q, tol, bricks, nbricks, offsets, store, vscale);
            break;
        case ESMF_PREC_FP16X2:
            k_brick_generate_l<2><<<grid, 256, 0, s>>>(b, Q, tol, bricks, nbricks, offsets, store, vscale);
            break;
        case ESMF_PREC_BF16X2:
            k_brick_generate_l<3><<<grid, 256, 0, s>>>(b, Q, tol, bricks, nbricks, offsets, store, vscale);
            break;
        default:
            set_error("unknown precision %d", precision);
            return ESMF_ERR_INVALID_ARG;
    }
    CKA(cudaGetLastError());
    return ESMF_OK;
}

}  // namespace esmf
