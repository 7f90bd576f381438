// Density-fitted J and K (the acceleration the paper names as future work,
// Sec. I), GB300 path: three- and two-centre integrals over auxiliary s
// Gaussians on the device, the Coulomb-metric fit folded into one factor
// B = L^-1 T (V = L L^T, T_P,pq = (pq|P)) at create time, and every build as
// dense GEMMs on cuBLAS (FP64 or FP32 arithmetic):
//   g_k = B vec(D_k),  J_k = B^T g_k            (J_pq = sum_P B_P,pq g_k,P)
//   K_k[p][q] = sum_{P,s} (B''_p D_k)[P][s] B''_q[P][s],  B''[p][P][r] = B_P,pr
// i.e. K_pq = sum_rs D_rs sum_P B_P,pr B_P,qs, Eq. (J_and_K) over the fitted
// integrals (pq|rs) ~ sum_P B_P,pq B_P,rs.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include "esmf_internal.cuh"
#include "integrals.cuh"

namespace esmf {

namespace {

#define CKD(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                    \
            return ESMF_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

#define CKB(call)                                                                  \
    do {                                                                           \
        cublasStatus_t s_ = (call);                                                \
        if (s_ != CUBLAS_STATUS_SUCCESS) {                                         \
            set_error("%s: cuBLAS status %d", #call, (int)s_);                     \
            return ESMF_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

// (pq|P) for p >= q (mirrored), one thread per (P, pair): the contracted sum
// over primitive pairs of the textbook [ab|c] closed form.
__global__ void k_df_eri3(DevBasis b, int naux, const double *acen, const double *aexp, double *T) {
    const int64_t npair = (int64_t)b.n * (b.n + 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npair * naux;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int P = (int)(t / npair);
        const int64_t pr = t % npair;
        int p = (int)((sqrt(8.0 * (double)pr + 1.0) - 1.0) * 0.5);
        while ((int64_t)p * (p + 1) / 2 > pr) --p;
        while ((int64_t)(p + 1) * (p + 2) / 2 <= pr) ++p;
        const int q = (int)(pr - (int64_t)p * (p + 1) / 2);
        const double c = aexp[P], cx = acen[3 * P], cy = acen[3 * P + 1], cz = acen[3 * P + 2];
        const double ax = b.center[3 * p], ay = b.center[3 * p + 1], az = b.center[3 * p + 2];
        const double bx = b.center[3 * q], by = b.center[3 * q + 1], bz = b.center[3 * q + 2];
        const double ab2 = (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
        double v = 0.0;
        for (int i = 0; i < b.nprim[p]; ++i)
            for (int j = 0; j < b.nprim[q]; ++j) {
                const double ea = b.exps[b.poff[p] + i], eb = b.exps[b.poff[q] + j];
                const double pe = ea + eb;
                const double px = (ea * ax + eb * bx) / pe, py = (ea * ay + eb * by) / pe, pz = (ea * az + eb * bz) / pe;
                const double pc2 = (px - cx) * (px - cx) + (py - cy) * (py - cy) + (pz - cz) * (pz - cz);
                v += b.w[b.poff[p] + i] * b.w[b.poff[q] + j] * exp(-ea * eb / pe * ab2) * kTwoPi52 /
                     (pe * c * sqrt(pe + c)) * boys0_d(pe * c / (pe + c) * pc2);
            }
        T[((int64_t)P * b.n + p) * b.n + q] = v;
        T[((int64_t)P * b.n + q) * b.n + p] = v;
    }
}

// (P|Q) between auxiliaries
__global__ void k_df_eri2(int naux, const double *acen, const double *aexp, double *V) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)naux * naux;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int P = (int)(t / naux), Q = (int)(t % naux);
        const double c = aexp[P], d = aexp[Q];
        const double dx = acen[3 * P] - acen[3 * Q], dy = acen[3 * P + 1] - acen[3 * Q + 1],
                     dz = acen[3 * P + 2] - acen[3 * Q + 2];
        V[t] = kTwoPi52 / (c * d * sqrt(c + d)) * boys0_d(c * d / (c + d) * (dx * dx + dy * dy + dz * dz));
    }
}

// B[P][p][q] -> B2[p][P][q], in the build's arithmetic type (B itself is
// also converted when the arithmetic is FP32: Bout may alias nothing).
template <typename T>
__global__ void k_df_layouts(int naux, int n, const double *B, T *Bout, T *B2) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)naux * nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int P = (int)(t / nn);
        const int64_t x = t % nn;
        const int p = (int)(x / n), q = (int)(x % n);
        const T v = (T)B[t];
        if (Bout) Bout[t] = v;
        B2[((int64_t)p * naux + P) * n + q] = v;
    }
}

template <typename T>
__global__ void k_to_type(int64_t cnt, const double *src, T *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// F = 2 J - K and t_k = D_k . F_k from the arithmetic-type J, K of a build;
// writes the caller's FP64 J, K (and F).  One block per (row p, density k).
template <typename T>
__global__ void k_df_finalize(int n, const double *D, const T *Jt, const T *Kt, double *J, double *K, double *F,
                              double *tsum) {
    const int p = blockIdx.x, k = blockIdx.y;
    const int64_t row = (int64_t)k * n * n + (int64_t)p * n;
    double part = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const double jv = (double)Jt[row + q], kv = (double)Kt[row + q];
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

int grid_of(int64_t work) {
    int64_t g = (work + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

int launch_df_integrals(const DevBasis &b, int naux, const double *acen, const double *aexp, double *T, double *V,
                        cudaStream_t s) {
    const int64_t npair = (int64_t)b.n * (b.n + 1) / 2;
    k_df_eri3<<<grid_of(npair * naux), 256, 0, s>>>(b, naux, acen, aexp, T);
    CKD(cudaGetLastError());
    k_df_eri2<<<grid_of((int64_t)naux * naux), 256, 0, s>>>(naux, acen, aexp, V);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

int launch_df_layouts(int naux, int n, const double *B, int fp32, void *Bout, void *B2, cudaStream_t s) {
    const int g = grid_of((int64_t)naux * n * n);
    if (fp32) k_df_layouts<float><<<g, 256, 0, s>>>(naux, n, B, (float *)Bout, (float *)B2);
    else k_df_layouts<double><<<g, 256, 0, s>>>(naux, n, B, nullptr, (double *)B2);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

// One density-fitted build (see the top of the file).  work: Dt, Jt, Kt
// (m n^2 each, arithmetic type; Dt unused in FP64), g (m naux), Y (naux n^2).
int df_build(const DfBuild &a, cudaStream_t s) {
    cublasHandle_t hb = (cublasHandle_t)a.cublas;
    CKB(cublasSetStream(hb, s));
    CKB(cublasSetPointerMode(hb, CUBLAS_POINTER_MODE_HOST));
    const int n = a.n, naux = a.naux, m = a.m;
    const int64_t nn = (int64_t)n * n;
    const cudaDataType_t ty = a.fp32 ? CUDA_R_32F : CUDA_R_64F;
    const cublasComputeType_t ct = a.fp32 ? CUBLAS_COMPUTE_32F : CUBLAS_COMPUTE_64F;
    const double one_d = 1.0, zero_d = 0.0;
    const float one_f = 1.0f, zero_f = 0.0f;
    const void *one = a.fp32 ? (const void *)&one_f : (const void *)&one_d;
    const void *zero = a.fp32 ? (const void *)&zero_f : (const void *)&zero_d;
    const void *Dw = a.D;
    if (a.fp32) {
        k_to_type<float><<<grid_of(m * nn), 256, 0, s>>>(m * nn, a.D, (float *)a.Dt);
        CKD(cudaGetLastError());
        Dw = a.Dt;
    }
    if (a.ev_start) CKD(cudaEventRecord(a.ev_start, s));
    // g (column-major naux x m) = B (naux x n^2, row-major) . D^T
    CKB(cublasGemmEx(hb, CUBLAS_OP_T, CUBLAS_OP_N, naux, m, (int)nn, one, a.B, ty, (int)nn, Dw, ty, (int)nn, zero,
                     a.g, ty, naux, ct, CUBLAS_GEMM_DEFAULT));
    // J (column-major n^2 x m) = B^T g
    CKB(cublasGemmEx(hb, CUBLAS_OP_N, CUBLAS_OP_N, (int)nn, m, naux, one, a.B, ty, (int)nn, a.g, ty, naux, zero,
                     a.Jt, ty, (int)nn, ct, CUBLAS_GEMM_DEFAULT));
    const size_t es = a.fp32 ? 4 : 8;
    for (int k = 0; k < m; ++k) {
        const void *Dk = (const char *)Dw + (size_t)k * nn * es;
        void *Kk = (char *)a.Kt + (size_t)k * nn * es;
        // Y (row-major (n naux) x n) = B'' (row-major (n naux) x n) . D_k
        CKB(cublasGemmEx(hb, CUBLAS_OP_N, CUBLAS_OP_N, n, n * naux, n, one, Dk, ty, n, a.B2, ty, n, zero, a.Y, ty,
                         n, ct, CUBLAS_GEMM_DEFAULT));
        // K_k (row-major n x n) = Y (n x naux n) . B''^T
        CKB(cublasGemmEx(hb, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n * naux, one, a.B2, ty, n * naux, a.Y, ty, n * naux,
                         zero, Kk, ty, n, ct, CUBLAS_GEMM_DEFAULT));
    }
    if (a.ev_stop) CKD(cudaEventRecord(a.ev_stop, s));
    return launch_factored_finalize(n, m, a.fp32, a.D, a.Jt, a.Kt, a.J, a.K, a.F, a.traces, s);
}

int launch_factored_finalize(int n, int m, int fp32, const double *D, const void *Jt, const void *Kt, double *J,
                             double *K, double *F, double *traces, cudaStream_t s) {
    if (traces) CKD(cudaMemsetAsync(traces, 0, sizeof(double) * m, s));
    const int threads = n <= 128 ? 128 : 256;
    if (fp32)
        k_df_finalize<float><<<dim3(n, m), threads, 0, s>>>(n, D, (const float *)Jt, (const float *)Kt, J, K, F,
                                                            traces);
    else
        k_df_finalize<double><<<dim3(n, m), threads, 0, s>>>(n, D, (const double *)Jt, (const double *)Kt, J, K, F,
                                                             traces);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

int df_gemm_fold(void *cublas, int naux, int64_t nn, const double *Linv, const double *T, double *B, cudaStream_t s) {
    cublasHandle_t hb = (cublasHandle_t)cublas;
    CKB(cublasSetStream(hb, s));
    const double one = 1.0, zero = 0.0;
    // B (row-major naux x n^2) = Linv (row-major naux x naux) . T (row-major naux x n^2);
    // column-major: B^T = T^T Linv^T
    CKB(cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, (int)nn, naux, naux, &one, T, (int)nn, Linv, naux, &zero, B,
                    (int)nn));
    return ESMF_OK;
}

int df_cublas_create(void **out) {
    cublasHandle_t hb = nullptr;
    CKB(cublasCreate(&hb));
    *out = hb;
    return ESMF_OK;
}

void df_cublas_destroy(void *h) {
    if (h) cublasDestroy((cublasHandle_t)h);
}

}  // namespace esmf
