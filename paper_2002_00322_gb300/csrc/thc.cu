// Least-squares tensor hypercontraction (THC) of the integrals, the other
// acceleration the paper names as future work (Sec. I), in the LS-THC form of
// Parrish, Hohenstein, Martinez and Sherrill (J. Chem. Phys. 137, 224106,
// 2012):  (pq|rs) ~ sum_PQ X_pP X_qP Z_PQ X_rQ X_sQ,  X_pP = phi_p(r_P).
//
// Create time (FP64): the collocation X on the device; the Coulomb matrix
// E_PQ = x_P^T J[x_Q x_Q^T] x_P of the grid's rank-one densities, from the
// library's own grouped J builds (this file forms the densities and reduces
// each J); S = (X^T X) o (X^T X); Z = (S + lam I)^-1 E (S + lam I)^-1 by four
// triangular solves against the host Cholesky factor of S + lam I, then
// symmetrised.  Every build is dense GEMMs plus elementwise kernels, per
// density k (Eq. J_and_K over the fitted integrals):
//   M_k = X^T D_k X                    M_PQ = sum_rs X_rP D_rs X_sQ
//   J_k = X diag(Z y_k) X^T,           y_k,Q = M_k,QQ
//   K_k = X (Z o M_k) X^T              K_pr = sum_PQ X_pP Z_PQ M_PQ X_rQ
// All matrices are row-major; a row-major A is the column-major A^T that
// cuBLAS sees, and every GEMM below is written for that view.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include "esmf_internal.cuh"

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

int grid_of(int64_t work) {
    int64_t g = (work + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

// X[p][P] = sum_k w_pk exp(-a_pk |r_P - A_p|^2), P fastest (coalesced writes)
__global__ void k_thc_collocate(DevBasis b, int G, const double *pts, double *X) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)b.n * G;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(t / G), P = (int)(t % G);
        const double dx = pts[3 * P] - b.center[3 * p], dy = pts[3 * P + 1] - b.center[3 * p + 1],
                     dz = pts[3 * P + 2] - b.center[3 * p + 2];
        const double d2 = dx * dx + dy * dy + dz * dz;
        double v = 0.0;
        for (int k = 0; k < b.nprim[p]; ++k) v += b.w[b.poff[p] + k] * exp(-b.exps[b.poff[p] + k] * d2);
        X[t] = v;
    }
}

// Dq[j][p][q] = X[p][q0 + j] X[q][q0 + j] for j < mq
__global__ void k_thc_rank_one(int n, int G, int q0, int mq, const double *X, double *Dq) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)mq * nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / nn);
        const int64_t x = t % nn;
        const int p = (int)(x / n), q = (int)(x % n);
        Dq[t] = X[(int64_t)p * G + q0 + j] * X[(int64_t)q * G + q0 + j];
    }
}

// E[P][q0 + j] = sum_p X[p][P] R_j[p][P], R_j = J_j X (n x G)
__global__ void k_thc_coulomb_cols(int n, int G, int q0, int mq, const double *X, const double *R, double *E) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)mq * G;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / G), P = (int)(t % G);
        const double *Rj = R + (int64_t)j * n * G;
        double e = 0.0;
        for (int p = 0; p < n; ++p) e += X[(int64_t)p * G + P] * Rj[(int64_t)p * G + P];
        E[(int64_t)P * G + q0 + j] = e;
    }
}

// Zout[i][j] = (T) ((W[i][j] + W[j][i]) / 2): symmetric to the last bit
template <typename T>
__global__ void k_thc_symmetrise(int G, const double *W, T *Zout) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)G * G;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / G), j = (int)(t % G);
        Zout[t] = (T)(0.5 * (W[t] + W[(int64_t)j * G + i]));
    }
}

template <typename T>
__global__ void k_thc_convert(int64_t cnt, const double *src, T *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// y[k][Q] = M[k][Q][Q]
template <typename T>
__global__ void k_thc_diag(int m, int G, const T *M, T *y) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)m * G;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / G), Q = (int)(t % G);
        y[t] = M[(int64_t)k * G * G + (int64_t)Q * G + Q];
    }
}

// Xz[k][p][P] = X[p][P] z[k][P]
template <typename T>
__global__ void k_thc_scale_cols(int m, int n, int G, const T *X, const T *z, T *Xz) {
    const int64_t nG = (int64_t)n * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)m * nG;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / nG);
        const int64_t x = t % nG;
        Xz[t] = X[x] * z[(int64_t)k * G + (int)(x % G)];
    }
}

// M[k][P][Q] *= Z[P][Q]
template <typename T>
__global__ void k_thc_hadamard(int m, int G, const T *Z, T *M) {
    const int64_t GG = (int64_t)G * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)m * GG;
         t += (int64_t)gridDim.x * blockDim.x)
        M[t] *= Z[t % GG];
}

}  // namespace

int launch_thc_collocate(const DevBasis &b, int G, const double *pts, double *X, cudaStream_t s) {
    k_thc_collocate<<<grid_of((int64_t)b.n * G), 256, 0, s>>>(b, G, pts, X);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

int launch_thc_rank_one(int n, int G, int q0, int mq, const double *X, double *Dq, cudaStream_t s) {
    k_thc_rank_one<<<grid_of((int64_t)mq * n * n), 256, 0, s>>>(n, G, q0, mq, X, Dq);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

// Columns q0 .. q0 + mq - 1 of E from the Coulomb matrices Jq (mq x n x n) of
// the rank-one densities: R_j = J_j X (batched), then the column reduction.
int thc_coulomb_columns(void *cublas, int n, int G, int q0, int mq, const double *X, const double *Jq, double *R,
                        double *E, cudaStream_t s) {
    cublasHandle_t hb = (cublasHandle_t)cublas;
    CKB(cublasSetStream(hb, s));
    CKB(cublasSetPointerMode(hb, CUBLAS_POINTER_MODE_HOST));
    const double one = 1.0, zero = 0.0;
    // R_j (row-major n x G) = J_j X; column-major R_j^T (G x n) = X^T J_j^T:
    // A = X seen as X^T (G x n, ld G), B = J_j seen as J_j^T (n x n, ld n)
    CKB(cublasDgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, G, n, n, &one, X, G, 0, Jq, n, (long long)n * n,
                                  &zero, R, G, (long long)n * G, mq));
    k_thc_coulomb_cols<<<grid_of((int64_t)mq * G), 256, 0, s>>>(n, G, q0, mq, X, R, E);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

// C (G x G) = X^T X
int thc_gram(void *cublas, int n, int G, const double *X, double *C, cudaStream_t s) {
    cublasHandle_t hb = (cublasHandle_t)cublas;
    CKB(cublasSetStream(hb, s));
    CKB(cublasSetPointerMode(hb, CUBLAS_POINTER_MODE_HOST));
    const double one = 1.0, zero = 0.0;
    // column-major C^T = X^T X: A = X seen as X^T (G x n, ld G), B = X^T transposed
    CKB(cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, G, G, n, &one, X, G, X, G, &zero, C, G));
    return ESMF_OK;
}

// W <- (L L^T)^-1 W (L L^T)^-1 in place, for symmetric W (the Coulomb matrix
// E), L lower triangular row-major (entries above the diagonal are ignored);
// then Zout = the symmetric part of W in the build arithmetic.  Column-major,
// the row-major L is the upper triangular U = L^T, and L L^T = U^T U:
//   W <- U^-T W,  W <- W U^-1,  W <- U^-1 W,  W <- W U^-T.
int thc_solve_z(void *cublas, int G, const double *L, double *W, int fp32, void *Zout, cudaStream_t s) {
    cublasHandle_t hb = (cublasHandle_t)cublas;
    CKB(cublasSetStream(hb, s));
    CKB(cublasSetPointerMode(hb, CUBLAS_POINTER_MODE_HOST));
    const double one = 1.0;
    CKB(cublasDtrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, G, G, &one, L,
                    G, W, G));
    CKB(cublasDtrsm(hb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, G, G, &one, L,
                    G, W, G));
    CKB(cublasDtrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, G, G, &one, L,
                    G, W, G));
    CKB(cublasDtrsm(hb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, G, G, &one, L,
                    G, W, G));
    if (fp32) k_thc_symmetrise<float><<<grid_of((int64_t)G * G), 256, 0, s>>>(G, W, (float *)Zout);
    else k_thc_symmetrise<double><<<grid_of((int64_t)G * G), 256, 0, s>>>(G, W, (double *)Zout);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

int launch_thc_convert(int64_t cnt, const double *src, float *dst, cudaStream_t s) {
    k_thc_convert<float><<<grid_of(cnt), 256, 0, s>>>(cnt, src, dst);
    CKD(cudaGetLastError());
    return ESMF_OK;
}

// One hypercontracted build of m densities (see the top of the file).  Work
// in the arithmetic type: Dt (m n^2, FP32 only), A (m n G: first X^T D_k,
// then X diag(z_k), then X (Z o M_k)), M (m G^2), y and z (m G each), Jt and
// Kt (m n^2 each); then J, K, F and the traces through the shared
// finalisation.
int thc_build(const ThcBuild &a, cudaStream_t s) {
    cublasHandle_t hb = (cublasHandle_t)a.cublas;
    CKB(cublasSetStream(hb, s));
    CKB(cublasSetPointerMode(hb, CUBLAS_POINTER_MODE_HOST));
    const int n = a.n, G = a.G, m = a.m;
    const long long nn = (long long)n * n, nG = (long long)n * G, GG = (long long)G * G;
    const cudaDataType_t ty = a.fp32 ? CUDA_R_32F : CUDA_R_64F;
    const cublasComputeType_t ct = a.fp32 ? CUBLAS_COMPUTE_32F : CUBLAS_COMPUTE_64F;
    const double one_d = 1.0, zero_d = 0.0;
    const float one_f = 1.0f, zero_f = 0.0f;
    const void *one = a.fp32 ? (const void *)&one_f : (const void *)&one_d;
    const void *zero = a.fp32 ? (const void *)&zero_f : (const void *)&zero_d;
    const void *Dw = a.D;
    if (a.fp32) {
        k_thc_convert<float><<<grid_of(m * nn), 256, 0, s>>>(m * nn, a.D, (float *)a.Dt);
        CKD(cudaGetLastError());
        Dw = a.Dt;
    }
    // A_k (row-major G x n) = X^T D_k; column-major A_k^T (n x G) = D_k^T X:
    // A = D_k seen as D_k^T (n x n, ld n), B = X seen as X^T (G x n, ld G) transposed
    CKB(cublasGemmStridedBatchedEx(hb, CUBLAS_OP_N, CUBLAS_OP_T, n, G, n, one, Dw, ty, n, nn, a.X, ty, G, 0, zero,
                                   a.A, ty, n, nG, m, ct, CUBLAS_GEMM_DEFAULT));
    // M_k (row-major G x G) = A_k X; column-major M_k^T = X^T A_k^T:
    // A = X seen as X^T (G x n, ld G), B = A_k seen as A_k^T (n x G, ld n)
    CKB(cublasGemmStridedBatchedEx(hb, CUBLAS_OP_N, CUBLAS_OP_N, G, G, n, one, a.X, ty, G, 0, a.A, ty, n, nG, zero,
                                   a.M, ty, G, GG, m, ct, CUBLAS_GEMM_DEFAULT));
    if (a.fp32) k_thc_diag<float><<<grid_of(m * (int64_t)G), 256, 0, s>>>(m, G, (const float *)a.M, (float *)a.y);
    else k_thc_diag<double><<<grid_of(m * (int64_t)G), 256, 0, s>>>(m, G, (const double *)a.M, (double *)a.y);
    CKD(cudaGetLastError());
    // z (row-major m x G) = y Z^T, z_k = Z y_k; column-major z^T (G x m) = Z y^T:
    // A = Z seen as Z^T (ld G) transposed, B = y seen as y^T (G x m, ld G)
    CKB(cublasGemmEx(hb, CUBLAS_OP_T, CUBLAS_OP_N, G, m, G, one, a.Z, ty, G, a.y, ty, G, zero, a.z, ty, G, ct,
                     CUBLAS_GEMM_DEFAULT));
    if (a.fp32)
        k_thc_scale_cols<float><<<grid_of(m * nG), 256, 0, s>>>(m, n, G, (const float *)a.X, (const float *)a.z,
                                                                 (float *)a.A);
    else
        k_thc_scale_cols<double><<<grid_of(m * nG), 256, 0, s>>>(m, n, G, (const double *)a.X, (const double *)a.z,
                                                                  (double *)a.A);
    CKD(cudaGetLastError());
    // J_k (row-major n x n) = (X diag z_k) X^T; column-major J_k^T = X (X diag z_k)^T:
    // A = X seen as X^T (ld G) transposed (n x G), B = X diag z_k seen as its transpose (G x n, ld G)
    CKB(cublasGemmStridedBatchedEx(hb, CUBLAS_OP_T, CUBLAS_OP_N, n, n, G, one, a.X, ty, G, 0, a.A, ty, G, nG, zero,
                                   a.Jt, ty, n, nn, m, ct, CUBLAS_GEMM_DEFAULT));
    if (a.fp32) k_thc_hadamard<float><<<grid_of(m * GG), 256, 0, s>>>(m, G, (const float *)a.Z, (float *)a.M);
    else k_thc_hadamard<double><<<grid_of(m * GG), 256, 0, s>>>(m, G, (const double *)a.Z, (double *)a.M);
    CKD(cudaGetLastError());
    // W_k (row-major n x G) = X (Z o M_k); column-major W_k^T (G x n) = (Z o M_k)^T X^T:
    // A = Z o M_k seen as its transpose (G x G, ld G), B = X seen as X^T (G x n, ld G)
    CKB(cublasGemmStridedBatchedEx(hb, CUBLAS_OP_N, CUBLAS_OP_N, G, n, G, one, a.M, ty, G, GG, a.X, ty, G, 0, zero,
                                   a.A, ty, G, nG, m, ct, CUBLAS_GEMM_DEFAULT));
    // K_k (row-major n x n) = W_k X^T; column-major K_k^T = X W_k^T:
    // A = X seen as X^T (ld G) transposed (n x G), B = W_k seen as W_k^T (G x n, ld G)
    CKB(cublasGemmStridedBatchedEx(hb, CUBLAS_OP_T, CUBLAS_OP_N, n, n, G, one, a.X, ty, G, 0, a.A, ty, G, nG, zero,
                                   a.Kt, ty, n, nn, m, ct, CUBLAS_GEMM_DEFAULT));
    return launch_factored_finalize(n, m, a.fp32, a.D, a.Jt, a.Kt, a.J, a.K, a.F, a.traces, s);
}

}  // namespace esmf
