// Kernels of the ESMF energy and gradient (Sec. II.B.2, Eqs. esmf_energy_1b,
// esmf_energy_2b and the appendix derivatives): an FP64 GEMM for the O(N^3)
// matrix products, the elementwise assembly of the derivative matrices and a
// deterministic reduction of the scalar inner products.  The Fock-like
// builds themselves are the library's grouped contraction.
//
// Notation: Theta = first N_o rows of V, Gamma = last N_v rows; P = Theta^T
// Theta, T = Theta^T sigma Gamma, A = Gamma^T sigma^T sigma Gamma -
// Theta^T sigma sigma^T Theta; F_X = F[X] = 2 J[X] - K[X]; Fk = G + F_P (the
// closed-shell Fock matrix of the rotated reference); N2 = c0^2 + 2 |sigma|^2.
// With E_HF = (G + Fk) . P, the energy is
//   E = (N2 E_HF + 4 c0 Fk . T + 2 Fk . A + 2 F_T . T) / N2
// (E1 + E2 of the paper, its last E2 term read as 2 F[T] . T).
#include <cuda_runtime.h>

#include "esmf_internal.cuh"

#define RET_IF(x)                  \
    do {                           \
        int r_ = (x);              \
        if (r_ != ESMF_OK) return r_; \
    } while (0)

namespace esmf {

namespace {

constexpr int GK = 32;             // K step of the GEMM tiles

// One problem of a grouped FP64 GEMM: C (M x N) = alpha op(A) op(B) + beta C,
// row-major; op(A) is M x K (A stored K x M when ta), op(B) is K x N (B stored
// N x K when tb).
struct GemmProblem {
    int M, N, K, lda, ldb, ldc, ta, tb;
    double alpha, beta;
    const double *A, *B;
    double *C;
};
constexpr int MAX_GROUP = 8;
struct GemmGroup {
    GemmProblem p[MAX_GROUP];
    int tiles[MAX_GROUP + 1];          // prefix sums of the problems' tile counts
    int count;
};

// Independent GEMMs in one launch.  GB300's FP64 pipe is narrow (about two
// FMAs per clock per SM), so the small O(N^3) products must spread over all
// SMs: tile T x T outputs, (T/R)^2 threads each owning an R x R strided patch
// (rows ty + (T/R) i, columns tx + (T/R) j); the tile's operand loads are
// unrolled so their latencies overlap.
template <int T, int R>
__global__ void __launch_bounds__((T / R) * (T / R)) k_gemm_group(const __grid_constant__ GemmGroup g) {
    constexpr int S = T / R, NT = S * S, LOADS = T * GK / NT;
    static_assert(T * GK % NT == 0, "tile loads");
    __shared__ double As[GK][T + 1];
    __shared__ double Bs[GK][T + 1];
    int q = 0;
    while (q + 1 < g.count && (int)blockIdx.x >= g.tiles[q + 1]) ++q;
    const GemmProblem &P = g.p[q];
    const int tile = blockIdx.x - g.tiles[q];
    const int tn = (P.N + T - 1) / T;
    const int m0 = (tile / tn) * T, n0 = (tile % tn) * T;
    const int t = threadIdx.x, tx = t % S, ty = t / S;
    double acc[R][R] = {};
    for (int k0 = 0; k0 < P.K; k0 += GK) {
        double va[LOADS], vb[LOADS];
#pragma unroll
        for (int r = 0; r < LOADS; ++r) {
            const int e = t + NT * r;
            const int mm = P.ta ? e % T : e / GK, kk = P.ta ? e / T : e % GK;
            const int gm = m0 + mm, gk = k0 + kk;
            va[r] = (gm < P.M && gk < P.K) ? (P.ta ? P.A[(size_t)gk * P.lda + gm] : P.A[(size_t)gm * P.lda + gk]) : 0.0;
            const int nn = P.tb ? e / GK : e % T, kb = P.tb ? e % GK : e / T;
            const int gn = n0 + nn, gkb = k0 + kb;
            vb[r] = (gn < P.N && gkb < P.K) ? (P.tb ? P.B[(size_t)gn * P.ldb + gkb] : P.B[(size_t)gkb * P.ldb + gn]) : 0.0;
        }
#pragma unroll
        for (int r = 0; r < LOADS; ++r) {
            const int e = t + NT * r;
            const int mm = P.ta ? e % T : e / GK, kk = P.ta ? e / T : e % GK;
            As[kk][mm] = va[r];
            const int nn = P.tb ? e / GK : e % T, kb = P.tb ? e % GK : e / T;
            Bs[kb][nn] = vb[r];
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GK; ++kk) {
            double a[R], b[R];
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = As[kk][ty + S * i];
#pragma unroll
            for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + S * j];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int gm = m0 + ty + S * i;
        if (gm >= P.M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int gn = n0 + tx + S * j;
            if (gn >= P.N) continue;
            double *c = P.C + (size_t)gm * P.ldc + gn;
            *c = P.beta == 0.0 ? P.alpha * acc[i][j] : fma(P.alpha, acc[i][j], P.beta * *c);
        }
    }
}

GemmProblem gp(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
               int ldb, double beta, double *C, int ldc) {
    GemmProblem p;
    p.M = M; p.N = N; p.K = K; p.lda = lda; p.ldb = ldb; p.ldc = ldc; p.ta = ta; p.tb = tb;
    p.alpha = alpha; p.beta = beta; p.A = A; p.B = B; p.C = C;
    return p;
}

int tiles_of(const GemmProblem &p, int T) { return ((p.M + T - 1) / T) * ((p.N + T - 1) / T); }

// Fk = G + F_P and M1 = 4 c0 (F_T + F_T^T) + 2 (F_A + F_A^T) (the Theta-derivative
// contributions of F[P] . T and F[P] . A through F[P]).
__global__ void k_energy_fock(int n, double c0, const double *__restrict__ G, const double *__restrict__ F,
                              double *__restrict__ Fk, double *__restrict__ M1, int with_grad) {
    const size_t nn = (size_t)n * n;
    const double *FP = F, *FT = F + nn, *FA = F + 2 * nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        Fk[e] = G[e] + FP[e];
        if (with_grad) {
            const size_t p = e / n, q = e % n, tr = q * n + p;
            M1[e] = 4.0 * c0 * (FT[e] + FT[tr]) + 2.0 * (FA[e] + FA[tr]);
        }
    }
}

// Per-block partial sums of the five scalars the energy needs:
// (G + Fk) . P, Fk . T, Fk . A, F_T . T and |sigma|^2.
constexpr int DOT_BLOCKS = 256;
__global__ void __launch_bounds__(256) k_energy_dots(int n, int nsig, const double *__restrict__ G,
                                                     const double *__restrict__ Fk, const double *__restrict__ F,
                                                     const double *__restrict__ D, const double *__restrict__ sigma,
                                                     double *__restrict__ partial) {
    const size_t nn = (size_t)n * n;
    const double *P = D, *T = D + nn, *A = D + 2 * nn, *FT = F + nn;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const double fk = Fk[e];
        s[0] += (G[e] + fk) * P[e];
        s[1] += fk * T[e];
        s[2] += fk * A[e];
        s[3] += FT[e] * T[e];
    }
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)nsig; e += (size_t)gridDim.x * blockDim.x)
        s[4] += sigma[e] * sigma[e];
    __shared__ double red[8][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        partial[blockIdx.x * 5 + threadIdx.x] = v;
    }
}

// Sums the partials in a fixed order (warp k sums scalar k) and forms E and
// dE/dc0 (Eq. eng_der_c0): out = {E, dE/dc0}; sc = {E_HF, E, N2, Fk . T}.
__global__ void k_energy_scalars(double c0, const double *__restrict__ partial, double *__restrict__ out,
                                 double *__restrict__ sc) {
    __shared__ double tot[5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < 5) {
        double v = 0.0;
        for (int b = lane; b < DOT_BLOCKS; b += 32) v += partial[b * 5 + warp];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) tot[warp] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double N2 = c0 * c0 + 2.0 * tot[4];
    const double ehf = tot[0];
    const double E = (N2 * ehf + 4.0 * c0 * tot[1] + 2.0 * tot[2] + 2.0 * tot[3]) / N2;
    out[0] = E;
    out[1] = (2.0 * c0 * ehf + 4.0 * tot[1]) / N2 - 2.0 * c0 * E / N2;
    sc[0] = ehf;
    sc[1] = E;
    sc[2] = N2;
    sc[3] = tot[1];
}

// Final assembly with the device scalars sc = {E_HF, E, N2}:
//   dE/dsigma = (4 c0 Z1a + 4 Z1b + 4 Z1c - 4 Z3 + 4 (E_HF - E) sigma) / N2   (Eq. eng_der_sigma_jb)
//   dE/dTheta = 4 X1 + (R1 + 4 R2 - 4 R3 + 4 c0 X2) / N2                       (dE/dTheta, from E)
//   dE/dGamma = (4 c0 X4 + 4 Rg1 + 4 Rg2) / N2                                 (Eq. eng_der_ucp)
// with X1 = Theta Fk, X2 = sigma Gamma Fk, X3 = Theta F_T, X4 = sigma^T Theta Fk,
// Z1a,b,c = X1,2,3 Gamma^T, Z3 = X1 Theta^T sigma, R1 = Theta M1,
// R2 = sigma Gamma F_T^T, R3 = sigma X4, Rg1 = sigma^T X2, Rg2 = sigma^T Theta F_T.
// dV holds Theta's rows then Gamma's.
__global__ void k_energy_finish(int n, int no, int nv, double c0, EnergyWork w, const double *__restrict__ sigma,
                                double *__restrict__ dsig, double *__restrict__ dV) {
    const double ehf = w.sc[0], E = w.sc[1], inv = 1.0 / w.sc[2];
    const size_t ns = (size_t)no * nv, nt = (size_t)no * n, ng = (size_t)nv * n;
    const size_t tot = ns + nt + ng;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        if (e < ns) {
            dsig[e] = (4.0 * c0 * w.Z1a[e] + 4.0 * w.Z1b[e] + 4.0 * w.Z1c[e] - 4.0 * w.Z3[e] +
                       4.0 * (ehf - E) * sigma[e]) * inv;
        } else if (e < ns + nt) {
            const size_t i = e - ns;
            dV[i] = 4.0 * w.X1[i] + (w.R1[i] + 4.0 * w.R2[i] - 4.0 * w.R3[i] + 4.0 * c0 * w.X2[i]) * inv;
        } else {
            const size_t i = e - ns - nt;
            dV[nt + i] = (4.0 * c0 * w.X4[i] + 4.0 * w.Rg1[i] + 4.0 * w.Rg2[i]) * inv;
        }
    }
}

// ---------------------------------------------------------------- GVP
// Up to 12 inner products x_k . y_k in one pass (per-block partials).
constexpr int MAX_DOTS = 12;
struct DotList {
    const double *x[MAX_DOTS], *y[MAX_DOTS];
    size_t len[MAX_DOTS];
    int count;
};
__global__ void __launch_bounds__(256) k_dot_list(const __grid_constant__ DotList L, double *__restrict__ partial) {
    __shared__ double red[8][MAX_DOTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < L.count; ++k) {
        double v = 0.0;
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < L.len[k]; e += (size_t)gridDim.x * blockDim.x)
            v += L.x[k][e] * L.y[k][e];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < L.count) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        partial[blockIdx.x * MAX_DOTS + threadIdx.x] = v;
    }
}

// Gx = Gam - Gam^T (the rotation gradient, Eq. redefine_U at X = 0) and, in
// place, X <- X + X^T for the two tangent densities built from one product.
__global__ void k_antisym(int n, const double *__restrict__ Gam, double *__restrict__ Gx) {
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const size_t p = e / n, q = e % n;
        Gx[e] = Gam[e] - Gam[q * n + p];
    }
}
__global__ void k_symmetrize2(int n, double *__restrict__ X, double *__restrict__ Y) {
    const size_t pairs = (size_t)n * (n + 1) / 2;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * pairs; e += (size_t)gridDim.x * blockDim.x) {
        double *M = e < pairs ? X : Y;
        size_t r = e < pairs ? e : e - pairs;
        size_t p = (size_t)((sqrt(8.0 * (double)r + 1.0) - 1.0) / 2.0);
        while (p * (p + 1) / 2 > r) --p;
        while ((p + 1) * (p + 2) / 2 <= r) ++p;
        const size_t q = r - p * (p + 1) / 2;   // q <= p
        const double v = M[p * n + q] + M[q * n + p];
        M[p * n + q] = v;
        M[q * n + p] = v;
    }
}

// M1' = 4 c0' (F_T + F_T^T) + 4 c0 (F_T' + F_T'^T) + 2 (F_A' + F_A'^T), c0' = dE/dc0 (device).
__global__ void k_gvp_m1t(int n, double c0, const double *__restrict__ gc0, const double *__restrict__ F,
                          const double *__restrict__ Ft, double *__restrict__ M1t) {
    const size_t nn = (size_t)n * n;
    const double c0t = gc0[1];
    const double *FT = F + nn, *FTt = Ft + nn, *FAt = Ft + 2 * nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const size_t p = e / n, q = e % n, tr = q * n + p;
        M1t[e] = 4.0 * c0t * (FT[e] + FT[tr]) + 4.0 * c0 * (FTt[e] + FTt[tr]) + 2.0 * (FAt[e] + FAt[tr]);
    }
}

// Scalars of the tangent pass and of the GVP objective (Eqs. esmf_gvb,
// esmf_l_gvp_der).  d = tangent inner products (see launch_gvp_finish);
// sc = {E_HF, E, N2, Fk . T}; scE = {E, dE/dc0}.
// out = {L, E, |grad E|^2, dL/dc0}; st = {c0', N2', E', s0', a, b}.
__global__ void k_gvp_scalars(double c0, double omega, double mu, double chi, const double *__restrict__ partial,
                              const double *__restrict__ sc, const double *__restrict__ scE,
                              double *__restrict__ out, double *__restrict__ st) {
    __shared__ double d[MAX_DOTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < MAX_DOTS; k += blockDim.x >> 5) {
        double v = 0.0;
        for (int b = lane; b < DOT_BLOCKS; b += 32) v += partial[b * MAX_DOTS + k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) d[k] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double s0 = sc[0], E = sc[1], N2 = sc[2], s1 = sc[3], gc0 = scE[1];
    const double s0t = d[0] + d[1] + d[2], s1t = d[3] + d[4], s2t = d[5] + d[6], s3t = d[7] + d[8];
    const double c0t = gc0;                                    // direction: the gradient itself
    const double N2t = 2.0 * c0 * c0t + 4.0 * d[9];
    const double numt = N2t * s0 + N2 * s0t + 4.0 * c0t * s1 + 4.0 * c0 * s1t + 2.0 * s2t + 2.0 * s3t;
    const double Et = (numt - E * N2t) / N2;
    const double Yct = 2.0 * c0t * s0 + 2.0 * c0 * s0t + 4.0 * s1t - 2.0 * c0t * E - 2.0 * c0 * Et;
    const double Hc0 = (Yct - gc0 * N2t) / N2;
    const double gn2 = gc0 * gc0 + d[10] + 0.5 * d[11];
    const double a = chi * (-2.0 * mu * (omega - E)) + (1.0 - chi);
    const double b = 2.0 * chi * (1.0 - mu);
    out[0] = chi * (mu * (omega - E) * (omega - E) + (1.0 - mu) * gn2) + (1.0 - chi) * E;
    out[1] = E;
    out[2] = gn2;
    out[3] = a * gc0 + b * Hc0;
    st[0] = c0t;
    st[1] = N2t;
    st[2] = Et;
    st[3] = s0t;
    st[4] = a;
    st[5] = b;
}

// Tangent of the gradient (the Hessian-vector product's c0/sigma/V parts):
//   Hs  = dsigma' = (4 c0' Z1a + 4 c0 Z1a' + 4 Z1b' + 4 Z1c' - 4 Z3' + 4 (s0' - E') sigma
//                    + 4 (s0 - E) g_s - N2' g_s) / N2
//   Mt  = [dTheta'; dGamma'] with
//   dTheta' = 4 X1' + (R1' + 4 R2' - 4 R3' + 4 c0' X2 + 4 c0 X2' - (g_Th - 4 X1) N2') / N2
//   dGamma' = (4 c0' X4 + 4 c0 X4' + 4 Rg1' + 4 Rg2' - g_Ga N2') / N2
__global__ void k_gvp_tangent(int n, int no, int nv, double c0, EnergyWork w, GvpWork v,
                              const double *__restrict__ sigma) {
    const double s0 = w.sc[0], E = w.sc[1], inv = 1.0 / w.sc[2];
    const double c0t = v.st[0], N2t = v.st[1], Et = v.st[2], s0t = v.st[3];
    const size_t ns = (size_t)no * nv, nt = (size_t)no * n, ng = (size_t)nv * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ns + nt + ng;
         e += (size_t)gridDim.x * blockDim.x) {
        if (e < ns) {
            v.Hs[e] = (4.0 * c0t * w.Z1a[e] + 4.0 * c0 * v.Z1a[e] + 4.0 * v.Z1b[e] + 4.0 * v.Z1c[e] - 4.0 * v.Z3[e] +
                       4.0 * (s0t - Et) * sigma[e] + 4.0 * (s0 - E) * v.gs[e] - N2t * v.gs[e]) * inv;
        } else if (e < ns + nt) {
            const size_t i = e - ns;
            v.Mt[i] = 4.0 * v.X1[i] + (v.R1[i] + 4.0 * v.R2[i] - 4.0 * v.R3[i] + 4.0 * c0t * w.X2[i] +
                                       4.0 * c0 * v.X2[i] - (v.gV[i] - 4.0 * w.X1[i]) * N2t) * inv;
        } else {
            const size_t i = e - ns - nt;
            v.Mt[nt + i] = (4.0 * c0t * w.X4[i] + 4.0 * c0 * v.X4[i] + 4.0 * v.Rg1[i] + 4.0 * v.Rg2[i] -
                            v.gV[nt + i] * N2t) * inv;
        }
    }
}

// dL/dsigma = a g_s + b Hs;  dL/dX = a Gx + b (Dd - Dd^T)   (Eq. esmf_l_gvp_der)
__global__ void k_gvp_out(int n, int no, int nv, GvpWork v, double *__restrict__ dLs, double *__restrict__ dLX) {
    const double a = v.st[4], b = v.st[5];
    const size_t ns = (size_t)no * nv, nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ns + nn; e += (size_t)gridDim.x * blockDim.x) {
        if (e < ns) {
            dLs[e] = a * v.gs[e] + b * v.Hs[e];
        } else {
            const size_t i = e - ns, p = i / n, q = i % n;
            dLX[i] = a * v.Gx[i] + b * (v.Dd[i] - v.Dd[q * n + p]);
        }
    }
}

int grid_for(size_t len) {
    size_t g = (len + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

int check(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return ESMF_ERR_CUDA;
    }
    return ESMF_OK;
}

// Launches up to MAX_GROUP independent GEMMs together, with the largest tile
// that still gives about four blocks per SM (GB300: 152 SMs).
int launch_group(const GemmProblem *ps, int count, cudaStream_t s) {
    GemmGroup g;
    g.count = 0;
    for (int i = 0; i < count; ++i)
        if (ps[i].M > 0 && ps[i].N > 0) g.p[g.count++] = ps[i];
    if (g.count == 0) return ESMF_OK;
    int T = 16;
    for (int cand : {64, 32}) {
        int tot = 0;
        for (int i = 0; i < g.count; ++i) tot += tiles_of(g.p[i], cand);
        if (tot >= 608) { T = cand; break; }
    }
    g.tiles[0] = 0;
    for (int i = 0; i < g.count; ++i) g.tiles[i + 1] = g.tiles[i] + tiles_of(g.p[i], T);
    const int blocks = g.tiles[g.count];
    if (T == 64) k_gemm_group<64, 4><<<blocks, 256, 0, s>>>(g);
    else if (T == 32) k_gemm_group<32, 4><<<blocks, 64, 0, s>>>(g);
    else k_gemm_group<16, 2><<<blocks, 64, 0, s>>>(g);
    return check("k_gemm_group");
}

}  // namespace

size_t energy_work_doubles(int n, int no) {
    const size_t nn = (size_t)n * n, nv = (size_t)(n - no);
    // D, J, K, F (3 each), Fk, M1, Wc, Wm; X1, X2, X3, R1, R2, R3 (no x n);
    // X4, Rg1, Rg2 (nv x n); Z1a, Z1b, Z1c, Z3 (no x nv); Z2 (no x no); partials, scalars
    return 16 * nn + 6 * (size_t)no * n + 3 * nv * n + 4 * (size_t)no * nv + (size_t)no * no +
           5 * DOT_BLOCKS + 8;
}

EnergyWork energy_work_layout(double *base, int n, int no) {
    const size_t nn = (size_t)n * n, nv = (size_t)(n - no), non = (size_t)no * n, nvn = nv * n;
    EnergyWork w;
    double *p = base;
    w.D = p; p += 3 * nn;
    w.J = p; p += 3 * nn;
    w.K = p; p += 3 * nn;
    w.F = p; p += 3 * nn;
    w.Fk = p; p += nn;
    w.M1 = p; p += nn;
    w.Wc = p; p += nn;
    w.Wm = p; p += nn;
    w.X1 = p; p += non;
    w.X2 = p; p += non;
    w.X3 = p; p += non;
    w.R1 = p; p += non;
    w.R2 = p; p += non;
    w.R3 = p; p += non;
    w.X4 = p; p += nvn;
    w.Rg1 = p; p += nvn;
    w.Rg2 = p; p += nvn;
    w.Z1a = p; p += (size_t)no * nv;
    w.Z1b = p; p += (size_t)no * nv;
    w.Z1c = p; p += (size_t)no * nv;
    w.Z3 = p; p += (size_t)no * nv;
    w.Z2 = p; p += (size_t)no * no;
    w.partial = p; p += 5 * DOT_BLOCKS;
    w.sc = p;
    return w;
}

// Densities of the grouped build: P, T and (for the energy's Fk . A) A, from
//   Wc = [sigma Gamma; sigma^T Theta] and Wm = [sigma Gamma; -sigma^T Theta]
// (W1 = sigma Gamma, W2 = sigma^T Theta):
//   P = Theta^T Theta, T = Theta^T W1, A = Wc^T Wm = W1^T W1 - W2^T W2.
int launch_energy_densities(int n, int no, const double *V, const double *sigma, const EnergyWork &w,
                            cudaStream_t s) {
    const int nv = n - no;
    const double *Th = V, *Ga = V + (size_t)no * n;
    const size_t nn = (size_t)n * n, non = (size_t)no * n;
    const GemmProblem g1[4] = {
        gp(false, false, no, n, nv, 1.0, sigma, nv, Ga, n, 0.0, w.Wc, n),
        gp(true, false, nv, n, no, 1.0, sigma, nv, Th, n, 0.0, w.Wc + non, n),
        gp(false, false, no, n, nv, 1.0, sigma, nv, Ga, n, 0.0, w.Wm, n),
        gp(true, false, nv, n, no, -1.0, sigma, nv, Th, n, 0.0, w.Wm + non, n)};
    RET_IF(launch_group(g1, 4, s));
    const GemmProblem g2[3] = {
        gp(true, false, n, n, no, 1.0, Th, n, Th, n, 0.0, w.D, n),
        gp(true, false, n, n, no, 1.0, Th, n, w.Wc, n, 0.0, w.D + nn, n),
        gp(true, false, n, n, n, 1.0, w.Wc, n, w.Wm, n, 0.0, w.D + 2 * nn, n)};
    return launch_group(g2, 3, s);
}

// Everything after the grouped build (F = [F_P, F_T, F_A] in w.F).
int launch_energy_finish(int n, int no, double c0, const double *G, const double *V, const double *sigma,
                         const EnergyWork &w, double *scalars, double *dsig, double *dV, cudaStream_t s) {
    const int nv = n - no;
    const size_t nn = (size_t)n * n, non = (size_t)no * n;
    const double *Th = V, *Ga = V + non, *FT = w.F + nn;
    const double *W1 = w.Wc, *W2 = w.Wc + non;
    const bool grad = dsig != nullptr;
    k_energy_fock<<<grid_for(nn), 256, 0, s>>>(n, c0, G, w.F, w.Fk, w.M1, grad ? 1 : 0);
    RET_IF(check("k_energy_fock"));
    k_energy_dots<<<DOT_BLOCKS, 256, 0, s>>>(n, no * nv, G, w.Fk, w.F, w.D, sigma, w.partial);
    RET_IF(check("k_energy_dots"));
    k_energy_scalars<<<1, 160, 0, s>>>(c0, w.partial, scalars, w.sc);
    RET_IF(check("k_energy_scalars"));
    if (!grad) return ESMF_OK;
    const GemmProblem g3[7] = {
        gp(false, false, no, n, n, 1.0, Th, n, w.Fk, n, 0.0, w.X1, n),
        gp(false, false, no, n, n, 1.0, W1, n, w.Fk, n, 0.0, w.X2, n),
        gp(false, false, no, n, n, 1.0, Th, n, FT, n, 0.0, w.X3, n),
        gp(false, false, nv, n, n, 1.0, W2, n, w.Fk, n, 0.0, w.X4, n),
        gp(false, false, no, n, n, 1.0, Th, n, w.M1, n, 0.0, w.R1, n),
        gp(false, true, no, n, n, 1.0, W1, n, FT, n, 0.0, w.R2, n),
        gp(false, false, nv, n, n, 1.0, W2, n, FT, n, 0.0, w.Rg2, n)};
    RET_IF(launch_group(g3, 7, s));
    const GemmProblem g4[6] = {
        gp(false, true, no, nv, n, 1.0, w.X1, n, Ga, n, 0.0, w.Z1a, nv),
        gp(false, true, no, nv, n, 1.0, w.X2, n, Ga, n, 0.0, w.Z1b, nv),
        gp(false, true, no, nv, n, 1.0, w.X3, n, Ga, n, 0.0, w.Z1c, nv),
        gp(false, true, no, no, n, 1.0, w.X1, n, Th, n, 0.0, w.Z2, no),
        gp(false, false, no, n, nv, 1.0, sigma, nv, w.X4, n, 0.0, w.R3, n),
        gp(true, false, nv, n, no, 1.0, sigma, nv, w.X2, n, 0.0, w.Rg1, n)};
    RET_IF(launch_group(g4, 6, s));
    const GemmProblem g5[1] = {gp(false, false, no, nv, no, 1.0, w.Z2, no, sigma, nv, 0.0, w.Z3, nv)};
    RET_IF(launch_group(g5, 1, s));
    const size_t tot = (size_t)no * nv + non + (size_t)nv * n;
    k_energy_finish<<<grid_for(tot), 256, 0, s>>>(n, no, nv, c0, w, sigma, dsig, dV);
    return check("k_energy_finish");
}

size_t gvp_work_doubles(int n, int no) {
    const size_t nn = (size_t)n * n, nv = (size_t)(n - no);
    // gs, Z1a, Z1b, Z1c, Z3, Hs (no x nv); gV, Gam, Gx, Vt, Wct, Wmt, M1t, Mt, Dd and
    // Dt, Jt, Kt, Ft (3 each): 21 N x N; six no x n, three nv x n, Z2; partials; scE, st
    return 21 * nn + 6 * (size_t)no * nv + 6 * (size_t)no * n + 3 * nv * n + (size_t)no * no +
           MAX_DOTS * DOT_BLOCKS + 16;
}

GvpWork gvp_work_layout(double *base, int n, int no) {
    const size_t nn = (size_t)n * n, nv = (size_t)(n - no), non = (size_t)no * n, nvn = nv * n,
                 nonv = (size_t)no * nv;
    GvpWork v;
    double *p = base;
    v.gs = p; p += nonv;
    v.gV = p; p += nn;
    v.Gam = p; p += nn;
    v.Gx = p; p += nn;
    v.Vt = p; p += nn;
    v.Wct = p; p += nn;
    v.Wmt = p; p += nn;
    v.Dt = p; p += 3 * nn;
    v.Jt = p; p += 3 * nn;
    v.Kt = p; p += 3 * nn;
    v.Ft = p; p += 3 * nn;
    v.M1t = p; p += nn;
    v.Mt = p; p += nn;
    v.Dd = p; p += nn;
    v.X1 = p; p += non;
    v.X2 = p; p += non;
    v.X3 = p; p += non;
    v.R1 = p; p += non;
    v.R2 = p; p += non;
    v.R3 = p; p += non;
    v.X4 = p; p += nvn;
    v.Rg1 = p; p += nvn;
    v.Rg2 = p; p += nvn;
    v.Z1a = p; p += nonv;
    v.Z1b = p; p += nonv;
    v.Z1c = p; p += nonv;
    v.Z3 = p; p += nonv;
    v.Hs = p; p += nonv;
    v.Z2 = p; p += (size_t)no * no;
    v.partial = p; p += MAX_DOTS * DOT_BLOCKS;
    v.scE = p; p += 8;
    v.st = p;
    return v;
}

// After the first pass (v.gs, v.gV, v.scE hold dE/dsigma, dE/dV, {E, dE/dc0}):
// the rotation gradient Gx = Gam - Gam^T (Gam = dE/dV V^T) and the tangent
// densities of the direction (c0', sigma', V') = (dE/dc0, dE/dsigma, Gx V):
//   W1' = sigma' Gamma + sigma Gamma', W2' = sigma'^T Theta + sigma^T Theta'
//   P' = Theta'^T Theta + (.)^T, T' = Theta'^T W1 + Theta^T W1',
//   A' = Wc'^T Wm + (.)^T   (Wc = [W1; W2], Wm = [W1; -W2])
int launch_gvp_tangent_densities(int n, int no, const double *V, const double *sigma, const EnergyWork &w,
                                 const GvpWork &v, cudaStream_t s) {
    const int nv = n - no;
    const size_t nn = (size_t)n * n, non = (size_t)no * n;
    const double *Th = V, *Ga = V + non, *Tht = v.Vt, *Gat = v.Vt + non;
    const GemmProblem a1[1] = {gp(false, true, n, n, n, 1.0, v.gV, n, V, n, 0.0, v.Gam, n)};
    RET_IF(launch_group(a1, 1, s));
    k_antisym<<<grid_for(nn), 256, 0, s>>>(n, v.Gam, v.Gx);
    RET_IF(check("k_antisym"));
    const GemmProblem a2[1] = {gp(false, false, n, n, n, 1.0, v.Gx, n, V, n, 0.0, v.Vt, n)};
    RET_IF(launch_group(a2, 1, s));
    const GemmProblem b0[4] = {
        gp(false, false, no, n, nv, 1.0, v.gs, nv, Ga, n, 0.0, v.Wct, n),
        gp(true, false, nv, n, no, 1.0, v.gs, nv, Th, n, 0.0, v.Wct + non, n),
        gp(false, false, no, n, nv, 1.0, v.gs, nv, Ga, n, 0.0, v.Wmt, n),
        gp(true, false, nv, n, no, -1.0, v.gs, nv, Th, n, 0.0, v.Wmt + non, n)};
    RET_IF(launch_group(b0, 4, s));
    const GemmProblem b1[4] = {
        gp(false, false, no, n, nv, 1.0, sigma, nv, Gat, n, 1.0, v.Wct, n),
        gp(true, false, nv, n, no, 1.0, sigma, nv, Tht, n, 1.0, v.Wct + non, n),
        gp(false, false, no, n, nv, 1.0, sigma, nv, Gat, n, 1.0, v.Wmt, n),
        gp(true, false, nv, n, no, -1.0, sigma, nv, Tht, n, 1.0, v.Wmt + non, n)};
    RET_IF(launch_group(b1, 4, s));
    const GemmProblem c0[3] = {
        gp(true, false, n, n, no, 1.0, Tht, n, Th, n, 0.0, v.Dt, n),
        gp(true, false, n, n, no, 1.0, Tht, n, w.Wc, n, 0.0, v.Dt + nn, n),
        gp(true, false, n, n, n, 1.0, v.Wct, n, w.Wm, n, 0.0, v.Dt + 2 * nn, n)};
    RET_IF(launch_group(c0, 3, s));
    const GemmProblem c1[1] = {gp(true, false, n, n, no, 1.0, Th, n, v.Wct, n, 1.0, v.Dt + nn, n)};
    RET_IF(launch_group(c1, 1, s));
    k_symmetrize2<<<grid_for(nn), 256, 0, s>>>(n, v.Dt, v.Dt + 2 * nn);
    return check("k_symmetrize2");
}

// Everything after the tangent build (v.Ft = [F_P', F_T', F_A']): tangent
// scalars and the objective, the tangent of the gradient, the rotation part
// of H g, dL/dx.
int launch_gvp_finish(int n, int no, double c0, double omega, double mu, double chi, const double *G,
                      const double *V, const double *sigma, const EnergyWork &w, const GvpWork &v,
                      double *scalars, double *dLs, double *dLX, cudaStream_t s) {
    const int nv = n - no;
    const size_t nn = (size_t)n * n, non = (size_t)no * n, nonv = (size_t)no * nv;
    const double *Th = V, *Ga = V + non, *Tht = v.Vt, *Gat = v.Vt + non;
    const double *FT = w.F + nn, *FPt = v.Ft, *FTt = v.Ft + nn;
    const double *W1 = w.Wc, *W2 = w.Wc + non, *W1t = v.Wct, *W2t = v.Wct + non;
    // tangent inner products: s0' = F_P'.P + G.P' + Fk.P', s1' = F_P'.T + Fk.T',
    // s2' = F_P'.A + Fk.A', s3' = F_T'.T + F_T.T', sigma.g_s, |g_s|^2, |Gx|^2
    DotList L;
    const double *xs[MAX_DOTS] = {FPt, G, w.Fk, FPt, w.Fk, FPt, w.Fk, FTt, FT, sigma, v.gs, v.Gx};
    const double *ys[MAX_DOTS] = {w.D, v.Dt, v.Dt, w.D + nn, v.Dt + nn, w.D + 2 * nn, v.Dt + 2 * nn, w.D + nn,
                                  v.Dt + nn, v.gs, v.gs, v.Gx};
    for (int k = 0; k < MAX_DOTS; ++k) {
        L.x[k] = xs[k];
        L.y[k] = ys[k];
        L.len[k] = (k == 9 || k == 10) ? nonv : nn;
    }
    L.count = MAX_DOTS;
    k_dot_list<<<DOT_BLOCKS, 256, 0, s>>>(L, v.partial);
    RET_IF(check("k_dot_list"));
    k_gvp_scalars<<<1, 384, 0, s>>>(c0, omega, mu, chi, v.partial, w.sc, v.scE, scalars, v.st);
    RET_IF(check("k_gvp_scalars"));
    k_gvp_m1t<<<grid_for(nn), 256, 0, s>>>(n, c0, v.scE, w.F, v.Ft, v.M1t);
    RET_IF(check("k_gvp_m1t"));
    const GemmProblem t3[7] = {
        gp(false, false, no, n, n, 1.0, Tht, n, w.Fk, n, 0.0, v.X1, n),
        gp(false, false, no, n, n, 1.0, W1t, n, w.Fk, n, 0.0, v.X2, n),
        gp(false, false, no, n, n, 1.0, Tht, n, FT, n, 0.0, v.X3, n),
        gp(false, false, nv, n, n, 1.0, W2t, n, w.Fk, n, 0.0, v.X4, n),
        gp(false, false, no, n, n, 1.0, Tht, n, w.M1, n, 0.0, v.R1, n),
        gp(false, true, no, n, n, 1.0, W1t, n, FT, n, 0.0, v.R2, n),
        gp(false, false, nv, n, n, 1.0, W2t, n, FT, n, 0.0, v.Rg2, n)};
    RET_IF(launch_group(t3, 7, s));
    const GemmProblem t4[7] = {
        gp(false, false, no, n, n, 1.0, Th, n, FPt, n, 1.0, v.X1, n),
        gp(false, false, no, n, n, 1.0, W1, n, FPt, n, 1.0, v.X2, n),
        gp(false, false, no, n, n, 1.0, Th, n, FTt, n, 1.0, v.X3, n),
        gp(false, false, nv, n, n, 1.0, W2, n, FPt, n, 1.0, v.X4, n),
        gp(false, false, no, n, n, 1.0, Th, n, v.M1t, n, 1.0, v.R1, n),
        gp(false, true, no, n, n, 1.0, W1, n, FTt, n, 1.0, v.R2, n),
        gp(false, false, nv, n, n, 1.0, W2, n, FTt, n, 1.0, v.Rg2, n)};
    RET_IF(launch_group(t4, 7, s));
    const GemmProblem t5[6] = {
        gp(false, true, no, nv, n, 1.0, v.X1, n, Ga, n, 0.0, v.Z1a, nv),
        gp(false, true, no, nv, n, 1.0, v.X2, n, Ga, n, 0.0, v.Z1b, nv),
        gp(false, true, no, nv, n, 1.0, v.X3, n, Ga, n, 0.0, v.Z1c, nv),
        gp(false, true, no, no, n, 1.0, v.X1, n, Th, n, 0.0, v.Z2, no),
        gp(false, false, no, n, nv, 1.0, v.gs, nv, w.X4, n, 0.0, v.R3, n),
        gp(true, false, nv, n, no, 1.0, v.gs, nv, w.X2, n, 0.0, v.Rg1, n)};
    RET_IF(launch_group(t5, 6, s));
    const GemmProblem t6[6] = {
        gp(false, true, no, nv, n, 1.0, w.X1, n, Gat, n, 1.0, v.Z1a, nv),
        gp(false, true, no, nv, n, 1.0, w.X2, n, Gat, n, 1.0, v.Z1b, nv),
        gp(false, true, no, nv, n, 1.0, w.X3, n, Gat, n, 1.0, v.Z1c, nv),
        gp(false, true, no, no, n, 1.0, w.X1, n, Tht, n, 1.0, v.Z2, no),
        gp(false, false, no, n, nv, 1.0, sigma, nv, v.X4, n, 1.0, v.R3, n),
        gp(true, false, nv, n, no, 1.0, sigma, nv, v.X2, n, 1.0, v.Rg1, n)};
    RET_IF(launch_group(t6, 6, s));
    const GemmProblem t7[1] = {gp(false, false, no, nv, no, 1.0, v.Z2, no, sigma, nv, 0.0, v.Z3, nv)};
    RET_IF(launch_group(t7, 1, s));
    const GemmProblem t8[1] = {gp(false, false, no, nv, no, 1.0, w.Z2, no, v.gs, nv, 1.0, v.Z3, nv)};
    RET_IF(launch_group(t8, 1, s));
    const size_t tot = nonv + non + (size_t)nv * n;
    k_gvp_tangent<<<grid_for(tot), 256, 0, s>>>(n, no, nv, c0, w, v, sigma);
    RET_IF(check("k_gvp_tangent"));
    // rotation part of H g: Dd = Mt V^T - (Gx Gam + Gam Gx) / 2
    const GemmProblem d0[1] = {gp(false, true, n, n, n, 1.0, v.Mt, n, V, n, 0.0, v.Dd, n)};
    RET_IF(launch_group(d0, 1, s));
    const GemmProblem d1[1] = {gp(false, false, n, n, n, -0.5, v.Gx, n, v.Gam, n, 1.0, v.Dd, n)};
    RET_IF(launch_group(d1, 1, s));
    const GemmProblem d2[1] = {gp(false, false, n, n, n, -0.5, v.Gam, n, v.Gx, n, 1.0, v.Dd, n)};
    RET_IF(launch_group(d2, 1, s));
    k_gvp_out<<<grid_for(nonv + nn), 256, 0, s>>>(n, no, nv, v, dLs, dLX);
    return check("k_gvp_out");
}

}  // namespace esmf
