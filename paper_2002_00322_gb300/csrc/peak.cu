// CUDA-core FMA throughput of the device (a measurement aid for the roofline
// of the CUDA-core contraction kernels; the paper has no counterpart).
//
// Every thread runs CHAINS independent fused multiply-add chains for `iters`
// iterations, enough independent work per warp to keep the FP32 or FP64 pipe
// issuing every cycle; the grid is a multiple of the SM count.  The result is
// stored only when a runtime flag (never set by the host) asks for it, so the
// compiler keeps the chains without the store costing anything.
#include <cuda_runtime.h>

#include <chrono>
#include <vector>

#include "esmf_internal.cuh"

namespace esmf {

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T a, T b, int iters, int store, T *out) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_chains(int blocks_per_sm, int iters, double *tflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("device query failed");
        return ESMF_ERR_CUDA;
    }
    const int grid = nsm * blocks_per_sm, threads = 256;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("stream/event creation failed");
        if (s) cudaStreamDestroy(s);
        if (e0) cudaEventDestroy(e0);
        return ESMF_ERR_CUDA;
    }
    // a: slightly below one, b: small, so the chains stay finite and normal
    const T a = (T)0.999999, b = (T)1e-7;
    float best = 0.f;
    int rc = ESMF_OK;
    for (int rep = 0; rep < 4 && rc == ESMF_OK; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<grid, threads, 0, s>>>(a, b, iters, 0, nullptr);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            set_error("FMA chain kernel failed");
            rc = ESMF_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;   // first launch is warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc != ESMF_OK) return rc;
    const double flops = 2.0 * grid * threads * (double)CHAINS * UNROLL * (double)iters;
    *tflops = flops / (best * 1e-3) / 1e12;
    return ESMF_OK;
}

}  // namespace

}  // namespace esmf

using namespace esmf;

extern "C" int esmf_measure_fma_peak(int precision, int device, double *tflops) {
    if (!tflops || (precision != ESMF_PREC_FP64 && precision != ESMF_PREC_FP32)) {
        set_error("esmf_measure_fma_peak: precision must be FP64 or FP32 and tflops non-NULL");
        return ESMF_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("device %d not available", device);
        return ESMF_ERR_INVALID_ARG;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
        set_error("cudaSetDevice(%d) failed", device);
        return ESMF_ERR_CUDA;
    }
    // about 0.1-0.3 s per timed launch at the part's rates
    const int rc = precision == ESMF_PREC_FP64 ? time_chains<double>(4, 3000, tflops)
                                               : time_chains<float>(8, 50000, tflops);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
