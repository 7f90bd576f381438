// Build entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at build time: code that runs while the
// host application owns every device allocation (a pool handed out by a
// framework or a serving process with a fixed memory plan), and latency-bound
// loops where a cudaMalloc/cudaFree pair would synchronise the device and
// stall other streams.  esmf_fock_build_noalloc serves them: for stored FP64
// and FP32 handles and integral-direct handles it runs the same CUDA-core
// contraction and finalisation kernels as esmf_fock_build; for split 16-bit
// stores it runs the CUDA-core kernel over the store (the tensor-core kernel
// needs density tiles in handle work memory), equal to esmf_fock_build within
// that precision's tolerance.  Its FP64 J/K accumulators (the contraction
// kernel's scratch memory) live in the file-scope device array below instead
// of handle memory grown on demand.
//
// The array is sized once, at library load, on every device the library is
// used on, and stays resident until the process exits.  All calls share it,
// so builds issued through this entry point must not overlap on the GPU.
#include <cuda_runtime.h>

#include <mutex>

#include "esmf_internal.cuh"

namespace esmf {
int handle_prepare_noalloc(esmf_fock_t *h, int m, const double *D, JKArgs *a, int *device,
                           bool *split);
}  // namespace esmf

using namespace esmf;

// J accumulators followed by K accumulators, m * np * np doubles each.
static __device__ __align__(256) double g_noalloc_scratch[ESMF_NOALLOC_MAX_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_dev[kMaxDevices] = {};

// The symbol's device address, looked up once per device with that device
// current.  In host code g_noalloc_scratch names a host-side shadow, never
// the device memory, so the kernels receive this address instead.
int scratch_address(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("device %d outside the supported range", device);
        return ESMF_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[device]) {
        double *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress(no-alloc scratch): %s", cudaGetErrorString(e));
            return ESMF_ERR_CUDA;
        }
        g_scratch_dev[device] = p;
    }
    *out = g_scratch_dev[device];
    return ESMF_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int esmf_fock_build_noalloc(esmf_fock_t *h, int m, const double *D, double *J,
                                       double *K, double *F, double *traces, void *stream) {
    if (!h) { set_error("handle is NULL"); return ESMF_ERR_INVALID_ARG; }
    if (m < 1 || m > ESMF_MAX_DENSITIES) { set_error("m = %d outside [1, %d]", m, ESMF_MAX_DENSITIES); return ESMF_ERR_INVALID_ARG; }
    if (!D || !J || !K) { set_error("D, J and K are required"); return ESMF_ERR_INVALID_ARG; }
    JKArgs a;
    int device = 0;
    bool split = false;
    int rc = handle_prepare_noalloc(h, m, D, &a, &device, &split);
    if (rc != ESMF_OK) return rc;
    const int64_t per = (int64_t)m * a.b.np * a.b.np;
    if (2 * per > (int64_t)ESMF_NOALLOC_MAX_SCRATCH_DOUBLES) {
        set_error("no-alloc build needs %lld scratch doubles (2 m Np^2 with m = %d, Np = %d); the "
                  "static limit is %lld", (long long)(2 * per), m, a.b.np,
                  (long long)ESMF_NOALLOC_MAX_SCRATCH_DOUBLES);
        return ESMF_ERR_INVALID_ARG;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
        set_error("cudaSetDevice(%d) failed", device);
        return ESMF_ERR_CUDA;
    }
    struct Restore {
        int prev, dev;
        ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
    } restore{prev, device};
    if (!on_device(D) || !on_device(J) || !on_device(K) || (F && !on_device(F)) ||
        (traces && !on_device(traces))) {
        set_error("D, J, K, F and traces must be device memory");
        return ESMF_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    if ((rc = scratch_address(device, &scratch)) != ESMF_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear what this call uses
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(double) * 2 * per, s);
    if (e == cudaSuccess && traces) e = cudaMemsetAsync(traces, 0, sizeof(double) * m, s);
    if (e != cudaSuccess) { set_error("clear scratch: %s", cudaGetErrorString(e)); return ESMF_ERR_CUDA; }
    a.Jacc = scratch;
    a.Kacc = scratch + per;
    if (a.nbricks > 0) {
        rc = split ? launch_jk_cuda_split(a, s) : launch_jk_cuda(a, s);
        if (rc != ESMF_OK) return rc;
    }
    return launch_finalize(a.b, m, D, a.Jacc, a.Kacc, J, K, F, traces, s);
}
