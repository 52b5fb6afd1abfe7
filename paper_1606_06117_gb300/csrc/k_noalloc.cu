// k_noalloc.cu -- sl_norms_static: the error-norm reduction of sl_norms with its
// scratch in a fixed device array instead of library-allocated memory, for
// callers that must not trigger any device allocation (see include/sl.h).
#include <cmath>
#include <mutex>

#include "sl.h"
#include "sl_internal.h"

namespace sl {
namespace {

// Block partials (kReduceBlocks rows) plus the folded row, 4 doubles each:
// 32.8 KB that every GPU loading the library keeps until the process exits.
// Host code must not use this name as a device address; it asks the runtime for
// the address once per device (norm_scratch below).
static __device__ __align__(256) double g_norm_scratch[(kReduceBlocks + 1) * 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_norm_scratch on the current device, resolved on the first
// call for that device (with that device current) and cached.
cudaError_t norm_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Turns the folded sums of the scratch into the three norms in the caller's
// device buffer: RMS, max, relative L2.
__global__ void k_norm_finish(const double *__restrict__ scratch, double inv_n, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double s2 = scratch[kReduceBlocks * 4 + 0];
        const double mx = scratch[kReduceBlocks * 4 + 1];
        const double r2 = scratch[kReduceBlocks * 4 + 2];
        out[0] = sqrt(s2 * inv_n);
        out[1] = mx;
        out[2] = r2 > 0.0 ? sqrt(s2 / r2) : sqrt(s2);
    }
}

}  // namespace
}  // namespace sl

extern "C" int sl_norms_static(const void *a, const void *b, int64_t n, int dtype, double *out, void *stream)
{
    using namespace sl;
    if (!a || !b || !out) return set_error(SL_ERR_ARG, "sl_norms_static: a, b and out must not be NULL");
    if (n < 1 || n > kNormsStaticMaxElems)
        return set_error(SL_ERR_ARG, "sl_norms_static: n must be in [1, 2^40] elements");
    if (dtype < SL_F32 || dtype > SL_F32_D64) return set_error(SL_ERR_ARG, "sl_norms_static: unknown dtype");
    double *scratch = nullptr;
    cudaError_t e = norm_scratch(&scratch);
    if (e != cudaSuccess) return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every partial slot read by the fold is written by this call first, so the
    // scratch needs no clearing between calls
    e = launch_norms(dtype == SL_F64 ? 1 : 0, a, b, n, scratch, st);
    if (e == cudaSuccess) {
        k_norm_finish<<<1, 32, 0, st>>>(scratch, 1.0 / (double)n, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    return SL_OK;
}
