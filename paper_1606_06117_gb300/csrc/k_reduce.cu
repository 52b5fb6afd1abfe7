// k_reduce.cu -- FP64 reductions: error norms between two fields and the
// maximum Courant number of a velocity.  Two passes: a grid-stride pass that
// leaves one partial per block, then one block that folds the partials.
#include "sl_internal.h"

namespace sl {
namespace {

constexpr int RT = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// partials[b*4 + {0,1,2}] = (sum (a-b)^2, max |a-b|, sum b^2) of block b.
template <typename T>
__global__ void __launch_bounds__(RT) k_norm_partial(const T *__restrict__ a, const T *__restrict__ b, int64_t n,
                                                      double *__restrict__ partials)
{
    double s2 = 0.0, mx = 0.0, r2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double x = double(a[i]), y = double(b[i]);
        const double d = x - y;
        s2 += d * d;
        r2 += y * y;
        mx = fmax(mx, fabs(d));
    }
    __shared__ double sh[3][RT / 32];
    s2 = warp_sum(s2);
    r2 = warp_sum(r2);
    mx = warp_max(mx);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = s2; sh[1][w] = mx; sh[2][w] = r2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < RT / 32; ++k) { t0 += sh[0][k]; t1 = fmax(t1, sh[1][k]); t2 += sh[2][k]; }
        partials[blockIdx.x * 4 + 0] = t0;
        partials[blockIdx.x * 4 + 1] = t1;
        partials[blockIdx.x * 4 + 2] = t2;
    }
}

// One block: folds nb partials into partials[kReduceBlocks*4 + {0,1,2}]
// (sum, max, sum) in a fixed order.
__global__ void __launch_bounds__(RT) k_fold(double *__restrict__ partials, int nb)
{
    double s0 = 0.0, m1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nb; i += RT) {
        s0 += partials[i * 4 + 0];
        m1 = fmax(m1, partials[i * 4 + 1]);
        s2 += partials[i * 4 + 2];
    }
    __shared__ double sh[3][RT / 32];
    s0 = warp_sum(s0);
    m1 = warp_max(m1);
    s2 = warp_sum(s2);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = s0; sh[1][w] = m1; sh[2][w] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < RT / 32; ++k) { t0 += sh[0][k]; t1 = fmax(t1, sh[1][k]); t2 += sh[2][k]; }
        partials[kReduceBlocks * 4 + 0] = t0;
        partials[kReduceBlocks * 4 + 1] = t1;
        partials[kReduceBlocks * 4 + 2] = t2;
    }
}

// partials[b*4 + 1] = max over the block's cells and components of |u_d| s_d.
template <typename T>
__global__ void __launch_bounds__(RT) k_courant_partial(const T *__restrict__ vel, int ndim, int64_t n, double s0,
                                                         double s1, double s2, double *__restrict__ partials)
{
    double mx = 0.0;
    const double sc[3] = {fabs(s0), fabs(s1), fabs(s2)};
    for (int d = 0; d < ndim; ++d) {
        const T *u = vel + d * n;
        double m = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
            m = fmax(m, fabs(double(u[i])));
        mx = fmax(mx, m * sc[d]);
    }
    __shared__ double sh[RT / 32];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < RT / 32; ++k) t = fmax(t, sh[k]);
        partials[blockIdx.x * 4 + 0] = 0.0;
        partials[blockIdx.x * 4 + 1] = t;
        partials[blockIdx.x * 4 + 2] = 0.0;
    }
}

int blocks_for(int64_t n)
{
    int64_t b = (n + RT - 1) / RT;
    if (b > kReduceBlocks) b = kReduceBlocks;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_norms(int dtype, const void *a, const void *b, int64_t n, double *partials, cudaStream_t st)
{
    const int nb = blocks_for(n);
    if (dtype == 1)
        k_norm_partial<double><<<nb, RT, 0, st>>>(static_cast<const double *>(a), static_cast<const double *>(b), n,
                                                 partials);
    else
        k_norm_partial<float><<<nb, RT, 0, st>>>(static_cast<const float *>(a), static_cast<const float *>(b), n,
                                                partials);
    k_fold<<<1, RT, 0, st>>>(partials, nb);
    return cudaGetLastError();
}

cudaError_t launch_courant(int dtype, const void *vel, int ndim, int64_t n, const double s[3], double *partials,
                           cudaStream_t st)
{
    const int nb = blocks_for(n);
    const double s2 = ndim == 3 ? s[2] : 0.0;
    if (dtype == 1)
        k_courant_partial<double><<<nb, RT, 0, st>>>(static_cast<const double *>(vel), ndim, n, s[0], s[1], s2,
                                                    partials);
    else
        k_courant_partial<float><<<nb, RT, 0, st>>>(static_cast<const float *>(vel), ndim, n, s[0], s[1], s2,
                                                   partials);
    k_fold<<<1, RT, 0, st>>>(partials, nb);
    return cudaGetLastError();
}

}  // namespace sl
