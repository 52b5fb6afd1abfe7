// sl_common.cuh -- device helpers shared by the fused advection kernels.
//
// Geometry of every fused kernel: the grid is cut into TX x TY columns of
// cells in the x-y plane and, in 3D, into chunks of TZ planes along z.  A CTA
// owns one (column tile, z chunk) item and marches along z, staging each x-y
// plane of the inputs (plus a periodic halo) in shared memory with 16-byte
// cp.async copies, so that every input element is read from HBM about once
// and every output element is written once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sl {

// ------------------------------------------------------------------ geometry
struct Geo {
    int nx, ny, nz;         // cells per axis
    int64_t plane;          // nx * ny
    int64_t ncell;          // nx * ny * nz
    double sx, sy, sz;      // dt / dx_d: Courant number = u_d * s_d
    int tiles_x, tiles_y;   // column tiles per axis
    int tz;                 // planes per z chunk
    int chunks;             // z chunks
    unsigned *status;       // device status word (SL_DEV_* bits)
};

__host__ __device__ __forceinline__ int wrapi(int v, int n)
{
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------------ async copies
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem)
{
    if constexpr (sizeof(T) == 4)
        cp_async4(smem, gmem);
    else
        cp_async8(smem, gmem);
}

// ----------------------------------------------------------- 1D CEC kernels
//
// One directional sweep of the combined scheme (Sec. 2 eqs. intro:FEC,
// intro:BEC, intro:CEC, intro:CECcoef) along a line, for |C| <= 1 where the
// CIR operator is (1 - U) Phi_i + U Phi_{i-s} (Sec. 3), s = sgn C, U = |C|.
// With l_j = L_U[Phi]_j - Phi_j = U_j (Phi_{j-s_j} - Phi_j) and
// delta_j = Phi_j - Phi_bar_j = -(l_j + U_j ((Phi_{j+s_j} - Phi_j)
//                                          + l_{j+s_j} - l_j)),
// the combination a FEC + b BEC with 3a = 2 - 1/U, b = 1 - a is
//   CEC_i = Phi_i + l_i + ((2 - U_i) delta_i + (1 + U_i) delta_{i-s_i}) / 6,
// which has no 1/U and is exact algebra on the definitions.  Every quantity
// is formed from neighbour differences, so delta does not cancel against Phi.
// D is the arithmetic type of l, delta and the combination.

// Upwind difference Phi_{j-s} - Phi_j from the forward differences
// dm = Phi_j - Phi_{j-1} and dp = Phi_{j+1} - Phi_j.
template <typename D>
__device__ __forceinline__ D upwind_diff(D C, D dm, D dp) { return C > D(0) ? -dm : dp; }

// Downwind difference Phi_{j+s} - Phi_j.
template <typename D>
__device__ __forceinline__ D downwind_diff(D C, D dm, D dp) { return C > D(0) ? dp : -dm; }

// Outputs o[0..R) of a line segment from p[0..R+6) = Phi at offsets -3..R+2
// and c[0..R+4) = Courant numbers at offsets -2..R+1.
template <typename T, typename D, int R>
__device__ __forceinline__ void cec_line(const T (&p)[R + 6], const D (&c)[R + 4], T (&o)[R])
{
    D dp[R + 5];                 // dp[j] = Phi(j-2) - Phi(j-3): forward difference at offset j-3
#pragma unroll
    for (int j = 0; j < R + 5; ++j) dp[j] = D(p[j + 1]) - D(p[j]);
    D l[R + 4];                  // l at offsets -2..R+1 (index m <-> offset m-2)
#pragma unroll
    for (int m = 0; m < R + 4; ++m) {
        // at offset m-2: dm = forward diff at offset m-3 -> dp[m], dp = dp[m+1]
        const D C = c[m];
        l[m] = fabs(C) * upwind_diff(C, dp[m], dp[m + 1]);
    }
    D del[R + 2];                // delta at offsets -1..R (index q <-> offset q-1)
#pragma unroll
    for (int q = 0; q < R + 2; ++q) {
        const int m = q + 1;     // same offset in l / c
        const D C = c[m];
        const D dd = C > D(0) ? dp[m + 1] + l[m + 1] - l[m] : -dp[m] + l[m - 1] - l[m];
        del[q] = -(l[m] + fabs(C) * dd);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int m = i + 2, q = i + 1;
        const D C = c[m];
        const D U = fabs(C);
        const D dup = C > D(0) ? del[q - 1] : (C < D(0) ? del[q + 1] : del[q]);
        o[i] = T(D(p[i + 3]) + l[m] + ((D(2) - U) * del[q] + (D(1) + U) * dup) * D(1.0 / 6.0));
    }
}

// Sliding window of the same sweep along z for one column: feed planes in
// order with push(); after plane p is pushed, out() is the result at p - 3.
template <typename T, typename D>
struct ZWin {
    D ph[4];   // Phi at p-3 .. p
    D l[3];    // l at p-3 .. p-1
    D del[3];  // delta at p-4 .. p-2
    D c[3];    // Courant at p-3 .. p-1

    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) ph[i] = D(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) l[i] = del[i] = c[i] = D(0);
    }

    // phi_p: Phi at plane p; c_pm1: Courant number at plane p-1.
    __device__ __forceinline__ T push(T phi_p, D c_pm1)
    {
        ph[0] = ph[1]; ph[1] = ph[2]; ph[2] = ph[3]; ph[3] = D(phi_p);
        c[0] = c[1]; c[1] = c[2]; c[2] = c_pm1;
        // l at p-1 (needs Phi p-2..p)
        const D dm1 = ph[2] - ph[1], dp1 = ph[3] - ph[2];
        const D lnew = fabs(c_pm1) * upwind_diff(c_pm1, dm1, dp1);
        l[0] = l[1]; l[1] = l[2]; l[2] = lnew;
        // delta at p-2 (needs Phi p-3..p-1, l p-3..p-1, Courant at p-2)
        const D C2 = c[1];
        const D dm2 = ph[1] - ph[0], dp2 = ph[2] - ph[1];
        const D dd = C2 > D(0) ? dp2 + l[2] - l[1] : -dm2 + l[0] - l[1];
        const D dnew = -(l[1] + fabs(C2) * dd);
        del[0] = del[1]; del[1] = del[2]; del[2] = dnew;
        // CEC at p-3 (needs delta p-4..p-2, l p-3, Courant at p-3)
        const D C3 = c[0];
        const D U = fabs(C3);
        const D dup = C3 > D(0) ? del[0] : (C3 < D(0) ? del[2] : del[1]);
        return T(ph[0] + l[0] + ((D(2) - U) * del[1] + (D(1) + U) * dup) * D(1.0 / 6.0));
    }
};

// ----------------------------------------------------------------- status
__device__ __forceinline__ void flag_cfl(unsigned *status, bool bad)
{
    // one atomic per warp that saw a violation
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicOr(status, 1u);
}

}  // namespace sl
