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
// intro:BEC, intro:CEC, intro:CECcoef) along a line, for |C| <= 1, with
// s = sgn C, U = |C| and W = 1 - U.  The CIR operator of Sec. 3 is written from
// the upwind neighbour (s = 0: the cell itself),
//   L_j     = Phi_{j-s_j} + W_j (Phi_j - Phi_{j-s_j}),
//   delta_j = Phi_j - L_{-U}[L]_j = (Phi_j - L_j) - U_j (L_{j+s_j} - L_j),
//   CEC_i   = a FEC_i + b BEC_i (3a = 2 - 1/U, b = 1 - a)
//           = L_i + delta_i / 2 + (1 + U_i)/6 (delta_{i-s_i} - delta_i),
// exact algebra on the definitions without 1/U.  Constant fields stay exact
// (every difference is zero), C = +-1 is an exact shift (W = 0) and C = 0
// keeps the cell.  D is the arithmetic type (float, or double with float
// storage for SL_F32_D64).

// by the sign of C: C > 0, C < 0, C == 0
template <typename D, typename V>
__device__ __forceinline__ V by_sign(D C, V pos, V neg, V zero) { return C > D(0) ? pos : (C < D(0) ? neg : zero); }

// Outputs o[0..R) of a line segment from p[0..R+6) = Phi at offsets -3..R+2
// and c[0..R+4) = Courant numbers at offsets -2..R+1.
template <typename T, typename D, int R>
__device__ __forceinline__ void cec_line(const T (&p)[R + 6], const D (&c)[R + 4], T (&o)[R])
{
    D L[R + 4];                  // offsets -2..R+1 (index m <-> offset m-2, Phi at p[m+1])
#pragma unroll
    for (int m = 0; m < R + 4; ++m) {
        const D nb = by_sign(c[m], D(p[m]), D(p[m + 2]), D(p[m + 1]));
        L[m] = nb + (D(1) - fabs(c[m])) * (D(p[m + 1]) - nb);
    }
    D del[R + 2];                // offsets -1..R (index q <-> offset q-1)
#pragma unroll
    for (int q = 0; q < R + 2; ++q) {
        const int m = q + 1;
        const D Ln = by_sign(c[m], L[m + 1], L[m - 1], L[m]);
        del[q] = (D(p[m + 1]) - L[m]) - fabs(c[m]) * (Ln - L[m]);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int m = i + 2, q = i + 1;
        const D U = fabs(c[m]);
        const D dn = by_sign(c[m], del[q - 1], del[q + 1], del[q]);
        o[i] = T(L[m] + D(0.5) * del[q] + (D(1) + U) * D(1.0 / 6.0) * (dn - del[q]));
    }
}

// Sliding window of the same sweep along z for one column: feed planes in
// order with push(); after plane p is pushed, the result is the value at p - 3.
// State after a push of plane p: Phi at p-1, p; L at p-2, p-1; Courant at p-2,
// p-1; delta at p-3, p-2.
template <typename T, typename D>
struct ZWin {
    D ph[2];   // Phi at p-2 (ph[0]), p-1 (ph[1])
    D L[2];    // L at p-3, p-2
    D c[2];    // Courant at p-3, p-2
    D dl[2];   // delta at p-4, p-3

    __device__ __forceinline__ void init()
    {
        ph[0] = ph[1] = L[0] = L[1] = c[0] = c[1] = dl[0] = dl[1] = D(0);
    }

    // phi_p: Phi at plane p; c_pm1: Courant number at plane p-1.
    __device__ __forceinline__ T push(T phi_p, D c_pm1)
    {
        const D phi = D(phi_p);
        // L at p-1 (Phi at p-2, p-1, p; Courant at p-1)
        const D nb = by_sign(c_pm1, ph[0], phi, ph[1]);
        const D Ln = nb + (D(1) - fabs(c_pm1)) * (ph[1] - nb);
        // delta at p-2 (Phi at p-2; L at p-3, p-2, p-1; Courant at p-2)
        const D C2 = c[1];
        const D Lb = by_sign(C2, Ln, L[0], L[1]);
        const D dn = (ph[0] - L[1]) - fabs(C2) * (Lb - L[1]);
        // CEC at p-3 (L at p-3; delta at p-4, p-3, p-2; Courant at p-3)
        const D C3 = c[0];
        const D dd = by_sign(C3, dl[0], dn, dl[1]);
        const T out = T(L[0] + D(0.5) * dl[1] + (D(1) + fabs(C3)) * D(1.0 / 6.0) * (dd - dl[1]));
        ph[0] = ph[1];
        ph[1] = phi;
        L[0] = L[1];
        L[1] = Ln;
        c[0] = C2;
        c[1] = c_pm1;
        dl[0] = dl[1];
        dl[1] = dn;
        return out;
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
