// k_cec_fast.cu -- the fused split third-order step (SL_CEC, FP32) for grids
// whose rows can be staged by the bulk-copy engine (nx % 4 == 0, nx >= 40,
// ny >= 38, 16-byte aligned buffers).  Same mathematics as k_split.cu (Sec. 2
// eqs. intro:FEC, intro:BEC, intro:CEC, intro:CECcoef, one 1D sweep per axis,
// Sec. 5 eqs. split:1-2), organised for instruction economy:
//
//  - Staging: each x-y plane of Phi and u (with its periodic halo) is copied
//    in 16-byte cp.async chunks whose source and destination offsets every
//    thread computes once per segment, double-buffered one plane ahead.
//  - Work split: persistent CTAs; the (column tile, plane) pairs of all grids
//    are numbered and every CTA takes one contiguous, equal share, walking
//    z inside each column tile, so every SM gets the same number of planes.
//  - The z sweep runs in per-column register windows (10 registers per column,
//    the plane loop unrolled by two so no value is ever moved); the x and y
//    sweeps run on runs of 8 / 4 cells in registers from shared memory.
#include <type_traits>

#include "sl_internal.h"

namespace sl {
namespace {

// ------------------------------------------------------------ 1D sweep math
// cec_run: outputs o[0..R) of a line from p[0..R+6) = Phi at offsets -3..R+2
// and c[0..R+4) = Courant numbers at offsets -2..R+1.  With D_j = Phi_{j+1} -
// Phi_j, l_j = L_U[Phi]_j - Phi_j = -C_j D_{j-1} (C_j > 0) or -C_j D_j,
// E_j = L_U[Phi]_{j+1} - L_U[Phi]_j = D_j + l_{j+1} - l_j, the round-trip
// difference is delta_j = Phi_j - Phi_bar_j = -l_j - C_j E_j (C_j > 0) or
// -l_j - C_j E_{j-1}, and the combination a FEC + b BEC (3a = 2 - 1/U,
// b = 1 - a) is Phi_i + l_i + ((2 - U_i) delta_i + (1 + U_i) delta_{i-s_i})/6.
template <int R>
__device__ __forceinline__ void cec_run(const float (&p)[R + 6], const float (&c)[R + 4], float (&o)[R])
{
    float dp[R + 5];
#pragma unroll
    for (int j = 0; j < R + 5; ++j) dp[j] = p[j + 1] - p[j];
    float l[R + 4];
#pragma unroll
    for (int m = 0; m < R + 4; ++m) l[m] = -c[m] * (c[m] > 0.f ? dp[m] : dp[m + 1]);
    float e[R + 3];
#pragma unroll
    for (int k = 0; k < R + 3; ++k) e[k] = dp[k + 1] + (l[k + 1] - l[k]);
    float del[R + 2];
#pragma unroll
    for (int q = 0; q < R + 2; ++q) del[q] = -l[q + 1] - c[q + 1] * (c[q + 1] > 0.f ? e[q + 1] : e[q]);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float C = c[i + 2], U = fabsf(C), d0 = del[i + 1];
        const float dup = C > 0.f ? del[i] : (C < 0.f ? del[i + 2] : d0);
        o[i] = (p[i + 3] + l[i + 2]) + (2.f * d0 + dup + U * (dup - d0)) * (1.f / 6.f);
    }
}

// The same run when every Courant number of it has the sign S (+1 or -1):
// the upwind side is fixed, so no comparison or selection is needed.
template <int R, int S>
__device__ __forceinline__ void cec_run_signed(const float (&p)[R + 6], const float (&c)[R + 4], float (&o)[R])
{
    float dp[R + 5];
#pragma unroll
    for (int j = 0; j < R + 5; ++j) dp[j] = p[j + 1] - p[j];
    float l[R + 4];
#pragma unroll
    for (int m = 0; m < R + 4; ++m) l[m] = -c[m] * (S > 0 ? dp[m] : dp[m + 1]);
    float e[R + 3];
#pragma unroll
    for (int k = 0; k < R + 3; ++k) e[k] = dp[k + 1] + (l[k + 1] - l[k]);
    float del[R + 2];
#pragma unroll
    for (int q = 0; q < R + 2; ++q) del[q] = -l[q + 1] - c[q + 1] * (S > 0 ? e[q + 1] : e[q]);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float U = S > 0 ? c[i + 2] : -c[i + 2], d0 = del[i + 1];
        const float dup = S > 0 ? del[i] : del[i + 2];
        o[i] = (p[i + 3] + l[i + 2]) + (2.f * d0 + dup + U * (dup - d0)) * (1.f / 6.f);
    }
}

// Picks the sign-specialised form when the whole warp's runs share one sign.
template <int R>
__device__ __forceinline__ void cec_run_auto(const float (&p)[R + 6], const float (&c)[R + 4], float (&o)[R])
{
    bool pos = true, neg = true;
#pragma unroll
    for (int k = 0; k < R + 4; ++k) {
        pos &= c[k] > 0.f;
        neg &= c[k] < 0.f;
    }
    const unsigned am = __activemask();
    if (__all_sync(am, pos))
        cec_run_signed<R, 1>(p, c, o);
    else if (__all_sync(am, neg))
        cec_run_signed<R, -1>(p, c, o);
    else
        cec_run<R>(p, c, o);
}

// z sweep window of one column.  push<P>(phi_p, c_{p-1}) returns the result at
// plane p-3; P alternates 0, 1 so that two-deep values change roles instead of
// being moved.
struct ZCol {
    float ph;       // Phi_{p-1}
    float d;        // D_{p-2}
    float l;        // l_{p-2}
    float e;        // E_{p-3}
    float c[2];     // Courant at p-3 / p-2 (roles swap with P)
    float L[2];     // L_U[Phi] at p-3 / p-2
    float dl[2];    // delta at p-4 / p-3

    __device__ __forceinline__ void init()
    {
        ph = d = l = e = 0.f;
        c[0] = c[1] = L[0] = L[1] = dl[0] = dl[1] = 0.f;
    }

    template <int P>
    __device__ __forceinline__ float push(float phi, float cn)
    {
        const float dn = phi - ph;                               // D_{p-1}
        const float ln = -cn * (cn > 0.f ? d : dn);              // l_{p-1}
        const float Ln = ph + ln;                                // L at p-1
        const float en = d + (ln - l);                           // E_{p-2}
        const float c2 = c[P ^ 1];                               // Courant at p-2
        const float dn2 = -l - c2 * (c2 > 0.f ? en : e);         // delta_{p-2}
        const float C = c[P], U = fabsf(C), d0 = dl[P ^ 1];      // output plane p-3
        const float dup = C > 0.f ? dl[P] : (C < 0.f ? dn2 : d0);
        const float out = L[P] + (2.f * d0 + dup + U * (dup - d0)) * (1.f / 6.f);
        ph = phi;
        d = dn;
        l = ln;
        e = en;
        c[P] = cn;       // becomes "p-2" at the next push
        L[P] = Ln;
        dl[P] = dn2;
        return out;
    }

    // push<P> when the Courant numbers at p-3, p-2 and p-1 all have sign S
    template <int P, int S>
    __device__ __forceinline__ float push_signed(float phi, float cn)
    {
        const float dn = phi - ph;
        const float ln = -cn * (S > 0 ? d : dn);
        const float Ln = ph + ln;
        const float en = d + (ln - l);
        const float c2 = c[P ^ 1];
        const float dn2 = -l - c2 * (S > 0 ? en : e);
        const float U = S > 0 ? c[P] : -c[P], d0 = dl[P ^ 1];
        const float dup = S > 0 ? dl[P] : dn2;
        const float out = L[P] + (2.f * d0 + dup + U * (dup - d0)) * (1.f / 6.f);
        ph = phi;
        d = dn;
        l = ln;
        e = en;
        c[P] = cn;
        L[P] = Ln;
        dl[P] = dn2;
        return out;
    }

    template <int P>
    __device__ __forceinline__ bool sign_pos(float cn) const { return cn > 0.f && c[0] > 0.f && c[1] > 0.f; }
    template <int P>
    __device__ __forceinline__ bool sign_neg(float cn) const { return cn < 0.f && c[0] < 0.f && c[1] < 0.f; }
};

// Pushes one plane into N windows, sign-specialised when the whole warp agrees.
template <int P, int N>
__device__ __forceinline__ void push_all(ZCol (&win)[N], const float (&phi)[N], const float (&cn)[N], float (&out)[N])
{
    bool pos = true, neg = true;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        pos &= win[i].template sign_pos<P>(cn[i]);
        neg &= win[i].template sign_neg<P>(cn[i]);
    }
    const unsigned am = __activemask();
    if (__all_sync(am, pos)) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = win[i].template push_signed<P, 1>(phi[i], cn[i]);
    } else if (__all_sync(am, neg)) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = win[i].template push_signed<P, -1>(phi[i], cn[i]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = win[i].template push<P>(phi[i], cn[i]);
    }
}

// ---------------------------------------------------------------- geometry
struct Seg {
    int inst, tx, ty, z0, z1;
};

// Walks a CTA's share [w, wend) of the numbered (column tile, plane) pairs.
// The pairs of one column tile are numbered from a tile-dependent plane phi
// (periodic in z), chosen so that the share boundaries of every tile fall on
// the same planes: CTAs that start together then process the same z plane of
// neighbouring tiles at about the same time, and the halo rows one tile stages
// are still in L2 when its neighbours stage them.
__device__ __forceinline__ bool next_seg(const FastInst *tab, int ninst, int64_t &w, int64_t wend, int &hint,
                                         double share, Seg &s)
{
    if (w >= wend) return false;
    while (hint + 1 < ninst && tab[hint + 1].w0 <= w) ++hint;
    const FastInst &I = tab[hint];
    const int64_t local = w - I.w0;
    const int t = (int)(local / I.nz);
    const int o = (int)(local - (int64_t)t * I.nz);
    const int64_t tile_w = I.w0 + (int64_t)t * I.nz;
    int phi = (int)(fmod((double)tile_w, share) + 0.5);
    phi = phi % I.nz;
    const int64_t tile_end = tile_w + I.nz;
    const int64_t e = wend < tile_end ? wend : tile_end;
    s.inst = hint;
    s.tx = t % I.tiles_x;
    s.ty = t / I.tiles_x;
    s.z0 = o + phi;                    // in [0, 2 nz); planes are taken modulo nz
    s.z1 = s.z0 + (int)(e - w);
    w = e;
    return true;
}

__device__ __forceinline__ int wrapz(int p, int nz) { return ((p % nz) + nz) % nz; }

// 16-byte chunks of one staged array: rows [r0, r0 + NR) relative to the
// tile, x range [x0 + c0, x0 + c0 + 4 CPR) (c0 and x0 multiples of 4, nx a
// multiple of 4, so no chunk straddles the periodic seam).  Thread tid owns
// chunks tid + k NT; the in-plane source offset and the shared-memory offset
// of each are computed once per segment.
template <int NT, int NR, int CPR, int LD>
struct Chunks {
    static constexpr int N = NR * CPR;
    static constexpr int K = (N + NT - 1) / NT;
    int src[K];
    int dst[K];

    __device__ __forceinline__ void setup(int tid, int x0, int y0, int r0, int c0, int nx, int ny)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int idx = tid + k * NT;
            if (idx < N) {
                const int row = idx / CPR, cc = idx - (idx / CPR) * CPR;
                int gy = y0 + r0 + row;
                gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
                int gx = x0 + c0 + 4 * cc;
                gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
                src[k] = gy * nx + gx;
                dst[k] = row * LD + 4 * cc;
            } else {
                src[k] = -1;
                dst[k] = 0;
            }
        }
    }

    __device__ __forceinline__ void issue(float *sdst, const float *gsrc) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (src[k] >= 0) cp_async16(sdst + dst[k], gsrc + src[k]);
    }
};

// ============================================================ order x, y, z
#ifndef SL_XYZ_MINB
#define SL_XYZ_MINB 2      // CTAs per SM the x,y,z kernel is compiled for
#endif
#ifndef SL_ZYX_NT
#define SL_ZYX_NT 256      // threads of the z,y,x kernel
#endif
#ifndef SL_ZYX_RX
#define SL_ZYX_RX 8        // x-sweep run length of the z,y,x kernel
#endif
#ifndef SL_XYZ_RX
#define SL_XYZ_RX 8        // x-sweep run length of the x,y,z kernel
#endif
#ifndef SL_ZYX_RY
#define SL_ZYX_RY 8        // y-sweep run length of the z,y,x kernel
#endif

namespace xyz {
constexpr int TX = 32, TY = 32, NT = 256, RX = SL_XYZ_RX, RY = 4;
constexpr int PH = TY + 6, PW = TX + 12;              // Phi / u_x rows [-3, TY+3), x [-4, TX+4), stride 44
constexpr int SZ_PHI = PH * PW;
constexpr int SZ_CY = (TY + 4) * TX;                  // u_y rows [-2, TY+2), x [0, TX)
constexpr int SZ_CZ = TY * TX;                        // u_z rows [0, TY)
constexpr int SLOT = 2 * SZ_PHI + SZ_CY + SZ_CZ;
constexpr int SZ_S1 = PH * TX;                        // x-swept rows
constexpr size_t SMEM = sizeof(float) * (2 * SLOT + SZ_S1) + 128;
}  // namespace xyz

template <bool BATCH>
__global__ void __launch_bounds__(xyz::NT, SL_XYZ_MINB)
k_cec_xyz_fast(const __grid_constant__ FastInst one, const FastInst *__restrict__ table, int ninst, int64_t total, unsigned *status)
{
    using namespace xyz;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *sS1 = buf + 2 * SLOT;

    const int tid = threadIdx.x;
    const FastInst *tab = BATCH ? table : &one;
    const int64_t G = gridDim.x;
    int64_t w = total * blockIdx.x / G;
    const int64_t wend = total * (blockIdx.x + 1) / G;
    bool bad = false;
    int hint = 0;
    Seg sg;
    const int cx = tid % TX, yr = (tid / TX) * RY;
    Chunks<NT, PH, (TX + 8) / 4, PW> chPhi;        // Phi and u_x: rows [-3, TY+3), x [-4, TX+4)
    Chunks<NT, TY + 4, TX / 4, TX> chCy;           // u_y: rows [-2, TY+2), x [0, TX)
    Chunks<NT, TY, TX / 4, TX> chCz;               // u_z: rows [0, TY)

    while (next_seg(tab, ninst, w, wend, hint, (double)total / (double)G, sg)) {
        const FastInst &I = tab[sg.inst];
        const int x0 = sg.tx * TX, y0 = sg.ty * TY;
        const float sx = I.sx, sy = I.sy, sz = I.sz;
        const int pfirst = sg.z0 - 3, plast = sg.z1 + 2;

        chPhi.setup(tid, x0, y0, -3, -4, I.nx, I.ny);
        chCy.setup(tid, x0, y0, -2, 0, I.nx, I.ny);
        chCz.setup(tid, x0, y0, 0, 0, I.nx, I.ny);
        // pz: plane index of the bundle, already reduced modulo nz
        auto issue = [&](int pz, int slot) {
            float *sb = buf + slot * SLOT;
            const int pz1 = pz == 0 ? I.nz - 1 : pz - 1;
            const float *vx = I.vel + (int64_t)pz * I.plane;
            chPhi.issue(sb, I.in + (int64_t)pz * I.plane);
            chPhi.issue(sb + SZ_PHI, vx);
            chCy.issue(sb + 2 * SZ_PHI, vx + I.ncell);
            chCz.issue(sb + 2 * SZ_PHI + SZ_CY, I.vel + 2 * I.ncell + (int64_t)pz1 * I.plane);
            cp_async_commit();
        };

        ZCol win[RY];
#pragma unroll
        for (int i = 0; i < RY; ++i) win[i].init();

        // one plane: x sweep into sS1, y sweep, z windows, store
        // p: unreduced plane; zw: p modulo nz
        auto plane = [&](auto PC, int p, int zw) {
            constexpr int P = decltype(PC)::value;
            const int slot = (p - pfirst) & 1;
            cp_async_wait_all();
            __syncthreads();
            if (p < plast) issue(zw + 1 == I.nz ? 0 : zw + 1, slot ^ 1);
            const float *sb = buf + slot * SLOT;
            const float *phiP = sb, *cxP = sb + SZ_PHI, *cyP = sb + 2 * SZ_PHI, *czP = sb + 2 * SZ_PHI + SZ_CY;
            constexpr int XR = TX / RX;
            for (int r = tid; r < PH * XR; r += NT) {
                const int row = r / XR, xr = (r % XR) * RX;
                const float4 *pr = reinterpret_cast<const float4 *>(phiP + row * PW + xr);
                const float4 *cr = reinterpret_cast<const float4 *>(cxP + row * PW + xr);
                float blk[RX + 8], pv[RX + 6], cv[RX + 4], o[RX];
#pragma unroll
                for (int k = 0; k < (RX + 8) / 4; ++k) {
                    const float4 v = pr[k];
                    blk[4 * k] = v.x; blk[4 * k + 1] = v.y; blk[4 * k + 2] = v.z; blk[4 * k + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < RX + 6; ++k) pv[k] = blk[k + 1];
#pragma unroll
                for (int k = 0; k < (RX + 8) / 4; ++k) {
                    const float4 v = cr[k];
                    blk[4 * k] = v.x; blk[4 * k + 1] = v.y; blk[4 * k + 2] = v.z; blk[4 * k + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < RX + 4; ++k) cv[k] = blk[k + 2] * sx;
#pragma unroll
                for (int k = 2; k < RX + 2; ++k) bad |= fabsf(cv[k]) > 1.f;
                cec_run_auto<RX>(pv, cv, o);
                float4 *dst = reinterpret_cast<float4 *>(sS1 + row * TX + xr);
#pragma unroll
                for (int k = 0; k < RX / 4; ++k) dst[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
            }
            __syncthreads();
            float pv[RY + 6], cv[RY + 4], o[RY];
#pragma unroll
            for (int k = 0; k < RY + 6; ++k) pv[k] = sS1[(yr + k) * TX + cx];
#pragma unroll
            for (int k = 0; k < RY + 4; ++k) cv[k] = cyP[(yr + k) * TX + cx] * sy;
#pragma unroll
            for (int k = 2; k < RY + 2; ++k) bad |= fabsf(cv[k]) > 1.f;
            cec_run_auto<RY>(pv, cv, o);
            const bool store = p - 3 >= sg.z0;
            const int kw = zw >= 3 ? zw - 3 : zw - 3 + I.nz;
            float *dst = I.out + (int64_t)kw * I.plane + (int64_t)(y0 + yr) * I.nx + x0 + cx;
            float cz[RY], res[RY];
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                cz[i] = czP[(yr + i) * TX + cx] * sz;
                bad |= fabsf(cz[i]) > 1.f;
            }
            push_all<P, RY>(win, o, cz, res);
            if (store) {
#pragma unroll
                for (int i = 0; i < RY; ++i) dst[(int64_t)i * I.nx] = res[i];
            }
        };

        int zw = wrapz(pfirst, I.nz);
        issue(zw, 0);
        for (int p = pfirst; p <= plast; p += 2) {
            plane(std::integral_constant<int, 0>(), p, zw);
            zw = zw + 1 == I.nz ? 0 : zw + 1;
            if (p + 1 <= plast) plane(std::integral_constant<int, 1>(), p + 1, zw);
            zw = zw + 1 == I.nz ? 0 : zw + 1;
        }
        __syncthreads();   // shared buffers are reused by the next segment
    }
    flag_cfl(status, bad);
}

// ============================================================ order z, y, x
namespace zyx {
constexpr int TX = 32, TY = 32, NT = SL_ZYX_NT, RX = SL_ZYX_RX, RY = SL_ZYX_RY;
constexpr int PH = TY + 6, PW = TX + 12;
constexpr int SZ_PHI = PH * PW;                      // Phi and u_z (plane p-1): rows [-3, TY+3)
constexpr int SZ_CY = (TY + 4) * PW;                 // u_y (plane p-3): rows [-2, TY+2)
constexpr int SZ_CX = TY * PW;                       // u_x (plane p-3): rows [0, TY)
constexpr int SLOT = 2 * SZ_PHI + SZ_CY + SZ_CX;
constexpr int NZC = (TX + 6) * (TY + 6);             // z-swept columns (x, y in [-3, T+3))
constexpr int NCOL = (NZC + NT - 1) / NT;
constexpr size_t SMEM = sizeof(float) * (2 * SLOT + SZ_PHI + SZ_CX) + 128;
}  // namespace zyx

template <bool BATCH>
__global__ void __launch_bounds__(zyx::NT, 512 / SL_ZYX_NT)
k_cec_zyx_fast(const __grid_constant__ FastInst one, const FastInst *__restrict__ table, int ninst, int64_t total,
               unsigned *status)
{
    using namespace zyx;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *sZ = buf + 2 * SLOT;                      // z-swept plane, rows [-3, TY+3)
    float *sS2 = sZ + SZ_PHI;                        // y-swept rows [0, TY)

    const int tid = threadIdx.x;
    const FastInst *tab = BATCH ? table : &one;
    const int64_t G = gridDim.x;
    int64_t w = total * blockIdx.x / G;
    const int64_t wend = total * (blockIdx.x + 1) / G;
    bool bad = false;
    int hint = 0;
    Seg sg;
    Chunks<NT, PH, (TX + 8) / 4, PW> chPhi;        // Phi and u_z: rows [-3, TY+3), x [-4, TX+4)
    Chunks<NT, TY + 4, (TX + 8) / 4, PW> chCy;     // u_y: rows [-2, TY+2)
    Chunks<NT, TY, (TX + 8) / 4, PW> chCx;         // u_x: rows [0, TY)

    // per-thread z columns: staged offsets (row = y + 3, col = x + 4)
    int zoff[NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
        const int r = tid + j * NT;
        zoff[j] = r < NZC ? (r / (TX + 6)) * PW + (r % (TX + 6)) + 1 : -1;
    }

    while (next_seg(tab, ninst, w, wend, hint, (double)total / (double)G, sg)) {
        const FastInst &I = tab[sg.inst];
        const int x0 = sg.tx * TX, y0 = sg.ty * TY;
        const float sx = I.sx, sy = I.sy, sz = I.sz;
        const int pfirst = sg.z0 - 3, plast = sg.z1 + 2;
        chPhi.setup(tid, x0, y0, -3, -4, I.nx, I.ny);
        chCy.setup(tid, x0, y0, -2, -4, I.nx, I.ny);
        chCx.setup(tid, x0, y0, 0, -4, I.nx, I.ny);

        // pz: plane index of the bundle, already reduced modulo nz
        auto issue = [&](int pz, int slot) {
            float *sb = buf + slot * SLOT;
            const int nz = I.nz;
            const int pz1 = pz == 0 ? nz - 1 : pz - 1;
            const float *vk = I.vel + (int64_t)(pz >= 3 ? pz - 3 : pz - 3 + nz) * I.plane;
            chPhi.issue(sb, I.in + (int64_t)pz * I.plane);
            chPhi.issue(sb + SZ_PHI, I.vel + 2 * I.ncell + (int64_t)pz1 * I.plane);
            chCy.issue(sb + 2 * SZ_PHI, vk + I.ncell);
            chCx.issue(sb + 2 * SZ_PHI + SZ_CY, vk);
            cp_async_commit();
        };

        ZCol win[NCOL];
#pragma unroll
        for (int j = 0; j < NCOL; ++j) win[j].init();

        auto plane = [&](auto PC, int p, int zw) {
            constexpr int P = decltype(PC)::value;
            const int slot = (p - pfirst) & 1;
            cp_async_wait_all();
            __syncthreads();
            if (p < plast) issue(zw + 1 == I.nz ? 0 : zw + 1, slot ^ 1);
            const float *sb = buf + slot * SLOT;
            const float *phiP = sb, *czP = sb + SZ_PHI, *cyP = sb + 2 * SZ_PHI, *cxP = sb + 2 * SZ_PHI + SZ_CY;
            // ---- z sweep on the halo-widened columns
#pragma unroll
            for (int j = 0; j < NCOL; ++j) {
                if (zoff[j] >= 0) {
                    const int o = zoff[j];
                    const float c = czP[o] * sz;
                    sZ[o] = win[j].push<P>(phiP[o], c);
                    const int row = o / PW, col = o - row * PW;
                    if (row >= 3 && row < TY + 3 && col >= 4 && col < TX + 4) bad |= fabsf(c) > 1.f;
                }
            }
            __syncthreads();
            if (p - 3 < sg.z0) return;
            const int kw = zw >= 3 ? zw - 3 : zw - 3 + I.nz;
            // ---- y sweep: columns x in [-3, TX+3), rows [0, TY) -> sS2
            for (int r = tid; r < (TX + 6) * (TY / RY); r += NT) {
                const int col = r % (TX + 6) + 1, yr = (r / (TX + 6)) * RY;
                float pv[RY + 6], cv[RY + 4], o[RY];
#pragma unroll
                for (int k = 0; k < RY + 6; ++k) pv[k] = sZ[(yr + k) * PW + col];
#pragma unroll
                for (int k = 0; k < RY + 4; ++k) cv[k] = cyP[(yr + k) * PW + col] * sy;
                if (col >= 4 && col < TX + 4) {
#pragma unroll
                    for (int k = 2; k < RY + 2; ++k) bad |= fabsf(cv[k]) > 1.f;
                }
                cec_run_auto<RY>(pv, cv, o);
#pragma unroll
                for (int i = 0; i < RY; ++i) sS2[(yr + i) * PW + col] = o[i];
            }
            __syncthreads();
            // ---- x sweep: rows [0, TY), cols [0, TX) -> global plane kz
            constexpr int XR = TX / RX;
            for (int r = tid; r < TY * XR; r += NT) {
                const int row = r / XR, xr = (r % XR) * RX;
                const float4 *pr = reinterpret_cast<const float4 *>(sS2 + row * PW + xr);
                const float4 *cr = reinterpret_cast<const float4 *>(cxP + row * PW + xr);
                float blk[RX + 8], pv[RX + 6], cv[RX + 4], o[RX];
#pragma unroll
                for (int k = 0; k < (RX + 8) / 4; ++k) {
                    const float4 v = pr[k];
                    blk[4 * k] = v.x; blk[4 * k + 1] = v.y; blk[4 * k + 2] = v.z; blk[4 * k + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < RX + 6; ++k) pv[k] = blk[k + 1];
#pragma unroll
                for (int k = 0; k < (RX + 8) / 4; ++k) {
                    const float4 v = cr[k];
                    blk[4 * k] = v.x; blk[4 * k + 1] = v.y; blk[4 * k + 2] = v.z; blk[4 * k + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < RX + 4; ++k) cv[k] = blk[k + 2] * sx;
#pragma unroll
                for (int k = 2; k < RX + 2; ++k) bad |= fabsf(cv[k]) > 1.f;
                cec_run_auto<RX>(pv, cv, o);
                float4 *dst = reinterpret_cast<float4 *>(I.out + (int64_t)kw * I.plane + (int64_t)(y0 + row) * I.nx +
                                                         x0 + xr);
#pragma unroll
                for (int k = 0; k < RX / 4; ++k) dst[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
            }
        };

        int zw = wrapz(pfirst, I.nz);
        issue(zw, 0);
        for (int p = pfirst; p <= plast; p += 2) {
            plane(std::integral_constant<int, 0>(), p, zw);
            zw = zw + 1 == I.nz ? 0 : zw + 1;
            if (p + 1 <= plast) plane(std::integral_constant<int, 1>(), p + 1, zw);
            zw = zw + 1 == I.nz ? 0 : zw + 1;
        }
        __syncthreads();
    }
    flag_cfl(status, bad);
}

// Shared-memory opt-in and persistent grid size of one kernel, once per device.
template <bool ZYX, bool BATCH>
cudaError_t prepare(int &grid)
{
    static int cached[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cached[dev] == 0) {
        auto kern = ZYX ? k_cec_zyx_fast<BATCH> : k_cec_xyz_fast<BATCH>;
        const size_t smem = ZYX ? zyx::SMEM : xyz::SMEM;
        const int nt = ZYX ? zyx::NT : xyz::NT;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        cached[dev] = sms * (per_sm > 0 ? per_sm : 1);
    }
    grid = cached[dev];
    return cudaSuccess;
}

template <bool ZYX, bool BATCH>
cudaError_t go_fast(const FastInst &one, const FastInst *tab, int ninst, int64_t total, unsigned *status,
                    int grid_req, cudaStream_t st)
{
    int grid = 0;
    cudaError_t e = prepare<ZYX, BATCH>(grid);
    if (e != cudaSuccess) return e;
    if (grid_req > 0) grid = grid_req;
    if (grid > total) grid = (int)total;
    if (ZYX)
        k_cec_zyx_fast<BATCH><<<grid, zyx::NT, zyx::SMEM, st>>>(one, tab, ninst, total, status);

    else
        k_cec_xyz_fast<BATCH><<<grid, xyz::NT, xyz::SMEM, st>>>(one, tab, ninst, total, status);
    return cudaGetLastError();
}

}  // namespace

bool fast_eligible(const int64_t dims[3], int ndim, int dtype, bool aligned)
{
    // whole 32 x 32 column tiles, a staged row wraps at most once (nx >= 40),
    // halo planes and rows wrap at most once (nz >= 8, ny >= 32)
    return dtype == 0 && ndim == 3 && aligned && dims[0] % 32 == 0 && dims[1] % 32 == 0 && dims[0] >= 64 &&
           dims[1] >= 32 && dims[2] >= 8;
}

void fast_fill(FastInst &f, const void *in, void *out, const void *vel, const int64_t dims[3], const double s[3],
               int64_t w0)
{
    f.in = static_cast<const float *>(in);
    f.out = static_cast<float *>(out);
    f.vel = static_cast<const float *>(vel);
    f.nx = (int)dims[0];
    f.ny = (int)dims[1];
    f.nz = (int)dims[2];
    f.plane = (int64_t)f.nx * f.ny;
    f.ncell = f.plane * f.nz;
    f.tiles_x = f.nx / 32;
    f.ntiles = f.tiles_x * (f.ny / 32);
    f.sx = (float)s[0];
    f.sy = (float)s[1];
    f.sz = (float)s[2];
    f.w0 = w0;
}

cudaError_t launch_cec_fast(const FastInst &one, const FastInst *dev_table, int ninst, int64_t total, int parity,
                            unsigned *status, int grid_req, cudaStream_t st)
{
    const bool zyx_order = parity & 1;
    if (dev_table)
        return zyx_order ? go_fast<true, true>(one, dev_table, ninst, total, status, grid_req, st)
                         : go_fast<false, true>(one, dev_table, ninst, total, status, grid_req, st);
    return zyx_order ? go_fast<true, false>(one, nullptr, 1, total, status, grid_req, st)
                     : go_fast<false, false>(one, nullptr, 1, total, status, grid_req, st);
}

int fast_grid(int parity)
{
    int g = 0;
    if (((parity & 1) ? prepare<true, false>(g) : prepare<false, false>(g)) != cudaSuccess) return 0;
    return g;
}

}  // namespace sl
