// k_cir_fast.cu -- unsplit CIR step (the multilinear operator L_U of Sec. 2,
// the 3D tensor-product form of eq. CIR2D) for FP32 3D grids, on groups of
// four x-adjacent cells.
//
// A CTA owns a 32 x TY column tile and marches along z.  Phi is staged plane
// by plane (tile plus one cell on each side, in 16-byte cp.async chunks) into
// a ring of 3 + PF planes, the velocity of the tile into a ring of 1 + PF
// planes; every input element is read from HBM about once per tile and every
// output element written once.
//
// One thread owns a group of four x-adjacent cells.  The value at the
// departure point x - C (|C| <= 1) mixes the cell with its neighbour at offset
// -sgn C on each axis, each lerp written from the neighbour, n + W (a - n)
// with W = 1 - |C|: |C| = 1 picks the neighbour exactly, C = 0 keeps the cell
// and a constant field stays constant.  When each Courant component has one
// nonzero sign over the group, the four cells share their stencil rows: each
// of the four corner rows (own / y-neighbour row, own / z-neighbour plane) is
// one 16-byte shared load plus one x-neighbour element, and the lerps run two
// cells at a time in packed f32x2 arithmetic.  A warp in which some group
// mixes signs (or has a zero component) evaluates its cells one by one with
// per-cell offsets.  Both forms perform the same roundings in the same order,
// so a cell's result does not depend on the form its warp took.
//
// Groups are numbered down the rows of the tile (with TY = 16 a warp holds two
// columns of 16 rows: a compact patch, so fewer warps straddle a sign
// change).  The shared rows have a pitch of 44 floats for Phi and 36 for the
// velocity, both 4 (mod 8) words, so that the 16-byte loads of eight
// consecutive rows issued by a quarter-warp fall on distinct banks.
#include "sl_internal.h"

// planes of Phi prefetched ahead, and resident CTAs per SM the register budget
// is compiled for (tile heights 16 and 32)
#ifndef SL_CIR_PF
#define SL_CIR_PF 2
#endif
#ifndef SL_CIR_MINB
#define SL_CIR_MINB 4
#endif
#ifndef SL_CIR_MINB32
#define SL_CIR_MINB32 2
#endif

namespace sl {
namespace {

constexpr int CTX = 32;      // tile width in cells
constexpr int CPP = 44;      // Phi row pitch (floats): columns [-4, 40)
constexpr int CPC = 36;      // velocity row pitch: columns [0, 32)

template <int TY_, int PF_>
struct CF {
    static constexpr int TY = TY_, PF = PF_;
    static constexpr int NT = 8 * TY;              // one thread per group of the tile
    static constexpr int RPHI = TY + 2;            // Phi rows [-1, TY + 1)
    static constexpr int NPHI = 3 + PF;            // Phi planes p-2, p-1, p + prefetch
    static constexpr int VS = 1 + PF;              // velocity planes p-1 + prefetch
    static constexpr int SPHI = RPHI * CPP, SC = TY * CPC;
    static constexpr int OFF_PHI = 4;              // 4-float guards before and after
    static constexpr int OFF_C = OFF_PHI + NPHI * SPHI;
    static constexpr int TOTAL = OFF_C + VS * 3 * SC + 4;
    static constexpr size_t smem() { return sizeof(float) * (size_t)TOTAL; }
    // staged 16-byte chunks: Phi columns [-4, 36) (10 per row), velocity [0, 32) (8 per row)
    static constexpr int N_PHI = RPHI * 10, N_C = TY * 8;
    static constexpr int K_PHI = (N_PHI + NT - 1) / NT, K_C = (N_C + NT - 1) / NT;
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float2 k2(float v) { return make_float2(v, v); }

// a - b as b * (-1) + a: the exact difference rounded once, like a subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, k2(-1.f), a); }
// n + w (a - n), the lerp from the neighbour n
__device__ __forceinline__ float2 lerp2(float2 w, float2 a, float2 n) { return __ffma2_rn(w, sub2(a, n), n); }
__device__ __forceinline__ float lerp1(float w, float a, float n) { return __fmaf_rn(w, __fsub_rn(a, n), n); }

__device__ __forceinline__ float min3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Courant numbers of a group and their sign class.
struct Grp {
    float2 v[6];   // uniform group: W = 1 - |C| (x01, x23, y01, y23, z01, z23); otherwise C itself
    int f;         // bit 0: every axis has one nonzero sign over the group; bits 1-3: C_x, C_y, C_z < 0
};

// Classify a group from its velocities; bad is set when some |C| > 1.
__device__ __forceinline__ Grp classify(float4 ux, float4 uy, float4 uz, float sx, float sy, float sz, bool &bad)
{
    const float2 cx01 = __fmul2_rn(lo2(ux), k2(sx)), cx23 = __fmul2_rn(hi2(ux), k2(sx));
    const float2 cy01 = __fmul2_rn(lo2(uy), k2(sy)), cy23 = __fmul2_rn(hi2(uy), k2(sy));
    const float2 cz01 = __fmul2_rn(lo2(uz), k2(sz)), cz23 = __fmul2_rn(hi2(uz), k2(sz));
    const float mnx = min3(cx01.x, cx01.y, fminf(cx23.x, cx23.y)), mxx = max3(cx01.x, cx01.y, fmaxf(cx23.x, cx23.y));
    const float mny = min3(cy01.x, cy01.y, fminf(cy23.x, cy23.y)), mxy = max3(cy01.x, cy01.y, fmaxf(cy23.x, cy23.y));
    const float mnz = min3(cz01.x, cz01.y, fminf(cz23.x, cz23.y)), mxz = max3(cz01.x, cz01.y, fmaxf(cz23.x, cz23.y));
    bad |= max3(mxx, mxy, mxz) > 1.f || min3(mnx, mny, mnz) < -1.f;
    // one nonzero sign per axis <=> min * max > 0 (an underflowing product only
    // sends the group to the per-cell form)
    const bool uni = min3(mnx * mxx, mny * mxy, mnz * mxz) > 0.f;
    Grp g;
    if (uni) {
        const float sxn = mnx > 0.f ? -1.f : 1.f, syn = mny > 0.f ? -1.f : 1.f, szn = mnz > 0.f ? -1.f : 1.f;
        g.v[0] = __ffma2_rn(k2(sxn), cx01, k2(1.f));
        g.v[1] = __ffma2_rn(k2(sxn), cx23, k2(1.f));
        g.v[2] = __ffma2_rn(k2(syn), cy01, k2(1.f));
        g.v[3] = __ffma2_rn(k2(syn), cy23, k2(1.f));
        g.v[4] = __ffma2_rn(k2(szn), cz01, k2(1.f));
        g.v[5] = __ffma2_rn(k2(szn), cz23, k2(1.f));
        g.f = 1 | (mnx < 0.f ? 2 : 0) | (mny < 0.f ? 4 : 0) | (mnz < 0.f ? 8 : 0);
    } else {
        g.v[0] = cx01;
        g.v[1] = cx23;
        g.v[2] = cy01;
        g.v[3] = cy23;
        g.v[4] = cz01;
        g.v[5] = cz23;
        g.f = 0;
    }
    return g;
}

// x lerps of one row of four cells whose x neighbours lie at offset DX
template <int DX>
__device__ __forceinline__ void xrow(const float *r, float2 w01, float2 w23, float2 &b01, float2 &b23)
{
    const float4 a = ld4(r);
    float2 n01, n23;
    if constexpr (DX < 0) {
        const float m = r[-1];
        n01 = make_float2(m, a.x);
        n23 = make_float2(a.y, a.z);
    } else {
        const float m = r[4];
        n01 = make_float2(a.y, a.z);
        n23 = make_float2(a.w, m);
    }
    b01 = lerp2(w01, lo2(a), n01);
    b23 = lerp2(w23, hi2(a), n23);
}

// Trilinear values of a uniform group from its four corner rows: r00 own row
// of the cell's plane, r01 the y-neighbour row, r10 / r11 the same rows of the
// z-neighbour plane.
template <int DX>
__device__ __forceinline__ float4 tri4(const float *r00, const float *r01, const float *r10, const float *r11,
                                       const Grp &g)
{
    float2 b00a, b00b, b01a, b01b, b10a, b10b, b11a, b11b;
    xrow<DX>(r00, g.v[0], g.v[1], b00a, b00b);
    xrow<DX>(r01, g.v[0], g.v[1], b01a, b01b);
    xrow<DX>(r10, g.v[0], g.v[1], b10a, b10b);
    xrow<DX>(r11, g.v[0], g.v[1], b11a, b11b);
    const float2 c0a = lerp2(g.v[2], b00a, b01a), c0b = lerp2(g.v[3], b00b, b01b);
    const float2 c1a = lerp2(g.v[2], b10a, b11a), c1b = lerp2(g.v[3], b10b, b11b);
    const float2 va = lerp2(g.v[4], c0a, c1a), vb = lerp2(g.v[5], c0b, c1b);
    return make_float4(va.x, va.y, vb.x, vb.y);
}

// The same value for one cell with its own offsets: p0 the cell in its plane,
// p1 the cell's position in the z-neighbour plane, dx / dyo the x / y
// neighbour offsets.  Same operations in the same order as tri4.
__device__ __forceinline__ float tri1(const float *p0, const float *p1, int dx, int dyo, float wx, float wy, float wz)
{
    const float b0 = lerp1(wx, p0[0], p0[dx]);
    const float b1 = lerp1(wx, p0[dyo], p0[dyo + dx]);
    const float e0 = lerp1(wx, p1[0], p1[dx]);
    const float e1 = lerp1(wx, p1[dyo], p1[dyo + dx]);
    return lerp1(wz, lerp1(wy, b0, b1), lerp1(wy, e0, e1));
}

__device__ __forceinline__ int sgn_off(float c) { return c > 0.f ? 1 : (c < 0.f ? -1 : 0); }
__device__ __forceinline__ float cell(const float2 *v, int a, int k)
{
    return k < 2 ? (k ? v[2 * a].y : v[2 * a].x) : (k == 3 ? v[2 * a + 1].y : v[2 * a + 1].x);
}

// L_U of the planes sm, s0, sp (q-1, q, q+1) at the group whose first cell
// sits at offset o; fast: every group of the warp is uniform.
__device__ __forceinline__ float4 interp(const Grp &g, bool fast, const float *sm, const float *s0, const float *sp, int o)
{
    if (fast) {
        const int dyo = (g.f & 4) ? CPP : -CPP;
        const float *r00 = s0 + o, *r01 = r00 + dyo;
        const float *r10 = ((g.f & 8) ? sp : sm) + o, *r11 = r10 + dyo;
        return (g.f & 2) ? tri4<1>(r00, r01, r10, r11, g) : tri4<-1>(r00, r01, r10, r11, g);
    }
    const bool uni = g.f & 1;
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float cx = cell(g.v, 0, k), cy = cell(g.v, 1, k), cz = cell(g.v, 2, k);
        int dx, dy, dz;
        float wx, wy, wz;
        if (uni) {   // v holds W; the neighbours lie at -sgn C of the group
            dx = (g.f & 2) ? 1 : -1;
            dy = (g.f & 4) ? 1 : -1;
            dz = (g.f & 8) ? 1 : -1;
            wx = cx;
            wy = cy;
            wz = cz;
        } else {     // v holds C
            dx = -sgn_off(cx);
            dy = -sgn_off(cy);
            dz = -sgn_off(cz);
            wx = __fsub_rn(1.f, fabsf(cx));
            wy = __fsub_rn(1.f, fabsf(cy));
            wz = __fsub_rn(1.f, fabsf(cz));
        }
        const float *p1 = (dz < 0 ? sm : (dz > 0 ? sp : s0)) + o + k;
        v[k] = tri1(s0 + o + k, p1, dx, dy * CPP, wx, wy, wz);
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

// In-plane source offsets and shared-memory destinations of a tile's staged
// 16-byte chunks (rows wrap at most once across the periodic seams).
template <int K_, int N, int CPR, int PITCH, int NT>
struct Chunks {
    int src[K_], dst[K_];
    __device__ __forceinline__ void setup(int tid, int x0, int y0, int r0, int c0, int nx, int ny)
    {
#pragma unroll
        for (int k = 0; k < K_; ++k) {
            const int idx = tid + k * NT;
            if (idx < N) {
                const int row = idx / CPR, cc = idx - row * CPR;
                int gy = y0 + r0 + row, gx = x0 + c0 + 4 * cc;
                gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
                gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
                src[k] = gy * nx + gx;
                dst[k] = row * PITCH + 4 * cc;
            } else {
                src[k] = -1;
                dst[k] = 0;
            }
        }
    }
    __device__ __forceinline__ void issue(float *sdst, const float *gsrc) const
    {
#pragma unroll
        for (int k = 0; k < K_; ++k)
            if (src[k] >= 0) cp_async16(sdst + dst[k], gsrc + src[k]);
    }
};

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int TY, int PF, int MINB>
__global__ void __launch_bounds__(CF<TY, PF>::NT, MINB)
k_cir_fast(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ vel, Geo g)
{
    using K = CF<TY, PF>;
    constexpr int NT = K::NT;
    extern __shared__ float4 smem4[];
    float *const sm = reinterpret_cast<float *>(smem4);
    float *const sPhi = sm + K::OFF_PHI;
    float *const sC = sm + K::OFF_C;
    const int tid = threadIdx.x;
    const float sx = (float)g.sx, sy = (float)g.sy, sz = (float)g.sz;
    bool bad = false;

    // this thread's group: column tid / TY (cells x .. x+3), row tid % TY
    const int x = 4 * (tid / TY), yy = tid % TY;
    const int o = (yy + 1) * CPP + x + 4;
    const int oc = yy * CPC + x;
    const int k1 = 1 % g.nz;

    // one (column tile, z chunk of g.tz planes) item per CTA
    const int64_t total = (int64_t)g.tiles_x * g.tiles_y * g.chunks;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int item = (int)w;
        const int t = item % (g.tiles_x * g.tiles_y);
        const int z0 = (item / (g.tiles_x * g.tiles_y)) * g.tz;
        const int z1 = min(z0 + g.tz, g.nz);
        const int x0 = (t % g.tiles_x) * CTX;
        const int y0 = (t / g.tiles_x) * TY;
        // Phi planes [z0 - 1, z1] are read; plane p - 1 is written in iteration p
        const int pfirst = z0 - 1, plast = z1;
        Chunks<K::K_PHI, K::N_PHI, 10, CPP, NT> chPhi;
        Chunks<K::K_C, K::N_C, 8, CPC, NT> chC;
        chPhi.setup(tid, x0, y0, -1, -4, g.nx, g.ny);
        chC.setup(tid, x0, y0, 0, 0, g.nx, g.ny);
        const bool gok = x0 + x < g.nx && y0 + yy < g.ny;
        float *const gout = out + (int64_t)(y0 + yy) * g.nx + x0 + x;

        // plane p of Phi and plane p - 1 of the velocity, into the next slots
        int pw_i = wrapi(pfirst, g.nz);
        int ph_i = 0, cv_i = 0;
        auto issue = [&](void) {
            chPhi.issue(sPhi + ph_i * K::SPHI, in + (int64_t)pw_i * g.plane);
            const float *cs = vel + (int64_t)(pw_i == 0 ? g.nz - 1 : pw_i - 1) * g.plane;
            float *cd = sC + cv_i * 3 * K::SC;
#pragma unroll
            for (int d = 0; d < 3; ++d) chC.issue(cd + d * K::SC, cs + d * g.ncell);
            ph_i = ph_i + 1 == K::NPHI ? 0 : ph_i + 1;
            cv_i = cv_i + 1 == K::VS ? 0 : cv_i + 1;
            pw_i = pw_i + 1 == g.nz ? 0 : pw_i + 1;
        };

#pragma unroll
        for (int j = 0; j < PF; ++j) {
            if (pfirst + j <= plast) issue();
            cp_async_commit();
        }
        int pw = wrapi(pfirst, g.nz);   // plane p modulo nz
        int sphi = 0, scv = 0;          // ring slots of plane p
        for (int p = pfirst; p <= plast; ++p) {
            cp_async_wait<PF - 1>();
            __syncthreads();
            if (p + PF <= plast) issue();
            cp_async_commit();
            if (p > pfirst + 1) {   // L_U[Phi] at plane p - 1: Phi planes p-2, p-1, p
                const int a1 = sphi == 0 ? K::NPHI - 1 : sphi - 1, a2 = a1 == 0 ? K::NPHI - 1 : a1 - 1;
                const float *cv = sC + scv * 3 * K::SC + oc;
                const Grp gr = classify(ld4(cv), ld4(cv + K::SC), ld4(cv + 2 * K::SC), sx, sy, sz, bad);
                const bool fast = __all_sync(0xffffffffu, gr.f & 1);
                const float4 v = interp(gr, fast, sPhi + a2 * K::SPHI, sPhi + a1 * K::SPHI, sPhi + sphi * K::SPHI, o);
                if (gok) {
                    const int q = pw - k1 < 0 ? pw - k1 + g.nz : pw - k1;
                    st4(gout + (int64_t)q * g.plane, v);
                }
            }
            pw = pw + 1 == g.nz ? 0 : pw + 1;
            sphi = sphi + 1 == K::NPHI ? 0 : sphi + 1;
            scv = scv + 1 == K::VS ? 0 : scv + 1;
        }
        __syncthreads();
    }
    flag_cfl(g.status, bad);
}

template <int TY, int PF, int MINB>
cudaError_t go_cir(Geo g, int grid, const float *in, float *out, const float *vel, cudaStream_t st)
{
    using K = CF<TY, PF>;
    auto kern = k_cir_fast<TY, PF, MINB>;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem());
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    g.tiles_x = (g.nx + CTX - 1) / CTX;
    g.tiles_y = (g.ny + TY - 1) / TY;
    const int64_t total = (int64_t)g.tiles_x * g.tiles_y * g.chunks;
    int gr = grid > 0 ? grid : (int)total;
    if (gr > total) gr = (int)total;
    kern<<<gr, K::NT, K::smem(), st>>>(in, out, vel, g);
    return cudaGetLastError();
}

}  // namespace

bool cir_fast_eligible(int dtype, int ndim, const int64_t dims[3], bool aligned)
{
    // FP32, 3D, 16-byte aligned rows of whole groups; Phi rows of a tile
    // (columns [-4, 36)) and rows [-1, TY + 1) wrap at most once (TY = 16, or
    // 32 where dims[1] >= 32)
    return dtype == 0 && ndim == 3 && aligned && dims[0] % 4 == 0 && dims[0] >= 40 && dims[1] >= 16 &&
           dims[0] * dims[1] < (int64_t(1) << 31);
}

cudaError_t launch_cir_fast(const void *in, void *out, const void *vel, const int64_t dims[3], const double s[3],
                            Launch lc, unsigned *status, cudaStream_t st)
{
    Geo g;
    g.nx = (int)dims[0];
    g.ny = (int)dims[1];
    g.nz = (int)dims[2];
    g.plane = (int64_t)g.nx * g.ny;
    g.ncell = g.plane * g.nz;
    g.sx = s[0];
    g.sy = s[1];
    g.sz = s[2];
    g.status = status;
    g.tz = lc.tz > 0 ? lc.tz : default_tz(0, 3, dims);
    if (g.tz > g.nz) g.tz = g.nz;
    g.chunks = (g.nz + g.tz - 1) / g.tz;
    const float *fi = static_cast<const float *>(in);
    const float *fv = static_cast<const float *>(vel);
    float *fo = static_cast<float *>(out);
    // tile height 32 where a tile fits (a launch-shape choice), else 16
    if (lc.ty == 32 && g.ny >= 32) return go_cir<32, SL_CIR_PF, SL_CIR_MINB32>(g, lc.grid, fi, fo, fv, st);
    return go_cir<16, SL_CIR_PF, SL_CIR_MINB>(g, lc.grid, fi, fo, fv, st);
}

}  // namespace sl
