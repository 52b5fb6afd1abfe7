// k_cec_fast.cu -- the fused split third-order step (SL_CEC, FP32) for grids
// of whole 32 x 32 column tiles (nx, ny multiples of 32, nx >= 64, nz >= 8,
// 16-byte aligned buffers): one persistent launch per step, one HBM read of
// Phi and u and one write of the result per cell.
//
// Mathematics (Sec. 2 eqs. intro:FEC, intro:BEC, intro:CEC, intro:CECcoef; one
// 1D sweep per axis as in Sec. 2 last paragraph and Sec. 5 eqs. split:1-2).
// Along a line with Courant numbers C_j (|C_j| <= 1), s_j = sgn C_j,
// U_j = |C_j| and W_j = 1 - U_j, the CIR operator of Sec. 3 is written from
// the upwind neighbour:
//   L_j     = Phi_{j-s_j} + W_j (Phi_j - Phi_{j-s_j})
//   delta_j = Phi_j - L_{-U}[L]_j = (Phi_j - L_j) - U_j (L_{j+s_j} - L_j)
//   CEC_i   = a FEC_i + b BEC_i  (3a = 2 - 1/U, b = 1 - a)
//           = L_i + delta_i / 2 + (1 + U_i)/6 (delta_{i-s_i} - delta_i),
// which has no 1/U and is exact algebra on the definitions.  This form keeps
// constant fields exactly (every difference is zero) and makes a Courant
// number of +-1 an exact shift (W = 0 picks the neighbour, delta is exactly
// zero); s_j = 0 gives L_j = Phi_j and CEC_j = Phi_j.
//
// When every Courant number a computation reads has one sign S, the upwind
// side is fixed: no comparison or selection, and a CEC output reads only the
// 4-point upwind stencil (Phi_{i-2..i+1} for S = +1).  Each warp votes on the
// signs of the Courant numbers it reads and takes the signed form when they
// all agree; the y sweep of the z,y,x order also has a lane-signed form (every
// line of one sign, the signs differing between lines: the upwind side is
// chosen once per line).  All forms perform the same roundings, so a cell's
// result does not depend on which form computed it (or on how the grid is
// split over CTAs).  The kernels carry mC = -C = u (-dt/dx) throughout.
//
// Organisation (both orders): persistent CTAs of 256 threads; the (column
// tile, plane) pairs of all grids are numbered and every CTA takes one
// contiguous, equal share, marching along z in each column tile.  Each plane
// bundle (the field and velocity rows a plane needs, with their periodic halo)
// is staged by the tensor-memory accelerator, one 2D box per array and row
// band, issued by one thread and counted by the slot's mbarrier; three slots
// are in flight.  One block barrier per plane in either order.
//   x,y,z: x sweep on the tile widened by the y halo (scalar runs of 8 in
//          registers, into a double-buffered shared plane); y sweep on pairs
//          of adjacent columns in packed f32x2 arithmetic, feeding per-column
//          z windows (packed pairs, 8 values per column) that output plane
//          p - 3.
//   z,y,x: z windows on pairs of columns of the tile widened by the x and y
//          halos, into a double-buffered shared plane; then each warp sweeps
//          its own 4 rows: y on column pairs (packed), x in scalar runs of 4,
//          handing over through shared memory within the warp.
// Only the window push is compiled once per window parity; the rest of the
// plane loop exists once (instruction-cache pressure measured on z,y,x).
#include <cuda.h>
#include <mutex>
#include <type_traits>

#include "sl_internal.h"

namespace sl {
namespace {

constexpr int TX = 32, TY = 32, NT = 256;

// ------------------------------------------------------- arithmetic lanes
// One lane type per form: float (one line) or float2 (two independent lines
// in one f32x2 instruction).  Every product that feeds a sum is an explicit
// fused multiply-add and every operation is rounded explicitly, so that the
// signed and general forms give bit-identical results.
// Per-line upwind side of the lane-signed form: pos (C > 0) and sg = +-1, so
// that -|mC| = mC sg.
struct LS1 {
    bool p;
    float sg;
};
struct LS2 {
    bool px, py;
    float2 sg;
};

struct L1 {
    using V = float;
    using LS = LS1;
    static __device__ __forceinline__ LS lsign(float mx) { return LS1{mx < 0.f, mx < 0.f ? 1.f : -1.f}; }
    static __device__ __forceinline__ V sel(const LS &s, V a, V b) { return s.p ? a : b; }
    static __device__ __forceinline__ V nabs(const LS &s, V m) { return __fmul_rn(m, s.sg); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ V k(float x) { return x; }
    static __device__ __forceinline__ V abs(V a) { return fabsf(a); }
    static __device__ __forceinline__ V neg(V a) { return -a; }
    // the sign of C (given as mC = -C), and a choice by it: C > 0, C < 0, C == 0
    struct Sg {
        bool p, n;
    };
    static __device__ __forceinline__ Sg sgn(V mc) { return Sg{mc < 0.f, mc > 0.f}; }
    static __device__ __forceinline__ V pick(const Sg &s, V cpos, V cneg, V czero)
    {
        return s.p ? cpos : (s.n ? cneg : czero);
    }
};

// a - b as b * (-1) + a: one rounding of the exact difference, as a subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

struct L2 {
    using V = float2;
    using LS = LS2;
    static __device__ __forceinline__ LS lsign(float mxx, float mxy)
    {
        return LS2{mxx < 0.f, mxy < 0.f, make_float2(mxx < 0.f ? 1.f : -1.f, mxy < 0.f ? 1.f : -1.f)};
    }
    static __device__ __forceinline__ V sel(const LS &s, V a, V b)
    {
        return make_float2(s.px ? a.x : b.x, s.py ? a.y : b.y);
    }
    static __device__ __forceinline__ V nabs(const LS &s, V m) { return __fmul2_rn(m, s.sg); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return sub2(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V k(float x) { return make_float2(x, x); }
    static __device__ __forceinline__ V abs(V a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
    static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
    struct Sg {
        L1::Sg x, y;
    };
    static __device__ __forceinline__ Sg sgn(V mc) { return Sg{L1::sgn(mc.x), L1::sgn(mc.y)}; }
    static __device__ __forceinline__ V pick(const Sg &s, V cpos, V cneg, V czero)
    {
        return make_float2(L1::pick(s.x, cpos.x, cneg.x, czero.x), L1::pick(s.y, cpos.y, cneg.y, czero.y));
    }
};

// three-input minimum / maximum
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Sign class of a set of mC values from their minimum and maximum: bit 0 =
// every C > 0, bit 1 = every C < 0 (neither for a zero or mixed signs).
__device__ __forceinline__ unsigned sign_bits(float mn, float mx)
{
    return (mx < 0.f ? 1u : 0u) | (mn > 0.f ? 2u : 0u);
}

// The same for pairs of lines from each line's minimum and maximum, plus bit 2
// = every line has one sign (the signs may differ from line to line).
__device__ __forceinline__ unsigned sign_bits2(float mnx, float mxx, float mny, float mxy)
{
    const bool px = mxx < 0.f, nx = mnx > 0.f, py = mxy < 0.f, ny = mny > 0.f;
    return (px && py ? 1u : 0u) | (nx && ny ? 2u : 0u) | ((px || nx) && (py || ny) ? 4u : 0u);
}

// Range of mC values: minimum and maximum (N >= 1), and whether |C| > 1.
template <int N>
__device__ __forceinline__ void mc_range(const float (&m)[N], float &mn, float &mx)
{
    mn = m[0];
    mx = m[0];
    int i = 1;
#pragma unroll
    for (; i + 1 < N; i += 2) {
        mn = min3f(mn, m[i], m[i + 1]);
        mx = max3f(mx, m[i], m[i + 1]);
    }
    if (i < N) {
        mn = fminf(mn, m[i]);
        mx = fmaxf(mx, m[i]);
    }
}

// ------------------------------------------------------------ 1D CEC runs
// Outputs o[0..R) of a line segment from p[k] = Phi at offset k - 3 (k in
// [0, R+6)) and m[k] = mC at offset k - 2 (k in [0, R+4)).  The signed forms
// read only p[1..R+4) and m[1..R+3) (offsets -2..R and -1..R).
template <class O, int R>
__device__ __forceinline__ void run_pos(const typename O::V (&p)[R + 6], const typename O::V (&m)[R + 4],
                                        typename O::V (&o)[R])
{
    using V = typename O::V;
    // every C > 0 (s = +1): L_j = Phi_{j-1} + W_j (Phi_j - Phi_{j-1}), W = 1 + mC
    V L[R + 2];   // offsets -1..R
#pragma unroll
    for (int j = 0; j < R + 2; ++j)
        L[j] = O::fma(O::add(O::k(1.f), m[j + 1]), O::sub(p[j + 2], p[j + 1]), p[j + 1]);
    V d[R + 1];   // delta at offsets -1..R-1: (Phi_j - L_j) + mC_j (L_{j+1} - L_j)
#pragma unroll
    for (int j = 0; j < R + 1; ++j) d[j] = O::fma(m[j + 1], O::sub(L[j + 1], L[j]), O::sub(p[j + 2], L[j]));
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const V w = O::fma(m[i + 2], O::k(-1.f / 6.f), O::k(1.f / 6.f));   // (1 + U)/6
        o[i] = O::fma(w, O::sub(d[i], d[i + 1]), O::fma(O::k(0.5f), d[i + 1], L[i + 1]));
    }
}

template <class O, int R>
__device__ __forceinline__ void run_neg(const typename O::V (&p)[R + 6], const typename O::V (&m)[R + 4],
                                        typename O::V (&o)[R])
{
    using V = typename O::V;
    // every C < 0 (s = -1): L_j = Phi_{j+1} - W_j (Phi_{j+1} - Phi_j), -W = mC - 1
    V L[R + 2];   // offsets -1..R
#pragma unroll
    for (int j = 0; j < R + 2; ++j)
        L[j] = O::fma(O::sub(m[j + 1], O::k(1.f)), O::sub(p[j + 3], p[j + 2]), p[j + 3]);
    V d[R + 1];   // delta at offsets 0..R: (Phi_j - L_j) + mC_j (L_j - L_{j-1})
#pragma unroll
    for (int j = 0; j < R + 1; ++j) d[j] = O::fma(m[j + 2], O::sub(L[j + 1], L[j]), O::sub(p[j + 3], L[j + 1]));
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const V w = O::fma(m[i + 2], O::k(1.f / 6.f), O::k(1.f / 6.f));    // (1 + U)/6
        o[i] = O::fma(w, O::sub(d[i + 1], d[i]), O::fma(O::k(0.5f), d[i], L[i + 1]));
    }
}

template <class O, int R>
__device__ __forceinline__ void run_any(const typename O::V (&p)[R + 6], const typename O::V (&m)[R + 4],
                                        typename O::V (&o)[R])
{
    using V = typename O::V;
    typename O::Sg sg[R + 4];   // signs at offsets -2..R+1, each compared once
#pragma unroll
    for (int j = 0; j < R + 4; ++j) sg[j] = O::sgn(m[j]);
    V L[R + 4];   // offsets -2..R+1
#pragma unroll
    for (int j = 0; j < R + 4; ++j) {
        const V nb = O::pick(sg[j], p[j], p[j + 2], p[j + 1]);           // Phi_{j - s_j}
        L[j] = O::fma(O::sub(O::k(1.f), O::abs(m[j])), O::sub(p[j + 1], nb), nb);
    }
    V d[R + 2];   // offsets -1..R: (Phi_j - L_j) - U_j (L_{j+s_j} - L_j)
#pragma unroll
    for (int j = 0; j < R + 2; ++j) {
        const V Ln = O::pick(sg[j + 1], L[j + 2], L[j], L[j + 1]);
        d[j] = O::fma(O::neg(O::abs(m[j + 1])), O::sub(Ln, L[j + 1]), O::sub(p[j + 2], L[j + 1]));
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const V w = O::fma(O::abs(m[i + 2]), O::k(1.f / 6.f), O::k(1.f / 6.f));
        const V dn = O::pick(sg[i + 2], d[i], d[i + 2], d[i + 1]);        // delta_{i - s_i}
        o[i] = O::fma(w, O::sub(dn, d[i + 1]), O::fma(O::k(0.5f), d[i + 1], L[i + 2]));
    }
}

// Every line of one sign, possibly different from line to line (ls): the
// upwind side is chosen once per line.  Reads p[1..R+5) and m[1..R+3) like the
// signed forms; delta at offset -1 is used by C > 0 lines only and delta at R
// by C < 0 lines only.
template <class O, int R>
__device__ __forceinline__ void run_lane(const typename O::LS &ls, const typename O::V (&p)[R + 6],
                                         const typename O::V (&m)[R + 4], typename O::V (&o)[R])
{
    using V = typename O::V;
    V nm[R + 2], L[R + 2], d[R + 2];   // offsets -1..R
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        nm[k] = O::nabs(ls, m[k + 1]);                                       // -U
        const V nb = O::sel(ls, p[k + 1], p[k + 3]);                          // Phi_{j - s}
        L[k] = O::fma(O::add(O::k(1.f), nm[k]), O::sub(p[k + 2], nb), nb);
    }
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        const V Ln = k == 0 ? L[1] : (k == R + 1 ? L[R] : O::sel(ls, L[k + 1], L[k - 1]));
        d[k] = O::fma(nm[k], O::sub(Ln, L[k]), O::sub(p[k + 2], L[k]));
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const V w = O::fma(nm[i + 1], O::k(-1.f / 6.f), O::k(1.f / 6.f));
        const V dn = O::sel(ls, d[i], d[i + 2]);                              // delta_{i - s}
        o[i] = O::fma(w, O::sub(dn, d[i + 1]), O::fma(O::k(0.5f), d[i + 1], L[i + 1]));
    }
}

// The form the warp's class allows (p[0], p[R+5], m[0] and m[R+3] are read by
// the general form only).
template <class O, int R>
__device__ __forceinline__ void run_cls(unsigned cls, const typename O::V (&p)[R + 6],
                                        const typename O::V (&m)[R + 4], typename O::V (&o)[R])
{
    if (cls & 1u)
        run_pos<O, R>(p, m, o);
    else if (cls & 2u)
        run_neg<O, R>(p, m, o);
    else
        run_any<O, R>(p, m, o);
}

// ------------------------------------------------------------- z windows
// Sliding window of the same sweep along z for one column (or a pair): feed
// planes in order; push<P>(Phi_p, mC_{p-1}) returns the result at plane p - 3.
// P alternates 0, 1 so that two-deep values change roles instead of moving:
// at a push of parity P, ph[P] = Phi_{p-2}, ph[P^1] = Phi_{p-1},
// L[P] = L_{p-3}, L[P^1] = L_{p-2}, m[P] = mC_{p-3}, m[P^1] = mC_{p-2},
// d[P] = delta_{p-4}, d[P^1] = delta_{p-3}.
template <class O>
struct ZWin {
    using V = typename O::V;
    V ph[2], L[2], m[2], d[2];

    __device__ __forceinline__ void init()
    {
        ph[0] = ph[1] = L[0] = L[1] = m[0] = m[1] = d[0] = d[1] = O::k(0.f);
    }

    template <int P, int S>
    __device__ __forceinline__ V push(V phi, V mn)
    {
        V Ln, dn, out;
        if constexpr (S > 0) {
            Ln = O::fma(O::add(O::k(1.f), mn), O::sub(ph[P ^ 1], ph[P]), ph[P]);         // L_{p-1}
            dn = O::fma(m[P ^ 1], O::sub(Ln, L[P ^ 1]), O::sub(ph[P], L[P ^ 1]));        // delta_{p-2}
            const V w = O::fma(m[P], O::k(-1.f / 6.f), O::k(1.f / 6.f));
            out = O::fma(w, O::sub(d[P], d[P ^ 1]), O::fma(O::k(0.5f), d[P ^ 1], L[P]));
        } else if constexpr (S < 0) {
            Ln = O::fma(O::sub(mn, O::k(1.f)), O::sub(phi, ph[P ^ 1]), phi);
            dn = O::fma(m[P ^ 1], O::sub(L[P ^ 1], L[P]), O::sub(ph[P], L[P ^ 1]));
            const V w = O::fma(m[P], O::k(1.f / 6.f), O::k(1.f / 6.f));
            out = O::fma(w, O::sub(dn, d[P ^ 1]), O::fma(O::k(0.5f), d[P ^ 1], L[P]));
        } else {
            const typename O::Sg s1 = O::sgn(mn), s2 = O::sgn(m[P ^ 1]), s3 = O::sgn(m[P]);
            const V nb = O::pick(s1, ph[P], phi, ph[P ^ 1]);
            Ln = O::fma(O::sub(O::k(1.f), O::abs(mn)), O::sub(ph[P ^ 1], nb), nb);
            const V Lnb = O::pick(s2, Ln, L[P], L[P ^ 1]);
            dn = O::fma(O::neg(O::abs(m[P ^ 1])), O::sub(Lnb, L[P ^ 1]), O::sub(ph[P], L[P ^ 1]));
            const V w = O::fma(O::abs(m[P]), O::k(1.f / 6.f), O::k(1.f / 6.f));
            const V dd = O::pick(s3, d[P], dn, d[P ^ 1]);
            out = O::fma(w, O::sub(dd, d[P ^ 1]), O::fma(O::k(0.5f), d[P ^ 1], L[P]));
        }
        ph[P] = phi;
        L[P] = Ln;
        m[P] = mn;
        d[P] = dn;
        return out;
    }
};

// Pushes one plane into N windows, sign-specialised when the whole warp agrees
// that the Courant numbers at p-1, p-2 and p-3 of all its windows share a sign.
// The two earlier planes' verdicts are carried as history bits: hist bit 0 / 1
// = all Courant numbers of the previous push > 0 / < 0, bits 2 / 3 the same
// one push earlier (zero at the start of a segment, like the windows' mC).
// lo / hi: minimum and maximum of mn over the thread's windows.
template <int P, class O, int N>
__device__ __forceinline__ void push_all(ZWin<O> (&win)[N], const typename O::V (&phi)[N],
                                         const typename O::V (&mn)[N], typename O::V (&out)[N], unsigned &hist,
                                         unsigned am, float lo, float hi)
{
    const unsigned now = sign_bits(lo, hi);
    const unsigned cls = __reduce_and_sync(am, now & hist & (hist >> 2));
    hist = ((hist & 3u) << 2) | now;
    if (cls == 1u) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = win[i].template push<P, 1>(phi[i], mn[i]);
    } else if (cls == 2u) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = win[i].template push<P, -1>(phi[i], mn[i]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = win[i].template push<P, 0>(phi[i], mn[i]);
    }
}

// One push of one pair window with its own warp vote (hist as in push_all).
template <int P>
__device__ __forceinline__ float2 push_voted(ZWin<L2> &w, float2 phi, float2 mn, unsigned &hist, float lo, float hi)
{
    const unsigned now = sign_bits(lo, hi);
    const unsigned cls = __reduce_and_sync(0xffffffffu, now & hist & (hist >> 2));
    hist = ((hist & 3u) << 2) | now;
    if (cls == 1u) return w.template push<P, 1>(phi, mn);
    if (cls == 2u) return w.template push<P, -1>(phi, mn);
    return w.template push<P, 0>(phi, mn);
}

// One push of each of a thread's z,y,x window sets, each set voting on its
// own (a warp's set k covers one compact patch of columns).
template <int P>
__device__ __forceinline__ void push_sets(ZWin<L2> (&win)[3], const float2 (&ph)[3], const float2 (&mz)[3],
                                          float2 (&res)[3], unsigned (&hist)[3], const float (&lo)[3],
                                          const float (&hi)[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) res[k] = push_voted<P>(win[k], ph[k], mz[k], hist[k], lo[k], hi[k]);
}

// ---------------------------------------------------------------- geometry
struct Seg {
    int inst, tx, ty, z0, z1;
};

// Walks a CTA's share [w, wend) of the numbered (column tile, plane) pairs;
// an instance numbers the output planes [zb, zb + nzr) of each column tile.
// Over all nz planes, the pairs of one column tile are numbered from a
// tile-dependent plane phi (periodic in z), chosen so that the share
// boundaries of every tile fall on the same planes: CTAs that start together
// then process the same z plane of neighbouring tiles at about the same time,
// and the halo rows one tile stages are still in L2 when its neighbours stage
// them.  A partial range is numbered from zb and never wraps.
__device__ __forceinline__ bool next_seg(const FastInst *tab, int ninst, int64_t &w, int64_t wend, int &hint,
                                         double share, Seg &s)
{
    if (w >= wend) return false;
    while (hint + 1 < ninst && tab[hint + 1].w0 <= w) ++hint;
    const FastInst &I = tab[hint];
    const int nzr = I.nzr;
    const int64_t local = w - I.w0;
    const int t = (int)(local / nzr);
    const int o = (int)(local - (int64_t)t * nzr);
    const int64_t tile_w = I.w0 + (int64_t)t * nzr;
    int phi = 0;
    if (nzr == I.nz) phi = (int)(fmod((double)tile_w, share) + 0.5) % I.nz;
    const int64_t tile_end = tile_w + nzr;
    const int64_t e = wend < tile_end ? wend : tile_end;
    s.inst = hint;
    s.tx = t % I.tiles_x;
    s.ty = t / I.tiles_x;
    s.z0 = I.zb + o + phi;             // in [0, 2 nz); planes are taken modulo nz
    s.z1 = s.z0 + (int)(e - w);
    w = e;
    return true;
}

__device__ __forceinline__ int wrapz(int p, int nz) { return ((p % nz) + nz) % nz; }

// ------------------------------------------------------------------ staging
// Staged rows of 44 floats run from x0 - 4 to x0 + 40 (row stride 44 floats,
// so the 16-byte blocks of runs in different rows fall on different banks).
// Rows are copied in bands [y0 - 8, y0), [y0, y0 + 32) and [y0 + 32, y0 + 32
// + b): each band lies within [0, ny) after the periodic wrap (ny is a
// multiple of 32) and starts on a 128-byte boundary in shared memory (8 rows
// of 176 bytes = 11 x 128).  At the periodic seam in x (x0 == 0 or x0 + 32 ==
// nx) the wide box reads zeros outside [0, nx); the four columns a sweep needs
// there are copied by 4-wide boxes into a side buffer (4 floats per row),
// which the sweeps read in their place.
constexpr unsigned kPolls = 1u << 20;   // bound of every mbarrier wait
constexpr int PW = 44;                  // staged row stride (floats)

__device__ __forceinline__ void bar_init(uint64_t *b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(b)) : "memory");
}

// the one arrival of a slot's phase, announcing the bytes its copies deliver
__device__ __forceinline__ void bar_arm(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *b, unsigned parity, unsigned polls)
{
    for (unsigned it = 0; it < polls; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// box (x, y, z) of a 3D tensor map into shared memory (128-byte aligned)
__device__ __forceinline__ void tma3(float *dst, const CUtensorMap *m, int x, int y, int z, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
        : "memory");
}

// Tensor maps of one instance: box shapes (width x rows) over the field
// tensor [nz][ny][nx] (F) and the velocity tensor [3 nz][ny][nx] (V).
enum {
    M_F44_8, M_F44_32, M_F44_3, M_F40_4, M_F40_32, M_F40_3, M_F4_8, M_F4_32, M_F4_3,
    M_V44_8, M_V44_32, M_V44_3, M_V40_4, M_V40_32, M_V40_3, M_V40_2, M_V4_8, M_V4_32, M_V4_3, M_V4_2,
    M_V32_2, M_V32_32, NMAPS
};
constexpr int NFMAPS = M_F4_3 + 1;   // the field's maps come first
struct FastMaps {
    CUtensorMap m[NMAPS];                          // field 0 and the velocity
    CUtensorMap fx[kFastFields - 1][NFMAPS];       // fields 1 .. nf-1
};
static_assert(sizeof(FastMaps) == kFastMapsBytes, "tensor map block size");

// Row bands of one staged array of rows [-8, 32 + nb) (nb = 2 or 3): wide
// boxes at x0 - 4 into dst, and at the seam the 4-wide side boxes at xs into
// side (4 floats per row).  m8/m32/mb are the wide maps, s8/s32/sb the narrow.
struct Band3 {
    int m8, m32, mb, s8, s32, sb, nb;
};

__device__ __forceinline__ void stage_rows(float *dst, float *side, const CUtensorMap *m, const Band3 &b, int x0,
                                           int xs, int yt, int y0, int yb, int z, bool seam, uint64_t *bar)
{
    tma3(dst, &m[b.m8], x0 - 4, yt, z, bar);
    tma3(dst + 8 * PW, &m[b.m32], x0 - 4, y0, z, bar);
    tma3(dst + 40 * PW, &m[b.mb], x0 - 4, yb, z, bar);
    if (seam) {
        tma3(side, &m[b.s8], xs, yt, z, bar);
        tma3(side + 32, &m[b.s32], xs, y0, z, bar);
        tma3(side + 160, &m[b.sb], xs, yb, z, bar);
    }
}

// A wait gave up (no copy arrived within kPolls polls): the issuing thread
// waits (bounded) for the phase of every slot it armed and that has not
// completed, so that no copy lands in shared memory after the CTA has left,
// and records the timeout.
template <int NS>
__device__ __forceinline__ void drain(uint64_t *bars, unsigned armed, unsigned par)
{
    for (int k = 0; k < NS; ++k)
        if ((armed >> k) & 1u) bar_wait(&bars[k], (par >> k) & 1u, kPolls);
}

// Offsets (floats, from the array base) of the 4 blocks [xr - 4, xr + 12) of
// one row whose column of x = -4 is at `row`: the first block comes from the
// side buffer `side` at the left seam (sl) and the last one at the right seam
// (sr); the middle blocks are at mid + 4 and mid + 8.  Fixed per segment.
struct Blocks {
    int b0, mid, b3;
    __device__ __forceinline__ void set(int row, int side, int xr, bool sl, bool sr)
    {
        mid = row + xr;
        b0 = sl && xr == 0 ? side : mid;
        b3 = sr && xr == TX - 8 ? side : mid + 12;
    }
    __device__ __forceinline__ void load(float (&v)[16], const float *base) const
    {
        const float4 q0 = *reinterpret_cast<const float4 *>(base + b0);
        const float4 q1 = *reinterpret_cast<const float4 *>(base + mid + 4);
        const float4 q2 = *reinterpret_cast<const float4 *>(base + mid + 8);
        const float4 q3 = *reinterpret_cast<const float4 *>(base + b3);
        v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
        v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
        v[8] = q2.x; v[9] = q2.y; v[10] = q2.z; v[11] = q2.w;
        v[12] = q3.x; v[13] = q3.y; v[14] = q3.z; v[15] = q3.w;
    }
};

// One x-run of 8 outputs (scalar): out[0..8) = the sweep at x in [xr, xr + 8)
// from the Phi row (pb, pbase) and the u_x row (ub, ubase).  Votes per warp on
// the signs of mC at offsets -1..8 and records |C| > 1 there in bad.
__device__ __forceinline__ void x_run(const float *pbase, const Blocks &pb, const float *ubase, const Blocks &ub,
                                      float ms, float (&o)[8], bool &bad)
{
    constexpr int R = 8;
    float blk[16], p[R + 6], m[R + 4];
    pb.load(blk, pbase);
#pragma unroll
    for (int k = 0; k < R + 6; ++k) p[k] = blk[k + 1];          // offsets -3..R+2
    ub.load(blk, ubase);
#pragma unroll
    for (int k = 0; k < R + 4; ++k) m[k] = __fmul_rn(blk[k + 2], ms);   // offsets -2..R+1
    float mv[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) mv[k] = m[k + 1];
    float mn, mx;
    mc_range(mv, mn, mx);
    bad |= (mn < -1.f) | (mx > 1.f);
    const unsigned cls = __reduce_and_sync(__activemask(), sign_bits(mn, mx));
    run_cls<L1, R>(cls, p, m, o);
}

// ============================================================ order x, y, z
namespace xyz {
constexpr int RX = 8, NXI = (TY + 6) * (TX / RX);    // 152 x-run items
// slot layout (floats; every part starts on a 128-byte boundary): Phi and u_x
// rows [-8, TY+3) at stride PW, u_y rows [-2, TY+2) and u_z rows [0, TY) at
// stride TX, and the seam side buffers of Phi and u_x (rows [-8, TY+3), 4 wide)
constexpr int O_PHI = 0, O_UX = 1920, O_UY = 3840, O_UZ = O_UY + (TY + 4) * TX, O_SP = O_UZ + TY * TX,
              O_SX = O_SP + 192, SLOT = O_SX + 192;
static_assert(43 * PW <= 1920 && 43 * 4 <= 192 && SLOT % 32 == 0, "slot layout");
constexpr int XW = 36;                                // x-swept row stride (bank-conflict-free stores)
constexpr int SZ_X = (TY + 6) * XW;                   // one x-swept plane, rows [-3, TY+3)
constexpr unsigned BYTES = 4u * (2 * 43 * PW + (TY + 4) * TX + TY * TX), BYTES_SEAM = 4u * 2 * 43 * 4;
template <int NS>
constexpr size_t smem() { return sizeof(float) * (NS * SLOT + 2 * SZ_X) + 128; }
}  // namespace xyz

// Stages the bundle of plane pz (reduced modulo nz) for the x,y,z order into
// slot sb: Phi, u_x and u_y at pz, u_z at pz - 1 (one thread).
__device__ __forceinline__ void xyz_issue(float *sb, uint64_t *b, const CUtensorMap *fm, const CUtensorMap *m,
                                          int x0, int y0, int nx, int ny, int nz, int pz, bool seam)
{
    using namespace xyz;
    const int yt = y0 - 8 < 0 ? y0 - 8 + ny : y0 - 8, yb = y0 + TY >= ny ? y0 + TY - ny : y0 + TY;
    const int yt2 = y0 - 2 < 0 ? y0 - 2 + ny : y0 - 2;
    const int pz1 = pz == 0 ? nz - 1 : pz - 1;
    const int xs = x0 == 0 ? nx - 4 : 0;
    bar_arm(b, BYTES + (seam ? BYTES_SEAM : 0u));
    const Band3 fb{M_F44_8, M_F44_32, M_F44_3, M_F4_8, M_F4_32, M_F4_3, 3};
    const Band3 vb{M_V44_8, M_V44_32, M_V44_3, M_V4_8, M_V4_32, M_V4_3, 3};
    stage_rows(sb + O_PHI, sb + O_SP, fm, fb, x0, xs, yt, y0, yb, pz, seam, b);
    stage_rows(sb + O_UX, sb + O_SX, m, vb, x0, xs, yt, y0, yb, pz, seam, b);
    tma3(sb + O_UY, &m[M_V32_2], x0, yt2, nz + pz, b);
    tma3(sb + O_UY + 2 * TX, &m[M_V32_32], x0, y0, nz + pz, b);
    tma3(sb + O_UY + 34 * TX, &m[M_V32_2], x0, yb, nz + pz, b);
    tma3(sb + O_UZ, &m[M_V32_32], x0, y0, 2 * nz + pz1, b);
}

#ifndef SL_XYZ_MINB
#define SL_XYZ_MINB 2      // CTAs per SM the x,y,z kernel is compiled for
#endif
#ifndef SL_ZYX_MINB
#define SL_ZYX_MINB 2      // CTAs per SM the z,y,x kernel is compiled for
#endif

// Dynamic shared memory rounded up to a 128-byte boundary, kept as a shared
// pointer (integer arithmetic on the address would turn every access into a
// generic one).
__device__ __forceinline__ float *smem_base()
{
    extern __shared__ float4 smem4[];
    float *const base = reinterpret_cast<float *>(smem4);
    return base + (((128u - (smem_u32(base) & 127u)) & 127u) >> 2);
}

template <bool BATCH, int NS>
__global__ void __launch_bounds__(NT, SL_XYZ_MINB)
k_cec_xyz_fast(const __grid_constant__ FastInst one, const __grid_constant__ FastMaps one_maps,
               const FastInst *__restrict__ table, int ninst, int64_t total, unsigned *status)
{
    using namespace xyz;
    float *const buf = smem_base();
    float *const sX = buf + NS * SLOT;                // two x-swept planes

    const int tid = threadIdx.x;
    const FastInst *tab = BATCH ? table : &one;
    // CTA groups of nf (one field each) share one (tile, plane) sequence
    const int nf = BATCH ? 1 : one.nf, fld = BATCH ? 0 : (int)(blockIdx.x % (unsigned)nf);
    const int64_t G = gridDim.x / nf, gb = blockIdx.x / nf;
    int64_t w = total * gb / G;
    const int64_t wend = total * (gb + 1) / G;
    bool bad = false;
    int hint = 0;
    Seg sg;
    // x phase: item tid < NXI -> row xrow (y = xrow - 3, staged row xrow + 5), run start xr
    const bool xact = tid < NXI;
    const int xrow = tid >> 2, xr = (tid & 3) * RX;
    const int xst = xrow * XW + xr;                   // its x-swept store offset
    // y/z phase: column pair cp (x = 2 cp, 2 cp + 1), rows yr, yr + 1
    const int cp = tid & 15, yr = (tid >> 4) * 2;
    const int yu = O_UY + yr * TX + 2 * cp;           // u_y of row yr - 2 (staged row y + 2)
    const int yx = yr * XW + 2 * cp;                  // x-swept row yr - 3 (row y + 3)
    const int zu = O_UZ + yr * TX + 2 * cp;           // u_z of row yr
    constexpr int ISSUER = NT - 1;                    // idle in the x phase
    __shared__ uint64_t bars[NS];
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) bar_init(&bars[k]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned par = 0;                     // bit k: parity of slot k's next completion
    unsigned armed = 0;                   // issuer: slots armed and not seen complete
    // Poll budget of a wait.  Once a wait has given up, later waits poll once
    // and the issuer stops issuing: the kernel runs to its end on stale shared
    // data (every access stays in bounds, every thread meets every barrier).
    unsigned polls = kPolls;
    bool tmo = false;
    int slot_seq = 0;                     // slot of the next staged plane

    while (next_seg(tab, ninst, w, wend, hint, (double)total / (double)G, sg)) {
        const FastInst &I = tab[sg.inst];
        const CUtensorMap *maps = BATCH ? static_cast<const FastMaps *>(I.maps)->m : one_maps.m;
        const CUtensorMap *fmaps = fld == 0 ? maps : one_maps.fx[fld - 1];
        const int x0 = sg.tx * TX, y0 = sg.ty * TY, nz = I.nz;
        const int64_t plane_n = I.plane;
        const float msx = -I.sx, msy = -I.sy, msz = -I.sz;
        const int pfirst = sg.z0 - 3, plast = sg.z1 + 2;
        const bool sl = x0 == 0, sr = x0 + TX == I.nx, seam = sl || sr;
        Blocks bp, bu;
        bp.set(O_PHI + (xrow + 5) * PW, O_SP + 4 * (xrow + 5), xr, sl, sr);
        bu.set(O_UX + (xrow + 5) * PW, O_SX + 4 * (xrow + 5), xr, sl, sr);
        float *const obase = (BATCH ? I.out : I.fout[fld]) + (int64_t)(y0 + yr) * I.nx + x0 + 2 * cp;
        const int onx = I.nx;
        auto issue = [&](int pz, int s) {
            if (tid == ISSUER && !tmo) {
                xyz_issue(buf + s * SLOT, &bars[s], fmaps, maps, x0, y0, I.nx, I.ny, nz, pz, seam);
                armed |= 1u << s;
            }
        };

        ZWin<L2> win[2];
        win[0].init();
        win[1].init();
        unsigned zhist = 0;

        // prefetch planes pfirst .. pfirst + NS - 2 (the previous segment ended
        // with a barrier, so every slot is free)
        int zw = wrapz(pfirst, nz);
        {
            int z = zw;
            for (int k = 0; k < NS - 1 && pfirst + k <= plast; ++k) {
                issue(z, (slot_seq + k) % NS);
                z = z + 1 == nz ? 0 : z + 1;
            }
        }

        // one plane: x sweep into sX[P], barrier, y sweep, z windows, store.
        // Only the window push is compiled once per parity P (the windows'
        // roles alternate); the rest of the plane exists once.
        auto plane = [&](int p, int zp) {
            const int P = (p - pfirst) & 1;
            const int s = slot_seq;
            slot_seq = s + 1 == NS ? 0 : s + 1;
            const float *sb = buf + s * SLOT;
            const bool ok = bar_wait(&bars[s], (par >> s) & 1u, polls);
            if (!ok) {
                polls = 1;
                tmo = true;
            } else if (tid == ISSUER) {
                armed &= ~(1u << s);
            }
            par ^= 1u << s;
            float *const sx = sX + P * SZ_X;
            if (xact) {
                float o[RX];
                x_run(sb, bp, sb, bu, msx, o, bad);
                float4 *dst = reinterpret_cast<float4 *>(sx + xst);
                dst[0] = make_float4(o[0], o[1], o[2], o[3]);
                dst[1] = make_float4(o[4], o[5], o[6], o[7]);
            }
            __syncthreads();
            // every thread is past the y/z phase of plane p - 1: the slot that
            // held it is refilled with plane p + NS - 1
            if (p + NS - 1 <= plast) {
                int z = zp + NS - 1;
                if (z >= nz) z -= nz;
                if (z >= nz) z -= nz;
                issue(z, s == 0 ? NS - 1 : s - 1);
            }
            // ---- y sweep: column pair cp, rows yr, yr + 1 (packed pairs)
            const float2 ms2 = make_float2(msy, msy);
            const float *uy = sb + yu;                   // u_y row yr - 2 + k at uy + k TX
            float2 m[6];                                 // mC at rows yr-2 .. yr+3
#pragma unroll
            for (int k = 1; k < 5; ++k) m[k] = __fmul2_rn(*reinterpret_cast<const float2 *>(uy + k * TX), ms2);
            float mn = min3f(m[1].x, m[1].y, m[2].x), mx = max3f(m[1].x, m[1].y, m[2].x);
            mn = min3f(mn, m[2].y, m[3].x);
            mx = max3f(mx, m[2].y, m[3].x);
            mn = min3f(mn, m[3].y, m[4].x);
            mx = max3f(mx, m[3].y, m[4].x);
            mn = fminf(mn, m[4].y);
            mx = fmaxf(mx, m[4].y);
            bad |= (mn < -1.f) | (mx > 1.f);
            const unsigned cls = __reduce_and_sync(0xffffffffu, sign_bits(mn, mx));
            const float *xs = sx + yx;                   // x-swept row yr - 3 + k at xs + k XW
            float2 pv[8], yo[2];                         // Phi at rows yr-3 .. yr+4
#pragma unroll
            for (int k = 1; k < 7; ++k) pv[k] = *reinterpret_cast<const float2 *>(xs + k * XW);
            if (cls == 1u) {
                run_pos<L2, 2>(pv, m, yo);
            } else if (cls == 2u) {
                run_neg<L2, 2>(pv, m, yo);
            } else {
                m[0] = __fmul2_rn(*reinterpret_cast<const float2 *>(uy), ms2);
                m[5] = __fmul2_rn(*reinterpret_cast<const float2 *>(uy + 5 * TX), ms2);
                pv[0] = *reinterpret_cast<const float2 *>(xs);
                pv[7] = *reinterpret_cast<const float2 *>(xs + 7 * XW);
                run_any<L2, 2>(pv, m, yo);
            }
            // ---- z windows: rows yr, yr + 1; output plane p - 3
            const float2 msz2 = make_float2(msz, msz);
            float2 mz[2], res[2];
            mz[0] = __fmul2_rn(*reinterpret_cast<const float2 *>(sb + zu), msz2);
            mz[1] = __fmul2_rn(*reinterpret_cast<const float2 *>(sb + zu + TX), msz2);
            const float zlo = min3f(mz[0].x, mz[0].y, fminf(mz[1].x, mz[1].y));
            const float zhi = max3f(mz[0].x, mz[0].y, fmaxf(mz[1].x, mz[1].y));
            bad |= (zlo < -1.f) | (zhi > 1.f);
            if (P == 0)
                push_all<0, L2, 2>(win, yo, mz, res, zhist, 0xffffffffu, zlo, zhi);
            else
                push_all<1, L2, 2>(win, yo, mz, res, zhist, 0xffffffffu, zlo, zhi);
            if (p - 3 >= sg.z0) {
                const int kw = zp >= 3 ? zp - 3 : zp - 3 + nz;
                float *dst = obase + (int64_t)kw * plane_n;
                *reinterpret_cast<float2 *>(dst) = res[0];
                *reinterpret_cast<float2 *>(dst + onx) = res[1];
            }
        };

        for (int p = pfirst; p <= plast; ++p) {
            plane(p, zw);
            zw = zw + 1 == nz ? 0 : zw + 1;
        }
        __syncthreads();   // shared buffers are reused by the next segment
    }
    if (tid == ISSUER && armed) drain<NS>(bars, armed, par);
    if (tmo) atomicOr(status, 2u);
    flag_cfl(status, bad);
}

// ============================================================ order z, y, x
namespace zyx {
constexpr int ZS = 40;                                // staged and swept row stride (x in [-4, 36))
constexpr int NZP = (TY + 6) * 20;                    // 760 z-window pairs (x in [-4, 36), y in [-3, 35))
constexpr int NZW = (NZP + NT - 1) / NT;              // 3 per thread
constexpr int RY = 4, RX = 4;                         // a warp's y and x sweeps cover rows [4 w, 4 w + 4)
// slot layout (floats, 128-byte aligned parts): Phi(p) and u_z(p-1) rows
// [-4, TY+3), u_y(p-3) rows [-4, TY+2), u_x(p-3) rows [0, TY), row r at
// (r + 4) ZS (u_x: r ZS); the seam side buffers hold row r at 32 + 4 r
// (rows from -8, so that the bands of 8, 32 and 2 or 3 rows are contiguous).
// u_z and its side buffer lie DZ after Phi and its side buffer.
constexpr int O_PHI = 0, O_SP = 1568, DZ = 1760, O_UZ = O_PHI + DZ, O_SZ = O_SP + DZ, O_UY = 3520, O_SY = 5056,
              O_UX = 5248, O_SX = 6528, SLOT = 6688;
static_assert(39 * ZS <= O_SP && O_SP + 192 <= DZ && O_SZ + 192 <= O_UY && O_UY + 38 * ZS <= O_SY &&
                  O_SY + 192 <= O_UX && O_UX + TY * ZS <= O_SX && O_SX + 160 <= SLOT && SLOT % 32 == 0,
              "slot layout");
constexpr int SZ_Z = (TY + 6) * ZS;                   // one z-swept plane, rows [-3, TY+3)
constexpr int SZ_Y = TY * ZS;                         // y-swept rows [0, TY)
constexpr unsigned BYTES = 4u * (39 + 39 + 38 + 32) * ZS, BYTES_SEAM = 4u * 4 * (43 + 43 + 42 + 32);
template <int NS>
constexpr size_t smem() { return sizeof(float) * (NS * SLOT + 2 * SZ_Z + SZ_Y) + 128; }
}  // namespace zyx

// Row zr in [0, 38) and pair column zc in [0, 20) of z-window pair q: the
// first 640 pairs form 20 blocks of 8 rows x 4 pairs (one warp's 32 lanes, so
// that a warp's sign vote covers a compact 8 x 8 patch of columns); the last
// 120 fill rows 32..37 row by row.
__device__ __forceinline__ void zpair(int q, int &zr, int &zc)
{
    if (q < 640) {
        const int b = q >> 5, l = q & 31;
        zr = 8 * (b / 5) + (l >> 2);
        zc = 4 * (b % 5) + (l & 3);
    } else {
        zr = 32 + (q - 640) / 20;
        zc = (q - 640) % 20;
    }
}

// One staged array of the z,y,x order: rows [-4, 32 + nb) in bands of 4, 32
// and nb rows (40 floats wide, from x0 - 4), and at the seam the side buffer
// rows [-8, 32 + nb) in bands of 8, 32 and nb.
__device__ __forceinline__ void stage40(float *dst, float *side, const CUtensorMap *m, int m4, int m32, int mb,
                                        int s8, int s32, int sb, int x0, int xs, int yt4, int yt8, int y0, int yb,
                                        int z, bool seam, uint64_t *bar)
{
    tma3(dst, &m[m4], x0 - 4, yt4, z, bar);
    tma3(dst + 4 * zyx::ZS, &m[m32], x0 - 4, y0, z, bar);
    tma3(dst + 36 * zyx::ZS, &m[mb], x0 - 4, yb, z, bar);
    if (seam) {
        tma3(side, &m[s8], xs, yt8, z, bar);
        tma3(side + 32, &m[s32], xs, y0, z, bar);
        tma3(side + 160, &m[sb], xs, yb, z, bar);
    }
}

// Stages the bundle of plane pz (reduced modulo nz) for the z,y,x order into
// slot sb: Phi at pz, u_z at pz - 1, u_y and u_x at pz - 3 (one thread).
__device__ __forceinline__ void zyx_issue(float *sb, uint64_t *b, const CUtensorMap *fm, const CUtensorMap *m,
                                          int x0, int y0, int nx, int ny, int nz, int pz, bool seam)
{
    using namespace zyx;
    const int yt4 = y0 - 4 < 0 ? y0 - 4 + ny : y0 - 4, yt8 = y0 - 8 < 0 ? y0 - 8 + ny : y0 - 8;
    const int yb = y0 + TY >= ny ? y0 + TY - ny : y0 + TY;
    const int pz1 = pz == 0 ? nz - 1 : pz - 1;
    const int pz3 = pz >= 3 ? pz - 3 : pz - 3 + nz;
    const int xs = x0 == 0 ? nx - 4 : 0;
    bar_arm(b, BYTES + (seam ? BYTES_SEAM : 0u));
    stage40(sb + O_PHI, sb + O_SP, fm, M_F40_4, M_F40_32, M_F40_3, M_F4_8, M_F4_32, M_F4_3, x0, xs, yt4, yt8, y0,
            yb, pz, seam, b);
    stage40(sb + O_UZ, sb + O_SZ, m, M_V40_4, M_V40_32, M_V40_3, M_V4_8, M_V4_32, M_V4_3, x0, xs, yt4, yt8, y0,
            yb, 2 * nz + pz1, seam, b);
    stage40(sb + O_UY, sb + O_SY, m, M_V40_4, M_V40_32, M_V40_2, M_V4_8, M_V4_32, M_V4_2, x0, xs, yt4, yt8, y0,
            yb, nz + pz3, seam, b);
    tma3(sb + O_UX, &m[M_V40_32], x0 - 4, y0, pz3, b);
    if (seam) tma3(sb + O_SX + 32, &m[M_V4_32], xs, y0, pz3, b);
}

// The 3 blocks [xr - 4, xr + 8) of a row for an x-run of 4 (offsets from the
// array base; the first / last block from the side buffer at the seam).
struct Blocks3 {
    int b0, mid, b2;
    __device__ __forceinline__ void set(int row, int side, int xr, bool sl, bool sr)
    {
        mid = row + xr + 4;
        b0 = sl && xr == 0 ? side : mid - 4;
        b2 = sr && xr == TX - 4 ? side : mid + 4;
    }
    __device__ __forceinline__ void load(float (&v)[12], const float *base) const
    {
        const float4 q0 = *reinterpret_cast<const float4 *>(base + b0);
        const float4 q1 = *reinterpret_cast<const float4 *>(base + mid);
        const float4 q2 = *reinterpret_cast<const float4 *>(base + b2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
        v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
        v[8] = q2.x; v[9] = q2.y; v[10] = q2.z; v[11] = q2.w;
    }
};

// One x-run of 4 outputs (scalar) at x in [xr, xr + 4); votes per warp on mC
// at offsets -1..4 and records |C| > 1 there in bad.
__device__ __forceinline__ void x_run4(const float *pbase, const Blocks3 &pb, const float *ubase, const Blocks3 &ub,
                                       float ms, float (&o)[4], bool &bad)
{
    constexpr int R = 4;
    float blk[12], p[R + 6], m[R + 4];
    pb.load(blk, pbase);
#pragma unroll
    for (int k = 0; k < R + 6; ++k) p[k] = blk[k + 1];
    ub.load(blk, ubase);
#pragma unroll
    for (int k = 0; k < R + 4; ++k) m[k] = __fmul_rn(blk[k + 2], ms);
    float mv[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) mv[k] = m[k + 1];
    float mn, mx;
    mc_range(mv, mn, mx);
    bad |= (mn < -1.f) | (mx > 1.f);
    const unsigned cls = __reduce_and_sync(0xffffffffu, sign_bits(mn, mx));
    run_cls<L1, R>(cls, p, m, o);
}

template <bool BATCH, int NS>
__global__ void __launch_bounds__(NT, SL_ZYX_MINB)
k_cec_zyx_fast(const __grid_constant__ FastInst one, const __grid_constant__ FastMaps one_maps,
               const FastInst *__restrict__ table, int ninst, int64_t total, unsigned *status)
{
    using namespace zyx;
    float *const buf = smem_base();
    float *const sZ = buf + NS * SLOT;                // two z-swept planes
    float *const sY = sZ + 2 * SZ_Z;                  // y-swept plane (each warp its own 4 rows)

    const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
    const FastInst *tab = BATCH ? table : &one;
    // CTA groups of nf (one field each) share one (tile, plane) sequence
    const int nf = BATCH ? 1 : one.nf, fld = BATCH ? 0 : (int)(blockIdx.x % (unsigned)nf);
    const int64_t G = gridDim.x / nf, gb = blockIdx.x / nf;
    int64_t w = total * gb / G;
    const int64_t wend = total * (gb + 1) / G;
    bool bad = false;
    int hint = 0;
    Seg sg;
    constexpr int ISSUER = NT - 1;                    // idle in the y phase
    __shared__ uint64_t bars[NS];
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) bar_init(&bars[k]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned par = 0, armed = 0, polls = kPolls;
    bool tmo = false;
    int slot_seq = 0;

    // z-window pairs q = tid + NT k at row zr (y = zr - 3) and pair column zc
    // (x = 2 zc - 4, 2 zc - 3); zst: z-swept store offset (-1: no pair)
    int zst[NZW];
#pragma unroll
    for (int k = 0; k < NZW; ++k) {
        int zr, zc;
        zpair(tid + NT * k, zr, zc);
        zst[k] = tid + NT * k < NZP ? zr * ZS + 2 * zc : -1;
    }
    // y items: lanes < 20 of warp wq, pair column lane (x = 2 lane - 4), rows
    // [yg, yg + 4); yo: z-swept row yg - 3 (index y + 3) and y-swept row yg
    const bool yact = lane < 20;
    const int yg = wq * RY;
    const int yo = yg * ZS + 2 * lane;
    // x items: row xrow = yg + lane / 8, run start xr
    const int xrow = yg + (lane >> 3), xr = (lane & 7) * RX;

    while (next_seg(tab, ninst, w, wend, hint, (double)total / (double)G, sg)) {
        const FastInst &I = tab[sg.inst];
        const CUtensorMap *maps = BATCH ? static_cast<const FastMaps *>(I.maps)->m : one_maps.m;
        const CUtensorMap *fmaps = fld == 0 ? maps : one_maps.fx[fld - 1];
        const int x0 = sg.tx * TX, y0 = sg.ty * TY, nz = I.nz;
        const int64_t plane_n = I.plane;
        const float msx = -I.sx, msy = -I.sy, msz = -I.sz;
        const int pfirst = sg.z0 - 3, plast = sg.z1 + 2;
        const bool sl = x0 == 0, sr = x0 + TX == I.nx, seam = sl || sr;
        const int edge = (sl ? 1 : 0) | (sr ? 2 : 0);
        auto issue = [&](int pz, int s) {
            if (tid == ISSUER && !tmo) {
                zyx_issue(buf + s * SLOT, &bars[s], fmaps, maps, x0, y0, I.nx, I.ny, nz, pz, seam);
                armed |= 1u << s;
            }
        };
        // Phi of window pair k at zop[k] (its u_z DZ further): wide row zr + 1,
        // or the side buffer row for the two pairs left / right at the seam
        int zop[NZW];
#pragma unroll
        for (int k = 0; k < NZW; ++k) {
            const int q = tid + NT * k;
            int zr, zc;
            zpair(q, zr, zc);
            const bool side = ((zc < 2 ? 1 : (zc >= 18 ? 2 : 0)) & edge) != 0;
            zop[k] = q >= NZP ? 0 : (side ? O_SP + 20 + 4 * zr + 2 * (zc & 1) : O_PHI + (zr + 1) * ZS + 2 * zc);
        }
        // u_y of the y item: row yg - 2 + k at uyo + k ust
        const bool yside = ((lane < 2 ? 1 : (lane >= 18 ? 2 : 0)) & edge) != 0;
        const int ust = yside ? 4 : ZS;
        const int uyo = yside ? O_SY + 24 + 4 * yg + 2 * (lane & 1) : O_UY + (yg + 2) * ZS + 2 * lane;
        Blocks3 bu;
        bu.set(O_UX + xrow * ZS, O_SX + 32 + 4 * xrow, xr, sl, sr);
        float *const obase = (BATCH ? I.out : I.fout[fld]) + (int64_t)(y0 + xrow) * I.nx + x0 + xr;

        ZWin<L2> win[NZW];
#pragma unroll
        for (int k = 0; k < NZW; ++k) win[k].init();
        unsigned zhist[NZW] = {0u, 0u, 0u};

        int zw = wrapz(pfirst, nz);
        {
            int z = zw;
            for (int k = 0; k < NS - 1 && pfirst + k <= plast; ++k) {
                issue(z, (slot_seq + k) % NS);
                z = z + 1 == nz ? 0 : z + 1;
            }
        }

        // one plane; only the window push is compiled once per parity P
        auto plane = [&](int p, int zp) {
            const int P = (p - pfirst) & 1;
            const int s = slot_seq;
            slot_seq = s + 1 == NS ? 0 : s + 1;
            const float *sb = buf + s * SLOT;
            const bool ok = bar_wait(&bars[s], (par >> s) & 1u, polls);
            if (!ok) {
                polls = 1;
                tmo = true;
            } else if (tid == ISSUER) {
                armed &= ~(1u << s);
            }
            par ^= 1u << s;
            float *const sz = sZ + P * SZ_Z;
            // ---- z windows on the widened columns -> sZ[P] (z-swept plane p - 3)
            {
                const float2 msz2 = make_float2(msz, msz);
                float2 ph[NZW], mz[NZW], res[NZW];
                float zlo[NZW], zhi[NZW];
#pragma unroll
                for (int k = 0; k < NZW; ++k) {
                    // a thread's last pair may not exist: it repeats the first
                    // (same signs, computed and discarded)
                    const int o = (k < NZW - 1 || zst[k] >= 0) ? zop[k] : zop[0];
                    ph[k] = *reinterpret_cast<const float2 *>(sb + o);
                    mz[k] = __fmul2_rn(*reinterpret_cast<const float2 *>(sb + o + DZ), msz2);
                    zlo[k] = fminf(mz[k].x, mz[k].y);
                    zhi[k] = fmaxf(mz[k].x, mz[k].y);
                }
                bad |= (min3f(zlo[0], zlo[1], zlo[2]) < -1.f) | (max3f(zhi[0], zhi[1], zhi[2]) > 1.f);
                if (P == 0)
                    push_sets<0>(win, ph, mz, res, zhist, zlo, zhi);
                else
                    push_sets<1>(win, ph, mz, res, zhist, zlo, zhi);
#pragma unroll
                for (int k = 0; k < NZW; ++k)
                    if (k < NZW - 1 || zst[k] >= 0) *reinterpret_cast<float2 *>(sz + zst[k]) = res[k];
            }
            __syncthreads();
            // every thread is past plane p - 1: its slot is refilled with plane p + NS - 1
            if (p + NS - 1 <= plast) {
                int z = zp + NS - 1;
                if (z >= nz) z -= nz;
                if (z >= nz) z -= nz;
                issue(z, s == 0 ? NS - 1 : s - 1);
            }
            if (p - 3 < sg.z0) return;   // warm-up planes: nothing to output (uniform over the CTA)
            // ---- y sweep (lanes < 20): pair column `lane`, rows [yg, yg + 4) -> sY
            if (yact) {
                const float2 ms2 = make_float2(msy, msy);
                const float *uy = sb + uyo;
                float2 m[RY + 4], pv[RY + 6], yv[RY];
#pragma unroll
                for (int k = 1; k < RY + 3; ++k) m[k] = __fmul2_rn(*reinterpret_cast<const float2 *>(uy + k * ust), ms2);
                // the columns x in [-3, 35) are real cells of this or a
                // neighbouring tile; x = -4 and x = 35 are computed but unused
                float mnx = m[1].x, mxx = m[1].x, mny = m[1].y, mxy = m[1].y;
#pragma unroll
                for (int k = 2; k + 1 < RY + 3; k += 2) {
                    mnx = min3f(mnx, m[k].x, m[k + 1].x);
                    mxx = max3f(mxx, m[k].x, m[k + 1].x);
                    mny = min3f(mny, m[k].y, m[k + 1].y);
                    mxy = max3f(mxy, m[k].y, m[k + 1].y);
                }
                mnx = fminf(mnx, m[RY + 2].x);
                mxx = fmaxf(mxx, m[RY + 2].x);
                mny = fminf(mny, m[RY + 2].y);
                mxy = fmaxf(mxy, m[RY + 2].y);
                bad |= (fminf(mnx, mny) < -1.f) | (fmaxf(mxx, mxy) > 1.f);
                const unsigned cls = __reduce_and_sync(0x000fffffu, sign_bits2(mnx, mxx, mny, mxy));
                const float *zs = sz + yo;               // z-swept row yg - 3 + k at zs + k ZS
#pragma unroll
                for (int k = 1; k < RY + 5; ++k) pv[k] = *reinterpret_cast<const float2 *>(zs + k * ZS);
                if (cls == 0u) {
                    m[0] = __fmul2_rn(*reinterpret_cast<const float2 *>(uy), ms2);
                    m[RY + 3] = __fmul2_rn(*reinterpret_cast<const float2 *>(uy + (RY + 3) * ust), ms2);
                    pv[0] = *reinterpret_cast<const float2 *>(zs);
                    pv[RY + 5] = *reinterpret_cast<const float2 *>(zs + (RY + 5) * ZS);
                }
                if (cls & 1u)
                    run_pos<L2, RY>(pv, m, yv);
                else if (cls & 2u)
                    run_neg<L2, RY>(pv, m, yv);
                else if (cls & 4u)
                    run_lane<L2, RY>(L2::lsign(mxx, mxy), pv, m, yv);
                else
                    run_any<L2, RY>(pv, m, yv);
#pragma unroll
                for (int i = 0; i < RY; ++i) *reinterpret_cast<float2 *>(sY + yo + i * ZS) = yv[i];
            }
            __syncwarp();
            // ---- x sweep (all lanes): row xrow, x in [xr, xr + 4) -> global plane p - 3
            float o[RX];
            Blocks3 bp;
            bp.mid = xrow * ZS + xr + 4;
            bp.b0 = bp.mid - 4;
            bp.b2 = bp.mid + 4;
            x_run4(sY, bp, sb, bu, msx, o, bad);
            const int kw = zp >= 3 ? zp - 3 : zp - 3 + nz;
            *reinterpret_cast<float4 *>(obase + (int64_t)kw * plane_n) = make_float4(o[0], o[1], o[2], o[3]);
        };

        for (int p = pfirst; p <= plast; ++p) {
            plane(p, zw);
            zw = zw + 1 == nz ? 0 : zw + 1;
        }
        __syncthreads();
    }
    if (tid == ISSUER && armed) drain<NS>(bars, armed, par);
    if (tmo) atomicOr(status, 2u);
    flag_cfl(status, bad);
}

#ifndef SL_XYZ_SLOTS
#define SL_XYZ_SLOTS 3     // staged plane slots per CTA, x,y,z order
#endif
#ifndef SL_ZYX_SLOTS
#define SL_ZYX_SLOTS 3     // staged plane slots per CTA, z,y,x order
#endif

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
        auto kern = ZYX ? k_cec_zyx_fast<BATCH, SL_ZYX_SLOTS> : k_cec_xyz_fast<BATCH, SL_XYZ_SLOTS>;
        const size_t smem = ZYX ? zyx::smem<SL_ZYX_SLOTS>() : xyz::smem<SL_XYZ_SLOTS>();
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        cached[dev] = sms * (per_sm > 0 ? per_sm : 1);
    }
    grid = cached[dev];
    return cudaSuccess;
}

template <bool ZYX, bool BATCH>
cudaError_t go_fast(const FastInst &one, const FastMaps &maps, const FastInst *tab, int ninst, int64_t total,
                    unsigned *status, int grid_req, cudaStream_t st)
{
    int grid = 0;
    cudaError_t e = prepare<ZYX, BATCH>(grid);
    if (e != cudaSuccess) return e;
    if (grid_req > 0) grid = grid_req;
    const int nf = tab ? 1 : one.nf;
    if (grid > total) grid = (int)total;
    grid = grid >= nf ? grid / nf * nf : nf;   // whole groups of nf CTAs
    if (grid > total * nf) grid = (int)(total * nf);
    if (ZYX)
        k_cec_zyx_fast<BATCH, SL_ZYX_SLOTS>
            <<<grid, NT, zyx::smem<SL_ZYX_SLOTS>(), st>>>(one, maps, tab, ninst, total, status);
    else
        k_cec_xyz_fast<BATCH, SL_XYZ_SLOTS>
            <<<grid, NT, xyz::smem<SL_XYZ_SLOTS>(), st>>>(one, maps, tab, ninst, total, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ tensor maps
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
    });
    return fn;
}

#ifndef SL_TMA_L2
#define SL_TMA_L2 CU_TENSOR_MAP_L2_PROMOTION_NONE   // measured: less DRAM traffic than 64-256 B promotion
#endif

// Encodes the box shapes of one instance: each field f.fin[i] as [nz][ny][nx]
// and the velocity f.vel as [3 nz][ny][nx] (FP32, row stride nx, plane stride
// nx ny).
cudaError_t encode_maps(FastMaps &fm, const FastInst &f)
{
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    static const int shape[NMAPS][3] = {
        {0, 44, 8}, {0, 44, 32}, {0, 44, 3}, {0, 40, 4}, {0, 40, 32}, {0, 40, 3}, {0, 4, 8}, {0, 4, 32}, {0, 4, 3},
        {1, 44, 8}, {1, 44, 32}, {1, 44, 3}, {1, 40, 4}, {1, 40, 32}, {1, 40, 3}, {1, 40, 2}, {1, 4, 8},
        {1, 4, 32}, {1, 4, 3}, {1, 4, 2}, {1, 32, 2}, {1, 32, 32}};
    for (int k = 0; k < NMAPS; ++k) {
        const bool v = shape[k][0] == 1;
        const cuuint64_t dims[3] = {(cuuint64_t)f.nx, (cuuint64_t)f.ny, (cuuint64_t)f.nz * (v ? 3 : 1)};
        const cuuint64_t strides[2] = {(cuuint64_t)f.nx * sizeof(float), (cuuint64_t)f.plane * sizeof(float)};
        const cuuint32_t box[3] = {(cuuint32_t)shape[k][1], (cuuint32_t)shape[k][2], 1u};
        const cuuint32_t step[3] = {1u, 1u, 1u};
        for (int fi = 0; fi < (v ? 1 : f.nf); ++fi) {
            void *base = const_cast<float *>(v ? f.vel : f.fin[fi]);
            CUtensorMap *dst = fi == 0 ? &fm.m[k] : &fm.fx[fi - 1][k];
            if (enc(dst, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, step,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, SL_TMA_L2,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
    }
    return cudaSuccess;
}

// Recently encoded maps of single-instance launches, keyed by buffers and sizes.
cudaError_t cached_maps(FastMaps &fm, const FastInst &f)
{
    struct Entry {
        const float *fin[kFastFields] = {};
        const float *vel = nullptr;
        int nx = 0, ny = 0, nz = 0, nf = 0;
        FastMaps maps;
    };
    static Entry cache[8];
    static int next = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    auto same = [&](const Entry &c) {
        if (c.nf != f.nf || c.vel != f.vel || c.nx != f.nx || c.ny != f.ny || c.nz != f.nz || !c.fin[0]) return false;
        for (int i = 0; i < f.nf; ++i)
            if (c.fin[i] != f.fin[i]) return false;
        return true;
    };
    for (const Entry &c : cache)
        if (same(c)) {
            fm = c.maps;
            return cudaSuccess;
        }
    Entry &c = cache[next];
    cudaError_t e = encode_maps(c.maps, f);
    if (e != cudaSuccess) {
        c.fin[0] = nullptr;
        return e;
    }
    for (int i = 0; i < kFastFields; ++i) c.fin[i] = i < f.nf ? f.fin[i] : nullptr;
    c.nf = f.nf;
    c.vel = f.vel;
    c.nx = f.nx;
    c.ny = f.ny;
    c.nz = f.nz;
    next = (next + 1) % 8;
    fm = c.maps;
    return cudaSuccess;
}

}  // namespace

cudaError_t fast_encode_maps(void *dst, const FastInst &f)
{
    return encode_maps(*static_cast<FastMaps *>(dst), f);
}

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
    f.maps = nullptr;
    f.zb = 0;
    f.nzr = f.nz;
    f.nf = 1;
    for (int i = 0; i < kFastFields; ++i) {
        f.fin[i] = i == 0 ? f.in : nullptr;
        f.fout[i] = i == 0 ? f.out : nullptr;
    }
}

cudaError_t launch_cec_fast(const FastInst &one, const FastInst *dev_table, int ninst, int64_t total, int parity,
                            unsigned *status, int grid_req, cudaStream_t st)
{
    const bool zyx_order = parity & 1;
    static FastMaps unused;   // batched launches read each instance's maps from the table
    if (dev_table)
        return zyx_order ? go_fast<true, true>(one, unused, dev_table, ninst, total, status, grid_req, st)
                         : go_fast<false, true>(one, unused, dev_table, ninst, total, status, grid_req, st);
    FastMaps maps;
    cudaError_t e = cached_maps(maps, one);
    if (e != cudaSuccess) return e;
    return zyx_order ? go_fast<true, false>(one, maps, nullptr, 1, total, status, grid_req, st)
                     : go_fast<false, false>(one, maps, nullptr, 1, total, status, grid_req, st);
}

int fast_grid(int parity)
{
    int g = 0;
    if (((parity & 1) ? prepare<true, false>(g) : prepare<false, false>(g)) != cudaSuccess) return 0;
    return g;
}

}  // namespace sl
