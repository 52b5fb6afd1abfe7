// k_wide.cu -- steps at any Courant number, with non-local interpolation: the
// corners of L_U bracket the departure point X = i - C (cell units) however far
// it is, so |C| > 1 needs no wider stencil than |C| < 1, only a gather from
// further away (Sec. 4: semi-Lagrangian schemes may exceed CFL 1 when the
// interpolation uses non-neighbouring points).
//
//   CIR, FEC, BEC  the operator compositions of Sec. 2 (eqs. intro:FEC,
//                  intro:BEC) with the unsplit multilinear L_U (eq. CIR2D and
//                  its 3D tensor product).
//   CEC            split 1D sweeps (Sec. 5 eqs. split:1-2, order x,y,z on even
//                  steps and z,y,x on odd steps) with the weights of eq.
//                  intro:CECcoefSL, 3a = 2 - 1/(U % 1), b = 1 - a, and the
//                  correction of the local scheme taken at the departure cell:
//                  with m = trunc(C), r = C - m, j = i - m, s = sgn r,
//                  CEC_i = L_U[Phi]_i + delta_j/2 + (1 + |r|)/6 (delta_{j-s} - delta_j).
//                  For constant velocity this is the local CEC at Courant
//                  number r shifted by m cells (third order); for |C| < 1 it
//                  is the local CEC.
//
// Unfused: one gather kernel per interpolation call, each with the scheme's
// pointwise combination as its epilogue, and one gather kernel for the CEC
// correction.  Intermediate fields live in a caller-owned workspace.
#include "sl_internal.h"

namespace sl {
namespace {

enum Epi { EPI_NONE = 0, EPI_FEC = 1, EPI_BEC_IN = 2, EPI_DELTA = 3 };

constexpr int kWideBlock = 128;

struct WideGeo {
    int n[3];          // cells per axis (x, y, z)
    int64_t ncell;     // n[0] n[1] n[2]
    double s[3];       // dt / dx_d: Courant number = u_d s_d
    unsigned *status;  // SL_DEV_CFL: a non-finite or huge departure point
};

// Integer part and fraction of a displacement D (cell units): D = fl + f,
// f in [0, 1).  A non-finite displacement, or one of 2^30 cells or more, is
// flagged and replaced by 0, so that every index below stays in 32 bits and
// in bounds (grid sizes are at most 2^30).
template <typename T>
__device__ __forceinline__ int floor_split(T D, T &f, bool &bad)
{
    if (!(fabs(D) < T(1073741824.0))) {
        bad = true;
        D = T(0);
    }
    const T fl = floor(D);
    f = D - fl;
    return (int)fl;
}

// v reduced into [0, n), for v = a cell index (< n <= 2^30) plus an offset of
// magnitude below 2^30, so v and v - n fit in 32 bits.  Departure points
// within one period take a compare and an add; the remainder only runs beyond.
__device__ __forceinline__ int wrapn(int v, int n)
{
    if (v < 0) {
        v += n;
        if (v >= 0) return v;
    } else if (v < n) {
        return v;
    } else {
        v -= n;
        if (v < n) return v;
    }
    const int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ int64_t cell_at(const WideGeo &g, int x, int y, int z)
{
    return ((int64_t)z * g.n[1] + y) * g.n[0] + x;
}

// Each thread takes the cells (x, y0 + k, z), k < kWideRows: a warp's loads of
// one k are coalesced along x, and the rows' loads are issued together (the
// velocity of all rows, then all corners), so that several independent gathers
// are in flight per thread.
constexpr int kWideRows = 4;

// out = epilogue(L_{dir U}[src]) at every cell.  AX < 0: the multilinear
// operator on NDIM axes; AX >= 0: the 1D operator along that axis.  dir = +1
// is L_U (departure i - C), dir = -1 is L_{-U} (departure i + C, -u at its own
// arrival cell).
template <typename T, int NDIM, int AX, int EPI>
__global__ void __launch_bounds__(kWideBlock)
k_wide_interp(T *__restrict__ out, const T *__restrict__ src, const T *__restrict__ vel, const T *__restrict__ aux0,
              const T *__restrict__ aux1, WideGeo g, int dir)
{
    constexpr int R = kWideRows;
    const int x = blockIdx.x * kWideBlock + threadIdx.x, y0 = blockIdx.y * R, z = blockIdx.z;
    bool bad = false;
    bool on[R];
    int64_t cell[R];
    T C[R][3];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        on[k] = x < g.n[0] && y0 + k < g.n[1];
        cell[k] = on[k] ? cell_at(g, x, y0 + k, z) : 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const bool moves = AX < 0 ? d < NDIM : d == AX;
            C[k][d] = moves && on[k] ? vel[(int64_t)d * g.ncell + cell[k]] * T(g.s[d]) : T(0);
        }
    }
    T val[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int pos[3] = {x, y0 + k, z};
        int b0[3] = {pos[0], pos[1], pos[2]}, b1[3] = {pos[0], pos[1], pos[2]};
        T f[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const bool moves = AX < 0 ? d < NDIM : d == AX;
            if (moves) {
                const int fl = floor_split<T>(T(-dir) * C[k][d], f[d], bad);
                b0[d] = wrapn(pos[d] + fl, g.n[d]);
                b1[d] = b0[d] + 1 == g.n[d] ? 0 : b0[d] + 1;
            }
        }
        val[k] = T(0);
        if (!on[k]) continue;
        if constexpr (AX >= 0) {
            int q0[3] = {pos[0], pos[1], pos[2]}, q1[3] = {pos[0], pos[1], pos[2]};
            q0[AX] = b0[AX];
            q1[AX] = b1[AX];
            const T a = src[cell_at(g, q0[0], q0[1], q0[2])], b = src[cell_at(g, q1[0], q1[1], q1[2])];
            val[k] = a + f[AX] * (b - a);
        } else {
            // corners weighted by prod_d (1 - f_d | f_d), lerped along x, then y, then z,
            // each lerp as a + f (b - a) so that a constant field stays exact
            T c[2];
#pragma unroll
            for (int h = 0; h < (NDIM == 3 ? 2 : 1); ++h) {
                const int zz = NDIM == 3 ? (h ? b1[2] : b0[2]) : z;
                const T a00 = src[cell_at(g, b0[0], b0[1], zz)], a10 = src[cell_at(g, b1[0], b0[1], zz)];
                const T a01 = src[cell_at(g, b0[0], b1[1], zz)], a11 = src[cell_at(g, b1[0], b1[1], zz)];
                const T e0 = a00 + f[0] * (a10 - a00);
                const T e1 = a01 + f[0] * (a11 - a01);
                c[h] = e0 + f[1] * (e1 - e0);
            }
            val[k] = NDIM == 3 ? c[0] + f[2] * (c[1] - c[0]) : c[0];
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        if (!on[k]) continue;
        const int64_t i = cell[k];
        const T v = val[k];
        if constexpr (EPI == EPI_NONE) out[i] = v;
        if constexpr (EPI == EPI_FEC) out[i] = aux1[i] + (aux0[i] - v) * T(0.5);
        if constexpr (EPI == EPI_BEC_IN) out[i] = aux0[i] + (aux0[i] - v) * T(0.5);
        if constexpr (EPI == EPI_DELTA) out[i] = aux0[i] - v;
    }
    flag_cfl(g.status, bad);
}

// The CEC sweep's output along AX from L_U[Phi] (lphi) and delta = Phi - Phi_bar:
// CEC_i = lphi_i + delta_j/2 + (1 + |r|)/6 (delta_{j-s} - delta_j), m = trunc(C_i),
// r = C_i - m, j = i - m, s = sgn r.
template <typename T, int AX>
__global__ void __launch_bounds__(kWideBlock)
k_wide_cec(T *__restrict__ out, const T *__restrict__ lphi, const T *__restrict__ delta, const T *__restrict__ vel,
           WideGeo g)
{
    constexpr int R = kWideRows;
    const int x = blockIdx.x * kWideBlock + threadIdx.x, y0 = blockIdx.y * R, z = blockIdx.z;
    bool bad = false;
    bool on[R];
    int64_t cell[R];
    T C[R], L[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        on[k] = x < g.n[0] && y0 + k < g.n[1];
        cell[k] = on[k] ? cell_at(g, x, y0 + k, z) : 0;
        C[k] = on[k] ? vel[(int64_t)AX * g.ncell + cell[k]] * T(g.s[AX]) : T(0);
        L[k] = on[k] ? lphi[cell[k]] : T(0);
    }
    T dj[R], du[R], r[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        T c = C[k];
        if (!(fabs(c) < T(1073741824.0))) {
            bad = true;
            c = T(0);
        }
        const T m = trunc(c);
        r[k] = c - m;
        const int s = (r[k] > T(0)) - (r[k] < T(0));
        const int pos[3] = {x, y0 + k, z};
        int qj[3] = {pos[0], pos[1], pos[2]}, qu[3] = {pos[0], pos[1], pos[2]};
        qj[AX] = wrapn(pos[AX] - (int)m, g.n[AX]);
        qu[AX] = wrapn(pos[AX] - (int)m - s, g.n[AX]);
        dj[k] = on[k] ? delta[cell_at(g, qj[0], qj[1], qj[2])] : T(0);
        du[k] = on[k] ? delta[cell_at(g, qu[0], qu[1], qu[2])] : T(0);
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (on[k]) out[cell[k]] = L[k] + dj[k] * T(0.5) + (T(1) + fabs(r[k])) * T(1.0 / 6.0) * (du[k] - dj[k]);
    flag_cfl(g.status, bad);
}

dim3 wide_grid(const WideGeo &g)
{
    return dim3((g.n[0] + kWideBlock - 1) / kWideBlock, (g.n[1] + kWideRows - 1) / kWideRows, g.n[2]);
}

// --------------------------------------------- fused sweep on whole lines
// A CEC sweep along AX only reads the line it works on: L_U[Phi] at a cell
// gathers Phi near the cell's departure point, delta gathers L_U[Phi] near the
// reversed departure point, and the correction gathers delta near the
// departure cell.  So a CTA holds W whole lines in shared memory (Phi, then
// delta in its place; the Courant numbers; L_U[Phi]) and writes the sweep's
// output: one read of Phi and u_AX and one write per cell (12 B in FP32), in
// place of the 44 B of the three gathers above.  Lines along x are rows
// (contiguous); lines along y or z are W adjacent x columns, so that every
// load and store of a warp is coalesced along x.
constexpr int kSweepThreads = 256;
// 24 KB per CTA (8 lines of 256 cells in FP32): measured fastest among 12,
// 24, 36, 48 and 96 KB, several CTAs per SM hiding each other's barriers
constexpr size_t kSweepSmem = 24 * 1024;

template <typename T, int AX, int W>
__global__ void __launch_bounds__(kSweepThreads)
k_wide_sweep(T *__restrict__ out, const T *__restrict__ src, const T *__restrict__ vel, WideGeo g, int64_t nlines)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = g.n[AX];
    T *S = reinterpret_cast<T *>(smem_raw);   // Phi, then delta
    T *V = S + (size_t)W * n;                 // Courant numbers along AX
    T *Lb = V + (size_t)W * n;                // L_U[Phi]
    const int tid = threadIdx.x;
    const T sc = T(g.s[AX]);
    bool bad = false;
    // first element of line w = 0, and the stride along the line
    int64_t base, stride, row0 = 0;
    if constexpr (AX == 0) {
        row0 = (int64_t)blockIdx.x * W;
        base = row0 * g.n[0];
        stride = 1;
    } else {
        const int xt = g.n[0] / W;
        const int64_t q = blockIdx.x / xt;                         // z (AX = 1) or y (AX = 2)
        const int x0 = (int)(blockIdx.x - q * xt) * W;
        base = (AX == 1 ? q * g.n[0] * (int64_t)g.n[1] : q * g.n[0]) + x0;
        stride = AX == 1 ? g.n[0] : (int64_t)g.n[0] * g.n[1];
    }
    auto sidx = [&](int w, int i) { return AX == 0 ? w * n + i : i * W + w; };
    auto gidx = [&](int w, int i) { return AX == 0 ? base + (int64_t)w * n + i : base + (int64_t)i * stride + w; };
    // rows of a power-of-two length take one flat loop with shifts
    const int lg = (n & (n - 1)) == 0 ? __ffs(n) - 1 : -1;
    const int rows = AX == 0 ? (int)min((int64_t)W, nlines - row0) : W;
    auto each = [&](auto f) {
        if constexpr (AX == 0) {
            if (lg >= 0) {
                for (int e = tid; e < (rows << lg); e += kSweepThreads) f(e >> lg, e & (n - 1));
            } else {
                for (int w = 0; w < rows; ++w)
                    for (int i = tid; i < n; i += kSweepThreads) f(w, i);
            }
        } else {
            for (int e = tid; e < W * n; e += kSweepThreads) f(e % W, e / W);
        }
    };
    // staging: each thread issues the loads of B elements before storing any,
    // so that B global loads of Phi and B of u_AX are in flight at once (4
    // measured fastest of 1, 2, 4, 8 and 16: more costs registers and CTAs)
    constexpr int B = 4;
    auto stage = [&](const int (&w)[B], const int (&i)[B], const bool (&ok)[B]) {
        T a[B], c[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int64_t q = ok[k] ? gidx(w[k], i[k]) : 0;
            a[k] = ok[k] ? src[q] : T(0);
            c[k] = ok[k] ? vel[(int64_t)AX * g.ncell + q] * sc : T(0);
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (!ok[k]) continue;
            if (!(fabs(c[k]) < T(1073741824.0))) {
                bad = true;
                c[k] = T(0);
            }
            S[sidx(w[k], i[k])] = a[k];
            V[sidx(w[k], i[k])] = c[k];
        }
    };
    if constexpr (AX == 0) {
        for (int w0 = 0; w0 < W; w0 += B)
            for (int i0 = tid; i0 < n; i0 += kSweepThreads) {
                int w[B], i[B];
                bool ok[B];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    w[k] = w0 + k;
                    i[k] = i0;
                    ok[k] = w[k] < W && row0 + w[k] < nlines;
                }
                stage(w, i, ok);
            }
    } else {
        for (int e0 = tid; e0 < W * n; e0 += kSweepThreads * B) {
            int w[B], i[B];
            bool ok[B];
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const int e = e0 + k * kSweepThreads;
                ok[k] = e < W * n;
                w[k] = e % W;
                i[k] = e / W;
            }
            stage(w, i, ok);
        }
    }
    __syncthreads();
    each([&](int w, int i) {                                          // L_U[Phi]
        T f;
        bool unused = false;
        const int b0 = wrapn(i + floor_split<T>(-V[sidx(w, i)], f, unused), n);
        const int b1 = b0 + 1 == n ? 0 : b0 + 1;
        const T a = S[sidx(w, b0)], b = S[sidx(w, b1)];
        Lb[sidx(w, i)] = a + f * (b - a);
    });
    __syncthreads();
    each([&](int w, int i) {                                          // delta = Phi - L_{-U}[L_U[Phi]]
        T f;
        bool unused = false;
        const int b0 = wrapn(i + floor_split<T>(V[sidx(w, i)], f, unused), n);
        const int b1 = b0 + 1 == n ? 0 : b0 + 1;
        const T a = Lb[sidx(w, b0)], b = Lb[sidx(w, b1)];
        S[sidx(w, i)] = S[sidx(w, i)] - (a + f * (b - a));
    });
    __syncthreads();
    each([&](int w, int i) {                                          // departure-cell correction
        const T c = V[sidx(w, i)], m = trunc(c), r = c - m;
        const int sg = (r > T(0)) - (r < T(0));
        const int j = wrapn(i - (int)m, n), ju = wrapn(i - (int)m - sg, n);
        const T dj = S[sidx(w, j)], du = S[sidx(w, ju)];
        out[gidx(w, i)] = Lb[sidx(w, i)] + dj * T(0.5) + (T(1) + fabs(r)) * T(1.0 / 6.0) * (du - dj);
    });
    flag_cfl(g.status, bad);
}

template <typename T, int AX, int W>
cudaError_t go_sweep(T *dst, const T *src, const T *vel, const WideGeo &g, cudaStream_t st)
{
    static int ready[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = 3 * sizeof(T) * (size_t)W * g.n[AX];
    if (!ready[dev]) {
        e = cudaFuncSetAttribute(k_wide_sweep<T, AX, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmem);
        if (e != cudaSuccess) return e;
        ready[dev] = 1;
    }
    const int64_t nlines = AX == 0 ? (int64_t)g.n[1] * g.n[2] : 0;
    const int64_t blocks = AX == 0 ? (nlines + W - 1) / W : (int64_t)(g.n[0] / W) * (AX == 1 ? g.n[2] : g.n[1]);
    k_wide_sweep<T, AX, W><<<(unsigned)blocks, kSweepThreads, smem, st>>>(dst, src, vel, g, nlines);
    return cudaGetLastError();
}

// The fused sweep with the most lines per CTA that fit kSweepSmem (W | nx for
// lines along y and z); false when not even one line fits.
template <typename T, int AX>
bool sweep_fused(T *dst, const T *src, const T *vel, const WideGeo &g, cudaStream_t st, cudaError_t &e)
{
    const size_t line = 3 * sizeof(T) * (size_t)g.n[AX];
    for (int W = 32; W >= 1; W /= 2) {
        if (W * line > kSweepSmem || (AX != 0 && g.n[0] % W != 0)) continue;
        const int64_t blocks = AX == 0 ? ((int64_t)g.n[1] * g.n[2] + W - 1) / W
                                       : (int64_t)(g.n[0] / W) * (AX == 1 ? g.n[2] : g.n[1]);
        if (blocks > 0x7fffffff) return false;
        switch (W) {
        case 32: e = go_sweep<T, AX, 32>(dst, src, vel, g, st); break;
        case 16: e = go_sweep<T, AX, 16>(dst, src, vel, g, st); break;
        case 8: e = go_sweep<T, AX, 8>(dst, src, vel, g, st); break;
        case 4: e = go_sweep<T, AX, 4>(dst, src, vel, g, st); break;
        case 2: e = go_sweep<T, AX, 2>(dst, src, vel, g, st); break;
        default: e = go_sweep<T, AX, 1>(dst, src, vel, g, st); break;
        }
        return true;
    }
    return false;
}

template <typename T, int NDIM, int AX, int EPI>
cudaError_t interp(T *out, const T *src, const T *vel, const T *aux0, const T *aux1, const WideGeo &g, int dir,
                   cudaStream_t st)
{
    k_wide_interp<T, NDIM, AX, EPI><<<wide_grid(g), kWideBlock, 0, st>>>(out, src, vel, aux0, aux1, g, dir);
    return cudaGetLastError();
}

// One CEC sweep: fused on whole lines when they fit in shared memory, else the
// three gathers through the workspace fields w0 (L_U[Phi]) and w1 (delta).
template <typename T, int AX>
cudaError_t sweep(T *dst, const T *src, const T *vel, T *w0, T *w1, const WideGeo &g, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (sweep_fused<T, AX>(dst, src, vel, g, st, e)) return e;
    e = interp<T, 3, AX, EPI_NONE>(w0, src, vel, nullptr, nullptr, g, +1, st);                        // L_U[Phi]
    if (e == cudaSuccess) e = interp<T, 3, AX, EPI_DELTA>(w1, w0, vel, src, nullptr, g, -1, st);       // delta
    if (e != cudaSuccess) return e;
    k_wide_cec<T, AX><<<wide_grid(g), kWideBlock, 0, st>>>(dst, w0, w1, vel, g);
    return cudaGetLastError();
}

template <typename T, int NDIM>
cudaError_t unsplit(int scheme, T *out, const T *in, const T *vel, T *w0, T *w1, const WideGeo &g, cudaStream_t st)
{
    if (scheme == 0) return interp<T, NDIM, -1, EPI_NONE>(out, in, vel, nullptr, nullptr, g, +1, st);
    cudaError_t e = interp<T, NDIM, -1, EPI_NONE>(w0, in, vel, nullptr, nullptr, g, +1, st);           // L_U[Phi]
    if (e != cudaSuccess) return e;
    if (scheme == 1) return interp<T, NDIM, -1, EPI_FEC>(out, w0, vel, in, w0, g, -1, st);
    e = interp<T, NDIM, -1, EPI_BEC_IN>(w1, w0, vel, in, nullptr, g, -1, st);                           // Phi + delta/2
    if (e != cudaSuccess) return e;
    return interp<T, NDIM, -1, EPI_NONE>(out, w1, vel, nullptr, nullptr, g, +1, st);
}

template <typename T>
cudaError_t run(int scheme, const void *in_v, void *out_v, const void *vel_v, int ndim, const WideGeo &g, int parity,
                void *work, cudaStream_t st)
{
    const T *in = static_cast<const T *>(in_v), *vel = static_cast<const T *>(vel_v);
    T *out = static_cast<T *>(out_v);
    const size_t fb = wide_field_bytes(g.ncell, sizeof(T));
    // the scheme's workspace fields (wide_fields of them; none for CIR, whose
    // workspace may be NULL)
    T *w[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < wide_fields(scheme, ndim); ++k) w[k] = reinterpret_cast<T *>(static_cast<char *>(work) + k * fb);
    if (scheme != 3) return ndim == 3 ? unsplit<T, 3>(scheme, out, in, vel, w[0], w[1], g, st)
                                      : unsplit<T, 2>(scheme, out, in, vel, w[0], w[1], g, st);
    // split CEC: in -> w2 (-> w3) -> out
    const T *src = in;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < ndim && e == cudaSuccess; ++k) {
        const int axis = (parity & 1) ? ndim - 1 - k : k;
        T *dst = k == ndim - 1 ? out : w[2 + (k & 1)];
        e = axis == 0 ? sweep<T, 0>(dst, src, vel, w[0], w[1], g, st)
                      : (axis == 1 ? sweep<T, 1>(dst, src, vel, w[0], w[1], g, st)
                                   : sweep<T, 2>(dst, src, vel, w[0], w[1], g, st));
        src = dst;
    }
    return e;
}

}  // namespace

size_t wide_field_bytes(int64_t ncell, size_t elem) { return ((size_t)ncell * elem + 255) & ~(size_t)255; }

int wide_fields(int scheme, int ndim)
{
    switch (scheme) {
    case 0: return 0;
    case 1: return 1;
    case 2: return 2;
    default: return ndim == 3 ? 4 : 3;
    }
}

cudaError_t launch_wide(int dtype, int scheme, const void *in, void *out, const void *vel, int ndim,
                        const int64_t dims[3], const double s[3], int parity, void *work, unsigned *status,
                        cudaStream_t st)
{
    WideGeo g;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = (int)dims[d];
        g.s[d] = d < ndim ? s[d] : 0.0;
    }
    g.ncell = dims[0] * dims[1] * dims[2];
    g.status = status;
    return dtype == 1 ? run<double>(scheme, in, out, vel, ndim, g, parity, work, st)
                      : run<float>(scheme, in, out, vel, ndim, g, parity, work, st);
}

}  // namespace sl
