// k_split.cu -- fused directionally split third-order step (SL_CEC).
//
// One kernel performs the three 1D CEC sweeps of a time step (Sec. 2 last
// paragraph, Sec. 5 eqs. split:1-2; per-axis coefficients of eq.
// intro:CECcoef) with a single HBM read of Phi and u and a single write of
// the result.  Each 1D sweep reads Phi three cells and u two cells away from
// its output, so the staged plane tiles carry a halo of 3 (Phi) and 2 (u).
//
//  - order x,y,z (even step): per plane, the x sweep runs on the staged tile
//    (rows widened by the y halo) into shared memory, the y sweep reads it and
//    feeds, per column, a register window that performs the z sweep three
//    planes behind the plane being loaded.
//  - order z,y,x (odd step): the z sweep runs first in register windows over
//    the halo-widened columns and writes each finished plane to shared
//    memory, where the y and x sweeps follow.
//
// Loads are 16-byte cp.async copies of whole aligned rows (x staged over
// [-4, TX+4)), double-buffered one plane ahead; periodic wrap-around is folded
// into per-thread source offsets computed once per work item.
#include "sl_internal.h"

namespace sl {
namespace {

template <typename T, int TX, int TY>
struct Shape {
    static constexpr int V = 16 / sizeof(T);             // elements per 16-byte copy
    static constexpr int HW = TX + 8;                    // staged x in [-4, TX+4)
    static constexpr int PW = HW + (sizeof(T) == 4 ? 4 : 2);   // row stride
    static constexpr int PH = TY + 6;                    // staged y in [-3, TY+3)
};

// N consecutive elements from 16-byte aligned shared memory.
template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T *src, T (&dst)[N])
{
    if constexpr (sizeof(T) == 4) {
        static_assert(N % 4 == 0, "");
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(src)[i];
            dst[4 * i] = v.x; dst[4 * i + 1] = v.y; dst[4 * i + 2] = v.z; dst[4 * i + 3] = v.w;
        }
    } else {
        static_assert(N % 2 == 0, "");
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 v = reinterpret_cast<const double2 *>(src)[i];
            dst[2 * i] = v.x; dst[2 * i + 1] = v.y;
        }
    }
}

template <typename T, int N>
__device__ __forceinline__ void sts_vec(T *dst, const T (&src)[N])
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4 *>(dst)[i] = make_float4(src[4 * i], src[4 * i + 1], src[4 * i + 2], src[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < N / 2; ++i)
            reinterpret_cast<double2 *>(dst)[i] = make_double2(src[2 * i], src[2 * i + 1]);
    }
}

// Stages a rectangle of rows [r0, r0+NR) (relative to the tile origin) and
// staged columns [-4, -4 + NC) of one plane into shared memory with row
// stride LD.  Vector path: NC multiple of V and nx multiple of V, so every
// 16-byte copy lies inside one period.  Offsets are per-thread and
// precomputed per work item.
template <typename T, int NT, int NR, int NC, int LD, bool VEC>
struct Stager {
    static constexpr int V = 16 / sizeof(T);
    static constexpr int CPR = NC / V;
    static constexpr int N = NR * CPR;
    static constexpr int K = VEC ? (N + NT - 1) / NT : 1;
    int off[K];

    __device__ __forceinline__ void setup(int tid, int x0, int y0, int r0, int c0, int nx, int ny)
    {
        if constexpr (VEC) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int idx = tid + k * NT;
                if (idx < N) {
                    const int row = idx / CPR, cc = idx - (idx / CPR) * CPR;
                    const int gy = wrapi(y0 + r0 + row, ny);
                    const int gx = wrapi(x0 + c0 + cc * V, nx);
                    off[k] = gy * nx + gx;
                } else {
                    off[k] = -1;
                }
            }
        }
    }

    __device__ __forceinline__ void issue(int tid, T *dst, const T *src, int x0, int y0, int r0, int c0, int nx,
                                          int ny) const
    {
        if constexpr (VEC) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int idx = tid + k * NT;
                if (off[k] >= 0) {
                    const int row = idx / CPR, cc = idx - (idx / CPR) * CPR;
                    cp_async16(dst + row * LD + cc * V, src + off[k]);
                }
            }
        } else {
            for (int idx = tid; idx < NR * NC; idx += NT) {
                const int row = idx / NC, col = idx - (idx / NC) * NC;
                const int gy = wrapi(y0 + r0 + row, ny);
                const int gx = wrapi(x0 + c0 + col, nx);
                cp_async_elem(dst + row * LD + col, src + (int64_t)gy * nx + gx);
            }
        }
    }
};

__device__ __forceinline__ void decode_item(int item, const Geo &g, int TX, int TY, int &x0, int &y0, int &z0,
                                            int &z1)
{
    const int tx = item % g.tiles_x;
    const int rest = item / g.tiles_x;
    const int ty = rest % g.tiles_y;
    const int cz = rest / g.tiles_y;
    x0 = tx * TX;
    y0 = ty * TY;
    z0 = cz * g.tz;
    z1 = min(z0 + g.tz, g.nz);
}

// ============================================================ order x, y, z
template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
struct XYZ {
    using S = Shape<T, TX, TY>;
    static constexpr int RX = 8, RY = 4;
    static constexpr int NT = TX * (TY / RY);
    static constexpr int NB = 2;
    static constexpr int SZ_PHI = S::PH * S::PW;
    static constexpr int SZ_CY = (TY + 4) * TX;
    static constexpr int SZ_CZ = HAS_Z ? TY * TX : 0;
    static constexpr int SZ_S1 = S::PH * TX;
    static constexpr size_t smem() { return sizeof(T) * (size_t)(NB * (2 * SZ_PHI + SZ_CY + SZ_CZ) + SZ_S1); }
};

template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
__device__ __forceinline__ void xyz_item(const Geo &g, int item, const T *__restrict__ in, T *__restrict__ out,
                                         const T *__restrict__ vel, unsigned char *smem_raw, bool &bad)
{
    using K = XYZ<T, D, TX, TY, HAS_Z, VEC>;
    using S = typename K::S;
    constexpr int RX = K::RX, RY = K::RY, NT = K::NT, NB = K::NB;
    T *sPhi = reinterpret_cast<T *>(smem_raw);
    T *sCx = sPhi + NB * K::SZ_PHI;
    T *sCy = sCx + NB * K::SZ_PHI;
    T *sCz = sCy + NB * K::SZ_CY;
    T *sS1 = sCz + NB * K::SZ_CZ;

    const int tid = threadIdx.x;
    const D sx = D(g.sx), sy = D(g.sy), sz = D(g.sz);

    Stager<T, NT, S::PH, S::HW, S::PW, VEC> stPhi;     // Phi and u_x: rows [-3,TY+3), cols [-4,TX+4)
    Stager<T, NT, TY + 4, TX, TX, VEC> stCy;           // u_y: rows [-2,TY+2), cols [0,TX)
    Stager<T, NT, TY, TX, TX, VEC> stCz;               // u_z: rows [0,TY), cols [0,TX)

    int x0, y0, z0, z1;
    decode_item(item, g, TX, TY, x0, y0, z0, z1);
    stPhi.setup(tid, x0, y0, -3, -4, g.nx, g.ny);
    stCy.setup(tid, x0, y0, -2, 0, g.nx, g.ny);
    if constexpr (HAS_Z) stCz.setup(tid, x0, y0, 0, 0, g.nx, g.ny);

    const int pfirst = HAS_Z ? z0 - 3 : 0;
    const int plast = HAS_Z ? z1 + 2 : 0;
    auto issue = [&](int p, int slot) {
        const int64_t base = (int64_t)wrapi(p, g.nz) * g.plane;
        stPhi.issue(tid, sPhi + slot * K::SZ_PHI, in + base, x0, y0, -3, -4, g.nx, g.ny);
        stPhi.issue(tid, sCx + slot * K::SZ_PHI, vel + base, x0, y0, -3, -4, g.nx, g.ny);
        stCy.issue(tid, sCy + slot * K::SZ_CY, vel + g.ncell + base, x0, y0, -2, 0, g.nx, g.ny);
        if constexpr (HAS_Z) {
            const int64_t bz = (int64_t)wrapi(p - 1, g.nz) * g.plane;
            stCz.issue(tid, sCz + slot * K::SZ_CZ, vel + 2 * g.ncell + bz, x0, y0, 0, 0, g.nx, g.ny);
        }
        cp_async_commit();
    };

    const int cx = tid % TX, yr = (tid / TX) * RY;     // y-sweep run / z columns of this thread
    ZWin<T, D> win[RY];
#pragma unroll
    for (int i = 0; i < RY; ++i) win[i].init();

    issue(pfirst, 0);
    for (int p = pfirst; p <= plast; ++p) {
        const int slot = (p - pfirst) & 1;
        cp_async_wait_all();
        __syncthreads();
        if (p < plast) issue(p + 1, slot ^ 1);

        // ---- x sweep: rows [-3, TY+3) x cols [0, TX) -> sS1
        const T *phiP = sPhi + slot * K::SZ_PHI;
        const T *cxP = sCx + slot * K::SZ_PHI;
        constexpr int XR = TX / RX;
        for (int r = tid; r < S::PH * XR; r += NT) {
            const int row = r / XR, xr = (r - (r / XR) * XR) * RX;
            T blk[RX + 8];
            lds_vec<T, RX + 8>(phiP + row * S::PW + xr, blk);
            T pv[RX + 6];
#pragma unroll
            for (int k = 0; k < RX + 6; ++k) pv[k] = blk[k + 1];
            lds_vec<T, RX + 8>(cxP + row * S::PW + xr, blk);
            D cv[RX + 4];
#pragma unroll
            for (int k = 0; k < RX + 4; ++k) cv[k] = D(blk[k + 2]) * sx;
#pragma unroll
            for (int k = 2; k < RX + 2; ++k) bad |= fabs(cv[k]) > D(1);
            T o[RX];
            cec_line<T, D, RX>(pv, cv, o);
            sts_vec<T, RX>(sS1 + row * TX + xr, o);
        }
        __syncthreads();

        // ---- y sweep of this thread's run, then z windows
        const T *cyP = sCy + slot * K::SZ_CY;
        T pv[RY + 6];
#pragma unroll
        for (int k = 0; k < RY + 6; ++k) pv[k] = sS1[(yr + k) * TX + cx];
        D cv[RY + 4];
#pragma unroll
        for (int k = 0; k < RY + 4; ++k) cv[k] = D(cyP[(yr + k) * TX + cx]) * sy;
#pragma unroll
        for (int k = 2; k < RY + 2; ++k) bad |= fabs(cv[k]) > D(1);
        T o[RY];
        cec_line<T, D, RY>(pv, cv, o);
        const int gx = x0 + cx;
        if constexpr (HAS_Z) {
            const T *czP = sCz + slot * K::SZ_CZ;
            const int kz = p - 3;
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const D c = D(czP[(yr + i) * TX + cx]) * sz;
                bad |= fabs(c) > D(1);
                const T v = win[i].push(o[i], c);
                const int gy = y0 + yr + i;
                if (kz >= z0 && gx < g.nx && gy < g.ny) out[(int64_t)kz * g.plane + (int64_t)gy * g.nx + gx] = v;
            }
        } else {
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int gy = y0 + yr + i;
                if (gx < g.nx && gy < g.ny) out[(int64_t)gy * g.nx + gx] = o[i];
            }
        }
    }
    __syncthreads();   // shared buffers are reused by the next item
}

template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
__global__ void __launch_bounds__(XYZ<T, D, TX, TY, HAS_Z, VEC>::NT)
k_cec_xyz(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ vel, Geo g, int64_t fin,
          int64_t fout)
{
    in += (int64_t)blockIdx.y * fin;   // field of this CTA (FieldSet)
    out += (int64_t)blockIdx.y * fout;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nitems = g.tiles_x * g.tiles_y * g.chunks;
    bool bad = false;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x)
        xyz_item<T, D, TX, TY, HAS_Z, VEC>(g, item, in, out, vel, smem_raw, bad);
    flag_cfl(g.status, bad);
}

// ============================================================ order z, y, x
template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
struct ZYX {
    using S = Shape<T, TX, TY>;
    static constexpr int RX = 4, RY = 4;
    static constexpr int NT = 256;
    static constexpr int NB = 2;
    static constexpr int NZC = (TX + 6) * (TY + 6);           // z-swept columns
    static constexpr int NCOL = HAS_Z ? (NZC + NT - 1) / NT : 1;
    static constexpr int SZ_PHI = S::PH * S::PW;
    static constexpr int SZ_CZ = HAS_Z ? S::PH * S::PW : 0;
    static constexpr int SZ_Z = HAS_Z ? S::PH * S::PW : 0;
    static constexpr int SZ_CY = (TY + 4) * S::PW;
    static constexpr int SZ_S2 = TY * S::PW;
    static constexpr int SZ_CX = TY * S::PW;
    static constexpr size_t smem()
    {
        return sizeof(T) * (size_t)(NB * (SZ_PHI + SZ_CZ + SZ_CY + SZ_CX) + SZ_Z + SZ_S2);
    }
};

template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
__device__ __forceinline__ void zyx_item(const Geo &g, int item, const T *__restrict__ in, T *__restrict__ out,
                                         const T *__restrict__ vel, unsigned char *smem_raw, bool &bad)
{
    using K = ZYX<T, D, TX, TY, HAS_Z, VEC>;
    using S = typename K::S;
    constexpr int RX = K::RX, RY = K::RY, NT = K::NT, NB = K::NB, NCOL = K::NCOL;
    T *sPhi = reinterpret_cast<T *>(smem_raw);
    T *sCz = sPhi + NB * K::SZ_PHI;
    T *sCy = sCz + NB * K::SZ_CZ;
    T *sCx = sCy + NB * K::SZ_CY;
    T *sZ = sCx + NB * K::SZ_CX;
    T *sS2 = sZ + K::SZ_Z;

    const int tid = threadIdx.x;
    const D sx = D(g.sx), sy = D(g.sy), sz = D(g.sz);

    Stager<T, NT, S::PH, S::HW, S::PW, VEC> stPhi;     // Phi, u_z: rows [-3,TY+3), cols [-4,TX+4)
    Stager<T, NT, TY + 4, S::HW, S::PW, VEC> stCy;     // u_y: rows [-2,TY+2)
    Stager<T, NT, TY, S::HW, S::PW, VEC> stCx;         // u_x: rows [0,TY)

    int x0, y0, z0, z1;
    decode_item(item, g, TX, TY, x0, y0, z0, z1);
    stPhi.setup(tid, x0, y0, -3, -4, g.nx, g.ny);
    stCy.setup(tid, x0, y0, -2, -4, g.nx, g.ny);
    stCx.setup(tid, x0, y0, 0, -4, g.nx, g.ny);

    const int pfirst = HAS_Z ? z0 - 3 : 0;
    const int plast = HAS_Z ? z1 + 2 : 0;
    auto issue = [&](int p, int slot) {
        const int64_t base = (int64_t)wrapi(p, g.nz) * g.plane;
        stPhi.issue(tid, sPhi + slot * K::SZ_PHI, in + base, x0, y0, -3, -4, g.nx, g.ny);
        int64_t bk = base;
        if constexpr (HAS_Z) {
            const int64_t bz = (int64_t)wrapi(p - 1, g.nz) * g.plane;
            stPhi.issue(tid, sCz + slot * K::SZ_CZ, vel + 2 * g.ncell + bz, x0, y0, -3, -4, g.nx, g.ny);
            bk = (int64_t)wrapi(p - 3, g.nz) * g.plane;
        }
        stCy.issue(tid, sCy + slot * K::SZ_CY, vel + g.ncell + bk, x0, y0, -2, -4, g.nx, g.ny);
        stCx.issue(tid, sCx + slot * K::SZ_CX, vel + bk, x0, y0, 0, -4, g.nx, g.ny);
        cp_async_commit();
    };

    ZWin<T, D> win[NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) win[j].init();

    issue(pfirst, 0);
    for (int p = pfirst; p <= plast; ++p) {
        const int slot = (p - pfirst) & 1;
        cp_async_wait_all();
        __syncthreads();
        if (p < plast) issue(p + 1, slot ^ 1);

        const T *zsrc = sPhi + slot * K::SZ_PHI;
        int kz = 0;
        if constexpr (HAS_Z) {
            // ---- z sweep over columns x in [-3, TX+3), y in [-3, TY+3)
            const T *czP = sCz + slot * K::SZ_CZ;
#pragma unroll
            for (int j = 0; j < NCOL; ++j) {
                const int r = tid + j * NT;
                if (r < K::NZC) {
                    const int row = r / (TX + 6), col = r - (r / (TX + 6)) * (TX + 6) + 1;
                    const D c = D(czP[row * S::PW + col]) * sz;
                    const T v = win[j].push(zsrc[row * S::PW + col], c);
                    sZ[row * S::PW + col] = v;
                    if (row >= 3 && row < TY + 3 && col >= 4 && col < TX + 4) bad |= fabs(c) > D(1);
                }
            }
            __syncthreads();
            kz = p - 3;
            if (kz < z0) continue;
            zsrc = sZ;
        }

        // ---- y sweep: columns x in [-3, TX+3), rows [0, TY) -> sS2
        const T *cyP = sCy + slot * K::SZ_CY;
        for (int r = tid; r < (TX + 6) * (TY / RY); r += NT) {
            const int col = r % (TX + 6) + 1, yr = (r / (TX + 6)) * RY;
            T pv[RY + 6];
#pragma unroll
            for (int k = 0; k < RY + 6; ++k) pv[k] = zsrc[(yr + k) * S::PW + col];
            D cv[RY + 4];
#pragma unroll
            for (int k = 0; k < RY + 4; ++k) cv[k] = D(cyP[(yr + k) * S::PW + col]) * sy;
            if (col >= 4 && col < TX + 4) {
#pragma unroll
                for (int k = 2; k < RY + 2; ++k) bad |= fabs(cv[k]) > D(1);
            }
            T o[RY];
            cec_line<T, D, RY>(pv, cv, o);
#pragma unroll
            for (int i = 0; i < RY; ++i) sS2[(yr + i) * S::PW + col] = o[i];
        }
        __syncthreads();

        // ---- x sweep: rows [0, TY), cols [0, TX) -> global plane kz
        const T *cxP = sCx + slot * K::SZ_CX;
        constexpr int XR = TX / RX;
        for (int r = tid; r < TY * XR; r += NT) {
            const int row = r / XR, xr = (r - (r / XR) * XR) * RX;
            T blk[RX + 8];
            lds_vec<T, RX + 8>(sS2 + row * S::PW + xr, blk);
            T pv[RX + 6];
#pragma unroll
            for (int k = 0; k < RX + 6; ++k) pv[k] = blk[k + 1];
            lds_vec<T, RX + 8>(cxP + row * S::PW + xr, blk);
            D cv[RX + 4];
#pragma unroll
            for (int k = 0; k < RX + 4; ++k) cv[k] = D(blk[k + 2]) * sx;
#pragma unroll
            for (int k = 2; k < RX + 2; ++k) bad |= fabs(cv[k]) > D(1);
            T o[RX];
            cec_line<T, D, RX>(pv, cv, o);
            const int gy = y0 + row;
            if (gy < g.ny) {
                T *dst = out + (int64_t)kz * g.plane + (int64_t)gy * g.nx + x0 + xr;
                if (VEC && x0 + xr + RX <= g.nx) {
                    if constexpr (sizeof(T) == 4) {
                        reinterpret_cast<float4 *>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
                    } else {
                        reinterpret_cast<double2 *>(dst)[0] = make_double2(o[0], o[1]);
                        reinterpret_cast<double2 *>(dst)[1] = make_double2(o[2], o[3]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < RX; ++i)
                        if (x0 + xr + i < g.nx) dst[i] = o[i];
                }
            }
        }
    }
    __syncthreads();
}

template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
__global__ void __launch_bounds__(256)
k_cec_zyx(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ vel, Geo g, int64_t fin,
          int64_t fout)
{
    in += (int64_t)blockIdx.y * fin;   // field of this CTA (FieldSet)
    out += (int64_t)blockIdx.y * fout;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nitems = g.tiles_x * g.tiles_y * g.chunks;
    bool bad = false;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x)
        zyx_item<T, D, TX, TY, HAS_Z, VEC>(g, item, in, out, vel, smem_raw, bad);
    flag_cfl(g.status, bad);
}

template <typename T, typename D, int TX, int TY, bool HAS_Z, bool VEC>
cudaError_t dispatch_order(int parity, const Geo &g, int grid, const void *in, void *out, const void *vel,
                           const FieldSet &fs, cudaStream_t st)
{
    const T *i = static_cast<const T *>(in);
    const T *v = static_cast<const T *>(vel);
    T *o = static_cast<T *>(out);
    if ((parity & 1) == 0) {
        using K = XYZ<T, D, TX, TY, HAS_Z, VEC>;
        auto kern = k_cec_xyz<T, D, TX, TY, HAS_Z, VEC>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem());
        if (e != cudaSuccess) return e;
        const int nitems = g.tiles_x * g.tiles_y * g.chunks;
        const int gr = grid > 0 && grid < nitems ? grid : nitems;
        kern<<<dim3(gr, fs.n), K::NT, K::smem(), st>>>(i, o, v, g, fs.fin, fs.fout);
    } else {
        using K = ZYX<T, D, TX, TY / 2, HAS_Z, VEC>;
        auto kern = k_cec_zyx<T, D, TX, TY / 2, HAS_Z, VEC>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem());
        if (e != cudaSuccess) return e;
        Geo g2 = g;
        g2.tiles_y = (g.ny + TY / 2 - 1) / (TY / 2);
        const int nitems = g2.tiles_x * g2.tiles_y * g2.chunks;
        const int gr = grid > 0 && grid < nitems ? grid : nitems;
        kern<<<dim3(gr, fs.n), K::NT, K::smem(), st>>>(i, o, v, g2, fs.fin, fs.fout);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ batched
// Persistent CTAs take (instance, tile, z-chunk) items from a device counter
// until the batch is exhausted; every item is the same fused step as above.
template <typename T, int TX, int TY, int PAR>
__global__ void __launch_bounds__(256)
k_cec_batched(const BatchRec *__restrict__ recs, int ninst, int nitems, unsigned *counter, unsigned *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    bool bad = false;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (recs[mid].item0[PAR] <= it) lo = mid; else hi = mid - 1;
        }
        const BatchRec &r = recs[lo];
        const Geo g = r.g[PAR];
        const T *in = static_cast<const T *>(PAR ? r.b : r.a);
        T *out = static_cast<T *>(PAR ? r.a : r.b);
        const T *vel = static_cast<const T *>(r.vel);
        if constexpr (PAR == 0)
            xyz_item<T, T, TX, TY, true, true>(g, it - r.item0[0], in, out, vel, smem_raw, bad);
        else
            zyx_item<T, T, TX, TY / 2, true, true>(g, it - r.item0[1], in, out, vel, smem_raw, bad);
    }
    flag_cfl(status, bad);
}

}  // namespace

int default_tz(int dtype, int ndim, const int64_t dims[3])
{
    (void)dtype;
    if (ndim == 2) return 1;
    // enough z chunks to give every SM two CTAs, but chunks of >= 16 planes
    const int64_t nz = dims[2];
    const int64_t cols = ((dims[0] + 31) / 32) * ((dims[1] + 31) / 32);
    int tz = (int)nz;
    const int64_t want = 2 * 152;
    while (tz > 16 && cols * ((nz + tz - 1) / tz) < want) tz = (tz + 1) / 2;
    return tz < 1 ? 1 : tz;
}

cudaError_t launch_split_cec(int dtype, const void *in, void *out, const void *vel, int ndim,
                             const int64_t dims[3], const double s[3], int parity, Launch lc,
                             unsigned *status, cudaStream_t st, FieldSet fs)
{
    constexpr int TX = 32;
    Geo g;
    g.nx = (int)dims[0];
    g.ny = (int)dims[1];
    g.nz = ndim == 3 ? (int)dims[2] : 1;
    g.plane = (int64_t)g.nx * g.ny;
    g.ncell = g.plane * g.nz;
    g.sx = s[0];
    g.sy = s[1];
    g.sz = ndim == 3 ? s[2] : 0.0;
    g.status = status;
    g.tz = ndim == 3 ? (lc.tz > 0 ? lc.tz : default_tz(dtype, ndim, dims)) : 1;
    if (g.tz > g.nz) g.tz = g.nz;
    g.chunks = (g.nz + g.tz - 1) / g.tz;
    g.tiles_x = (g.nx + TX - 1) / TX;
    const bool has_z = ndim == 3;
    if (dtype == 1) {   // SL_F64
        constexpr int TY = 16;
        g.tiles_y = (g.ny + TY - 1) / TY;
        const bool vec = lc.aligned && g.nx % 2 == 0;
        if (has_z)
            return vec ? dispatch_order<double, double, TX, TY, true, true>(parity, g, lc.grid, in, out, vel, fs, st)
                       : dispatch_order<double, double, TX, TY, true, false>(parity, g, lc.grid, in, out, vel, fs, st);
        return vec ? dispatch_order<double, double, TX, TY, false, true>(parity, g, lc.grid, in, out, vel, fs, st)
                   : dispatch_order<double, double, TX, TY, false, false>(parity, g, lc.grid, in, out, vel, fs, st);
    }
    constexpr int TY = 32;
    g.tiles_y = (g.ny + TY - 1) / TY;
    const bool vec = lc.aligned && g.nx % 4 == 0;
    if (dtype == 2) {   // SL_F32_D64
        if (has_z)
            return vec ? dispatch_order<float, double, TX, TY, true, true>(parity, g, lc.grid, in, out, vel, fs, st)
                       : dispatch_order<float, double, TX, TY, true, false>(parity, g, lc.grid, in, out, vel, fs, st);
        return vec ? dispatch_order<float, double, TX, TY, false, true>(parity, g, lc.grid, in, out, vel, fs, st)
                   : dispatch_order<float, double, TX, TY, false, false>(parity, g, lc.grid, in, out, vel, fs, st);
    }
    if (has_z)
        return vec ? dispatch_order<float, float, TX, TY, true, true>(parity, g, lc.grid, in, out, vel, fs, st)
                   : dispatch_order<float, float, TX, TY, true, false>(parity, g, lc.grid, in, out, vel, fs, st);
    return vec ? dispatch_order<float, float, TX, TY, false, true>(parity, g, lc.grid, in, out, vel, fs, st)
               : dispatch_order<float, float, TX, TY, false, false>(parity, g, lc.grid, in, out, vel, fs, st);
}

size_t batched_smem(int parity)
{
    return parity ? ZYX<float, float, 32, 16, true, true>::smem() : XYZ<float, float, 32, 32, true, true>::smem();
}

void batched_tiles(int parity, int &tx, int &ty)
{
    tx = 32;
    ty = parity ? 16 : 32;
}

cudaError_t launch_batched_cec(const BatchRec *dev_recs, int ninst, int nitems, int parity, unsigned *counter,
                               unsigned *status, int grid, cudaStream_t st)
{
    const size_t smem = batched_smem(parity);
    if (parity) {
        auto kern = k_cec_batched<float, 32, 32, 1>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, 256, smem, st>>>(dev_recs, ninst, nitems, counter, status);
    } else {
        auto kern = k_cec_batched<float, 32, 32, 0>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, 256, smem, st>>>(dev_recs, ninst, nitems, counter, status);
    }
    return cudaGetLastError();
}

int batched_blocks_per_sm(int parity)
{
    int nb = 0;
    const size_t smem = batched_smem(parity);
    cudaError_t e;
    if (parity) {
        auto kern = k_cec_batched<float, 32, 32, 1>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
    } else {
        auto kern = k_cec_batched<float, 32, 32, 0>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
    }
    return e == cudaSuccess && nb > 0 ? nb : 1;
}

}  // namespace sl
