// k_unsplit.cu -- fused unsplit CIR / FEC / BEC step.
//
// The multilinear operator L_U (Sec. 2; eq. CIR2D and its 3D tensor-product
// analogue) is applied 1, 2 or 3 times (Table 1, "Nb of calls"):
//   stage 1  L_U[Phi]                         on the tile + (NST-1) halo
//   stage 2  Phi_bar = L_{-U}[L_U[Phi]]        on the tile + (NST-2) halo,
//            FEC = L_U[Phi] + (Phi - Phi_bar)/2 (eq. intro:FEC) or
//            Psi = Phi + (Phi - Phi_bar)/2       (BEC input)
//   stage 3  BEC = L_U[Psi]                   on the tile (eq. intro:BEC)
// so the halo of Phi grows by one cell per stage (NST cells) and that of u
// by NST-1.  The CTA marches along z; a plane of stage s is produced s planes
// behind the newest loaded plane, and each stage keeps the three planes its
// successor reads in a shared-memory ring.  One HBM read of Phi and u and one
// write of the result per cell.
#include "sl_internal.h"

namespace sl {
namespace {

// Multilinear value at a departure point with |C| <= 1 in the sign form of
// Sec. 3: on each axis the corners are the cell itself and its neighbour at
// offset `o_d` (= -s_d for L_U, +s_d for L_{-U}; 0 when C_d = 0), weighted
// W_d = 1 - U_d and U_d.  Each lerp is written from the neighbour, n + W (c - n),
// so that U = 1 picks the neighbour exactly, C = 0 (o_d = 0) the cell, and a
// constant field stays constant.  q0 is the cell's plane, q1 the neighbouring
// plane on z (q0 itself when C_z = 0); wx, wy, wz are the W_d.
template <typename A, bool HAS_Z, typename S>
__device__ __forceinline__ A mlerp(const S *q0, const S *q1, int o, int ox, int oy, A wx, A wy, A wz)
{
    const A a00 = A(q0[o]), a10 = A(q0[o + ox]), a01 = A(q0[o + oy]), a11 = A(q0[o + oy + ox]);
    const A b0 = a10 + wx * (a00 - a10);
    const A b1 = a11 + wx * (a01 - a11);
    const A c0 = b1 + wy * (b0 - b1);
    if constexpr (!HAS_Z) {
        return c0;
    } else {
        const A e00 = A(q1[o]), e10 = A(q1[o + ox]), e01 = A(q1[o + oy]), e11 = A(q1[o + oy + ox]);
        const A f0 = e10 + wx * (e00 - e10);
        const A f1 = e11 + wx * (e01 - e11);
        const A c1 = f1 + wy * (f0 - f1);
        return c1 + wz * (c0 - c1);
    }
}

template <typename T, typename D, int NST, int TX, int TY, bool HAS_Z>
struct Cfg {
    static constexpr int NT = 256;
    static constexpr int H = NST;                          // Phi halo
    static constexpr int HW = TX + 8;                      // staged x in [-4, TX+4)
    // row stride; FP32 BEC rows are unpadded so that three CTAs fit on an SM
    static constexpr int PW = HW + (sizeof(T) == 4 ? (NST == 3 ? 0 : 4) : 2);
    static constexpr int PH = TY + 2 * H;                  // staged y in [-H, TY+H)
    static constexpr int SLOT = PH * PW;
    static constexpr int NPHI = HAS_Z ? 4 : 1;             // Phi ring: planes p-2..p + prefetch
    static constexpr int NCS = HAS_Z ? NST + 1 : 1;        // u ring
    static constexpr int NC = HAS_Z ? 3 : 2;               // velocity components
    static constexpr int NL = NST >= 2 ? (HAS_Z ? 3 : 1) : 0;   // L_U[Phi] ring (type D)
    static constexpr int NP = NST >= 3 ? (HAS_Z ? 3 : 1) : 0;   // Psi ring
    // The other rings hold only the rows they use: u rows [-(H-1), TY+H-1),
    // L_U[Phi] (stage 1 output) rows [-(NST-1), TY+NST-1), Psi (stage 2 output)
    // rows [-(NST-2), TY+NST-2).  Their ring pointers are shifted back by the
    // missing top rows (SHC, SHL, SHP), so that one offset o = (y + H) PW + x + 4
    // addresses the same cell in every ring.
    static constexpr int SHC = 1, SHL = H - (NST - 1), SHP = H - (NST - 2);
    static constexpr int SC = (TY + 2 * (H - 1)) * PW;
    static constexpr int SLL = (TY + 2 * (NST - 1)) * PW;
    static constexpr int SLP = NST >= 2 ? (TY + 2 * (NST - 2)) * PW : 0;
    static constexpr size_t smem()
    {
        return sizeof(T) * ((size_t)SLOT * NPHI + (size_t)SC * NCS * NC + (size_t)SLP * NP) +
               sizeof(D) * (size_t)SLL * NL;
    }
};

// Stage rows [r0, r0 + nr) x staged columns [-4, TX+4) of one plane.
template <typename T, int NT, int TX, int PW, bool VEC>
__device__ __forceinline__ void stage_rows(int tid, T *dst, const T *src, int x0, int y0, int r0, int nr, int H,
                                           int nx, int ny)
{
    constexpr int HW = TX + 8;
    if constexpr (VEC) {
        constexpr int V = 16 / sizeof(T);
        constexpr int CPR = HW / V;
        for (int idx = tid; idx < nr * CPR; idx += NT) {
            const int row = idx / CPR, cc = idx - (idx / CPR) * CPR;
            const int gy = wrapi(y0 + r0 + row, ny);
            const int gx = wrapi(x0 - 4 + cc * V, nx);
            cp_async16(dst + (r0 + row + H) * PW + cc * V, src + (int64_t)gy * nx + gx);
        }
    } else {
        for (int idx = tid; idx < nr * HW; idx += NT) {
            const int row = idx / HW, col = idx - (idx / HW) * HW;
            const int gy = wrapi(y0 + r0 + row, ny);
            const int gx = wrapi(x0 - 4 + col, nx);
            cp_async_elem(dst + (r0 + row + H) * PW + col, src + (int64_t)gy * nx + gx);
        }
    }
}

// 16-byte chunks of the staged rows [r0, r0 + NR) x columns [-4, TX+4) of a
// tile, when a row crosses the periodic seams at most once (nx >= TX + 8 and
// ny >= TY + NST): thread tid owns chunks tid + k NT, whose in-plane source and
// shared-memory offsets are computed once per tile.
template <typename T, int NT, int TX, int NR, int PW>
struct RowChunks {
    static constexpr int V = 16 / sizeof(T), CPR = (TX + 8) / V, N = NR * CPR, K = (N + NT - 1) / NT;
    int src[K];
    int dst[K];

    __device__ __forceinline__ void setup(int tid, int x0, int y0, int r0, int H, int nx, int ny)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int idx = tid + k * NT;
            if (idx < N) {
                const int row = idx / CPR, cc = idx - row * CPR;
                int gy = y0 + r0 + row, gx = x0 - 4 + cc * V;
                gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
                gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
                src[k] = gy * nx + gx;
                dst[k] = (r0 + row + H) * PW + cc * V;
            } else {
                src[k] = -1;
                dst[k] = 0;
            }
        }
    }

    __device__ __forceinline__ void issue(T *sdst, const T *gsrc) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (src[k] >= 0) cp_async16(sdst + dst[k], gsrc + src[k]);
    }
};

template <typename T, typename D, int NST, int TX, int TY, bool HAS_Z, bool VEC>
__global__ void __launch_bounds__(256)
k_unsplit(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ vel, Geo g, int64_t fin, int64_t fout)
{
    in += (int64_t)blockIdx.y * fin;   // field of this CTA (FieldSet)
    out += (int64_t)blockIdx.y * fout;
    using K = Cfg<T, D, NST, TX, TY, HAS_Z>;
    constexpr int NT = K::NT, H = K::H, PW = K::PW, SLOT = K::SLOT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int SC = K::SC, SLL = K::SLL, SLP = K::SLP;
    T *sPhi = reinterpret_cast<T *>(smem_raw);                 // [NPHI][SLOT]
    T *sC = sPhi + K::NPHI * SLOT;                             // [NCS][NC][SC]
    T *sP = sC + K::NCS * K::NC * SC;                          // [NP][SLP]
    D *sL = reinterpret_cast<D *>(sP + K::NP * SLP);           // [NL][SLL]

    const int tid = threadIdx.x;
    const D sxd = D(g.sx), syd = D(g.sy), szd = D(g.sz);
    bool bad = false;
    // Work split.  BEC (three stages; its shared memory allows two CTAs per SM):
    // persistent CTAs; the (column tile, plane) pairs are numbered tile by tile
    // and every CTA takes one contiguous, equal share, walking z inside each
    // tile.  A tile's pairs are numbered from a tile-dependent plane, so that
    // the share boundaries of all tiles fall on the same planes (neighbouring
    // tiles are then processed at the same z and their shared halo rows stay in
    // L2); planes are taken modulo nz.  CIR and FEC (more CTAs per SM): one
    // (column tile, z chunk of g.tz planes) item per CTA, items over the grid.
    constexpr bool PERSIST = NST == 3 && HAS_Z;
    const int nzz = HAS_Z ? g.nz : 1;
    const int64_t total = PERSIST ? (int64_t)g.tiles_x * g.tiles_y * nzz : (int64_t)g.tiles_x * g.tiles_y * g.chunks;
    const int64_t G = gridDim.x;
    int64_t w = PERSIST ? total * blockIdx.x / G : blockIdx.x;
    const int64_t wend = PERSIST ? total * (blockIdx.x + 1) / G : total;
    const double share = (double)total / (double)G;

    while (w < wend) {
        int t, z0, z1;
        if constexpr (PERSIST) {
            t = (int)(w / nzz);
            const int64_t tile_w = (int64_t)t * nzz;
            const int o = (int)(w - tile_w);
            const int rot = (int)(fmod((double)tile_w, share) + 0.5) % nzz;
            const int64_t e = wend < tile_w + nzz ? wend : tile_w + nzz;
            z0 = o + rot;                   // in [0, 2 nz)
            z1 = z0 + (int)(e - w);
            w = e;
        } else {
            const int item = (int)w;
            t = item % (g.tiles_x * g.tiles_y);
            z0 = (item / (g.tiles_x * g.tiles_y)) * g.tz;
            z1 = min(z0 + g.tz, g.nz);
            w += G;
        }
        const int x0 = (t % g.tiles_x) * TX;
        const int y0 = (t / g.tiles_x) * TY;
        const int pfirst = HAS_Z ? z0 - NST : 0;
        const int plast = HAS_Z ? z1 + NST - 1 : 0;
        // per-tile chunk offsets when rows wrap at most once (the common case)
        const bool once = VEC && g.nx >= TX + 8 && g.ny >= TY + NST;
        RowChunks<T, NT, TX, TY + 2 * H, PW> chPhi;
        RowChunks<T, NT, TX, TY + 2 * (H - 1), PW> chC;
        if (once) {
            chPhi.setup(tid, x0, y0, -H, H, g.nx, g.ny);
            chC.setup(tid, x0, y0, -(H - 1), H, g.nx, g.ny);
        }

        auto issue = [&](int p) {
            const int b = p - pfirst;
            const int64_t base = (int64_t)wrapi(p, g.nz) * g.plane;
            const int64_t bc = HAS_Z ? (int64_t)wrapi(p - 1, g.nz) * g.plane : base;
            T *cdst = sC + (b % K::NCS) * K::NC * SC - K::SHC * PW;
            if (once) {
                chPhi.issue(sPhi + (b % K::NPHI) * SLOT, in + base);
#pragma unroll
                for (int d = 0; d < K::NC; ++d) chC.issue(cdst + d * SC, vel + d * g.ncell + bc);
            } else {
                stage_rows<T, NT, TX, PW, VEC>(tid, sPhi + (b % K::NPHI) * SLOT, in + base, x0, y0, -H, TY + 2 * H,
                                               H, g.nx, g.ny);
#pragma unroll
                for (int d = 0; d < K::NC; ++d)
                    stage_rows<T, NT, TX, PW, VEC>(tid, cdst + d * SC, vel + d * g.ncell + bc, x0, y0, -(H - 1),
                                                   TY + 2 * (H - 1), H, g.nx, g.ny);
            }
            cp_async_commit();
        };
        // ring slots of plane q
        auto sl_phi = [&](int q) { return sPhi + ((q - pfirst) % K::NPHI) * SLOT; };
        auto sl_c = [&](int q) { return sC + ((q + 1 - pfirst) % K::NCS) * K::NC * SC - K::SHC * PW; };
        auto sl_l = [&](int q) { return sL + (K::NL > 1 ? ((q + 1 - pfirst) % 3) : 0) * SLL - K::SHL * PW; };
        auto sl_p = [&](int q) { return sP + (K::NP > 1 ? ((q + 1 - pfirst) % 3) : 0) * SLP - K::SHP * PW; };

        issue(pfirst);
        for (int p = pfirst; p <= plast; ++p) {
            cp_async_wait_all();
            __syncthreads();
            if (p < plast) issue(p + 1);

            // ------------------------------------------------ stage 1: L_U[Phi]
            if (!HAS_Z || p >= z0 - NST + 2) {
                const int q = HAS_Z ? p - 1 : 0;
                constexpr int h = NST - 1;
                constexpr int RW = TX + 2 * h, RH = TY + 2 * h;
                const T *phi0 = sl_phi(q);
                const T *cP = sl_c(q);
                const T *phim = HAS_Z ? sl_phi(q - 1) : phi0, *php = HAS_Z ? sl_phi(q + 1) : phi0;
                D *const lq = sl_l(q);
                int yy = tid / RW, xx = tid - (tid / RW) * RW;
                for (int r = tid; r < RW * RH; r += NT, xx += NT % RW, yy += NT / RW) {
                    if (xx >= RW) {
                        xx -= RW;
                        ++yy;
                    }
                    const int o = (yy - h + H) * PW + (xx - h + 4);
                    const D cx = D(cP[o]) * sxd, cy = D(cP[SC + o]) * syd;
                    const D cz = HAS_Z ? D(cP[2 * SC + o]) * szd : D(0);
                    const int ox = by_sign(cx, -1, 1, 0), oy = by_sign(cy, -PW, PW, 0);
                    const T *phi1 = HAS_Z ? by_sign<D, const T *>(cz, phim, php, phi0) : phi0;
                    const D v = mlerp<D, HAS_Z>(phi0, phi1, o, ox, oy, D(1) - fabs(cx), D(1) - fabs(cy),
                                                D(1) - fabs(cz));
                    if constexpr (NST == 1) {
                        bad |= fabs(cx) > D(1) || fabs(cy) > D(1) || fabs(cz) > D(1);
                        const int gx = x0 + xx, gy = y0 + yy;
                        if (gx < g.nx && gy < g.ny) out[(int64_t)(q >= g.nz ? q - g.nz : q) * g.plane + (int64_t)gy * g.nx + gx] = T(v);
                    } else {
                        lq[o] = v;
                    }
                }
            }
            if constexpr (NST >= 2) {
                __syncthreads();
                // -------------------------------- stage 2: Phi_bar and the correction
                if (!HAS_Z || p >= z0 - NST + 4) {
                    const int q = HAS_Z ? p - 2 : 0;
                    constexpr int h = NST - 2;
                    constexpr int RW = TX + 2 * h, RH = TY + 2 * h;
                    const T *phiq = sl_phi(q);
                    const T *cP = sl_c(q);
                    const D *l0 = sl_l(q);
                    const D *lp = HAS_Z ? sl_l(q + 1) : l0, *lm = HAS_Z ? sl_l(q - 1) : l0;
                    T *const pq = sl_p(q);
                    int yy = tid / RW, xx = tid - (tid / RW) * RW;
                    for (int r = tid; r < RW * RH; r += NT, xx += NT % RW, yy += NT / RW) {
                        if (xx >= RW) {
                            xx -= RW;
                            ++yy;
                        }
                        const int o = (yy - h + H) * PW + (xx - h + 4);
                        const D cx = D(cP[o]) * sxd, cy = D(cP[SC + o]) * syd;
                        const D cz = HAS_Z ? D(cP[2 * SC + o]) * szd : D(0);
                        // reversed flow: departure x + u dt, corners toward +s
                        const int ox = by_sign(cx, 1, -1, 0), oy = by_sign(cy, PW, -PW, 0);
                        const D *l1 = HAS_Z ? by_sign<D, const D *>(cz, lp, lm, l0) : l0;
                        const D bar = mlerp<D, HAS_Z>(l0, l1, o, ox, oy, D(1) - fabs(cx), D(1) - fabs(cy),
                                                      D(1) - fabs(cz));
                        const D delta = D(phiq[o]) - bar;
                        if constexpr (NST == 2) {
                            bad |= fabs(cx) > D(1) || fabs(cy) > D(1) || fabs(cz) > D(1);
                            const int gx = x0 + xx, gy = y0 + yy;
                            if (gx < g.nx && gy < g.ny)
                                out[(int64_t)(q >= g.nz ? q - g.nz : q) * g.plane + (int64_t)gy * g.nx + gx] = T(l0[o] + delta * D(0.5));
                        } else {
                            pq[o] = T(D(phiq[o]) + delta * D(0.5));
                        }
                    }
                }
            }
            if constexpr (NST >= 3) {
                __syncthreads();
                // -------------------------------------------- stage 3: L_U[Psi]
                if (!HAS_Z || p >= z0 + 3) {
                    const int q = HAS_Z ? p - 3 : 0;
                    const T *cP = sl_c(q);
                    const T *p0 = sl_p(q);
                    const T *pm = HAS_Z ? sl_p(q - 1) : p0, *pp = HAS_Z ? sl_p(q + 1) : p0;
                    for (int r = tid; r < TX * TY; r += NT) {
                        const int yy = r / TX, xx = r - (r / TX) * TX;
                        const int o = (yy + H) * PW + (xx + 4);
                        const T cx = T(D(cP[o]) * sxd), cy = T(D(cP[SC + o]) * syd);
                        const T cz = HAS_Z ? T(D(cP[2 * SC + o]) * szd) : T(0);
                        bad |= fabs(cx) > T(1) || fabs(cy) > T(1) || fabs(cz) > T(1);
                        const int ox = by_sign(cx, -1, 1, 0), oy = by_sign(cy, -PW, PW, 0);
                        const T *p1 = HAS_Z ? by_sign<T, const T *>(cz, pm, pp, p0) : p0;
                        const T v = mlerp<T, HAS_Z>(p0, p1, o, ox, oy, T(1) - fabs(cx), T(1) - fabs(cy),
                                                    T(1) - fabs(cz));
                        const int gx = x0 + xx, gy = y0 + yy;
                        if (gx < g.nx && gy < g.ny) out[(int64_t)(q >= g.nz ? q - g.nz : q) * g.plane + (int64_t)gy * g.nx + gx] = v;
                    }
                }
            }
        }
        __syncthreads();
    }
    flag_cfl(g.status, bad);
}

template <typename T, typename D, int NST, int TX, int TY, bool HAS_Z, bool VEC>
cudaError_t go(Geo g, int grid, const void *in, void *out, const void *vel, const FieldSet &fs, cudaStream_t st)
{
    using K = Cfg<T, D, NST, TX, TY, HAS_Z>;
    auto kern = k_unsplit<T, D, NST, TX, TY, HAS_Z, VEC>;
    // shared-memory opt-in and resident CTAs per SM, once per device
    static int per_dev[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (per_dev[dev] == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem());
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::NT, K::smem());
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        per_dev[dev] = sms * (per_sm > 0 ? per_sm : 1);
    }
    g.tiles_y = (g.ny + TY - 1) / TY;
    const bool persist = NST == 3 && HAS_Z;
    const int64_t total = (int64_t)g.tiles_x * g.tiles_y * (persist ? g.nz : g.chunks);
    int gr = grid > 0 ? grid : (persist ? per_dev[dev] : (int)total);
    if (gr > total) gr = (int)total;
    kern<<<dim3(gr, fs.n), K::NT, K::smem(), st>>>(static_cast<const T *>(in), static_cast<T *>(out),
                                                   static_cast<const T *>(vel), g, fs.fin, fs.fout);
    return cudaGetLastError();
}

template <typename T, typename D, int TY, bool HAS_Z, bool VEC>
cudaError_t by_scheme(int scheme, const Geo &g, int grid, const void *in, void *out, const void *vel,
                      const FieldSet &fs, cudaStream_t st)
{
    switch (scheme) {
    case 0: return go<T, D, 1, 32, TY, HAS_Z, VEC>(g, grid, in, out, vel, fs, st);
    case 1: return go<T, D, 2, 32, TY, HAS_Z, VEC>(g, grid, in, out, vel, fs, st);
    default: return go<T, D, 3, 32, TY, HAS_Z, VEC>(g, grid, in, out, vel, fs, st);
    }
}

template <typename T, typename D, int TY>
cudaError_t by_shape(int scheme, bool has_z, bool vec, const Geo &g, int grid, const void *in, void *out,
                     const void *vel, const FieldSet &fs, cudaStream_t st)
{
    if (has_z)
        return vec ? by_scheme<T, D, TY, true, true>(scheme, g, grid, in, out, vel, fs, st)
                   : by_scheme<T, D, TY, true, false>(scheme, g, grid, in, out, vel, fs, st);
    return vec ? by_scheme<T, D, TY, false, true>(scheme, g, grid, in, out, vel, fs, st)
               : by_scheme<T, D, TY, false, false>(scheme, g, grid, in, out, vel, fs, st);
}

}  // namespace

cudaError_t launch_unsplit(int dtype, int scheme, const void *in, void *out, const void *vel, int ndim,
                           const int64_t dims[3], const double s[3], Launch lc, unsigned *status, cudaStream_t st,
                           FieldSet fs)
{
    if (scheme == 0 && cir_fast_eligible(dtype, ndim, dims, lc.aligned)) {
        const size_t es = dtype == 1 ? 8 : 4;
        for (int f = 0; f < fs.n; ++f) {
            const cudaError_t e = launch_cir_fast(static_cast<const char *>(in) + f * fs.fin * es,
                                                  static_cast<char *>(out) + f * fs.fout * es, vel, dims, s, lc,
                                                  status, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
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
    g.tiles_x = (g.nx + 31) / 32;
    const bool has_z = ndim == 3;
    if (dtype == 1) return by_shape<double, double, 8>(scheme, has_z, lc.aligned && g.nx % 2 == 0, g, lc.grid, in, out, vel, fs, st);
    if (dtype == 2) return by_shape<float, double, 16>(scheme, has_z, lc.aligned && g.nx % 4 == 0, g, lc.grid, in, out, vel, fs, st);
    const bool vec = lc.aligned && g.nx % 4 == 0;
    // FP32 3D grids with vector staging: tile heights 8 and 32 besides 16 (a
    // launch-shape choice; a cell's arithmetic does not depend on it)
    if (has_z && vec && lc.ty == 8) return by_scheme<float, float, 8, true, true>(scheme, g, lc.grid, in, out, vel, fs, st);
    if (has_z && vec && lc.ty == 32) return by_scheme<float, float, 32, true, true>(scheme, g, lc.grid, in, out, vel, fs, st);
    return by_shape<float, float, 16>(scheme, has_z, vec, g, lc.grid, in, out, vel, fs, st);
}

}  // namespace sl
