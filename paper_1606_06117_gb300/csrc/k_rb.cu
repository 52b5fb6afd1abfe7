// k_rb.cu -- the Rayleigh-Benard driver of Sec. 6 (eqs. e:nsnd, e:Tnd, e:mnd,
// e:poisson, e:proj) on the GPU: a 2D box with walls on all four sides, the
// velocity U = (u, w) and the temperature perturbation theta advected
// semi-Lagrangian by U with one of the paper's schemes, explicit buoyancy and
// diffusion, and a pressure-correction projection.
//
// Discretisation (cell-centred, nx x nz cells of Lx x Lz):
//  * the fields live on a grid padded by G = 3 ghost layers (the reach of the
//    split CEC stencil); before each step the ghosts are the walls' mirror
//    images: u and w change sign across every wall (no slip), theta changes
//    sign across the plates (theta = 0) and keeps it across the side walls
//    (d theta / dx = 0);
//  * the advection is sl_advect on the padded grid with the padded velocity:
//    the periodic wrap of the step kernels only ever reaches ghost cells;
//  * u2 = L[u] + dt Pr lap u, w2 = L[w] + dt (Ra Pr theta + Pr lap w),
//    theta' = L[theta] + dt (w + lap theta), 5-point Laplacians of the step-n
//    fields;
//  * projection: face velocities are averages of the two adjacent cells (zero
//    on the walls), their divergence D is the right-hand side of lap phi = D
//    with the compact Neumann Laplacian, solved in its eigenbasis: the
//    orthonormal DCT-II matrices C_x, C_z diagonalise it with eigenvalues
//    -(4/h^2) sin^2(pi j / 2 n) per axis, so phi = C_z^T [(C_z D C_x^T) / lam] C_x
//    with the constant mode set to zero.  Cells take the average of their
//    two faces' gradient corrections.
//
// GB300 runs FP64 at a small fraction of its FP32 rate (about two FMAs per
// clock and SM), so the step is arranged to spend few FP64 operations and to
// spread them over many SMs: each producer writes its cells' ghost images
// itself (no separate fill pass), the forces kernel also gives the divergence,
// the transforms run one CTA per mode row with coalesced or broadcast loads,
// the per-cell kernels use small CTAs, and long runs replay the step from a
// CUDA graph (5 launches per step: the advection of the three fields in one
// launch, forces, two transforms, projection).
#include <cmath>
#include <new>
#include <vector>

#include "sl.h"
#include "sl_internal.h"

namespace sl {
namespace {

constexpr int RBG = 3;   // ghost layers

// Padded row length: G ghost columns on the left, G on the right and one more
// there when nx is odd, so that a padded plane has an even number of cells
// and the three state planes, back to back, share one 16-byte alignment.
__host__ __device__ constexpr int rb_px(int nx) { return nx + 2 * RBG + (nx & 1); }

// Ghost cell (k, i) of a padded (nz + 2G) x (nx + 2G) plane: the mirror image
// of an interior cell across the nearer wall(s), with sign sx per side-wall
// crossing and sz per plate crossing.  Interior cells are left alone.
template <typename T>
__global__ void k_rb_ghosts(T *p, int nplanes, int nx, int nz, int64_t pstride, const int *sx, const int *sz)
{
    const int px = rb_px(nx), pz = nz + 2 * RBG;
    const int64_t n = (int64_t)px * pz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nplanes;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(idx / n);
        const int64_t r = idx - (int64_t)f * n;
        const int k = (int)(r / px), i = (int)(r - (int64_t)k * px);
        const int ki = k - RBG, ii = i - RBG;
        const bool gk = ki < 0 || ki >= nz, gi = ii < 0 || ii >= nx;
        if (!gk && !gi) continue;
        const int mk = ki < 0 ? -1 - ki : (ki >= nz ? 2 * nz - 1 - ki : ki);
        const int mi = ii < 0 ? -1 - ii : (ii >= nx ? 2 * nx - 1 - ii : ii);
        const int s = (gk ? sz[f] : 1) * (gi ? sx[f] : 1);
        T *pl = p + f * pstride;
        pl[r] = T(s) * pl[(int64_t)(mk + RBG) * px + mi + RBG];
    }
}

// Stores v at interior cell (k, i) of a padded plane and at each ghost cell
// whose mirror image it is (sign sx per side-wall crossing, sz per plate
// crossing): the same values the ghost fill gives, written by the producer.
template <typename T>
__device__ __forceinline__ void store_mirrored(T *pl, int k, int i, T v, int nx, int nz, T sx, T sz)
{
    const int px = rb_px(nx), gr = px - nx - RBG;   // gr ghost columns on the right
    pl[(int64_t)(k + RBG) * px + i + RBG] = v;
    const int gi = i < RBG ? -1 - i : (i >= nx - gr ? 2 * nx - 1 - i : INT32_MIN);
    const int gk = k < RBG ? -1 - k : (k >= nz - RBG ? 2 * nz - 1 - k : INT32_MIN);
    // a cell near both side walls (small nx) has two x images
    const int gi2 = (i < RBG && i >= nx - gr) ? 2 * nx - 1 - i : INT32_MIN;
    const int gk2 = (k < RBG && k >= nz - RBG) ? 2 * nz - 1 - k : INT32_MIN;
    const int xs[3] = {i, gi, gi2}, zs[3] = {k, gk, gk2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if ((a == 0 && b == 0) || xs[a] == INT32_MIN || zs[b] == INT32_MIN) continue;
            const T sg = (a ? sx : T(1)) * (b ? sz : T(1));
            pl[(int64_t)(zs[b] + RBG) * px + xs[a] + RBG] = sg * v;
        }
}

// The explicit forces on the interior, from the advected fields a* and the
// step-n fields (ghosts filled): u2, w2 into o_u, o_w (interior only),
// theta' into o_t with its ghost images, and the divergence of the face
// velocities (averages of the adjacent cells of (u2, w2), zero on the walls)
// into d (nz x nx).  A cell evaluates u2 and w2 of its neighbours itself (the
// same expressions), so that no second pass is needed for the divergence.
template <typename T>
__global__ void k_rb_forces(const T *u, const T *w, const T *th, const T *au, const T *aw, const T *at, T *o_u, T *o_w,
                            T *o_t, T *d, int nx, int nz, T dt, T Ra, T Pr, T idx2, T idz2, T idx, T idz)
{
    const int px = rb_px(nx);
    const int n = nx * nz;
    auto lap = [&](const T *f, int64_t o) {
        return (f[o + 1] - T(2) * f[o] + f[o - 1]) * idx2 + (f[o + px] - T(2) * f[o] + f[o - px]) * idz2;
    };
    auto u2 = [&](int64_t o) { return au[o] + dt * (Pr * lap(u, o)); };
    auto w2 = [&](int64_t o) { return aw[o] + dt * (Ra * Pr * th[o] + Pr * lap(w, o)); };
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int k = c / nx, i = c - (c / nx) * nx;
        const int64_t o = (int64_t)(k + RBG) * px + i + RBG;
        const T uc = u2(o), wc = w2(o);
        o_u[o] = uc;
        o_w[o] = wc;
        store_mirrored(o_t, k, i, at[o] + dt * (w[o] + lap(th, o)), nx, nz, T(1), T(-1));
        const T ue = i + 1 < nx ? T(0.5) * (uc + u2(o + 1)) : T(0);
        const T uw = i > 0 ? T(0.5) * (u2(o - 1) + uc) : T(0);
        const T wn = k + 1 < nz ? T(0.5) * (wc + w2(o + px)) : T(0);
        const T ws = k > 0 ? T(0.5) * (w2(o - px) + wc) : T(0);
        d[c] = (ue - uw) * idx + (wn - ws) * idz;
    }
}

// out(c) = sum_{t < K} a[t * as] B[t * ldb + c] for c < N, by the CTA's 256
// threads: 64 columns at a time, each column's sum split over four thread
// groups (t = g mod 4, two terms in flight per group) and combined in fixed
// order in shared memory (part, 256 elements).
template <typename T, typename Store>
__device__ __forceinline__ void rb_vecmat(const T *a, int64_t as, const T *B, int64_t ldb, int K, int N, T *part,
                                          Store store)
{
    const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
    for (int c0 = 0; c0 < N; c0 += 64) {
        const int col = c0 + c;
        T acc0 = T(0), acc1 = T(0);
        if (col < N) {
            int t = g;
#pragma unroll 4
            for (; t + 4 < K; t += 8) {
                acc0 += a[t * as] * B[t * ldb + col];
                acc1 += a[(t + 4) * as] * B[(t + 4) * ldb + col];
            }
            if (t < K) acc0 += a[t * as] * B[t * ldb + col];
        }
        part[g * 64 + c] = acc0 + acc1;
        __syncthreads();
        if (g == 0 && col < N) store(col, (part[c] + part[64 + c]) + (part[128 + c] + part[192 + c]));
        __syncthreads();
    }
}

constexpr int kRbRowThreads = 256;

// Forward transform and solve, one CTA per z mode k:
//   R[i] = sum_m C_z[k][m] D[m][i],  F[k][j] = sum_i R[i] C_x[j][i] / lam_kj
// (lam_kj = lz[k] + lx[j]; the constant mode F[0][0] = 0).  Every load is
// coalesced across the threads or a broadcast (C_x enters transposed, cxT).
template <typename T>
__global__ void __launch_bounds__(kRbRowThreads)
k_rb_forward(const T *D, const T *cz, const T *cxT, const T *lx, const T *lz, T *F, int nx, int nz)
{
    extern __shared__ __align__(16) unsigned char rb_smem[];
    T *part = reinterpret_cast<T *>(rb_smem), *R = part + kRbRowThreads;
    const int k = blockIdx.x;
    rb_vecmat(cz + (int64_t)k * nz, 1, D, nx, nz, nx, part, [&](int i, T v) { R[i] = v; });
    T *Fk = F + (int64_t)k * nx;
    const T lk = lz[k];
    rb_vecmat(R, 1, cxT, nx, nx, nx, part,
              [&](int j, T v) { Fk[j] = (k == 0 && j == 0) ? T(0) : v / (lk + lx[j]); });
}

// Inverse transform, one CTA per row m of phi:
//   R[j] = sum_k C_z[k][m] F[k][j],  phi[m][i] = sum_j R[j] C_x[j][i].
template <typename T>
__global__ void __launch_bounds__(kRbRowThreads)
k_rb_inverse(const T *F, const T *cz, const T *cx, T *phi, int nx, int nz)
{
    extern __shared__ __align__(16) unsigned char rb_smem[];
    T *part = reinterpret_cast<T *>(rb_smem), *R = part + kRbRowThreads;
    const int m = blockIdx.x;
    rb_vecmat(cz + m, nz, F, nx, nz, nx, part, [&](int j, T v) { R[j] = v; });
    T *pm = phi + (int64_t)m * nx;
    rb_vecmat(R, 1, cx, nx, nx, nx, part, [&](int i, T v) { pm[i] = v; });
}

// Copies n elements from global to shared memory: 16-byte chunks by cp.async
// (both bases 16-byte aligned), the tail by plain loads.
template <typename T>
__device__ __forceinline__ void rb_stage(T *dst, const T *src, int64_t n)
{
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = n / V;
    for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) cp_async16(dst + c * V, src + c * V);
    for (int64_t i = nv * V + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Elements a staged operand block takes, rounded up to a 16-byte multiple.
template <typename T>
__host__ __device__ constexpr int64_t rb_pad(int64_t n)
{
    return (n + 16 / (int64_t)sizeof(T) - 1) / (16 / (int64_t)sizeof(T)) * (16 / (int64_t)sizeof(T));
}

// The same transforms with their matrix operands staged in shared memory
// first (small boxes: D or F and C_x^T or C_x fit), so that the sums read
// shared memory instead of waiting on L2; same summation order, same results.
template <typename T>
__global__ void __launch_bounds__(kRbRowThreads)
k_rb_forward_s(const T *D, const T *cz, const T *cxT, const T *lx, const T *lz, T *F, int nx, int nz)
{
    extern __shared__ __align__(16) unsigned char rb_smem[];
    T *part = reinterpret_cast<T *>(rb_smem), *R = part + kRbRowThreads;
    T *sD = R + rb_pad<T>(nx), *sC = sD + rb_pad<T>((int64_t)nz * nx);
    rb_stage(sD, D, (int64_t)nz * nx);
    rb_stage(sC, cxT, (int64_t)nx * nx);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int k = blockIdx.x;
    rb_vecmat(cz + (int64_t)k * nz, 1, sD, nx, nz, nx, part, [&](int i, T v) { R[i] = v; });
    T *Fk = F + (int64_t)k * nx;
    const T lk = lz[k];
    rb_vecmat(R, 1, sC, nx, nx, nx, part,
              [&](int j, T v) { Fk[j] = (k == 0 && j == 0) ? T(0) : v / (lk + lx[j]); });
}

template <typename T>
__global__ void __launch_bounds__(kRbRowThreads)
k_rb_inverse_s(const T *F, const T *cz, const T *cx, T *phi, int nx, int nz)
{
    extern __shared__ __align__(16) unsigned char rb_smem[];
    T *part = reinterpret_cast<T *>(rb_smem), *R = part + kRbRowThreads;
    T *sF = R + rb_pad<T>(nx), *sC = sF + rb_pad<T>((int64_t)nz * nx);
    rb_stage(sF, F, (int64_t)nz * nx);
    rb_stage(sC, cx, (int64_t)nx * nx);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int m = blockIdx.x;
    rb_vecmat(cz + m, nz, sF, nx, nz, nx, part, [&](int j, T v) { R[j] = v; });
    T *pm = phi + (int64_t)m * nx;
    rb_vecmat(R, 1, sC, nx, nx, nx, part, [&](int i, T v) { pm[i] = v; });
}

// Shared memory of the staged transforms, and the largest the box uses them for.
template <typename T>
size_t rb_staged_smem(int nx, int nz)
{
    return sizeof(T) * (size_t)(kRbRowThreads + rb_pad<T>(nx) + rb_pad<T>((int64_t)nz * nx) + (int64_t)nx * nx);
}
constexpr size_t kRbStagedMax = 96 * 1024;

// Projection: cells take the average of their two faces' gradient corrections
// (face gradient (phi_{i+1} - phi_i) / dx inside, zero on the walls); the
// result is the new u, w with their ghost images.
template <typename T>
__global__ void k_rb_project(const T *u2, const T *w2, const T *phi, T *u, T *w, int nx, int nz, T idx, T idz)
{
    const int px = rb_px(nx);
    const int n = nx * nz;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int k = c / nx, i = c - (c / nx) * nx;
        const int64_t o = (int64_t)(k + RBG) * px + i + RBG;
        const T ge = i + 1 < nx ? (phi[c + 1] - phi[c]) * idx : T(0);
        const T gw = i > 0 ? (phi[c] - phi[c - 1]) * idx : T(0);
        const T gn = k + 1 < nz ? (phi[c + nx] - phi[c]) * idz : T(0);
        const T gs = k > 0 ? (phi[c] - phi[c - nx]) * idz : T(0);
        store_mirrored(u, k, i, u2[o] - T(0.5) * (gw + ge), nx, nz, T(-1), T(-1));
        store_mirrored(w, k, i, w2[o] - T(0.5) * (gs + gn), nx, nz, T(-1), T(-1));
    }
}

// interior <-> padded copies
template <typename T>
__global__ void k_rb_copy(const T *src, T *dst, int nx, int nz, bool to_padded)
{
    const int px = rb_px(nx);
    const int n = nx * nz;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int k = c / nx, i = c - (c / nx) * nx;
        const int64_t o = (int64_t)(k + RBG) * px + i + RBG;
        if (to_padded)
            dst[o] = src[c];
        else
            dst[c] = src[o];
    }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// Threads per CTA for the per-cell kernels: FP64 arithmetic is scarce per SM,
// so small boxes spread over as many SMs as the device has before CTAs grow.
int cell_block(int64_t n, int sms)
{
    int b = 32;
    while (b < 256 && (n + b - 1) / b > 4 * sms) b *= 2;
    return b;
}
int cell_grid(int64_t n, int b) { return (int)std::min<int64_t>((n + b - 1) / b, 4096); }

}  // namespace
}  // namespace sl

using namespace sl;

struct sl_rb {
    int device = -1, sms = 1;
    bool staged = false;   // transforms with staged operands (small boxes)
    int nx = 0, nz = 0, scheme = SL_CEC, dtype = SL_F64;
    double Lx = 2.0, Lz = 1.0, Ra = 0.0, Pr = 1.0;
    int64_t step = 0;
    size_t esz = 8;
    int64_t plane = 0;     // padded plane: rb_px(nx) (nz + 2G) elements
    int cur = 0;           // which of the two state buffers holds step n
    void *mem = nullptr;   // one device allocation
    // padded planes: two states (u, w, theta back to back, so that (u, w) is
    // the velocity argument of the advection), the advected fields, (u2, w2)
    void *S[2] = {nullptr, nullptr}, *A = nullptr, *W = nullptr;
    // interior arrays (nz x nx): the face divergence D, its transform F, phi
    void *d = nullptr, *F = nullptr, *phi = nullptr;
    // orthonormal DCT-II matrices C_x (and its transpose), C_z; eigenvalues per axis
    void *cx = nullptr, *cxT = nullptr, *cz = nullptr, *lx = nullptr, *lz = nullptr;
    int *signs = nullptr;   // sx of (u, w, theta), then sz of (u, w, theta)
    // long runs replay kRbGraphSteps steps from one CUDA graph, captured for
    // one dt and one starting buffer on a stream of the box's own
    cudaStream_t cs = nullptr;
    cudaGraphExec_t exec = nullptr;
    double graph_dt = 0.0;
    int graph_cur = -1;
};

namespace {

template <typename T>
int rb_step_t(sl_rb *r, double dt, int nsteps, cudaStream_t st)
{
    const int nx = r->nx, nz = r->nz, n = nx * nz;
    const int px = rb_px(nx), pz = nz + 2 * RBG;
    const int64_t P = r->plane;
    T *A = static_cast<T *>(r->A), *Wk = static_cast<T *>(r->W);
    T *d = static_cast<T *>(r->d), *F = static_cast<T *>(r->F), *phi = static_cast<T *>(r->phi);
    const T *cx = static_cast<const T *>(r->cx), *cxT = static_cast<const T *>(r->cxT);
    const T *cz = static_cast<const T *>(r->cz);
    const T *lx = static_cast<const T *>(r->lx), *lz = static_cast<const T *>(r->lz);
    const double dx = r->Lx / nx, dz = r->Lz / nz;
    const int64_t pdims[3] = {px, pz, 1};
    const double sp[3] = {dx, dz, 1.0};
    const int cbk = cell_block(n, r->sms), cgr = cell_grid(n, cbk);
    const size_t rsm = sizeof(T) * (kRbRowThreads + nx), ssm = rb_staged_smem<T>(nx, nz);
    for (int s = 0; s < nsteps; ++s) {
        // S0 holds step n with its ghost layers (the walls' mirror images)
        T *S0 = static_cast<T *>(r->S[r->cur]), *S1 = static_cast<T *>(r->S[r->cur ^ 1]);
        // semi-Lagrangian advection of u, w, theta by U^n on the padded box;
        // CEC alternates its sweep order with the step index
        const void *ins[3] = {S0, S0 + P, S0 + 2 * P};
        void *outs[3] = {A, A + P, A + 2 * P};
        int rc = sl_advect_multi(outs, ins, 3, S0, 2, pdims, sp, dt, r->scheme, r->dtype, (int)(r->step & 1), st);
        if (rc) return rc;
        // forces: u2, w2 into the work planes, theta' (with ghosts) into the
        // next state, the face divergence D into d
        k_rb_forces<T><<<cgr, cbk, 0, st>>>(S0, S0 + P, S0 + 2 * P, A, A + P, A + 2 * P, Wk, Wk + P, S1 + 2 * P, d, nx,
                                            nz, T(dt), T(r->Ra), T(r->Pr), T(1.0 / (dx * dx)), T(1.0 / (dz * dz)),
                                            T(1.0 / dx), T(1.0 / dz));
        // phi = C_z^T [(C_z D C_x^T) / lam] C_x
        if (r->staged) {
            k_rb_forward_s<T><<<nz, kRbRowThreads, ssm, st>>>(d, cz, cxT, lx, lz, F, nx, nz);
            k_rb_inverse_s<T><<<nz, kRbRowThreads, ssm, st>>>(F, cz, cx, phi, nx, nz);
        } else {
            k_rb_forward<T><<<nz, kRbRowThreads, rsm, st>>>(d, cz, cxT, lx, lz, F, nx, nz);
            k_rb_inverse<T><<<nz, kRbRowThreads, rsm, st>>>(F, cz, cx, phi, nx, nz);
        }
        // the projected u, w (with ghosts) of the next state
        k_rb_project<T><<<cgr, cbk, 0, st>>>(Wk, Wk + P, phi, S1, S1 + P, nx, nz, T(1.0 / dx), T(1.0 / dz));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
        r->cur ^= 1;
        ++r->step;
    }
    return SL_OK;
}

template <typename T>
int rb_copy_t(sl_rb *r, const void *u, const void *w, const void *t, void *ou, void *ow, void *ot, cudaStream_t st)
{
    const int cb = blocks_for((int64_t)r->nx * r->nz);
    T *S = static_cast<T *>(r->S[r->cur]);
    const int64_t P = r->plane;
    if (u) {
        k_rb_copy<T><<<cb, 256, 0, st>>>(static_cast<const T *>(u), S, r->nx, r->nz, true);
        k_rb_copy<T><<<cb, 256, 0, st>>>(static_cast<const T *>(w), S + P, r->nx, r->nz, true);
        k_rb_copy<T><<<cb, 256, 0, st>>>(static_cast<const T *>(t), S + 2 * P, r->nx, r->nz, true);
        k_rb_ghosts<T><<<blocks_for(3 * P), 256, 0, st>>>(S, 3, r->nx, r->nz, P, r->signs, r->signs + 3);
    } else {
        k_rb_copy<T><<<cb, 256, 0, st>>>(S, static_cast<T *>(ou), r->nx, r->nz, false);
        k_rb_copy<T><<<cb, 256, 0, st>>>(S + P, static_cast<T *>(ow), r->nx, r->nz, false);
        k_rb_copy<T><<<cb, 256, 0, st>>>(S + 2 * P, static_cast<T *>(ot), r->nx, r->nz, false);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SL_OK : set_error(SL_ERR_CUDA, cudaGetErrorString(e));
}

constexpr int kRbGraphSteps = 8;   // even: the graph ends on the buffer and sweep order it starts on

int rb_eager(sl_rb *r, double dt, int nsteps, cudaStream_t st)
{
    return r->dtype == SL_F64 ? rb_step_t<double>(r, dt, nsteps, st) : rb_step_t<float>(r, dt, nsteps, st);
}

// The graph of kRbGraphSteps steps from the current buffer with this dt
// (captured again when either differs from the cached graph's).
int rb_graph(sl_rb *r, double dt)
{
    if (r->exec && r->graph_dt == dt && r->graph_cur == r->cur) return SL_OK;
    if (r->exec) {
        cudaGraphExecDestroy(r->exec);
        r->exec = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!r->cs) e = cudaStreamCreateWithFlags(&r->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    const int cur0 = r->cur;
    const int64_t step0 = r->step;
    e = cudaStreamBeginCapture(r->cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    const int rc = rb_eager(r, dt, kRbGraphSteps, r->cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(r->cs, &g);
    r->cur = cur0;   // nothing ran yet
    r->step = step0;
    if (rc != SL_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != SL_OK ? rc : set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&r->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        r->exec = nullptr;
        return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    }
    r->graph_dt = dt;
    r->graph_cur = cur0;
    return SL_OK;
}

// orthonormal DCT-II matrix, row j: s_j cos(pi j (i + 1/2) / n)
void dct_matrix(std::vector<double> &c, int n)
{
    c.resize((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            c[(size_t)j * n + i] = std::sqrt((j == 0 ? 1.0 : 2.0) / n) * std::cos(M_PI * j * (i + 0.5) / n);
}

}  // namespace

extern "C" {

int sl_rb_create(sl_rb **out, int nx, int nz, double Lx, double Lz, double Ra, double Pr, int scheme, int dtype)
{
    if (!out) return set_error(SL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 4 || nz < 4 || nx > 4096 || nz > 4096) return set_error(SL_ERR_ARG, "nx and nz must be in [4, 4096]");
    if (!(Lx > 0) || !(Lz > 0) || !std::isfinite(Lx) || !std::isfinite(Lz) || !std::isfinite(Ra) ||
        !std::isfinite(Pr) || Pr < 0)
        return set_error(SL_ERR_ARG, "Lx, Lz must be > 0; Ra, Pr finite, Pr >= 0");
    if (scheme < SL_CIR || scheme > SL_CEC) return set_error(SL_ERR_ARG, "unknown scheme");
    if (dtype != SL_F32 && dtype != SL_F64) return set_error(SL_ERR_UNSUPPORTED, "the box runs in SL_F32 or SL_F64");
    DevCtx *c = ctx_get();
    if (!c) return set_error(SL_ERR_CUDA, "could not create the device context");
    sl_rb *r = new (std::nothrow) sl_rb();
    if (!r) return set_error(SL_ERR_NOMEM, "host allocation");
    r->device = c->device;
    r->sms = c->num_sms > 0 ? c->num_sms : 1;
    r->nx = nx;
    r->nz = nz;
    r->Lx = Lx;
    r->Lz = Lz;
    r->Ra = Ra;
    r->Pr = Pr;
    r->scheme = scheme;
    r->dtype = dtype;
    r->esz = dtype == SL_F64 ? 8 : 4;
    // the planes of one state are contiguous (the advection's velocity is
    // (u, w)); every buffer starts on a 512-byte boundary
    r->plane = (int64_t)rb_px(nx) * (nz + 2 * RBG);
    auto round64 = [](int64_t k) { return (k + 63) / 64 * 64; };
    const int64_t n = (int64_t)nx * nz;
    const int64_t elems = 4 * round64(3 * r->plane) + 3 * round64(n) + 2 * round64((int64_t)nx * nx) +
                          round64((int64_t)nz * nz) + round64(nx) + round64(nz) + 64;
    if (cudaMalloc(&r->mem, r->esz * elems) != cudaSuccess) {
        delete r;
        return set_error(SL_ERR_NOMEM, "device buffers of the box");
    }
    char *p = static_cast<char *>(r->mem);
    auto take = [&](int64_t k) {
        void *q = p;
        p += r->esz * round64(k);
        return q;
    };
    r->S[0] = take(3 * r->plane);
    r->S[1] = take(3 * r->plane);
    r->A = take(3 * r->plane);
    r->W = take(3 * r->plane);
    r->d = take(n);
    r->F = take(n);
    r->phi = take(n);
    r->cx = take((int64_t)nx * nx);
    r->cxT = take((int64_t)nx * nx);
    r->cz = take((int64_t)nz * nz);
    r->lx = take(nx);
    r->lz = take(nz);
    r->signs = reinterpret_cast<int *>(p);
    std::vector<double> cxm, czm, cxt((size_t)nx * nx), lxv(nx), lzv(nz);
    dct_matrix(cxm, nx);
    for (int j = 0; j < nx; ++j)
        for (int i = 0; i < nx; ++i) cxt[(size_t)i * nx + j] = cxm[(size_t)j * nx + i];
    dct_matrix(czm, nz);
    const double dx = Lx / nx, dz = Lz / nz;
    for (int j = 0; j < nx; ++j) lxv[j] = -4.0 / (dx * dx) * std::pow(std::sin(M_PI * j / (2.0 * nx)), 2);
    for (int k = 0; k < nz; ++k) lzv[k] = -4.0 / (dz * dz) * std::pow(std::sin(M_PI * k / (2.0 * nz)), 2);
    const int signs[6] = {-1, -1, 1, -1, -1, -1};   // sx of u, w, theta; sz of u, w, theta
    cudaError_t e = cudaMemset(r->mem, 0, r->esz * elems);
    auto up = [&](void *dst, const std::vector<double> &v) {
        if (e != cudaSuccess) return;
        if (dtype == SL_F64) {
            e = cudaMemcpy(dst, v.data(), 8 * v.size(), cudaMemcpyHostToDevice);
        } else {
            const std::vector<float> f(v.begin(), v.end());
            e = cudaMemcpy(dst, f.data(), 4 * f.size(), cudaMemcpyHostToDevice);
        }
    };
    up(r->cx, cxm);
    up(r->cxT, cxt);
    up(r->cz, czm);
    up(r->lx, lxv);
    up(r->lz, lzv);
    if (e == cudaSuccess) e = cudaMemcpy(r->signs, signs, sizeof signs, cudaMemcpyHostToDevice);
    // small boxes stage the transforms' matrix operands in shared memory; the
    // kernels' limit is per function, not per box, so it is raised to the cap
    // that every staged box fits under
    const size_t ssm = dtype == SL_F64 ? rb_staged_smem<double>(nx, nz) : rb_staged_smem<float>(nx, nz);
    if (e == cudaSuccess && ssm <= kRbStagedMax) {
        const int cap = (int)kRbStagedMax;
        if (dtype == SL_F64) {
            e = cudaFuncSetAttribute(k_rb_forward_s<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_rb_inverse_s<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        } else {
            e = cudaFuncSetAttribute(k_rb_forward_s<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_rb_inverse_s<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        }
        r->staged = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        cudaFree(r->mem);
        delete r;
        return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = r;
    return SL_OK;
}

int sl_rb_set_state(sl_rb *r, const void *u, const void *w, const void *theta, void *stream)
{
    if (!r || !u || !w || !theta) return set_error(SL_ERR_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    r->step = 0;
    return r->dtype == SL_F64 ? rb_copy_t<double>(r, u, w, theta, nullptr, nullptr, nullptr, st)
                              : rb_copy_t<float>(r, u, w, theta, nullptr, nullptr, nullptr, st);
}

int sl_rb_get_state(sl_rb *r, void *u, void *w, void *theta, void *stream)
{
    if (!r || !u || !w || !theta) return set_error(SL_ERR_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return r->dtype == SL_F64 ? rb_copy_t<double>(r, nullptr, nullptr, nullptr, u, w, theta, st)
                              : rb_copy_t<float>(r, nullptr, nullptr, nullptr, u, w, theta, st);
}

int sl_rb_step(sl_rb *r, double dt, int nsteps, void *stream)
{
    if (!r || nsteps < 0 || !std::isfinite(dt)) return set_error(SL_ERR_ARG, "bad argument");
    DevCtx *c = ctx_get();
    if (!c || c->device != r->device) return set_error(SL_ERR_ARG, "the box belongs to another device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int left = nsteps, rc = SL_OK;
    if (left >= 2 * kRbGraphSteps) {
        if (r->step & 1) {   // graphs start on an even step (CEC's x-first sweep)
            rc = rb_eager(r, dt, 1, st);
            if (rc) return rc;
            --left;
        }
        rc = rb_graph(r, dt);
        if (rc) return rc;
        for (; left >= kRbGraphSteps; left -= kRbGraphSteps) {
            const cudaError_t e = cudaGraphLaunch(r->exec, st);
            if (e != cudaSuccess) return set_error(SL_ERR_CUDA, cudaGetErrorString(e));
            r->step += kRbGraphSteps;
        }
    }
    return left ? rb_eager(r, dt, left, st) : SL_OK;
}

int sl_rb_destroy(sl_rb *r)
{
    if (!r) return SL_OK;
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->cs) cudaStreamDestroy(r->cs);
    if (r->mem) cudaFree(r->mem);
    delete r;
    return SL_OK;
}

}  // extern "C"
