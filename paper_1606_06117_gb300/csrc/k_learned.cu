// k_learned.cu -- learned one-pass corrector: a 67 -> 64 -> 64 -> 1 MLP that
// maps each cell's 4 x 4 x 4 upwind neighbourhood and its fractional departure
// offsets to the third-order correction, so that one step is
//     Phi_new = L_U[Phi] + s * MLP(features),
// with L_U the multilinear (CIR) value at the departure point (Sec. 3, eq.
// CIR2D) and the target of training the combined scheme of eqs. intro:CEC /
// intro:CECcoef.  No counterpart in the paper: a throughput form whose error
// is judged against the plain scheme.
//
// Features of cell i (index space, |C| <= 1): X_d = i_d - C_d, base
// b_d = min(floor(X_d), i_d), f_d = X_d - b_d in [0, 1]; the 64 values
// Phi(b + (a, b', c)), a, b', c in {-1, 0, 1, 2} (x fastest); m = the trilinear
// value of the inner 2 x 2 x 2 at f (= CIR); s = max |Phi_k - m| (floored);
// inputs x_k = (Phi_k - m)/s, x_{64+d} = f_d - 1/2; output Phi_new = m + s y.
//
// Kernels: feature extraction for training samples, an FP32 minibatch
// forward/backward kernel with an Adam update, and the inference step whose
// two GEMMs run on the tensor cores (tcgen05.mma, BF16 operands staged in
// shared memory, FP32 accumulators in tensor memory).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <random>
#include <vector>

#include "sl.h"
#include "sl_internal.h"

namespace sl {
namespace lrn {

constexpr int NIN = 67, KP1 = 80, NH = 64;   // inputs, padded K of layer 1, hidden width
constexpr int NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1;   // 8577
// offsets of the parameters in the FP32 parameter vector
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH, O_W3 = O_B2 + NH,
              O_B3 = O_W3 + NH;

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

// three-input max / min (one instruction each on sm_100 and later)
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------------- features
// Computes the 67 inputs, the CIR value m and the scale s of one cell from a
// periodic field; phi is read through `at(x, y, z)` (wrapped by the caller).
template <typename At>
__device__ __forceinline__ void cell_features(At at, int x, int y, int z, float cx, float cy, float cz,
                                              float (&feat)[NIN], float &m, float &s)
{
    const float X[3] = {x - cx, y - cy, z - cz};
    const int I[3] = {x, y, z};
    int b[3];
    float f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int fl = (int)floorf(X[d]);
        if (fl > I[d]) fl = I[d];
        b[d] = fl;
        f[d] = X[d] - (float)fl;
    }
    float v[64];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb)
#pragma unroll
            for (int a = 0; a < 4; ++a) v[a + 4 * bb + 16 * c] = at(b[0] - 1 + a, b[1] - 1 + bb, b[2] - 1 + c);
    // trilinear value of the inner cube (indices 1, 2 on each axis)
    float e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {   // (y, z) pairs of the inner cube
        const int yy = 1 + (q & 1), zz = 1 + (q >> 1);
        const float lo = v[1 + 4 * yy + 16 * zz], hi = v[2 + 4 * yy + 16 * zz];
        e[q] = lo + f[0] * (hi - lo);
    }
    const float g0 = e[0] + f[1] * (e[1] - e[0]);
    const float g1 = e[2] + f[1] * (e[3] - e[2]);
    m = g0 + f[2] * (g1 - g0);
    // max |v_k - m| = max(max v - m, m - min v): rounding is monotonic, so this
    // is exactly the largest rounded difference; four chains each for ILP
    float hi[4], lo[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {   // chain c: v[c], v[c + 4], ..., v[c + 60]
        hi[c] = lo[c] = v[c + 60];
#pragma unroll
        for (int k = c; k < 60; k += 8) {
            hi[c] = max3f(hi[c], v[k], v[k + 4]);
            lo[c] = min3f(lo[c], v[k], v[k + 4]);
        }
    }
    const float vmax = fmaxf(fmaxf(hi[0], hi[1]), fmaxf(hi[2], hi[3]));
    const float vmin = fminf(fminf(lo[0], lo[1]), fminf(lo[2], lo[3]));
    s = fmaxf(fmaxf(vmax - m, m - vmin), 1e-30f);
    const float inv = 1.f / s;
    // feat = (v - m) / s as v inv - m inv, two cells' worth per packed FFMA2
    const float2 inv2 = make_float2(inv, inv), nm2 = make_float2(-m * inv, -m * inv);
#pragma unroll
    for (int k = 0; k < 64; k += 2) {
        const float2 r = __ffma2_rn(make_float2(v[k], v[k + 1]), inv2, nm2);
        feat[k] = r.x;
        feat[k + 1] = r.y;
    }
    feat[64] = f[0] - 0.5f;
    feat[65] = f[1] - 0.5f;
    feat[66] = f[2] - 0.5f;
}

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Training samples at pseudo-random cells: rows of 68 floats (67 inputs, target
// y = (target_field - m) / s).
__global__ void k_samples(const float *__restrict__ phi, const float *__restrict__ target,
                          const float *__restrict__ vel, int nx, int ny, int nz, float sx, float sy, float sz,
                          int nsamples, uint32_t seed, float *__restrict__ rows)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nsamples) return;
    const int64_t plane = (int64_t)nx * ny, ncell = plane * nz;
    const uint32_t h = hash32(seed * 0x9E3779B9u + (uint32_t)j);
    const int64_t cell = (int64_t)(((uint64_t)h * (uint64_t)hash32(h ^ 0x5bd1e995u)) % (uint64_t)ncell);
    const int z = (int)(cell / plane), y = (int)((cell / nx) % ny), x = (int)(cell % nx);
    auto at = [&](int xx, int yy, int zz) {
        return phi[(int64_t)wrapc(zz, nz) * plane + (int64_t)wrapc(yy, ny) * nx + wrapc(xx, nx)];
    };
    float feat[NIN], m, s;
    cell_features(at, x, y, z, vel[cell] * sx, vel[ncell + cell] * sy, vel[2 * ncell + cell] * sz, feat, m, s);
    float *r = rows + (int64_t)j * 68;
#pragma unroll
    for (int k = 0; k < NIN; ++k) r[k] = feat[k];
    r[67] = (target[cell] - m) / s;
}

// --------------------------------------------------------------- training
// One minibatch: each CTA takes SB samples, runs forward and backward in FP32
// and adds its parameter gradients (and squared-error sum) into grad/loss.
constexpr int SB = 64, TT = 256;

__global__ void __launch_bounds__(TT) k_train(const float *__restrict__ params, const float *__restrict__ rows,
                                              int nrows, int batch, uint32_t seed, float *__restrict__ grad,
                                              float *__restrict__ loss)
{
    extern __shared__ __align__(16) float sm[];
    float *W = sm;                         // parameters, NPARAM
    float *X = W + ((NPARAM + 3) & ~3);    // SB x 68
    float *H1 = X + SB * 68;               // SB x NH
    float *H2 = H1 + SB * NH;
    float *D2 = H2 + SB * NH;              // dL/d(pre-activation 2)
    float *D1 = D2 + SB * NH;              // dL/d(pre-activation 1)
    float *DY = D1 + SB * NH;              // SB
    const int tid = threadIdx.x;
    for (int i = tid; i < NPARAM; i += TT) W[i] = params[i];
    const int s0 = blockIdx.x * SB;
    for (int i = tid; i < SB * 68; i += TT) {
        const int sidx = s0 + i / 68;
        float v = 0.f;
        if (sidx < batch) {
            const uint32_t r = hash32(seed * 0x85ebca6bu + (uint32_t)sidx) % (uint32_t)nrows;
            v = rows[(int64_t)r * 68 + i % 68];
        }
        X[i] = v;
    }
    __syncthreads();
    // layer 1
    for (int i = tid; i < SB * NH; i += TT) {
        const int s = i / NH, j = i % NH;
        float a = W[O_B1 + j];
        const float *w = W + O_W1 + j * NIN;
        const float *x = X + s * 68;
        for (int k = 0; k < NIN; ++k) a += w[k] * x[k];
        H1[i] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int i = tid; i < SB * NH; i += TT) {
        const int s = i / NH, j = i % NH;
        float a = W[O_B2 + j];
        const float *w = W + O_W2 + j * NH;
        const float *h = H1 + s * NH;
        for (int k = 0; k < NH; ++k) a += w[k] * h[k];
        H2[i] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (tid < SB) {
        float y = W[O_B3];
        for (int k = 0; k < NH; ++k) y += W[O_W3 + k] * H2[tid * NH + k];
        const bool valid = s0 + tid < batch;
        const float e = valid ? y - X[tid * 68 + 67] : 0.f;
        DY[tid] = 2.f * e / (float)batch;
        atomicAdd(loss, e * e);
    }
    __syncthreads();
    for (int i = tid; i < SB * NH; i += TT) {
        const int s = i / NH, j = i % NH;
        D2[i] = H2[i] > 0.f ? DY[s] * W[O_W3 + j] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < SB * NH; i += TT) {
        const int s = i / NH, k = i % NH;
        float a = 0.f;
        for (int j = 0; j < NH; ++j) a += D2[s * NH + j] * W[O_W2 + j * NH + k];
        D1[i] = H1[i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients summed over the CTA's samples
    for (int p = tid; p < NPARAM; p += TT) {
        float g = 0.f;
        if (p < O_B1) {
            const int j = p / NIN, k = p % NIN;
            for (int s = 0; s < SB; ++s) g += D1[s * NH + j] * X[s * 68 + k];
        } else if (p < O_W2) {
            const int j = p - O_B1;
            for (int s = 0; s < SB; ++s) g += D1[s * NH + j];
        } else if (p < O_B2) {
            const int j = (p - O_W2) / NH, k = (p - O_W2) % NH;
            for (int s = 0; s < SB; ++s) g += D2[s * NH + j] * H1[s * NH + k];
        } else if (p < O_W3) {
            const int j = p - O_B2;
            for (int s = 0; s < SB; ++s) g += D2[s * NH + j];
        } else if (p < O_B3) {
            const int j = p - O_W3;
            for (int s = 0; s < SB; ++s) g += DY[s] * H2[s * NH + j];
        } else {
            for (int s = 0; s < SB; ++s) g += DY[s];
        }
        atomicAdd(grad + p, g);
    }
}

// Adam step on the FP32 parameters; clears the gradient.
__global__ void k_adam(float *__restrict__ params, float *__restrict__ grad, float *__restrict__ mom,
                       float *__restrict__ var, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i];
    const float m = b1 * mom[i] + (1.f - b1) * g;
    const float v = b2 * var[i] + (1.f - b2) * g * g;
    mom[i] = m;
    var[i] = v;
    params[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    grad[i] = 0.f;
}

// ------------------------------------------------- inference (tensor cores)
// Shared-memory operand layout (no swizzle, K-major): 8 x 16-byte core
// matrices; the core matrix of rows [8r, 8r+8) and K elements [8k, 8k+8) sits
// at ((k * RG + r) * 128) bytes, RG = rows / 8.  Hence the byte distance
// between core matrices adjacent along K ("leading") is RG * 128 and along
// M/N ("stride") is 128.
__device__ __forceinline__ uint32_t core_off(int row, int kg, int rg) { return (uint32_t)((kg * rg + row / 8) * 128 + (row % 8) * 16); }

__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // start >> 4 in bits 0-13, leading offset >> 4 in 16-29, stride offset >> 4
    // in 32-45, descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0)
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4)                          // D format: F32
           | (1u << 7)                        // A format: BF16
           | (1u << 10)                       // B format: BF16
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init1(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned it = 0; it < (1u << 20); ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 32 lanes x 32 consecutive TMEM columns into v[0..32) (this thread's lane).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// pack_bf16(max(a, 0), max(b, 0)) in one conversion (rounding and the clamp at
// zero commute, so the result is the same)
__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

constexpr int MT = 128;                      // cells per tile (MMA M)
constexpr int BX = 32, BY = 4;               // tile = 32 x 4 cells of one plane
constexpr int HX = BX + 8, HY = BY + 4, HZ = 5;   // staged block: x halo 4 (16-byte chunks), y, z halo 2
constexpr int CPR = HX / 4;                         // 16-byte chunks per staged row
constexpr int A1_BYTES = MT * KP1 * 2, A2_BYTES = MT * NH * 2;
constexpr int W1_BYTES = NH * KP1 * 2, W2_BYTES = NH * NH * 2;
constexpr int BLK_FLOATS = HX * HY * HZ;
// layout of the dynamic shared memory (bytes); about 54 KB, so four CTAs fit on
// an SM and take all 512 of its tensor-memory columns.  The layer-2 operand A2
// reuses A1's space: layer 1's MMA has finished reading A1 (its commit was
// waited for) before epilogue 1 writes A2, and layer 2's MMA has finished
// before the next tile's features are written to A1.
constexpr int CTAS_PER_SM = 4;
static_assert(CTAS_PER_SM * 128 <= 512, "tensor-memory columns of the resident CTAs");
static_assert(A2_BYTES <= A1_BYTES, "A2 fits in A1's space");
constexpr int S_A1 = 0, S_A2 = S_A1, S_W1 = S_A1 + A1_BYTES, S_W2 = S_W1 + W1_BYTES;
constexpr int S_F = S_W2 + W2_BYTES;                          // FP32: b1, b2, w3, b3
constexpr int STAGE_FLOATS = BLK_FLOATS + 3 * MT;              // Phi block + the tile's three u components
constexpr int S_BLK = S_F + 4 * (3 * NH + 4);                  // two stages (double buffer)
constexpr int S_BAR = S_BLK + 2 * 4 * STAGE_FLOATS;
constexpr int S_TM = S_BAR + 16;
constexpr int SMEM_BYTES = S_TM + 16;
// a fifth resident CTA would wait forever for tensor-memory columns; its shared
// memory (with the 1 KB per-CTA reserve) cannot fit in the SM's 228 KB
static_assert((CTAS_PER_SM + 1) * (SMEM_BYTES + 1024) > 228 * 1024, "at most CTAS_PER_SM resident CTAs");

// One learned step over the grid; persistent CTAs of 128 threads (4 warps),
// one cell per thread per tile.  wb points at the BF16 operand images of W1
// and W2 (already in the core-matrix layout) followed by b1, b2, w3, b3 in FP32.
__global__ void __launch_bounds__(MT) k_learned_step(const float *__restrict__ phi, float *__restrict__ out,
                                                     const float *__restrict__ vel, int nx, int ny, int nz,
                                                     float sx, float sy, float sz,
                                                     const unsigned char *__restrict__ wb, unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S_BAR);
    uint32_t *tm_slot = reinterpret_cast<uint32_t *>(smem + S_TM);
    float *fw = reinterpret_cast<float *>(smem + S_F);
    float *blk = reinterpret_cast<float *>(smem + S_BLK);
    const int64_t plane = (int64_t)nx * ny, ncell = plane * nz;

    // weights once per CTA (operand images are copied verbatim)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(wb);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + S_W1);
        for (int i = tid; i < (W1_BYTES + W2_BYTES) / 16; i += MT) dst[i] = src[i];
        const float *fsrc = reinterpret_cast<const float *>(wb + W1_BYTES + W2_BYTES);
        for (int i = tid; i < 3 * NH + 1; i += MT) fw[i] = fsrc[i];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(tm_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) mbar_init1(bar);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tm_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = instr_desc(MT, NH);
    const uint32_t a1 = smem_u32(smem + S_A1), a2 = smem_u32(smem + S_A2);
    const uint32_t w1 = smem_u32(smem + S_W1), w2 = smem_u32(smem + S_W2);
    unsigned phase = 0;
    bool timeout = false;

    const int tiles_x = nx / BX, tiles_y = ny / BY;
    const int64_t ntiles = (int64_t)tiles_x * tiles_y * nz;
    // the Phi block x in [x0-2, x0+34), y in [y0-2, y0+6), z in [z-2, z+3) and
    // the tile's velocity, staged with 4-byte cp.async one tile ahead
    auto issue_block = [&](int64_t tt, int b) {
        const int tx_ = (int)(tt % tiles_x);
        const int ty_ = (int)((tt / tiles_x) % tiles_y);
        const int z_ = (int)(tt / ((int64_t)tiles_x * tiles_y));
        float *dst = blk + b * STAGE_FLOATS;
        // x in [x0-4, x0+36) in 16-byte chunks: nx is a multiple of 32, so a
        // chunk never straddles the periodic seam and every source is aligned
        for (int i = tid; i < BLK_FLOATS / 4; i += MT) {
            const int cx4 = i % CPR, row = i / CPR, by = row % HY, bz = row / HY;
            int gx = tx_ * BX - 4 + 4 * cx4, gy = ty_ * BY - 2 + by, gz = z_ - 2 + bz;   // at most one period away
            gx += gx < 0 ? nx : (gx >= nx ? -nx : 0);
            gy += gy < 0 ? ny : (gy >= ny ? -ny : 0);
            gz += gz < 0 ? nz : (gz >= nz ? -nz : 0);
            cp_async16(dst + 4 * i, phi + (int64_t)gz * plane + (int64_t)gy * nx + gx);
        }
        const int64_t cell_ = (int64_t)z_ * plane + (int64_t)(ty_ * BY + tid / BX) * nx + tx_ * BX + tid % BX;
        cp_async4(dst + BLK_FLOATS + tid, vel + cell_);
        cp_async4(dst + BLK_FLOATS + MT + tid, vel + ncell + cell_);
        cp_async4(dst + BLK_FLOATS + 2 * MT + tid, vel + 2 * ncell + cell_);
        cp_async_commit();
    };
    if ((int64_t)blockIdx.x < ntiles) issue_block(blockIdx.x, 0);
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles && !timeout; t += gridDim.x, ++it) {
        const int tx = (int)(t % tiles_x);
        const int ty = (int)((t / tiles_x) % tiles_y);
        const int z = (int)(t / ((int64_t)tiles_x * tiles_y));
        const int x0 = tx * BX, y0 = ty * BY;
        const float *sb = blk + (it & 1) * STAGE_FLOATS;
        cp_async_wait_all();
        __syncthreads();
        if (t + gridDim.x < ntiles) issue_block(t + gridDim.x, (it & 1) ^ 1);
        // ---- features of this thread's cell -> row tid of A1 (BF16)
        const int cxl = tid % BX, cyl = tid / BX;
        const int64_t cell = (int64_t)z * plane + (int64_t)(y0 + cyl) * nx + x0 + cxl;
        const float cx = sb[BLK_FLOATS + tid] * sx, cy = sb[BLK_FLOATS + MT + tid] * sy,
                    cz = sb[BLK_FLOATS + 2 * MT + tid] * sz;
        if (fabsf(cx) > 1.f || fabsf(cy) > 1.f || fabsf(cz) > 1.f) atomicOr(status, 1u);
        const float ccx = fminf(fmaxf(cx, -1.f), 1.f), ccy = fminf(fmaxf(cy, -1.f), 1.f),
                    ccz = fminf(fmaxf(cz, -1.f), 1.f);
        auto at = [&](int xx, int yy, int zz) {
            // xx, yy, zz are global indices within 2 cells of the cell
            return sb[((zz - z + 2) * HY + (yy - y0 + 2)) * HX + (xx - x0 + 4)];
        };
        float feat[NIN], m, s;
        cell_features(at, x0 + cxl, y0 + cyl, z, ccx, ccy, ccz, feat, m, s);
        {
            unsigned char *A = smem + S_A1;
#pragma unroll
            for (int kg = 0; kg < KP1 / 8; ++kg) {
                float q[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) q[e] = (kg * 8 + e < NIN) ? feat[kg * 8 + e] : 0.f;
                uint4 pk = make_uint4(pack_bf16(q[0], q[1]), pack_bf16(q[2], q[3]), pack_bf16(q[4], q[5]),
                                      pack_bf16(q[6], q[7]));
                *reinterpret_cast<uint4 *>(A + core_off(tid, kg, MT / 8)) = pk;
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 1 on the tensor cores: D[0:64) = A1 (128 x 80) * W1^T
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < KP1 / 16; ++k) {
                const uint64_t da = smem_desc(a1 + k * 2 * (MT / 8) * 128, (MT / 8) * 128, 128);
                const uint64_t db = smem_desc(w1 + k * 2 * (NH / 8) * 128, (NH / 8) * 128, 128);
                mma_bf16(tmem, da, db, idesc, k > 0);
            }
            mma_commit(bar);
        }
        if (!mbar_wait_bounded(bar, phase)) timeout = true;
        phase ^= 1u;
        tc_fence_after();
        // ---- epilogue 1: bias, ReLU, BF16 -> A2
        {
            unsigned char *A = smem + S_A2;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float v[32];
                tmem_ld32(lane_base + half * 32, v);
                const float4 *b1v = reinterpret_cast<const float4 *>(fw + half * 32);
#pragma unroll
                for (int kg = 0; kg < 4; ++kg) {
                    const float4 ba = b1v[2 * kg], bb = b1v[2 * kg + 1];
                    const float2 bias[4] = {make_float2(ba.x, ba.y), make_float2(ba.z, ba.w), make_float2(bb.x, bb.y),
                                            make_float2(bb.z, bb.w)};
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {   // bias on pairs (FADD2), ReLU folded into the conversion
                        const float2 h = __fadd2_rn(make_float2(v[kg * 8 + 2 * e], v[kg * 8 + 2 * e + 1]), bias[e]);
                        w[e] = pack_bf16_relu(h.x, h.y);
                    }
                    const uint4 pk = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(A + core_off(tid, half * 4 + kg, MT / 8)) = pk;
                }
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 2: D[64:128) = A2 (128 x 64) * W2^T
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NH / 16; ++k) {
                const uint64_t da = smem_desc(a2 + k * 2 * (MT / 8) * 128, (MT / 8) * 128, 128);
                const uint64_t db = smem_desc(w2 + k * 2 * (NH / 8) * 128, (NH / 8) * 128, 128);
                mma_bf16(tmem + NH, da, db, idesc, k > 0);
            }
            mma_commit(bar);
        }
        if (!mbar_wait_bounded(bar, phase)) timeout = true;
        phase ^= 1u;
        tc_fence_after();
        // ---- epilogue 2: bias, ReLU, output layer, Phi_new = m + s y
        float2 ya01 = make_float2(fw[3 * NH], 0.f), ya23 = make_float2(0.f, 0.f);   // four accumulation chains
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tmem_ld32(lane_base + NH + half * 32, v);
            const float4 *b2v = reinterpret_cast<const float4 *>(fw + NH + half * 32);
            const float4 *w3v = reinterpret_cast<const float4 *>(fw + 2 * NH + half * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                // bias and weight pairs: packed FADD2 / FFMA2, ReLU per lane
                const float4 bb = b2v[q], ww = w3v[q];
                float2 h01 = __fadd2_rn(make_float2(v[4 * q], v[4 * q + 1]), make_float2(bb.x, bb.y));
                float2 h23 = __fadd2_rn(make_float2(v[4 * q + 2], v[4 * q + 3]), make_float2(bb.z, bb.w));
                h01 = make_float2(fmaxf(h01.x, 0.f), fmaxf(h01.y, 0.f));
                h23 = make_float2(fmaxf(h23.x, 0.f), fmaxf(h23.y, 0.f));
                ya01 = __ffma2_rn(h01, make_float2(ww.x, ww.y), ya01);
                ya23 = __ffma2_rn(h23, make_float2(ww.z, ww.w), ya23);
            }
        }
        const float y = (ya01.x + ya01.y) + (ya23.x + ya23.y);
        out[cell] = m + s * y;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        timeout = __syncthreads_or(timeout);
    }
    cp_async_wait_all();   // a block prefetched for a tile that was not run
    if (timeout && tid == 0) atomicOr(status, 2u);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
}

// Failure-detection self-test: waits on an mbarrier that no thread or copy
// ever completes, gives up after `polls` polls like every bounded wait of the
// library, and records SL_DEV_TIMEOUT.  Faults, traps or hangs nothing.
__global__ void k_wait_selftest(unsigned polls, unsigned *status, unsigned *gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init1(&bar);   // expects one arrival that never comes
    __syncthreads();
    bool ok = false;
    for (unsigned it = 0; it < polls && !ok; ++it) {
        unsigned r;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(r)
            : "r"(smem_u32(&bar)), "r"(0u)
            : "memory");
        ok = r != 0;
    }
    if (!ok && threadIdx.x == 0) {
        atomicOr(status, 2u);
        atomicAdd(gave_up, 1u);
    }
}

// FP32 parameters -> the inference weight image: W1 (64 x 80, K zero-padded)
// and W2 (64 x 64) as BF16 K-major core matrices, then b1, b2, w3, b3 in FP32.
__global__ void k_pack(const float *__restrict__ params, unsigned char *__restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(wb);
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(wb + W1_BYTES);
    float *f = reinterpret_cast<float *>(wb + W1_BYTES + W2_BYTES);
    if (i < NH * KP1) {
        const int n = i / KP1, k = i % KP1;
        const float v = k < NIN ? params[O_W1 + n * NIN + k] : 0.f;
        w1[core_off(n, k / 8, NH / 8) / 2 + k % 8] = __float2bfloat16_rn(v);
    }
    if (i < NH * NH) {
        const int n = i / NH, k = i % NH;
        w2[core_off(n, k / 8, NH / 8) / 2 + k % 8] = __float2bfloat16_rn(params[O_W2 + n * NH + k]);
    }
    if (i < NH) {
        f[i] = params[O_B1 + i];
        f[NH + i] = params[O_B2 + i];
        f[2 * NH + i] = params[O_W3 + i];
    }
    if (i == 0) f[3 * NH] = params[O_B3];
}

}  // namespace lrn
}  // namespace sl

// ============================================================== host side
using namespace sl;
using namespace sl::lrn;

struct sl_corrector {
    int device = -1;
    float *params = nullptr;   // NPARAM FP32 (layout: W1 64x67, b1, W2 64x64, b2, w3, b3)
    float *grad = nullptr;
    float *mom = nullptr;
    float *var = nullptr;
    float *loss = nullptr;     // 1 float
    unsigned char *wb = nullptr;   // inference weight image
    float *rows = nullptr;     // training rows, 68 floats each
    int64_t nrows = 0, cap = 0;
    int64_t adam_t = 0;
    void *scratch = nullptr;   // two fields for the checked step
    size_t scratch_bytes = 0;
    bool plain = false;        // sticky fallback to the plain scheme
};

namespace {

int lfail(int code, const char *msg) { return set_error(code, msg); }

bool learned_geometry_ok(int ndim, const int64_t dims[3]) {
    return ndim == 3 && dims[0] % BX == 0 && dims[1] % BY == 0 && dims[2] >= 3 && dims[0] >= 32 && dims[1] >= 4;
}

int pack(sl_corrector *c, cudaStream_t st) {
    k_pack<<<(NH * KP1 + 255) / 256, 256, 0, st>>>(c->params, c->wb);
    return cudaGetLastError() == cudaSuccess ? SL_OK : lfail(SL_ERR_CUDA, "weight packing launch failed");
}

}  // namespace

extern "C" {

int sl_corrector_create(sl_corrector **out, uint64_t seed)
{
    if (!out) return lfail(SL_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    DevCtx *ctx = ctx_get();
    if (!ctx) return lfail(SL_ERR_CUDA, "could not create the device context");
    sl_corrector *c = new (std::nothrow) sl_corrector();
    if (!c) return lfail(SL_ERR_NOMEM, "host allocation");
    c->device = ctx->device;
    const size_t wbytes = W1_BYTES + W2_BYTES + 4 * (3 * NH + 4);
    void *p = nullptr;
    if (cudaMalloc(&p, 4 * (size_t)NPARAM * 4 + 256 + wbytes) != cudaSuccess) {
        delete c;
        return lfail(SL_ERR_NOMEM, "device parameters");
    }
    c->params = static_cast<float *>(p);
    c->grad = c->params + NPARAM;
    c->mom = c->grad + NPARAM;
    c->var = c->mom + NPARAM;
    c->loss = c->var + NPARAM;
    c->wb = reinterpret_cast<unsigned char *>(c->var + NPARAM) + 256;
    // He initialisation, zero biases (host RNG, seeded)
    std::vector<float> h(NPARAM, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int i = 0; i < NH * NIN; ++i) h[O_W1 + i] = nd(rng) * std::sqrt(2.f / NIN);
    for (int i = 0; i < NH * NH; ++i) h[O_W2 + i] = nd(rng) * std::sqrt(2.f / NH);
    for (int i = 0; i < NH; ++i) h[O_W3 + i] = nd(rng) * std::sqrt(1.f / NH);
    cudaError_t e = cudaMemcpy(c->params, h.data(), 4 * NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->grad, 0, 4 * (size_t)NPARAM * 3 + 4);
    if (e != cudaSuccess || pack(c, nullptr) != SL_OK || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(p);
        delete c;
        return lfail(SL_ERR_CUDA, "corrector initialisation");
    }
    *out = c;
    return SL_OK;
}

int sl_corrector_destroy(sl_corrector *c)
{
    if (!c) return SL_OK;
    cudaFree(c->params);
    if (c->rows) cudaFree(c->rows);
    if (c->scratch) cudaFree(c->scratch);
    delete c;
    return SL_OK;
}

int sl_corrector_param_count(void) { return NPARAM; }

int sl_corrector_get_params(sl_corrector *c, float *host, int n)
{
    if (!c || !host || n != NPARAM) return lfail(SL_ERR_ARG, "need the corrector and a buffer of sl_corrector_param_count() floats");
    return cudaMemcpy(host, c->params, 4 * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? SL_OK
                                                                                         : lfail(SL_ERR_CUDA, "copy");
}

int sl_corrector_set_params(sl_corrector *c, const float *host, int n)
{
    if (!c || !host || n != NPARAM) return lfail(SL_ERR_ARG, "need the corrector and sl_corrector_param_count() floats");
    if (cudaMemcpy(c->params, host, 4 * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return lfail(SL_ERR_CUDA, "copy");
    c->plain = false;
    int rc = pack(c, nullptr);
    if (rc) return rc;
    return cudaDeviceSynchronize() == cudaSuccess ? SL_OK : lfail(SL_ERR_CUDA, "weight packing");
}

int sl_corrector_add_samples(sl_corrector *c, const void *phi, const void *target, const void *vel,
                             const int64_t dims[3], const double spacing[3], double dt, int nsamples, uint64_t seed,
                             void *stream)
{
    if (!c || !phi || !target || !vel || !dims || !spacing || nsamples < 1)
        return lfail(SL_ERR_ARG, "NULL argument or nsamples < 1");
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1 || !(spacing[d] > 0.0)) return lfail(SL_ERR_ARG, "bad dims or spacing");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (c->nrows + nsamples > c->cap) {
        const int64_t ncap = std::max<int64_t>(2 * c->cap, c->nrows + nsamples);
        float *nr = nullptr;
        if (cudaMalloc(&nr, (size_t)ncap * 68 * 4) != cudaSuccess) return lfail(SL_ERR_NOMEM, "sample buffer");
        if (c->rows) {
            if (cudaMemcpyAsync(nr, c->rows, (size_t)c->nrows * 68 * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                cudaFree(nr);
                return lfail(SL_ERR_CUDA, "sample copy");
            }
            cudaFree(c->rows);
        }
        c->rows = nr;
        c->cap = ncap;
    }
    k_samples<<<(nsamples + 255) / 256, 256, 0, st>>>(
        static_cast<const float *>(phi), static_cast<const float *>(target), static_cast<const float *>(vel),
        (int)dims[0], (int)dims[1], (int)dims[2], (float)(dt / spacing[0]), (float)(dt / spacing[1]),
        (float)(dt / spacing[2]), nsamples, (uint32_t)(seed ^ (seed >> 32)), c->rows + c->nrows * 68);
    if (cudaGetLastError() != cudaSuccess) return lfail(SL_ERR_CUDA, "sample launch");
    c->nrows += nsamples;
    return SL_OK;
}

int sl_corrector_get_rows(sl_corrector *c, float *host, int64_t first, int64_t n)
{
    if (!c || !host || first < 0 || n < 0 || first + n > c->nrows) return lfail(SL_ERR_ARG, "row range outside the training set");
    if (n == 0) return SL_OK;
    return cudaMemcpy(host, c->rows + first * 68, (size_t)n * 68 * 4, cudaMemcpyDeviceToHost) == cudaSuccess
               ? SL_OK
               : lfail(SL_ERR_CUDA, "copy");
}

int sl_corrector_train(sl_corrector *c, int iters, int batch, float lr, uint64_t seed, float *last_loss, void *stream)
{
    if (!c || iters < 1 || batch < 1 || !(lr > 0.f)) return lfail(SL_ERR_ARG, "bad training arguments");
    if (c->nrows < 1) return lfail(SL_ERR_ARG, "no training samples (sl_corrector_add_samples)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t smem = 4 * (size_t)(((NPARAM + 3) & ~3) + SB * 68 + 4 * SB * NH + SB);
    if (cudaFuncSetAttribute(k_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return lfail(SL_ERR_CUDA, "training kernel shared memory");
    const float b1 = 0.9f, b2 = 0.999f;
    for (int it = 0; it < iters; ++it) {
        ++c->adam_t;
        const float c1 = 1.f - std::pow(b1, (float)c->adam_t), c2 = 1.f - std::pow(b2, (float)c->adam_t);
        if (cudaMemsetAsync(c->loss, 0, 4, st) != cudaSuccess) return lfail(SL_ERR_CUDA, "memset");
        k_train<<<(batch + SB - 1) / SB, TT, smem, st>>>(c->params, c->rows, (int)std::min<int64_t>(c->nrows, 1 << 30),
                                                        batch, (uint32_t)(seed * 2654435761u + it), c->grad, c->loss);
        k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(c->params, c->grad, c->mom, c->var, lr, b1, b2, 1e-8f, c1, c2);
    }
    int rc = pack(c, st);
    if (rc) return rc;
    float l = 0.f;
    if (cudaMemcpyAsync(&l, c->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return lfail(SL_ERR_CUDA, "training");
    if (last_loss) *last_loss = l / (float)batch;
    return SL_OK;
}

int sl_selftest_wait_timeout(unsigned polls, void *stream)
{
    if (polls < 1 || polls > (1u << 20)) return lfail(SL_ERR_ARG, "polls must be in [1, 2^20]");
    DevCtx *ctx = ctx_get();
    if (!ctx) return lfail(SL_ERR_CUDA, "no device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *gave_up = ctx->counters + 255;
    if (cudaMemsetAsync(gave_up, 0, 4, st) != cudaSuccess) return lfail(SL_ERR_CUDA, "memset");
    k_wait_selftest<<<1, 32, 0, st>>>(polls, ctx->status, gave_up);
    unsigned h = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, gave_up, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return lfail(SL_ERR_CUDA, "self-test launch");
    return h == 1 ? SL_ERR_TIMEOUT : lfail(SL_ERR_CUDA, "the self-test wait completed unexpectedly");
}

int sl_corrector_reset(sl_corrector *c)
{
    if (!c) return lfail(SL_ERR_ARG, "corrector is NULL");
    c->plain = false;
    return SL_OK;
}

int sl_advect_learned(sl_corrector *c, void *out, const void *in, const void *vel, int ndim, const int64_t dims[3],
                      const double spacing[3], double dt, int step_parity, int check, double fallback_ratio,
                      int *used_plain, double errs[2], void *stream)
{
    if (!c || !out || !in || !vel || !dims || !spacing) return lfail(SL_ERR_ARG, "NULL argument");
    if (!learned_geometry_ok(ndim, dims))
        return lfail(SL_ERR_UNSUPPORTED, "learned steps need ndim = 3, dims[0] % 32 == 0, dims[1] % 4 == 0, dims[2] >= 3");
    if (reinterpret_cast<uintptr_t>(in) % 16 != 0)
        return lfail(SL_ERR_UNSUPPORTED, "learned steps need a 16-byte aligned input field");
    for (int d = 0; d < 3; ++d)
        if (!(spacing[d] > 0.0)) return lfail(SL_ERR_ARG, "spacing must be > 0");
    const int64_t n = dims[0] * dims[1] * dims[2];
    const size_t fb = (size_t)n * 4;
    const char *po = static_cast<const char *>(out), *pi = static_cast<const char *>(in);
    if (po < pi + fb && pi < po + fb) return lfail(SL_ERR_ALIAS, "out overlaps in");
    DevCtx *ctx = ctx_get();
    if (!ctx) return lfail(SL_ERR_CUDA, "no device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto learned = [&](void *dst) {
        static int smem_set[64] = {};
        if (!smem_set[ctx->device]) {
            if (cudaFuncSetAttribute(k_learned_step, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess)
                return cudaErrorInvalidValue;
            // all of the SM's unified L1 / shared memory as shared, so four CTAs fit
            if (cudaFuncSetAttribute(k_learned_step, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
                return cudaErrorInvalidValue;
            smem_set[ctx->device] = 1;
        }
        const int64_t tiles = (dims[0] / BX) * (dims[1] / BY) * dims[2];
        int grid = ctx->num_sms * CTAS_PER_SM;   // never more: each CTA holds 128 TMEM columns
        if (grid > tiles) grid = (int)tiles;
        k_learned_step<<<grid, MT, SMEM_BYTES, st>>>(
            static_cast<const float *>(in), static_cast<float *>(dst), static_cast<const float *>(vel), (int)dims[0],
            (int)dims[1], (int)dims[2], (float)(dt / spacing[0]), (float)(dt / spacing[1]), (float)(dt / spacing[2]),
            c->wb, ctx->status);
        return cudaGetLastError();
    };
    if (used_plain) *used_plain = c->plain ? 1 : 0;
    if (!check) {
        if (c->plain) return sl_advect(out, in, vel, ndim, dims, spacing, dt, SL_CEC, SL_F32, step_parity, stream);
        return learned(out) == cudaSuccess ? SL_OK : lfail(SL_ERR_CUDA, "learned step launch");
    }
    // checked step: plain CEC into out, BEC and learned into scratch, compare
    if (c->scratch_bytes < 2 * fb + 256) {
        if (c->scratch) cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
        if (cudaMalloc(&c->scratch, 2 * fb + 256) != cudaSuccess) return lfail(SL_ERR_NOMEM, "check scratch");
        c->scratch_bytes = 2 * fb + 256;
    }
    char *s0 = static_cast<char *>(c->scratch);
    void *bec = s0, *lrn = s0 + ((fb + 255) & ~(size_t)255);
    int rc = sl_advect(out, in, vel, ndim, dims, spacing, dt, SL_CEC, SL_F32, step_parity, stream);
    if (rc) return rc;
    rc = sl_advect(bec, in, vel, ndim, dims, spacing, dt, SL_BEC, SL_F32, step_parity, stream);
    if (rc) return rc;
    if (learned(lrn) != cudaSuccess) return lfail(SL_ERR_CUDA, "learned step launch");
    double nl[3], np[3];
    rc = sl_norms(lrn, out, n, SL_F32, nl, stream);
    if (rc) return rc;
    rc = sl_norms(bec, out, n, SL_F32, np, stream);
    if (rc) return rc;
    if (errs) {
        errs[0] = nl[2];
        errs[1] = np[2];
    }
    if (!c->plain && nl[2] <= fallback_ratio * np[2]) {
        if (cudaMemcpyAsync(out, lrn, fb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return lfail(SL_ERR_CUDA, "copy");
    } else {
        c->plain = true;
    }
    if (used_plain) *used_plain = c->plain ? 1 : 0;
    return SL_OK;
}

}  // extern "C"
