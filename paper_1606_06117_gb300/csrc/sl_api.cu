// sl_api.cu -- the extern "C" entry points of libsl (declared in include/sl.h):
// argument validation, the per-device context, error reporting and dispatch
// to the fused kernels.  No C++ exception crosses these functions.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "sl.h"
#include "sl_internal.h"

namespace sl {
namespace {

thread_local std::string g_err;
std::mutex g_mu;
constexpr int kMaxDev = 64;
DevCtx g_ctx[kMaxDev];

struct Staging {
    void *buf = nullptr;
    size_t bytes = 0;
};
Staging g_stage[kMaxDev];
std::mutex g_host_mu[kMaxDev];   // host-buffer steps of one device share its staging buffer

// z slabs of a host-buffer step: each slab's inputs are copied in, its planes
// stepped and its output copied back on three streams, so that the copies of
// later slabs overlap the kernels and read-back of earlier ones.
constexpr int kMaxSlabs = 8;
constexpr int64_t kMinSlabPlanes = 32;
struct HostPipe {
    bool ready = false;
    cudaStream_t in = nullptr, run = nullptr, back = nullptr;
    cudaEvent_t start = nullptr, copied[kMaxSlabs] = {}, stepped[kMaxSlabs] = {};
    int64_t max_pitch = 0;   // largest row pitch of a 2D copy
};
HostPipe g_pipe[kMaxDev];

void pipe_destroy(HostPipe &p)
{
    for (cudaStream_t *s : {&p.in, &p.run, &p.back})
        if (*s) cudaStreamDestroy(*s);
    if (p.start) cudaEventDestroy(p.start);
    for (int k = 0; k < kMaxSlabs; ++k) {
        if (p.copied[k]) cudaEventDestroy(p.copied[k]);
        if (p.stepped[k]) cudaEventDestroy(p.stepped[k]);
    }
    p = HostPipe();
}

bool pipe_ready(HostPipe &p)
{
    if (p.ready) return true;
    bool ok = true;
    for (cudaStream_t *s : {&p.in, &p.run, &p.back})
        ok = ok && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < kMaxSlabs; ++k)
        ok = cudaEventCreateWithFlags(&p.copied[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.stepped[k], cudaEventDisableTiming) == cudaSuccess;
    int dev = 0, pitch = 0;
    ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&pitch, cudaDevAttrMaxPitch, dev) == cudaSuccess;
    if (!ok) {
        pipe_destroy(p);
        return false;
    }
    p.max_pitch = pitch;
    p.ready = true;
    return true;
}

// autotuned launch shapes per (nx, ny, nz, scheme, dtype)
using TuneKey = std::tuple<int64_t, int64_t, int64_t, int, int>;
std::map<TuneKey, sl_tuning> g_tuned;

bool tuned_get(const int64_t dims[3], int scheme, int dtype, sl_tuning &t)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(TuneKey(dims[0], dims[1], dims[2], scheme, dtype));
    if (it == g_tuned.end()) return false;
    t = it->second;
    return true;
}

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t elem_size(int dtype) { return dtype == SL_F64 ? 8 : 4; }

bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Validates the geometry arguments shared by the step entry points and
// computes Courant scale factors s_d = dt / dx_d.
int check_geometry(int ndim, const int64_t dims[3], const double spacing[3], double dt, int dtype, double s[3])
{
    if (ndim != 2 && ndim != 3) return fail(SL_ERR_ARG, "ndim must be 2 or 3 (got %d)", ndim);
    if (!dims || !spacing) return fail(SL_ERR_ARG, "dims and spacing must not be NULL");
    if (dtype < SL_F32 || dtype > SL_F32_D64) return fail(SL_ERR_ARG, "unknown dtype %d", dtype);
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1 || dims[d] > (int64_t)1 << 30) return fail(SL_ERR_ARG, "dims[%d] = %lld out of range", d, (long long)dims[d]);
    if (ndim == 2 && dims[2] != 1) return fail(SL_ERR_ARG, "dims[2] must be 1 when ndim = 2");
    if (dims[0] * dims[1] > ((int64_t)1 << 31) - 1) return fail(SL_ERR_ARG, "an x-y plane must hold fewer than 2^31 cells");
    if (dims[0] * dims[1] * dims[2] > ((int64_t)1 << 40)) return fail(SL_ERR_ARG, "grid too large");
    if (!std::isfinite(dt)) return fail(SL_ERR_ARG, "dt must be finite");
    for (int d = 0; d < ndim; ++d) {
        if (!(spacing[d] > 0.0) || !std::isfinite(spacing[d])) return fail(SL_ERR_ARG, "spacing[%d] must be > 0", d);
        s[d] = dt / spacing[d];
    }
    if (ndim == 2) s[2] = 0.0;
    return SL_OK;
}

int64_t ncell_of(const int64_t dims[3]) { return dims[0] * dims[1] * dims[2]; }

// The kernel family that serves a request (fixed by the request; the tuner
// only chooses among launch shapes of that family).
int family_of(int scheme, int dtype, int ndim, const int64_t dims[3], bool aligned)
{
    if (scheme == SL_CEC) return fast_eligible(dims, ndim, dtype, aligned) ? SL_KERNEL_CEC_FAST : SL_KERNEL_CEC_SPLIT;
    if (scheme == SL_CIR && cir_fast_eligible(dtype, ndim, dims, aligned)) return SL_KERNEL_CIR_GROUPS;
    return SL_KERNEL_UNSPLIT;
}

// Tile height of a family's launch with no height chosen (the kernels' defaults).
int default_ty(int fam, int dtype)
{
    switch (fam) {
    case SL_KERNEL_CEC_FAST: return 32;
    case SL_KERNEL_CEC_SPLIT: return dtype == SL_F64 ? 16 : 32;
    case SL_KERNEL_CIR_GROUPS: return 16;
    default: return dtype == SL_F64 ? 8 : 16;
    }
}

// The launch shape of a request: the cached choice when it was tuned on the
// family that serves the request, else the family's defaults.
Launch launch_for(int fam, const int64_t dims[3], int scheme, int dtype, bool aligned, const DevCtx *c)
{
    Launch lc;
    lc.aligned = aligned;
    sl_tuning t;
    if (tuned_get(dims, scheme, dtype, t) && t.kernel == fam) {
        lc.tz = t.tile_z;
        lc.ty = t.tile_y;
        lc.grid = t.ctas_per_sm > 0 ? t.ctas_per_sm * c->num_sms : 0;
    }
    return lc;
}

cudaError_t launch_family(int fam, const Launch &lc, void *out, const void *in, const void *vel, int ndim,
                          const int64_t dims[3], const double s[3], int scheme, int dtype, int parity,
                          cudaStream_t st, DevCtx *c, FieldSet fs = FieldSet())
{
    if (fam == SL_KERNEL_CEC_FAST) {
        FastInst one;
        fast_fill(one, in, out, vel, dims, s, 0);
        return launch_cec_fast(one, nullptr, 1, (int64_t)one.ntiles * one.nz, parity, c->status, lc.grid, st);
    }
    if (fam == SL_KERNEL_CEC_SPLIT)
        return launch_split_cec(dtype, in, out, vel, ndim, dims, s, parity, lc, c->status, st, fs);
    return launch_unsplit(dtype, scheme, in, out, vel, ndim, dims, s, lc, c->status, st, fs);
}

int launch_step(void *out, const void *in, const void *vel, int ndim, const int64_t dims[3], const double s[3],
                int scheme, int dtype, int parity, cudaStream_t st, DevCtx *c)
{
    const bool aligned = aligned16(out) && aligned16(in) && aligned16(vel);
    const int fam = family_of(scheme, dtype, ndim, dims, aligned);
    const Launch lc = launch_for(fam, dims, scheme, dtype, aligned, c);
    const cudaError_t e = launch_family(fam, lc, out, in, vel, ndim, dims, s, scheme, dtype, parity, st, c);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SL_OK;
}

}  // namespace

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

DevCtx *ctx_get()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DevCtx &c = g_ctx[dev];
    if (c.device == dev) return &c;
    void *p = nullptr;
    const size_t bytes = 256 + sizeof(double) * (kReduceBlocks + 1) * 4 + 256 * sizeof(unsigned);
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, bytes) != cudaSuccess) {
        cudaFree(p);
        return nullptr;
    }
    c.status = static_cast<unsigned *>(p);
    c.partials = reinterpret_cast<double *>(static_cast<char *>(p) + 256);
    c.counters = reinterpret_cast<unsigned *>(c.partials + (kReduceBlocks + 1) * 4);
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    c.device = dev;
    return &c;
}

}  // namespace sl

using namespace sl;

struct sl_batch {
    int device = -1;
    int n = 0;
    int scheme = SL_CEC;
    int dtype = SL_F32;
    bool fast = false;             // every instance takes the fast persistent path
    BatchRec *dev_recs = nullptr;  // generic path: work-queue records
    FastInst *dev_fast = nullptr;  // fast path: [2][n] tables (even: a -> b, odd: b -> a)
    int64_t fast_total = 0;
    unsigned *counter = nullptr;   // owns the device allocation
    int nitems[2] = {0, 0};
    int grid[2] = {0, 0};
    int fast_grid = 0;             // fast path: CTAs (0 = the kernel's default)
    sl_tuning tuning{};            // current launch shape, as reported
};

extern "C" {

int sl_version(void) { return 10000; }

const char *sl_last_error(void) { return g_err.c_str(); }

int sl_init(void)
{
    if (!ctx_get()) return fail(SL_ERR_CUDA, "could not create the device context");
    return SL_OK;
}

int sl_advect(void *out, const void *in, const void *vel, int ndim, const int64_t dims[3], const double spacing[3],
              double dt, int scheme, int dtype, int step_parity, void *stream)
{
    if (!out || !in || !vel) return fail(SL_ERR_ARG, "out, in and vel must not be NULL");
    if (scheme < SL_CIR || scheme > SL_CEC) return fail(SL_ERR_ARG, "unknown scheme %d", scheme);
    double s[3];
    int rc = check_geometry(ndim, dims, spacing, dt, dtype, s);
    if (rc) return rc;
    const size_t es = elem_size(dtype);
    const size_t fb = (size_t)ncell_of(dims) * es;
    if (overlap(out, fb, in, fb)) return fail(SL_ERR_ALIAS, "out overlaps in");
    if (overlap(out, fb, vel, fb * ndim)) return fail(SL_ERR_ALIAS, "out overlaps vel");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    return launch_step(out, in, vel, ndim, dims, s, scheme, dtype, step_parity, static_cast<cudaStream_t>(stream), c);
}

int sl_advect_multi(void *const *outs, const void *const *ins, int nfields, const void *vel, int ndim,
                    const int64_t dims[3], const double spacing[3], double dt, int scheme, int dtype,
                    int step_parity, void *stream)
{
    if (!outs || !ins || nfields < 1) return fail(SL_ERR_ARG, "outs/ins must hold nfields >= 1 pointers");
    if (!vel) return fail(SL_ERR_ARG, "vel must not be NULL");
    if (scheme < SL_CIR || scheme > SL_CEC) return fail(SL_ERR_ARG, "unknown scheme %d", scheme);
    double s[3];
    int rc = check_geometry(ndim, dims, spacing, dt, dtype, s);
    if (rc) return rc;
    const size_t fb = (size_t)ncell_of(dims) * elem_size(dtype);
    for (int f = 0; f < nfields; ++f) {
        if (!outs[f] || !ins[f]) return fail(SL_ERR_ARG, "field %d pointer is NULL", f);
        if (overlap(outs[f], fb, vel, fb * ndim)) return fail(SL_ERR_ALIAS, "outs[%d] overlaps vel", f);
        for (int h = 0; h < nfields; ++h) {
            if (overlap(outs[f], fb, ins[h], fb)) return fail(SL_ERR_ALIAS, "outs[%d] overlaps ins[%d]", f, h);
            if (h != f && overlap(outs[f], fb, outs[h], fb)) return fail(SL_ERR_ALIAS, "outs[%d] overlaps outs[%d]", f, h);
        }
    }
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool aligned = aligned16(vel);
    for (int f = 0; f < nfields; ++f) aligned = aligned && aligned16(ins[f]) && aligned16(outs[f]);
    if (scheme == SL_CEC && fast_eligible(dims, ndim, dtype, aligned)) {
        // groups of up to kFastFields fields per launch: the CTAs of a group
        // share one velocity read through L2
        const Launch lc = launch_for(SL_KERNEL_CEC_FAST, dims, scheme, dtype, aligned, c);
        for (int f0 = 0; f0 < nfields; f0 += kFastFields) {
            const int nf = std::min(kFastFields, nfields - f0);
            FastInst one;
            fast_fill(one, ins[f0], outs[f0], vel, dims, s, 0);
            one.nf = nf;
            for (int i = 0; i < nf; ++i) {
                one.fin[i] = static_cast<const float *>(ins[f0 + i]);
                one.fout[i] = static_cast<float *>(outs[f0 + i]);
            }
            const cudaError_t e = launch_cec_fast(one, nullptr, 1, (int64_t)one.ntiles * one.nz, step_parity,
                                                  c->status, lc.grid, st);
            if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        }
        return SL_OK;
    }
    // fields at uniform strides that share one alignment: one launch whose
    // CTAs of field f do what a launch for field f alone does
    const ptrdiff_t es = (ptrdiff_t)elem_size(dtype);
    const char *i0 = static_cast<const char *>(ins[0]), *o0 = static_cast<const char *>(outs[0]);
    const bool al0 = aligned16(ins[0]) && aligned16(outs[0]);
    const ptrdiff_t din = nfields > 1 ? static_cast<const char *>(ins[1]) - i0 : 0;
    const ptrdiff_t dout = nfields > 1 ? static_cast<const char *>(outs[1]) - o0 : 0;
    bool uniform = nfields > 1 && nfields <= 65535 && din % es == 0 && dout % es == 0;
    for (int f = 0; f < nfields && uniform; ++f)
        uniform = static_cast<const char *>(ins[f]) - i0 == f * din &&
                  static_cast<const char *>(outs[f]) - o0 == f * dout &&
                  (aligned16(ins[f]) && aligned16(outs[f])) == al0;
    if (uniform) {
        const bool al = al0 && aligned16(vel);
        const int fam = family_of(scheme, dtype, ndim, dims, al);
        if (fam != SL_KERNEL_CEC_FAST) {
            const Launch lc = launch_for(fam, dims, scheme, dtype, al, c);
            FieldSet fs;
            fs.n = nfields;
            fs.fin = din / es;
            fs.fout = dout / es;
            const cudaError_t e = launch_family(fam, lc, outs[0], ins[0], vel, ndim, dims, s, scheme, dtype,
                                                step_parity, st, c, fs);
            if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
            return SL_OK;
        }
    }
    for (int f = 0; f < nfields; ++f) {
        rc = launch_step(outs[f], ins[f], vel, ndim, dims, s, scheme, dtype, step_parity, st, c);
        if (rc) return rc;
    }
    return SL_OK;
}

int sl_advect_host(void *out, const void *in, const void *vel, int ndim, const int64_t dims[3],
                   const double spacing[3], double dt, int scheme, int dtype, int step_parity, void *stream)
{
    if (!out || !in || !vel) return fail(SL_ERR_ARG, "out, in and vel must not be NULL");
    if (scheme < SL_CIR || scheme > SL_CEC) return fail(SL_ERR_ARG, "unknown scheme %d", scheme);
    double s[3];
    int rc = check_geometry(ndim, dims, spacing, dt, dtype, s);
    if (rc) return rc;
    const size_t fb = (size_t)ncell_of(dims) * elem_size(dtype);
    if (overlap(out, fb, in, fb) || overlap(out, fb, vel, fb * ndim)) return fail(SL_ERR_ALIAS, "out overlaps an input");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    std::lock_guard<std::mutex> hold(g_host_mu[c->device]);
    const size_t need = fb * (2 + ndim) + 512;
    Staging &sg = g_stage[c->device];
    if (sg.bytes < need) {
        if (sg.buf) cudaFree(sg.buf);
        sg.buf = nullptr;
        sg.bytes = 0;
        if (cudaMalloc(&sg.buf, need) != cudaSuccess) return fail(SL_ERR_NOMEM, "device staging of %zu bytes", need);
        sg.bytes = need;
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *base = static_cast<char *>(sg.buf);
    char *d_in = base;
    char *d_out = base + al(fb);
    char *d_vel = base + 2 * al(fb);
    const char *h_in = static_cast<const char *>(in), *h_vel = static_cast<const char *>(vel);
    char *h_out = static_cast<char *>(out);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const int64_t nz = dims[2];
    const int nslab = (int)std::min<int64_t>(kMaxSlabs, nz / kMinSlabPlanes);
    HostPipe &pp = g_pipe[c->device];
    if (scheme != SL_CEC || nslab < 2 || !fast_eligible(dims, ndim, dtype, true) || !pipe_ready(pp)) {
        // one stream: copy in, step, copy back
        cudaError_t e = cudaMemcpyAsync(d_in, in, fb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_vel, vel, fb * ndim, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "host to device copy");
        rc = launch_step(d_out, d_in, d_vel, ndim, dims, s, scheme, dtype, step_parity, st, c);
        if (rc) return rc;
        e = cudaMemcpyAsync(out, d_out, fb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
        return SL_OK;
    }

    // Slab k writes the output planes [zk, zk+1) and reads the input planes
    // [zk - 6, zk+1 + 3) modulo nz.  The input copies run in z order, starting
    // with the six top planes that slab 0 reads across the periodic boundary;
    // slab k's kernel waits for the copy that completes its planes, and its
    // read-back waits for its kernel.  Slabs hold at least 32 planes, so every
    // copy range below is well ordered.
    const size_t pb = (size_t)dims[0] * (size_t)dims[1] * sizeof(float);
    auto zk = [&](int k) { return nz * k / nslab; };
    // planes [p0, p1) of the field, then of the velocity components: one 2D
    // copy of ndim rows (pitch fb) where fb is a valid pitch (fewer, larger
    // copies; each copy costs a few microseconds), else one copy per component
    auto put = [&](int64_t p0, int64_t p1) {
        cudaError_t e = cudaSuccess;
        if (p1 <= p0) return e;
        const size_t off = (size_t)p0 * pb, n = (size_t)(p1 - p0) * pb;
        e = cudaMemcpyAsync(d_in + off, h_in + off, n, cudaMemcpyHostToDevice, pp.in);
        if (e != cudaSuccess) return e;
        if ((int64_t)fb <= pp.max_pitch)
            return cudaMemcpy2DAsync(d_vel + off, fb, h_vel + off, fb, n, ndim, cudaMemcpyHostToDevice, pp.in);
        for (int d = 0; d < ndim && e == cudaSuccess; ++d)
            e = cudaMemcpyAsync(d_vel + d * fb + off, h_vel + d * fb + off, n, cudaMemcpyHostToDevice, pp.in);
        return e;
    };
    const Launch lc_fast = launch_for(SL_KERNEL_CEC_FAST, dims, scheme, dtype, true, c);
    cudaError_t e = cudaEventRecord(pp.start, st);
    for (cudaStream_t q : {pp.in, pp.run, pp.back})
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q, pp.start, 0);
    const char *what = "host to device copy";
    for (int k = 0; k < nslab && e == cudaSuccess; ++k) {
        const int64_t a = zk(k), b = zk(k + 1), top = nz - kFastHaloBelow;
        if (k == 0) {
            e = put(top, nz);
            if (e == cudaSuccess) e = put(0, std::min(b + kFastHaloAbove, top));
        } else {
            e = put(a + kFastHaloAbove, k + 1 < nslab ? b + kFastHaloAbove : top);
        }
        if (e == cudaSuccess) e = cudaEventRecord(pp.copied[k], pp.in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(pp.run, pp.copied[k], 0);
        if (e != cudaSuccess) break;
        FastInst one;
        fast_fill(one, d_in, d_out, d_vel, dims, s, 0);
        one.zb = (int)a;
        one.nzr = (int)(b - a);
        e = launch_cec_fast(one, nullptr, 1, (int64_t)one.ntiles * one.nzr, step_parity, c->status, lc_fast.grid, pp.run);
        if (e != cudaSuccess) {
            what = "kernel launch";
            break;
        }
        e = cudaEventRecord(pp.stepped[k], pp.run);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(pp.back, pp.stepped[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out + (size_t)a * pb, d_out + (size_t)a * pb, (size_t)(b - a) * pb,
                                cudaMemcpyDeviceToHost, pp.back);
        if (e != cudaSuccess) what = "device to host copy";
    }
    // every stream is drained before returning, also after a failed call
    for (cudaStream_t q : {pp.in, pp.run, pp.back}) {
        const cudaError_t f = cudaStreamSynchronize(q);
        if (e == cudaSuccess && f != cudaSuccess) {
            e = f;
            what = "host-buffer step";
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, what);
    return SL_OK;
}

int sl_release_host_staging(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return fail(SL_ERR_CUDA, "no device");
    std::lock_guard<std::mutex> hold(g_host_mu[dev]);
    if (g_stage[dev].buf) cudaFree(g_stage[dev].buf);
    g_stage[dev] = Staging();
    return SL_OK;
}

int sl_courant_max(const void *vel, int ndim, const int64_t dims[3], const double spacing[3], double dt, int dtype,
                   double *out_max, void *stream)
{
    if (!vel || !out_max) return fail(SL_ERR_ARG, "vel and out_max must not be NULL");
    double s[3];
    int rc = check_geometry(ndim, dims, spacing, dt, dtype, s);
    if (rc) return rc;
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_courant(dtype == SL_F64 ? 1 : 0, vel, ndim, ncell_of(dims), s, c->partials, st);
    double res[4];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res, c->partials + kReduceBlocks * 4, sizeof res, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "courant reduction");
    *out_max = res[1];
    return SL_OK;
}

int sl_norms(const void *a, const void *b, int64_t n, int dtype, double out[3], void *stream)
{
    if (!a || !b || !out || n < 1) return fail(SL_ERR_ARG, "a, b, out must be non-NULL and n >= 1");
    if (dtype < SL_F32 || dtype > SL_F32_D64) return fail(SL_ERR_ARG, "unknown dtype %d", dtype);
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_norms(dtype == SL_F64 ? 1 : 0, a, b, n, c->partials, st);
    double res[4];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res, c->partials + kReduceBlocks * 4, sizeof res, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "norm reduction");
    out[0] = std::sqrt(res[0] / (double)n);
    out[1] = res[1];
    out[2] = res[2] > 0.0 ? std::sqrt(res[0] / res[2]) : std::sqrt(res[0]);
    return SL_OK;
}

int sl_device_status(void *stream, unsigned *out_bits)
{
    if (!out_bits) return fail(SL_ERR_ARG, "out_bits must not be NULL");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->status, sizeof v, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof v, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    *out_bits = v;
    return SL_OK;
}

int sl_batch_create(sl_batch **out, const sl_instance *inst, int n, int scheme, int dtype, int tile_z)
{
    if (!out || !inst || n < 1) return fail(SL_ERR_ARG, "out and inst must be non-NULL and n >= 1");
    *out = nullptr;
    if (scheme != SL_CEC || dtype != SL_F32)
        return fail(SL_ERR_UNSUPPORTED, "batched steps serve SL_CEC with SL_F32");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    std::vector<BatchRec> recs(n);
    int total[2] = {0, 0};
    for (int i = 0; i < n; ++i) {
        const sl_instance &in = inst[i];
        double s[3];
        int rc = check_geometry(3, in.dims, in.spacing, in.dt, dtype, s);
        if (rc) return rc;
        if (!in.a || !in.b || !in.vel) return fail(SL_ERR_ARG, "instance %d has a NULL pointer", i);
        if (in.dims[0] % 4 || !aligned16(in.a) || !aligned16(in.b) || !aligned16(in.vel))
            return fail(SL_ERR_UNSUPPORTED, "instance %d: batched steps need dims[0] %% 4 == 0 and 16-byte aligned buffers", i);
        const size_t fb = (size_t)ncell_of(in.dims) * 4;
        if (overlap(in.a, fb, in.b, fb) || overlap(in.b, fb, in.vel, 3 * fb) || overlap(in.a, fb, in.vel, 3 * fb))
            return fail(SL_ERR_ALIAS, "instance %d: buffers overlap", i);
        // planes per work item: the argument, else the choice cached for the
        // generic split kernel on this grid, else 32
        int tz_cached = 32;
        sl_tuning tc;
        if (tuned_get(in.dims, SL_CEC, dtype, tc) && tc.kernel == SL_KERNEL_CEC_SPLIT && tc.tile_z > 0)
            tz_cached = tc.tile_z;
        BatchRec &r = recs[i];
        r.a = in.a;
        r.b = in.b;
        r.vel = in.vel;
        for (int par = 0; par < 2; ++par) {
            int tx, ty;
            batched_tiles(par, tx, ty);
            Geo &g = r.g[par];
            g.nx = (int)in.dims[0];
            g.ny = (int)in.dims[1];
            g.nz = (int)in.dims[2];
            g.plane = (int64_t)g.nx * g.ny;
            g.ncell = g.plane * g.nz;
            g.sx = s[0];
            g.sy = s[1];
            g.sz = s[2];
            g.status = c->status;
            g.tz = tile_z > 0 ? std::min(tile_z, g.nz) : std::min(tz_cached, g.nz);
            g.chunks = (g.nz + g.tz - 1) / g.tz;
            g.tiles_x = (g.nx + tx - 1) / tx;
            g.tiles_y = (g.ny + ty - 1) / ty;
            r.item0[par] = total[par];
            total[par] += g.tiles_x * g.tiles_y * g.chunks;
        }
    }
    bool fast = true;
    std::vector<FastInst> ftab(2 * (size_t)n);
    int64_t ftotal = 0;
    for (int i = 0; i < n; ++i) {
        const sl_instance &in = inst[i];
        double s[3] = {in.dt / in.spacing[0], in.dt / in.spacing[1], in.dt / in.spacing[2]};
        if (!fast_eligible(in.dims, 3, dtype, true)) fast = false;
        fast_fill(ftab[i], in.a, in.b, in.vel, in.dims, s, ftotal);
        fast_fill(ftab[n + i], in.b, in.a, in.vel, in.dims, s, ftotal);
        ftotal += (int64_t)ftab[i].ntiles * ftab[i].nz;
    }
    sl_batch *b = new (std::nothrow) sl_batch();
    if (!b) return fail(SL_ERR_NOMEM, "host allocation");
    b->fast = fast;
    b->fast_total = ftotal;
    b->device = c->device;
    b->n = n;
    b->scheme = scheme;
    b->dtype = dtype;
    b->nitems[0] = total[0];
    b->nitems[1] = total[1];
    for (int par = 0; par < 2; ++par) b->grid[par] = std::min(total[par], c->num_sms * batched_blocks_per_sm(par));
    b->tuning.kernel = fast ? SL_KERNEL_CEC_FAST : SL_KERNEL_CEC_SPLIT;
    b->tuning.tile_x = 32;
    b->tuning.tile_y = 32;
    b->tuning.tile_z = fast ? 0 : recs[0].g[0].tz;
    b->tuning.ctas_per_sm = fast ? std::max(1, fast_grid(0) / c->num_sms) : batched_blocks_per_sm(0);
    b->tuning.ms = 0.f;
    void *p = nullptr;
    const size_t rec_bytes = (sizeof(BatchRec) * n + 255) & ~(size_t)255;
    const size_t fast_bytes = (sizeof(FastInst) * 2 * n + 255) & ~(size_t)255;
    const size_t map_bytes = fast ? kFastMapsBytes * 2 * n : 0;
    if (cudaMalloc(&p, 256 + rec_bytes + fast_bytes + map_bytes) != cudaSuccess) {
        delete b;
        return fail(SL_ERR_NOMEM, "device instance table");
    }
    b->counter = static_cast<unsigned *>(p);
    b->dev_recs = reinterpret_cast<BatchRec *>(static_cast<char *>(p) + 256);
    b->dev_fast = reinterpret_cast<FastInst *>(static_cast<char *>(p) + 256 + rec_bytes);
    cudaError_t e = cudaSuccess;
    if (fast) {
        // tensor maps of both directions of every instance, after the tables
        char *dev_maps = static_cast<char *>(p) + 256 + rec_bytes + fast_bytes;
        std::vector<unsigned char> maps(map_bytes);
        for (size_t k = 0; k < 2 * (size_t)n && e == cudaSuccess; ++k) {
            e = fast_encode_maps(maps.data() + k * kFastMapsBytes, ftab[k]);
            ftab[k].maps = dev_maps + k * kFastMapsBytes;
        }
        if (e == cudaSuccess) e = cudaMemcpy(dev_maps, maps.data(), map_bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->dev_recs, recs.data(), sizeof(BatchRec) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dev_fast, ftab.data(), sizeof(FastInst) * 2 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->counter, 0, 256);
    if (e != cudaSuccess) {
        cudaFree(p);
        delete b;
        return cuda_fail(e, "instance table upload");
    }
    *out = b;
    return SL_OK;
}

int sl_batch_step(sl_batch *b, int step_index, void *stream)
{
    if (!b) return fail(SL_ERR_ARG, "batch is NULL");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    if (c->device != b->device) return fail(SL_ERR_ARG, "batch belongs to device %d", b->device);
    const int par = step_index & 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (b->fast) {
        FastInst dummy{};
        e = launch_cec_fast(dummy, b->dev_fast + (size_t)par * b->n, b->n, b->fast_total, par, c->status, b->fast_grid, st);
    } else {
        e = cudaMemsetAsync(b->counter, 0, sizeof(unsigned), st);
        if (e == cudaSuccess)
            e = launch_batched_cec(b->dev_recs, b->n, b->nitems[par], par, b->counter, c->status, b->grid[par], st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    return SL_OK;
}

int sl_batch_autotune(sl_batch *b, sl_tuning *best, void *stream)
{
    if (!b) return fail(SL_ERR_ARG, "batch is NULL");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    if (c->device != b->device) return fail(SL_ERR_ARG, "batch belongs to device %d", b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // candidate CTAs per SM within the kernel's occupancy (even steps only: A -> B)
    const int occ = b->fast ? std::max(1, fast_grid(0) / c->num_sms) : batched_blocks_per_sm(0);
    std::vector<int> cands;
    for (int k : {1, 2, 4})
        if (k <= occ) cands.push_back(k);
    const int saved_fast = b->fast_grid, saved0 = b->grid[0], saved1 = b->grid[1];
    auto set = [&](int k) {
        if (b->fast) {
            b->fast_grid = k * c->num_sms;
        } else {
            b->grid[0] = std::min(b->nitems[0], k * c->num_sms);
            b->grid[1] = std::min(b->nitems[1], std::min(k, batched_blocks_per_sm(1)) * c->num_sms);
        }
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(SL_ERR_CUDA, "events");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(SL_ERR_CUDA, "events");
    }
    float best_ms = 1e30f;
    int best_k = cands.front();
    int rc = SL_OK;
    for (int k : cands) {
        set(k);
        rc = sl_batch_step(b, 0, stream);   // warm-up
        float ms = 0.f;
        cudaError_t e = rc ? cudaSuccess : cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && !rc && e == cudaSuccess; ++r) rc = sl_batch_step(b, 0, stream);
        if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "batch autotune");
        if (rc) break;
        if (ms / 3.f < best_ms) {
            best_ms = ms / 3.f;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        b->fast_grid = saved_fast;
        b->grid[0] = saved0;
        b->grid[1] = saved1;
        return rc;
    }
    set(best_k);
    b->tuning.ctas_per_sm = best_k;
    b->tuning.ms = best_ms;
    if (best) *best = b->tuning;
    return SL_OK;
}

int sl_batch_tuning(const sl_batch *b, sl_tuning *out)
{
    if (!b || !out) return fail(SL_ERR_ARG, "batch and out must not be NULL");
    *out = b->tuning;
    return SL_OK;
}

int sl_batch_destroy(sl_batch *b)
{
    if (!b) return SL_OK;
    if (b->counter) cudaFree(b->counter);
    delete b;
    return SL_OK;
}

int64_t sl_advect_wide_workspace(int ndim, const int64_t dims[3], int scheme, int dtype)
{
    if (scheme < SL_CIR || scheme > SL_CEC) return fail(SL_ERR_ARG, "unknown scheme %d", scheme);
    if (dtype != SL_F32 && dtype != SL_F64) return fail(SL_ERR_UNSUPPORTED, "wide steps take SL_F32 or SL_F64");
    const double unit[3] = {1.0, 1.0, 1.0};
    double s[3];
    int rc = check_geometry(ndim, dims, unit, 1.0, dtype, s);
    if (rc) return rc;
    return (int64_t)wide_fields(scheme, ndim) * (int64_t)wide_field_bytes(ncell_of(dims), elem_size(dtype));
}

int sl_advect_wide(void *out, const void *in, const void *vel, int ndim, const int64_t dims[3],
                   const double spacing[3], double dt, int scheme, int dtype, int step_parity, void *workspace,
                   int64_t workspace_bytes, void *stream)
{
    if (!out || !in || !vel) return fail(SL_ERR_ARG, "out, in and vel must not be NULL");
    const int64_t need = sl_advect_wide_workspace(ndim, dims, scheme, dtype);
    if (need < 0) return (int)need;
    double s[3];
    int rc = check_geometry(ndim, dims, spacing, dt, dtype, s);
    if (rc) return rc;
    if (dims[1] > 65535 || dims[2] > 65535) return fail(SL_ERR_UNSUPPORTED, "wide steps need dims[1], dims[2] <= 65535");
    if (workspace_bytes < need || (need > 0 && !workspace))
        return fail(SL_ERR_ARG, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (need > 0 && (reinterpret_cast<uintptr_t>(workspace) & 255u)) return fail(SL_ERR_ARG, "workspace must be 256-byte aligned");
    const size_t fb = (size_t)ncell_of(dims) * elem_size(dtype);
    if (overlap(out, fb, in, fb) || overlap(out, fb, vel, fb * ndim)) return fail(SL_ERR_ALIAS, "out overlaps an input");
    if (need > 0 && (overlap(workspace, (size_t)need, in, fb) || overlap(workspace, (size_t)need, vel, fb * ndim) ||
                     overlap(workspace, (size_t)need, out, fb)))
        return fail(SL_ERR_ALIAS, "workspace overlaps a field");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    const cudaError_t e = launch_wide(dtype, scheme, in, out, vel, ndim, dims, s, step_parity, workspace, c->status,
                                      static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "wide step launch");
    return SL_OK;
}

int sl_autotune_scheme(void *out, const void *in, const void *vel, int ndim, const int64_t dims[3],
                       const double spacing[3], double dt, int scheme, int dtype, sl_tuning *best, void *stream)
{
    if (!out || !in || !vel) return fail(SL_ERR_ARG, "out, in and vel must not be NULL");
    if (scheme < SL_CIR || scheme > SL_CEC) return fail(SL_ERR_ARG, "unknown scheme %d", scheme);
    double s[3];
    int rc = check_geometry(ndim, dims, spacing, dt, dtype, s);
    if (rc) return rc;
    const size_t fb = (size_t)ncell_of(dims) * elem_size(dtype);
    if (overlap(out, fb, in, fb) || overlap(out, fb, vel, fb * ndim)) return fail(SL_ERR_ALIAS, "out overlaps an input");
    DevCtx *c = ctx_get();
    if (!c) return fail(SL_ERR_CUDA, "could not create the device context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool aligned = aligned16(out) && aligned16(in) && aligned16(vel);
    const int fam = family_of(scheme, dtype, ndim, dims, aligned);

    // candidates: (tile height, planes per item, CTAs per SM); 0 = the default
    struct Cand {
        int ty, tz, ctas;
    };
    std::vector<Cand> cands;
    std::vector<int> tzs;
    if (ndim == 3) {
        for (int tz : {8, 16, 32, 64, 128, 256})
            if (tz < dims[2]) tzs.push_back(tz);
        tzs.push_back((int)dims[2]);
    } else {
        tzs.push_back(1);
    }
    if (fam == SL_KERNEL_CEC_FAST) {
        const int occ = std::max(1, fast_grid(0) / c->num_sms);
        for (int k = 1; k <= std::min(occ, 2); ++k) cands.push_back({0, 0, k});
    } else if (fam == SL_KERNEL_CEC_SPLIT) {
        for (int tz : tzs) cands.push_back({0, tz, 0});
    } else if (fam == SL_KERNEL_CIR_GROUPS) {
        for (int ty : {16, 32})
            if (ty == 16 || dims[1] >= 32)
                for (int tz : tzs) cands.push_back({ty, tz, 0});
    } else {
        std::vector<int> tys = {0};
        if (dtype == SL_F32 && ndim == 3 && aligned && dims[0] % 4 == 0) tys = {8, 16, 32};
        for (int ty : tys) {
            if (scheme == SL_BEC && ndim == 3)
                for (int k = 1; k <= 3; ++k) cands.push_back({ty, 0, k});
            else
                for (int tz : tzs) cands.push_back({ty, tz, 0});
        }
    }

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(SL_ERR_CUDA, "events");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(SL_ERR_CUDA, "events");
    }
    const int reps = scheme == SL_CEC ? 4 : 3;   // both sweep orders for SL_CEC
    float best_ms = 1e30f;
    Cand pick = cands.front();
    cudaError_t e = cudaSuccess;
    for (const Cand &cd : cands) {
        Launch lc;
        lc.aligned = aligned;
        lc.ty = cd.ty;
        lc.tz = cd.tz;
        lc.grid = cd.ctas > 0 ? cd.ctas * c->num_sms : 0;
        e = launch_family(fam, lc, out, in, vel, ndim, dims, s, scheme, dtype, 0, st, c);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = launch_family(fam, lc, out, in, vel, ndim, dims, s, scheme, dtype, r & 1, st, c);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        if (ms / reps < best_ms) {
            best_ms = ms / reps;
            pick = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    sl_tuning t;
    t.kernel = fam;
    t.tile_x = 32;
    t.tile_y = pick.ty > 0 ? pick.ty : default_ty(fam, dtype);
    if (fam == SL_KERNEL_CIR_GROUPS && t.tile_y == 32 && dims[1] < 32) t.tile_y = 16;
    t.tile_z = pick.tz;
    t.ctas_per_sm = pick.ctas;
    t.ms = best_ms;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[TuneKey(dims[0], dims[1], dims[2], scheme, dtype)] = t;
    }
    if (best) *best = t;
    return SL_OK;
}

int sl_autotune(void *out, const void *in, const void *vel, int ndim, const int64_t dims[3], const double spacing[3],
                double dt, int dtype, int *tile_z, void *stream)
{
    if (!tile_z) return fail(SL_ERR_ARG, "NULL argument");
    sl_tuning t;
    const int rc = sl_autotune_scheme(out, in, vel, ndim, dims, spacing, dt, SL_CEC, dtype, &t, stream);
    if (rc) return rc;
    if (t.kernel == SL_KERNEL_CEC_FAST) {
        DevCtx *c = ctx_get();
        *tile_z = t.ctas_per_sm * (c ? c->num_sms : 1);
    } else {
        *tile_z = t.tile_z;
    }
    return SL_OK;
}

int sl_tuning_get(const int64_t dims[3], int scheme, int dtype, sl_tuning *out)
{
    if (!dims || !out) return fail(SL_ERR_ARG, "dims and out must not be NULL");
    if (!tuned_get(dims, scheme, dtype, *out)) return fail(SL_ERR_ARG, "no launch shape cached for this grid");
    return SL_OK;
}

int sl_tuning_clear(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned.clear();
    return SL_OK;
}

int sl_tuning_save(const char *path)
{
    if (!path) return fail(SL_ERR_ARG, "path is NULL");
    std::vector<std::pair<TuneKey, sl_tuning>> all;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        all.assign(g_tuned.begin(), g_tuned.end());
    }
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(SL_ERR_ARG, "cannot write %s", path);
    char name[256] = "unknown";
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
        std::snprintf(name, sizeof name, "%s", prop.name);
    else
        cudaGetLastError();   // no device: clear the error and write the entries anyway
    std::fprintf(f, "# libsl launch shapes, timed on %s: nx ny nz scheme dtype kernel tile_x tile_y tile_z ctas_per_sm ms\n", name);
    for (const auto &kv : all) {
        const sl_tuning &t = kv.second;
        std::fprintf(f, "%lld %lld %lld %d %d %d %d %d %d %d %.6g\n", (long long)std::get<0>(kv.first),
                     (long long)std::get<1>(kv.first), (long long)std::get<2>(kv.first), std::get<3>(kv.first),
                     std::get<4>(kv.first), t.kernel, t.tile_x, t.tile_y, t.tile_z, t.ctas_per_sm, (double)t.ms);
    }
    const bool ok = std::ferror(f) == 0;
    if (std::fclose(f) != 0 || !ok) return fail(SL_ERR_ARG, "write error on %s", path);
    return SL_OK;
}

int sl_tuning_load(const char *path)
{
    if (!path) return fail(SL_ERR_ARG, "path is NULL");
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(SL_ERR_ARG, "cannot read %s", path);
    std::vector<std::pair<TuneKey, sl_tuning>> got;
    char line[512];
    int lineno = 0;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        const char *q = line;
        while (*q == ' ' || *q == '\t') ++q;
        if (*q == '#' || *q == '\n' || *q == '\0') continue;
        long long nx, ny, nz;
        int scheme, dtype, kernel, tx, ty, tz, ctas;
        double ms;
        char extra;
        const int n = std::sscanf(q, "%lld %lld %lld %d %d %d %d %d %d %d %lf %c", &nx, &ny, &nz, &scheme, &dtype,
                                  &kernel, &tx, &ty, &tz, &ctas, &ms, &extra);
        const bool ok = n == 11 && nx >= 1 && ny >= 1 && nz >= 1 && nx <= (1ll << 30) && ny <= (1ll << 30) &&
                        nz <= (1ll << 30) && scheme >= SL_CIR && scheme <= SL_CEC && dtype >= SL_F32 &&
                        dtype <= SL_F32_D64 && kernel >= SL_KERNEL_CEC_FAST && kernel <= SL_KERNEL_UNSPLIT &&
                        tx == 32 && (ty == 8 || ty == 16 || ty == 32) && tz >= 0 && tz <= (1 << 30) && ctas >= 0 &&
                        ctas <= 32 && std::isfinite(ms);
        if (!ok) {
            std::fclose(f);
            return fail(SL_ERR_ARG, "%s line %d: malformed launch shape", path, lineno);
        }
        sl_tuning t;
        t.kernel = kernel;
        t.tile_x = tx;
        t.tile_y = ty;
        t.tile_z = tz;
        t.ctas_per_sm = ctas;
        t.ms = (float)ms;
        got.emplace_back(TuneKey(nx, ny, nz, scheme, dtype), t);
    }
    std::fclose(f);
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto &kv : got) g_tuned[kv.first] = kv.second;
    return SL_OK;
}

}  // extern "C"
