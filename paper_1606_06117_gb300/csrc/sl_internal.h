// sl_internal.h -- declarations shared by the host entry points and the kernel
// translation units of libsl.  Not part of the public ABI (see include/sl.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sl_common.cuh"

namespace sl {

// Per-device context: status word and small work areas.
struct DevCtx {
    int device = -1;
    unsigned *status = nullptr;      // SL_DEV_* bits
    double *partials = nullptr;      // reduction partials (kReduceBlocks x 4)
    unsigned *counters = nullptr;    // work counters for batched launches
    int num_sms = 0;
};

constexpr int kReduceBlocks = 1024;

DevCtx *ctx_get();   // context of the current device, created on demand

// Launch configuration chosen for a fused kernel.
struct Launch {
    int tz = 0;          // z chunk (planes per work item); 0 = default
    int ty = 0;          // column tile height among a kernel's compiled variants; 0 = default
    int grid = 0;        // CTAs; 0 = one per item (persistent kernels: their occupancy)
    bool aligned = true; // all base pointers 16-byte aligned (vector staging allowed)
};

// Several fields advected by one velocity in one launch: field f reads
// in + f * fin and writes out + f * fout (elements); the launch's grid gains
// a y extent of n, and each field's CTAs do exactly what a launch for that
// field alone does.
struct FieldSet {
    int n = 1;
    int64_t fin = 0, fout = 0;
};

// Fused single-step kernels; return a cudaError_t of the launch.
cudaError_t launch_split_cec(int dtype, const void *in, void *out, const void *vel, int ndim,
                             const int64_t dims[3], const double s[3], int parity,
                             Launch lc, unsigned *status, cudaStream_t st, FieldSet fs = FieldSet());
cudaError_t launch_unsplit(int dtype, int scheme, const void *in, void *out, const void *vel,
                           int ndim, const int64_t dims[3], const double s[3], Launch lc,
                           unsigned *status, cudaStream_t st, FieldSet fs = FieldSet());
// FP32 3D CIR kernel on four-cell groups (k_cir_fast.cu); launch_unsplit routes
// eligible CIR steps to it.
bool cir_fast_eligible(int dtype, int ndim, const int64_t dims[3], bool aligned);
cudaError_t launch_cir_fast(const void *in, void *out, const void *vel, const int64_t dims[3], const double s[3],
                            Launch lc, unsigned *status, cudaStream_t st);

// Reductions (synchronous results through host pointers after a stream sync).
cudaError_t launch_norms(int dtype, const void *a, const void *b, int64_t n, double *partials,
                         cudaStream_t st);
cudaError_t launch_courant(int dtype, const void *vel, int ndim, int64_t n, const double s[3],
                           double *partials, cudaStream_t st);

// Batched persistent CEC step (FP32, 3D) over an instance table in device
// memory.  Record i owns global items [item0[par], item0[par] + items) of the
// x,y,z (par 0) or z,y,x (par 1) decomposition.
struct BatchRec {
    void *a;
    void *b;
    const void *vel;
    Geo g[2];
    int item0[2];
};
void batched_tiles(int parity, int &tx, int &ty);
int batched_blocks_per_sm(int parity);
cudaError_t launch_batched_cec(const BatchRec *dev_recs, int ninst, int nitems, int parity, unsigned *counter,
                               unsigned *status, int grid, cudaStream_t st);

int default_tz(int dtype, int ndim, const int64_t dims[3]);

// Fast FP32 CEC path (k_cec_fast.cu): one periodic grid of whole 32 x 32 column
// tiles; w0 numbers its first (column tile, plane) pair in a batch.  A launch
// writes the output planes [zb, zb + nzr) (fast_fill: all nz planes) and reads
// the input planes [zb - 6, zb + nzr + 3), taken modulo nz.
// A single-instance launch may advance nf <= kFastFields fields with one
// velocity: its CTAs form groups of nf that take the same (column tile, plane)
// sequence, one field each, so the group's velocity reads are served from L2.
constexpr int kFastFields = 4;
struct FastInst {
    const float *in;
    float *out;
    const float *vel;
    int nx, ny, nz;
    int tiles_x, ntiles;
    int64_t plane, ncell;
    float sx, sy, sz;
    int64_t w0;
    const void *maps;   // batched tables: device address of this instance's tensor maps
    int zb, nzr;        // output planes [zb, zb + nzr); 0 <= zb, 1 <= nzr, zb + nzr <= nz
    int nf;             // fields (1 in batched tables); fin[0] = in, fout[0] = out
    const float *fin[kFastFields];
    float *fout[kFastFields];
};
// Input planes a fast launch reads below and above its output planes.
constexpr int kFastHaloBelow = 6, kFastHaloAbove = 3;
// Bytes of one instance's tensor maps (22 maps of the first field and the
// velocity, 9 for each further field; 128 bytes each, 64-byte aligned).
constexpr size_t kFastMapsBytes = (22 + 9 * (kFastFields - 1)) * 128;
// Encodes the tensor maps of an instance into dst (host memory, kFastMapsBytes).
cudaError_t fast_encode_maps(void *dst, const FastInst &f);
bool fast_eligible(const int64_t dims[3], int ndim, int dtype, bool aligned);
void fast_fill(FastInst &f, const void *in, void *out, const void *vel, const int64_t dims[3], const double s[3],
               int64_t w0);
cudaError_t launch_cec_fast(const FastInst &one, const FastInst *dev_table, int ninst, int64_t total, int parity,
                            unsigned *status, int grid_req, cudaStream_t st);
int fast_grid(int parity);

// Steps at any Courant number (k_wide.cu): non-local interpolation, unfused
// kernels, intermediate fields in a caller-owned workspace of wide_fields()
// fields of wide_field_bytes() each (256-byte aligned).  Grids launch as
// (x blocks, ny, nz), so ny and nz must be at most 65535.
size_t wide_field_bytes(int64_t ncell, size_t elem);
int wide_fields(int scheme, int ndim);
cudaError_t launch_wide(int dtype, int scheme, const void *in, void *out, const void *vel, int ndim,
                        const int64_t dims[3], const double s[3], int parity, void *work, unsigned *status,
                        cudaStream_t st);

// Records a thread-local error message (read by sl_last_error) and returns code.
int set_error(int code, const char *msg);

// Largest element count sl_norms_static accepts.
constexpr int64_t kNormsStaticMaxElems = (int64_t)1 << 40;

}  // namespace sl
