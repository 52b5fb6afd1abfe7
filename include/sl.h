/*
 * sl.h -- C ABI of libsl, the GB300 (sm_103a) implementation of the
 * multi-stage semi-Lagrangian advection schemes of Cameron, Raynaud & Dormy,
 * "Multi-stage high order semi-Lagrangian schemes for incompressible flows in
 * Cartesian geometries" (arXiv 1606.06117).
 *
 * The library advances a passive scalar Phi by one time step of
 * d_t Phi + (u . grad) Phi = 0 (Sec. 2, eq. intro:adv) on a uniform periodic
 * Cartesian grid, with one of four schemes built from the multilinear
 * semi-Lagrangian operator L_U[Phi](x) = Phi~(x - u dt) (Sec. 2):
 *
 *   SL_CIR  L_U[Phi]                                   (Sec. 3; eq. CIR2D)
 *   SL_FEC  L_U[Phi] + (Phi - Phi_bar)/2,
 *           Phi_bar = L_{-U}[L_U[Phi]]                 (eq. intro:FEC)
 *   SL_BEC  L_U[Phi + (Phi - Phi_bar)/2]               (eq. intro:BEC)
 *   SL_CEC  a FEC + b BEC per axis, 3a = 2 - dx/(|u|dt), b = 1 - a
 *           (eqs. intro:CEC, intro:CECcoef), applied direction by direction
 *           (Sec. 2 last paragraph, Sec. 5 eqs. split:1-2); the sweep order is
 *           x,y,z for an even step_parity and z,y,x for an odd one.
 *
 * CIR, FEC and BEC use the unsplit multilinear operator on all axes.  The
 * velocity is taken at the arrival cell; the departure point is the straight
 * backtrace x_i - u_i dt.  Every step of sl_advect is one fused kernel: one
 * read of Phi and u and one write of Phi per cell.
 *
 * Conventions shared by all entry points
 *   - Fields are C-contiguous [z][y][x] arrays (x fastest) of dims[2] x dims[1]
 *     x dims[0] cells.  For ndim = 2 set dims[2] = 1.
 *   - vel points to ndim component planes of prod(dims) elements each (x
 *     component first), the same element type as the field (SoA).
 *   - spacing[d] is the cell size dx_d; the Courant number of a cell is
 *     C_d = u_d dt / dx_d.  The schemes need |C_d| <= 1 (Table 1 stability);
 *     larger values are reported through the device status word (bit
 *     SL_DEV_CFL) and the result is then undefined but stays in bounds.
 *     sl_advect_wide takes any Courant number (non-local interpolation).
 *   - Pointers are device pointers owned by the caller unless the entry point
 *     says otherwise.  out must not alias in (SL_ERR_ALIAS).
 *   - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *     stream) unless stated otherwise.  No C++ exception crosses the ABI.
 *   - The return value is an sl_status.  On failure sl_last_error() gives a
 *     thread-local message.  The library keeps a small per-device context
 *     (status word and work counters) that it allocates on the first call on a
 *     device; make that first call outside CUDA graph capture, or call
 *     sl_init() first.
 */
#ifndef SL_H
#define SL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SL_CIR = 0, SL_FEC = 1, SL_BEC = 2, SL_CEC = 3 } sl_scheme;

/* Element type and arithmetic.  SL_F32: float storage and arithmetic, the
 * round-trip difference Phi - Phi_bar evaluated from neighbour differences so
 * that it does not cancel.  SL_F64: double throughout.  SL_F32_D64: float
 * storage with L_U[Phi], Phi_bar and Phi - Phi_bar evaluated in double. */
typedef enum { SL_F32 = 0, SL_F64 = 1, SL_F32_D64 = 2 } sl_dtype;

typedef enum {
    SL_OK = 0,
    SL_ERR_ARG = -1,         /* bad pointer, size, enum or spacing      */
    SL_ERR_ALIAS = -2,       /* out overlaps in                          */
    SL_ERR_CFL = -3,         /* a Courant number exceeds 1 (host checks) */
    SL_ERR_CUDA = -4,        /* a CUDA runtime call failed               */
    SL_ERR_TIMEOUT = -5,     /* a bounded device wait ran out            */
    SL_ERR_UNSUPPORTED = -6, /* valid request the library does not serve */
    SL_ERR_NOMEM = -7        /* device or host allocation failed         */
} sl_status;

/* Bits of the device status word (see sl_device_status). */
#define SL_DEV_CFL 1u        /* a kernel saw |C_d| > 1 (sl_advect), or a
                                non-finite C_d or |C_d| >= 2^30 (sl_advect_wide) */
#define SL_DEV_TIMEOUT 2u    /* a bounded device wait gave up       */

/* Library version, major * 10000 + minor * 100 + patch. */
int sl_version(void);

/* Thread-local text of the last error returned on this thread ("" if none). */
const char *sl_last_error(void);

/* Create the per-device context of the current device (idempotent).  Safe to
 * call before any stream capture; the other entry points call it lazily. */
int sl_init(void);

/*
 * One time step of one scheme: out = S[in].
 *   out, in      device arrays of prod(dims) elements (type per dtype).
 *   vel          device array, ndim planes of prod(dims) elements.
 *   ndim         2 or 3.
 *   dims         cells per axis (x, y, z); each >= 1, dims[2] = 1 when ndim = 2.
 *   spacing      cell size per axis (x, y, z), > 0 (spacing[2] unused in 2D).
 *   dt           time step (any sign; a negative dt reverses the flow).
 *   scheme       sl_scheme.   dtype  sl_dtype.
 *   step_parity  only read by SL_CEC: sweep order x,y,z (even) or z,y,x (odd).
 *   stream       cudaStream_t or NULL.
 * Errors: SL_ERR_ARG, SL_ERR_ALIAS, SL_ERR_CUDA (launch failure).
 */
int sl_advect(void *out, const void *in, const void *vel, int ndim,
              const int64_t dims[3], const double spacing[3], double dt,
              int scheme, int dtype, int step_parity, void *stream);

/*
 * The same step applied to nfields fields advected by one velocity (e.g. the
 * three velocity components and a scalar).  outs[f] = S[ins[f]], equal bit for
 * bit to one sl_advect call per field.  Same arguments and errors as
 * sl_advect; every outs[f] must differ from every ins[g] and from the other
 * outs.  Since L_U is linear in Phi for a fixed velocity (Sec. 2), every field
 * shares the departure points and CEC weights; an SL_CEC step in FP32 on the
 * geometry of the persistent kernel (see sl_autotune) advances up to 4 fields
 * per launch: the launch's CTAs form groups, one CTA per field, that walk the
 * same (column tile, plane) sequence, so that a group's velocity reads can be
 * served from L2 after the first one.  Otherwise fields stored at uniform
 * strides (ins[f] = ins[0] + f * a, outs[f] = outs[0] + f * b, whole elements)
 * whose buffers share one 16-byte alignment run in one launch of the generic
 * kernels, a row of CTAs per field; other field sets take a launch per field.
 */
int sl_advect_multi(void *const *outs, const void *const *ins, int nfields,
                    const void *vel, int ndim, const int64_t dims[3],
                    const double spacing[3], double dt, int scheme, int dtype,
                    int step_parity, void *stream);

/*
 * sl_advect on HOST buffers: copies in and vel to the device, runs the step
 * and copies the result back into out; returns once out holds the result.
 * The library keeps a device staging buffer per device that grows to the
 * largest request (freed by sl_release_host_staging); calls on one device run
 * one at a time.  Host buffers may be pageable; page-locked buffers copy
 * faster.
 * Work order: the work runs after everything already queued on stream.  An
 * SL_CEC step in FP32 on the fast geometry (whole 32 x 32 column tiles,
 * nx >= 64, ndim = 3) with nz >= 64 is cut into z slabs of at least 32
 * planes (at most 8 slabs) on three library-owned streams: a slab's kernel
 * starts once the input planes it reads are on the device, and its output
 * planes are copied back while later slabs' inputs are still being copied
 * in.  The result equals sl_advect's bit for bit.  Other steps run on stream:
 * copy in, step, copy back.
 * Errors: those of sl_advect; SL_ERR_NOMEM (staging).  Every copy and kernel
 * of the call has ended when it returns, also after an error.
 */
int sl_advect_host(void *out, const void *in, const void *vel, int ndim,
                   const int64_t dims[3], const double spacing[3], double dt,
                   int scheme, int dtype, int step_parity, void *stream);
int sl_release_host_staging(void);

/*
 * Host-side Courant check: max_d max_cells |u_d| dt / dx_d of a device
 * velocity, reduced on the device in double and returned synchronously.
 */
int sl_courant_max(const void *vel, int ndim, const int64_t dims[3],
                   const double spacing[3], double dt, int dtype,
                   double *out_max, void *stream);

/*
 * Error norms of a device field a against a device field b (n elements of
 * dtype), accumulated in double on the device and returned synchronously:
 * out[0] = RMS of a - b, out[1] = max |a - b|, out[2] = ||a - b||_2 / ||b||_2.
 */
int sl_norms(const void *a, const void *b, int64_t n, int dtype, double out[3],
             void *stream);

/*
 * sl_norms for callers that cannot allocate device memory: the same FP64
 * reduction, but its scratch is a fixed 32.8 KB array compiled into the
 * library (resident on every GPU that loads it until the process exits), and
 * the three results go to the caller's DEVICE buffer out (3 doubles, same order
 * as sl_norms) asynchronously on the stream; nothing is copied to the host and
 * the stream is not synchronised.  The paper has no counterpart: this is a
 * library-interface variant.
 *
 * Who needs it: code that runs while a CUDA stream is being captured into a
 * graph (cudaMalloc is not permitted there), applications whose device memory
 * is handed out by their own pool and must see no driver allocation inside a
 * time loop, and callbacks with a fixed memory budget.  sl_norms itself
 * creates the library's device context with cudaMalloc on its first call and
 * synchronises the stream, which those callers cannot accept.
 *
 * The first call on a device resolves the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The resolved address is kept for the life of the process: after a
 * device reset (cudaDeviceReset, or the primary context torn down and made
 * again) it no longer points at mapped memory, so do not call this function on
 * that device after such a reset.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 * n must be in [1, 2^40]; larger or smaller values return SL_ERR_ARG.  All calls
 * share the one array: calls whose kernels overlap on the GPU (e.g. on two
 * streams at once) race and may return wrong norms; serialise them.
 */
int sl_norms_static(const void *a, const void *b, int64_t n, int dtype, double *out,
                    void *stream);

/*
 * Failure-detection self-test of the bounded device waits: one CTA waits on an
 * mbarrier that nothing completes, gives up after `polls` polls (1 .. 2^20),
 * sets SL_DEV_TIMEOUT in the device status word and exits normally; the
 * context stays usable.  Returns SL_ERR_TIMEOUT when the wait ran out as
 * intended (synchronous).  The paper has no counterpart.
 */
int sl_selftest_wait_timeout(unsigned polls, void *stream);

/*
 * Read and clear the device status word of the current device (SL_DEV_*
 * bits).  Synchronises the stream first.
 */
int sl_device_status(void *stream, unsigned *out_bits);

/*
 * Checkpoints of a field for long runs (no counterpart in the paper).
 * sl_field_save copies the device field (prod(dims) elements of dtype's
 * storage type: float for SL_F32 and SL_F32_D64, double for SL_F64) to the
 * file at path: one JSON header line (format, version, ndim, dims, dtype,
 * step, payload bytes, FNV-1a 64 checksum of the payload) followed by the raw
 * little-endian payload.  sl_field_load checks that the file holds exactly
 * that grid and type, that the payload is complete and its checksum matches,
 * then copies it into the device field and returns the saved step in *step
 * (may be NULL).  Both synchronise the stream and return when done.
 * Errors: SL_ERR_ARG (NULL argument, bad geometry, unreadable / unwritable
 * file, another grid or type, a truncated or corrupted payload: the device
 * field is not touched then), SL_ERR_NOMEM (host buffer), SL_ERR_CUDA.
 */
int sl_field_save(const char *path, const void *field, int ndim, const int64_t dims[3],
                  int dtype, int64_t step, void *stream);
int sl_field_load(const char *path, void *field, int ndim, const int64_t dims[3],
                  int dtype, int64_t *step, void *stream);

/*
 * Autotuning of launch shapes (no counterpart in the paper).
 *
 * The kernel that serves a step is fixed by the request (scheme, dtype,
 * dimensionality, sizes, 16-byte alignment); the autotuner chooses, by timing
 * on the caller's buffers, among launch shapes of that kernel that change only
 * how cells are grouped into work, never a cell's arithmetic, so every choice
 * gives bitwise the same results:
 *   SL_KERNEL_CEC_FAST     persistent FP32 split CEC kernel (32 x 32 column
 *                          tiles): CTAs per SM, 1 or 2.
 *   SL_KERNEL_CEC_SPLIT    generic split CEC kernel: planes per work item.
 *   SL_KERNEL_CIR_GROUPS   FP32 CIR kernel on four-cell groups: tile height
 *                          16 or 32, planes per work item.
 *   SL_KERNEL_UNSPLIT      generic CIR / FEC / BEC kernel: tile height 8, 16 or
 *                          32 (FP32 3D grids with dims[0] % 4 == 0 and aligned
 *                          buffers; otherwise the dtype's fixed height) and
 *                          planes per work item, or for 3D BEC (persistent
 *                          equal shares) CTAs per SM, 1 to 3.
 * A choice is cached per (dims, scheme, dtype) in the process and used by
 * sl_advect, sl_advect_multi, sl_advect_host and sl_batch_create whenever the
 * request is served by the kernel it was tuned for.
 */
enum {
    SL_KERNEL_CEC_FAST = 1,
    SL_KERNEL_CEC_SPLIT = 2,
    SL_KERNEL_CIR_GROUPS = 3,
    SL_KERNEL_UNSPLIT = 4
};

typedef struct {
    int kernel;       /* SL_KERNEL_*                                         */
    int tile_x;       /* column tile of a work item, cells along x           */
    int tile_y;       /*                             cells along y           */
    int tile_z;       /* planes per work item; 0: persistent equal shares    */
    int ctas_per_sm;  /* CTAs per SM of a persistent launch; 0: one per item  */
    float ms;         /* measured time of one step, milliseconds             */
} sl_tuning;

/* --------------------------------------------------------------------------
 * Batched advection of independent periodic 3D problems of uneven sizes in one
 * persistent launch per step (no counterpart in the paper: a throughput form
 * of the same SL_CEC step).
 */
typedef struct {
    void *a;            /* field buffer A (device)                         */
    void *b;            /* field buffer B (device), same size as A         */
    const void *vel;    /* 3 velocity planes (device)                      */
    int64_t dims[3];    /* x, y, z cells                                   */
    double spacing[3];  /* dx, dy, dz                                      */
    double dt;          /* time step                                       */
} sl_instance;

typedef struct sl_batch sl_batch;

/*
 * Build a batch plan for n instances (copied; the device pointers must stay
 * valid while the plan is used).  The plan owns a device instance table and a
 * work counter.  When every instance fits the persistent FP32 CEC kernel (see
 * sl_autotune) the plan launches it over all instances; otherwise a generic
 * work-queue kernel whose items are (column tile, z chunk) pairs.  tile_z is
 * the z extent of one such item; 0 takes, per instance, the planes per work
 * item cached by sl_autotune_scheme for (its dims, SL_CEC, dtype) on the
 * generic split kernel, else 32.
 */
int sl_batch_create(sl_batch **out, const sl_instance *inst, int n, int scheme,
                    int dtype, int tile_z);
/*
 * Time the plan's candidate CTA counts (1, 2 or 4 CTAs per SM, within the
 * kernel's occupancy) on even steps and keep the fastest in the plan; *best
 * (may be NULL) receives the choice, with kernel SL_KERNEL_CEC_FAST or
 * SL_KERNEL_CEC_SPLIT and the plan's tile.  Every instance's B buffer is
 * overwritten (A is only read).  Results of later steps are bitwise those of
 * the untuned plan.  sl_batch_tuning reports the plan's current launch shape.
 */
int sl_batch_autotune(sl_batch *b, sl_tuning *best, void *stream);
int sl_batch_tuning(const sl_batch *b, sl_tuning *out);
/*
 * One step of every instance: even step_index reads A and writes B with sweep
 * order x,y,z; odd step_index reads B and writes A with order z,y,x.  Only a
 * memset and a kernel launch are issued, so the call can be captured in a
 * CUDA graph.
 */
int sl_batch_step(sl_batch *b, int step_index, void *stream);
int sl_batch_destroy(sl_batch *b);

/*
 * One time step at any Courant number (Sec. 4: semi-Lagrangian schemes may
 * exceed CFL 1 when the interpolation uses non-neighbouring points).  The
 * interpolation is non-local: its corners bracket the departure point
 * X = i - C (cell units) however far it is, so an integer C is an exact shift.
 *   SL_CIR, SL_FEC, SL_BEC  the operator compositions of Sec. 2 (eqs.
 *                  intro:FEC, intro:BEC) with the unsplit multilinear
 *                  interpolation (eq. CIR2D and its 3D tensor product).
 *   SL_CEC         split 1D sweeps (order as sl_advect) with the weights of
 *                  eq. intro:CECcoefSL, 3a = 2 - 1/(U % 1), b = 1 - a, and the
 *                  correction of the local scheme taken at the departure cell:
 *                  m = trunc(C), r = C - m, j = i - m, s = sgn r,
 *                  CEC_i = L_U[Phi]_i + delta_j/2 + (1 + |r|)/6 (delta_{j-s} - delta_j).
 *                  For constant velocity this is the upwind cubic Lagrange
 *                  interpolation at the departure point (third order at every
 *                  CFL); for |C| < 1 it equals sl_advect's SL_CEC up to rounding.
 * Same arguments as sl_advect, with dtype SL_F32 or SL_F64 (SL_F32_D64 returns
 * SL_ERR_UNSUPPORTED), and dims[1], dims[2] <= 65535 (else SL_ERR_UNSUPPORTED).
 *   workspace        device memory of at least sl_advect_wide_workspace()
 *                    bytes, 256-byte aligned, owned by the caller; it holds
 *                    intermediate fields and is overwritten.  May be NULL when
 *                    that size is 0 (SL_CIR).
 *   workspace_bytes  its size.
 * The call allocates nothing and only enqueues kernels on stream (one per
 * interpolation call: 1 / 2 / 3 for CIR / FEC / BEC; for CEC one per axis
 * when a line of the grid fits the fused sweep, else 3 per axis).  A
 * non-finite Courant number, or one of magnitude 2^30 or more, sets SL_DEV_CFL
 * and is replaced by 0 (the arrival cell).
 * Errors: those of sl_advect; SL_ERR_ARG for a workspace that is too small or
 * misaligned; SL_ERR_ALIAS when out, in, vel and workspace overlap (out and
 * workspace must each be disjoint from every other buffer).
 */
int64_t sl_advect_wide_workspace(int ndim, const int64_t dims[3], int scheme, int dtype);
int sl_advect_wide(void *out, const void *in, const void *vel, int ndim,
                   const int64_t dims[3], const double spacing[3], double dt,
                   int scheme, int dtype, int step_parity, void *workspace,
                   int64_t workspace_bytes, void *stream);

/*
 * Time every candidate launch shape of the kernel serving (scheme, dtype,
 * ndim, dims, alignment of the buffers) on the given stream, cache the
 * fastest and return it in *best (may be NULL).  The buffers are the caller's
 * device memory, laid out as for sl_advect; out is overwritten (each candidate
 * runs a few steps, both sweep orders for SL_CEC), in and vel are only read.
 * Errors: those of sl_advect.
 */
int sl_autotune_scheme(void *out, const void *in, const void *vel, int ndim,
                       const int64_t dims[3], const double spacing[3], double dt,
                       int scheme, int dtype, sl_tuning *best, void *stream);

/*
 * The cached choice for (dims, scheme, dtype) in *out: SL_OK, or SL_ERR_ARG
 * when nothing is cached.
 */
int sl_tuning_get(const int64_t dims[3], int scheme, int dtype, sl_tuning *out);

/*
 * Write every cached choice to the text file at path (one line per entry:
 * nx ny nz scheme dtype kernel tile_x tile_y tile_z ctas_per_sm ms, after a
 * comment line naming the device), or read such a file back into the cache
 * (entries replace cached ones with the same key).  A choice depends on the GPU
 * model that timed it; load only files written on the same model.  Errors:
 * SL_ERR_ARG (NULL path, unreadable / unwritable file, or a malformed line:
 * nothing of the file is loaded then).  sl_tuning_clear empties the cache.
 */
int sl_tuning_save(const char *path);
int sl_tuning_load(const char *path);
int sl_tuning_clear(void);

/*
 * Former interface, kept: sl_autotune_scheme for SL_CEC; *tile_z receives the
 * chosen planes per work item of the generic kernel, or the chosen CTA count
 * (CTAs per SM times SMs) of the persistent FP32 kernel (used when dims[0] and
 * dims[1] are multiples of 32, dims[0] >= 64, dims[2] >= 8 and the buffers are
 * 16-byte aligned).
 */
int sl_autotune(void *out, const void *in, const void *vel, int ndim,
                const int64_t dims[3], const double spacing[3], double dt,
                int dtype, int *tile_z, void *stream);

/* --------------------------------------------------------------------------
 * Learned one-pass corrector (no counterpart in the paper: a throughput form
 * of the third-order step whose error is judged against the plain scheme).
 *
 * One learned step is Phi_new = L_U[Phi] + s * MLP(x), where L_U[Phi] is the
 * multilinear (CIR) value at the departure point (Sec. 3, eq. CIR2D), and the
 * MLP (67 -> 64 -> 64 -> 1, ReLU, BF16 operands with FP32 accumulation on the
 * tensor cores) reads x = the cell's 4 x 4 x 4 upwind neighbourhood
 * Phi(b - 1 .. b + 2) around the departure base b = min(floor(i - C), i),
 * shifted by L_U[Phi] and divided by s = max |Phi_k - L_U[Phi]|, plus the three
 * fractional offsets f - 1/2.  It is trained on pairs produced by the plain
 * third-order step (eqs. intro:CEC, intro:CECcoef): target (CEC - L_U[Phi])/s.
 *
 * Parameter vector (FP32, sl_corrector_param_count() = 8577 values):
 * W1 (64 x 67, row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
 */
typedef struct sl_corrector sl_corrector;

int sl_corrector_param_count(void);
/* He-initialised weights from a seeded generator; device buffers owned by c. */
int sl_corrector_create(sl_corrector **out, uint64_t seed);
int sl_corrector_destroy(sl_corrector *c);
int sl_corrector_get_params(sl_corrector *c, float *host, int n);
/* Also clears the fallback flag. */
int sl_corrector_set_params(sl_corrector *c, const float *host, int n);
/*
 * Append nsamples training rows taken at pseudo-random cells (seeded) of the
 * FP32 3D field phi with velocity vel: 67 inputs and the target
 * (target - L_U[Phi]) / s, where target is the plain SL_CEC step of phi
 * computed by the caller with the same vel, spacing and dt.  The corrector
 * keeps the rows on the device (grown as needed).
 */
int sl_corrector_add_samples(sl_corrector *c, const void *phi, const void *target, const void *vel,
                             const int64_t dims[3], const double spacing[3], double dt,
                             int nsamples, uint64_t seed, void *stream);
/* Copy rows [first, first + n) of the training set to host (68 floats each). */
int sl_corrector_get_rows(sl_corrector *c, float *host, int64_t first, int64_t n);
/*
 * iters Adam steps (beta 0.9 / 0.999) on minibatches of batch rows drawn with
 * the seed; FP32 forward and backward on the CUDA cores.  *last_loss (may be
 * NULL) receives the mean squared error of the last minibatch.  Synchronous.
 */
int sl_corrector_train(sl_corrector *c, int iters, int batch, float lr, uint64_t seed,
                       float *last_loss, void *stream);
/* Clear the fallback flag (learned steps resume). */
int sl_corrector_reset(sl_corrector *c);
/*
 * Save the network's parameters to the file at path, or load them from one
 * written by sl_corrector_save (a JSON header line, then the 8577 FP32 values
 * and their FNV-1a checksum, as sl_field_save).  Loading replaces the
 * parameters as sl_corrector_set_params does (and clears the fallback state).
 * Errors: SL_ERR_ARG (NULL argument, unreadable / unwritable file, a file of
 * another kind or network, a short payload, trailing bytes or a checksum
 * mismatch: nothing is loaded then), SL_ERR_CUDA.  Synchronous.
 */
int sl_corrector_save(sl_corrector *c, const char *path);
int sl_corrector_load(sl_corrector *c, const char *path);
/*
 * One step with the corrector: FP32 fields, ndim = 3, dims[0] % 32 == 0,
 * dims[1] % 4 == 0, dims[2] >= 3, in 16-byte aligned (else SL_ERR_UNSUPPORTED).
 * With check == 0 the learned step runs
 * (or the plain SL_CEC step with step_parity once the corrector has fallen
 * back).  With check != 0 the plain SL_CEC and SL_BEC steps of the same input
 * are also computed; the learned error is ||learned - CEC|| / ||CEC|| and the
 * plain error ||BEC - CEC|| / ||CEC|| (the distance of the second-order
 * scheme from the third-order one).  If the learned error exceeds
 * fallback_ratio times the plain error, out receives the plain step and the
 * corrector falls back for good (until sl_corrector_reset).  errs (may be NULL)
 * receives the two errors; *used_plain (may be NULL) the fallback flag.
 * A checked step synchronises the stream.
 */
int sl_advect_learned(sl_corrector *c, void *out, const void *in, const void *vel, int ndim,
                      const int64_t dims[3], const double spacing[3], double dt, int step_parity,
                      int check, double fallback_ratio, int *used_plain, double errs[2], void *stream);

/* ------------------------------------------------------------------------
 * Rayleigh-Benard box (Sec. 6, eqs. e:nsnd, e:Tnd, e:mnd, e:poisson, e:proj).
 *
 * A 2D box of nx x nz cells over Lx x Lz (x fastest, z upwards; the paper's
 * box has Lz / Lx = 0.5, Pr = 1), no-slip impermeable walls, theta = 0 on the
 * plates and d theta / dx = 0 on the side walls.  The state is the velocity
 * U = (u, w) and the temperature perturbation theta, cell-centred.  One step
 * from step n:
 *   ghost layers (3 per side) of u, w, theta := the walls' mirror images
 *     (u, w change sign across every wall, theta across the plates only);
 *   (u1, w1, theta1) := the chosen scheme's step of u, w and theta by U^n on
 *     the padded grid (the SL_CEC sweep order alternates with the step index);
 *   u2 = u1 + dt Pr lap u^n, w2 = w1 + dt (Ra Pr theta^n + Pr lap w^n),
 *   theta^{n+1} = theta1 + dt (w^n + lap theta^n)   (5-point Laplacians);
 *   faces: averages of the adjacent cells of (u2, w2), zero on the walls;
 *   lap phi = div faces with d phi / dn = 0, zero-mean phi;
 *   U^{n+1} = U2 - (cell average of the two face gradients of phi).
 * The projected faces are divergence-free up to rounding.
 *
 * sl_rb_create: nx, nz in [4, 4096]; Lx, Lz > 0; Ra finite; Pr >= 0;
 *   scheme sl_scheme; dtype SL_F64 or SL_F32 (the arithmetic of every step).
 *   Allocates all device buffers on the current device (about
 *   12 (nx + 6)(nz + 6) + 3 nx nz + 2 nx^2 + nz^2 elements); the state starts at
 *   rest (U = 0, theta = 0).  Errors: SL_ERR_ARG, SL_ERR_UNSUPPORTED,
 *   SL_ERR_NOMEM, SL_ERR_CUDA.
 * sl_rb_set_state / sl_rb_get_state: DEVICE arrays of nz x nx elements of the
 *   box's dtype (row-major, x fastest) for u, w and theta, copied in / out on
 *   stream; set_state also resets the step index to 0.  Errors: SL_ERR_ARG.
 * sl_rb_step: nsteps steps of size dt on stream (enqueued, not waited for).
 *   Runs of 16 steps or more replay a CUDA graph of 8 steps, captured on the
 *   box's own stream for this dt (again when dt changes); the results equal
 *   those of single steps bit for bit.
 *   The advection needs |u| dt / dx and |w| dt / dz below 1 (the kernels'
 *   stencil reach; sl_device_status flags a violation).  Errors: SL_ERR_ARG
 *   (NULL box, nsteps < 0, non-finite dt, a box of another device), and those
 *   of sl_advect_multi.
 * sl_rb_destroy: frees the box (NULL is a no-op); the caller makes sure none
 *   of its steps is still running.
 */
typedef struct sl_rb sl_rb;
int sl_rb_create(sl_rb **out, int nx, int nz, double Lx, double Lz, double Ra, double Pr, int scheme,
                 int dtype);
int sl_rb_set_state(sl_rb *rb, const void *u, const void *w, const void *theta, void *stream);
int sl_rb_get_state(sl_rb *rb, void *u, void *w, void *theta, void *stream);
int sl_rb_step(sl_rb *rb, double dt, int nsteps, void *stream);
int sl_rb_destroy(sl_rb *rb);

#ifdef __cplusplus
}
#endif

#endif /* SL_H */
