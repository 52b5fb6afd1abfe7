// sl_io.cu -- checkpoint files of fields and of the learned corrector's
// weights (declared in include/sl.h).  The paper has no counterpart: long
// runs (the 2000-step time-reversal run, trained weights) need to stop and
// resume.
//
// A file is one JSON header line followed by the raw little-endian payload:
//   {"format": "libsl-field", "version": 1, "ndim": 3, "dims": [nx, ny, nz],
//    "dtype": "f32", "step": k, "bytes": N, "fnv1a64": "0123456789abcdef"}
//   {"format": "libsl-corrector", "version": 1, "params": 8577, "bytes": N,
//    "fnv1a64": "..."}
// The checksum is the 64-bit FNV-1a hash of the payload (Fowler, Noll and Vo:
// offset basis 14695981039346656037, prime 1099511628211), so that a
// truncated or corrupted file is refused instead of loaded.
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sl.h"
#include "sl_internal.h"

namespace sl {
namespace {

uint64_t fnv1a64(const unsigned char *p, size_t n)
{
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

const char *dtype_name(int dtype) { return dtype == SL_F64 ? "f64" : (dtype == SL_F32_D64 ? "f32_d64" : "f32"); }

int io_fail(int code, const char *fmt, const char *a = "", long long b = 0)
{
    char buf[512];
    std::snprintf(buf, sizeof buf, fmt, a, b);
    return set_error(code, buf);
}

// Write header + payload to path; returns SL_OK or SL_ERR_ARG.
int write_file(const char *path, const char *header, const std::vector<unsigned char> &payload)
{
    FILE *f = std::fopen(path, "wb");
    if (!f) return io_fail(SL_ERR_ARG, "cannot write %s", path);
    bool ok = std::fputs(header, f) >= 0;
    ok = ok && std::fwrite(payload.data(), 1, payload.size(), f) == payload.size();
    ok = std::fclose(f) == 0 && ok;
    return ok ? SL_OK : io_fail(SL_ERR_ARG, "write error on %s", path);
}

// Read the header line (at most 511 characters) and exactly `bytes` payload
// bytes, and check the payload's FNV-1a hash against `hash_hex`.
int read_payload(FILE *f, const char *path, int64_t bytes, const char *hash_hex, std::vector<unsigned char> &payload)
{
    payload.resize((size_t)bytes);
    if (bytes > 0 && std::fread(payload.data(), 1, (size_t)bytes, f) != (size_t)bytes)
        return io_fail(SL_ERR_ARG, "%s: payload shorter than its header says", path);
    if (std::fgetc(f) != EOF) return io_fail(SL_ERR_ARG, "%s: trailing bytes after the payload", path);
    char want[17];
    std::snprintf(want, sizeof want, "%016" PRIx64, fnv1a64(payload.data(), payload.size()));
    if (std::strcmp(want, hash_hex) != 0) return io_fail(SL_ERR_ARG, "%s: payload checksum mismatch", path);
    return SL_OK;
}

bool read_header(FILE *f, char (&line)[512])
{
    if (!std::fgets(line, sizeof line, f)) return false;
    const size_t n = std::strlen(line);
    return n > 0 && line[n - 1] == '\n';
}

}  // namespace
}  // namespace sl

using namespace sl;

extern "C" {

int sl_field_save(const char *path, const void *field, int ndim, const int64_t dims[3], int dtype, int64_t step,
                  void *stream)
{
    if (!path || !field || !dims) return io_fail(SL_ERR_ARG, "path, field and dims must not be NULL%s", "");
    if (ndim != 2 && ndim != 3) return io_fail(SL_ERR_ARG, "ndim must be 2 or 3%s", "");
    if (dtype < SL_F32 || dtype > SL_F32_D64) return io_fail(SL_ERR_ARG, "unknown dtype%s", "");
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1 || dims[d] > (int64_t(1) << 30)) return io_fail(SL_ERR_ARG, "dims out of range%s", "");
    if (ndim == 2 && dims[2] != 1) return io_fail(SL_ERR_ARG, "dims[2] must be 1 when ndim = 2%s", "");
    const int64_t ncell = dims[0] * dims[1] * dims[2];
    if (ncell > (int64_t(1) << 40)) return io_fail(SL_ERR_ARG, "grid too large%s", "");
    const int64_t bytes = ncell * (dtype == SL_F64 ? 8 : 4);
    std::vector<unsigned char> payload;
    try {
        payload.resize((size_t)bytes);
    } catch (...) {
        return io_fail(SL_ERR_NOMEM, "host buffer of %s%lld bytes", "", (long long)bytes);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(payload.data(), field, (size_t)bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return io_fail(SL_ERR_CUDA, "device to host copy: %s", cudaGetErrorString(e));
    char header[512];
    std::snprintf(header, sizeof header,
                  "{\"format\": \"libsl-field\", \"version\": 1, \"ndim\": %d, \"dims\": [%lld, %lld, %lld], "
                  "\"dtype\": \"%s\", \"step\": %lld, \"bytes\": %lld, \"fnv1a64\": \"%016" PRIx64 "\"}\n",
                  ndim, (long long)dims[0], (long long)dims[1], (long long)dims[2], dtype_name(dtype),
                  (long long)step, (long long)bytes, fnv1a64(payload.data(), payload.size()));
    return write_file(path, header, payload);
}

int sl_field_load(const char *path, void *field, int ndim, const int64_t dims[3], int dtype, int64_t *step,
                  void *stream)
{
    if (!path || !field || !dims) return io_fail(SL_ERR_ARG, "path, field and dims must not be NULL%s", "");
    FILE *f = std::fopen(path, "rb");
    if (!f) return io_fail(SL_ERR_ARG, "cannot read %s", path);
    char line[512];
    int nd = 0;
    long long nx = 0, ny = 0, nz = 0, stp = 0, bytes = -1;
    char dt[16] = {0}, hash[32] = {0};
    const bool parsed =
        read_header(f, line) &&
        std::sscanf(line,
                    "{\"format\": \"libsl-field\", \"version\": 1, \"ndim\": %d, \"dims\": [%lld, %lld, %lld], "
                    "\"dtype\": \"%15[a-z0-9_]\", \"step\": %lld, \"bytes\": %lld, \"fnv1a64\": \"%16[0-9a-f]\"}",
                    &nd, &nx, &ny, &nz, dt, &stp, &bytes, hash) == 8;
    if (!parsed) {
        std::fclose(f);
        return io_fail(SL_ERR_ARG, "%s: not a libsl field file", path);
    }
    if (nd != ndim || nx != dims[0] || ny != dims[1] || nz != dims[2] || std::strcmp(dt, dtype_name(dtype)) != 0) {
        std::fclose(f);
        return io_fail(SL_ERR_ARG, "%s: the file holds another grid or type", path);
    }
    const int64_t want = dims[0] * dims[1] * dims[2] * (dtype == SL_F64 ? 8 : 4);
    if (bytes != want) {
        std::fclose(f);
        return io_fail(SL_ERR_ARG, "%s: payload size does not match the grid", path);
    }
    std::vector<unsigned char> payload;
    int rc;
    try {
        rc = read_payload(f, path, want, hash, payload);
    } catch (...) {
        rc = io_fail(SL_ERR_NOMEM, "host buffer of %s%lld bytes", "", (long long)want);
    }
    std::fclose(f);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(field, payload.data(), (size_t)want, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return io_fail(SL_ERR_CUDA, "host to device copy: %s", cudaGetErrorString(e));
    if (step) *step = stp;
    return SL_OK;
}

int sl_corrector_save(sl_corrector *c, const char *path)
{
    if (!c || !path) return io_fail(SL_ERR_ARG, "corrector and path must not be NULL%s", "");
    const int n = sl_corrector_param_count();
    std::vector<unsigned char> payload((size_t)n * 4);
    int rc = sl_corrector_get_params(c, reinterpret_cast<float *>(payload.data()), n);
    if (rc) return rc;
    char header[256];
    std::snprintf(header, sizeof header,
                  "{\"format\": \"libsl-corrector\", \"version\": 1, \"params\": %d, \"bytes\": %d, "
                  "\"fnv1a64\": \"%016" PRIx64 "\"}\n",
                  n, 4 * n, fnv1a64(payload.data(), payload.size()));
    return write_file(path, header, payload);
}

int sl_corrector_load(sl_corrector *c, const char *path)
{
    if (!c || !path) return io_fail(SL_ERR_ARG, "corrector and path must not be NULL%s", "");
    FILE *f = std::fopen(path, "rb");
    if (!f) return io_fail(SL_ERR_ARG, "cannot read %s", path);
    char line[512];
    int np = 0, bytes = -1;
    char hash[32] = {0};
    const bool parsed =
        read_header(f, line) &&
        std::sscanf(line,
                    "{\"format\": \"libsl-corrector\", \"version\": 1, \"params\": %d, \"bytes\": %d, "
                    "\"fnv1a64\": \"%16[0-9a-f]\"}",
                    &np, &bytes, hash) == 3;
    const int n = sl_corrector_param_count();
    if (!parsed || np != n || bytes != 4 * n) {
        std::fclose(f);
        return io_fail(SL_ERR_ARG, "%s: not a libsl corrector file of this network", path);
    }
    std::vector<unsigned char> payload;
    const int rc = read_payload(f, path, 4 * n, hash, payload);
    std::fclose(f);
    if (rc) return rc;
    return sl_corrector_set_params(c, reinterpret_cast<const float *>(payload.data()), n);
}

}  // extern "C"
