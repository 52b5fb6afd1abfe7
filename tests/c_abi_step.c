/* A plain C user of libsl: two CEC steps (both sweep orders) of a seeded
 * field on a 64 x 64 x 32 grid with constant Courant numbers, through device
 * buffers (sl_advect) and through host buffers (sl_advect_host).  The two
 * results must agree bit for bit (checked here); the device result is
 * written to argv[1] as raw floats for the test to compare with the Python
 * binding and the FP64 oracle.  Exit status: 0 on success.
 *
 * Built by tests/test_gpu_c_abi.py:
 *   gcc -O1 c_abi_step.c -I include -I <cuda>/include -L <lib dir> -lsl -L <cuda>/lib64 -lcudart */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "sl.h"

#define NX 64
#define NY 64
#define NZ 32
#define NCELL (NX * NY * NZ)

/* the seeded inputs: a 32-bit LCG mapped to [-1, 1) */
static float lcg(uint32_t *s)
{
    *s = *s * 1664525u + 1013904223u;
    return (float)((*s >> 8) * (1.0 / 16777216.0)) * 2.0f - 1.0f;
}

static int check(int rc, const char *what)
{
    if (rc != SL_OK) fprintf(stderr, "%s: %d %s\n", what, rc, sl_last_error());
    return rc != SL_OK;
}

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    const size_t fb = sizeof(float) * NCELL;
    float *phi = malloc(fb), *vel = malloc(3 * fb), *out_h = malloc(fb), *out_d = malloc(fb);
    if (!phi || !vel || !out_h || !out_d) return 3;
    uint32_t s = 12345u;
    for (int i = 0; i < NCELL; ++i) phi[i] = lcg(&s);
    const double spacing[3] = {0.5, 0.25, 2.0}, dt = 0.1;
    const double courant[3] = {0.3, -0.2, 0.45};
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < NCELL; ++i) vel[(size_t)d * NCELL + i] = (float)(courant[d] * spacing[d] / dt);
    const int64_t dims[3] = {NX, NY, NZ};

    float *d_a, *d_b, *d_v;
    if (cudaMalloc((void **)&d_a, fb) || cudaMalloc((void **)&d_b, fb) || cudaMalloc((void **)&d_v, 3 * fb)) return 4;
    if (cudaMemcpy(d_a, phi, fb, cudaMemcpyHostToDevice) || cudaMemcpy(d_v, vel, 3 * fb, cudaMemcpyHostToDevice))
        return 4;
    /* step 0 (x,y,z) then step 1 (z,y,x) on the device */
    if (check(sl_advect(d_b, d_a, d_v, 3, dims, spacing, dt, SL_CEC, SL_F32, 0, NULL), "sl_advect 0")) return 5;
    if (check(sl_advect(d_a, d_b, d_v, 3, dims, spacing, dt, SL_CEC, SL_F32, 1, NULL), "sl_advect 1")) return 5;
    if (cudaMemcpy(out_d, d_a, fb, cudaMemcpyDeviceToHost)) return 4;
    /* the same two steps on host buffers */
    if (check(sl_advect_host(out_h, phi, vel, 3, dims, spacing, dt, SL_CEC, SL_F32, 0, NULL), "host 0")) return 5;
    memcpy(phi, out_h, fb);
    if (check(sl_advect_host(out_h, phi, vel, 3, dims, spacing, dt, SL_CEC, SL_F32, 1, NULL), "host 1")) return 5;
    if (memcmp(out_h, out_d, fb) != 0) {
        fprintf(stderr, "host and device results differ\n");
        return 6;
    }
    unsigned status = 0;
    if (check(sl_device_status(NULL, &status), "status") || status != 0) return 7;
    FILE *f = fopen(argv[1], "wb");
    if (!f || fwrite(out_d, sizeof(float), NCELL, f) != NCELL) return 8;
    fclose(f);
    cudaFree(d_a);
    cudaFree(d_b);
    cudaFree(d_v);
    printf("C_ABI_OK\n");
    return 0;
}
