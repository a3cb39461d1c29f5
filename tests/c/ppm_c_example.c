/* The library through its C ABI alone, as a C program would use it: device
 * arrays from the CUDA runtime, no Python.  A 64 x 64 grid of hit points on
 * the plane z = 0 and 100,000 photons per iteration, uniform on the unit
 * square with flux 1/J and none for x > 0.5 (a shadow).  Checks the
 * estimate against the known irradiance (1 where lit, exactly 0 in the
 * shadow), the counters, host-fed iterations and the error codes.
 * Exit status 0 on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "ppm.h"

#define NSIDE 64
#define NH (NSIDE * NSIDE)
#define J 100000
#define ITERS 8
#define R0 0.02f

static int fail(const char* what, int code)
{
    fprintf(stderr, "FAIL: %s (%d: %s)\n", what, code, ppm_strerror(code));
    return 1;
}

#define CHECK(call)                                   \
    do {                                              \
        int rc_ = (call);                             \
        if (rc_ != PPM_OK) return fail(#call, rc_);   \
    } while (0)

#define CUDA(call)                                                            \
    do {                                                                      \
        if ((call) != cudaSuccess) { fprintf(stderr, "FAIL: %s\n", #call); return 1; } \
    } while (0)

/* xorshift64*: a small seeded generator for the photon positions */
static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static float uniform01(void)
{
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return (float)((rng_state * 0x2545F4914F6CDD1Dull) >> 40) * (1.0f / 16777216.0f);
}

static void make_photons(float* pos, float* flux)
{
    for (int i = 0; i < J; ++i) {
        const float x = uniform01(), y = uniform01();
        pos[3 * i] = x;
        pos[3 * i + 1] = y;
        pos[3 * i + 2] = 0.f;
        flux[i] = x > 0.5f ? 0.f : 1.0f / J;
    }
}

int main(void)
{
    /* hit points, host side */
    static float hpos[NH * 3], hu[NH * 3], hv[NH * 3];
    for (int j = 0; j < NSIDE; ++j)
        for (int i = 0; i < NSIDE; ++i) {
            const int h = j * NSIDE + i;
            hpos[3 * h] = (i + 0.5f) / NSIDE;
            hpos[3 * h + 1] = (j + 0.5f) / NSIDE;
            hpos[3 * h + 2] = 0.f;
            hu[3 * h] = 1.f; hu[3 * h + 1] = 0.f; hu[3 * h + 2] = 0.f;
            hv[3 * h] = 0.f; hv[3 * h + 1] = 1.f; hv[3 * h + 2] = 0.f;
        }
    float *d_pos, *d_u, *d_v, *d_ppos, *d_flux, *d_L;
    CUDA(cudaMalloc((void**)&d_pos, sizeof(hpos)));
    CUDA(cudaMalloc((void**)&d_u, sizeof(hu)));
    CUDA(cudaMalloc((void**)&d_v, sizeof(hv)));
    CUDA(cudaMalloc((void**)&d_ppos, sizeof(float) * 3 * J));
    CUDA(cudaMalloc((void**)&d_flux, sizeof(float) * J));
    CUDA(cudaMalloc((void**)&d_L, sizeof(float) * NH));
    CUDA(cudaMemcpy(d_pos, hpos, sizeof(hpos), cudaMemcpyHostToDevice));
    CUDA(cudaMemcpy(d_u, hu, sizeof(hu), cudaMemcpyHostToDevice));
    CUDA(cudaMemcpy(d_v, hv, sizeof(hv), cudaMemcpyHostToDevice));

    /* errors are codes, never crashes */
    ppm_ctx* ctx = NULL;
    if (ppm_create(NULL, R0, 0.75f, NULL, NULL, &ctx) != PPM_EINVAL || ctx != NULL)
        return fail("ppm_create(NULL hit points) must be PPM_EINVAL", -99);

    ppm_hitpoints hp = {NH, d_pos, d_u, d_v, NULL, NULL};
    ppm_params prm;
    ppm_default_params(&prm);
    CHECK(ppm_create(&hp, R0, 0.75f, &prm, NULL, &ctx));

    float* ppos = (float*)malloc(sizeof(float) * 3 * J);
    float* pflux = (float*)malloc(sizeof(float) * J);
    if (!ppos || !pflux) return fail("malloc", -98);
    ppm_photons ph = {J, J, d_ppos, d_flux, 1, 0, NULL, NULL, NULL};
    for (int it = 1; it <= ITERS; ++it) {
        make_photons(ppos, pflux);
        CUDA(cudaMemcpy(d_ppos, ppos, sizeof(float) * 3 * J, cudaMemcpyHostToDevice));
        CUDA(cudaMemcpy(d_flux, pflux, sizeof(float) * J, cudaMemcpyHostToDevice));
        CHECK(ppm_build_grid(ctx, &ph));
        CHECK(ppm_gather_test_update(ctx, it));
    }
    if (ppm_gather_test_update(ctx, ITERS + 1) != PPM_ESTATE)      /* no grid built since */
        return fail("gather without a new grid must be PPM_ESTATE", -97);

    /* two more iterations fed from host memory */
    for (int it = ITERS + 1; it <= ITERS + 2; ++it) {
        make_photons(ppos, pflux);
        ppm_photons hph = {J, J, ppos, pflux, 1, 0, NULL, NULL, NULL};
        CHECK(ppm_iterate_host(ctx, &hph, it));
        ppm_iter_stats hs;
        CHECK(ppm_stats_host(ctx, it, &hs));           /* the arrays may change after this */
        if (hs.iter != it || hs.pairs <= 0) return fail("host-fed counters", -96);
    }
    ppm_iter_stats st;
    CHECK(ppm_stats(ctx, &st));
    if (st.iter != ITERS + 2 || st.pairs <= 0 || st.flags != 0) return fail("counters", -95);

    /* the estimate: irradiance 1 where the whole disk is lit, 0 where dark */
    static float L[NH];
    CHECK(ppm_radiance(ctx, d_L));
    CUDA(cudaMemcpy(L, d_L, sizeof(L), cudaMemcpyDeviceToHost));
    double sum = 0.0;
    int lit = 0, dark = 0;
    for (int h = 0; h < NH; ++h) {
        const float x = hpos[3 * h], y = hpos[3 * h + 1];
        const int inside = y > R0 && y < 1.f - R0 && x > R0;
        if (inside && x < 0.5f - R0) {
            if (!(L[h] > 0.5f && L[h] < 1.5f)) return fail("lit estimate out of range", -94);
            sum += L[h];
            ++lit;
        } else if (x > 0.5f + R0 && L[h] != 0.f) {
            return fail("shadowed estimate not zero", -93);
        } else if (x > 0.5f + R0) {
            ++dark;
        }
    }
    const double mean = sum / lit;
    if (fabs(mean - 1.0) > 0.02) return fail("mean lit estimate not within 2% of 1", -92);
    printf("ok: %d hit points, %d iterations, %lld pairs in the last; lit mean %.4f over %d, %d dark at 0\n",
           NH, ITERS + 2, (long long)st.pairs, mean, lit, dark);

    ppm_destroy(ctx);
    free(ppos);
    free(pflux);
    cudaFree(d_pos); cudaFree(d_u); cudaFree(d_v); cudaFree(d_ppos); cudaFree(d_flux); cudaFree(d_L);
    return 0;
}
