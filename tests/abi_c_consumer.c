/* A plain C program using the gather through its C ABI only (include/ssilvb.h): CUDA runtime
 * allocations, ssilvb_create / ssilvb_gather / ssilvb_get_status / ssilvb_destroy, and the error
 * path.  The scene is a fronto-parallel plane, which occludes nothing (Section 3.1): with slices on
 * multiples of pi/4 and no noise every sample lies in the tangent plane, so AO = 1 and GI = 0
 * exactly.  Prints "OK" and exits 0 on success. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "ssilvb.h"

#define CHECK(x)                                                                      \
    do {                                                                              \
        if (!(x)) {                                                                   \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #x);           \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

int main(void) {
    const int W = 64, H = 48;
    const size_t npx = (size_t)W * H;
    float *h_depth = (float *)malloc(npx * 4), *h_px = (float *)malloc(npx * 16), *h_out = (float *)malloc(npx * 16);
    CHECK(h_depth && h_px && h_out);
    for (size_t i = 0; i < npx; ++i) {
        h_depth[i] = 5.0f;
        h_px[4 * i + 0] = 0.0f;
        h_px[4 * i + 1] = 0.0f;
        h_px[4 * i + 2] = 1.0f;  /* normal facing the camera; reused as radiance (0, 0, 1) */
        h_px[4 * i + 3] = 0.0f;
    }
    float *d_depth = NULL, *d_px = NULL, *d_out = NULL;
    CHECK(cudaMalloc((void **)&d_depth, npx * 4) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_px, npx * 16) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_out, npx * 16) == cudaSuccess);
    CHECK(cudaMemcpy(d_depth, h_depth, npx * 4, cudaMemcpyHostToDevice) == cudaSuccess);
    CHECK(cudaMemcpy(d_px, h_px, npx * 16, cudaMemcpyHostToDevice) == cudaSuccess);

    ssilvb_ctx *ctx = NULL;
    CHECK(ssilvb_create(&ctx, 0) == SSILVB_OK && ctx != NULL);

    ssilvb_gbuffer g;
    memset(&g, 0, sizeof(g));
    g.width = W;
    g.height = H;
    g.depth = d_depth;
    g.depth_pitch = (size_t)W * 4;
    g.normal = d_px;
    g.normal_pitch = (size_t)W * 16;
    g.normal_fmt = SSILVB_FMT_F32X4;
    g.radiance = d_px;
    g.radiance_pitch = (size_t)W * 16;
    g.radiance_fmt = SSILVB_FMT_F32X4;
    ssilvb_camera cam = {32.0f, 32.0f, 32.0f, 24.0f, {1, 0, 0, 0, 1, 0, 0, 0, 1}};
    ssilvb_params p;
    memset(&p, 0, sizeof(p));
    p.num_slices = 4;
    p.steps_per_side = 8;
    p.radius = 2.0f;
    p.thickness = 0.5f;
    p.sector_count = 32;
    p.compute_gi = 1;
    p.noise_mode = 0;
    ssilvb_output o;
    memset(&o, 0, sizeof(o));
    o.out0 = d_out;
    o.out0_pitch = (size_t)W * 16;

    CHECK(ssilvb_gather(ctx, &g, &cam, &p, &o, NULL) == SSILVB_OK);
    CHECK(ssilvb_get_status(ctx, NULL) == SSILVB_OK);
    CHECK(cudaMemcpy(h_out, d_out, npx * 16, cudaMemcpyDeviceToHost) == cudaSuccess);
    for (size_t i = 0; i < npx; ++i) {
        CHECK(h_out[4 * i + 0] == 0.0f && h_out[4 * i + 1] == 0.0f && h_out[4 * i + 2] == 0.0f);
        CHECK(h_out[4 * i + 3] == 1.0f);
    }

    /* the error path: an invalid parameter enqueues nothing and says why */
    p.num_slices = 0;
    CHECK(ssilvb_gather(ctx, &g, &cam, &p, &o, NULL) == SSILVB_ERR_INVALID_ARG);
    CHECK(strlen(ssilvb_last_error(ctx)) > 0);
    CHECK(strcmp(ssilvb_status_string(SSILVB_ERR_INVALID_ARG), "SSILVB_ERR_INVALID_ARG") == 0);

    CHECK(ssilvb_destroy(ctx) == SSILVB_OK);
    cudaFree(d_depth);
    cudaFree(d_px);
    cudaFree(d_out);
    free(h_depth);
    free(h_px);
    free(h_out);
    printf("OK\n");
    return 0;
}
