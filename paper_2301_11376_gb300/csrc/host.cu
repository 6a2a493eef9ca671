// Host-buffer entry points: ssilvb_gather_host (synchronous) and ssilvb_gather_host_async.
//
// A frame's G-buffer goes host to device into staging the context owns, the gather runs in row
// bands, and each band's outputs go back to the host while later bands still compute (every band
// reads the whole frame's inputs, so the inputs go first).  The synchronous call borrows the
// caller's stream for its inputs and every other band and returns when the outputs are in host
// memory.  The asynchronous call alternates between two lanes on context streams and returns at
// once, so one frame's copies overlap its neighbours' gathers; ssilvb_synchronize waits for them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ssilvb {

static void release_lane(HostLane &L) {
    for (cudaEvent_t &ev : L.band_done)
        if (ev) cudaEventDestroy(ev), ev = nullptr;
    for (cudaEvent_t *ev : {&L.inputs_ready, &L.comp1_done, &L.done})
        if (*ev) cudaEventDestroy(*ev), *ev = nullptr;
    if (L.stage) cudaFree(L.stage), L.stage = nullptr;
    L.stage_bytes = 0;
    L.pending = false;
}

static cudaError_t create_lane_events(HostLane &L) {
    cudaError_t e = cudaSuccess;
    for (cudaEvent_t &ev : L.band_done)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (cudaEvent_t *ev : {&L.inputs_ready, &L.comp1_done, &L.done})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    return e;
}

void release_host_resources(ssilvb_ctx *ctx) {
    release_lane(ctx->sync_lane);
    for (HostLane &L : ctx->async_lane) release_lane(L);
    for (cudaStream_t *s : {&ctx->host_band, &ctx->host_copy, &ctx->async_in, &ctx->async_comp[0],
                            &ctx->async_comp[1], &ctx->async_out})
        if (*s) cudaStreamDestroy(*s), *s = nullptr;
    if (ctx->host_entry) cudaEventDestroy(ctx->host_entry), ctx->host_entry = nullptr;
    ctx->host_ready = false;
}

// Streams and events of both host-buffer paths, all or none (a partial set is released).
static cudaError_t create_host_resources(ssilvb_ctx *ctx) {
    cudaError_t e = cudaSuccess;
    for (cudaStream_t *s : {&ctx->host_band, &ctx->host_copy, &ctx->async_in, &ctx->async_comp[0],
                            &ctx->async_comp[1], &ctx->async_out})
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->host_entry, cudaEventDisableTiming);
    if (e == cudaSuccess) e = create_lane_events(ctx->sync_lane);
    for (HostLane &L : ctx->async_lane) {
        if (e == cudaSuccess) e = create_lane_events(L);
        L.in = ctx->async_in;
        L.comp[0] = ctx->async_comp[0];
        L.comp[1] = ctx->async_comp[1];
        L.out = ctx->async_out;
    }
    ctx->sync_lane.comp[1] = ctx->host_band;
    ctx->sync_lane.out = ctx->host_copy;
    if (e != cudaSuccess) release_host_resources(ctx);
    else ctx->host_ready = true;
    return e;
}

ssilvb_status wait_host_async(ssilvb_ctx *ctx) {
    for (HostLane &L : ctx->async_lane) {
        if (!L.pending) continue;
        const cudaError_t e = cudaEventSynchronize(L.done);
        L.pending = false;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "asynchronous host-buffer gather");
    }
    return SSILVB_OK;
}

// Wait (on the host) for everything the lane has enqueued; used before its staging is replaced
// and after a failed enqueue, so that no copy writes the caller's buffers after the call returns.
static void drain_lane(HostLane &L) {
    for (cudaStream_t s : {L.in, L.comp[0], L.comp[1], L.out})
        if (s) cudaStreamSynchronize(s);
    L.pending = false;
}

// Enqueue one frame on lane L: staging (grown on demand), host-to-device copies on L.in, row bands
// alternating between L.comp[0] and L.comp[1], each band's outputs back on L.out; L.done marks the
// end.  Inputs were validated by the caller.
static ssilvb_status enqueue_frame(ssilvb_ctx *ctx, HostLane &L, const ssilvb_gbuffer *gbuffer,
                                   const ssilvb_camera *camera, const ssilvb_params *params,
                                   const ssilvb_output *out) {
    const size_t W = gbuffer->width, H = gbuffer->height;
    // bytes per pixel of one normal / radiance plane; F16X8 is one plane holding both
    const bool nr16 = gbuffer->normal_fmt == SSILVB_FMT_F16X8;
    const size_t px = gbuffer->normal_fmt == SSILVB_FMT_F16X4 ? 8 : 16;
    const int na = params->ambient_cones;
    const size_t melem = params->sector_count / 8;
    const size_t mask_bytes = out->masks ? (size_t)params->num_slices * W * H * melem : 0;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t b_depth = up(W * H * 4), b_px = up(W * H * px), b_out = up(W * H * 16);
    const size_t b_light = out->light_out ? up(W * H * px) : 0;
    const size_t b_direct = (out->light_out && gbuffer->direct) ? up(W * H * px) : 0;
    const size_t need = b_depth + (nr16 ? 1 : 2) * b_px + b_out + (na > 0 ? b_out : 0) + up(mask_bytes) + b_light +
                        b_direct;
    if (need > L.stage_bytes) {
        if (L.stage) {
            drain_lane(L);
            cudaFree(L.stage);
            L.stage = nullptr;
            L.stage_bytes = 0;
        }
        if (cudaMalloc(&L.stage, need) != cudaSuccess) {
            cudaGetLastError();
            L.stage = nullptr;
            return fail(ctx, SSILVB_ERR_OUT_OF_MEMORY, "staging allocation of %zu bytes failed", need);
        }
        L.stage_bytes = need;
    }
    char *base = static_cast<char *>(L.stage);
    float *d_depth = reinterpret_cast<float *>(base);
    char *d_normal = base + b_depth;
    char *d_rad = nr16 ? d_normal : d_normal + b_px;
    char *d_out0 = d_rad + b_px;
    char *d_out1 = na > 0 ? d_out0 + b_out : nullptr;
    char *d_masks = out->masks ? d_out0 + b_out + (na > 0 ? b_out : 0) : nullptr;
    char *d_light = out->light_out ? d_out0 + b_out + (na > 0 ? b_out : 0) + up(mask_bytes) : nullptr;
    char *d_direct = b_direct ? d_out0 + b_out + (na > 0 ? b_out : 0) + up(mask_bytes) + b_light : nullptr;

    cudaError_t e = cudaMemcpy2DAsync(d_depth, W * 4, gbuffer->depth, gbuffer->depth_pitch, W * 4, H,
                                      cudaMemcpyHostToDevice, L.in);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_normal, W * px, gbuffer->normal, gbuffer->normal_pitch, W * px, H,
                              cudaMemcpyHostToDevice, L.in);
    if (e == cudaSuccess && !nr16)
        e = cudaMemcpy2DAsync(d_rad, W * px, gbuffer->radiance, gbuffer->radiance_pitch, W * px, H,
                              cudaMemcpyHostToDevice, L.in);
    if (e == cudaSuccess && d_direct)
        e = cudaMemcpy2DAsync(d_direct, W * px, gbuffer->direct, gbuffer->direct_pitch, W * px, H,
                              cudaMemcpyHostToDevice, L.in);
    if (e == cudaSuccess) e = cudaEventRecord(L.inputs_ready, L.in);
    for (cudaStream_t c : L.comp)
        if (e == cudaSuccess && c != L.in) e = cudaStreamWaitEvent(c, L.inputs_ready, 0);

    ssilvb_gbuffer dg = *gbuffer;
    dg.depth = d_depth;
    dg.depth_pitch = W * 4;
    dg.normal = d_normal;
    dg.normal_pitch = W * px;
    dg.radiance = d_rad;
    dg.radiance_pitch = W * px;
    dg.direct = d_direct;
    dg.direct_pitch = d_direct ? W * px : 0;
    const ssilvb_output dout = {reinterpret_cast<float *>(d_out0), W * 16, reinterpret_cast<float *>(d_out1), W * 16,
                                d_masks, d_light, W * px};
    GatherParams P;
    fill_params(P, &dg, camera, params, &dout);
    const KernelChoice k = resolve_choice(ctx, tune_key(gbuffer, params, 0));
    // Row bands, one launch each, for frames of 512+ rows.  Bands alternate between two streams, so
    // that one band's last wave overlaps the next band's first instead of draining the GPU between
    // launches.  Band b gets a share of the rows proportional to 10 - b: the last band, whose copy
    // nothing hides, is the smallest.
    const int bands = (int)std::max<size_t>(1, std::min<size_t>(kMaxHostBands, H / 256));
    size_t cut[kMaxHostBands + 1] = {0};
    {
        size_t wsum = 0, w = 0;
        for (int b = 0; b < bands; ++b) wsum += 10 - b;
        for (int b = 0; b < bands; ++b) {
            w += 10 - b;
            cut[b + 1] = H * w / wsum;
        }
    }
    for (int b = 0; b < bands && e == cudaSuccess; ++b) {
        const size_t y0 = cut[b], y1 = cut[b + 1], n = y1 - y0;
        cudaStream_t ls = L.comp[b & 1];
        P.y0 = (int)y0;
        P.y1 = (int)y1;
        e = launch_single(P, params->sector_count, gbuffer->normal_fmt,
                          std::isinf(params->thickness), k, ls);
        if (e == cudaSuccess) e = cudaEventRecord(L.band_done[b], ls);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(L.out, L.band_done[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(reinterpret_cast<char *>(out->out0) + y0 * out->out0_pitch, out->out0_pitch,
                                  d_out0 + y0 * W * 16, W * 16, W * 16, n, cudaMemcpyDeviceToHost, L.out);
        if (e == cudaSuccess && na > 0)
            e = cudaMemcpy2DAsync(reinterpret_cast<char *>(out->out1) + y0 * out->out1_pitch, out->out1_pitch,
                                  d_out1 + y0 * W * 16, W * 16, W * 16, n, cudaMemcpyDeviceToHost, L.out);
        for (int i = 0; e == cudaSuccess && out->masks && i < params->num_slices; ++i) {
            const size_t o = ((size_t)i * H + y0) * W * melem;  // [N_d][H][W] words: rows y0..y1 of slice i
            e = cudaMemcpyAsync(static_cast<char *>(out->masks) + o, d_masks + o, n * W * melem,
                                cudaMemcpyDeviceToHost, L.out);
        }
        if (e == cudaSuccess && out->light_out)
            e = cudaMemcpy2DAsync(static_cast<char *>(out->light_out) + y0 * out->light_out_pitch,
                                  out->light_out_pitch, d_light + y0 * W * px, W * px, W * px, n,
                                  cudaMemcpyDeviceToHost, L.out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(L.comp1_done, L.comp[1]);
    if (e == cudaSuccess) e = cudaEventRecord(L.done, L.out);
    if (e != cudaSuccess) {
        drain_lane(L);
        return cuda_fail(ctx, e, "host-buffer gather enqueue");
    }
    L.pending = true;
    return SSILVB_OK;
}

}  // namespace ssilvb

using namespace ssilvb;

extern "C" {

ssilvb_status ssilvb_gather_host(ssilvb_ctx *ctx, const ssilvb_gbuffer *gbuffer, const ssilvb_camera *camera,
                                 const ssilvb_params *params, const ssilvb_output *out,
                                 struct CUstream_st *stream) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->last_error.clear();
    DeviceGuard dg(ctx->device);
    ssilvb_status s = validate(ctx, gbuffer, camera, params, out, false);
    if (s != SSILVB_OK) return s;
    if (!ctx->host_ready) {
        const cudaError_t e = create_host_resources(ctx);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "host-buffer stream set-up");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HostLane &L = ctx->sync_lane;
    L.in = st;
    L.comp[0] = st;
    s = enqueue_frame(ctx, L, gbuffer, camera, params, out);
    if (s != SSILVB_OK) return s;
    cudaError_t e = cudaStreamWaitEvent(st, L.comp1_done, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, L.done, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    L.pending = false;
    if (e != cudaSuccess) {
        drain_lane(L);
        return cuda_fail(ctx, e, "gather execution");
    }
    return SSILVB_OK;
}

ssilvb_status ssilvb_gather_host_async(ssilvb_ctx *ctx, const ssilvb_gbuffer *gbuffer,
                                       const ssilvb_camera *camera, const ssilvb_params *params,
                                       const ssilvb_output *out, struct CUstream_st *stream) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->last_error.clear();
    DeviceGuard dg(ctx->device);
    ssilvb_status s = validate(ctx, gbuffer, camera, params, out, false);
    if (s != SSILVB_OK) return s;
    if (!ctx->host_ready) {
        const cudaError_t e = create_host_resources(ctx);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "host-buffer stream set-up");
    }
    HostLane &L = ctx->async_lane[ctx->async_next];
    // start after the work already on the caller's stream, and after this lane's previous frame
    // (whose gather and copies read the staging this frame overwrites)
    cudaError_t e = cudaEventRecord(ctx->host_entry, reinterpret_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.in, ctx->host_entry, 0);
    if (e == cudaSuccess && L.pending) e = cudaStreamWaitEvent(L.in, L.done, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "asynchronous host-buffer gather ordering");
    s = enqueue_frame(ctx, L, gbuffer, camera, params, out);
    if (s != SSILVB_OK) return s;
    ctx->async_next ^= 1;
    return SSILVB_OK;
}

}  // extern "C"
