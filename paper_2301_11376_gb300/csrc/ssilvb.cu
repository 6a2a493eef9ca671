// Host side of the ssilvb C ABI: argument validation, per-launch constants and
// kernel launches for the visibility-bitmask gather (arXiv 2301.11376,
// Algorithm 1, Sections 3.1-3.3).  The declarations and their contracts are in
// include/ssilvb.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

#define SSILVB_VERSION 10100

namespace ssilvb {

namespace {
thread_local std::string g_create_error;
}  // namespace

ssilvb_status fail(ssilvb_ctx *ctx, ssilvb_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->last_error = buf;
    else g_create_error = buf;
    return s;
}

ssilvb_status cuda_fail(ssilvb_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, SSILVB_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

ssilvb_status validate(ssilvb_ctx *ctx, const ssilvb_gbuffer *g, const ssilvb_camera *c, const ssilvb_params *p,
                       const ssilvb_output *o, bool device_ptrs) {
    if (!g || !c || !p || !o) return fail(ctx, SSILVB_ERR_INVALID_ARG, "null gbuffer, camera, params or output");
    if (g->width < 1 || g->height < 1 || g->width > 16384 || g->height > 16384)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "image size %dx%d outside 1..16384", g->width, g->height);
    if (!g->depth || !g->normal || !g->radiance) return fail(ctx, SSILVB_ERR_INVALID_ARG, "null G-buffer plane");
    if (g->normal_fmt != SSILVB_FMT_F32X4 && g->normal_fmt != SSILVB_FMT_F16X4 && g->normal_fmt != SSILVB_FMT_F16X8)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "unknown normal format %d", g->normal_fmt);
    if (g->radiance_fmt != SSILVB_FMT_F32X4 && g->radiance_fmt != SSILVB_FMT_F16X4 &&
        g->radiance_fmt != SSILVB_FMT_F16X8)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "unknown radiance format %d", g->radiance_fmt);
    if (g->normal_fmt != g->radiance_fmt)
        return fail(ctx, SSILVB_ERR_UNSUPPORTED, "normal and radiance formats must match");
    const bool nr16 = g->normal_fmt == SSILVB_FMT_F16X8;
    if (nr16 && (g->radiance != g->normal || g->radiance_pitch != g->normal_pitch))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "F16X8: radiance must be the normal plane (same pointer and pitch)");
    if (nr16 && o->light_out)
        return fail(ctx, SSILVB_ERR_UNSUPPORTED, "the multi-bounce light buffer needs F32X4 or F16X4 planes");
    const size_t px = g->normal_fmt == SSILVB_FMT_F16X4 ? 8 : 16;
    const size_t W = (size_t)g->width;
    if (g->depth_pitch < W * 4 || g->depth_pitch % 4)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "depth pitch %zu invalid for width %zu", g->depth_pitch, W);
    if ((g->depth_pitch / 4) * (size_t)g->height >= ((size_t)1 << 31))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "depth plane larger than 2^31 elements");
    if (g->normal_pitch < W * px || g->normal_pitch % px || g->radiance_pitch < W * px || g->radiance_pitch % px)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "normal/radiance pitch invalid (pixel size %zu)", px);
    if (!aligned(g->depth, 16) || !aligned(g->normal, 16) || !aligned(g->radiance, 16))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "G-buffer planes must be 16-byte aligned");
    if (!(c->fx > 0.0f) || !(c->fy > 0.0f) || !std::isfinite(c->fx) || !std::isfinite(c->fy) ||
        !std::isfinite(c->cx) || !std::isfinite(c->cy))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "camera intrinsics must be finite with fx, fy > 0");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(c->view_to_world[i])) return fail(ctx, SSILVB_ERR_INVALID_ARG, "view_to_world not finite");
    if (p->num_slices < 1 || p->num_slices > ssilvb::kMaxSlices)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "num_slices %d outside 1..16", p->num_slices);
    if (p->steps_per_side < 1 || p->steps_per_side > 64)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "steps_per_side %d outside 1..64", p->steps_per_side);
    if (!(p->radius > 0.0f) || !std::isfinite(p->radius))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "radius must be finite and > 0");
    if (!(p->thickness > 0.0f) || (std::isfinite(p->thickness) && p->thickness > 1e6f))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "thickness must be in (0, 1e6] or +INF");
    if (!(p->thickness_slope >= 0.0f) || !std::isfinite(p->thickness_slope))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "thickness_slope must be finite and >= 0");
    if (p->sector_count != 32 && p->sector_count != 64 && p->sector_count != 128)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "sector_count %d not in {32, 64, 128}", p->sector_count);
    if (p->hit_rule != 0 && p->hit_rule != 1) return fail(ctx, SSILVB_ERR_INVALID_ARG, "hit_rule must be 0 or 1");
    if (p->step_mode != 0 && p->step_mode != 1) return fail(ctx, SSILVB_ERR_INVALID_ARG, "step_mode must be 0 or 1");
    if (p->compute_gi != 0 && p->compute_gi != 1) return fail(ctx, SSILVB_ERR_INVALID_ARG, "compute_gi must be 0 or 1");
    const int na = p->ambient_cones;
    if (na != 0 && na != 1 && na != 2 && na != 4 && na != 8)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "ambient_cones %d not in {0,1,2,4,8}", na);
    if (na > 0 && !p->sh_rgb) return fail(ctx, SSILVB_ERR_INVALID_ARG, "sh_rgb required when ambient_cones > 0");
    if (p->noise_mode < 0 || p->noise_mode > 2)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "noise_mode %d not in {0, 1, 2}", p->noise_mode);
    if (p->noise_mode == 2 && !p->noise_table)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "noise_mode 2 needs noise_table");
    if (p->noise_mode != 2 && p->noise_table)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "noise_table is read only with noise_mode 2 (got mode %d)",
                    p->noise_mode);
    if (p->noise_mode == 1 && p->noise_frame < 0)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "noise_frame %d must be >= 0", p->noise_frame);
    if (p->noise_mode == 2)
        for (int i = 0; i < 32; ++i)
            if (!(p->noise_table[i] >= 0.0f && p->noise_table[i] < 1.0f))
                return fail(ctx, SSILVB_ERR_INVALID_ARG, "noise_table[%d] not in [0, 1)", i);
    if (p->sh_rgb && na > 0)
        for (int i = 0; i < 27; ++i)
            if (!std::isfinite(p->sh_rgb[i])) return fail(ctx, SSILVB_ERR_INVALID_ARG, "sh_rgb not finite");
    if (!o->out0) return fail(ctx, SSILVB_ERR_INVALID_ARG, "out0 is required");
    if (o->out0_pitch < W * 16 || o->out0_pitch % 16 || !aligned(o->out0, 16))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "out0 must be 16-byte aligned with pitch >= 16*width, multiple of 16");
    if (na > 0 && (!o->out1 || o->out1_pitch < W * 16 || o->out1_pitch % 16 || !aligned(o->out1, 16)))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "out1 (16-byte aligned, pitch >= 16*width) required with ambient cones");
    if (o->masks && !aligned(o->masks, p->sector_count == 128 ? 16 : 8))
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "masks must be aligned to their element size");
    if (o->light_out) {
        if (!aligned(o->light_out, 16) || o->light_out_pitch < W * px || o->light_out_pitch % px)
            return fail(ctx, SSILVB_ERR_INVALID_ARG, "light_out: 16-byte aligned, pitch a multiple of %zu >= width", px);
        if (o->light_out == g->radiance || (g->direct && o->light_out == g->direct))
            return fail(ctx, SSILVB_ERR_INVALID_ARG, "light_out must not be an input plane (use two buffers)");
        if (g->direct && (!aligned(g->direct, 16) || g->direct_pitch < W * px || g->direct_pitch % px))
            return fail(ctx, SSILVB_ERR_INVALID_ARG, "direct: 16-byte aligned, pitch a multiple of %zu >= width", px);
        if (!(p->bounce_gain >= 0.0f) || !std::isfinite(p->bounce_gain))
            return fail(ctx, SSILVB_ERR_INVALID_ARG, "bounce_gain must be finite and >= 0");
    }
    if (device_ptrs) {
        const void *ptrs[] = {g->depth, g->normal, g->radiance, o->out0, na > 0 ? o->out1 : nullptr, o->masks,
                              o->light_out, o->light_out ? g->direct : nullptr};
        for (const void *q : ptrs) {
            if (!q) continue;
            cudaPointerAttributes a;
            cudaError_t e = cudaPointerGetAttributes(&a, q);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, SSILVB_ERR_INVALID_ARG, "pointer %p is not CUDA memory", q);
            }
            if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
                return fail(ctx, SSILVB_ERR_INVALID_ARG, "pointer %p is not device memory", q);
            if (a.device != ctx->device)
                return fail(ctx, SSILVB_ERR_INVALID_ARG, "pointer %p is on device %d, context on %d", q, a.device,
                            ctx->device);
        }
    }
    return SSILVB_OK;
}

// The built-in noise table (noise_mode 1): per 4x4 pixel class, xi_phi = interleaved gradient
// noise (Jimenez, "Next Generation Post Processing in Call of Duty: Advanced Warfare", SIGGRAPH
// 2014), IGN(x, y) = frac(52.9829189 frac(0.06711056 x + 0.00583715 y)), at the class's pixel
// offset by 5.588238 (frame mod 64) pixels along both axes for temporal variation, and
// xi_s = frac(xi_phi + 1/2); FP64, each rounded once to binary32, a value that rounds to 1 taken as 0.
static void builtin_noise(int frame, float table[32]) {
    const double off = 5.588238 * (double)(frame % 64);
    for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x) {
            const double px = x + off, py = y + off;
            const double f = std::fmod(0.06711056 * px + 0.00583715 * py, 1.0);
            const double xi = std::fmod(52.9829189 * f, 1.0);
            float a = (float)xi, b = (float)std::fmod(xi + 0.5, 1.0);
            table[2 * (y * 4 + x)] = a >= 1.0f ? 0.0f : a;
            table[2 * (y * 4 + x) + 1] = b >= 1.0f ? 0.0f : b;
        }
}

// The 3-band SH environment (coefficients sh[3 m + channel], m the real SH basis y00, y1-1, y10,
// y11, y2-2, y2-1, y20, y21, y22 with the usual normalisation) as a quadratic form of the view-space
// direction a (Section 3.2's ambient light).  For a unit world direction w = R a the sum of
// sh_m Y_m(w) is c + b_w.w + w^T M w: c holds band 0 and the constant term of y20, b_w = Y1 (sh3,
// sh1, sh2) band 1, M band 2.  The constant goes on the diagonal (c |a|^2 = c), so b = R^T b_w and
// Q = R^T M R + c I.  FP64, each coefficient rounded once to binary32; Q kept as (xx, yy, zz, xy, xz, yz).
static void ambient_form(const float R[9], const float *sh, float b_out[3][3], float q_out[3][6]) {
    const double y0 = 0.5 * std::sqrt(1.0 / M_PI), y1 = std::sqrt(3.0 / (4.0 * M_PI));
    const double y2 = 0.5 * std::sqrt(15.0 / M_PI), y3 = 0.25 * std::sqrt(5.0 / M_PI);
    const double y4 = 0.25 * std::sqrt(15.0 / M_PI);
    double Rd[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rd[i][j] = (double)R[3 * i + j];
    for (int ch = 0; ch < 3; ++ch) {
        double h[9];
        for (int m = 0; m < 9; ++m) h[m] = (double)sh[3 * m + ch];
        const double c = y0 * h[0] - y3 * h[6];
        const double bw[3] = {y1 * h[3], y1 * h[1], y1 * h[2]};
        const double Mw[3][3] = {{y4 * h[8], 0.5 * y2 * h[4], 0.5 * y2 * h[7]},
                                 {0.5 * y2 * h[4], -(y4 * h[8]), 0.5 * y2 * h[5]},
                                 {0.5 * y2 * h[7], 0.5 * y2 * h[5], 3.0 * y3 * h[6]}};
        double T[3][3], Q[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) T[i][k] = (Mw[i][0] * Rd[0][k] + Mw[i][1] * Rd[1][k]) + Mw[i][2] * Rd[2][k];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) Q[j][k] = (Rd[0][j] * T[0][k] + Rd[1][j] * T[1][k]) + Rd[2][j] * T[2][k];
        for (int j = 0; j < 3; ++j) {
            b_out[ch][j] = (float)((Rd[0][j] * bw[0] + Rd[1][j] * bw[1]) + Rd[2][j] * bw[2]);
            Q[j][j] = Q[j][j] + c;
        }
        q_out[ch][0] = (float)Q[0][0];
        q_out[ch][1] = (float)Q[1][1];
        q_out[ch][2] = (float)Q[2][2];
        q_out[ch][3] = (float)Q[0][1];
        q_out[ch][4] = (float)Q[0][2];
        q_out[ch][5] = (float)Q[1][2];
    }
}

// Per-launch constants.  Every expression is written out exactly as the method's binary32
// specification fixes it (the same expressions any other IEEE implementation evaluates).
void fill_params(ssilvb::GatherParams &P, const ssilvb_gbuffer *g, const ssilvb_camera *c, const ssilvb_params *p,
                 const ssilvb_output *o) {
    std::memset(&P, 0, sizeof(P));
    P.depth = g->depth;
    P.normal = static_cast<const char *>(g->normal);
    P.radiance = static_cast<const char *>(g->radiance);
    P.out0 = o->out0;
    P.out1 = p->ambient_cones > 0 ? o->out1 : nullptr;
    P.masks = o->masks;
    P.light_out = static_cast<char *>(o->light_out);
    P.light_pitch = o->light_out ? o->light_out_pitch : 0;
    P.gain = o->light_out ? p->bounce_gain : 0.0f;
    const bool own_direct = o->light_out && g->direct;
    P.direct = own_direct ? static_cast<const char *>(g->direct) : static_cast<const char *>(g->radiance);
    P.direct_pitch = own_direct ? g->direct_pitch : g->radiance_pitch;
    P.depth_pitch = g->depth_pitch / 4;
    P.normal_pitch = g->normal_pitch;
    P.radiance_pitch = g->radiance_pitch;
    P.out0_pitch = o->out0_pitch / 4;
    P.out1_pitch = p->ambient_cones > 0 ? o->out1_pitch / 4 : 0;
    P.W = g->width;
    P.H = g->height;
    P.y0 = 0;
    P.y1 = g->height;
    // Frames of 2^22 pixels or more (4K) run their class-mapped patches in bands of about 32 patch
    // rows (27 at 2160 rows): measured at 4K 4 % faster (N_b 64: 4 %); at 1080p and 1440p the raster
    // order (bands of one patch row) is 2-4 % faster, so smaller frames keep it.
    P.band_rows = (long long)g->width * g->height >= (1LL << 22) ? 32 : 1;
    P.nd = p->num_slices;
    P.ns = p->steps_per_side;
    P.na = p->ambient_cones;
    P.hit_rule = p->hit_rule;
    P.step_mode = p->step_mode;
    P.gi = p->compute_gi;
    const int nb = p->sector_count, nd = p->num_slices, ns = p->steps_per_side, na = p->ambient_cones;
    P.inv_fx = 1.0f / c->fx;
    P.inv_fy = 1.0f / c->fy;
    P.kx0 = -(c->cx * P.inv_fx);
    P.ninv_fy = -P.inv_fy;
    P.ky0 = c->cy * P.inv_fy;
    P.Rfx = p->radius * c->fx;
    P.dn = 1.0f / (float)(ns + 1);
    P.K = (float)((double)nb / M_PI);
    P.half_nb = 0.5f * (float)nb;
    P.f_nb = (float)nb;
    P.inv_nb = 1.0f / (float)nb;
    P.inv_nd = 1.0f / (float)nd;
    P.edge_hi = p->hit_rule == 0 ? P.f_nb - 0.5f : std::nextafter(P.f_nb, 0.0f);
    P.edge_lo = p->hit_rule == 0 ? 0.5f : std::nextafter(0.0f, 1.0f);
    const double del = p->hit_rule == 0 ? M_PI / (2.0 * nb) : 0.0;
    P.sdel = (float)std::sin(del);
    P.cdel = (float)std::cos(del);
    P.t0 = p->thickness;
    P.kt = p->thickness_slope;
    float noise[32] = {};
    if (p->noise_mode == 1) builtin_noise(p->noise_frame, noise);
    else if (p->noise_mode == 2) std::memcpy(noise, p->noise_table, sizeof(noise));
    for (int cl = 0; cl < 16; ++cl) {
        const float xi_phi = noise[2 * cl];
        P.xi_s[cl] = noise[2 * cl + 1];
        for (int i = 0; i < nd; ++i) {
            const double phi = ((double)i + (double)xi_phi) * M_PI / (double)nd;
            P.dcos[cl][i] = (float)std::cos(phi);
            P.dsin[cl][i] = (float)std::sin(phi);
        }
    }
    for (int k = 0; k < na; ++k) {
        const double th = -0.5 * M_PI + (k + 0.5) * M_PI / na;
        P.ccos[k] = (float)std::cos(th);
        P.csin[k] = (float)std::sin(th);
    }
    if (na > 0) ambient_form(c->view_to_world, p->sh_rgb, P.amb_b, P.amb_q);
}

cudaError_t launch_single(const GatherParams &P0, int nb, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s) {
    GatherParams P = P0;  // passed to the kernel by value
    apply_order(P, k);
    if (nb == 32) return launch_single_nb32(P, fmt, inf_t, k, s);
    if (nb == 64) return launch_single_nb64(P, fmt, inf_t, k, s);
    return launch_single_nb128(P, fmt, inf_t, k, s);
}

void single_kernel_node(const GatherParams &P, int nb, int fmt, bool inf_t, const KernelChoice &k, const void **fn,
                        dim3 *grid, dim3 *block) {
    if (nb == 32) single_node_nb32(P, fmt, inf_t, k, fn, grid, block);
    else if (nb == 64) single_node_nb64(P, fmt, inf_t, k, fn, grid, block);
    else single_node_nb128(P, fmt, inf_t, k, fn, grid, block);
}

cudaError_t launch_batch_nb(int nb, const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt,
                            bool inf_t, int step_mode, const KernelChoice &k, int grid, cudaStream_t s) {
    if (nb == 32) return launch_batch_nb32(hdr, frames, queue, fmt, inf_t, step_mode, k, grid, s);
    if (nb == 64) return launch_batch_nb64(hdr, frames, queue, fmt, inf_t, step_mode, k, grid, s);
    return launch_batch_nb128(hdr, frames, queue, fmt, inf_t, step_mode, k, grid, s);
}

int batch_occ(int nb, int fmt, bool inf_t, int minb) {
    if (nb == 32) return batch_occ_nb32(fmt, inf_t, minb);
    if (nb == 64) return batch_occ_nb64(fmt, inf_t, minb);
    return batch_occ_nb128(fmt, inf_t, minb);
}

TuneKey tune_key(const ssilvb_gbuffer *g, const ssilvb_params *p, int batch) {
    TuneKey k;
    k.nb = p->sector_count;
    k.fmt = g->normal_fmt;
    k.inf_t = std::isinf(p->thickness) ? 1 : 0;
    const double px = (double)g->width * g->height;
    k.size_class = (int)std::ceil(std::log2(px > 1.0 ? px : 1.0));
    k.nd = p->num_slices;
    k.ns = p->steps_per_side;
    k.batch = batch;
    return k;
}

KernelChoice resolve_choice(const ssilvb_ctx *ctx, const TuneKey &key) {
    KernelChoice k;
    // size_class = ceil(log2(pixels)): 23 and up is more than 2^22 pixels (3840 x 2160 is 2^22.98)
    k.minb = default_minb(key.nb, key.batch == 0 && key.size_class >= 23);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) k = it->second;
    const ssilvb_tuning &t = ctx->tuning;
    if (t.mapping != SSILVB_MAP_AUTO) k.mapping = t.mapping;
    if (t.occupancy) k.minb = t.occupancy;
    if (t.rows_per_tile) k.rows = t.rows_per_tile;
    if (t.ctas_per_sm) k.ctas_per_sm = t.ctas_per_sm;
    if (t.use_graph) k.graph = t.use_graph == 1;
    if (t.batch_mode) k.batch_mode = t.batch_mode;
    if (t.block_order) k.order = t.block_order;
    return k;
}

}  // namespace ssilvb

using namespace ssilvb;

extern "C" {

int ssilvb_version(void) { return SSILVB_VERSION; }

const char *ssilvb_status_string(ssilvb_status s) {
    switch (s) {
        case SSILVB_OK: return "SSILVB_OK";
        case SSILVB_ERR_INVALID_ARG: return "SSILVB_ERR_INVALID_ARG";
        case SSILVB_ERR_UNSUPPORTED: return "SSILVB_ERR_UNSUPPORTED";
        case SSILVB_ERR_OUT_OF_MEMORY: return "SSILVB_ERR_OUT_OF_MEMORY";
        case SSILVB_ERR_CUDA: return "SSILVB_ERR_CUDA";
        case SSILVB_ERR_TIMEOUT: return "SSILVB_ERR_TIMEOUT";
        case SSILVB_ERR_DEVICE_CHECK: return "SSILVB_ERR_DEVICE_CHECK";
    }
    return "SSILVB_UNKNOWN_STATUS";
}

const char *ssilvb_last_error(const ssilvb_ctx *ctx) {
    return ctx ? ctx->last_error.c_str() : ssilvb::g_create_error.c_str();
}

ssilvb_status ssilvb_create(ssilvb_ctx **out_ctx, int cuda_device) {
    if (!out_ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "out_ctx is NULL");
    *out_ctx = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (cuda_device < 0 || cuda_device >= n)
        return fail(nullptr, SSILVB_ERR_INVALID_ARG, "device %d outside 0..%d", cuda_device, n - 1);
    ssilvb_ctx *ctx = new (std::nothrow) ssilvb_ctx();
    if (!ctx) return fail(nullptr, SSILVB_ERR_OUT_OF_MEMORY, "host allocation failed");
    ctx->device = cuda_device;
    DeviceGuard dg(cuda_device);
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, cuda_device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        ssilvb_status s = cuda_fail(nullptr, e, "context set-up");
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? SSILVB_ERR_OUT_OF_MEMORY : s;
    }
    *out_ctx = ctx;
    return SSILVB_OK;
}

ssilvb_status ssilvb_destroy(ssilvb_ctx *ctx) {
    if (!ctx) return SSILVB_OK;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->d_status) cudaFree(ctx->d_status);
    release_batch_slots(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    release_host_resources(ctx);
    delete ctx;
    return SSILVB_OK;
}

ssilvb_status ssilvb_gather(ssilvb_ctx *ctx, const ssilvb_gbuffer *gbuffer, const ssilvb_camera *camera,
                            const ssilvb_params *params, const ssilvb_output *out, struct CUstream_st *stream) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->last_error.clear();
    DeviceGuard dg(ctx->device);
    ssilvb_status s = validate(ctx, gbuffer, camera, params, out, true);
    if (s != SSILVB_OK) return s;
    ssilvb::GatherParams P;
    fill_params(P, gbuffer, camera, params, out);
    const KernelChoice k = resolve_choice(ctx, tune_key(gbuffer, params, 0));
    cudaError_t e = launch_single(P, params->sector_count, gbuffer->normal_fmt,
                                  std::isinf(params->thickness), k, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather launch");
    return SSILVB_OK;
}

ssilvb_status ssilvb_set_tuning(ssilvb_ctx *ctx, const ssilvb_tuning *tuning) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    if (!tuning) return fail(ctx, SSILVB_ERR_INVALID_ARG, "tuning is NULL");
    if (tuning->mapping < SSILVB_MAP_AUTO || tuning->mapping > SSILVB_MAP_CLASS)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "unknown mapping %d", tuning->mapping);
    if (tuning->occupancy != 0 && tuning->occupancy != 8 && tuning->occupancy != 9)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "occupancy must be 0, 8 or 9");
    if (tuning->rows_per_tile < 0 || tuning->rows_per_tile > 8)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "rows_per_tile must be 0..8");
    if (tuning->ctas_per_sm < 0 || tuning->ctas_per_sm > 16)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "ctas_per_sm must be 0..16");
    if (tuning->use_graph < 0 || tuning->use_graph > 2)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "use_graph must be 0, 1 or 2");
    if (tuning->batch_mode < 0 || tuning->batch_mode > 2)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "batch_mode must be 0, 1 or 2");
    if (tuning->block_order < 0 || tuning->block_order > 2)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "block_order must be 0, 1 or 2");
    if (tuning->reserved) return fail(ctx, SSILVB_ERR_INVALID_ARG, "reserved tuning field must be zero");
    ctx->tuning = *tuning;
    return SSILVB_OK;
}

ssilvb_status ssilvb_synchronize(ssilvb_ctx *ctx, struct CUstream_st *stream) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream execution");
    const ssilvb_status hs = wait_host_async(ctx);
    if (hs != SSILVB_OK) return hs;
    int st = 0;
    e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (st != 0) {
        cudaMemset(ctx->d_status, 0, sizeof(int));
        if (st == SSILVB_ERR_TIMEOUT) return fail(ctx, SSILVB_ERR_TIMEOUT, "a bounded device wait gave up");
        return fail(ctx, SSILVB_ERR_DEVICE_CHECK, "device check failed (code %d)", st);
    }
    return SSILVB_OK;
}

ssilvb_status ssilvb_get_status(ssilvb_ctx *ctx, struct CUstream_st *stream) { return ssilvb_synchronize(ctx, stream); }

}  // extern "C"
