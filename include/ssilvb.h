/*
 * ssilvb: screen-space indirect lighting with a visibility bitmask, on GB300.
 *
 * C ABI of the GPU gather of Therrien, Levesque and Gilet, "Screen Space
 * Indirect Lighting with Visibility Bitmask" (arXiv 2301.11376).  For every
 * pixel and every slice direction around the view vector the gather marches
 * depth samples on both sides, turns each sample's front and back elevation
 * (the back one from a constant thickness t) into a run of sectors of an
 * N_b-bit visibility mask, adds the newly occluded sectors' share of the
 * sample's direct radiance into indirect diffuse light, and ORs the run into
 * the slice mask, which gives ambient occlusion and the directionally
 * occluded ambient light (Algorithm 1 of Section 3.1; Sections 3.2 and 3.3).
 *
 * Conventions shared by every entry point
 *   - Plain pointers and sizes only.  Device pointers are CUDA device memory
 *     on the context's device; "host" pointers are ordinary CPU memory.
 *   - Every argument is validated before anything is enqueued; on any error
 *     nothing is launched and the call returns a status != SSILVB_OK, with a
 *     human-readable detail in ssilvb_last_error().
 *   - Calls that take a stream are asynchronous on that stream (a
 *     cudaStream_t; NULL = the legacy default stream) unless stated otherwise.
 *   - The caller owns every buffer it passes.  The library keeps no pointer
 *     to them after the work enqueued by the call has finished.
 *   - A context is not thread-safe: use one per host thread.  No C++
 *     exception crosses this boundary.
 *
 * Geometry conventions
 *   View space is right-handed, camera at the origin looking along -z, +y up.
 *   Image rows go down.  The centre of pixel (x, y) is (x + 0.5, y + 0.5) and
 *   projects from view position P as u = cx + fx * P.x / (-P.z),
 *   v = cy - fy * P.y / (-P.z).  Depth is linear: z = -P.z > 0.  A depth value
 *   that is not in (0, +INF) (including +INF and NaN) marks sky: such pixels
 *   output AO = 1, GI = 0, ambient = 0 and are never used as samples.
 */
#ifndef SSILVB_H
#define SSILVB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t is struct CUstream_st* */

typedef struct ssilvb_ctx ssilvb_ctx; /* opaque, owned by the library */

typedef enum {
    SSILVB_OK = 0,
    SSILVB_ERR_INVALID_ARG = 1,   /* null pointer, bad size, alignment or pitch, parameter out of range */
    SSILVB_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement (e.g. mixed formats) */
    SSILVB_ERR_OUT_OF_MEMORY = 3, /* a context allocation failed */
    SSILVB_ERR_CUDA = 4,          /* a CUDA runtime or driver call failed; see ssilvb_last_error */
    SSILVB_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    SSILVB_ERR_DEVICE_CHECK = 6   /* a device-side consistency check failed */
} ssilvb_status;

/* Storage of normals and radiance.  F32X4 / F16X4: two planes, 4 components per pixel (xyz / rgb,
 * the 4th ignored), 32-bit float or IEEE binary16.  F16X8: one interleaved plane of 8 binary16 per
 * pixel, (n.x, n.y, n.z, c.r, c.g, c.b, unused, unused), 16 bytes, the footprint of the two F16X4
 * planes: a sample's normal and radiance then share one 32-byte memory sector, which halves the
 * sectors the indirect-light fetches read (the values, and so every result, are those of F16X4). */
typedef enum { SSILVB_FMT_F32X4 = 0, SSILVB_FMT_F16X4 = 1, SSILVB_FMT_F16X8 = 2 } ssilvb_format;

/* The G-buffer the gather reads (Algorithm 1 inputs p, n_p and the light buffer of
 * Section 3.3: depth, view-space normals and direct radiance "with shadows").
 * Device pointers, row-major with a row pitch in BYTES; base pointers 16-byte
 * aligned; depth pitch a multiple of 4, normal/radiance pitch a multiple of the
 * pixel size (16 for F32X4, 8 for F16X4, 16 for F16X8).  normal_fmt must equal radiance_fmt.
 * F16X8: normal and radiance are the same pointer and pitch (the interleaved plane); the
 * multi-bounce light buffer (light_out, direct) is not available with it (UNSUPPORTED). */
typedef struct {
    int width, height;            /* 1 .. 16384 each */
    const float *depth;           /* [height][pitch] linear view depth */
    size_t depth_pitch;
    const void *normal;           /* view-space unit normal, xyz used */
    size_t normal_pitch;
    int normal_fmt;               /* ssilvb_format */
    const void *radiance;         /* light buffer, rgb used: direct radiance (plus the previous
                                     frame's injected bounce under multi-bounce) */
    size_t radiance_pitch;
    int radiance_fmt;             /* ssilvb_format */
    const void *direct;           /* optional, multi-bounce only: this frame's direct radiance, in
                                     the radiance format; NULL = the radiance plane is direct light */
    size_t direct_pitch;
} ssilvb_gbuffer;

/* Pinhole intrinsics in pixels (fx, fy > 0) and the row-major view->world
 * rotation, used only to look up the ambient environment in world space. */
typedef struct {
    float fx, fy, cx, cy;
    float view_to_world[9];
} ssilvb_camera;

/* Parameters of the method (Algorithm 1; Sections 3.1-3.3, 4.1-4.3). */
typedef struct {
    int num_slices;        /* N_d, 1..16: slice directions per pixel, azimuth (i + xi_phi) pi / N_d */
    int steps_per_side;    /* N_s, 1..64: samples on each side of the slice */
    float radius;          /* R > 0 (view-space units): projected radius r = R fx / z pixels */
    float thickness;       /* t > 0; +INF = infinite thickness (horizon-based occlusion) */
    float thickness_slope; /* k_t >= 0: thickness grows linearly with depth, t(z) = t + k_t z */
    int sector_count;      /* N_b: 32, 64 or 128 (Section 4.1 compares 32 and 128) */
    int hit_rule;          /* 0: a sector is occluded when at least half covered (Section 3.1);
                              1: floor/ceil run of Algorithm 1 */
    int step_mode;         /* 0: constant steps r (j+1+xi_s)/(N_s+1);
                              1: quadratic ("exponential") steps r ((j+1+xi_s)/(N_s+1))^2 */
    int ambient_cones;     /* N_a in {0, 1, 2, 4, 8} dividing N_b: ambient cones per slice, 0 = off */
    int compute_gi;        /* 1 = indirect diffuse (reads normal and radiance at samples), 0 = off */
    int noise_mode;        /* per-pixel slice rotation xi_phi and step jitter xi_s ("directions with random
                              offset", Section 3.1; spatial and temporal jitter, Section 4.3), one pair per
                              4x4 pixel class, row (y&3)*4 + (x&3):
                              0 = none (both 0);
                              1 = built in: xi_phi = Jimenez's interleaved gradient noise at the class's
                                  pixel offset by 5.588238 (noise_frame mod 64) pixels along x and y,
                                  xi_s = frac(xi_phi + 1/2), each computed in FP64 and rounded to binary32
                                  once (a value that rounds to 1 becomes 0);
                              2 = the caller's noise_table */
    int noise_frame;       /* noise_mode 1: frame index of the temporal rotation (>= 0) */
    const float *noise_table; /* HOST, noise_mode 2 only (else NULL): 16 x (xi_phi, xi_s) in [0,1) */
    const float *sh_rgb;   /* HOST, 9 x 3 real SH radiance coefficients [m][rgb] of the ambient
                              environment (order Y00, Y1-1, Y10, Y11, Y2-2, Y2-1, Y20, Y21, Y22);
                              required iff ambient_cones > 0 */
    float bounce_gain;     /* multi-bounce (Section 4.3): g >= 0, finite; used only with out->light_out */
} ssilvb_params;

/* Outputs, device pointers.  out0 (required): float4 per pixel = (GI.r, GI.g, GI.b, AO),
 * AO = mean over slices of the unoccluded sector fraction (1 = fully visible).
 * out1 (required iff ambient_cones > 0): float4 = (ambient.r, .g, .b, 0).
 * Pitches in bytes, multiples of 16; bases 16-byte aligned.
 * masks (optional, NULL = not written): the final slice bitmasks, dense
 * [num_slices][height][width] of uint32 (N_b = 32), uint64 (N_b = 64) or 4 x uint32 (N_b = 128,
 * sector k in bit k % 32 of word k / 32), aligned to that element size.
 * light_out (optional, NULL = not written): the light buffer for the next frame of the
 * multi-bounce scheme of Section 4.3, direct + bounce_gain * GI per channel (4th = 0), where
 * direct is gbuffer->direct (or the radiance plane when that is NULL), in the radiance plane's
 * format and pitch rules; it must not be the radiance or direct plane (the caller alternates
 * two light buffers between frames).  A gain below 1 keeps the feedback bounded. */
typedef struct {
    float *out0;
    size_t out0_pitch;
    float *out1;
    size_t out1_pitch;
    void *masks;
    void *light_out;
    size_t light_out_pitch;
} ssilvb_output;

/* Launch choices.  None of them changes any result: every choice gives bit-identical output.
 * A zero field means "automatic": the autotuner's choice for this kind of call if
 * ssilvb_autotune has run, else the library default. */
typedef enum {
    SSILVB_MAP_AUTO = 0,  /* library default */
    SSILVB_MAP_TILE = 1,  /* one thread per pixel, 32 x 8 pixel tiles */
    SSILVB_MAP_CLASS = 2  /* one thread per pixel; the 32 lanes of a warp share a 4x4 noise class */
} ssilvb_mapping;

typedef struct {
    int mapping;          /* ssilvb_mapping, single-frame calls */
    int occupancy;        /* 0 (default: 8 for N_b 32, else 9), or 8 / 9: blocks of 128 threads per SM the register budget is sized for */
    int rows_per_tile;    /* batch: 0, or 1..8 patch rows per work item (a patch row is 16 pixel rows of
                             one 32-pixel-wide patch column, one row class of 4) */
    int ctas_per_sm;      /* batch: 0 (as many as fit), or 1..16 blocks per SM in the persistent grid */
    int use_graph;        /* batch, persistent mode: 0 auto, 1 launch through a cached CUDA graph, 2 plain */
    int batch_mode;       /* batch: 0 auto, 1 one persistent kernel over a tile queue,
                             2 one CUDA graph of independent per-frame kernels */
    int block_order;      /* class mapping, single frames and graph-of-kernels batches: 0 auto (bands for
                             frames of 2^22 pixels or more, else raster), 1 patches in raster order,
                             2 patches in bands of about 32 patch rows, column by column within a band (the
                             blocks resident at once cover a compact region; results are identical) */
    int reserved;         /* must be zero */
} ssilvb_tuning;

/* One frame of a batch: its G-buffer, camera, parameters and outputs, with the same meaning
 * and rules as the arguments of ssilvb_gather. */
typedef struct {
    ssilvb_gbuffer gbuffer;
    ssilvb_camera camera;
    ssilvb_params params;
    ssilvb_output out;
} ssilvb_frame;

/* Library version, major * 10000 + minor * 100 + patch. */
int ssilvb_version(void);

/* Human-readable name of a status code (static storage). */
const char *ssilvb_status_string(ssilvb_status s);

/* Detail of the context's last failure ("" if none); valid until the next call on ctx.
 * NULL ctx returns the detail of the last failed ssilvb_create in this thread. */
const char *ssilvb_last_error(const ssilvb_ctx *ctx);

/* Create a context on CUDA device cuda_device.  *out_ctx receives the context,
 * or NULL on failure.  Allocates a device status word; errors:
 * INVALID_ARG (null out_ctx, bad device), CUDA, OUT_OF_MEMORY. */
ssilvb_status ssilvb_create(ssilvb_ctx **out_ctx, int cuda_device);

/* Destroy a context and free what it owns (NULL is allowed).  Synchronises the device. */
ssilvb_status ssilvb_destroy(ssilvb_ctx *ctx);

/* The visibility-bitmask gather over one frame (Algorithm 1 per pixel, with the
 * ambient cones of Section 3.2 and indirect diffuse of Section 3.3).  All G-buffer
 * and output pointers are device memory; host pointers inside params are read
 * during the call only.  Enqueues the work on stream and returns. */
ssilvb_status ssilvb_gather(ssilvb_ctx *ctx, const ssilvb_gbuffer *gbuffer, const ssilvb_camera *camera,
                            const ssilvb_params *params, const ssilvb_output *out, struct CUstream_st *stream);

/* The same gather on HOST buffers: gbuffer and out point to host memory (pinned
 * memory gives the fastest copies).  The context stages the frame in device
 * buffers it owns (grown on demand and kept for reuse) and copies the inputs host
 * to device on stream.  A frame of 512 rows or more then runs as up to 8 row bands,
 * alternating between stream and a second stream the context owns, and each band's
 * outputs are copied back on a third context stream while later bands compute.
 * The results equal one ssilvb_gather launch bit for bit.  The call returns after
 * the outputs are in host memory, with stream ordered after all of this work (the
 * call synchronises stream). */
ssilvb_status ssilvb_gather_host(ssilvb_ctx *ctx, const ssilvb_gbuffer *gbuffer, const ssilvb_camera *camera,
                                 const ssilvb_params *params, const ssilvb_output *out,
                                 struct CUstream_st *stream);

/* ssilvb_gather_host for streams of frames: the same work and results, enqueued on streams the
 * context owns, and the call returns at once.  Work starts after what is already enqueued on
 * stream.  Consecutive calls alternate between two staging lanes, so one frame's copies overlap
 * its neighbours' gathers.  The host buffers of a call must stay valid and unchanged, and its
 * outputs are complete, only once ssilvb_synchronize(ctx, ...) has returned; that call waits for
 * every frame enqueued this way.  Errors as ssilvb_gather_host, reported by this call (invalid
 * arguments, enqueue failures) or by ssilvb_synchronize (execution errors). */
ssilvb_status ssilvb_gather_host_async(ssilvb_ctx *ctx, const ssilvb_gbuffer *gbuffer,
                                       const ssilvb_camera *camera, const ssilvb_params *params,
                                       const ssilvb_output *out, struct CUstream_st *stream);

/* The gather over many frames of uneven sizes in ONE persistent launch (Algorithm 1 per pixel
 * of every frame).  All frames must share sector_count, the storage format of normal and
 * radiance, step_mode, and whether the thickness is infinite (else UNSUPPORTED); every other parameter,
 * the size, the camera and the noise may differ per frame.  Output regions of different frames
 * must not overlap.  Each frame's results are bit-identical to an ssilvb_gather of that frame.
 * Two launch forms (ssilvb_tuning.batch_mode; the autotuner picks): (1) one persistent kernel:
 * a work item is rows_per_tile patch rows (16 pixel rows each) of one 32-pixel-wide patch column
 * and one of its 4 row classes (a block of 128 threads, each warp 8 x 4 pixels at stride 4);
 * the items of all frames are concatenated and handed to the resident blocks through a queue
 * counter the context owns, launched through a CUDA graph the context caches; (2) one CUDA graph
 * whose independent nodes are the frames' kernels, so the frames run concurrently.  Asynchronous on stream.  The context keeps up to 4
 * batches in flight; a call that needs a busy slot first waits on the host for that slot's
 * previous batch.  1 <= n_frames <= 4096; frames is host memory read during the call. */
ssilvb_status ssilvb_gather_batch(ssilvb_ctx *ctx, const ssilvb_frame *frames, int n_frames,
                                  struct CUstream_st *stream);

/* Autotuner: times the launch choices (register budget, rows per work item, CUDA graph or not,
 * block order; for n_frames == 1 also the single-frame mapping) on these frames, synchronising stream, and
 * remembers the fastest for calls of the same kind (sector count, storage, thickness mode,
 * pixel-count class, largest N_d and N_s, single or batch).  The frames' outputs are written
 * (valid results).  *chosen (may be NULL) receives the winner. */
ssilvb_status ssilvb_autotune(ssilvb_ctx *ctx, const ssilvb_frame *frames, int n_frames, struct CUstream_st *stream,
                              ssilvb_tuning *chosen);

/* The batch gather of ssilvb_gather_batch (persistent-kernel form) for callers that cannot
 * allocate device memory when they call it: an engine that reserves its whole GPU budget up
 * front and forbids driver allocations in its frame loop, or a plug-in whose host application
 * owns all device memory; cudaMalloc also synchronises the device, which a real-time loop
 * cannot afford.  The paper has no counterpart: this is an interface choice only.
 * No context: it runs on the CURRENT device, and its scratch (the work list and the tile-queue
 * counter) lives in a fixed array inside the library, about 44 KB that every GPU loading the
 * library holds until the process exits.  The call allocates nothing (no cudaMalloc,
 * cudaFree, graph or event); the caller still passes all inputs and outputs, with the same
 * rules as ssilvb_gather_batch.  At most 16 frames (INVALID_ARG beyond, with the limit in the
 * message).  The first call on a device looks up the array's device address (and loads the
 * kernels if CUDA loads modules lazily), so make it before any stream capture.  The work list
 * is uploaded from host memory on the calling thread's stack with cudaMemcpyAsync.  Every call
 * shares the array and overwrites the previous call's work list and counter.  Calls whose work
 * overlaps on the GPU therefore race: a running kernel can read another call's frame table,
 * mixing one frame's sizes and pitches with another frame's pointers, and so read and write
 * out of the bounds of any buffer passed in.  The caller must order the calls: issue them on
 * one stream, or make each wait for the previous one with an event.
 * Asynchronous on stream; the host frame array is read during the call only.  Error detail:
 * ssilvb_last_error(NULL) in the calling thread. */
ssilvb_status ssilvb_gather_batch_noalloc(const ssilvb_frame *frames, int n_frames, struct CUstream_st *stream);

/* Set the context's launch choices for later calls (copied).  INVALID_ARG on an unknown value. */
ssilvb_status ssilvb_set_tuning(ssilvb_ctx *ctx, const ssilvb_tuning *tuning);

/* Wait for the work enqueued on stream, and for every frame enqueued by
 * ssilvb_gather_host_async, and report a failure of it: CUDA (asynchronous launch or
 * execution error) or DEVICE_CHECK / TIMEOUT from the context's device status word, which
 * the call then clears.  The current kernels
 * neither wait on the device nor check anything there (every argument is checked on
 * the host before a launch), so those two codes are reserved and never returned. */
ssilvb_status ssilvb_synchronize(ssilvb_ctx *ctx, struct CUstream_st *stream);

/* The same call under the name of the status query in the gather's interface description: waits
 * for stream (and the asynchronous host-buffer frames) and reports their status, exactly as
 * ssilvb_synchronize. */
ssilvb_status ssilvb_get_status(ssilvb_ctx *ctx, struct CUstream_st *stream);

#ifdef __cplusplus
}
#endif
#endif /* SSILVB_H */
