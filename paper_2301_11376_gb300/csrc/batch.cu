// Batched gather (many frames, one persistent launch) and the autotuner.  Declarations and
// contracts: include/ssilvb.h (ssilvb_gather_batch, ssilvb_autotune).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace ssilvb {

namespace {

constexpr int kRing = 4;
constexpr int kMaxFrames = 4096;

size_t table_bytes(int cap) { return sizeof(BatchHeader) + (size_t)cap * sizeof(FrameDesc); }

void free_frame_graph(BatchSlot &s) {
    if (s.fexec) cudaGraphExecDestroy(s.fexec);
    if (s.fgraph) cudaGraphDestroy(s.fgraph);
    s.fexec = nullptr;
    s.fgraph = nullptr;
    s.fnodes.clear();
}

void free_slot(BatchSlot &s) {
    free_frame_graph(s);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.d_table) cudaFree(s.d_table);
    if (s.d_queue) cudaFree(s.d_queue);
    if (s.h_table) cudaFreeHost(s.h_table);
    s.exec = nullptr;
    s.d_table = nullptr;
    s.d_queue = nullptr;
    s.h_table = nullptr;
    s.cap = 0;
    s.exec_key = std::make_tuple(-1, -1, -1, -1, -1, -1, -1);
}

// Wait (host) until the slot's previous batch has finished reading its tables.
ssilvb_status wait_slot(ssilvb_ctx *ctx, BatchSlot &s) {
    if (!s.pending) return SSILVB_OK;
    cudaError_t e = cudaEventSynchronize(s.done);
    s.pending = false;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "previous batch");
    return SSILVB_OK;
}

ssilvb_status ensure_slot(ssilvb_ctx *ctx, BatchSlot &s, int n) {
    if (!s.done) {
        cudaError_t e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event create");
    }
    if (s.cap >= n) return SSILVB_OK;
    free_slot(s);
    int cap = 64;
    while (cap < n) cap *= 2;
    cudaError_t e = cudaMalloc(&s.d_table, table_bytes(cap));
    if (e == cudaSuccess) e = cudaMalloc(&s.d_queue, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_table, table_bytes(cap));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_slot(s);
        return fail(ctx, SSILVB_ERR_OUT_OF_MEMORY, "batch tables for %d frames: %s", cap, cudaGetErrorString(e));
    }
    s.cap = cap;
    return SSILVB_OK;
}

// The enqueue sequence of one batch: work list host->device, queue counter to zero, kernel.
cudaError_t enqueue_batch(ssilvb_ctx *ctx, BatchSlot &s, size_t bytes, int nb, int fmt, bool inf_t, int sm,
                          const KernelChoice &k, int grid, cudaStream_t st) {
    const BatchHeader *hdr = reinterpret_cast<const BatchHeader *>(s.d_table);
    const FrameDesc *frames = reinterpret_cast<const FrameDesc *>(s.d_table + sizeof(BatchHeader));
    cudaError_t e = cudaMemcpyAsync(s.d_table, s.h_table, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.d_queue, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = launch_batch_nb(nb, hdr, frames, s.d_queue, fmt, inf_t, sm, k, grid, st);
    (void)ctx;
    return e;
}

int occupancy(int nb, int fmt, bool inf_t, int minb) { return batch_occ(nb, fmt, inf_t, minb); }

ssilvb_status run_batch(ssilvb_ctx *ctx, const ssilvb_frame *frames, int n, cudaStream_t st, const KernelChoice *force) {
    if (!frames || n < 1 || n > kMaxFrames)
        return fail(ctx, SSILVB_ERR_INVALID_ARG, "n_frames %d outside 1..%d (or frames NULL)", n, kMaxFrames);
    const int nb = frames[0].params.sector_count;
    const int fmt = frames[0].gbuffer.normal_fmt;
    const bool inf_t = std::isinf(frames[0].params.thickness);
    const int sm = frames[0].params.step_mode;
    int max_nd = 0, max_ns = 0;
    double px = 0.0;
    for (int i = 0; i < n; ++i) {
        const ssilvb_frame &f = frames[i];
        ssilvb_status s = validate(ctx, &f.gbuffer, &f.camera, &f.params, &f.out, true);
        if (s != SSILVB_OK) {
            std::string d = ctx->last_error;
            return fail(ctx, s, "frame %d: %s", i, d.c_str());
        }
        if (f.params.sector_count != nb || f.gbuffer.normal_fmt != fmt ||
            (bool)std::isinf(f.params.thickness) != inf_t || f.params.step_mode != sm)
            return fail(ctx, SSILVB_ERR_UNSUPPORTED,
                        "frame %d: sector count, storage format, infinite thickness and step mode must match frame 0",
                        i);
        max_nd = std::max(max_nd, f.params.num_slices);
        max_ns = std::max(max_ns, f.params.steps_per_side);
        px += (double)f.gbuffer.width * f.gbuffer.height;
    }
    TuneKey key;
    key.nb = nb;
    key.fmt = fmt;
    key.inf_t = inf_t;
    key.size_class = (int)std::ceil(std::log2(px > 1.0 ? px : 1.0));
    key.nd = max_nd;
    key.ns = max_ns;
    key.batch = 1;
    const KernelChoice k = force ? *force : resolve_choice(ctx, key);

    if ((int)ctx->slots.size() < kRing) ctx->slots.resize(kRing);
    BatchSlot &s = ctx->slots[ctx->next_slot];
    ctx->next_slot = (ctx->next_slot + 1) % kRing;
    ssilvb_status rs = wait_slot(ctx, s);
    if (rs == SSILVB_OK) rs = ensure_slot(ctx, s, n);
    if (rs != SSILVB_OK) return rs;

    if (k.batch_mode == 2) {
        // One graph, one independent kernel node per frame (the single-frame kernel with its
        // parameters as a grid constant): the frames run concurrently, no tile queue.
        s.fparams.resize(n);
        for (int i = 0; i < n; ++i) {
            fill_params(s.fparams[i], &frames[i].gbuffer, &frames[i].camera, &frames[i].params, &frames[i].out);
            apply_order(s.fparams[i], k);
        }
        auto node_params = [&](int i, cudaKernelNodeParams &kp, void **args) {
            const void *fn = nullptr;
            dim3 grid, block;
            single_kernel_node(s.fparams[i], nb, fmt, inf_t, k, &fn, &grid, &block);
            args[0] = &s.fparams[i];
            kp.func = const_cast<void *>(fn);
            kp.gridDim = grid;
            kp.blockDim = block;
            kp.sharedMemBytes = 0;
            kp.kernelParams = args;
            kp.extra = nullptr;
        };
        bool rebuild = !s.fexec || (int)s.fnodes.size() != n;
        if (!rebuild) {
            for (int i = 0; i < n && !rebuild; ++i) {
                cudaKernelNodeParams kp;
                void *args[1];
                node_params(i, kp, args);
                if (cudaGraphExecKernelNodeSetParams(s.fexec, s.fnodes[i], &kp) != cudaSuccess) {
                    cudaGetLastError();
                    rebuild = true;
                }
            }
        }
        cudaError_t e = cudaSuccess;
        if (rebuild) {
            free_frame_graph(s);
            e = cudaGraphCreate(&s.fgraph, 0);
            s.fnodes.resize(n);
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                cudaKernelNodeParams kp;
                void *args[1];
                node_params(i, kp, args);
                e = cudaGraphAddKernelNode(&s.fnodes[i], s.fgraph, nullptr, 0, &kp);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&s.fexec, s.fgraph, 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                free_frame_graph(s);
                return cuda_fail(ctx, e, "frame graph");
            }
        }
        e = cudaGraphLaunch(s.fexec, st);
        if (e == cudaSuccess) e = cudaEventRecord(s.done, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "frame graph launch");
        s.pending = true;
        return SSILVB_OK;
    }

    // Work list: every frame's tiles (k.rows patch rows of one patch column and row class; see
    // gather_batch_kernel), concatenated in frame order.
    BatchHeader *hdr = reinterpret_cast<BatchHeader *>(s.h_table);
    FrameDesc *fd = reinterpret_cast<FrameDesc *>(s.h_table + sizeof(BatchHeader));
    long long tiles = 0;
    for (int i = 0; i < n; ++i) {
        const ssilvb_frame &f = frames[i];
        std::memset(&fd[i], 0, sizeof(FrameDesc));
        fill_params(fd[i].P, &f.gbuffer, &f.camera, &f.params, &f.out);
        fd[i].tiles_x = 4 * ((f.gbuffer.width + 31) / 32);
        fd[i].rows = k.rows;
        fd[i].tile_begin = (int)tiles;
        tiles += (long long)fd[i].tiles_x * ((f.gbuffer.height + 16 * k.rows - 1) / (16 * k.rows));
    }
    if (tiles >= (1LL << 31) - (1LL << 24)) return fail(ctx, SSILVB_ERR_INVALID_ARG, "batch has too many work items");
    std::memset(hdr, 0, sizeof(BatchHeader));
    hdr->n_frames = n;
    hdr->total_tiles = (int)tiles;

    const int per_sm = k.ctas_per_sm ? k.ctas_per_sm : std::max(1, occupancy(nb, fmt, inf_t, k.minb));
    const int grid = std::max(1, per_sm * ctx->num_sms);  // blocks beyond the work list exit at once
    cudaError_t e;
    if (k.graph) {
        // One cached graph per slot: it always copies the slot's whole table, so it stays valid
        // for any batch that fits; rebuilt only when the slot, kernel variant or grid changes.
        const auto ek = std::make_tuple(nb, fmt, (int)inf_t, sm, k.minb, grid, s.cap);
        if (!s.exec || s.exec_key != ek) {
            if (s.exec) cudaGraphExecDestroy(s.exec);
            s.exec = nullptr;
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = enqueue_batch(ctx, s, table_bytes(s.cap), nb, fmt, inf_t, sm, k, grid, ctx->cap_stream);
                e = cudaStreamEndCapture(ctx->cap_stream, &g);
                if (e1 != cudaSuccess) e = e1;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&s.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s.exec = nullptr;
                return cuda_fail(ctx, e, "batch graph");
            }
            s.exec_key = ek;
        }
        e = cudaGraphLaunch(s.exec, st);
    } else {
        e = enqueue_batch(ctx, s, table_bytes(n), nb, fmt, inf_t, sm, k, grid, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.done, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch launch");
    s.pending = true;
    return SSILVB_OK;
}

float time_runs(ssilvb_ctx *ctx, const ssilvb_frame *frames, int n, cudaStream_t st, const KernelChoice &k,
                bool single, bool *ok) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    *ok = true;
    for (int r = 0; r < 4 && *ok; ++r) {
        cudaEventRecord(a, st);
        ssilvb_status s;
        if (single) {
            GatherParams P;
            fill_params(P, &frames[0].gbuffer, &frames[0].camera, &frames[0].params, &frames[0].out);
            cudaError_t e = launch_single(P, frames[0].params.sector_count,
                                          frames[0].gbuffer.normal_fmt,
                                          std::isinf(frames[0].params.thickness), k, st);
            s = e == cudaSuccess ? SSILVB_OK : cuda_fail(ctx, e, "autotune launch");
        } else {
            s = run_batch(ctx, frames, n, st, &k);
        }
        cudaEventRecord(b, st);
        if (s != SSILVB_OK || cudaEventSynchronize(b) != cudaSuccess) {
            *ok = false;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) best = std::min(best, ms);  // the first run is a warm-up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace

void release_batch_slots(ssilvb_ctx *ctx) {
    for (BatchSlot &s : ctx->slots) {
        if (s.pending) cudaEventSynchronize(s.done);
        free_slot(s);
        if (s.done) cudaEventDestroy(s.done);
        s.done = nullptr;
    }
    ctx->slots.clear();
}

}  // namespace ssilvb

using namespace ssilvb;

extern "C" {

ssilvb_status ssilvb_gather_batch(ssilvb_ctx *ctx, const ssilvb_frame *frames, int n_frames,
                                  struct CUstream_st *stream) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->last_error.clear();
    DeviceGuard dg(ctx->device);
    return run_batch(ctx, frames, n_frames, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

ssilvb_status ssilvb_autotune(ssilvb_ctx *ctx, const ssilvb_frame *frames, int n_frames, struct CUstream_st *stream,
                              ssilvb_tuning *chosen) {
    if (!ctx) return fail(nullptr, SSILVB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->last_error.clear();
    DeviceGuard dg(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // validate once through a plain batch run with the current choice
    ssilvb_status s0 = run_batch(ctx, frames, n_frames, st, nullptr);
    if (s0 != SSILVB_OK) return s0;
    cudaError_t e0 = cudaStreamSynchronize(st);
    if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "autotune warm-up");

    std::vector<KernelChoice> cands;
    for (int minb : {8, 9}) {
        KernelChoice k;
        k.mapping = SSILVB_MAP_CLASS;
        k.minb = minb;
        k.batch_mode = 2;
        for (int order : {1, 2}) {  // the frames' blocks in raster order or in bands
            k.order = order;
            cands.push_back(k);
        }
        k.order = 0;  // the persistent kernel hands out its own work items
        for (int rows : {1, 2, 4})
            for (int graph : {1, 0}) {
                k.batch_mode = 1;
                k.rows = rows;
                k.graph = graph;
                cands.push_back(k);
            }
    }
    KernelChoice best_b;
    float t_best_b = 1e30f;
    for (const KernelChoice &k : cands) {
        bool ok;
        const float t = time_runs(ctx, frames, n_frames, st, k, false, &ok);
        if (!ok) return ctx->last_error.empty() ? fail(ctx, SSILVB_ERR_CUDA, "autotune run failed") : SSILVB_ERR_CUDA;
        if (t < t_best_b) {
            t_best_b = t;
            best_b = k;
        }
    }
    double px = 0.0;
    int max_nd = 0, max_ns = 0;
    for (int i = 0; i < n_frames; ++i) {
        px += (double)frames[i].gbuffer.width * frames[i].gbuffer.height;
        max_nd = std::max(max_nd, frames[i].params.num_slices);
        max_ns = std::max(max_ns, frames[i].params.steps_per_side);
    }
    TuneKey kb;
    kb.nb = frames[0].params.sector_count;
    kb.fmt = frames[0].gbuffer.normal_fmt;
    kb.inf_t = std::isinf(frames[0].params.thickness) ? 1 : 0;
    kb.size_class = (int)std::ceil(std::log2(px > 1.0 ? px : 1.0));
    kb.nd = max_nd;
    kb.ns = max_ns;
    kb.batch = 1;
    ctx->tuned[kb] = best_b;
    KernelChoice best = best_b;
    if (n_frames == 1) {
        KernelChoice best_s;
        float t_best_s = 1e30f;
        for (int mapping : {SSILVB_MAP_CLASS, SSILVB_MAP_TILE})
            for (int minb : {8, 9})
                for (int order : {1, 2}) {
                    if (mapping == SSILVB_MAP_TILE && (minb == 8 || order == 2)) continue;
                    KernelChoice k;
                    k.mapping = mapping;
                    k.minb = minb;
                    k.order = mapping == SSILVB_MAP_CLASS ? order : 0;
                    bool ok;
                    const float t = time_runs(ctx, frames, 1, st, k, true, &ok);
                    if (!ok) return SSILVB_ERR_CUDA;
                    if (t < t_best_s) { t_best_s = t; best_s = k; }
                }
        ctx->tuned[tune_key(&frames[0].gbuffer, &frames[0].params, 0)] = best_s;
        best = best_s;
        best.rows = best_b.rows;
        best.graph = best_b.graph;
        best.batch_mode = best_b.batch_mode;
    }
    if (chosen) {
        std::memset(chosen, 0, sizeof(*chosen));
        chosen->mapping = best.mapping;
        chosen->occupancy = best.minb;
        chosen->rows_per_tile = best.rows;
        chosen->ctas_per_sm = best.ctas_per_sm;
        chosen->use_graph = best.graph ? 1 : 2;
        chosen->batch_mode = best.batch_mode;
        chosen->block_order = best.order;
    }
    return SSILVB_OK;
}

}  // extern "C"
