// Host-side internals shared by the ssilvb translation units: the context, argument
// validation, per-launch constants and the kernel launch wrappers (one unit per N_b, so the
// CUDA build compiles them in parallel).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "gather_kernel.cuh"
#include "ssilvb.h"

namespace ssilvb {

// ssilvb_gather_host splits a frame into at most this many row bands (one launch each).
constexpr int kMaxHostBands = 8;

// One host-buffer frame in flight: device staging for its inputs and outputs, the streams its
// inputs, row bands and output copies run on, and the events that order them.
struct HostLane {
    void *stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t in = nullptr, comp[2] = {nullptr, nullptr}, out = nullptr;
    cudaEvent_t inputs_ready = nullptr, comp1_done = nullptr, done = nullptr;
    cudaEvent_t band_done[kMaxHostBands] = {};
    bool pending = false;  // `done` is recorded and may still be outstanding
};

// A resolved launch choice.  Every choice gives bit-identical results.
struct KernelChoice {
    int mapping = SSILVB_MAP_CLASS;  // single frame: SSILVB_MAP_TILE or SSILVB_MAP_CLASS
    int minb = 9;                    // class/batch kernels: 8 (64 registers) or 9 (56) blocks of 128 threads per SM
    int rows = 1;                    // batch: rows per tile
    int ctas_per_sm = 0;             // batch: resident blocks per SM of the persistent grid (0 = occupancy)
    int graph = 1;                   // batch, persistent mode: launch through a CUDA graph
    int batch_mode = 2;              // batch: 1 persistent tile queue, 2 graph of per-frame kernels
    int order = 0;                   // class mapping: 0 by frame size (fill_params), 1 raster, 2 bands
};

// Apply a launch choice's block order to a frame's parameters (order 0 keeps fill_params's choice).
inline void apply_order(GatherParams &P, const KernelChoice &k) {
    if (k.order == 1) P.band_rows = 1;
    else if (k.order == 2) P.band_rows = 32;
}

// Default register budget of the class and batch kernels (CUDA events): 8 blocks of 128 threads per
// SM for N_b = 32 (at 4K 3.99 against 4.21 ms with 9); for N_b = 64 and 128, 8 on single frames of
// 2^22 pixels or more (at 4K 4.31 against 4.36 ms and 4.72 against 4.77 ms) and 9 otherwise (the
// 1080p trend rows at N_b 128 are 5-10 % faster with 9).
inline int default_minb(int nb, bool large_frame = false) { return nb == 32 || large_frame ? 8 : 9; }

cudaError_t launch_single_nb32(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s);
cudaError_t launch_single_nb64(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s);
cudaError_t launch_batch_nb32(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt, bool inf_t,
                              int step_mode, const KernelChoice &k, int grid, cudaStream_t s);
cudaError_t launch_batch_nb64(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt, bool inf_t,
                              int step_mode, const KernelChoice &k, int grid, cudaStream_t s);
cudaError_t launch_single_nb128(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s);
cudaError_t launch_batch_nb128(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt, bool inf_t,
                               int step_mode, const KernelChoice &k, int grid, cudaStream_t s);
int batch_occ_nb128(int fmt, bool inf_t, int minb);
void single_node_nb128(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, const void **fn, dim3 *grid,
                       dim3 *block);
// Dispatch on the sector count (32, 64 or 128).
cudaError_t launch_batch_nb(int nb, const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt,
                            bool inf_t, int step_mode, const KernelChoice &k, int grid, cudaStream_t s);
int batch_occ(int nb, int fmt, bool inf_t, int minb);
// The single-frame kernel of a variant and its launch shape (for graph kernel nodes).
void single_kernel_node(const GatherParams &P, int nb, int fmt, bool inf_t, const KernelChoice &k, const void **fn,
                        dim3 *grid, dim3 *block);
// Resident 128-thread blocks per SM of a batch kernel variant (occupancy calculator).
int batch_occ_nb32(int fmt, bool inf_t, int minb);
void single_node_nb32(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, const void **fn, dim3 *grid,
                      dim3 *block);
void single_node_nb64(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, const void **fn, dim3 *grid,
                      dim3 *block);
int batch_occ_nb64(int fmt, bool inf_t, int minb);

// One in-flight batch: device work list and queue counter, pinned host staging of the work
// list, the event that marks the batch's kernel done, and its cached CUDA graph.
struct BatchSlot {
    int cap = 0;
    char *d_table = nullptr;     // BatchHeader + FrameDesc[cap]
    unsigned *d_queue = nullptr;
    char *h_table = nullptr;     // pinned
    cudaEvent_t done = nullptr;
    bool pending = false;
    cudaGraphExec_t exec = nullptr;
    std::tuple<int, int, int, int, int, int, int> exec_key{-1, -1, -1, -1, -1, -1, -1};
    // graph of per-frame kernels: its instantiation and node handles (reused while the count matches)
    cudaGraph_t fgraph = nullptr;
    cudaGraphExec_t fexec = nullptr;
    std::vector<cudaGraphNode_t> fnodes;
    std::vector<GatherParams> fparams;  // argument storage of the nodes
};

struct TuneKey {
    int nb, fmt, inf_t, size_class, nd, ns, batch;  // fmt: the storage format code (ssilvb_format)
    bool operator<(const TuneKey &o) const {
        return std::tie(nb, fmt, inf_t, size_class, nd, ns, batch) <
               std::tie(o.nb, o.fmt, o.inf_t, o.size_class, o.nd, o.ns, o.batch);
    }
};

}  // namespace ssilvb

struct ssilvb_ctx {
    int device = 0;
    int num_sms = 0;
    int *d_status = nullptr;  // device status word (device-side checks and bounded waits)
    std::string last_error;
    // Host-buffer paths (host.cu), created on first use: the synchronous call's lane borrows the
    // caller's stream for its inputs and first band stream; the asynchronous calls alternate between
    // two lanes on context streams, so one frame's copies overlap the next frame's gather.
    bool host_ready = false;
    cudaStream_t host_band = nullptr, host_copy = nullptr;               // synchronous lane
    cudaStream_t async_in = nullptr, async_comp[2] = {}, async_out = nullptr;
    cudaEvent_t host_entry = nullptr;
    ssilvb::HostLane sync_lane, async_lane[2];
    int async_next = 0;
    ssilvb_tuning tuning = {SSILVB_MAP_AUTO, 0, 0, 0, 0, 0, 0, 0};
    cudaStream_t cap_stream = nullptr;     // private stream the batch graphs are captured on
    std::vector<ssilvb::BatchSlot> slots;  // ring of in-flight batches
    int next_slot = 0;
    std::map<ssilvb::TuneKey, ssilvb::KernelChoice> tuned;  // autotuner results
};

namespace ssilvb {

ssilvb_status fail(ssilvb_ctx *ctx, ssilvb_status s, const char *fmt, ...);
ssilvb_status cuda_fail(ssilvb_ctx *ctx, cudaError_t e, const char *what);
ssilvb_status validate(ssilvb_ctx *ctx, const ssilvb_gbuffer *g, const ssilvb_camera *c, const ssilvb_params *p,
                       const ssilvb_output *o, bool device_ptrs);
void fill_params(GatherParams &P, const ssilvb_gbuffer *g, const ssilvb_camera *c, const ssilvb_params *p,
                 const ssilvb_output *o);
TuneKey tune_key(const ssilvb_gbuffer *g, const ssilvb_params *p, int batch);
// The launch choice for a call: explicit tuning fields win, then autotuned results, then defaults.
KernelChoice resolve_choice(const ssilvb_ctx *ctx, const TuneKey &key);
cudaError_t launch_single(const GatherParams &P, int nb, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s);
void release_batch_slots(ssilvb_ctx *ctx);
// Host-buffer paths (host.cu): free their streams, events and staging; wait for asynchronous frames.
void release_host_resources(ssilvb_ctx *ctx);
ssilvb_status wait_host_async(ssilvb_ctx *ctx);

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace ssilvb
