// ssilvb_gather_batch_noalloc: the persistent batch gather without any device allocation.
//
// Some callers cannot allocate GPU memory at the point where they want to run the gather:
// a renderer or engine that reserves its whole device-memory budget up front and forbids
// driver allocations inside the frame loop, or a plug-in hosted by an application that owns
// all device memory.  cudaMalloc also synchronises the device, which a real-time frame loop
// cannot afford.  For them this entry point keeps the persistent kernel's scratch (its work
// list and tile-queue counter) in a fixed array that lives in the library image itself, so a
// call allocates nothing: no context, no cudaMalloc, no cudaFree, no graph, no event.  Calls
// share that array, so the caller must order them (one stream, or an event between them);
// calls that overlap on the GPU can mix frame tables and access memory out of bounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace ssilvb {
namespace {

constexpr int kNoAllocMaxFrames = 16;
constexpr size_t kQueueOffset = sizeof(BatchHeader) + kNoAllocMaxFrames * sizeof(FrameDesc);
constexpr size_t kScratchBytes = (kQueueOffset + sizeof(unsigned) + 255) & ~(size_t)255;

// The scratch of every call on a device: BatchHeader, FrameDesc[16], the queue counter.
// Every GPU that loads the library holds one copy (about 44 KB) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
// The name of the array is only a host-side stand-in; kernels must receive this address.
ssilvb_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, SSILVB_ERR_UNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(nullptr, e, "cudaGetSymbolAddress of the scratch array");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SSILVB_OK;
}

}  // namespace
}  // namespace ssilvb

using namespace ssilvb;

extern "C" ssilvb_status ssilvb_gather_batch_noalloc(const ssilvb_frame *frames, int n_frames,
                                                     struct CUstream_st *stream) {
    if (!frames || n_frames < 1 || n_frames > kNoAllocMaxFrames)
        return fail(nullptr, SSILVB_ERR_INVALID_ARG,
                    "ssilvb_gather_batch_noalloc takes 1..%d frames (got %d, or frames is NULL)", kNoAllocMaxFrames,
                    n_frames);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    void *scratch = nullptr;
    ssilvb_status st = scratch_address(dev, &scratch);
    if (st != SSILVB_OK) return st;

    // Validation through the same rules as every other entry point, against the current device.
    ssilvb_ctx probe;
    probe.device = dev;
    const int nb = frames[0].params.sector_count;
    const int fmt = frames[0].gbuffer.normal_fmt;
    const bool inf_t = std::isinf(frames[0].params.thickness);
    const int sm = frames[0].params.step_mode;
    for (int i = 0; i < n_frames; ++i) {
        const ssilvb_frame &f = frames[i];
        st = validate(&probe, &f.gbuffer, &f.camera, &f.params, &f.out, true);
        if (st != SSILVB_OK) return fail(nullptr, st, "frame %d: %s", i, probe.last_error.c_str());
        if (f.params.sector_count != nb || f.gbuffer.normal_fmt != fmt ||
            (bool)std::isinf(f.params.thickness) != inf_t || f.params.step_mode != sm)
            return fail(nullptr, SSILVB_ERR_UNSUPPORTED,
                        "frame %d: sector count, storage format, infinite thickness and step mode must match frame 0",
                        i);
    }

    // The work list, built on this call's stack (no heap), then copied into the scratch.
    KernelChoice k;  // library defaults: class-strided warps, one row per work item
    k.rows = 1;
    k.minb = default_minb(nb);
    alignas(16) unsigned char host[kQueueOffset];
    BatchHeader *hdr = reinterpret_cast<BatchHeader *>(host);
    FrameDesc *fd = reinterpret_cast<FrameDesc *>(host + sizeof(BatchHeader));
    long long tiles = 0;
    for (int i = 0; i < n_frames; ++i) {
        const ssilvb_frame &f = frames[i];
        std::memset(&fd[i], 0, sizeof(FrameDesc));
        fill_params(fd[i].P, &f.gbuffer, &f.camera, &f.params, &f.out);
        fd[i].tiles_x = 4 * ((f.gbuffer.width + 31) / 32);
        fd[i].rows = k.rows;
        fd[i].tile_begin = (int)tiles;
        tiles += (long long)fd[i].tiles_x * ((f.gbuffer.height + 15) / 16);
    }
    std::memset(hdr, 0, sizeof(BatchHeader));
    hdr->n_frames = n_frames;
    hdr->total_tiles = (int)tiles;

    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
    per_sm = batch_occ(nb, fmt, inf_t, k.minb);
    const int grid = std::max(1, std::max(1, per_sm) * sms);

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *base = static_cast<unsigned char *>(scratch);
    const size_t bytes = sizeof(BatchHeader) + (size_t)n_frames * sizeof(FrameDesc);
    // From pageable memory the copy returns once the bytes are staged, so `host` may be reused.
    e = cudaMemcpyAsync(base, host, bytes, cudaMemcpyHostToDevice, s);
    // The counter keeps the previous call's value: it must start at zero.
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kQueueOffset, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "work-list upload");
    const BatchHeader *d_hdr = reinterpret_cast<const BatchHeader *>(base);
    const FrameDesc *d_frames = reinterpret_cast<const FrameDesc *>(base + sizeof(BatchHeader));
    unsigned *d_queue = reinterpret_cast<unsigned *>(base + kQueueOffset);
    e = launch_batch_nb(nb, d_hdr, d_frames, d_queue, fmt, inf_t, sm, k, grid, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch launch");
    return SSILVB_OK;
}
