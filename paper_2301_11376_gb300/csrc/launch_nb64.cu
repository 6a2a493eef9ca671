// Kernel instantiations and launch wrappers for N_b = 64.
#include "launch_impl.cuh"

namespace ssilvb {

cudaError_t launch_single_nb64(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s) {
    return launch_single_nb<64>(P, fmt, inf_t, k, s);
}

cudaError_t launch_batch_nb64(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt, bool inf_t,
                              int step_mode, const KernelChoice &k, int grid, cudaStream_t s) {
    return launch_batch_nb<64>(hdr, frames, queue, fmt, inf_t, step_mode, k, grid, s);
}

int batch_occ_nb64(int fmt, bool inf_t, int minb) { return batch_occ_nb<64>(fmt, inf_t, minb); }

void single_node_nb64(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, const void **fn, dim3 *grid,
                     dim3 *block) {
    single_node_nb<64>(P, fmt, inf_t, k, fn, grid, block);
}

}  // namespace ssilvb
