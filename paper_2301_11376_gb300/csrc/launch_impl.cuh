// Launch wrappers for one sector count (included by launch_nb32.cu, launch_nb64.cu and launch_nb128.cu).
#pragma once

#include "internal.h"

namespace ssilvb {

// Launch grid of the class mapping: (4 row classes x TH patch rows, patch columns, bands of TH patch
// rows), TH = 1 for the raster order, else the band height closest to P.band_rows that splits the
// launch's patch rows into equal bands (the last one at most a row short).
inline dim3 class_grid(const GatherParams &P) {
    const int px = (P.W + 31) / 32, py = (P.y1 - P.y0 + 15) / 16;
    int th = 1;
    if (P.band_rows > 1) {
        const int nbands = (py + P.band_rows - 1) / P.band_rows;
        th = (py + nbands - 1) / nbands;
    }
    return dim3(4 * th, px, (py + th - 1) / th);
}

template <int NB, int FMT, bool INF_T, int SM>
cudaError_t launch_single_t(const GatherParams &P, const KernelChoice &k, cudaStream_t s) {
    if (k.mapping == SSILVB_MAP_TILE) {
        dim3 grid((P.W + 31) / 32, (P.y1 - P.y0 + 7) / 8);
        gather_tile_kernel<NB, FMT, INF_T, SM><<<grid, 256, 0, s>>>(P);
    } else {
        // 32 x 16 pixel patches, 4 row classes each (see gather_class_kernel)
        const dim3 grid = class_grid(P);
        if (k.minb == 8) gather_class_kernel<NB, FMT, INF_T, SM, 8><<<grid, 128, 0, s>>>(P);
        else gather_class_kernel<NB, FMT, INF_T, SM, 9><<<grid, 128, 0, s>>>(P);
    }
    return cudaGetLastError();
}

template <int NB, int FMT, bool INF_T>
cudaError_t launch_single_s(const GatherParams &P, const KernelChoice &k, cudaStream_t s) {
    return P.step_mode == 0 ? launch_single_t<NB, FMT, INF_T, 0>(P, k, s) : launch_single_t<NB, FMT, INF_T, 1>(P, k, s);
}

// fmt: the storage format code (0 binary32 planes, 1 binary16 planes, 2 interleaved binary16 plane)
template <int NB, int FMT>
cudaError_t launch_single_f(const GatherParams &P, bool inf_t, const KernelChoice &k, cudaStream_t s) {
    return inf_t ? launch_single_s<NB, FMT, true>(P, k, s) : launch_single_s<NB, FMT, false>(P, k, s);
}

template <int NB>
cudaError_t launch_single_nb(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, cudaStream_t s) {
    if (fmt == kFmtF16x8) return launch_single_f<NB, kFmtF16x8>(P, inf_t, k, s);
    if (fmt == kFmtF16) return launch_single_f<NB, kFmtF16>(P, inf_t, k, s);
    return launch_single_f<NB, kFmtF32>(P, inf_t, k, s);
}

template <int NB, int FMT, bool INF_T, int SM>
void single_node_t(const GatherParams &P, const KernelChoice &k, const void **fn, dim3 *grid, dim3 *block) {
    if (k.mapping == SSILVB_MAP_TILE) {
        *fn = reinterpret_cast<const void *>(gather_tile_kernel<NB, FMT, INF_T, SM>);
        *grid = dim3((P.W + 31) / 32, (P.y1 - P.y0 + 7) / 8);
        *block = dim3(256);
    } else {
        *fn = k.minb == 8 ? reinterpret_cast<const void *>(gather_class_kernel<NB, FMT, INF_T, SM, 8>)
                          : reinterpret_cast<const void *>(gather_class_kernel<NB, FMT, INF_T, SM, 9>);
        *grid = class_grid(P);
        *block = dim3(128);
    }
}

template <int NB, int FMT>
void single_node_f(const GatherParams &P, bool inf_t, const KernelChoice &k, const void **fn, dim3 *grid,
                   dim3 *block) {
    const bool s1 = P.step_mode != 0;
    if (inf_t) s1 ? single_node_t<NB, FMT, true, 1>(P, k, fn, grid, block) : single_node_t<NB, FMT, true, 0>(P, k, fn, grid, block);
    else s1 ? single_node_t<NB, FMT, false, 1>(P, k, fn, grid, block) : single_node_t<NB, FMT, false, 0>(P, k, fn, grid, block);
}

template <int NB>
void single_node_nb(const GatherParams &P, int fmt, bool inf_t, const KernelChoice &k, const void **fn, dim3 *grid,
                    dim3 *block) {
    if (fmt == kFmtF16x8) single_node_f<NB, kFmtF16x8>(P, inf_t, k, fn, grid, block);
    else if (fmt == kFmtF16) single_node_f<NB, kFmtF16>(P, inf_t, k, fn, grid, block);
    else single_node_f<NB, kFmtF32>(P, inf_t, k, fn, grid, block);
}

template <int NB, int FMT, bool INF_T, int SM>
cudaError_t launch_batch_t(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, const KernelChoice &k,
                           int grid, cudaStream_t s) {
    if (k.minb == 8) gather_batch_kernel<NB, FMT, INF_T, SM, 8><<<grid, 128, 0, s>>>(hdr, frames, queue);
    else gather_batch_kernel<NB, FMT, INF_T, SM, 9><<<grid, 128, 0, s>>>(hdr, frames, queue);
    return cudaGetLastError();
}

template <int NB, int FMT, bool INF_T>
cudaError_t launch_batch_s(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int step_mode,
                           const KernelChoice &k, int grid, cudaStream_t s) {
    return step_mode == 0 ? launch_batch_t<NB, FMT, INF_T, 0>(hdr, frames, queue, k, grid, s)
                          : launch_batch_t<NB, FMT, INF_T, 1>(hdr, frames, queue, k, grid, s);
}

template <int NB, int FMT>
cudaError_t launch_batch_f(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, bool inf_t, int step_mode,
                           const KernelChoice &k, int grid, cudaStream_t s) {
    return inf_t ? launch_batch_s<NB, FMT, true>(hdr, frames, queue, step_mode, k, grid, s)
                 : launch_batch_s<NB, FMT, false>(hdr, frames, queue, step_mode, k, grid, s);
}

template <int NB>
cudaError_t launch_batch_nb(const BatchHeader *hdr, const FrameDesc *frames, unsigned *queue, int fmt, bool inf_t,
                            int step_mode, const KernelChoice &k, int grid, cudaStream_t s) {
    if (fmt == kFmtF16x8) return launch_batch_f<NB, kFmtF16x8>(hdr, frames, queue, inf_t, step_mode, k, grid, s);
    if (fmt == kFmtF16) return launch_batch_f<NB, kFmtF16>(hdr, frames, queue, inf_t, step_mode, k, grid, s);
    return launch_batch_f<NB, kFmtF32>(hdr, frames, queue, inf_t, step_mode, k, grid, s);
}

template <int NB, int FMT, bool INF_T>
int batch_occ_t(int minb) {
    int n = 0;
    cudaError_t e = minb == 8
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_batch_kernel<NB, FMT, INF_T, 0, 8>, 128, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_batch_kernel<NB, FMT, INF_T, 0, 9>, 128, 0);
    return e == cudaSuccess ? n : 0;
}

template <int NB>
int batch_occ_nb(int fmt, bool inf_t, int minb) {
    if (fmt == kFmtF16x8) return inf_t ? batch_occ_t<NB, kFmtF16x8, true>(minb) : batch_occ_t<NB, kFmtF16x8, false>(minb);
    if (fmt == kFmtF16) return inf_t ? batch_occ_t<NB, kFmtF16, true>(minb) : batch_occ_t<NB, kFmtF16, false>(minb);
    return inf_t ? batch_occ_t<NB, kFmtF32, true>(minb) : batch_occ_t<NB, kFmtF32, false>(minb);
}

}  // namespace ssilvb
