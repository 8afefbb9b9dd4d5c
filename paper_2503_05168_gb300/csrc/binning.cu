// binning.cu -- tile instances (Sec. 3.1: "the preprocessing stage ...
// identifies the intersection between Gaussians and rendering tiles") and
// per-tile ranges into the sorted instance list.
#include "common.cuh"
#include "kernels.h"

namespace seele {

// One thread per visible record in depth order: writes (global tile, record)
// for every tile of its rect, row-major.  Emission in depth order means the
// later stable sort by tile leaves each tile's list front to back.
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offsets,
                                                   const uint2* __restrict__ rect, const CamDev* __restrict__ cams,
                                                   int n_gauss, const DeviceStatus* __restrict__ st,
                                                   uint32_t* __restrict__ inst_tile, uint32_t* __restrict__ inst_rec) {
    const uint32_t n = st->n_visible;
    if (st->error != kOk) return;  // capacity overflow: nothing fits, outputs undefined
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const uint32_t r = __ldg(order + j);
        uint32_t o = __ldg(offsets + j);
        const uint2 bx = __ldg(rect + r);
        const CamDev& C = cams[r / (uint32_t)n_gauss];
        const uint32_t x0 = bx.x & 0xffffu, y0 = bx.x >> 16, x1 = bx.y & 0xffffu, y1 = bx.y >> 16;
        for (uint32_t ty = y0; ty <= y1; ++ty) {
            const uint32_t row = C.tile_offset + ty * (uint32_t)C.tiles_x;
            for (uint32_t tx = x0; tx <= x1; ++tx) {
                inst_tile[o] = row + tx;
                inst_rec[o] = r;
                ++o;
            }
        }
    }
}

// ranges[t] = [first, last + 1) of tile t in the sorted list; tiles without
// instances keep the [0, 0) the caller cleared them to.
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ inst_tile,
                                                     const DeviceStatus* __restrict__ st, uint2* __restrict__ ranges) {
    if (st->error != kOk) return;
    const uint32_t K = st->n_inst_valid;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
        const uint32_t t = __ldg(inst_tile + i);
        const uint32_t prev = i > 0 ? __ldg(inst_tile + i - 1) : 0xffffffffu;
        const uint32_t next = i + 1 < K ? __ldg(inst_tile + i + 1) : 0xffffffffu;
        if (t != prev) ranges[t].x = i;
        if (t != next) ranges[t].y = i + 1;
    }
}

void launch_emit(const uint32_t* order, const uint32_t* offsets, const uint2* rect, const CamDev* cams, int n_gauss,
                 const DeviceStatus* st, uint32_t* inst_tile, uint32_t* inst_rec, int blocks, cudaStream_t s) {
    emit_kernel<<<blocks, 256, 0, s>>>(order, offsets, rect, cams, n_gauss, st, inst_tile, inst_rec);
}

void launch_ranges(const uint32_t* inst_tile, const DeviceStatus* st, uint2* ranges, int blocks, cudaStream_t s) {
    ranges_kernel<<<blocks, 256, 0, s>>>(inst_tile, st, ranges);
}

}  // namespace seele
