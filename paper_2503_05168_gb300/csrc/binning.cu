// binning.cu -- tile instances (Sec. 3.1: "the preprocessing stage ...
// identifies the intersection between Gaussians and rendering tiles") and
// per-tile ranges into the sorted instance list.
#include "common.cuh"
#include "kernels.h"

namespace seele {

// A warp takes 32 consecutive visible records in depth order and writes all
// their (global tile, record) instances as one contiguous, coalesced run:
// lane l writes outputs l, l + 32, ... of the run and finds the record it
// belongs to by a binary search over the warp's exclusive counts.  Emission in
// depth order means the later stable sort by tile leaves each tile's list
// front to back; within one record the tiles of its rect go row-major.
template <typename KeyT>
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offsets,
                                                   const uint2* __restrict__ rect, const CamDev* __restrict__ cams,
                                                   int n_gauss, const DeviceStatus* __restrict__ st,
                                                   KeyT* __restrict__ inst_tile, uint32_t* __restrict__ inst_rec) {
    if (st->error != kOk) return;  // capacity overflow: nothing fits, outputs undefined
    const uint32_t n = st->n_visible;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wb = warp * 32; wb < n; wb += nwarps * 32) {
        const uint32_t j = wb + lane;
        uint32_t r = 0, x0 = 0, y0 = 0, w = 1, cnt = 0, row0 = 0, tx_n = 0;
        if (j < n) {
            r = __ldg(order + j);
            const uint2 b = __ldg(rect + r);
            x0 = b.x & 0xffffu;
            y0 = b.x >> 16;
            w = (b.y & 0xffffu) - x0 + 1;
            cnt = w * ((b.y >> 16) - y0 + 1);
            const CamDev& C = cams[r / (uint32_t)n_gauss];
            tx_n = (uint32_t)C.tiles_x;
            row0 = C.tile_offset;
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - cnt;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t base = __shfl_sync(0xffffffffu, j < n ? __ldg(offsets + j) : 0u, 0);
        // warp-uniform trip count: every shuffle below has all 32 lanes present
        for (uint32_t o0 = 0; o0 < total; o0 += 32) {
            const uint32_t o = o0 + lane;
            // largest lane s with excl_s <= o (lanes past the run search harmlessly)
            int s = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, excl, s + step);
                if (e <= o) s += step;
            }
            const uint32_t es = __shfl_sync(0xffffffffu, excl, s);
            const uint32_t ws = __shfl_sync(0xffffffffu, w, s);
            const uint32_t rs = __shfl_sync(0xffffffffu, row0, s);
            const uint32_t ys = __shfl_sync(0xffffffffu, y0, s);
            const uint32_t ns = __shfl_sync(0xffffffffu, tx_n, s);
            const uint32_t xs = __shfl_sync(0xffffffffu, x0, s);
            const uint32_t rr = __shfl_sync(0xffffffffu, r, s);
            if (o < total) {
                const uint32_t lt = o - es;
                const uint32_t ty = lt / ws, tx = lt - ty * ws;
                inst_tile[base + o] = (KeyT)(rs + (ys + ty) * ns + xs + tx);
                inst_rec[base + o] = rr;
            }
        }
    }
}

template <typename KeyT>
void launch_emit(const uint32_t* order, const uint32_t* offsets, const uint2* rect, const CamDev* cams, int n_gauss,
                 const DeviceStatus* st, KeyT* inst_tile, uint32_t* inst_rec, int blocks, cudaStream_t s) {
    emit_kernel<KeyT><<<blocks, 256, 0, s>>>(order, offsets, rect, cams, n_gauss, st, inst_tile, inst_rec);
}

template void launch_emit<uint16_t>(const uint32_t*, const uint32_t*, const uint2*, const CamDev*, int,
                                    const DeviceStatus*, uint16_t*, uint32_t*, int, cudaStream_t);
template void launch_emit<uint32_t>(const uint32_t*, const uint32_t*, const uint2*, const CamDev*, int,
                                    const DeviceStatus*, uint32_t*, uint32_t*, int, cudaStream_t);

}  // namespace seele
