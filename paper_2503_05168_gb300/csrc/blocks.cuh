// blocks.cuh -- the tile blocks a visible record reaches, in emission order.
//
// Block binning (Sec. 3.1's tile intersection at the granularity of
// kBlockW x kBlockH tile blocks): per block row of the record's tile rect, the
// spans of its tile rows (the ellipse test of tiletest.cuh, or the whole rect
// row) are computed once, and every block met by their union becomes one
// instance carrying the mask of the block's tiles that the rows cover (bit
// q * kBlockW + i for tile column i of tile row q).  Block rows go top to
// bottom and blocks left to right.  Preprocessing counted exactly these blocks
// from the same stored floats (the same row_span calls), so the emitter's
// count always equals the record's scanned instance count.
#pragma once

#include "common.cuh"
#include "tiletest.cuh"

namespace seele {

__device__ __forceinline__ const CamDev& record_camera(const CamDev* __restrict__ cams, uint32_t r, int n_gauss) {
    return cams[r < (uint32_t)n_gauss ? 0u : r / (uint32_t)n_gauss];
}

// Calls f(k, unit, mask) for the k-th block instance of record r (unit = the
// global tile-block id) and returns the number of instances.
template <typename F>
__device__ __forceinline__ uint32_t for_each_block(const float4* __restrict__ rec, uint32_t r,
                                                   const CamDev* __restrict__ cams, int n_gauss, int tile_w,
                                                   int tile_h, int ellipse, F&& f) {
    const uint2 bx2 = rec_tile_box(rec, r);
    const int x0 = (int)(bx2.x & 0xffffu), y0 = (int)(bx2.x >> 16);
    const int x1 = (int)(bx2.y & 0xffffu), y1 = (int)(bx2.y >> 16);
    const CamDev& C = record_camera(cams, r, n_gauss);
    const uint32_t boff = C.block_offset, bx_n = (uint32_t)C.blocks_x;
    Ellipse E{};
    if (ellipse) E = make_ellipse(__ldg(rec + (size_t)kRecF4 * r), __ldg(rec + (size_t)kRecF4 * r + 1));
    uint32_t k = 0;
    for (int by = y0 / kBlockH; by <= y1 / kBlockH; ++by) {
        int lo[kBlockH], hi[kBlockH];
        int blo = 1 << 30, bhi = -1;
#pragma unroll
        for (int q = 0; q < kBlockH; ++q) {
            const int ty = by * kBlockH + q;
            lo[q] = 1;
            hi[q] = 0;
            if (ty < y0 || ty > y1) continue;
            int l = x0, h = x1;
            if (ellipse && !row_span(E, ty, tile_w, tile_h, x0, x1, &l, &h)) continue;
            lo[q] = l;
            hi[q] = h;
            blo = min(blo, l);
            bhi = max(bhi, h);
        }
        if (bhi < blo) continue;
        const uint32_t row_base = boff + (uint32_t)by * bx_n;
        for (int bx = blo / kBlockW; bx <= bhi / kBlockW; ++bx) {
            const int c0 = bx * kBlockW, c1 = c0 + kBlockW - 1;
            uint32_t mask = 0;
#pragma unroll
            for (int q = 0; q < kBlockH; ++q) {
                const int a = max(lo[q], c0), b = min(hi[q], c1);
                if (a <= b) mask |= ((0xffu >> (kBlockW - 1 - (b - a))) << (a - c0)) << (kBlockW * q);
            }
            f(k, row_base + (uint32_t)bx, mask);
            ++k;
        }
    }
    return k;
}

}  // namespace seele
