// raster.cu -- launches of the tile rasterizer (raster_impl.cuh): one CTA per
// list unit, or the persistent queue kernels of raster_queue.cu.
#include "raster_impl.cuh"

namespace seele {

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool COUNT, bool BLOCKS>
static void launch_variant(const RasterArgs& a, cudaStream_t s) {
    constexpr int NT = (TW / PW) * (TH / PH);
    if (!COUNT && a.queue != nullptr) {
        launch_raster_queue<TW, TH, PW, PH, GW, GH, CR, BLOCKS>(a, s);
        return;
    }
    const uint32_t grid = BLOCKS ? 32 * a.n_blocks : a.n_tiles;
    launch_pdl(raster_fwd_kernel<TW, TH, PW, PH, GW, GH, CR, COUNT, BLOCKS>, dim3(grid), dim3(NT), 0, s,
               a.starts, a.ends, a.inst_rec, a.inst_mask, a.mask_summary, a.block_order, a.rec, a.cams, a.n_cams,
               a.fp, a.out_rgb, a.out_T, a.out_nc, COUNT ? a.count_into : a.status, a.view_end, a.view_done,
               (COUNT || BLOCKS) ? nullptr : a.ckpt, (COUNT || BLOCKS) ? nullptr : a.cfin);
}

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR>
static void launch_one(const RasterArgs& a, cudaStream_t s) {
    const bool blocks = a.inst_mask != nullptr;
    if (a.count_into) {
        if (blocks) launch_variant<TW, TH, PW, PH, GW, GH, CR, true, true>(a, s);
        else launch_variant<TW, TH, PW, PH, GW, GH, CR, true, false>(a, s);
    } else {
        if (blocks) launch_variant<TW, TH, PW, PH, GW, GH, CR, false, true>(a, s);
        else launch_variant<TW, TH, PW, PH, GW, GH, CR, false, false>(a, s);
    }
}

template <int TW, int TH>
static bool launch_shape(const RasterArgs& a, cudaStream_t s) {
    if (!a.cr) launch_one<TW, TH, 2, 2, 1, 1, false>(a, s);
    else if (a.group_w == 2 && a.group_h == 2) launch_one<TW, TH, 2, 2, 2, 2, true>(a, s);
    else if (a.group_w == 1 && a.group_h == 1) launch_one<TW, TH, 2, 2, 1, 1, true>(a, s);
    else if (a.group_w == 2 && a.group_h == 4) launch_one<TW, TH, 2, 4, 2, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 4) launch_one<TW, TH, 2, 2, 4, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 8) launch_one<TW, TH, 2, 4, 4, 8, true>(a, s);
    else return false;
    return true;
}

// 8x8 tiles: a pair of pixels in a row per thread, one warp per tile; a group
// of two or more columns is whole threads
static bool launch_shape_8x8(const RasterArgs& a, cudaStream_t s) {
    if (!a.cr) launch_one<8, 8, 2, 1, 1, 1, false>(a, s);
    else if (a.group_w == 2 && a.group_h == 2) launch_one<8, 8, 2, 1, 2, 2, true>(a, s);
    else if (a.group_w == 1 && a.group_h == 1) launch_one<8, 8, 2, 1, 1, 1, true>(a, s);
    else if (a.group_w == 2 && a.group_h == 4) launch_one<8, 8, 2, 1, 2, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 4) launch_one<8, 8, 2, 1, 4, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 8) launch_one<8, 8, 2, 1, 4, 8, true>(a, s);
    else return false;
    return true;
}

bool launch_raster_fwd(const RasterArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return true;
    if (a.fp.tile_w == 8 && a.fp.tile_h == 8) return launch_shape_8x8(a, s);
    if (a.fp.tile_w == 16 && a.fp.tile_h == 16) return launch_shape<16, 16>(a, s);
    if (a.fp.tile_w == 32 && a.fp.tile_h == 8) return launch_shape<32, 8>(a, s);
    if (a.fp.tile_w == 32 && a.fp.tile_h == 16) return launch_shape<32, 16>(a, s);
    return false;
}

}  // namespace seele
