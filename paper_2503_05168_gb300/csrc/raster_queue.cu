// raster_queue.cu -- the persistent, queue-driven launches of the tile
// rasterizer (raster_impl.cuh): one resident wave of CTAs pulls list units
// from an atomic counter in the order the frame's unit order gives (longest
// lists first, or cameras in groups, see launch_view_order).
#include "raster_impl.cuh"

namespace seele {

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool BLOCKS>
void launch_raster_queue(const RasterArgs& a, cudaStream_t s) {
    constexpr int NT = (TW / PW) * (TH / PH);
    auto kernel = raster_queue_kernel<TW, TH, PW, PH, GW, GH, CR, BLOCKS>;
    static int per_sm = 0, sms = 0;  // resident CTAs of this variant, SMs of the device
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, 0);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    const uint32_t n_items = BLOCKS ? 32 * a.n_blocks : a.n_tiles;
    const uint32_t grid = std::min<uint32_t>(n_items, (uint32_t)(per_sm * sms));
    launch_pdl(kernel, dim3(std::max<uint32_t>(grid, 1u)), dim3(NT), 0, s, a.starts, a.ends, a.inst_rec, a.inst_mask,
               a.mask_summary, a.block_order, a.rec, a.cams, a.n_cams, a.fp, a.out_rgb, a.out_T, a.out_nc,
               a.status, a.view_end, a.view_done, BLOCKS ? nullptr : a.ckpt,
               BLOCKS ? nullptr : a.cfin, n_items, a.queue);
}

#define SEELE_QUEUE_SHAPE(TW, TH, PW, PH)                                                      \
    template void launch_raster_queue<TW, TH, PW, PH, 1, 1, false, false>(const RasterArgs&, cudaStream_t); \
    template void launch_raster_queue<TW, TH, PW, PH, 1, 1, false, true>(const RasterArgs&, cudaStream_t);  \
    template void launch_raster_queue<TW, TH, PW, PH, 1, 1, true, false>(const RasterArgs&, cudaStream_t);  \
    template void launch_raster_queue<TW, TH, PW, PH, 1, 1, true, true>(const RasterArgs&, cudaStream_t);

// the variants launch_shape and launch_shape_8x8 dispatch to
SEELE_QUEUE_SHAPE(16, 16, 2, 2)
SEELE_QUEUE_SHAPE(32, 8, 2, 2)
SEELE_QUEUE_SHAPE(32, 16, 2, 2)
SEELE_QUEUE_SHAPE(8, 8, 2, 1)
#define SEELE_QUEUE_CR(TW, TH, PW, PH, GW, GH)                                                          \
    template void launch_raster_queue<TW, TH, PW, PH, GW, GH, true, false>(const RasterArgs&, cudaStream_t); \
    template void launch_raster_queue<TW, TH, PW, PH, GW, GH, true, true>(const RasterArgs&, cudaStream_t);
#define SEELE_QUEUE_CR_SHAPE(TW, TH)     \
    SEELE_QUEUE_CR(TW, TH, 2, 2, 2, 2)   \
    SEELE_QUEUE_CR(TW, TH, 2, 4, 2, 4)   \
    SEELE_QUEUE_CR(TW, TH, 2, 2, 4, 4)   \
    SEELE_QUEUE_CR(TW, TH, 2, 4, 4, 8)
SEELE_QUEUE_CR_SHAPE(16, 16)
SEELE_QUEUE_CR_SHAPE(32, 8)
SEELE_QUEUE_CR_SHAPE(32, 16)
SEELE_QUEUE_CR(8, 8, 2, 1, 2, 2)
SEELE_QUEUE_CR(8, 8, 2, 1, 2, 4)
SEELE_QUEUE_CR(8, 8, 2, 1, 4, 4)
SEELE_QUEUE_CR(8, 8, 2, 1, 4, 8)

}  // namespace seele
