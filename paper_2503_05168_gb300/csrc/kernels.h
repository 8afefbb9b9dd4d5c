// kernels.h -- host-side launchers of the Seele kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace seele {

void launch_repack(int n, int nc, const float* means, const float* log_scales, const float* quats,
                   const float* logits, const float* sh, float4* pos_logit, float4* quat, float4* log_scale,
                   float4* shp, cudaStream_t s);

void launch_preprocess(const SceneDev& sc, const CamDev* cams, const FrameParams& fp, const ProjOut& out,
                       cudaStream_t s);

uint32_t scan_tiles_per_launch();
// cnt: per-record instance counts (0 = culled); pack: carry them in the
// values' top bits (R <= 2^24).
void launch_compact_visible(const uint32_t* cnt, bool pack, const float* depth, uint32_t R,
                            const uint32_t* chunk_vis, uint32_t* keys, uint32_t* vals, DeviceStatus* st,
                            cudaStream_t s);
// Instance offsets of the depth-ordered records and K (capacity check):
// cnt_sorted[j] is the instance count of the j-th record in depth order;
// chunk_sum: scratch of ceil(max_n / kChunkItems) words.
void launch_scan_tiles(const uint32_t* cnt_sorted, uint32_t* chunk_sum, uint32_t max_n, uint32_t* offsets,
                       DeviceStatus* st, uint32_t capacity, cudaStream_t s);

// Exclusive scan of a rows x stride row-major count matrix given its row
// totals (no look-back); a radix pass has 256 rows, one per digit.  With
// count_ptr the matrix is dense: its stride is ceil(*count_ptr / col_items)
// (at least 1; the launch's stride is the maximum) and the rest is not read.
void launch_digit_scan(const uint32_t* in, uint32_t stride, const uint32_t* row_total, uint32_t* out,
                       cudaStream_t s, uint32_t rows = 256, const uint32_t* count_ptr = nullptr,
                       uint32_t col_items = 1);
// Single-pass scan with decoupled look-back (in 16-byte aligned).  status:
// one word per block (exclusive_scan_blocks), entries of other epochs read as
// unpublished; st->ticket[ticket] must be zero.  spin_limit: polls of a
// predecessor before giving up (0: kSpinLimit); withhold: a test hook, the
// block with this ticket publishes nothing (UINT32_MAX: none).
void launch_exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint64_t* status, uint32_t epoch,
                           DeviceStatus* st, int ticket, cudaStream_t s, uint32_t spin_limit = 0,
                           uint32_t withhold = 0xffffffffu);
uint32_t exclusive_scan_blocks(uint32_t n);

// Spatial order of a scene (order.cu): Morton order of the means, stable;
// returns the ping-pong index holding the order in vals (0), or -1.
// bb: 6 words of scratch; count_ptr: device word holding n.
int launch_spatial_order(const float4* pos, int n, uint32_t* bb, uint32_t* keys[2], uint32_t* vals[2],
                         const uint32_t* count_ptr, uint32_t* counts, uint32_t* offsets, uint32_t* digit_totals,
                         cudaStream_t s);
void launch_gather_planes(const float4* src, float4* dst, int n, int planes, const uint32_t* order, cudaStream_t s);
void launch_gather_u32(const uint32_t* src, uint32_t* dst, int n, const uint32_t* order, cudaStream_t s);
void launch_scatter_u32(const uint32_t* src, uint32_t* dst, int n, const uint32_t* order, cudaStream_t s);

uint32_t sort_tile_items();
void launch_radix_upsweep_u32(const uint32_t* keys, const uint32_t* count_ptr, int shift, uint32_t* counts,
                              uint32_t stride, cudaStream_t s);
// keys_out == nullptr: write values only.
void launch_radix_downsweep_u32(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                uint32_t* vals_out, const uint32_t* count_ptr, int shift, int nbits,
                                const uint32_t* offsets, uint32_t stride, uint32_t* run_start, uint32_t* run_end,
                                cudaStream_t s);
// Words of one count matrix for a pass over max_n elements with digits of
// radix_bits bits.
uint32_t radix_count_words(uint32_t max_n, int radix_bits = 8);
// Digit width of the last pass of radix_sort_pairs for key_bits significant
// bits of a key_bytes-byte key: 9 or 10 (one pass) for 16-bit keys of that
// many bits, else 8.
int radix_last_bits(int key_bits, int key_bytes);
// Last-pass counts: out[o] = the instance count of sorted record o.  packed:
// the values carry the count in their top bits (kPackedIdBits; saturated
// counts are read from src) and the pass writes bare record ids; otherwise
// the count is src[value].
struct SortGather {
    const uint32_t* src = nullptr;
    uint32_t* out = nullptr;
    bool packed = false;
};
// Stable LSD sort of (keys[0], vals[0]) by their low `key_bits` bits in 8-bit
// digits (one 9- or 10-bit digit for 16-bit keys of that many bits); returns the index of the buffer pair holding the result, or -1 on a
// launch error.  With run_start / run_end (cleared to all-ones / zero, one
// word per key value) the last pass also records [first, last + 1) of every
// key value present -- the per-tile ranges.  With aux (two buffers, like vals)
// a second 32-bit payload is permuted with the values.  With gather (and no
// aux) the last pass also lays out the records' instance counts in sorted
// order (SortGather).
// digit_totals: 256 words per pass (1 << radix_last_bits for a one-pass
// wide sort), cleared by the caller; counts and offsets: radix_count_words
// (max_n, radix_last_bits) words each.
template <typename KeyT>
int radix_sort_pairs(KeyT* keys[2], uint32_t* vals[2], const uint32_t* count_ptr, uint32_t max_n, int key_bits,
                     bool keys_after_last, uint32_t* counts, uint32_t* offsets, uint32_t* digit_totals,
                     int& launches, cudaStream_t s, uint32_t* run_start = nullptr, uint32_t* run_end = nullptr,
                     uint32_t* const* aux = nullptr, const SortGather* gather = nullptr);

template <typename KeyT>
void launch_emit_blocks(const uint32_t* order, const uint32_t* offsets, const float4* rec,
                        const CamDev* cams, int n_gauss, int tile_w, int tile_h, int ellipse, DeviceStatus* st,
                        KeyT* inst_block, uint32_t* inst_rec, uint32_t* inst_mask, int blocks, cudaStream_t s);

// Tile binning through the blocks (binning.cu): the tile lists in tile
// order, made from the sorted block lists (each block's list filtered by
// each tile's bit, in order), and the tiles' ranges (starts[n_tiles], then
// ends), with K_t checked against the capacity.  Scratch: map (n_ids -
// n_blocks words, cleared to all-ones), C and Co (32 n_ids words each), Lt
// (32 ceil(n_tiles / 32) words, cleared), chunk_total (ceil(n_tiles / 32)
// words, cleared), St (like Lt); n_ids = expand_chunk_ids(capacity,
// n_blocks).
uint32_t expand_chunk_ids(uint64_t capacity, uint64_t n_blocks);
void launch_tile_expand(const uint32_t* rec_ids, const uint32_t* mask, const uint32_t* bstart, const uint32_t* bend,
                        uint32_t n_blocks, const CamDev* cams, int n_cams, uint32_t n_tiles, uint32_t n_ids,
                        uint32_t capacity, DeviceStatus* st, uint32_t* map, uint32_t* C, uint32_t* Co, uint32_t* Lt,
                        uint32_t* chunk_total, uint32_t* St, uint32_t* out_rec, uint32_t* ranges, cudaStream_t s);

// Block binning: OR of the tile masks of every 32 list entries, and the
// order in which the rasterizer visits tile blocks (longest lists first).
void launch_mask_summary(const uint32_t* mask, const DeviceStatus* st, uint32_t* summary, uint32_t max_groups,
                         cudaStream_t s);
void launch_block_order(const uint32_t* bstart, const uint32_t* bend, uint32_t n_blocks, uint32_t* order,
                        cudaStream_t s);
// The unit order for the persistent rasterizer: cameras in groups of `depth`
// (least total work first; 0: one group of all), longest lists first within
// a group.  Needs n_cams <= kViewOrderMaxCams.
constexpr int kViewOrderMaxCams = 1024;
void launch_view_order(const uint32_t* bstart, const uint32_t* bend, uint32_t n_units, const CamDev* cams, int n_cams,
                       bool blocks, int depth, uint32_t* order, cudaStream_t s);

// Offline view-dependent representation (views.cu).  k-means of n 6-D
// double points (one CTA); top-k contributors of a frame's tile lists ORed
// into the per-Gaussian cluster mask.
void launch_kmeans(const double* x, int n, int k, const double* u, int max_iter, double* cent, int* assign,
                   double* scratch, int* iters, cudaStream_t s);
// Contribution skew per pixel over the tile lists (seele_contribution_skew).
bool launch_skew(const uint32_t* starts, const uint32_t* ends, const uint32_t* inst_rec, const float4* rec,
                 const CamDev* cams, int n_cams, uint32_t n_tiles, const FrameParams& fp, double frac,
                 uint32_t* out_m, uint32_t* out_blended, uint32_t* out_walked, float* out_total,
                 uint32_t* out_listed, cudaStream_t s);

bool launch_topk(const uint32_t* starts, const uint32_t* ends, const uint32_t* inst_rec, const float4* rec,
                 const CamDev* cams, int n_cams, uint32_t n_tiles, const FrameParams& fp, int k,
                 const int* cam_cluster, uint32_t* mask, cudaStream_t s);

struct RasterArgs {
    const uint32_t* starts;     // [n_units]: unit u's list is [starts[u], ends[u]) (empty if start >= end);
    const uint32_t* ends;       //   units are tiles, or tile blocks with block binning
    const uint32_t* inst_rec;
    // block binning (else nullptr): per entry the tiles of its block it reaches,
    // and per 32 entries the OR of those masks; block_order: the order CTAs
    // visit the units (blocks, or tiles with tile binning) in
    const uint32_t* inst_mask;
    const uint32_t* mask_summary;
    const uint32_t* block_order;
    uint32_t n_blocks;
    const float4* rec;
    const CamDev* cams;
    int n_cams;
    uint32_t n_tiles;
    FrameParams fp;
    bool cr;
    int group_w, group_h;
    float* out_rgb;
    float* out_T;
    uint32_t* out_nc;
    DeviceStatus* count_into;   // non-null: run the counting variant
    DeviceStatus* status = nullptr;  // the frame's status word (checked build: index checks)
    unsigned long long* view_end;  // [n_cams] time the camera's last tile finished (%globaltimer)
    uint32_t* view_done;        // [n_cams] finished tiles, cleared per frame
    // tile binning (else nullptr): transmittance checkpoints, [slots][tile pixels]
    // (see kCkptShift), and every pixel's final (T, r, g, b)
    float4* ckpt;
    float4* cfin;
    // non-null: the persistent rasterizer, taking units in block_order's order
    // through this counter (zero at the frame's start); the counting variant
    // always runs one CTA per unit
    uint32_t* queue = nullptr;
};
bool launch_raster_fwd(const RasterArgs& a, cudaStream_t s);

// The multi-view autotuner's cache (tune_cache.cu): one configuration per key.
struct TuneEntry {
    int tile_w = 16, tile_h = 16, schedule = 0, batch_depth = 0;
    float batch_ms = 0.f, p50_ms = 0.f, p99_ms = 0.f;
};
bool tune_cache_lookup(const char* path, const std::string& key, TuneEntry* out);
bool tune_cache_store(const char* path, const std::string& key, const TuneEntry& e);

struct RasterBwdArgs {
    const uint32_t* starts;
    const uint32_t* ends;
    const uint32_t* inst_rec;
    const float4* rec;
    const CamDev* cams;
    int n_cams;
    uint32_t n_tiles;
    FrameParams fp;
    bool cr;
    int group_w, group_h;
    const float* dL_drgb;       // planar, the forward's output layout
    const float* T_final;
    const uint32_t* n_contrib;
    float* grad_rec;            // [R][12]: d(u, v, cA, cB, cC, log2 o, r, g, b), zeroed by the caller
    const uint32_t* tile_order; // nullable: CTA i walks tile tile_order[i] (longest lists first)
    // checkpoints of the forward pass (nullptr: each CTA walks a whole list):
    // CTAs n_tiles + i walk chunk i - (start >> kCkptShift) of tile chunk_map[i]
    const float4* ckpt;
    const float4* cfin;
    const uint32_t* chunk_map;
    uint32_t n_map;
};
void launch_chunk_map(const uint32_t* starts, const uint32_t* ends, uint32_t n_tiles, uint32_t* map, uint32_t n_map,
                      cudaStream_t s);
bool launch_raster_bwd(const RasterBwdArgs& a, cudaStream_t s);
// order (nullable): caller index of each resident Gaussian (spatial order)
void launch_preprocess_bwd(const SceneDev& sc, const CamDev* cams, const FrameParams& fp, const uint32_t* tiles,
                           const float* grad_rec, float* d_means, float* d_ls, float* d_quat, float* d_logit,
                           float* d_sh, const uint32_t* order, cudaStream_t s);

}  // namespace seele
