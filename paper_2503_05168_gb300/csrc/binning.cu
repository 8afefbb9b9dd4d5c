// binning.cu -- tile instances (Sec. 3.1: the tile intersections found in
// preprocessing become per-tile lists) and their ranges: block instances
// emitted in depth order, and -- for tile binning -- the sorted block lists
// expanded into tile lists.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "blocks.cuh"
#include "tiletest.cuh"

namespace seele {

// Block binning: one thread per depth-ordered record writes its (block,
// record, mask) entries (blocks.cuh) at the record's scanned offset -- a
// record reaches about two tile blocks on average, too few to be worth a warp.
template <typename KeyT>
__global__ void __launch_bounds__(256) emit_blocks_kernel(const uint32_t* __restrict__ order,
                                                          const uint32_t* __restrict__ offsets,
                                                          const float4* __restrict__ rec,
                                                          const CamDev* __restrict__ cams, int n_gauss, int tile_w,
                                                          int tile_h, int ellipse, DeviceStatus* st,
                                                          KeyT* __restrict__ inst_block,
                                                          uint32_t* __restrict__ inst_rec,
                                                          uint32_t* __restrict__ inst_mask) {
    pdl_enter();
    if (st->error != kOk) return;
    const uint32_t n = st->n_visible;
    const uint32_t n_inst = st->n_instances;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const uint32_t r = __ldg(order + j);
        const uint32_t pos = __ldg(offsets + j);
        const uint32_t end = j + 1 < n ? __ldg(offsets + j + 1) : n_inst;
        const uint32_t got = for_each_block(rec, r, cams, n_gauss, tile_w, tile_h, ellipse,
                                            [&](uint32_t k, uint32_t unit, uint32_t mask) {
                                                if (pos + k < end) {
                                                    inst_block[pos + k] = (KeyT)unit;
                                                    inst_rec[pos + k] = r;
                                                    inst_mask[pos + k] = mask;
                                                }
                                            });
        if (pos + got != end) {
            // never expected: both counts come from the same row_span on the
            // same stored floats.  Report it and keep every slot a valid entry.
            record_error(st, kErrInternal, 8);
            const uint32_t boff = record_camera(cams, r, n_gauss).block_offset;
            for (uint32_t p = pos + got; p < end; ++p) {
                inst_block[p] = (KeyT)boff;
                inst_rec[p] = r;
                inst_mask[p] = 0u;
            }
        }
    }
}

// Tile binning through the blocks: a tile's list is its block's list kept
// where the entry's mask has the tile's bit, in order (the (tile, depth,
// record) order of Sec. 3.1), so the tile lists are made by expanding the
// sorted block lists -- about a quarter as many entries to sort as tile
// instances.  A block's list is cut into chunks of kExpandChunk entries.
// Chunk 0 of block b has id b; chunk i >= 1 has id n_blocks + (start_b >>
// kExpandShift) + i, unique because the block lists are disjoint (the last
// of these ids of a block lies below the first of the next block), so no
// scan is needed to place them.
//   expand_map:     id of a later chunk -> block;
//   expand_count:   per chunk, the entries of each of its block's 32 tiles;
//   expand_offsets: per block and tile bit, each chunk's start inside the
//                   tile's list, the tile's count at its global tile id (Lt)
//                   and its 32-tile chunk's total; an exclusive scan of Lt
//                   then gives the list starts (St), so the lists lie in tile
//                   order, as a sort by tile would leave them;
//   expand_write:   per chunk, staged in shared memory, warp t keeps the
//                   entries with bit t (tile t % 8, t / 8 of the block) and
//                   writes them at their places; the block's first chunk
//                   writes the tiles' ranges; K_t is checked against the
//                   capacity.
constexpr int kExpandShift = 11;
constexpr uint32_t kExpandChunk = 1u << kExpandShift;
constexpr int kExpandThreads = 256;   // expand_write: 8 warps of 8 groups of 32 entries
constexpr int kExpandGroups = kExpandChunk / kExpandThreads;
static_assert(kExpandGroups == 8 && kBlockW * kBlockH == 32, "a lane per tile of the block");
constexpr int kCountThreads = 256;    // expand_count: 8 entries per thread
static_assert(kExpandChunk == 8 * kCountThreads, "eight counted entries per thread");

// chunk ids: n_blocks first chunks, then the later-chunk slots
uint32_t expand_chunk_ids(uint64_t capacity, uint64_t n_blocks) {
    return (uint32_t)(n_blocks + (capacity >> kExpandShift) + 2);
}

// The global id of tile bit t of block b, or UINT32_MAX where the block
// overhangs its camera's tile grid.
__device__ __forceinline__ uint32_t block_tile(const CamDev* __restrict__ cams, int n_cams, uint32_t b, int t) {
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].block_offset <= b) lo = mid; else hi = mid - 1;
    }
    const CamDev& C = cams[lo];
    const uint32_t lb = b - C.block_offset;
    const int tx = (int)(lb % (uint32_t)C.blocks_x) * kBlockW + t % kBlockW;
    const int ty = (int)(lb / (uint32_t)C.blocks_x) * kBlockH + t / kBlockW;
    if (tx >= C.tiles_x || ty >= C.tiles_y) return 0xffffffffu;
    return C.tile_offset + (uint32_t)(ty * C.tiles_x + tx);
}

__device__ __forceinline__ uint2 block_range(const uint32_t* __restrict__ bstart, const uint32_t* __restrict__ bend,
                                             uint32_t b) {
    const uint32_t s = __ldg(bstart + b), e = __ldg(bend + b);
    return s < e ? make_uint2(s, e) : make_uint2(0u, 0u);
}

// The chunk behind CTA id: its block (UINT32_MAX: none) and index.
__device__ __forceinline__ uint32_t chunk_block(uint32_t id, uint32_t n_blocks, const uint32_t* __restrict__ map) {
    return id < n_blocks ? id : __ldg(map + (id - n_blocks));
}

__device__ __forceinline__ uint32_t chunk_id(uint32_t b, uint32_t start, uint32_t i, uint32_t n_blocks) {
    return i == 0 ? b : n_blocks + (start >> kExpandShift) + i;
}

// map[slot] = block for every chunk i >= 1 (slot = (start_b >> kExpandShift)
// + i; the map is cleared to UINT32_MAX first).
__global__ void expand_map_kernel(const uint32_t* __restrict__ bstart, const uint32_t* __restrict__ bend,
                                  uint32_t n_blocks, const DeviceStatus* __restrict__ st, uint32_t n_slots,
                                  uint32_t* __restrict__ map) {
    pdl_enter();
    if (st->error != kOk) return;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks; b += gridDim.x * blockDim.x) {
        const uint2 r = block_range(bstart, bend, b);
        const uint32_t n = (r.y - r.x + kExpandChunk - 1) >> kExpandShift;
        for (uint32_t i = 1; i < n; ++i) {
            const uint32_t slot = (r.x >> kExpandShift) + i;
            if (slot < n_slots) map[slot] = b;
        }
    }
}

// 32 x 32 bit transpose across a warp: lane l brings word x (bit t = entry
// l's tile bit t) and gets back the word whose bit e is bit l of lane e's
// word -- for lane t, which of the warp's 32 entries reach tile t.  Five
// exchanges, each swapping the off-diagonal sub-blocks of the next smaller
// scale between lane pairs.  Every lane of the warp calls it together.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    constexpr uint32_t kM[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const uint32_t other = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? (x & ~kM[k]) | ((other >> j) & kM[k]) : (x & kM[k]) | ((other & kM[k]) << j);
    }
    return x;
}

// The chunk ids in use: the first chunks, then the later-chunk slots below
// the block instances' end (K_b, on the device).
__device__ __forceinline__ uint32_t chunk_ids_used(const DeviceStatus* st, uint32_t n_blocks, uint32_t n_ids) {
    const uint32_t kb = *(volatile const int32_t*)&st->error == kOk ? *(volatile const uint32_t*)&st->n_inst_valid
                                                                    : 0u;
    return min(n_ids, n_blocks + (kb >> kExpandShift) + 2u);
}

__global__ void __launch_bounds__(kCountThreads) expand_count_kernel(const uint32_t* __restrict__ mask,
                                                                     const uint32_t* __restrict__ bstart,
                                                                     const uint32_t* __restrict__ bend,
                                                                     uint32_t n_blocks, uint32_t n_ids,
                                                                     const DeviceStatus* __restrict__ st,
                                                                     const uint32_t* __restrict__ map,
                                                                     uint32_t* __restrict__ C) {
    __shared__ uint32_t s_c[32];
    __shared__ uint32_t s_used;
    pdl_enter();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_used = chunk_ids_used(st, n_blocks, n_ids);
    __syncthreads();
    const uint32_t used = s_used;
    for (uint32_t id = blockIdx.x; id < used; id += gridDim.x) {
        const uint32_t b = chunk_block(id, n_blocks, map);
        if (b == 0xffffffffu) continue;
        if (threadIdx.x < 32) s_c[threadIdx.x] = 0u;
        __syncthreads();
        const uint2 r = block_range(bstart, bend, b);
        const uint32_t i = id < n_blocks ? 0u : id - n_blocks - (r.x >> kExpandShift);
        const uint32_t c0 = r.x + i * kExpandChunk, c1 = min(r.y, c0 + kExpandChunk);
        // lane t counts bit t over the warp's 8 groups of 32 entries
        uint32_t m[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t j = c0 + (uint32_t)(256 * w + 32 * q + lane);
            m[q] = j < c1 ? __ldg(mask + j) : 0u;
        }
        uint32_t n = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) n += __popc(warp_transpose32(m[q], lane));
        atomicAdd(&s_c[lane], n);
        __syncthreads();
        if (threadIdx.x < 32) C[(size_t)id * 32 + threadIdx.x] = s_c[threadIdx.x];
        __syncthreads();
    }
}

// One warp per block, lane t for tile bit t.
__global__ void expand_offsets_kernel(const uint32_t* __restrict__ bstart, const uint32_t* __restrict__ bend,
                                      uint32_t n_blocks, const CamDev* __restrict__ cams, int n_cams,
                                      const DeviceStatus* __restrict__ st, const uint32_t* __restrict__ C,
                                      uint32_t* __restrict__ Co, uint32_t* __restrict__ Lt,
                                      uint32_t* __restrict__ chunk_total) {
    pdl_enter();
    if (st->error != kOk) return;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < n_blocks; b += warps) {
        const uint2 r = block_range(bstart, bend, b);
        const uint32_t n = (r.y - r.x + kExpandChunk - 1) >> kExpandShift;
        uint32_t run = 0;
        for (uint32_t i = 0; i < n; ++i) {
            const size_t k = (size_t)chunk_id(b, r.x, i, n_blocks) * 32 + lane;
            const uint32_t v = __ldg(C + k);
            Co[k] = run;
            run += v;
        }
        const uint32_t g = block_tile(cams, n_cams, b, lane);
        if (g != 0xffffffffu) {
            Lt[g] = run;
            if (run != 0u) atomicAdd(chunk_total + (g >> 5), run);
        }
    }
}

__global__ void __launch_bounds__(kExpandThreads) expand_write_kernel(
    const uint32_t* __restrict__ rec_ids, const uint32_t* __restrict__ mask, const uint32_t* __restrict__ bstart,
    const uint32_t* __restrict__ bend, uint32_t n_blocks, uint32_t n_ids, const uint32_t* __restrict__ map,
    const uint32_t* __restrict__ Co,
    const uint32_t* __restrict__ Lt, const uint32_t* __restrict__ St, const CamDev* __restrict__ cams, int n_cams,
    uint32_t n_tiles, uint32_t capacity, DeviceStatus* st, uint32_t* __restrict__ out_rec,
    uint32_t* __restrict__ ranges) {
    __shared__ uint32_t s_wc[kExpandThreads / 32][33];  // per warp and tile: count, then start
    __shared__ int32_t s_err;
    __shared__ uint32_t s_used;
    pdl_enter();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // K_t = the last tile's start plus its count; every CTA checks it alike
    const uint32_t K = __ldg(St + n_tiles - 1) + __ldg(Lt + n_tiles - 1);
    // read once for the whole CTA: CTA 0 replaces the instance count below
    // (a CTA that reads it afterwards only visits more empty chunk ids)
    if (threadIdx.x == 0) {
        s_err = *(volatile const int32_t*)&st->error;
        s_used = chunk_ids_used(st, n_blocks, n_ids);
    }
    __syncthreads();
    if (s_err != kOk) return;
    if (K > capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->n_instances = K;
            st->capacity = capacity;
            record_error(st, kErrCapacity, 11);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->n_instances = K;
        st->capacity = capacity;
        st->n_inst_valid = K;
    }
    const uint32_t used = s_used;
    for (uint32_t id = blockIdx.x; id < used; id += gridDim.x) {
        const uint32_t b = chunk_block(id, n_blocks, map);
        if (b == 0xffffffffu) continue;
        const uint2 r = block_range(bstart, bend, b);
        const uint32_t i = id < n_blocks ? 0u : id - n_blocks - (r.x >> kExpandShift);
        const uint32_t c0 = r.x + i * kExpandChunk, c1 = min(r.y, c0 + kExpandChunk), n = c1 - c0;
        // warp w takes entries [256 w, 256 w + 256) of the chunk, 8 groups of
        // 32, in registers; after the transpose lane t holds, per group,
        // which of them reach tile t.  First each warp's count per tile, then,
        // from the tiles' list starts, the warps' own starts, then the writes.
        uint32_t col[kExpandGroups], rq[kExpandGroups], cnt = 0;
#pragma unroll
        for (int q = 0; q < kExpandGroups; ++q) {
            const uint32_t k = 32u * (kExpandGroups * (uint32_t)w + (uint32_t)q) + (uint32_t)lane;
            const bool ok = k < n;
            rq[q] = ok ? __ldg(rec_ids + c0 + k) : 0u;
            col[q] = warp_transpose32(ok ? __ldg(mask + c0 + k) : 0u, lane);
            cnt += __popc(col[q]);
        }
        __syncthreads();  // the previous chunk's starts have been read
        s_wc[w][lane] = cnt;
        __syncthreads();
        if (w == 0) {
            const uint32_t g0 = block_tile(cams, n_cams, b, lane);
            uint32_t run = g0 == 0xffffffffu ? 0u : __ldg(St + g0) + __ldg(Co + (size_t)id * 32 + lane);
            if (g0 != 0xffffffffu && i == 0) {
                ranges[g0] = __ldg(St + g0);
                ranges[n_tiles + g0] = __ldg(St + g0) + __ldg(Lt + g0);
            }
#pragma unroll
            for (int ww = 0; ww < kExpandThreads / 32; ++ww) {
                const uint32_t x = s_wc[ww][lane];
                s_wc[ww][lane] = run;
                run += x;
            }
        }
        __syncthreads();
        // the warp writes one tile's run at a time (coalesced): lane e stores
        // its own entry when it reaches the tile; every tile in turn,
        // unrolled, so that the shuffles of different tiles overlap
        const uint32_t pos = s_wc[w][lane];
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int tt = 0; tt < 32; ++tt) {
            uint32_t p = __shfl_sync(0xffffffffu, pos, tt);
#pragma unroll
            for (int q = 0; q < kExpandGroups; ++q) {
                const uint32_t c = __shfl_sync(0xffffffffu, col[q], tt);
                if ((c >> lane) & 1u) {
                    const uint32_t o = p + __popc(c & lt);
                    if (o < capacity) out_rec[o] = rq[q];
                }
                p += __popc(c);
            }
        }
    }
}

void launch_tile_expand(const uint32_t* rec_ids, const uint32_t* mask, const uint32_t* bstart, const uint32_t* bend,
                        uint32_t n_blocks, const CamDev* cams, int n_cams, uint32_t n_tiles, uint32_t n_ids,
                        uint32_t capacity, DeviceStatus* st, uint32_t* map, uint32_t* C, uint32_t* Co, uint32_t* Lt,
                        uint32_t* chunk_total, uint32_t* St, uint32_t* out_rec, uint32_t* ranges, cudaStream_t s) {
    const uint32_t nb = std::max<uint32_t>(n_blocks, 1u);
    launch_pdl(expand_map_kernel, dim3(std::min<uint32_t>((nb + 255) / 256, 1024u)), dim3(256), 0, s, bstart, bend,
               n_blocks, (const DeviceStatus*)st, n_ids - n_blocks, map);
    int sms = 152;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    launch_pdl(expand_count_kernel, dim3(std::min<uint32_t>(n_ids, 8u * (uint32_t)sms)), dim3(kCountThreads), 0, s,
               mask, bstart, bend, n_blocks, n_ids, (const DeviceStatus*)st, (const uint32_t*)map, C);
    launch_pdl(expand_offsets_kernel, dim3(std::min<uint32_t>((nb + 7) / 8, 2048u)), dim3(256), 0, s, bstart, bend,
               n_blocks, cams, n_cams, (const DeviceStatus*)st, (const uint32_t*)C, Co, Lt, chunk_total);
    const uint32_t chunks = (n_tiles + 31) / 32;
    launch_digit_scan(Lt, 32, chunk_total, St, s, chunks);
    launch_pdl(expand_write_kernel, dim3(std::min<uint32_t>(n_ids, 8u * (uint32_t)sms)), dim3(kExpandThreads), 0, s,
               rec_ids, mask, bstart, bend, n_blocks, n_ids, (const uint32_t*)map, (const uint32_t*)Co, (const uint32_t*)Lt, (const uint32_t*)St, cams, n_cams,
               n_tiles, capacity, st, out_rec, ranges);
}

// After the block sort: the OR of the tile masks of every 32 consecutive
// entries (aligned to the list array), so a tile's rasterizer can skip 32
// entries of its block list with one load when none of them reaches it.
__global__ void mask_summary_kernel(const uint32_t* __restrict__ mask, const DeviceStatus* __restrict__ st,
                                    uint32_t* __restrict__ summary, uint32_t max_groups) {
    constexpr int kInFlight = 8;  // groups per warp with their loads issued together
    pdl_enter();
    const uint32_t n = st->error == kOk ? st->n_inst_valid : 0u;
    const uint32_t groups = min((n + 31) / 32, max_groups);
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g0 < groups; g0 += kInFlight * warps) {
        uint32_t m[kInFlight];
#pragma unroll
        for (int q = 0; q < kInFlight; ++q) {
            const uint32_t j = 32 * (g0 + q * warps) + lane;
            m[q] = j < n ? __ldg(mask + j) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kInFlight; ++q) {
            const uint32_t g = g0 + q * warps;
            const uint32_t o = __reduce_or_sync(0xffffffffu, m[q]);
            if (lane == 0 && g < groups) summary[g] = o;
        }
    }
}

void launch_mask_summary(const uint32_t* mask, const DeviceStatus* st, uint32_t* summary, uint32_t max_groups,
                         cudaStream_t s) {
    const uint32_t blocks = std::max<uint32_t>(1u, std::min<uint32_t>((max_groups + 7) / 8, 152u * 16u));
    launch_pdl(mask_summary_kernel, dim3(blocks), dim3(256), 0, s, mask, st, summary, max_groups);
}

// Longest lists first: the raster grid walks tile blocks in decreasing order
// of their list length (a counting sort on a log-scale bucket of the length,
// one CTA), so the longest-running tiles start early and no straggler is
// left for the end of the kernel.  Order within a bucket is free.
constexpr int kOrderBuckets = 64;

constexpr uint32_t kOrderCache = 32768;  // units whose buckets stay in shared memory

__global__ void __launch_bounds__(1024) block_order_kernel(const uint32_t* __restrict__ bstart,
                                                           const uint32_t* __restrict__ bend, uint32_t n_blocks,
                                                           uint32_t* __restrict__ order) {
    __shared__ uint32_t s_hist[kOrderBuckets];
    __shared__ uint32_t s_pos[kOrderBuckets];
    __shared__ uint8_t s_bucket[kOrderCache];
    pdl_enter();
    auto bucket_of = [](uint32_t s, uint32_t e) -> int {
        const uint32_t len = s < e ? e - s : 0u;
        // 4 buckets per octave, longest lists in bucket 0
        const uint32_t v = len + 1u;
        const int lg = 31 - __clz(v);
        const int frac = lg >= 2 ? (int)((v >> (lg - 2)) & 3u) : (int)((v << (2 - lg)) & 3u);
        return kOrderBuckets - 1 - min(kOrderBuckets - 1, lg * 4 + frac);
    };
    auto bucket = [&](uint32_t b) -> int { return bucket_of(__ldg(bstart + b), __ldg(bend + b)); };
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    // the units' buckets, computed once and kept in shared memory when they
    // fit; each thread issues the loads of 16 units before using any
    const bool cached = n_blocks <= kOrderCache;
    constexpr int kPer = 16;
    for (uint32_t base = 0; base < n_blocks; base += kPer * blockDim.x) {
        uint32_t sv[kPer], ev[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t b = base + (uint32_t)q * blockDim.x + threadIdx.x;
            sv[q] = b < n_blocks ? __ldg(bstart + b) : 0u;
            ev[q] = b < n_blocks ? __ldg(bend + b) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t b = base + (uint32_t)q * blockDim.x + threadIdx.x;
            if (b < n_blocks) {
                const int k = bucket_of(sv[q], ev[q]);
                if (cached) s_bucket[b] = (uint8_t)k;
                atomicAdd(&s_hist[k], 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < kOrderBuckets; ++i) {
            s_pos[i] = run;
            run += s_hist[i];
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < n_blocks; b += blockDim.x)
        order[atomicAdd(&s_pos[cached ? (int)s_bucket[b] : bucket(b)], 1u)] = b;
}

void launch_block_order(const uint32_t* bstart, const uint32_t* bend, uint32_t n_blocks, uint32_t* order,
                        cudaStream_t s) {
    launch_pdl(block_order_kernel, dim3(1), dim3(1024), 0, s, bstart, bend, n_blocks, order);
}

// Cameras in groups for the persistent rasterizer (Sec. 3.1's tiles of many
// views from one queue): the cameras are ranked by their rasterization work,
// least first -- the list length of each unit times the tiles that walk it
// (one for a tile, the image's tiles of a tile block) -- and cut into groups
// of `depth`; the queue takes group after
// group, each with its longest lists first, so the views of an early group
// finish before later groups start (per-view latency) while each group still
// balances its own tiles.  depth 0 (or >= n_cams): one group, the plain
// longest-lists-first order.  One CTA: a counting sort on (group, bucket).
constexpr int kOrderGroups = 64;

__global__ void __launch_bounds__(1024) view_order_kernel(const uint32_t* __restrict__ bstart,
                                                          const uint32_t* __restrict__ bend, uint32_t n_units,
                                                          const CamDev* __restrict__ cams, int n_cams, int blocks,
                                                          int depth, uint32_t* __restrict__ order) {
    __shared__ unsigned long long s_tot[kViewOrderMaxCams];
    __shared__ uint8_t s_group[kViewOrderMaxCams];
    __shared__ uint32_t s_hist[kOrderGroups * kOrderBuckets];
    __shared__ uint32_t s_warp[32];
    pdl_enter();
    const int t = threadIdx.x;
    auto cam_of = [&](uint32_t u) {
        int lo = 0, hi = n_cams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const uint32_t off = blocks ? cams[mid].block_offset : cams[mid].tile_offset;
            if (off <= u) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    auto length = [&](uint32_t u) {
        const uint32_t s = __ldg(bstart + u), e = __ldg(bend + u);
        return s < e ? e - s : 0u;
    };
    auto bucket = [&](uint32_t len) {  // 4 buckets per octave, longest lists in bucket 0
        const uint32_t v = len + 1u;
        const int lg = 31 - __clz(v);
        const int frac = lg >= 2 ? (int)((v >> (lg - 2)) & 3u) : (int)((v << (2 - lg)) & 3u);
        return kOrderBuckets - 1 - min(kOrderBuckets - 1, lg * 4 + frac);
    };
    // tiles that walk unit u's list
    auto walkers = [&](uint32_t u, int c) -> uint32_t {
        if (!blocks) return 1u;
        const CamDev& C = cams[c];
        const uint32_t lb = u - C.block_offset;
        const int bx = (int)(lb % (uint32_t)C.blocks_x) * kBlockW, by = (int)(lb / (uint32_t)C.blocks_x) * kBlockH;
        return (uint32_t)(min(kBlockW, C.tiles_x - bx) * min(kBlockH, C.tiles_y - by));
    };
    for (int i = t; i < n_cams; i += blockDim.x) s_tot[i] = 0;
    for (int i = t; i < kOrderGroups * kOrderBuckets; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (uint32_t u = t; u < n_units; u += blockDim.x) {
        const int c = cam_of(u);
        atomicAdd(&s_tot[c], (unsigned long long)length(u) * walkers(u, c));
    }
    __syncthreads();
    // rank by total (ties to the lower index), then the group of the rank
    const int d = (depth <= 0 || depth >= n_cams) ? n_cams : max(depth, (n_cams + kOrderGroups - 1) / kOrderGroups);
    for (int c = t; c < n_cams; c += blockDim.x) {
        const unsigned long long mine = s_tot[c];
        int rank = 0;
        for (int o = 0; o < n_cams; ++o) rank += (s_tot[o] < mine || (s_tot[o] == mine && o < c)) ? 1 : 0;
        s_group[c] = (uint8_t)(rank / d);
    }
    __syncthreads();
    for (uint32_t u = t; u < n_units; u += blockDim.x)
        atomicAdd(&s_hist[s_group[cam_of(u)] * kOrderBuckets + bucket(length(u))], 1u);
    __syncthreads();
    // exclusive scan of the histogram: four entries per thread
    constexpr int kPer = kOrderGroups * kOrderBuckets / 1024;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        v[i] = s_hist[t * kPer + i];
        sum += v[i];
    }
    const int lane = t & 31, w = t >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t x = s_warp[lane], xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        s_warp[lane] = xi - x;
    }
    __syncthreads();
    uint32_t run = s_warp[w] + incl - sum;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        s_hist[t * kPer + i] = run;
        run += v[i];
    }
    __syncthreads();
    for (uint32_t u = t; u < n_units; u += blockDim.x)
        order[atomicAdd(&s_hist[s_group[cam_of(u)] * kOrderBuckets + bucket(length(u))], 1u)] = u;
}

void launch_view_order(const uint32_t* bstart, const uint32_t* bend, uint32_t n_units, const CamDev* cams, int n_cams,
                       bool blocks, int depth, uint32_t* order, cudaStream_t s) {
    launch_pdl(view_order_kernel, dim3(1), dim3(1024), 0, s, bstart, bend, n_units, cams, n_cams, blocks ? 1 : 0,
               depth, order);
}

template <typename KeyT>
void launch_emit_blocks(const uint32_t* order, const uint32_t* offsets, const float4* rec,
                        const CamDev* cams, int n_gauss, int tile_w, int tile_h, int ellipse, DeviceStatus* st,
                        KeyT* inst_block, uint32_t* inst_rec, uint32_t* inst_mask, int blocks, cudaStream_t s) {
    launch_pdl(emit_blocks_kernel<KeyT>, dim3(blocks), dim3(256), 0, s, order, offsets, rec, cams, n_gauss, tile_w,
               tile_h, ellipse, st, inst_block, inst_rec, inst_mask);
}

template void launch_emit_blocks<uint16_t>(const uint32_t*, const uint32_t*, const float4*,
                                           const CamDev*, int, int, int, int, DeviceStatus*, uint16_t*, uint32_t*,
                                           uint32_t*, int, cudaStream_t);
template void launch_emit_blocks<uint32_t>(const uint32_t*, const uint32_t*, const float4*,
                                           const CamDev*, int, int, int, int, DeviceStatus*, uint32_t*, uint32_t*,
                                           uint32_t*, int, cudaStream_t);

}  // namespace seele
