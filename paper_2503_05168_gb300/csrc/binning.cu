// binning.cu -- tile instances (Sec. 3.1: "the preprocessing stage ...
// identifies the intersection between Gaussians and rendering tiles") and
// per-tile ranges into the sorted instance list.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "blocks.cuh"
#include "tiletest.cuh"

namespace seele {

// A warp takes 32 consecutive visible records in depth order and writes all
// their (global tile, record) instances as one contiguous, coalesced run.
// The records' tile rows are expanded 32 at a time (lane -> (record, row) by a
// binary search over the exclusive row counts); each row lane finds its span
// of tiles with the ellipse test of tiletest.cuh (or takes the whole rect row),
// and the warp then writes the rows' tiles cooperatively: lane l writes
// outputs l, l + 32, ... and finds its row by a second binary search.
// Emission in depth order means the later stable sort by tile leaves each
// tile's list front to back; within one record tiles go row-major.  Every
// write stays inside the warp's run [offsets[wb], offsets[wb + 32]); a span
// sum that disagrees with the preprocessing count is reported as kErrInternal.
__device__ __forceinline__ int warp_search(uint32_t excl, uint32_t o) {
    // largest lane s with excl_s <= o (excl non-decreasing over the lanes)
    int s = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint32_t e = __shfl_sync(0xffffffffu, excl, s + step);
        if (e <= o) s += step;
    }
    return s;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename KeyT>
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offsets,
                                                   const float4* __restrict__ rec,
                                                   const CamDev* __restrict__ cams, int n_gauss, int tile_w,
                                                   int tile_h, int ellipse, DeviceStatus* st,
                                                   KeyT* __restrict__ inst_tile, uint32_t* __restrict__ inst_rec) {
    pdl_enter();
    if (st->error != kOk) return;  // capacity overflow: nothing fits, outputs undefined
    const uint32_t n = st->n_visible;
    const uint32_t n_inst = st->n_instances;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wb = warp * 32; wb < n; wb += nwarps * 32) {
        const uint32_t j = wb + lane;
        uint32_t r = 0, x0 = 0, x1 = 0, y0 = 0, rows = 0, row0 = 0, tx_n = 0;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (j < n) {
            r = __ldg(order + j);
            const uint2 b = rec_tile_box(rec, r);
            x0 = b.x & 0xffffu;
            y0 = b.x >> 16;
            x1 = b.y & 0xffffu;
            rows = (b.y >> 16) - y0 + 1;
            const CamDev& C = cams[r < (uint32_t)n_gauss ? 0u : r / (uint32_t)n_gauss];
            tx_n = (uint32_t)C.tiles_x;
            row0 = C.tile_offset;
            if (ellipse) {
                r0 = __ldg(rec + (size_t)kRecF4 * r);
                r1 = __ldg(rec + (size_t)kRecF4 * r + 1);
            }
        }
        const uint32_t rincl = warp_incl_scan(rows, lane);
        const uint32_t rexcl = rincl - rows;
        const uint32_t rtotal = __shfl_sync(0xffffffffu, rincl, 31);
        const uint32_t base = __shfl_sync(0xffffffffu, j < n ? __ldg(offsets + j) : 0u, 0);
        const uint32_t end = wb + 32 < n ? __ldg(offsets + wb + 32) : n_inst;
        uint32_t pos = base;
        // warp-uniform trip counts: every shuffle below has all 32 lanes present
        for (uint32_t c0 = 0; c0 < rtotal; c0 += 32) {
            const uint32_t ro = c0 + lane;
            const int s = warp_search(rexcl, ro);
            const uint32_t rs = __shfl_sync(0xffffffffu, r, s);
            const uint32_t es = __shfl_sync(0xffffffffu, rexcl, s);
            const int xs0 = (int)__shfl_sync(0xffffffffu, x0, s);
            const int xs1 = (int)__shfl_sync(0xffffffffu, x1, s);
            const uint32_t ys0 = __shfl_sync(0xffffffffu, y0, s);
            const uint32_t ns = __shfl_sync(0xffffffffu, tx_n, s);
            const uint32_t os = __shfl_sync(0xffffffffu, row0, s);
            float4 q0, q1;
            q0.x = __shfl_sync(0xffffffffu, r0.x, s);
            q0.y = __shfl_sync(0xffffffffu, r0.y, s);
            q0.z = __shfl_sync(0xffffffffu, r0.z, s);
            q0.w = __shfl_sync(0xffffffffu, r0.w, s);
            q1.x = __shfl_sync(0xffffffffu, r1.x, s);
            q1.w = __shfl_sync(0xffffffffu, r1.w, s);
            q1.y = q1.z = 0.f;
            int lo = 0, hi = -1;
            uint32_t ty = 0;
            if (ro < rtotal) {
                ty = ys0 + (ro - es);
                if (ellipse) {
                    const Ellipse E = make_ellipse(q0, q1);
                    row_span(E, (int)ty, tile_w, tile_h, xs0, xs1, &lo, &hi);
                } else {
                    lo = xs0;
                    hi = xs1;
                }
            }
            const uint32_t cnt = hi >= lo ? (uint32_t)(hi - lo + 1) : 0u;
            const uint32_t cincl = warp_incl_scan(cnt, lane);
            const uint32_t cexcl = cincl - cnt;
            const uint32_t ctotal = __shfl_sync(0xffffffffu, cincl, 31);
            const uint32_t first = os + ty * ns + (uint32_t)lo;  // global id of the row's first kept tile
            for (uint32_t o0 = 0; o0 < ctotal; o0 += 32) {
                const uint32_t o = o0 + lane;
                const int t = warp_search(cexcl, o);
                const uint32_t et = __shfl_sync(0xffffffffu, cexcl, t);
                const uint32_t ft = __shfl_sync(0xffffffffu, first, t);
                const uint32_t rt = __shfl_sync(0xffffffffu, rs, t);
                const uint32_t p = pos + o;
                if (o < ctotal && p < end) {
                    inst_tile[p] = (KeyT)(ft + (o - et));
                    inst_rec[p] = rt;
                }
            }
            pos += ctotal;
        }
        if (pos != end) {
            // never expected: both counts come from the same row_span on the
            // same stored floats.  Report it and keep every slot a valid
            // (tile, record) pair so that the sort and the rasterizer stay in
            // bounds.
            if (lane == 0) record_error(st, kErrInternal, 7);
            const uint32_t t0 = __shfl_sync(0xffffffffu, row0, 0), rr0 = __shfl_sync(0xffffffffu, r, 0);
            for (uint32_t p = pos + lane; p < end; p += 32) {
                inst_tile[p] = (KeyT)t0;
                inst_rec[p] = rr0;
            }
        }
    }
}

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

// After the block sort: the OR of the tile masks of every 32 consecutive
// entries (aligned to the list array), so a tile's rasterizer can skip 32
// entries of its block list with one load when none of them reaches it.
__global__ void mask_summary_kernel(const uint32_t* __restrict__ mask, const DeviceStatus* __restrict__ st,
                                    uint32_t* __restrict__ summary, uint32_t max_groups) {
    pdl_enter();
    const uint32_t n = st->error == kOk ? st->n_inst_valid : 0u;
    const uint32_t groups = (n + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < groups && g < max_groups;
         g += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t j = 32 * g + lane;
        const uint32_t m = j < n ? __ldg(mask + j) : 0u;
        const uint32_t o = __reduce_or_sync(0xffffffffu, m);
        if (lane == 0) summary[g] = o;
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

__global__ void __launch_bounds__(1024) block_order_kernel(const uint32_t* __restrict__ bstart,
                                                           const uint32_t* __restrict__ bend, uint32_t n_blocks,
                                                           uint32_t* __restrict__ order) {
    __shared__ uint32_t s_hist[kOrderBuckets];
    __shared__ uint32_t s_pos[kOrderBuckets];
    pdl_enter();
    auto bucket = [&](uint32_t b) -> int {
        const uint32_t s = __ldg(bstart + b), e = __ldg(bend + b);
        const uint32_t len = s < e ? e - s : 0u;
        // 4 buckets per octave, longest lists in bucket 0
        const uint32_t v = len + 1u;
        const int lg = 31 - __clz(v);
        const int frac = lg >= 2 ? (int)((v >> (lg - 2)) & 3u) : (int)((v << (2 - lg)) & 3u);
        return kOrderBuckets - 1 - min(kOrderBuckets - 1, lg * 4 + frac);
    };
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < n_blocks; b += blockDim.x) atomicAdd(&s_hist[bucket(b)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < kOrderBuckets; ++i) {
            s_pos[i] = run;
            run += s_hist[i];
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < n_blocks; b += blockDim.x) order[atomicAdd(&s_pos[bucket(b)], 1u)] = b;
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
void launch_emit(const uint32_t* order, const uint32_t* offsets, const float4* rec,
                 const CamDev* cams, int n_gauss, int tile_w, int tile_h, int ellipse, DeviceStatus* st,
                 KeyT* inst_tile, uint32_t* inst_rec, int blocks, cudaStream_t s) {
    launch_pdl(emit_kernel<KeyT>, dim3(blocks), dim3(256), 0, s, order, offsets, rec, cams, n_gauss, tile_w, tile_h,
               ellipse, st, inst_tile, inst_rec);
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
template void launch_emit<uint16_t>(const uint32_t*, const uint32_t*, const float4*, const CamDev*,
                                    int, int, int, int, DeviceStatus*, uint16_t*, uint32_t*, int, cudaStream_t);
template void launch_emit<uint32_t>(const uint32_t*, const uint32_t*, const float4*, const CamDev*,
                                    int, int, int, int, DeviceStatus*, uint32_t*, uint32_t*, int, cudaStream_t);

}  // namespace seele
