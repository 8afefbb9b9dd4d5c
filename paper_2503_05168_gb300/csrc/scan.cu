// scan.cu -- single-pass prefix scans with decoupled look-back.
//
//  compact_visible: ordered stream compaction of the visible records (tiles
//                   touched > 0) into (depth bits, record id) pairs -- the input
//                   of the depth sort, in record-id order so that the stable
//                   sort breaks depth ties by id.  Preprocessing has counted
//                   the visible records of each 4096-record chunk, so a CTA
//                   adds up its predecessors' counts directly.
//  scan_tiles:      exclusive scan of the instance counts in depth order,
//                   giving each visible record the start of its instances and
//                   K; the depth sort's last pass has laid the counts out in
//                   depth order; chunk sums first, then each CTA adds up its
//                   predecessors' sums directly.
//  digit_scan:      exclusive scan of a radix sort's digit-major count matrix
//                   from its row totals, without look-back.
//  exclusive_scan:  generic single-pass scan with decoupled look-back: each
//                   block takes a dynamic ticket (so every predecessor has
//                   already started and will publish), reduces its tile,
//                   publishes the aggregate and walks back over its
//                   predecessors one warp-width at a time.  Every wait is
//                   bounded.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace seele {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kChunkItems, "scan tiles are the counting chunks");

// Exclusive prefix of `aggregate` over the preceding tiles (all threads call).
// A predecessor is polled at most spin_limit times; then the wait records a
// timeout and takes that predecessor as an inclusive zero.  publish = false
// (a test hook) makes this tile keep its sums to itself, so that its
// successor's wait runs out.
__device__ uint32_t lookback_prefix(uint64_t* status, uint32_t tile, uint32_t aggregate, uint32_t epoch,
                                    DeviceStatus* st, uint32_t site, uint32_t spin_limit, bool publish) {
    __shared__ uint32_t s_prefix;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0 && publish)
            st_release_u64(status + tile, pack_status(epoch, tile == 0 ? kFlagInclusive : kFlagAggregate, aggregate));
        uint32_t prefix = 0;
        int64_t window = (int64_t)tile - 1;
        while (window >= 0) {
            const int64_t idx = window - lane;
            uint32_t flag = kFlagInclusive, value = 0;
            if (idx >= 0) {
                uint32_t spins = 0;
                uint64_t s;
                do {
                    s = ld_acquire_u64(status + idx);
                    flag = status_flag(s, epoch);
                } while (flag == 0 && ++spins < spin_limit);
                if (flag == 0) {
                    record_error(st, kErrTimeout, site);
                    flag = kFlagInclusive;
                    s = 0;
                }
                value = (uint32_t)s;
            }
            const uint32_t incl = __ballot_sync(0xffffffffu, flag == kFlagInclusive);
            const int stop = incl ? __ffs(incl) - 1 : 31;
            uint32_t v = lane <= stop ? value : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            prefix += v;
            if (incl) break;
            window -= 32;
        }
        if (lane == 0) {
            if (tile > 0 && publish) st_release_u64(status + tile, pack_status(epoch, kFlagInclusive, prefix + aggregate));
            s_prefix = prefix;
        }
    }
    __syncthreads();
    return s_prefix;
}

// Block-wide exclusive scan of one value per thread; also returns the total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* total) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = t;
    }
    __syncthreads();
    const uint32_t warp_excl = w > 0 ? s_warp[w - 1] : 0u;
    *total = s_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_excl + incl - x;
}

__device__ __forceinline__ uint32_t take_ticket(uint32_t* counter) {
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    return s_tile;
}

// Sum of counts[0, c) by the whole block (every thread gets it).  Chunk
// counts are few (one per 4096 items), so each CTA adds up its predecessors
// directly instead of waiting on them.
__device__ __forceinline__ uint32_t chunk_prefix(const uint32_t* __restrict__ counts, uint32_t c) {
    __shared__ uint32_t s_part[kScanThreads / 32];
    uint32_t v = 0;
    for (uint32_t i = threadIdx.x; i < c; i += kScanThreads) v += __ldg(counts + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) total += s_part[w];
    __syncthreads();
    return total;
}

// Exclusive offsets of the block's warps from their totals (every thread).
__device__ __forceinline__ uint32_t warp_offset(uint32_t warp_total, uint32_t* block_total) {
    __shared__ uint32_t s_w[kScanThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) s_w[w] = warp_total;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int ww = 0; ww < kScanThreads / 32; ++ww) {
        const uint32_t v = s_w[ww];
        before += ww < w ? v : 0u;
        all += v;
    }
    *block_total = all;
    return before;
}

// Ordered compaction of chunk c: items are warp-striped (item k of lane l of
// warp w is c * 4096 + w * 512 + 32 k + l), ranked by one ballot per k, and
// placed after the visible records of all earlier chunks.  A record is
// visible when its instance count cnt[i] is not zero; with pack, each value
// carries min(cnt[i], 255) in its top 8 bits (record ids < 2^24).
__global__ void __launch_bounds__(kScanThreads) compact_visible_kernel(const uint32_t* __restrict__ cnt, int pack,
                                                                       const float* __restrict__ depth, uint32_t R,
                                                                       const uint32_t* __restrict__ chunk_vis,
                                                                       uint32_t* keys, uint32_t* vals,
                                                                       DeviceStatus* st) {
    pdl_enter();
    const uint32_t c = blockIdx.x;
    const uint32_t nchunks = (R + kChunkItems - 1) / kChunkItems;
    const uint32_t prefix = chunk_prefix(chunk_vis, c);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wbase = c * kChunkItems + (uint32_t)w * 32 * kScanItems;
    uint32_t bal[kScanItems], cv[kScanItems], wtot = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = wbase + 32 * k + lane;
        cv[k] = i < R ? __ldg(cnt + i) : 0u;
        bal[k] = __ballot_sync(0xffffffffu, cv[k] > 0u);
        wtot += __popc(bal[k]);
    }
    uint32_t total;
    uint32_t pos = prefix + warp_offset(wtot, &total);
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = wbase + 32 * k + lane;
        if ((bal[k] >> lane) & 1u) {
            const uint32_t o = pos + __popc(bal[k] & lt);
            keys[o] = __float_as_uint(__ldg(depth + i));
            vals[o] = pack ? (i | (min(cv[k], kPackedCountMax) << kPackedIdBits)) : i;
        }
        pos += __popc(bal[k]);
    }
    if (c == nchunks - 1 && threadIdx.x == 0) st->n_visible = prefix + total;
}

// Per chunk of 4096 depth-ordered records: the sum of their counts.
__global__ void __launch_bounds__(kScanThreads) chunk_sums_kernel(const uint32_t* __restrict__ cnt,
                                                                  const DeviceStatus* __restrict__ st,
                                                                  uint32_t* __restrict__ chunk_sum) {
    __shared__ uint32_t s_part[kScanThreads / 32];
    pdl_enter();
    const uint32_t n = st->n_visible;
    const uint32_t base = blockIdx.x * kChunkItems;
    if (base >= n) return;
    uint32_t v = 0;
    if (base + kChunkItems <= n) {
        const uint4* p4 = reinterpret_cast<const uint4*>(cnt + base) + threadIdx.x;
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 x = __ldg(p4 + q * kScanThreads);
            v += x.x + x.y + x.z + x.w;
        }
    } else {
        for (uint32_t j = base + threadIdx.x; j < n; j += kScanThreads) v += __ldg(cnt + j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_part[w];
        chunk_sum[blockIdx.x] = t;
    }
}

// Exclusive scan of the counts of the depth-ordered records (their instance
// offsets), chunk by chunk after the sums of the earlier chunks; the last
// chunk sets K and compares it with the capacity.
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const uint32_t* __restrict__ cnt,
                                                                  const uint32_t* __restrict__ chunk_sum,
                                                                  uint32_t* offsets, DeviceStatus* st,
                                                                  uint32_t capacity) {
    pdl_enter();
    const uint32_t n = st->n_visible;
    const uint32_t nchunks = (n + kChunkItems - 1) / kChunkItems;
    const uint32_t c = blockIdx.x;
    if (c >= nchunks) {
        if (n == 0 && c == 0 && threadIdx.x == 0) {
            st->n_instances = 0;
            st->capacity = capacity;
        }
        return;
    }
    const uint32_t prefix = chunk_prefix(chunk_sum, c);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wbase = c * kChunkItems + (uint32_t)w * 32 * kScanItems;
    uint32_t v[kScanItems], wtot = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t j = wbase + 32 * k + lane;
        v[k] = j < n ? __ldg(cnt + j) : 0u;
        wtot += v[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wtot += __shfl_xor_sync(0xffffffffu, wtot, o);
    uint32_t total;
    uint32_t pos = prefix + warp_offset(wtot, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        uint32_t incl = v[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t j = wbase + 32 * k + lane;
        if (j < n) offsets[j] = pos + incl - v[k];
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (c == nchunks - 1 && threadIdx.x == 0) {
        const uint32_t K = prefix + total;
        st->n_instances = K;
        st->capacity = capacity;
        if (K > capacity) record_error(st, kErrCapacity, 3);
        else st->n_inst_valid = K;
    }
}

// Exclusive scan of the row-major count matrix in[d * stride + t] (rows of
// stride: a radix pass's 256 digits, or the tile blocks of tile binning with
// their 32 tiles each) given its row totals: the elements before scan tile s
// are the whole rows d < d0 and the first t0 entries of row d0, so each
// block adds those up itself and no block waits on another.
__global__ void __launch_bounds__(kScanThreads) digit_scan_kernel(const uint32_t* __restrict__ in, uint32_t stride,
                                                                  uint32_t rows,
                                                                  const uint32_t* __restrict__ row_total,
                                                                  uint32_t* __restrict__ out,
                                                                  const uint32_t* __restrict__ count_ptr,
                                                                  uint32_t col_items) {
    __shared__ uint32_t s_part[kScanThreads / 32];
    pdl_enter();
    // a dense matrix: one column per col_items of the device count
    if (count_ptr != nullptr) stride = max((*count_ptr + col_items - 1u) / col_items, 1u);
    const uint32_t n = rows * stride;
    const uint32_t first = blockIdx.x * kScanTile;
    if (first >= n) return;
    const uint32_t base = first + threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    if (base + kScanItems <= n) {
        const uint4* p4 = reinterpret_cast<const uint4*>(in + base);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 v = __ldg(p4 + q);
            c[4 * q] = v.x;
            c[4 * q + 1] = v.y;
            c[4 * q + 2] = v.z;
            c[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) c[k] = base + k < n ? __ldg(in + base + k) : 0u;
    }
    const uint32_t d0 = first / stride, t0 = first - d0 * stride;
    uint32_t part = 0;
    for (uint32_t d = threadIdx.x; d < d0; d += kScanThreads) part += __ldg(row_total + d);
    const uint32_t* row = in + (size_t)d0 * stride;
    for (uint32_t t = threadIdx.x; t < t0; t += kScanThreads) part += __ldg(row + t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    uint32_t prefix = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) prefix += s_part[w];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += c[k];
    uint32_t total;
    uint32_t pos = prefix + block_exclusive_scan(sum, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pos;
        pos += c[k];
    }
}

// Exclusive scan of n uint32 values (n known on the host).
__global__ void __launch_bounds__(kScanThreads) exclusive_scan_kernel(const uint32_t* __restrict__ in, uint32_t n,
                                                                      uint32_t* __restrict__ out, uint64_t* status,
                                                                      uint32_t epoch, DeviceStatus* st, int ticket,
                                                                      uint32_t spin_limit, uint32_t withhold) {
    const uint32_t tile = take_ticket(&st->ticket[ticket]);
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (tile >= ntiles) return;
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    uint32_t sum = 0;
    if (base + kScanItems <= n) {
        const uint4* p4 = reinterpret_cast<const uint4*>(in + base);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 v = __ldg(p4 + q);
            c[4 * q] = v.x;
            c[4 * q + 1] = v.y;
            c[4 * q + 2] = v.z;
            c[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) c[k] = base + k < n ? __ldg(in + base + k) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += c[k];
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(sum, &total);
    const uint32_t prefix = lookback_prefix(status, tile, total, epoch, st, 4, spin_limit, tile != withhold);
    uint32_t pos = prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pos;
        pos += c[k];
    }
}

void launch_digit_scan(const uint32_t* in, uint32_t stride, const uint32_t* row_total, uint32_t* out,
                       cudaStream_t s, uint32_t rows, const uint32_t* count_ptr, uint32_t col_items) {
    const uint32_t blocks = std::max<uint32_t>((rows * stride + kScanTile - 1) / kScanTile, 1u);
    launch_pdl(digit_scan_kernel, dim3(blocks), dim3(kScanThreads), 0, s, in, stride, rows, row_total, out,
               count_ptr, count_ptr ? col_items : 1u);
}

void launch_exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint64_t* status, uint32_t epoch,
                           DeviceStatus* st, int ticket, cudaStream_t s, uint32_t spin_limit, uint32_t withhold) {
    const uint32_t blocks = (n + kScanTile - 1) / kScanTile;
    exclusive_scan_kernel<<<blocks > 0 ? blocks : 1, kScanThreads, 0, s>>>(in, n, out, status, epoch, st, ticket,
                                                                            spin_limit ? spin_limit : kSpinLimit,
                                                                            withhold);
}

uint32_t exclusive_scan_blocks(uint32_t n) { return std::max<uint32_t>((n + kScanTile - 1) / kScanTile, 1u); }

uint32_t scan_tiles_per_launch() { return kScanTile; }

void launch_compact_visible(const uint32_t* cnt, bool pack, const float* depth, uint32_t R,
                            const uint32_t* chunk_vis, uint32_t* keys, uint32_t* vals, DeviceStatus* st,
                            cudaStream_t s) {
    const uint32_t blocks = (R + kChunkItems - 1) / kChunkItems;
    launch_pdl(compact_visible_kernel, dim3(blocks > 0 ? blocks : 1), dim3(kScanThreads), 0, s, cnt, pack ? 1 : 0,
               depth, R, chunk_vis, keys, vals, st);
}

void launch_scan_tiles(const uint32_t* cnt_sorted, uint32_t* chunk_sum, uint32_t max_n, uint32_t* offsets,
                       DeviceStatus* st, uint32_t capacity, cudaStream_t s) {
    const uint32_t blocks = std::max<uint32_t>((max_n + kChunkItems - 1) / kChunkItems, 1u);
    launch_pdl(chunk_sums_kernel, dim3(blocks), dim3(kScanThreads), 0, s, cnt_sorted, st, chunk_sum);
    launch_pdl(scan_tiles_kernel, dim3(blocks), dim3(kScanThreads), 0, s, cnt_sorted, chunk_sum, offsets, st,
               capacity);
}

}  // namespace seele
