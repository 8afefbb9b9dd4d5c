// scan.cu -- single-pass prefix scans with decoupled look-back.
//
//  compact_visible: ordered stream compaction of the visible records (tiles
//                   touched > 0) into (depth bits, record id) pairs -- the input
//                   of the depth sort, in record-id order so that the stable
//                   sort breaks depth ties by id.
//  scan_tiles:      exclusive scan of tiles touched in depth order, giving each
//                   visible record the start of its tile instances and K.
//
// Each block takes a dynamic ticket (so every predecessor has already started
// and will publish), reduces its tile, publishes the aggregate and walks back
// over its predecessors one warp-width at a time.  Every wait is bounded.
#include "common.cuh"
#include "kernels.h"

namespace seele {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive prefix of `aggregate` over the preceding tiles (all threads call).
__device__ uint32_t lookback_prefix(uint64_t* status, uint32_t tile, uint32_t aggregate, uint32_t epoch,
                                    DeviceStatus* st, uint32_t site) {
    __shared__ uint32_t s_prefix;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) st_release_u64(status + tile, pack_status(epoch, tile == 0 ? kFlagInclusive : kFlagAggregate, aggregate));
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
                } while (flag == 0 && ++spins < kSpinLimit);
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
            if (tile > 0) st_release_u64(status + tile, pack_status(epoch, kFlagInclusive, prefix + aggregate));
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

__global__ void __launch_bounds__(kScanThreads) compact_visible_kernel(const uint32_t* __restrict__ tiles,
                                                                       const float* __restrict__ depth, uint32_t R,
                                                                       uint32_t* keys, uint32_t* vals,
                                                                       uint64_t* status, uint32_t epoch,
                                                                       DeviceStatus* st, int ticket) {
    const uint32_t tile = take_ticket(&st->ticket[ticket]);
    const uint32_t ntiles = (R + kScanTile - 1) / kScanTile;
    if (tile >= ntiles) return;
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = base + k;
        const bool vis = i < R && __ldg(tiles + i) > 0u;
        flags |= (uint32_t)vis << k;
        cnt += vis;
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(cnt, &total);
    const uint32_t prefix = lookback_prefix(status, tile, total, epoch, st, 1);
    uint32_t pos = prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (flags >> k & 1u) {
            keys[pos] = __float_as_uint(__ldg(depth + base + k));
            vals[pos] = base + k;
            ++pos;
        }
    if (tile == ntiles - 1 && threadIdx.x == 0) st->n_visible = prefix + total;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const uint32_t* __restrict__ tiles,
                                                                  const uint32_t* __restrict__ order,
                                                                  uint32_t* offsets, uint64_t* status, uint32_t epoch,
                                                                  DeviceStatus* st, int ticket, uint32_t capacity) {
    const uint32_t tile = take_ticket(&st->ticket[ticket]);
    const uint32_t n = st->n_visible;
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (tile >= ntiles) {
        if (n == 0 && tile == 0 && threadIdx.x == 0) st->n_instances = 0;
        return;
    }
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t j = base + k;
        c[k] = j < n ? __ldg(tiles + __ldg(order + j)) : 0u;
        sum += c[k];
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(sum, &total);
    const uint32_t prefix = lookback_prefix(status, tile, total, epoch, st, 2);
    uint32_t pos = prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) offsets[base + k] = pos;
        pos += c[k];
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) {
        const uint32_t K = prefix + total;
        st->n_instances = K;
        st->capacity = capacity;
        if (K > capacity) record_error(st, kErrCapacity, 3);
        else st->n_inst_valid = K;
    }
}

// Exclusive scan of n uint32 values (n known on the host).
__global__ void __launch_bounds__(kScanThreads) exclusive_scan_kernel(const uint32_t* __restrict__ in, uint32_t n,
                                                                      uint32_t* __restrict__ out, uint64_t* status,
                                                                      uint32_t epoch, DeviceStatus* st, int ticket) {
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
    const uint32_t prefix = lookback_prefix(status, tile, total, epoch, st, 4);
    uint32_t pos = prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pos;
        pos += c[k];
    }
}

void launch_exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint64_t* status, uint32_t epoch,
                           DeviceStatus* st, int ticket, cudaStream_t s) {
    const uint32_t blocks = (n + kScanTile - 1) / kScanTile;
    exclusive_scan_kernel<<<blocks > 0 ? blocks : 1, kScanThreads, 0, s>>>(in, n, out, status, epoch, st, ticket);
}

uint32_t scan_tiles_per_launch() { return kScanTile; }

void launch_compact_visible(const uint32_t* tiles, const float* depth, uint32_t R, uint32_t* keys, uint32_t* vals,
                            uint64_t* status, uint32_t epoch, DeviceStatus* st, int ticket, cudaStream_t s) {
    const uint32_t blocks = (R + kScanTile - 1) / kScanTile;
    compact_visible_kernel<<<blocks > 0 ? blocks : 1, kScanThreads, 0, s>>>(tiles, depth, R, keys, vals, status,
                                                                            epoch, st, ticket);
}

void launch_scan_tiles(const uint32_t* tiles, const uint32_t* order, uint32_t max_n, uint32_t* offsets,
                       uint64_t* status, uint32_t epoch, DeviceStatus* st, int ticket, uint32_t capacity,
                       cudaStream_t s) {
    const uint32_t blocks = (max_n + kScanTile - 1) / kScanTile;
    scan_tiles_kernel<<<blocks > 0 ? blocks : 1, kScanThreads, 0, s>>>(tiles, order, offsets, status, epoch, st,
                                                                       ticket, capacity);
}

}  // namespace seele
