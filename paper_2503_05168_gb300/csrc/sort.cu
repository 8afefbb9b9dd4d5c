// sort.cu -- stable least-significant-digit radix sort of (uint32 key,
// uint32 value) pairs, one kernel per 8-bit digit ("onesweep": per-tile
// ranking, per-digit decoupled look-back, shared-memory staged scatter).
//
// Used twice per frame: on the visible records keyed by fp32 depth bits (31
// significant bits, 4 passes) and on the tile instances keyed by global tile
// id (ceil(bits / 8) passes).  Stability is what makes the composition give
// the (tile, depth, record id) order of Sec. 3.1 "Sorting".
//
// The element count lives on the device (it is produced by the previous
// kernel), so the grid is sized for the capacity and surplus blocks exit.
#include "common.cuh"
#include "kernels.h"

namespace seele {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kRadix = 256;
constexpr int kWarps = kSortThreads / 32;

// Histograms of every pass at once (the digit multiset of a pass does not
// depend on the order the previous passes leave behind).
__global__ void __launch_bounds__(kSortThreads) radix_histogram_kernel(const uint32_t* __restrict__ keys,
                                                                       const uint32_t* __restrict__ count_ptr,
                                                                       int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_hist[4][kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += kSortThreads) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n = *count_ptr;
    for (uint32_t i = blockIdx.x * kSortThreads + threadIdx.x; i < n; i += gridDim.x * kSortThreads) {
        const uint32_t k = __ldg(keys + i);
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) {
        const uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(hist + i, v);
    }
}

__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(const uint32_t* __restrict__ keys_in,
                                                                const uint32_t* __restrict__ vals_in,
                                                                uint32_t* __restrict__ keys_out,
                                                                uint32_t* __restrict__ vals_out,
                                                                const uint32_t* __restrict__ count_ptr, int shift,
                                                                const uint32_t* __restrict__ hist, uint64_t* status,
                                                                uint32_t epoch, DeviceStatus* st, int ticket) {
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_wcount[kWarps][kRadix + 1];  // per-warp digit counters, then exclusive prefixes
    __shared__ uint32_t s_local_base[kRadix];          // digit start inside this tile
    __shared__ uint32_t s_global_base[kRadix];         // digit start in the output for this tile
    __shared__ uint32_t s_tile;

    if (threadIdx.x == 0) s_tile = atomicAdd(&st->ticket[ticket], 1u);
    for (int i = threadIdx.x; i < kWarps * (kRadix + 1); i += kSortThreads) (&s_wcount[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t n = *count_ptr;
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    if (tile >= ntiles) return;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wbase = tile * kSortTile + w * (32 * kSortItems);
    const uint32_t lt_mask = (1u << lane) - 1u;

    // load warp-striped: item k of lane l is element wbase + 32 k + l, so the
    // order (k, lane) is the input order and ranking in that order is stable
    uint32_t key[kSortItems], val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t i = wbase + 32 * k + lane;
        const bool ok = i < n;
        key[k] = ok ? __ldg(keys_in + i) : 0u;
        val[k] = ok ? __ldg(vals_in + i) : 0u;
        const uint32_t d = ok ? (key[k] >> shift) & 0xffu : (uint32_t)kRadix;  // sentinel bucket
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = s_wcount[w][d];
        __syncwarp();
        if ((peers & lt_mask) == 0u) s_wcount[w][d] = before + __popc(peers);
        __syncwarp();
        rank[k] = before + __popc(peers & lt_mask);
    }
    __syncthreads();

    // per digit: totals over warps, per-warp exclusive offsets, publish + look back
    const uint32_t d = threadIdx.x;  // kSortThreads == kRadix
    uint32_t total = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t c = s_wcount[ww][d];
        s_wcount[ww][d] = total;
        total += c;
    }
    uint64_t* my = status + (size_t)tile * kRadix + d;
    st_release_u64(my, pack_status(epoch, tile == 0 ? kFlagInclusive : kFlagAggregate, total));

    // tile-local digit starts (exclusive scan of totals over digits)
    {
        __shared__ uint32_t s_scan[kSortThreads / 32];
        uint32_t incl = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_scan[w] = incl;
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < w; ++ww) add += s_scan[ww];
        s_local_base[d] = add + incl - total;
    }

    // global digit start: exclusive prefix of the pass histogram
    uint32_t gstart;
    {
        __shared__ uint32_t s_scan2[kSortThreads / 32];
        const uint32_t h = __ldg(hist + d);
        uint32_t incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_scan2[w] = incl;
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < w; ++ww) add += s_scan2[ww];
        gstart = add + incl - h;
    }

    // decoupled look-back over preceding tiles for this digit
    __shared__ int s_gave_up;
    if (threadIdx.x == 0) s_gave_up = 0;
    __syncthreads();
    uint32_t prefix = 0;
    if (tile > 0) {
        int64_t t = (int64_t)tile - 1;
        while (t >= 0) {
            uint32_t spins = 0, flag;
            uint64_t s;
            do {
                s = ld_acquire_u64(status + (size_t)t * kRadix + d);
                flag = status_flag(s, epoch);
            } while (flag == 0 && ++spins < kSpinLimit);
            if (flag == 0) {
                record_error(st, kErrTimeout, 10 + (uint32_t)shift);
                s_gave_up = 1;
                break;
            }
            prefix += (uint32_t)s;
            if (flag == kFlagInclusive) break;
            --t;
        }
        st_release_u64(my, pack_status(epoch, kFlagInclusive, prefix + total));
    }
    s_global_base[d] = gstart + prefix;
    __syncthreads();
    if (s_gave_up) return;  // offsets unknown: write nothing rather than guess

    // stage the tile in shared memory sorted by digit, then write out runs
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t i = wbase + 32 * k + lane;
        if (i < n) {
            const uint32_t dg = (key[k] >> shift) & 0xffu;
            const uint32_t p = s_local_base[dg] + s_wcount[w][dg] + rank[k];
            s_keys[p] = key[k];
            s_vals[p] = val[k];
        }
    }
    __syncthreads();
    const uint32_t tile_n = min((uint32_t)kSortTile, n - tile * kSortTile);
    for (uint32_t i = threadIdx.x; i < tile_n; i += kSortThreads) {
        const uint32_t k = s_keys[i];
        const uint32_t dg = (k >> shift) & 0xffu;
        const uint32_t o = s_global_base[dg] + (i - s_local_base[dg]);
        if (o < n) {
            keys_out[o] = k;
            vals_out[o] = s_vals[i];
        }
    }
}

uint32_t sort_tile_items() { return kSortTile; }

void launch_radix_histogram(const uint32_t* keys, const uint32_t* count_ptr, int passes, uint32_t* hist,
                            int blocks, cudaStream_t s) {
    radix_histogram_kernel<<<blocks, kSortThreads, 0, s>>>(keys, count_ptr, passes, hist);
}

void launch_onesweep(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                     const uint32_t* count_ptr, uint32_t max_n, int shift, const uint32_t* hist, uint64_t* status,
                     uint32_t epoch, DeviceStatus* st, int ticket, cudaStream_t s) {
    const uint32_t blocks = (max_n + kSortTile - 1) / kSortTile;
    onesweep_kernel<<<blocks > 0 ? blocks : 1, kSortThreads, 0, s>>>(keys_in, vals_in, keys_out, vals_out,
                                                                      count_ptr, shift, hist, status, epoch, st,
                                                                      ticket);
}

}  // namespace seele
