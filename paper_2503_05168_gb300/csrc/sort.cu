// sort.cu -- stable least-significant-digit radix sort of (key, uint32 value)
// pairs with 8-bit digits, as reduce-then-scan passes:
//   upsweep:   each tile of 4096 elements counts its digits into a
//              digit-major matrix counts[d * stride + tile];
//   scan:      one device-wide exclusive scan of that matrix gives, for every
//              (digit, tile), where the tile's run of that digit starts (the
//              upsweep also adds up each digit's total, so every scan block
//              finds the sum of the elements before it directly);
//   downsweep: each tile ranks its elements stably (warp match + per-warp
//              counters), stages them in shared memory by digit and writes
//              each digit's run contiguously.
// No block waits on another inside the sort.
// Ranking uses one warp ballot per significant digit bit.  Used twice per
// frame: on the visible records keyed by fp32 depth bits (31 bits, 4 passes)
// and on the tile instances keyed by global tile id (16-bit keys when the
// frame has <= 65536 tiles); the last pass of each writes values only.
// 16-bit keys of 9 or 10 significant bits (257 to 1024 tile blocks) take one
// pass with 9- or 10-bit digits instead of an 8-bit pass and a 1- or 2-bit
// one: the per-warp digit counters are 16-bit then, so the pass's shared
// memory still fits a CTA's static 48 KB.
// Stability is what makes the two sorts compose into the (tile, depth,
// record id) order of Sec. 3.1 "Sorting".  The depth sort's last pass also
// lays out each record's instance count in depth order (SortGather).
//
// Element counts live on the device (they are produced by the previous
// kernel), so grids are sized for the capacity.  In the render path's sorts
// the count matrix is dense in the tiles that hold elements: its stride is
// ceil(n / 4096) for the device count n, which the upsweep, the scan and the
// downsweep each derive from the same word, and surplus tiles return at once
// (no zero counts written or scanned for the unused capacity).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace seele {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kRadix = 256;
constexpr int kWarps = kSortThreads / 32;

// Per-tile digit counts, digit-major.  Counting ignores order, so each thread
// reads 16 consecutive keys with vector loads and adds them to its warp's
// shared counters.  RB: digit width in bits.
// The count matrix's stride: the launch's (grid) stride, or with `dense` the
// number of tiles that hold elements.
__device__ __forceinline__ uint32_t count_stride(uint32_t n, uint32_t stride, int dense) {
    return dense ? max((n + (uint32_t)kSortTile - 1u) / (uint32_t)kSortTile, 1u) : stride;
}

template <typename KeyT, int RB>
__global__ void __launch_bounds__(kSortThreads) upsweep_kernel(const KeyT* __restrict__ keys,
                                                               const uint32_t* __restrict__ count_ptr, int shift,
                                                               uint32_t* __restrict__ counts, uint32_t stride,
                                                               uint32_t* __restrict__ row_total, int dense) {
    static_assert(kSortItems * sizeof(KeyT) % 16 == 0, "vector loads");
    constexpr uint32_t R = 1u << RB;
    static_assert(R % kSortThreads == 0, "whole digits per thread");
    __shared__ uint32_t s_w[kWarps][R];
    pdl_enter();
    const uint32_t tile = blockIdx.x;
    const uint32_t n = *count_ptr;
    stride = count_stride(n, stride, dense);
    if (tile >= stride) return;  // surplus tile of a dense matrix
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * (int)R; i += kSortThreads) (&s_w[0][0])[i] = 0;
    __syncthreads();
    const uint32_t base = tile * kSortTile + threadIdx.x * kSortItems;
    if (base + kSortItems <= n) {
        constexpr int NV = kSortItems * sizeof(KeyT) / 16;
        const uint4* p = reinterpret_cast<const uint4*>(keys + base);
        uint4 v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = __ldg(p + q);
        const KeyT* kk = reinterpret_cast<const KeyT*>(v);
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) atomicAdd(&s_w[w][((uint32_t)kk[k] >> shift) & (R - 1u)], 1u);
    } else {
        for (int k = 0; k < kSortItems; ++k)
            if (base + k < n) atomicAdd(&s_w[w][((uint32_t)__ldg(keys + base + k) >> shift) & (R - 1u)], 1u);
    }
    __syncthreads();
#pragma unroll
    for (uint32_t q = 0; q < R / kSortThreads; ++q) {
        const uint32_t d = threadIdx.x + q * kSortThreads;
        uint32_t total = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) total += s_w[ww][d];
        counts[(size_t)d * stride + tile] = total;
        if (row_total != nullptr && total != 0u) atomicAdd(row_total + d, total);
    }
}

// AUX: a second 32-bit payload travels with each pair; it is staged through
// the same shared buffer as the values after they have been written.
// RB: digit width in bits; thread t owns digits [t DPT, (t + 1) DPT).
template <typename KeyT, bool WRITE_KEYS, bool AUX, int RB>
__global__ void __launch_bounds__(kSortThreads) downsweep_kernel(const KeyT* __restrict__ keys_in,
                                                                 const uint32_t* __restrict__ vals_in,
                                                                 KeyT* __restrict__ keys_out,
                                                                 uint32_t* __restrict__ vals_out,
                                                                 const uint32_t* __restrict__ count_ptr, int shift,
                                                                 int nbits, const uint32_t* __restrict__ offsets,
                                                                 uint32_t stride, uint32_t* __restrict__ run_start,
                                                                 uint32_t* __restrict__ run_end,
                                                                 const uint32_t* __restrict__ aux_in,
                                                                 uint32_t* __restrict__ aux_out,
                                                                 SortGather gather, int dense) {
    constexpr uint32_t R = 1u << RB;
    constexpr int DPT = (int)R / kSortThreads;
    static_assert(DPT >= 1 && (int)R == DPT * kSortThreads, "whole digits per thread");
    static_assert(RB == 8 || sizeof(KeyT) == 2, "wide digits only with 16-bit keys (shared memory)");
    // counts inside a tile are <= 4096: 16-bit counters for the wide digits
    using CntT = typename std::conditional<(RB > 8), uint16_t, uint32_t>::type;
    __shared__ KeyT s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ CntT s_wcount[kWarps][R + 1];  // per-warp digit counters, then exclusive prefixes
    __shared__ CntT s_local_base[R];          // digit start inside this tile
    __shared__ uint32_t s_global_base[R];     // digit start in the output for this tile
    __shared__ uint32_t s_scan[kWarps];

    pdl_enter();
    const uint32_t tile = blockIdx.x;
    const uint32_t n = *count_ptr;
    if (tile * (uint32_t)kSortTile >= n) return;
    stride = count_stride(n, stride, dense);
    const uint32_t t0 = threadIdx.x * DPT;  // this thread's first digit
    for (int i = threadIdx.x; i < kWarps * (int)(R + 1); i += kSortThreads) (&s_wcount[0][0])[i] = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) s_global_base[t0 + q] = __ldg(offsets + (size_t)(t0 + q) * stride + tile);
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t wbase = tile * kSortTile + w * (32 * kSortItems);
    const uint32_t lt_mask = (1u << lane) - 1u;

    // load warp-striped: item k of lane l is element wbase + 32 k + l, so the
    // order (k, lane) is the input order and ranking in that order is stable
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t i = wbase + 32 * k + lane;
        const bool ok = i < n;
        key[k] = ok ? (uint32_t)__ldg(keys_in + i) : 0xffffffffu;
        val[k] = ok ? __ldg(vals_in + i) : 0u;
    }
    // lanes holding the same digit: one ballot per significant digit bit plus
    // one for validity (elements past n form their own group)
    const uint32_t valid_base = __ballot_sync(0xffffffffu, true);
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const bool ok = key[k] != 0xffffffffu;
        const uint32_t dg = ok ? (key[k] >> shift) & (R - 1u) : R;  // sentinel bucket
        const uint32_t okm = __ballot_sync(0xffffffffu, ok);
        uint32_t peers = ok ? okm : (valid_base & ~okm);
        for (int b = 0; b < nbits; ++b) {
            const uint32_t bm = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
            peers &= ((dg >> b) & 1u) ? bm : ~bm;
        }
        const uint32_t before = s_wcount[w][dg];
        __syncwarp();
        if ((peers & lt_mask) == 0u) s_wcount[w][dg] = (CntT)(before + __popc(peers));
        __syncwarp();
        rank[k] = before + __popc(peers & lt_mask);
    }
    __syncthreads();

    // per digit: per-warp exclusive offsets and the tile-local digit start
    uint32_t tot[DPT];
    uint32_t total = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        uint32_t acc = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = s_wcount[ww][t0 + q];
            s_wcount[ww][t0 + q] = (CntT)acc;
            acc += c;
        }
        tot[q] = acc;
        total += acc;
    }
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
    uint32_t lb = add + incl - total;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        s_local_base[t0 + q] = (CntT)lb;
        lb += tot[q];
    }
    __syncthreads();

    // stage the tile in shared memory sorted by digit, then write out runs
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        if (key[k] != 0xffffffffu) {
            const uint32_t dg = (key[k] >> shift) & (R - 1u);
            const uint32_t p = (uint32_t)s_local_base[dg] + s_wcount[w][dg] + rank[k];
            s_keys[p] = (KeyT)key[k];
            s_vals[p] = val[k];
        }
    }
    __syncthreads();
    const uint32_t tile_n = min((uint32_t)kSortTile, n - tile * kSortTile);
    const bool counts = !AUX && gather.src != nullptr;
    const bool packed = counts && gather.packed;
    const uint32_t vmask = packed ? (1u << kPackedIdBits) - 1u : 0xffffffffu;
    for (uint32_t i = threadIdx.x; i < tile_n; i += kSortThreads) {
        const uint32_t k = s_keys[i];
        const uint32_t dg = (k >> shift) & (R - 1u);
        const uint32_t o = s_global_base[dg] + (i - (uint32_t)s_local_base[dg]);
        if (o < n) {
            if (WRITE_KEYS) keys_out[o] = (KeyT)k;
            const uint32_t v = s_vals[i];
            vals_out[o] = v & vmask;
            if (counts) {
                // the record's instance count: carried in the value, or read
                uint32_t c = packed ? v >> kPackedIdBits : kPackedCountMax;
                if (c == kPackedCountMax) c = __ldg(gather.src + (v & vmask));
                gather.out[o] = c;
            }
            // last pass: within a digit run the staged keys are in the lower
            // digits' sorted order, so equal whole keys are adjacent; each
            // block reports where its runs of a key begin and end
            if (run_start != nullptr) {
                if (i == 0 || (uint32_t)s_keys[i - 1] != k) atomicMin(run_start + k, o);
                if (i + 1 == tile_n || (uint32_t)s_keys[i + 1] != k) atomicMax(run_end + k, o + 1);
            }
        }
    }
    if (AUX) {
        // read again here rather than held in registers through the ranking
        uint32_t aux[kSortItems];
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t i = wbase + 32 * k + lane;
            aux[k] = key[k] != 0xffffffffu ? __ldg(aux_in + i) : 0u;
        }
        __syncthreads();  // every value has been read out of s_vals
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            if (key[k] != 0xffffffffu) {
                const uint32_t dg = (key[k] >> shift) & (R - 1u);
                s_vals[(uint32_t)s_local_base[dg] + s_wcount[w][dg] + rank[k]] = aux[k];
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < tile_n; i += kSortThreads) {
            const uint32_t dg = ((uint32_t)s_keys[i] >> shift) & (R - 1u);
            const uint32_t o = s_global_base[dg] + (i - (uint32_t)s_local_base[dg]);
            if (o < n) aux_out[o] = s_vals[i];
        }
    }
}

uint32_t sort_tile_items() { return kSortTile; }

// Single passes of the sort, for callers that manage their own buffers.
void launch_radix_upsweep_u32(const uint32_t* keys, const uint32_t* count_ptr, int shift, uint32_t* counts,
                              uint32_t stride, cudaStream_t s) {
    upsweep_kernel<uint32_t, 8><<<stride, kSortThreads, 0, s>>>(keys, count_ptr, shift, counts, stride, nullptr, 0);
}

void launch_radix_downsweep_u32(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                uint32_t* vals_out, const uint32_t* count_ptr, int shift, int nbits,
                                const uint32_t* offsets, uint32_t stride, uint32_t* run_start, uint32_t* run_end,
                                cudaStream_t s) {
    if (keys_out)
        downsweep_kernel<uint32_t, true, false, 8><<<stride, kSortThreads, 0, s>>>(
            keys_in, vals_in, keys_out, vals_out, count_ptr, shift, nbits, offsets, stride, run_start, run_end,
            nullptr, nullptr, SortGather{}, 0);
    else
        downsweep_kernel<uint32_t, false, false, 8><<<stride, kSortThreads, 0, s>>>(
            keys_in, vals_in, keys_out, vals_out, count_ptr, shift, nbits, offsets, stride, run_start, run_end,
            nullptr, nullptr, SortGather{}, 0);
}

int radix_last_bits(int key_bits, int key_bytes) {
    return (key_bytes == 2 && key_bits > 8 && key_bits <= 10) ? key_bits : 8;
}

uint32_t radix_count_words(uint32_t max_n, int radix_bits) {
    return (1u << radix_bits) * std::max<uint32_t>((max_n + kSortTile - 1) / kSortTile, 1u);
}

template <typename KeyT, bool WK, bool AUX, int RB>
static void launch_downsweep(KeyT* keys[2], uint32_t* vals[2], uint32_t* const* aux, int a, int b,
                             const uint32_t* count_ptr, int shift, int nbits, const uint32_t* offsets, uint32_t stride,
                             uint32_t* rs, uint32_t* re, const SortGather& gather, cudaStream_t s) {
    launch_pdl(downsweep_kernel<KeyT, WK, AUX, RB>, dim3(stride), dim3(kSortThreads), 0, s, keys[a], vals[a], keys[b],
               vals[b], count_ptr, shift, nbits, offsets, stride, rs, re, AUX ? aux[a] : nullptr,
               AUX ? aux[b] : nullptr, gather, 1);
}

template <typename KeyT, int RB>
static void launch_pass(KeyT* keys[2], uint32_t* vals[2], uint32_t* const* aux, int a, int b, bool wk,
                        const uint32_t* count_ptr, int shift, int nbits, uint32_t* counts, uint32_t* offsets,
                        uint32_t* totals, uint32_t stride, uint32_t* rs, uint32_t* re, const SortGather& g,
                        cudaStream_t s) {
    launch_pdl(upsweep_kernel<KeyT, RB>, dim3(stride), dim3(kSortThreads), 0, s, keys[a], count_ptr, shift, counts,
               stride, totals, 1);
    launch_digit_scan(counts, stride, totals, offsets, s, 1u << RB, count_ptr, kSortTile);
    if (aux) {
        if (wk) launch_downsweep<KeyT, true, true, RB>(keys, vals, aux, a, b, count_ptr, shift, nbits, offsets, stride,
                                                        rs, re, g, s);
        else launch_downsweep<KeyT, false, true, RB>(keys, vals, aux, a, b, count_ptr, shift, nbits, offsets, stride,
                                                      rs, re, g, s);
    } else {
        if (wk) launch_downsweep<KeyT, true, false, RB>(keys, vals, aux, a, b, count_ptr, shift, nbits, offsets,
                                                         stride, rs, re, g, s);
        else launch_downsweep<KeyT, false, false, RB>(keys, vals, aux, a, b, count_ptr, shift, nbits, offsets,
                                                       stride, rs, re, g, s);
    }
}

template <typename KeyT>
int radix_sort_pairs(KeyT* keys[2], uint32_t* vals[2], const uint32_t* count_ptr, uint32_t max_n, int key_bits,
                     bool keys_after_last, uint32_t* counts, uint32_t* offsets, uint32_t* digit_totals,
                     int& launches, cudaStream_t s, uint32_t* run_start, uint32_t* run_end, uint32_t* const* aux,
                     const SortGather* gather) {
    const uint32_t stride = std::max<uint32_t>((max_n + kSortTile - 1) / kSortTile, 1u);
    const int wide = radix_last_bits(key_bits, (int)sizeof(KeyT));  // digit width of the last pass
    const int passes = wide > 8 ? 1 : std::max(1, (key_bits + 7) / 8);
    for (int p = 0; p < passes; ++p) {
        const int a = p & 1, b = a ^ 1;
        const int nbits = wide > 8 ? wide : std::max(1, std::min(8, key_bits - 8 * p));
        const bool last = p == passes - 1;
        uint32_t* rs = last ? run_start : nullptr;
        uint32_t* re = last ? run_end : nullptr;
        const SortGather g = (last && gather) ? *gather : SortGather{};
        uint32_t* totals = digit_totals + (size_t)p * kRadix;
        const bool wk = !last || keys_after_last;
        if constexpr (sizeof(KeyT) == 2) {
            if (wide == 9) {
                launch_pass<KeyT, 9>(keys, vals, aux, a, b, wk, count_ptr, 0, nbits, counts, offsets, totals, stride,
                                     rs, re, g, s);
            } else if (wide == 10) {
                launch_pass<KeyT, 10>(keys, vals, aux, a, b, wk, count_ptr, 0, nbits, counts, offsets, totals, stride,
                                      rs, re, g, s);
            } else {
                launch_pass<KeyT, 8>(keys, vals, aux, a, b, wk, count_ptr, 8 * p, nbits, counts, offsets, totals,
                                     stride, rs, re, g, s);
            }
        } else {
            launch_pass<KeyT, 8>(keys, vals, aux, a, b, wk, count_ptr, 8 * p, nbits, counts, offsets, totals, stride,
                                 rs, re, g, s);
        }
        if (cudaPeekAtLastError() != cudaSuccess) return -1;
        launches += 3;
    }
    return passes & 1;
}
template int radix_sort_pairs<uint32_t>(uint32_t* [2], uint32_t* [2], const uint32_t*, uint32_t, int, bool,
                                        uint32_t*, uint32_t*, uint32_t*, int&, cudaStream_t, uint32_t*,
                                        uint32_t*, uint32_t* const*, const SortGather*);
template int radix_sort_pairs<uint16_t>(uint16_t* [2], uint32_t* [2], const uint32_t*, uint32_t, int, bool,
                                        uint32_t*, uint32_t*, uint32_t*, int&, cudaStream_t, uint32_t*,
                                        uint32_t*, uint32_t* const*, const SortGather*);

}  // namespace seele
