// order.cu -- spatial order of a loaded scene (SEELE_SCENE_SPATIAL).
//
// Preprocessing reads every attribute plane as float4 per Gaussian, and DRAM
// delivers 64-byte chunks: four neighbouring Gaussians share a chunk, so a
// culled Gaussian next to a visible one costs its bytes anyway.  Storing the
// scene in Morton (Z-curve) order of the means puts Gaussians that the frustum
// keeps or culls together next to each other, and whole chunks of culled ones
// are never read.  The order is computed once at load: the bounding box of the
// means (order-preserving integer atomics), a 30-bit Morton code per Gaussian
// (10 bits per axis), a stable radix sort of (code, index), then a gather of
// every plane.  Ties keep the caller's order.
#include "common.cuh"
#include "kernels.h"

namespace seele {

namespace {

// float -> uint32 with the same order (negative values flipped)
__device__ __forceinline__ uint32_t ordered_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered_bits(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// spreads the low 10 bits of x to every third bit
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

}  // namespace

// bb[0..2]: smallest x, y, z; bb[3..5]: largest (ordered bits; start at
// all-ones / zero)
__global__ void bbox_kernel(const float4* __restrict__ pos, int n, uint32_t* __restrict__ bb) {
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const float4 p = __ldg(pos + g);
        const uint32_t b[3] = {ordered_bits(p.x), ordered_bits(p.y), ordered_bits(p.z)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], b[a]);
            hi[a] = max(hi[a], b[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(bb + a, lo[a]);
            atomicMax(bb + 3 + a, hi[a]);
        }
}

__global__ void morton_kernel(const float4* __restrict__ pos, int n, const uint32_t* __restrict__ bb,
                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 p = __ldg(pos + g);
    const float c[3] = {p.x, p.y, p.z};
    uint32_t code = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = from_ordered_bits(bb[a]), hi = from_ordered_bits(bb[3 + a]);
        const float ext = hi - lo;
        float t = ext > 0.f ? (c[a] - lo) / ext : 0.f;
        t = fminf(fmaxf(t, 0.f), 1.f);
        code |= spread3(min((uint32_t)(t * 1024.f), 1023u)) << a;
    }
    keys[g] = code;
    vals[g] = (uint32_t)g;
}

// dst[j * n + i] = src[j * n + order[i]] for `planes` float4 planes
__global__ void gather_planes_kernel(const float4* __restrict__ src, float4* __restrict__ dst, int n, int planes,
                                     const uint32_t* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t g = __ldg(order + i);
    for (int j = 0; j < planes; ++j) dst[(size_t)j * n + i] = __ldg(src + (size_t)j * n + g);
}

__global__ void gather_u32_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int n,
                                  const uint32_t* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __ldg(src + __ldg(order + i));
}

// dst[order[i]] = src[i]: back to the caller's order
__global__ void scatter_u32_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int n,
                                   const uint32_t* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[__ldg(order + i)] = __ldg(src + i);
}

int launch_spatial_order(const float4* pos, int n, uint32_t* bb, uint32_t* keys[2], uint32_t* vals[2],
                         const uint32_t* count_ptr, uint32_t* counts, uint32_t* offsets, uint32_t* digit_totals,
                         cudaStream_t s) {
    if (cudaMemsetAsync(bb, 0xff, 12, s) != cudaSuccess || cudaMemsetAsync(bb + 3, 0, 12, s) != cudaSuccess)
        return -1;
    bbox_kernel<<<152 * 4, 256, 0, s>>>(pos, n, bb);
    morton_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos, n, bb, keys[0], vals[0]);
    if (cudaMemsetAsync(digit_totals, 0, 4 * 4 * 256, s) != cudaSuccess) return -1;
    int launches = 0;
    return radix_sort_pairs<uint32_t>(keys, vals, count_ptr, (uint32_t)n, 30, false, counts, offsets, digit_totals,
                                      launches, s);
}

void launch_gather_planes(const float4* src, float4* dst, int n, int planes, const uint32_t* order, cudaStream_t s) {
    gather_planes_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, dst, n, planes, order);
}

void launch_gather_u32(const uint32_t* src, uint32_t* dst, int n, const uint32_t* order, cudaStream_t s) {
    gather_u32_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, dst, n, order);
}

void launch_scatter_u32(const uint32_t* src, uint32_t* dst, int n, const uint32_t* order, cudaStream_t s) {
    scatter_u32_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, dst, n, order);
}

}  // namespace seele
