// noalloc.cu -- seele_sort_tile_instances_noalloc: the tile-instance sort of
// the render path for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host application or engine
// that owns the whole device memory budget and forbids allocations outside
// its own pool, a real-time loop where an allocation (which can synchronise
// the device) would stall a frame, or code that must keep its footprint fixed
// and known up front.  For them this entry point keeps every byte of scratch
// in one file-scope device array, reserved when the library is loaded; the
// caller passes inputs and outputs only.
//
// The array is shared by every call on a device and keeps the last call's
// contents, so calls that overlap on the GPU (different streams, or threads)
// race on it; the call clears what must start at zero itself.
#include <atomic>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "seele.h"

namespace {

using namespace seele;

constexpr uint32_t kSortTileItems = 4096;  // elements per sort tile (matches sort.cu)
constexpr uint32_t kStride = SEELE_NOALLOC_MAX_INSTANCES / kSortTileItems;
constexpr uint32_t kCountWords = 256 * kStride;
constexpr uint32_t kLookbackEntries = 1024;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kOffStatus = 0;
constexpr size_t kOffCount = 256;                                        // element count read by the kernels
constexpr size_t kOffKeys = 512;                                         // pass-1 keys
constexpr size_t kOffVals = kOffKeys + 4ull * SEELE_NOALLOC_MAX_INSTANCES;  // pass-1 values
constexpr size_t kOffCounts = kOffVals + 4ull * SEELE_NOALLOC_MAX_INSTANCES;
constexpr size_t kOffOffsets = kOffCounts + 4ull * kCountWords;
constexpr size_t kOffLookback = kOffOffsets + 4ull * kCountWords;
constexpr size_t kScratchBytes = kOffLookback + 8ull * kLookbackEntries;
static_assert(sizeof(DeviceStatus) <= 256, "status fits its slot");

// Reserved on every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Clears the status word and tickets and stores the element count.  Device
// code can name the array directly.
__global__ void noalloc_prepare_kernel(uint32_t n) {
    uint32_t* w = reinterpret_cast<uint32_t*>(g_scratch + kOffStatus);
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) w[i] = 0u;
    if (threadIdx.x == 0) *reinterpret_cast<uint32_t*>(g_scratch + kOffCount) = n;
}

// Tile ids must be below n_tiles: the sort ranks only the bits such ids have
// and indexes the range arrays with them.  An id outside that range zeroes the
// element count the sort kernels read (so they touch nothing) and records an
// argument error.
__global__ void noalloc_check_kernel(const uint32_t* __restrict__ tile, uint32_t n, uint32_t n_tiles) {
    uint32_t bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        bad |= __ldg(tile + i) >= n_tiles ? 1u : 0u;
    if (__syncthreads_or(bad) && threadIdx.x == 0) {
        DeviceStatus* st = reinterpret_cast<DeviceStatus*>(g_scratch + kOffStatus);
        atomicCAS(&st->error, kOk, kErrArg);
        atomicExch(reinterpret_cast<uint32_t*>(g_scratch + kOffCount), 0u);
    }
}

// Host code must not take &g_scratch (that is a host-side stand-in): the
// device address comes from cudaGetSymbolAddress, once per device, with that
// device current.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};
std::atomic<uint32_t> g_epoch[kMaxDevices];

seele_status scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return SEELE_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
        g_epoch[dev].store(1);
    }
    *out = g_addr[dev];
    return SEELE_OK;
}

int bits_needed(uint32_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

}  // namespace

extern "C" seele_status seele_sort_tile_instances_noalloc(const uint32_t* inst_tile, const uint32_t* inst_record,
                                                           uint32_t n_instances, uint32_t n_tiles,
                                                           uint32_t* sorted_record, uint32_t* tile_start,
                                                           uint32_t* tile_end, void* cuda_stream) {
    if (n_tiles < 1 || n_tiles > SEELE_NOALLOC_MAX_TILES) return SEELE_ERR_ARG;
    if (n_instances > SEELE_NOALLOC_MAX_INSTANCES) return SEELE_ERR_ARG;
    if (!tile_start || !tile_end) return SEELE_ERR_ARG;
    if (n_instances > 0 && (!inst_tile || !inst_record || !sorted_record)) return SEELE_ERR_ARG;
    // the first pass reads the tile ids as 16-byte vectors
    if (reinterpret_cast<uintptr_t>(inst_tile) & 15u) return SEELE_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return SEELE_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    seele_status st0 = scratch_address(dev, &base);
    if (st0 != SEELE_OK) return st0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    DeviceStatus* st = reinterpret_cast<DeviceStatus*>(base + kOffStatus);
    const uint32_t* count = reinterpret_cast<const uint32_t*>(base + kOffCount);
    uint32_t* keys_tmp = reinterpret_cast<uint32_t*>(base + kOffKeys);
    uint32_t* vals_tmp = reinterpret_cast<uint32_t*>(base + kOffVals);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(base + kOffOffsets);
    uint64_t* lookback = reinterpret_cast<uint64_t*>(base + kOffLookback);

    noalloc_prepare_kernel<<<1, 64, 0, s>>>(n_instances);
    if (n_instances > 0) {
        const uint32_t blocks = (n_instances + 255) / 256 < 1216 ? (n_instances + 255) / 256 : 1216;
        noalloc_check_kernel<<<blocks, 256, 0, s>>>(inst_tile, n_instances, n_tiles);
    }
    if (cudaMemsetAsync(tile_start, 0xff, 4ull * n_tiles, s) != cudaSuccess ||
        cudaMemsetAsync(tile_end, 0, 4ull * n_tiles, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return SEELE_ERR_CUDA;
    }
    const uint32_t stride = n_instances == 0 ? 1u : (n_instances + kSortTileItems - 1) / kSortTileItems;
    const int key_bits = bits_needed(n_tiles - 1) > 0 ? bits_needed(n_tiles - 1) : 1;
    const int passes = (key_bits + 7) / 8;  // 1 or 2
    for (int p = 0; p < passes; ++p) {
        const bool last = p == passes - 1;
        const uint32_t* kin = p == 0 ? inst_tile : keys_tmp;
        const uint32_t* vin = p == 0 ? inst_record : vals_tmp;
        const int nbits = key_bits - 8 * p < 8 ? key_bits - 8 * p : 8;
        launch_radix_upsweep_u32(kin, count, 8 * p, counts, stride, s);
        launch_exclusive_scan(counts, 256 * stride, offsets, lookback, g_epoch[dev].fetch_add(1), st, p, s);
        launch_radix_downsweep_u32(kin, vin, last ? nullptr : keys_tmp, last ? sorted_record : vals_tmp, count,
                                   8 * p, nbits, offsets, stride, last ? tile_start : nullptr,
                                   last ? tile_end : nullptr, s);
    }
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return SEELE_ERR_CUDA;
    }
    // wait, then read the status word back (a plain copy; nothing is allocated)
    int32_t err = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(&err, base + kOffStatus, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return SEELE_ERR_CUDA;
    }
    if (err == kOk) return SEELE_OK;
    if (err == kErrTimeout) return SEELE_ERR_TIMEOUT;
    if (err == kErrArg) return SEELE_ERR_ARG;
    return SEELE_ERR_INTERNAL;
}
