// common.cuh -- device-side types shared by the Seele kernels (sm_103a).
//
// One frame of the hot path, for all cameras at once (record id
// r = camera * n + g indexes every per-(camera, Gaussian) array):
//   preprocess    -> records, rect, tiles_touched, depth        (Sec. 3.1, 3.3)
//   compact       -> visible record ids in id order, depth keys
//   depth sort    -> visible ids in (fp32 depth, id) order       (Sec. 3.1 "Sorting")
//   tile scan     -> instance offsets in depth order, K
//   emit          -> (global tile, record id) pairs, depth-ordered
//   tile sort     -> stable by tile: (tile, depth, id) order
//   ranges        -> [start, end) per global tile
//   raster        -> image, final T, n_contrib                   (Eqns. 1-2, Alg. 1)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace seele {

constexpr float kLog2e = 1.4426950408889634f;

// Device status word: the first error a kernel meets is kept.
enum : int32_t { kOk = 0, kErrArg = 1, kErrCapacity = 4, kErrTimeout = 5, kErrInternal = 7 };

struct DeviceStatus {
    int32_t error;
    uint32_t n_visible;      // visible records
    uint32_t n_instances;    // K
    uint32_t capacity;       // instance capacity the scan compared K against
    uint32_t n_inst_valid;   // K if it fits the capacity, else 0 (what the tile sort reads)
    uint32_t timeout_site;   // which wait gave up (diagnostics)
    uint32_t queue;          // list units taken by the persistent rasterizer
    uint32_t pad[2];
    uint32_t ticket[16];     // dynamic block tickets of the look-back kernels
    unsigned long long work[4];  // rasterizer work counters (counting variant only)
};

// Per-camera constants, built on the host.
struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float campos[3];
    float lim_x, lim_y;      // 1.3 * W / (2 fx), 1.3 * H / (2 fy)
    float near_z;
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    uint32_t tile_offset;    // first global tile id of this camera
    uint32_t pix_offset;     // sum of W*H of the previous cameras
    uint32_t sel_bits;       // selected view clusters
    uint32_t block_offset;   // first global tile-block id of this camera (block binning)
    int32_t blocks_x;        // tile blocks per row: ceil(tiles_x / kBlockW)
    uint32_t slot_ok[2];     // streamed scene: slots (bit s of word s / 32) ready to read that
                             // hold part of a selected cluster
    int32_t pad;
};

// Records are counted in chunks of this many for the ordered compaction and
// scans (a chunk is one CTA of those kernels).
constexpr uint32_t kChunkItems = 4096;
// Packed (record id, instance count) sort values: ids below 2^kPackedIdBits,
// counts saturated at kPackedCountMax (the true count is then read again).
constexpr int kPackedIdBits = 24;
constexpr uint32_t kPackedCountMax = 255u;
// Transmittance checkpoints of tile-binned renders: every kCkptL entries of
// a tile's list, each pixel's (T, r, g, b) so far.  Tile t's checkpoint c
// (c >= 1, at list position c * kCkptL < its length) is slot
// (start_t >> kCkptShift) + c: lists are disjoint, so slots never collide
// and there are at most capacity / kCkptL + 2 of them.  The backward pass
// walks each kCkptL-entry chunk of a list in a CTA of its own from them.
constexpr uint32_t kCkptShift = 8;
constexpr uint32_t kCkptL = 1u << kCkptShift;

// Block binning: a tile block is kBlockW x kBlockH tiles; its instances carry a
// 32-bit mask of the block's tiles that the Gaussian reaches (bit j * kBlockW + i
// for tile (i, j) of the block).
constexpr int kBlockW = 8;
constexpr int kBlockH = 4;
static_assert(kBlockW * kBlockH == 32, "one mask word per block instance");

struct FrameParams {
    int32_t n;               // Gaussians
    int32_t n_cams;
    int32_t sh_degree;
    int32_t tile_w, tile_h;
    int32_t opacity_filter;
    int32_t tile_test;       // 1: ellipse tile test, 0: every tile of the rect
    int32_t binning;         // 0: tile instances, 1: tile-block instances with tile masks
    int32_t use_mask;
    float alpha_min, alpha_max, t_stop;
    float log_alpha_min, log2_alpha_min;  // ln and log2 of alpha_min
    float dilation;
    float frustum_slack;
    uint32_t n_tiles_total;
    uint32_t n_shared;       // streamed scene: resident shared Gaussians, then slots of slot_cap
    uint32_t slot_cap;       // 0: the whole scene is resident
};

// Scene in the library's layout (structure of arrays, 16-byte aligned).
struct SceneDev {
    const float4* pos_logit = nullptr;   // (x, y, z, opacity logit)
    const float4* quat = nullptr;        // (w, x, y, z)
    const float4* log_scale = nullptr;   // (lx, ly, lz, 0)
    const float4* sh = nullptr;          // plane-major: sh[j * n + g], j < ceil(3 nc / 4)
    const uint32_t* mask = nullptr;      // [n] or nullptr
    const uint32_t* veto = nullptr;      // streamed scene: [n] clusters that take precedence, or nullptr
    // a BORROW scene read in place (else nullptr): the caller's arrays in the
    // layout of seele_scene_desc, quats and sh 16-byte aligned
    const float* means = nullptr;        // [n][3]
    const float* log_scales = nullptr;   // [n][3]
    const float* quats = nullptr;        // [n][4]
    const float* logits = nullptr;       // [n]
    const float* shc = nullptr;          // [n][nc][3]
};

// One Gaussian's attributes from the planes, or (AOS) from the caller's arrays.
template <bool AOS>
__device__ __forceinline__ float4 scene_pos_logit(const SceneDev& sc, int g) {
    if constexpr (AOS)
        return make_float4(__ldg(sc.means + 3 * (size_t)g), __ldg(sc.means + 3 * (size_t)g + 1),
                           __ldg(sc.means + 3 * (size_t)g + 2), __ldg(sc.logits + g));
    else
        return __ldg(sc.pos_logit + g);
}

template <bool AOS>
__device__ __forceinline__ float4 scene_quat(const SceneDev& sc, int g) {
    if constexpr (AOS)
        return __ldg(reinterpret_cast<const float4*>(sc.quats) + g);
    else
        return __ldg(sc.quat + g);
}

template <bool AOS>
__device__ __forceinline__ float4 scene_log_scale(const SceneDev& sc, int g) {
    if constexpr (AOS)
        return make_float4(__ldg(sc.log_scales + 3 * (size_t)g), __ldg(sc.log_scales + 3 * (size_t)g + 1),
                           __ldg(sc.log_scales + 3 * (size_t)g + 2), 0.f);
    else
        return __ldg(sc.log_scale + g);
}

// SH coefficients 4j .. 4j + 3 of Gaussian g (zero past 3 nc), the j-th plane
template <bool AOS, int NC>
__device__ __forceinline__ float4 scene_sh4(const SceneDev& sc, int n, int g, int j) {
    if constexpr (AOS) {
        const float* row = sc.shc + (size_t)g * (3 * NC);
        if constexpr ((3 * NC) % 4 == 0) {
            return __ldg(reinterpret_cast<const float4*>(row) + j);  // 16-byte rows
        } else {
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = 4 * j + i < 3 * NC ? __ldg(row + 4 * j + i) : 0.f;
            return make_float4(v[0], v[1], v[2], v[3]);
        }
    } else {
        return __ldg(sc.sh + (size_t)j * n + g);
    }
}

// Raster record: kRecF4 float4 per record, one 64-byte line:
//   (u, v, cA, cB), (cC, log2 o, e_thr, T_tile), (r, g, b, clamp flag),
//   (tile box x0 | y0 << 16, x1 | y1 << 16, 0, 0) as integer bits.
constexpr int kRecF4 = 4;

__device__ __forceinline__ uint2 rec_tile_box(const float4* rec, uint32_t r) {
    const float4 b = __ldg(rec + (size_t)kRecF4 * r + 3);
    return make_uint2(__float_as_uint(b.x), __float_as_uint(b.y));
}

// Per-record outputs of preprocessing.
struct ProjOut {
    float4* rec;               // [kRecF4 * R] raster records
    uint32_t* tiles;           // [R] tiles touched (0 = culled)
    uint32_t* blocks;          // [R] tile-block instances (0 = culled; block binning only, else unused)
    float* depth;              // [R] camera-space Z
    unsigned long long* t_frame;  // receives the frame's start time (%globaltimer, ns)
    uint32_t* chunk_vis;       // [ceil(R / kChunkItems)] visible records per chunk (cleared per frame)
};

// Programmatic dependent launch: a frame kernel launched with launch_pdl may
// start while its predecessor drains; it waits for the predecessor's
// completion (and memory) before anything else, and lets its own successor
// launch at once.  Both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded spin for the decoupled look-back: about a second at most, then the
// waiting block records a timeout and gives up instead of hanging the GPU.
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ void record_error(DeviceStatus* st, int32_t code, uint32_t site) {
    if (atomicCAS(&st->error, kOk, code) == kOk) st->timeout_site = site;
}

// The checked build (SEELE_CHECKED, libseele_checked.so) validates every
// index a kernel gathers with before the access; a bad one records
// kErrInternal with the site below and is replaced by a valid one, so the
// kernel stays in bounds and the host reports SEELE_ERR_INTERNAL.  The
// ordinary build compiles the checks away.
#ifdef SEELE_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
enum : uint32_t { kSiteRasterRange = 20, kSiteRasterRecord = 21, kSiteRasterBlock = 22 };

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Look-back status word: [epoch:30][flag:2][value:32].  Entries of another
// epoch read as "not yet published", so the status arrays need no clearing
// between scans.
constexpr uint32_t kFlagAggregate = 1u, kFlagInclusive = 2u;

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint32_t flag, uint32_t value) {
    return ((uint64_t)(epoch & 0x3fffffffu) << 34) | ((uint64_t)flag << 32) | value;
}

__device__ __forceinline__ uint32_t status_flag(uint64_t s, uint32_t epoch) {
    return ((uint32_t)(s >> 34) == (epoch & 0x3fffffffu)) ? (uint32_t)(s >> 32) & 3u : 0u;
}

}  // namespace seele
