// api.cu -- the C ABI of include/seele.h: context, scene and camera state,
// workspace management and the per-frame kernel sequence.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "seele.h"
#include "kernels.h"

using namespace seele;

namespace {

// NVTX ranges: one per public call, and within a frame's enqueue one per
// stage (host-side, where each stage is issued; free when no tool listens).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
const char* const kStageNvtx[SEELE_NUM_STAGES] = {"preprocess", "compact", "depth_sort", "tile_scan",
                                                   "emit", "tile_sort", "ranges", "raster"};
struct NvtxStages {
    bool open = false;
    void next(int k) {
        if (open) nvtxRangePop();
        nvtxRangePushA(kStageNvtx[k]);
        open = true;
    }
    ~NvtxStages() {
        if (open) nvtxRangePop();
    }
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Device memory of a COPY scene that several contexts render
// (seele_share_scene): the planes, the cluster mask and the spatial order,
// freed when the last context lets go.
struct SharedScene {
    int device = 0;
    void* p[6] = {};
    ~SharedScene() {
        int prev = 0;
        const bool had = cudaGetDevice(&prev) == cudaSuccess;
        cudaSetDevice(device);
        for (void* q : p)
            if (q) cudaFree(q);
        if (had) cudaSetDevice(prev);
    }
};

constexpr int kMaxCams = 4096;
constexpr uint64_t kShortKeyMaxTiles = 65536;   // 16-bit tile keys

}  // namespace

struct seele_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // scene
    bool has_scene = false;
    int64_t n = 0;
    int sh_degree = 0;
    int scene_flags = 0;
    seele_scene_desc borrowed{};
    DevBuf pos_logit, quat, log_scale, sh, mask, staging, veto;
    // spatial order (SEELE_SCENE_SPATIAL): caller index of each resident
    // Gaussian, the planes before the gather, a few words of scratch
    DevBuf order, unordered, order_scratch;
    bool spatial = false;
    // set while the scene's memory is shared: pos_logit, quat, log_scale,
    // sh, mask and order are then views of it, not owned
    std::shared_ptr<SharedScene> shared;
    bool has_mask = false;
    int n_clusters = 0;
    std::vector<double> centroids;
    double pos_scale = 1.0;

    // cameras
    std::vector<seele_camera> cams;
    std::vector<CamDev> camdev;
    DevBuf cams_dev;

    // frame workspace
    DevBuf rec, tiles, blocks, depth, visk[2], visv[2], offs, instk[2], instv[2], instm[2], ranges, msum,
        border, chunkv, chunks, vbuf, status, hist, digtot, T, nc, rgb_tmp, sortcnt, grad_rec, cnts, torder,
        ckpt, cfin, bmap, branges, tcnt, toff, emap, ecnt;
    // the last render wrote transmittance checkpoints for ckpt_slots slots
    bool ckpt_valid = false;
    // the last render left its tiles' longest-list-first order in border
    bool border_tiles = false;
    uint64_t ckpt_slots = 0;
    DeviceStatus* h_status = nullptr;  // pinned mirror of the device status
    cudaEvent_t ev[SEELE_NUM_STAGES + 1] = {};
    bool profiling = false;

    // pinned staging ring for camera constants (no pageable copies in a frame)
    struct CamSlot {
        CamDev* host = nullptr;
        size_t cap = 0;
        cudaEvent_t done = nullptr;
        bool used = false;
    } cam_ring[4];
    int cam_next = 0;

    // per-view completion times: [frame start][end per camera][done tiles per camera]
    DevBuf viewt;

    // captured frame (SEELE_RENDER_GRAPH)
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;   // capture happens here (the legacy stream cannot capture)
    std::vector<uint64_t> gkey;
    int g_launches = 0, g_fin = 0;
    uint64_t scene_gen = 0;
    uint64_t capacity = 0;
    bool status_pending = false;

    // last render
    bool rendered = false;
    seele_options last_opt{};
    int inst_final = 0;
    uint32_t n_tiles_total = 0;
    uint32_t n_units_total = 0;   // list units: tiles, or tile blocks with block binning
    uint64_t n_pix_total = 0;
    FrameParams last_fp{};

    // view-representation builder: while set, frames end in the top-k
    // contributor pass instead of the rasterizer
    int topk_k = 0;
    const int* topk_cluster = nullptr;   // device, cluster of each camera of the frame
    uint32_t* topk_mask = nullptr;       // device, [n]
    // contribution-skew statistic: while skew_frac > 0, frames end in the
    // skew pass, writing [pixels] m, blended, walked (u32), total (f32) and
    // listed (u32)
    double skew_frac = 0.0;
    DevBuf skew;

    // Streamed scene (Sec. 3.3 "Scene Prefetching"): every view cluster's
    // Gaussians stay in pinned host memory, cut into chunks of at most
    // slot_cap; the device holds the shared Gaussians and n_slots slots of
    // slot_cap Gaussians, each holding one chunk.  A frame loads the chunks of
    // the clusters its cameras select that are not resident (on its own
    // stream); after it, the chunks of the clusters selected for the cameras'
    // linearly extrapolated poses are prefetched on the copy stream.
    struct Streamed {
        bool on = false;
        int n_slots = 0, ahead = 1, planes = 0;   // planes: float4 per Gaussian
        uint32_t n_shared = 0, cap = 0;
        int64_t n_full = 0;                       // Gaussians of the whole scene
        float4* host = nullptr;                   // pinned, [planes][copies]
        uint32_t* host_mask = nullptr;            // pinned, [copies]: the copy's cluster bit
        uint32_t* host_veto = nullptr;            // pinned, [copies]: the Gaussian's lower clusters
        size_t copies = 0;
        std::vector<size_t> seg;                  // [C + 2]: cluster c is [seg[c], seg[c + 1]), shared last
        std::vector<int> chunk_begin;             // [C + 1]: cluster c's chunks are [chunk_begin[c], ..[c + 1])
        std::vector<int> chunk_cluster;           // per chunk
        std::vector<size_t> chunk_at;             // per chunk: first copy
        std::vector<uint32_t> chunk_n;            // per chunk: copies
        std::vector<int> slot_cluster;            // per slot: the chunk it holds, -1: empty
        std::vector<bool> slot_async;             // filled on the copy stream, not yet waited for
        std::vector<uint64_t> slot_stamp;         // last frame that used or filled it
        std::vector<cudaEvent_t> slot_ready, slot_used;
        cudaStream_t copy = nullptr;
        uint64_t frame = 0;
        std::vector<std::vector<double>> prev;    // per camera: position and view direction last frame
        int64_t loads_sync = 0, loads_prefetch = 0, prefetch_hits = 0, resident_hits = 0;
    } st;
};

namespace {

seele_status fail(seele_ctx* c, seele_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define SEELE_CUDA(ctx, call)                                                                              \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            (void)cudaGetLastError();                                                                      \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SEELE_ERR_OOM : SEELE_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
        }                                                                                                  \
    } while (0)

#define SEELE_LAUNCHED(ctx) SEELE_CUDA(ctx, cudaGetLastError())

cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (cudaMallocHost,
// cudaHostRegister), which kernels read and write over the host link; NULL
// for any other pointer.
const void* mapped_host(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <class T>
T* ptr(DevBuf& b) {
    return static_cast<T*>(b.p);
}

#define SEELE_MARK_EXT(ctx, k) \
    if ((ctx)->profiling) cudaEventRecord((ctx)->ev[k], (ctx)->stream)

// Camera centre and unit viewing direction (the third row of R).
void camera_pose(const seele_camera& cam, double pos[3], double dir[3]) {
    const float* w = cam.world_to_cam;
    const double R[9] = {w[0], w[1], w[2], w[4], w[5], w[6], w[8], w[9], w[10]};
    const double t[3] = {w[3], w[7], w[11]};
    for (int i = 0; i < 3; ++i) pos[i] = -(R[i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2]);
    for (int i = 0; i < 3; ++i) dir[i] = R[6 + i];
}

// Runtime cluster selection (Sec. 3.3 "Algorithm"): nearest centroid to the
// camera feature (position / s, unit viewing direction), then the M centroids
// nearest to that centroid; ties go to the lower index.
uint32_t select_clusters_at(const seele_ctx* c, const double pos[3], const double dir[3], int M) {
    if (c->n_clusters <= 0) return 0xffffffffu;
    double f[6] = {pos[0] / c->pos_scale, pos[1] / c->pos_scale, pos[2] / c->pos_scale, dir[0], dir[1], dir[2]};
    const int C = c->n_clusters;
    auto dist2 = [&](const double* a, const double* b) {
        double s = 0;
        for (int i = 0; i < 6; ++i) s += (a[i] - b[i]) * (a[i] - b[i]);
        return s;
    };
    int best = 0;
    double bd = INFINITY;
    for (int k = 0; k < C; ++k) {
        double d = dist2(f, &c->centroids[6 * k]);
        if (d < bd) {
            bd = d;
            best = k;
        }
    }
    uint32_t bits = 1u << best;
    for (int pick = 0; pick < M && pick < C - 1; ++pick) {
        int arg = -1;
        double ad = INFINITY;
        for (int k = 0; k < C; ++k) {
            if (bits >> k & 1u) continue;
            double d = dist2(&c->centroids[6 * best], &c->centroids[6 * k]);
            if (d < ad) {
                ad = d;
                arg = k;
            }
        }
        bits |= 1u << arg;
    }
    return bits;
}

uint32_t select_clusters(const seele_ctx* c, const seele_camera& cam, int M) {
    double pos[3], dir[3];
    camera_pose(cam, pos, dir);
    return select_clusters_at(c, pos, dir, M);
}

// Digit totals of the sorts' passes, 256 words per pass: the depth sort's
// four, then up to four of the tile sort (or the 512 or 1024 of its one wide
// pass).
constexpr uint32_t kDepthSortTotals = 4 * 256;
constexpr uint32_t kDigitTotalWords = 8 * 256;

// ------------------------------------------------------- spatial order --

// Reorders the planes built in c->unordered (and the cluster mask) into
// Morton order of the means; c->order keeps each one's caller index.
seele_status spatial_order(seele_ctx* c, int64_t n, int planes) {
    cudaStream_t s = c->stream;
    SEELE_CUDA(c, ensure(c->order, 4 * n));
    SEELE_CUDA(c, ensure(c->order_scratch, 64));
    for (int i = 0; i < 2; ++i) {
        SEELE_CUDA(c, ensure(c->visk[i], 4 * n));
        SEELE_CUDA(c, ensure(c->visv[i], 4 * n));
    }
    const uint32_t words = radix_count_words((uint32_t)n);
    SEELE_CUDA(c, ensure(c->sortcnt, 8ull * words));
    SEELE_CUDA(c, ensure(c->digtot, 4 * kDigitTotalWords));
    uint32_t* bb = ptr<uint32_t>(c->order_scratch);
    const uint32_t count = (uint32_t)n;
    SEELE_CUDA(c, cudaMemcpy(bb + 6, &count, 4, cudaMemcpyHostToDevice));
    uint32_t* keys[2] = {ptr<uint32_t>(c->visk[0]), ptr<uint32_t>(c->visk[1])};
    uint32_t* vals[2] = {ptr<uint32_t>(c->visv[0]), ptr<uint32_t>(c->visv[1])};
    const float4* P0 = ptr<float4>(c->unordered);
    const int fin = launch_spatial_order(P0, (int)n, bb, keys, vals, bb + 6, ptr<uint32_t>(c->sortcnt),
                                         ptr<uint32_t>(c->sortcnt) + words, ptr<uint32_t>(c->digtot), s);
    if (fin < 0) return fail(c, SEELE_ERR_CUDA, "spatial order: %s", cudaGetErrorString(cudaGetLastError()));
    const uint32_t* ord = vals[fin];
    SEELE_CUDA(c, cudaMemcpyAsync(c->order.p, ord, 4 * n, cudaMemcpyDeviceToDevice, s));
    launch_gather_planes(P0, ptr<float4>(c->pos_logit), (int)n, 1, ord, s);
    launch_gather_planes(P0 + n, ptr<float4>(c->quat), (int)n, 1, ord, s);
    launch_gather_planes(P0 + 2 * n, ptr<float4>(c->log_scale), (int)n, 1, ord, s);
    launch_gather_planes(P0 + 3 * n, ptr<float4>(c->sh), (int)n, planes, ord, s);
    if (c->has_mask) {
        SEELE_CUDA(c, cudaMemcpyAsync(keys[1], c->mask.p, 4 * n, cudaMemcpyDeviceToDevice, s));
        launch_gather_u32(keys[1], ptr<uint32_t>(c->mask), (int)n, ord, s);
    }
    SEELE_LAUNCHED(c);
    return SEELE_OK;
}

// The scene as the kernels read it: the planes, or a BORROW scene's own
// arrays in place when quats and sh are 16-byte aligned (else the frame
// repacks them into the planes first).
SceneDev scene_dev(seele_ctx* c) {
    SceneDev sc;
    sc.pos_logit = ptr<float4>(c->pos_logit);
    sc.quat = ptr<float4>(c->quat);
    sc.log_scale = ptr<float4>(c->log_scale);
    sc.sh = ptr<float4>(c->sh);
    if (c->scene_flags == SEELE_SCENE_BORROW) {
        const seele_scene_desc& b = c->borrowed;
        if (((uintptr_t)b.quats & 15u) == 0 && ((uintptr_t)b.sh & 15u) == 0) {
            sc.means = b.means;
            sc.log_scales = b.log_scales;
            sc.quats = b.quats;
            sc.logits = b.opacity_logits;
            sc.shc = b.sh;
        }
    }
    return sc;
}

// ------------------------------------------------------- shared scene --

DevBuf* scene_bufs(seele_ctx* c, int i) {
    DevBuf* b[6] = {&c->pos_logit, &c->quat, &c->log_scale, &c->sh, &c->mask, &c->order};
    return b[i];
}

// Lets go of a shared scene's memory (freed here if this was the last
// context holding it); the scene buffers start empty again.
void scene_unshare(seele_ctx* c) {
    if (!c->shared) return;
    for (int i = 0; i < 6; ++i) *scene_bufs(c, i) = DevBuf{};
    c->shared.reset();
}

// ------------------------------------------------------- streamed scene --

void stream_release(seele_ctx* c) {
    auto& S = c->st;
    if (S.copy) cudaStreamSynchronize(S.copy);
    for (cudaEvent_t e : S.slot_ready)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : S.slot_used)
        if (e) cudaEventDestroy(e);
    if (S.copy) cudaStreamDestroy(S.copy);
    if (S.host) cudaFreeHost(S.host);
    if (S.host_mask) cudaFreeHost(S.host_mask);
    if (S.host_veto) cudaFreeHost(S.host_veto);
    S = seele_ctx::Streamed{};
}

// Copies m Gaussians from pool position b to resident position `at`, and
// clears the rest of a slot of `room`.
seele_status stream_copy(seele_ctx* c, size_t b, size_t m, uint32_t at, uint32_t room, cudaStream_t s) {
    auto& S = c->st;
    const size_t n = (size_t)c->n;
    float4* planes[3] = {ptr<float4>(c->pos_logit), ptr<float4>(c->quat), ptr<float4>(c->log_scale)};
    for (int p = 0; p < S.planes; ++p) {
        float4* dst = p < 3 ? planes[p] + at : ptr<float4>(c->sh) + (size_t)(p - 3) * n + at;
        if (m) SEELE_CUDA(c, cudaMemcpyAsync(dst, S.host + (size_t)p * S.copies + b, 16 * m, cudaMemcpyHostToDevice, s));
    }
    if (m) {
        SEELE_CUDA(c, cudaMemcpyAsync(ptr<uint32_t>(c->mask) + at, S.host_mask + b, 4 * m, cudaMemcpyHostToDevice, s));
        SEELE_CUDA(c, cudaMemcpyAsync(ptr<uint32_t>(c->veto) + at, S.host_veto + b, 4 * m, cudaMemcpyHostToDevice, s));
    }
    if (room > m) SEELE_CUDA(c, cudaMemsetAsync(ptr<uint32_t>(c->mask) + at + m, 0, 4 * (room - m), s));
    return SEELE_OK;
}

// A slot to (re)fill: empty first, else the least recently used one whose
// chunk's cluster is not in `keep`.
int stream_victim(const seele_ctx* c, uint32_t keep) {
    const auto& S = c->st;
    int best = -1;
    for (int s = 0; s < S.n_slots; ++s) {
        const int ch = S.slot_cluster[s];
        if (ch >= 0 && ((keep >> S.chunk_cluster[ch]) & 1u)) continue;
        if (ch < 0) return s;
        if (best < 0 || S.slot_stamp[s] < S.slot_stamp[best]) best = s;
    }
    return best;
}

int stream_slot_of(const seele_ctx* c, int ch) {
    for (int s = 0; s < c->st.n_slots; ++s)
        if (c->st.slot_cluster[s] == ch) return s;
    return -1;
}

int stream_chunks(const seele_ctx* c, uint32_t clusters) {
    int n = 0;
    for (int k = 0; k < c->n_clusters; ++k)
        if ((clusters >> k) & 1u) n += c->st.chunk_begin[k + 1] - c->st.chunk_begin[k];
    return n;
}

// Before a frame: every cluster the cameras select is made resident (loaded
// on the frame's stream when it is not), the frame waits for slots the copy
// stream filled, and each camera learns which slots it may read.
seele_status stream_prepare(seele_ctx* c) {
    auto& S = c->st;
    uint32_t need = 0;
    for (const CamDev& d : c->camdev) need |= d.sel_bits;
    need &= c->n_clusters >= 32 ? 0xffffffffu : ((1u << c->n_clusters) - 1u);
    if (stream_chunks(c, need) > S.n_slots)
        return fail(c, SEELE_ERR_ARG, "the cameras select %d clusters in %d chunks, more than the %d slots",
                    __builtin_popcount(need), stream_chunks(c, need), S.n_slots);
    ++S.frame;
    for (int ch = 0; ch < (int)S.chunk_cluster.size(); ++ch) {
        if (!((need >> S.chunk_cluster[ch]) & 1u)) continue;
        int s = stream_slot_of(c, ch);
        if (s >= 0) {
            if (S.slot_async[s]) {
                SEELE_CUDA(c, cudaStreamWaitEvent(c->stream, S.slot_ready[s], 0));
                S.slot_async[s] = false;
                ++S.prefetch_hits;
            } else {
                ++S.resident_hits;
            }
        } else {
            s = stream_victim(c, need);
            if (S.slot_async[s]) SEELE_CUDA(c, cudaStreamWaitEvent(c->stream, S.slot_ready[s], 0));
            S.slot_async[s] = false;
            const seele_status r =
                stream_copy(c, S.chunk_at[ch], S.chunk_n[ch], S.n_shared + (uint32_t)s * S.cap, S.cap, c->stream);
            if (r != SEELE_OK) return r;
            S.slot_cluster[s] = ch;
            ++S.loads_sync;
        }
        S.slot_stamp[s] = S.frame;
    }
    for (CamDev& d : c->camdev) {
        d.slot_ok[0] = d.slot_ok[1] = 0;
        for (int s = 0; s < S.n_slots; ++s) {
            const int ch = S.slot_cluster[s];
            if (ch >= 0 && ((d.sel_bits >> S.chunk_cluster[ch]) & 1u)) d.slot_ok[s >> 5] |= 1u << (s & 31);
        }
    }
    return SEELE_OK;
}

// After a frame is enqueued: mark the slots it reads as used by it, then
// prefetch the clusters selected for each camera's pose extrapolated
// `ahead` frames (position and viewing direction, linearly from the last two
// frames) into slots the frame does not read, on the copy stream.
seele_status stream_prefetch(seele_ctx* c, int M) {
    auto& S = c->st;
    uint32_t used[2] = {0u, 0u};
    for (const CamDev& d : c->camdev) {
        used[0] |= d.slot_ok[0];
        used[1] |= d.slot_ok[1];
    }
    for (int s = 0; s < S.n_slots; ++s)
        if ((used[s >> 5] >> (s & 31)) & 1u) SEELE_CUDA(c, cudaEventRecord(S.slot_used[s], c->stream));
    uint32_t now = 0, want = 0;
    for (const CamDev& d : c->camdev) now |= d.sel_bits;
    if (S.prev.size() != c->cams.size()) S.prev.assign(c->cams.size(), std::vector<double>());
    for (size_t i = 0; i < c->cams.size(); ++i) {
        double pos[3], dir[3];
        camera_pose(c->cams[i], pos, dir);
        if (S.prev[i].size() == 6) {
            double p[3], v[3], len = 0;
            for (int j = 0; j < 3; ++j) {
                p[j] = pos[j] + S.ahead * (pos[j] - S.prev[i][j]);
                v[j] = dir[j] + S.ahead * (dir[j] - S.prev[i][3 + j]);
                len += v[j] * v[j];
            }
            len = std::sqrt(len);
            if (len > 0)
                for (int j = 0; j < 3; ++j) v[j] /= len;
            want |= select_clusters_at(c, p, v, M);
        }
        S.prev[i] = {pos[0], pos[1], pos[2], dir[0], dir[1], dir[2]};
    }
    want &= ~now;
    for (int ch = 0; ch < (int)S.chunk_cluster.size(); ++ch) {
        if (!((want >> S.chunk_cluster[ch]) & 1u) || stream_slot_of(c, ch) >= 0) continue;
        const int s = stream_victim(c, now | want);
        if (s < 0) break;
        // the copy waits for the last frame that read the slot
        SEELE_CUDA(c, cudaStreamWaitEvent(S.copy, S.slot_used[s], 0));
        const seele_status r =
            stream_copy(c, S.chunk_at[ch], S.chunk_n[ch], S.n_shared + (uint32_t)s * S.cap, S.cap, S.copy);
        if (r != SEELE_OK) return r;
        SEELE_CUDA(c, cudaEventRecord(S.slot_ready[s], S.copy));
        S.slot_cluster[s] = ch;
        S.slot_async[s] = true;
        S.slot_stamp[s] = S.frame;
        ++S.loads_prefetch;
    }
    return SEELE_OK;
}

bool group_supported(int gw, int gh) {
    return (gw == 2 && gh == 2) || (gw == 1 && gh == 1) || (gw == 2 && gh == 4) || (gw == 4 && gh == 4) ||
           (gw == 4 && gh == 8);
}

int bits_for(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

struct FrameInfo {
    int ncam = 0;
    uint64_t R = 0, tiles_total = 0, blocks_total = 0, pix_total = 0, cap = 0;
    uint64_t units_total = 0;  // list units: tiles, or tile blocks with block binning
    bool blocks = false, short_keys = false, rgb_dev = true, T_dev = true;
    int tile_bits = 1;         // key bits of a list unit id
    uint32_t cnt_words = 0;
    bool queue = false;        // the persistent rasterizer, units in camera groups
    int batch_depth = 0;
    bool expand = false;       // tile binning made by expanding the sorted block lists
    int block_bits = 1;        // key bits of a tile-block id
    FrameParams fp{};
};

// Emission of (block, record, tile mask) instances in depth order, their
// stable radix sort by block and the block ranges (from the last pass).
// Block binning: then the mask summaries and the order in which the
// rasterizer visits the blocks.  Tile binning: then the block lists expanded
// into the tile lists (in tile order) and the tiles' ranges and visiting
// order.  Returns the ping-pong buffer holding the final lists, or -1 on a
// launch error.
template <typename KeyT>
int enqueue_tile_sort(seele_ctx* c, const FrameInfo& f, const uint32_t* order, const float4* rec,
                      const CamDev* cams, DeviceStatus* st, const uint32_t* n_inst, uint64_t cap, int emit_blocks,
                      uint32_t* dtot, uint32_t* scnt, uint32_t* soff, int& launches, cudaStream_t s) {
    const FrameParams& fp = f.fp;
    KeyT* keys[2] = {ptr<KeyT>(c->instk[0]), ptr<KeyT>(c->instk[1])};
    uint32_t* vals[2] = {ptr<uint32_t>(c->instv[0]), ptr<uint32_t>(c->instv[1])};
    uint32_t* masks[2] = {ptr<uint32_t>(c->instm[0]), ptr<uint32_t>(c->instm[1])};
    if (f.expand) {
        // tile lists from the block lists: block instances, their stable sort
        // by block, then each block's list split into its tiles' lists
        launch_emit_blocks<KeyT>(order, ptr<uint32_t>(c->offs), rec, cams, (int)c->n, fp.tile_w, fp.tile_h,
                                 fp.tile_test, st, keys[0], vals[0], masks[0], emit_blocks, s);
        if (cudaPeekAtLastError() != cudaSuccess) return -1;
        ++launches;
        SEELE_MARK_EXT(c, SEELE_STAGE_TILE_SORT);
        const uint32_t B = (uint32_t)f.blocks_total;
        uint32_t* brun = ptr<uint32_t>(c->branges);
        const int bfin = radix_sort_pairs<KeyT>(keys, vals, n_inst, (uint32_t)cap, f.block_bits, false, scnt, soff,
                                                dtot, launches, s, brun, brun + B, masks);
        if (bfin < 0) return -1;
        SEELE_MARK_EXT(c, SEELE_STAGE_RANGES);
        const uint64_t tiles = f.tiles_total;
        const uint32_t chunks = (uint32_t)((tiles + 31) / 32);
        const uint32_t n_ids = expand_chunk_ids(cap, B);
        uint32_t* Lt = ptr<uint32_t>(c->tcnt);
        uint32_t* chunk_total = Lt + 32 * (size_t)chunks;
        uint32_t* St = ptr<uint32_t>(c->toff);
        uint32_t* C = ptr<uint32_t>(c->ecnt);
        uint32_t* Co = C + 32 * (size_t)n_ids;
        uint32_t* run = ptr<uint32_t>(c->ranges);
        launch_tile_expand(vals[bfin], masks[bfin], brun, brun + B, B, cams, f.ncam, (uint32_t)tiles, n_ids,
                           (uint32_t)std::min<uint64_t>(cap, 0xffffffffu), st, ptr<uint32_t>(c->emap), C, Co, Lt,
                           chunk_total, St, vals[bfin ^ 1], run, s);
        if (f.queue)
            launch_view_order(run, run + tiles, (uint32_t)tiles, cams, f.ncam, 0, f.batch_depth,
                              ptr<uint32_t>(c->border), s);
        else
            launch_block_order(run, run + tiles, (uint32_t)tiles, ptr<uint32_t>(c->border), s);
        if (cudaPeekAtLastError() != cudaSuccess) return -1;
        launches += 6;
        return bfin ^ 1;
    }
    launch_emit_blocks<KeyT>(order, ptr<uint32_t>(c->offs), rec, cams, (int)c->n, fp.tile_w, fp.tile_h,
                             fp.tile_test, st, keys[0], vals[0], masks[0], emit_blocks, s);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    ++launches;
    SEELE_MARK_EXT(c, SEELE_STAGE_TILE_SORT);
    uint32_t* run = ptr<uint32_t>(c->ranges);
    const uint64_t units = f.units_total;
    const int fin = radix_sort_pairs<KeyT>(keys, vals, n_inst, (uint32_t)cap, f.tile_bits, false, scnt, soff, dtot,
                                           launches, s, run, run + units, f.blocks ? masks : nullptr);
    if (fin < 0) return -1;
    SEELE_MARK_EXT(c, SEELE_STAGE_RANGES);
    if (f.blocks) {
        launch_mask_summary(masks[fin], st, ptr<uint32_t>(c->msum), (uint32_t)(cap / 32 + 1), s);
        ++launches;
    }
    // CTAs take the units with the longest lists first (the persistent
    // rasterizer: camera group by camera group)
    if (f.queue)
        launch_view_order(run, run + units, (uint32_t)units, cams, f.ncam, f.blocks, f.batch_depth,
                          ptr<uint32_t>(c->border), s);
    else
        launch_block_order(run, run + units, (uint32_t)units, ptr<uint32_t>(c->border), s);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    ++launches;
    return fin;
}

bool tile_supported(int w, int h) {
    return (w == 8 && h == 8) || (w == 16 && h == 16) || (w == 32 && h == 8) || (w == 32 && h == 16);
}

seele_status check_options(seele_ctx* c, const seele_options* opt) {
    if (opt->mode != SEELE_MODE_PLAIN && opt->mode != SEELE_MODE_CR) return fail(c, SEELE_ERR_ARG, "bad mode");
    if (!tile_supported(opt->tile_w, opt->tile_h))
        return fail(c, SEELE_ERR_ARG, "tile size %dx%d not supported (8x8, 16x16, 32x8, 32x16)", opt->tile_w, opt->tile_h);
    if (opt->mode == SEELE_MODE_CR && !group_supported(opt->group_w, opt->group_h))
        return fail(c, SEELE_ERR_ARG, "pixel group %dx%d not supported (1x1, 2x2, 2x4, 4x4, 4x8)", opt->group_w, opt->group_h);
    if (!(opt->alpha_min > 0 && opt->alpha_min < opt->alpha_max && opt->alpha_max <= 1.0f))
        return fail(c, SEELE_ERR_ARG, "need 0 < alpha_min < alpha_max <= 1");
    if (!(opt->t_stop > 0 && opt->t_stop < 1)) return fail(c, SEELE_ERR_ARG, "need 0 < t_stop < 1");
    if (opt->cluster_filter && (c->n_clusters <= 0 || !c->has_mask))
        return fail(c, SEELE_ERR_STATE, "cluster_filter needs a scene with view clusters");
    if (opt->n_neighbors < 0) return fail(c, SEELE_ERR_ARG, "n_neighbors must be >= 0");
    if (opt->tile_test != SEELE_TILES_RECT && opt->tile_test != SEELE_TILES_ELLIPSE)
        return fail(c, SEELE_ERR_ARG, "bad tile_test");
    if (opt->binning != SEELE_BIN_TILES && opt->binning != SEELE_BIN_BLOCKS)
        return fail(c, SEELE_ERR_ARG, "bad binning");
    if (opt->schedule != SEELE_SCHEDULE_GRID && opt->schedule != SEELE_SCHEDULE_QUEUE)
        return fail(c, SEELE_ERR_ARG, "bad schedule");
    if (opt->batch_depth < 0) return fail(c, SEELE_ERR_ARG, "batch_depth must be >= 0");
    return SEELE_OK;
}

// Camera constants for the options' tile size (host only).
void build_cameras(seele_ctx* c, const seele_options* opt, uint64_t& tiles_total, uint64_t& blocks_total,
                   uint64_t& pix_total) {
    const int ncam = (int)c->cams.size();
    c->camdev.resize(ncam);
    tiles_total = 0;
    blocks_total = 0;
    pix_total = 0;
    for (int i = 0; i < ncam; ++i) {
        const seele_camera& k = c->cams[i];
        CamDev& d = c->camdev[i];
        std::memset(&d, 0, sizeof d);
        const float* w = k.world_to_cam;
        const float Rm[9] = {w[0], w[1], w[2], w[4], w[5], w[6], w[8], w[9], w[10]};
        const float t[3] = {w[3], w[7], w[11]};
        std::memcpy(d.R, Rm, sizeof Rm);
        std::memcpy(d.t, t, sizeof t);
        d.fx = k.fx;
        d.fy = k.fy;
        d.cx = k.cx;
        d.cy = k.cy;
        for (int j = 0; j < 3; ++j)
            d.campos[j] = (float)(-((double)Rm[j] * t[0] + (double)Rm[3 + j] * t[1] + (double)Rm[6 + j] * t[2]));
        d.lim_x = (float)(1.3 * k.width / (2.0 * k.fx));
        d.lim_y = (float)(1.3 * k.height / (2.0 * k.fy));
        d.near_z = k.near_z;
        d.W = k.width;
        d.H = k.height;
        d.tiles_x = (k.width + opt->tile_w - 1) / opt->tile_w;
        d.tiles_y = (k.height + opt->tile_h - 1) / opt->tile_h;
        d.tile_offset = (uint32_t)tiles_total;
        d.pix_offset = (uint32_t)pix_total;
        d.sel_bits = opt->cluster_filter ? select_clusters(c, k, opt->n_neighbors) : 0xffffffffu;
        d.blocks_x = (d.tiles_x + kBlockW - 1) / kBlockW;
        d.block_offset = (uint32_t)blocks_total;
        blocks_total += (uint64_t)d.blocks_x * ((d.tiles_y + kBlockH - 1) / kBlockH);
        tiles_total += (uint64_t)d.tiles_x * d.tiles_y;
        pix_total += (uint64_t)k.width * k.height;
    }
}

void fill_params(seele_ctx* c, const seele_options* opt, FrameInfo& f) {
    FrameParams& fp = f.fp;
    fp = FrameParams{};
    fp.n = (int32_t)c->n;
    fp.n_cams = f.ncam;
    fp.sh_degree = c->sh_degree;
    fp.tile_w = opt->tile_w;
    fp.tile_h = opt->tile_h;
    fp.opacity_filter = opt->opacity_filter ? 1 : 0;
    fp.tile_test = opt->tile_test == SEELE_TILES_ELLIPSE ? 1 : 0;
    fp.binning = (f.blocks || f.expand) ? 1 : 0;  // preprocessing counts the block instances
    fp.use_mask = opt->cluster_filter ? 1 : 0;
    fp.alpha_min = opt->alpha_min;
    fp.log_alpha_min = std::log(opt->alpha_min);
    fp.log2_alpha_min = std::log2(opt->alpha_min);
    fp.alpha_max = opt->alpha_max;
    fp.t_stop = opt->t_stop;
    fp.dilation = 0.3f;
    fp.frustum_slack = 1.3f;
    fp.n_tiles_total = (uint32_t)f.tiles_total;
    fp.n_shared = c->st.on ? c->st.n_shared : 0u;
    fp.slot_cap = c->st.on ? c->st.cap : 0u;
}

// Sizes every buffer of a frame at the current capacity (may allocate).
seele_status size_frame(seele_ctx* c, FrameInfo& f) {
    const uint64_t R = f.R, cap = f.cap;
    SEELE_CUDA(c, ensure(c->cams_dev, sizeof(CamDev) * f.ncam));
    SEELE_CUDA(c, ensure(c->rec, 16ull * kRecF4 * R));
    SEELE_CUDA(c, ensure(c->tiles, 4 * R));
    SEELE_CUDA(c, ensure(c->depth, 4 * R));
    for (int i = 0; i < 2; ++i) {
        SEELE_CUDA(c, ensure(c->visk[i], 4 * R));
        SEELE_CUDA(c, ensure(c->visv[i], 4 * R));
        SEELE_CUDA(c, ensure(c->instk[i], 4 * cap));
        SEELE_CUDA(c, ensure(c->instv[i], 4 * cap));
        if (f.blocks || f.expand) SEELE_CUDA(c, ensure(c->instm[i], 4 * (cap + 32)));  // whole 32-entry groups
    }
    if (f.expand) {
        SEELE_CUDA(c, ensure(c->blocks, 4 * R));
        const uint64_t chunks = (f.tiles_total + 31) / 32;
        SEELE_CUDA(c, ensure(c->branges, 8 * f.blocks_total));  // block list starts, then ends
        const uint64_t ids = expand_chunk_ids(cap, f.blocks_total);
        SEELE_CUDA(c, ensure(c->tcnt, 4 * 33 * chunks));        // tile counts (whole chunks), chunk totals
        SEELE_CUDA(c, ensure(c->toff, 4 * 32 * chunks));        // tile list starts
        SEELE_CUDA(c, ensure(c->emap, 4 * (ids - f.blocks_total)));  // later chunks -> block
        SEELE_CUDA(c, ensure(c->ecnt, 8 * 32 * ids));           // per-chunk tile counts, then their offsets
    }
    if (f.blocks) {
        SEELE_CUDA(c, ensure(c->blocks, 4 * R));
        SEELE_CUDA(c, ensure(c->msum, 4 * (cap / 32 + 2)));
    }
    SEELE_CUDA(c, ensure(c->border, 4 * f.units_total));
    SEELE_CUDA(c, ensure(c->offs, 4 * R));
    SEELE_CUDA(c, ensure(c->cnts, 4 * R));
    SEELE_CUDA(c, ensure(c->chunkv, 4 * (R / kChunkItems + 1)));
    SEELE_CUDA(c, ensure(c->chunks, 4 * (R / kChunkItems + 1)));
    SEELE_CUDA(c, ensure(c->ranges, 8 * f.units_total));  // starts[n_units], then ends[n_units]
    SEELE_CUDA(c, ensure(c->status, sizeof(DeviceStatus)));
    SEELE_CUDA(c, ensure(c->T, 4 * f.pix_total));
    SEELE_CUDA(c, ensure(c->nc, 4 * f.pix_total));
    SEELE_CUDA(c, ensure(c->viewt, 12ull * f.ncam + 8));
    if (!f.rgb_dev) SEELE_CUDA(c, ensure(c->rgb_tmp, 12 * f.pix_total));
    if (!f.blocks) {
        // transmittance checkpoints for the backward pass (tile binning)
        SEELE_CUDA(c, ensure(c->ckpt, 16ull * ((cap >> kCkptShift) + 2) * (uint64_t)f.fp.tile_w * f.fp.tile_h));
        SEELE_CUDA(c, ensure(c->cfin, 16 * f.pix_total));
    }
    // count matrices: the depth sort's 8-bit passes over R records, the tile
    // or block sort's passes over cap instances (one wide pass at 257 to
    // 1024 units with 16-bit keys)
    const int wide = radix_last_bits(f.expand ? f.block_bits : f.tile_bits, f.short_keys ? 2 : 4);
    f.cnt_words = std::max(radix_count_words((uint32_t)R), radix_count_words((uint32_t)cap, wide));
    SEELE_CUDA(c, ensure(c->sortcnt, 8ull * f.cnt_words));
    // digit totals of the sorts' passes (cleared every frame)
    SEELE_CUDA(c, ensure(c->digtot, 4 * kDigitTotalWords));
    return SEELE_OK;
}

// Copies the camera constants through a ring of pinned staging buffers; a
// slot is refilled only once its previous copy has run.
seele_status upload_cameras(seele_ctx* c) {
    auto& slot = c->cam_ring[c->cam_next];
    c->cam_next = (c->cam_next + 1) % 4;
    const size_t bytes = sizeof(CamDev) * c->camdev.size();
    if (!slot.done) SEELE_CUDA(c, cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming));
    if (slot.used) SEELE_CUDA(c, cudaEventSynchronize(slot.done));
    if (slot.cap < bytes) {
        if (slot.host) cudaFreeHost(slot.host);
        slot.host = nullptr;
        slot.cap = 0;
        SEELE_CUDA(c, cudaMallocHost(&slot.host, bytes));
        slot.cap = bytes;
    }
    std::memcpy(slot.host, c->camdev.data(), bytes);
    SEELE_CUDA(c, cudaMemcpyAsync(c->cams_dev.p, slot.host, bytes, cudaMemcpyHostToDevice, c->stream));
    SEELE_CUDA(c, cudaEventRecord(slot.done, c->stream));
    slot.used = true;
    return SEELE_OK;
}

// Everything a captured frame depends on besides the camera poses.
std::vector<uint64_t> graph_key(const seele_ctx* c, const seele_options* opt, const FrameInfo& f,
                                const float* rgb_target, const float* T_copy) {
    std::vector<uint64_t> k;
    k.push_back(c->scene_gen);
    k.push_back((uint64_t)f.ncam);
    for (const auto& cam : c->cams) k.push_back(((uint64_t)cam.width << 32) | (uint32_t)cam.height);
    seele_options o = *opt;
    o.flags = 0;
    uint64_t words[(sizeof o + 7) / 8] = {};
    std::memcpy(words, &o, sizeof o);
    for (uint64_t w : words) k.push_back(w);
    k.push_back(f.cap);
    k.push_back((uint64_t)(uintptr_t)rgb_target);
    k.push_back((uint64_t)(uintptr_t)T_copy);
    k.push_back((uint64_t)(uintptr_t)c->rec.p);
    k.push_back((uint64_t)(uintptr_t)c->instk[0].p);
    k.push_back((uint64_t)(uintptr_t)c->instm[0].p);
    k.push_back((uint64_t)(uintptr_t)c->border.p);
    k.push_back((uint64_t)(uintptr_t)c->ckpt.p);
    k.push_back((uint64_t)(uintptr_t)c->cfin.p);
    return k;
}

// Enqueues one frame on the context's stream: clears, kernels, status
// read-back.  Allocates nothing and never waits, so it can be captured.
seele_status enqueue_frame(seele_ctx* c, const seele_options* opt, const FrameInfo& f, float* rgb_target,
                           float* T_copy, bool count, int& launches, int& fin) {
    const uint64_t R = f.R, cap = f.cap, tiles_total = f.tiles_total, units_total = f.units_total;
    const int ncam = f.ncam;
    cudaStream_t s = c->stream;
    DeviceStatus* st = ptr<DeviceStatus>(c->status);
    uint32_t* dtot = ptr<uint32_t>(c->digtot);
    launches = 0;
    NvtxStages nvtx_stages;
#define SEELE_MARK(k)                                               \
    if ((k) < SEELE_NUM_STAGES) nvtx_stages.next(k);                \
    if (c->profiling) SEELE_CUDA(c, cudaEventRecord(c->ev[k], s))

    SEELE_CUDA(c, cudaMemsetAsync(st, 0, sizeof(DeviceStatus), s));
    SEELE_CUDA(c, cudaMemsetAsync(c->chunkv.p, 0, 4 * (R / kChunkItems + 1), s));
    SEELE_CUDA(c, cudaMemsetAsync(dtot, 0, 4 * kDigitTotalWords, s));
    SEELE_CUDA(c, cudaMemsetAsync(c->viewt.p, 0, 12ull * ncam + 8, s));
    SEELE_CUDA(c, cudaMemsetAsync(c->ranges.p, 0xff, 4 * units_total, s));
    SEELE_CUDA(c, cudaMemsetAsync(ptr<uint32_t>(c->ranges) + units_total, 0, 4 * units_total, s));
    if (f.expand) {
        SEELE_CUDA(c, cudaMemsetAsync(c->branges.p, 0xff, 4 * f.blocks_total, s));
        SEELE_CUDA(c, cudaMemsetAsync(ptr<uint32_t>(c->branges) + f.blocks_total, 0, 4 * f.blocks_total, s));
        SEELE_CUDA(c, cudaMemsetAsync(c->tcnt.p, 0, 4 * 33 * ((tiles_total + 31) / 32), s));
        SEELE_CUDA(c, cudaMemsetAsync(c->emap.p, 0xff, 4 * (expand_chunk_ids(cap, f.blocks_total) - f.blocks_total),
                                      s));
    }
    SEELE_MARK(SEELE_STAGE_PREPROCESS);
    SceneDev sc = scene_dev(c);
    if (c->scene_flags == SEELE_SCENE_BORROW && sc.means == nullptr) {
        const seele_scene_desc& b = c->borrowed;
        const int ncoef = (c->sh_degree + 1) * (c->sh_degree + 1);
        launch_repack((int)c->n, ncoef, b.means, b.log_scales, b.quats, b.opacity_logits, b.sh,
                      ptr<float4>(c->pos_logit), ptr<float4>(c->quat), ptr<float4>(c->log_scale), ptr<float4>(c->sh),
                      s);
        SEELE_LAUNCHED(c);
        ++launches;
    }
    sc.mask = c->has_mask ? (c->scene_flags == SEELE_SCENE_BORROW ? c->borrowed.cluster_mask
                                                                  : ptr<const uint32_t>(c->mask))
                          : nullptr;
    sc.veto = c->st.on ? ptr<const uint32_t>(c->veto) : nullptr;
    unsigned long long* vt = ptr<unsigned long long>(c->viewt);
    ProjOut po{ptr<float4>(c->rec), ptr<uint32_t>(c->tiles),
               (f.blocks || f.expand) ? ptr<uint32_t>(c->blocks) : nullptr, ptr<float>(c->depth), vt,
               ptr<uint32_t>(c->chunkv)};
    const CamDev* cams = ptr<const CamDev>(c->cams_dev);
    launch_preprocess(sc, cams, f.fp, po, s);
    SEELE_LAUNCHED(c);
    ++launches;

    // visible records -> (depth bits, id), then the stable depth sort
    SEELE_MARK(SEELE_STAGE_COMPACT);
    // with ids below 2^24 the sort values also carry the instance counts
    const uint32_t* cnt_src = (f.blocks || f.expand) ? po.blocks : po.tiles;
    const bool packed = R <= (1ull << kPackedIdBits);
    launch_compact_visible(cnt_src, packed, po.depth, (uint32_t)R, po.chunk_vis, ptr<uint32_t>(c->visk[0]),
                           ptr<uint32_t>(c->visv[0]), st, s);
    SEELE_LAUNCHED(c);
    ++launches;
    const uint32_t* n_vis = &st->n_visible;
    SEELE_MARK(SEELE_STAGE_DEPTH_SORT);
    uint32_t* scnt = ptr<uint32_t>(c->sortcnt);
    uint32_t* soff = scnt + f.cnt_words;
    {
        uint32_t* vk[2] = {ptr<uint32_t>(c->visk[0]), ptr<uint32_t>(c->visk[1])};
        uint32_t* vv[2] = {ptr<uint32_t>(c->visv[0]), ptr<uint32_t>(c->visv[1])};
        // positive fp32 depths order like their bit patterns, sign bit clear:
        // 31 bits; the last pass also lays the records' instance counts out
        // in depth order
        SortGather gather;
        gather.src = cnt_src;
        gather.out = ptr<uint32_t>(c->cnts);
        gather.packed = packed;
        if (radix_sort_pairs<uint32_t>(vk, vv, n_vis, (uint32_t)R, 31, false, scnt, soff, dtot, launches, s, nullptr,
                                       nullptr, nullptr, &gather) != 0)
            return fail(c, SEELE_ERR_CUDA, "depth sort launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    // sorted ids are back in buffer 0 after an even number of passes
    const uint32_t* order = ptr<uint32_t>(c->visv[0]);
    SEELE_MARK(SEELE_STAGE_TILE_SCAN);
    launch_scan_tiles(ptr<uint32_t>(c->cnts), ptr<uint32_t>(c->chunks), (uint32_t)R, ptr<uint32_t>(c->offs), st,
                      (uint32_t)std::min<uint64_t>(cap, 0xffffffffu), s);
    SEELE_LAUNCHED(c);
    launches += 2;
    const int emit_blocks = (int)std::max<uint64_t>(std::min<uint64_t>((R + 255) / 256, 8 * 152), 1);
    SEELE_MARK(SEELE_STAGE_EMIT);
    const uint32_t* n_inst = &st->n_inst_valid;
    if (f.short_keys)
        fin = enqueue_tile_sort<uint16_t>(c, f, order, po.rec, cams, st, n_inst, cap, emit_blocks,
                                          dtot + kDepthSortTotals, scnt, soff, launches, s);
    else
        fin = enqueue_tile_sort<uint32_t>(c, f, order, po.rec, cams, st, n_inst, cap, emit_blocks,
                                          dtot + kDepthSortTotals, scnt, soff, launches, s);
    if (fin < 0) return fail(c, SEELE_ERR_CUDA, "tile sort launch failed: %s", cudaGetErrorString(cudaGetLastError()));

    RasterArgs ra;
    ra.starts = ptr<uint32_t>(c->ranges);
    ra.ends = ptr<uint32_t>(c->ranges) + units_total;
    ra.inst_rec = ptr<uint32_t>(c->instv[fin]);
    ra.inst_mask = f.blocks ? ptr<uint32_t>(c->instm[fin]) : nullptr;
    ra.mask_summary = f.blocks ? ptr<uint32_t>(c->msum) : nullptr;
    ra.block_order = ptr<uint32_t>(c->border);
    ra.n_blocks = (uint32_t)f.blocks_total;
    ra.rec = ptr<float4>(c->rec);
    ra.cams = cams;
    ra.n_cams = ncam;
    ra.n_tiles = (uint32_t)tiles_total;
    ra.fp = f.fp;
    ra.cr = opt->mode == SEELE_MODE_CR;
    ra.group_w = opt->group_w;
    ra.group_h = opt->group_h;
    ra.out_rgb = rgb_target;
    ra.out_T = ptr<float>(c->T);
    ra.out_nc = ptr<uint32_t>(c->nc);
    ra.count_into = count ? st : nullptr;
    ra.status = st;
    ra.view_end = vt + 1;
    ra.view_done = reinterpret_cast<uint32_t*>(vt + 1 + ncam);
    const bool ckpt = !f.blocks && !count && c->skew_frac <= 0.0 && c->topk_k <= 0;
    ra.ckpt = ckpt ? ptr<float4>(c->ckpt) : nullptr;
    ra.cfin = ckpt ? ptr<float4>(c->cfin) : nullptr;
    ra.queue = (f.queue && !count) ? &st->queue : nullptr;
    SEELE_MARK(SEELE_STAGE_RASTER);
    if (c->skew_frac > 0.0) {
        uint32_t* sk = ptr<uint32_t>(c->skew);
        if (!launch_skew(ra.starts, ra.ends, ra.inst_rec, ra.rec, cams, ncam, ra.n_tiles, f.fp, c->skew_frac, sk,
                         sk + f.pix_total, sk + 2 * f.pix_total, reinterpret_cast<float*>(sk + 3 * f.pix_total),
                         sk + 4 * f.pix_total, s))
            return fail(c, SEELE_ERR_ARG, "no skew pass for these options");
    } else if (c->topk_k > 0) {
        if (!launch_topk(ra.starts, ra.ends, ra.inst_rec, ra.rec, cams, ncam, ra.n_tiles, f.fp, c->topk_k,
                         c->topk_cluster, c->topk_mask, s))
            return fail(c, SEELE_ERR_ARG, "no top-k pass for these options");
    } else if (!launch_raster_fwd(ra, s)) {
        return fail(c, SEELE_ERR_ARG, "no rasterizer for these options");
    }
    SEELE_LAUNCHED(c);
    ++launches;
    SEELE_MARK(SEELE_NUM_STAGES);
#undef SEELE_MARK
    if (T_copy) SEELE_CUDA(c, cudaMemcpyAsync(T_copy, c->T.p, 4 * f.pix_total, cudaMemcpyDeviceToDevice, s));
    SEELE_CUDA(c, cudaMemcpyAsync(c->h_status, st, sizeof(DeviceStatus), cudaMemcpyDeviceToHost, s));
    return SEELE_OK;
}

}  // namespace

extern "C" {

void seele_default_options(seele_options* o) {
    if (!o) return;
    o->mode = SEELE_MODE_PLAIN;
    o->group_w = 2;
    o->group_h = 2;
    o->tile_w = 16;
    o->tile_h = 16;
    o->opacity_filter = 0;
    o->cluster_filter = 0;
    o->n_neighbors = 3;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->t_stop = 1e-4f;
    o->flags = 0;
    o->tile_test = SEELE_TILES_ELLIPSE;
    o->binning = SEELE_BIN_BLOCKS;
    o->schedule = SEELE_SCHEDULE_GRID;
    o->batch_depth = 0;
}

seele_status seele_create(seele_ctx** out, int device, void* cuda_stream) {
    if (!out) return SEELE_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        (void)cudaGetLastError();
        return SEELE_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SEELE_ERR_CUDA;
    seele_ctx* c = new (std::nothrow) seele_ctx();
    if (!c) return SEELE_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMallocHost(&c->h_status, sizeof(DeviceStatus)) != cudaSuccess) {
        delete c;
        return SEELE_ERR_OOM;
    }
    std::memset(c->h_status, 0, sizeof(DeviceStatus));
    *out = c;
    return SEELE_OK;
}

void seele_destroy(seele_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    scene_unshare(c);
    DevBuf* all[] = {&c->pos_logit, &c->quat, &c->log_scale, &c->sh, &c->mask, &c->staging, &c->cams_dev,
                     &c->rec, &c->tiles, &c->depth, &c->visk[0], &c->visk[1], &c->visv[0],
                     &c->visv[1], &c->offs, &c->instk[0], &c->instk[1], &c->instv[0], &c->instv[1],
                     &c->ranges, &c->status, &c->hist, &c->digtot, &c->T, &c->nc, &c->rgb_tmp, &c->sortcnt,
                     &c->grad_rec, &c->blocks, &c->instm[0], &c->instm[1], &c->msum, &c->border, &c->chunkv,
                     &c->chunks, &c->vbuf, &c->cnts, &c->skew, &c->veto, &c->order, &c->unordered,
                     &c->order_scratch, &c->torder, &c->ckpt, &c->cfin, &c->bmap, &c->branges, &c->tcnt, &c->toff, &c->emap, &c->ecnt};
    for (DevBuf* b : all) release(*b);
    stream_release(c);
    release(c->viewt);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto& slot : c->cam_ring) {
        if (slot.host) cudaFreeHost(slot.host);
        if (slot.done) cudaEventDestroy(slot.done);
    }
    if (c->h_status) cudaFreeHost(c->h_status);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

seele_status seele_set_stream(seele_ctx* c, void* cuda_stream) {
    if (!c) return SEELE_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return SEELE_OK;
}

const char* seele_last_error(const seele_ctx* c) { return c ? c->err.c_str() : "null context"; }

seele_status seele_load_scene(seele_ctx* c, const seele_scene_desc* d) {
    const NvtxRange nvtx_call("seele_load_scene");
    if (!c) return SEELE_ERR_ARG;
    if (!d) return fail(c, SEELE_ERR_ARG, "scene descriptor is NULL");
    if (d->n < 1 || d->n > (int64_t)65535 * 256)
        return fail(c, SEELE_ERR_ARG, "n = %lld out of range (1 .. 16776960)", (long long)d->n);
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(c, SEELE_ERR_ARG, "sh_degree must be 0..3");
    if (!d->means || !d->log_scales || !d->quats || !d->opacity_logits || !d->sh)
        return fail(c, SEELE_ERR_ARG, "scene attribute pointer is NULL");
    const bool spatial = (d->flags & SEELE_SCENE_SPATIAL) != 0;
    const int32_t mode = d->flags & ~SEELE_SCENE_SPATIAL;
    if (mode != SEELE_SCENE_COPY && mode != SEELE_SCENE_BORROW)
        return fail(c, SEELE_ERR_ARG, "flags must be COPY or BORROW, optionally with SPATIAL");
    if (spatial && mode == SEELE_SCENE_BORROW) return fail(c, SEELE_ERR_ARG, "SPATIAL needs a COPY scene");
    if (d->n_clusters < 0 || d->n_clusters > 32) return fail(c, SEELE_ERR_ARG, "n_clusters must be 0..32");
    if (d->n_clusters > 0 && (!d->centroids || !(d->pos_scale > 0)))
        return fail(c, SEELE_ERR_ARG, "centroids and a positive pos_scale are required with clusters");
    SEELE_CUDA(c, cudaSetDevice(c->device));
    c->has_scene = false;
    c->rendered = false;
    ++c->scene_gen;
    stream_release(c);
    scene_unshare(c);
    const int64_t n = d->n;
    const int nc = (d->sh_degree + 1) * (d->sh_degree + 1);
    const int planes = (3 * nc + 3) / 4;
    SEELE_CUDA(c, ensure(c->pos_logit, 16 * n));
    SEELE_CUDA(c, ensure(c->quat, 16 * n));
    SEELE_CUDA(c, ensure(c->log_scale, 16 * n));
    SEELE_CUDA(c, ensure(c->sh, 16 * n * planes));
    c->has_mask = d->cluster_mask != nullptr;
    c->spatial = false;
    if (mode == SEELE_SCENE_BORROW) {
        const void* ps[] = {d->means, d->log_scales, d->quats, d->opacity_logits, d->sh};
        for (const void* p : ps)
            if (!is_device_ptr(p)) return fail(c, SEELE_ERR_ARG, "BORROW needs device pointers");
        if (d->cluster_mask && !is_device_ptr(d->cluster_mask))
            return fail(c, SEELE_ERR_ARG, "BORROW needs a device cluster_mask");
        c->borrowed = *d;
    } else {
        // the repack reads device and page-locked host attributes where they
        // are; other host attributes go through one device staging area
        const float* src[5] = {d->means, d->log_scales, d->quats, d->opacity_logits, d->sh};
        const size_t cnt[5] = {(size_t)n * 3, (size_t)n * 3, (size_t)n * 4, (size_t)n, (size_t)n * nc * 3};
        size_t stage_floats = 0;
        const float* direct[5];
        for (int i = 0; i < 5; ++i) {
            direct[i] = is_device_ptr(src[i]) ? src[i] : static_cast<const float*>(mapped_host(src[i]));
            if (!direct[i]) stage_floats += cnt[i];
        }
        if (stage_floats) SEELE_CUDA(c, ensure(c->staging, stage_floats * 4));
        const float* use[5];
        size_t off = 0;
        for (int i = 0; i < 5; ++i) {
            if (direct[i]) {
                use[i] = direct[i];
            } else {
                float* dst = ptr<float>(c->staging) + off;
                SEELE_CUDA(c, cudaMemcpyAsync(dst, src[i], cnt[i] * 4, cudaMemcpyHostToDevice, c->stream));
                use[i] = dst;
                off += cnt[i];
            }
        }
        // with SPATIAL the planes are built aside, then gathered in Morton order
        if (spatial) SEELE_CUDA(c, ensure(c->unordered, 16ull * n * (3 + planes)));
        float4* P0 = spatial ? ptr<float4>(c->unordered) : ptr<float4>(c->pos_logit);
        float4* P1 = spatial ? P0 + n : ptr<float4>(c->quat);
        float4* P2 = spatial ? P0 + 2 * n : ptr<float4>(c->log_scale);
        float4* P3 = spatial ? P0 + 3 * n : ptr<float4>(c->sh);
        launch_repack((int)n, nc, use[0], use[1], use[2], use[3], use[4], P0, P1, P2, P3, c->stream);
        SEELE_LAUNCHED(c);
        if (c->has_mask) {
            SEELE_CUDA(c, ensure(c->mask, 4 * n));
            SEELE_CUDA(c, cudaMemcpyAsync(c->mask.p, d->cluster_mask, 4 * n, cudaMemcpyDefault, c->stream));
        }
        if (spatial) {
            const seele_status r = spatial_order(c, n, planes);
            if (r != SEELE_OK) return r;
        }
        SEELE_CUDA(c, cudaStreamSynchronize(c->stream));
        if (spatial) release(c->unordered);
        c->spatial = spatial;
    }
    c->n = n;
    c->sh_degree = d->sh_degree;
    c->scene_flags = mode;
    c->n_clusters = d->n_clusters;
    c->pos_scale = d->pos_scale;
    c->centroids.assign(d->centroids ? d->centroids : nullptr, d->centroids ? d->centroids + 6 * d->n_clusters : nullptr);
    c->has_scene = true;
    return SEELE_OK;
}

seele_status seele_load_scene_streamed(seele_ctx* c, const seele_scene_desc* d, int32_t n_slots,
                                       int64_t slot_gaussians, int32_t ahead) {
    if (!c) return SEELE_ERR_ARG;
    if (!d) return fail(c, SEELE_ERR_ARG, "scene descriptor is NULL");
    if (d->flags != SEELE_SCENE_COPY) return fail(c, SEELE_ERR_ARG, "a streamed scene is copied (COPY)");
    if (d->n < 1 || d->n > (int64_t)65535 * 256)
        return fail(c, SEELE_ERR_ARG, "n = %lld out of range (1 .. 16776960)", (long long)d->n);
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(c, SEELE_ERR_ARG, "sh_degree must be 0..3");
    if (d->n_clusters < 1 || d->n_clusters > 32 || !d->cluster_mask || !d->centroids || !(d->pos_scale > 0))
        return fail(c, SEELE_ERR_ARG, "a streamed scene needs 1..32 view clusters, masks, centroids and pos_scale");
    if (n_slots < 1 || n_slots > 64) return fail(c, SEELE_ERR_ARG, "n_slots must be 1..64");
    if (slot_gaussians < 0) return fail(c, SEELE_ERR_ARG, "slot_gaussians must be >= 0");
    if (ahead < 1) return fail(c, SEELE_ERR_ARG, "ahead must be >= 1");
    const void* hp[] = {d->means, d->log_scales, d->quats, d->opacity_logits, d->sh, d->cluster_mask};
    for (const void* q : hp)
        if (!q || is_device_ptr(q)) return fail(c, SEELE_ERR_ARG, "a streamed scene is read from host memory");
    SEELE_CUDA(c, cudaSetDevice(c->device));
    SEELE_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_scene = false;
    c->rendered = false;
    ++c->scene_gen;
    stream_release(c);
    scene_unshare(c);
    auto& S = c->st;
    const int64_t n = d->n;
    const int C = d->n_clusters, nc = (d->sh_degree + 1) * (d->sh_degree + 1), np = (3 * nc + 3) / 4;
    const uint32_t all = C >= 32 ? 0xffffffffu : ((1u << C) - 1u);
    // segments: cluster k holds every Gaussian with bit k (a Gaussian of
    // several clusters is copied into each), the shared ones (every bit) last
    std::vector<std::vector<uint32_t>> seg(C + 1);
    for (int64_t g = 0; g < n; ++g) {
        const uint32_t m = d->cluster_mask[g] & all;
        if (m == 0u) continue;
        if (m == all) {
            seg[C].push_back((uint32_t)g);
            continue;
        }
        for (int k = 0; k < C; ++k)
            if ((m >> k) & 1u) seg[k].push_back((uint32_t)g);
    }
    S.planes = 3 + np;
    S.seg.assign(C + 2, 0);
    for (int k = 0; k <= C; ++k) S.seg[k + 1] = S.seg[k] + seg[k].size();
    S.copies = S.seg[C + 1];
    S.n_shared = (uint32_t)seg[C].size();
    // slot size: as asked, else the largest cluster (one chunk per cluster)
    uint64_t largest = 1;
    for (int k = 0; k < C; ++k) largest = std::max<uint64_t>(largest, seg[k].size());
    S.cap = (uint32_t)std::min<uint64_t>(slot_gaussians > 0 ? (uint64_t)slot_gaussians : largest, largest);
    S.chunk_begin.assign(C + 1, 0);
    for (int k = 0; k < C; ++k) {
        S.chunk_begin[k] = (int)S.chunk_cluster.size();
        for (size_t b = 0; b < seg[k].size(); b += S.cap) {
            S.chunk_cluster.push_back(k);
            S.chunk_at.push_back(S.seg[k] + b);
            S.chunk_n.push_back((uint32_t)std::min<size_t>(S.cap, seg[k].size() - b));
        }
    }
    S.chunk_begin[C] = (int)S.chunk_cluster.size();
    S.n_slots = n_slots;
    S.ahead = ahead;
    S.n_full = n;
    const uint64_t n_res = (uint64_t)S.n_shared + (uint64_t)n_slots * S.cap;
    SEELE_CUDA(c, cudaMallocHost(&S.host, 16 * (size_t)S.planes * std::max<size_t>(S.copies, 1)));
    SEELE_CUDA(c, cudaMallocHost(&S.host_mask, 4 * std::max<size_t>(S.copies, 1)));
    SEELE_CUDA(c, cudaMallocHost(&S.host_veto, 4 * std::max<size_t>(S.copies, 1)));
    // plane-major copies in the library's layout (planes of float4)
    for (int k = 0; k <= C; ++k)
        for (size_t i = 0; i < seg[k].size(); ++i) {
            const size_t at = S.seg[k] + i, g = seg[k][i];
            float4* H = S.host;
            H[at] = make_float4(d->means[3 * g], d->means[3 * g + 1], d->means[3 * g + 2], d->opacity_logits[g]);
            H[S.copies + at] = make_float4(d->quats[4 * g], d->quats[4 * g + 1], d->quats[4 * g + 2], d->quats[4 * g + 3]);
            H[2 * S.copies + at] =
                make_float4(d->log_scales[3 * g], d->log_scales[3 * g + 1], d->log_scales[3 * g + 2], 0.f);
            const float* sh = d->sh + g * 3 * nc;
            for (int j = 0; j < np; ++j) {
                float v[4];
                for (int q = 0; q < 4; ++q) v[q] = 4 * j + q < 3 * nc ? sh[4 * j + q] : 0.f;
                H[(size_t)(3 + j) * S.copies + at] = make_float4(v[0], v[1], v[2], v[3]);
            }
            const uint32_t m = d->cluster_mask[g] & all;
            S.host_mask[at] = k == C ? 0xffffffffu : (1u << k);
            S.host_veto[at] = k == C ? 0u : (m & ((1u << k) - 1u));
        }
    c->n = (int64_t)n_res;
    SEELE_CUDA(c, ensure(c->pos_logit, 16 * n_res));
    SEELE_CUDA(c, ensure(c->quat, 16 * n_res));
    SEELE_CUDA(c, ensure(c->log_scale, 16 * n_res));
    SEELE_CUDA(c, ensure(c->sh, 16 * n_res * np));
    SEELE_CUDA(c, ensure(c->mask, 4 * n_res));
    SEELE_CUDA(c, ensure(c->veto, 4 * n_res));
    SEELE_CUDA(c, cudaMemsetAsync(c->mask.p, 0, 4 * n_res, c->stream));
    SEELE_CUDA(c, cudaMemsetAsync(c->veto.p, 0, 4 * n_res, c->stream));
    const seele_status r = stream_copy(c, S.seg[C], S.n_shared, 0, S.n_shared, c->stream);
    if (r != SEELE_OK) return r;
    S.slot_cluster.assign(n_slots, -1);
    S.slot_async.assign(n_slots, false);
    S.slot_stamp.assign(n_slots, 0);
    S.slot_ready.assign(n_slots, nullptr);
    S.slot_used.assign(n_slots, nullptr);
    for (int s = 0; s < n_slots; ++s) {
        SEELE_CUDA(c, cudaEventCreateWithFlags(&S.slot_ready[s], cudaEventDisableTiming));
        SEELE_CUDA(c, cudaEventCreateWithFlags(&S.slot_used[s], cudaEventDisableTiming));
    }
    SEELE_CUDA(c, cudaStreamCreateWithFlags(&S.copy, cudaStreamNonBlocking));
    SEELE_CUDA(c, cudaStreamSynchronize(c->stream));
    S.on = true;
    c->spatial = false;
    c->sh_degree = d->sh_degree;
    c->scene_flags = SEELE_SCENE_COPY;
    c->has_mask = true;
    c->n_clusters = C;
    c->pos_scale = d->pos_scale;
    c->centroids.assign(d->centroids, d->centroids + 6 * C);
    c->has_scene = true;
    return SEELE_OK;
}

seele_status seele_share_scene(seele_ctx* dst, const seele_ctx* src_c) {
    if (!dst) return SEELE_ERR_ARG;
    if (!src_c || src_c == dst) return fail(dst, SEELE_ERR_ARG, "src must be another context");
    seele_ctx* src = const_cast<seele_ctx*>(src_c);   // only its ownership record changes
    if (src->device != dst->device) return fail(dst, SEELE_ERR_ARG, "src and dst are on different devices");
    if (!src->has_scene) return fail(dst, SEELE_ERR_STATE, "src holds no scene");
    if (src->st.on) return fail(dst, SEELE_ERR_STATE, "a streamed scene cannot be shared: its slots change every frame");
    SEELE_CUDA(dst, cudaSetDevice(dst->device));
    SEELE_CUDA(dst, dst->stream ? cudaStreamSynchronize(dst->stream) : cudaDeviceSynchronize());
    dst->has_scene = false;
    dst->rendered = false;
    ++dst->scene_gen;
    stream_release(dst);
    scene_unshare(dst);
    const int64_t n = src->n;
    if (src->scene_flags == SEELE_SCENE_COPY) {
        if (!src->shared) {
            auto h = std::make_shared<SharedScene>();
            h->device = src->device;
            for (int i = 0; i < 6; ++i) h->p[i] = scene_bufs(src, i)->p;
            src->shared = h;
        }
        for (int i = 0; i < 6; ++i) {
            release(*scene_bufs(dst, i));
            *scene_bufs(dst, i) = *scene_bufs(src, i);
        }
        dst->shared = src->shared;
    } else {
        // BORROW: the caller's arrays, repacked into dst's own planes per frame
        const int planes = (3 * (src->sh_degree + 1) * (src->sh_degree + 1) + 3) / 4;
        SEELE_CUDA(dst, ensure(dst->pos_logit, 16 * n));
        SEELE_CUDA(dst, ensure(dst->quat, 16 * n));
        SEELE_CUDA(dst, ensure(dst->log_scale, 16 * n));
        SEELE_CUDA(dst, ensure(dst->sh, 16 * n * planes));
        dst->borrowed = src->borrowed;
    }
    dst->n = n;
    dst->sh_degree = src->sh_degree;
    dst->scene_flags = src->scene_flags;
    dst->spatial = src->spatial;
    dst->has_mask = src->has_mask;
    dst->n_clusters = src->n_clusters;
    dst->pos_scale = src->pos_scale;
    dst->centroids = src->centroids;
    dst->has_scene = true;
    return SEELE_OK;
}

seele_status seele_get_stream_stats(const seele_ctx* c, seele_stream_stats* out) {
    if (!c || !out) return SEELE_ERR_ARG;
    seele_ctx* m = const_cast<seele_ctx*>(c);
    if (!c->st.on) return fail(m, SEELE_ERR_STATE, "no streamed scene loaded");
    const auto& S = c->st;
    const int64_t per = 16 * S.planes + 4;  // attribute planes and the cluster mask
    out->full_bytes = per * S.n_full;
    out->resident_bytes = (per + 4) * c->n;  // plus the precedence mask
    out->n_shared = S.n_shared;
    out->slot_capacity = S.cap;
    out->n_slots = S.n_slots;
    out->n_chunks = (int64_t)S.chunk_cluster.size();
    out->frames = (int64_t)S.frame;
    out->loads_sync = S.loads_sync;
    out->loads_prefetched = S.loads_prefetch;
    out->prefetch_hits = S.prefetch_hits;
    out->resident_hits = S.resident_hits;
    return SEELE_OK;
}

seele_status seele_set_cameras(seele_ctx* c, const seele_camera* cams, int32_t n) {
    if (!c) return SEELE_ERR_ARG;
    if (!cams || n < 1 || n > kMaxCams) return fail(c, SEELE_ERR_ARG, "need 1..%d cameras", kMaxCams);
    for (int i = 0; i < n; ++i) {
        const seele_camera& k = cams[i];
        if (k.width < 1 || k.height < 1 || k.width > 16384 || k.height > 16384)
            return fail(c, SEELE_ERR_ARG, "camera %d: size %dx%d out of range", i, k.width, k.height);
        if (!(k.fx > 0) || !(k.fy > 0) || !(k.near_z > 0))
            return fail(c, SEELE_ERR_ARG, "camera %d: fx, fy and near_z must be positive", i);
    }
    c->cams.assign(cams, cams + n);
    c->rendered = false;
    return SEELE_OK;
}

seele_status seele_synchronize(seele_ctx* c) {
    if (!c) return SEELE_ERR_ARG;
    SEELE_CUDA(c, cudaSetDevice(c->device));
    SEELE_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!c->status_pending) return SEELE_OK;
    c->status_pending = false;
    const DeviceStatus& h = *c->h_status;
    if (h.error == kErrCapacity) {
        c->capacity = std::max<uint64_t>(c->capacity, (uint64_t)h.n_instances + h.n_instances / 4 + 1024);
        c->rendered = false;
        return fail(c, SEELE_ERR_CAPACITY, "tile instances %u exceed capacity %u", h.n_instances, h.capacity);
    }
    if (h.error == kErrTimeout) {
        c->rendered = false;
        return fail(c, SEELE_ERR_TIMEOUT, "device wait gave up at site %u", h.timeout_site);
    }
    if (h.error == kErrInternal) {
        c->rendered = false;
        return fail(c, SEELE_ERR_INTERNAL, "device consistency check failed at site %u", h.timeout_site);
    }
    return SEELE_OK;
}

seele_status seele_render(seele_ctx* c, const seele_options* opt, float* out_rgb, float* out_T, seele_stats* stats) {
    const NvtxRange nvtx_call("seele_render");
    if (!c) return SEELE_ERR_ARG;
    if (!c->has_scene) return fail(c, SEELE_ERR_STATE, "no scene loaded");
    if (c->cams.empty()) return fail(c, SEELE_ERR_STATE, "no cameras set");
    if (!opt || !out_rgb) return fail(c, SEELE_ERR_ARG, "options and out_rgb are required");
    seele_status st0 = check_options(c, opt);
    if (st0 != SEELE_OK) return st0;
    const bool async = (opt->flags & SEELE_RENDER_ASYNC) != 0;
    const bool profile = (opt->flags & SEELE_RENDER_PROFILE) != 0;
    const bool count = (opt->flags & SEELE_RENDER_COUNT) != 0;
    const bool graph = (opt->flags & SEELE_RENDER_GRAPH) != 0;
    if ((async || graph) && (profile || count))
        return fail(c, SEELE_ERR_ARG, "PROFILE and COUNT need a synchronous render without GRAPH");
    SEELE_CUDA(c, cudaSetDevice(c->device));
    FrameInfo f;
    f.rgb_dev = is_device_ptr(out_rgb);
    f.T_dev = out_T ? is_device_ptr(out_T) : true;
    // host outputs are read back on the stream after the frame; only
    // page-locked ones asynchronously
    if ((async || graph) && ((!f.rgb_dev && !mapped_host(out_rgb)) || (!f.T_dev && !mapped_host(out_T))))
        return fail(c, SEELE_ERR_ARG, "ASYNC and GRAPH renders need device or page-locked host outputs");
    f.ncam = (int)c->cams.size();
    f.R = (uint64_t)c->n * f.ncam;
    if (f.R >= (1ull << 31)) return fail(c, SEELE_ERR_ARG, "cameras x Gaussians must be < 2^31");
    build_cameras(c, opt, f.tiles_total, f.blocks_total, f.pix_total);
    if (f.tiles_total >= (1ull << 31) || f.pix_total >= (1ull << 31))
        return fail(c, SEELE_ERR_ARG, "too many tiles or pixels in one render");
    if (c->st.on) {
        if (!opt->cluster_filter) return fail(c, SEELE_ERR_ARG, "a streamed scene renders with the cluster filter");
        const seele_status sp = stream_prepare(c);
        if (sp != SEELE_OK) return sp;
    }
    f.blocks = opt->binning == SEELE_BIN_BLOCKS;
    f.queue = opt->schedule == SEELE_SCHEDULE_QUEUE && f.ncam <= kViewOrderMaxCams;
    f.batch_depth = opt->batch_depth;
    f.units_total = f.blocks ? f.blocks_total : f.tiles_total;
    f.short_keys = f.units_total <= kShortKeyMaxTiles;
    f.tile_bits = std::max(1, bits_for(f.units_total > 0 ? f.units_total - 1 : 0));
    f.expand = !f.blocks;
    f.block_bits = std::max(1, bits_for(f.blocks_total > 0 ? f.blocks_total - 1 : 0));
    fill_params(c, opt, f);
    if (profile && !c->ev[0])
        for (cudaEvent_t& e : c->ev) SEELE_CUDA(c, cudaEventCreate(&e));
    c->profiling = profile;
    if (c->capacity == 0) c->capacity = std::max<uint64_t>(1u << 20, 4 * f.R);

    int retries = 0, launches = 0, fin = 0;
    for (int attempt = 0;; ++attempt) {
        f.cap = c->capacity;
        seele_status s1 = size_frame(c, f);
        if (s1 != SEELE_OK) return s1;
        s1 = upload_cameras(c);
        if (s1 != SEELE_OK) return s1;
        float* rgb_target = f.rgb_dev ? out_rgb : ptr<float>(c->rgb_tmp);
        float* T_copy = (out_T && f.T_dev) ? out_T : nullptr;
        if (graph) {
            const std::vector<uint64_t> key = graph_key(c, opt, f, rgb_target, T_copy);
            if (!c->gexec || key != c->gkey) {
                if (c->gexec) cudaGraphExecDestroy(c->gexec);  // freed once any replay in flight ends
                c->gexec = nullptr;
                if (!c->cap_stream) SEELE_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
                cudaStream_t user = c->stream;
                c->stream = c->cap_stream;
                if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    c->stream = user;
                    (void)cudaGetLastError();
                    return fail(c, SEELE_ERR_CUDA, "stream capture could not begin");
                }
                const seele_status se = enqueue_frame(c, opt, f, rgb_target, T_copy, false, launches, fin);
                cudaGraph_t g = nullptr;
                const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
                c->stream = user;
                if (se != SEELE_OK) {
                    if (g) cudaGraphDestroy(g);
                    return se;
                }
                if (ee != cudaSuccess || !g) {
                    (void)cudaGetLastError();
                    return fail(c, SEELE_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ee));
                }
                const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
                cudaGraphDestroy(g);
                if (ei != cudaSuccess) {
                    (void)cudaGetLastError();
                    c->gexec = nullptr;
                    return fail(c, SEELE_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
                }
                c->gkey = key;
                c->g_launches = launches;
                c->g_fin = fin;
            }
            SEELE_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
            launches = c->g_launches;
            fin = c->g_fin;
        } else {
            const seele_status se = enqueue_frame(c, opt, f, rgb_target, T_copy, count, launches, fin);
            if (se != SEELE_OK) return se;
        }
        c->inst_final = fin;
        c->n_tiles_total = (uint32_t)f.tiles_total;
        c->n_units_total = (uint32_t)f.units_total;
        c->n_pix_total = f.pix_total;
        c->last_opt = *opt;
        c->last_fp = f.fp;
        // the frame (enqueued or replayed) wrote checkpoints for the backward pass
        c->ckpt_valid = !f.blocks && !count && c->skew_frac <= 0.0 && c->topk_k <= 0;
        c->ckpt_slots = (f.cap >> kCkptShift) + 2;
        c->border_tiles = !f.blocks && !f.queue;
        if (!f.rgb_dev)
            SEELE_CUDA(c, cudaMemcpyAsync(out_rgb, c->rgb_tmp.p, 12 * f.pix_total, cudaMemcpyDeviceToHost, c->stream));
        if (out_T && !f.T_dev)
            SEELE_CUDA(c, cudaMemcpyAsync(out_T, c->T.p, 4 * f.pix_total, cudaMemcpyDeviceToHost, c->stream));
        if (async) {
            c->status_pending = true;
            c->rendered = true;
            break;
        }
        SEELE_CUDA(c, cudaStreamSynchronize(c->stream));
        const DeviceStatus& h = *c->h_status;
        // grow to what the overflowing stage counted and render again; with
        // tile binning the block instances and then the (more numerous) tile
        // instances can each overflow once
        if (h.error == kErrCapacity && attempt < 2) {
            c->capacity = std::max<uint64_t>(c->capacity, (uint64_t)h.n_instances + h.n_instances / 4 + 1024);
            ++retries;
            continue;
        }
        if (h.error == kErrCapacity) return fail(c, SEELE_ERR_CAPACITY, "capacity still exceeded after growth");
        if (h.error == kErrTimeout) return fail(c, SEELE_ERR_TIMEOUT, "device wait gave up at site %u", h.timeout_site);
        if (h.error == kErrInternal)
            return fail(c, SEELE_ERR_INTERNAL, "device consistency check failed at site %u", h.timeout_site);
        c->rendered = true;
        break;
    }

    if (c->st.on) {
        const seele_status sp = stream_prefetch(c, opt->n_neighbors);
        if (sp != SEELE_OK) return sp;
    }
    if (stats) {
        std::memset(stats->stage_ms, 0, sizeof stats->stage_ms);
        if (profile)
            for (int k = 0; k < SEELE_NUM_STAGES; ++k)
                SEELE_CUDA(c, cudaEventElapsedTime(&stats->stage_ms[k], c->ev[k], c->ev[k + 1]));
        stats->leader_tests = count ? (int64_t)c->h_status->work[0] : 0;
        stats->pairs_evaluated = count ? (int64_t)c->h_status->work[1] : 0;
        stats->pairs_blended = count ? (int64_t)c->h_status->work[2] : 0;
        stats->n_visible = async ? -1 : (int64_t)c->h_status->n_visible;
        stats->n_instances = async ? -1 : (int64_t)c->h_status->n_instances;
        stats->capacity = (int64_t)c->capacity;
        stats->retries = retries;
        stats->n_kernels = launches;
    }
    return SEELE_OK;
}

seele_status seele_get_view_times(const seele_ctx* c, float* out_ms, int32_t n) {
    if (!c || !out_ms) return SEELE_ERR_ARG;
    seele_ctx* m = const_cast<seele_ctx*>(c);
    if (!c->rendered) return fail(m, SEELE_ERR_STATE, "no completed render");
    const int ncam = (int)c->cams.size();
    if (n != ncam) return fail(m, SEELE_ERR_ARG, "n must equal the number of cameras (%d)", ncam);
    SEELE_CUDA(m, cudaSetDevice(c->device));
    SEELE_CUDA(m, cudaStreamSynchronize(c->stream));
    std::vector<unsigned long long> t(1 + ncam);
    SEELE_CUDA(m, cudaMemcpy(t.data(), c->viewt.p, 8ull * (1 + ncam), cudaMemcpyDeviceToHost));
    for (int i = 0; i < ncam; ++i) out_ms[i] = t[1 + i] >= t[0] ? (float)((t[1 + i] - t[0]) * 1e-6) : 0.f;
    return SEELE_OK;
}

seele_status seele_autotune(seele_ctx* c, seele_options* inout, float* best_ms) {
    const NvtxRange nvtx_call("seele_autotune");
    if (!c || !inout) return SEELE_ERR_ARG;
    if (!c->has_scene || c->cams.empty()) return fail(c, SEELE_ERR_STATE, "autotune needs a scene and cameras");
    static const int shapes[][2] = {{16, 16}, {32, 8}, {32, 16}, {8, 8}};
    std::vector<float> out;
    size_t pix = 0;
    for (const auto& k : c->cams) pix += (size_t)k.width * k.height;
    float* dev_out = nullptr;
    if (cudaMalloc(&dev_out, 12 * pix) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, SEELE_ERR_OOM, "autotune output buffer");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = INFINITY;
    int bw = inout->tile_w, bh = inout->tile_h;
    seele_status result = SEELE_OK;
    for (const auto& sh : shapes) {
        seele_options o = *inout;
        o.tile_w = sh[0];
        o.tile_h = sh[1];
        o.flags = 0;
        seele_status st = SEELE_OK;
        for (int w = 0; w < 2 && st == SEELE_OK; ++w) st = seele_render(c, &o, dev_out, nullptr, nullptr);
        if (st != SEELE_OK) {
            result = st;
            break;
        }
        o.flags = SEELE_RENDER_ASYNC;
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 5 && st == SEELE_OK; ++r) st = seele_render(c, &o, dev_out, nullptr, nullptr);
        cudaEventRecord(e1, c->stream);
        if (st == SEELE_OK) st = seele_synchronize(c);
        if (st != SEELE_OK) {
            result = st;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 5.f;
        if (ms < best) {
            best = ms;
            bw = sh[0];
            bh = sh[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dev_out);
    if (result != SEELE_OK) return result;
    inout->tile_w = bw;
    inout->tile_h = bh;
    if (best_ms) *best_ms = best;
    c->rendered = false;
    return SEELE_OK;
}

// The batched multi-view autotuner: tile shape (GRID, batch time), then
// schedule and batch depth for the objective; see seele.h.
seele_status seele_autotune_ex(seele_ctx* c, seele_options* inout, int32_t objective, const char* cache_path,
                               seele_tune_result* result) {
    const NvtxRange nvtx_call("seele_autotune_ex");
    if (!c || !inout) return SEELE_ERR_ARG;
    if (objective < SEELE_TUNE_BATCH_MS || objective > SEELE_TUNE_VIEW_P99)
        return fail(c, SEELE_ERR_ARG, "bad objective");
    if (!c->has_scene || c->cams.empty()) return fail(c, SEELE_ERR_STATE, "autotune needs a scene and cameras");
    seele_status st0 = check_options(c, inout);
    if (st0 != SEELE_OK) return st0;
    SEELE_CUDA(c, cudaSetDevice(c->device));
    const int ncam = (int)c->cams.size();
    // cache key: device, scene size bucket, resolutions, work-shaping options, objective
    std::string key;
    {
        cudaDeviceProp prop{};
        SEELE_CUDA(c, cudaGetDeviceProperties(&prop, c->device));
        std::string name = prop.name;
        for (char& ch : name)
            if (ch == '"' || ch == '\\' || ch == ' ') ch = '_';
        int lg = 0;
        while ((1ll << lg) < c->n) ++lg;
        std::vector<std::pair<int, int>> res;
        for (const auto& k : c->cams) res.push_back({k.width, k.height});
        std::sort(res.begin(), res.end());
        char buf[256];
        std::snprintf(buf, sizeof buf, "%s|sm%d|n2^%d|deg%d|mode%d|g%dx%d|op%d|cl%d|bin%d|tt%d|obj%d|cams", name.c_str(),
                      prop.multiProcessorCount, lg, c->sh_degree, inout->mode, inout->group_w, inout->group_h,
                      inout->opacity_filter, inout->cluster_filter, inout->binning, inout->tile_test, objective);
        key = buf;
        for (size_t i = 0; i < res.size();) {
            size_t j = i;
            while (j < res.size() && res[j] == res[i]) ++j;
            std::snprintf(buf, sizeof buf, ":%dx%dx%d", (int)(j - i), res[i].first, res[i].second);
            key += buf;
            i = j;
        }
    }
    seele_tune_result r{};
    TuneEntry hit;
    if (tune_cache_lookup(cache_path, key, &hit)) {
        inout->tile_w = hit.tile_w;
        inout->tile_h = hit.tile_h;
        inout->schedule = hit.schedule;
        inout->batch_depth = hit.batch_depth;
        r.batch_ms = hit.batch_ms;
        r.view_p50_ms = hit.p50_ms;
        r.view_p99_ms = hit.p99_ms;
        r.from_cache = 1;
        if (result) *result = r;
        return SEELE_OK;
    }
    size_t pix = 0;
    for (const auto& k : c->cams) pix += (size_t)k.width * k.height;
    float* dev_out = nullptr;
    if (cudaMalloc(&dev_out, 12 * pix) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, SEELE_ERR_OOM, "autotune output buffer");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    struct Measured {
        float batch = INFINITY, p50 = INFINITY, p99 = INFINITY;
        float score(int obj) const { return obj == SEELE_TUNE_VIEW_P50 ? p50 : obj == SEELE_TUNE_VIEW_P99 ? p99 : batch; }
    };
    std::vector<float> views(ncam);
    auto measure = [&](seele_options o, Measured* m) -> seele_status {
        o.flags = 0;
        seele_status st = SEELE_OK;
        for (int w = 0; w < 2 && st == SEELE_OK; ++w) st = seele_render(c, &o, dev_out, nullptr, nullptr);
        o.flags = SEELE_RENDER_ASYNC | SEELE_RENDER_GRAPH;
        if (st == SEELE_OK) st = seele_render(c, &o, dev_out, nullptr, nullptr);  // captures the graph
        if (st == SEELE_OK) st = seele_synchronize(c);
        if (st != SEELE_OK) return st;
        cudaEventRecord(e0, c->stream);
        for (int k = 0; k < 5 && st == SEELE_OK; ++k) st = seele_render(c, &o, dev_out, nullptr, nullptr);
        cudaEventRecord(e1, c->stream);
        if (st == SEELE_OK) st = seele_synchronize(c);
        if (st != SEELE_OK) return st;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        m->batch = ms / 5.f;
        std::vector<float> all;
        for (int k = 0; k < 3 && st == SEELE_OK; ++k) {
            st = seele_render(c, &o, dev_out, nullptr, nullptr);
            if (st == SEELE_OK) st = seele_get_view_times(c, views.data(), ncam);
            all.insert(all.end(), views.begin(), views.end());
        }
        if (st != SEELE_OK) return st;
        std::sort(all.begin(), all.end());
        m->p50 = all[all.size() / 2];
        m->p99 = all[std::min(all.size() - 1, (size_t)std::ceil(0.99 * all.size()) - 1)];
        ++r.candidates;
        return SEELE_OK;
    };
    seele_status status = SEELE_OK;
    seele_options best = *inout;
    Measured bm;
    // stage 1: the tile shape, GRID schedule, batch time
    static const int shapes[][2] = {{16, 16}, {32, 8}, {32, 16}, {8, 8}};
    for (const auto& sh : shapes) {
        seele_options o = *inout;
        o.tile_w = sh[0];
        o.tile_h = sh[1];
        o.schedule = SEELE_SCHEDULE_GRID;
        o.batch_depth = 0;
        Measured m;
        status = measure(o, &m);
        if (status != SEELE_OK) break;
        if (m.batch < bm.batch) {
            bm = m;
            best = o;
        }
    }
    // stage 2: schedule and batch depth with that shape, for the objective
    if (status == SEELE_OK && ncam <= kViewOrderMaxCams) {
        std::vector<int> depths = {0};
        for (int d = ncam / 2; d >= 1 && depths.size() < 8; d /= 2) depths.push_back(d);
        const seele_options base = best;
        for (int d : depths) {
            seele_options o = base;
            o.schedule = SEELE_SCHEDULE_QUEUE;
            o.batch_depth = d;
            Measured m;
            status = measure(o, &m);
            if (status != SEELE_OK) break;
            if (m.score(objective) < bm.score(objective)) {
                bm = m;
                best = o;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dev_out);
    c->rendered = false;
    if (status != SEELE_OK) return status;
    inout->tile_w = best.tile_w;
    inout->tile_h = best.tile_h;
    inout->schedule = best.schedule;
    inout->batch_depth = best.batch_depth;
    r.batch_ms = bm.batch;
    r.view_p50_ms = bm.p50;
    r.view_p99_ms = bm.p99;
    if (result) *result = r;
    if (cache_path) {
        TuneEntry e;
        e.tile_w = best.tile_w;
        e.tile_h = best.tile_h;
        e.schedule = best.schedule;
        e.batch_depth = best.batch_depth;
        e.batch_ms = bm.batch;
        e.p50_ms = bm.p50;
        e.p99_ms = bm.p99;
        if (!tune_cache_store(cache_path, key, e)) return fail(c, SEELE_ERR_ARG, "cannot write the cache file");
    }
    return SEELE_OK;
}

seele_status seele_render_backward(seele_ctx* c, const float* dL_drgb, const seele_grads* g) {
    const NvtxRange nvtx_call("seele_render_backward");
    if (!c) return SEELE_ERR_ARG;
    if (!c->rendered) return fail(c, SEELE_ERR_STATE, "no render to differentiate");
    if (c->st.on) return fail(c, SEELE_ERR_STATE, "gradients need the whole scene resident (seele_load_scene)");
    if (!dL_drgb || !g || !g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh)
        return fail(c, SEELE_ERR_ARG, "dL_drgb and every gradient buffer are required");
    SEELE_CUDA(c, cudaSetDevice(c->device));
    const void* dev_ptrs[] = {dL_drgb, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh};
    for (const void* p : dev_ptrs)
        if (!is_device_ptr(p)) return fail(c, SEELE_ERR_ARG, "backward buffers must be device memory");
    if (c->last_opt.binning == SEELE_BIN_BLOCKS) {
        // the backward walks per-tile lists: bin the same frame by tiles
        // (same image, same per-pixel list positions) and continue from it
        seele_options o = c->last_opt;
        o.binning = SEELE_BIN_TILES;
        o.flags = 0;
        SEELE_CUDA(c, ensure(c->rgb_tmp, 12 * c->n_pix_total));
        const seele_status r = seele_render(c, &o, ptr<float>(c->rgb_tmp), nullptr, nullptr);
        if (r != SEELE_OK) return r;
    }
    const int ncam = (int)c->cams.size();
    const uint64_t R = (uint64_t)c->n * ncam;
    SEELE_CUDA(c, ensure(c->grad_rec, 48 * R));
    cudaStream_t s = c->stream;
    SEELE_CUDA(c, cudaMemsetAsync(c->grad_rec.p, 0, 48 * R, s));
    RasterBwdArgs a;
    a.starts = ptr<uint32_t>(c->ranges);
    a.ends = ptr<uint32_t>(c->ranges) + c->n_tiles_total;
    a.inst_rec = ptr<uint32_t>(c->instv[c->inst_final]);
    a.rec = ptr<float4>(c->rec);
    a.cams = ptr<const CamDev>(c->cams_dev);
    a.n_cams = ncam;
    a.n_tiles = c->n_tiles_total;
    a.fp = c->last_fp;
    a.cr = c->last_opt.mode == SEELE_MODE_CR;
    a.group_w = c->last_opt.group_w;
    a.group_h = c->last_opt.group_h;
    a.dL_drgb = dL_drgb;
    a.T_final = ptr<float>(c->T);
    a.n_contrib = ptr<uint32_t>(c->nc);
    a.grad_rec = ptr<float>(c->grad_rec);
    // tiles with the longest lists first, as in the forward pass (whose
    // order of these very ranges is reused when it made one)
    if (c->border_tiles) {
        a.tile_order = ptr<const uint32_t>(c->border);
    } else {
        SEELE_CUDA(c, ensure(c->torder, 4ull * c->n_tiles_total));
        launch_block_order(a.starts, a.ends, c->n_tiles_total, ptr<uint32_t>(c->torder), s);
        SEELE_LAUNCHED(c);
        a.tile_order = ptr<const uint32_t>(c->torder);
    }
    // long lists are walked in kCkptL-entry chunks from the forward pass's
    // checkpoints, one CTA each
    a.ckpt = nullptr;
    a.cfin = nullptr;
    a.chunk_map = nullptr;
    a.n_map = 0;
    if (c->ckpt_valid) {
        a.n_map = (uint32_t)c->ckpt_slots;
        SEELE_CUDA(c, ensure(c->bmap, 4ull * a.n_map));
        SEELE_CUDA(c, cudaMemsetAsync(c->bmap.p, 0xff, 4ull * a.n_map, s));
        launch_chunk_map(a.starts, a.ends, c->n_tiles_total, ptr<uint32_t>(c->bmap), a.n_map, s);
        SEELE_LAUNCHED(c);
        a.ckpt = ptr<const float4>(c->ckpt);
        a.cfin = ptr<const float4>(c->cfin);
        a.chunk_map = ptr<const uint32_t>(c->bmap);
    }
    if (!launch_raster_bwd(a, s)) return fail(c, SEELE_ERR_ARG, "no backward rasterizer for these options");
    SEELE_LAUNCHED(c);
    SceneDev sc = scene_dev(c);
    sc.mask = nullptr;
    launch_preprocess_bwd(sc, a.cams, c->last_fp, ptr<uint32_t>(c->tiles), a.grad_rec, g->means, g->log_scales,
                          g->quats, g->opacity_logits, g->sh, c->spatial ? ptr<const uint32_t>(c->order) : nullptr,
                          s);
    SEELE_LAUNCHED(c);
    return SEELE_OK;
}

seele_status seele_get_debug_view(const seele_ctx* c, seele_debug_view* out) {
    if (!c || !out) return SEELE_ERR_ARG;
    if (!c->rendered) return SEELE_ERR_STATE;
    seele_ctx* m = const_cast<seele_ctx*>(c);
    std::memset(out, 0, sizeof *out);
    out->n_records = (int64_t)c->n * (int64_t)c->cams.size();
    out->n_visible = c->h_status->n_visible;
    out->n_instances = c->h_status->n_inst_valid;
    const bool blk = c->last_opt.binning == SEELE_BIN_BLOCKS;
    out->n_tiles = c->n_units_total;
    out->inst_record = ptr<const uint32_t>(m->instv[c->inst_final]);
    out->tile_start = ptr<const uint32_t>(m->ranges);
    out->tile_end = ptr<const uint32_t>(m->ranges) + c->n_units_total;
    out->inst_mask = blk ? ptr<const uint32_t>(m->instm[c->inst_final]) : nullptr;
    out->tiles_touched = ptr<const uint32_t>(m->tiles);
    out->records = ptr<const float>(m->rec);
    out->depth = ptr<const float>(m->depth);
    out->n_contrib = ptr<const uint32_t>(m->nc);
    out->scene_order = c->spatial ? ptr<const uint32_t>(m->order) : nullptr;
    out->mask_summary = blk ? ptr<const uint32_t>(m->msum) : nullptr;
    return SEELE_OK;
}

seele_status seele_contribution_skew(seele_ctx* c, const seele_options* opt, float frac, uint32_t* out_m,
                                     uint32_t* out_blended, uint32_t* out_walked, float* out_total,
                                     uint32_t* out_listed) {
    const NvtxRange nvtx_call("seele_contribution_skew");
    if (!c) return SEELE_ERR_ARG;
    if (!c->has_scene) return fail(c, SEELE_ERR_STATE, "no scene loaded");
    if (c->st.on) return fail(c, SEELE_ERR_STATE, "the skew statistic needs the whole scene resident");
    if (c->cams.empty()) return fail(c, SEELE_ERR_STATE, "no cameras");
    if (!(frac > 0.f && frac <= 1.f)) return fail(c, SEELE_ERR_ARG, "frac must be in (0, 1]");
    if (!out_m || !out_blended || !out_walked || !out_total) return fail(c, SEELE_ERR_ARG, "every output is required");
    SEELE_CUDA(c, cudaSetDevice(c->device));
    seele_options o;
    if (opt) o = *opt;
    else seele_default_options(&o);
    o.mode = SEELE_MODE_PLAIN;
    o.opacity_filter = 0;
    o.cluster_filter = 0;
    o.binning = SEELE_BIN_TILES;
    o.flags = 0;
    uint64_t pix = 0;
    for (const auto& cam : c->cams) pix += (uint64_t)cam.width * cam.height;
    SEELE_CUDA(c, ensure(c->skew, 20 * pix));
    SEELE_CUDA(c, ensure(c->rgb_tmp, 12 * pix));
    c->skew_frac = frac;
    const seele_status r = seele_render(c, &o, ptr<float>(c->rgb_tmp), nullptr, nullptr);
    c->skew_frac = 0.0;
    c->rendered = false;
    if (r != SEELE_OK) return r;
    cudaStream_t s = c->stream;
    const uint32_t* sk = ptr<uint32_t>(c->skew);
    SEELE_CUDA(c, cudaMemcpyAsync(out_m, sk, 4 * pix, cudaMemcpyDefault, s));
    SEELE_CUDA(c, cudaMemcpyAsync(out_blended, sk + pix, 4 * pix, cudaMemcpyDefault, s));
    SEELE_CUDA(c, cudaMemcpyAsync(out_walked, sk + 2 * pix, 4 * pix, cudaMemcpyDefault, s));
    SEELE_CUDA(c, cudaMemcpyAsync(out_total, sk + 3 * pix, 4 * pix, cudaMemcpyDefault, s));
    if (out_listed) SEELE_CUDA(c, cudaMemcpyAsync(out_listed, sk + 4 * pix, 4 * pix, cudaMemcpyDefault, s));
    SEELE_CUDA(c, cudaStreamSynchronize(s));
    return SEELE_OK;
}

seele_status seele_build_view_clusters(seele_ctx* c, const seele_camera* poses, int32_t n_poses, int32_t n_clusters,
                                       int32_t top_k, const double* uniforms, int32_t max_iter, float* out_centroids,
                                       float* out_pos_scale, uint32_t* out_mask, int32_t* out_assign) {
    const NvtxRange nvtx_call("seele_build_view_clusters");
    if (!c) return SEELE_ERR_ARG;
    if (!c->has_scene) return fail(c, SEELE_ERR_STATE, "no scene loaded");
    if (c->st.on) return fail(c, SEELE_ERR_STATE, "the builder needs the whole scene resident");
    if (!poses || !uniforms || !out_centroids || !out_pos_scale || !out_mask)
        return fail(c, SEELE_ERR_ARG, "poses, uniforms and the outputs are required");
    if (n_clusters < 1 || n_clusters > 32 || n_poses < n_clusters)
        return fail(c, SEELE_ERR_ARG, "need 1 <= n_clusters <= 32 and n_poses >= n_clusters");
    if (top_k < 1 || top_k > 64) return fail(c, SEELE_ERR_ARG, "top_k must be in [1, 64]");
    if (max_iter < 0) return fail(c, SEELE_ERR_ARG, "max_iter must be >= 0");
    for (int j = 0; j < n_clusters; ++j)
        if (!(uniforms[j] >= 0.0 && uniforms[j] < 1.0)) return fail(c, SEELE_ERR_ARG, "uniforms must lie in [0, 1)");
    for (int i = 0; i < n_poses; ++i)
        if (poses[i].width < 1 || poses[i].height < 1 || poses[i].width > 16384 || poses[i].height > 16384)
            return fail(c, SEELE_ERR_ARG, "pose %d: bad image size", i);
    SEELE_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t s = c->stream;

    // pose features (x / s, v), s = the largest camera distance of the samples
    std::vector<double> feat(6 * (size_t)n_poses);
    double scale = 0.0;
    for (int i = 0; i < n_poses; ++i) {
        const float* w = poses[i].world_to_cam;
        const double R[9] = {w[0], w[1], w[2], w[4], w[5], w[6], w[8], w[9], w[10]};
        const double t[3] = {w[3], w[7], w[11]};
        for (int a = 0; a < 3; ++a) feat[6 * i + a] = -(R[a] * t[0] + R[3 + a] * t[1] + R[6 + a] * t[2]);
        for (int a = 0; a < 3; ++a) feat[6 * i + 3 + a] = R[6 + a];
        scale = std::max(scale, std::sqrt(feat[6 * i] * feat[6 * i] + feat[6 * i + 1] * feat[6 * i + 1] +
                                          feat[6 * i + 2] * feat[6 * i + 2]));
    }
    if (!(scale > 0.0)) return fail(c, SEELE_ERR_ARG, "every pose sits at the origin");
    for (int i = 0; i < n_poses; ++i)
        for (int a = 0; a < 3; ++a) feat[6 * i + a] /= scale;

    // device layout: features, uniforms, centroids, assignment, seeding scratch,
    // iteration count, then the per-camera clusters of a batch and the mask
    const size_t nf = 6 * (size_t)n_poses, nk = (size_t)n_clusters;
    const size_t off_u = 8 * nf, off_c = off_u + 8 * nk, off_a = off_c + 48 * nk;
    const size_t off_d = off_a + 8 * (size_t)n_poses, off_it = off_d + 8 * (size_t)n_poses;
    const size_t off_cl = off_it + 16, off_m = off_cl + 4 * (size_t)kMaxCams + 256;
    SEELE_CUDA(c, ensure(c->vbuf, off_m + 4 * (size_t)c->n + 16));
    unsigned char* vb = static_cast<unsigned char*>(c->vbuf.p);
    SEELE_CUDA(c, cudaMemcpyAsync(vb, feat.data(), 8 * nf, cudaMemcpyHostToDevice, s));
    SEELE_CUDA(c, cudaMemcpyAsync(vb + off_u, uniforms, 8 * nk, cudaMemcpyHostToDevice, s));
    launch_kmeans(reinterpret_cast<double*>(vb), n_poses, n_clusters, reinterpret_cast<double*>(vb + off_u),
                  max_iter, reinterpret_cast<double*>(vb + off_c), reinterpret_cast<int*>(vb + off_a),
                  reinterpret_cast<double*>(vb + off_d), reinterpret_cast<int*>(vb + off_it), s);
    SEELE_LAUNCHED(c);
    std::vector<double> cent(6 * nk);
    std::vector<int> assign(n_poses);
    SEELE_CUDA(c, cudaMemcpyAsync(cent.data(), vb + off_c, 48 * nk, cudaMemcpyDeviceToHost, s));
    SEELE_CUDA(c, cudaMemcpyAsync(assign.data(), vb + off_a, 4 * (size_t)n_poses, cudaMemcpyDeviceToHost, s));
    SEELE_CUDA(c, cudaStreamSynchronize(s));

    // top-k contributors of every pose, a batch of cameras per frame
    uint32_t* mask = reinterpret_cast<uint32_t*>(vb + off_m);
    int* cl = reinterpret_cast<int*>(vb + off_cl);
    SEELE_CUDA(c, cudaMemsetAsync(mask, 0, 4 * (size_t)c->n, s));
    std::vector<seele_camera> saved = c->cams;
    seele_options o;
    seele_default_options(&o);
    o.binning = SEELE_BIN_TILES;
    seele_status result = SEELE_OK;
    const int batch = 32;
    for (int b0 = 0; b0 < n_poses && result == SEELE_OK; b0 += batch) {
        const int nb = std::min(batch, n_poses - b0);
        c->cams.assign(poses + b0, poses + b0 + nb);
        uint64_t pix = 0;
        for (int i = 0; i < nb; ++i) pix += (uint64_t)poses[b0 + i].width * poses[b0 + i].height;
        SEELE_CUDA(c, cudaMemcpyAsync(cl, assign.data() + b0, 4 * (size_t)nb, cudaMemcpyHostToDevice, s));
        SEELE_CUDA(c, ensure(c->rgb_tmp, 12 * pix));
        c->topk_k = top_k;
        c->topk_cluster = cl;
        c->topk_mask = mask;
        result = seele_render(c, &o, ptr<float>(c->rgb_tmp), nullptr, nullptr);
        c->topk_k = 0;
    }
    c->cams = saved;
    c->rendered = false;
    if (result != SEELE_OK) return result;
    const uint32_t* mask_out = mask;
    if (c->spatial) {
        // back to the caller's order of the Gaussians
        SEELE_CUDA(c, ensure(c->visk[1], 4 * (size_t)c->n));
        launch_scatter_u32(mask, ptr<uint32_t>(c->visk[1]), (int)c->n, ptr<const uint32_t>(c->order), s);
        SEELE_LAUNCHED(c);
        mask_out = ptr<const uint32_t>(c->visk[1]);
    }
    SEELE_CUDA(c, cudaMemcpyAsync(out_mask, mask_out, 4 * (size_t)c->n, cudaMemcpyDefault, s));
    SEELE_CUDA(c, cudaStreamSynchronize(s));
    for (size_t i = 0; i < 6 * nk; ++i) out_centroids[i] = (float)cent[i];
    *out_pos_scale = (float)scale;
    if (out_assign)
        for (int i = 0; i < n_poses; ++i) out_assign[i] = assign[i];
    return SEELE_OK;
}

}  // extern "C"
