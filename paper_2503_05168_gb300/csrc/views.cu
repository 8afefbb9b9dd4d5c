// views.cu -- the offline view-dependent representation (Sec. 3.3 "Offline
// Clustering"): sampled camera poses are clustered on the feature (x / s, v)
// by k-means, and a Gaussian joins cluster c when, for some pixel of some pose
// of c, it is among the k Gaussians with the largest contribution
// Gamma_i alpha_i (the transmittance in front of it times its alpha).  The
// runtime reads the result as one bit per cluster per Gaussian; Gaussians of
// every cluster are the shared ones, Gaussians of none are dropped.
#include "common.cuh"
#include "kernels.h"

namespace seele {

// --------------------------------------------------------------- k-means --

// One CTA, double precision.  k-means++ seeding from the uniforms u[0..k):
// the first centre is point floor(u[0] n); centre j is the first point at
// which the running sum of squared distances to the nearest chosen centre
// exceeds u[j] times their total (floor(u[j] n) if the total is zero).
// Lloyd iterations then assign each point to its nearest centre (ties to the
// lower index) and move each centre to the mean of its points in index order
// (an empty cluster keeps its centre), until an assignment step changes
// nothing or max_iter updates have run.
constexpr int kKmThreads = 256;

__global__ void __launch_bounds__(kKmThreads) kmeans_kernel(const double* __restrict__ x, int n, int k,
                                                            const double* __restrict__ u, int max_iter,
                                                            double* __restrict__ cent, int* __restrict__ assign,
                                                            double* __restrict__ d2, int* __restrict__ iters) {
    constexpr int D = 6;
    __shared__ int s_pick;
    __shared__ int s_changed;
    const int t = threadIdx.x;
    if (t == 0) s_pick = min(n - 1, (int)floor(u[0] * n));
    __syncthreads();
    for (int c = t; c < D; c += kKmThreads) cent[c] = x[s_pick * D + c];
    __syncthreads();
    for (int i = t; i < n; i += kKmThreads) {
        double d = 0.0;
        for (int c = 0; c < D; ++c) d += (x[i * D + c] - cent[c]) * (x[i * D + c] - cent[c]);
        d2[i] = d;
    }
    __syncthreads();
    for (int j = 1; j < k; ++j) {
        if (t == 0) {
            // the running sum in index order, as the definition reads
            double total = 0.0;
            for (int i = 0; i < n; ++i) total += d2[i];
            int pick = n - 1;
            if (total > 0.0) {
                const double target = u[j] * total;
                double run = 0.0;
                for (int i = 0; i < n; ++i) {
                    run += d2[i];
                    if (run > target) {
                        pick = i;
                        break;
                    }
                }
            } else {
                pick = min(n - 1, (int)floor(u[j] * n));
            }
            s_pick = pick;
        }
        __syncthreads();
        for (int c = t; c < D; c += kKmThreads) cent[j * D + c] = x[s_pick * D + c];
        __syncthreads();
        for (int i = t; i < n; i += kKmThreads) {
            double d = 0.0;
            for (int c = 0; c < D; ++c) d += (x[i * D + c] - cent[j * D + c]) * (x[i * D + c] - cent[j * D + c]);
            if (d < d2[i]) d2[i] = d;
        }
        __syncthreads();
    }
    for (int i = t; i < n; i += kKmThreads) assign[i] = -1;
    __syncthreads();
    int it = 0;
    for (; it < max_iter; ++it) {
        if (t == 0) s_changed = 0;
        __syncthreads();
        for (int i = t; i < n; i += kKmThreads) {
            int best = 0;
            double bd = 0.0;
            for (int c = 0; c < D; ++c) bd += (x[i * D + c] - cent[c]) * (x[i * D + c] - cent[c]);
            for (int j = 1; j < k; ++j) {
                double d = 0.0;
                for (int c = 0; c < D; ++c) d += (x[i * D + c] - cent[j * D + c]) * (x[i * D + c] - cent[j * D + c]);
                if (d < bd) {
                    bd = d;
                    best = j;
                }
            }
            if (assign[i] != best) {
                assign[i] = best;
                s_changed = 1;
            }
        }
        __syncthreads();
        if (!s_changed) break;
        // one thread per cluster sums its points in index order
        for (int j = t; j < k; j += kKmThreads) {
            double sum[D] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int m = 0;
            for (int i = 0; i < n; ++i)
                if (assign[i] == j) {
                    for (int c = 0; c < D; ++c) sum[c] += x[i * D + c];
                    ++m;
                }
            if (m > 0)
                for (int c = 0; c < D; ++c) cent[j * D + c] = sum[c] / m;
        }
        __syncthreads();
    }
    if (t == 0) *iters = it;
}

void launch_kmeans(const double* x, int n, int k, const double* u, int max_iter, double* cent, int* assign,
                   double* scratch, int* iters, cudaStream_t s) {
    kmeans_kernel<<<1, kKmThreads, 0, s>>>(x, n, k, u, max_iter, cent, assign, scratch, iters);
}

// ------------------------------------------------------ top-k contributors --

__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (w, g) ranks above (w2, g2): larger contribution, ties to the lower index
__device__ __forceinline__ bool better(float w, uint32_t g, float w2, uint32_t g2) {
    return w > w2 || (w == w2 && g < g2);
}

// One CTA per tile, one thread per pixel.  Every pixel walks its tile list
// front to back under the plain blending rules of the rasterizer (support and
// alpha_theta as one exponent threshold, stop before crossing Gamma_theta)
// and keeps its k best (contribution, Gaussian) pairs in shared memory
// (slot-major, so threads never share a bank row); at the end each kept
// Gaussian's cluster bit is ORed into its mask.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) topk_kernel(const uint32_t* __restrict__ starts,
                                                       const uint32_t* __restrict__ ends,
                                                       const uint32_t* __restrict__ inst_rec,
                                                       const float4* __restrict__ rec,
                                                       const CamDev* __restrict__ cams, int n_cams, FrameParams fp,
                                                       int k, const int* __restrict__ cam_cluster,
                                                       uint32_t* __restrict__ mask) {
    constexpr int NT = TW * TH;
    extern __shared__ uint32_t s_dyn[];
    float* s_w = reinterpret_cast<float*>(s_dyn);   // [k][NT]
    uint32_t* s_g = s_dyn + (size_t)k * NT;          // [k][NT]
    __shared__ float4 s0[NT], s1[NT];
    __shared__ uint32_t s_r[NT];

    const uint32_t gtile = blockIdx.x;
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_offset <= gtile) lo = mid; else hi = mid - 1;
    }
    const CamDev& C = cams[lo];
    const uint32_t lt = gtile - C.tile_offset;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    bool live = px < C.W && py < C.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    float T = 1.f;
    int m = 0, worst = 0;  // slots used; slot of the worst kept pair once full

    uint2 rg = make_uint2(__ldg(starts + gtile), __ldg(ends + gtile));
    if (rg.x >= rg.y) rg = make_uint2(0u, 0u);
    for (uint32_t base = rg.x; base < rg.y; base += NT) {
        if (__syncthreads_and(!live)) break;
        const uint32_t j = base + t;
        if (j < rg.y) {
            const uint32_t r = __ldg(inst_rec + j);
            s_r[t] = r;
            s0[t] = __ldg(rec + (size_t)kRecF4 * r);
            s1[t] = __ldg(rec + (size_t)kRecF4 * r + 1);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)NT, rg.y - base);
        for (int q = 0; q < cnt && live; ++q) {
            const float4 A = s0[q];
            const float4 B = s1[q];
            const float dx = fx - A.x, dy = fy - A.y;
            const float e = fmaf(fmaf(A.z, dx, A.w * dy), dx, fmaf(B.x * dy, dy, B.y));
            if (e < B.z) continue;  // outside the support or alpha < alpha_theta
            const float al = fminf(fp.alpha_max, ex2_fast(e));
            const float w = al * T;
            const float Tn = T - w;
            if (Tn < fp.t_stop) {
                live = false;
                break;
            }
            T = Tn;
            const uint32_t g = s_r[q] % (uint32_t)fp.n;
            if (m < k) {
                s_w[m * NT + t] = w;
                s_g[m * NT + t] = g;
                ++m;
                if (m == k) {
                    worst = 0;
                    for (int i = 1; i < k; ++i)
                        if (better(s_w[worst * NT + t], s_g[worst * NT + t], s_w[i * NT + t], s_g[i * NT + t]))
                            worst = i;
                }
            } else if (better(w, g, s_w[worst * NT + t], s_g[worst * NT + t])) {
                s_w[worst * NT + t] = w;
                s_g[worst * NT + t] = g;
                worst = 0;
                for (int i = 1; i < k; ++i)
                    if (better(s_w[worst * NT + t], s_g[worst * NT + t], s_w[i * NT + t], s_g[i * NT + t]))
                        worst = i;
            }
        }
    }
    const uint32_t bit = 1u << (uint32_t)cam_cluster[lo];
    for (int i = 0; i < m; ++i) atomicOr(mask + s_g[i * NT + t], bit);
}

bool launch_topk(const uint32_t* starts, const uint32_t* ends, const uint32_t* inst_rec, const float4* rec,
                 const CamDev* cams, int n_cams, uint32_t n_tiles, const FrameParams& fp, int k,
                 const int* cam_cluster, uint32_t* mask, cudaStream_t s) {
    if (n_tiles == 0) return true;
    auto run = [&](auto kernel, int nt) -> bool {
        const size_t dyn = (size_t)k * nt * 8;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
            return false;
        kernel<<<n_tiles, nt, dyn, s>>>(starts, ends, inst_rec, rec, cams, n_cams, fp, k, cam_cluster, mask);
        return true;
    };
    if (fp.tile_w == 8 && fp.tile_h == 8) return run(topk_kernel<8, 8>, 64);
    if (fp.tile_w == 16 && fp.tile_h == 16) return run(topk_kernel<16, 16>, 256);
    if (fp.tile_w == 32 && fp.tile_h == 8) return run(topk_kernel<32, 8>, 256);
    return false;
}

}  // namespace seele
