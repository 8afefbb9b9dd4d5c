// skew.cu -- contribution skew of a plain render (Sec. 1 "Rendering
// Inefficiency", Sec. 3.4 "Motivation"): per pixel, sorting the contributions
// Gamma_i alpha_i of the Gaussians it blends in descending order, the smallest
// number m of them that sum to frac of their total.  The paper finds m to be
// about 1.5% of the Gaussians of a pixel, which motivates Alg. 1.
//
// One CTA per tile and one thread per pixel walk the tile list under the plain
// blending rules (support and alpha_theta as one exponent threshold, stop
// before crossing T_stop).  The first walk counts the contributions, the list
// entries examined and their total; m then follows without storing or sorting
// the contributions: the sum of the contributions at or above a threshold
// falls as the threshold rises, so a bisection on the threshold's float bits
// (positive floats order like their bits) finds the largest threshold whose
// sum still reaches frac of the total, one walk per step, and m is the count
// at or above it.  Sums are kept in double precision.
#include "common.cuh"
#include "kernels.h"

namespace seele {

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kSkewSteps = 31;  // bisection steps over [0, bits(1.0f)] < 2^30

}  // namespace

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) skew_kernel(const uint32_t* __restrict__ starts,
                                                       const uint32_t* __restrict__ ends,
                                                       const uint32_t* __restrict__ inst_rec,
                                                       const float4* __restrict__ rec, const CamDev* __restrict__ cams,
                                                       int n_cams, FrameParams fp, double frac,
                                                       uint32_t* __restrict__ out_m,
                                                       uint32_t* __restrict__ out_blended,
                                                       uint32_t* __restrict__ out_walked,
                                                       float* __restrict__ out_total,
                                                       uint32_t* __restrict__ out_listed) {
    constexpr int NT = TW * TH;
    __shared__ float4 s0[NT], s1[NT];

    const uint32_t gtile = blockIdx.x;
    int lo_c = 0, hi_c = n_cams - 1;
    while (lo_c < hi_c) {
        const int mid = (lo_c + hi_c + 1) >> 1;
        if (cams[mid].tile_offset <= gtile) lo_c = mid; else hi_c = mid - 1;
    }
    const CamDev& C = cams[lo_c];
    const uint32_t lt = gtile - C.tile_offset;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const bool inside = px < C.W && py < C.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    uint2 rg = make_uint2(__ldg(starts + gtile), __ldg(ends + gtile));
    if (rg.x >= rg.y) rg = make_uint2(0u, 0u);

    // One walk of the tile list.  Every thread takes part in the staging;
    // a pixel stops at T_stop, the block once every pixel has.  With
    // thr_bits = 0 it also counts the entries examined and the largest
    // contribution's bits.
    auto walk = [&](uint32_t thr_bits, double& sum, uint32_t& count, uint32_t& walked, uint32_t& wmax) {
        float T = 1.f;
        bool live = inside;
        sum = 0.0;
        count = 0;
        walked = 0;
        wmax = 0;
        for (uint32_t base = rg.x; base < rg.y; base += NT) {
            if (__syncthreads_and(!live)) break;
            const uint32_t j = base + t;
            if (j < rg.y) {
                const uint32_t r = __ldg(inst_rec + j);
                s0[t] = __ldg(rec + (size_t)kRecF4 * r);
                s1[t] = __ldg(rec + (size_t)kRecF4 * r + 1);
            }
            __syncthreads();
            const int cnt = (int)min((uint32_t)NT, rg.y - base);
            for (int q = 0; q < cnt && live; ++q) {
                ++walked;
                const float4 A = s0[q];
                const float4 B = s1[q];
                const float dx = fx - A.x, dy = fy - A.y;
                const float e = fmaf(fmaf(A.z, dx, A.w * dy), dx, fmaf(B.x * dy, dy, B.y));
                if (e < B.z) continue;  // outside the support or alpha < alpha_theta
                const float al = fminf(fp.alpha_max, ex2_approx(e));
                const float w = al * T;
                const float Tn = T - w;
                if (Tn < fp.t_stop) {
                    live = false;
                    break;
                }
                T = Tn;
                const uint32_t wb = __float_as_uint(w);
                if (wb >= thr_bits) {
                    sum += (double)w;
                    ++count;
                }
                wmax = max(wmax, wb);
            }
            __syncthreads();
        }
    };

    double total;
    uint32_t blended, walked, wmax;
    walk(0u, total, blended, walked, wmax);
    // largest threshold lo with sum(>= lo) >= frac * total; sum(>= hi) falls short
    const double target = frac * total;
    uint32_t lo = 0, hi = wmax + 1, m = blended;
    for (int step = 0; step < kSkewSteps; ++step) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        double sum;
        uint32_t count, wk, wm;
        walk(mid, sum, count, wk, wm);
        if (hi - lo > 1) {
            if (sum >= target) {
                lo = mid;
                m = count;
            } else {
                hi = mid;
            }
        }
    }
    if (inside) {
        const size_t p = (size_t)C.pix_offset + (size_t)py * C.W + px;
        out_m[p] = blended > 0 ? m : 0u;
        out_blended[p] = blended;
        out_walked[p] = walked;
        out_total[p] = (float)total;
        out_listed[p] = rg.y - rg.x;
    }
}

bool launch_skew(const uint32_t* starts, const uint32_t* ends, const uint32_t* inst_rec, const float4* rec,
                 const CamDev* cams, int n_cams, uint32_t n_tiles, const FrameParams& fp, double frac,
                 uint32_t* out_m, uint32_t* out_blended, uint32_t* out_walked, float* out_total,
                 uint32_t* out_listed, cudaStream_t s) {
    if (n_tiles == 0) return true;
    if (fp.tile_w == 8 && fp.tile_h == 8)
        skew_kernel<8, 8><<<n_tiles, 64, 0, s>>>(starts, ends, inst_rec, rec, cams, n_cams, fp, frac, out_m,
                                                 out_blended, out_walked, out_total, out_listed);
    else if (fp.tile_w == 16 && fp.tile_h == 16)
        skew_kernel<16, 16><<<n_tiles, 256, 0, s>>>(starts, ends, inst_rec, rec, cams, n_cams, fp, frac, out_m,
                                                    out_blended, out_walked, out_total, out_listed);
    else if (fp.tile_w == 32 && fp.tile_h == 8)
        skew_kernel<32, 8><<<n_tiles, 256, 0, s>>>(starts, ends, inst_rec, rec, cams, n_cams, fp, frac, out_m,
                                                   out_blended, out_walked, out_total, out_listed);
    else if (fp.tile_w == 32 && fp.tile_h == 16)
        skew_kernel<32, 16><<<n_tiles, 512, 0, s>>>(starts, ends, inst_rec, rec, cams, n_cams, fp, frac, out_m,
                                                    out_blended, out_walked, out_total, out_listed);
    else
        return false;
    return true;
}

}  // namespace seele
