// raster.cu -- tile rasterization, forward (Sec. 3.1 "Rasterization",
// Eqns. 1-2) and contribution-aware (Sec. 3.4, Algorithm 1).
//
// One CTA per tile; each thread owns a PW x PH block of pixels, so a Gaussian
// staged in shared memory is loaded once per 4 (or 8) pixels and the pixels of
// a thread give four independent dependency chains.  Pixel groups of Alg. 1
// are GW x GH sub-blocks of a thread's block with the top-left pixel as
// leader (Sec. 4.1): the leader's exponent decides for its group, the
// remaining pixels then apply the per-pixel rules.  A warp skips a Gaussian
// outright when every group it holds rejects it -- the divergence-free skip of
// Sec. 3.4 "GPU Parallelism".
//
// Work per (pixel, Gaussian) pair: ~11 FP32-pipe instructions and one MUFU
// ex2; the kernel is bound by FP32 issue, not by memory.
#include "common.cuh"
#include "kernels.h"

namespace seele {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool COUNT>
__global__ void __launch_bounds__((TW / PW) * (TH / PH))
    raster_fwd_kernel(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ ends,
                      const uint32_t* __restrict__ inst_rec,
                      const float4* __restrict__ rec, const CamDev* __restrict__ cams, int n_cams, FrameParams fp,
                      float* __restrict__ out_rgb, float* __restrict__ out_T, uint32_t* __restrict__ out_nc,
                      DeviceStatus* __restrict__ counters, unsigned long long* __restrict__ view_end,
                      uint32_t* __restrict__ view_done) {
    constexpr int NT = (TW / PW) * (TH / PH);
    constexpr int NP = PW * PH;
    constexpr int TXN = TW / PW;
    static_assert(PW % GW == 0 && PH % GH == 0, "groups must tile the thread block");
    __shared__ float4 s0[NT], s1[NT], s2[NT];

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
    const int bx = tx * TW + (t % TXN) * PW, by = ty * TH + (t / TXN) * PH;

    float T[NP], cr[NP], cg[NP], cb[NP];
    uint32_t nc[NP];
    uint32_t live = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T[p] = 1.f;
        cr[p] = cg[p] = cb[p] = 0.f;
        nc[p] = 0;
        if (bx + p % PW < C.W && by + p / PW < C.H) live |= 1u << p;
    }
    uint2 rg = make_uint2(__ldg(starts + gtile), __ldg(ends + gtile));
    if (rg.x >= rg.y) rg = make_uint2(0u, 0u);  // tile without instances
    const float fx0 = (float)bx + 0.5f, fy0 = (float)by + 0.5f;
    const float amax = fp.alpha_max, tstop = fp.t_stop;
    uint32_t n_lead = 0, n_eval = 0, n_blend = 0;  // counting variant only

    for (uint32_t base = rg.x; base < rg.y; base += NT) {
        if (__syncthreads_and(live == 0u)) break;
        const uint32_t j = base + t;
        if (j < rg.y) {
            const uint32_t r = __ldg(inst_rec + j);
            s0[t] = __ldg(rec + 3 * (size_t)r);
            s1[t] = __ldg(rec + 3 * (size_t)r + 1);
            s2[t] = __ldg(rec + 3 * (size_t)r + 2);
        }
        __syncthreads();
        const int cnt = min((uint32_t)NT, rg.y - base);
        if (CR && GW == PW && GH == PH) {
            // Alg. 1 with one group per thread.  Phase 1: the leader (pixel 0)
            // tests every staged Gaussian -- independent of the blending state,
            // so the tests run back to back.  Phase 2: only the Gaussians the
            // leader kept are blended, in list order, by the group's pixels.
            if (live == 0u) continue;
            for (int c0 = 0; c0 < cnt && live != 0u; c0 += 64) {
            const int c1 = min(cnt, c0 + 64);
            uint64_t pass = 0;
#pragma unroll 8
            for (int k = c0; k < c1; ++k) {
                const float4 A = s0[k];
                const float4 B = s1[k];
                const float dx = fx0 - A.x, dy = fy0 - A.y;
                const float e0 = fmaf(fmaf(A.z, dx, A.w * dy), dx, fmaf(B.x * dy, dy, B.y));
                if (COUNT) ++n_lead;
                pass |= (uint64_t)(e0 >= B.z) << (k - c0);
            }
            while (pass != 0ull && live != 0u) {
                const int k = c0 + __ffsll((long long)pass) - 1;
                pass &= pass - 1ull;
                const float4 A = s0[k];
                const float4 B = s1[k];
                const float4 Cc = s2[k];
                const float dx = fx0 - A.x, dy = fy0 - A.y;
                const uint32_t pos1 = base + (uint32_t)k - rg.x + 1u;
#pragma unroll
                for (int jj = 0; jj < PH; ++jj) {
                    const float ddy = dy + (float)jj;
                    const float rb = A.w * ddy, rc = fmaf(B.x * ddy, ddy, B.y);
#pragma unroll
                    for (int i = 0; i < PW; ++i) {
                        const int p = jj * PW + i;
                        if (!(live >> p & 1u)) continue;
                        if (COUNT) ++n_eval;
                        const float ddx = dx + (float)i;
                        const float e = fmaf(fmaf(A.z, ddx, rb), ddx, rc);
                        if (e < B.z) continue;  // per-pixel alpha_theta / support rule
                        const float al = fminf(amax, ex2_approx(e));
                        const float Tn = T[p] * (1.f - al);
                        if (Tn < tstop) {
                            live &= ~(1u << p);
                            continue;
                        }
                        const float wgt = al * T[p];
                        cr[p] = fmaf(wgt, Cc.x, cr[p]);
                        cg[p] = fmaf(wgt, Cc.y, cg[p]);
                        cb[p] = fmaf(wgt, Cc.z, cb[p]);
                        T[p] = Tn;
                        nc[p] = pos1;
                        if (COUNT) ++n_blend;
                    }
                }
            }
            }
            continue;
        }
        for (int k = 0; k < cnt; ++k) {
            if (live == 0u) break;
            const float4 A = s0[k];
            const float4 B = s1[k];
            const float dx = fx0 - A.x, dy = fy0 - A.y;
            const uint32_t pos1 = base + (uint32_t)k - rg.x + 1u;
            // exponent of alpha = 2^e at pixel offset (i, j) of this thread
            auto expo = [&](int i, int jj) {
                const float ddx = dx + (float)i, ddy = dy + (float)jj;
                return fmaf(fmaf(A.z, ddx, A.w * ddy), ddx, fmaf(B.x * ddy, ddy, B.y));
            };
            auto blend = [&](int p, float e) {
                if (COUNT) ++n_eval;
                if (e < B.z) return;  // outside the support or alpha < alpha_theta
                const float al = fminf(amax, ex2_approx(e));
                const float Tn = T[p] * (1.f - al);
                if (Tn < tstop) {     // stop before crossing Gamma_theta
                    live &= ~(1u << p);
                    return;
                }
                const float4 Cc = s2[k];
                const float wgt = al * T[p];
                cr[p] = fmaf(wgt, Cc.x, cr[p]);
                cg[p] = fmaf(wgt, Cc.y, cg[p]);
                cb[p] = fmaf(wgt, Cc.z, cb[p]);
                T[p] = Tn;
                nc[p] = pos1;
                if (COUNT) ++n_blend;
            };
            if (CR && GW == PW && GH == PH) {
                // handled by the two-phase path below
            } else if (CR) {
#pragma unroll
                for (int gy = 0; gy < PH / GH; ++gy)
#pragma unroll
                    for (int gx = 0; gx < PW / GW; ++gx) {
                        uint32_t gmask = 0;
#pragma unroll
                        for (int jj = 0; jj < GH; ++jj)
#pragma unroll
                            for (int i = 0; i < GW; ++i) gmask |= 1u << ((gy * GH + jj) * PW + gx * GW + i);
                        if ((live & gmask) == 0u) continue;
                        if (COUNT) ++n_lead;
                        const float e0 = expo(gx * GW, gy * GH);
                        if (e0 < B.z) continue;  // leader rejects: the whole group skips g
#pragma unroll
                        for (int jj = 0; jj < GH; ++jj)
#pragma unroll
                            for (int i = 0; i < GW; ++i) {
                                const int p = (gy * GH + jj) * PW + gx * GW + i;
                                if (!(live >> p & 1u)) continue;
                                blend(p, (i == 0 && jj == 0) ? e0 : expo(gx * GW + i, gy * GH + jj));
                            }
                    }
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    if (live >> p & 1u) blend(p, expo(p % PW, p / PW));
            }
        }
    }

    if (COUNT) {
        atomicAdd(&counters->work[0], (unsigned long long)n_lead);
        atomicAdd(&counters->work[1], (unsigned long long)n_eval);
        atomicAdd(&counters->work[2], (unsigned long long)n_blend);
    }
    const size_t plane = (size_t)C.W * C.H;
    float* img = out_rgb + 3 * (size_t)C.pix_offset;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int x = bx + p % PW, y = by + p / PW;
        if (x < C.W && y < C.H) {
            const size_t o = (size_t)y * C.W + x;
            img[o] = cr[p];
            img[plane + o] = cg[p];
            img[2 * plane + o] = cb[p];
            out_T[C.pix_offset + o] = T[p];
            out_nc[C.pix_offset + o] = nc[p];
        }
    }
    // the CTA that finishes a camera's last tile stamps the view's end time
    if (view_done) {
        __syncthreads();
        if (t == 0 && atomicAdd(view_done + lo, 1u) + 1u == (uint32_t)(C.tiles_x * C.tiles_y))
            view_end[lo] = global_ns();
    }
}

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR>
static void launch_one(const RasterArgs& a, cudaStream_t s) {
    constexpr int NT = (TW / PW) * (TH / PH);
    if (a.count_into)
        raster_fwd_kernel<TW, TH, PW, PH, GW, GH, CR, true><<<a.n_tiles, NT, 0, s>>>(
            a.starts, a.ends, a.inst_rec, a.rec, a.cams, a.n_cams, a.fp, a.out_rgb, a.out_T, a.out_nc, a.count_into,
            a.view_end, a.view_done);
    else
        raster_fwd_kernel<TW, TH, PW, PH, GW, GH, CR, false><<<a.n_tiles, NT, 0, s>>>(
            a.starts, a.ends, a.inst_rec, a.rec, a.cams, a.n_cams, a.fp, a.out_rgb, a.out_T, a.out_nc, nullptr,
            a.view_end, a.view_done);
}

template <int TW, int TH>
static bool launch_shape(const RasterArgs& a, cudaStream_t s) {
    if (!a.cr) launch_one<TW, TH, 2, 2, 1, 1, false>(a, s);
    else if (a.group_w == 2 && a.group_h == 2) launch_one<TW, TH, 2, 2, 2, 2, true>(a, s);
    else if (a.group_w == 1 && a.group_h == 1) launch_one<TW, TH, 2, 2, 1, 1, true>(a, s);
    else if (a.group_w == 2 && a.group_h == 4) launch_one<TW, TH, 2, 4, 2, 4, true>(a, s);
    else return false;
    return true;
}

bool launch_raster_fwd(const RasterArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return true;
    if (a.fp.tile_w == 16 && a.fp.tile_h == 16) return launch_shape<16, 16>(a, s);
    if (a.fp.tile_w == 32 && a.fp.tile_h == 8) return launch_shape<32, 8>(a, s);
    if (a.fp.tile_w == 32 && a.fp.tile_h == 16) return launch_shape<32, 16>(a, s);
    return false;
}

}  // namespace seele
