// raster_impl.cuh -- tile rasterization, forward (Sec. 3.1 "Rasterization",
// Eqns. 1-2) and contribution-aware (Sec. 3.4, Algorithm 1): the body shared
// by the one-CTA-per-unit kernels (raster.cu) and the persistent queue
// kernels (raster_queue.cu).
//
// One CTA per tile; each thread owns a PW x PH block of pixels, so a Gaussian
// staged in shared memory is loaded once per 4 (or 8) pixels and the pixels of
// a thread give four independent dependency chains.  Pixel groups of Alg. 1
// are GW x GH sub-blocks of a thread's block, or unions of whole thread
// blocks, with the top-left pixel as leader (Sec. 4.1): the leader's exponent
// decides for its group, the remaining pixels then apply the per-pixel rules.
// A group spanning several threads has each of them evaluate the leader's
// exponent itself (the same FP32 operations on the same inputs).  A warp skips a Gaussian
// outright when every group it holds rejects it -- the divergence-free skip of
// Sec. 3.4 "GPU Parallelism".
//
// Work per (pixel, Gaussian) pair: ~10 FP32-pipe instructions, three
// compares and one MUFU ex2; the kernel is bound by instruction issue, not by
// memory.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace seele {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One (pixel, Gaussian) pair under the per-pixel rules: outside the support
// or below alpha_theta (e < thr) nothing happens; otherwise the pixel either
// blends (T (1 - alpha) stays at or above its stop bound) or stops without
// blending.  A pixel's stop bound `tau` is Gamma_theta while it is live and 2
// once it has stopped, so that a stopped pixel never blends again (T <= 1 <
// 2) and stopping again changes nothing: liveness costs no flag per pair.
// Written as predicated PTX so that the pair costs three compares and no
// branch or select: blend under (e >= thr and T' >= tau), stop under
// (e >= thr and T' < tau).
// CLAMP: the record's alpha can reach alpha_max (else 2^e < alpha_max).
template <bool CLAMP>
__device__ __forceinline__ void blend_pair(float& T, float& cr, float& cg, float& cb, uint32_t& nc, float& tau,
                                           float e, float thr, const float4& c, uint32_t pos1, float amax) {
    if (CLAMP)
        asm("{\n\t.reg .pred pon, ptk, pst;\n\t.reg .f32 al, wg, tn;\n\t"
            "ex2.approx.ftz.f32 al, %6;\n\t"
            "min.f32 al, al, %12;\n\t"
            "mul.rn.f32 wg, al, %0;\n\t"
            "sub.rn.f32 tn, %0, wg;\n\t"
            "setp.ge.f32 pon, %6, %7;\n\t"
            "setp.ge.and.f32 ptk, tn, %5, pon;\n\t"
            "setp.lt.and.f32 pst, tn, %5, pon;\n\t"
            "@ptk fma.rn.f32 %1, wg, %8, %1;\n\t"
            "@ptk fma.rn.f32 %2, wg, %9, %2;\n\t"
            "@ptk fma.rn.f32 %3, wg, %10, %3;\n\t"
            "@ptk mov.f32 %0, tn;\n\t"
            "@ptk mov.b32 %4, %11;\n\t"
            "@pst mov.f32 %5, 0f40000000;\n\t}"
            : "+f"(T), "+f"(cr), "+f"(cg), "+f"(cb), "+r"(nc), "+f"(tau)
            : "f"(e), "f"(thr), "f"(c.x), "f"(c.y), "f"(c.z), "r"(pos1), "f"(amax));
    else
        asm("{\n\t.reg .pred pon, ptk, pst;\n\t.reg .f32 al, wg, tn;\n\t"
            "ex2.approx.ftz.f32 al, %6;\n\t"
            "mul.rn.f32 wg, al, %0;\n\t"
            "sub.rn.f32 tn, %0, wg;\n\t"
            "setp.ge.f32 pon, %6, %7;\n\t"
            "setp.ge.and.f32 ptk, tn, %5, pon;\n\t"
            "setp.lt.and.f32 pst, tn, %5, pon;\n\t"
            "@ptk fma.rn.f32 %1, wg, %8, %1;\n\t"
            "@ptk fma.rn.f32 %2, wg, %9, %2;\n\t"
            "@ptk fma.rn.f32 %3, wg, %10, %3;\n\t"
            "@ptk mov.f32 %0, tn;\n\t"
            "@ptk mov.b32 %4, %11;\n\t"
            "@pst mov.f32 %5, 0f40000000;\n\t}"
            : "+f"(T), "+f"(cr), "+f"(cg), "+f"(cb), "+r"(nc), "+f"(tau)
            : "f"(e), "f"(thr), "f"(c.x), "f"(c.y), "f"(c.z), "r"(pos1), "f"(amax));
}

// The counting variant: the same rules in plain code, counting the pairs
// evaluated (pixel live) and blended.
template <bool CLAMP>
__device__ __forceinline__ void blend_pair_counted(float& T, float& cr, float& cg, float& cb, uint32_t& nc,
                                                   float& tau, float e, float thr, const float4& c, uint32_t pos1,
                                                   float amax, uint32_t& n_eval, uint32_t& n_blend) {
    n_eval += tau <= 1.f ? 1u : 0u;
    float al = ex2_approx(e);
    if (CLAMP) al = fminf(amax, al);
    const float wgt = __fmul_rn(al, T);
    const float Tn = __fsub_rn(T, wgt);
    if (e >= thr) {
        if (Tn >= tau) {
            cr = fmaf(wgt, c.x, cr);
            cg = fmaf(wgt, c.y, cg);
            cb = fmaf(wgt, c.z, cb);
            T = Tn;
            nc = pos1;
            ++n_blend;
        } else {
            tau = 2.f;
        }
    }
}

template <bool CLAMP, bool COUNT>
__device__ __forceinline__ void blend_one(float& T, float& cr, float& cg, float& cb, uint32_t& nc, float& tau, float e,
                                          float thr, const float4& c, uint32_t pos1, float amax, uint32_t& n_eval,
                                          uint32_t& n_blend) {
    if (COUNT)
        blend_pair_counted<CLAMP>(T, cr, cg, cb, nc, tau, e, thr, c, pos1, amax, n_eval, n_blend);
    else
        blend_pair<CLAMP>(T, cr, cg, cb, nc, tau, e, thr, c, pos1, amax);
}

// BLOCKS (block binning): CTA i rasterizes tile i % 32 of the tile block
// block_order[i / 32].  Its list is the block's list filtered by the tile's
// mask bit: a window of 32 * NT entries at a time, one 32-entry group per
// thread, skipped with one load when the group's OR-summary lacks the bit.
// The kept entries, in list order, are exactly the tile's own list.
template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool COUNT, bool BLOCKS>
__device__ __forceinline__ void raster_unit(uint32_t item, const uint32_t* __restrict__ starts,
                                            const uint32_t* __restrict__ ends, const uint32_t* __restrict__ inst_rec,
                                            const uint32_t* __restrict__ inst_mask,
                                            const uint32_t* __restrict__ mask_summary,
                                            const uint32_t* __restrict__ block_order, const float4* __restrict__ rec,
                                            const CamDev* __restrict__ cams, int n_cams, const FrameParams& fp,
                                            float* __restrict__ out_rgb, float* __restrict__ out_T,
                                            uint32_t* __restrict__ out_nc, DeviceStatus* __restrict__ counters,
                                            unsigned long long* __restrict__ view_end,
                                            uint32_t* __restrict__ view_done, float4* __restrict__ ckpt,
                                            float4* __restrict__ cfin) {
    constexpr int NT = (TW / PW) * (TH / PH);
    constexpr int NP = PW * PH;
    constexpr int TXN = TW / PW;
    constexpr int WIN = BLOCKS ? 32 * NT : 1;  // list entries filtered per window
    static_assert((PW % GW == 0 && PH % GH == 0) || (GW % PW == 0 && GH % PH == 0),
                  "groups tile the thread block or are tiled by thread blocks");
    constexpr bool WHOLE = GW % PW == 0 && GH % PH == 0;  // a group is one or more whole thread blocks
    static_assert(NT % 32 == 0 && kBlockW * kBlockH == 32, "whole warps; one mask word per block entry");
    __shared__ float4 s0[NT], s1[NT], s2[NT];
    // CR with whole-thread groups: the leader tests read the fields they need
    // field by field (negated mean, conic, offset, threshold), four records
    // per vector load, and evaluate two records per packed FP32 instruction.
    constexpr bool LEAD2 = CR && WHOLE;
    __shared__ __align__(16) float sL[LEAD2 ? 7 : 1][LEAD2 ? NT : 4];
    __shared__ uint32_t s_idx[WIN];          // block binning: list indices of the window's tile entries
    __shared__ uint32_t s_wsum[NT / 32];

    uint32_t gtile, unit, bit = 0;
    int lo = 0, tx, ty;
    if (BLOCKS) {
        uint32_t b = __ldg(block_order + (item >> 5));
        if (kChecked && b >= cams[n_cams - 1].block_offset + (uint32_t)(cams[n_cams - 1].blocks_x *
                                                                          ((cams[n_cams - 1].tiles_y + kBlockH - 1) / kBlockH))) {
            if (threadIdx.x == 0) record_error(counters, kErrInternal, kSiteRasterBlock);
            b = 0;
        }
        bit = item & 31u;
        int hi = n_cams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cams[mid].block_offset <= b) lo = mid; else hi = mid - 1;
        }
        const CamDev& Cb = cams[lo];
        const uint32_t lb = b - Cb.block_offset;
        tx = (int)(lb % (uint32_t)Cb.blocks_x) * kBlockW + (int)(bit % kBlockW);
        ty = (int)(lb / (uint32_t)Cb.blocks_x) * kBlockH + (int)(bit / kBlockW);
        if (tx >= Cb.tiles_x || ty >= Cb.tiles_y) return;  // padding tile of a partial block
        gtile = Cb.tile_offset + (uint32_t)(ty * Cb.tiles_x + tx);
        unit = b;
    } else {
        gtile = block_order ? __ldg(block_order + item) : item;  // longest lists first
        int hi = n_cams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cams[mid].tile_offset <= gtile) lo = mid; else hi = mid - 1;
        }
        const uint32_t lt = gtile - cams[lo].tile_offset;
        tx = (int)(lt % (uint32_t)cams[lo].tiles_x);
        ty = (int)(lt / (uint32_t)cams[lo].tiles_x);
        unit = gtile;
    }
    const CamDev& C = cams[lo];
    const int t = threadIdx.x;
    const int bx = tx * TW + (t % TXN) * PW, by = ty * TH + (t / TXN) * PH;

    float T[NP], cr[NP], cg[NP], cb[NP], tau[NP];
    uint32_t nc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T[p] = 1.f;
        cr[p] = cg[p] = cb[p] = 0.f;
        nc[p] = 0;
        tau[p] = (bx + p % PW < C.W && by + p / PW < C.H) ? fp.t_stop : 2.f;  // pixels off the image never blend
    }
    // every pixel of the thread has stopped (the stop bounds are t_stop < 1 or 2)
    auto all_stopped = [&]() {
        float sum = 0.f;
#pragma unroll
        for (int p = 0; p < NP; ++p) sum += tau[p];
        return sum > 2.f * NP - 0.5f;
    };
    // bit p set while pixel p has not stopped
    auto live_mask = [&]() {
        uint32_t m = 0;
#pragma unroll
        for (int p = 0; p < NP; ++p) m |= tau[p] <= 1.f ? 1u << p : 0u;
        return m;
    };
    uint2 rg = make_uint2(__ldg(starts + unit), __ldg(ends + unit));
    if (rg.x >= rg.y) rg = make_uint2(0u, 0u);  // no instances
    if (kChecked && rg.y > counters->n_inst_valid) {
        if (threadIdx.x == 0) record_error(counters, kErrInternal, kSiteRasterRange);
        rg = make_uint2(0u, 0u);
    }
    const uint32_t n_records = (uint32_t)fp.n * (uint32_t)n_cams;
    // a record id of the list, validated in the checked build
    auto record_of = [&](uint32_t j) {
        uint32_t r = __ldg(inst_rec + j);
        if (kChecked && r >= n_records) {
            record_error(counters, kErrInternal, kSiteRasterRecord);
            r = 0;
        }
        return r;
    };
    // thread t stages record r in slot t
    auto stage = [&](uint32_t r) {
        const float4 v0 = __ldg(rec + (size_t)kRecF4 * r);
        const float4 v1 = __ldg(rec + (size_t)kRecF4 * r + 1);
        s0[t] = v0;
        s1[t] = v1;
        s2[t] = __ldg(rec + (size_t)kRecF4 * r + 2);
        if constexpr (LEAD2) {
            sL[0][t] = -v0.x;  // lx0 + (-mx) is lx0 - mx exactly
            sL[1][t] = -v0.y;
            sL[2][t] = v0.z;
            sL[3][t] = v0.w;
            sL[4][t] = v1.x;
            sL[5][t] = v1.y;
            sL[6][t] = v1.z;
        }
    };
    const float fx0 = (float)bx + 0.5f, fy0 = (float)by + 0.5f;
    // the leader pixel of the group holding this thread's block (WHOLE groups)
    const float lx0 = (float)(bx / GW * GW) + 0.5f, ly0 = (float)(by / GH * GH) + 0.5f;
    const float amax = fp.alpha_max;
    uint32_t n_lead = 0, n_eval = 0, n_blend = 0;  // counting variant only

    uint32_t cursor = BLOCKS ? rg.x >> 5 : rg.x;  // next list entry (tiles) or 32-entry group (blocks)
    const uint32_t cursor_end = BLOCKS ? (rg.y + 31u) >> 5 : rg.y;
    uint32_t pos0 = 0;           // tile-list position of staged entry 0
    int n_idx = 0, idx_pos = 0;  // block binning: window entries kept / staged
    while (true) {
        if (__syncthreads_and(all_stopped())) break;
        int cnt;
        if (!BLOCKS) {
            if (cursor >= cursor_end) break;
            const uint32_t j = cursor + t;
            if (j < rg.y) stage(record_of(j));
            cnt = (int)min((uint32_t)NT, rg.y - cursor);
            cursor += NT;
            __syncthreads();
        } else {
            if (idx_pos == n_idx) {
                if (cursor >= cursor_end) break;
                // thread t filters group cursor + t; group order is list order
                const uint32_t g = cursor + (uint32_t)t;
                uint32_t hits = 0;
                if (g < cursor_end && ((__ldg(mask_summary + g) >> bit) & 1u)) {
                    const uint4* mg = reinterpret_cast<const uint4*>(inst_mask + 32 * (size_t)g);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint4 v = __ldg(mg + q);
                        hits |= (((v.x >> bit) & 1u) | (((v.y >> bit) & 1u) << 1) | (((v.z >> bit) & 1u) << 2) |
                                 (((v.w >> bit) & 1u) << 3)) << (4 * q);
                    }
                    // entries of neighbouring lists share the edge groups
                    const uint32_t e0 = 32 * g;
                    if (e0 < rg.x) hits &= 0xffffffffu << (rg.x - e0);
                    if (e0 + 32 > rg.y) hits &= 0xffffffffu >> (e0 + 32 - rg.y);
                }
                const uint32_t c = __popc(hits);
                uint32_t incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((t & 31) >= o) incl += y;
                }
                if ((t & 31) == 31) s_wsum[t >> 5] = incl;
                __syncthreads();
                uint32_t off = incl - c, total = 0;
#pragma unroll
                for (int ww = 0; ww < NT / 32; ++ww) {
                    const uint32_t v = s_wsum[ww];
                    off += ww < (t >> 5) ? v : 0u;
                    total += v;
                }
                while (hits) {
                    const int q = __ffs(hits) - 1;
                    hits &= hits - 1u;
                    s_idx[off++] = 32 * g + (uint32_t)q;
                }
                n_idx = (int)total;
                idx_pos = 0;
                cursor += NT;
                __syncthreads();
                if (n_idx == 0) continue;
            }
            cnt = min(NT, n_idx - idx_pos);
            if (t < cnt) stage(record_of(s_idx[idx_pos + t]));
            idx_pos += cnt;
            __syncthreads();
        }
        do {
        if constexpr (CR && WHOLE) {
            // Alg. 1 with the thread's pixels inside one group.  Phase 1: the
            // group's leader tests every staged Gaussian -- independent of the
            // blending state, so the tests run back to back.  Phase 2: only the
            // Gaussians the leader kept are blended, in list order, by the
            // thread's pixels (branch-free over the pixels: almost every pixel
            // of a kept Gaussian blends, and their chains interleave).
            if (all_stopped()) continue;
            const float2 L2x = make_float2(lx0, lx0), L2y = make_float2(ly0, ly0);
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const int n32 = min(32, cnt - c0);
                // the leader's exponent for all 32 slots, two records per
                // packed instruction: each lane rounds as the scalar
                // fma(fma(a, dx, b dy), dx, fma(c dy, dy, off)) does, so the
                // decisions are those of the scalar form bit for bit; slots
                // past the batch hold stale values and are masked off
                uint32_t pass = 0;
#pragma unroll 1
                for (int i = 0; i < 32; i += 4) {
                    const float4 nx = *reinterpret_cast<const float4*>(&sL[0][c0 + i]);
                    const float4 ny = *reinterpret_cast<const float4*>(&sL[1][c0 + i]);
                    const float4 ca = *reinterpret_cast<const float4*>(&sL[2][c0 + i]);
                    const float4 cb2 = *reinterpret_cast<const float4*>(&sL[3][c0 + i]);
                    const float4 cc = *reinterpret_cast<const float4*>(&sL[4][c0 + i]);
                    const float4 of = *reinterpret_cast<const float4*>(&sL[5][c0 + i]);
                    const float4 th = *reinterpret_cast<const float4*>(&sL[6][c0 + i]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 X = h ? make_float2(nx.z, nx.w) : make_float2(nx.x, nx.y);
                        const float2 Y = h ? make_float2(ny.z, ny.w) : make_float2(ny.x, ny.y);
                        const float2 Ca = h ? make_float2(ca.z, ca.w) : make_float2(ca.x, ca.y);
                        const float2 Cb = h ? make_float2(cb2.z, cb2.w) : make_float2(cb2.x, cb2.y);
                        const float2 Cc2 = h ? make_float2(cc.z, cc.w) : make_float2(cc.x, cc.y);
                        const float2 Of = h ? make_float2(of.z, of.w) : make_float2(of.x, of.y);
                        const float2 Th = h ? make_float2(th.z, th.w) : make_float2(th.x, th.y);
                        const float2 dx = __fadd2_rn(L2x, X), dy = __fadd2_rn(L2y, Y);
                        const float2 e0 = __ffma2_rn(__ffma2_rn(Ca, dx, __fmul2_rn(Cb, dy)), dx,
                                                     __ffma2_rn(__fmul2_rn(Cc2, dy), dy, Of));
                        pass |= (e0.x >= Th.x ? 1u << (i + 2 * h) : 0u) | (e0.y >= Th.y ? 2u << (i + 2 * h) : 0u);
                    }
                }
                if (n32 < 32) pass &= (1u << n32) - 1u;
                if (COUNT) n_lead += (uint32_t)n32;
                while (pass != 0u) {
                    const int k = c0 + __ffs(pass) - 1;
                    pass &= pass - 1u;
                    const float4 A = s0[k];
                    const float4 B = s1[k];
                    const float4 Cc = s2[k];
                    const float dx = fx0 - A.x, dy = fy0 - A.y;
                    const uint32_t pos1 = pos0 + (uint32_t)k + 1u;
                    auto pixels = [&](auto clamp) {
#pragma unroll
                        for (int jj = 0; jj < PH; ++jj) {
                            const float ddy = dy + (float)jj;
                            const float rb = A.w * ddy, rc = fmaf(B.x * ddy, ddy, B.y);
#pragma unroll
                            for (int i = 0; i < PW; ++i) {
                                const int p = jj * PW + i;
                                const float ddx = dx + (float)i;
                                const float e = fmaf(fmaf(A.z, ddx, rb), ddx, rc);
                                blend_one<decltype(clamp)::value, COUNT>(T[p], cr[p], cg[p], cb[p], nc[p], tau[p],
                                                                         e, B.z, Cc, pos1, amax, n_eval, n_blend);
                            }
                        }
                    };
                    if (Cc.w != 0.f) pixels(std::true_type{});
                    else pixels(std::false_type{});
                    // with four or more pixels a thread leaves its kept list
                    // once they have all stopped (a stopped pixel never
                    // blends again, so with fewer the test costs more than
                    // the rest of the batch's kept list)
                    if (NP >= 4 && all_stopped()) break;
                }
                if (all_stopped()) break;
            }
            continue;
        }
        if constexpr (!(CR && WHOLE))
        for (int k = 0; k < cnt; ++k) {
            // group liveness for Alg. 1; the plain rule only stops the walk
            const uint32_t live = CR ? live_mask() : (all_stopped() ? 0u : 1u);
            if (live == 0u) break;
            const float4 A = s0[k];
            const float4 B = s1[k];
            const float4 Cc = s2[k];
            const bool clamp = Cc.w != 0.f;
            const float dx = fx0 - A.x, dy = fy0 - A.y;
            const uint32_t pos1 = pos0 + (uint32_t)k + 1u;
            // exponent of alpha = 2^e at pixel offset (i, j) of this thread
            auto expo = [&](int i, int jj) {
                const float ddx = dx + (float)i, ddy = dy + (float)jj;
                return fmaf(fmaf(A.z, ddx, A.w * ddy), ddx, fmaf(B.x * ddy, ddy, B.y));
            };
            auto blend = [&](int p, float e) {
                if (clamp)
                    blend_one<true, COUNT>(T[p], cr[p], cg[p], cb[p], nc[p], tau[p], e, B.z, Cc, pos1, amax, n_eval,
                                           n_blend);
                else
                    blend_one<false, COUNT>(T[p], cr[p], cg[p], cb[p], nc[p], tau[p], e, B.z, Cc, pos1, amax, n_eval,
                                            n_blend);
            };
            if (CR) {
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
                                blend(p, (i == 0 && jj == 0) ? e0 : expo(gx * GW + i, gy * GH + jj));
                            }
                    }
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p) blend(p, expo(p % PW, p / PW));
            }
        }
        } while (0);
        pos0 += (uint32_t)cnt;
        if (!BLOCKS && ckpt != nullptr && (pos0 & (kCkptL - 1u)) == 0u && pos0 < rg.y - rg.x) {
            float4* slot = ckpt + (size_t)((rg.x >> kCkptShift) + (pos0 >> kCkptShift)) * (TW * TH);
#pragma unroll
            for (int p = 0; p < NP; ++p)
                if (bx + p % PW < C.W && by + p / PW < C.H)
                    slot[(by - ty * TH + p / PW) * TW + (bx - tx * TW + p % PW)] = make_float4(T[p], cr[p], cg[p], cb[p]);
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
            if (cfin != nullptr) cfin[C.pix_offset + o] = make_float4(T[p], cr[p], cg[p], cb[p]);
        }
    }
    // the CTA that finishes a camera's last tile stamps the view's end time
    if (view_done) {
        __syncthreads();
        if (t == 0 && atomicAdd(view_done + lo, 1u) + 1u == (uint32_t)(C.tiles_x * C.tiles_y))
            view_end[lo] = global_ns();
    }
}


// Persistent launch of the variant (raster_queue.cu): a.queue counts the
// units taken, a.block_order gives their order.
template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool BLOCKS>
void launch_raster_queue(const RasterArgs& a, cudaStream_t s);

#define SEELE_RASTER_PARAMS                                                                                      \
    const uint32_t *__restrict__ starts, const uint32_t *__restrict__ ends, const uint32_t *__restrict__ inst_rec, \
        const uint32_t *__restrict__ inst_mask, const uint32_t *__restrict__ mask_summary,                       \
        const uint32_t *__restrict__ block_order, const float4 *__restrict__ rec, const CamDev *__restrict__ cams,  \
        int n_cams, FrameParams fp, float *__restrict__ out_rgb, float *__restrict__ out_T,                      \
        uint32_t *__restrict__ out_nc, DeviceStatus *__restrict__ counters,                                      \
        unsigned long long *__restrict__ view_end, uint32_t *__restrict__ view_done, float4 *__restrict__ ckpt,   \
        float4 *__restrict__ cfin
#define SEELE_RASTER_ARGS                                                                                         \
    starts, ends, inst_rec, inst_mask, mask_summary, block_order, rec, cams, n_cams, fp, out_rgb, out_T, out_nc, \
        counters, view_end, view_done, ckpt, cfin

// One CTA per list unit (tile, or tile of a block), in the order of blockIdx.
template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool COUNT, bool BLOCKS>
__global__ void __launch_bounds__((TW / PW) * (TH / PH)) raster_fwd_kernel(SEELE_RASTER_PARAMS) {
    pdl_enter();
    raster_unit<TW, TH, PW, PH, GW, GH, CR, COUNT, BLOCKS>(blockIdx.x, SEELE_RASTER_ARGS);
}

// Persistent: as many CTAs as fit the SMs at once; each takes the next unit
// from an atomic queue (the order block_order gives) until none is left, so
// the units are started strictly in queue order and no CTA launch is paid
// per unit.
template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR, bool BLOCKS>
__global__ void __launch_bounds__((TW / PW) * (TH / PH))
    raster_queue_kernel(SEELE_RASTER_PARAMS, uint32_t n_items, uint32_t* __restrict__ queue) {
    __shared__ uint32_t s_item;
    pdl_enter();
    for (;;) {
        __syncthreads();  // every thread has read the previous item; shared staging is free
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) break;
        raster_unit<TW, TH, PW, PH, GW, GH, CR, false, BLOCKS>(item, SEELE_RASTER_ARGS);
    }
}

}  // namespace seele
