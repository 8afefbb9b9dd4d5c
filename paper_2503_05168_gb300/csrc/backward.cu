// backward.cu -- gradients of the render for fine-tuning (Sec. 3.5: the
// hybrid preprocessing and the contribution-aware skips are left out of the
// gradient; every skip and stop decision of the forward pass is replayed and
// held fixed).
//
// raster_bwd_kernel: one CTA per 256-entry chunk of a tile's list (one per
//   tile for lists that short), the same 2x2-pixels-per-thread layout as
//   the forward pass.  Each pixel walks its chunk back to front from its
//   last blended entry; the transmittance before an entry is recomputed by
//   T_j = T_{j+1} / (1 - alpha_j) from the state at the chunk's end (the
//   final T, or the forward pass's checkpoint there), and S, the colour
//   accumulated behind entry j, gives
//     dC/dc_j = T_j alpha_j,   dC/dalpha_j = T_j c_j - S / (1 - alpha_j).
//   Only g . dC/dalpha_j enters the gradient (g = dL/dC of the pixel), so a
//   pixel keeps the scalar g . S instead of S.  Gradients w.r.t. the record
//   (u, v, cA, cB, cC, log2 o, r, g, b) are summed over the warp's pixels and
//   added with one atomic per value; the exponent's terms are summed as
//   moments of the pixel offsets (sum de dx, de dy, de dx^2, ...) and turned
//   into du, dv once per entry.  The pixels of a thread run branch-free under
//   a per-pixel predicate.
//   8x8 tiles (one warp per tile, two pixels per lane) sum in two phases:
//   the lanes write each blended entry's per-pixel terms (de, colour weight)
//   to one of eight shared-memory slots; once the slots are full, lane
//   (e, q) adds up entry e over the pixels of columns q and q + 4, with the
//   pixel offsets as constants, and four lanes combine an entry's totals --
//   instead of nine per-pixel accumulations and a nine-value warp sum per
//   entry.
// preprocess_bwd_kernel: one thread per Gaussian, summing over cameras, runs
//   the chain rule back through the raster record, the conic, the EWA
//   projection, the covariance, the quaternion and the SH colour.
#include "common.cuh"
#include "kernels.h"

namespace seele {

constexpr float kLn2 = 0.69314718055994531f;

__device__ __forceinline__ float ex2_approx_b(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx_b(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Warp totals of nine per-lane values.  Values 0..7 are reduced by
// recursive halving: at each exchange a lane sends the half of its values
// that its partner keeps and adds the half it keeps, so after the exchanges
// over lane bits 4, 3 and 2 (then 1 and 0 on the one value left) lane l
// holds the total of value (l >> 2) & 7 -- 9 shuffles instead of 40.  Value
// 8 takes a plain butterfly.  Returns (total of value (l >> 2) & 7, total of
// value 8).
__device__ __forceinline__ float2 warp_sum9(const float (&v)[9], int lane) {
    constexpr unsigned kAll = 0xffffffffu;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 16;
        a[i] = (hi ? v[i + 4] : v[i]) + __shfl_xor_sync(kAll, hi ? v[i] : v[i + 4], 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 8;
        a[i] = (hi ? a[i + 2] : a[i]) + __shfl_xor_sync(kAll, hi ? a[i] : a[i + 2], 8);
    }
    {
        const bool hi = lane & 4;
        a[0] = (hi ? a[1] : a[0]) + __shfl_xor_sync(kAll, hi ? a[0] : a[1], 4);
    }
    a[0] += __shfl_xor_sync(kAll, a[0], 2);
    a[0] += __shfl_xor_sync(kAll, a[0], 1);
    float w = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kAll, w, o);
    return make_float2(a[0], w);
}

// Slots of the two-phase sum (8x8 tiles): 8 entries of 64 pixel pairs
// (de, weight); the stride of 132 floats keeps the phase-B loads of a
// half-warp in distinct banks.
constexpr int kSlots = 8;
constexpr int kSlotStride = 132;

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR>
__global__ void __launch_bounds__((TW / PW) * (TH / PH))
    raster_bwd_kernel(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ ends,
                      const uint32_t* __restrict__ inst_rec, const float4* __restrict__ rec,
                      const CamDev* __restrict__ cams, int n_cams, FrameParams fp, const float* __restrict__ dL_drgb,
                      const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
                      float* __restrict__ grad_rec, const uint32_t* __restrict__ tile_order,
                      const float4* __restrict__ ckpt, const float4* __restrict__ cfin,
                      const uint32_t* __restrict__ chunk_map, uint32_t n_tiles) {
    constexpr int NT = (TW / PW) * (TH / PH);
    constexpr int NP = PW * PH;
    constexpr int TXN = TW / PW;
    // a group is a sub-block of the thread's pixels, or one or more whole
    // thread blocks (the forward pass's rule); GWL x GHL is its part here
    constexpr bool WHOLE = GW % PW == 0 && GH % PH == 0;
    constexpr int GWL = WHOLE ? PW : GW, GHL = WHOLE ? PH : GH;
    // two-phase sum: one warp per 8x8 tile, lane l holds pixels 2l, 2l + 1
    constexpr bool SLOTS = TW == 8 && TH == 8 && PW == 2 && PH == 1;
    static_assert(!SLOTS || NT == 32, "one warp per tile");
    __shared__ float4 s0[NT], s1[NT], s2[NT];
    __shared__ uint32_t s_r[NT];
    __shared__ uint32_t s_max;
    __shared__ __align__(16) float s_x[SLOTS ? kSlots * kSlotStride : 4];
    __shared__ float4 s_g[SLOTS ? TW * TH : 1];  // dL/dC of the tile's pixels
    __shared__ int s_slot[kSlots];

    // CTA -> (tile, chunk): the first n_tiles CTAs take chunk 0 of every
    // tile, the others the later chunks of long lists (see kCkptShift)
    uint32_t gtile, chunk = 0;
    if (blockIdx.x < n_tiles) {
        gtile = tile_order ? __ldg(tile_order + blockIdx.x) : blockIdx.x;
    } else {
        gtile = __ldg(chunk_map + (blockIdx.x - n_tiles));
        if (gtile == 0xffffffffu) return;
        chunk = (blockIdx.x - n_tiles) - (__ldg(starts + gtile) >> kCkptShift);
    }
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_offset <= gtile) lo = mid; else hi = mid - 1;
    }
    const CamDev& C = cams[lo];
    const uint32_t lt = gtile - C.tile_offset;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int t = threadIdx.x, lane = t & 31;
    const int bx = tx * TW + (t % TXN) * PW, by = ty * TH + (t / TXN) * PH;
    uint32_t start = __ldg(starts + gtile), end = __ldg(ends + gtile);
    if (start >= end) start = end = 0;

    const size_t plane = (size_t)C.W * C.H;
    const float* gimg = dL_drgb + 3 * (size_t)C.pix_offset;
    float T[NP], g0[NP], g1[NP], g2[NP], gS[NP];  // gS = g . (colour behind)
    uint32_t last[NP];
    uint32_t my_max = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int x = bx + p % PW, y = by + p / PW;
        T[p] = 1.f;
        g0[p] = g1[p] = g2[p] = 0.f;
        gS[p] = 0.f;
        last[p] = 0;
        if (x < C.W && y < C.H) {
            const size_t o = (size_t)y * C.W + x;
            T[p] = __ldg(T_final + C.pix_offset + o);
            last[p] = __ldg(n_contrib + C.pix_offset + o);
            g0[p] = __ldg(gimg + o);
            g1[p] = __ldg(gimg + plane + o);
            g2[p] = __ldg(gimg + 2 * plane + o);
            my_max = max(my_max, last[p]);
        }
        if constexpr (SLOTS) s_g[NP * t + p] = make_float4(g0[p], g1[p], g2[p], 0.f);
    }
    if (t == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, my_max);
    __syncthreads();
    const uint32_t lmax = min(s_max, end - start);
    // this CTA's part of the list; with checkpoints, chunk [c L, (c + 1) L)
    const uint32_t wlo = ckpt ? chunk * kCkptL : 0u;
    const uint32_t whi = ckpt ? min(lmax, (chunk + 1u) * kCkptL) : lmax;
    if (wlo >= whi) return;
    if (whi < lmax) {
        // start from the state the forward pass saved at the chunk's end:
        // T there, and the colour behind it = final colour - colour so far
        const float4* slot = ckpt + (size_t)((start >> kCkptShift) + chunk + 1u) * (TW * TH);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int x = bx + p % PW, y = by + p / PW;
            if (x < C.W && y < C.H) {
                const float4 k = __ldg(slot + (y - ty * TH) * TW + (x - tx * TW));
                const float4 f = __ldg(cfin + C.pix_offset + (size_t)y * C.W + x);
                T[p] = k.x;
                gS[p] = g0[p] * (f.y - k.y) + g1[p] * (f.z - k.z) + g2[p] * (f.w - k.w);
            }
        }
    }
    const float fx0 = (float)bx + 0.5f, fy0 = (float)by + 0.5f;
    const float Xc = (float)(tx * TW) + 0.5f * TW, Yc = (float)(ty * TH) + 0.5f * TH;  // the tile's centre
    // Phase B of the two-phase sum over the ns filled slots.  Lane (e, q)
    // takes pixels q + 4 i (column q + 4 (i & 1), row i >> 1): moments of de
    // about column q and its colour sums, moved to the tile's centre,
    // summed over the entry's four lanes, then about the Gaussian's centre.
    auto flush = [&](int ns) {
        constexpr unsigned kAll = 0xffffffffu;
        __syncwarp();
        const int e = lane & 7, q = lane >> 3;
        float N0 = 0.f, Nx = 0.f, Ny = 0.f, Nxx = 0.f, Nxy = 0.f, Nyy = 0.f, cr = 0.f, cg = 0.f, cb = 0.f;
        if (e < ns) {
            const float* xr = s_x + e * kSlotStride + 2 * q;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float2 xv = *reinterpret_cast<const float2*>(xr + 8 * i);
                const float4 g = s_g[q + 4 * i];
                const float oy = (float)(i >> 1) - 3.5f;  // row offset from the centre
                N0 += xv.x;
                Ny = fmaf(xv.x, oy, Ny);
                Nyy = fmaf(xv.x, oy * oy, Nyy);
                if (i & 1) {  // column q + 4: 4 right of column q
                    const float t4 = 4.f * xv.x;
                    Nx += t4;
                    Nxx = fmaf(t4, 4.f, Nxx);
                    Nxy = fmaf(t4, oy, Nxy);
                }
                cr = fmaf(xv.y, g.x, cr);
                cg = fmaf(xv.y, g.y, cg);
                cb = fmaf(xv.y, g.z, cb);
            }
        }
        const float cq = (float)q - 3.5f;  // column q's offset from the centre
        float M[9] = {N0, fmaf(cq, N0, Nx), Ny, fmaf(cq, fmaf(2.f, Nx, cq * N0), Nxx), fmaf(cq, Ny, Nxy), Nyy,
                      cr, cg, cb};
#pragma unroll
        for (int v = 0; v < 9; ++v) {
            M[v] += __shfl_xor_sync(kAll, M[v], 8);
            M[v] += __shfl_xor_sync(kAll, M[v], 16);
        }
        if (e < ns) {
            const int k = s_slot[e];
            const float4 A = s0[k];
            const float cC = s1[k].x;
            const float U = Xc - A.x, V = Yc - A.y;  // pixel offset dx = ox + U, dy = oy + V
            const float sx = fmaf(U, M[0], M[1]), sy = fmaf(V, M[0], M[2]);
            const float sxx = fmaf(U, fmaf(U, M[0], 2.f * M[1]), M[3]);
            const float sxy = fmaf(U, fmaf(V, M[0], M[2]), fmaf(V, M[1], M[4]));
            const float syy = fmaf(V, fmaf(V, M[0], 2.f * M[2]), M[5]);
            // de/du = -(2 cA dx + cB dy), de/dv = -(cB dx + 2 cC dy); the
            // slots hold de / ln 2
            const float du = -fmaf(2.f * A.z, sx, A.w * sy) * kLn2;
            const float dv = -fmaf(A.w, sx, 2.f * cC * sy) * kLn2;
            const float a0 = q == 0 ? du : q == 1 ? dv : q == 2 ? sxx * kLn2 : sxy * kLn2;
            const float a1 = q == 0 ? syy * kLn2 : q == 1 ? M[0] * kLn2 : q == 2 ? M[6] : M[7];
            float* G = grad_rec + 12 * (size_t)s_r[k];
            if (a0 != 0.f) atomicAdd(G + q, a0);
            if (a1 != 0.f) atomicAdd(G + 4 + q, a1);
            if (q == 0 && M[8] != 0.f) atomicAdd(G + 8, M[8]);
        }
        __syncwarp();
    };
    const float lx0 = (float)(bx / GW * GW) + 0.5f, ly0 = (float)(by / GH * GH) + 0.5f;  // the group's leader
    const float amax = fp.alpha_max;

    int n_slot = 0;  // filled slots (warp-uniform)
    for (int b1 = (int)whi; b1 > (int)wlo; b1 -= NT) {
        const int b0 = max((int)wlo, b1 - NT);
        __syncthreads();
        if (t < b1 - b0) {
            const uint32_t r = __ldg(inst_rec + start + b0 + t);
            s_r[t] = r;
            s0[t] = __ldg(rec + (size_t)kRecF4 * r);
            s1[t] = __ldg(rec + (size_t)kRecF4 * r + 1);
            s2[t] = __ldg(rec + (size_t)kRecF4 * r + 2);
        }
        __syncthreads();
        for (int k = b1 - b0 - 1; k >= 0; --k) {
            const uint32_t j = (uint32_t)(b0 + k);  // list position
            const float4 A = s0[k];
            const float4 B = s1[k];
            const float4 Cc = s2[k];
            const float dx = fx0 - A.x, dy = fy0 - A.y;
            // the forward pass's exponent, bit for bit
            auto expo = [&](int i, int jj) {
                const float ddx = dx + (float)i, ddy = dy + (float)jj;
                return fmaf(fmaf(A.z, ddx, A.w * ddy), ddx, fmaf(B.x * ddy, ddy, B.y));
            };
            // per lane: sums of de, de dx, de dy, de dx^2, de dx dy, de dy^2 and
            // of the colour weights
            float sde = 0.f, sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
            const bool clampable = Cc.w != 0.f;  // the record's alpha can reach alpha_max
            // Which of the thread's pixels did the forward pass blend this
            // entry into (before its last blend, inside the support, alpha >=
            // alpha_theta, its group kept the entry)?  Cheap; the gradient
            // terms below run only when some lane of the warp has one.
            float ev[NP];
            uint32_t mbits = 0;
#pragma unroll
            for (int gy = 0; gy < PH / GHL; ++gy)
#pragma unroll
                for (int gx = 0; gx < PW / GWL; ++gx) {
                    bool need = false;
#pragma unroll
                    for (int jj = 0; jj < GHL; ++jj)
#pragma unroll
                        for (int i = 0; i < GWL; ++i) need |= j < last[(gy * GHL + jj) * PW + gx * GWL + i];
                    bool lead = need;
                    if (CR && need) {
                        if (WHOLE) {
                            const float lx = lx0 - A.x, ly = ly0 - A.y;
                            lead = fmaf(fmaf(A.z, lx, A.w * ly), lx, fmaf(B.x * ly, ly, B.y)) >= B.z;
                        } else {
                            lead = expo(gx * GW, gy * GH) >= B.z;
                        }
                    }
#pragma unroll
                    for (int jj = 0; jj < GHL; ++jj)
#pragma unroll
                        for (int i = 0; i < GWL; ++i) {
                            const int pi = gx * GWL + i, pj = gy * GHL + jj;
                            const int p = pj * PW + pi;
                            ev[p] = expo(pi, pj);
                            mbits |= (lead && j < last[p] && ev[p] >= B.z) ? 1u << p : 0u;
                        }
                }
            if (!__any_sync(0xffffffffu, mbits != 0u)) continue;
            if constexpr (SLOTS) {
                // phase A: the pixels' de / ln 2 and colour weights into a slot
                float de[NP], wg[NP];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const bool m = (mbits >> p) & 1u;
                    float al = ex2_approx_b(ev[p]);
                    if (clampable) al = fminf(amax, al);
                    const float inv = rcp_approx_b(1.f - al);
                    const float Tb = T[p] * inv;
                    wg[p] = m ? Tb * al : 0.f;
                    const float gc = fmaf(g2[p], Cc.z, fmaf(g1[p], Cc.y, g0[p] * Cc.x));
                    const float dal = fmaf(Tb, gc, -gS[p] * inv);
                    gS[p] = fmaf(wg[p], gc, gS[p]);
                    T[p] = m ? Tb : T[p];
                    de[p] = (m && (!clampable || al < amax)) ? dal * al : 0.f;
                }
                *reinterpret_cast<float4*>(s_x + n_slot * kSlotStride + 4 * lane) =
                    make_float4(de[0], wg[0], de[1], wg[1]);
                if (lane == 0) s_slot[n_slot] = k;
                if (++n_slot == kSlots) {
                    flush(n_slot);
                    n_slot = 0;
                }
                continue;
            }
            // One pixel of the entry, branch-free: for a pixel the entry was
            // not blended into every update below adds zero or keeps the value.
            auto pixel = [&](int p, int pi, int pj) {
                const bool m = (mbits >> p) & 1u;
                float al = ex2_approx_b(ev[p]);
                if (clampable) al = fminf(amax, al);
                // 1 - alpha >= 0.01 (the clamp): the approximate reciprocal
                // keeps T_before within a few ulp per entry
                const float inv = rcp_approx_b(1.f - al);
                const float Tb = T[p] * inv;  // transmittance before this entry
                const float wgt = m ? Tb * al : 0.f;
                const float gc = fmaf(g2[p], Cc.z, fmaf(g1[p], Cc.y, g0[p] * Cc.x));
                const float dal = fmaf(Tb, gc, -gS[p] * inv);
                dr = fmaf(wgt, g0[p], dr);
                dg = fmaf(wgt, g1[p], dg);
                db = fmaf(wgt, g2[p], db);
                gS[p] = fmaf(wgt, gc, gS[p]);
                T[p] = m ? Tb : T[p];
                // at the clamp alpha is constant: no gradient through e
                const float de = (m && (!clampable || al < amax)) ? dal * al * kLn2 : 0.f;
                const float ddx = dx + (float)pi, ddy = dy + (float)pj;
                const float ex = de * ddx, ey = de * ddy;
                sde += de;
                sx += ex;
                sy += ey;
                sxx = fmaf(ex, ddx, sxx);
                sxy = fmaf(ex, ddy, sxy);
                syy = fmaf(ey, ddy, syy);
            };
#pragma unroll
            for (int pj = 0; pj < PH; ++pj)
#pragma unroll
                for (int pi = 0; pi < PW; ++pi) pixel(pj * PW + pi, pi, pj);
            // e = cA dx^2 + cB dx dy + cC dy^2 + log2 o with dx = x - u:
            // de/du = -(2 cA dx + cB dy), de/dv = -(cB dx + 2 cC dy)
            const float du = -fmaf(2.f * A.z, sx, A.w * sy);
            const float dv = -fmaf(A.w, sx, 2.f * B.x * sy);
            const float v[9] = {du, dv, sxx, sxy, syy, sde, dr, dg, db};
            const float2 tot = warp_sum9(v, lane);
            float* G = grad_rec + 12 * (size_t)s_r[k];
            if ((lane & 3) == 0 && tot.x != 0.f) atomicAdd(G + (lane >> 2), tot.x);
            if (lane == 1 && tot.y != 0.f) atomicAdd(G + 8, tot.y);
        }
        if constexpr (SLOTS) {
            // the staged records are replaced next: sum the filled slots now
            if (n_slot > 0) flush(n_slot);
            n_slot = 0;
        }
    }
}

// d/d(x, y, z) of the real SH basis of preprocess.cu (same polynomials).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float (*dY)[3]) {
    constexpr float c0 = 0.28209479177387814f, c1 = 0.48860251190291992f, c2a = 1.0925484305920792f,
                    c2b = 0.31539156525252005f, c2c = 0.54627421529603959f, c3a = 0.59004358992664352f,
                    c3b = 2.8906114426405538f, c3c = 0.45704579946446572f, c3d = 0.37317633259011540f,
                    c3e = 1.4453057213202769f;
    Y[0] = c0;
    dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    if (DEG > 0) {
        Y[1] = -c1 * y; dY[1][0] = 0.f; dY[1][1] = -c1; dY[1][2] = 0.f;
        Y[2] = c1 * z;  dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = c1;
        Y[3] = -c1 * x; dY[3][0] = -c1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    }
    if (DEG > 1) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = c2a * x * y;  dY[4][0] = c2a * y; dY[4][1] = c2a * x; dY[4][2] = 0.f;
        Y[5] = -c2a * y * z; dY[5][0] = 0.f; dY[5][1] = -c2a * z; dY[5][2] = -c2a * y;
        Y[6] = c2b * (2.f * zz - xx - yy);
        dY[6][0] = -2.f * c2b * x; dY[6][1] = -2.f * c2b * y; dY[6][2] = 4.f * c2b * z;
        Y[7] = -c2a * x * z; dY[7][0] = -c2a * z; dY[7][1] = 0.f; dY[7][2] = -c2a * x;
        Y[8] = c2c * (xx - yy); dY[8][0] = 2.f * c2c * x; dY[8][1] = -2.f * c2c * y; dY[8][2] = 0.f;
        if (DEG > 2) {
            Y[9] = -c3a * y * (3.f * xx - yy);
            dY[9][0] = -6.f * c3a * x * y; dY[9][1] = -c3a * (3.f * xx - 3.f * yy); dY[9][2] = 0.f;
            Y[10] = c3b * x * y * z;
            dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
            Y[11] = -c3c * y * (4.f * zz - xx - yy);
            dY[11][0] = 2.f * c3c * x * y; dY[11][1] = -c3c * (4.f * zz - xx - 3.f * yy);
            dY[11][2] = -8.f * c3c * y * z;
            Y[12] = c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            dY[12][0] = -6.f * c3d * x * z; dY[12][1] = -6.f * c3d * y * z;
            dY[12][2] = c3d * (6.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -c3c * x * (4.f * zz - xx - yy);
            dY[13][0] = -c3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * c3c * x * y;
            dY[13][2] = -8.f * c3c * x * z;
            Y[14] = c3e * z * (xx - yy);
            dY[14][0] = 2.f * c3e * x * z; dY[14][1] = -2.f * c3e * y * z; dY[14][2] = c3e * (xx - yy);
            Y[15] = -c3a * x * (xx - 3.f * yy);
            dY[15][0] = -c3a * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * c3a * x * y; dY[15][2] = 0.f;
        }
    }
}

// ONE: a single camera (the training step).  Its SH gradients are written
// once, so they go through shared memory and leave as whole rows; with
// several cameras they are summed in registers over the cameras.
template <int DEG, bool ONE>
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(SceneDev sc, const CamDev* __restrict__ cams,
                                                             FrameParams fp, const uint32_t* __restrict__ tiles,
                                                             const float* __restrict__ grad_rec,
                                                             float* __restrict__ d_means, float* __restrict__ d_ls,
                                                             float* __restrict__ d_quat, float* __restrict__ d_logit,
                                                             float* __restrict__ d_sh,
                                                             const uint32_t* __restrict__ order) {
    constexpr int NC = (DEG + 1) * (DEG + 1);
    constexpr int NF = 3 * NC;
    // One camera: each thread's SH gradient row leaves through shared memory
    // (whole rows per CTA).  With 16-byte rows, a borrowed scene's SH rows
    // also come in through the same slot, copied asynchronously when the
    // thread starts, so that the loads overlap the projection's recompute;
    // the row stride is then a multiple of 16 bytes and odd in 16-byte units
    // (float4 accesses in distinct banks), else odd in words.
    constexpr bool STAGE = ONE && NF % 4 == 0;
    constexpr int RS = STAGE ? ((NF / 4) % 2 == 0 ? NF + 4 : NF) : (NF | 1);
    __shared__ __align__(16) float s_sh[ONE ? 128 * RS : 4];
    const int t = threadIdx.x;
    const int g = blockIdx.x * blockDim.x + t;
    const bool aos = sc.means != nullptr;  // a BORROW scene read in place
    const bool staged = STAGE && aos;
    if (staged && g < fp.n) {
        const float4* src = reinterpret_cast<const float4*>(sc.shc + (size_t)g * NF);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_sh + t * RS);
#pragma unroll
        for (int jp = 0; jp < NF / 4; ++jp)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * jp), "l"(src + jp) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const float4* my_sh = reinterpret_cast<const float4*>(s_sh + t * RS);
    bool wrote = false;
    if (g < fp.n) {
    float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
    float gsh[ONE ? 1 : NF];
    if constexpr (!ONE) {
#pragma unroll
        for (int i = 0; i < NF; ++i) gsh[i] = 0.f;
    }
    const float4 pl = aos ? scene_pos_logit<true>(sc, g) : scene_pos_logit<false>(sc, g);
    const float4 q4 = aos ? scene_quat<true>(sc, g) : scene_quat<false>(sc, g);
    const float4 ls = aos ? scene_log_scale<true>(sc, g) : scene_log_scale<false>(sc, g);

    for (int ci = 0; ci < (ONE ? 1 : fp.n_cams); ++ci) {
        const size_t rid = (size_t)ci * fp.n + g;
        if (__ldg(tiles + rid) == 0u) continue;
        // the record's 9 gradients, 48-byte aligned: two 16-byte loads and one word
        const float* G = grad_rec + 12 * rid;
        const float4 G0 = __ldg(reinterpret_cast<const float4*>(G));
        const float4 G1 = __ldg(reinterpret_cast<const float4*>(G) + 1);
        const float gu = G0.x, gv = G0.y, gcA = G0.z, gcB = G0.w, gcC = G1.x, glo = G1.y;
        const float grgb[3] = {G1.z, G1.w, __ldg(G + 8)};
        const CamDev& C = cams[ci];

        // ---- recompute the forward quantities
        const float X = fmaf(C.R[0], pl.x, fmaf(C.R[1], pl.y, fmaf(C.R[2], pl.z, C.t[0])));
        const float Y = fmaf(C.R[3], pl.x, fmaf(C.R[4], pl.y, fmaf(C.R[5], pl.z, C.t[1])));
        const float Z = fmaf(C.R[6], pl.x, fmaf(C.R[7], pl.y, fmaf(C.R[8], pl.z, C.t[2])));
        const float xz = X / Z, yz = Y / Z;
        const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
        const float qinv = rsqrtf(qn2);
        const float qw = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
        const float s[3] = {expf(ls.x), expf(ls.y), expf(ls.z)};
        float R[9];
        R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
        R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
        R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
        float WM[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                WM[3 * i + j] = (C.R[3 * i] * R[j] + C.R[3 * i + 1] * R[3 + j] + C.R[3 * i + 2] * R[6 + j]) * s[j];
        const float jx = C.fx / Z, jy = C.fy / Z;
        float N0[3], N1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            N0[j] = jx * (WM[j] - xz * WM[6 + j]);
            N1[j] = jy * (WM[3 + j] - yz * WM[6 + j]);
        }
        const float a = N0[0] * N0[0] + N0[1] * N0[1] + N0[2] * N0[2] + fp.dilation;
        const float b = N0[0] * N1[0] + N0[1] * N1[1] + N0[2] * N1[2];
        const float c = N1[0] * N1[0] + N1[1] * N1[1] + N1[2] * N1[2] + fp.dilation;
        const float det = a * c - b * b;
        const float inv = 1.f / det;
        const float Pa = c * inv, Pb = -b * inv, Pc = a * inv;  // conic [[Pa, Pb], [Pb, Pc]]

        // ---- record -> conic: cA = -L/2 Pa, cB = -L Pb, cC = -L/2 Pc
        const float gPa = -0.5f * kLog2e * gcA, gPb = -kLog2e * gcB, gPc = -0.5f * kLog2e * gcC;
        // conic = Sigma'^-1: dL/dSigma' = -P Gs P with Gs the symmetric gradient
        // [[gPa, gPb/2], [gPb/2, gPc]]
        const float h = 0.5f * gPb;
        const float m00 = gPa * Pa + h * Pb, m01 = gPa * Pb + h * Pc;  // (Gs P) row 0
        const float m10 = h * Pa + gPc * Pb, m11 = h * Pb + gPc * Pc;  // (Gs P) row 1
        const float S00 = -(Pa * m00 + Pb * m10);
        const float S01 = -(Pa * m01 + Pb * m11);
        const float S11 = -(Pb * m01 + Pc * m11);
        // Sigma' = [N0.N0, N0.N1; N1.N0, N1.N1] + dilation
        float gN0[3], gN1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gN0[j] = 2.f * S00 * N0[j] + 2.f * S01 * N1[j];
            gN1[j] = 2.f * S11 * N1[j] + 2.f * S01 * N0[j];
        }
        // N0 = jx (WM0 - xz WM2), N1 = jy (WM1 - yz WM2)
        float gWM[9];
        float gjx = 0.f, gjy = 0.f, gxz = 0.f, gyz = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gjx += gN0[j] * (WM[j] - xz * WM[6 + j]);
            gjy += gN1[j] * (WM[3 + j] - yz * WM[6 + j]);
            gxz -= gN0[j] * jx * WM[6 + j];
            gyz -= gN1[j] * jy * WM[6 + j];
            gWM[j] = gN0[j] * jx;
            gWM[3 + j] = gN1[j] * jy;
            gWM[6 + j] = -gN0[j] * jx * xz - gN1[j] * jy * yz;
        }
        // screen position u = fx xz + cx, v = fy yz + cy
        gxz += gu * C.fx;
        gyz += gv * C.fy;
        // xz = X / Z, yz = Y / Z, jx = fx / Z, jy = fy / Z
        const float iz = 1.f / Z;
        const float gX = gxz * iz, gY = gyz * iz;
        const float gZ = -(gxz * xz + gyz * yz) * iz - (gjx * jx + gjy * jy) * iz;
        // X_cam = W m + t
#pragma unroll
        for (int i = 0; i < 3; ++i) gm[i] += C.R[i] * gX + C.R[3 + i] * gY + C.R[6 + i] * gZ;
        // WM = W R diag(s): gM = W^T gWM, then split into R and s
        float gRs[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) gRs[3 * i + j] = C.R[i] * gWM[j] + C.R[3 + i] * gWM[3 + j] + C.R[6 + i] * gWM[6 + j];
        float gR[9];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                gR[3 * i + j] = gRs[3 * i + j] * s[j];
                acc += gRs[3 * i + j] * R[3 * i + j];
            }
            gls[j] += acc * s[j];  // d/d log s = s d/ds
        }
        // rotation of the unit quaternion, then the normalisation
        const float gqw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
        const float gqx = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - qw * gR[5] + qz * gR[6] +
                                 qw * gR[7] - 2.f * qx * gR[8]);
        const float gqy = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + qw * gR[2] + qx * gR[3] + qz * gR[5] - qw * gR[6] +
                                 qz * gR[7] - 2.f * qy * gR[8]);
        const float gqz = 2.f * (-2.f * qz * gR[0] - qw * gR[1] + qx * gR[2] + qw * gR[3] - 2.f * qz * gR[4] +
                                 qy * gR[5] + qx * gR[6] + qy * gR[7]);
        const float dotq = qw * gqw + qx * gqx + qy * gqy + qz * gqz;
        gq[0] += (gqw - qw * dotq) * qinv;
        gq[1] += (gqx - qx * dotq) * qinv;
        gq[2] += (gqy - qy * dotq) * qinv;
        gq[3] += (gqz - qz * dotq) * qinv;
        // opacity: log2 o = -log2(1 + e^-l)  ->  d/dl = (1 - o) / ln 2
        const float o = 1.f / (1.f + expf(-pl.w));
        glogit += glo * (1.f - o) / kLn2;
        // colour: rgb = max(0, sum_k sh_k Y_k(d) + 0.5), d = unit(m - campos)
        float dd[3] = {pl.x - C.campos[0], pl.y - C.campos[1], pl.z - C.campos[2]};
        const float rn = rsqrtf(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        dd[0] *= rn;
        dd[1] *= rn;
        dd[2] *= rn;
        float Yb[NC], dY[NC][3];
        sh_basis_grad<DEG>(dd[0], dd[1], dd[2], Yb, dY);
        // the coefficients stream in twice (the second time from L1):
        // first the raw colour, then w_k = sum_c gc_c sh_kc, so that the
        // direction gradient is sum_k w_k grad Y_k
        constexpr int NPL = (NF + 3) / 4;
        if (staged) asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's own row
        auto sh4 = [&](int jp) {
            if (staged) return my_sh[jp];
            return aos ? scene_sh4<true, NC>(sc, fp.n, g, jp) : scene_sh4<false, NC>(sc, fp.n, g, jp);
        };
        float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int jp = 0; jp < NPL; ++jp) {
            const float4 vv = sh4(jp);
            const float e4[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * jp + i < NF) raw[(4 * jp + i) % 3] = fmaf(e4[i], Yb[(4 * jp + i) / 3], raw[(4 * jp + i) % 3]);
        }
        const float gc[3] = {raw[0] > 0.f ? grgb[0] : 0.f, raw[1] > 0.f ? grgb[1] : 0.f,
                             raw[2] > 0.f ? grgb[2] : 0.f};
        float w[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) w[k] = 0.f;
#pragma unroll
        for (int jp = 0; jp < NPL; ++jp) {
            const float4 vv = sh4(jp);
            const float e4[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * jp + i < NF) w[(4 * jp + i) / 3] = fmaf(e4[i], gc[(4 * jp + i) % 3], w[(4 * jp + i) / 3]);
        }
        if constexpr (STAGE) {
            // the input row has been read: the gradient row replaces it
#pragma unroll
            for (int jp = 0; jp < NF / 4; ++jp)
                reinterpret_cast<float4*>(s_sh + t * RS)[jp] =
                    make_float4(Yb[(4 * jp) / 3] * gc[(4 * jp) % 3], Yb[(4 * jp + 1) / 3] * gc[(4 * jp + 1) % 3],
                                Yb[(4 * jp + 2) / 3] * gc[(4 * jp + 2) % 3], Yb[(4 * jp + 3) / 3] * gc[(4 * jp + 3) % 3]);
            wrote = true;
        } else if constexpr (ONE) {
#pragma unroll
            for (int f = 0; f < NF; ++f) s_sh[t * RS + f] = Yb[f / 3] * gc[f % 3];
            wrote = true;
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) gsh[f] = fmaf(Yb[f / 3], gc[f % 3], gsh[f]);
        }
        float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            gdir[0] = fmaf(w[k], dY[k][0], gdir[0]);
            gdir[1] = fmaf(w[k], dY[k][1], gdir[1]);
            gdir[2] = fmaf(w[k], dY[k][2], gdir[2]);
        }
        const float dot = dd[0] * gdir[0] + dd[1] * gdir[1] + dd[2] * gdir[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) gm[i] += (gdir[i] - dd[i] * dot) * rn;
    }
    // gradients go to the caller's index of the Gaussian
    const size_t go = order != nullptr ? (size_t)__ldg(order + g) : (size_t)g;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        d_means[3 * go + i] = gm[i];
        d_ls[3 * go + i] = gls[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) d_quat[4 * go + i] = gq[i];
    d_logit[go] = glogit;
    if constexpr (!ONE) {
#pragma unroll
        for (int i = 0; i < NF; ++i) d_sh[go * NF + i] = gsh[i];
    }
    }  // g < n
    if constexpr (ONE) {
        // a row copied in but not replaced (no tile reached): its copy lands first
        if (staged) asm volatile("cp.async.wait_all;" ::: "memory");
        if (!wrote)
            for (int f = 0; f < NF; ++f) s_sh[t * RS + f] = 0.f;
        __syncthreads();
        const size_t g0 = (size_t)blockIdx.x * blockDim.x;
        const int cnt = (int)min((size_t)blockDim.x, (size_t)fp.n - g0);
        if (order == nullptr) {
            // the block's rows are one contiguous span of the output
            for (int i = t; i < cnt * NF; i += blockDim.x) d_sh[g0 * NF + i] = s_sh[(i / NF) * RS + i % NF];
        } else {
            // rows at the caller's indices: one warp per row
            const int lane = t & 31;
            for (int r = t >> 5; r < cnt; r += (int)(blockDim.x >> 5)) {
                float* dst = d_sh + (size_t)__ldg(order + g0 + r) * NF;
                for (int f = lane; f < NF; f += 32) dst[f] = s_sh[r * RS + f];
            }
        }
    }
}

template <int TW, int TH, int PW, int PH, int GW, int GH, bool CR>
static void launch_bwd_one(const RasterBwdArgs& a, cudaStream_t s) {
    constexpr int NT = (TW / PW) * (TH / PH);
    raster_bwd_kernel<TW, TH, PW, PH, GW, GH, CR><<<a.n_tiles + (a.ckpt ? a.n_map : 0u), NT, 0, s>>>(
        a.starts, a.ends, a.inst_rec, a.rec, a.cams, a.n_cams, a.fp, a.dL_drgb, a.T_final, a.n_contrib,
        a.grad_rec, a.tile_order, a.ckpt, a.cfin, a.chunk_map, a.n_tiles);
}

template <int TW, int TH>
static bool launch_bwd_shape(const RasterBwdArgs& a, cudaStream_t s) {
    if (!a.cr) launch_bwd_one<TW, TH, 2, 2, 1, 1, false>(a, s);
    else if (a.group_w == 2 && a.group_h == 2) launch_bwd_one<TW, TH, 2, 2, 2, 2, true>(a, s);
    else if (a.group_w == 1 && a.group_h == 1) launch_bwd_one<TW, TH, 2, 2, 1, 1, true>(a, s);
    else if (a.group_w == 2 && a.group_h == 4) launch_bwd_one<TW, TH, 2, 4, 2, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 4) launch_bwd_one<TW, TH, 2, 2, 4, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 8) launch_bwd_one<TW, TH, 2, 4, 4, 8, true>(a, s);
    else return false;
    return true;
}

// 8x8 tiles: one warp per tile, two pixels (a row pair) per lane, so each
// list entry is tested once per tile rather than once per half tile.
static bool launch_bwd_shape_8x8(const RasterBwdArgs& a, cudaStream_t s) {
    if (!a.cr) launch_bwd_one<8, 8, 2, 1, 1, 1, false>(a, s);
    else if (a.group_w == 2 && a.group_h == 2) launch_bwd_one<8, 8, 2, 1, 2, 2, true>(a, s);
    else if (a.group_w == 1 && a.group_h == 1) launch_bwd_one<8, 8, 2, 1, 1, 1, true>(a, s);
    else if (a.group_w == 2 && a.group_h == 4) launch_bwd_one<8, 8, 2, 1, 2, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 4) launch_bwd_one<8, 8, 2, 1, 4, 4, true>(a, s);
    else if (a.group_w == 4 && a.group_h == 8) launch_bwd_one<8, 8, 2, 1, 4, 8, true>(a, s);
    else return false;
    return true;
}

bool launch_raster_bwd(const RasterBwdArgs& a, cudaStream_t s) {
    if (a.n_tiles == 0) return true;
    if (a.fp.tile_w == 8 && a.fp.tile_h == 8) return launch_bwd_shape_8x8(a, s);
    if (a.fp.tile_w == 16 && a.fp.tile_h == 16) return launch_bwd_shape<16, 16>(a, s);
    if (a.fp.tile_w == 32 && a.fp.tile_h == 8) return launch_bwd_shape<32, 8>(a, s);
    if (a.fp.tile_w == 32 && a.fp.tile_h == 16) return launch_bwd_shape<32, 16>(a, s);
    return false;
}

// Chunk map of the backward pass: slot (start_t >> kCkptShift) + c -> t for
// the chunks c >= 1 of every list longer than kCkptL (slots of different
// lists never collide; unused slots stay all-ones).
__global__ void chunk_map_kernel(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ ends,
                                 uint32_t n_tiles, uint32_t* __restrict__ map, uint32_t n_map) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
        const uint32_t s = __ldg(starts + t), e = __ldg(ends + t);
        if (s >= e) continue;
        const uint32_t n = (e - s + kCkptL - 1u) >> kCkptShift;
        for (uint32_t c = 1; c < n; ++c) {
            const uint32_t i = (s >> kCkptShift) + c;
            if (i < n_map) map[i] = t;
        }
    }
}

void launch_chunk_map(const uint32_t* starts, const uint32_t* ends, uint32_t n_tiles, uint32_t* map, uint32_t n_map,
                      cudaStream_t s) {
    if (n_tiles == 0) return;
    chunk_map_kernel<<<std::min<uint32_t>((n_tiles + 255) / 256, 152u * 4u), 256, 0, s>>>(starts, ends, n_tiles, map,
                                                                                         n_map);
}

void launch_preprocess_bwd(const SceneDev& sc, const CamDev* cams, const FrameParams& fp, const uint32_t* tiles,
                           const float* grad_rec, float* d_means, float* d_ls, float* d_quat, float* d_logit,
                           float* d_sh, const uint32_t* order, cudaStream_t s) {
    const int blocks = (fp.n + 127) / 128;
    if (fp.n_cams == 1) {
        switch (fp.sh_degree) {
            case 0: preprocess_bwd_kernel<0, true><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
            case 1: preprocess_bwd_kernel<1, true><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
            case 2: preprocess_bwd_kernel<2, true><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
            default: preprocess_bwd_kernel<3, true><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
        }
        return;
    }
    switch (fp.sh_degree) {
        case 0: preprocess_bwd_kernel<0, false><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
        case 1: preprocess_bwd_kernel<1, false><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
        case 2: preprocess_bwd_kernel<2, false><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
        default: preprocess_bwd_kernel<3, false><<<blocks, 128, 0, s>>>(sc, cams, fp, tiles, grad_rec, d_means, d_ls, d_quat, d_logit, d_sh, order); break;
    }
}

}  // namespace seele
