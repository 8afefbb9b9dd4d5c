// preprocess.cu -- per-(camera, Gaussian) preprocessing (Sec. 3.1
// "Preprocessing", Sec. 3.3 view-cluster filter and online filtering,
// Eqns. 3-5) and the scene repack into the structure-of-arrays layout.
//
// One thread per (camera, Gaussian); every load is a 16-byte vector load of
// a structure-of-arrays plane, so a warp reads 512 contiguous bytes per
// plane.  The kernel is HBM-bound: 64 B of geometry + 16..192 B of SH per
// selected Gaussian in, 64 B of record/rect/count/depth out.
#include "common.cuh"
#include "tiletest.cuh"
#include "kernels.h"

namespace seele {

// Real spherical harmonics with the Condon-Shortley phase, k = l*l + l + m,
// written as polynomials of the unit direction (x, y, z).  Constants are the
// closed-form normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
// Legendre/trigonometric factors:
//   l=0: 1/(2 sqrt(pi))
//   l=1: sqrt(3/(4 pi))                     (-y, z, -x)
//   l=2: sqrt(15/(4 pi)) (xy, -yz, -xz), sqrt(5/(16 pi)) (2zz-xx-yy), sqrt(15/(16 pi)) (xx-yy)
//   l=3: sqrt(35/(32 pi)) (-y(3xx-yy), -x(xx-3yy)), sqrt(105/(4 pi)) xyz,
//        sqrt(21/(32 pi)) (-y(4zz-xx-yy), -x(4zz-xx-yy)), sqrt(7/(16 pi)) z(2zz-3xx-3yy),
//        sqrt(105/(16 pi)) z(xx-yy)
struct ShConst {
    static constexpr float c0 = 0.28209479177387814f;
    static constexpr float c1 = 0.48860251190291992f;
    static constexpr float c2a = 1.0925484305920792f;
    static constexpr float c2b = 0.31539156525252005f;
    static constexpr float c2c = 0.54627421529603959f;
    static constexpr float c3a = 0.59004358992664352f;
    static constexpr float c3b = 2.8906114426405538f;
    static constexpr float c3c = 0.45704579946446572f;
    static constexpr float c3d = 0.37317633259011540f;
    static constexpr float c3e = 1.4453057213202769f;
};

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = ShConst::c0;
    if (DEG > 0) {
        Y[1] = -ShConst::c1 * y;
        Y[2] = ShConst::c1 * z;
        Y[3] = -ShConst::c1 * x;
    }
    if (DEG > 1) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = ShConst::c2a * x * y;
        Y[5] = -ShConst::c2a * y * z;
        Y[6] = ShConst::c2b * (2.f * zz - xx - yy);
        Y[7] = -ShConst::c2a * x * z;
        Y[8] = ShConst::c2c * (xx - yy);
        if (DEG > 2) {
            Y[9] = -ShConst::c3a * y * (3.f * xx - yy);
            Y[10] = ShConst::c3b * x * y * z;
            Y[11] = -ShConst::c3c * y * (4.f * zz - xx - yy);
            Y[12] = ShConst::c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -ShConst::c3c * x * (4.f * zz - xx - yy);
            Y[14] = ShConst::c3e * z * (xx - yy);
            Y[15] = -ShConst::c3a * x * (xx - 3.f * yy);
        }
    }
}

template <int DEG, bool AOS>
__device__ __forceinline__ void load_sh(const SceneDev& sc, int n, int g, float* f) {
    constexpr int NC = (DEG + 1) * (DEG + 1);
    constexpr int NP = (3 * NC + 3) / 4;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float4 v = scene_sh4<AOS, NC>(sc, n, g, j);
        f[4 * j + 0] = v.x;
        f[4 * j + 1] = v.y;
        f[4 * j + 2] = v.z;
        f[4 * j + 3] = v.w;
    }
}

// a*c - b*b with one rounding error (Kahan's fma formulation of a 2x2
// determinant); keeps the conic accurate for elongated footprints.
__device__ __forceinline__ float det2_sym(float a, float b, float c) {
    float w = b * b;
    float e = fmaf(-b, b, w);
    float f = fmaf(a, c, -w);
    return f + e;
}

template <int DEG, bool AOS>
__global__ void __launch_bounds__(256) preprocess_kernel(SceneDev sc, const CamDev* __restrict__ cams,
                                                         FrameParams fp, ProjOut out) {
    // cameras vary fastest over the grid, so the blocks that read one slice
    // of the scene run together and share it through L2
    const int g = blockIdx.y * blockDim.x + threadIdx.x;
    const int ci = blockIdx.x;
    if (g == 0 && ci == 0 && out.t_frame) *out.t_frame = global_ns();
    if (g >= fp.n) return;
    const size_t rid = (size_t)ci * fp.n + g;
    const CamDev& C = cams[ci];
    uint32_t ntiles = 0, nblocks = 0;
    do {
        // view-cluster filter: selected clusters plus shared Gaussians (Sec. 3.3);
        // a streamed scene's slot is read only when it holds a selected cluster
        // and is ready, and a Gaussian held by several selected clusters' slots
        // is kept in the slot of the lowest one (veto: the lower clusters)
        if (fp.use_mask) {
            if (fp.slot_cap != 0u && (uint32_t)g >= fp.n_shared) {
                const uint32_t slot = ((uint32_t)g - fp.n_shared) / fp.slot_cap;
                if (!((C.slot_ok[slot >> 5] >> (slot & 31u)) & 1u)) break;
            }
            if ((__ldg(sc.mask + g) & C.sel_bits) == 0u) break;
            if (sc.veto != nullptr && (__ldg(sc.veto + g) & C.sel_bits) != 0u) break;
        }
        const float4 pl = scene_pos_logit<AOS>(sc, g);
        const float X = fmaf(C.R[0], pl.x, fmaf(C.R[1], pl.y, fmaf(C.R[2], pl.z, C.t[0])));
        const float Y = fmaf(C.R[3], pl.x, fmaf(C.R[4], pl.y, fmaf(C.R[5], pl.z, C.t[1])));
        const float Z = fmaf(C.R[6], pl.x, fmaf(C.R[7], pl.y, fmaf(C.R[8], pl.z, C.t[2])));
        if (!(Z > C.near_z)) break;
        const float iz = __frcp_rn(Z);
        const float xz = X * iz, yz = Y * iz;
        if (fabsf(xz) > C.lim_x || fabsf(yz) > C.lim_y) break;

        // opacity and the support threshold t_g (Eqn. 3, or Eqn. 5 when filtering)
        // (hardware exp/log/reciprocal: a few ulp, inside the FP32 margins)
        const float o = __frcp_rn(1.f + __expf(-pl.w));
        float tg = 9.f;
        if (fp.opacity_filter) {
            if (!(o > fp.alpha_min)) break;
            tg = fminf(2.f * (__logf(o) - fp.log_alpha_min), 9.f);
        }

        // Sigma' = J W R S (J W R S)^T + dilation: build N = J W R S (2x3)
        const float4 q4 = scene_quat<AOS>(sc, g);
        const float qinv = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
        const float qw = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
        const float4 ls = scene_log_scale<AOS>(sc, g);
        const float s0 = __expf(ls.x), s1 = __expf(ls.y), s2 = __expf(ls.z);
        float M[9];  // R(q) diag(s)
        M[0] = (1.f - 2.f * (qy * qy + qz * qz)) * s0;
        M[1] = 2.f * (qx * qy - qw * qz) * s1;
        M[2] = 2.f * (qx * qz + qw * qy) * s2;
        M[3] = 2.f * (qx * qy + qw * qz) * s0;
        M[4] = (1.f - 2.f * (qx * qx + qz * qz)) * s1;
        M[5] = 2.f * (qy * qz - qw * qx) * s2;
        M[6] = 2.f * (qx * qz - qw * qy) * s0;
        M[7] = 2.f * (qy * qz + qw * qx) * s1;
        M[8] = (1.f - 2.f * (qx * qx + qy * qy)) * s2;
        float WM[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                WM[3 * i + j] = fmaf(C.R[3 * i + 0], M[j], fmaf(C.R[3 * i + 1], M[3 + j], C.R[3 * i + 2] * M[6 + j]));
        const float jx = C.fx * iz, jy = C.fy * iz;
        float N0[3], N1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            N0[j] = jx * fmaf(-xz, WM[6 + j], WM[j]);
            N1[j] = jy * fmaf(-yz, WM[6 + j], WM[3 + j]);
        }
        const float a = fmaf(N0[0], N0[0], fmaf(N0[1], N0[1], N0[2] * N0[2])) + fp.dilation;
        const float b = fmaf(N0[0], N1[0], fmaf(N0[1], N1[1], N0[2] * N1[2]));
        const float c = fmaf(N1[0], N1[0], fmaf(N1[1], N1[1], N1[2] * N1[2])) + fp.dilation;
        const float det = det2_sym(a, b, c);
        if (!(det > 0.f)) break;
        const float inv = __frcp_rn(det);

        const float u = fmaf(C.fx, xz, C.cx);
        const float v = fmaf(C.fy, yz, C.cy);

        // rect: the support ellipse q <= t_g lies within sqrt(t_g lambda_max)
        const float hd = 0.5f * (a - c);
        const float lmax = 0.5f * (a + c) + sqrtf(fmaxf(fmaf(hd, hd, b * b), 0.f));
        const float r = ceilf(sqrtf(tg * lmax));
        float fx0 = floorf(u - 0.5f - r), fx1 = ceilf(u - 0.5f + r);
        float fy0 = floorf(v - 0.5f - r), fy1 = ceilf(v - 0.5f + r);
        fx0 = fmaxf(fx0, 0.f);
        fy0 = fmaxf(fy0, 0.f);
        fx1 = fminf(fx1, (float)(C.W - 1));
        fy1 = fminf(fy1, (float)(C.H - 1));
        if (fx0 > fx1 || fy0 > fy1) break;
        const int sw = __ffs(fp.tile_w) - 1, sh = __ffs(fp.tile_h) - 1;  // tile sizes are powers of two
        const int tx0 = (int)fx0 >> sw, tx1 = (int)fx1 >> sw;
        const int ty0 = (int)fy0 >> sh, ty1 = (int)fy1 >> sh;

        // raster record: exponent e = log2(o) - q log2(e) / 2 and one threshold
        // for "inside the support and alpha >= alpha_theta" (both are e >= bound);
        // the last slot holds the tile test's bound on -(cA dx^2 + cB dx dy + cC dy^2)
        const float lo = __log2f(o);
        const float thr = fmaxf(fmaf(-0.5f * kLog2e, tg, lo), fp.log2_alpha_min);
        const float4 rec0 = make_float4(u, v, -0.5f * kLog2e * c * inv, kLog2e * b * inv);
        const float4 rec1 = make_float4(-0.5f * kLog2e * a * inv, lo, thr,
                                        __fmul_rn(tg, 0.5f * kLog2e * (1.f + kTileInflate)));
        // tiles touched, and for block binning the tile-block instances: per
        // block row, the blocks spanned by the union of its tile rows' spans
        if (fp.tile_test) {
            const Ellipse E = make_ellipse(rec0, rec1);
            int cur = ty0 / kBlockH, blo = 1 << 30, bhi = -1;
            for (int ty = ty0; ty <= ty1; ++ty) {
                if (ty / kBlockH != cur) {
                    if (bhi >= blo) nblocks += (uint32_t)(bhi / kBlockW - blo / kBlockW + 1);
                    cur = ty / kBlockH;
                    blo = 1 << 30;
                    bhi = -1;
                }
                int l, h;
                if (row_span(E, ty, fp.tile_w, fp.tile_h, tx0, tx1, &l, &h)) {
                    ntiles += (uint32_t)(h - l + 1);
                    blo = min(blo, l);
                    bhi = max(bhi, h);
                }
            }
            if (bhi >= blo) nblocks += (uint32_t)(bhi / kBlockW - blo / kBlockW + 1);
            if (ntiles == 0) break;
        } else {
            ntiles = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
            nblocks = (uint32_t)((tx1 / kBlockW - tx0 / kBlockW + 1) * (ty1 / kBlockH - ty0 / kBlockH + 1));
        }

        // colour: SH in the direction from the camera centre to the mean
        float dxw = pl.x - C.campos[0], dyw = pl.y - C.campos[1], dzw = pl.z - C.campos[2];
        const float dn = rsqrtf(dxw * dxw + dyw * dyw + dzw * dzw);
        dxw *= dn;
        dyw *= dn;
        dzw *= dn;
        constexpr int NC = (DEG + 1) * (DEG + 1);
        float Yb[NC];
        sh_basis<DEG>(dxw, dyw, dzw, Yb);
        float shf[((3 * NC + 3) / 4) * 4];
        load_sh<DEG, AOS>(sc, fp.n, g, shf);
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < NC; ++k) s = fmaf(shf[3 * k + ch], Yb[k], s);
            rgb[ch] = fmaxf(s, 0.f);
        }

        float4* ro = out.rec + (size_t)kRecF4 * rid;
        ro[0] = rec0;
        ro[1] = rec1;
        // the last slot flags the Gaussians whose alpha can reach the clamp
        // (o within 1e-4 in log2 of alpha_max): only their blends need the
        // min(), for every other one 2^e < alpha_max wherever e <= log2 o
        ro[2] = make_float4(rgb[0], rgb[1], rgb[2], lo > __log2f(fp.alpha_max) - 1e-4f ? 1.f : 0.f);
        ro[3] = make_float4(__uint_as_float((uint32_t)tx0 | ((uint32_t)ty0 << 16)),
                            __uint_as_float((uint32_t)tx1 | ((uint32_t)ty1 << 16)), 0.f, 0.f);
        out.depth[rid] = Z;
    } while (0);
    out.tiles[rid] = ntiles;
    if (fp.binning) out.blocks[rid] = nblocks;  // > 0 exactly when ntiles > 0
    // visible records per 4096-record chunk (for the compaction); the valid
    // lanes of a warp are a prefix and hold consecutive records, so they span
    // at most two chunks
    const int lane = threadIdx.x & 31;
    const int valid = min(32, fp.n - (g - lane));
    const uint32_t am = valid >= 32 ? 0xffffffffu : ((1u << valid) - 1u);
    const uint32_t chunk = (uint32_t)(rid / kChunkItems);
    const uint32_t c0 = __shfl_sync(am, chunk, 0);
    const uint32_t vis = __ballot_sync(am, ntiles > 0u);
    const uint32_t hi = __ballot_sync(am, ntiles > 0u && chunk != c0);
    if (lane == 0) {
        if (vis & ~hi) atomicAdd(out.chunk_vis + c0, (uint32_t)__popc(vis & ~hi));
        if (hi) atomicAdd(out.chunk_vis + c0 + 1, (uint32_t)__popc(hi));
    }
}

// Scene repack: caller layout (arrays of structures) -> library planes.  A
// block takes kRepackG consecutive Gaussians: it reads their contiguous
// spans of every input array with consecutive threads on consecutive words
// (also when the inputs are page-locked host memory read over the
// host link), parks them in shared memory (SH rows padded to an odd
// stride, so a warp reading one column hits 32 banks), then writes the
// float4 planes, one Gaussian per thread.
constexpr int kRepackG = 128;

template <int NC>
__global__ void __launch_bounds__(256) repack_kernel(int n, const float* __restrict__ means,
                                                     const float* __restrict__ log_scales,
                                                     const float* __restrict__ quats,
                                                     const float* __restrict__ logits,
                                                     const float* __restrict__ sh, float4* __restrict__ pos_logit,
                                                     float4* __restrict__ quat, float4* __restrict__ log_scale,
                                                     float4* __restrict__ shp) {
    constexpr int NF = 3 * NC, NP = (NF + 3) / 4, RS = NF | 1;
    __shared__ float4 s_q[kRepackG];
    __shared__ float s_sh[kRepackG * RS], s_m[3 * kRepackG], s_s[3 * kRepackG], s_o[kRepackG];
    const size_t g0 = (size_t)blockIdx.x * kRepackG;
    const int cnt = (int)min((size_t)kRepackG, (size_t)n - g0);
    const int t = threadIdx.x;
    for (int i = t; i < cnt * NF; i += 256) s_sh[(i / NF) * RS + i % NF] = __ldg(sh + g0 * NF + i);
    for (int i = t; i < cnt * 3; i += 256) {
        s_m[i] = __ldg(means + g0 * 3 + i);
        s_s[i] = __ldg(log_scales + g0 * 3 + i);
    }
    float* q = reinterpret_cast<float*>(s_q);
    for (int i = t; i < cnt * 4; i += 256) q[i] = __ldg(quats + g0 * 4 + i);
    for (int i = t; i < cnt; i += 256) s_o[i] = __ldg(logits + g0 + i);
    __syncthreads();
    if (t < cnt) {
        pos_logit[g0 + t] = make_float4(s_m[3 * t], s_m[3 * t + 1], s_m[3 * t + 2], s_o[t]);
        quat[g0 + t] = s_q[t];
        log_scale[g0 + t] = make_float4(s_s[3 * t], s_s[3 * t + 1], s_s[3 * t + 2], 0.f);
    }
    for (int k = t; k < NP * kRepackG; k += 256) {
        const int j = k / kRepackG, gl = k % kRepackG;
        if (gl >= cnt) continue;
        const float* row = s_sh + gl * RS + 4 * j;
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (4 * j + i < NF) ? row[i] : 0.f;
        shp[(size_t)j * n + g0 + gl] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

void launch_preprocess(const SceneDev& sc, const CamDev* cams, const FrameParams& fp, const ProjOut& out,
                       cudaStream_t s) {
    dim3 grid(fp.n_cams, (fp.n + 255) / 256);
    const bool aos = sc.means != nullptr;
    switch (fp.sh_degree) {
        case 0:
            if (aos) preprocess_kernel<0, true><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            else preprocess_kernel<0, false><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            break;
        case 1:
            if (aos) preprocess_kernel<1, true><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            else preprocess_kernel<1, false><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            break;
        case 2:
            if (aos) preprocess_kernel<2, true><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            else preprocess_kernel<2, false><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            break;
        default:
            if (aos) preprocess_kernel<3, true><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            else preprocess_kernel<3, false><<<grid, 256, 0, s>>>(sc, cams, fp, out);
            break;
    }
}

void launch_repack(int n, int nc, const float* means, const float* log_scales, const float* quats,
                   const float* logits, const float* sh, float4* pos_logit, float4* quat, float4* log_scale,
                   float4* shp, cudaStream_t s) {
    const int blocks = (n + kRepackG - 1) / kRepackG;
    switch (nc) {
        case 1: repack_kernel<1><<<blocks, 256, 0, s>>>(n, means, log_scales, quats, logits, sh, pos_logit, quat,
                                                        log_scale, shp); break;
        case 4: repack_kernel<4><<<blocks, 256, 0, s>>>(n, means, log_scales, quats, logits, sh, pos_logit, quat,
                                                        log_scale, shp); break;
        case 9: repack_kernel<9><<<blocks, 256, 0, s>>>(n, means, log_scales, quats, logits, sh, pos_logit, quat,
                                                        log_scale, shp); break;
        default: repack_kernel<16><<<blocks, 256, 0, s>>>(n, means, log_scales, quats, logits, sh, pos_logit,
                                                          quat, log_scale, shp); break;
    }
}

}  // namespace seele
