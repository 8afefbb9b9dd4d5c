// tiletest.cuh -- which tiles of a Gaussian's rect its support ellipse reaches.
//
// Sec. 3.3's online filtering bounds each Gaussian by the rect of its support
// radius; this test tightens the rect to the ellipse itself.  Per tile row, the
// ellipse Q(dx, dy) <= T cut by the row's band of pixel-centre y values is
// convex, so its x-extent is one interval: the largest x over the band lies at
// the ellipse's rightmost point (dy = -b x_r / c) clamped to the band, the
// smallest at the leftmost point (dy = +b x_r / c) clamped.  A tile is kept
// when its pixel-centre x-range, widened by kTileSlack px, meets that
// interval; the band is widened by the same slack.  T carries a 0.1% inflation
// of the support.  The two slacks keep the test conservative under FP32
// rounding, so no pixel that the rasterizer would blend is dropped.
//
// The record stores the scaled conic of the exponent (cA, cB, cC with
// e = log2(o) + cA dx^2 + cB dx dy + cC dy^2), so Q = -(cA dx^2 + cB dx dy +
// cC dy^2) = a dx^2 + 2 b dx dy + c dy^2 with a = -cA, b = -cB / 2, c = -cC.
// Counting (preprocessing) and enumeration (emission) both call row_span on
// the same stored floats, and every operation below is an explicitly rounded
// intrinsic, so the two see identical spans.
#pragma once
#include <cstdint>

namespace seele {

constexpr float kTileInflate = 1e-3f;
constexpr float kTileSlack = 1.f / 256.f;

// Hardware approximations (about one ulp); the slack above covers their error,
// and both kernels issue the same instructions on the same inputs.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Ellipse {
    float u, v;        // centre (px)
    float a, b, c;     // Q = a dx^2 + 2 b dx dy + c dy^2
    float det;         // a c - b^2
    float inv_a;       // 1 / a
    float xr, yr;      // half extents of Q <= T along x and y
    float k;           // the rightmost point is at dy = -k, the leftmost at +k
};

__device__ __forceinline__ Ellipse make_ellipse(float4 r0, float4 r1) {
    Ellipse E;
    E.u = r0.x;
    E.v = r0.y;
    E.a = -r0.z;
    E.b = __fmul_rn(-0.5f, r0.w);
    E.c = -r1.x;
    const float T = r1.w;
    // Kahan's a c - b^2 with one rounding error
    const float w = __fmul_rn(E.b, E.b);
    const float e = __fmaf_rn(-E.b, E.b, w);
    const float f = __fmaf_rn(E.a, E.c, -w);
    E.det = __fadd_rn(f, e);
    E.inv_a = rcp_approx(E.a);
    const float inv_det = rcp_approx(E.det);
    E.xr = sqrt_approx(__fmul_rn(__fmul_rn(T, E.c), inv_det));
    E.yr = sqrt_approx(__fmul_rn(__fmul_rn(T, E.a), inv_det));
    E.k = __fmul_rn(__fmul_rn(E.b, E.xr), rcp_approx(E.c));
    return E;
}

// x offset from the centre of the ellipse's boundary at height dy (|dy| <= yr);
// side = +1 right, -1 left.  The root uses det (yr - dy)(yr + dy) = a T - det dy^2
// without the cancellation of the expanded form.
__device__ __forceinline__ float boundary_x(const Ellipse& E, float dy, float side) {
    const float s = __fmul_rn(E.det, __fmul_rn(__fsub_rn(E.yr, dy), __fadd_rn(E.yr, dy)));
    const float root = sqrt_approx(fmaxf(s, 0.f));
    return __fmul_rn(__fmaf_rn(side, root, __fmul_rn(-E.b, dy)), E.inv_a);
}

// Tiles [*lo, *hi] of tile row ty within the rect columns [rx0, rx1]; false
// when the row holds none.  A conic whose FP32 determinant is not positive (a
// needle so thin that rounding swamps a c - b^2) keeps the whole rect row.
// Tile sizes are powers of two, so multiplying by 1 / TW is exact.
__device__ __forceinline__ bool row_span(const Ellipse& E, int ty, int TW, int TH, int rx0, int rx1, int* lo,
                                         int* hi) {
    if (!(E.det > 0.f && E.a > 0.f && E.c > 0.f)) {
        *lo = rx0;
        *hi = rx1;
        return true;
    }
    const float y0 = (float)(ty * TH), x_w = (float)TW, inv_w = 1.f / (float)TW;
    const float ya = __fsub_rn(__fadd_rn(y0, 0.5f - kTileSlack), E.v);
    const float yb = __fsub_rn(__fadd_rn(y0, (float)TH - 0.5f + kTileSlack), E.v);
    const float blo = fmaxf(ya, -E.yr), bhi = fminf(yb, E.yr);
    if (blo > bhi) return false;
    const float dr = fminf(fmaxf(-E.k, blo), bhi), dl = fminf(fmaxf(E.k, blo), bhi);
    const float xR = __fadd_rn(E.u, boundary_x(E, dr, 1.f));
    const float xL = __fadd_rn(E.u, boundary_x(E, dl, -1.f));
    const float fr = __fmul_rn(__fadd_rn(xR, kTileSlack - 0.5f), inv_w);
    const float fl = __fmul_rn(__fsub_rn(xL, x_w - 0.5f + kTileSlack), inv_w);
    const int a = max(rx0, (int)ceilf(fmaxf(fl, -1.f)));
    const int b = min(rx1, (int)floorf(fminf(fr, 65536.f)));
    *lo = a;
    *hi = b;
    return b >= a;
}

}  // namespace seele
