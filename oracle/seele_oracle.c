/*
 * seele_oracle.c -- plain FP64 CPU oracle for the Seele hot path
 * (arxiv 2503.05168, "Seele: A Unified Acceleration Framework for Real-Time
 * Gaussian Splatting on Mobile Devices").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Everything is computed in double precision, one Gaussian / one pixel at a
 * time, in the order the paper states the method.  Where the paper is silent
 * the 3DGS conventions it builds on are used (Sec. 3.1 cites 3DGS and EWA):
 *
 *   camera    x right, y down, z forward; X_cam = R * x_world + t;
 *             u = fx * X / Z + cx,  v = fy * Y / Z + cy (continuous pixel
 *             coordinates); pixel (px, py) is sampled at (px + .5, py + .5).
 *   culling   Z <= near, or |X/Z| > 1.3 * W / (2 fx), or |Y/Z| > 1.3 * H / (2 fy)
 *             ("filters out Gaussians outside the current view frustum", Sec. 3.1).
 *   Sigma     R(q) diag(exp(log_scale))^2 R(q)^T, q = (w, x, y, z) normalised.
 *   EWA       Sigma' = J W Sigma W^T J^T + 0.3 I (Sec. 3.1, Eqn. 2 with the EWA
 *             projection of Zwicker et al.; 0.3 is the 3DGS low-pass term).
 *   colour    rgb = max(0, sum_lm k_lm Y_lm(d) + 0.5), d = unit(mean - campos),
 *             real spherical harmonics with the Condon-Shortley phase,
 *             coefficient index k = l*l + l + m (Sec. 3.1: the colour of a
 *             Gaussian comes from its SH coefficients).
 *   alpha     alpha = min(0.99, o * exp(-q / 2)), q = d^T Sigma'^-1 d (Eqn. 2),
 *             o = sigmoid(logit).
 *   support   a pixel only receives a Gaussian when q <= t_g, with t_g = 9 (the
 *             3-sigma envelope of Eqn. 3) or, with the opacity-aware online
 *             filter, t_g = min(2 ln(o / alpha_theta), 9) (Eqns. 4-5); in that
 *             mode o <= alpha_theta culls the Gaussian.
 *   rect      r = ceil(sqrt(t_g * lambda_max(Sigma'))); pixel box
 *             [floor(u - .5 - r), ceil(u - .5 + r)] clipped to the image, mapped
 *             to tiles by integer division (Sec. 3.3 "Online Filtering").
 *   tiles     with the ellipse tile test, a tile of the rect is kept only if
 *             the ellipse q <= t_g (1 + 1e-3) meets the rectangle spanned by
 *             the tile's pixel centres widened by 1/256 px on every side; the
 *             relative and absolute slack keep the test conservative under
 *             FP32 rounding.  Every pixel with q <= t_g lies in a kept tile, so
 *             the image does not depend on the test.
 *   blending  front to back in (fp32 depth, index) order (Sec. 3.1 "Sorting");
 *             skip alpha < alpha_theta; T' = T (1 - alpha); if T' < Gamma_theta
 *             the pixel stops without blending; otherwise C += T alpha c,
 *             T = T' (Eqn. 1 and the two rules after Eqn. 2).
 *   CR        Algorithm 1: every w x h pixel group has its top-left pixel as
 *             leader (Sec. 4.1 takes the group's first pixel); the leader's
 *             alpha decides for the whole group, pixels of a passing group
 *             apply the per-pixel rules above (Sec. 3.4: a passing group is
 *             rasterized as in the plain method).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Plain data types, mirrored by numpy dtypes in oracle/__init__.py           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double R[9];        /* world -> camera rotation, row-major */
    double t[3];        /* world -> camera translation */
    double fx, fy, cx, cy;
    int32_t width, height;
    double near_z;
} oc_camera;

typedef struct {
    int32_t tile_w, tile_h;
    int32_t opacity_filter;   /* 1: support t_g of Eqn. 5 instead of 9 (Eqn. 3) */
    int32_t cr;               /* 1: contribution-aware rasterization (Alg. 1) */
    int32_t group_w, group_h; /* pixel group P of Alg. 1 */
    int32_t use_mask;         /* 1: view-cluster filter of Sec. 3.3 */
    uint32_t sel_bits;        /* clusters selected for this camera */
    int32_t tile_test;        /* 0: every tile of the rect; 1: tiles the support ellipse reaches */
    double alpha_min;         /* alpha_theta = 1/255 (Sec. 3.1) */
    double alpha_max;         /* 0.99 clamp */
    double t_stop;            /* Gamma_theta */
    double dilation;          /* 0.3 */
    double frustum_slack;     /* 1.3 */
} oc_options;

typedef struct {
    int32_t visible;     /* passes every cull and touches at least one tile */
    int32_t radius;      /* r of the rect rule, pixels */
    int32_t rect[4];     /* tile x0, y0, x1, y1, inclusive */
    int32_t ntiles;
    float depth32;       /* Z rounded to fp32: the sort key */
    double mean_cam[3];  /* X, Y, Z */
    double uv[2];
    double cov2[3];      /* Sigma' = [[a, b], [b, c]], dilation included */
    double conic[3];     /* Sigma'^-1 = [[A, B], [B, C]] */
    double opacity;
    double rgb_raw[3];   /* before the max(0, .) clamp */
    double rgb[3];
    double tg;           /* support threshold on q */
    double margin_px;    /* distance of the rect decisions to a rounding flip, px */
    double margin_rel;   /* relative distance of the cull decisions to their threshold */
} oc_proj;

/* counters: 0 visible, 1 instances, 2 alpha evaluations, 3 blended pairs,
 *           4 leader tests, 5 leader skips, 6 pixels terminated early,
 *           7 blended pairs whose alpha sat at the 0.99 clamp */
#define OC_NCOUNT 8

/* ------------------------------------------------------------------------ */
/* Small linear algebra                                                      */
/* ------------------------------------------------------------------------ */

static void mat3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat3_transpose(const double* A, double* B) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * j + i] = A[3 * i + j];
}

/* Rotation matrix of the unit quaternion (w, x, y, z): R v = q v q*. */
static void quat_to_rot(const double* qn, double* R) {
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Camera centre in world coordinates: c = -R^T t. */
static void camera_centre(const oc_camera* cam, double* c) {
    for (int i = 0; i < 3; ++i)
        c[i] = -(cam->R[0 * 3 + i] * cam->t[0] + cam->R[1 * 3 + i] * cam->t[1] + cam->R[2 * 3 + i] * cam->t[2]);
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics from their closed form                           */
/* ------------------------------------------------------------------------ */
/*
 * Y_lm for m > 0: sqrt(2) K_lm P_l^m(z) Re((x + i y)^m) / sin^m
 *            m < 0: sqrt(2) K_l|m| P_l^|m|(z) Im((x + i y)^|m|) / sin^|m|
 *            m = 0: K_l0 P_l(z)
 * with K_lm = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!) and P_l^m the
 * associated Legendre function including the Condon-Shortley phase (-1)^m.
 * Writing P_l^m(z) = sin^m(theta) Q_l^m(z), Q follows from the textbook
 * recurrence in l, and (x + i y)^m = sin^m e^{i m phi}, so each basis function
 * is a polynomial in (x, y, z).  The recurrence is carried in forward-mode
 * (value and gradient) so the backward pass gets dY/dd from the same
 * definition.  Valid on the unit sphere (r = 1 is used in the recurrence).
 */
typedef struct { double v, dx, dy, dz; } dual3;

static dual3 d3(double v, double dx, double dy, double dz) { dual3 r = {v, dx, dy, dz}; return r; }
static dual3 d3_add(dual3 a, dual3 b) { return d3(a.v + b.v, a.dx + b.dx, a.dy + b.dy, a.dz + b.dz); }
static dual3 d3_scale(dual3 a, double s) { return d3(a.v * s, a.dx * s, a.dy * s, a.dz * s); }
static dual3 d3_mul(dual3 a, dual3 b) {
    return d3(a.v * b.v, a.dx * b.v + a.v * b.dx, a.dy * b.v + a.v * b.dy, a.dz * b.v + a.v * b.dz);
}

static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* Y[k] and its gradient for k = l*l + l + m, l <= lmax (<= 3). */
static void sh_basis(int lmax, const double* d, dual3* Y) {
    dual3 X = d3(d[0], 1, 0, 0), Yv = d3(d[1], 0, 1, 0), Z = d3(d[2], 0, 0, 1);
    /* C_m + i S_m = (x + i y)^m */
    dual3 Cm[4], Sm[4];
    Cm[0] = d3(1, 0, 0, 0); Sm[0] = d3(0, 0, 0, 0);
    for (int m = 1; m <= lmax; ++m) {
        Cm[m] = d3_add(d3_mul(X, Cm[m - 1]), d3_scale(d3_mul(Yv, Sm[m - 1]), -1.0));
        Sm[m] = d3_add(d3_mul(X, Sm[m - 1]), d3_mul(Yv, Cm[m - 1]));
    }
    for (int m = 0; m <= lmax; ++m) {
        /* Q_m^m = (-1)^m (2m - 1)!!;  Q_{m+1}^m = (2m + 1) z Q_m^m;
           Q_l^m = ((2l - 1) z Q_{l-1}^m - (l + m - 1) Q_{l-2}^m) / (l - m) */
        dual3 Q[4];
        double dfact = 1.0;
        for (int i = 1; i <= 2 * m - 1; i += 2) dfact *= i;
        Q[m] = d3((m % 2) ? -dfact : dfact, 0, 0, 0);
        if (m + 1 <= lmax) Q[m + 1] = d3_scale(d3_mul(Z, Q[m]), 2.0 * m + 1.0);
        for (int l = m + 2; l <= lmax; ++l)
            Q[l] = d3_scale(d3_add(d3_scale(d3_mul(Z, Q[l - 1]), 2.0 * l - 1.0),
                                   d3_scale(Q[l - 2], -(double)(l + m - 1))),
                            1.0 / (double)(l - m));
        for (int l = m; l <= lmax; ++l) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            if (m == 0) {
                Y[l * l + l] = d3_scale(Q[l], K);
            } else {
                Y[l * l + l + m] = d3_scale(d3_mul(Q[l], Cm[m]), sqrt(2.0) * K);
                Y[l * l + l - m] = d3_scale(d3_mul(Q[l], Sm[m]), sqrt(2.0) * K);
            }
        }
    }
}

/* Exported for the basis pins (orthonormality, library comparison). */
void oc_sh_eval(int lmax, int64_t npts, const double* dirs, double* out_y, double* out_grad) {
    int nc = (lmax + 1) * (lmax + 1);
    for (int64_t i = 0; i < npts; ++i) {
        dual3 Y[16];
        sh_basis(lmax, dirs + 3 * i, Y);
        for (int k = 0; k < nc; ++k) {
            out_y[i * nc + k] = Y[k].v;
            if (out_grad) {
                out_grad[(i * nc + k) * 3 + 0] = Y[k].dx;
                out_grad[(i * nc + k) * 3 + 1] = Y[k].dy;
                out_grad[(i * nc + k) * 3 + 2] = Y[k].dz;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Preprocessing: one Gaussian (Sec. 3.1 "Preprocessing", Sec. 3.3)          */
/* ------------------------------------------------------------------------ */

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static double frac_dist(double x) { return fabs(x - nearbyint(x)); }

#define OC_TILE_INFLATE 1e-3
#define OC_TILE_SLACK (1.0 / 256.0)

/* Tiles [*lo, *hi] of tile row ty that the tile-test ellipse q <= t reaches,
 * within the rect.  The ellipse cut by the row's band of pixel-centre y values
 * is convex, so its x-range is one interval: the largest x over the band is at
 * the ellipse's rightmost point (dy = -B x_r / C) clamped to the band, the
 * smallest at the leftmost point (dy = +B x_r / C) clamped, and a tile is kept
 * when its pixel-centre x-range overlaps that interval.  Returns 0 for an
 * empty row.  *margin receives the distance (px) of these decisions to a
 * flip. */
static int row_span(const oc_proj* P, const oc_options* opt, int ty, int* lo, int* hi, double* margin) {
    if (!opt->tile_test) {
        *lo = P->rect[0];
        *hi = P->rect[2];
        return 1;
    }
    const double A = P->conic[0], B = P->conic[1], C = P->conic[2];
    const double t = P->tg * (1.0 + OC_TILE_INFLATE);
    const double det = A * C - B * B;
    const double xr = sqrt(t * C / det), yr = sqrt(t * A / det);
    const int TW = opt->tile_w, TH = opt->tile_h;
    const double sl_px = OC_TILE_SLACK;
    const double ya = ty * TH + 0.5 - sl_px - P->uv[1], yb = ty * TH + TH - 0.5 + sl_px - P->uv[1];
    double m = fabs(ya - yr);
    if (fabs(yb + yr) < m) m = fabs(yb + yr);
    if (m < *margin) *margin = m;
    const double blo = ya > -yr ? ya : -yr, bhi = yb < yr ? yb : yr;
    if (blo > bhi) return 0;
    double dr = -B * xr / C, dl = B * xr / C;
    dr = dr < blo ? blo : (dr > bhi ? bhi : dr);
    dl = dl < blo ? blo : (dl > bhi ? bhi : dl);
    double sr = A * t - det * dr * dr, sl = A * t - det * dl * dl;
    const double xR = P->uv[0] + (-B * dr + sqrt(sr > 0 ? sr : 0)) / A;
    const double xL = P->uv[0] + (-B * dl - sqrt(sl > 0 ? sl : 0)) / A;
    const double fr = (xR + sl_px - 0.5) / TW, fl = (xL - sl_px - TW + 0.5) / TW;
    if (frac_dist(fr) * TW < *margin) *margin = frac_dist(fr) * TW;
    if (frac_dist(fl) * TW < *margin) *margin = frac_dist(fl) * TW;
    int a = (int)ceil(fl), b = (int)floor(fr);
    if (a < P->rect[0]) a = P->rect[0];
    if (b > P->rect[2]) b = P->rect[2];
    *lo = a;
    *hi = b;
    return b >= a;
}

static void project_one(int64_t g, int sh_degree, const double* means, const double* log_scales,
                        const double* quats, const double* logits, const double* sh,
                        const uint32_t* mask, const oc_camera* cam, const oc_options* opt,
                        oc_proj* P) {
    memset(P, 0, sizeof(*P));
    P->margin_px = INFINITY;
    P->margin_rel = INFINITY;
    int nc = (sh_degree + 1) * (sh_degree + 1);

    /* view-cluster filter (Sec. 3.3 "Algorithm"): Gaussians of the selected
       1 + M clusters, shared Gaussians carry every cluster bit */
    if (opt->use_mask && mask && (mask[g] & opt->sel_bits) == 0u) return;

    const double* m = means + 3 * g;
    double Xc[3];
    for (int i = 0; i < 3; ++i)
        Xc[i] = cam->R[3 * i + 0] * m[0] + cam->R[3 * i + 1] * m[1] + cam->R[3 * i + 2] * m[2] + cam->t[i];
    double X = Xc[0], Y = Xc[1], Z = Xc[2];
    memcpy(P->mean_cam, Xc, sizeof(Xc));

    /* frustum cull */
    if (Z <= cam->near_z) return;
    double limx = opt->frustum_slack * cam->width / (2.0 * cam->fx);
    double limy = opt->frustum_slack * cam->height / (2.0 * cam->fy);
    if (fabs(X / Z) > limx || fabs(Y / Z) > limy) return;
    double mrel = fabs(Z - cam->near_z) / cam->near_z;
    double mx = fabs(fabs(X / Z) - limx) / limx, my = fabs(fabs(Y / Z) - limy) / limy;
    if (mx < mrel) mrel = mx;
    if (my < mrel) mrel = my;

    /* opacity */
    double o = sigmoid(logits[g]);
    double tg = 9.0;
    if (opt->opacity_filter) {
        /* Eqn. 4-5: beyond q = 2 ln(o / alpha_theta) the alpha is below alpha_theta */
        if (o <= opt->alpha_min) return;
        double lim = 2.0 * log(o / opt->alpha_min);
        if (lim < tg) tg = lim;
        double mo = fabs(o - opt->alpha_min) / opt->alpha_min;
        if (mo < mrel) mrel = mo;
    }

    /* 3D covariance Sigma = R S S^T R^T */
    const double* q = quats + 4 * g;
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qu[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
    double Rq[9], S2[9] = {0}, tmp[9], RqT[9], Sigma[9];
    quat_to_rot(qu, Rq);
    for (int i = 0; i < 3; ++i) S2[4 * i] = exp(2.0 * log_scales[3 * g + i]);
    mat3_mul(Rq, S2, tmp);
    mat3_transpose(Rq, RqT);
    mat3_mul(tmp, RqT, Sigma);

    /* camera-space covariance W Sigma W^T */
    double WT[9], Sc[9];
    mat3_transpose(cam->R, WT);
    mat3_mul(cam->R, Sigma, tmp);
    mat3_mul(tmp, WT, Sc);

    /* EWA: Jacobian of (fx X / Z + cx, fy Y / Z + cy) at the mean */
    double J[6] = {cam->fx / Z, 0.0, -cam->fx * X / (Z * Z),
                   0.0, cam->fy / Z, -cam->fy * Y / (Z * Z)};
    double JS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += J[3 * i + k] * Sc[3 * k + j];
            JS[3 * i + j] = s;
        }
    double C2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += JS[3 * i + k] * J[3 * j + k];
            C2[2 * i + j] = s;
        }
    double a = C2[0] + opt->dilation, b = 0.5 * (C2[1] + C2[2]), c = C2[3] + opt->dilation;
    double det = a * c - b * b;
    if (det <= 0.0) return;
    P->cov2[0] = a; P->cov2[1] = b; P->cov2[2] = c;
    P->conic[0] = c / det; P->conic[1] = -b / det; P->conic[2] = a / det;

    /* screen position */
    double u = cam->fx * X / Z + cam->cx;
    double v = cam->fy * Y / Z + cam->cy;
    P->uv[0] = u; P->uv[1] = v;

    /* rect: the support ellipse q <= t_g lies inside sqrt(t_g lambda_max) */
    double mid = 0.5 * (a + c);
    double disc = 0.25 * (a - c) * (a - c) + b * b;
    if (disc < 0.0) disc = 0.0;
    double lmax = mid + sqrt(disc);
    double rr = sqrt(tg * lmax);
    int r = (int)ceil(rr);
    P->radius = r;
    int px0 = (int)floor(u - 0.5 - r), px1 = (int)ceil(u - 0.5 + r);
    int py0 = (int)floor(v - 0.5 - r), py1 = (int)ceil(v - 0.5 + r);
    double mpx = frac_dist(rr);
    double mu = frac_dist(u - 0.5), mv = frac_dist(v - 0.5);
    if (mu < mpx) mpx = mu;
    if (mv < mpx) mpx = mv;
    if (px0 < 0) px0 = 0;
    if (py0 < 0) py0 = 0;
    if (px1 > cam->width - 1) px1 = cam->width - 1;
    if (py1 > cam->height - 1) py1 = cam->height - 1;
    P->margin_rel = mrel;
    P->tg = tg;
    if (px0 > px1 || py0 > py1) {
        P->margin_px = mpx;
        return;
    }
    P->rect[0] = px0 / opt->tile_w; P->rect[1] = py0 / opt->tile_h;
    P->rect[2] = px1 / opt->tile_w; P->rect[3] = py1 / opt->tile_h;
    P->ntiles = 0;
    for (int ty = P->rect[1]; ty <= P->rect[3]; ++ty) {
        int lo, hi;
        if (row_span(P, opt, ty, &lo, &hi, &mpx)) P->ntiles += hi - lo + 1;
    }
    P->margin_px = mpx;
    if (P->ntiles == 0) return;

    /* colour from SH in the view direction */
    double cc[3];
    camera_centre(cam, cc);
    double dir[3] = {m[0] - cc[0], m[1] - cc[1], m[2] - cc[2]};
    double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int i = 0; i < 3; ++i) dir[i] /= dn;
    dual3 Yb[16];
    sh_basis(sh_degree, dir, Yb);
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5;
        for (int k = 0; k < nc; ++k) s += sh[(g * nc + k) * 3 + ch] * Yb[k].v;
        P->rgb_raw[ch] = s;
        P->rgb[ch] = s > 0.0 ? s : 0.0;
    }

    P->opacity = o;
    P->depth32 = (float)Z;
    P->visible = 1;
}

void oc_preprocess(int64_t n, int sh_degree, const double* means, const double* log_scales,
                   const double* quats, const double* logits, const double* sh, const uint32_t* mask,
                   const oc_camera* cam, const oc_options* opt, oc_proj* out, int nthreads) {
#ifdef _OPENMP
    #pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t g = 0; g < n; ++g)
        project_one(g, sh_degree, means, log_scales, quats, logits, sh, mask, cam, opt, out + g);
    (void)nthreads;
}

/* ------------------------------------------------------------------------ */
/* Tile lists (Sec. 3.1 "Sorting"): (tile, fp32 depth, index) order          */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t tile; uint32_t dbits; int32_t gid; } oc_inst;

static int inst_cmp(const void* pa, const void* pb) {
    const oc_inst* a = (const oc_inst*)pa;
    const oc_inst* b = (const oc_inst*)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

int64_t oc_count_instances(int64_t n, const oc_proj* proj) {
    int64_t K = 0;
    for (int64_t g = 0; g < n; ++g)
        if (proj[g].visible) K += proj[g].ntiles;
    return K;
}

/* Writes the sorted instance list (tile id, Gaussian id) and the per-tile
   [start, end) ranges; tile id = ty * tiles_x + tx. */
void oc_build_instances(int64_t n, const oc_proj* proj, const oc_options* opt, int tiles_x, int tiles_y,
                        int32_t* out_tile, int32_t* out_gid, int64_t* out_ranges) {
    int64_t K = oc_count_instances(n, proj);
    oc_inst* inst = (oc_inst*)malloc(sizeof(oc_inst) * (K > 0 ? K : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        const oc_proj* P = proj + g;
        if (!P->visible) continue;
        uint32_t bits;
        memcpy(&bits, &P->depth32, 4);
        for (int ty = P->rect[1]; ty <= P->rect[3]; ++ty) {
            int lo, hi;
            double mdummy = INFINITY;
            if (!row_span(P, opt, ty, &lo, &hi, &mdummy)) continue;
            for (int tx = lo; tx <= hi; ++tx) {
                inst[k].tile = ty * tiles_x + tx;
                inst[k].dbits = bits;
                inst[k].gid = (int32_t)g;
                ++k;
            }
        }
    }
    qsort(inst, (size_t)K, sizeof(oc_inst), inst_cmp);
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t < ntiles; ++t) { out_ranges[2 * t] = 0; out_ranges[2 * t + 1] = 0; }
    for (int64_t i = 0; i < K; ++i) {
        out_tile[i] = inst[i].tile;
        out_gid[i] = inst[i].gid;
        int t = inst[i].tile;
        if (i == 0 || inst[i - 1].tile != t) out_ranges[2 * t] = i;
        if (i == K - 1 || inst[i + 1].tile != t) out_ranges[2 * t + 1] = i + 1;
    }
    free(inst);
}

/* ------------------------------------------------------------------------ */
/* Blending (Eqns. 1-2) and contribution-aware rasterization (Alg. 1)        */
/* ------------------------------------------------------------------------ */

typedef struct {
    double C[3];
    double T;
    int64_t ncontrib;    /* 1 + list position of the last blended entry, 0 if none */
    int done;
    double margin;       /* min relative distance of a decision to its threshold */
} px_state;

static void px_init(px_state* s) {
    s->C[0] = s->C[1] = s->C[2] = 0.0;
    s->T = 1.0;
    s->ncontrib = 0;
    s->done = 0;
    s->margin = INFINITY;
}

static void upd_margin(double* m, double v) { if (v < *m) *m = v; }

/* q = d^T Sigma'^-1 d at the sample point (x, y), d = (x, y) - (u, v). */
static double quad_at(const oc_proj* P, double x, double y) {
    double dx = x - P->uv[0], dy = y - P->uv[1];
    return P->conic[0] * dx * dx + 2.0 * P->conic[1] * dx * dy + P->conic[2] * dy * dy;
}

/* Eqn. 2 with the 0.99 clamp. */
static double alpha_of_q(const oc_proj* P, const oc_options* opt, double q) {
    double al = P->opacity * exp(-0.5 * q);
    return al < opt->alpha_max ? al : opt->alpha_max;
}

/* The per-pixel rule: outside the support or alpha < alpha_theta the entry is
   skipped; once T (1 - alpha) falls below Gamma_theta the pixel stops without
   blending it; otherwise C += T alpha c.  Returns 1 if blended. */
static int px_blend(px_state* s, const oc_proj* P, const oc_options* opt, double x, double y,
                    int64_t pos, int64_t* cnt) {
    double q = quad_at(P, x, y);
    cnt[2]++;
    upd_margin(&s->margin, fabs(q - P->tg) / P->tg);
    if (q > P->tg) return 0;
    double al = alpha_of_q(P, opt, q);
    upd_margin(&s->margin, fabs(al - opt->alpha_min) / opt->alpha_min);
    if (al < opt->alpha_min) return 0;
    double Tn = s->T * (1.0 - al);
    upd_margin(&s->margin, fabs(Tn - opt->t_stop) / opt->t_stop);
    if (Tn < opt->t_stop) { s->done = 1; cnt[6]++; return 0; }
    for (int ch = 0; ch < 3; ++ch) s->C[ch] += s->T * al * P->rgb[ch];
    s->T = Tn;
    s->ncontrib = pos + 1;
    cnt[3]++;
    if (al >= opt->alpha_max) cnt[7]++;
    return 1;
}

/* Leader test of Alg. 1: does the group's first pixel see alpha >= alpha_theta?
   A leader outside the support sees alpha = 0. */
static int leader_pass(const oc_proj* P, const oc_options* opt, double x, double y, double* margin) {
    double q = quad_at(P, x, y);
    upd_margin(margin, fabs(q - P->tg) / P->tg);
    if (q > P->tg) return 0;
    double al = alpha_of_q(P, opt, q);
    upd_margin(margin, fabs(al - opt->alpha_min) / opt->alpha_min);
    return al >= opt->alpha_min;
}

static void write_px(const px_state* s, int W, int H, int x, int y, double* rgb, double* Tout,
                     int64_t* nc, double* margin) {
    int64_t p = (int64_t)y * W + x;
    for (int ch = 0; ch < 3; ++ch) rgb[(int64_t)ch * W * H + p] = s->C[ch];
    Tout[p] = s->T;
    nc[p] = s->ncontrib;
    margin[p] = s->margin;
}

/* One tile: plain blending, every pixel walks the tile list (Sec. 3.1). */
static void render_tile_plain(const oc_proj* proj, const int32_t* gid, int64_t start, int64_t end,
                              int x0, int y0, int x1, int y1, int W, int H, const oc_options* opt,
                              double* rgb, double* Tout, int64_t* nc, double* margin, int64_t* cnt) {
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            px_state s;
            px_init(&s);
            for (int64_t i = start; i < end && !s.done; ++i)
                px_blend(&s, proj + gid[i], opt, x + 0.5, y + 0.5, i - start, cnt);
            write_px(&s, W, H, x, y, rgb, Tout, nc, margin);
        }
}

/* One tile under Algorithm 1: pixel groups of group_w x group_h, leader =
   first (top-left) pixel.  The leader's alpha is computed for every entry
   while any pixel of the group is live, even once the leader itself is done. */
static void render_tile_cr(const oc_proj* proj, const int32_t* gid, int64_t start, int64_t end,
                           int x0, int y0, int x1, int y1, int W, int H, const oc_options* opt,
                           double* rgb, double* Tout, int64_t* nc, double* margin, int64_t* cnt) {
    int gw = opt->group_w, gh = opt->group_h;
    px_state st[64];
    for (int gy = y0; gy < y1; gy += gh)
        for (int gx = x0; gx < x1; gx += gw) {
            int npx = 0;
            int xs[64], ys[64];
            for (int dy = 0; dy < gh; ++dy)
                for (int dx = 0; dx < gw; ++dx) {
                    int x = gx + dx, y = gy + dy;
                    if (x >= x1 || y >= y1) continue;
                    xs[npx] = x; ys[npx] = y;
                    px_init(&st[npx]);
                    ++npx;
                }
            double gmargin = INFINITY;
            for (int64_t i = start; i < end; ++i) {
                int live = 0;
                for (int k = 0; k < npx; ++k) live |= !st[k].done;
                if (!live) break;
                const oc_proj* P = proj + gid[i];
                cnt[4]++;
                if (!leader_pass(P, opt, gx + 0.5, gy + 0.5, &gmargin)) { cnt[5]++; continue; }
                for (int k = 0; k < npx; ++k)
                    if (!st[k].done) px_blend(&st[k], P, opt, xs[k] + 0.5, ys[k] + 0.5, i - start, cnt);
            }
            for (int k = 0; k < npx; ++k) {
                upd_margin(&st[k].margin, gmargin);
                write_px(&st[k], W, H, xs[k], ys[k], rgb, Tout, nc, margin);
            }
        }
}

/* Tiled render of one camera from the sorted instance list.  Output RGB is
   planar [3][H][W]; T and ncontrib are [H][W]. */
void oc_render_tiled(const oc_proj* proj, const int32_t* gid, const int64_t* ranges, int W, int H,
                     const oc_options* opt, double* rgb, double* Tout, int64_t* nc, double* margin,
                     int64_t* counters, int nthreads) {
    int tw = opt->tile_w, th = opt->tile_h;
    int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int nt = nthreads > 0 ? nthreads : 1;
    int64_t* cnt = (int64_t*)calloc((size_t)nt * OC_NCOUNT, sizeof(int64_t));
#ifdef _OPENMP
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t t = 0; t < ntiles; ++t) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
        int x0 = tx * tw, y0 = ty * th;
        int x1 = x0 + tw < W ? x0 + tw : W, y1 = y0 + th < H ? y0 + th : H;
        if (opt->cr)
            render_tile_cr(proj, gid, ranges[2 * t], ranges[2 * t + 1], x0, y0, x1, y1, W, H, opt, rgb,
                           Tout, nc, margin, cnt + tid * OC_NCOUNT);
        else
            render_tile_plain(proj, gid, ranges[2 * t], ranges[2 * t + 1], x0, y0, x1, y1, W, H, opt, rgb,
                              Tout, nc, margin, cnt + tid * OC_NCOUNT);
    }
    for (int k = 0; k < OC_NCOUNT; ++k) {
        int64_t s = 0;
        for (int i = 0; i < nt; ++i) s += cnt[i * OC_NCOUNT + k];
        counters[k] += s;
    }
    free(cnt);
}

/* ------------------------------------------------------------------------ */
/* Outcomes of a pixel under near-threshold decisions                        */
/* ------------------------------------------------------------------------ */

/* A decision that double precision takes within a relative distance `tol` of
   its threshold may go the other way in a single-precision render.  For one
   pixel, every outcome (C, T) reachable by taking either branch of any such
   decision is enumerated by a depth-first walk of the pixel's tile list: both
   branches are followed at a near decision, the double-precision branch
   everywhere else.  The decisions are the pixel rule's (support q <= t_g and
   alpha >= alpha_theta, taken together as one test; the stop test on
   T (1 - alpha)) and, under Algorithm 1, the group leader's test.  A leader
   pixel's own support and alpha test is the leader test on the same sample
   point and is not branched a second time.  The double-precision branch is
   always followed first, so outcome 0 is the ordinary render's pixel. */

typedef struct {
    const oc_proj* proj;
    const int32_t* gid;
    int64_t end;
    const oc_options* opt;
    double px, py;        /* the pixel's sample point */
    double lx, ly;        /* its group leader's sample point (Algorithm 1) */
    int is_leader;
    double tol;
    int max_out;
    int n_out;            /* outcomes written; max_out + 1 once there are more */
    double* out;          /* [max_out][4]: r, g, b, T */
} po_walk;

/* The values "q <= t_g and alpha >= alpha_theta" at (x, y) can take when
   either near component may flip: bit 0 set = false reachable, bit 1 = true
   reachable.  *base = the double-precision value. */
static int po_on(const po_walk* w, const oc_proj* P, double x, double y, int* base) {
    double q = quad_at(P, x, y);
    double al = alpha_of_q(P, w->opt, q);
    int s = q <= P->tg, a = al >= w->opt->alpha_min;
    int s_near = fabs(q - P->tg) / P->tg < w->tol;
    int a_near = fabs(al - w->opt->alpha_min) / w->opt->alpha_min < w->tol;
    *base = s && a;
    int vals = 0;
    for (int fs = 0; fs <= s_near; ++fs)
        for (int fa = 0; fa <= a_near; ++fa) vals |= 1 << ((fs ? !s : s) && (fa ? !a : a));
    return vals;
}

static void po_leaf(po_walk* w, const double* C, double T) {
    if (w->n_out >= w->max_out) { w->n_out = w->max_out + 1; return; }
    double* o = w->out + 4 * (int64_t)w->n_out;
    o[0] = C[0]; o[1] = C[1]; o[2] = C[2]; o[3] = T;
    w->n_out++;
}

/* Continue at list entry i, at stage `stage` of that entry's decisions:
   0 the leader test (Algorithm 1 only), 1 the pixel's support and alpha
   test, 2 the stop test and the blend. */
static void po_walk_from(po_walk* w, int64_t i, int stage, const double* C0, double T) {
    double C[3] = {C0[0], C0[1], C0[2]};
    while (i < w->end) {
        if (w->n_out > w->max_out) return;
        const oc_proj* P = w->proj + w->gid[i];
        int base, v;
        if (stage == 0) {
            if (w->opt->cr) {
                v = po_on(w, P, w->lx, w->ly, &base);
                if (v == 3) {
                    if (base) { po_walk_from(w, i, 1, C, T); po_walk_from(w, i + 1, 0, C, T); }
                    else { po_walk_from(w, i + 1, 0, C, T); po_walk_from(w, i, 1, C, T); }
                    return;
                }
                if (!base) { ++i; continue; }     /* the whole group skips entry i */
            }
            stage = 1;
        }
        if (stage == 1) {
            if (!(w->opt->cr && w->is_leader)) {
                v = po_on(w, P, w->px, w->py, &base);
                if (v == 3) {
                    if (base) { po_walk_from(w, i, 2, C, T); po_walk_from(w, i + 1, 0, C, T); }
                    else { po_walk_from(w, i + 1, 0, C, T); po_walk_from(w, i, 2, C, T); }
                    return;
                }
                if (!base) { ++i; stage = 0; continue; }
            }
            stage = 2;
        }
        double al = alpha_of_q(P, w->opt, quad_at(P, w->px, w->py));
        double Tn = T * (1.0 - al);
        int stop = Tn < w->opt->t_stop;
        double Cn[3];
        for (int ch = 0; ch < 3; ++ch) Cn[ch] = C[ch] + T * al * P->rgb[ch];
        if (fabs(Tn - w->opt->t_stop) / w->opt->t_stop < w->tol) {
            if (stop) { po_leaf(w, C, T); po_walk_from(w, i + 1, 0, Cn, Tn); }
            else { po_walk_from(w, i + 1, 0, Cn, Tn); po_leaf(w, C, T); }
            return;
        }
        if (stop) { po_leaf(w, C, T); return; }
        C[0] = Cn[0]; C[1] = Cn[1]; C[2] = Cn[2];
        T = Tn;
        ++i;
        stage = 0;
    }
    po_leaf(w, C, T);
}

/* Outcomes of the pixels pix[k] = y * W + x of a tiled render (the lists and
   ranges of oc_build_instances): out[k][j][0..3] = (r, g, b, T) of outcome j,
   n_out[k] = the number of outcomes, or -1 when there are more than max_out. */
void oc_pixel_outcomes(const oc_proj* proj, const int32_t* gid, const int64_t* ranges, int W, int H,
                       const oc_options* opt, const int64_t* pix, int64_t npix, double tol, int max_out,
                       double* out, int32_t* n_out, int nthreads) {
    int tw = opt->tile_w, th = opt->tile_h;
    int tiles_x = (W + tw - 1) / tw;
    int gw = opt->cr ? opt->group_w : 1, gh = opt->cr ? opt->group_h : 1;
    (void)H;
#ifdef _OPENMP
    #pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t k = 0; k < npix; ++k) {
        int x = (int)(pix[k] % W), y = (int)(pix[k] / W);
        int tx = x / tw, ty = y / th;
        int64_t t = (int64_t)ty * tiles_x + tx;
        int x0 = tx * tw, y0 = ty * th;
        int gx = x0 + (x - x0) / gw * gw, gy = y0 + (y - y0) / gh * gh;
        po_walk w;
        w.proj = proj;
        w.gid = gid;
        w.end = ranges[2 * t + 1];
        w.opt = opt;
        w.px = x + 0.5; w.py = y + 0.5;
        w.lx = gx + 0.5; w.ly = gy + 0.5;
        w.is_leader = gx == x && gy == y;
        w.tol = tol;
        w.max_out = max_out;
        w.n_out = 0;
        w.out = out + (int64_t)4 * max_out * k;
        double C0[3] = {0.0, 0.0, 0.0};
        if (ranges[2 * t] < ranges[2 * t + 1]) po_walk_from(&w, ranges[2 * t], 0, C0, 1.0);
        else po_leaf(&w, C0, 1.0);
        n_out[k] = w.n_out > max_out ? -1 : w.n_out;
    }
}

/* ------------------------------------------------------------------------ */
/* Brute-force render: no tiles, no rects.  Every pixel walks every visible  */
/* Gaussian in global (fp32 depth, index) order under the same rules.        */
/* ------------------------------------------------------------------------ */

static int depth_cmp(const void* pa, const void* pb) {
    const oc_inst* a = (const oc_inst*)pa;
    const oc_inst* b = (const oc_inst*)pb;
    if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

void oc_render_bruteforce(int64_t n, const oc_proj* proj, int W, int H, const oc_options* opt,
                          double* rgb, double* Tout, int64_t* nc, int nthreads) {
    oc_inst* ord = (oc_inst*)malloc(sizeof(oc_inst) * (n > 0 ? n : 1));
    int64_t nv = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (!proj[g].visible) continue;
        memcpy(&ord[nv].dbits, &proj[g].depth32, 4);
        ord[nv].gid = (int32_t)g;
        ord[nv].tile = 0;
        ++nv;
    }
    qsort(ord, (size_t)nv, sizeof(oc_inst), depth_cmp);
    int32_t* gid = (int32_t*)malloc(sizeof(int32_t) * (nv > 0 ? nv : 1));
    for (int64_t i = 0; i < nv; ++i) gid[i] = ord[i].gid;
    free(ord);
    int gw = opt->cr ? opt->group_w : 1, gh = opt->cr ? opt->group_h : 1;
    int ngx = (W + gw - 1) / gw, ngy = (H + gh - 1) / gh;
    double* margin = (double*)malloc(sizeof(double) * (size_t)W * H);
#ifdef _OPENMP
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int gy = 0; gy < ngy; ++gy) {
        int64_t cnt[OC_NCOUNT] = {0};
        for (int gx = 0; gx < ngx; ++gx) {
            int x0 = gx * gw, y0 = gy * gh;
            int x1 = x0 + gw < W ? x0 + gw : W, y1 = y0 + gh < H ? y0 + gh : H;
            if (opt->cr)
                render_tile_cr(proj, gid, 0, nv, x0, y0, x1, y1, W, H, opt, rgb, Tout, nc, margin, cnt);
            else
                render_tile_plain(proj, gid, 0, nv, x0, y0, x1, y1, W, H, opt, rgb, Tout, nc, margin, cnt);
        }
    }
    (void)nthreads;
    free(margin);
    free(gid);
}

/* ------------------------------------------------------------------------ */
/* Backward of the blending (for the fine-tuning of Sec. 3.5)                */
/* ------------------------------------------------------------------------ */
/*
 * With C = sum_j T_j alpha_j c_j over the blended entries j and
 * T_j = prod_{k<j, blended} (1 - alpha_k):
 *   dC/dc_j     = T_j alpha_j
 *   dC/dalpha_j = T_j c_j - S_j / (1 - alpha_j),  S_j = sum_{k>j} T_k alpha_k c_k
 * and alpha = o exp(-q / 2) unless clamped at 0.99 (then constant).  The skip
 * and stop decisions of the forward pass are held fixed (HP and CR "do not
 * participate in gradient descent", Sec. 3.5).  Per Gaussian the result is
 * dL/d(u, v, A, B, C, o, r, g, b) in g2d[9 * gid].
 */
typedef struct { int64_t pos; double T, al; int clamped; double x, y; } bw_rec;

static void backward_pixel(const oc_proj* proj, const int32_t* gid, int64_t start, int64_t end,
                           const int* leader_pass, double x, double y, const oc_options* opt,
                           const double* dC, double* g2d, bw_rec* rec) {
    /* forward replay, recording the blended entries */
    double T = 1.0;
    int64_t nb = 0;
    for (int64_t i = start; i < end; ++i) {
        if (leader_pass && !leader_pass[i - start]) continue;
        const oc_proj* P = proj + gid[i];
        double q = quad_at(P, x, y);
        if (q > P->tg) continue;
        double al = alpha_of_q(P, opt, q);
        if (al < opt->alpha_min) continue;
        double Tn = T * (1.0 - al);
        if (Tn < opt->t_stop) break;
        rec[nb].pos = i;
        rec[nb].T = T;
        rec[nb].al = al;
        rec[nb].clamped = (al >= opt->alpha_max);
        rec[nb].x = x; rec[nb].y = y;
        ++nb;
        T = Tn;
    }
    double S[3] = {0, 0, 0};
    for (int64_t j = nb - 1; j >= 0; --j) {
        const oc_proj* P = proj + gid[rec[j].pos];
        double* G = g2d + 9 * (int64_t)gid[rec[j].pos];
        double Tj = rec[j].T, al = rec[j].al;
        double dal = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            G[6 + ch] += Tj * al * dC[ch];
            dal += dC[ch] * (Tj * P->rgb[ch] - S[ch] / (1.0 - al));
        }
        for (int ch = 0; ch < 3; ++ch) S[ch] += Tj * al * P->rgb[ch];
        if (rec[j].clamped) continue;
        double dx = x - P->uv[0], dy = y - P->uv[1];
        double A = P->conic[0], B = P->conic[1], Cc = P->conic[2];
        double q = A * dx * dx + 2.0 * B * dx * dy + Cc * dy * dy;
        double Gs = exp(-0.5 * q);
        G[5] += dal * Gs;                       /* d alpha / d o */
        double dq = dal * (-0.5 * al);          /* d alpha / d q */
        G[2] += dq * dx * dx;
        G[3] += dq * 2.0 * dx * dy;
        G[4] += dq * dy * dy;
        G[0] += dq * (-(2.0 * A * dx + 2.0 * B * dy));
        G[1] += dq * (-(2.0 * B * dx + 2.0 * Cc * dy));
    }
}

void oc_backward_raster(int64_t n, const oc_proj* proj, const int32_t* gid, const int64_t* ranges, int W,
                        int H, const oc_options* opt, const double* dL_drgb, double* g2d) {
    (void)n;
    int tw = opt->tile_w, th = opt->tile_h;
    int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    for (int t = 0; t < tiles_x * tiles_y; ++t) {
        int64_t start = ranges[2 * t], end = ranges[2 * t + 1];
        int64_t len = end - start;
        bw_rec* rec = (bw_rec*)malloc(sizeof(bw_rec) * (len > 0 ? len : 1));
        int* lp = (int*)malloc(sizeof(int) * (len > 0 ? len : 1));
        int tx = t % tiles_x, ty = t / tiles_x;
        int x0 = tx * tw, y0 = ty * th;
        int x1 = x0 + tw < W ? x0 + tw : W, y1 = y0 + th < H ? y0 + th : H;
        int gw = opt->cr ? opt->group_w : 1, gh = opt->cr ? opt->group_h : 1;
        for (int gy = y0; gy < y1; gy += gh)
            for (int gx = x0; gx < x1; gx += gw) {
                if (opt->cr) {
                    /* the leader decisions of Alg. 1, replayed; entries after the
                       whole group stopped are never blended anyway */
                    for (int64_t i = 0; i < len; ++i) {
                        double mdummy = INFINITY;
                        lp[i] = leader_pass(proj + gid[start + i], opt, gx + 0.5, gy + 0.5, &mdummy);
                    }
                }
                for (int y = gy; y < gy + gh && y < y1; ++y)
                    for (int x = gx; x < gx + gw && x < x1; ++x) {
                        double dC[3];
                        for (int ch = 0; ch < 3; ++ch) dC[ch] = dL_drgb[(int64_t)ch * W * H + (int64_t)y * W + x];
                        backward_pixel(proj, gid, start, end, opt->cr ? lp : NULL, x + 0.5, y + 0.5, opt, dC,
                                       g2d, rec);
                    }
            }
        free(rec);
        free(lp);
    }
}

/* ------------------------------------------------------------------------ */
/* Backward of the preprocessing (chain rule through Sec. 3.1's projection)  */
/* ------------------------------------------------------------------------ */

void oc_backward_preprocess(int64_t n, int sh_degree, const double* means, const double* log_scales,
                            const double* quats, const double* logits, const double* sh,
                            const oc_camera* cam, const oc_options* opt, const oc_proj* proj,
                            const double* g2d, double* d_means, double* d_log_scales, double* d_quats,
                            double* d_logits, double* d_sh) {
    (void)opt;
    int nc = (sh_degree + 1) * (sh_degree + 1);
    double cc[3];
    camera_centre(cam, cc);
    const double* W = cam->R;
    for (int64_t g = 0; g < n; ++g) {
        const oc_proj* P = proj + g;
        for (int i = 0; i < 3; ++i) { d_means[3 * g + i] = 0; d_log_scales[3 * g + i] = 0; }
        for (int i = 0; i < 4; ++i) d_quats[4 * g + i] = 0;
        d_logits[g] = 0;
        for (int k = 0; k < nc * 3; ++k) d_sh[g * nc * 3 + k] = 0;
        if (!P->visible) continue;
        const double* G = g2d + 9 * g;
        const double* m = means + 3 * g;
        double X = P->mean_cam[0], Y = P->mean_cam[1], Z = P->mean_cam[2];
        double fx = cam->fx, fy = cam->fy;
        double dXc[3] = {0, 0, 0};

        /* colour: rgb = max(0, sum_k sh_k Y_k(d) + .5), d = unit(m - campos) */
        double v[3] = {m[0] - cc[0], m[1] - cc[1], m[2] - cc[2]};
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
        dual3 Yb[16];
        sh_basis(sh_degree, dir, Yb);
        double ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            double dr = P->rgb_raw[ch] > 0.0 ? G[6 + ch] : 0.0;
            for (int k = 0; k < nc; ++k) {
                d_sh[(g * nc + k) * 3 + ch] = Yb[k].v * dr;
                double s = sh[(g * nc + k) * 3 + ch] * dr;
                ddir[0] += s * Yb[k].dx; ddir[1] += s * Yb[k].dy; ddir[2] += s * Yb[k].dz;
            }
        }
        double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
        for (int i = 0; i < 3; ++i) d_means[3 * g + i] += (ddir[i] - dir[i] * dd) / vn;

        /* opacity */
        double o = P->opacity;
        d_logits[g] = G[5] * o * (1.0 - o);

        /* conic (A, B, C) = (c, -b, a) / (a c - b^2) */
        double a = P->cov2[0], b = P->cov2[1], c = P->cov2[2];
        double D = a * c - b * b, D2 = D * D;
        double gA = G[2], gB = G[3], gC = G[4];
        double da = gA * (-c * c / D2) + gB * (b * c / D2) + gC * (-b * b / D2);
        double db = gA * (2.0 * b * c / D2) + gB * (-(D + 2.0 * b * b) / D2) + gC * (2.0 * a * b / D2);
        double dc = gA * (-b * b / D2) + gB * (a * b / D2) + gC * (-a * a / D2);
        /* Sigma' = J Sc J^T + dilation: symmetric gradient M */
        double M[4] = {da, 0.5 * db, 0.5 * db, dc};

        /* recompute Sigma, Sc and J */
        const double* q = quats + 4 * g;
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qu[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
        double Rq[9], RqT[9], S2[9] = {0}, tmp[9], Sigma[9], WT[9], Sc[9];
        double s[3];
        for (int i = 0; i < 3; ++i) { s[i] = exp(log_scales[3 * g + i]); S2[4 * i] = s[i] * s[i]; }
        quat_to_rot(qu, Rq);
        mat3_mul(Rq, S2, tmp);
        mat3_transpose(Rq, RqT);
        mat3_mul(tmp, RqT, Sigma);
        mat3_transpose(W, WT);
        mat3_mul(W, Sigma, tmp);
        mat3_mul(tmp, WT, Sc);
        double J[6] = {fx / Z, 0.0, -fx * X / (Z * Z), 0.0, fy / Z, -fy * Y / (Z * Z)};

        /* dL/dSc = J^T M J */
        double dSc[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) acc += J[3 * k + i] * M[2 * k + l] * J[3 * l + j];
                dSc[3 * i + j] = acc;
            }
        /* dL/dJ = 2 M J Sc */
        double dJ[6];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 3; ++l) acc += M[2 * i + k] * J[3 * k + l] * Sc[3 * l + j];
                dJ[3 * i + j] = 2.0 * acc;
            }
        dXc[0] += dJ[2] * (-fx / (Z * Z));
        dXc[1] += dJ[5] * (-fy / (Z * Z));
        dXc[2] += dJ[0] * (-fx / (Z * Z)) + dJ[2] * (2.0 * fx * X / (Z * Z * Z)) + dJ[4] * (-fy / (Z * Z)) +
                  dJ[5] * (2.0 * fy * Y / (Z * Z * Z));
        /* screen position u = fx X / Z + cx, v = fy Y / Z + cy */
        dXc[0] += G[0] * fx / Z;
        dXc[1] += G[1] * fy / Z;
        dXc[2] += G[0] * (-fx * X / (Z * Z)) + G[1] * (-fy * Y / (Z * Z));
        /* X_cam = W m + t */
        for (int i = 0; i < 3; ++i)
            d_means[3 * g + i] += W[0 * 3 + i] * dXc[0] + W[1 * 3 + i] * dXc[1] + W[2 * 3 + i] * dXc[2];

        /* Sc = W Sigma W^T  ->  dSigma = W^T dSc W */
        double dSigma[9];
        mat3_mul(WT, dSc, tmp);
        mat3_mul(tmp, W, dSigma);
        /* Sigma = sum_i s_i^2 r_i r_i^T with r_i the columns of Rq */
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) acc += Rq[3 * j + i] * dSigma[3 * j + k] * Rq[3 * k + i];
            d_log_scales[3 * g + i] = 2.0 * s[i] * s[i] * acc;   /* dL/ds_i * s_i */
        }
        /* dL/dRq = 2 dSigma Rq S^2 */
        double dR[9];
        mat3_mul(dSigma, Rq, tmp);
        mat3_mul(tmp, S2, dR);
        for (int i = 0; i < 9; ++i) dR[i] *= 2.0;
        /* dRq / d(unit quaternion) from the closed form of quat_to_rot */
        double w = qu[0], x = qu[1], y = qu[2], z = qu[3];
        double dq[4];
        dq[0] = dR[1] * (-2 * z) + dR[2] * (2 * y) + dR[3] * (2 * z) + dR[5] * (-2 * x) + dR[6] * (-2 * y) +
                dR[7] * (2 * x);
        dq[1] = dR[1] * (2 * y) + dR[2] * (2 * z) + dR[3] * (2 * y) + dR[4] * (-4 * x) + dR[5] * (-2 * w) +
                dR[6] * (2 * z) + dR[7] * (2 * w) + dR[8] * (-4 * x);
        dq[2] = dR[0] * (-4 * y) + dR[1] * (2 * x) + dR[2] * (2 * w) + dR[3] * (2 * x) + dR[5] * (2 * z) +
                dR[6] * (-2 * w) + dR[7] * (2 * z) + dR[8] * (-4 * y);
        dq[3] = dR[0] * (-4 * z) + dR[1] * (-2 * w) + dR[2] * (2 * x) + dR[3] * (2 * w) + dR[4] * (-4 * z) +
                dR[5] * (2 * y) + dR[6] * (2 * x) + dR[7] * (2 * y);
        /* normalisation q / |q| */
        double qd = qu[0] * dq[0] + qu[1] * dq[1] + qu[2] * dq[2] + qu[3] * dq[3];
        for (int i = 0; i < 4; ++i) d_quats[4 * g + i] = (dq[i] - qu[i] * qd) / qn;
    }
}

/* ------------------------------------------------------------------------ */
/* Runtime cluster selection (Sec. 3.3 "Algorithm")                          */
/* ------------------------------------------------------------------------ */
/*
 * Feature of a pose: (x / s, v) with x the camera position, s the position
 * normalisation of the offline clustering, v the unit viewing direction
 * (beta = 1).  The nearest centroid is chosen, then the M centroids nearest
 * to it; ties go to the lower cluster index.  Returns the cluster bit set.
 */
uint32_t oc_select_clusters(int nclusters, const double* centroids, double pos_scale, const oc_camera* cam,
                            int M) {
    if (nclusters <= 0) return 0xffffffffu;
    double c[3];
    camera_centre(cam, c);
    double f[6] = {c[0] / pos_scale, c[1] / pos_scale, c[2] / pos_scale, cam->R[6], cam->R[7], cam->R[8]};
    int best = 0;
    double bd = INFINITY;
    for (int k = 0; k < nclusters; ++k) {
        double d = 0.0;
        for (int i = 0; i < 6; ++i) d += (f[i] - centroids[6 * k + i]) * (f[i] - centroids[6 * k + i]);
        if (d < bd) { bd = d; best = k; }
    }
    uint32_t bits = 1u << best;
    for (int pick = 0; pick < M && pick < nclusters - 1; ++pick) {
        int arg = -1;
        double ad = INFINITY;
        for (int k = 0; k < nclusters; ++k) {
            if (bits & (1u << k)) continue;
            double d = 0.0;
            for (int i = 0; i < 6; ++i)
                d += (centroids[6 * best + i] - centroids[6 * k + i]) * (centroids[6 * best + i] - centroids[6 * k + i]);
            if (d < ad) { ad = d; arg = k; }
        }
        bits |= 1u << arg;
    }
    return bits;
}

/* ------------------------------------------------------------------------ */
/* Offline view-dependent representation (Sec. 3.3 "Offline Clustering").    */
/* Sampled camera poses are clustered on the feature (x / s, v); for every    */
/* pixel of every pose the Gaussians with the k largest contributions         */
/* Gamma_i alpha_i are found, and a Gaussian belongs to cluster c when it is  */
/* such a top contributor for some pose of c.  (Readings: k-means with        */
/* beta = 1, s = the largest camera distance of the samples; shared = the     */
/* Gaussians of every cluster; a Gaussian of no cluster is dropped.)          */
/* ------------------------------------------------------------------------ */

/* Pose feature: camera centre over the position scale, then the unit viewing
   direction (the camera's +z axis in world coordinates). */
void oc_pose_feature(const oc_camera* cam, double pos_scale, double* f) {
    double c[3];
    camera_centre(cam, c);
    for (int i = 0; i < 3; ++i) f[i] = c[i] / pos_scale;
    for (int i = 0; i < 3; ++i) f[3 + i] = cam->R[6 + i];
}

static double sqdist(const double* a, const double* b, int dim) {
    double d = 0.0;
    for (int i = 0; i < dim; ++i) d += (a[i] - b[i]) * (a[i] - b[i]);
    return d;
}

/* k-means of n points of `dim` coordinates into k clusters.  Seeding is
   k-means++ driven by the uniforms u[0..k): the first centre is point
   floor(u[0] n); centre j is the first point at which the running sum of the
   squared distances to the nearest chosen centre exceeds u[j] times their
   total (floor(u[j] n) if that total is zero).  Lloyd iterations then assign
   every point to its nearest centre (ties to the lower index) and move every
   centre to the mean of its points (an empty cluster keeps its centre),
   stopping once an assignment step changes nothing or after max_iter
   updates.  Returns the number of updates made. */
int oc_kmeans(int n, int dim, const double* x, int k, const double* u, int max_iter, double* cent,
              int32_t* assign) {
    double* d2 = (double*)malloc((size_t)n * sizeof(double));
    int first = (int)floor(u[0] * n);
    if (first >= n) first = n - 1;
    memcpy(cent, x + (size_t)first * dim, (size_t)dim * sizeof(double));
    for (int i = 0; i < n; ++i) d2[i] = sqdist(x + (size_t)i * dim, cent, dim);
    for (int j = 1; j < k; ++j) {
        double total = 0.0;
        for (int i = 0; i < n; ++i) total += d2[i];
        int pick = n - 1;
        if (total > 0.0) {
            const double target = u[j] * total;
            double run = 0.0;
            for (int i = 0; i < n; ++i) {
                run += d2[i];
                if (run > target) { pick = i; break; }
            }
        } else {
            pick = (int)floor(u[j] * n);
            if (pick >= n) pick = n - 1;
        }
        memcpy(cent + (size_t)j * dim, x + (size_t)pick * dim, (size_t)dim * sizeof(double));
        for (int i = 0; i < n; ++i) {
            const double d = sqdist(x + (size_t)i * dim, cent + (size_t)j * dim, dim);
            if (d < d2[i]) d2[i] = d;
        }
    }
    free(d2);
    for (int i = 0; i < n; ++i) assign[i] = -1;
    double* sum = (double*)malloc((size_t)k * dim * sizeof(double));
    int* cnt = (int*)malloc((size_t)k * sizeof(int));
    int it = 0;
    for (; it < max_iter; ++it) {
        int changed = 0;
        for (int i = 0; i < n; ++i) {
            int best = 0;
            double bd = sqdist(x + (size_t)i * dim, cent, dim);
            for (int j = 1; j < k; ++j) {
                const double d = sqdist(x + (size_t)i * dim, cent + (size_t)j * dim, dim);
                if (d < bd) { bd = d; best = j; }
            }
            if (assign[i] != best) { assign[i] = best; changed = 1; }
        }
        if (!changed) break;
        memset(sum, 0, (size_t)k * dim * sizeof(double));
        memset(cnt, 0, (size_t)k * sizeof(int));
        for (int i = 0; i < n; ++i) {
            for (int c = 0; c < dim; ++c) sum[(size_t)assign[i] * dim + c] += x[(size_t)i * dim + c];
            cnt[assign[i]]++;
        }
        for (int j = 0; j < k; ++j)
            if (cnt[j] > 0)
                for (int c = 0; c < dim; ++c) cent[(size_t)j * dim + c] = sum[(size_t)j * dim + c] / cnt[j];
    }
    free(sum);
    free(cnt);
    return it;
}

typedef struct {
    double w;
    int32_t g;
} oc_contrib;

static int contrib_cmp(const void* a, const void* b) {
    const oc_contrib* x = (const oc_contrib*)a;
    const oc_contrib* y = (const oc_contrib*)b;
    if (x->w != y->w) return x->w > y->w ? -1 : 1;
    return (x->g > y->g) - (x->g < y->g);
}

/* Per-pixel top-k contributors of a plain render (Sec. 3.3): every pixel
   walks its tile list under the rules of px_blend; a blended Gaussian
   contributes Gamma_i alpha_i = T alpha (T before it).  The k largest, ties
   to the lower Gaussian index, descending: out_ids / out_w [H W][k] (unused
   slots -1 / 0), out_count [H W], and out_margin [H W] = the smaller of the
   pixel's decision margin and the relative gap between the k-th and
   (k+1)-th contribution (INFINITY with k or fewer contributors). */
void oc_topk_contributors(const oc_proj* proj, const int32_t* gid, const int64_t* ranges, int W, int H,
                          const oc_options* opt, int k, int32_t* out_ids, double* out_w, int32_t* out_count,
                          double* out_margin, int nthreads) {
    int tw = opt->tile_w, th = opt->tile_h;
    int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int nt = nthreads > 0 ? nthreads : 1;
    (void)nt;
#ifdef _OPENMP
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t t = 0; t < ntiles; ++t) {
        int64_t cnt[OC_NCOUNT] = {0};
        int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
        int64_t start = ranges[2 * t], end = ranges[2 * t + 1];
        oc_contrib* buf = (oc_contrib*)malloc((size_t)(end > start ? end - start : 1) * sizeof(oc_contrib));
        for (int y = ty * th; y < ty * th + th && y < H; ++y)
            for (int x = tx * tw; x < tx * tw + tw && x < W; ++x) {
                px_state s;
                px_init(&s);
                int m = 0;
                for (int64_t i = start; i < end && !s.done; ++i) {
                    const double T = s.T;
                    const oc_proj* P = proj + gid[i];
                    if (px_blend(&s, P, opt, x + 0.5, y + 0.5, i - start, cnt)) {
                        buf[m].w = T * alpha_of_q(P, opt, quad_at(P, x + 0.5, y + 0.5));
                        buf[m].g = gid[i];
                        ++m;
                    }
                }
                qsort(buf, (size_t)m, sizeof(oc_contrib), contrib_cmp);
                const int64_t p = (int64_t)y * W + x;
                const int c = m < k ? m : k;
                for (int j = 0; j < k; ++j) {
                    out_ids[p * k + j] = j < c ? buf[j].g : -1;
                    out_w[p * k + j] = j < c ? buf[j].w : 0.0;
                }
                out_count[p] = c;
                double mg = s.margin;
                if (m > k) {
                    const double gap = (buf[k - 1].w - buf[k].w) / buf[k - 1].w;
                    if (gap < mg) mg = gap;
                }
                out_margin[p] = mg;
            }
        free(buf);
    }
}

/* Contribution skew (Sec. 1 "Rendering Inefficiency", Sec. 3.4 "Motivation"):
   every pixel walks its tile list under the plain rules of px_blend, the
   contributions Gamma_i alpha_i of the blended Gaussians are sorted in
   descending order, and out_m [H W] is the smallest number of them whose sum
   reaches frac times their total (0 for a pixel nothing blends into).  Also
   out_blended (contributions), out_walked (list entries the pixel examined:
   up to and including the one whose blending would have crossed T_stop, else
   the whole list), out_total (the sum), and out_margin = the smaller of the
   pixel's decision margin and the relative distance of frac * total from the
   two prefix sums that bracket it. */
void oc_contribution_skew(const oc_proj* proj, const int32_t* gid, const int64_t* ranges, int W, int H,
                          const oc_options* opt, double frac, int32_t* out_m, int32_t* out_blended,
                          int32_t* out_walked, double* out_total, double* out_margin, int nthreads) {
    int tw = opt->tile_w, th = opt->tile_h;
    int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int nt = nthreads > 0 ? nthreads : 1;
    (void)nt;
#ifdef _OPENMP
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t t = 0; t < ntiles; ++t) {
        int64_t cnt[OC_NCOUNT] = {0};
        int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
        int64_t start = ranges[2 * t], end = ranges[2 * t + 1];
        oc_contrib* buf = (oc_contrib*)malloc((size_t)(end > start ? end - start : 1) * sizeof(oc_contrib));
        for (int y = ty * th; y < ty * th + th && y < H; ++y)
            for (int x = tx * tw; x < tx * tw + tw && x < W; ++x) {
                px_state s;
                px_init(&s);
                int m = 0;
                int64_t walked = 0;
                for (int64_t i = start; i < end && !s.done; ++i) {
                    const double T = s.T;
                    const oc_proj* P = proj + gid[i];
                    ++walked;
                    if (px_blend(&s, P, opt, x + 0.5, y + 0.5, i - start, cnt)) {
                        buf[m].w = T * alpha_of_q(P, opt, quad_at(P, x + 0.5, y + 0.5));
                        buf[m].g = gid[i];
                        ++m;
                    }
                }
                qsort(buf, (size_t)m, sizeof(oc_contrib), contrib_cmp);
                double total = 0.0;
                for (int j = 0; j < m; ++j) total += buf[j].w;
                const double target = frac * total;
                int need = 0;
                double before = 0.0, upto = 0.0;
                if (m > 0) {
                    while (need < m && upto < target) {
                        before = upto;
                        upto += buf[need].w;
                        ++need;
                    }
                }
                const int64_t p = (int64_t)y * W + x;
                out_m[p] = need;
                out_blended[p] = m;
                out_walked[p] = (int32_t)walked;
                out_total[p] = total;
                double mg = s.margin;
                if (m > 0 && total > 0.0) {
                    const double above = (upto - target) / total, below = (target - before) / total;
                    if (above < mg) mg = above;
                    if (need > 1 && below < mg) mg = below;
                }
                out_margin[p] = mg;
            }
        free(buf);
    }
}
