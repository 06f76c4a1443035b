/*
 * raster.c -- FP64 oracle of the 3DGS image synthesis of Section II-A: each
 * Gaussian projected into a pinhole camera (Eq. 3 for the covariance, the
 * point projection pi for the mean) and the projections alpha-blended front
 * to back at each pixel in depth order (Eq. 4).
 *
 * TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU leg use it; the
 * product library never does.  It shares no code with the CUDA path.  The
 * 3D covariances come in from the query oracle (Eq. 2, already pinned).
 *
 * Readings of what the paper leaves open:
 *  - camera: x_c = R x_w + t, looking along +z; u = fx x/z + cx,
 *    v = fy y/z + cy; pixel (i, j) samples the image point (i + 0.5, j + 0.5);
 *  - J = d(u, v)/d(x_c) at the mean; Sigma' = J R Sigma R^T J^T + dilation I
 *    (a screen-space low-pass of `dilation` px^2 keeps Sigma' invertible for
 *    disks seen edge on); a Gaussian with det(Sigma') <= 0 is not drawn;
 *  - G2D(x) = exp(-(x - mu')^T Sigma'^-1 (x - mu') / 2), peak 1;
 *  - a Gaussian counts at a pixel when alpha G >= 1/255; alpha G is clamped
 *    at 0.99; blending stops before the Gaussian that would bring the
 *    transmittance below 1e-4;
 *  - Gaussians whose camera-frame depth is below near_plane are not drawn;
 *  - order: increasing camera-frame depth of the mean computed in float32 with
 *    the operations ((r20 x + r21 y) + r22 z) + t2 in that order (the same
 *    rounding as the device, so both take the same order), ties by index;
 *  - depth output: the blended Euclidean distance of the mean from the camera
 *    centre (the colour replaced by the splat's distance, Section II-A).
 *
 * For the comparison with FP32 results each pixel also reports
 *  - flags: bit 0 some alpha G within the decision band of 1/255, bit 1 the
 *    stopping test within its band of 1e-4, bit 2 two contributing Gaussians
 *    with the same float32 depth (their order is a tie);
 *  - cond = sum_k w_k (1 + q_k kappa_k), w_k = alpha_k G_k T_k the blending
 *    weight, q_k the quadratic form, kappa_k the condition number of Sigma'_k:
 *    the relative FP32 error of alpha_k G_k is at most a constant times
 *    u (1 + q_k kappa_k), and an output moves by at most 2 T_k per unit of
 *    alpha_k G_k, so the output error is bounded by a constant times u cond;
 *  - slack = sum over the Gaussians of bit 0 of 2 (1/255) (1 + band) T_k: the
 *    most an output can move when such a Gaussian is drawn on one side and
 *    not on the other (its weight plus its share of the later transmittance).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t width, height;
    double near_plane;
    double dilation;
    double bg[3];
    double band_rel;   /* fixed relative width of the decision bands */
    double band_cond;  /* plus band_cond * 2^-24 * (1 + q kappa) per Gaussian */
} orc_rdesc;

typedef struct {
    double u, v;          /* mu' */
    double ia, ib, ic;    /* Sigma'^-1 = [[ia, ib], [ib, ic]] */
    double kappa;         /* condition number of Sigma' */
    double dist;          /* |x_c| */
    float z32;            /* sort key */
    int64_t idx;
} proj_t;

static int cmp_proj(const void *pa, const void *pb) {
    const proj_t *a = (const proj_t *)pa, *b = (const proj_t *)pb;
    if (a->z32 < b->z32) return -1;
    if (a->z32 > b->z32) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* float32 depth of a mean, rounded after every operation in a fixed order */
static float depth32(const float *cam, const float *m) {
    volatile float p0 = cam[6] * m[0];
    volatile float p1 = cam[7] * m[1];
    volatile float s = p0 + p1;
    volatile float p2 = cam[8] * m[2];
    volatile float s2 = s + p2;
    volatile float z = s2 + cam[11];
    return z;
}

/* Project every Gaussian into camera `cam` (16 floats: R row-major, t, fx,
 * fy, cx, cy); returns the number drawn, sorted front to back. */
static int64_t project_all(int64_t n, const float *means, const double *sig, const float *cam,
                           const orc_rdesc *d, proj_t *out) {
    double R[9], t[3];
    for (int k = 0; k < 9; ++k) R[k] = cam[k];
    for (int k = 0; k < 3; ++k) t[k] = cam[9 + k];
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const float near32 = (float)d->near_plane;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        const float z32 = depth32(cam, means + 3 * i);
        if (!(z32 >= near32)) continue;
        double xw[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
        double xc[3];
        for (int a = 0; a < 3; ++a) xc[a] = R[3 * a] * xw[0] + R[3 * a + 1] * xw[1] + R[3 * a + 2] * xw[2] + t[a];
        const double z = xc[2];
        /* J (2x3) and M = J R (2x3) */
        double J[2][3] = {{fx / z, 0.0, -fx * xc[0] / (z * z)}, {0.0, fy / z, -fy * xc[1] / (z * z)}};
        double M[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = J[r][0] * R[c] + J[r][1] * R[3 + c] + J[r][2] * R[6 + c];
        const double *S = sig + 9 * i;
        double MS[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) MS[r][c] = M[r][0] * S[c] + M[r][1] * S[3 + c] + M[r][2] * S[6 + c];
        double a = MS[0][0] * M[0][0] + MS[0][1] * M[0][1] + MS[0][2] * M[0][2] + d->dilation;
        double b = MS[0][0] * M[1][0] + MS[0][1] * M[1][1] + MS[0][2] * M[1][2];
        double c = MS[1][0] * M[1][0] + MS[1][1] * M[1][1] + MS[1][2] * M[1][2] + d->dilation;
        const double det = a * c - b * b;
        if (!(det > 0.0)) continue;
        proj_t p;
        p.u = fx * xc[0] / z + cx;
        p.v = fy * xc[1] / z + cy;
        p.ia = c / det;
        p.ib = -b / det;
        p.ic = a / det;
        const double tr = 0.5 * (a + c), disc = sqrt(0.25 * (a - c) * (a - c) + b * b);
        p.kappa = (tr + disc) / (tr - disc);
        p.dist = sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
        p.z32 = z32;
        p.idx = i;
        out[m++] = p;
    }
    qsort(out, (size_t)m, sizeof(proj_t), cmp_proj);
    return m;
}

static void blend_pixel(const proj_t *P, int64_t m, const double *opacity, const double *color,
                        const orc_rdesc *d, int32_t x, int32_t y, double *rgb, double *depth, double *alpha,
                        int32_t *ncontrib, int32_t *flags, double *cond, double *slack) {
    const double u = x + 0.5, v = y + 0.5;
    const double thr = 1.0 / 255.0, t_stop = 1e-4, u32 = ldexp(1.0, -24);
    double T = 1.0, c[3] = {0, 0, 0}, dd = 0.0, cd = 0.0, tband = 0.0, sl = 0.0;
    int32_t K = 0, fl = 0;
    float last_z = 0.f;
    int have_last = 0;
    for (int64_t k = 0; k < m; ++k) {
        const proj_t *p = &P[k];
        const double dx = u - p->u, dy = v - p->v;
        const double q = p->ia * dx * dx + 2.0 * p->ib * dx * dy + p->ic * dy * dy;
        const double A = opacity[p->idx] * exp(-0.5 * q);
        const double eps = d->band_cond * u32 * (1.0 + q * p->kappa);
        const double band = d->band_rel + eps;
        if (fabs(A - thr) <= band * thr) {
            fl |= 1;
            sl += 2.0 * thr * (1.0 + band) * T;
        }
        if (A < thr) continue;
        const double a = A < 0.99 ? A : 0.99;
        const double Tn = T * (1.0 - a);
        /* relative error of Tn: the errors of the factors so far */
        const double tb = tband + (A < 0.99 ? eps * a / (1.0 - a) : 0.0) + 4.0 * u32;
        if (fabs(Tn - t_stop) <= (d->band_rel + tb) * t_stop) fl |= 2;
        if (Tn < t_stop) break;
        if (have_last && p->z32 == last_z) fl |= 4;
        last_z = p->z32;
        have_last = 1;
        const double w = a * T;
        for (int ch = 0; ch < 3; ++ch) c[ch] += w * color[3 * p->idx + ch];
        dd += w * p->dist;
        cd += w * (1.0 + q * p->kappa);
        T = Tn;
        tband = tb;
        ++K;
    }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = c[ch] + T * d->bg[ch];
    *depth = dd;
    *alpha = 1.0 - T;
    *ncontrib = K;
    *flags = fl;
    *cond = cd;
    *slack = sl;
}

/* Render the listed pixels (npix triples: view, x, y). */
int orc_render_pixels(int64_t n, const float *means, const double *sig, const double *opacity,
                      const double *color, int32_t nviews, const float *cams, const orc_rdesc *d,
                      int64_t npix, const int32_t *pix, double *rgb, double *depth, double *alpha,
                      int32_t *ncontrib, int32_t *flags, double *cond, double *slack) {
    proj_t *P = (proj_t *)malloc(sizeof(proj_t) * (size_t)(n > 0 ? n : 1));
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npix > 0 ? npix : 1));
    if (!P || !list) {
        free(P);
        free(list);
        return -1;
    }
    for (int32_t vw = 0; vw < nviews; ++vw) {
        int64_t cnt = 0;
        for (int64_t i = 0; i < npix; ++i)
            if (pix[3 * i] == vw) list[cnt++] = i;
        if (cnt == 0) continue;
        const int64_t m = project_all(n, means, sig, cams + 16 * (size_t)vw, d, P);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (int64_t j = 0; j < cnt; ++j) {
            const int64_t i = list[j];
            blend_pixel(P, m, opacity, color, d, pix[3 * i + 1], pix[3 * i + 2], rgb + 3 * i, depth + i, alpha + i,
                        ncontrib + i, flags + i, cond + i, slack + i);
        }
    }
    free(P);
    free(list);
    return 0;
}
