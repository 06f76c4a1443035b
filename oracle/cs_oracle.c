/*
 * cs_oracle.c -- FP64 brute-force CPU oracle for the CollisionSplatting
 * conservative collision metric.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every query is evaluated against every Gaussian (no cull, no blocking, no
 * reordering), in double precision, from the single-precision inputs.  The
 * steps follow the paper's Section II in its own order:
 *
 *   Eq. 2   Sigma_i = R(q_i) S_i S_i^T R(q_i)^T,  S_i = diag(scale_i)
 *   Eq. 6   A_j = R_E P_j R_E^T,  P_j = diag(1/a^2, 1/b^2, 1/c^2)
 *           (a sphere of radius r is a = b = c = r, R_E = I)
 *   Eq. 5   s^2_ij = (mu_i - mu_j)^T A_j (mu_i - mu_j)
 *   Eq. 7   sigma^2_ij = g Sigma_i g^T,  g = d s^2 / dX at X = mu_i
 *   Eq. 8   st^2_ij = max(0, s^2_ij - n_sigma sqrt(sigma^2_ij))
 *   Eq. 11  dc_ij = d_max exp(-gamma max(st^2_ij - s_min, 0))
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - neighbour set N_j = { i kept : st^2_ij <= S_cut },
 *     S_cut = s_min + ln(1/eps)/gamma, so every dropped cost term is below
 *     eps * d_max (Section II-D averages Eq. 11 over "neighbouring splats"
 *     without giving the radius);
 *   - mean cost = (sum over N_j of dc) / |N_j|, 0 when N_j is empty;
 *   - collision count = #{ i in N_j : st^2 < 1 } (Section II-E counts
 *     s^2 < 1, and the Eq. 8 metric is the one used for checking);
 *   - min over N_j of st^2 (+inf when empty);
 *   - softmin_tau = -tau ln sum_{N_j} exp(-st^2/tau) (+inf when empty),
 *     the "recursive softmin" of Section II-B written in closed form;
 *   - floater filter (Section II-C): drop a Gaussian when its opacity is below
 *     opacity_min AND its largest scale exceeds extent_max;
 *   - quaternions are (w, x, y, z) and are normalised here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double gamma;       /* Eq. 11 decay */
    double d_max;       /* Eq. 11 maximum cost per splat */
    double s_min;       /* Eq. 11 minimum allowed scaling factor */
    double eps;         /* truncation bound for the neighbour set */
    double tau;         /* softmin temperature */
    int64_t k_thr;      /* collide iff count_in > k_thr (Section II-E) */
    double opacity_min; /* floater filter (Section II-C) */
    double extent_max;
    int32_t use_filter;
    int32_t nthreads;   /* <= 0: OpenMP default */
    double band;        /* width of the reporting bands below (<= 0: 1e-5) */
    int32_t exact_variance; /* 1: the exact variance of Eq. 5 under the Gaussian instead of
                               the linearisation of Eq. 7 (adds 2 tr((A Sigma)^2)) */
} orc_params;

/* Per-query outputs.  Any pointer may be NULL. */
typedef struct {
    double *sum_cost;   /* sum of dc over N_j */
    double *mean_cost;  /* sum / |N_j| (0 when empty) */
    int64_t *count_nbr; /* |N_j| */
    int64_t *count_in;  /* #{i in N_j: st^2 < 1} */
    uint8_t *collide;   /* count_in > k_thr */
    double *min_s2;     /* min over N_j of st^2 (+inf if empty) */
    double *softmin;    /* -tau ln sum exp(-st^2/tau) (+inf if empty) */
    /* diagnostics used by the parity tests */
    int64_t *band_cut;  /* pairs with |st^2 - S_cut| <= band S_cut (band = 1e-5 by default) */
    int64_t *band_in;   /* pairs with |st^2 - 1| <= band */
    double *cond;       /* max over N_j of s^2 + n_sigma sqrt(sigma^2) */
    double *min_cond;   /* s^2 + n_sigma sqrt(sigma^2) of the argmin pair */
    int64_t *band_kink; /* pairs near a kink of the gradient: |st^2 - s_min| <= band or
                           the Eq. 8 clamp within band of its switching point */
    double *cond_cost;  /* max of s^2 + n_sigma sqrt(sigma^2) over the pairs of N_j whose
                           Eq. 11 cost can feel it: st^2 >= s_min - band (s^2 + n sqrt(sigma^2));
                           below s_min the cost is flat (d_max), so rounding there is harmless */
} orc_outputs;

/* ---- geometry -------------------------------------------------------- */

/* Rotation matrix of the unit quaternion (w, x, y, z) after normalising. */
static void rot_from_quat(const float *qf, double R[3][3])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    double nrm = sqrt(w * w + x * x + y * y + z * z);
    if (nrm == 0.0) { w = 1.0; x = y = z = 0.0; nrm = 1.0; }
    w /= nrm; x /= nrm; y /= nrm; z /= nrm;
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

/* out = R D R^T with D = diag(dg). */
static void rotate_diag(const double R[3][3], const double dg[3], double out[3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += R[a][k] * dg[k] * R[b][k];
            out[a][b] = s;
        }
}

/* Eq. 2: Sigma = R S S^T R^T with S = diag(scale). */
static void gaussian_covariance(const float *scale, const float *quat, double Sig[3][3])
{
    double R[3][3];
    rot_from_quat(quat, R);
    double s2[3] = {(double)scale[0] * scale[0], (double)scale[1] * scale[1],
                    (double)scale[2] * scale[2]};
    rotate_diag(R, s2, Sig);
}

/* Eq. 6: centre and shape matrix A of a robot primitive.
 * type 0: sphere   {cx, cy, cz, r}
 * type 1: ellipsoid {cx, cy, cz, qw, qx, qy, qz, a, b, c}            */
static int robot_primitive(int type, const float *p, double c[3], double A[3][3])
{
    c[0] = p[0]; c[1] = p[1]; c[2] = p[2];
    if (type == 0) {
        double r = p[3];
        if (!(r > 0.0)) return -1;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] = (a == b) ? 1.0 / (r * r) : 0.0;
        return 0;
    }
    if (type == 1) {
        double ax = p[7], bx = p[8], cx = p[9];
        if (!(ax > 0.0) || !(bx > 0.0) || !(cx > 0.0)) return -1;
        double R[3][3];
        rot_from_quat(p + 3, R);
        double P[3] = {1.0 / (ax * ax), 1.0 / (bx * bx), 1.0 / (cx * cx)};
        rotate_diag(R, P, A);
        return 0;
    }
    return -1;
}

static int keep_gaussian(const orc_params *prm, const float *scale, const float *opacity, int64_t i)
{
    if (!prm->use_filter || opacity == NULL) return 1;
    double smax = fmax(fmax(scale[0], scale[1]), scale[2]);
    return !(opacity[i] < prm->opacity_min && smax > prm->extent_max);
}

/* Eq. 5, Eq. 7, Eq. 8 for one (Gaussian, primitive) pair. */
typedef struct {
    double s2;    /* Eq. 5 */
    double var;   /* Eq. 7 */
    double st2;   /* Eq. 8 */
    double raw;   /* s2 - n_sigma sqrt(var), before the clamp */
} pair_terms;

/* tr((A Sigma)^2) = sum_ab (A Sigma)_ab (A Sigma)_ba: for X ~ N(mu, Sigma) the
 * quadratic form s^2(X) = (X - c)^T A (X - c) has variance
 * 4 d^T A Sigma A d + 2 tr((A Sigma)^2); Eq. 7 keeps the first term only. */
static double trace_asas(const double A[3][3], const double Sig[3][3])
{
    double M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = A[a][0] * Sig[0][b] + A[a][1] * Sig[1][b] + A[a][2] * Sig[2][b];
    double t = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) t += M[a][b] * M[b][a];
    return t;
}

static pair_terms evaluate_pair(const double mu[3], const double Sig[3][3], const double c[3],
                                const double A[3][3], double nsigma, int exact)
{
    pair_terms t;
    double d[3] = {mu[0] - c[0], mu[1] - c[1], mu[2] - c[2]};
    /* Eq. 5 */
    double Ad[3];
    for (int a = 0; a < 3; ++a) Ad[a] = A[a][0] * d[0] + A[a][1] * d[1] + A[a][2] * d[2];
    t.s2 = d[0] * Ad[0] + d[1] * Ad[1] + d[2] * Ad[2];
    /* Eq. 7: the gradient of Eq. 5 with respect to X at X = mu is 2 A d
     * (A symmetric), and the variance is that row vector sandwiching Sigma. */
    double g[3] = {2.0 * Ad[0], 2.0 * Ad[1], 2.0 * Ad[2]};
    double Sg[3];
    for (int a = 0; a < 3; ++a) Sg[a] = Sig[a][0] * g[0] + Sig[a][1] * g[1] + Sig[a][2] * g[2];
    t.var = g[0] * Sg[0] + g[1] * Sg[1] + g[2] * Sg[2];
    if (exact) t.var += 2.0 * trace_asas(A, Sig);
    if (t.var < 0.0) t.var = 0.0; /* Sigma is PSD; guards round-off only */
    /* Eq. 8 */
    t.raw = t.s2 - nsigma * sqrt(t.var);
    t.st2 = t.raw > 0.0 ? t.raw : 0.0;
    return t;
}

/* Eq. 11 */
static double pair_cost(const orc_params *prm, double st2)
{
    double e = st2 - prm->s_min;
    if (e < 0.0) e = 0.0;
    return prm->d_max * exp(-prm->gamma * e);
}

static double cutoff(const orc_params *prm)
{
    return prm->s_min + log(1.0 / prm->eps) / prm->gamma;
}

/* ---- public entry points -------------------------------------------- */

/* Terms of a single pair: out = {s2, sigma2, st2, dc, raw}. */
int orc_pair(const float *mean, const float *scale, const float *quat, int prim_type,
             const float *prim, double nsigma, const orc_params *prm, double *out)
{
    double Sig[3][3], c[3], A[3][3];
    gaussian_covariance(scale, quat, Sig);
    if (robot_primitive(prim_type, prim, c, A) != 0) return -1;
    double mu[3] = {mean[0], mean[1], mean[2]};
    pair_terms t = evaluate_pair(mu, Sig, c, A, nsigma, prm->exact_variance);
    out[0] = t.s2;
    out[1] = t.var;
    out[2] = t.st2;
    out[3] = pair_cost(prm, t.st2);
    out[4] = t.raw;
    return 0;
}

/* Covariance of every Gaussian (Eq. 2), row-major 3x3 per Gaussian, and the
 * floater-filter decision. */
int orc_covariances(int64_t n, const float *scales, const float *quats, const float *opacity,
                    const orc_params *prm, double *sig_out /* [n*9] */, uint8_t *keep_out)
{
    for (int64_t i = 0; i < n; ++i) {
        double Sig[3][3];
        gaussian_covariance(scales + 3 * i, quats + 4 * i, Sig);
        if (sig_out)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) sig_out[9 * i + 3 * a + b] = Sig[a][b];
        if (keep_out) keep_out[i] = (uint8_t)keep_gaussian(prm, scales + 3 * i, opacity, i);
    }
    return 0;
}

/* Every query against every kept Gaussian.  nsigma has Q entries. */
int orc_query(int64_t n, const float *means, const float *scales, const float *quats,
              const float *opacity, int prim_type, const float *prims, int64_t Q,
              const double *nsigma, const orc_params *prm, orc_outputs *out)
{
    const int stride = prim_type == 0 ? 4 : 10;
    const double S_cut = cutoff(prm);
    const double band = prm->band > 0.0 ? prm->band : 1e-5;
    double *Sig = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    uint8_t *keep = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!Sig || !keep) { free(Sig); free(keep); return -2; }
    orc_covariances(n, scales, quats, opacity, prm, Sig, keep);
    int bad = 0;

#ifdef _OPENMP
    int nt = prm->nthreads > 0 ? prm->nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : bad)
#endif
    for (int64_t j = 0; j < Q; ++j) {
        double c[3], A[3][3];
        if (robot_primitive(prim_type, prims + (size_t)stride * j, c, A) != 0) { bad += 1; continue; }
        double ns = nsigma[j];
        double sum = 0.0, mn = INFINITY, mn_cond = 0.0, cond = 0.0, ccost = 0.0;
        int64_t cnt = 0, cin = 0, bcut = 0, bin = 0, bkink = 0;
        /* softmin: shift by the running minimum so the sum stays in range */
        double sm_m = INFINITY, sm_acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (!keep[i]) continue;
            const double *S = Sig + 9 * i;
            double Sg[3][3] = {{S[0], S[1], S[2]}, {S[3], S[4], S[5]}, {S[6], S[7], S[8]}};
            double mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
            pair_terms t = evaluate_pair(mu, Sg, c, A, ns, prm->exact_variance);
            if (fabs(t.st2 - S_cut) <= band * S_cut) ++bcut;
            if (fabs(t.st2 - 1.0) <= band) ++bin;
            if (t.st2 <= S_cut * (1.0 + band) &&
                (fabs(t.st2 - prm->s_min) <= band * fmax(1.0, fabs(prm->s_min)) ||
                 fabs(t.raw) <= band * (t.s2 + ns * sqrt(t.var))))
                ++bkink;
            if (!(t.st2 <= S_cut)) continue;
            ++cnt;
            sum += pair_cost(prm, t.st2);
            if (t.st2 < 1.0) ++cin;
            double cnd = t.s2 + ns * sqrt(t.var);
            if (cnd > cond) cond = cnd;
            if (t.st2 >= prm->s_min - band * cnd && cnd > ccost) ccost = cnd;
            if (t.st2 < mn) { mn = t.st2; mn_cond = cnd; }
            double x = t.st2 / prm->tau;
            if (x < sm_m) { sm_acc = sm_acc * exp(x - sm_m) + 1.0; sm_m = x; }
            else sm_acc += exp(sm_m - x);
        }
        if (out->sum_cost) out->sum_cost[j] = sum;
        if (out->mean_cost) out->mean_cost[j] = cnt > 0 ? sum / (double)cnt : 0.0;
        if (out->count_nbr) out->count_nbr[j] = cnt;
        if (out->count_in) out->count_in[j] = cin;
        if (out->collide) out->collide[j] = (uint8_t)(cin > prm->k_thr);
        if (out->min_s2) out->min_s2[j] = mn;
        if (out->softmin) out->softmin[j] = cnt > 0 ? prm->tau * (sm_m - log(sm_acc)) : INFINITY;
        if (out->band_cut) out->band_cut[j] = bcut;
        if (out->band_in) out->band_in[j] = bin;
        if (out->cond) out->cond[j] = cond;
        if (out->min_cond) out->min_cond[j] = mn_cond;
        if (out->band_kink) out->band_kink[j] = bkink;
        if (out->cond_cost) out->cond_cost[j] = ccost;
    }
    free(Sig);
    free(keep);
    return bad ? -1 : 0;
}

/* ---- analytic gradient ---------------------------------------------- */

/* d st^2 / d c for one pair (zero where the Eq. 8 clamp is active or the
 * variance vanishes).  With d = mu - c, w = A d:
 *   d s^2 / d c            = -2 w
 *   sqrt(sigma^2)          = 2 sqrt(w^T Sigma w)
 *   d sqrt(sigma^2) / d c  = -2 A Sigma w / sqrt(w^T Sigma w)               */
static void st2_grad(const double mu[3], const double Sig[3][3], const double c[3],
                     const double A[3][3], double nsigma, int exact, double *st2_out, double gvec[3],
                     double *gmag)
{
    double d[3] = {mu[0] - c[0], mu[1] - c[1], mu[2] - c[2]};
    double w[3];
    for (int a = 0; a < 3; ++a) w[a] = A[a][0] * d[0] + A[a][1] * d[1] + A[a][2] * d[2];
    double s2 = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
    double Sw[3];
    for (int a = 0; a < 3; ++a) Sw[a] = Sig[a][0] * w[0] + Sig[a][1] * w[1] + Sig[a][2] * w[2];
    double wSw = w[0] * Sw[0] + w[1] * Sw[1] + w[2] * Sw[2];
    if (wSw < 0.0) wSw = 0.0;
    /* sqrt(sigma^2) / 2; the exact variance adds tr((A Sigma)^2) / 2 under the
     * root, a term that does not depend on c */
    double root = sqrt(wSw + (exact ? 0.5 * trace_asas(A, Sig) : 0.0));
    double raw = s2 - nsigma * 2.0 * root;
    *st2_out = raw > 0.0 ? raw : 0.0;
    for (int a = 0; a < 3; ++a) gvec[a] = 0.0;
    *gmag = 0.0;
    if (!(raw > 0.0)) return;
    double ASw[3];
    for (int a = 0; a < 3; ++a) ASw[a] = A[a][0] * Sw[0] + A[a][1] * Sw[1] + A[a][2] * Sw[2];
    double m1 = 0.0, m2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double p1 = -2.0 * w[a], p2 = root > 0.0 ? nsigma * 2.0 * ASw[a] / root : 0.0;
        gvec[a] = p1 + p2;
        m1 += p1 * p1;
        m2 += p2 * p2;
    }
    /* size of the two parts, which may cancel: the conditioning of the term */
    *gmag = sqrt(m1) + sqrt(m2);
}

/* Gradient of the per-query metric with respect to the primitive centre.
 * mode 0: mean cost, 1: summed cost, 2: min st^2, 3: softmin st^2.
 * grad_out: [Q] upstream gradient (NULL = ones).  grad: [Q*3]. */
int orc_grad(int64_t n, const float *means, const float *scales, const float *quats,
             const float *opacity, int prim_type, const float *prims, int64_t Q,
             const double *nsigma, const orc_params *prm, int mode, const double *grad_out,
             double *grad, double *gscale)
{
    const int stride = prim_type == 0 ? 4 : 10;
    const double S_cut = cutoff(prm);
    double *Sig = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    uint8_t *keep = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!Sig || !keep) { free(Sig); free(keep); return -2; }
    orc_covariances(n, scales, quats, opacity, prm, Sig, keep);
    int bad = 0;

#ifdef _OPENMP
    int nt = prm->nthreads > 0 ? prm->nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : bad)
#endif
    for (int64_t j = 0; j < Q; ++j) {
        double c[3], A[3][3];
        grad[3 * j] = grad[3 * j + 1] = grad[3 * j + 2] = 0.0;
        if (gscale) gscale[j] = 0.0;
        if (robot_primitive(prim_type, prims + (size_t)stride * j, c, A) != 0) { bad += 1; continue; }
        double ns = nsigma[j];
        double acc[3] = {0, 0, 0};
        double mag = 0.0; /* sum of the norms of the summed terms */
        int64_t cnt = 0;
        double best = INFINITY, best_g[3] = {0, 0, 0};
        /* softmin: weights exp(-st2/tau) / sum, accumulated with a running
         * shift (the minimum seen so far). */
        double sm_m = INFINITY, sm_acc = 0.0, sm_g[3] = {0, 0, 0};
        for (int64_t i = 0; i < n; ++i) {
            if (!keep[i]) continue;
            const double *S = Sig + 9 * i;
            double Sg[3][3] = {{S[0], S[1], S[2]}, {S[3], S[4], S[5]}, {S[6], S[7], S[8]}};
            double mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
            double st2, g[3], gm;
            st2_grad(mu, Sg, c, A, ns, prm->exact_variance, &st2, g, &gm);
            if (!(st2 <= S_cut)) continue;
            ++cnt;
            if (mode == 0 || mode == 1) {
                /* Eq. 11: flat (= d_max) below s_min, exponential above */
                if (st2 > prm->s_min) {
                    double dc = pair_cost(prm, st2);
                    for (int a = 0; a < 3; ++a) acc[a] += -prm->gamma * dc * g[a];
                    mag += prm->gamma * dc * gm;
                }
            } else if (mode == 2) {
                if (st2 < best) {
                    best = st2; best_g[0] = g[0]; best_g[1] = g[1]; best_g[2] = g[2];
                    mag = gm;
                }
            } else {
                double x = st2 / prm->tau;
                if (x < sm_m) {
                    double r = exp(x - sm_m);
                    sm_acc = sm_acc * r + 1.0;
                    for (int a = 0; a < 3; ++a) sm_g[a] = sm_g[a] * r + g[a];
                    mag = mag * r + gm;
                    sm_m = x;
                } else {
                    double e = exp(sm_m - x);
                    sm_acc += e;
                    for (int a = 0; a < 3; ++a) sm_g[a] += e * g[a];
                    mag += e * gm;
                }
            }
        }
        double up = grad_out ? grad_out[j] : 1.0;
        double out[3] = {0, 0, 0};
        if (mode == 0) {
            if (cnt > 0) for (int a = 0; a < 3; ++a) out[a] = acc[a] / (double)cnt;
            if (cnt > 0) mag /= (double)cnt;
        } else if (mode == 1) {
            for (int a = 0; a < 3; ++a) out[a] = acc[a];
        } else if (mode == 2) {
            for (int a = 0; a < 3; ++a) out[a] = best_g[a];
        } else if (cnt > 0) {
            for (int a = 0; a < 3; ++a) out[a] = sm_g[a] / sm_acc;
            mag /= sm_acc;
        }
        for (int a = 0; a < 3; ++a) grad[3 * j + a] = up * out[a];
        if (gscale) gscale[j] = fabs(up) * mag;
    }
    free(Sig);
    free(keep);
    return bad ? -1 : 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
