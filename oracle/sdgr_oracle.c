/*
 * sdgr_oracle.c -- FP64 CPU oracle for the SAR Differentiable Gaussian
 * Rasterizer (SDGR) of SAR-GS (arXiv 2506.21633).
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the tests, by the smoke check
 * and by the CPU-baseline leg of the benchmark; the product path never links
 * or calls it.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * Plain, slow and brute force: every ray of the computation plane and every
 * pixel of the imaging plane is evaluated against every Gaussian, in double
 * precision, following the paper's steps in its order:
 *   Section II-A-1 (Mapping and Projection Algorithm): the world->radar
 *     transform W = [R_r T_r] (eqs. "transformation matrix", R_r), the 3D
 *     Gaussian (eq. G(x)), the projected covariance (eq. Sigmaprime) and the
 *     projection matrices P_C (eq. x_C) and P_I (eq. x_i);
 *   Section II-A-2 (scattering intensities, eq. I_i with delta^{p,q});
 *   Section II-A-3 (imaging, eq. S_{n,m});
 *   Section II-B (gradients of the imaging process, of the intensity
 *     computation and of the Gaussian parameters), derived afresh by the
 *     chain rule because the printed forms drop a factor 1/2 and the inverse.
 *
 * Readings of passages that are garbled or silent (each is also listed in the
 * design notes):
 *   R1  theta is the grazing angle and enters R_r literally.
 *   R2  x_r = R_r (x_w - c) + T_r, T_r = (0, 0, R0), R0 = h / sin(theta),
 *       h = 10 000 m (Section III-B-3); the projections are orthographic; the
 *       slant-range row of P_I uses 2/(dR N_R) (the printed tan(theta) would
 *       not cancel the -2h/(dR N_R sin(theta)) offset).  NDC -> pixel uses
 *       pixel = (ndc + 1) N / 2 - 1/2, i.e. pixel centres at integers.
 *   R3  computation plane = (x_r, y_r) with N_R x N_A cells of dA x dR tan(theta)
 *       and one ray per cell centre; imaging plane = (x_r, z_r - R0).
 *   R4  Sigma' = J (R_r Sigma R_r^T) J^T, J = the 2x3 Jacobian of the pixel
 *       coordinates with respect to x_r.
 *   R5  alpha_i = o_i exp(-delta/2) with o_i = sigmoid(opacity logit) standing
 *       for 1 - exp(-(k_e+ + k_e-) ...) (the two extinctions only enter as a
 *       sum); T_i = prod_{j<i} (1 - alpha_j); I_i = P_i sum_rays alpha_i T_i.
 *       Variant (alpha_mode 1, Beer-Lambert): the extinction exponent of the
 *       paper's attenuation factor is an optical depth tau_i times the
 *       Gaussian's profile along the ray, alpha_i = 1 - exp(-tau_i
 *       exp(-delta/2)), with tau_i = softplus(opacity logit) =
 *       -log(1 - sigmoid(logit)): the peak opacity equals o_i of the default.
 *   R6  beta = c_i exp(-delta/2), delta = d^T Sigma'^{-1} d, c_i = 1 / (2 pi
 *       sqrt(det Sigma'_I)) (energy mode) or 1 (peak mode).
 *   R7  contributions with delta > K^2 are zero on both planes (K <= 0: no
 *       cutoff).
 *   R8  eps (px^2) is added to both 2D covariances.
 *   R9  one depth order per view: ascending fl32(z_r - R0) (the float32
 *       rounding of the slant-range offset, the precision the GPU kernel
 *       decides the order in), ties broken by Gaussian index.
 *   R10 rays stop only when T_min > 0 and T < T_min (default: never).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -o liboracle.so sdgr_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ALTITUDE 10000.0 /* radar altitude h (m), Section III-B-3 */
#define ORC_PI 3.14159265358979323846

typedef struct {
    double phi, theta; /* radar azimuth angle, grazing angle (rad) */
    double dA, dR;     /* azimuth and slant-range resolution (m) */
    int32_t NA, NR;    /* image columns (azimuth) and rows (slant range) */
    int32_t pad0, pad1;
    double center[3];  /* world point the beam is centred on (m) */
} orc_view;

typedef struct {
    double K;          /* cutoff radius in standard deviations, <= 0: none */
    double eps;        /* dilation added to both 2D covariances (px^2) */
    double T_min;      /* ray stops once T < T_min (0: never) */
    int32_t norm_mode; /* 0: energy-normalised beta, 1: peak (c_i = 1) */
    int32_t sh_degree; /* 0..3: degree of the view-dependent scattering */
    int32_t alpha_mode; /* 0: alpha = o G; 1: alpha = 1 - exp(-tau G) (R5) */
    int32_t pad;
    const double *sh;  /* [N][16] SH coefficients of degrees 1..3 (NULL: none) */
    double *dsh;       /* [N][16] out: dL/dsh (orc_grad only; NULL: not wanted) */
    double *duI;       /* [V][N][2] out: dL/du_I per view (orc_grad only; NULL: not wanted) */
} orc_cfg;

/* View-dependent scattering (the phase function of Section II-B-3, "from the
 * centre and the spherical harmonic coefficients").  With plane-wave
 * geometry the direction is the same for every Gaussian of a view: the unit
 * vector d from the scene toward the radar (the negative line of sight).
 * P_i(view) = P_i + sum_{l=1..degree} sum_m sh_i[l^2 - 1 + l + m] Y_lm(d),
 * with the real orthonormal spherical harmonics (no Condon-Shortley phase):
 *   l=1: c1 (y, z, x),                           c1 = sqrt(3/(4 pi))
 *   l=2: c2 xy, c2 yz, c20 (3z^2 - 1), c2 xz, c22 (x^2 - y^2)
 *        c2 = sqrt(15/pi)/2, c20 = sqrt(5/pi)/4, c22 = sqrt(15/pi)/4
 *   l=3: c33 y(3x^2 - y^2), c32 xyz, c31 y(5z^2 - 1), c30 z(5z^2 - 3),
 *        c31 x(5z^2 - 1), c32/2 z(x^2 - y^2), c33 x(x^2 - 3y^2)
 *        c33 = sqrt(35/(2 pi))/4, c32 = sqrt(105/pi)/2, c31 = sqrt(21/(2 pi))/4,
 *        c30 = sqrt(7/pi)/4 */
static void sh_basis(const double d[3], double Y[15]) {
    const double pi = ORC_PI;
    const double x = d[0], y = d[1], z = d[2];
    const double c1 = sqrt(3.0 / (4.0 * pi));
    const double c2 = sqrt(15.0 / pi) / 2.0, c20 = sqrt(5.0 / pi) / 4.0, c22 = sqrt(15.0 / pi) / 4.0;
    const double c33 = sqrt(35.0 / (2.0 * pi)) / 4.0, c32 = sqrt(105.0 / pi) / 2.0;
    const double c31 = sqrt(21.0 / (2.0 * pi)) / 4.0, c30 = sqrt(7.0 / pi) / 4.0;
    Y[0] = c1 * y; Y[1] = c1 * z; Y[2] = c1 * x;
    Y[3] = c2 * x * y; Y[4] = c2 * y * z; Y[5] = c20 * (3 * z * z - 1); Y[6] = c2 * x * z; Y[7] = c22 * (x * x - y * y);
    Y[8] = c33 * y * (3 * x * x - y * y); Y[9] = c32 * x * y * z; Y[10] = c31 * y * (5 * z * z - 1);
    Y[11] = c30 * z * (5 * z * z - 3); Y[12] = c31 * x * (5 * z * z - 1); Y[13] = 0.5 * c32 * z * (x * x - y * y);
    Y[14] = c33 * x * (x * x - 3 * y * y);
}

static int sh_count(int degree) { return degree <= 0 ? 0 : (degree >= 3 ? 15 : (degree == 1 ? 3 : 8)); }

/* SH basis of the direction toward the radar of a view, for tests. */
int orc_sh_basis(const double *d, double *Y) {
    sh_basis(d, Y);
    return 0;
}

typedef struct {
    /* activations (C1) */
    double s[3], qhat[4], qlen, o, P;
    double tau;       /* optical depth softplus(logit) (alpha_mode 1) */
    double R[3][3];   /* rotation of the Gaussian */
    double Sig[3][3]; /* 3D covariance Sigma = R diag(s^2) R^T */
    /* radar frame (eqs. W, R_r, x_r) */
    double Rr[3][3];
    double xr[3];
    double R0;
    double Sr[3][3]; /* R_r Sigma R_r^T */
    double key;      /* depth key, reading R9 */
    /* plane 0 = computation plane (P_C), plane 1 = imaging plane (P_I) */
    double u[2][2];      /* pixel coordinates (column, row) */
    double J[2][2][3];   /* d pixel / d x_r */
    double S2[2][2][2];  /* 2D covariance incl. dilation */
    double C2[2][2][2];  /* its inverse */
    double det[2];
    double cnorm;        /* imaging-plane normaliser c_i */
    double Ysh[15];      /* SH basis of this view's direction (zeros past the degree) */
    int bb[2][4];        /* inclusive pixel box x0, x1, y0, y1 (culled mode) */
} orc_gauss;

static int g_threads = 0;

int orc_set_threads(int n) {
    g_threads = n;
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int n_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int thread_id(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

static double cutoff2(const orc_cfg *cfg) { return cfg->K > 0.0 ? cfg->K * cfg->K : INFINITY; }

/* World -> radar rotation R_r (Section II-A-1, eq. R_r): rows are the azimuth
 * axis, the in-plane "elevation" axis and the line of sight. */
static void radar_rotation(double phi, double theta, double Rr[3][3]) {
    double sp = sin(phi), cp = cos(phi), st = sin(theta), ct = cos(theta);
    Rr[0][0] = -sp;      Rr[0][1] = -cp;     Rr[0][2] = 0.0;
    Rr[1][0] = -st * cp; Rr[1][1] = st * sp; Rr[1][2] = ct;
    Rr[2][0] = -ct * cp; Rr[2][1] = ct * sp; Rr[2][2] = -st;
}

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static double mahal(const double C[2][2], double dx, double dy) {
    return C[0][0] * dx * dx + (C[0][1] + C[1][0]) * dx * dy + C[1][1] * dy * dy;
}

/* Mapping and Projection Algorithm for one Gaussian and one view. */
static void project(const double *p, const orc_view *v, const orc_cfg *cfg, orc_gauss *g, const double *sh_row) {
    int a, b, k;
    /* activations */
    for (k = 0; k < 3; ++k) g->s[k] = exp(p[4 + k]);
    g->qlen = sqrt(p[8] * p[8] + p[9] * p[9] + p[10] * p[10] + p[11] * p[11]);
    for (k = 0; k < 4; ++k) g->qhat[k] = p[8 + k] / g->qlen;
    g->o = 1.0 / (1.0 + exp(-p[3]));
    g->tau = p[3] > 0.0 ? p[3] + log1p(exp(-p[3])) : log1p(exp(p[3]));
    g->P = p[7];
    quat_to_rot(g->qhat, g->R);
    memset(g->Ysh, 0, sizeof(g->Ysh));
    if (sh_row && cfg->sh_degree > 0) {
        double st = sin(v->theta), ct = cos(v->theta), sp = sin(v->phi), cp = cos(v->phi);
        const double d[3] = {ct * cp, -ct * sp, st}; /* toward the radar */
        int k, nk = sh_count(cfg->sh_degree);
        sh_basis(d, g->Ysh);
        for (k = nk; k < 15; ++k) g->Ysh[k] = 0.0;
        for (k = 0; k < nk; ++k) g->P += sh_row[k] * g->Ysh[k];
    }
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (k = 0; k < 3; ++k) acc += g->R[a][k] * g->s[k] * g->s[k] * g->R[b][k];
            g->Sig[a][b] = acc;
        }
    /* x_r = R_r (x_w - c) + T_r  (reading R2) */
    radar_rotation(v->phi, v->theta, g->Rr);
    g->R0 = ORC_ALTITUDE / sin(v->theta);
    double d[3] = {p[0] - v->center[0], p[1] - v->center[1], p[2] - v->center[2]};
    for (a = 0; a < 3; ++a) g->xr[a] = g->Rr[a][0] * d[0] + g->Rr[a][1] * d[1] + g->Rr[a][2] * d[2];
    g->xr[2] += g->R0;
    /* Sigma_r = R_r Sigma R_r^T */
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            double acc = 0.0;
            int i, j;
            for (i = 0; i < 3; ++i)
                for (j = 0; j < 3; ++j) acc += g->Rr[a][i] * g->Sig[i][j] * g->Rr[b][j];
            g->Sr[a][b] = acc;
        }
    /* depth key (R9): float32 rounding of the slant-range offset */
    g->key = (double)(float)(g->Rr[2][0] * d[0] + g->Rr[2][1] * d[1] + g->Rr[2][2] * d[2]);

    /* P_C: ndc_x = 2/(dA NA) x_r, ndc_y = 2/(dR NR tan(theta)) y_r */
    double tt = tan(v->theta);
    double ndcC[2] = {2.0 / (v->dA * v->NA) * g->xr[0], 2.0 / (v->dR * v->NR * tt) * g->xr[1]};
    /* P_I: ndc_x as above, ndc_y = 2/(dR NR) z_r - 2h/(dR NR sin(theta))  (R2) */
    double ndcI[2] = {2.0 / (v->dA * v->NA) * g->xr[0],
                      2.0 / (v->dR * v->NR) * g->xr[2] - 2.0 * ORC_ALTITUDE / (v->dR * v->NR * sin(v->theta))};
    int Ns[2] = {v->NA, v->NR};
    for (k = 0; k < 2; ++k) {
        g->u[0][k] = (ndcC[k] + 1.0) * Ns[k] * 0.5 - 0.5;
        g->u[1][k] = (ndcI[k] + 1.0) * Ns[k] * 0.5 - 0.5;
    }
    /* Jacobians of the pixel coordinates with respect to x_r */
    memset(g->J, 0, sizeof(g->J));
    g->J[0][0][0] = 1.0 / v->dA;
    g->J[0][1][1] = 1.0 / (v->dR * tt);
    g->J[1][0][0] = 1.0 / v->dA;
    g->J[1][1][2] = 1.0 / v->dR;
    /* Sigma' = J Sigma_r J^T + eps I  (R4, R8) and its inverse */
    int pl;
    for (pl = 0; pl < 2; ++pl) {
        for (a = 0; a < 2; ++a)
            for (b = 0; b < 2; ++b) {
                double acc = 0.0;
                int i, j;
                for (i = 0; i < 3; ++i)
                    for (j = 0; j < 3; ++j) acc += g->J[pl][a][i] * g->Sr[i][j] * g->J[pl][b][j];
                g->S2[pl][a][b] = acc + (a == b ? cfg->eps : 0.0);
            }
        double det = g->S2[pl][0][0] * g->S2[pl][1][1] - g->S2[pl][0][1] * g->S2[pl][1][0];
        g->det[pl] = det;
        g->C2[pl][0][0] = g->S2[pl][1][1] / det;
        g->C2[pl][1][1] = g->S2[pl][0][0] / det;
        g->C2[pl][0][1] = -g->S2[pl][0][1] / det;
        g->C2[pl][1][0] = -g->S2[pl][1][0] / det;
        /* bounding box of the K-ellipse (used only to skip pixels in culled mode) */
        double K = cfg->K > 0.0 ? cfg->K : 1e30;
        double rx = K * sqrt(g->S2[pl][0][0]) + 1e-9, ry = K * sqrt(g->S2[pl][1][1]) + 1e-9;
        double x0 = ceil(g->u[pl][0] - rx), x1 = floor(g->u[pl][0] + rx);
        double y0 = ceil(g->u[pl][1] - ry), y1 = floor(g->u[pl][1] + ry);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > v->NA - 1) x1 = v->NA - 1;
        if (y1 > v->NR - 1) y1 = v->NR - 1;
        g->bb[pl][0] = (int)x0; g->bb[pl][1] = (int)x1;
        g->bb[pl][2] = (int)y0; g->bb[pl][3] = (int)y1;
    }
    g->cnorm = cfg->norm_mode == 0 ? 1.0 / (2.0 * ORC_PI * sqrt(g->det[1])) : 1.0;
}

static const orc_gauss *g_sort_base;
static int cmp_depth(const void *pa, const void *pb) {
    int ia = *(const int *)pa, ib = *(const int *)pb;
    double ka = g_sort_base[ia].key, kb = g_sort_base[ib].key;
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

static void depth_order(const orc_gauss *g, int N, int *order) {
    int i;
    for (i = 0; i < N; ++i) order[i] = i;
    g_sort_base = g;
    qsort(order, (size_t)N, sizeof(int), cmp_depth);
}

/* Candidate lists for the brute-force loops.  Brute-force mode: every pixel
 * visits every Gaussian (in the given order).  Culled mode: the image is cut
 * into 8x8-pixel cells and each cell lists, in the given order, the
 * Gaussians whose K-ellipse bounding box reaches it; a pixel then visits its
 * cell's list and skips the Gaussians whose box misses the pixel.  Every
 * skipped pair has delta > K^2, so both modes add the same terms in the same
 * order. */
#define ORC_CELL 8
typedef struct {
    int culled;
    int N;
    int cx; /* cells per row */
    int64_t *start;
    int *idx;
} cand_lists;

static void build_cands(const orc_gauss *g, int N, const int *order, const orc_view *v, int pl, int culled,
                        cand_lists *cl) {
    int k;
    cl->culled = culled;
    cl->N = N;
    cl->cx = (v->NA + ORC_CELL - 1) / ORC_CELL;
    if (!culled) {
        cl->start = NULL;
        cl->idx = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
        for (k = 0; k < N; ++k) cl->idx[k] = order[k];
        return;
    }
    int cy = (v->NR + ORC_CELL - 1) / ORC_CELL;
    int64_t ncell = (int64_t)cl->cx * cy, c;
    cl->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (k = 0; k < N; ++k) {
        const orc_gauss *q = &g[order[k]];
        if (q->bb[pl][0] > q->bb[pl][1] || q->bb[pl][2] > q->bb[pl][3]) continue;
        int a, b;
        for (b = q->bb[pl][2] / ORC_CELL; b <= q->bb[pl][3] / ORC_CELL; ++b)
            for (a = q->bb[pl][0] / ORC_CELL; a <= q->bb[pl][1] / ORC_CELL; ++a) cl->start[(int64_t)b * cl->cx + a + 1]++;
    }
    for (c = 0; c < ncell; ++c) cl->start[c + 1] += cl->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
    for (c = 0; c < ncell; ++c) fill[c] = cl->start[c];
    cl->idx = (int *)malloc(sizeof(int) * (size_t)(cl->start[ncell] > 0 ? cl->start[ncell] : 1));
    for (k = 0; k < N; ++k) {
        const orc_gauss *q = &g[order[k]];
        if (q->bb[pl][0] > q->bb[pl][1] || q->bb[pl][2] > q->bb[pl][3]) continue;
        int a, b;
        for (b = q->bb[pl][2] / ORC_CELL; b <= q->bb[pl][3] / ORC_CELL; ++b)
            for (a = q->bb[pl][0] / ORC_CELL; a <= q->bb[pl][1] / ORC_CELL; ++a)
                cl->idx[fill[(int64_t)b * cl->cx + a]++] = order[k];
    }
    free(fill);
}

static void cand_range(const cand_lists *cl, int m, int n, int64_t *b, int64_t *e) {
    if (!cl->culled) { *b = 0; *e = cl->N; return; }
    int64_t c = (int64_t)(n / ORC_CELL) * cl->cx + m / ORC_CELL;
    *b = cl->start[c];
    *e = cl->start[c + 1];
}

static int outside_box(const orc_gauss *q, int pl, int m, int n) {
    return m < q->bb[pl][0] || m > q->bb[pl][1] || n < q->bb[pl][2] || n > q->bb[pl][3];
}

static void free_cands(cand_lists *cl) { free(cl->start); free(cl->idx); }

/* Section II-A-2: scattering intensities.  For every ray (cell centre (m, n))
 * of the computation plane the Gaussians are visited front to back; the ray
 * deposits alpha_i T_i on Gaussian i and is attenuated by (1 - alpha_i).
 * A[i] = sum over rays of alpha_i T_i; I_i = P_i A_i. */
/* Opacity of Gaussian q on a ray where its profile exp(-delta/2) is G
 * (reading R5 and its Beer-Lambert variant). */
static double alpha_of(const orc_gauss *q, const orc_cfg *cfg, double G) {
    return cfg->alpha_mode ? -expm1(-q->tau * G) : q->o * G;
}

static void intensity_pass(const orc_gauss *g, int N, const int *order, const orc_view *v, const orc_cfg *cfg,
                           int culled, double *A, double *Tfin) {
    int nt = n_threads();
    double K2 = cutoff2(cfg);
    double *part = (double *)calloc((size_t)nt * (size_t)(N > 0 ? N : 1), sizeof(double));
    cand_lists cl;
    build_cands(g, N, order, v, 0, culled, &cl);
    int n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < v->NR; ++n) {
        double *Ap = part + (size_t)thread_id() * (size_t)N;
        int m;
        for (m = 0; m < v->NA; ++m) {
            double T = 1.0;
            int64_t k, b, e;
            cand_range(&cl, m, n, &b, &e);
            for (k = b; k < e; ++k) {
                int i = cl.idx[k];
                const orc_gauss *q = &g[i];
                if (culled && outside_box(q, 0, m, n)) continue;
                double dx = m - q->u[0][0], dy = n - q->u[0][1];
                double delta = mahal(q->C2[0], dx, dy);
                if (delta > K2) continue;
                double alpha = alpha_of(q, cfg, exp(-0.5 * delta));
                Ap[i] += alpha * T;
                T *= (1.0 - alpha);
                if (cfg->T_min > 0.0 && T < cfg->T_min) break;
            }
            if (Tfin) Tfin[(size_t)n * v->NA + m] = T;
        }
    }
    int t, i;
    for (i = 0; i < N; ++i) A[i] = 0.0;
    for (t = 0; t < nt; ++t)
        for (i = 0; i < N; ++i) A[i] += part[(size_t)t * N + i];
    free(part);
    free_cands(&cl);
}

/* Section II-A-3: imaging.  S_{n,m} = sum_i beta_i^{n,m} I_i (order-free). */
static void imaging_pass(const orc_gauss *g, int N, const double *I, const orc_view *v, const orc_cfg *cfg, int culled,
                         double *S) {
    double K2 = cutoff2(cfg);
    int *ident = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int i, n;
    for (i = 0; i < N; ++i) ident[i] = i;
    cand_lists cl;
    build_cands(g, N, ident, v, 1, culled, &cl);
#pragma omp parallel for schedule(static)
    for (n = 0; n < v->NR; ++n) {
        int m;
        for (m = 0; m < v->NA; ++m) {
            double acc = 0.0;
            int64_t k, b, e;
            cand_range(&cl, m, n, &b, &e);
            for (k = b; k < e; ++k) {
                int j = cl.idx[k];
                const orc_gauss *q = &g[j];
                if (culled && outside_box(q, 1, m, n)) continue;
                double dx = m - q->u[1][0], dy = n - q->u[1][1];
                double delta = mahal(q->C2[1], dx, dy);
                if (delta > K2) continue;
                acc += q->cnorm * exp(-0.5 * delta) * I[j];
            }
            S[(size_t)n * v->NA + m] = acc;
        }
    }
    free_cands(&cl);
    free(ident);
}

static int view_forward(const double *params, int N, const orc_view *v, const orc_cfg *cfg, int culled, orc_gauss *g,
                        int *order, double *A, double *I, double *S, double *Tfin) {
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) project(params + 12 * (size_t)i, v, cfg, &g[i], cfg->sh ? cfg->sh + 16 * (size_t)i : NULL);
    depth_order(g, N, order);
    intensity_pass(g, N, order, v, cfg, culled, A, Tfin);
    for (i = 0; i < N; ++i) I[i] = g[i].P * A[i];
    if (S) imaging_pass(g, N, I, v, cfg, culled, S);
    return 0;
}

static int check_args(const double *params, int N, const orc_view *views, int V, const orc_cfg *cfg) {
    int v;
    if (N < 0 || V < 0 || (N > 0 && !params) || (V > 0 && !views) || !cfg) return 1;
    for (v = 0; v < V; ++v) {
        if (views[v].NA <= 0 || views[v].NR <= 0) return 1;
        if (!(views[v].dA > 0.0) || !(views[v].dR > 0.0)) return 1;
        if (!(views[v].theta > 0.0) || !(views[v].theta < ORC_PI / 2)) return 1;
    }
    return 0;
}

/* Projected quantities of every Gaussian for one view; 16 doubles each:
 * uC(2) SigmaC(xx,xy,yy) uI(2) SigmaI(xx,xy,yy) key cnorm o z_r detC detI */
int orc_project(const double *params, int32_t N, const orc_view *v, const orc_cfg *cfg, double *out) {
    if (check_args(params, N, v, 1, cfg)) return 1;
    int i;
    for (i = 0; i < N; ++i) {
        orc_gauss g;
        project(params + 12 * (size_t)i, v, cfg, &g, cfg->sh ? cfg->sh + 16 * (size_t)i : NULL);
        double *o = out + 16 * (size_t)i;
        o[0] = g.u[0][0]; o[1] = g.u[0][1];
        o[2] = g.S2[0][0][0]; o[3] = g.S2[0][0][1]; o[4] = g.S2[0][1][1];
        o[5] = g.u[1][0]; o[6] = g.u[1][1];
        o[7] = g.S2[1][0][0]; o[8] = g.S2[1][0][1]; o[9] = g.S2[1][1][1];
        o[10] = g.key; o[11] = g.cnorm; o[12] = g.o; o[13] = g.xr[2];
        o[14] = g.det[0]; o[15] = g.det[1];
    }
    return 0;
}

/* Forward render of V views of one scene.  images: views concatenated, each
 * NR x NA row-major (row = slant-range bin, near to far; column = azimuth
 * bin).  A: [V][N] ray sums (I = P A).  Tfinal (optional): per ray final
 * transmittance, laid out like images. */
int orc_render(const double *params, int32_t N, const orc_view *views, int32_t V, const orc_cfg *cfg,
               int32_t culled, double *images, double *A, double *Tfinal) {
    if (check_args(params, N, views, V, cfg)) return 1;
    if (cfg->K <= 0.0) culled = 0;
    orc_gauss *g = (orc_gauss *)malloc(sizeof(orc_gauss) * (size_t)(N > 0 ? N : 1));
    int *order = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    double *I = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    size_t pix = 0;
    int v;
    for (v = 0; v < V; ++v) {
        view_forward(params, N, &views[v], cfg, culled, g, order, A + (size_t)v * N, I, images + pix,
                     Tfinal ? Tfinal + pix : NULL);
        pix += (size_t)views[v].NA * views[v].NR;
    }
    free(g); free(order); free(I);
    return 0;
}

/* Depth order of one view (indices, front to back), for tests. */
int orc_depth_order(const double *params, int32_t N, const orc_view *v, const orc_cfg *cfg, int32_t *order) {
    if (check_args(params, N, v, 1, cfg)) return 1;
    orc_gauss *g = (orc_gauss *)malloc(sizeof(orc_gauss) * (size_t)(N > 0 ? N : 1));
    int *o = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int i;
    for (i = 0; i < N; ++i) project(params + 12 * (size_t)i, v, cfg, &g[i], cfg->sh ? cfg->sh + 16 * (size_t)i : NULL);
    depth_order(g, N, o);
    for (i = 0; i < N; ++i) order[i] = o[i];
    free(g); free(o);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Backward (Section II-B).  Given dL/dS for every pixel of every view, the
 * gradient of L with respect to the 12 raw parameters of every Gaussian,
 * summed over views.  dLdI (optional) receives dL/dI_i per view, [V][N].
 * ------------------------------------------------------------------------- */

/* dL/dq from dL/dR for R = R(q/|q|). */
static void rot_backward(const orc_gauss *g, const double G[3][3], double dq[4]) {
    double w = g->qhat[0], x = g->qhat[1], y = g->qhat[2], z = g->qhat[3];
    double dw = 2 * (-z * G[0][1] + y * G[0][2] + z * G[1][0] - x * G[1][2] - y * G[2][0] + x * G[2][1]);
    double dx = 2 * (y * G[0][1] + z * G[0][2] + y * G[1][0] - 2 * x * G[1][1] - w * G[1][2] + z * G[2][0] +
                     w * G[2][1] - 2 * x * G[2][2]);
    double dy = 2 * (-2 * y * G[0][0] + x * G[0][1] + w * G[0][2] + x * G[1][0] + z * G[1][2] - w * G[2][0] +
                     z * G[2][1] - 2 * y * G[2][2]);
    double dz = 2 * (-2 * z * G[0][0] - w * G[0][1] + x * G[0][2] + w * G[1][0] - 2 * z * G[1][1] + y * G[1][2] +
                     x * G[2][0] + y * G[2][1]);
    double dh[4] = {dw, dx, dy, dz};
    double dot = g->qhat[0] * dh[0] + g->qhat[1] * dh[1] + g->qhat[2] * dh[2] + g->qhat[3] * dh[3];
    int k;
    for (k = 0; k < 4; ++k) dq[k] = (dh[k] - g->qhat[k] * dot) / g->qlen;
}

/* Per-Gaussian adjoint accumulators of one view. */
typedef struct {
    double gI;       /* dL/dI_i */
    double uI[2];    /* dL/du on the imaging plane */
    double CI[2][2]; /* dL/d(conic) on the imaging plane, general-matrix form */
    double cI;       /* dL/dc_i */
    double uC[2];    /* dL/du on the computation plane */
    double CC[2][2]; /* dL/d(conic) on the computation plane */
    double o;        /* dL/do (alpha_mode 1: dL/dtau) */
} orc_adj;

/* Adjoint of one view, given its forward state (projections g, depth order,
 * ray sums A, intensities I); adds the view's gradient into grads. */
static int view_adjoint(int N, const orc_view *v, const orc_cfg *cfg, int culled, const orc_gauss *g,
                        const int *order, const double *A, const double *I, const double *dLdS, double *grads,
                        double *dLdI_out, double *duI_out) {
    double K2 = cutoff2(cfg);
    orc_adj *adj = (orc_adj *)calloc((size_t)(N > 0 ? N : 1), sizeof(orc_adj));
    int i;

    /* Gradient of the imaging process: S = sum_i c_i e_i I_i with
     * e_i = exp(-delta_i / 2), delta_i = d^T C_I d, d = pixel - u_I. */
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < N; ++i) {
        const orc_gauss *q = &g[i];
        orc_adj *ad = &adj[i];
        int x0 = 0, x1 = v->NA - 1, y0 = 0, y1 = v->NR - 1;
        if (culled) { x0 = q->bb[1][0]; x1 = q->bb[1][1]; y0 = q->bb[1][2]; y1 = q->bb[1][3]; }
        int n, m;
        for (n = y0; n <= y1; ++n)
            for (m = x0; m <= x1; ++m) {
                double d[2] = {m - q->u[1][0], n - q->u[1][1]};
                double delta = mahal(q->C2[1], d[0], d[1]);
                if (delta > K2) continue;
                double e = exp(-0.5 * delta);
                double gS = dLdS[(size_t)n * v->NA + m];
                ad->gI += gS * q->cnorm * e;                 /* dS/dI_i = beta */
                double gE = gS * q->cnorm * I[i];            /* dL/de */
                double Cd0 = q->C2[1][0][0] * d[0] + q->C2[1][0][1] * d[1];
                double Cd1 = q->C2[1][1][0] * d[0] + q->C2[1][1][1] * d[1];
                ad->uI[0] += gE * e * Cd0;                   /* de/du = e C d */
                ad->uI[1] += gE * e * Cd1;
                int a, b;
                for (a = 0; a < 2; ++a)
                    for (b = 0; b < 2; ++b) ad->CI[a][b] += gE * (-0.5 * e * d[a] * d[b]);
                ad->cI += gS * e * I[i];                     /* dS/dc_i */
            }
    }

    /* Gradient of the intensity computation.  Per ray, the ray's share of
     * L is sum_i chat_i alpha_i T_i with chat_i = dL/dI_i P_i, so
     * dL/dalpha_i = T_i (chat_i - B_i),
     * B_i = sum_{j>i} chat_j alpha_j prod_{i<k<j} (1 - alpha_k),
     * a suffix sum taken back to front (no division by 1 - alpha). */
    double *chat = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (i = 0; i < N; ++i) chat[i] = adj[i].gI * g[i].P;
    int nt = n_threads();
    double *part = (double *)calloc((size_t)nt * (size_t)(N > 0 ? N : 1) * 7, sizeof(double));
    cand_lists cl;
    build_cands(g, N, order, v, 0, culled, &cl);
    int n;
#pragma omp parallel for schedule(static)
    for (n = 0; n < v->NR; ++n) {
        double *Pp = part + (size_t)thread_id() * (size_t)N * 7;
        int64_t cap = N > 0 ? N : 1;
        int *hit = (int *)malloc(sizeof(int) * (size_t)cap);
        double *al = (double *)malloc(sizeof(double) * (size_t)cap);
        double *Ts = (double *)malloc(sizeof(double) * (size_t)cap);
        int m;
        for (m = 0; m < v->NA; ++m) {
            /* front to back: the Gaussians this ray meets, their alpha and T */
            int64_t cnt = 0, k, b, e;
            double T = 1.0;
            cand_range(&cl, m, n, &b, &e);
            for (k = b; k < e; ++k) {
                int j = cl.idx[k];
                const orc_gauss *q = &g[j];
                if (culled && outside_box(q, 0, m, n)) continue;
                double dx = m - q->u[0][0], dy = n - q->u[0][1];
                double delta = mahal(q->C2[0], dx, dy);
                if (delta > K2) continue;
                double alpha = alpha_of(q, cfg, exp(-0.5 * delta));
                hit[cnt] = j; al[cnt] = alpha; Ts[cnt] = T; ++cnt;
                T *= (1.0 - alpha);
                if (cfg->T_min > 0.0 && T < cfg->T_min) break;
            }
            /* back to front: suffix sums B and dL/dalpha */
            double B = 0.0;
            for (k = cnt - 1; k >= 0; --k) {
                int j = hit[k];
                const orc_gauss *q = &g[j];
                double galpha = Ts[k] * (chat[j] - B);
                B = chat[j] * al[k] + (1.0 - al[k]) * B;
                double d[2] = {m - q->u[0][0], n - q->u[0][1]};
                double e1 = exp(-0.5 * mahal(q->C2[0], d[0], d[1])); /* exp(-delta/2) */
                double *acc = Pp + (size_t)j * 7;
                double gE;                                            /* dL/de */
                if (cfg->alpha_mode) {
                    /* alpha = 1 - exp(-tau e): d alpha/d tau = e (1 - alpha), d alpha/d e = tau (1 - alpha) */
                    acc[0] += galpha * e1 * (1.0 - al[k]);            /* dL/dtau */
                    gE = galpha * q->tau * (1.0 - al[k]);
                } else {
                    acc[0] += galpha * e1;                            /* dL/do */
                    gE = galpha * q->o;
                }
                acc[1] += gE * e1 * (q->C2[0][0][0] * d[0] + q->C2[0][0][1] * d[1]);
                acc[2] += gE * e1 * (q->C2[0][1][0] * d[0] + q->C2[0][1][1] * d[1]);
                acc[3] += gE * (-0.5 * e1 * d[0] * d[0]);
                acc[4] += gE * (-0.5 * e1 * d[0] * d[1]);
                acc[5] += gE * (-0.5 * e1 * d[1] * d[0]);
                acc[6] += gE * (-0.5 * e1 * d[1] * d[1]);
            }
        }
        free(hit); free(al); free(Ts);
    }
    int t;
    for (t = 0; t < nt; ++t)
        for (i = 0; i < N; ++i) {
            const double *acc = part + ((size_t)t * N + i) * 7;
            adj[i].o += acc[0];
            adj[i].uC[0] += acc[1]; adj[i].uC[1] += acc[2];
            adj[i].CC[0][0] += acc[3]; adj[i].CC[0][1] += acc[4];
            adj[i].CC[1][0] += acc[5]; adj[i].CC[1][1] += acc[6];
        }
    free(part);
    free_cands(&cl);

    /* Gradient of the Gaussian parameters: conic -> 2D covariance ->
     * Sigma_r -> Sigma -> (scale, rotation); pixel centres -> x_r -> mean. */
    for (i = 0; i < N; ++i) {
        const orc_gauss *q = &g[i];
        const orc_adj *ad = &adj[i];
        double *gr = grads + 12 * (size_t)i;
        double dS2[2][2][2];
        int pl, a, b, k, l;
        for (pl = 0; pl < 2; ++pl) {
            const double(*C)[2] = q->C2[pl];
            const double(*G)[2] = pl == 0 ? ad->CC : ad->CI;
            /* C = Sigma'^{-1}:  dL/dSigma' = -C^T G C^T */
            for (a = 0; a < 2; ++a)
                for (b = 0; b < 2; ++b) {
                    double acc = 0.0;
                    for (k = 0; k < 2; ++k)
                        for (l = 0; l < 2; ++l) acc -= C[k][a] * G[k][l] * C[b][l];
                    dS2[pl][a][b] = acc;
                }
        }
        if (cfg->norm_mode == 0) {
            /* c = 1/(2 pi sqrt(det Sigma'_I)):  dc/dSigma'_I = -c/2 Sigma'_I^{-T} */
            for (a = 0; a < 2; ++a)
                for (b = 0; b < 2; ++b) dS2[1][a][b] += ad->cI * (-0.5 * q->cnorm * q->C2[1][b][a]);
        }
        /* Sigma' = J Sigma_r J^T + eps I:  dL/dSigma_r = J^T dL/dSigma' J */
        double dSr[3][3] = {{0}};
        for (pl = 0; pl < 2; ++pl)
            for (a = 0; a < 3; ++a)
                for (b = 0; b < 3; ++b)
                    for (k = 0; k < 2; ++k)
                        for (l = 0; l < 2; ++l) dSr[a][b] += q->J[pl][k][a] * dS2[pl][k][l] * q->J[pl][l][b];
        /* Sigma_r = R_r Sigma R_r^T:  dL/dSigma = R_r^T dL/dSigma_r R_r */
        double dSig[3][3] = {{0}};
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b)
                for (k = 0; k < 3; ++k)
                    for (l = 0; l < 3; ++l) dSig[a][b] += q->Rr[k][a] * dSr[k][l] * q->Rr[l][b];
        /* Sigma = M M^T, M = R diag(s):  dL/dM = (G + G^T) M */
        double M[3][3], dM[3][3];
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) M[a][b] = q->R[a][b] * q->s[b];
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (k = 0; k < 3; ++k) acc += (dSig[a][k] + dSig[k][a]) * M[k][b];
                dM[a][b] = acc;
            }
        double dR[3][3], ds[3];
        for (b = 0; b < 3; ++b) {
            ds[b] = 0.0;
            for (a = 0; a < 3; ++a) {
                ds[b] += dM[a][b] * q->R[a][b];
                dR[a][b] = dM[a][b] * q->s[b];
            }
        }
        double dq[4];
        rot_backward(q, dR, dq);
        /* pixel centres: u = J x_r + const, x_r = R_r (mu - c) + T_r */
        double dxr[3] = {0, 0, 0};
        for (a = 0; a < 3; ++a)
            for (k = 0; k < 2; ++k) dxr[a] += q->J[0][k][a] * ad->uC[k] + q->J[1][k][a] * ad->uI[k];
        for (a = 0; a < 3; ++a) gr[a] += q->Rr[0][a] * dxr[0] + q->Rr[1][a] * dxr[1] + q->Rr[2][a] * dxr[2];
        /* d o / d logit = o (1 - o); d tau / d logit = sigmoid(logit) = o */
        gr[3] += ad->o * (cfg->alpha_mode ? q->o : q->o * (1.0 - q->o));
        for (k = 0; k < 3; ++k) gr[4 + k] += ds[k] * q->s[k];
        gr[7] += ad->gI * A[i];
        if (cfg->dsh) {
            int kk;
            for (kk = 0; kk < 15; ++kk) cfg->dsh[16 * (size_t)i + kk] += ad->gI * A[i] * q->Ysh[kk];
        }
        for (k = 0; k < 4; ++k) gr[8 + k] += dq[k];
        if (dLdI_out) dLdI_out[i] = ad->gI;
        if (duI_out) { duI_out[2 * (size_t)i] = ad->uI[0]; duI_out[2 * (size_t)i + 1] = ad->uI[1]; }
    }
    free(chat); free(adj);
    return 0;
}

static int view_backward(const double *params, int N, const orc_view *v, const orc_cfg *cfg, int culled,
                         const double *dLdS, double *grads, double *dLdI_out, double *duI_out) {
    orc_gauss *g = (orc_gauss *)malloc(sizeof(orc_gauss) * (size_t)(N > 0 ? N : 1));
    int *order = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    double *A = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *I = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    view_forward(params, N, v, cfg, culled, g, order, A, I, NULL, NULL);
    view_adjoint(N, v, cfg, culled, g, order, A, I, dLdS, grads, dLdI_out, duI_out);
    free(g); free(order); free(A); free(I);
    return 0;
}

int orc_grad(const double *params, int32_t N, const orc_view *views, int32_t V, const orc_cfg *cfg, int32_t culled,
             const double *dLdS, double *grads, double *dLdI) {
    if (check_args(params, N, views, V, cfg) || !dLdS || !grads) return 1;
    if (cfg->K <= 0.0) culled = 0;
    size_t pix = 0;
    int v;
    memset(grads, 0, sizeof(double) * 12 * (size_t)N);
    if (cfg->dsh) memset(cfg->dsh, 0, sizeof(double) * 16 * (size_t)N);
    for (v = 0; v < V; ++v) {
        view_backward(params, N, &views[v], cfg, culled, dLdS + pix, grads, dLdI ? dLdI + (size_t)v * N : NULL,
                      cfg->duI ? cfg->duI + (size_t)v * N * 2 : NULL);
        pix += (size_t)views[v].NA * views[v].NR;
    }
    return 0;
}

/* One optimisation step's rendering work for V views of one scene: forward
 * (images), the L1 loss against targets (mean over all pixels of all views),
 * and the adjoint reusing each view's forward state.  images: out, laid out
 * as in orc_render; grads: out [N][12].  Returns the loss (NaN on bad
 * arguments). */
double orc_l1(const double *S, const double *target, int64_t npix, double *dLdS);

double orc_step(const double *params, int32_t N, const orc_view *views, int32_t V, const orc_cfg *cfg, int32_t culled,
                const double *targets, double *images, double *grads) {
    if (check_args(params, N, views, V, cfg) || !targets || !images || !grads) return NAN;
    if (cfg->K <= 0.0) culled = 0;
    size_t n1 = (size_t)(N > 0 ? N : 1);
    orc_gauss **g = (orc_gauss **)malloc(sizeof(orc_gauss *) * (size_t)(V > 0 ? V : 1));
    int **order = (int **)malloc(sizeof(int *) * (size_t)(V > 0 ? V : 1));
    double **A = (double **)malloc(sizeof(double *) * (size_t)(V > 0 ? V : 1));
    double **I = (double **)malloc(sizeof(double *) * (size_t)(V > 0 ? V : 1));
    size_t pix = 0, *poff = (size_t *)malloc(sizeof(size_t) * (size_t)(V + 1));
    int v;
    for (v = 0; v < V; ++v) {
        g[v] = (orc_gauss *)malloc(sizeof(orc_gauss) * n1);
        order[v] = (int *)malloc(sizeof(int) * n1);
        A[v] = (double *)malloc(sizeof(double) * n1);
        I[v] = (double *)malloc(sizeof(double) * n1);
        poff[v] = pix;
        view_forward(params, N, &views[v], cfg, culled, g[v], order[v], A[v], I[v], images + pix, NULL);
        pix += (size_t)views[v].NA * views[v].NR;
    }
    double *dLdS = (double *)malloc(sizeof(double) * (pix > 0 ? pix : 1));
    double loss = orc_l1(images, targets, (int64_t)pix, dLdS);
    memset(grads, 0, sizeof(double) * 12 * (size_t)N);
    if (cfg->dsh) memset(cfg->dsh, 0, sizeof(double) * 16 * (size_t)N);
    for (v = 0; v < V; ++v) {
        view_adjoint(N, &views[v], cfg, culled, g[v], order[v], A[v], I[v], dLdS + poff[v], grads, NULL, NULL);
        free(g[v]); free(order[v]); free(A[v]); free(I[v]);
    }
    free(g); free(order); free(A); free(I); free(poff); free(dLdS);
    return loss;
}

/* Adam (Kingma & Ba), with the bias corrections and eps added to the square
 * root of the corrected second moment, one learning rate per parameter
 * group: lr[0] means, lr[1] log-scales, lr[2] quaternions, lr[3] opacity
 * logit, lr[4] P.  step is 1-based. */
int orc_adam(double *params, const double *grads, double *m, double *v, int64_t N, const double lr[5], double b1,
             double b2, double eps, int32_t step) {
    static const int group[12] = {0, 0, 0, 3, 1, 1, 1, 4, 2, 2, 2, 2};
    if (N < 0 || step < 1) return 1;
    double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
    int64_t i;
    for (i = 0; i < N * 12; ++i) {
        double g = grads[i];
        m[i] = b1 * m[i] + (1.0 - b1) * g;
        v[i] = b2 * v[i] + (1.0 - b2) * g * g;
        double mh = m[i] / bc1, vh = v[i] / bc2;
        params[i] -= lr[group[i % 12]] * mh / (sqrt(vh) + eps);
    }
    return 0;
}

/* L1 loss, mean over every pixel of every view, and its gradient
 * dL/dS = sign(S - S*) / (number of pixels), sign(0) = 0. */
double orc_l1(const double *S, const double *target, int64_t npix, double *dLdS) {
    double acc = 0.0;
    int64_t k;
    for (k = 0; k < npix; ++k) {
        double r = S[k] - target[k];
        acc += fabs(r);
        if (dLdS) dLdS[k] = (r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0)) / (double)npix;
    }
    return acc / (double)npix;
}
