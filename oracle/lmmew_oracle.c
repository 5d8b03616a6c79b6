/*
 * FP64 CPU oracle of the list-mode multi-energy-window (LM-MEW) path model
 * and its LM-OSEM reconstruction (Rahman et al., arXiv 2305.17111).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * links, includes or calls it, and it shares no code with that library.
 *
 * Everything is double precision, in plain loops, following the paper:
 *   - path sensitivity s(P, E_0^w)          Eq. (s_p), with n = 0 and n = 1
 *   - path integral gamma(r_u, r_v, E)      Eq. (radpath)
 *   - event density pr(A_j | lambda)         Eq. (Aj_expansion) and (pr_path_1)
 *   - LM-MLEM / LM-OSEM update               Eq. (lm_mlem), (os-lm-mlem), (z_bar_update_os)
 *   - observed-data log-likelihood           Eq. (lll_med)
 * with the steps of Algorithm 1 (precompute path integrals and path
 * sensitivities, then per subset the event sums, then the update).
 *
 * Readings of the paper where it is silent (the same readings the CUDA path
 * implements, written here independently):
 *   - detector response pr(A|P,E): collimator bin probability (Gaussian whose
 *     FWHM grows linearly with depth, integrated over the bin) times the
 *     energy-resolution Gaussian density at the recorded energy;
 *   - scatter subpaths: a grid of scatter cells (cell density = mean of its
 *     pixels), point quadrature with weight A_p / (2 pi d) (the polar area
 *     element of the in-plane emission), the cell that contains the emission
 *     voxel is skipped;
 *   - Klein-Nishina "normalised to a 2-D plane": in-plane density
 *     K(theta) / integral_0^{2pi} K, times 2 pi so that isotropy gives 1;
 *   - scatter probability per unit length = mu (total attenuation);
 *   - constant collimator acceptance and solid-angle factors = 1;
 *   - sensitivity = integral of the row over the detector and the windows;
 *   - subsets interleave angles: s(a) = a mod N_s;
 *   - a line integral that runs exactly along a pixel edge takes the mean of
 *     the two pixels on either side.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ME_C2_KEV 510.99895
#define ORC_PI 3.14159265358979323846

typedef struct {
    /* scanner and grid */
    int n;              /* image is n x n pixels */
    double h;           /* pixel size, cm */
    int n_angles;       /* detector angles over 360 degrees */
    int n_bins;         /* detector bins */
    double bin_w;       /* bin width, cm; bins span [-n_bins*bin_w/2, +n_bins*bin_w/2) */
    double r_det;       /* detector face distance from the centre, cm */
    double fwhm0;       /* collimator FWHM at the face, cm */
    double fwhm_slope;  /* collimator FWHM growth per cm of depth */
    double scan_time;   /* T */
    /* attenuation */
    const float* rho;   /* n*n relative density, [iy*n + ix] */
    int n_knots;
    double knot_e[16];
    double knot_mu[16];
    int scatter_n;      /* scatter grid is scatter_n x scatter_n cells; 0 = no scatter */
    /* spectrum */
    int n_lines;
    double line_e[16];
    double line_yield[16];
    /* energy model */
    double fwhm_frac, e_ref, fwhm_expo;
    int n_windows;
    double win_lo[16], win_hi[16];
    /* voxel set: n*n mask, nonzero = voxel belongs to the model */
    const uint8_t* support;
} orc_params;

typedef struct {
    orc_params p;
    float* rho;          /* own copy */
    int nq;              /* support voxels */
    int* q_pix;          /* pixel index of each support voxel */
    int np;              /* scatter points with positive density */
    double* p_x;         /* scatter point position, pixel units from the corner */
    double* p_y;
    double* p_rho;       /* mean density of the cell */
    int* p_cell;         /* cell index my*S + mx */
    double cell_area;    /* cm^2 */
    double* cos_a;       /* detector direction n_a per angle */
    double* sin_a;
    double* gam_qp;      /* [nq][np] integral of rho along q -> p, cm */
    double* dist_qp;     /* [nq][np] |r_p - r_q|, cm */
    double* gam_det_q;   /* [A][nq] integral of rho from q to the detector, cm */
    double* gam_det_p;   /* [A][np] integral of rho from p to the detector, cm */
    double kn_norm[16];  /* per line: integral over [0, 2 pi) of the KN shape */
} orc_model;

/* ------------------------------------------------------------------ */
/* Physics of the energy axis                                          */
/* ------------------------------------------------------------------ */

/* Mass of a Gaussian N(mean, sigma^2) on [lo, hi].  Written with erfc on the
 * side of the tail so that far-tail masses keep their relative accuracy. */
static double gauss_interval(double lo, double hi, double mean, double sigma) {
    double s = sqrt(2.0) * sigma;
    double zl = (lo - mean) / s, zh = (hi - mean) / s;
    if (zl >= 0.0) return 0.5 * (erfc(zl) - erfc(zh));
    if (zh <= 0.0) return 0.5 * (erfc(-zh) - erfc(-zl));
    return 0.5 * (erf(zh) - erf(zl));
}

/* Water attenuation coefficient (1/cm) at energy e: linear through the
 * knots, end segments extended (the paper assumes mu piecewise linear in E). */
double orc_mu_water(const orc_model* m, double e) {
    const orc_params* p = &m->p;
    if (p->n_knots == 1) return p->knot_mu[0];
    int s = 0;
    while (s < p->n_knots - 2 && e >= p->knot_e[s + 1]) s++;
    double t = (e - p->knot_e[s]) / (p->knot_e[s + 1] - p->knot_e[s]);
    return p->knot_mu[s] + t * (p->knot_mu[s + 1] - p->knot_mu[s]);
}

/* Energy resolution: FWHM/E = frac * (E/E_ref)^exponent; returns sigma, keV. */
double orc_sigma_e(const orc_model* m, double e) {
    const orc_params* p = &m->p;
    double fwhm = p->fwhm_frac * e * pow(e / p->e_ref, p->fwhm_expo);
    return fwhm / (2.0 * sqrt(2.0 * log(2.0)));
}

/* Density (1/keV) of recording energy e_hat for a photon of energy e. */
double orc_energy_density(const orc_model* m, double e_hat, double e) {
    double s = orc_sigma_e(m, e);
    double z = (e_hat - e) / s;
    return exp(-0.5 * z * z) / (sqrt(2.0 * ORC_PI) * s);
}

/* Probability that a photon of energy e is recorded inside some window. */
double orc_window_mass(const orc_model* m, double e) {
    double s = orc_sigma_e(m, e);
    double tot = 0.0;
    for (int k = 0; k < m->p.n_windows; k++)
        tot += gauss_interval(m->p.win_lo[k], m->p.win_hi[k], e, s);
    return tot;
}

/* Klein-Nishina angular shape (E'/E)^2 (E'/E + E/E' - sin^2 theta). */
double orc_kn_shape(double e, double cos_t) {
    double ratio = 1.0 / (1.0 + (e / ORC_ME_C2_KEV) * (1.0 - cos_t));
    return ratio * ratio * (ratio + 1.0 / ratio - (1.0 - cos_t * cos_t));
}

/* Integral of the KN shape over in-plane angles [0, 2 pi): periodic
 * trapezoid rule, which converges geometrically for this analytic periodic
 * integrand. */
double orc_kn_plane_norm(double e) {
    const int nodes = 8192;
    double sum = 0.0;
    for (int i = 0; i < nodes; i++) sum += orc_kn_shape(e, cos(2.0 * ORC_PI * i / nodes));
    return sum * 2.0 * ORC_PI / nodes;
}

double orc_compton_energy(double e, double cos_t) {
    return e / (1.0 + (e / ORC_ME_C2_KEV) * (1.0 - cos_t));
}

/* ------------------------------------------------------------------ */
/* Collimator / position response                                      */
/* ------------------------------------------------------------------ */

double orc_sigma_coll(const orc_model* m, double depth) {
    return (m->p.fwhm0 + m->p.fwhm_slope * depth) / (2.0 * sqrt(2.0 * log(2.0)));
}

/* Probability that a photon whose ideal detector coordinate is u lands in
 * bin b, for a Gaussian blur sigma. */
double orc_bin_prob(const orc_model* m, int b, double u, double sigma) {
    double lo = -0.5 * m->p.n_bins * m->p.bin_w + b * m->p.bin_w;
    double hi = lo + m->p.bin_w;
    return gauss_interval(lo, hi, u, sigma);
}

/* Probability that it lands anywhere on the detector. */
double orc_detector_mass(const orc_model* m, double u, double sigma) {
    double half = 0.5 * m->p.n_bins * m->p.bin_w;
    return gauss_interval(-half, half, u, sigma);
}

/* ------------------------------------------------------------------ */
/* Line integrals of rho (exact for the pixelwise-constant map)        */
/* ------------------------------------------------------------------ */

static double rho_pix(const orc_model* m, int ix, int iy) {
    int n = m->p.n;
    if (ix < 0 || iy < 0 || ix >= n || iy >= n) return 0.0;
    return m->rho[iy * n + ix];
}

/* Density at a point (pixel units from the corner).  A point on a grid line
 * of an axis-parallel ray is handled by the caller. */
static double rho_at(const orc_model* m, double x, double y) {
    return rho_pix(m, (int)floor(x), (int)floor(y));
}

/* Integral of rho along the segment (x0,y0)->(x1,y1), both in pixel units,
 * returned in pixel units of length.  Parametric form r(t) = r0 + t (r1-r0):
 * every crossing of a pixel edge splits the segment, and each piece lies in
 * one pixel whose density is read at the piece's midpoint.  A ray that runs
 * exactly along a grid line takes the mean of the pixels on both sides. */
static double seg_integral_pix(const orc_model* m, double x0, double y0, double x1, double y1) {
    const int n = m->p.n;
    double dx = x1 - x0, dy = y1 - y0;
    double len = sqrt(dx * dx + dy * dy);
    if (len == 0.0) return 0.0;
    /* clip t to the image square [0, n]^2 */
    double tmin = 0.0, tmax = 1.0;
    if (dx == 0.0) {
        if (x0 < 0.0 || x0 > n) return 0.0;
    } else {
        double ta = (0.0 - x0) / dx, tb = (n - x0) / dx;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > tmin) tmin = ta;
        if (tb < tmax) tmax = tb;
    }
    if (dy == 0.0) {
        if (y0 < 0.0 || y0 > n) return 0.0;
    } else {
        double ta = (0.0 - y0) / dy, tb = (n - y0) / dy;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > tmin) tmin = ta;
        if (tb < tmax) tmax = tb;
    }
    if (tmax <= tmin) return 0.0;
    /* axis-parallel ray on a grid line */
    int on_x_line = (dx == 0.0 && x0 == floor(x0));
    int on_y_line = (dy == 0.0 && y0 == floor(y0));

    /* crossing parameters of vertical (x = k) and horizontal (y = k) lines */
    int cap = 2 * n + 4;
    double* tx = (double*)malloc(sizeof(double) * cap);
    double* ty = (double*)malloc(sizeof(double) * cap);
    int nx = 0, ny = 0;
    if (dx != 0.0) {
        for (int k = 0; k <= n; k++) {
            double t = (k - x0) / dx;
            if (t > tmin && t < tmax) tx[nx++] = t;
        }
        if (dx < 0.0)  /* make increasing */
            for (int i = 0; i < nx / 2; i++) { double t = tx[i]; tx[i] = tx[nx - 1 - i]; tx[nx - 1 - i] = t; }
    }
    if (dy != 0.0) {
        for (int k = 0; k <= n; k++) {
            double t = (k - y0) / dy;
            if (t > tmin && t < tmax) ty[ny++] = t;
        }
        if (dy < 0.0)
            for (int i = 0; i < ny / 2; i++) { double t = ty[i]; ty[i] = ty[ny - 1 - i]; ty[ny - 1 - i] = t; }
    }
    /* merge the two increasing lists and sum piece lengths x density */
    double total = 0.0, t_prev = tmin;
    int i = 0, j = 0;
    for (;;) {
        double t_next;
        if (i < nx && (j >= ny || tx[i] <= ty[j])) t_next = tx[i++];
        else if (j < ny) t_next = ty[j++];
        else t_next = tmax;
        if (t_next > t_prev) {
            double tm = 0.5 * (t_prev + t_next);
            double px = x0 + tm * dx, py = y0 + tm * dy;
            double r;
            if (on_x_line) r = 0.5 * (rho_pix(m, (int)x0 - 1, (int)floor(py)) + rho_pix(m, (int)x0, (int)floor(py)));
            else if (on_y_line) r = 0.5 * (rho_pix(m, (int)floor(px), (int)y0 - 1) + rho_pix(m, (int)floor(px), (int)y0));
            else r = rho_at(m, px, py);
            total += (t_next - t_prev) * len * r;
        }
        t_prev = t_next;
        if (t_next >= tmax) break;
    }
    free(tx);
    free(ty);
    return total;
}

/* Integral of rho (cm) along the segment between two points given in cm. */
double orc_line_integral(const orc_model* m, double x0, double y0, double x1, double y1) {
    double c = 0.5 * m->p.n, h = m->p.h;
    return h * seg_integral_pix(m, x0 / h + c, y0 / h + c, x1 / h + c, y1 / h + c);
}

/* Integral of rho (cm) from a point (pixel units) to the edge of the image,
 * along the direction (cx, cy). */
static double det_integral_pix(const orc_model* m, double x, double y, double cx, double cy) {
    double far = 4.0 * m->p.n + 8.0;
    return m->p.h * seg_integral_pix(m, x, y, x + far * cx, y + far * cy);
}

/* Same, from a point in cm, along the direction of detector angle a. */
double orc_detector_integral(const orc_model* m, double x_cm, double y_cm, int a) {
    double c = 0.5 * m->p.n, h = m->p.h;
    return det_integral_pix(m, x_cm / h + c, y_cm / h + c, m->cos_a[a], m->sin_a[a]);
}

/* ------------------------------------------------------------------ */
/* Model construction: voxel set, scatter points, path integrals        */
/* ------------------------------------------------------------------ */

void orc_destroy(orc_model* m) {
    if (!m) return;
    free(m->rho); free(m->q_pix); free(m->p_x); free(m->p_y); free(m->p_rho); free(m->p_cell);
    free(m->cos_a); free(m->sin_a); free(m->gam_qp); free(m->dist_qp);
    free(m->gam_det_q); free(m->gam_det_p);
    free(m);
}

static void voxel_xy_pix(const orc_model* m, int q, double* x, double* y) {
    int pix = m->q_pix[q];
    *x = (pix % m->p.n) + 0.5;
    *y = (pix / m->p.n) + 0.5;
}

orc_model* orc_create(const orc_params* params) {
    orc_model* m = (orc_model*)calloc(1, sizeof(orc_model));
    m->p = *params;
    const int n = m->p.n, A = m->p.n_angles;
    m->rho = (float*)malloc(sizeof(float) * n * n);
    memcpy(m->rho, params->rho, sizeof(float) * n * n);
    m->p.rho = m->rho;
    m->p.support = NULL;

    m->q_pix = (int*)malloc(sizeof(int) * n * n);
    m->nq = 0;
    for (int i = 0; i < n * n; i++)
        if (params->support[i]) m->q_pix[m->nq++] = i;

    /* detector directions; quarter turns are exact */
    m->cos_a = (double*)malloc(sizeof(double) * A);
    m->sin_a = (double*)malloc(sizeof(double) * A);
    for (int a = 0; a < A; a++) {
        if ((4 * a) % A == 0) {
            int k = (4 * a) / A;
            double c[4] = {1, 0, -1, 0}, s[4] = {0, 1, 0, -1};
            m->cos_a[a] = c[k];
            m->sin_a[a] = s[k];
        } else {
            double th = 2.0 * ORC_PI * a / A;
            m->cos_a[a] = cos(th);
            m->sin_a[a] = sin(th);
        }
    }

    /* scatter points: centres of the cells with positive mean density */
    const int S = m->p.scatter_n;
    m->np = 0;
    if (S > 0) {
        int f = n / S;
        m->cell_area = (f * m->p.h) * (f * m->p.h);
        m->p_x = (double*)malloc(sizeof(double) * S * S);
        m->p_y = (double*)malloc(sizeof(double) * S * S);
        m->p_rho = (double*)malloc(sizeof(double) * S * S);
        m->p_cell = (int*)malloc(sizeof(int) * S * S);
        for (int my = 0; my < S; my++)
            for (int mx = 0; mx < S; mx++) {
                double sum = 0.0;
                for (int iy = my * f; iy < (my + 1) * f; iy++)
                    for (int ix = mx * f; ix < (mx + 1) * f; ix++) sum += m->rho[iy * n + ix];
                double mean = sum / (f * f);
                if (mean > 0.0) {
                    m->p_x[m->np] = (mx + 0.5) * f;
                    m->p_y[m->np] = (my + 0.5) * f;
                    m->p_rho[m->np] = mean;
                    m->p_cell[m->np] = my * S + mx;
                    m->np++;
                }
            }
    }

    const int nq = m->nq, np = m->np;
    m->gam_det_q = (double*)malloc(sizeof(double) * (size_t)A * nq);
    m->gam_det_p = (double*)malloc(sizeof(double) * (size_t)A * (np > 0 ? np : 1));
    m->gam_qp = (double*)malloc(sizeof(double) * (size_t)nq * (np > 0 ? np : 1));
    m->dist_qp = (double*)malloc(sizeof(double) * (size_t)nq * (np > 0 ? np : 1));

    /* Algorithm 1: compute and store the path integrals */
#pragma omp parallel for schedule(dynamic, 4)
    for (int a = 0; a < A; a++) {
        for (int q = 0; q < nq; q++) {
            double x, y;
            voxel_xy_pix(m, q, &x, &y);
            m->gam_det_q[(size_t)a * nq + q] = det_integral_pix(m, x, y, m->cos_a[a], m->sin_a[a]);
        }
        for (int p = 0; p < np; p++)
            m->gam_det_p[(size_t)a * np + p] = det_integral_pix(m, m->p_x[p], m->p_y[p], m->cos_a[a], m->sin_a[a]);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < nq; q++) {
        double x, y;
        voxel_xy_pix(m, q, &x, &y);
        for (int p = 0; p < np; p++) {
            double dx = m->p_x[p] - x, dy = m->p_y[p] - y;
            m->gam_qp[(size_t)q * np + p] = m->p.h * seg_integral_pix(m, x, y, m->p_x[p], m->p_y[p]);
            m->dist_qp[(size_t)q * np + p] = m->p.h * sqrt(dx * dx + dy * dy);
        }
    }
    for (int w = 0; w < m->p.n_lines; w++) m->kn_norm[w] = orc_kn_plane_norm(m->p.line_e[w]);
    return m;
}

int orc_num_voxels(const orc_model* m) { return m->nq; }
int orc_num_scatter_points(const orc_model* m) { return m->np; }
void orc_voxel_pixels(const orc_model* m, int32_t* out) {
    for (int q = 0; q < m->nq; q++) out[q] = m->q_pix[q];
}

/* ------------------------------------------------------------------ */
/* Path sensitivities s(P, E_0^w) for one detector angle (Eq. s_p)      */
/* ------------------------------------------------------------------ */

typedef struct {
    int a;
    double* s_prim;   /* [W][nq]     s of the unscattered path q -> detector */
    double* s_scat;   /* [W][nq][np] s of the path q -> p -> detector */
    double* e_scat;   /* [W][nq][np] photon energy after the scatter */
    double* u_q;      /* [nq] detector coordinate of the voxel */
    double* sig_q;    /* [nq] collimator blur at the voxel's depth */
    double* u_p;      /* [np] */
    double* sig_p;    /* [np] */
} angle_paths;

static void voxel_xy_cm(const orc_model* m, int q, double* x, double* y) {
    double xp, yp;
    voxel_xy_pix(m, q, &xp, &yp);
    *x = (xp - 0.5 * m->p.n) * m->p.h;
    *y = (yp - 0.5 * m->p.n) * m->p.h;
}

static void angle_paths_build(const orc_model* m, int a, angle_paths* ap) {
    const int nq = m->nq, np = m->np, W = m->p.n_lines;
    const double ca = m->cos_a[a], sa = m->sin_a[a];
    ap->a = a;
    ap->s_prim = (double*)malloc(sizeof(double) * W * nq);
    ap->s_scat = (double*)malloc(sizeof(double) * (size_t)W * nq * (np > 0 ? np : 1));
    ap->e_scat = (double*)malloc(sizeof(double) * (size_t)W * nq * (np > 0 ? np : 1));
    ap->u_q = (double*)malloc(sizeof(double) * nq);
    ap->sig_q = (double*)malloc(sizeof(double) * nq);
    ap->u_p = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    ap->sig_p = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    for (int q = 0; q < nq; q++) {
        double x, y;
        voxel_xy_cm(m, q, &x, &y);
        ap->u_q[q] = -x * sa + y * ca;
        ap->sig_q[q] = orc_sigma_coll(m, m->p.r_det - (x * ca + y * sa));
    }
    for (int p = 0; p < np; p++) {
        double x = (m->p_x[p] - 0.5 * m->p.n) * m->p.h, y = (m->p_y[p] - 0.5 * m->p.n) * m->p.h;
        ap->u_p[p] = -x * sa + y * ca;
        ap->sig_p[p] = orc_sigma_coll(m, m->p.r_det - (x * ca + y * sa));
    }
    const int f = (m->p.scatter_n > 0) ? m->p.n / m->p.scatter_n : 1;
#pragma omp parallel for schedule(static)
    for (int q = 0; q < nq; q++) {
        double xq, yq;
        voxel_xy_pix(m, q, &xq, &yq);
        int pix = m->q_pix[q];
        int own_cell = (m->p.scatter_n > 0) ? ((pix / m->p.n) / f) * m->p.scatter_n + (pix % m->p.n) / f : -1;
        for (int w = 0; w < W; w++) {
            double e0 = m->p.line_e[w];
            double mu0 = orc_mu_water(m, e0);
            /* n = 0: exp(-gamma(r_0, r_d, E_0)) */
            ap->s_prim[w * nq + q] = exp(-mu0 * m->gam_det_q[(size_t)a * nq + q]);
            for (int p = 0; p < np; p++) {
                size_t k = ((size_t)w * nq + q) * np + p;
                if (m->p_cell[p] == own_cell) {
                    ap->s_scat[k] = 0.0;
                    ap->e_scat[k] = e0;
                    continue;
                }
                double d = m->dist_qp[(size_t)q * np + p];
                double ux = (m->p_x[p] - xq) * m->p.h / d, uy = (m->p_y[p] - yq) * m->p.h / d;
                double cos_t = ux * ca + uy * sa;
                double e1 = orc_compton_energy(e0, cos_t);
                double mu1 = orc_mu_water(m, e1);
                /* n = 1: exp(-gamma(r_0,r_1,E_0) - gamma(r_1,r_d,E_1)) x Delta x K */
                double att = exp(-mu0 * m->gam_qp[(size_t)q * np + p]
                                 - mu1 * m->gam_det_p[(size_t)a * np + p]);
                double interact = m->p_rho[p] * mu0 * m->cell_area / (2.0 * ORC_PI * d);
                double kn = 2.0 * ORC_PI * orc_kn_shape(e0, cos_t) / m->kn_norm[w];
                ap->s_scat[k] = att * interact * kn;
                ap->e_scat[k] = e1;
            }
        }
    }
}

static void angle_paths_free(angle_paths* ap) {
    free(ap->s_prim); free(ap->s_scat); free(ap->e_scat);
    free(ap->u_q); free(ap->sig_q); free(ap->u_p); free(ap->sig_p);
}

/* Row of the system matrix for one event at angle ap->a:
 *   row[q] = sum_w alpha_w sum_{P in P_q} pr(A_j | P, E_0^w) s(P, E_0^w)
 * (the per-voxel numerator terms of Eq. z_bar_update_os without lambda). */
static void event_row(const orc_model* m, const angle_paths* ap, int b, double e_hat,
                      double* row, double* c_p /* scratch [np] */) {
    const int nq = m->nq, np = m->np, W = m->p.n_lines;
    for (int p = 0; p < np; p++) c_p[p] = orc_bin_prob(m, b, ap->u_p[p], ap->sig_p[p]);
    for (int q = 0; q < nq; q++) {
        double c_q = orc_bin_prob(m, b, ap->u_q[q], ap->sig_q[q]);
        double acc = 0.0;
        for (int w = 0; w < W; w++) {
            double e0 = m->p.line_e[w];
            double sum_w = ap->s_prim[w * nq + q] * c_q * orc_energy_density(m, e_hat, e0);
            const double* s = ap->s_scat + ((size_t)w * nq + q) * np;
            const double* e1 = ap->e_scat + ((size_t)w * nq + q) * np;
            for (int p = 0; p < np; p++)
                if (s[p] != 0.0) sum_w += s[p] * c_p[p] * orc_energy_density(m, e_hat, e1[p]);
            acc += m->p.line_yield[w] * sum_w;
        }
        row[q] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Public event-level operations                                        */
/* ------------------------------------------------------------------ */

/* One row (support voxels in raster order). */
void orc_row(const orc_model* m, int a, int b, double e_hat, double* out_row) {
    angle_paths ap;
    angle_paths_build(m, a, &ap);
    double* c_p = (double*)malloc(sizeof(double) * (m->np > 0 ? m->np : 1));
    event_row(m, &ap, b, e_hat, out_row, c_p);
    free(c_p);
    angle_paths_free(&ap);
}

/* Single-scatter part of one line's row for one event:
 *   out[q] = alpha_w sum_{P, n = 1} pr(A_j | P, E_0^w) s(P, E_0^w)
 * i.e. the n = 1 paths of Eq. (s_p) summed over the scatter points, times the
 * detector response (the quantity the learned surrogate is trained on). */
void orc_scatter_line_row(const orc_model* m, int a, int b, double e_hat, int w, double* out_row) {
    angle_paths ap;
    angle_paths_build(m, a, &ap);
    const int nq = m->nq, np = m->np;
    double* c_p = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    for (int p = 0; p < np; p++) c_p[p] = orc_bin_prob(m, b, ap.u_p[p], ap.sig_p[p]);
    for (int q = 0; q < nq; q++) {
        const double* s = ap.s_scat + ((size_t)w * nq + q) * np;
        const double* e1 = ap.e_scat + ((size_t)w * nq + q) * np;
        double acc = 0.0;
        for (int p = 0; p < np; p++)
            if (s[p] != 0.0) acc += s[p] * c_p[p] * orc_energy_density(m, e_hat, e1[p]);
        out_row[q] = m->p.line_yield[w] * acc;
    }
    free(c_p);
    angle_paths_free(&ap);
}

/* Path sensitivities of one detector angle, as angle_paths holds them:
 * s_prim [W][nq] and s_scat, e_scat [W][nq][np] (Eq. s_p with n = 0 and
 * n = 1; s_scat is 0 for the emission voxel's own cell), the detector
 * coordinate and collimator blur of every voxel (u_q, sig_q [nq]) and scatter
 * point (u_p, sig_p [np]).  Used by the model-consistent event sampler. */
void orc_angle_paths(const orc_model* m, int a, double* s_prim, double* s_scat, double* e_scat,
                     double* u_q, double* sig_q, double* u_p, double* sig_p) {
    const size_t W = (size_t)m->p.n_lines, nq = (size_t)m->nq, np = (size_t)m->np;
    angle_paths ap;
    angle_paths_build(m, a, &ap);
    memcpy(s_prim, ap.s_prim, sizeof(double) * W * nq);
    if (np > 0) {
        memcpy(s_scat, ap.s_scat, sizeof(double) * W * nq * np);
        memcpy(e_scat, ap.e_scat, sizeof(double) * W * nq * np);
        memcpy(u_p, ap.u_p, sizeof(double) * np);
        memcpy(sig_p, ap.sig_p, sizeof(double) * np);
    }
    memcpy(u_q, ap.u_q, sizeof(double) * nq);
    memcpy(sig_q, ap.sig_q, sizeof(double) * nq);
    angle_paths_free(&ap);
}

/* Visit events angle by angle: build s(P) for that angle once, then hand
 * each event's row to a callback together with the index of the thread that
 * computed it (callbacks keep per-thread partial sums). */
typedef void (*row_fn)(void* ctx, int tid, int64_t j, const double* row);

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

static void for_each_row(const orc_model* m, int64_t n_ev, const uint16_t* angle,
                         const uint16_t* bin, const float* energy, const uint8_t* use,
                         row_fn fn, void* ctx) {
    const int A = m->p.n_angles;
    int64_t* count = (int64_t*)calloc(A + 1, sizeof(int64_t));
    for (int64_t j = 0; j < n_ev; j++) if (!use || use[j]) count[angle[j] + 1]++;
    for (int a = 0; a < A; a++) count[a + 1] += count[a];
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (count[A] > 0 ? count[A] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * A);
    for (int a = 0; a < A; a++) fill[a] = count[a];
    for (int64_t j = 0; j < n_ev; j++) if (!use || use[j]) order[fill[angle[j]]++] = j;
    for (int a = 0; a < A; a++) {
        if (count[a + 1] == count[a]) continue;
        angle_paths ap;
        angle_paths_build(m, a, &ap);
#pragma omp parallel
        {
            double* row = (double*)malloc(sizeof(double) * (m->nq > 0 ? m->nq : 1));
            double* c_p = (double*)malloc(sizeof(double) * (m->np > 0 ? m->np : 1));
            int tid = thread_id();
#pragma omp for schedule(dynamic, 1)
            for (int64_t k = count[a]; k < count[a + 1]; k++) {
                int64_t j = order[k];
                event_row(m, &ap, bin[j], energy[j], row, c_p);
                fn(ctx, tid, j, row);
            }
            free(row); free(c_p);
        }
        angle_paths_free(&ap);
    }
    free(count); free(order); free(fill);
}

typedef struct { const orc_model* m; const double* lam; double* y; } fwd_ctx;
static void fwd_cb(void* c, int tid, int64_t j, const double* row) {
    fwd_ctx* x = (fwd_ctx*)c;
    (void)tid;
    double s = 0.0;
    for (int q = 0; q < x->m->nq; q++) s += row[q] * x->lam[x->m->q_pix[q]];
    x->y[j] = s;
}

/* y_j = sum_q row_j[q] lambda_q (the denominator of Eq. z_bar_update_os). */
void orc_forward(const orc_model* m, int64_t n_ev, const uint16_t* angle, const uint16_t* bin,
                 const float* energy, const double* lam, double* y) {
    fwd_ctx c = {m, lam, y};
    for_each_row(m, n_ev, angle, bin, energy, NULL, fwd_cb, &c);
}

/* per-thread partial sums over voxels, added in thread order at the end */
static double* partials_new(const orc_model* m) {
    return (double*)calloc((size_t)n_threads() * (m->nq > 0 ? m->nq : 1), sizeof(double));
}
static void partials_reduce(const orc_model* m, const double* part, double* acc) {
    for (int q = 0; q < m->nq; q++) acc[q] = 0.0;
    for (int t = 0; t < n_threads(); t++)
        for (int q = 0; q < m->nq; q++) acc[q] += part[(size_t)t * m->nq + q];
}

typedef struct { const orc_model* m; const double* wt; double* part; } bp_ctx;
static void bp_cb(void* c, int tid, int64_t j, const double* row) {
    bp_ctx* x = (bp_ctx*)c;
    double* acc = x->part + (size_t)tid * x->m->nq;
    if (x->wt[j] == 0.0) return;
    for (int q = 0; q < x->m->nq; q++) acc[q] += x->wt[j] * row[q];
}

/* out[pixel(q)] = sum_j weight_j row_j[q]; pixels outside the voxel set = 0. */
void orc_backproject(const orc_model* m, int64_t n_ev, const uint16_t* angle, const uint16_t* bin,
                     const float* energy, const double* weight, double* out) {
    double* part = partials_new(m);
    double* acc = (double*)calloc(m->nq > 0 ? m->nq : 1, sizeof(double));
    bp_ctx c = {m, weight, part};
    for_each_row(m, n_ev, angle, bin, energy, NULL, bp_cb, &c);
    partials_reduce(m, part, acc);
    memset(out, 0, sizeof(double) * m->p.n * m->p.n);
    for (int q = 0; q < m->nq; q++) out[m->q_pix[q]] = acc[q];
    free(acc); free(part);
}

/* Sensitivity of subset `subset` (angles a with a mod n_subsets == subset;
 * subset < 0 = all angles):
 *   sens[q] = T sum_{a in subset} sum_w alpha_w sum_{P in P_q} s(P, E_0^w)
 *             x (probability that pr(A|P,E) falls on the detector and inside a window)
 * i.e. the denominator of Eq. os-lm-mlem. */
void orc_sensitivity(const orc_model* m, int subset, int n_subsets, double* out) {
    const int nq = m->nq, np = m->np, W = m->p.n_lines;
    double* acc = (double*)calloc(nq > 0 ? nq : 1, sizeof(double));
    for (int a = 0; a < m->p.n_angles; a++) {
        if (subset >= 0 && (a % n_subsets) != subset) continue;
        angle_paths ap;
        angle_paths_build(m, a, &ap);
#pragma omp parallel for schedule(static)
        for (int q = 0; q < nq; q++) {
            double tot = 0.0;
            for (int w = 0; w < W; w++) {
                double e0 = m->p.line_e[w];
                double sum_w = ap.s_prim[w * nq + q] * orc_detector_mass(m, ap.u_q[q], ap.sig_q[q])
                               * orc_window_mass(m, e0);
                const double* s = ap.s_scat + ((size_t)w * nq + q) * np;
                const double* e1 = ap.e_scat + ((size_t)w * nq + q) * np;
                for (int p = 0; p < np; p++)
                    if (s[p] != 0.0)
                        sum_w += s[p] * orc_detector_mass(m, ap.u_p[p], ap.sig_p[p]) * orc_window_mass(m, e1[p]);
                tot += m->p.line_yield[w] * sum_w;
            }
            acc[q] += m->p.scan_time * tot;
        }
        angle_paths_free(&ap);
    }
    memset(out, 0, sizeof(double) * m->p.n * m->p.n);
    for (int q = 0; q < nq; q++) out[m->q_pix[q]] = acc[q];
    free(acc);
}

/* LM-OSEM, Eq. (os-lm-mlem) with (z_bar_update_os):
 *   for it in [start_iter, n_iters), s in [start_subset (first it only), N_s):
 *     y_j   = sum_q row_j[q] lambda_q                      (j in subset s)
 *     num_q = sum_{j in s, y_j > 0} row_j[q] / y_j
 *     lambda_q <- lambda_q num_q / sens_s[q]   (0 where sens_s[q] = 0)
 *   loglik[it*N_s + s] (optional) = sum_{j in s, y_j > 0} log y_j - sum_q lambda_q sens_s[q],
 *   evaluated at the image entering the sub-iteration (Eq. lll_med without the
 *   constants J log T - log J!).
 * Each event's row is built once per sub-iteration: y_j needs only that row,
 * and row / y_j is then added to the back projection.
 * lam is the n*n image, updated in place; pixels outside the voxel set are 0. */
typedef struct { const orc_model* m; const double* lam; double* y; double* part; } em_ctx;
static void em_cb(void* c, int tid, int64_t j, const double* row) {
    em_ctx* x = (em_ctx*)c;
    double s = 0.0;
    for (int q = 0; q < x->m->nq; q++) s += row[q] * x->lam[x->m->q_pix[q]];
    x->y[j] = s;
    if (!(s > 0.0)) return;
    double r = 1.0 / s;
    double* acc = x->part + (size_t)tid * x->m->nq;
    for (int q = 0; q < x->m->nq; q++) acc[q] += row[q] * r;
}

void orc_osem(const orc_model* m, int64_t n_ev, const uint16_t* angle, const uint16_t* bin,
              const float* energy, int n_subsets, int n_iters, int start_iter, int start_subset,
              double* lam, double* loglik) {
    const int nq = m->nq, npix = m->p.n * m->p.n;
    double* sens = (double*)malloc(sizeof(double) * (size_t)n_subsets * npix);
    for (int s = 0; s < n_subsets; s++) orc_sensitivity(m, s, n_subsets, sens + (size_t)s * npix);
    double* y = (double*)calloc(n_ev > 0 ? n_ev : 1, sizeof(double));
    double* acc = (double*)malloc(sizeof(double) * (nq > 0 ? nq : 1));
    double* part = partials_new(m);
    uint8_t* use = (uint8_t*)malloc(n_ev > 0 ? n_ev : 1);
    {
        uint8_t* in = (uint8_t*)calloc(npix, 1);
        for (int q = 0; q < nq; q++) in[m->q_pix[q]] = 1;
        for (int i = 0; i < npix; i++) if (!in[i]) lam[i] = 0.0;
        free(in);
    }
    for (int it = start_iter; it < n_iters; it++) {
        for (int s = (it == start_iter ? start_subset : 0); s < n_subsets; s++) {
            for (int64_t j = 0; j < n_ev; j++) use[j] = (angle[j] % n_subsets) == s;
            memset(part, 0, sizeof(double) * (size_t)n_threads() * (nq > 0 ? nq : 1));
            em_ctx c = {m, lam, y, part};
            for_each_row(m, n_ev, angle, bin, energy, use, em_cb, &c);
            partials_reduce(m, part, acc);
            const double* sn = sens + (size_t)s * npix;
            if (loglik) {
                double ll = 0.0;
                for (int64_t j = 0; j < n_ev; j++) if (use[j] && y[j] > 0.0) ll += log(y[j]);
                for (int q = 0; q < nq; q++) ll -= lam[m->q_pix[q]] * sn[m->q_pix[q]];
                loglik[(size_t)it * n_subsets + s] = ll;
            }
            for (int q = 0; q < nq; q++) {
                int pix = m->q_pix[q];
                lam[pix] = (sn[pix] > 0.0) ? lam[pix] * acc[q] / sn[pix] : 0.0;
            }
        }
    }
    free(sens); free(y); free(acc); free(part); free(use);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the calling thread's later parallel regions (for timing the
 * oracle on one core and on all of them); ignored without OpenMP or n < 1. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
