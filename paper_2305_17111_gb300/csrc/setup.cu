// Model set-up on the GPU (once per lm_create): exact line integrals through
// the density map (Eq. radpath), path sensitivities s(P, E_0^w) of Eq. (s_p)
// for the unscattered and single-scatter paths of every (angle, voxel,
// scatter point, line), the collimator tables and the per-angle sensitivity
// image (denominator of Eq. os-lm-mlem).  Arithmetic is FP64, and every sum
// is accumulated in FP64; inside each scatter-path term the window masses,
// the attenuation factor's 2^-fraction and the mantissa's log2 are FP32
// (about 2e-7 relative per term).  The tables the hot kernel streams are
// rounded to FP32 at the end.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMeC2 = 510.99895;     // electron rest energy, keV
constexpr double kLog2e = 1.4426950408889634;

__device__ __forceinline__ double mu_water(const ModelConst& m, double e) {
    if (m.n_knots == 1) return m.knot_mu[0];
    int s = 0;
    while (s < m.n_knots - 2 && e >= m.knot_e[s + 1]) ++s;
    return m.knot_mu[s] + (e - m.knot_e[s]) * m.knot_slope[s];
}

// sigma of the energy response: FWHM = frac * E * (E / E_ref)^expo.  For the
// usual expo = -1/2 this is frac * sqrt(E * E_ref): a square root instead of
// an FP64 power (the same value to rounding).
__host__ __device__ __forceinline__ double sigma_energy(double frac, double e_ref, double expo,
                                                        double e) {
    const double fwhm = expo == -0.5 ? frac * sqrt(e * e_ref) : frac * e * pow(e / e_ref, expo);
    return fwhm / (2.0 * sqrt(2.0 * log(2.0)));
}

// 1/x and 1/sqrt(x) for positive normal x well inside the FP32 range: the
// FP32 estimate y refined by one Newton-Raphson step in FP64, for 1/x
// y (2 - x y) and for 1/sqrt(x) y (3/2 - x y^2 / 2).  A relative error e of y
// becomes about e^2 (1.5 e^2 for the square root), here ~1e-13: far below
// the FP32 rounding of every table entry they feed.
__device__ __forceinline__ double recip_nr(double x) {
    const double y = (double)(1.0f / (float)x);
    return y * fma(-x, y, 2.0);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
    const double y = (double)rsqrtf((float)x);
    return y * fma(-0.5 * x * y, y, 1.5);
}

// 1 / sigma of the energy response; for expo = -1/2 one reciprocal square root.
__device__ __forceinline__ double inv_sigma_energy(double frac, double e_ref, double expo,
                                                   double e) {
    constexpr double kFwhmToSigma = 2.3548200450309493;   // 2 sqrt(2 ln 2)
    if (expo == -0.5) return rsqrt_nr(e * e_ref) * (kFwhmToSigma / frac);
    return 1.0 / sigma_energy(frac, e_ref, expo, e);
}

// 2^-t: t = n + f with n = floor(t) taken exactly in FP64, 2^-f of the
// fraction in FP32, then scaled by 2^-n exactly.  Relative error about 2e-7
// whatever the size of t; 0 once t >= 1000 (and for NaN).
__device__ __forceinline__ double pow2_neg(double t) {
    if (!(t < 1000.0)) return 0.0;
    const double n = floor(t);
    return ldexp((double)exp2f(-(float)(t - n)), -(int)n);
}

// log2 z for a positive FP32 z: z = mant * 2^e exactly (frexpf), log2 of
// the mantissa in [0.5, 1).  Absolute error about 1e-7 whatever the size of z.
__device__ __forceinline__ double log2_pos_f(float z) {
    int e;
    const float mant = frexpf(z, &e);
    return (double)e + (double)log2f(mant);
}

__device__ __forceinline__ double sigma_coll(const ModelConst& m, double depth) {
    return (m.fwhm0 + m.slope * depth) / (2.0 * sqrt(2.0 * log(2.0)));
}

// Gaussian mass on [lo, hi]; erfc on the tail side keeps small masses accurate.
__device__ __forceinline__ double gauss_mass(double lo, double hi, double mean, double sigma) {
    const double inv = 1.0 / (sqrt(2.0) * sigma);
    const double a = (lo - mean) * inv, b = (hi - mean) * inv;
    if (a >= 0.0) return 0.5 * (erfc(a) - erfc(b));
    if (b <= 0.0) return 0.5 * (erfc(-b) - erfc(-a));
    return 0.5 * (erf(b) - erf(a));
}

// Mass of the energy response to E (sigma s) inside the windows.
__device__ __forceinline__ double window_mass(const ModelConst& m, double e, double s) {
    double t = 0.0;
    for (int k = 0; k < m.n_win; ++k) t += gauss_mass(m.win_lo[k], m.win_hi[k], e, s);
    return t;
}
__device__ __forceinline__ double window_mass(const ModelConst& m, double e) {
    return window_mass(m, e, sigma_energy(m.fwhm_frac, m.e_ref, m.expo, e));
}

// The same window mass in FP32 (a per-term probability of the sensitivity;
// the sensitivity itself is accumulated in FP64).
__device__ __forceinline__ float gauss_mass_f(float lo, float hi, float mean, float sigma) {
    const float inv = 1.0f / (1.41421356f * sigma);
    const float a = (lo - mean) * inv, b = (hi - mean) * inv;
    if (a >= 0.f) return 0.5f * (erfcf(a) - erfcf(b));
    if (b <= 0.f) return 0.5f * (erfcf(-b) - erfcf(-a));
    return 0.5f * (erff(b) - erff(a));
}
__device__ __forceinline__ float window_mass_f(const ModelConst& m, float e, float s) {
    float t = 0.f;
    for (int k = 0; k < m.n_win; ++k) t += gauss_mass_f((float)m.win_lo[k], (float)m.win_hi[k], e, s);
    return t;
}


// Integral over [0, 2 pi) of the KN shape, in closed form: with a = 1 + k,
// b = k, D = a^2 - b^2, int dth/(a - b cos) = 2 pi / sqrt(D),
// int dth/(a - b cos)^3 = pi (2a^2 + b^2) / D^(5/2) and, by parts,
// int sin^2/(a - b cos)^2 = (a int 1/(a - b cos) - 2 pi) / b^2.
__device__ double kn_plane_norm(double e) {
    const double k = e / kMeC2;
    if (k < 1e-4) return 3.0 * kPi * (1.0 - 2.0 * k);   // Thomson limit + first order
    const double a = 1.0 + k, b = k, d = 1.0 + 2.0 * k;
    const double i1 = 2.0 * kPi / sqrt(d);
    const double i3 = kPi * (2.0 * a * a + b * b) * pow(d, -2.5);
    return i3 + i1 - (a * i1 - 2.0 * kPi) / (b * b);
}

__device__ __forceinline__ double rho_pix(const float* rho, int n, int ix, int iy) {
    return (ix < 0 || iy < 0 || ix >= n || iy >= n) ? 0.0 : (double)rho[iy * n + ix];
}

// Exact integral of the pixelwise-constant density along the segment
// (x0,y0)->(x1,y1), pixel units from the image corner, result in pixel
// lengths.  Incremental grid walk: the next vertical and horizontal grid
// crossings are tracked, every piece between consecutive crossings lies in
// one pixel (looked up at the piece's midpoint).  A ray running exactly
// along a grid line takes the mean of the pixels on its two sides.
__device__ double seg_integral(const float* rho, int n, double x0, double y0, double x1,
                               double y1) {
    const double dx = x1 - x0, dy = y1 - y0;
    const double len = sqrt(dx * dx + dy * dy);
    if (len == 0.0) return 0.0;
    double tmin = 0.0, tmax = 1.0;
    if (dx == 0.0) {
        if (x0 < 0.0 || x0 > n) return 0.0;
    } else {
        double ta = -x0 / dx, tb = (n - x0) / dx;
        if (ta > tb) { const double t = ta; ta = tb; tb = t; }
        tmin = fmax(tmin, ta);
        tmax = fmin(tmax, tb);
    }
    if (dy == 0.0) {
        if (y0 < 0.0 || y0 > n) return 0.0;
    } else {
        double ta = -y0 / dy, tb = (n - y0) / dy;
        if (ta > tb) { const double t = ta; ta = tb; tb = t; }
        tmin = fmax(tmin, ta);
        tmax = fmin(tmax, tb);
    }
    if (!(tmax > tmin)) return 0.0;
    const bool vline = (dx == 0.0 && x0 == floor(x0));
    const bool hline = (dy == 0.0 && y0 == floor(y0));
    const int sx = dx > 0.0 ? 1 : (dx < 0.0 ? -1 : 0);
    const int sy = dy > 0.0 ? 1 : (dy < 0.0 ? -1 : 0);
    const double xs = x0 + tmin * dx, ys = y0 + tmin * dy;
    int kx = sx > 0 ? (int)floor(xs) + 1 : (int)ceil(xs) - 1;
    int ky = sy > 0 ? (int)floor(ys) + 1 : (int)ceil(ys) - 1;
    double tx = sx ? (kx - x0) / dx : 2.0 * tmax + 1.0;
    double ty = sy ? (ky - y0) / dy : 2.0 * tmax + 1.0;
    double t = tmin, acc = 0.0;
    for (int guard = 0; guard < 4 * n + 16 && t < tmax; ++guard) {
        const double tn = fmin(fmin(tx, ty), tmax);
        if (tn > t) {
            const double tm = 0.5 * (t + tn);
            const double px = x0 + tm * dx, py = y0 + tm * dy;
            double r;
            if (vline) {
                const int ix = (int)x0, iy = (int)floor(py);
                r = 0.5 * (rho_pix(rho, n, ix - 1, iy) + rho_pix(rho, n, ix, iy));
            } else if (hline) {
                const int iy = (int)y0, ix = (int)floor(px);
                r = 0.5 * (rho_pix(rho, n, ix, iy - 1) + rho_pix(rho, n, ix, iy));
            } else {
                r = rho_pix(rho, n, (int)floor(px), (int)floor(py));
            }
            acc += (tn - t) * r;
        }
        t = tn;
        if (sx && tn == tx) { kx += sx; tx = (kx - x0) / dx; }
        if (sy && tn == ty) { ky += sy; ty = (ky - y0) / dy; }
    }
    return acc * len;
}

__device__ __forceinline__ int n_of(const ModelConst& m) { return m.n; }

__device__ __forceinline__ double det_integral(const float* rho, int n, double x, double y,
                                               double c, double s) {
    const double far = 4.0 * n + 8.0;
    return seg_integral(rho, n, x, y, x + far * c, y + far * s);
}

// ---------------------------------------------------------------- kernels

__global__ void k_line_consts(ModelConst m, double* out /* [W][4] */) {
    const int w = threadIdx.x;
    if (w >= m.W) return;
    const double e = m.line_e[w];
    const double s = sigma_energy(m.fwhm_frac, m.e_ref, m.expo, e);
    out[w * 4 + 0] = kn_plane_norm(e);
    out[w * 4 + 1] = -kLog2e / (2.0 * s * s);
    out[w * 4 + 2] = 1.0 / (sqrt(2.0 * kPi) * s);
    out[w * 4 + 3] = mu_water(m, e);
}

__global__ void k_cell_means(const float* rho, int n, int S, double* mean) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S * S) return;
    const int f = n / S, mx = c % S, my = c / S;
    double sum = 0.0;
    for (int iy = my * f; iy < (my + 1) * f; ++iy)
        for (int ix = mx * f; ix < (mx + 1) * f; ++ix) sum += rho[iy * n + ix];
    mean[c] = sum / (double)(f * f);
}

// Detector-leg path integrals (cm) for voxels and scatter points.
__global__ void k_gamma_det(ModelConst m, const float* rho, const double* cs_a,
                            const int* q_pix, const int* p_cell, double* g_q, double* g_p) {
    const int a = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.nq + m.np) return;
    double x, y;
    if (i < m.nq) {
        const int pix = q_pix[i];
        x = (pix % m.n) + 0.5;
        y = (pix / m.n) + 0.5;
    } else {
        const int c = p_cell[i - m.nq];
        x = ((c % m.S) + 0.5) * m.f;
        y = ((c / m.S) + 0.5) * m.f;
    }
    const double g = m.h * det_integral(rho, m.n, x, y, cs_a[2 * a], cs_a[2 * a + 1]);
    if (i < m.nq) g_q[(size_t)a * m.nq + i] = g;
    else g_p[(size_t)a * m.np + (i - m.nq)] = g;
}

// Path features of the learned scatter surrogate: for every (angle, voxel)
// the line integral of rho (cm) from the voxel centre to the image edge along
// the 8 directions theta_a + k pi/4.
__global__ void k_gamma8(ModelConst m, const float* rho, const int* q_pix, float* g8) {
    const int a = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m.nq) return;
    const int pix = q_pix[q];
    const double x = (pix % m.n) + 0.5, y = (pix / m.n) + 0.5;
    for (int k = 0; k < 8; ++k) {
        const double th = 2.0 * kPi * a / m.A + k * 0.25 * kPi;
        g8[((size_t)a * m.nq + q) * 8 + k] = (float)(m.h * det_integral(rho, n_of(m), x, y, cos(th), sin(th)));
    }
}

// Emission-to-scatter path integrals and distances (cm).
__global__ void k_gamma_qp(ModelConst m, const float* rho, const int* q_pix, const int* p_cell,
                           double* g_qp, double* d_qp) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)m.nq * m.np) return;
    const int q = (int)(k / m.np), p = (int)(k % m.np);
    const int pix = q_pix[q], c = p_cell[p];
    const double xq = (pix % m.n) + 0.5, yq = (pix / m.n) + 0.5;
    const double xp = ((c % m.S) + 0.5) * m.f, yp = ((c / m.S) + 0.5) * m.f;
    g_qp[k] = m.h * seg_integral(rho, m.n, xq, yq, xp, yp);
    d_qp[k] = m.h * sqrt((xp - xq) * (xp - xq) + (yp - yq) * (yp - yq));
}

__device__ __forceinline__ void point_cm(const ModelConst& m, bool voxel, int idx, const int* q_pix,
                                         const int* p_cell, double* x, double* y) {
    if (voxel) {
        const int pix = q_pix[idx];
        *x = ((pix % m.n) + 0.5 - 0.5 * m.n) * m.h;
        *y = ((pix / m.n) + 0.5 - 0.5 * m.n) * m.h;
    } else {
        const int c = p_cell[idx];
        *x = (((c % m.S) + 0.5) * m.f - 0.5 * m.n) * m.h;
        *y = (((c / m.S) + 0.5) * m.f - 0.5 * m.n) * m.h;
    }
}

// Per angle, the scatter points in ascending order of their detector
// coordinate u (ties by index): inv[a][r] = point of rank r.  In this order
// the points a bin can see form one contiguous run.
__global__ void k_point_order(ModelConst m, const double* cs_a, const int* p_cell, int* inv) {
    const int a = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.np) return;
    const double c = cs_a[2 * a], s = cs_a[2 * a + 1];
    double x, y;
    point_cm(m, false, p, nullptr, p_cell, &x, &y);
    const double u = -x * s + y * c;
    int rank = 0;
    for (int o = 0; o < m.np; ++o) {
        double xo, yo;
        point_cm(m, false, o, nullptr, p_cell, &xo, &yo);
        const double uo = -xo * s + yo * c;
        rank += (uo < u || (uo == u && o < p)) ? 1 : 0;
    }
    inv[(size_t)a * m.np + rank] = p;
}

// Collimator bin probabilities: voxels [A][B][nq], scatter points [A][npc][B][kCPad]
// with the points of each angle in the order of k_point_order (k_chunk_range
// then applies the floor to the scatter points).
__global__ void k_collimator(ModelConst m, const double* cs_a, const int* q_pix,
                             const int* p_cell, const int* inv, float* cv, float* csp) {
    const int a = blockIdx.z, b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_p_pad = m.npc * kPC;
    if (i >= m.nq + n_p_pad) return;
    const double c = cs_a[2 * a], s = cs_a[2 * a + 1];
    const double lo = -0.5 * m.B * m.bin_w + b * m.bin_w, hi = lo + m.bin_w;
    if (i < m.nq) {
        double x, y;
        point_cm(m, true, i, q_pix, p_cell, &x, &y);
        const double u = -x * s + y * c, sg = sigma_coll(m, m.r_det - (x * c + y * s));
        cv[((size_t)a * m.B + b) * m.nq + i] = (float)gauss_mass(lo, hi, u, sg);
    } else {
        const int r = i - m.nq;   // rank of the point in this angle's order
        float val = 0.f;
        if (r < m.np) {
            double x, y;
            point_cm(m, false, inv[(size_t)a * m.np + r], q_pix, p_cell, &x, &y);
            const double u = -x * s + y * c, sg = sigma_coll(m, m.r_det - (x * c + y * s));
            val = (float)gauss_mass(lo, hi, u, sg);
        }
        const int pc = r / kPC, pl = r % kPC;
        csp[(((size_t)a * m.npc + pc) * m.B + b) * kCPad + pl] = val;
    }
}

// For every (angle, bin): the floor on the scatter points' collimator
// probabilities, then the run of ordered points whose probability for that
// bin is non-zero, as [first, last + 1) (0, 0 if none).
__global__ void k_chunk_range(ModelConst m, float* csp, int2* range) {
    const int a = blockIdx.y;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m.B) return;
    auto at = [&](int r) -> float& {
        return csp[(((size_t)a * m.npc + r / kPC) * m.B + b) * kCPad + (r % kPC)];
    };
    // probabilities below kCollimatorFloorRel of this (angle, bin)'s largest become 0
    float vmax = 0.f;
    for (int r = 0; r < m.np; ++r) vmax = fmaxf(vmax, at(r));
    const float floor_ab = kCollimatorFloorRel * vmax;
    int first = -1, last = -1;
    for (int r = 0; r < m.np; ++r) {
        float& v = at(r);
        if (v < floor_ab) v = 0.f;
        if (v != 0.f) {
            if (first < 0) first = r;
            last = r;
        }
    }
    range[(size_t)a * m.B + b] = first < 0 ? make_int2(0, 0) : make_int2(first, last + 1);
}

// Unscattered paths: prim[a][w][q] = alpha_w exp(-mu_w(E_w) gamma_det) and the
// primary part of the per-angle sensitivity.
__global__ void k_primary(ModelConst m, const double* cs_a, const int* q_pix, const double* g_q,
                          const double* mu_line, float* prim, double* sens_a) {
    const int a = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m.nq) return;
    double x, y;
    point_cm(m, true, q, q_pix, nullptr, &x, &y);
    const double c = cs_a[2 * a], s = cs_a[2 * a + 1];
    const double u = -x * s + y * c, sg = sigma_coll(m, m.r_det - (x * c + y * s));
    const double on_det = gauss_mass(-0.5 * m.B * m.bin_w, 0.5 * m.B * m.bin_w, u, sg);
    double sens = 0.0;
    for (int w = 0; w < m.W; ++w) {
        const double v = m.alpha[w] * exp(-mu_line[w] * g_q[(size_t)a * m.nq + q]);
        prim[((size_t)a * m.W + w) * m.nq + q] = (float)v;
        sens += v * on_det * window_mass(m, m.line_e[w]);
    }
    sens_a[(size_t)a * m.nq + q] = m.T * sens;
}

// Single-scatter paths.  One warp per (angle, voxel), lanes over scatter
// points.  Writes the FP32 hot-kernel tables in the square-root form of the
// energy Gaussian, alpha_w s(P) g(E_hat; E') = 2^-(d^2 + nlh) with
//   d = sr E_hat + m,  sr = sqrt(log2(e) / 2) / sigma_E(E'),  m = -sr E',
//   nlh = -log2(alpha_w s(P) / (sqrt(2 pi) sigma_E(E')))
// (sr and m rounded once from FP64, so sr E_hat + m in one FMA carries the
// same error as E_hat - E' with E' rounded), and adds sum_w alpha_w sum_p s(P) Prob(detector) Prob(window | E') to the
// per-angle sensitivity.
// Collimator mass on the whole detector of every scatter point at every
// angle (it does not depend on the emission voxel): on_det[a][p].
__global__ void k_on_detector(ModelConst m, const double* cs_a, const int* p_cell, double* on_det) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (p >= m.np) return;
    const double c = cs_a[2 * a], s = cs_a[2 * a + 1];
    const int cell = p_cell[p];
    const double xp = ((cell % m.S) + 0.5) * m.f, yp = ((cell / m.S) + 0.5) * m.f;
    const double xpc = (xp - 0.5 * m.n) * m.h, ypc = (yp - 0.5 * m.n) * m.h;
    const double half_det = 0.5 * m.B * m.bin_w;
    on_det[(size_t)a * m.np + p] =
        gauss_mass(-half_det, half_det, -xpc * s + ypc * c,
                   sigma_coll(m, m.r_det - (xpc * c + ypc * s)));
}

// Block (x, y): 8 voxels (a warp each) of angle a0 + y astep, whose tables go
// to slot y of tab; with kSens the angle's scatter sensitivity is added to
// sens_a (the set-up pass over every angle), without it only the tables are
// written (a streamed angle block rebuilt; the same table values).
template <bool kSens>
__global__ void __launch_bounds__(256) k_scatter(ModelConst m, int a0, int astep,
                                                 const double* cs_a, const int* q_pix,
                                                 const int* p_cell, const double* p_rho,
                                                 const double* g_qp, const double* d_qp,
                                                 const double* g_p, const double* mu_line,
                                                 const int* inv, const double* on_det, float* tab,
                                                 double* sens_a) {
    const int slot = blockIdx.y, a = a0 + slot * astep;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 8 + warp;
    if (q >= m.nq) return;
    const double c = cs_a[2 * a], s = cs_a[2 * a + 1];
    const int pix = q_pix[q];
    const int qx = pix % m.n, qy = pix / m.n;
    const int own_cell = (qy / m.f) * m.S + (qx / m.f);
    const double xq = qx + 0.5, yq = qy + 0.5;
    const int qt = q / kQT, ql = q % kQT;
    // per line: 1 / (in-plane KN normaliser) and E_w / (m_e c^2)
    float inv_kn[LMMEW_MAX_LINES];
    double k0[LMMEW_MAX_LINES];
    for (int w = 0; w < m.W; ++w) {
        inv_kn[w] = (float)(1.0 / m.kn_norm[w]);
        k0[w] = m.line_e[w] / kMeC2;
    }
    double sens = 0.0;
    for (int pc = 0; pc < m.npc; ++pc) {
        const int r = pc * kPC + lane;   // slot in this angle's point order
        float* base = tab + (((size_t)slot * m.nqt + qt) * m.npc + pc) * (size_t)(3 * m.W * kQT * kPC);
        if (r >= m.np) {
            for (int w = 0; w < m.W; ++w) {
                base[((0 * m.W + w) * kQT + ql) * kPC + lane] = kPosHuge;
                base[((1 * m.W + w) * kQT + ql) * kPC + lane] = 0.f;
                base[((2 * m.W + w) * kQT + ql) * kPC + lane] = 0.f;
            }
            continue;
        }
        const int p = inv[(size_t)a * m.np + r];
        const int cell = p_cell[p];
        if (cell == own_cell) {   // the emission voxel's own cell carries no path
            for (int w = 0; w < m.W; ++w) {
                base[((0 * m.W + w) * kQT + ql) * kPC + lane] = kPosHuge;
                base[((1 * m.W + w) * kQT + ql) * kPC + lane] = 0.f;
                base[((2 * m.W + w) * kQT + ql) * kPC + lane] = 0.f;
            }
            continue;
        }
        const double xp = ((cell % m.S) + 0.5) * m.f, yp = ((cell / m.S) + 0.5) * m.f;
        const size_t k = (size_t)q * m.np + p;
        const double d = d_qp[k];
        const double inv_d = 1.0 / d;
        const double ux = (xp - xq) * m.h * inv_d, uy = (yp - yq) * m.h * inv_d;
        const double cos_t = ux * c + uy * s;
        const double od = on_det[(size_t)a * m.np + p];
        const double gqp = g_qp[k], gp = g_p[(size_t)a * m.np + p];
        // rho_p A_p / (2 pi d) times the 2 pi of the in-plane KN density
        const float inter = (float)(p_rho[p] * m.cell_area * inv_d);
        const float sin2 = (float)(1.0 - cos_t * cos_t);
        for (int w = 0; w < m.W; ++w) {
            // s(P) = 2^-att * pre: att the attenuation of both legs in bits
            // (FP64: it is exponentiated), pre the scatter density, the KN
            // weight and the geometry (FP32 factors, ~2e-7 relative)
            const double e0 = m.line_e[w];
            const double den = 1.0 + k0[w] * (1.0 - cos_t);   // E_w / E'
            const double r = recip_nr(den);
            const double e1 = e0 * r;
            const double mu0 = mu_line[w], mu1 = mu_water(m, e1);
            // Klein-Nishina angular shape r^2 (r + 1/r - sin^2), r = E'/E_w
            const float rf = (float)r;
            const float kn = rf * rf * (rf + (float)den - sin2);
            const double att = (mu0 * gqp + mu1 * gp) * kLog2e;
            const float pre = inter * (float)mu0 * kn * inv_kn[w];
            const double path = pow2_neg(att) * (double)pre;
            const double inv_sg = inv_sigma_energy(m.fwhm_frac, m.e_ref, m.expo, e1);
            const float pref = (float)(m.alpha[w] * inv_sg) * 0.3989422804f;   // / sqrt(2 pi)
            const double wgt = (double)pref * path;
            const double sr = sqrt(0.5 * kLog2e) * inv_sg;
            // -log2(wgt) = att - log2(pref pre), without forming 2^-att
            base[((0 * m.W + w) * kQT + ql) * kPC + lane] =
                wgt > 0.0 ? (float)(att - log2_pos_f(pref * pre)) : kPosHuge;
            base[((1 * m.W + w) * kQT + ql) * kPC + lane] = wgt > 0.0 ? (float)sr : 0.f;
            base[((2 * m.W + w) * kQT + ql) * kPC + lane] = wgt > 0.0 ? (float)(-sr * e1) : 0.f;
            if (kSens && path > 0.0)
                sens += m.alpha[w] * path * od *
                        (double)window_mass_f(m, (float)e1, 1.0f / (float)inv_sg);
        }
    }
    if (kSens) {
        for (int o = 16; o > 0; o >>= 1) sens += __shfl_xor_sync(0xffffffffu, sens, o);
        if (lane == 0) sens_a[(size_t)a * m.nq + q] += m.T * sens;
    }
}

__global__ void k_sum_subsets(const double* sens_a, int A, int nq, int parts, double* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (q >= nq) return;
    double acc = 0.0;
    for (int a = s; a < A; a += parts) acc += sens_a[(size_t)a * nq + q];
    out[(size_t)s * nq + q] = acc;
}

__global__ void k_sum_all(const double* sens_a, int A, int nq, double* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double acc = 0.0;
    for (int a = 0; a < A; ++a) acc += sens_a[(size_t)a * nq + q];
    out[q] = acc;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace

int subset_sensitivity(lm_handle* h, int parts, cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int prim_only = h->scatter_model == 2 ? 1 : 0;
    if (h->sens_parts != parts || h->sens_prim_only != prim_only) {
        const double* src = prim_only ? h->d_sens_a_prim : h->d_sens_a;
        if (h->d_sens_sub) { cudaFree(h->d_sens_sub); h->d_sens_sub = nullptr; }
        const size_t bytes = sizeof(double) * (size_t)(parts + 1) * m.nq;
        if (cudaMalloc(&h->d_sens_sub, bytes) != cudaSuccess)
            return set_error(LMMEW_ERR_OOM, "cannot allocate subset sensitivities");
        dim3 g((m.nq + 255) / 256, parts);
        k_sum_subsets<<<g, 256, 0, st>>>(src, m.A, m.nq, parts, h->d_sens_sub);
        ++h->launches;
        k_sum_all<<<(m.nq + 255) / 256, 256, 0, st>>>(src, m.A, m.nq,
                                                       h->d_sens_sub + (size_t)parts * m.nq);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
        h->sens_parts = parts;
        h->sens_prim_only = prim_only;
    }
    return LMMEW_OK;
}

int build_tables(lm_handle* h, const float* rho_host, const uint8_t* support_host) {
    ModelConst& m = h->mc;
    const int n = m.n;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, 0);

    // support voxel list (raster order)
    std::vector<int> q_pix;
    for (int i = 0; i < n * n; ++i)
        if (support_host ? support_host[i] != 0 : rho_host[i] > 0.f) q_pix.push_back(i);
    m.nq = (int)q_pix.size();
    if (m.nq == 0) return set_error(LMMEW_ERR_INVALID_ARG, "the support holds no voxel");
    m.nqt = (m.nq + kQT - 1) / kQT;

    DevBuf d_rho, d_cs_a, d_cell_mean, d_p_cell, d_p_rho, d_gq, d_gp, d_gqp, d_dqp, d_lc;
    LMMEW_CUDA(cudaMalloc(&d_rho.p, sizeof(float) * n * n));
    LMMEW_CUDA(cudaMemcpy(d_rho.p, rho_host, sizeof(float) * n * n, cudaMemcpyHostToDevice));
    const float* rho = (const float*)d_rho.p;

    // scatter points: cells with positive mean density (raster order)
    std::vector<int> p_cell;
    std::vector<double> p_rho;
    if (m.S > 0) {
        LMMEW_CUDA(cudaMalloc(&d_cell_mean.p, sizeof(double) * m.S * m.S));
        k_cell_means<<<(m.S * m.S + 255) / 256, 256>>>(rho, n, m.S, (double*)d_cell_mean.p);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
        std::vector<double> mean(m.S * m.S);
        LMMEW_CUDA(cudaMemcpy(mean.data(), d_cell_mean.p, sizeof(double) * m.S * m.S,
                              cudaMemcpyDeviceToHost));
        for (int c = 0; c < m.S * m.S; ++c)
            if (mean[c] > 0.0) { p_cell.push_back(c); p_rho.push_back(mean[c]); }
    }
    m.np = (int)p_cell.size();
    m.npc = (m.np + kPC - 1) / kPC;

    // The single-scatter path tables hold 3 floats per (angle, line, voxel,
    // scatter point), padded to 32-voxel x 32-point blocks: A W Q P x 12
    // bytes, next to the voxel-to-point line integrals and distances (Q P x
    // 16 bytes, kept to rebuild tables).  All angles stay resident when they
    // fit 90 % of the free memory (and the table budget); otherwise the
    // buffer holds as many angles as fit half of it (or the budget) and the
    // row launches rebuild the tables of the angles they need (streamed).
    // A model whose set-up and the tables of one angle do not fit is refused
    // here, before anything large is allocated.
    int tab_slots = m.A;
    const size_t per_angle = sizeof(float) * (size_t)m.nqt * m.npc * 3 * m.W * kQT * kPC;
    if (m.np) {
        const size_t tab = per_angle * (size_t)m.A;
        const size_t inter = 2 * sizeof(double) * (size_t)m.nq * m.np;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const bool over_budget = g_table_budget > 0 && tab > (size_t)g_table_budget;
            if (tab + inter > free_b / 10 * 9 || over_budget) {
                size_t cap = free_b > inter ? (free_b - inter) / 2 : 0;
                if (g_table_budget > 0) cap = std::min(cap, (size_t)g_table_budget);
                tab_slots = (int)std::min<size_t>((size_t)m.A, cap / per_angle);
            }
            if (tab_slots < 1)
                return set_error(LMMEW_ERR_OOM,
                                 "the path tables of one angle need " +
                                     std::to_string(per_angle >> 20) +
                                     " MiB (12 bytes x lines x voxels x scatter points) and their "
                                     "set-up " + std::to_string(inter >> 20) +
                                     " MiB more, beyond what the " + std::to_string(free_b >> 20) +
                                     " MiB free on the device (or the table budget) allow; use a "
                                     "coarser scatter grid");
        }
    }

    // collimator blur must stay positive for every point and angle
    {
        double rmax = 0.0;
        for (int pix : q_pix) {
            const double x = ((pix % n) + 0.5 - 0.5 * n) * m.h, y = ((pix / n) + 0.5 - 0.5 * n) * m.h;
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
        for (int c : p_cell) {
            const double x = (((c % m.S) + 0.5) * m.f - 0.5 * n) * m.h;
            const double y = (((c / m.S) + 0.5) * m.f - 0.5 * n) * m.h;
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
        const double lo = m.fwhm0 + m.slope * (m.r_det - rmax);
        const double hi = m.fwhm0 + m.slope * (m.r_det + rmax);
        if (!(lo > 0.0 && hi > 0.0))
            return set_error(LMMEW_ERR_INVALID_ARG,
                             "collimator FWHM is not positive at some depth of the model");
    }

    // detector directions, quarter turns exact
    std::vector<double> cs_a(2 * m.A);
    for (int a = 0; a < m.A; ++a) {
        if ((4 * a) % m.A == 0) {
            const int k = (4 * a) / m.A;
            const double cc[4] = {1, 0, -1, 0}, ss[4] = {0, 1, 0, -1};
            cs_a[2 * a] = cc[k];
            cs_a[2 * a + 1] = ss[k];
        } else {
            cs_a[2 * a] = cos(2.0 * kPi * a / m.A);
            cs_a[2 * a + 1] = sin(2.0 * kPi * a / m.A);
        }
    }
    LMMEW_CUDA(cudaMalloc(&d_cs_a.p, sizeof(double) * 2 * m.A));
    LMMEW_CUDA(cudaMemcpy(d_cs_a.p, cs_a.data(), sizeof(double) * 2 * m.A, cudaMemcpyHostToDevice));
    const double* dcs = (const double*)d_cs_a.p;

    LMMEW_CUDA(cudaMalloc(&h->d_q_pix, sizeof(int) * m.nq));
    LMMEW_CUDA(cudaMemcpy(h->d_q_pix, q_pix.data(), sizeof(int) * m.nq, cudaMemcpyHostToDevice));
    const int np_alloc = std::max(m.np, 1);
    LMMEW_CUDA(cudaMalloc(&d_p_cell.p, sizeof(int) * np_alloc));
    LMMEW_CUDA(cudaMalloc(&d_p_rho.p, sizeof(double) * np_alloc));
    if (m.np) {
        LMMEW_CUDA(cudaMemcpy(d_p_cell.p, p_cell.data(), sizeof(int) * m.np, cudaMemcpyHostToDevice));
        LMMEW_CUDA(cudaMemcpy(d_p_rho.p, p_rho.data(), sizeof(double) * m.np, cudaMemcpyHostToDevice));
    }

    // per-line constants: KN plane normaliser, energy response, mu at the line
    LMMEW_CUDA(cudaMalloc(&d_lc.p, sizeof(double) * 4 * LMMEW_MAX_LINES));
    k_line_consts<<<1, 32>>>(m, (double*)d_lc.p);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    double lc[4 * LMMEW_MAX_LINES];
    LMMEW_CUDA(cudaMemcpy(lc, d_lc.p, sizeof(lc), cudaMemcpyDeviceToHost));
    double mu_line_h[LMMEW_MAX_LINES];
    for (int w = 0; w < m.W; ++w) {
        m.kn_norm[w] = lc[4 * w + 0];
        h->lc.e[w] = (float)m.line_e[w];
        h->lc.nk[w] = (float)lc[4 * w + 1];
        h->lc.norm[w] = (float)lc[4 * w + 2];
        mu_line_h[w] = lc[4 * w + 3];
    }
    DevBuf d_mu_line;
    LMMEW_CUDA(cudaMalloc(&d_mu_line.p, sizeof(mu_line_h)));
    LMMEW_CUDA(cudaMemcpy(d_mu_line.p, mu_line_h, sizeof(mu_line_h), cudaMemcpyHostToDevice));
    const double* mu_line = (const double*)d_mu_line.p;

    for (int w = 0; w < m.W; ++w) h->mu_line[w] = mu_line_h[w];
    // surrogate path features and the density map they look up
    if (cudaMalloc(&h->d_g8, sizeof(float) * (size_t)m.A * m.nq * 8) != cudaSuccess ||
        cudaMalloc(&h->d_rho, sizeof(float) * (size_t)n * n) != cudaSuccess)
        return set_error(LMMEW_ERR_OOM, "cannot allocate path features");
    LMMEW_CUDA(cudaMemcpy(h->d_rho, rho, sizeof(float) * (size_t)n * n, cudaMemcpyDeviceToDevice));
    {
        dim3 g((m.nq + 127) / 128, m.A);
        k_gamma8<<<g, 128>>>(m, rho, h->d_q_pix, h->d_g8);
        LMMEW_CUDA(cudaGetLastError());
    }

    // path integrals
    LMMEW_CUDA(cudaMalloc(&d_gq.p, sizeof(double) * (size_t)m.A * m.nq));
    LMMEW_CUDA(cudaMalloc(&d_gp.p, sizeof(double) * (size_t)m.A * np_alloc));
    {
        dim3 g((m.nq + m.np + 127) / 128, m.A);
        k_gamma_det<<<g, 128>>>(m, rho, dcs, h->d_q_pix, (const int*)d_p_cell.p,
                                (double*)d_gq.p, (double*)d_gp.p);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
    }
    if (m.np) {
        const size_t k = (size_t)m.nq * m.np;
        LMMEW_CUDA(cudaMalloc(&d_gqp.p, sizeof(double) * k));
        LMMEW_CUDA(cudaMalloc(&d_dqp.p, sizeof(double) * k));
        k_gamma_qp<<<(unsigned)((k + 127) / 128), 128>>>(m, rho, h->d_q_pix,
                                                         (const int*)d_p_cell.p,
                                                         (double*)d_gqp.p, (double*)d_dqp.p);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
    }

    // per-angle point order
    DevBuf d_inv;
    LMMEW_CUDA(cudaMalloc(&d_inv.p, sizeof(int) * (size_t)m.A * np_alloc));
    if (m.np) {
        dim3 g((m.np + 127) / 128, m.A);
        k_point_order<<<g, 128>>>(m, dcs, (const int*)d_p_cell.p, (int*)d_inv.p);
        LMMEW_CUDA(cudaGetLastError());
    }
    const int* inv = (const int*)d_inv.p;

    // collimator tables
    const size_t cv_n = (size_t)m.A * m.B * m.nq;
    const size_t cs_n = (size_t)m.A * std::max(m.npc, 1) * m.B * kCPad;
    if (cudaMalloc(&h->d_cv, sizeof(float) * cv_n) != cudaSuccess ||
        cudaMalloc(&h->d_cs, sizeof(float) * cs_n) != cudaSuccess)
        return set_error(LMMEW_ERR_OOM, "cannot allocate collimator tables");
    LMMEW_CUDA(cudaMemset(h->d_cs, 0, sizeof(float) * cs_n));
    {
        dim3 g((m.nq + m.npc * kPC + 127) / 128, m.B, m.A);
        k_collimator<<<g, 128>>>(m, dcs, h->d_q_pix, (const int*)d_p_cell.p, inv, h->d_cv,
                                 h->d_cs);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
    }
    if (cudaMalloc(&h->d_crange, sizeof(int2) * (size_t)m.A * m.B) != cudaSuccess)
        return set_error(LMMEW_ERR_OOM, "cannot allocate chunk ranges");
    if (m.np) {
        dim3 g((m.B + 127) / 128, m.A);
        k_chunk_range<<<g, 128>>>(m, h->d_cs, h->d_crange);
        LMMEW_CUDA(cudaGetLastError());
    } else {
        LMMEW_CUDA(cudaMemset(h->d_crange, 0, sizeof(int2) * (size_t)m.A * m.B));
    }

    // unscattered paths + per-angle sensitivity
    if (cudaMalloc(&h->d_prim, sizeof(float) * (size_t)m.A * m.W * m.nq) != cudaSuccess ||
        cudaMalloc(&h->d_sens_a, sizeof(double) * (size_t)m.A * m.nq) != cudaSuccess)
        return set_error(LMMEW_ERR_OOM, "cannot allocate primary tables");
    {
        dim3 g((m.nq + 127) / 128, m.A);
        k_primary<<<g, 128>>>(m, dcs, h->d_q_pix, (const double*)d_gq.p, mu_line, h->d_prim,
                              h->d_sens_a);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
        // keep the unscattered part alone for the model without scatter
        if (cudaMalloc(&h->d_sens_a_prim, sizeof(double) * (size_t)m.A * m.nq) != cudaSuccess)
            return set_error(LMMEW_ERR_OOM, "cannot allocate primary sensitivity");
        LMMEW_CUDA(cudaMemcpy(h->d_sens_a_prim, h->d_sens_a, sizeof(double) * (size_t)m.A * m.nq,
                              cudaMemcpyDeviceToDevice));
    }

    // single-scatter paths: every angle once, in blocks of the table buffer's
    // size, for the sensitivity; the tables of the last block stay resident
    if (m.np) {
        h->tab_slots = tab_slots < m.A ? tab_slots : 0;
        h->tab_bytes = per_angle * (size_t)tab_slots;
        if (cudaMalloc(&h->d_tab, h->tab_bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(LMMEW_ERR_OOM, "cannot allocate scatter tables (" +
                                                std::to_string(h->tab_bytes >> 20) + " MiB)");
        }
        LMMEW_CUDA(cudaMemset(h->d_tab, 0, h->tab_bytes));
        DevBuf d_on_det;
        LMMEW_CUDA(cudaMalloc(&d_on_det.p, sizeof(double) * (size_t)m.A * m.np));
        k_on_detector<<<dim3((m.np + 127) / 128, m.A), 128>>>(m, dcs, (const int*)d_p_cell.p,
                                                               (double*)d_on_det.p);
        ++h->launches;
        for (int a0 = 0; a0 < m.A; a0 += tab_slots) {
            const int cnt = std::min(tab_slots, m.A - a0);
            k_scatter<true><<<dim3((m.nq + 7) / 8, cnt), 256>>>(
                m, a0, 1, dcs, h->d_q_pix, (const int*)d_p_cell.p, (const double*)d_p_rho.p,
                (const double*)d_gqp.p, (const double*)d_dqp.p, (const double*)d_gp.p, mu_line,
                inv, (const double*)d_on_det.p, h->d_tab, h->d_sens_a);
            ++h->launches;
            LMMEW_CUDA(cudaGetLastError());
            h->tab_a0 = a0;
            h->tab_astep = 1;
            h->tab_count = cnt;
        }
        if (h->tab_slots && cudaMalloc(&h->d_clip, sizeof(ChunkRange)) != cudaSuccess)
            return set_error(LMMEW_ERR_OOM, "cannot allocate the clipped row range");
        // kept for rebuilding streamed tables
        auto keep = [](DevBuf& b) {
            void* p = b.p;
            b.p = nullptr;
            return p;
        };
        h->d_on_det = (double*)keep(d_on_det);
        h->d_gqp = (double*)keep(d_gqp);
        h->d_dqp = (double*)keep(d_dqp);
    }
    h->d_cs_a = (double*)d_cs_a.p;
    d_cs_a.p = nullptr;
    h->d_p_cell = (int*)d_p_cell.p;
    d_p_cell.p = nullptr;
    h->d_p_rho = (double*)d_p_rho.p;
    d_p_rho.p = nullptr;
    h->d_gp = (double*)d_gp.p;
    d_gp.p = nullptr;
    h->d_inv = (int*)d_inv.p;
    d_inv.p = nullptr;
    h->d_mu_line = (double*)d_mu_line.p;
    d_mu_line.p = nullptr;
    LMMEW_CUDA(cudaMalloc(&h->d_status, sizeof(int)));
    LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    cudaEventRecord(e1, 0);
    LMMEW_CUDA(cudaDeviceSynchronize());
    cudaEventElapsedTime(&h->setup_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return subset_sensitivity(h, h->n_subsets_default, 0) == LMMEW_OK
               ? (cudaDeviceSynchronize() == cudaSuccess ? LMMEW_OK
                                                         : set_error(LMMEW_ERR_CUDA, "set-up"))
               : LMMEW_ERR_OOM;
}

int64_t g_table_budget = 0;

int stream_tables(lm_handle* h, int a0, int astep, int count, cudaStream_t st) {
    const ModelConst& m = h->mc;
    if (m.np == 0 || h->tab_slots == 0 || count <= 0) return LMMEW_OK;
    if (count > h->tab_slots)
        return set_error(LMMEW_ERR_INVALID_ARG, "an angle block larger than the table buffer");
    // resident already: the same step (or one angle) inside the resident block
    const int last = a0 + (count - 1) * astep;
    const int r_last = h->tab_a0 + (h->tab_count - 1) * h->tab_astep;
    if (h->tab_count > 0 && (astep == h->tab_astep || count == 1) && a0 >= h->tab_a0 &&
        last <= r_last && (a0 - h->tab_a0) % h->tab_astep == 0 &&
        (last - h->tab_a0) % h->tab_astep == 0)
        return LMMEW_OK;
    k_scatter<false><<<dim3((m.nq + 7) / 8, count), 256, 0, st>>>(
        m, a0, astep, h->d_cs_a, h->d_q_pix, h->d_p_cell, h->d_p_rho, h->d_gqp, h->d_dqp, h->d_gp,
        h->d_mu_line, h->d_inv, h->d_on_det, h->d_tab, nullptr);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    h->tab_a0 = a0;
    h->tab_astep = astep;
    h->tab_count = count;
    return LMMEW_OK;
}

int set_table_streaming(lm_handle* h, int max_angles) {
    const ModelConst& m = h->mc;
    if (max_angles < 0) return set_error(LMMEW_ERR_INVALID_ARG, "max_angles must be >= 0");
    if (m.np == 0) return LMMEW_OK;   // no single-scatter tables
    const int slots = (max_angles == 0 || max_angles >= m.A) ? m.A : max_angles;
    const int cur = h->tab_slots ? h->tab_slots : m.A;
    if (slots == cur) return LMMEW_OK;
    if (slots < m.A && h->prec != 0)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED,
                         "the reduced-precision form needs every angle's tables resident; "
                         "switch the scatter precision to FP32 first");
    const size_t per_angle = sizeof(float) * (size_t)m.nqt * m.npc * 3 * m.W * kQT * kPC;
    // launches already queued may still read the old buffer
    LMMEW_CUDA(cudaDeviceSynchronize());
    float* buf = nullptr;
    if (cudaMalloc(&buf, per_angle * (size_t)slots) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LMMEW_ERR_OOM, "cannot allocate the path tables of " +
                                            std::to_string(slots) + " angles (" +
                                            std::to_string((per_angle * slots) >> 20) + " MiB)");
    }
    if (slots < m.A && !h->d_clip && cudaMalloc(&h->d_clip, sizeof(ChunkRange)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return set_error(LMMEW_ERR_OOM, "cannot allocate the clipped row range");
    }
    LMMEW_CUDA(cudaMemset(buf, 0, per_angle * (size_t)slots));
    cudaFree(h->d_tab);
    h->d_tab = buf;
    h->tab_bytes = per_angle * (size_t)slots;
    h->tab_count = 0;
    if (slots == m.A) {   // every angle, once
        h->tab_slots = m.A;
        const int rc = stream_tables(h, 0, 1, m.A, 0);
        h->tab_slots = 0;
        if (rc != LMMEW_OK) return rc;
    } else {
        h->tab_slots = slots;
    }
    LMMEW_CUDA(cudaDeviceSynchronize());
    return LMMEW_OK;
}

}  // namespace lmmew
