/*
 * FP64 CPU oracle for list-mode OSEM attenuation-and-scatter compensation
 * (Rahman, Laforest, Jha, "A list-mode OSEM-based attenuation and scatter
 * compensation method for SPECT", ISBI 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * What it computes (paper Section 2.1-2.2, Eqs. 2, 4, 7, 8):
 *   p_jn  = sum over paths P starting in pixel n of  pr(A_j|P) s_eff(P)
 *   s_n^i = sum over paths P starting in pixel n that reach the detector at an
 *           angle of subset i of s_eff(P)
 * The paper leaves s_eff(P) and pr(A|P) to an earlier reference; this oracle
 * uses the 2-D in-plane first-order model (primary path (n) and single
 * Compton scatter paths (n,m)) that the design document freezes:
 *   primary   w = exp(-L_det(p_n, a, E0))
 *             k = phi(u; u_a(p_n), s_u(d_a(p_n))) phi(E; E0, s_E(E0))
 *   scatter   w = D^2 mu_m Kt(psi) exp(-L(p_n->p_m)) exp(-r(E') L_det(p_m,a,E0)) / (2 pi |p_m-p_n|)
 *             k = phi(u; u_a(p_m), s_u(d_a(p_m))) phi(E; E', s_E(E'))
 *   pr(A|P) s_eff(P) = w k,   s_eff(P) = w D_u D_E.
 * Only first-order, in-plane scatter is kept (paper Section 2.2, last
 * paragraph before the GPU description).
 * For binned attributes (paper Section 4) orc_model_binned integrates k over
 * the bin: each Gaussian density becomes its mass on the bin.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, brute-force path enumeration, quadrature, invariants of the
 * EM update).  The absolute path weights are pinned against physics: photon
 * counts per scatter order from an independent Monte-Carlo converge to the
 * sensitivities restricted to each path type as the pixel shrinks.  The
 * full reconstruction is pinned only through those invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MEC2_KEV 510.99895
#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t nx, ny;          /* image grid, row-major pixel n = iy*nx + ix        */
    double pixel_mm;         /* pixel pitch D                                      */
    int32_t n_angles;        /* detector angles theta_a = angle0 + 2 pi a / n_angles */
    double angle0_rad;
    int32_t n_bins;          /* detector extent U = n_bins * bin_mm, |u| <= U/2    */
    double bin_mm;
    double radius_mm;        /* detector face distance R from the rotation axis    */
    double coll_fwhm0_mm;    /* collimator response FWHM_u(d) = f0 + f1 d          */
    double coll_fwhm_slope;
    double e0_kev;           /* photopeak energy                                   */
    double fwhm_frac_e0;     /* energy FWHM at E0 as a fraction of E0              */
    double e_lo_kev, e_hi_kev; /* acceptance window                                */
    double pos_cut;          /* scatter terms with (du/s_u)^2/2 above this are skipped */
} orc_geom;

/* ------------------------------------------------------------------ */
/* Photon physics                                                      */
/* ------------------------------------------------------------------ */

/* Compton energy of a photon of energy e after deflection by psi. */
double orc_compton_energy(double e_kev, double cos_psi)
{
    return e_kev / (1.0 + (e_kev / ORC_MEC2_KEV) * (1.0 - cos_psi));
}

/* Klein-Nishina angular shape K = P^2 (P + 1/P - sin^2 psi) / 2, P = E'/E.
 * K(0) = 1; for E -> 0 it tends to the Thomson shape (1 + cos^2 psi)/2. */
double orc_kn_shape(double e_kev, double cos_psi)
{
    double P = orc_compton_energy(e_kev, cos_psi) / e_kev;
    double sin2 = 1.0 - cos_psi * cos_psi;
    return 0.5 * P * P * (P + 1.0 / P - sin2);
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on the
 * three-term Legendre recurrence. */
static void orc_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Mean of the in-plane Klein-Nishina shape over the circle,
 * Kbar = (1/2pi) int_0^{2pi} K(psi) dpsi, Gauss-Legendre with 2048 nodes.
 * Kt = K / Kbar is then a probability density of 2 pi per radian. */
double orc_kn_mean(double e_kev)
{
    enum { NQ = 2048 };
    static double xs[NQ], ws[NQ];
    static int ready = 0;
    if (!ready) {
        orc_gauss_legendre(NQ, xs, ws);
        ready = 1;
    }
    double acc = 0.0;
    for (int i = 0; i < NQ; ++i) {
        double psi = ORC_PI * (xs[i] + 1.0); /* [-1,1] -> [0, 2 pi] */
        acc += ws[i] * ORC_PI * orc_kn_shape(e_kev, cos(psi));
    }
    return acc / (2.0 * ORC_PI);
}

/* Total Klein-Nishina cross section in units of 2 pi r_e^2 (textbook closed
 * form).  Only ratios are used: mu(E) = mu(E0) sigma(E)/sigma(E0). */
double orc_sigma_kn(double e_kev)
{
    double k = e_kev / ORC_MEC2_KEV;
    double l = log(1.0 + 2.0 * k);
    double a = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k);
    return a + l / (2.0 * k) - (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k));
}

/* ------------------------------------------------------------------ */
/* Line integrals through the pixelised mu-map                         */
/* ------------------------------------------------------------------ */

static int orc_cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Exact line integral of the piecewise-constant map mu (zero outside the
 * grid) along the segment (x0,y0)-(x1,y1).  Siddon's parametrisation: every
 * crossing of a grid line is an alpha in [0,1]; between consecutive crossings
 * the segment lies in one pixel, found from the midpoint. */
double orc_line_integral(const double* mu, int nx, int ny, double dpx,
                         double x0, double y0, double x1, double y1)
{
    double xmin = -0.5 * nx * dpx, ymin = -0.5 * ny * dpx;
    double dx = x1 - x0, dy = y1 - y0;
    double len = sqrt(dx * dx + dy * dy);
    if (len == 0.0) return 0.0;
    double* al = (double*)malloc(sizeof(double) * (size_t)(nx + ny + 4));
    int na = 0;
    al[na++] = 0.0;
    al[na++] = 1.0;
    if (dx != 0.0)
        for (int k = 0; k <= nx; ++k) {
            double a = (xmin + k * dpx - x0) / dx;
            if (a > 0.0 && a < 1.0) al[na++] = a;
        }
    if (dy != 0.0)
        for (int k = 0; k <= ny; ++k) {
            double a = (ymin + k * dpx - y0) / dy;
            if (a > 0.0 && a < 1.0) al[na++] = a;
        }
    qsort(al, (size_t)na, sizeof(double), orc_cmp_double);
    double acc = 0.0;
    for (int i = 0; i + 1 < na; ++i) {
        double da = al[i + 1] - al[i];
        if (da <= 0.0) continue;
        double am = 0.5 * (al[i] + al[i + 1]);
        double xm = x0 + am * dx, ym = y0 + am * dy;
        int ix = (int)floor((xm - xmin) / dpx);
        int iy = (int)floor((ym - ymin) / dpx);
        if (ix < 0 || ix >= nx || iy < 0 || iy >= ny) continue;
        acc += mu[(size_t)iy * nx + ix] * da * len;
    }
    free(al);
    return acc;
}

/* Line integral from (x0,y0) along the unit direction (ux,uy) to beyond the
 * grid (the map is zero outside, so any far end point gives the same value). */
double orc_ray_to_edge(const double* mu, int nx, int ny, double dpx,
                       double x0, double y0, double ux, double uy)
{
    double far = (nx + ny + 2) * dpx;
    return orc_line_integral(mu, nx, ny, dpx, x0, y0, x0 + far * ux, y0 + far * uy);
}

/* ------------------------------------------------------------------ */
/* Geometry helpers                                                    */
/* ------------------------------------------------------------------ */

static void orc_pixel_centre(const orc_geom* g, int pix, double* x, double* y)
{
    int ix = pix % g->nx, iy = pix / g->nx;
    *x = (ix + 0.5 - 0.5 * g->nx) * g->pixel_mm;
    *y = (iy + 0.5 - 0.5 * g->ny) * g->pixel_mm;
}

static double orc_fwhm_to_sigma(double fwhm) { return fwhm / (2.0 * sqrt(2.0 * log(2.0))); }

/* Depth-dependent collimator response width. */
static double orc_sigma_u(const orc_geom* g, double depth)
{
    return orc_fwhm_to_sigma(g->coll_fwhm0_mm + g->coll_fwhm_slope * depth);
}

/* Energy resolution: FWHM_E(E) = f_E sqrt(E0 E). */
static double orc_sigma_e(const orc_geom* g, double e_kev)
{
    return orc_fwhm_to_sigma(g->fwhm_frac_e0 * sqrt(g->e0_kev * e_kev));
}

static double orc_gauss(double x, double m, double s)
{
    double z = (x - m) / s;
    return exp(-0.5 * z * z) / (s * sqrt(2.0 * ORC_PI));
}

/* Probability mass of N(m, s^2) inside [lo, hi]. */
static double orc_gauss_mass(double lo, double hi, double m, double s)
{
    return 0.5 * erfc(-(hi - m) / (s * sqrt(2.0))) - 0.5 * erfc(-(lo - m) / (s * sqrt(2.0)));
}

double orc_det_u(const orc_geom* g, int a, double x, double y)
{
    double th = g->angle0_rad + 2.0 * ORC_PI * a / g->n_angles;
    return -x * sin(th) + y * cos(th);
}

double orc_det_depth(const orc_geom* g, int a, double x, double y)
{
    double th = g->angle0_rad + 2.0 * ORC_PI * a / g->n_angles;
    return g->radius_mm - (x * cos(th) + y * sin(th));
}

/* ------------------------------------------------------------------ */
/* Attenuation tables                                                  */
/* ------------------------------------------------------------------ */

/* l_edge[a*npix + pix]: integral of mu(E0) from the centre of every pixel along
 * omega_a to the grid edge.  l_pair[i*n_scat + k]: integral of mu(E0) between
 * the centres of support pixel sup[i] and scatter pixel scat[k]. */
void orc_build_tables(const orc_geom* g, const double* mu, const int32_t* sup, int n_sup,
                      const int32_t* scat, int n_scat, double* l_edge, double* l_pair)
{
    int npix = g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < g->n_angles * npix; ++q) {
        int a = q / npix, pix = q % npix;
        double th = g->angle0_rad + 2.0 * ORC_PI * a / g->n_angles;
        double x, y;
        orc_pixel_centre(g, pix, &x, &y);
        l_edge[q] = orc_ray_to_edge(mu, g->nx, g->ny, g->pixel_mm, x, y, cos(th), sin(th));
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n_sup; ++i) {
        double xn, yn;
        orc_pixel_centre(g, sup[i], &xn, &yn);
        for (int k = 0; k < n_scat; ++k) {
            double xm, ym;
            orc_pixel_centre(g, scat[k], &xm, &ym);
            l_pair[(size_t)i * n_scat + k] =
                orc_line_integral(mu, g->nx, g->ny, g->pixel_mm, xn, yn, xm, ym);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Path weights                                                        */
/* ------------------------------------------------------------------ */

/* Scatter path (n, m) at angle a: weight w (the part of pr(A|P) s_eff(P) that
 * does not depend on the event), scattered energy E', and the detector-side
 * centre u_c and depth of the position kernel.  Returns 0 for m == n. */
static int orc_scatter_path(const orc_geom* g, const double* mu, int a, int pix_n, int pix_m,
                            double l_nm, double l_edge_m, double kbar, double sig0,
                            double* w, double* eprime)
{
    if (pix_n == pix_m) return 0;
    double xn, yn, xm, ym;
    orc_pixel_centre(g, pix_n, &xn, &yn);
    orc_pixel_centre(g, pix_m, &xm, &ym);
    double vx = xm - xn, vy = ym - yn;
    double r = sqrt(vx * vx + vy * vy);
    double th = g->angle0_rad + 2.0 * ORC_PI * a / g->n_angles;
    double cos_psi = (vx * cos(th) + vy * sin(th)) / r;
    double e1 = orc_compton_energy(g->e0_kev, cos_psi);
    double kt = orc_kn_shape(g->e0_kev, cos_psi) / kbar;
    double ratio = orc_sigma_kn(e1) / sig0;
    *w = g->pixel_mm * g->pixel_mm * mu[pix_m] * kt * exp(-l_nm) * exp(-ratio * l_edge_m) /
         (2.0 * ORC_PI * r);
    *eprime = e1;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Event model p_jn (Eq. 2 with Eq. 4: the per-event mixture over paths)  */
/* ------------------------------------------------------------------ */

/* p_out[j*n_sup + i] = sum over paths from sup[i] at angle ev_angle[j] of
 * w(P) k(u_j, E_j | P).  Tables from orc_build_tables. */
void orc_model(const orc_geom* g, const double* mu, const int32_t* sup, int n_sup,
               const int32_t* scat, int n_scat, const double* l_edge, const double* l_pair,
               const int32_t* ev_angle, const double* ev_u, const double* ev_e, int64_t n_ev,
               double* p_out, int parts /* bit 0: primary path, bit 1: scatter paths */)
{
    int npix = g->nx * g->ny;
    double kbar = orc_kn_mean(g->e0_kev);
    double sig0 = orc_sigma_kn(g->e0_kev);
    double se0 = orc_sigma_e(g, g->e0_kev);
    size_t tab = (size_t)n_sup * n_scat;
    double* w = (double*)malloc(sizeof(double) * tab);   /* [k][i] */
    double* ep = (double*)malloc(sizeof(double) * tab);  /* [k][i] */
    double* ucen = (double*)malloc(sizeof(double) * (size_t)n_scat);
    double* usig = (double*)malloc(sizeof(double) * (size_t)n_scat);
    memset(p_out, 0, sizeof(double) * (size_t)n_ev * n_sup);

    for (int a = 0; a < g->n_angles; ++a) {
        int64_t cnt = 0;
        for (int64_t j = 0; j < n_ev; ++j) cnt += (ev_angle[j] == a);
        if (cnt == 0) continue;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n_scat; ++k) {
            double xm, ym;
            orc_pixel_centre(g, scat[k], &xm, &ym);
            ucen[k] = orc_det_u(g, a, xm, ym);
            usig[k] = orc_sigma_u(g, orc_det_depth(g, a, xm, ym));
            for (int i = 0; i < n_sup; ++i) {
                double wv = 0.0, e1 = g->e0_kev;
                orc_scatter_path(g, mu, a, sup[i], scat[k], l_pair[(size_t)i * n_scat + k],
                                 l_edge[(size_t)a * npix + scat[k]], kbar, sig0, &wv, &e1);
                w[(size_t)k * n_sup + i] = wv;
                ep[(size_t)k * n_sup + i] = e1;
            }
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t j = 0; j < n_ev; ++j) {
            if (ev_angle[j] != a) continue;
            double* row = p_out + (size_t)j * n_sup;
            double u = ev_u[j], e = ev_e[j];
            /* primary path (n) */
            for (int i = 0; i < n_sup && (parts & 1); ++i) {
                double xn, yn;
                orc_pixel_centre(g, sup[i], &xn, &yn);
                double su = orc_sigma_u(g, orc_det_depth(g, a, xn, yn));
                row[i] = exp(-l_edge[(size_t)a * npix + sup[i]]) *
                         orc_gauss(u, orc_det_u(g, a, xn, yn), su) * orc_gauss(e, g->e0_kev, se0);
            }
            if (!(parts & 2)) continue;
            /* first-order scatter paths (n, m) */
            for (int k = 0; k < n_scat; ++k) {
                double z = (u - ucen[k]) / usig[k];
                if (0.5 * z * z > g->pos_cut) continue;
                double pu = orc_gauss(u, ucen[k], usig[k]);
                const double* wk = w + (size_t)k * n_sup;
                const double* ek = ep + (size_t)k * n_sup;
                for (int i = 0; i < n_sup; ++i) {
                    if (wk[i] == 0.0) continue;
                    row[i] += wk[i] * pu * orc_gauss(e, ek[i], orc_sigma_e(g, ek[i]));
                }
            }
        }
    }
    free(w);
    free(ep);
    free(ucen);
    free(usig);
}

/* ------------------------------------------------------------------ */
/* Subset sensitivity (denominator of Eq. 7)                           */
/* ------------------------------------------------------------------ */

/* s_out[i*n_sup + q] = sum over angles a with a mod n_subsets == i of the
 * detection probability of every path from sup[q]:
 *   exp(-L_det) D_u D_E(E0)  +  sum_m w(n,m) D_u(m) D_E(E').
 * parts: bit 0 keeps the primary path, bit 1 the scatter paths (3: both). */
void orc_sensitivity(const orc_geom* g, const double* mu, const int32_t* sup, int n_sup,
                     const int32_t* scat, int n_scat, const double* l_edge, const double* l_pair,
                     int n_subsets, double* s_out, int parts)
{
    int npix = g->nx * g->ny;
    double kbar = orc_kn_mean(g->e0_kev);
    double sig0 = orc_sigma_kn(g->e0_kev);
    double se0 = orc_sigma_e(g, g->e0_kev);
    double half = 0.5 * g->n_bins * g->bin_mm;
    double de0 = orc_gauss_mass(g->e_lo_kev, g->e_hi_kev, g->e0_kev, se0);
    memset(s_out, 0, sizeof(double) * (size_t)n_subsets * n_sup);
    for (int a = 0; a < g->n_angles; ++a) {
        int sub = a % n_subsets;
#pragma omp parallel for schedule(dynamic, 4)
        for (int i = 0; i < n_sup; ++i) {
            double xn, yn;
            orc_pixel_centre(g, sup[i], &xn, &yn);
            double acc = 0.0;
            if (parts & 1)
                acc = exp(-l_edge[(size_t)a * npix + sup[i]]) *
                      orc_gauss_mass(-half, half, orc_det_u(g, a, xn, yn),
                                     orc_sigma_u(g, orc_det_depth(g, a, xn, yn))) *
                      de0;
            for (int k = 0; k < n_scat && (parts & 2); ++k) {
                double wv, e1;
                if (!orc_scatter_path(g, mu, a, sup[i], scat[k], l_pair[(size_t)i * n_scat + k],
                                      l_edge[(size_t)a * npix + scat[k]], kbar, sig0, &wv, &e1))
                    continue;
                double xm, ym;
                orc_pixel_centre(g, scat[k], &xm, &ym);
                double du = orc_gauss_mass(-half, half, orc_det_u(g, a, xm, ym),
                                           orc_sigma_u(g, orc_det_depth(g, a, xm, ym)));
                double dE = orc_gauss_mass(g->e_lo_kev, g->e_hi_kev, e1, orc_sigma_e(g, e1));
                acc += wv * du * dE;
            }
            s_out[(size_t)sub * n_sup + i] += acc;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Binned attributes (paper Section 4: position binned into the        */
/* detector's bins, energy into a few bins)                            */
/* ------------------------------------------------------------------ */

/* Mass of N(m, s^2) inside [lo, hi], written so that a bin far out in either
 * tail keeps its relative accuracy (the erfc of the nearer edge minus that of
 * the farther one); equal to orc_gauss_mass up to rounding. */
static double orc_gauss_mass_tail(double lo, double hi, double m, double s)
{
    double zl = (lo - m) / (s * sqrt(2.0)), zh = (hi - m) / (s * sqrt(2.0));
    if (zl >= 0.0) return 0.5 * (erfc(zl) - erfc(zh));
    if (zh <= 0.0) return 0.5 * (erfc(-zh) - erfc(-zl));
    return 1.0 - 0.5 * (erfc(-zl) + erfc(zh));
}

/* p_out[r*n_sup + i]: probability that an emission in sup[i] is detected at
 * angle row_angle[r] with its position in detector bin row_pos[r]
 * ([-U/2 + b bin_mm, -U/2 + (b+1) bin_mm]) and its energy in
 * [e_edges[row_e[r]], e_edges[row_e[r] + 1]].  This is the event model of
 * orc_model with each Gaussian density replaced by its mass on the bin:
 *   primary   w mass_u(bin; u_a(p_n), s_u) mass_E(bin; E0, s_E(E0))
 *   scatter   w mass_u(bin; u_a(p_m), s_u) mass_E(bin; E', s_E(E'))
 * A scatter path is skipped when the whole position bin lies beyond the
 * position cut of its kernel (the cut of orc_model, at the bin's nearest
 * point). */
void orc_model_binned(const orc_geom* g, const double* mu, const int32_t* sup, int n_sup,
                      const int32_t* scat, int n_scat, const double* l_edge, const double* l_pair,
                      const int32_t* row_angle, const int32_t* row_pos, const int32_t* row_e,
                      int64_t n_rows, const double* e_edges, double* p_out, int parts)
{
    int npix = g->nx * g->ny;
    double kbar = orc_kn_mean(g->e0_kev);
    double sig0 = orc_sigma_kn(g->e0_kev);
    double se0 = orc_sigma_e(g, g->e0_kev);
    double half = 0.5 * g->n_bins * g->bin_mm;
    size_t tab = (size_t)n_sup * n_scat;
    double* w = (double*)malloc(sizeof(double) * tab);   /* [k][i] */
    double* ep = (double*)malloc(sizeof(double) * tab);  /* [k][i] */
    double* ucen = (double*)malloc(sizeof(double) * (size_t)n_scat);
    double* usig = (double*)malloc(sizeof(double) * (size_t)n_scat);
    memset(p_out, 0, sizeof(double) * (size_t)n_rows * n_sup);

    for (int a = 0; a < g->n_angles; ++a) {
        int64_t cnt = 0;
        for (int64_t r = 0; r < n_rows; ++r) cnt += (row_angle[r] == a);
        if (cnt == 0) continue;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n_scat; ++k) {
            double xm, ym;
            orc_pixel_centre(g, scat[k], &xm, &ym);
            ucen[k] = orc_det_u(g, a, xm, ym);
            usig[k] = orc_sigma_u(g, orc_det_depth(g, a, xm, ym));
            for (int i = 0; i < n_sup; ++i) {
                double wv = 0.0, e1 = g->e0_kev;
                orc_scatter_path(g, mu, a, sup[i], scat[k], l_pair[(size_t)i * n_scat + k],
                                 l_edge[(size_t)a * npix + scat[k]], kbar, sig0, &wv, &e1);
                w[(size_t)k * n_sup + i] = wv;
                ep[(size_t)k * n_sup + i] = e1;
            }
        }
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t r = 0; r < n_rows; ++r) {
            if (row_angle[r] != a) continue;
            double* row = p_out + (size_t)r * n_sup;
            double u0 = -half + row_pos[r] * g->bin_mm, u1 = u0 + g->bin_mm;
            double e0 = e_edges[row_e[r]], e1 = e_edges[row_e[r] + 1];
            for (int i = 0; i < n_sup && (parts & 1); ++i) {
                double xn, yn;
                orc_pixel_centre(g, sup[i], &xn, &yn);
                double su = orc_sigma_u(g, orc_det_depth(g, a, xn, yn));
                row[i] = exp(-l_edge[(size_t)a * npix + sup[i]]) *
                         orc_gauss_mass_tail(u0, u1, orc_det_u(g, a, xn, yn), su) *
                         orc_gauss_mass_tail(e0, e1, g->e0_kev, se0);
            }
            if (!(parts & 2)) continue;
            for (int k = 0; k < n_scat; ++k) {
                double dn = ucen[k] < u0 ? u0 - ucen[k] : (ucen[k] > u1 ? ucen[k] - u1 : 0.0);
                double z = dn / usig[k];
                if (0.5 * z * z > g->pos_cut) continue;
                double pu = orc_gauss_mass_tail(u0, u1, ucen[k], usig[k]);
                const double* wk = w + (size_t)k * n_sup;
                const double* ek = ep + (size_t)k * n_sup;
                for (int i = 0; i < n_sup; ++i) {
                    if (wk[i] == 0.0) continue;
                    row[i] += wk[i] * pu * orc_gauss_mass_tail(e0, e1, ek[i], orc_sigma_e(g, ek[i]));
                }
            }
        }
    }
    free(w);
    free(ep);
    free(ucen);
    free(usig);
}
