// Subset sensitivity (row a6 of the hot path): the denominator of paper
// Eq. 7, T sum over paths from pixel q reaching the detector at an angle of
// subset i of s_eff(P), with s_eff(P) = w(P) D_u(P) D_E(P): the path weight
// times the probability that the collimator response falls on the detector
// extent and the energy response inside the acquisition window.
//
// One thread per (angle, support pixel) sums the primary path and every
// scatter path; terms are FP32, partial sums of 32 terms are added into an
// FP64 accumulator, and the per-angle results are reduced per subset in
// angle order (deterministic).
#include <math.h>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

struct SensArgs {
    int nx, ny, npix;
    float dpx;
    const int32_t* sup;
    int n_sup, ld_w;
    const int32_t* scat;
    const float4* scat_geo;  // (x_m, y_m, mu_m, pixel index bits)
    int n_scat;
    const float* mu;
    const float2* trig;
    const float* l_edge;
    const float* l_pair;
    const float2* compton;
    const float4* ppar;   // .w = D_u of the primary
    const float* du_m;    // [a][m]
    float eps0, inv_kbar;
    float w_const;        // D^2 / (2 pi)
    float de0;            // window mass of the photopeak
    double* sens_angle;   // [a][n]
};

__global__ void k_sens_angle(SensArgs A) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int a = blockIdx.y;
    if (n >= A.n_sup) return;
    int pn = A.sup[n];
    const float xn = pixel_x(pn, A.nx, A.dpx), yn = pixel_y(pn, A.nx, A.ny, A.dpx);
    float2 trig = A.trig[a];
    double acc = (double)(expf(-A.l_edge[(size_t)a * A.npix + pn]) *
                          A.ppar[(size_t)a * A.ld_w + n].w * A.de0);
    const float* lp = A.l_pair + n;
    const float* le = A.l_edge + (size_t)a * A.npix;
    const float* du = A.du_m + (size_t)a * A.n_scat;
    float part = 0.0f;
    for (int k = 0; k < A.n_scat; ++k) {
        const float4 gm = __ldg(A.scat_geo + k);
        const int pm = __float_as_int(gm.w);
        float cpsi, rinv;
        if (path_geometry_xy(xn, yn, gm.x, gm.y, pn == pm, trig, &cpsi, &rinv)) {
            float P, kt;
            compton(cpsi, A.eps0, A.inv_kbar, &P, &kt);
            float2 cr = compton_lookup(A.compton, cpsi);  // (mu ratio, window mass)
            float att = fmaf(cr.x, __ldg(le + pm), lp[(size_t)k * A.n_sup]);
            float w = A.w_const * gm.z * kt * rinv * __expf(-att);
            part = fmaf(w, __ldg(du + k) * cr.y, part);
        }
        if ((k & 31) == 31) {
            acc += (double)part;
            part = 0.0f;
        }
    }
    acc += (double)part;
    A.sens_angle[(size_t)a * A.n_sup + n] = acc;
}

__global__ void k_sens_reduce(const double* __restrict__ sens_angle, int n_angles, int n_sup,
                              int n_subsets, double* __restrict__ sens, double* __restrict__ total) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_sup) return;
    double tot = 0.0;
    for (int i = 0; i < n_subsets; ++i) {
        double s = 0.0;
        for (int a = i; a < n_angles; a += n_subsets) s += sens_angle[(size_t)a * n_sup + n];
        sens[(size_t)i * n_sup + n] = s;
        tot += s;
    }
    total[n] = tot;
}

}  // namespace

lmosem_status compute_sensitivity(lmosem_ctx* c, int n_subsets) {
    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_sens_angle, (size_t)c->n_angles * c->n_sup))) return st;
    if ((st = dev_alloc(c, &c->d_sens, (size_t)(n_subsets + 1) * c->n_sup))) return st;
    SensArgs A;
    A.nx = c->nx;
    A.ny = c->ny;
    A.npix = c->npix;
    A.dpx = (float)c->dpx;
    A.sup = c->d_sup;
    A.n_sup = c->n_sup;
    A.ld_w = c->ld_w;
    A.scat = c->d_scat;
    A.scat_geo = c->d_scat_geo;
    A.n_scat = c->n_scat;
    A.mu = c->d_mu;
    A.trig = c->d_trig;
    A.l_edge = c->d_l_edge;
    A.l_pair = c->d_l_pair;
    A.compton = c->d_compton;
    A.ppar = c->d_ppar;
    A.du_m = c->d_du_m;
    A.eps0 = (float)(c->e0 / kMec2Kev);
    A.inv_kbar = (float)(1.0 / c->kbar);
    A.w_const = (float)(c->dpx * c->dpx / (2.0 * kPi));
    A.de0 = (float)c->de0;
    A.sens_angle = c->d_sens_angle;
    if (wtab_all_fits(c)) {
        // the scatter-weight planes of every angle fit the table budget: build
        // them in the same pass (same terms) and keep them for the model build
        if ((st = wtab_all_with_sens(c, c->d_sens_angle, A.w_const, A.de0))) return st;
    } else {
        dev_free(c, &c->d_wtab_all);
        LMOSEM_PROF_BEGIN(c);
        k_sens_angle<<<dim3((c->n_sup + 127) / 128, c->n_angles), 128, 0, c->stream>>>(A);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SENS);
    }
    // rows 0..n_subsets-1: s^i; row n_subsets: s = sum_i s^i
    LMOSEM_PROF_BEGIN(c);
    k_sens_reduce<<<(c->n_sup + 255) / 256, 256, 0, c->stream>>>(
        c->d_sens_angle, c->n_angles, c->n_sup, n_subsets, c->d_sens,
        c->d_sens + (size_t)n_subsets * c->n_sup);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SENS);
    c->sens_subsets = n_subsets;
    return LMOSEM_OK;
}

}  // namespace lmosem
