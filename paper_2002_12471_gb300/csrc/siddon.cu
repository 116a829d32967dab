// Attenuation and geometry tables (row a1 of the hot path): line integrals
// of mu(E0) through the pixelised map from every pixel centre to the grid
// edge along omega_a and between every scatter and support pixel centre,
// the per-angle position-kernel parameters, and the cos(psi) table of the
// energy-dependent Compton quantities.
//
// The attenuation of the paper's s_eff(P) (Section 2.1, Eq. 4 and the text
// after it) is exp(-integral of mu) along the photon path; the scattered leg
// uses mu(E') = mu(E0) sigma_KN(E') / sigma_KN(E0).
#include <math.h>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

// Integral of the piecewise-constant map along the ray that starts at the
// centre of pixel (ix, iy) and runs in the unit direction (dx, dy) for tmax
// (infinity: to the grid edge).  Siddon's parametrisation: the ray is cut at
// every grid line it crosses, each crossing distance computed afresh from
// its integer line index (no drift); the segment sum is Neumaier-compensated.
__device__ float ray_from_centre(const float* __restrict__ mu, int nx, int ny, float dpx, int ix,
                                 int iy, float dx, float dy, float tmax) {
    const float xmin = -0.5f * (float)nx * dpx, ymin = -0.5f * (float)ny * dpx;
    const float x0 = xmin + ((float)ix + 0.5f) * dpx;
    const float y0 = ymin + ((float)iy + 0.5f) * dpx;
    const int sx = dx > 0.0f ? 1 : (dx < 0.0f ? -1 : 0);
    const int sy = dy > 0.0f ? 1 : (dy < 0.0f ? -1 : 0);
    const float idx = sx ? 1.0f / dx : 0.0f, idy = sy ? 1.0f / dy : 0.0f;
    float t = 0.0f, sum = 0.0f, comp = 0.0f;
    for (int step = 0; step < nx + ny + 2; ++step) {
        float tx = sx ? (xmin + (float)(ix + (sx > 0)) * dpx - x0) * idx : INFINITY;
        float ty = sy ? (ymin + (float)(iy + (sy > 0)) * dpx - y0) * idy : INFINITY;
        float tn = fminf(fminf(tx, ty), tmax);
        float seg = fmaxf(tn - t, 0.0f) * __ldg(mu + iy * nx + ix);
        float s2 = sum + seg;
        comp += (fabsf(sum) >= fabsf(seg)) ? (sum - s2) + seg : (seg - s2) + sum;
        sum = s2;
        if (tn >= tmax) break;
        if (tx <= ty) ix += sx;
        if (ty <= tx) iy += sy;
        if (ix < 0 || ix >= nx || iy < 0 || iy >= ny) break;
        t = tn;
    }
    return sum + comp;
}

__global__ void k_l_edge(const float* __restrict__ mu, int nx, int ny, float dpx,
                         const float2* __restrict__ trig, float* __restrict__ l_edge) {
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    int a = blockIdx.y;
    int npix = nx * ny;
    if (pix >= npix) return;
    float2 cs = trig[a];
    l_edge[(size_t)a * npix + pix] =
        ray_from_centre(mu, nx, ny, dpx, pix % nx, pix / nx, cs.x, cs.y, INFINITY);
}

__global__ void k_l_pair(const float* __restrict__ mu, int nx, int ny, float dpx,
                         const int32_t* __restrict__ sup, int n_sup,
                         const int32_t* __restrict__ scat, float* __restrict__ l_pair) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (i >= n_sup) return;
    int pn = sup[i], pm = scat[k];
    float v = 0.0f;
    if (pn != pm) {
        float vx = pixel_x(pm, nx, dpx) - pixel_x(pn, nx, dpx);
        float vy = pixel_y(pm, nx, ny, dpx) - pixel_y(pn, nx, ny, dpx);
        float r = sqrtf(vx * vx + vy * vy);
        v = ray_from_centre(mu, nx, ny, dpx, pn % nx, pn / nx, vx / r, vy / r, r);
    }
    l_pair[(size_t)k * n_sup + i] = v;
}

// Per-angle position-kernel parameters.  For a detector position u and a
// pixel centre p at depth d: the Gaussian collimator response
// phi(u; p.t_a, sigma_u(d)) = 2^(lq - ((u - u_c) q)^2), q = sqrt(log2 e / 2) / sigma,
// lq = log2(1 / (sigma sqrt(2 pi))); cut = k_sigma sigma; D_u = mass of the
// Gaussian on the detector extent.
struct PosPar {
    float u, q, lq, cut, du;
};

__device__ PosPar pos_par(float x, float y, float2 cs, float radius, float f0, float f1,
                          float k_sigma, float half_ext) {
    PosPar p;
    p.u = -x * cs.y + y * cs.x;
    float depth = radius - (x * cs.x + y * cs.y);
    float sig = (f0 + f1 * depth) * 0.42466090014400953f;  // FWHM -> sigma
    p.q = 0.8493218002880191f / sig;                         // sqrt(log2(e)/2)/sigma
    p.lq = -log2f(sig) - 1.3257480647361593f;                 // -log2(sqrt(2 pi))
    p.cut = k_sigma * sig;
    float s2 = 0.7071067811865476f / sig;
    p.du = 0.5f * (erfcf((p.u - half_ext) * s2) - erfcf((p.u + half_ext) * s2));
    return p;
}

__global__ void k_angle_params(int nx, int ny, float dpx, const float2* __restrict__ trig,
                               const int32_t* __restrict__ sup, int n_sup, int ld_w,
                               const int32_t* __restrict__ scat, int n_scat,
                               const float* __restrict__ l_edge, float radius, float f0, float f1,
                               float k_sigma, float half_ext, float4* __restrict__ mpar,
                               float* __restrict__ du_m, float4* __restrict__ ppar) {
    int a = blockIdx.y;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    float2 cs = trig[a];
    int npix = nx * ny;
    if (k < n_scat) {
        int pm = scat[k];
        PosPar p = pos_par(pixel_x(pm, nx, dpx), pixel_y(pm, nx, ny, dpx), cs, radius, f0, f1,
                           k_sigma, half_ext);
        mpar[(size_t)a * n_scat + k] = make_float4(p.u, p.q, p.lq, p.cut);
        du_m[(size_t)a * n_scat + k] = p.du;
    }
    if (k < ld_w) {
        float4 v = make_float4(0.0f, 0.0f, -INFINITY, 0.0f);
        if (k < n_sup) {
            int pn = sup[k];
            PosPar p = pos_par(pixel_x(pn, nx, dpx), pixel_y(pn, nx, ny, dpx), cs, radius, f0, f1,
                               k_sigma, half_ext);
            float lp = p.lq - l_edge[(size_t)a * npix + pn] * kLog2e;
            v = make_float4(p.u, p.q, lp, p.du);
        }
        ppar[(size_t)a * ld_w + k] = v;
    }
}

// Total Klein-Nishina cross section (textbook closed form; units of
// 2 pi r_e^2, only ratios are used).
__host__ __device__ double sigma_kn_total(double e_kev) {
    double k = e_kev / kMec2Kev;
    double l = log1p(2.0 * k);
    return (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k) + l / (2.0 * k) -
           (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k));
}

// cos(psi) table: (sigma_KN(E') / sigma_KN(E0), window mass of the energy
// blur at E') at kComptonNodes nodes on [-1, 1], in FP64
__global__ void k_compton_table(double e0, double fwhm_frac, double e_lo, double e_hi, double sig0,
                                float2* __restrict__ comp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kComptonNodes) return;
    const double fw2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    const double cp = -1.0 + 2.0 * k / (kComptonNodes - 1);
    const double e1 = e0 / (1.0 + e0 / kMec2Kev * (1.0 - cp));
    const double se = fwhm_frac * sqrt(e0 * e1) * fw2s;
    const double de = 0.5 * (erfc((e_lo - e1) / (sqrt(2.0) * se)) - erfc((e_hi - e1) / (sqrt(2.0) * se)));
    comp[k] = make_float2((float)(sigma_kn_total(e1) / sig0), (float)de);
}

double kn_shape_host(double e0, double c) {
    double p = 1.0 / (1.0 + e0 / kMec2Kev * (1.0 - c));
    return 0.5 * p * p * (p + 1.0 / p - (1.0 - c * c));
}

}  // namespace

lmosem_status build_tables(lmosem_ctx* c) {
    lmosem_status st;
    const int npix = c->npix;

    // host: trig table, Klein-Nishina circle mean, cos(psi) table
    std::vector<float2> trig(c->n_angles);
    for (int a = 0; a < c->n_angles; ++a) {
        double th = c->angle0 + 2.0 * kPi * a / c->n_angles;
        trig[a] = make_float2((float)cos(th), (float)sin(th));
    }
    // periodic trapezoid rule: exponentially convergent for the analytic
    // 2 pi-periodic Klein-Nishina shape
    {
        const int nq = 8192;
        double acc = 0.0;
        for (int k = 0; k < nq; ++k) acc += kn_shape_host(c->e0, cos(2.0 * kPi * k / nq));
        c->kbar = acc / nq;
    }
    const double fw2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    {
        double s0 = c->fwhm_frac * c->e0 * fw2s;
        c->de0 = 0.5 * (erfc((c->e_lo - c->e0) / (sqrt(2.0) * s0)) -
                        erfc((c->e_hi - c->e0) / (sqrt(2.0) * s0)));
    }
    const double sig0 = sigma_kn_total(c->e0);

    if ((st = dev_alloc(c, &c->d_trig, c->n_angles))) return st;
    if ((st = dev_alloc(c, &c->d_compton, kComptonNodes))) return st;
    if ((st = dev_alloc(c, &c->d_l_edge, (size_t)c->n_angles * npix))) return st;
    if ((st = dev_alloc(c, &c->d_l_pair, (size_t)c->n_scat * c->n_sup))) return st;
    if ((st = dev_alloc(c, &c->d_mpar, (size_t)c->n_angles * c->n_scat))) return st;
    if ((st = dev_alloc(c, &c->d_du_m, (size_t)c->n_angles * c->n_scat))) return st;
    if ((st = dev_alloc(c, &c->d_ppar, (size_t)c->n_angles * c->ld_w))) return st;
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_trig, trig.data(), trig.size() * sizeof(float2),
                                 cudaMemcpyHostToDevice, c->stream));
    // the cos(psi) table on the device (FP64; 16k nodes would cost the host ~1 ms)
    LMOSEM_PROF_BEGIN(c);
    k_compton_table<<<(kComptonNodes + 255) / 256, 256, 0, c->stream>>>(c->e0, c->fwhm_frac, c->e_lo, c->e_hi,
                                                                         sig0, c->d_compton);
    LMOSEM_LAUNCHED(c, LMOSEM_K_TABLES);

    float dpx = (float)c->dpx;
    LMOSEM_PROF_BEGIN(c);
    k_l_edge<<<dim3((npix + 255) / 256, c->n_angles), 256, 0, c->stream>>>(
        c->d_mu, c->nx, c->ny, dpx, c->d_trig, c->d_l_edge);
    LMOSEM_LAUNCHED(c, LMOSEM_K_TABLES);
    LMOSEM_PROF_BEGIN(c);
    k_l_pair<<<dim3((c->n_sup + 255) / 256, c->n_scat), 256, 0, c->stream>>>(
        c->d_mu, c->nx, c->ny, dpx, c->d_sup, c->n_sup, c->d_scat, c->d_l_pair);
    LMOSEM_LAUNCHED(c, LMOSEM_K_TABLES);
    int wmax = c->n_scat > c->ld_w ? c->n_scat : c->ld_w;
    LMOSEM_PROF_BEGIN(c);
    k_angle_params<<<dim3((wmax + 255) / 256, c->n_angles), 256, 0, c->stream>>>(
        c->nx, c->ny, dpx, c->d_trig, c->d_sup, c->n_sup, c->ld_w, c->d_scat, c->n_scat,
        c->d_l_edge, (float)c->radius, (float)c->fwhm0, (float)c->fwhm_slope, c->k_sigma,
        (float)(0.5 * c->n_bins * c->bin_mm), c->d_mpar, c->d_du_m, c->d_ppar);
    LMOSEM_LAUNCHED(c, LMOSEM_K_TABLES);
    // no host wait: a copy from pageable memory returns once its source has
    // been staged, so the host vectors above may go
    return LMOSEM_OK;
}

}  // namespace lmosem
