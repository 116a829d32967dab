// Support initialiser: a crude OSEM reconstruction of the binned sinogram
// whose thresholded image bounds the emission support (the paper reduces the
// list-mode cost, which grows with the non-zero voxels, by estimating the
// object's boundary this way first; Sec. 2.2, last paragraph).
//
// Reading (the paper gives no details):
//   * sinogram c[a][k]: events of angle a in position bin k = floor((u + U/2)/w)
//     (u = U/2 goes to the last bin), every energy of the window;
//   * crude projector over the whole grid: the collimator response of pixel n
//     integrated over bin k, no attenuation, no scatter, no energy,
//       A[a][k][n] = (erf((hi_k - u_a(p_n)) q) - erf((lo_k - u_a(p_n)) q)) / 2,
//       q = 1 / (sqrt(2) sigma_u(d_a(p_n)));
//   * ordered subsets by angle (a mod N_s), s^i_n = sum_{a in A_i, k} A[a][k][n],
//     uniform start f_n = sum c / sum_n s_n, update
//       f_n <- f_n / s^i_n sum_{a in A_i, k} A[a][k][n] c[a][k] / y[a][k], y = A f
//     (bins with y = 0 contribute nothing, s^i_n = 0 gives f_n = 0);
//   * support = {n : f_n >= threshold max f}, dilated by `dilate` pixels.
// Every reduction runs in a fixed order, so the result is deterministic.
#include <math.h>

#include <algorithm>
#include <vector>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kBsThreads = 256;
constexpr float kErfReach = 5.0f;  // |z| beyond which erf(z) = +-1 to FP32 precision

// per (angle, grid pixel): (u_a(p_n), 1 / (sqrt 2 sigma_u(d_a(p_n))))
__global__ void k_bs_geom(const float2* __restrict__ trig, int nx, int ny, float dpx, int n_angles,
                          float radius, float fwhm0, float slope, float2* __restrict__ geo) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    const int npix = nx * ny;
    if (n >= npix || a >= n_angles) return;
    const float x = pixel_x(n, nx, dpx), y = pixel_y(n, nx, ny, dpx);
    const float2 cs = trig[a];
    const float u = -x * cs.y + y * cs.x;
    const float depth = radius - (x * cs.x + y * cs.y);
    const float sigma = (fwhm0 + slope * depth) * 0.42466090014400953f;  // FWHM / (2 sqrt(2 ln 2))
    geo[(size_t)a * npix + n] = make_float2(u, 0.70710678118654752f / sigma);
}

// one event per thread; the bin index in FP64 (exact for FP32 positions)
__global__ void k_bs_sino(const int32_t* __restrict__ angle, const float* __restrict__ u, int64_t n, int n_bins,
                          double w, double half, unsigned int* __restrict__ sino) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = (int)floor(((double)u[i] + half) / w);
    k = min(max(k, 0), n_bins - 1);
    atomicAdd(&sino[(size_t)angle[i] * n_bins + k], 1u);
}

// s^i_n: the bins of an angle telescope to the extent's mass
__global__ void k_bs_sens(const float2* __restrict__ geo, int n_angles, int npix, float half, int n_subsets,
                          float* __restrict__ sens) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (n >= npix) return;
    double s = 0.0;
    for (int a = i; a < n_angles; a += n_subsets) {
        const float2 g = geo[(size_t)a * npix + n];
        s += 0.5 * ((double)erff((half - g.x) * g.y) - (double)erff((-half - g.x) * g.y));
    }
    sens[(size_t)i * npix + n] = (float)s;
}

// y[a][k] = sum_n A[a][k][n] f_n for the angles of subset i (one block per bin)
__global__ void k_bs_fwd(const float2* __restrict__ geo, const float* __restrict__ f, int npix, int n_bins,
                         float w, float half, int i, int n_subsets, float* __restrict__ y) {
    __shared__ float red[kBsThreads];
    const int k = blockIdx.x;
    const int a = i + blockIdx.y * n_subsets;
    const float lo = -half + k * w, hi = lo + w;
    float acc = 0.0f;
    for (int n = threadIdx.x; n < npix; n += kBsThreads) {
        const float2 g = geo[(size_t)a * npix + n];
        const float zl = (lo - g.x) * g.y, zh = (hi - g.x) * g.y;
        if (zl > kErfReach || zh < -kErfReach) continue;
        acc = fmaf(0.5f * (erff(zh) - erff(zl)), f[n], acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kBsThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) y[(size_t)a * n_bins + k] = red[0];
}

// f_n <- f_n / s^i_n sum_{a in A_i, k} A[a][k][n] c[a][k] / y[a][k]
__global__ void k_bs_update(const float2* __restrict__ geo, const unsigned int* __restrict__ sino,
                            const float* __restrict__ y, const float* __restrict__ sens_i, int npix, int n_angles,
                            int n_bins, float w, float half, int i, int n_subsets, float* __restrict__ f) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= npix) return;
    float back = 0.0f;
    for (int a = i; a < n_angles; a += n_subsets) {
        const float2 g = geo[(size_t)a * npix + n];
        // bins within reach of this pixel's response
        const float reach = kErfReach / g.y;
        const int k0 = max(0, (int)floorf((g.x - reach + half) / w));
        const int k1 = min(n_bins - 1, (int)floorf((g.x + reach + half) / w));
        if (k0 > k1) continue;
        float e_lo = erff((-half + k0 * w - g.x) * g.y);
        for (int k = k0; k <= k1; ++k) {
            const float e_hi = erff((-half + (k + 1) * w - g.x) * g.y);
            const size_t b = (size_t)a * n_bins + k;
            const float yb = y[b];
            if (yb > 0.0f) back = fmaf(0.5f * (e_hi - e_lo), (float)sino[b] / yb, back);
            e_lo = e_hi;
        }
    }
    const float s = sens_i[n];
    f[n] = s > 0.0f ? f[n] * back / s : 0.0f;
}

__global__ void k_bs_init(float* __restrict__ f, int npix, const unsigned int* __restrict__ sino, int nsino,
                          const float* __restrict__ sens, int n_subsets) {
    __shared__ double r1[kBsThreads], r2[kBsThreads];
    double c = 0.0, s = 0.0;
    for (int b = threadIdx.x; b < nsino; b += kBsThreads) c += sino[b];
    for (int n = threadIdx.x; n < npix; n += kBsThreads)
        for (int i = 0; i < n_subsets; ++i) s += sens[(size_t)i * npix + n];
    r1[threadIdx.x] = c;
    r2[threadIdx.x] = s;
    __syncthreads();
    for (int h = kBsThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            r1[threadIdx.x] += r1[threadIdx.x + h];
            r2[threadIdx.x] += r2[threadIdx.x + h];
        }
        __syncthreads();
    }
    const float v = r2[0] > 0.0 ? (float)(r1[0] / r2[0]) : 0.0f;
    for (int n = threadIdx.x; n < npix; n += kBsThreads) f[n] = v;
}

__global__ void k_bs_mask(const float* __restrict__ f, int nx, int ny, float threshold, int dilate,
                          uint8_t* __restrict__ mask) {
    __shared__ float red[kBsThreads];
    const int npix = nx * ny;
    float m = 0.0f;
    for (int n = threadIdx.x; n < npix; n += kBsThreads) m = fmaxf(m, f[n]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = kBsThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    const float thr = threshold * red[0];
    for (int n = threadIdx.x; n < npix; n += kBsThreads) {
        const int ix = n % nx, iy = n / nx;
        uint8_t in = 0;
        for (int dy = -dilate; dy <= dilate && !in; ++dy)
            for (int dx = -dilate; dx <= dilate && !in; ++dx) {
                const int jx = ix + dx, jy = iy + dy;
                if (jx >= 0 && jx < nx && jy >= 0 && jy < ny && f[jy * nx + jx] >= thr) in = 1;
            }
        mask[n] = in;
    }
}

}  // namespace

lmosem_status run_binned_support(lmosem_ctx* c, const int32_t* d_angle, const float* d_u, int64_t n,
                                 int n_subsets, int n_iters, double threshold, int dilate,
                                 uint8_t* h_support, float* d_image) {
    lmosem_status st;
    const int npix = c->npix, nb = c->n_bins, na = c->n_angles;
    const float w = (float)c->bin_mm, half = (float)(0.5 * c->n_bins * c->bin_mm);
    float2* geo = nullptr;
    unsigned int* sino = nullptr;
    float *sens = nullptr, *y = nullptr, *fown = nullptr;
    uint8_t* mask = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&geo, (size_t)na * npix)) || (st = tmp.alloc(&sino, (size_t)na * nb)) ||
        (st = tmp.alloc(&sens, (size_t)n_subsets * npix)) || (st = tmp.alloc(&y, (size_t)na * nb)) ||
        (st = tmp.alloc(&mask, npix)) || (!d_image && (st = tmp.alloc(&fown, npix))))
        return st;
    float* f = d_image ? d_image : fown;
    LMOSEM_CK(c, cudaMemsetAsync(sino, 0, sizeof(unsigned int) * na * nb, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(y, 0, sizeof(float) * na * nb, c->stream));
    LMOSEM_PROF_BEGIN(c);
    k_bs_geom<<<dim3((npix + 255) / 256, na), 256, 0, c->stream>>>(c->d_trig, c->nx, c->ny, (float)c->dpx, na,
                                                                  (float)c->radius, (float)c->fwhm0,
                                                                  (float)c->fwhm_slope, geo);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    LMOSEM_PROF_BEGIN(c);
    k_bs_sino<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(d_angle, d_u, n, nb, c->bin_mm,
                                                                  0.5 * c->n_bins * c->bin_mm, sino);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    LMOSEM_PROF_BEGIN(c);
    k_bs_sens<<<dim3((npix + 255) / 256, n_subsets), 256, 0, c->stream>>>(geo, na, npix, half, n_subsets, sens);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    LMOSEM_PROF_BEGIN(c);
    k_bs_init<<<1, kBsThreads, 0, c->stream>>>(f, npix, sino, na * nb, sens, n_subsets);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    for (int t = 0; t < n_iters; ++t)
        for (int i = 0; i < n_subsets; ++i) {
            const int n_a = (na - i + n_subsets - 1) / n_subsets;  // angles a = i, i + N_s, ...
            LMOSEM_PROF_BEGIN(c);
            k_bs_fwd<<<dim3(nb, n_a), kBsThreads, 0, c->stream>>>(geo, f, npix, nb, w, half, i, n_subsets, y);
            LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
            LMOSEM_PROF_BEGIN(c);
            k_bs_update<<<(npix + 255) / 256, 256, 0, c->stream>>>(geo, sino, y, sens + (size_t)i * npix, npix, na,
                                                                   nb, w, half, i, n_subsets, f);
            LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
        }
    LMOSEM_PROF_BEGIN(c);
    k_bs_mask<<<1, kBsThreads, 0, c->stream>>>(f, c->nx, c->ny, (float)threshold, dilate, mask);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    LMOSEM_CK(c, cudaMemcpyAsync(h_support, mask, npix, cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    return LMOSEM_OK;
}

}  // namespace lmosem
