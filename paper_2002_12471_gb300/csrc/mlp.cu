// Learned scatter surrogate (row a9 of the hot path).
//
// The first-order scatter part of the per-event path sum (paper Eq. 2 over
// the scatter paths of Section 2.2),
//     p^scat_jn = sum_{m in strip(j)} U_jm W_a(n, m) phi(E_j; E'_a(n, m), sigma_E),
// is replaced by a multilayer perceptron of eight inputs (pixel x, y,
// detector angle, event position, event energy, and three attenuation
// features: mu(E0) integrated from the pixel to the detector, along the
// event's detector line from the pixel's depth to the detector, and along
// that whole line), 8 -> 256 -> 256 -> 256 -> 256 -> 1 with ReLU, whose output
// is the standardised natural log of p^scat_jn.  The network is trained on
// exact scatter path sums made by the exact path (k_pathsum with the primary
// left out) and evaluated inside the model build, where p_jn = primary_jn +
// exp(mu + sigma y_jn).
//
// Matrix products run on the 5th-generation tensor cores (tcgen05, the
// kernel in mlp_tc.cu) in BF16 with FP32 accumulation in TMEM:
// C[M x N] = A[M x K] B[N x K]^T with both operands K-contiguous (the
// backward products use explicit transposes; the weight gradients split K
// over the SMs), fused bias / ReLU / ReLU-mask epilogues.  Parameters are
// kept in FP32 (Adam state too) with BF16 copies for the products.
#include <cuda_bf16.h>
#include <math.h>
#include <float.h>

#include <algorithm>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kIn = 8, kInPad = 16, kH = 256;
constexpr int kBaseIn = 6;  // inputs of the quadratic baseline (the first six)
constexpr int64_t kOffW1 = 0;
constexpr int64_t kOffB1 = kOffW1 + kH * kIn;
constexpr int64_t kOffW2 = kOffB1 + kH;
constexpr int64_t kOffB2 = kOffW2 + kH * kH;
constexpr int64_t kOffW3 = kOffB2 + kH;
constexpr int64_t kOffB3 = kOffW3 + kH * kH;
constexpr int64_t kOffW4 = kOffB3 + kH;
constexpr int64_t kOffB4 = kOffW4 + kH * kH;
constexpr int64_t kOffW5 = kOffB4 + kH;
constexpr int64_t kOffB5 = kOffW5 + kH;
// coefficients of the quadratic baseline of the log target in the first six
// scaled inputs (1, x_i, x_i x_j for i <= j): 28 values, fitted by least
// squares, or zero; the network learns the standardised residual
constexpr int kBasis = 28;
constexpr int64_t kOffBase = kOffB5 + 1;
constexpr int64_t kOffMu = kOffBase + kBasis;
constexpr int64_t kOffSigma = kOffMu + 1;
constexpr int64_t kParams = kOffSigma + 1;
static_assert(kParams == LMOSEM_SURROGATE_PARAMS, "parameter blob layout");
static_assert(kBasis == 1 + kBaseIn + kBaseIn * (kBaseIn + 1) / 2, "quadratic basis size");
static_assert(kIn <= kInPad, "inputs fit the padded operand");

__device__ __forceinline__ void basis(const float* x, float* phi) {
    phi[0] = 1.0f;
#pragma unroll
    for (int i = 0; i < kBaseIn; ++i) phi[1 + i] = x[i];
    int k = 1 + kBaseIn;
#pragma unroll
    for (int i = 0; i < kBaseIn; ++i)
#pragma unroll
        for (int j = i; j < kBaseIn; ++j) phi[k++] = x[i] * x[j];
}

// the baseline of the log scatter at scaled inputs x (FP32)
__device__ __forceinline__ float baseline(const float* __restrict__ blob, const float* x) {
    float phi[kBasis];
    basis(x, phi);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kBasis; ++k) s = fmaf(blob[kOffBase + k], phi[k], s);
    return s;
}

// ---------------------------------------------------------------- products

enum Epi { EPI_F32 = 0, EPI_RELU_BF16 = 1, EPI_MASK_BF16 = 2 };

// out[c][r] = in[r][c] (BF16), 32 x 32 tiles
__global__ void k_transpose(const __nv_bfloat16* __restrict__ in, int64_t rows, int cols, int64_t ldi,
                            __nv_bfloat16* __restrict__ out, int64_t ldo) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k;
        const int c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? in[r * ldi + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(int64_t)c * ldo + r] = tile[threadIdx.x][k];
    }
}

// ---------------------------------------------------------------- small kernels

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// minibatch rows (seeded, with replacement): scaled features as BF16 (padded
// to 16 columns) and standardised targets
// element index of input (row i, column k) in the row-major M x 16 layout of
// the chain of separate products or, for the fused tcgen05 kernel, the tile-major layout:
// 128-row tiles of 2048 elements, each the K = 16 operand layout (row group g
// of 8 rows at 128 elements, its two 8-column groups 64 elements apart)
__device__ __forceinline__ int64_t x_index(int64_t i, int k, bool tiled) {
    if (!tiled) return i * kInPad + k;
    const int r = (int)(i & 127);
    return (i >> 7) * (128 * kInPad) + (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// (step_ptr: the step index lives on the device, for a captured training step)
// (cdf: inclusive prefix sums of sampling weights, n FP64 values: row i is
// drawn with probability weight_i / total, by bisection; nullptr: uniform)
__global__ void k_gather(const float* __restrict__ feat, const float* __restrict__ targ, int64_t n,
                         int B, uint64_t seed, int step, const int* __restrict__ step_ptr,
                         const double* __restrict__ cdf, const float* __restrict__ blob,
                         const float* __restrict__ floor, __nv_bfloat16* __restrict__ X, float* __restrict__ t,
                         bool tiled) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (step_ptr) step = *step_ptr;
    const uint64_t h = seed == 0 ? 0 : splitmix64(seed ^ ((uint64_t)step * 0x100000001B3ull + b));
    int64_t i;
    if (seed == 0) {
        i = (int64_t)b % n;
    } else if (cdf) {
        const double x = (double)(h >> 11) * 0x1.0p-53 * cdf[n - 1];
        int64_t lo = 0, hi = n - 1;  // smallest i with cdf[i] > x
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > x) hi = mid;
            else lo = mid + 1;
        }
        i = lo;
    } else {
        i = (int64_t)(h % (uint64_t)n);
    }
    float x[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = feat[i * kIn + k];
#pragma unroll
    for (int k = 0; k < kInPad; ++k) X[x_index(b, k, tiled)] = __float2bfloat16_rn(k < kIn ? x[k] : 0.0f);
    const float ti = floor ? fmaxf(targ[i], *floor) : targ[i];
    t[b] = (ti - baseline(blob, x) - blob[kOffMu]) / blob[kOffSigma];
}

// y = H4 w5 + b5 (one warp per row)
__global__ void k_out_fwd(const __nv_bfloat16* __restrict__ H, int64_t M, const float* __restrict__ blob,
                          float* __restrict__ y) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    float s = 0.0f;
    for (int k = lane; k < kH; k += 32) s = fmaf(__bfloat162float(H[row * kH + k]), blob[kOffW5 + k], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + blob[kOffB5];
}

// dy = 2 (y - t) / B; dz4 = dy w5 where H4 > 0; loss sum into loss[step]
// (FP64; step = *step_ptr, or 0)
__global__ void k_out_bwd(const float* __restrict__ y, const float* __restrict__ t,
                          const __nv_bfloat16* __restrict__ H4, int B, const float* __restrict__ blob,
                          float* __restrict__ dy, __nv_bfloat16* __restrict__ dz4, double* __restrict__ loss,
                          const int* __restrict__ step_ptr) {
    const int b = blockIdx.x;
    if (step_ptr) loss += *step_ptr;
    const float r = y[b] - t[b];
    const float d = 2.0f * r / (float)B;
    if (threadIdx.x == 0) {
        dy[b] = d;
        atomicAdd(loss, (double)r * (double)r / (double)B);
    }
    for (int k = threadIdx.x; k < kH; k += blockDim.x) {
        const bool on = __bfloat162float(H4[(int64_t)b * kH + k]) > 0.0f;
        dz4[(int64_t)b * kH + k] = __float2bfloat16_rn(on ? d * blob[kOffW5 + k] : 0.0f);
    }
}

// dW5[k] = sum_b dy_b H4[b][k], db5 = sum_b dy_b: block z sums its share of
// the rows (thread k = column k, coalesced across the block; thread kH the
// bias) into part[z][k]; k_out_wgrad_sum adds the shares in order
constexpr int kOutSplits = 32;
__global__ void __launch_bounds__(kH + 32) k_out_wgrad(const float* __restrict__ dy,
                                                       const __nv_bfloat16* __restrict__ H4, int B,
                                                       float* __restrict__ part) {
    const int k = threadIdx.x;
    if (k > kH) return;
    const int per = (B + kOutSplits - 1) / kOutSplits;
    const int b0 = blockIdx.x * per, b1 = min(B, b0 + per);
    float s = 0.0f;
    for (int b = b0; b < b1; ++b) s += dy[b] * (k < kH ? __bfloat162float(H4[(int64_t)b * kH + k]) : 1.0f);
    part[blockIdx.x * (kH + 1) + k] = s;
}

__global__ void k_out_wgrad_sum(const float* __restrict__ part, float* __restrict__ grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kH) return;
    float s = 0.0f;
    for (int z = 0; z < kOutSplits; ++z) s += part[z * (kH + 1) + k];
    grad[k < kH ? kOffW5 + k : kOffB5] = s;
}

// db[r] = sum of row r of dZ^T (rows x B), one warp per row, fixed order
__global__ void k_rowsum(const __nv_bfloat16* __restrict__ ZT, int rows, int B, int64_t ld,
                         float* __restrict__ out) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.0f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(ZT[(int64_t)r * ld + b]);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
}

// a gradient block [rows x cols] into the blob: the sum, in split order, of
// the K splits of a GEMM result with ld (split_stride elements apart)
__global__ void k_copy_grad(const float* __restrict__ src, int rows, int cols, int64_t lds, int splits,
                            int64_t split_stride, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += src[z * split_stride + (int64_t)(i / cols) * lds + (i % cols)];
    dst[i] = s;
}

// learning rate and Adam bias corrections of the step *step_ptr (the last
// 20% of the steps at lr / 10): sc = (lr_s, 1 - b1^(s+1), 1 - b2^(s+1))
__global__ void k_step_scalars(const int* __restrict__ step_ptr, int steps, float lr, float b1, float b2,
                               float* __restrict__ sc) {
    const int s = *step_ptr;
    sc[0] = s < steps * 0.8 ? lr : lr * 0.1f;
    sc[1] = (float)(1.0 - pow((double)b1, (double)(s + 1)));
    sc[2] = (float)(1.0 - pow((double)b2, (double)(s + 1)));
}

// Adam (bias-corrected moments) over the whole blob except (mu, sigma); the
// step's scalars from sc; thread 0 then advances the device step counter (no
// later kernel of the step reads it)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, const float* __restrict__ sc, float b1, float b2,
                       float eps, int* __restrict__ step_ptr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *step_ptr += 1;
    if (i >= n) return;
    const float lr = sc[0], c1 = sc[1], c2 = sc[2];
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of the weights: W1 padded to 16 columns, W2..W4 and their
// transposes (for the input gradients)
__global__ void k_weights_bf16(const float* __restrict__ blob, __nv_bfloat16* __restrict__ w1,
                               __nv_bfloat16* __restrict__ w234, __nv_bfloat16* __restrict__ w234t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kH * kInPad) {
        const int o = i / kInPad, k = i % kInPad;
        w1[i] = __float2bfloat16_rn(k < kIn ? blob[kOffW1 + o * kIn + k] : 0.0f);
    }
    if (i < 3 * kH * kH) {
        const int l = i / (kH * kH), r = i % (kH * kH);
        const int o = r / kH, k = r % kH;
        const float val = blob[kOffW2 + (int64_t)l * (kH * kH + kH) + r];
        w234[i] = __float2bfloat16_rn(val);
        w234t[(int64_t)l * kH * kH + k * kH + o] = __float2bfloat16_rn(val);
    }
}

// with floor_below > 0 the targets are raised to (largest - floor_below):
// that level into *floor (else -FLT_MAX); one block
__global__ void k_target_floor(const float* __restrict__ t, int64_t n, float floor_below, float* __restrict__ floor) {
    __shared__ float smax[256];
    float fl = -FLT_MAX;
    if (floor_below > 0.0f) {
        float m = -FLT_MAX;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, t[i]);
        smax[threadIdx.x] = m;
        __syncthreads();
        for (int k = 0; k < (int)blockDim.x; ++k) fl = fmaxf(fl, smax[k]);
        fl -= floor_below;
    }
    if (threadIdx.x == 0) *floor = fl;
}

// mean and standard deviation of the (floored) targets minus the baseline
// (FP64, one block, fixed order) into the blob's mu and sigma
__global__ void k_target_stats(const float* __restrict__ t, const float* __restrict__ feat, int64_t n,
                               const float* __restrict__ floor, float* __restrict__ blob) {
    __shared__ double s1[256], s2[256];
    const float fl = *floor;
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double ti = fmaxf(t[i], fl) - baseline(blob, feat + i * kIn);
        a += ti;
        b += ti * ti;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, Bq = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            A += s1[k];
            Bq += s2[k];
        }
        const double mu = A / n;
        const double var = fmax(Bq / n - mu * mu, 1e-12);
        blob[kOffMu] = (float)mu;
        blob[kOffSigma] = (float)sqrt(var);
    }
}

// least squares of the baseline: for m rows evenly spaced over the samples,
// block (i, j) (j <= i) sums phi_i phi_j and block (i, kBasis) sums phi_i t
// (floored), FP64 in a fixed order
__global__ void k_basis_normal(const float* __restrict__ feat, const float* __restrict__ t, int64_t n, int64_t m,
                               const float* __restrict__ floor, double* __restrict__ out /* kBasis x (kBasis+1) */) {
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bj < kBasis && bj > bi) return;
    __shared__ double sh[256];
    const float fl = *floor;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
        const int64_t i = (int64_t)((double)r * (double)n / (double)m);
        float phi[kBasis];
        basis(feat + i * kIn, phi);
        const double pj = bj < kBasis ? (double)phi[bj] : (double)fmaxf(t[i], fl);
        acc += (double)phi[bi] * pj;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) s += sh[k];
        out[bi * (kBasis + 1) + bj] = s;
    }
}

// ---------------------------------------------------------------- features

struct FeatArgs {
    const int32_t* a_s;      // sorted angles
    const float* u_s;
    const float* e_s;
    const int32_t* sup;
    int n_sup, nx, ny, npix;
    float dpx;
    const float* l_edge;     // [a][pixel]
    float angle0, dtheta;
    const float* line;       // [a][iu][is]: mu(E0) integrated from depth s to the detector along u
    int line_nu, line_ns;
    float line_u0, line_s0, line_inv_h;
};

// attenuation along the detector line u of angle a from depth s on (bilinear
// in the table's nodes; u and s clamped to the table)
__device__ __forceinline__ float line_att(const FeatArgs& F, int a, float u, float s) {
    const float fu = fminf(fmaxf((u - F.line_u0) * F.line_inv_h, 0.0f), (float)(F.line_nu - 1) - 1e-3f);
    const float fs = fminf(fmaxf((s - F.line_s0) * F.line_inv_h, 0.0f), (float)(F.line_ns - 1) - 1e-3f);
    const int iu = (int)fu, is = (int)fs;
    const float wu = fu - (float)iu, ws = fs - (float)is;
    const float* t = F.line + ((size_t)a * F.line_nu + iu) * F.line_ns + is;
    const float lo = fmaf(ws, t[1] - t[0], t[0]);
    const float hi = fmaf(ws, t[F.line_ns + 1] - t[F.line_ns], t[F.line_ns]);
    return fmaf(wu, hi - lo, lo);
}

// network inputs in the detector frame of the event's angle: offset of the
// event from the pixel's projection, the pixel's coordinate along the flight
// direction and its projection, the angle, the energy, the pixel-to-detector
// attenuation, and the attenuation along the event's detector line from the
// pixel's depth to the detector and along the whole line, each scaled to O(1)
__device__ __forceinline__ void features(const FeatArgs& F, int64_t row, int q, float* out) {
    const int a = F.a_s[row];
    const int pix = F.sup[q];
    const float x = pixel_x(pix, F.nx, F.dpx), y = pixel_y(pix, F.nx, F.ny, F.dpx);
    const float th = F.angle0 + F.dtheta * a;
    float sn, cs;
    sincosf(th, &sn, &cs);
    const float u_a = -x * sn + y * cs;
    const float s_a = x * cs + y * sn;
    const float u = F.u_s[row];
    out[0] = (u - u_a) / 50.0f;
    out[1] = s_a / 100.0f;
    out[2] = u_a / 100.0f;
    out[3] = (th - 3.14159265358979f) / 3.14159265358979f;
    out[4] = (F.e_s[row] - 137.5f) / 37.5f;
    out[5] = (F.l_edge[(size_t)a * F.npix + pix] - 1.5f) / 1.5f;
    out[6] = (line_att(F, a, u, s_a) - 1.5f) / 1.5f;
    out[7] = (line_att(F, a, u, F.line_s0) - 1.5f) / 1.5f;
}

// Attenuation along detector lines: for angle a, lateral position
// u_i = u0 + i h and depth s_k = s0 + k h (point s omega_a + u t_a), the
// integral of the piecewise-constant mu(E0) map from s_k to the end of the
// line (beyond the grid), i.e. towards the detector.  One thread walks one
// line from s0 upwards through the merged sequences of vertical and
// horizontal grid-line crossings and table nodes, adding mu times the length
// of every piece (the pixel of a piece from its midpoint), in FP64: the node
// values are exact integrals of the map up to rounding.
__global__ void k_line_table(const float* __restrict__ mu, int nx, int ny, double dpx, int n_angles,
                             double angle0, int nu, int ns, double u0, double s0, double h,
                             float* __restrict__ out) {
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= n_angles * nu) return;
    const int a = line / nu, iu = line % nu;
    const double th = angle0 + 2.0 * kPi * a / n_angles;
    const double c = cos(th), sn = sin(th);
    const double u = u0 + iu * h;
    const double xmin = -0.5 * nx * dpx, ymin = -0.5 * ny * dpx;
    // x(s) = s c - u sn, y(s) = s sn + u c; the k-th crossing of an axis's
    // grid lines comes at an s that increases with k
    const bool hx = fabs(c) > 1e-12, hy = fabs(sn) > 1e-12;
    auto sx = [&](int k) { const int i = c > 0 ? k : nx - k; return (xmin + i * dpx + u * sn) / c; };
    auto sy = [&](int k) { const int i = sn > 0 ? k : ny - k; return (ymin + i * dpx - u * c) / sn; };
    float* row = out + (size_t)line * ns;
    // pass 0: the whole line's integral; pass 1: integral from each node on
    double total = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        int kx = 0, ky = 0;
        double cur = s0, acc = 0.0;
        for (int k = 0; k < ns;) {
            double nxt = s0 + k * h;
            if (hx && kx <= nx && sx(kx) < nxt) nxt = sx(kx);
            if (hy && ky <= ny && sy(ky) < nxt) nxt = sy(ky);
            if (nxt > cur) {
                const double mid = 0.5 * (cur + nxt);
                const double px = mid * c - u * sn, py = mid * sn + u * c;
                const int ix = (int)floor((px - xmin) / dpx), iy = (int)floor((py - ymin) / dpx);
                if (ix >= 0 && ix < nx && iy >= 0 && iy < ny) acc += (double)mu[(size_t)iy * nx + ix] * (nxt - cur);
                cur = nxt;
            }
            if (hx && kx <= nx && sx(kx) <= cur) {
                ++kx;
                continue;
            }
            if (hy && ky <= ny && sy(ky) <= cur) {
                ++ky;
                continue;
            }
            if (pass == 1) row[k] = (float)(total - acc);  // integral over [s_k, end)
            ++k;
        }
        total = acc;  // the last node lies beyond the grid
    }
}

// training samples: scaled features and log of the exact scatter entry for
// (event ids[k], every support pixel); rows of the caller's order
__global__ void k_samples(FeatArgs F, const float* __restrict__ model, int64_t ld,
                          const int64_t* __restrict__ rank, int64_t n_ev, float* __restrict__ feat,
                          float* __restrict__ targ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ev * F.n_sup) return;
    const int64_t k = i / F.n_sup;
    const int q = (int)(i % F.n_sup);
    const int64_t row = rank[k];
    float f[kIn];
    features(F, row, q, f);
#pragma unroll
    for (int c = 0; c < kIn; ++c) feat[i * kIn + c] = f[c];
    targ[i] = logf(fmaxf(model[row * ld + q], 1e-30f));
}

// rel[k * n_sup + q] = targ[k * n_sup + q] - max over q' of targ[k * n_sup + q']
// (one block per event row)
__global__ void k_row_rel(const float* __restrict__ targ, int n_sup, float* __restrict__ rel) {
    __shared__ float sm[256];
    const float* row = targ + (int64_t)blockIdx.x * n_sup;
    float m = -FLT_MAX;
    for (int q = threadIdx.x; q < n_sup; q += blockDim.x) m = fmaxf(m, row[q]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    m = sm[0];
    for (int q = threadIdx.x; q < n_sup; q += blockDim.x) rel[(int64_t)blockIdx.x * n_sup + q] = row[q] - m;
}

// targets floored per event row: t_i raised to (its row's largest - F), the
// row maximum being t_i - rel_i
__global__ void k_row_floor(const float* __restrict__ t, const float* __restrict__ rel, int64_t n, float F,
                            float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ti = t[i];
        out[i] = rel[i] < -F ? ti - rel[i] - F : ti;
    }
}

// inclusive prefix sums of w_i = exp(alpha rel_i) in FP64: per-chunk sums,
// their scan (one block, in order), then each chunk's scan from its offset
constexpr int kCdfChunk = 4096;
__global__ void k_cdf_chunks(const float* __restrict__ rel, int64_t n, float alpha, double* __restrict__ csum) {
    __shared__ double sh[256];
    const int64_t c0 = (int64_t)blockIdx.x * kCdfChunk;
    double a = 0.0;
    for (int64_t i = c0 + threadIdx.x; i < min(n, c0 + kCdfChunk); i += blockDim.x) a += exp((double)alpha * rel[i]);
    sh[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) s += sh[k];
        csum[blockIdx.x] = s;
    }
}
__global__ void k_cdf_offsets(double* __restrict__ csum, int64_t nchunks) {
    if (threadIdx.x != 0) return;
    double acc = 0.0;  // exclusive scan in place
    for (int64_t k = 0; k < nchunks; ++k) {
        const double v = csum[k];
        csum[k] = acc;
        acc += v;
    }
}
__global__ void k_cdf_fill(const float* __restrict__ rel, int64_t n, float alpha, const double* __restrict__ off,
                           double* __restrict__ cdf) {
    if (threadIdx.x != 0) return;  // one thread per chunk, in order
    const int64_t c0 = (int64_t)blockIdx.x * kCdfChunk;
    double acc = off[blockIdx.x];
    for (int64_t i = c0; i < min(n, c0 + kCdfChunk); ++i) {
        acc += exp((double)alpha * rel[i]);
        cdf[i] = acc;
    }
}

// surrogate inputs of rows [r0, r0 + nrows) x all support pixels, BF16; with
// a row list, of its entries r0 .. r0 + nrows - 1 instead
__global__ void k_surr_inputs(FeatArgs F, const int64_t* __restrict__ rows, int64_t r0, int64_t nrows,
                              __nv_bfloat16* __restrict__ X, bool tiled) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows * F.n_sup) return;
    const int64_t k = r0 + i / F.n_sup;
    float f[kIn];
    features(F, rows ? rows[k] : k, (int)(i % F.n_sup), f);
#pragma unroll
    for (int k = 0; k < kInPad; ++k) X[x_index(i, k, tiled)] = __float2bfloat16_rn(k < kIn ? f[k] : 0.0f);
}

// p_jn = primary_jn + exp(mu + sigma y_jn) into the FP32 model rows (rows as
// in k_surr_inputs)
__global__ void k_surr_combine(FeatArgs F, const int64_t* __restrict__ rows, const float* __restrict__ y,
                               int64_t r0, int64_t nrows, int n_sup, int64_t ld, const int32_t* __restrict__ a_s,
                               const float* __restrict__ u_s, const float* __restrict__ e_s,
                               const float4* __restrict__ ppar, int ld_w, float e0, float sE0, float lE0,
                               const float* __restrict__ blob, float* __restrict__ model) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows * ld) return;
    const int64_t row = rows ? rows[r0 + i / ld] : r0 + i / ld;
    const int q = (int)(i % ld);
    float v = 0.0f;
    if (q < n_sup) {
        const int a = a_s[row];
        const float4 pp = ppar[(size_t)a * ld_w + q];
        const float te = (e_s[row] - e0) * sE0;
        const float t = (u_s[row] - pp.x) * pp.y;
        const float prim = ex2_approx(fmaf(-t, t, pp.z + fmaf(-te, te, lE0)));
        float x[kIn];
        features(F, row, q, x);
        const float ls = baseline(blob, x) + blob[kOffMu] + blob[kOffSigma] * y[(i / ld) * n_sup + q];
        v = prim + expf(ls);
    }
    model[row * ld + q] = v;
}

// ---------------------------------------------------------------- host helpers

struct MlpBufs {
    __nv_bfloat16 *w1 = nullptr, *w234 = nullptr, *w234t = nullptr;
    unsigned char* wimg = nullptr;  // hidden weights in the operand layout of the tcgen05 kernel
};


// the products run on the tcgen05 kernel (mlp_tc.cu); splits > 1 splits K,
// each split writing its own FP32 slice of C (M ldc elements apart)
lmosem_status gemm(lmosem_ctx* c, int epi, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B,
                   int64_t ldb, void* C, int64_t ldc, const float* bias, const __nv_bfloat16* mask,
                   int64_t ldm, int64_t M, int N, int K, int splits = 1) {
    GemmTcArgs G;
    G.A = A;
    G.lda = lda;
    G.B = B;
    G.ldb = ldb;
    G.C = C;
    G.ldc = ldc;
    G.split_stride = M * ldc;
    G.bias = bias;
    G.mask = mask;
    G.ldm = ldm;
    G.M = M;
    G.N = N;
    G.K = K;
    G.k_per_split = K;
    G.status = nullptr;
    G.budget = 0;
    return gemm_tc(c, epi, G, splits);
}

lmosem_status transpose(lmosem_ctx* c, const __nv_bfloat16* in, int64_t rows, int cols, int64_t ldi,
                        __nv_bfloat16* out, int64_t ldo) {
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    LMOSEM_PROF_BEGIN(c);
    k_transpose<<<grid, dim3(32, 8), 0, c->stream>>>(in, rows, cols, ldi, out, ldo);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    return LMOSEM_OK;
}

lmosem_status weights_bf16(lmosem_ctx* c, const float* blob, MlpBufs& w) {
    LMOSEM_PROF_BEGIN(c);
    k_weights_bf16<<<(3 * kH * kH + 255) / 256, 256, 0, c->stream>>>(blob, w.w1, w.w234, w.w234t);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    return LMOSEM_OK;
}

// BF16 weights for inference: the row-major copies and, for the tcgen05
// kernel, the chunked operand image
lmosem_status infer_weights(lmosem_ctx* c, const float* blob, MlpBufs& w, Scratch& tmp) {
    lmosem_status st;
    if ((st = weights_bf16(c, blob, w))) return st;
    if (c->surrogate_kernel == 1) return LMOSEM_OK;
    if ((st = tmp.alloc(&w.wimg, (size_t)3 * kH * kH * 2))) return st;
    return weights_img(c, w.w234, w.wimg);
}

// forward of M rows: X (M x 16) -> H[0..3] (M x 256 each) -> y (M)
lmosem_status forward(lmosem_ctx* c, const float* blob, const MlpBufs& w, const __nv_bfloat16* X,
                      __nv_bfloat16* const H[4], float* y, int64_t M) {
    lmosem_status st;
    if ((st = gemm(c, EPI_RELU_BF16, X, kInPad, w.w1, kInPad, H[0], kH, blob + kOffB1, nullptr, 0, M, kH, kInPad)))
        return st;
    for (int l = 0; l < 3; ++l)
        if ((st = gemm(c, EPI_RELU_BF16, H[l], kH, w.w234 + (int64_t)l * kH * kH, kH, H[l + 1], kH,
                       blob + kOffB2 + (int64_t)l * (kH * kH + kH), nullptr, 0, M, kH, kH)))
            return st;
    LMOSEM_PROF_BEGIN(c);
    k_out_fwd<<<(unsigned)((M + 7) / 8), 256, 0, c->stream>>>(H[3], M, blob, y);
    LMOSEM_LAUNCHED(c, LMOSEM_K_MLP);
    return LMOSEM_OK;
}

// inference: the tcgen05 kernel (mlp_tc.cu) unless the options select the
// chain of separate tcgen05 products (surrogate_kernel == 1), which the training uses
lmosem_status forward_infer(lmosem_ctx* c, const float* blob, const MlpBufs& w, const __nv_bfloat16* X,
                            __nv_bfloat16* const H[4], float* y, int64_t M) {
    if (c->surrogate_kernel != 1) return forward_tc(c, blob, w.w1, w.wimg, X, y, M);
    return forward(c, blob, w, X, H, y, M);
}

// batch rows of the transposed operands (a multiple of the product's K step)
inline int padded_batch(int B) { return (B + 15) / 16 * 16; }
// K splits of the weight-gradient products (K = the batch): about 256 rows
// each, so that the 2 x 2 output tiles of a layer occupy the SMs
inline int wgrad_splits(int Bp) { return std::max(1, std::min(32, Bp / 256)); }

struct TrainBufs {
    __nv_bfloat16 *X = nullptr, *XT = nullptr, *H = nullptr, *HT = nullptr, *dz = nullptr, *dzT = nullptr;
    float *t = nullptr, *y = nullptr, *dy = nullptr, *gtmp = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    double* loss = nullptr;
    int* step = nullptr;  // device step counter of a captured training step (nullptr: loss[0])
};

// loss and gradient of one minibatch into tb.grad (blob layout)
lmosem_status loss_grad(lmosem_ctx* c, const float* blob, const MlpBufs& w, TrainBufs& tb, int B) {
    lmosem_status st;
    __nv_bfloat16* H[4] = {tb.H, tb.H + (int64_t)B * kH, tb.H + 2 * (int64_t)B * kH, tb.H + 3 * (int64_t)B * kH};
    if ((st = forward(c, blob, w, tb.X, H, tb.y, B))) return st;
    __nv_bfloat16* dz = tb.dz;                       // B x 256, current layer
    LMOSEM_PROF_BEGIN(c);
    k_out_bwd<<<B, 128, 0, c->stream>>>(tb.y, tb.t, H[3], B, blob, tb.dy, dz, tb.loss, tb.step);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    LMOSEM_PROF_BEGIN(c);
    k_out_wgrad<<<kOutSplits, kH + 32, 0, c->stream>>>(tb.dy, H[3], B, tb.gtmp);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    LMOSEM_PROF_BEGIN(c);
    k_out_wgrad_sum<<<2, 256, 0, c->stream>>>(tb.gtmp, tb.grad);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    for (int l = 3; l >= 0; --l) {                   // hidden layer l + 1 (0-based l)
        // dW = dz^T h_prev, db = row sums of dz^T
        // (the transposes keep their rows Bp = B rounded up to 16 long; the
        // tail columns stay zero, so K = Bp adds nothing)
        const int Bp = padded_batch(B);
        if ((st = transpose(c, dz, B, kH, kH, tb.dzT, Bp))) return st;
        const int in = l == 0 ? kInPad : kH;
        const __nv_bfloat16* hprev = l == 0 ? tb.X : H[l - 1];
        if ((st = transpose(c, hprev, B, in, in, tb.HT, Bp))) return st;
        const int splits = wgrad_splits(Bp);
        if ((st = gemm(c, EPI_F32, tb.dzT, Bp, tb.HT, Bp, tb.gtmp, in, nullptr, nullptr, 0, kH, in, Bp, splits)))
            return st;
        const int64_t offW = l == 0 ? kOffW1 : kOffW2 + (int64_t)(l - 1) * (kH * kH + kH);
        const int64_t offB = l == 0 ? kOffB1 : offW + kH * kH;
        const int cols = l == 0 ? kIn : kH;
        LMOSEM_PROF_BEGIN(c);
        k_copy_grad<<<(kH * cols + 255) / 256, 256, 0, c->stream>>>(tb.gtmp, kH, cols, in, splits,
                                                                     (int64_t)kH * in, tb.grad + offW);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        LMOSEM_PROF_BEGIN(c);
        k_rowsum<<<kH / 8, 256, 0, c->stream>>>(tb.dzT, kH, B, Bp, tb.grad + offB);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        if (l > 0) {
            // dz_prev = (dz W_l) where h_prev > 0
            __nv_bfloat16* nxt = dz == tb.dz ? tb.dz + (int64_t)B * kH : tb.dz;
            if ((st = gemm(c, EPI_MASK_BF16, dz, kH, w.w234t + (int64_t)(l - 1) * kH * kH, kH, nxt, kH, nullptr,
                           hprev, kH, B, kH, kH)))
                return st;
            dz = nxt;
        }
    }
    return LMOSEM_OK;
}

}  // namespace

// ---------------------------------------------------------------- entry points

lmosem_status run_surrogate_grad(lmosem_ctx* c, const float* blob, const float* feat, const float* targ,
                                 int64_t n, float* grad_out, double* h_loss) {
    lmosem_status st;
    if ((st = gemm_tc_setup(c))) return st;
    const int B = (int)n;
    MlpBufs w;
    TrainBufs tb;
    Scratch tmp(c);
    if ((st = tmp.alloc(&w.w1, kH * kInPad)) || (st = tmp.alloc(&w.w234, 3 * kH * kH)) ||
        (st = tmp.alloc(&w.w234t, 3 * kH * kH)) || (st = tmp.alloc(&tb.X, (size_t)B * kInPad)) ||
        (st = tmp.alloc(&tb.XT, (size_t)B * kInPad)) || (st = tmp.alloc(&tb.H, (size_t)4 * B * kH)) ||
        (st = tmp.alloc(&tb.HT, (size_t)padded_batch(B) * kH)) || (st = tmp.alloc(&tb.dz, (size_t)2 * B * kH)) ||
        (st = tmp.alloc(&tb.dzT, (size_t)padded_batch(B) * kH)) || (st = tmp.alloc(&tb.t, B)) ||
        (st = tmp.alloc(&tb.y, B)) || (st = tmp.alloc(&tb.dy, B)) ||
        (st = tmp.alloc(&tb.gtmp, (size_t)wgrad_splits(padded_batch(B)) * kH * kH)) || (st = tmp.alloc(&tb.loss, 1)))
        return st;
    LMOSEM_CK(c, cudaMemsetAsync(tb.HT, 0, sizeof(__nv_bfloat16) * padded_batch(B) * kH, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(tb.dzT, 0, sizeof(__nv_bfloat16) * padded_batch(B) * kH, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(grad_out, 0, sizeof(float) * kParams, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(tb.loss, 0, sizeof(double), c->stream));
    if ((st = weights_bf16(c, blob, w))) return st;
    LMOSEM_PROF_BEGIN(c);
    k_gather<<<(B + 255) / 256, 256, 0, c->stream>>>(feat, targ, n, B, 0, 0, nullptr, nullptr, blob, nullptr, tb.X,
                                                     tb.t, false);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    tb.grad = grad_out;
    if ((st = loss_grad(c, blob, w, tb, B))) return st;
    double h = 0.0;
    LMOSEM_CK(c, cudaMemcpyAsync(&h, tb.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (h_loss) *h_loss = h;
    return LMOSEM_OK;
}

// The quadratic baseline's coefficients into the blob: a least-squares fit
// to the floored targets of up to 2^20 evenly spaced samples (FP64 normal
// equations, Cholesky with a relative ridge of 1e-10), or zeros.
lmosem_status fit_baseline(lmosem_ctx* c, const float* feat, const float* targ, int64_t n, const float* d_floor,
                           bool fit, float* blob) {
    float coef[kBasis] = {};
    if (fit) {
        const int64_t m = std::min<int64_t>(n, int64_t(1) << 20);
        double* d_ne = nullptr;
        Scratch tmp(c);
        lmosem_status st;
        if ((st = tmp.alloc(&d_ne, (size_t)kBasis * (kBasis + 1)))) return st;
        LMOSEM_CK(c, cudaMemsetAsync(d_ne, 0, sizeof(double) * kBasis * (kBasis + 1), c->stream));
        LMOSEM_PROF_BEGIN(c);
        k_basis_normal<<<dim3(kBasis, kBasis + 1), 256, 0, c->stream>>>(feat, targ, n, m, d_floor, d_ne);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        double ne[kBasis * (kBasis + 1)];
        LMOSEM_CK(c, cudaMemcpyAsync(ne, d_ne, sizeof(ne), cudaMemcpyDeviceToHost, c->stream));
        LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
        // A = sum phi phi^T (lower triangle), r = sum phi t; A x = r by Cholesky
        double A[kBasis][kBasis], L[kBasis][kBasis] = {}, r[kBasis], x[kBasis];
        double tr = 0.0;
        for (int i = 0; i < kBasis; ++i) {
            for (int j = 0; j <= i; ++j) A[i][j] = A[j][i] = ne[i * (kBasis + 1) + j];
            r[i] = ne[i * (kBasis + 1) + kBasis];
            tr += A[i][i];
        }
        for (int i = 0; i < kBasis; ++i) A[i][i] += 1e-10 * tr / kBasis;
        for (int i = 0; i < kBasis; ++i) {
            for (int j = 0; j <= i; ++j) {
                double sum = A[i][j];
                for (int k = 0; k < j; ++k) sum -= L[i][k] * L[j][k];
                if (i == j) {
                    if (!(sum > 0.0)) return fail(c, LMOSEM_ENUMERIC, "baseline fit: singular normal equations");
                    L[i][i] = sqrt(sum);
                } else {
                    L[i][j] = sum / L[j][j];
                }
            }
        }
        for (int i = 0; i < kBasis; ++i) {  // L z = r, then L^T x = z
            double sum = r[i];
            for (int k = 0; k < i; ++k) sum -= L[i][k] * x[k];
            x[i] = sum / L[i][i];
        }
        for (int i = kBasis - 1; i >= 0; --i) {
            double sum = x[i];
            for (int k = i + 1; k < kBasis; ++k) sum -= L[k][i] * x[k];
            x[i] = sum / L[i][i];
        }
        for (int i = 0; i < kBasis; ++i) coef[i] = (float)x[i];
    }
    LMOSEM_CK(c, cudaMemcpyAsync(blob + kOffBase, coef, sizeof(coef), cudaMemcpyHostToDevice, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));  // coef is on this stack frame
    return LMOSEM_OK;
}

lmosem_status run_surrogate_train(lmosem_ctx* c, const float* feat, const float* targ, const float* rel,
                                  int64_t n, int steps, int B, float lr, uint64_t seed, float floor_below,
                                  bool residual_fit, float magnitude_power, float* blob, double* h_loss_curve) {
    lmosem_status st;
    if ((st = gemm_tc_setup(c))) return st;
    MlpBufs w;
    TrainBufs tb;
    double* d_curve = nullptr;
    float* d_floor = nullptr;
    int* d_step = nullptr;
    float* d_sc = nullptr;
    double *d_cdf = nullptr, *d_csum = nullptr;
    float* tf = nullptr;  // (Scratch keeps the address of the pointer: same scope as tmp)
    Scratch tmp(c);
    if (rel && floor_below > 0.0f) {  // floor per event row: the targets floored once
        if ((st = tmp.alloc(&tf, (size_t)n))) return st;
        LMOSEM_PROF_BEGIN(c);
        k_row_floor<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, c->stream>>>(targ, rel, n,
                                                                                               floor_below, tf);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        targ = tf;
        floor_below = 0.0f;
    }
    if ((st = tmp.alloc(&w.w1, kH * kInPad)) || (st = tmp.alloc(&w.w234, 3 * kH * kH)) ||
        (st = tmp.alloc(&w.w234t, 3 * kH * kH)) || (st = tmp.alloc(&tb.X, (size_t)B * kInPad)) ||
        (st = tmp.alloc(&tb.H, (size_t)4 * B * kH)) || (st = tmp.alloc(&tb.HT, (size_t)padded_batch(B) * kH)) ||
        (st = tmp.alloc(&tb.dz, (size_t)2 * B * kH)) || (st = tmp.alloc(&tb.dzT, (size_t)padded_batch(B) * kH)) ||
        (st = tmp.alloc(&tb.t, B)) || (st = tmp.alloc(&tb.y, B)) || (st = tmp.alloc(&tb.dy, B)) ||
        (st = tmp.alloc(&tb.gtmp, (size_t)wgrad_splits(padded_batch(B)) * kH * kH)) ||
        (st = tmp.alloc(&tb.grad, kParams)) ||
        (st = tmp.alloc(&tb.m, kParams)) || (st = tmp.alloc(&tb.v, kParams)) ||
        (st = tmp.alloc(&d_curve, std::max(1, steps))) || (st = tmp.alloc(&d_floor, 1)) ||
        (st = tmp.alloc(&d_step, 1)) || (st = tmp.alloc(&d_sc, 3)))
        return st;
    LMOSEM_CK(c, cudaMemsetAsync(tb.m, 0, sizeof(float) * kParams, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(tb.v, 0, sizeof(float) * kParams, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(d_curve, 0, sizeof(double) * std::max(1, steps), c->stream));
    LMOSEM_PROF_BEGIN(c);
    k_target_floor<<<1, 256, 0, c->stream>>>(targ, n, floor_below, d_floor);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    if ((st = fit_baseline(c, feat, targ, n, d_floor, residual_fit, blob))) return st;
    LMOSEM_PROF_BEGIN(c);
    k_target_stats<<<1, 256, 0, c->stream>>>(targ, feat, n, d_floor, blob);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    const float b1 = 0.9f, b2 = 0.999f;
    // one training step: its scalars (minibatch index, loss slot, learning
    // rate, bias corrections) come from the device step counter, so the step
    // is captured once as a CUDA graph and replayed (direct launches on a
    // stream that cannot be captured)
    LMOSEM_CK(c, cudaMemsetAsync(d_step, 0, sizeof(int), c->stream));
    if ((st = ensure_status(c))) return st;  // before any capture: the products report to it
    if (rel && magnitude_power > 0.0f) {    // sampling weights (entry / row maximum)^alpha
        const int64_t nchunks = (n + kCdfChunk - 1) / kCdfChunk;
        if ((st = tmp.alloc(&d_cdf, (size_t)n)) || (st = tmp.alloc(&d_csum, (size_t)nchunks))) return st;
        LMOSEM_PROF_BEGIN(c);
        k_cdf_chunks<<<(unsigned)nchunks, 256, 0, c->stream>>>(rel, n, magnitude_power, d_csum);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        LMOSEM_PROF_BEGIN(c);
        k_cdf_offsets<<<1, 32, 0, c->stream>>>(d_csum, nchunks);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        LMOSEM_PROF_BEGIN(c);
        k_cdf_fill<<<(unsigned)nchunks, 32, 0, c->stream>>>(rel, n, magnitude_power, d_csum, d_cdf);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    }
    tb.loss = d_curve;
    tb.step = d_step;
    auto enqueue_step = [&]() -> lmosem_status {
        lmosem_status s2;
        if ((s2 = weights_bf16(c, blob, w))) return s2;
        LMOSEM_PROF_BEGIN(c);
        k_gather<<<(B + 255) / 256, 256, 0, c->stream>>>(feat, targ, n, B, seed | 1ull, 0, d_step, d_cdf, blob,
                                                         d_floor, tb.X, tb.t, false);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        if ((s2 = loss_grad(c, blob, w, tb, B))) return s2;
        LMOSEM_PROF_BEGIN(c);
        k_step_scalars<<<1, 1, 0, c->stream>>>(d_step, steps, lr, b1, b2, d_sc);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        LMOSEM_PROF_BEGIN(c);
        k_adam<<<(unsigned)((kOffBase + 255) / 256), 256, 0, c->stream>>>(blob, tb.grad, tb.m, tb.v, kOffBase, d_sc, b1,
                                                                       b2, 1e-8f, d_step);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        return LMOSEM_OK;
    };
    cudaGraphExec_t exec = nullptr;
    int64_t step_launches = 0;
    if (steps > 1 && c->stream != nullptr && c->profile != 1 &&
        cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int64_t before = c->launches;
        c->capturing = true;
        st = enqueue_step();
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (!st && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st) return st;
        if (e != cudaSuccess) return cuda_fail(c, e, "training-step graph");
        step_launches = c->launches - before;
        c->launches = before;
    } else {
        cudaGetLastError();
    }
    for (int s = 0; s < steps; ++s) {
        if (exec) {
            cudaError_t e = cudaGraphLaunch(exec, c->stream);
            if (e != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return cuda_fail(c, e, "cudaGraphLaunch");
            }
            c->launches += step_launches;
        } else if ((st = enqueue_step())) {
            return st;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (h_loss_curve && steps > 0)
        LMOSEM_CK(c, cudaMemcpyAsync(h_loss_curve, d_curve, sizeof(double) * steps, cudaMemcpyDeviceToHost,
                                     c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    return LMOSEM_OK;
}

lmosem_status run_surrogate_infer(lmosem_ctx* c, const float* blob, const float* feat, int64_t n,
                                  float* out) {
    lmosem_status st;
    if ((st = gemm_tc_setup(c))) return st;
    MlpBufs w;
    __nv_bfloat16 *X = nullptr, *H = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&w.w1, kH * kInPad)) || (st = tmp.alloc(&w.w234, 3 * kH * kH)) ||
        (st = tmp.alloc(&w.w234t, 3 * kH * kH)) || (st = tmp.alloc(&X, (size_t)((n + 127) / 128 * 128) * kInPad)) ||
        (c->surrogate_kernel == 1 && (st = tmp.alloc(&H, (size_t)4 * n * kH))))
        return st;
    if ((st = infer_weights(c, blob, w, tmp))) return st;
    LMOSEM_PROF_BEGIN(c);
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(feat, feat, n, (int)n, 0, 0, nullptr, nullptr, blob, nullptr, X, out,
                                                                 c->surrogate_kernel != 1);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    __nv_bfloat16* Hs[4] = {H, H + n * kH, H + 2 * n * kH, H + 3 * n * kH};
    if ((st = forward_infer(c, blob, w, X, Hs, out, n))) return st;
    st = take_status(c);   // synchronises
    return st;
}

// The detector-line attenuation table of the surrogate's inputs (built once
// per context): nodes h = half a pixel apart across the detector extent,
// starting 3h/4 before it (so that no node line runs along a grid line at
// the axis angles), and along a line's whole crossing of the grid.
lmosem_status ensure_line_table(lmosem_ctx* c) {
    if (c->d_line) return LMOSEM_OK;
    const double h = 0.5 * c->dpx;
    const double U = 0.5 * c->n_bins * c->bin_mm + 0.75 * h;
    const double S = 0.5 * c->dpx * sqrt((double)c->nx * c->nx + (double)c->ny * c->ny) + h;
    const int nu = (int)ceil(2.0 * U / h) + 1, ns = (int)ceil(2.0 * S / h) + 1;
    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_line, (size_t)c->n_angles * nu * ns))) return st;
    c->line_nu = nu;
    c->line_ns = ns;
    c->line_u0 = -U;
    c->line_s0 = -S;
    c->line_h = h;
    const int lines = c->n_angles * nu;
    LMOSEM_PROF_BEGIN(c);
    k_line_table<<<(lines + 127) / 128, 128, 0, c->stream>>>(c->d_mu, c->nx, c->ny, c->dpx, c->n_angles, c->angle0,
                                                             nu, ns, -U, -S, h, c->d_line);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    return LMOSEM_OK;
}

FeatArgs feat_args(lmosem_ctx* c) {
    FeatArgs F;
    F.line = c->d_line;
    F.line_nu = c->line_nu;
    F.line_ns = c->line_ns;
    F.line_u0 = (float)c->line_u0;
    F.line_s0 = (float)c->line_s0;
    F.line_inv_h = (float)(1.0 / c->line_h);
    F.a_s = c->d_a_s;
    F.u_s = c->d_u_s;
    F.e_s = c->d_e_s;
    F.sup = c->d_sup;
    F.n_sup = c->n_sup;
    F.nx = c->nx;
    F.ny = c->ny;
    F.npix = c->npix;
    F.dpx = (float)c->dpx;
    F.l_edge = c->d_l_edge;
    F.angle0 = (float)c->angle0;
    F.dtheta = (float)(2.0 * kPi / c->n_angles);
    return F;
}

// features and log exact scatter of every (event, support pixel) of the
// current (scatter-only, FP32) model, in the caller's event order
lmosem_status run_surrogate_samples(lmosem_ctx* c, float* feat, float* targ, float* rel) {
    const int64_t total = c->J * c->n_sup;
    lmosem_status st;
    if ((st = ensure_line_table(c))) return st;
    // the sort's rank maps the caller's event k to its model row
    LMOSEM_PROF_BEGIN(c);
    k_samples<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(
        feat_args(c), reinterpret_cast<const float*>(c->d_model), c->ld_model, c->d_rank, c->J, feat, targ);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    if (rel) {
        LMOSEM_PROF_BEGIN(c);
        k_row_rel<<<(unsigned)c->J, 256, 0, c->stream>>>(targ, c->n_sup, rel);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    }
    return LMOSEM_OK;
}

// model rows with the surrogate scatter term, in chunks of whole rows: all J
// rows (d_rows == nullptr) or the n sorted rows d_rows lists
lmosem_status build_model_surrogate_rows(lmosem_ctx* c, const int64_t* d_rows, int64_t n) {
    lmosem_status st;
    const int64_t n_rows = d_rows ? n : c->J;
    if ((st = gemm_tc_setup(c))) return st;
    if ((st = ensure_line_table(c))) return st;
    // pairs per chunk: the product chain keeps two 256-wide BF16 activations
    // per pair in HBM, the fused tcgen05 kernel none
    const int64_t max_pairs = int64_t(1) << (c->surrogate_kernel == 1 ? 20 : 24);
    const int64_t rows_per = std::max<int64_t>(1, max_pairs / c->n_sup);
    const int64_t M = rows_per * c->n_sup;
    MlpBufs w;
    __nv_bfloat16 *X = nullptr, *H = nullptr;
    float* y = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&w.w1, kH * kInPad)) || (st = tmp.alloc(&w.w234, 3 * kH * kH)) ||
        (st = tmp.alloc(&w.w234t, 3 * kH * kH)) || (st = tmp.alloc(&X, (size_t)((M + 127) / 128 * 128) * kInPad)) ||
        (c->surrogate_kernel == 1 && (st = tmp.alloc(&H, (size_t)2 * M * kH))) || (st = tmp.alloc(&y, M)))
        return st;
    if ((st = infer_weights(c, c->d_surrogate, w, tmp))) return st;
    const double fw2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    const double se0 = fw2s * c->fwhm_frac * c->e0;
    __nv_bfloat16* Hs[4] = {H, H + M * kH, H, H + M * kH};  // ping-pong
    for (int64_t r0 = 0; r0 < n_rows; r0 += rows_per) {
        const int64_t nr = std::min(rows_per, n_rows - r0);
        const int64_t m = nr * c->n_sup;
        LMOSEM_PROF_BEGIN(c);
        k_surr_inputs<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(feat_args(c), d_rows, r0, nr, X,
                                                                          c->surrogate_kernel != 1);
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
        if ((st = forward_infer(c, c->d_surrogate, w, X, Hs, y, m))) return st;
        LMOSEM_PROF_BEGIN(c);
        k_surr_combine<<<(unsigned)((nr * c->ld_model + 255) / 256), 256, 0, c->stream>>>(
            feat_args(c), d_rows, y, r0, nr, c->n_sup, c->ld_model, c->d_a_s, c->d_u_s, c->d_e_s, c->d_ppar, c->ld_w, (float)c->e0,
            (float)(0.8493218002880191 / se0), (float)(-log2(se0 * sqrt(2.0 * kPi))), c->d_surrogate,
            reinterpret_cast<float*>(c->d_model));
        LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    }
    st = take_status(c);   // synchronises
    return st;
}

lmosem_status build_model_surrogate(lmosem_ctx* c) { return build_model_surrogate_rows(c, nullptr, 0); }

}  // namespace lmosem
