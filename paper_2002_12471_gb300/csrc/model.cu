// System-model build (rows a2-a5 of the hot path): the per-event path sum
//
//   p_jn = w_0(n) k_0(u_j, E_j | n)
//        + sum_{m in strip(j)} U_jm W_a(n, m) phi(E_j; E'_a(n, m), sigma_E(E'))
//
// of paper Eq. 2 with Eq. 4 (pr(A_j|P) s_eff(P) summed over the primary path
// (n) and the first-order in-plane scatter paths (n, m), Section 2.2), where
// U_jm = phi(u_j; u_a(m), sigma_u(d_a(m))) is the collimator response at the
// scatter pixel, W_a(n, m) the attenuated, Klein-Nishina-weighted scatter
// weight and E' the Compton energy.  The denominator of Eq. 8 is y_j =
// sum_n p_jn f_n, so caching p turns every OSEM sub-iteration into a
// streaming pass.
//
// Per angle a, three planes s, b and -lw are tabulated for every (m, n), with
// lw = log2(W / (sigma_E(E') sqrt(2 pi))), s = sqrt(log2 e / 2) / sigma_E(E')
// and b = -E' s, so that every term is
//     U_jm * 2^-(t^2 - lw),   t = E_j s + b,
// i.e. one FMA for t, one for t^2 - lw, one MUFU ex2 and one FMA into the
// accumulator.  The FMAs run as packed FP32x2 instructions (two support
// pixels per instruction), so a pair of terms costs three FFMA2 and two
// ex2: the kernel is bound by the MUFU pipe.
//
// A CTA owns 64 events of one angle (consecutive in position) x 128 support
// pixels and walks the scatter pixels whose kernel reaches any of its events
// (|u_j - u_m| <= k_sigma sigma_u(m)); terms outside that cut for a given
// event are exactly zero.  The table slices of the next 16 scatter pixels are
// copied into shared memory with cp.async while the current 16 are summed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kStage = 16;  // scatter pixels per pipeline stage

struct WTabArgs {
    int nx, ny, npix;
    float dpx;
    const int32_t* sup;
    int n_sup, ld_w;
    const int32_t* scat;
    int n_scat;
    const float* mu;
    const float2* trig;
    const float* l_edge;
    const float* l_pair;
    const float2* compton;
    const int32_t* slot_angle;  // angle of each sorted slot
    int s0;                     // first slot of the group
    float eps0, inv_kbar, e0;
    float w_const;              // D^2 / (2 pi sqrt(2 pi kappa)), sigma_E^2 = kappa E
    float cE;                   // s = cE / sqrt(E')
    float* wtab;                // [slot - s0][plane s, b, -lw][m][ld_w]
};

// planes (s, b, -lw) of the scatter path (n, m) at the angle of one slot
__global__ void k_wtable(WTabArgs A) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    int g = blockIdx.z;
    if (n >= A.ld_w) return;
    float s = 0.0f, b = 0.0f, nlw = INFINITY;
    if (n < A.n_sup) {
        int a = A.slot_angle[A.s0 + g];
        int pn = A.sup[n], pm = A.scat[k];
        float cpsi, rinv;
        if (path_geometry(pn, pm, A.nx, A.ny, A.dpx, A.trig[a], &cpsi, &rinv)) {
            float P, kt;
            compton(cpsi, A.eps0, A.inv_kbar, &P, &kt);
            float e1 = A.e0 * P;
            float ratio = compton_lookup(A.compton, cpsi).x;
            float att = A.l_pair[(size_t)k * A.n_sup + n] + ratio * A.l_edge[(size_t)a * A.npix + pm];
            float ri = rsqrtf(e1);
            nlw = att * kLog2e - log2f(A.w_const * A.mu[pm] * kt * rinv * ri);
            s = A.cE * ri;
            b = -e1 * s;
        }
    }
    size_t plane = (size_t)A.n_scat * A.ld_w;
    float* base = A.wtab + (size_t)g * 3 * plane + (size_t)k * A.ld_w + n;
    base[0] = s;
    base[plane] = b;
    base[2 * plane] = nlw;
}

// Every angle's planes (s, b, -lw) (indexed by angle) and, in the same pass,
// the per-angle subset-sensitivity sum of s_eff = w D_u D_E over the primary
// and every scatter path of support pixel n (paper Eq. 7 denominator): the
// terms are formed as in k_wtable and k_sens_angle (FP32 terms, added into
// an FP64 accumulator every 32 scatter pixels), so both results are bitwise
// those of the two separate kernels.
struct WSensArgs {
    WTabArgs w;
    const float4* ppar;   // .w = D_u of the primary
    const float* du_m;    // [a][m]
    float w_const_sens;   // D^2 / (2 pi)
    float de0;            // window mass of the photopeak
    double* sens_angle;   // [a][n]
};

__global__ void k_wtable_sens(WSensArgs S) {
    const WTabArgs& A = S.w;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (n >= A.ld_w) return;
    const size_t plane = (size_t)A.n_scat * A.ld_w;
    float* base = A.wtab + (size_t)a * 3 * plane + n;
    if (n >= A.n_sup) {  // padding columns: no path
        for (int k = 0; k < A.n_scat; ++k) {
            base[(size_t)k * A.ld_w] = 0.0f;
            base[plane + (size_t)k * A.ld_w] = 0.0f;
            base[2 * plane + (size_t)k * A.ld_w] = INFINITY;
        }
        return;
    }
    const int pn = A.sup[n];
    const float2 trig = A.trig[a];
    double acc = (double)(expf(-A.l_edge[(size_t)a * A.npix + pn]) * S.ppar[(size_t)a * A.ld_w + n].w * S.de0);
    const float* lp = A.l_pair + n;
    const float* le = A.l_edge + (size_t)a * A.npix;
    const float* du = S.du_m + (size_t)a * A.n_scat;
    float part = 0.0f;
    for (int k = 0; k < A.n_scat; ++k) {
        const int pm = __ldg(A.scat + k);
        float s = 0.0f, b = 0.0f, nlw = INFINITY;
        float cpsi, rinv;
        if (path_geometry(pn, pm, A.nx, A.ny, A.dpx, trig, &cpsi, &rinv)) {
            float P, kt;
            compton(cpsi, A.eps0, A.inv_kbar, &P, &kt);
            const float2 cr = compton_lookup(A.compton, cpsi);  // (mu ratio, window mass)
            const float att = lp[(size_t)k * A.n_sup] + cr.x * __ldg(le + pm);
            const float mu = __ldg(A.mu + pm);
            const float e1 = A.e0 * P;
            const float ri = rsqrtf(e1);
            nlw = att * kLog2e - log2f(A.w_const * mu * kt * rinv * ri);
            s = A.cE * ri;
            b = -e1 * s;
            const float w = S.w_const_sens * mu * kt * rinv * expf(-att);
            part = fmaf(w, __ldg(du + k) * cr.y, part);
        }
        base[(size_t)k * A.ld_w] = s;
        base[plane + (size_t)k * A.ld_w] = b;
        base[2 * plane + (size_t)k * A.ld_w] = nlw;
        if ((k & 31) == 31) {
            acc += (double)part;
            part = 0.0f;
        }
    }
    acc += (double)part;
    S.sens_angle[(size_t)a * A.n_sup + n] = acc;
}

struct PathSumArgs {
    const float* u_s;
    const float* e_s;
    // entries (realisation, angle) of this launch, in sorted-row order
    const int32_t* ent_angle;    // detector angle
    const int32_t* ent_wpos;     // slot of its scatter tables in the group
    const int32_t* ent_row0;     // first sorted row
    const int32_t* ent_cnt;      // rows
    const int32_t* tile_prefix;  // cumulative event tiles, tile_prefix[0] = 0
    int n_ent;
    int n_ptiles;
    const float* wtab;
    int ld_w, n_scat;
    const float4* mpar;          // [a][m]
    const float4* ppar;          // [a][n]
    float e0, sE0, lE0;          // primary energy factor 2^(lE0 - ((E - e0) sE0)^2)
    float* out;                  // FP32 rows
    int64_t ld_out;
    int64_t row_base;            // out row = sorted row - row_base
    int n_store;                 // columns to store (padded row width)
    int scatter_only;            // 1: leave the primary path out
};

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// shared-memory layout of k_pathsum, in floats
constexpr int kPlaneF = kStage * kTN;                 // one plane of one stage
constexpr int kOffPlanes = 0;                         // [2][3][kStage][kTN]
constexpr int kOffU = kOffPlanes + 2 * 3 * kPlaneF;   // [kStage][kTJ] float2
constexpr int kOffMp = kOffU + 2 * kStage * kTJ;      // [2][kStage] float4
constexpr int kOffEv = kOffMp + 2 * kStage * 4;       // u[kTJ], e[kTJ]
constexpr int kOffMisc = kOffEv + 2 * kTJ;            // 16 ints
constexpr int kOffList = kOffMisc + 16;               // n_scat ints

__global__ void __launch_bounds__(kBuildThreads, 2) k_pathsum(PathSumArgs A) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* planes = sm + kOffPlanes;
    float2* sU = reinterpret_cast<float2*>(sm + kOffU);
    float4* mp = reinterpret_cast<float4*>(sm + kOffMp);
    float* ev_u = sm + kOffEv;
    float* ev_e = ev_u + kTJ;
    int* misc = reinterpret_cast<int*>(sm + kOffMisc);
    int* mlist = reinterpret_cast<int*>(sm + kOffList);
    float* red = reinterpret_cast<float*>(misc);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int et = blockIdx.x / A.n_ptiles, pt = blockIdx.x % A.n_ptiles;

    // entry (realisation, angle) of this event tile
    int lo = 0, hi = A.n_ent - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (A.tile_prefix[mid] <= et) lo = mid; else hi = mid - 1;
    }
    const int ent = lo;
    const int a = A.ent_angle[ent];
    const int tile = et - A.tile_prefix[ent];
    const int64_t r0 = (int64_t)A.ent_row0[ent] + (int64_t)tile * kTJ;
    const int nr = min(kTJ, A.ent_cnt[ent] - tile * kTJ);
    const int n0 = pt * kTN;

    if (tid < kTJ) {
        ev_u[tid] = tid < nr ? A.u_s[r0 + tid] : 1e30f;
        ev_e[tid] = tid < nr ? A.e_s[r0 + tid] : 0.0f;
    }
    __syncthreads();
    // position range of the tile's events
    if (warp == 0) {
        float mn = INFINITY, mx = -INFINITY;
        for (int j = lane; j < nr; j += 32) {
            mn = fminf(mn, ev_u[j]);
            mx = fmaxf(mx, ev_u[j]);
        }
        for (int o = 16; o; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            red[8] = mn;
            red[9] = mx;
        }
    }
    __syncthreads();
    const float umin = red[8], umax = red[9];
    __syncthreads();

    // scatter pixels whose cut interval reaches the tile (block compaction)
    const float4* mp_a = A.mpar + (size_t)a * A.n_scat;
    int nm = 0;
    for (int m0 = 0; m0 < A.n_scat; m0 += kBuildThreads) {
        int m = m0 + tid;
        bool in = false;
        if (m < A.n_scat) {
            float4 q = __ldg(mp_a + m);
            in = (q.x + q.w >= umin) && (q.x - q.w <= umax);
        }
        unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) misc[warp] = __popc(bal);
        __syncthreads();
        int off = nm, total = 0;
        for (int w = 0; w < kBuildThreads / 32; ++w) {
            int cw = misc[w];
            if (w < warp) off += cw;
            total += cw;
        }
        if (in) mlist[off + __popc(bal & ((1u << lane) - 1u))] = m;
        __syncthreads();
        nm += total;
    }

    // accumulators (pairs of adjacent support pixels), initialised with the
    // primary path
    float2 E2[8];
    float2 acc[8][2];
    {
        const float4* pp_a = A.ppar + (size_t)a * A.ld_w + n0 + 4 * lane;
        float4 pp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) pp[q] = __ldg(pp_a + q);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            float uj = ev_u[8 * warp + jj];
            float ej = ev_e[8 * warp + jj];
            E2[jj] = make_float2(ej, ej);
            float te = (ej - A.e0) * A.sE0;
            float le = fmaf(-te, te, A.lE0);
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float t = (uj - pp[q].x) * pp[q].y;
                v[q] = A.scatter_only ? 0.0f : ex2_approx(fmaf(-t, t, pp[q].z + le));
            }
            acc[jj][0] = make_float2(v[0], v[1]);
            acc[jj][1] = make_float2(v[2], v[3]);
        }
    }

    // strip staging: three table planes and the position parameters of
    // kStage scatter pixels per stage, double-buffered with cp.async
    const size_t plane = (size_t)A.n_scat * A.ld_w;
    const float* tab = A.wtab + (size_t)A.ent_wpos[ent] * 3 * plane + n0;
    auto issue = [&](int c0, int buf) {
        for (int k = tid; k < 3 * kStage * (kTN / 4); k += kBuildThreads) {
            int p = k / (kStage * (kTN / 4));
            int r = k - p * (kStage * (kTN / 4));
            int mc = r / (kTN / 4), q = r - mc * (kTN / 4);
            float* dst = planes + ((buf * 3 + p) * kStage + mc) * kTN + 4 * q;
            if (c0 + mc < nm) {
                cp_async16(dst, tab + p * plane + (size_t)mlist[c0 + mc] * A.ld_w + 4 * q);
            } else {
                float v = p == 2 ? INFINITY : 0.0f;
                *reinterpret_cast<float4*>(dst) = make_float4(v, v, v, v);
            }
        }
        if (tid < kStage) {
            float4* dst = mp + buf * kStage + tid;
            if (c0 + tid < nm) cp_async16(dst, mp_a + mlist[c0 + tid]);
            else *dst = make_float4(0.0f, 0.0f, -INFINITY, -1.0f);  // cut < 0: U = 0
        }
        cp_async_commit();
    };

    const int nchunks = (nm + kStage - 1) / kStage;
    if (nchunks > 0) issue(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) {
            issue((c + 1) * kStage, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // U_jm of this stage, duplicated into FP32 pairs
        for (int k = tid; k < kStage * kTJ; k += kBuildThreads) {
            int mc = k / kTJ, j = k - mc * kTJ;
            float4 q = mp[buf * kStage + mc];
            float d = ev_u[j] - q.x;
            float z = d * q.y;
            float U = fabsf(d) <= q.w ? ex2_approx(fmaf(-z, z, q.z)) : 0.0f;
            sU[mc * kTJ + j] = make_float2(U, U);
        }
        __syncthreads();
        const float* pS = planes + (buf * 3 + 0) * kPlaneF + 4 * lane;
        const float* pB = planes + (buf * 3 + 1) * kPlaneF + 4 * lane;
        const float* pW = planes + (buf * 3 + 2) * kPlaneF + 4 * lane;
        const float4* pU = reinterpret_cast<const float4*>(sU + 8 * warp);
#pragma unroll 2
        for (int mc = 0; mc < kStage; ++mc) {
            const float4 S = *reinterpret_cast<const float4*>(pS + mc * kTN);
            const float4 B = *reinterpret_cast<const float4*>(pB + mc * kTN);
            const float4 W = *reinterpret_cast<const float4*>(pW + mc * kTN);
            const float4* up = pU + mc * (kTJ / 2);
            float2 U[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 v = up[k];
                U[2 * k] = make_float2(v.x, v.y);
                U[2 * k + 1] = make_float2(v.z, v.w);
            }
            const float2 S01 = make_float2(S.x, S.y), S23 = make_float2(S.z, S.w);
            const float2 B01 = make_float2(B.x, B.y), B23 = make_float2(B.z, B.w);
            const float2 W01 = make_float2(W.x, W.y), W23 = make_float2(W.z, W.w);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                float2 t0 = ffma2(E2[jj], S01, B01);
                float2 t1 = ffma2(E2[jj], S23, B23);
                float2 z0 = ffma2(t0, t0, W01);
                float2 z1 = ffma2(t1, t1, W23);
                float2 e0 = make_float2(ex2_approx(-z0.x), ex2_approx(-z0.y));
                float2 e1 = make_float2(ex2_approx(-z1.x), ex2_approx(-z1.y));
                acc[jj][0] = ffma2(U[jj], e0, acc[jj][0]);
                acc[jj][1] = ffma2(U[jj], e1, acc[jj][1]);
            }
        }
        __syncthreads();
    }

    // store the tile (columns past the support are exact zeros)
    const int n = n0 + 4 * lane;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        int j = 8 * warp + jj;
        if (j >= nr) continue;
        float* row = A.out + (r0 + j - A.row_base) * A.ld_out;
        float v[4] = {acc[jj][0].x, acc[jj][0].y, acc[jj][1].x, acc[jj][1].y};
        if (n + 3 < A.n_store) {
            *reinterpret_cast<float4*>(row + n) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (n + q < A.n_store) row[n + q] = v[q];
        }
    }
}

// Row scaling and rounding of FP32 staged rows: p_jn = c_j h_jn with
// max_n h_jn = hmax (2^15 for FP16 keeps entries down to ~2e-9 of the row
// maximum in the normal range; 1 for BF16).  The scale cancels in the EM
// update (paper Eq. 8: y_j and p_jq scale together) and enters only the
// log-likelihood.
template <typename H>
__global__ void k_quantize(const float* __restrict__ stage, int64_t ld_stage, int64_t rows,
                           int n_cols, int64_t ld_out, H* __restrict__ out, int64_t row0,
                           float* __restrict__ scale, float hmax) {
    int warps = blockDim.x >> 5;
    int64_t r = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float* src = stage + r * ld_stage;
    float mx = 0.0f;
    for (int n = lane; n < n_cols; n += 32) mx = fmaxf(mx, src[n]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float c = mx > 0.0f ? mx / hmax : 1.0f;
    float ic = 1.0f / c;
    H* dst = out + (row0 + r) * ld_out;
    for (int n = lane; n < ld_out; n += 32) {
        float v = n < n_cols ? src[n] * ic : 0.0f;
        if constexpr (std::is_same<H, __half>::value)
            dst[n] = __float2half_rn(v);
        else
            dst[n] = __float2bfloat16_rn(v);
    }
    if (lane == 0) scale[row0 + r] = c;
}

// scatter-table arguments of the context (sigma_E^2 = kappa E)
WTabArgs wtab_args(const lmosem_ctx* c, float* wtab, const int32_t* slot_angle, int s0) {
    const double fw2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    const double kappa = pow(c->fwhm_frac * fw2s, 2.0) * c->e0;
    WTabArgs W;
    W.nx = c->nx;
    W.ny = c->ny;
    W.npix = c->npix;
    W.dpx = (float)c->dpx;
    W.sup = c->d_sup;
    W.n_sup = c->n_sup;
    W.ld_w = c->ld_w;
    W.scat = c->d_scat;
    W.n_scat = c->n_scat;
    W.mu = c->d_mu;
    W.trig = c->d_trig;
    W.l_edge = c->d_l_edge;
    W.l_pair = c->d_l_pair;
    W.compton = c->d_compton;
    W.slot_angle = slot_angle;
    W.s0 = s0;
    W.eps0 = (float)(c->e0 / kMec2Kev);
    W.inv_kbar = (float)(1.0 / c->kbar);
    W.e0 = (float)c->e0;
    W.w_const = (float)(c->dpx * c->dpx / (2.0 * kPi * sqrt(2.0 * kPi * kappa)));
    W.cE = (float)sqrt(1.4426950408889634 / (2.0 * kappa));
    W.wtab = wtab;
    return W;
}

int64_t wtab_angle_floats(const lmosem_ctx* c) { return (int64_t)3 * c->n_scat * c->ld_w; }

}  // namespace

bool wtab_all_fits(const lmosem_ctx* c) {
    return (int64_t)c->n_angles * wtab_angle_floats(c) * (int64_t)sizeof(float) <= c->table_budget;
}

lmosem_status wtab_all_with_sens(lmosem_ctx* c, double* sens_angle, float w_const_sens, float de0) {
    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_wtab_all, (size_t)c->n_angles * wtab_angle_floats(c)))) return st;
    WSensArgs S;
    S.w = wtab_args(c, c->d_wtab_all, nullptr, 0);
    S.ppar = c->d_ppar;
    S.du_m = c->d_du_m;
    S.w_const_sens = w_const_sens;
    S.de0 = de0;
    S.sens_angle = sens_angle;
    LMOSEM_PROF_BEGIN(c);
    k_wtable_sens<<<dim3((c->ld_w + 127) / 128, c->n_angles), 128, 0, c->stream>>>(S);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SENS);
    return LMOSEM_OK;
}

lmosem_status build_model_rows(lmosem_ctx* c) {
    if (c->use_surrogate) {
        dev_free(c, &c->d_wtab_all);  // the surrogate form has no use for the tables
        return build_model_surrogate(c);
    }
    lmosem_status st;
    const int n_ptiles = c->ld_w / kTN;
    const int group = (c->n_angles + c->n_subsets - 1) / c->n_subsets;
    const int n_slots = c->n_subsets * group;

    // angles in sorted-slot order (empty slots skipped)
    std::vector<int32_t> slot_angle;
    for (int s = 0; s < n_slots; ++s) {
        int a = (s / group) + c->n_subsets * (s % group);
        if (a < c->n_angles) slot_angle.push_back(a);
    }
    const int ns = (int)slot_angle.size();

    // angle groups bounded by the scatter-table budget (three FP32 planes);
    // one group indexed by angle when the sensitivity pass left every
    // angle's planes behind
    const bool pre = c->d_wtab_all != nullptr;
    const int64_t per_angle = wtab_angle_floats(c) * (int64_t)sizeof(float);
    const int gsz = pre ? ns : (int)std::max<int64_t>(1, std::min<int64_t>(ns, c->table_budget / per_angle));
    const int n_groups = (ns + gsz - 1) / gsz;

    // launch entries (realisation, angle) of every group, in sorted-row order
    // within a realisation; one host array for all groups, copied once
    std::vector<int32_t> e_angle, e_wpos, e_row0, e_cnt, e_tiles, g_first(n_groups + 1, 0);
    std::vector<int64_t> g_rows(n_groups, 0), g_row0(n_groups, -1);
    for (int gi = 0; gi < n_groups; ++gi) {
        const int s0 = gi * gsz, s1 = std::min(ns, s0 + gsz);
        g_first[gi] = (int32_t)e_angle.size();
        for (int r = 0; r < c->n_real; ++r) {
            for (int s = s0; s < s1; ++s) {
                const int a = slot_angle[s];
                const size_t k = (size_t)r * c->n_angles + a;
                const int64_t cnt = c->h_angle_cnt[k];
                if (cnt == 0) continue;
                if (g_row0[gi] < 0) g_row0[gi] = c->h_angle_row0[k];
                e_angle.push_back(a);
                e_wpos.push_back(pre ? a : s - s0);
                e_row0.push_back((int32_t)c->h_angle_row0[k]);
                e_cnt.push_back((int32_t)cnt);
                e_tiles.push_back((int32_t)((cnt + kTJ - 1) / kTJ));
                g_rows[gi] += cnt;
            }
        }
    }
    g_first[n_groups] = (int32_t)e_angle.size();
    const int n_ent = (int)e_angle.size();
    // per-group exclusive tile prefix, stored per entry (+1 slot per group end)
    std::vector<int32_t> e_prefix(n_ent + n_groups, 0);
    std::vector<int32_t> g_tiles(n_groups, 0);
    for (int gi = 0; gi < n_groups; ++gi) {
        int32_t acc = 0;
        for (int e = g_first[gi]; e < g_first[gi + 1]; ++e) {
            e_prefix[e + gi] = acc;
            acc += e_tiles[e];
        }
        e_prefix[g_first[gi + 1] + gi] = acc;
        g_tiles[gi] = acc;
    }
    std::vector<int32_t> host_all;
    host_all.reserve((size_t)4 * n_ent + e_prefix.size() + ns);
    host_all.insert(host_all.end(), e_angle.begin(), e_angle.end());
    host_all.insert(host_all.end(), e_wpos.begin(), e_wpos.end());
    host_all.insert(host_all.end(), e_row0.begin(), e_row0.end());
    host_all.insert(host_all.end(), e_cnt.begin(), e_cnt.end());
    host_all.insert(host_all.end(), e_prefix.begin(), e_prefix.end());
    host_all.insert(host_all.end(), slot_angle.begin(), slot_angle.end());
    int32_t* d_all = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&d_all, host_all.size()))) return st;
    LMOSEM_CK(c, cudaMemcpyAsync(d_all, host_all.data(), host_all.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, c->stream));
    const int32_t* d_ent_angle = d_all;
    const int32_t* d_ent_wpos = d_all + n_ent;
    const int32_t* d_ent_row0 = d_all + 2 * n_ent;
    const int32_t* d_ent_cnt = d_all + 3 * n_ent;
    const int32_t* d_prefix = d_all + 4 * n_ent;
    const int32_t* d_slot_angle = d_all + 4 * n_ent + e_prefix.size();

    if (!pre && (st = dev_alloc(c, &c->d_wtab, (size_t)gsz * wtab_angle_floats(c)))) return st;
    float* wtab = pre ? c->d_wtab_all : c->d_wtab;
    const bool scaled = c->fmt != LMOSEM_MODEL_FP32;
    if (scaled) {
        // scaled rows are staged per group: one realisation, contiguous rows
        int64_t max_group_rows = 1;
        for (int gi = 0; gi < n_groups; ++gi) max_group_rows = std::max(max_group_rows, g_rows[gi]);
        if ((st = dev_alloc(c, &c->d_stage, (size_t)max_group_rows * c->ld_model))) return st;
    }

    const double fw2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    const double kappa = pow(c->fwhm_frac * fw2s, 2.0) * c->e0;  // sigma_E^2 = kappa E
    const double se0 = sqrt(kappa * c->e0);
    const size_t smem = sizeof(float) * ((size_t)kOffList + c->n_scat);
    LMOSEM_CK(c, cudaFuncSetAttribute(k_pathsum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));

    for (int gi = 0; gi < n_groups; ++gi) {
        const int s0 = gi * gsz, s1 = std::min(ns, s0 + gsz);
        if (!pre) {
            WTabArgs W = wtab_args(c, c->d_wtab, d_slot_angle, s0);
            LMOSEM_PROF_BEGIN(c);
            k_wtable<<<dim3((c->ld_w + 255) / 256, c->n_scat, s1 - s0), 256, 0, c->stream>>>(W);
            LMOSEM_LAUNCHED(c, LMOSEM_K_WTABLE);
        }

        const int tiles = g_tiles[gi];
        if (tiles == 0) continue;
        const int e0 = g_first[gi];
        PathSumArgs P;
        P.u_s = c->d_u_s;
        P.e_s = c->d_e_s;
        P.ent_angle = d_ent_angle + e0;
        P.ent_wpos = d_ent_wpos + e0;
        P.ent_row0 = d_ent_row0 + e0;
        P.ent_cnt = d_ent_cnt + e0;
        P.tile_prefix = d_prefix + e0 + gi;
        P.n_ent = g_first[gi + 1] - e0;
        P.n_ptiles = n_ptiles;
        P.wtab = wtab;
        P.ld_w = c->ld_w;
        P.n_scat = c->n_scat;
        P.mpar = c->d_mpar;
        P.ppar = c->d_ppar;
        P.e0 = (float)c->e0;
        P.sE0 = (float)(0.8493218002880191 / se0);
        P.lE0 = (float)(-log2(se0 * sqrt(2.0 * kPi)));
        P.ld_out = c->ld_model;
        P.n_store = (int)c->ld_model;
        P.scatter_only = c->scatter_only ? 1 : 0;
        const int64_t grow0 = g_row0[gi], grows = g_rows[gi];
        if (scaled) {
            P.out = c->d_stage;
            P.row_base = grow0;
        } else {
            P.out = reinterpret_cast<float*>(c->d_model);
            P.row_base = 0;
        }
        LMOSEM_PROF_BEGIN(c);
        k_pathsum<<<(unsigned)((int64_t)tiles * n_ptiles), kBuildThreads, smem, c->stream>>>(P);
        LMOSEM_LAUNCHED(c, LMOSEM_K_PATHSUM);
        if (scaled) {
            const int qthreads = 256;
            unsigned qblocks = (unsigned)((grows + qthreads / 32 - 1) / (qthreads / 32));
            LMOSEM_PROF_BEGIN(c);
            if (c->fmt == LMOSEM_MODEL_FP16_SCALED)
                k_quantize<__half><<<qblocks, qthreads, 0, c->stream>>>(
                    c->d_stage, c->ld_model, grows, c->n_sup, c->ld_model,
                    reinterpret_cast<__half*>(c->d_model), grow0, c->d_scale, 32768.0f);
            else
                k_quantize<__nv_bfloat16><<<qblocks, qthreads, 0, c->stream>>>(
                    c->d_stage, c->ld_model, grows, c->n_sup, c->ld_model,
                    reinterpret_cast<__nv_bfloat16*>(c->d_model), grow0, c->d_scale, 1.0f);
            LMOSEM_LAUNCHED(c, LMOSEM_K_QUANTIZE);
        }
    }
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    dev_free(c, &c->d_wtab);
    dev_free(c, &c->d_wtab_all);  // consumed
    dev_free(c, &c->d_stage);
    return LMOSEM_OK;
}

}  // namespace lmosem
