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
// event are exactly zero.  The table slices of 16 scatter pixels at a time
// are copied into shared memory with cp.async, two stages ahead of the one
// being summed (three buffers, one CTA barrier per stage).  A warp (8 events)
// skips the staged scatter pixels outside the cut of all of its events, and a
// last column tile with few live columns runs in a tail form (one event per
// thread); both leave every result bit unchanged.
//
// Energy cut: the table kernels also record, per scatter pixel m and column
// tile, the hull [lo, hi] of E' -/+ e_sigma sigma_E(E') over the tile's paths
// (n, m).  An event whose energy lies outside it takes U_jm = 0 for the tile:
// each term so dropped is below 2^(-e_sigma^2 log2(e) / 2) of its value at
// E_j = E' (1.5e-8 at the default 6 sigma, the same width as the position
// cut).  It drops the backscatter paths of photopeak events; the event sort
// puts the photopeak class in tiles of its own, so whole warps skip them.
//
// The binned form (paper Section 4) integrates the same model over position
// and energy bins; it reads the same planes (k_binned, below).
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
    const float4* scat_geo;     // (x_m, y_m, mu_m, pixel index bits)
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
    // energy hull of the scatter pixel m over the support pixels of a column
    // tile: [slot - s0][column tile][m] = (bits of lo, ~bits of hi), where
    // [lo, hi] covers E' -/+ e_sigma sigma_E(E') of every path (n, m) of the
    // tile; both words start at 0xffffffff and take atomicMin (the bits of
    // non-negative floats order as unsigned integers)
    uint2* hull;
    int n_ptiles;
    float hK;                   // e_sigma sqrt(kappa): half-width = hK sqrt(E'); inf: no cut
};

// (lo, hi) of one path in hull encoding
__device__ __forceinline__ uint2 hull_bits(float e1, float ri, float hK) {
    const float h = hK * (e1 * ri);  // e_sigma sigma_E(E'), sigma_E^2 = kappa E'
    return make_uint2(__float_as_uint(fmaxf(e1 - h, 0.0f)), ~__float_as_uint(e1 + h));
}

// warp-combine the lanes' hull words (lanes without a path hold 0xffffffff)
// and fold them into the table entry
__device__ __forceinline__ void hull_fold(uint2* dst, uint2 v) {
    const unsigned lo = __reduce_min_sync(0xffffffffu, v.x);
    const unsigned hi = __reduce_min_sync(0xffffffffu, v.y);
    if ((threadIdx.x & 31) == 0) {
        if (lo != 0xffffffffu) atomicMin(&dst->x, lo);
        if (hi != 0xffffffffu) atomicMin(&dst->y, hi);
    }
}

// planes (s, b, -lw) of the scatter path (n, m) at the angles of the group's
// slots: one thread per (n, m) walks the slots, so the angle-free inputs
// (the pair integral, the scatter pixel) are read once for all of them
__global__ void k_wtable(WTabArgs A, int n_slots) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (n >= A.ld_w) return;
    const size_t plane = (size_t)A.n_scat * A.ld_w;
    float* base = A.wtab + (size_t)k * A.ld_w + n;
    const bool real = n < A.n_sup;
    const int pn = real ? A.sup[n] : 0;
    const float4 gm = __ldg(A.scat_geo + k);
    const int pm = __float_as_int(gm.w);
    const float lpair = real ? A.l_pair[(size_t)k * A.n_sup + n] : 0.0f;
    const float xn = pixel_x(pn, A.nx, A.dpx), yn = pixel_y(pn, A.nx, A.ny, A.dpx);
    for (int g = 0; g < n_slots; ++g) {
        float s = 0.0f, b = 0.0f, nlw = INFINITY;
        uint2 hb = make_uint2(0xffffffffu, 0xffffffffu);
        if (real) {
            int a = A.slot_angle[A.s0 + g];
            float cpsi, rinv;
            if (path_geometry_xy(xn, yn, gm.x, gm.y, pn == pm, A.trig[a], &cpsi, &rinv)) {
                float P, kt;
                compton(cpsi, A.eps0, A.inv_kbar, &P, &kt);
                float e1 = A.e0 * P;
                float ratio = compton_lookup(A.compton, cpsi).x;
                float att = fmaf(ratio, A.l_edge[(size_t)a * A.npix + pm], lpair);
                float ri = rsqrtf(e1);
                nlw = fmaf(att, kLog2e, -__log2f(A.w_const * gm.z * kt * rinv * ri));
                s = A.cE * ri;
                b = -e1 * s;
                hb = hull_bits(e1, ri, A.hK);
            }
        }
        float* out = base + (size_t)g * 3 * plane;
        out[0] = s;
        out[plane] = b;
        out[2 * plane] = nlw;
        // whole warps share k and a 32-column slice of one tile (ld_w is a
        // multiple of kTN and the grid's surplus threads are whole warps)
        hull_fold(A.hull + ((size_t)g * A.n_ptiles + n / kTN) * A.n_scat + k, hb);
    }
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
    if (n >= A.ld_w) return;  // never splits a warp: ld_w is a multiple of kTN
    const size_t plane = (size_t)A.n_scat * A.ld_w;
    float* base = A.wtab + (size_t)a * 3 * plane + n;
    uint2* hull = A.hull + ((size_t)a * A.n_ptiles + n / kTN) * A.n_scat;
    const bool real = n < A.n_sup;  // padding columns: no path, but they join the warp's hull fold
    const int pn = real ? A.sup[n] : 0;
    const float xn = pixel_x(pn, A.nx, A.dpx), yn = pixel_y(pn, A.nx, A.ny, A.dpx);
    const float2 trig = A.trig[a];
    double acc = 0.0;
    if (real)
        acc = (double)(expf(-A.l_edge[(size_t)a * A.npix + pn]) * S.ppar[(size_t)a * A.ld_w + n].w * S.de0);
    const float* lp = A.l_pair + (real ? n : 0);
    const float* le = A.l_edge + (size_t)a * A.npix;
    const float* du = S.du_m + (size_t)a * A.n_scat;
    float part = 0.0f;
    for (int k = 0; k < A.n_scat; ++k) {
        const float4 gm = __ldg(A.scat_geo + k);
        const int pm = __float_as_int(gm.w);
        float s = 0.0f, b = 0.0f, nlw = INFINITY;
        uint2 hb = make_uint2(0xffffffffu, 0xffffffffu);
        float cpsi, rinv;
        if (real && path_geometry_xy(xn, yn, gm.x, gm.y, pn == pm, trig, &cpsi, &rinv)) {
            float P, kt;
            compton(cpsi, A.eps0, A.inv_kbar, &P, &kt);
            const float2 cr = compton_lookup(A.compton, cpsi);  // (mu ratio, window mass)
            const float att = fmaf(cr.x, __ldg(le + pm), lp[(size_t)k * A.n_sup]);
            const float mu = gm.z;
            const float e1 = A.e0 * P;
            const float ri = rsqrtf(e1);
            nlw = fmaf(att, kLog2e, -__log2f(A.w_const * mu * kt * rinv * ri));
            s = A.cE * ri;
            b = -e1 * s;
            hb = hull_bits(e1, ri, A.hK);
            const float w = S.w_const_sens * mu * kt * rinv * __expf(-att);
            part = fmaf(w, __ldg(du + k) * cr.y, part);
        }
        base[(size_t)k * A.ld_w] = s;
        base[plane + (size_t)k * A.ld_w] = b;
        base[2 * plane + (size_t)k * A.ld_w] = nlw;
        hull_fold(hull + k, hb);
        if ((k & 31) == 31) {
            acc += (double)part;
            part = 0.0f;
        }
    }
    acc += (double)part;
    if (real) S.sens_angle[(size_t)a * A.n_sup + n] = acc;
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
    int pt0, n_pt;               // column tiles pt0 .. pt0 + n_pt - 1 in this launch
    int n_tiles;                 // event tiles of this launch (all entries)
    int nq_tail;                 // narrow form: live 4-column groups of its tile
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
    // energy cut: hull of each scatter pixel over a column tile's paths,
    // [slot][column tile][m] (see WTabArgs); an event whose energy lies
    // outside it takes U_jm = 0 for that tile, so its terms there are exact
    // zeros in every form
    const uint2* hull;
    int n_ptiles;
    int e_cut;                   // 1: apply the energy cut
    int n_sup;                   // real support columns (for the term count)
    unsigned long long* n_terms; // terms kept by both cuts, summed over the launch
};

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}

// true when energy e lies outside the staged hull h (lo, ~hi bits): every
// term of the event at this scatter pixel and column tile is then dropped
__device__ __forceinline__ bool energy_cut(float e, uint2 h) {
    return e < __uint_as_float(h.x) || e > __uint_as_float(~h.y);
}

// hull words of stage rows c0 .. c0 + kStage - 1 into hl[buf * kStage + t],
// one row per thread t in [0, kStage) (padded rows: no cut, their U is 0)
template <typename TI>
__device__ __forceinline__ void stage_hull(int t, const TI& T, const int* mlist, const uint2* hull_a, uint2* hl,
                                           int c0, int buf) {
    if (t >= 0 && t < kStage) {
        uint2* dst = hl + buf * kStage + t;
        if (c0 + t < T.nm) cp_async8(dst, hull_a + mlist[c0 + t]);
        else *dst = make_uint2(0u, 0u);
    }
}

// real support columns of the column tile starting at n0
__device__ __forceinline__ int tile_cols(const PathSumArgs& A, int n0) { return max(0, min(kTN, A.n_sup - n0)); }

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

// ---- per-tile setup shared by both forms

// Where a CTA's event tile sits, and the scatter pixels whose cut interval
// reaches any of its events (the strip union), compacted into mlist.
struct TileInfo {
    int ent, a, nr, n0, nm;
    int64_t r0;
};

template <int NT = kBuildThreads>
__device__ __forceinline__ TileInfo tile_setup(const PathSumArgs& A, int et, int pt, float* ev_u,
                                               float* ev_e, int* misc, int* mlist) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* red = reinterpret_cast<float*>(misc);
    TileInfo T;
    int lo = 0, hi = A.n_ent - 1;  // entry (realisation, angle) of the event tile
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (A.tile_prefix[mid] <= et) lo = mid; else hi = mid - 1;
    }
    T.ent = lo;
    T.a = A.ent_angle[lo];
    const int tile = et - A.tile_prefix[lo];
    T.r0 = (int64_t)A.ent_row0[lo] + (int64_t)tile * kTJ;
    T.nr = min(kTJ, A.ent_cnt[lo] - tile * kTJ);
    T.n0 = pt * kTN;

    if (tid < kTJ) {
        ev_u[tid] = tid < T.nr ? A.u_s[T.r0 + tid] : 1e30f;
        ev_e[tid] = tid < T.nr ? A.e_s[T.r0 + tid] : 0.0f;
    }
    __syncthreads();
    if (warp == 0) {  // position range of the tile's events
        float mn = INFINITY, mx = -INFINITY;
        for (int j = lane; j < T.nr; j += 32) {
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

    const float4* mp_a = A.mpar + (size_t)T.a * A.n_scat;
    static_assert(NT >= kTJ && NT % 32 == 0 && NT <= 256, "64 to 256 threads");
    constexpr int nwarps = NT / 32;
    int nm = 0;
    for (int m0 = 0; m0 < A.n_scat; m0 += NT) {  // block compaction
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
        for (int w = 0; w < nwarps; ++w) {
            int cw = misc[w];
            if (w < warp) off += cw;
            total += cw;
        }
        if (in) mlist[off + __popc(bal & ((1u << lane) - 1u))] = m;
        __syncthreads();
        nm += total;
    }
    T.nm = nm;
    return T;
}

// primary path of event (uj, ej) at 4 support pixels
__device__ __forceinline__ void primary4(const PathSumArgs& A, const float4* pp, float uj, float ej,
                                         float2& lo, float2& hi) {
    const float te = (ej - A.e0) * A.sE0;
    const float le = fmaf(-te, te, A.lE0);
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float t = (uj - pp[q].x) * pp[q].y;
        v[q] = A.scatter_only ? 0.0f : ex2_approx(fmaf(-t, t, pp[q].z + le));
    }
    lo = make_float2(v[0], v[1]);
    hi = make_float2(v[2], v[3]);
}

// U_jm of one event (position u) at scatter pixel parameters q
__device__ __forceinline__ float strip_weight(float u, float4 q) {
    const float d = u - q.x;
    const float z = d * q.y;
    return fabsf(d) <= q.w ? ex2_approx(fmaf(-z, z, q.z)) : 0.0f;
}

// Scatter terms of one event at 4 support pixels (two packed pairs):
// acc += U 2^-((E s + b)^2 + w).  Both forms call this, so a column's bits do
// not depend on the form that computed it.
__device__ __forceinline__ void terms4(float2 E2, float2 U, float4 S, float4 B, float4 W, float2& lo,
                                       float2& hi) {
    const float2 t0 = ffma2(E2, make_float2(S.x, S.y), make_float2(B.x, B.y));
    const float2 t1 = ffma2(E2, make_float2(S.z, S.w), make_float2(B.z, B.w));
    const float2 z0 = ffma2(t0, t0, make_float2(W.x, W.y));
    const float2 z1 = ffma2(t1, t1, make_float2(W.z, W.w));
    const float2 e0 = make_float2(ex2_approx(-z0.x), ex2_approx(-z0.y));
    const float2 e1 = make_float2(ex2_approx(-z1.x), ex2_approx(-z1.y));
    lo = ffma2(U, e0, lo);
    hi = ffma2(U, e1, hi);
}

__device__ __forceinline__ void store4(const PathSumArgs& A, float* row, int n, float2 lo, float2 hi) {
    if (n + 3 < A.n_store) {
        *reinterpret_cast<float4*>(row + n) = make_float4(lo.x, lo.y, hi.x, hi.y);
    } else {
        const float v[4] = {lo.x, lo.y, hi.x, hi.y};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (n + q < A.n_store) row[n + q] = v[q];
    }
}

// ---- staging shared by both forms
//
// Shared-memory layout, in floats: the three table planes and the position
// parameters of kStage scatter pixels per stage, double-buffered with
// cp.async; U_jm of the stage; the tile's events; scratch; the strip union.
constexpr int kPlaneF = kStage * kTN;                 // one plane of one stage
constexpr int kOffPlanes = 0;                         // [2][3][kStage][kTN]
constexpr int kOffU = kOffPlanes + 2 * 3 * kPlaneF;   // [kStage][kTJ] float2
constexpr int kOffMp = kOffU + 2 * kStage * kTJ;      // [2][kStage] float4
constexpr int kOffHl = kOffMp + 2 * kStage * 4;       // [2][kStage] uint2 (energy hull)
constexpr int kOffEv = kOffHl + 2 * kStage * 2;       // u[kTJ], e[kTJ]
constexpr int kOffMisc = kOffEv + 2 * kTJ;            // 16 ints
constexpr int kOffList = kOffMisc + 16;               // n_scat ints

// stage c0 .. c0 + kStage - 1 of the strip union into buffer buf: the first
// nq 4-column groups of each plane row, rows `row` floats apart (padded
// scatter pixels get s = b = 0, w = inf and a negative cut, i.e. exact
// zeros), then commit the group
template <int NT = kBuildThreads>
__device__ __forceinline__ void stage_issue(const TileInfo& T, const int* mlist, const float* tab,
                                            size_t plane, int ld_w, const float4* mp_a, float* planes,
                                            float4* mp, int c0, int buf, int nq, int row = kTN,
                                            const uint2* hull_a = nullptr, uint2* hl = nullptr) {
    const int tid = threadIdx.x;
    for (int k = tid; k < 3 * kStage * nq; k += NT) {
        const int p = k / (kStage * nq);
        const int r = k - p * (kStage * nq);
        const int mc = r / nq, q = r - mc * nq;
        float* dst = planes + ((buf * 3 + p) * kStage + mc) * row + 4 * q;
        if (c0 + mc < T.nm) {
            cp_async16(dst, tab + p * plane + (size_t)mlist[c0 + mc] * ld_w + 4 * q);
        } else {
            const float v = p == 2 ? INFINITY : 0.0f;
            *reinterpret_cast<float4*>(dst) = make_float4(v, v, v, v);
        }
    }
    if (tid < kStage) {
        float4* dst = mp + buf * kStage + tid;
        if (c0 + tid < T.nm) cp_async16(dst, mp_a + mlist[c0 + tid]);
        else *dst = make_float4(0.0f, 0.0f, -INFINITY, -1.0f);  // cut < 0: U = 0
    }
    if (hull_a) stage_hull(tid - kStage, T, mlist, hull_a, hl, c0, buf);
    cp_async_commit();
}

// ---- narrow form: a last column tile of at most kNarrowQ x 4 live columns
//
// Each thread holds one event and up to kNarrowQ / 4 groups of 4 columns
// (instead of 8 events x 4 columns of a 128-column tile with most lanes
// idle).
constexpr int kNarrowQ = 16;
static_assert(kBuildThreads == 4 * kTJ, "narrow form: 64 events x 4 column groups per pass");

__global__ void __launch_bounds__(kBuildThreads, 2) k_pathsum_narrow(PathSumArgs A) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* planes = sm + kOffPlanes;
    float2* sU = reinterpret_cast<float2*>(sm + kOffU);
    float4* mp = reinterpret_cast<float4*>(sm + kOffMp);
    uint2* hl = reinterpret_cast<uint2*>(sm + kOffHl);
    float* ev_u = sm + kOffEv;
    float* ev_e = ev_u + kTJ;
    int* misc = reinterpret_cast<int*>(sm + kOffMisc);
    int* mlist = reinterpret_cast<int*>(sm + kOffList);
    const int tid = threadIdx.x;
    const TileInfo T = tile_setup(A, blockIdx.x, A.pt0, ev_u, ev_e, misc, mlist);
    const uint2* hull_a = A.hull + ((size_t)A.ent_wpos[T.ent] * A.n_ptiles + T.n0 / kTN) * A.n_scat;
    const int nq = A.nq_tail;
    constexpr int kQ = kNarrowQ / 4;
    const int jn = tid & (kTJ - 1), qs = tid / kTJ;  // event, first column group
    const float2 E2 = make_float2(ev_e[jn], ev_e[jn]);
    float2 acc[kQ][2];
#pragma unroll
    for (int qi = 0; qi < kQ; ++qi) {
        const int q = qs + 4 * qi;
        acc[qi][0] = acc[qi][1] = make_float2(0.0f, 0.0f);
        if (q < nq) {
            const float4* pp_a = A.ppar + (size_t)T.a * A.ld_w + T.n0 + 4 * q;
            float4 pp[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) pp[c] = __ldg(pp_a + c);
            primary4(A, pp, ev_u[jn], ev_e[jn], acc[qi][0], acc[qi][1]);
        }
    }

    const size_t plane = (size_t)A.n_scat * A.ld_w;
    const float* tab = A.wtab + (size_t)A.ent_wpos[T.ent] * 3 * plane + T.n0;
    const float4* mp_a = A.mpar + (size_t)T.a * A.n_scat;
    const int nchunks = (T.nm + kStage - 1) / kStage;
    unsigned kept = 0;  // (event, scatter pixel) pairs with U != 0 formed by this thread
    if (nchunks > 0) stage_issue(T, mlist, tab, plane, A.ld_w, mp_a, planes, mp, 0, 0, nq, kTN, hull_a, hl);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) {
            stage_issue(T, mlist, tab, plane, A.ld_w, mp_a, planes, mp, (c + 1) * kStage, buf ^ 1, nq, kTN, hull_a,
                        hl);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        for (int k = tid; k < kStage * kTJ; k += kBuildThreads) {
            const int mc = k / kTJ, j = k - mc * kTJ;
            const float U = (A.e_cut && energy_cut(ev_e[j], hl[buf * kStage + mc])) ? 0.0f
                                                                        : strip_weight(ev_u[j], mp[buf * kStage + mc]);
            kept += U != 0.0f;
            sU[mc * kTJ + j] = make_float2(U, U);
        }
        __syncthreads();
        const float* pS = planes + (buf * 3 + 0) * kPlaneF;
        const float* pB = planes + (buf * 3 + 1) * kPlaneF;
        const float* pW = planes + (buf * 3 + 2) * kPlaneF;
#pragma unroll 2
        for (int mc = 0; mc < kStage; ++mc) {
            const float2 Uj = sU[mc * kTJ + jn];
#pragma unroll
            for (int qi = 0; qi < kQ; ++qi) {
                const int q = qs + 4 * qi;
                if (q >= nq) break;
                const int o = mc * kTN + 4 * q;
                terms4(E2, Uj, *reinterpret_cast<const float4*>(pS + o),
                       *reinterpret_cast<const float4*>(pB + o), *reinterpret_cast<const float4*>(pW + o),
                       acc[qi][0], acc[qi][1]);
            }
        }
        __syncthreads();
    }
    if (A.n_terms) {
        const unsigned long long cols = (unsigned long long)tile_cols(A, T.n0);
        const unsigned w = __reduce_add_sync(0xffffffffu, kept);
        if ((tid & 31) == 0 && w) atomicAdd(A.n_terms, cols * w);
        if (tid == 0 && !A.scatter_only) atomicAdd(A.n_terms, cols * (unsigned long long)T.nr);
    }

    if (jn >= T.nr) return;
    float* row = A.out + (T.r0 + jn - A.row_base) * A.ld_out;
#pragma unroll
    for (int qi = 0; qi < kQ; ++qi) {
        const int q = qs + 4 * qi;
        if (q >= nq) break;
        store4(A, row, T.n0 + 4 * q, acc[qi][0], acc[qi][1]);
    }
    const int ngs = (min(A.n_store - T.n0, kTN) + 3) / 4;  // stored groups of the tile
    for (int q = qs; q < ngs; q += 4)
        if (q >= nq) store4(A, row, T.n0 + 4 * q, make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f));
}

// ---- tail form: a last column tile of at most kTailQ x 4 live columns
//
// One event per thread and 64 threads per CTA: the thread forms its event's
// U_jm itself (one ex2 per scatter pixel, skipped pixels are exact zeros)
// and its nq <= kTailQ groups of 4 columns; three compact stage buffers and
// one barrier per stage.  Same term operations as the other forms.
constexpr int kTailQ = 4;
constexpr int kTRow = 4 * kTailQ;                                 // floats per staged plane row
constexpr int kTOffPlanes = 0;                                    // [3][3][kStage][kTRow]
constexpr int kTOffMp = kTOffPlanes + 3 * 3 * kStage * kTRow;     // [3][kStage] float4
constexpr int kTOffHl = kTOffMp + 3 * kStage * 4;                 // [3][kStage] uint2 (energy hull)
constexpr int kTOffEv = kTOffHl + 3 * kStage * 2;                 // u[kTJ], e[kTJ]
constexpr int kTOffMisc = kTOffEv + 2 * kTJ;                      // 16 ints
constexpr int kTOffList = kTOffMisc + 16;                         // n_scat ints

__global__ void __launch_bounds__(kTJ) k_pathsum_tail(PathSumArgs A) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* planes = sm + kTOffPlanes;
    float4* mp = reinterpret_cast<float4*>(sm + kTOffMp);
    uint2* hl = reinterpret_cast<uint2*>(sm + kTOffHl);
    float* ev_u = sm + kTOffEv;
    float* ev_e = ev_u + kTJ;
    int* misc = reinterpret_cast<int*>(sm + kTOffMisc);
    int* mlist = reinterpret_cast<int*>(sm + kTOffList);
    const int j = threadIdx.x;
    const TileInfo T = tile_setup<kTJ>(A, blockIdx.x, A.pt0, ev_u, ev_e, misc, mlist);
    const uint2* hull_a = A.hull + ((size_t)A.ent_wpos[T.ent] * A.n_ptiles + T.n0 / kTN) * A.n_scat;
    const int nq = A.nq_tail;
    const float uj = ev_u[j], ej = ev_e[j];
    const float2 E2 = make_float2(ej, ej);
    float2 acc[kTailQ][2];
#pragma unroll
    for (int q = 0; q < kTailQ; ++q) {
        acc[q][0] = acc[q][1] = make_float2(0.0f, 0.0f);
        if (q < nq) {
            const float4* pp_a = A.ppar + (size_t)T.a * A.ld_w + T.n0 + 4 * q;
            float4 pp[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) pp[c] = __ldg(pp_a + c);
            primary4(A, pp, uj, ej, acc[q][0], acc[q][1]);
        }
    }

    const size_t plane = (size_t)A.n_scat * A.ld_w;
    const float* tab = A.wtab + (size_t)A.ent_wpos[T.ent] * 3 * plane + T.n0;
    const float4* mp_a = A.mpar + (size_t)T.a * A.n_scat;
    const int nchunks = (T.nm + kStage - 1) / kStage;
    unsigned kept = 0;  // scatter pixels with U != 0 for this thread's event
    for (int q = 0; q < min(2, nchunks); ++q)
        stage_issue<kTJ>(T, mlist, tab, plane, A.ld_w, mp_a, planes, mp, q * kStage, q, nq, kTRow, hull_a, hl);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c % 3;
        if (c + 1 < nchunks) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();  // stage c landed everywhere; every thread is done with stage c - 1
        if (c + 2 < nchunks)
            stage_issue<kTJ>(T, mlist, tab, plane, A.ld_w, mp_a, planes, mp, (c + 2) * kStage, (c + 2) % 3, nq,
                             kTRow, hull_a, hl);
        const float* pS = planes + (buf * 3 + 0) * kStage * kTRow;
        const float* pB = planes + (buf * 3 + 1) * kStage * kTRow;
        const float* pW = planes + (buf * 3 + 2) * kStage * kTRow;
        for (int mc = 0; mc < kStage; ++mc) {
            const float U =
                (A.e_cut && energy_cut(ej, hl[buf * kStage + mc])) ? 0.0f : strip_weight(uj, mp[buf * kStage + mc]);
            if (U == 0.0f) continue;
            ++kept;
            const float2 U2 = make_float2(U, U);
#pragma unroll
            for (int q = 0; q < kTailQ; ++q) {
                if (q >= nq) break;
                const int o = mc * kTRow + 4 * q;
                terms4(E2, U2, *reinterpret_cast<const float4*>(pS + o), *reinterpret_cast<const float4*>(pB + o),
                       *reinterpret_cast<const float4*>(pW + o), acc[q][0], acc[q][1]);
            }
        }
    }

    if (A.n_terms) {  // 64 threads: two whole warps
        const unsigned long long cols = (unsigned long long)tile_cols(A, T.n0);
        const unsigned w = __reduce_add_sync(0xffffffffu, kept);
        if ((j & 31) == 0 && w) atomicAdd(A.n_terms, cols * w);
        if (j == 0 && !A.scatter_only) atomicAdd(A.n_terms, cols * (unsigned long long)T.nr);
    }

    if (j >= T.nr) return;
    float* row = A.out + (T.r0 + j - A.row_base) * A.ld_out;
#pragma unroll
    for (int q = 0; q < kTailQ; ++q) {
        if (q >= nq) break;
        store4(A, row, T.n0 + 4 * q, acc[q][0], acc[q][1]);
    }
    const int ngs = (min(A.n_store - T.n0, kTN) + 3) / 4;  // stored groups of the tile
    for (int q = nq; q < ngs; ++q) store4(A, row, T.n0 + 4 * q, make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f));
}

// ---- wide form: 64 events x 128 columns, 8 events x 4 columns per thread
//
// Three stage buffers: at the top of stage c one CTA barrier both publishes
// stage c (landed by cp.async) and retires stage c - 1, whose buffer then
// takes stage c + 2.  Each warp forms the U_jm of its own 8 events (events
// 8w .. 8w + 7) and a 16-bit mask of the stage's scatter pixels whose cut
// reaches any of them; it skips the others, whose terms are exact zeros for
// all of its events.  One barrier per stage, no shared atomics.
constexpr int kWBuf = 3;
constexpr int kWarps = kBuildThreads / 32;
constexpr int kWOffPlanes = 0;                                   // [kWBuf][3][kStage][kTN]
constexpr int kWOffMp = kWOffPlanes + kWBuf * 3 * kPlaneF;       // [kWBuf][kStage] float4
constexpr int kWOffHl = kWOffMp + kWBuf * kStage * 4;            // [kWBuf][kStage] uint2 (energy hull)
constexpr int kWOffU = kWOffHl + kWBuf * kStage * 2;             // [warp][kStage][8] float2
constexpr int kWOffEv = kWOffU + kWarps * kStage * 8 * 2;        // u[kTJ], e[kTJ]
constexpr int kWOffMisc = kWOffEv + 2 * kTJ;                     // 16 ints
constexpr int kWOffList = kWOffMisc + 16;                        // n_scat ints
static_assert(kWOffMp % 4 == 0 && kWOffU % 4 == 0 && kWOffHl % 2 == 0, "aligned stage buffers");
static_assert(kTJ == 8 * kWarps && kStage == 16, "8 events per warp; 16-bit live masks; 4 U per lane");
static_assert(kBuildThreads == 256 && kTN == 128 && kStage == 2 * kWarps, "one column group, two stage rows per thread");

// The wide form's staging: the copies of stage_issue with the per-thread
// parts of the addresses hoisted out of the stage loop.  Thread t copies the
// 16-byte column group t % 32 of stage rows t / 32 and t / 32 + 8 of the
// three planes (tab_q = the table row start + that group's offset, dst_q =
// its slot in plane 0 of buffer 0); threads t < kStage the position
// parameters of stage row t.
__device__ __forceinline__ void stage_issue_wide(const TileInfo& T, const int* mlist, const float* tab_q,
                                                 size_t plane, int ld_w, const float4* mp_a, float* dst_q,
                                                 float4* mp, const uint2* hull_a, uint2* hl, int c0, int buf) {
    const int tid = threadIdx.x, mc0 = tid >> 5;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int mc = mc0 + 8 * h;
        float* d = dst_q + (buf * 3 * kStage + 8 * h) * kTN;
        if (c0 + mc < T.nm) {
            const float* src = tab_q + (size_t)mlist[c0 + mc] * ld_w;
            cp_async16(d, src);
            cp_async16(d + kPlaneF, src + plane);
            cp_async16(d + 2 * kPlaneF, src + 2 * plane);
        } else {
            const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            *reinterpret_cast<float4*>(d) = z;
            *reinterpret_cast<float4*>(d + kPlaneF) = z;
            *reinterpret_cast<float4*>(d + 2 * kPlaneF) = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
        }
    }
    if (tid < kStage) {
        float4* dst = mp + buf * kStage + tid;
        if (c0 + tid < T.nm) cp_async16(dst, mp_a + mlist[c0 + tid]);
        else *dst = make_float4(0.0f, 0.0f, -INFINITY, -1.0f);  // cut < 0: U = 0
    }
    stage_hull(tid - kStage, T, mlist, hull_a, hl, c0, buf);
    cp_async_commit();
}

__global__ void __launch_bounds__(kBuildThreads, 2) k_pathsum(PathSumArgs A) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* planes = sm + kWOffPlanes;
    float4* mp = reinterpret_cast<float4*>(sm + kWOffMp);
    uint2* hl = reinterpret_cast<uint2*>(sm + kWOffHl);
    float* ev_u = sm + kWOffEv;
    float* ev_e = ev_u + kTJ;
    int* misc = reinterpret_cast<int*>(sm + kWOffMisc);
    int* mlist = reinterpret_cast<int*>(sm + kWOffList);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2* sUw = reinterpret_cast<float2*>(sm + kWOffU) + warp * kStage * 8;
    // the event tile is the fast index: the CTAs resident at one time share a
    // column tile, whose planes for an angle (12 B x 128 per scatter pixel, a
    // few MB) stay in L2 for all of that angle's event tiles
    const TileInfo T = tile_setup(A, blockIdx.x % A.n_tiles, A.pt0 + blockIdx.x / A.n_tiles, ev_u, ev_e, misc,
                                  mlist);
    const uint2* hull_a = A.hull + ((size_t)A.ent_wpos[T.ent] * A.n_ptiles + T.n0 / kTN) * A.n_scat;
    // accumulators (pairs of adjacent support pixels), initialised with the
    // primary path
    float2 E2[8];
    float2 acc[8][2];
    {
        const float4* pp_a = A.ppar + (size_t)T.a * A.ld_w + T.n0 + 4 * lane;
        float4 pp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) pp[q] = __ldg(pp_a + q);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const float uj = ev_u[8 * warp + jj], ej = ev_e[8 * warp + jj];
            E2[jj] = make_float2(ej, ej);
            primary4(A, pp, uj, ej, acc[jj][0], acc[jj][1]);
        }
    }

    const size_t plane = (size_t)A.n_scat * A.ld_w;
    const float* tab = A.wtab + (size_t)A.ent_wpos[T.ent] * 3 * plane + T.n0;
    const float4* mp_a = A.mpar + (size_t)T.a * A.n_scat;
    const int nchunks = (T.nm + kStage - 1) / kStage;
    const float* tab_q = tab + 4 * lane;
    float* dst_q = planes + warp * kTN + 4 * lane;
    for (int q = 0; q < min(2, nchunks); ++q)
        stage_issue_wide(T, mlist, tab_q, plane, A.ld_w, mp_a, dst_q, mp, hull_a, hl, q * kStage, q);
    const float uw = ev_u[8 * warp + (lane & 7)];  // this lane's event in the U step
    const float ew = ev_e[8 * warp + (lane & 7)];
    unsigned kept = 0;  // (event, scatter pixel) pairs of the warp with U != 0
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c % kWBuf;
        if (c + 1 < nchunks) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();  // stage c landed everywhere; every warp is done with stage c - 1
        if (c + 2 < nchunks)
            stage_issue_wide(T, mlist, tab_q, plane, A.ld_w, mp_a, dst_q, mp, hull_a, hl, (c + 2) * kStage,
                             (c + 2) % kWBuf);
        // U_jm of this warp's events: lane holds event lane % 8 at scatter
        // pixels lane / 8 + 4 i
        unsigned live = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int mc = (lane >> 3) + 4 * i;
            const float U =
                (A.e_cut && energy_cut(ew, hl[buf * kStage + mc])) ? 0.0f : strip_weight(uw, mp[buf * kStage + mc]);
            sUw[mc * 8 + (lane & 7)] = make_float2(U, U);
            const unsigned bal = __ballot_sync(0xffffffffu, U != 0.0f);
            kept += __popc(bal);
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if ((bal >> (8 * g)) & 0xffu) live |= 1u << (g + 4 * i);
        }
        __syncwarp();
        const float* pS = planes + (buf * 3 + 0) * kPlaneF + 4 * lane;
        const float* pB = planes + (buf * 3 + 1) * kPlaneF + 4 * lane;
        const float* pW = planes + (buf * 3 + 2) * kPlaneF + 4 * lane;
#pragma unroll 1  // measured: 1% faster than unrolling by 2 (the body is 32 MUFU + 48 FFMA2 already)
        for (int mc = 0; mc < kStage; ++mc) {
            if (!((live >> mc) & 1u)) continue;
            const float4 S = *reinterpret_cast<const float4*>(pS + mc * kTN);
            const float4 B = *reinterpret_cast<const float4*>(pB + mc * kTN);
            const float4 W = *reinterpret_cast<const float4*>(pW + mc * kTN);
            const float4* up = reinterpret_cast<const float4*>(sUw + mc * 8);
            float2 U[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = up[k];
                U[2 * k] = make_float2(v.x, v.y);
                U[2 * k + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) terms4(E2[jj], U[jj], S, B, W, acc[jj][0], acc[jj][1]);
        }
    }

    if (A.n_terms && lane == 0) {
        const unsigned long long cols = (unsigned long long)tile_cols(A, T.n0);
        const int real = max(0, min(8, T.nr - 8 * warp));
        const unsigned long long t = cols * (kept + (A.scatter_only ? 0u : (unsigned)real));
        if (t) atomicAdd(A.n_terms, t);
    }
    const int n = T.n0 + 4 * lane;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const int j = 8 * warp + jj;
        if (j < T.nr) store4(A, A.out + (T.r0 + j - A.row_base) * A.ld_out, n, acc[jj][0], acc[jj][1]);
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
// ---- binned rows (the paper's binning experiment, Section 4)
//
// A row is a bin (angle a, detector position bin b, energy bin k).  Its model
// is the event model integrated over the bin, each Gaussian density replaced
// by its mass on the bin:
//   p_(abk),n = w_0(n) M_u(b; u_n) M_E(k; E0)
//             + sum_m M_u(b; u_m) W_a(n, m) M_E(k; E'_a(n, m)).
// For one (a, k) the scatter part is a product over m of the position-bin
// masses (bins x scatter pixels) with C_k = W M_E (scatter pixels x support
// pixels).  A CTA owns 64 position bins x 128 support pixels of one (a, k).
// For each stage of 16 scatter pixels it forms C_k from the (s, b, -lw)
// planes (sigma_E sqrt(2 pi) = sqrt(pi log2 e) / s, E' = -b / s, and
// (E - E') / (sigma_E sqrt 2) = (E s + b) sqrt(ln 2)) and the bin masses from
// the position parameters, then accumulates 8 bins x 4 pixels per thread; a
// warp skips the scatter pixels whose cut misses all 8 of its bins.
constexpr int kMaxEBins = 8;
constexpr float kSqrtLn2 = 0.83255461115769776f;     // q sqrt(ln 2) = 1 / (sigma sqrt 2)
constexpr float kSqrtPiLog2e = 2.1289340388624524f;  // sigma sqrt(2 pi) = sqrt(pi log2 e) / q

struct BinnedArgs {
    const float* wtab;
    int ld_w, n_scat;
    int a0;                       // first angle of the launch
    int wslot_by_angle;           // 1: planes indexed by angle, else by a - a0
    const float4* mpar;           // [a][m] (u_m, q_m, lq_m, cut_m)
    const float4* ppar;           // [a][n] (u_n, q_n, lp_n, D_u)
    int n_bins;
    float bin_mm, half;           // detector position bins
    int n_ebins;
    float e_edge[kMaxEBins + 1];  // energy bin edges
    float pe_mass[kMaxEBins];     // photopeak mass of each energy bin
    int n_btiles, n_ptiles;
    const int32_t* rowmap;        // [a][b][k] -> sorted row, or -1
    float* out;
    int64_t ld_out;
    int n_store;
    int scatter_only;
};

// mass of a unit Gaussian on [zl, zh] in units of sigma sqrt 2, keeping its
// relative accuracy far out in either tail
__device__ __forceinline__ float bin_mass(float zl, float zh) {
    if (zl >= 0.0f) return 0.5f * (erfcf(zl) - erfcf(zh));
    if (zh <= 0.0f) return 0.5f * (erfcf(-zh) - erfcf(-zl));
    return 1.0f - 0.5f * (erfcf(-zl) + erfcf(zh));
}

constexpr int kBOffPlanes = 0;                          // [2][3][kStage][kTN]
constexpr int kBOffMp = kBOffPlanes + 2 * 3 * kPlaneF;  // [2][kStage] float4
constexpr int kBOffC = kBOffMp + 2 * kStage * 4;        // [kStage][kTN]  C_k of the stage
constexpr int kBOffM = kBOffC + kStage * kTN;           // [kStage][kTJ]  bin masses of the stage
constexpr int kBOffMisc = kBOffM + kStage * kTJ;        // 16 ints
constexpr int kBOffList = kBOffMisc + 16;               // n_scat ints

__global__ void __launch_bounds__(kBuildThreads, 2) k_binned(BinnedArgs A) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* planes = sm + kBOffPlanes;
    float4* mp = reinterpret_cast<float4*>(sm + kBOffMp);
    float* Cm = sm + kBOffC;
    float* Mb = sm + kBOffM;
    int* misc = reinterpret_cast<int*>(sm + kBOffMisc);
    unsigned* live = reinterpret_cast<unsigned*>(misc) + 8;
    int* mlist = reinterpret_cast<int*>(sm + kBOffList);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    int idx = blockIdx.x;
    const int pt = idx % A.n_ptiles;
    idx /= A.n_ptiles;
    const int bt = idx % A.n_btiles;
    idx /= A.n_btiles;
    const int k = idx % A.n_ebins;
    const int a = A.a0 + idx / A.n_ebins;
    const int b0 = bt * kTJ, n0 = pt * kTN;
    const int nb = min(kTJ, A.n_bins - b0);
    const int32_t* rmap = A.rowmap + (size_t)a * A.n_bins * A.n_ebins + k;

    // nothing to do unless one of the CTA's bins holds a row
    bool has = false;
    for (int bl = tid; bl < nb; bl += kBuildThreads) has |= rmap[(size_t)(b0 + bl) * A.n_ebins] >= 0;
    if (!__syncthreads_or(has)) return;

    // scatter pixels whose cut interval reaches the CTA's bins
    const float umin = -A.half + b0 * A.bin_mm, umax = -A.half + (b0 + nb) * A.bin_mm;
    const float4* mp_a = A.mpar + (size_t)a * A.n_scat;
    int nm = 0;
    for (int m0 = 0; m0 < A.n_scat; m0 += kBuildThreads) {
        const int m = m0 + tid;
        bool in = false;
        if (m < A.n_scat) {
            const float4 q = __ldg(mp_a + m);
            in = (q.x + q.w >= umin) && (q.x - q.w <= umax);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) misc[warp] = __popc(bal);
        __syncthreads();
        int off = nm, total = 0;
        for (int w = 0; w < kBuildThreads / 32; ++w) {
            const int cw = misc[w];
            if (w < warp) off += cw;
            total += cw;
        }
        if (in) mlist[off + __popc(bal & ((1u << lane) - 1u))] = m;
        __syncthreads();
        nm += total;
    }

    // primary path: w_0 M_u(b; u_n) M_E(k; E0), 8 bins x 4 pixels per thread
    float2 acc[8][2];
    {
        const float4* pp_a = A.ppar + (size_t)a * A.ld_w + n0 + 4 * lane;
        float w0[4], s2[4], un[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 pp = __ldg(pp_a + q);
            w0[q] = (pp.y > 0.0f && !A.scatter_only) ? ex2_approx(pp.z) * kSqrtPiLog2e / pp.y * A.pe_mass[k]
                                                     : 0.0f;
            s2[q] = pp.y * kSqrtLn2;
            un[q] = pp.x;
        }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int b = b0 + 8 * warp + jj;
            const float ulo = -A.half + b * A.bin_mm, uhi = ulo + A.bin_mm;
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[q] = (b < A.n_bins && w0[q] != 0.0f)
                           ? w0[q] * bin_mass((ulo - un[q]) * s2[q], (uhi - un[q]) * s2[q])
                           : 0.0f;
            acc[jj][0] = make_float2(v[0], v[1]);
            acc[jj][1] = make_float2(v[2], v[3]);
        }
    }

    const size_t plane = (size_t)A.n_scat * A.ld_w;
    const int slot = A.wslot_by_angle ? a : a - A.a0;
    const float* tab = A.wtab + (size_t)slot * 3 * plane + n0;
    TileInfo T;
    T.nm = nm;
    const float el = A.e_edge[k], eh = A.e_edge[k + 1];
    const int nchunks = (nm + kStage - 1) / kStage;
    if (nchunks > 0) stage_issue(T, mlist, tab, plane, A.ld_w, mp_a, planes, mp, 0, 0, kTN / 4);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (tid < kBuildThreads / 32) live[tid] = 0u;
        if (c + 1 < nchunks) {
            stage_issue(T, mlist, tab, plane, A.ld_w, mp_a, planes, mp, (c + 1) * kStage, buf ^ 1, kTN / 4);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // bin masses of the stage: lanes hold bins 32 (warp & 1) + lane of one mc
        for (int kk = tid; kk < kStage * kTJ; kk += kBuildThreads) {
            const int mc = kk / kTJ, bl = kk - mc * kTJ;
            const float4 q = mp[buf * kStage + mc];
            const float ulo = -A.half + (b0 + bl) * A.bin_mm, uhi = ulo + A.bin_mm;
            const float dn = q.x < ulo ? ulo - q.x : (q.x > uhi ? q.x - uhi : 0.0f);
            const float s2 = q.y * kSqrtLn2;
            const float M = (bl < nb && dn <= q.w) ? bin_mass((ulo - q.x) * s2, (uhi - q.x) * s2) : 0.0f;
            Mb[mc * kTJ + bl] = M;
            const unsigned bal = __ballot_sync(0xffffffffu, M != 0.0f);
            if (lane < 4 && ((bal >> (8 * lane)) & 0xffu)) atomicOr(live + 4 * (warp & 1) + lane, 1u << mc);
        }
        // C_k = W M_E(k; E') of the stage
        const float* pS = planes + (buf * 3 + 0) * kPlaneF;
        const float* pB = planes + (buf * 3 + 1) * kPlaneF;
        const float* pW = planes + (buf * 3 + 2) * kPlaneF;
        for (int kk = tid; kk < kStage * kTN; kk += kBuildThreads) {
            const float sv = pS[kk], bv = pB[kk], nlw = pW[kk];
            float Cv = 0.0f;
            if (sv > 0.0f && nlw < INFINITY)
                Cv = ex2_approx(-nlw) * kSqrtPiLog2e / sv *
                     bin_mass(fmaf(el, sv, bv) * kSqrtLn2, fmaf(eh, sv, bv) * kSqrtLn2);
            Cm[kk] = Cv;
        }
        __syncthreads();
        const unsigned wlive = live[warp];
        for (int mc = 0; mc < kStage; ++mc) {
            if (!((wlive >> mc) & 1u)) continue;
            const float4 C = *reinterpret_cast<const float4*>(Cm + mc * kTN + 4 * lane);
            const float4 M0 = *reinterpret_cast<const float4*>(Mb + mc * kTJ + 8 * warp);
            const float4 M1 = *reinterpret_cast<const float4*>(Mb + mc * kTJ + 8 * warp + 4);
            const float Mv[8] = {M0.x, M0.y, M0.z, M0.w, M1.x, M1.y, M1.z, M1.w};
            const float2 C01 = make_float2(C.x, C.y), C23 = make_float2(C.z, C.w);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const float2 m2 = make_float2(Mv[jj], Mv[jj]);
                acc[jj][0] = ffma2(m2, C01, acc[jj][0]);
                acc[jj][1] = ffma2(m2, C23, acc[jj][1]);
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const int b = b0 + 8 * warp + jj;
        if (b >= A.n_bins) continue;
        const int32_t r = rmap[(size_t)b * A.n_ebins];
        if (r >= 0) {
            float* row = A.out + (int64_t)r * A.ld_out;
            const int n = n0 + 4 * lane;
            if (n + 3 < A.n_store) {
                *reinterpret_cast<float4*>(row + n) =
                    make_float4(acc[jj][0].x, acc[jj][0].y, acc[jj][1].x, acc[jj][1].y);
            } else {
                const float v[4] = {acc[jj][0].x, acc[jj][0].y, acc[jj][1].x, acc[jj][1].y};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (n + q < A.n_store) row[n + q] = v[q];
            }
        }
    }
}

int64_t wtab_angle_floats(const lmosem_ctx* c);

// planes of a buffer of n_buf slots, followed by the slots' energy hulls
WTabArgs wtab_args(const lmosem_ctx* c, float* wtab, int n_buf, const int32_t* slot_angle, int s0) {
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
    W.scat_geo = c->d_scat_geo;
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
    W.n_ptiles = c->ld_w / kTN;
    W.hull = reinterpret_cast<uint2*>(wtab + (size_t)n_buf * 3 * c->n_scat * c->ld_w);
    W.hK = c->e_sigma > 0.0f ? (float)(c->e_sigma * sqrt(kappa)) : INFINITY;
    return W;
}

// per angle: three planes of n_scat x ld_w floats, then the energy hulls of
// n_scat x (ld_w / kTN) column tiles (two words each)
int64_t wtab_angle_floats(const lmosem_ctx* c) {
    return (int64_t)3 * c->n_scat * c->ld_w + (int64_t)2 * c->n_scat * (c->ld_w / kTN);
}

// hull words of n slots to their starting value (0xffffffff: no path yet)
lmosem_status hull_reset(lmosem_ctx* c, const WTabArgs& W, int n) {
    LMOSEM_CK(c, cudaMemsetAsync(W.hull, 0xff, sizeof(uint2) * (size_t)n * W.n_ptiles * c->n_scat, c->stream));
    return LMOSEM_OK;
}

}  // namespace

bool wtab_all_fits(const lmosem_ctx* c) {
    return (int64_t)c->n_angles * wtab_angle_floats(c) * (int64_t)sizeof(float) <= c->table_budget;
}

lmosem_status wtab_all_with_sens(lmosem_ctx* c, double* sens_angle, float w_const_sens, float de0) {
    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_wtab_all, (size_t)c->n_angles * wtab_angle_floats(c)))) return st;
    WSensArgs S;
    S.w = wtab_args(c, c->d_wtab_all, c->n_angles, nullptr, 0);
    if ((st = hull_reset(c, S.w, c->n_angles))) return st;
    S.ppar = c->d_ppar;
    S.du_m = c->d_du_m;
    S.w_const_sens = w_const_sens;
    S.de0 = de0;
    S.sens_angle = sens_angle;
    LMOSEM_PROF_BEGIN(c);
    // 64-thread blocks: every (column block, angle) resident at once
    k_wtable_sens<<<dim3((c->ld_w + 63) / 64, c->n_angles), 64, 0, c->stream>>>(S);
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
    if (!c->d_terms && (st = dev_alloc(c, &c->d_terms, 1))) return st;
    LMOSEM_CK(c, cudaMemsetAsync(c->d_terms, 0, sizeof(unsigned long long), c->stream));
    c->terms_valid = true;

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
    const uint2* hull = wtab_args(c, wtab, pre ? c->n_angles : gsz, nullptr, 0).hull;
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
    const size_t smem_w = sizeof(float) * ((size_t)kWOffList + c->n_scat);
    const size_t smem_n = sizeof(float) * ((size_t)kOffList + c->n_scat);
    const size_t smem_t = sizeof(float) * ((size_t)kTOffList + c->n_scat);
    LMOSEM_CK(c, cudaFuncSetAttribute(k_pathsum_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_pathsum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_pathsum_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_n));
    // a last column tile with few live columns takes the narrow form
    const int nq_tail = (c->n_sup - (n_ptiles - 1) * kTN + 3) / 4;
    const bool narrow_tail = nq_tail <= kNarrowQ;
    const int n_wide = narrow_tail ? n_ptiles - 1 : n_ptiles;

    for (int gi = 0; gi < n_groups; ++gi) {
        const int s0 = gi * gsz, s1 = std::min(ns, s0 + gsz);
        if (!pre) {
            WTabArgs W = wtab_args(c, c->d_wtab, gsz, d_slot_angle, s0);
            if ((st = hull_reset(c, W, s1 - s0))) return st;
            LMOSEM_PROF_BEGIN(c);
            k_wtable<<<dim3((c->ld_w + 255) / 256, c->n_scat), 256, 0, c->stream>>>(W, s1 - s0);
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
        P.pt0 = 0;
        P.n_pt = n_wide;
        P.n_tiles = tiles;
        P.nq_tail = nq_tail;
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
        P.hull = hull;
        P.n_ptiles = n_ptiles;
        P.e_cut = c->e_sigma > 0.0f ? 1 : 0;
        P.n_sup = c->n_sup;
        P.n_terms = c->d_terms;
        const int64_t grow0 = g_row0[gi], grows = g_rows[gi];
        if (scaled) {
            P.out = c->d_stage;
            P.row_base = grow0;
        } else {
            P.out = reinterpret_cast<float*>(c->d_model);
            P.row_base = 0;
        }
        if (n_wide > 0) {
            LMOSEM_PROF_BEGIN(c);
            k_pathsum<<<(unsigned)((int64_t)tiles * n_wide), kBuildThreads, smem_w, c->stream>>>(P);
            LMOSEM_LAUNCHED(c, LMOSEM_K_PATHSUM);
        }
        if (narrow_tail) {
            P.pt0 = n_ptiles - 1;
            P.n_pt = 1;
            LMOSEM_PROF_BEGIN(c);
            if (nq_tail <= kTailQ)
                k_pathsum_tail<<<(unsigned)tiles, kTJ, smem_t, c->stream>>>(P);
            else
                k_pathsum_narrow<<<(unsigned)tiles, kBuildThreads, smem_n, c->stream>>>(P);
            LMOSEM_LAUNCHED(c, LMOSEM_K_PATHSUM);
        }
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
    // stream-ordered frees: no host wait (the caller's events were consumed
    // before the sort's last synchronisation)
    dev_free(c, &c->d_wtab);
    dev_free(c, &c->d_wtab_all);  // consumed
    dev_free(c, &c->d_stage);
    return LMOSEM_OK;
}

namespace {

__global__ void k_judge_gather(const int32_t* __restrict__ a_s, const float* __restrict__ u_s,
                                const float* __restrict__ e_s, const int64_t* __restrict__ rows, int64_t K,
                                int32_t* __restrict__ a_o, float* __restrict__ u_o, float* __restrict__ e_o) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t r = rows[k];
    a_o[k] = a_s[r];
    u_o[k] = u_s[r];
    e_o[k] = e_s[r];
}

// sampled row k: sum over the support of (surrogate - exact)^2 and exact^2,
// FP64, in a fixed order (one CTA per row)
__global__ void __launch_bounds__(256) k_judge_rows(const float* __restrict__ model, int64_t ld,
                                                    const int64_t* __restrict__ rows,
                                                    const float* __restrict__ exact, int n_sup,
                                                    double* __restrict__ out) {
    __shared__ double sh[2][8];
    const int64_t k = blockIdx.x;
    const float* ps = model + rows[k] * ld;
    const float* pe = exact + k * ld;
    double d2 = 0.0, e2 = 0.0;
    for (int n = threadIdx.x; n < n_sup; n += blockDim.x) {
        const double e = pe[n], d = (double)ps[n] - e;
        d2 += d * d;
        e2 += e * e;
    }
    for (int o = 16; o; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][warp] = d2;
        sh[1][warp] = e2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        out[2 * k] = a;
        out[2 * k + 1] = b;
    }
}

}  // namespace

// Exact FP32 rows (primary and every first-order scatter path) of K sorted
// model rows h_rows (increasing; d_rows their device copy) into d_out
// (K x ld_model): the rows' events are gathered and built by the exact path
// sum in place of the model's events, and the model's event state is put back
// after.  The rows of a (realisation, angle) stay contiguous in the sample,
// and a row's bits do not depend on the other events of its tiles, so every
// row equals the one the exact build of all events gives.  h_e (K floats, may
// be NULL) receives the rows' event energies.
lmosem_status exact_rows(lmosem_ctx* c, const std::vector<int64_t>& h_rows, const int64_t* d_rows, float* d_out,
                         float* h_e) {
    const int64_t K = (int64_t)h_rows.size();
    if (K == 0) return LMOSEM_OK;
    lmosem_status st;
    int32_t* d_a = nullptr;
    float *d_u = nullptr, *d_e = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&d_a, K)) || (st = tmp.alloc(&d_u, K)) || (st = tmp.alloc(&d_e, K))) return st;
    LMOSEM_PROF_BEGIN(c);
    k_judge_gather<<<(unsigned)((K + 255) / 256), 256, 0, c->stream>>>(c->d_a_s, c->d_u_s, c->d_e_s, d_rows, K,
                                                                        d_a, d_u, d_e);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    std::vector<int32_t> h_a(K);
    LMOSEM_CK(c, cudaMemcpyAsync(h_a.data(), d_a, K * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    if (h_e) LMOSEM_CK(c, cudaMemcpyAsync(h_e, d_e, K * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    std::vector<int64_t> s_row0((size_t)c->n_real * c->n_angles, 0), s_cnt((size_t)c->n_real * c->n_angles, 0);
    int r = 0;
    for (int64_t k = 0; k < K; ++k) {
        while (r + 1 < c->n_real && h_rows[k] >= c->h_real_row0[r + 1]) ++r;
        const size_t i = (size_t)r * c->n_angles + h_a[k];
        if (s_cnt[i]++ == 0) s_row0[i] = k;
    }
    const int64_t J0 = c->J;
    int32_t* a0 = c->d_a_s;
    float *u0 = c->d_u_s, *e0 = c->d_e_s;
    void* m0 = c->d_model;
    const int fmt0 = c->fmt;
    const bool sur0 = c->use_surrogate;
    std::vector<int64_t> row0_0, cnt0;
    row0_0.swap(c->h_angle_row0);
    cnt0.swap(c->h_angle_cnt);
    c->h_angle_row0 = s_row0;
    c->h_angle_cnt = s_cnt;
    c->J = K;
    c->d_a_s = d_a;
    c->d_u_s = d_u;
    c->d_e_s = d_e;
    c->d_model = d_out;
    c->fmt = LMOSEM_MODEL_FP32;
    c->use_surrogate = false;
    st = build_model_rows(c);
    c->use_surrogate = sur0;
    c->fmt = fmt0;
    c->d_model = m0;
    c->d_e_s = e0;
    c->d_u_s = u0;
    c->d_a_s = a0;
    c->J = J0;
    c->h_angle_row0.swap(row0_0);
    c->h_angle_cnt.swap(cnt0);
    return st;
}

namespace {

// model row rows[k] <- src row k (FP32, ld4 float4 per row)
__global__ void k_scatter_rows(const float4* __restrict__ src, const int64_t* __restrict__ rows, int64_t ld4,
                               float4* __restrict__ model) {
    const int64_t k = blockIdx.x;
    const float4* in = src + k * ld4;
    float4* out = model + rows[k] * ld4;
    for (int64_t i = threadIdx.x; i < ld4; i += blockDim.x) out[i] = in[i];
}

}  // namespace

// The exact judge of a surrogate build: K sorted rows evenly spaced over the
// model ((k + 1/2) J / K, so every subset and angle group is sampled) are
// rebuilt with the exact path sum into scratch rows and compared with the
// surrogate's rows.  row_sums (2K: squared difference and squared exact
// norm of every sampled row) and row_e (K event energies) may be NULL.
std::vector<int64_t> judge_sample_rows(const lmosem_ctx* c) {
    const int64_t J = c->J;
    const int64_t K = std::min<int64_t>(J, c->sur_check_rows);
    std::vector<int64_t> rows(K);
    for (int64_t k = 0; k < K; ++k) rows[k] = (int64_t)(((double)k + 0.5) * (double)J / (double)K);
    return rows;
}

lmosem_status judge_surrogate(lmosem_ctx* c, double* rel_err, double* row_max, std::vector<double>* row_sums,
                              std::vector<float>* row_e) {
    const std::vector<int64_t> rows = judge_sample_rows(c);
    const int64_t K = (int64_t)rows.size();
    lmosem_status st;
    int64_t* d_rows = nullptr;
    float* d_ex = nullptr;
    double* d_sums = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&d_rows, K)) || (st = tmp.alloc(&d_ex, (size_t)K * c->ld_model)) ||
        (st = tmp.alloc(&d_sums, 2 * K)))
        return st;
    LMOSEM_CK(c, cudaMemcpyAsync(d_rows, rows.data(), K * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    std::vector<float> energies(K);
    if ((st = exact_rows(c, rows, d_rows, d_ex, energies.data()))) return st;
    LMOSEM_PROF_BEGIN(c);
    k_judge_rows<<<(unsigned)K, 256, 0, c->stream>>>(reinterpret_cast<const float*>(c->d_model), c->ld_model,
                                                      d_rows, d_ex, c->n_sup, d_sums);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    std::vector<double> sums(2 * K);
    LMOSEM_CK(c, cudaMemcpyAsync(sums.data(), d_sums, 2 * K * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    double d2 = 0.0, e2 = 0.0, mx = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        d2 += sums[2 * k];
        e2 += sums[2 * k + 1];
        if (sums[2 * k + 1] > 0.0) mx = std::max(mx, sqrt(sums[2 * k] / sums[2 * k + 1]));
        else if (sums[2 * k] > 0.0) mx = INFINITY;
    }
    *rel_err = e2 > 0.0 ? sqrt(d2 / e2) : (d2 > 0.0 ? INFINITY : 0.0);
    *row_max = mx;
    if (row_sums) row_sums->swap(sums);
    if (row_e) row_e->swap(energies);
    return LMOSEM_OK;
}

// The sorted rows whose event energy lies at or above e_cut (every row when
// e_cut is the window's lower edge), built by the surrogate network.
lmosem_status build_surrogate_rows_above(lmosem_ctx* c, double e_cut, int64_t* n_built) {
    const int64_t J = c->J;
    if (e_cut <= c->e_lo) {
        *n_built = J;
        return build_model_surrogate_rows(c, nullptr, 0);
    }
    std::vector<float> e(J);
    LMOSEM_CK(c, cudaMemcpyAsync(e.data(), c->d_e_s, J * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    std::vector<int64_t> rows;
    for (int64_t r = 0; r < J; ++r)
        if (!((double)e[r] < e_cut)) rows.push_back(r);
    *n_built = (int64_t)rows.size();
    if (rows.empty()) return LMOSEM_OK;
    lmosem_status st;
    int64_t* d_rows = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&d_rows, rows.size()))) return st;
    LMOSEM_CK(c, cudaMemcpyAsync(d_rows, rows.data(), rows.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 c->stream));
    st = build_model_surrogate_rows(c, d_rows, (int64_t)rows.size());  // synchronises before rows is freed
    return st;
}

// The rows of the current (FP32) model whose event energy lies below e_cut,
// replaced by exact rows: the rows are rebuilt by the exact path sum in
// chunks of at most 8 GiB of scratch rows and copied over the model's.
lmosem_status rebuild_rows_below(lmosem_ctx* c, double e_cut, int64_t* n_rebuilt) {
    const int64_t J = c->J;
    std::vector<float> e(J);
    LMOSEM_CK(c, cudaMemcpyAsync(e.data(), c->d_e_s, J * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    std::vector<int64_t> rows;
    for (int64_t r = 0; r < J; ++r)
        if ((double)e[r] < e_cut) rows.push_back(r);
    *n_rebuilt = (int64_t)rows.size();
    if (rows.empty()) return LMOSEM_OK;
    if (c->ld_model % 4) return fail(c, LMOSEM_ESTATE, "model rows not 16-byte aligned");
    const int64_t row_bytes = c->ld_model * (int64_t)sizeof(float);
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>((int64_t)rows.size(), (int64_t(8) << 30) / row_bytes));
    lmosem_status st;
    int64_t* d_rows = nullptr;
    float* d_ex = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&d_rows, per)) || (st = tmp.alloc(&d_ex, (size_t)per * c->ld_model))) return st;
    for (int64_t k0 = 0; k0 < (int64_t)rows.size(); k0 += per) {
        const int64_t K = std::min<int64_t>(per, (int64_t)rows.size() - k0);
        std::vector<int64_t> part(rows.begin() + k0, rows.begin() + k0 + K);
        LMOSEM_CK(c, cudaMemcpyAsync(d_rows, part.data(), K * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
        if ((st = exact_rows(c, part, d_rows, d_ex, nullptr))) return st;
        LMOSEM_PROF_BEGIN(c);
        k_scatter_rows<<<(unsigned)K, 256, 0, c->stream>>>(reinterpret_cast<const float4*>(d_ex), d_rows,
                                                           c->ld_model / 4, reinterpret_cast<float4*>(c->d_model));
        LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
        // the host copy of this chunk's rows must outlive the copy above
        LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    }
    return LMOSEM_OK;
}

lmosem_status build_binned_rows(lmosem_ctx* c, const int32_t* d_rowmap, int n_ebins, const double* e_edges) {
    if (n_ebins < 1 || n_ebins > kMaxEBins) return fail(c, LMOSEM_EINVAL, "1..8 energy bins");
    lmosem_status st;
    const int n_ptiles = c->ld_w / kTN;
    const int n_btiles = (c->n_bins + kTJ - 1) / kTJ;
    const bool pre = c->d_wtab_all != nullptr;
    const int64_t per_angle = wtab_angle_floats(c) * (int64_t)sizeof(float);
    const int gsz = pre ? c->n_angles
                        : (int)std::max<int64_t>(1, std::min<int64_t>(c->n_angles, c->table_budget / per_angle));

    BinnedArgs B;
    B.ld_w = c->ld_w;
    B.n_scat = c->n_scat;
    B.wslot_by_angle = pre ? 1 : 0;
    B.mpar = c->d_mpar;
    B.ppar = c->d_ppar;
    B.n_bins = c->n_bins;
    B.bin_mm = (float)c->bin_mm;
    B.half = (float)(0.5 * c->n_bins * c->bin_mm);
    B.n_ebins = n_ebins;
    const double fw2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    const double kappa = pow(c->fwhm_frac * fw2s, 2.0) * c->e0;  // sigma_E^2 = kappa E
    const double se0 = sqrt(kappa * c->e0);
    for (int k = 0; k <= n_ebins; ++k) B.e_edge[k] = (float)e_edges[k];
    for (int k = 0; k < n_ebins; ++k)
        B.pe_mass[k] = (float)(0.5 * erfc(-(e_edges[k + 1] - c->e0) / (se0 * sqrt(2.0))) -
                               0.5 * erfc(-(e_edges[k] - c->e0) / (se0 * sqrt(2.0))));
    B.n_btiles = n_btiles;
    B.n_ptiles = n_ptiles;
    B.rowmap = d_rowmap;
    B.out = reinterpret_cast<float*>(c->d_model);
    B.ld_out = c->ld_model;
    B.n_store = (int)c->ld_model;
    B.scatter_only = c->scatter_only ? 1 : 0;

    // identity slot -> angle map for the per-group table kernel
    Scratch tmp(c);
    int32_t* d_ang = nullptr;
    if (!pre) {
        if ((st = tmp.alloc(&d_ang, c->n_angles))) return st;
        std::vector<int32_t> ident(c->n_angles);
        for (int a = 0; a < c->n_angles; ++a) ident[a] = a;
        LMOSEM_CK(c, cudaMemcpyAsync(d_ang, ident.data(), ident.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, c->stream));
        if ((st = dev_alloc(c, &c->d_wtab, (size_t)gsz * wtab_angle_floats(c)))) return st;
    }
    const size_t smem = sizeof(float) * ((size_t)kBOffList + c->n_scat);
    LMOSEM_CK(c, cudaFuncSetAttribute(k_binned, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int a0 = 0; a0 < c->n_angles; a0 += gsz) {
        const int na = std::min(gsz, c->n_angles - a0);
        if (!pre) {
            WTabArgs W = wtab_args(c, c->d_wtab, gsz, d_ang, a0);
            if ((st = hull_reset(c, W, na))) return st;  // written by the table kernel, unused here
            LMOSEM_PROF_BEGIN(c);
            k_wtable<<<dim3((c->ld_w + 255) / 256, c->n_scat), 256, 0, c->stream>>>(W, na);
            LMOSEM_LAUNCHED(c, LMOSEM_K_WTABLE);
        }
        B.wtab = pre ? c->d_wtab_all : c->d_wtab;
        B.a0 = a0;
        LMOSEM_PROF_BEGIN(c);
        k_binned<<<(unsigned)((int64_t)na * n_ebins * n_btiles * n_ptiles), kBuildThreads, smem, c->stream>>>(B);
        LMOSEM_LAUNCHED(c, LMOSEM_K_PATHSUM);
    }
    dev_free(c, &c->d_wtab);      // stream-ordered frees: no host wait
    dev_free(c, &c->d_wtab_all);  // consumed
    return LMOSEM_OK;
}

}  // namespace lmosem
