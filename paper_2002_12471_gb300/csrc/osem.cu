// OS-LM-MLEM iterations on the cached model (rows a7-a8 of the hot path).
//
// Paper Eq. 8 gives the E-step zbar_{j,P_q} = f_q p_jq / y_j with
// y_j = sum_n p_jn f_n, and Eq. 7 the subset update
//     f_q <- sum_{j in S_i} zbar_{j,P_q} / (T s^i_q) = f_q b_q / (T s^i_q),
//     b_q = sum_{j in S_i, y_j > 0} p_jq / y_j.
// Each sub-iteration is one streaming pass over the subset's model rows:
// every row is loaded once from HBM into registers (the next rows are
// already in flight while the current ones are reduced; for wide FP32 rows
// they are staged through a cp.async ring instead), y_j is formed by a CTA
// reduction, and the same registers are back-projected into the CTA's
// private b (registers, FP32).  A second kernel reduces the per-CTA b in a
// fixed order (deterministic) and applies the update with T s^i_q formed in
// FP64.  Binned rows carry a count that weights their back-projection and
// log-likelihood terms.
// The log-likelihood of Eq. 3 (without log J!) has its own pass: log(y_j) in
// FP32, reduced in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kMaxPassThreads = 256;

// 16-byte vector of model elements -> floats
template <typename H>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int N = 4;
    __device__ static void cvt(const uint4& v, float* out) {
        out[0] = __uint_as_float(v.x);
        out[1] = __uint_as_float(v.y);
        out[2] = __uint_as_float(v.z);
        out[3] = __uint_as_float(v.w);
    }
};
template <>
struct Vec<__half> {
    static constexpr int N = 8;
    __device__ static void cvt(const uint4& v, float* out) {
        const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __half22float2(h[k]);
            out[2 * k] = f.x;
            out[2 * k + 1] = f.y;
        }
    }
};
template <>
struct Vec<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ static void cvt(const uint4& v, float* out) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(h[k]);
            out[2 * k] = f.x;
            out[2 * k + 1] = f.y;
        }
    }
};

// (a.x b.x + c.x, a.y b.y + c.y) in one packed FP32x2 FMA
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

// Programmatic dependent launch: a sub-iteration's pass and update are
// launched with programmatic stream serialisation, so a kernel can start
// while its predecessor finishes.  pdl_wait() blocks until the preceding
// kernel of the stream has completed and its writes are visible (a no-op
// without such a launch); pdl_trigger() lets the next kernel be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

struct PassArgs {
    const void* model;
    int64_t ld_bytes;        // row stride in bytes
    int64_t nvec;            // 16-byte vectors per row
    int64_t r0, r1;          // rows of this pass
    int64_t rows_per_cta;
    const float* f;
    const float* scale;      // row scales (scaled forms) or nullptr
    const float* weight;     // row counts (binned rows) or nullptr (events: 1)
    int n_sup;
    double log_T;
    float* bpart;            // [cta][n_sup]
    double* llpart;          // [cta]
    int prefetch;            // register pass: row groups fetched into L2 this many groups ahead (0: none)
};

// rows [r, min(r + R, re)) of the model into L2, one bulk prefetch per row
// (the row's nvec 16-byte vectors: 16-byte aligned start and size)
template <int R>
__device__ __forceinline__ void prefetch_rows_l2(const char* model, int64_t ld_bytes, int64_t nvec, int64_t r,
                                                 int64_t re, int warp, int nwarps, int lane) {
    if (lane != 0) return;
    for (int i = warp; i < R; i += nwarps) {
        if (r + i >= re) return;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(model + (r + i) * ld_bytes),
                     "r"((unsigned)(nvec * 16))
                     : "memory");
    }
}

// One pass over rows [r0, r1): thread t owns the 16-byte column vectors
// t, t + NT, ... (VPT of them); groups of R rows are double-buffered in
// registers.  BACK: accumulate b; otherwise accumulate the log-likelihood.
// Rows per pipeline step (R) and minimum CTAs per SM of the register pass,
// per instance, as measured on GB300 (ms per OSEM iteration, one box):
//  * FP32, up to 4 vectors per thread: R = 4 or 2, no register cap (a cap
//    of two CTAs shortens the schedule: 64x64 rows 0.25 vs 0.31 ms);
//  * FP32, 6 or 8 vectors: R = 1 and two CTAs per SM (one CTA otherwise:
//    128x128 rows 1.03 vs 1.29 ms);
//  * 2-byte rows with 3 vectors per thread (twice the elements, and the
//    registers, per vector): R = 1 and two CTAs per SM, so the conversion
//    chains of one CTA overlap the other's (128x128 FP16 0.70 vs 0.76 ms);
//  * other 2-byte shapes: as FP32.
template <typename H, int VPT>
constexpr bool pass_half3() { return !std::is_same<H, float>::value && VPT == 3; }
template <typename H, int VPT>
constexpr int pass_min_ctas() {
    return pass_half3<H, VPT>() || (std::is_same<H, float>::value && VPT >= 6) ? 2 : 1;
}
template <typename H, int VPT>
constexpr int pass_rows() {
    return pass_half3<H, VPT>() ? 1 : (VPT >= 6 ? 1 : (VPT >= 3 ? 2 : 4));
}

// W: rows carry counts (binned rows; A.weight), compiled apart so that the
// list-mode pass keeps its exact instruction stream.
template <typename H, int VPT, int R, bool BACK, bool W>
__global__ void __launch_bounds__(kMaxPassThreads, pass_min_ctas<H, VPT>()) k_pass(PassArgs A) {
    constexpr int EPV = Vec<H>::N;
    static_assert(kMaxPassThreads / 32 == 8, "eight per-warp partials per row");
    __shared__ __align__(16) float red[2][R][kMaxPassThreads / 32];
    __shared__ double llred[kMaxPassThreads / 32];
    const int NT = blockDim.x, NW = NT >> 5;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const char* model = reinterpret_cast<const char*>(A.model);
    // the partial slots no warp writes hold +0 (read by sum8_in_order; the
    // first row group's barrier orders these stores before any read)
    for (int k = t; k < 2 * R * 8; k += NT)
        if ((k & 7) >= NW) (&red[0][0][0])[k] = 0.0f;

    float fr[VPT][EPV], br[VPT][EPV];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
        for (int e = 0; e < EPV; ++e) br[v][e] = 0.0f;
    // the image, once the kernel that wrote it has finished (the first rows
    // are already in flight: they do not depend on it)
    auto load_f = [&]() {
        pdl_wait();
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int col0 = EPV * (t + NT * v);
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
                int col = col0 + e;
                fr[v][e] = col < A.n_sup ? A.f[col] : 0.0f;
            }
        }
    };
    const int64_t rb = A.r0 + (int64_t)blockIdx.x * A.rows_per_cta;
    const int64_t re = min(A.r1, rb + A.rows_per_cta);
    double ll = 0.0;
    double npos = 0.0;  // weight of the rows with y > 0

    auto load = [&](int64_t r, uint4 (&dst)[R][VPT]) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                int64_t vec = t + (int64_t)NT * v;
                if (r + i < re && vec < A.nvec)
                    dst[i][v] = __ldcs(reinterpret_cast<const uint4*>(model + (r + i) * A.ld_bytes) + vec);
                else
                    dst[i][v] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    };
    auto process = [&](int64_t r, const uint4 (&raw)[R][VPT], int rb_) {
        float d[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            float2 s2 = make_float2(0.0f, 0.0f);  // even and odd columns
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                float p[EPV];
                Vec<H>::cvt(raw[i][v], p);
#pragma unroll
                for (int e = 0; e < EPV; e += 2)
                    s2 = ffma2(make_float2(p[e], p[e + 1]), make_float2(fr[v][e], fr[v][e + 1]), s2);
            }
            float s = s2.x + s2.y;
#pragma unroll
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            d[i] = s;
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < R; ++i) red[rb_][i][warp] = d[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const float y = sum8_in_order(red[rb_][i]);
            const bool ok = r + i < re && y > 0.0f;
            if constexpr (BACK) {
                float inv = ok ? 1.0f / y : 0.0f;
                if constexpr (W) inv *= A.weight[r + i];  // a binned row counts its photons
                const float2 inv2 = make_float2(inv, inv);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float p[EPV];
                    Vec<H>::cvt(raw[i][v], p);
#pragma unroll
                    for (int e = 0; e < EPV; e += 2) {
                        const float2 b2 = ffma2(make_float2(p[e], p[e + 1]), inv2,
                                                make_float2(br[v][e], br[v][e + 1]));
                        br[v][e] = b2.x;
                        br[v][e + 1] = b2.y;
                    }
                }
            } else {
                if (ok && t == i) {
                    const float c = A.scale ? A.scale[r + i] : 1.0f;
                    if constexpr (W) {
                        const double w = (double)A.weight[r + i];
                        ll += w * (double)logf(c * y);
                        npos += w;
                    } else {
                        ll += (double)logf(c * y);
                        npos += 1.0;
                    }
                }
            }
        }
    };

    // register double buffer: group g + 1 loads while group g is processed;
    // with A.prefetch = D, group g + 1 + D is requested into L2 at the same
    // time, so D more groups are in flight than the registers hold
    const int64_t ahead = (int64_t)A.prefetch * R;
    uint4 P0[R][VPT], P1[R][VPT];
    if (rb < re) load(rb, P0);
    for (int64_t k = 1; k <= A.prefetch; ++k)
        prefetch_rows_l2<R>(model, A.ld_bytes, A.nvec, rb + k * R, re, warp, NW, lane);
    load_f();
    for (int64_t r = rb; r < re; r += 2 * R) {
        if (ahead) prefetch_rows_l2<R>(model, A.ld_bytes, A.nvec, r + R + ahead, re, warp, NW, lane);
        if (r + R < re) load(r + R, P1);
        process(r, P0, 0);
        if (r + R >= re) break;
        if (ahead) prefetch_rows_l2<R>(model, A.ld_bytes, A.nvec, r + 2 * R + ahead, re, warp, NW, lane);
        if (r + 2 * R < re) load(r + 2 * R, P0);
        process(r + R, P1, 1);
    }
    pdl_trigger();
    if constexpr (BACK) {
        float* bp = A.bpart + (size_t)blockIdx.x * A.n_sup;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int col0 = EPV * (t + NT * v);
#pragma unroll
            for (int e = 0; e < EPV; ++e)
                if (col0 + e < A.n_sup) bp[col0 + e] = br[v][e];
        }
    } else {
        // per-CTA partial: sum_j w_j (log(c_j y_j) + log T), fixed order
        ll += npos * A.log_T;
        for (int o = 16; o; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
        if (lane == 0) llred[warp] = ll;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += llred[w];
            A.llpart[blockIdx.x] = s;
        }
    }
}

// The same pass with the rows staged through shared memory by cp.async:
// thread t copies, and later reads, only its own 16-byte vectors of each row,
// so its slots of the S-stage ring are private (no barrier guards them) and
// S - 1 row groups stay in flight per thread instead of the one the
// register double buffer allows.  The arithmetic is that of k_pass, in the
// same order.
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most n of this thread's newest copy groups are pending (n < 8)
__device__ __forceinline__ void cpa_wait(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
        case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
    }
}
constexpr int kCpaMaxStages = 8;
// Row groups the register pass prefetches into L2 ahead of its loads, unless
// the context sets a distance: for one-row groups (the wide rows), about
// 48 KB ahead per CTA, as measured on GB300 (ms per OSEM iteration, one box,
// 1M events at 128x128): FP16 rows (12 KB) 2.50 without, 1.98 / 1.89 / 1.87 /
// 1.88 / 2.09 ms at 1 / 2 / 4 / 6 / 12 rows ahead; FP32 rows (24 KB) 3.41 ms
// at 2 rows ahead and 3.47 at 4, against 3.64 for the cp.async ring.  The
// 64x64 FP32 groups of 4 rows gain nothing (0.266 ms without, 0.267 / 0.269 /
// 0.281 at 1 / 2 / 4 groups ahead): none there.
constexpr int64_t kPrefetchBytes = 48 << 10;
inline int auto_prefetch(int requested, int rows_per_group, int64_t ld_bytes) {
    if (requested < 0) return 0;
    if (requested > 0) return requested;
    if (rows_per_group != 1) return 0;
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, (kPrefetchBytes + ld_bytes / 2) / ld_bytes));
}

template <typename H, int VPT, int R, bool BACK, bool W>
__global__ void __launch_bounds__(kMaxPassThreads, pass_min_ctas<H, VPT>()) k_pass_cpa(PassArgs A, int S) {
    constexpr int EPV = Vec<H>::N;
    extern __shared__ __align__(128) unsigned char cring[];
    static_assert(kMaxPassThreads / 32 == 8, "eight per-warp partials per row");
    __shared__ __align__(16) float red[2][R][kMaxPassThreads / 32];
    __shared__ double llred[kMaxPassThreads / 32];
    const int NT = blockDim.x, NW = NT >> 5;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const char* model = reinterpret_cast<const char*>(A.model);
    // the partial slots no warp writes hold +0 (read by sum8_in_order; the
    // first row group's barrier orders these stores before any read)
    for (int k = t; k < 2 * R * 8; k += NT)
        if ((k & 7) >= NW) (&red[0][0][0])[k] = 0.0f;

    float fr[VPT][EPV], br[VPT][EPV];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
        for (int e = 0; e < EPV; ++e) br[v][e] = 0.0f;
    const int64_t rb = A.r0 + (int64_t)blockIdx.x * A.rows_per_cta;
    const int64_t re = min(A.r1, rb + A.rows_per_cta);
    const int64_t ngroups = re > rb ? (re - rb + R - 1) / R : 0;
    const size_t gbytes = (size_t)R * A.ld_bytes;
    double ll = 0.0;
    double npos = 0.0;

    auto issue = [&](int64_t g) {
        unsigned char* dst = cring + (size_t)(g % S) * gbytes;
        const int64_t r0 = rb + g * R;
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int64_t vec = t + (int64_t)NT * v;
                if (r0 + i < re && vec < A.nvec)
                    cpa16(dst + i * A.ld_bytes + vec * 16, model + (r0 + i) * A.ld_bytes + vec * 16);
            }
        }
        cpa_commit();
    };
    for (int64_t g = 0; g < min((int64_t)S - 1, ngroups); ++g) issue(g);
    // the image, once the kernel that wrote it has finished (the first row
    // groups are already in flight)
    pdl_wait();
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        int col0 = EPV * (t + NT * v);
#pragma unroll
        for (int e = 0; e < EPV; ++e) {
            int col = col0 + e;
            fr[v][e] = col < A.n_sup ? A.f[col] : 0.0f;
        }
    }
    for (int64_t g = 0; g < ngroups; ++g) {
        const int64_t issued = min(ngroups, g + S - 1);
        cpa_wait((int)(issued - 1 - g));  // this thread's copies of group g have landed
        if (g + S - 1 < ngroups) issue(g + S - 1);  // into the slots of group g - 1, read by this thread only
        const unsigned char* st = cring + (size_t)(g % S) * gbytes;
        const int64_t r = rb + g * R;
        const int rb_ = (int)(g & 1);
        uint4 raw[R][VPT];
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int64_t vec = t + (int64_t)NT * v;
                raw[i][v] = (r + i < re && vec < A.nvec)
                                ? *reinterpret_cast<const uint4*>(st + i * A.ld_bytes + vec * 16)
                                : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        float d[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            float2 s2 = make_float2(0.0f, 0.0f);  // even and odd columns
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                float p[EPV];
                Vec<H>::cvt(raw[i][v], p);
#pragma unroll
                for (int e = 0; e < EPV; e += 2)
                    s2 = ffma2(make_float2(p[e], p[e + 1]), make_float2(fr[v][e], fr[v][e + 1]), s2);
            }
            float sum = s2.x + s2.y;
#pragma unroll
            for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            d[i] = sum;
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < R; ++i) red[rb_][i][warp] = d[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const float y = sum8_in_order(red[rb_][i]);
            const bool ok = r + i < re && y > 0.0f;
            if constexpr (BACK) {
                float inv = ok ? 1.0f / y : 0.0f;
                if constexpr (W) inv *= A.weight[r + i];
                const float2 inv2 = make_float2(inv, inv);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float p[EPV];
                    Vec<H>::cvt(raw[i][v], p);
#pragma unroll
                    for (int e = 0; e < EPV; e += 2) {
                        const float2 b2 = ffma2(make_float2(p[e], p[e + 1]), inv2,
                                                make_float2(br[v][e], br[v][e + 1]));
                        br[v][e] = b2.x;
                        br[v][e + 1] = b2.y;
                    }
                }
            } else {
                if (ok && t == i) {
                    const float c = A.scale ? A.scale[r + i] : 1.0f;
                    if constexpr (W) {
                        const double w = (double)A.weight[r + i];
                        ll += w * (double)logf(c * y);
                        npos += w;
                    } else {
                        ll += (double)logf(c * y);
                        npos += 1.0;
                    }
                }
            }
        }
    }
    pdl_trigger();
    if constexpr (BACK) {
        float* bp = A.bpart + (size_t)blockIdx.x * A.n_sup;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int col0 = EPV * (t + NT * v);
#pragma unroll
            for (int e = 0; e < EPV; ++e)
                if (col0 + e < A.n_sup) bp[col0 + e] = br[v][e];
        }
    } else {
        ll += npos * A.log_T;
        for (int o = 16; o; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
        if (lane == 0) llred[warp] = ll;
        __syncthreads();
        if (t == 0) {
            double sm = 0.0;
            for (int w = 0; w < NW; ++w) sm += llred[w];
            A.llpart[blockIdx.x] = sm;
        }
    }
}

// b_q = sum of the per-CTA partials, then f_q <- f_q b_q / (T s^i_q).  One
// CTA of kUpdWarps warps per 32 support pixels; warp w sums the partials
// w, w + kUpdWarps, ... with eight loads in flight, then warp 0 adds the warp
// sums in warp order (fixed order: deterministic).
constexpr int kUpdWarps = 32;
__global__ void __launch_bounds__(kUpdWarps * 32) k_update(const float* __restrict__ bpart, int nparts,
                                                          int n_sup, float* __restrict__ f,
                                                          const double* __restrict__ sens_i, double T,
                                                          const int* __restrict__ status) {
    if (status && *status) return;  // the pass was abandoned: keep the image
    __shared__ float sh[kUpdWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;  // <= kUpdWarps
    const int n = blockIdx.x * 32 + lane;
    float b = 0.0f;
    if (n < n_sup) {
        int c = warp;
        for (; c + 7 * nw < nparts; c += 8 * nw) {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = bpart[(size_t)(c + k * nw) * n_sup + n];
#pragma unroll
            for (int k = 0; k < 8; ++k) b += v[k];
        }
        for (; c < nparts; c += nw) b += bpart[(size_t)c * n_sup + n];
    }
    sh[warp][lane] = b;
    __syncthreads();
    if (warp == 0 && n < n_sup) {
        float s = 0.0f;
        for (int w = 0; w < nw; ++w) s += sh[w][lane];
        double sd = sens_i[n];
        float ts = (float)(T * sd);
        f[n] = sd > 0.0 ? f[n] * s / ts : 0.0f;
    }
}

// b_q over the per-CTA partials with every SM busy: a CTA owns 8 support
// pixels, its 32 groups of 8 threads sum the partials g, g + 32, ... (one
// 32-byte sector per load), then group 0 adds the 32 group sums in order.
constexpr int kUpdPix = 8, kUpdGroups = 32;
__global__ void __launch_bounds__(kUpdPix * kUpdGroups) k_update_px(const float* __restrict__ bpart, int nparts,
                                                                  int n_sup, float* __restrict__ f,
                                                                  const double* __restrict__ sens_i, double T,
                                                                  const int* __restrict__ status) {
    pdl_trigger();  // the next pass may start loading its rows (they do not depend on f)
    pdl_wait();     // the pass that wrote the partials has finished
    if (status && *status) return;
    __shared__ float sh[kUpdGroups][kUpdPix + 1];
    const int p = threadIdx.x % kUpdPix, g = threadIdx.x / kUpdPix;
    const int n = blockIdx.x * kUpdPix + p;
    float b = 0.0f;
    if (n < n_sup) {
        int c = g;
        for (; c + 7 * kUpdGroups < nparts; c += 8 * kUpdGroups) {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = bpart[(size_t)(c + k * kUpdGroups) * n_sup + n];
#pragma unroll
            for (int k = 0; k < 8; ++k) b += v[k];
        }
        for (; c < nparts; c += kUpdGroups) b += bpart[(size_t)c * n_sup + n];
    }
    sh[g][p] = b;
    __syncthreads();
    if (g == 0 && n < n_sup) {
        float s = 0.0f;
        for (int k = 0; k < kUpdGroups; ++k) s += sh[k][p];
        const double sd = sens_i[n];
        const float ts = (float)(T * sd);
        f[n] = sd > 0.0 ? f[n] * s / ts : 0.0f;
    }
}

// T sum_q s^i_q f_q for every subset i (FP64; one CTA per subset, fixed order)
__global__ void k_subset_totals(const double* __restrict__ sens, int n_sup, const float* __restrict__ f,
                                double T, double* __restrict__ out) {
    __shared__ double sh[256];
    const double* s = sens + (size_t)blockIdx.x * n_sup;
    double acc = 0.0;
    for (int n = threadIdx.x; n < n_sup; n += blockDim.x) acc += s[n] * (double)f[n];
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) t += sh[k];
        out[blockIdx.x] = T * t;
    }
}

// loglik = sum of the per-CTA partials - T sum_q s_q f_q (FP64, one block)
__global__ void k_ll_final(const double* __restrict__ llpart, int nparts,
                           const double* __restrict__ s_total, const float* __restrict__ f,
                           int n_sup, double T, double* __restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int n = threadIdx.x; n < n_sup; n += blockDim.x) acc += s_total[n] * (double)f[n];
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sf = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) sf += sh[k];
        double ll = 0.0;
        for (int k = 0; k < nparts; ++k) ll += llpart[k];
        *out = ll - T * sf;
    }
}

__global__ void k_init_image(const double* __restrict__ s_total, int n_sup, double J, double T,
                             float* __restrict__ f) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int n = threadIdx.x; n < n_sup; n += blockDim.x) acc += s_total[n];
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) s += sh[k];
        sh[0] = s;
    }
    __syncthreads();
    float v = (float)(J / (T * sh[0]));
    for (int n = threadIdx.x; n < n_sup; n += blockDim.x) f[n] = v;
}

template <typename H>
__global__ void k_model_rows(const H* __restrict__ model, int64_t ld, const float* __restrict__ scale,
                             const int64_t* __restrict__ rank, const int64_t* __restrict__ ids,
                             int64_t n, int n_sup, float* __restrict__ out) {
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n_sup) return;
    for (int64_t k = blockIdx.y; k < n; k += gridDim.y) {
        int64_t r = rank[ids[k]];
        float v;
        if constexpr (std::is_same<H, float>::value) v = model[r * ld + col];
        else if constexpr (std::is_same<H, __half>::value) v = __half2float(model[r * ld + col]);
        else v = __bfloat162float(model[r * ld + col]);
        if (scale) v *= scale[r];
        out[k * n_sup + col] = v;
    }
}

// ---------------------------------------------------------------------------
// Streaming pass through a shared-memory ring filled by bulk (TMA) copies.
//
// A CTA owns a contiguous chunk of rows.  Its rows come in groups of G
// consecutive rows (one cp.async.bulk of G row strides each) into S ring
// stages; every stage has an mbarrier that completes when the copy's bytes
// have landed.  Up to S groups are in flight while the CTA reduces the
// current one, so the pass streams at HBM rate without holding rows in
// registers.  Every wait is bounded: a wait that outlasts its clock budget
// sets *status = 1, waits (bounded) for the CTA's copies still in flight and
// returns without writing results.
constexpr int kRingMaxStages = 8;
constexpr int kRingMaxG = 8;

struct RingArgs {
    const char* model;
    int64_t ld_bytes;        // row stride, bytes (multiple of 16)
    int64_t nvec;            // 16-byte vectors per row holding the support
    int64_t r0, r1;          // rows of this pass
    int64_t rows_per_cta;
    int G, S;                // rows per stage, stages
    const float* f;
    const float* scale;      // row scales (scaled forms) or nullptr
    const float* weight;     // row counts (binned rows) or nullptr
    int n_sup;
    double log_T;
    float* bpart;            // [cta][n_sup]
    double* llpart;          // [cta]
    int* status;             // set to 1 on a wait timeout
    long long wait_budget;   // clock cycles per wait
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm_and_copy(uint64_t* bar, void* dst, const void* src,
                                                  unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false when the budget ran out.  The non-blocking test comes
// before every budget check (try_wait may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long budget) {
    const long long t0 = clock64();
    while (true) {
        if (mbar_test_wait(bar, parity)) return true;
        if (clock64() - t0 > budget) return false;
        if (mbar_try_wait(bar, parity)) return true;
    }
}

template <typename H, int VPT, bool BACK>
__global__ void __launch_bounds__(kMaxPassThreads) k_pass_ring(RingArgs A) {
    constexpr int EPV = Vec<H>::N;
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ __align__(8) uint64_t bar[kRingMaxStages];
    __shared__ float red[kRingMaxG][kMaxPassThreads / 32];
    __shared__ double llred[kMaxPassThreads / 32];
    const int NT = blockDim.x, NW = NT >> 5;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int G = A.G, S = A.S;
    const int64_t stage_bytes = (int64_t)G * A.ld_bytes;

    float fr[VPT][EPV], br[VPT][EPV];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        int col0 = EPV * (t + NT * v);
#pragma unroll
        for (int e = 0; e < EPV; ++e) {
            int col = col0 + e;
            fr[v][e] = col < A.n_sup ? A.f[col] : 0.0f;
            br[v][e] = 0.0f;
        }
    }
    const int64_t rb = A.r0 + (int64_t)blockIdx.x * A.rows_per_cta;
    const int64_t re = min(A.r1, rb + A.rows_per_cta);
    const int64_t ngroups = re > rb ? (re - rb + G - 1) / G : 0;

    if (t == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t g) {  // thread 0 only
        const int s = (int)(g % S);
        const int64_t row = rb + g * G;
        const int64_t nrow = min((int64_t)G, re - row);
        mbar_arm_and_copy(&bar[s], ring + s * stage_bytes, A.model + row * A.ld_bytes,
                          (unsigned)(nrow * A.ld_bytes));
    };
    if (t == 0)
        for (int64_t g = 0; g < min((int64_t)S, ngroups); ++g) issue(g);

    double ll = 0.0;
    double npos = 0.0;  // weight of the rows with y > 0
    bool aborted = false;
    int64_t g = 0;
    for (; g < ngroups; ++g) {
        const int s = (int)(g % S);
        const unsigned parity = (unsigned)((g / S) & 1);
        bool ok = mbar_wait_bounded(&bar[s], parity, A.wait_budget);
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        const int64_t row = rb + g * G;
        const int nrow = (int)min((int64_t)G, re - row);
        const unsigned char* st = ring + s * stage_bytes;
        for (int i = 0; i < nrow; ++i) {
            const uint4* rp = reinterpret_cast<const uint4*>(st + i * A.ld_bytes);
            float sdot = 0.0f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                int64_t vec = t + (int64_t)NT * v;
                if (vec < A.nvec) {
                    float p[EPV];
                    Vec<H>::cvt(rp[vec], p);
#pragma unroll
                    for (int e = 0; e < EPV; ++e) sdot = fmaf(p[e], fr[v][e], sdot);
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
            if (lane == 0) red[i][warp] = sdot;
        }
        __syncthreads();
        for (int i = 0; i < nrow; ++i) {
            float y = 0.0f;
            for (int w = 0; w < NW; ++w) y += red[i][w];
            if constexpr (BACK) {
                float inv = y > 0.0f ? 1.0f / y : 0.0f;
                if (A.weight) inv *= A.weight[row + i];  // a binned row counts its photons
                const uint4* rp = reinterpret_cast<const uint4*>(st + i * A.ld_bytes);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    int64_t vec = t + (int64_t)NT * v;
                    if (vec < A.nvec) {
                        float p[EPV];
                        Vec<H>::cvt(rp[vec], p);
#pragma unroll
                        for (int e = 0; e < EPV; ++e) br[v][e] = fmaf(p[e], inv, br[v][e]);
                    }
                }
            } else {
                if (t == (i & (kMaxPassThreads - 1)) && y > 0.0f) {
                    const float c = A.scale ? A.scale[row + i] : 1.0f;
                    const double w = A.weight ? (double)A.weight[row + i] : 1.0;
                    ll += w * (double)logf(c * y);
                    npos += w;
                }
            }
        }
        __syncthreads();  // stage s and red[] are free again
        if (t == 0 && g + S < ngroups) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue(g + S);
        }
    }
    if (aborted) {
        if (t == 0) {
            atomicExch(A.status, 1);
            // copies still in flight target this CTA's shared memory: wait for
            // them (bounded) before the CTA exits
            for (int64_t q = g; q < min(ngroups, g + S); ++q)
                mbar_wait_bounded(&bar[q % S], (unsigned)((q / S) & 1), A.wait_budget * 4 + 4000000000LL);
        }
        __syncthreads();
        return;
    }
    if constexpr (BACK) {
        float* bp = A.bpart + (size_t)blockIdx.x * A.n_sup;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int col0 = EPV * (t + NT * v);
#pragma unroll
            for (int e = 0; e < EPV; ++e)
                if (col0 + e < A.n_sup) bp[col0 + e] = br[v][e];
        }
    } else {
        ll += npos * A.log_T;
        for (int o = 16; o; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
        if (lane == 0) llred[warp] = ll;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += llred[w];
            A.llpart[blockIdx.x] = s;
        }
    }
}

// ---- persistent OS-EM: the sub-iterations of n_iters iterations in one
// cooperative launch.
//
// Every CTA streams its share of each subset's rows through the thread-
// private cp.async ring of k_pass_cpa (same arithmetic per row), writes its
// partial b, and meets the other CTAs at a grid barrier.  CTA c then sums
// the partials of its slice of the support in CTA order (fixed, so the image
// is reproducible) and applies f_q <- f_q b_q / (T s^i_q); a second barrier
// publishes the new image.  The ring is not drained at subset boundaries:
// copies of the next subset's first rows (which do not depend on f) are in
// flight while the CTAs wait at the barriers and reduce.  Both barriers are
// bounded: a wait that runs out sets the status word, and every CTA leaves.
struct CoopArgs {
    const void* model;
    int64_t ld_bytes;
    int64_t nvec;
    const int64_t* sub_row0;  // n_subsets + 1 sorted-row offsets of the subsets
    int n_subsets, n_iters;
    float* f;                 // image, updated in place
    const double* sens;       // [n_subsets][n_sup] subset sensitivities (without T)
    double T;
    const float* weight;      // row counts (binned rows) or nullptr
    int n_sup;
    float* bpart;             // [grid][n_sup] partial back-projections
    unsigned* bar;            // arrivals, completed barriers (zero at launch)
    int* status;
    long long budget;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `target` (1, 2, ...) of the launch.  Returns false when
// this CTA's wait ran out (status set) or another CTA has given up.
__device__ __forceinline__ bool coop_barrier(const CoopArgs& A, unsigned target, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        __threadfence();  // this CTA's partials and image writes before the arrival
        const unsigned arrived = atomicAdd(&A.bar[0], 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&A.bar[0], 0u);
            __threadfence();
            atomicAdd(&A.bar[1], 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_u32(&A.bar[1]) < target) {
                if (*reinterpret_cast<volatile int*>(A.status)) {
                    good = 0;
                    break;
                }
                if (clock64() - t0 > A.budget) {
                    atomicExch(A.status, 1);
                    good = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_ok = good;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <typename H, int VPT>
constexpr int coop_rows() {
    // rows per ring stage, about 12 to 25 KB of row data
    return std::is_same<H, float>::value ? (VPT <= 2 ? 4 : (VPT <= 4 ? 2 : 1)) : (VPT <= 1 ? 4 : (VPT <= 3 ? 2 : 1));
}

template <typename H, int VPT>
constexpr int coop_min_ctas() {
    // two CTAs per SM, except 2-byte rows of 6 or 8 vectors per thread (over
    // 8192 columns), whose image and partial registers need the whole file
    return !std::is_same<H, float>::value && VPT >= 6 ? 1 : 2;
}

template <typename H, int VPT, int R, bool W>
__global__ void __launch_bounds__(kMaxPassThreads, coop_min_ctas<H, VPT>()) k_osem_coop(CoopArgs A, int S) {
    constexpr int EPV = Vec<H>::N;
    extern __shared__ __align__(128) unsigned char cring[];
    __shared__ float red[2][R][kMaxPassThreads / 32];
    __shared__ int s_ok;
    const int NT = blockDim.x, NW = NT >> 5;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int G = gridDim.x, cta = blockIdx.x;
    const char* model = reinterpret_cast<const char*>(A.model);
    const size_t gbytes = (size_t)R * A.ld_bytes;
    const int K = A.n_iters * A.n_subsets;
    if (*reinterpret_cast<volatile int*>(A.status)) return;  // an earlier wait ran out

    // this CTA's rows of sub-iteration k (the subsets split in R-row chunks)
    auto rows_of = [&](int k, int64_t& rb, int64_t& re) {
        const int i = k % A.n_subsets;
        const int64_t r0 = A.sub_row0[i], r1 = A.sub_row0[i + 1];
        int64_t chunk = (r1 - r0 + G - 1) / G;
        chunk = (chunk + R - 1) / R * R;
        rb = min(r1, r0 + (int64_t)cta * chunk);
        re = min(r1, rb + chunk);
    };
    // issue cursor: the next row group to copy, across sub-iterations
    int ki = 0;
    int64_t rbi, rei;
    rows_of(0, rbi, rei);
    int64_t ri = rbi;
    int64_t issued = 0;
    auto issue_next = [&]() {
        while (ki < K && ri >= rei) {
            if (++ki < K) {
                rows_of(ki, rbi, rei);
                ri = rbi;
            }
        }
        if (ki >= K) return;
        unsigned char* dst = cring + (size_t)(issued % S) * gbytes;
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int64_t vec = t + (int64_t)NT * v;
                if (ri + i < rei && vec < A.nvec)
                    cpa16(dst + i * A.ld_bytes + vec * 16, model + (ri + i) * A.ld_bytes + vec * 16);
            }
        }
        cpa_commit();
        ri += R;
        ++issued;
    };
    for (int s = 0; s < S - 1; ++s) issue_next();

    int64_t consumed = 0;
    unsigned barriers = 0;
    const int P = (A.n_sup + G - 1) / G;  // support pixels reduced by each CTA
    const int q0 = min(A.n_sup, cta * P), q1 = min(A.n_sup, q0 + P);
    for (int k = 0; k < K; ++k) {
        const int isub = k % A.n_subsets;
        float fr[VPT][EPV], br[VPT][EPV];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col0 = EPV * (t + NT * v);
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
                const int col = col0 + e;
                fr[v][e] = col < A.n_sup ? __ldcg(A.f + col) : 0.0f;  // written by other CTAs
                br[v][e] = 0.0f;
            }
        }
        int64_t rb, re;
        rows_of(k, rb, re);
        for (int64_t r = rb; r < re; r += R, ++consumed) {
            cpa_wait((int)min((int64_t)7, issued - 1 - consumed));  // this group has landed
            issue_next();  // into the slots of the previous group, read by this thread only
            const unsigned char* st = cring + (size_t)(consumed % S) * gbytes;
            const int rb_ = (int)(consumed & 1);
            uint4 raw[R][VPT];
#pragma unroll
            for (int i = 0; i < R; ++i) {
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int64_t vec = t + (int64_t)NT * v;
                    raw[i][v] = (r + i < re && vec < A.nvec)
                                    ? *reinterpret_cast<const uint4*>(st + i * A.ld_bytes + vec * 16)
                                    : make_uint4(0u, 0u, 0u, 0u);
                }
            }
            float d[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                float2 s2 = make_float2(0.0f, 0.0f);  // even and odd columns
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float p[EPV];
                    Vec<H>::cvt(raw[i][v], p);
#pragma unroll
                    for (int e = 0; e < EPV; e += 2)
                        s2 = ffma2(make_float2(p[e], p[e + 1]), make_float2(fr[v][e], fr[v][e + 1]), s2);
                }
                float sum = s2.x + s2.y;
#pragma unroll
                for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                d[i] = sum;
            }
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < R; ++i) red[rb_][i][warp] = d[i];
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < R; ++i) {
                float y = 0.0f;
                for (int w = 0; w < NW; ++w) y += red[rb_][i][w];
                const bool ok = r + i < re && y > 0.0f;
                float inv = ok ? 1.0f / y : 0.0f;
                if constexpr (W) inv *= ok ? A.weight[r + i] : 0.0f;
                const float2 inv2 = make_float2(inv, inv);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    float p[EPV];
                    Vec<H>::cvt(raw[i][v], p);
#pragma unroll
                    for (int e = 0; e < EPV; e += 2) {
                        const float2 b2 = ffma2(make_float2(p[e], p[e + 1]), inv2,
                                                make_float2(br[v][e], br[v][e + 1]));
                        br[v][e] = b2.x;
                        br[v][e + 1] = b2.y;
                    }
                }
            }
        }
        {
            float* bp = A.bpart + (size_t)cta * A.n_sup;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int col0 = EPV * (t + NT * v);
#pragma unroll
                for (int e = 0; e < EPV; ++e)
                    if (col0 + e < A.n_sup) __stcg(bp + col0 + e, br[v][e]);
            }
        }
        if (!coop_barrier(A, ++barriers, &s_ok)) break;
        // b_q of this CTA's slice: warp w takes the pixels q0 + w, q0 + w + NW,
        // ...; lane l sums the partials l, l + 32, ... in order and the lanes
        // are added in a fixed pattern (deterministic); T s^i_q in FP64
        const double* si = A.sens + (size_t)isub * A.n_sup;
        for (int q = q0 + warp; q < q1; q += NW) {
            float acc = 0.0f;
#pragma unroll 4
            for (int g = lane; g < G; g += 32) acc += __ldcg(A.bpart + (size_t)g * A.n_sup + q);
#pragma unroll
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const double sd = si[q];
                const float ts = (float)(A.T * sd);
                __stcg(A.f + q, sd > 0.0 ? __ldcg(A.f + q) * acc / ts : 0.0f);
            }
        }
        if (!coop_barrier(A, ++barriers, &s_ok)) break;
    }
    cpa_wait(0);  // no copy outlives the CTA (an abandoned launch included)
}

// launch with programmatic stream serialisation (see pdl_wait)
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct PassShape {
    int vpt, nt;
    int64_t nvec;
};

PassShape pass_shape(const lmosem_ctx* c) {
    int epv = c->fmt == LMOSEM_MODEL_FP32 ? 4 : 8;
    int64_t nvec = (c->ld_model + epv - 1) / epv;
    const int opts[] = {1, 2, 3, 4, 6, 8};
    int vpt = 8;
    for (int v : opts)
        if ((nvec + v - 1) / v <= kMaxPassThreads) {
            vpt = v;
            break;
        }
    int nt = (int)(((nvec + vpt - 1) / vpt + 31) / 32 * 32);
    return {vpt, nt, nvec};
}

// register-pipelined pass (pass_variant 0 or 1)
template <typename H, int VPT, bool BACK, bool W>
lmosem_status launch_pass_reg_t(lmosem_ctx* c, PassArgs A, int64_t rows, int nt) {
    constexpr int R = pass_rows<H, VPT>();
    auto kern = k_pass<H, VPT, R, BACK, W>;
    int per_sm = 0, dev = 0, sms = 0;
    LMOSEM_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0));
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = std::max(1, per_sm) * (int64_t)sms;
    grid = std::min<int64_t>(grid, c->pass_ctas);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, (rows + R - 1) / R));
    A.rows_per_cta = (rows + grid - 1) / grid;
    A.rows_per_cta = (A.rows_per_cta + R - 1) / R * R;
    grid = std::max<int64_t>(1, (rows + A.rows_per_cta - 1) / A.rows_per_cta);
    c->pass_grid = (int)grid;
    A.prefetch = auto_prefetch(A.prefetch, R, A.ld_bytes);
    LMOSEM_PROF_BEGIN(c);
    LMOSEM_CK(c, launch_pdl(kern, dim3((unsigned)grid), dim3(nt), 0, c->stream, A));
    LMOSEM_LAUNCHED(c, LMOSEM_K_PASS);
    return LMOSEM_OK;
}

// cp.async ring pass (pass_variant 3): stages of R rows, S stages per CTA
template <typename H, int VPT, bool BACK, bool W>
lmosem_status launch_pass_cpa_t(lmosem_ctx* c, PassArgs A, int64_t rows, int nt) {
    constexpr int R = pass_rows<H, VPT>();
    auto kern = k_pass_cpa<H, VPT, R, BACK, W>;
    const size_t gbytes = (size_t)R * A.ld_bytes;
    // about 104 KB of ring per CTA (two CTAs per SM), 3 to kCpaMaxStages stages
    int S = (int)std::max<int64_t>(3, std::min<int64_t>(kCpaMaxStages, (int64_t)(104 << 10) / (int64_t)gbytes));
    int dev = 0, sms = 0, smem_max = 0;
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    while (S > 2 && (size_t)S * gbytes > (size_t)smem_max) --S;
    if ((size_t)S * gbytes > (size_t)smem_max) return launch_pass_reg_t<H, VPT, BACK, W>(c, A, rows, nt);
    const size_t smem = (size_t)S * gbytes;
    LMOSEM_CK(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LMOSEM_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
    int64_t grid = std::max(1, per_sm) * (int64_t)sms;
    grid = std::min<int64_t>(grid, c->pass_ctas);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, (rows + R - 1) / R));
    A.rows_per_cta = (rows + grid - 1) / grid;
    A.rows_per_cta = (A.rows_per_cta + R - 1) / R * R;
    grid = std::max<int64_t>(1, (rows + A.rows_per_cta - 1) / A.rows_per_cta);
    c->pass_grid = (int)grid;
    LMOSEM_PROF_BEGIN(c);
    LMOSEM_CK(c, launch_pdl(kern, dim3((unsigned)grid), dim3(nt), smem, c->stream, A, S));
    LMOSEM_LAUNCHED(c, LMOSEM_K_PASS);
    return LMOSEM_OK;
}

// bulk-copy ring pass (pass_variant 2)
template <typename H, int VPT, bool BACK, bool W>
lmosem_status launch_pass_t(lmosem_ctx* c, PassArgs A0, int64_t rows, int nt) {
    // automatic: the register pass, with its L2 prefetch for wide rows (at
    // 128x128 FP32 3.41 ms per iteration against 3.64 for the cp.async ring;
    // without the prefetch the ring was the faster of the two)
    if (c->pass_variant == 3) return launch_pass_cpa_t<H, VPT, BACK, W>(c, A0, rows, nt);
    if (c->pass_variant != 2) return launch_pass_reg_t<H, VPT, BACK, W>(c, A0, rows, nt);
    auto kern = k_pass_ring<H, VPT, BACK>;
    // ring shape: stages of G rows (~24 KB), ~96 KB of stages per CTA unless set
    const int64_t rb = A0.ld_bytes;
    int G = (int)std::max<int64_t>(1, std::min<int64_t>(kRingMaxG, (24 << 10) / rb));
    if (c->ring_rows > 0) G = std::min(kRingMaxG, c->ring_rows);
    int S = (int)std::max<int64_t>(2, std::min<int64_t>(kRingMaxStages, (96 << 10) / (G * rb)));
    if (c->ring_stages > 0) S = std::max(2, std::min(kRingMaxStages, c->ring_stages));
    // a caller-chosen shape is cut to the shared memory a CTA may opt into:
    // fewer stages first (at least two), then fewer rows per stage
    int dev0 = 0, smem_max = 0;
    LMOSEM_CK(c, cudaGetDevice(&dev0));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0));
    while ((int64_t)S * G * rb > smem_max && S > 2) --S;
    while ((int64_t)S * G * rb > smem_max && G > 1) --G;
    if ((int64_t)S * G * rb > smem_max)  // two stages of one row do not fit: use the register pass
        return launch_pass_reg_t<H, VPT, BACK, W>(c, A0, rows, nt);
    const size_t smem = (size_t)S * G * rb;
    LMOSEM_CK(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    LMOSEM_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = std::max(1, per_sm) * (int64_t)sms;
    grid = std::min<int64_t>(grid, c->pass_ctas);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, (rows + G - 1) / G));
    RingArgs A;
    A.model = reinterpret_cast<const char*>(A0.model);
    A.ld_bytes = A0.ld_bytes;
    A.nvec = A0.nvec;
    A.r0 = A0.r0;
    A.r1 = A0.r1;
    A.rows_per_cta = (rows + grid - 1) / grid;
    A.rows_per_cta = (A.rows_per_cta + G - 1) / G * G;
    grid = std::max<int64_t>(1, (rows + A.rows_per_cta - 1) / A.rows_per_cta);
    A.G = G;
    A.S = S;
    A.f = A0.f;
    A.scale = A0.scale;
    A.weight = A0.weight;
    A.n_sup = A0.n_sup;
    A.log_T = A0.log_T;
    A.bpart = A0.bpart;
    A.llpart = A0.llpart;
    A.status = c->d_status;
    A.wait_budget = c->wait_budget;
    c->pass_grid = (int)grid;
    LMOSEM_PROF_BEGIN(c);
    kern<<<(unsigned)grid, nt, smem, c->stream>>>(A);
    LMOSEM_LAUNCHED(c, LMOSEM_K_PASS);
    return LMOSEM_OK;
}

template <typename H, bool BACK, bool W = false>
lmosem_status launch_pass_h(lmosem_ctx* c, const PassArgs& A, int64_t rows, PassShape s) {
    switch (s.vpt) {
        case 1: return launch_pass_t<H, 1, BACK, W>(c, A, rows, s.nt);
        case 2: return launch_pass_t<H, 2, BACK, W>(c, A, rows, s.nt);
        case 3: return launch_pass_t<H, 3, BACK, W>(c, A, rows, s.nt);
        case 4: return launch_pass_t<H, 4, BACK, W>(c, A, rows, s.nt);
        case 6: return launch_pass_t<H, 6, BACK, W>(c, A, rows, s.nt);
        default: return launch_pass_t<H, 8, BACK, W>(c, A, rows, s.nt);
    }
}

template <bool BACK>
lmosem_status launch_pass(lmosem_ctx* c, int64_t r0, int64_t r1, const float* f, double T) {
    PassShape s = pass_shape(c);
    int64_t rows = r1 - r0;
    if (rows <= 0) {
        c->pass_grid = 0;   // the reduction then sees b = 0 / an empty sum
        return LMOSEM_OK;
    }
    PassArgs A;
    A.model = c->d_model;
    A.ld_bytes = c->ld_model * (c->fmt == LMOSEM_MODEL_FP32 ? 4 : 2);
    A.nvec = s.nvec;
    A.r0 = r0;
    A.r1 = r1;
    A.rows_per_cta = 0;
    A.f = f;
    A.scale = c->fmt == LMOSEM_MODEL_FP32 ? nullptr : c->d_scale;
    A.weight = c->d_weight;
    A.n_sup = c->n_sup;
    A.log_T = log(T);
    A.bpart = c->d_bpart;
    A.llpart = c->d_llpart;
    A.prefetch = c->prefetch_groups;  // resolved by the register pass's launch
    if (c->d_weight) {  // binned rows: FP32 only
        if (c->fmt != LMOSEM_MODEL_FP32) return fail(c, LMOSEM_ESTATE, "binned rows are FP32");
        return launch_pass_h<float, BACK, true>(c, A, rows, s);
    }
    if (c->fmt == LMOSEM_MODEL_FP32) return launch_pass_h<float, BACK>(c, A, rows, s);
    if (c->fmt == LMOSEM_MODEL_FP16_SCALED) return launch_pass_h<__half, BACK>(c, A, rows, s);
    return launch_pass_h<__nv_bfloat16, BACK>(c, A, rows, s);
}

// the persistent cooperative form of n_iters iterations (one launch)
template <typename H, int VPT, bool W>
lmosem_status launch_coop_t(lmosem_ctx* c, CoopArgs A, int nt) {
    constexpr int R = coop_rows<H, VPT>();
    auto kern = k_osem_coop<H, VPT, R, W>;
    const size_t gbytes = (size_t)R * A.ld_bytes;
    // about 100 KB of ring per CTA (two CTAs per SM), 2 to kCpaMaxStages stages
    int S = (int)std::max<int64_t>(2, std::min<int64_t>(kCpaMaxStages, (int64_t)(100 << 10) / (int64_t)gbytes));
    int dev = 0, sms = 0, smem_max = 0;
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    while (S > 2 && (size_t)S * gbytes > (size_t)smem_max) --S;
    if ((size_t)S * gbytes > (size_t)smem_max) return fail(c, LMOSEM_ENOTIMPL, "rows too wide for the ring");
    const size_t smem = (size_t)S * gbytes;
    LMOSEM_CK(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LMOSEM_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
    if (per_sm < 1) return fail(c, LMOSEM_ENOTIMPL, "the persistent pass does not fit an SM");
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, c->pass_ctas);
    LMOSEM_CK(c, cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), c->stream));
    void* args[] = {&A, &S};
    c->pass_grid = grid;
    LMOSEM_PROF_BEGIN(c);
    LMOSEM_CK(c, cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3((unsigned)nt), args,
                                             smem, c->stream));
    LMOSEM_LAUNCHED(c, LMOSEM_K_PASS);
    return LMOSEM_OK;
}

template <typename H, bool W = false>
lmosem_status launch_coop_h(lmosem_ctx* c, const CoopArgs& A, PassShape s) {
    switch (s.vpt) {
        case 1: return launch_coop_t<H, 1, W>(c, A, s.nt);
        case 2: return launch_coop_t<H, 2, W>(c, A, s.nt);
        case 3: return launch_coop_t<H, 3, W>(c, A, s.nt);
        case 4: return launch_coop_t<H, 4, W>(c, A, s.nt);
        case 6: return launch_coop_t<H, 6, W>(c, A, s.nt);
        default: return launch_coop_t<H, 8, W>(c, A, s.nt);
    }
}

lmosem_status run_coop(lmosem_ctx* c, int n_iters, double T, float* d_f) {
    if (n_iters < 1) return LMOSEM_OK;
    lmosem_status st;
    const size_t words = (size_t)c->n_subsets + 2;  // subset offsets, then the barrier words
    if (c->coop_words < words) {
        if ((st = dev_alloc(c, &c->d_coop, words))) return st;
        c->coop_words = words;
    }
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_coop, c->h_subset_row0.data(), ((size_t)c->n_subsets + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, c->stream));
    PassShape s = pass_shape(c);
    CoopArgs A;
    A.model = c->d_model;
    A.ld_bytes = c->ld_model * (c->fmt == LMOSEM_MODEL_FP32 ? 4 : 2);
    A.nvec = s.nvec;
    A.sub_row0 = c->d_coop;
    A.n_subsets = c->n_subsets;
    A.n_iters = n_iters;
    A.f = d_f;
    A.sens = c->d_sens;
    A.T = T;
    A.weight = c->d_weight;
    A.n_sup = c->n_sup;
    A.bpart = c->d_bpart;
    A.bar = reinterpret_cast<unsigned*>(c->d_coop + c->n_subsets + 1);
    A.status = c->d_status;
    A.budget = c->wait_budget;
    if (c->d_weight) {  // binned rows: FP32 only
        if (c->fmt != LMOSEM_MODEL_FP32) return fail(c, LMOSEM_ESTATE, "binned rows are FP32");
        return launch_coop_h<float, true>(c, A, s);
    }
    if (c->fmt == LMOSEM_MODEL_FP32) return launch_coop_h<float>(c, A, s);
    if (c->fmt == LMOSEM_MODEL_FP16_SCALED) return launch_coop_h<__half>(c, A, s);
    return launch_coop_h<__nv_bfloat16>(c, A, s);
}

lmosem_status ll_final(lmosem_ctx* c, double T, const float* d_f, double* out) {
    LMOSEM_PROF_BEGIN(c);
    k_ll_final<<<1, 256, 0, c->stream>>>(c->d_llpart, c->pass_grid,
                                         c->d_sens + (size_t)c->n_subsets * c->n_sup, d_f,
                                         c->n_sup, T, out);
    LMOSEM_LAUNCHED(c, LMOSEM_K_UPDATE);
    return LMOSEM_OK;
}

}  // namespace

// capacity of the per-CTA partial buffers of the streaming pass
lmosem_status setup_pass(lmosem_ctx* c) {
    int dev = 0, sms = 0;
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    c->pass_ctas = sms * 8;
    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_bpart, (size_t)c->pass_ctas * c->n_sup))) return st;
    if ((st = dev_alloc(c, &c->d_llpart, (size_t)c->pass_ctas))) return st;
    return ensure_status(c);
}

lmosem_status ensure_status(lmosem_ctx* c) {
    if (c->d_status) return LMOSEM_OK;
    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_status, 4))) return st;
    LMOSEM_CK(c, cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), c->stream));
    return LMOSEM_OK;
}

namespace {

// the kernels of one global iteration: N_s passes and updates
lmosem_status enqueue_iteration(lmosem_ctx* c, double T, float* d_f) {
    lmosem_status st;
    for (int i = 0; i < c->n_subsets; ++i) {
        if ((st = launch_pass<true>(c, c->h_subset_row0[i], c->h_subset_row0[i + 1], d_f, T)))
            return st;
        LMOSEM_PROF_BEGIN(c);
        LMOSEM_CK(c, launch_pdl(k_update_px, dim3((c->n_sup + kUpdPix - 1) / kUpdPix), dim3(kUpdPix * kUpdGroups),
                                0, c->stream, (const float*)c->d_bpart, c->pass_grid, c->n_sup, d_f,
                                (const double*)(c->d_sens + (size_t)i * c->n_sup), T, (const int*)c->d_status));
        LMOSEM_LAUNCHED(c, LMOSEM_K_UPDATE);
    }
    return LMOSEM_OK;
}

// One iteration captured as a CUDA graph and replayed (no per-kernel launch
// overhead between the 2 N_s dependent kernels).  Used on a non-default
// stream without profiling; the graph is rebuilt when the image or T change.
lmosem_status iterate_graph(lmosem_ctx* c, int n_iters, double T, float* d_f, bool* done) {
    *done = false;
    if (c->profile == 1 || c->stream == nullptr || n_iters < 1) return LMOSEM_OK;
    if (!c->graph_exec || c->graph_f != d_f || c->graph_T != T) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        const int64_t before = c->launches;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return LMOSEM_OK;  // not capturable: launch directly
        }
        c->capturing = true;
        lmosem_status st = enqueue_iteration(c, T, d_f);
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->graph_exec = nullptr;
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
        c->graph_launches = c->launches - before;
        c->launches = before;
        c->graph_f = d_f;
        c->graph_T = T;
    }
    for (int it = 0; it < n_iters; ++it) {
        LMOSEM_CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
        c->launches += c->graph_launches;
    }
    *done = true;
    return LMOSEM_OK;
}

}  // namespace

lmosem_status run_iterations(lmosem_ctx* c, int n_iters, double T, float* d_f, double* d_ll) {
    lmosem_status st;
    // the persistent form when asked for (pass_variant 4), unless a
    // log-likelihood is taken after every iteration
    if (!d_ll && !c->batch_model && c->pass_variant == 4) return run_coop(c, n_iters, T, d_f);
    if (!d_ll) {
        bool done = false;
        if ((st = iterate_graph(c, n_iters, T, d_f, &done))) return st;
        if (done) return LMOSEM_OK;
    }
    for (int it = 0; it < n_iters; ++it) {
        if ((st = enqueue_iteration(c, T, d_f))) return st;
        if (d_ll) {
            if ((st = launch_pass<false>(c, 0, c->J, d_f, T))) return st;
            if ((st = ll_final(c, T, d_f, d_ll + it))) return st;
        }
    }
    return LMOSEM_OK;
}

lmosem_status run_loglik(lmosem_ctx* c, double T, const float* d_f, double* d_out) {
    lmosem_status st;
    if ((st = launch_pass<false>(c, 0, c->J, d_f, T))) return st;
    return ll_final(c, T, d_f, d_out);
}

lmosem_status run_subset_totals(lmosem_ctx* c, double T, const float* d_f, double* d_out) {
    LMOSEM_PROF_BEGIN(c);
    k_subset_totals<<<c->sens_subsets, 256, 0, c->stream>>>(c->d_sens, c->n_sup, d_f, T, d_out);
    LMOSEM_LAUNCHED(c, LMOSEM_K_UPDATE);
    return LMOSEM_OK;
}

lmosem_status run_init_image(lmosem_ctx* c, double T, float* d_f) {
    LMOSEM_PROF_BEGIN(c);
    k_init_image<<<1, 256, 0, c->stream>>>(c->d_sens + (size_t)c->sens_subsets * c->n_sup,
                                           c->n_sup, c->d_weight ? c->n_counts : (double)c->J, T, d_f);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    return LMOSEM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free sub-iteration (lmosem_osem_subiter_noalloc).
//
// The per-CTA partial back-projections live in one file-scope device array
// instead of a context buffer.  Its host-side name is only a stand-in, so
// the device address is looked up once per device with cudaGetSymbolAddress
// (with that device current) and cached.  Every call shares the array; each
// CTA overwrites its own slot before the reduction reads it, so nothing needs
// clearing, but calls that overlap on the GPU race on it.
namespace {

constexpr int64_t kNoAllocScratchFloats = int64_t(1) << 20;  // 4 MiB
// The register pass holds at most 8 four-float vectors per thread in
// kMaxPassThreads threads, so rows (and the support) are at most 8192 wide;
// the array then still holds 128 per-CTA partials.
constexpr int kNoAllocMaxVpt = 8;
constexpr int64_t kNoAllocMaxLd = int64_t(kMaxPassThreads) * kNoAllocMaxVpt * 4;
constexpr int kNoAllocMaxSupport = (int)kNoAllocMaxLd;
static_assert(kNoAllocScratchFloats / kNoAllocMaxSupport >= 64, "too few partial slots");
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};

template <int VPT>
inline auto noalloc_kernel() {
    return k_pass<float, VPT, VPT >= 6 ? 1 : (VPT >= 3 ? 2 : 4), true, false>;
}

// First call on a device: the array's address, and every kernel this entry
// point can launch loaded now (module loading is lazy by default), so that
// later calls with another row width load nothing.
cudaError_t noalloc_setup() {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    const void* kerns[] = {(const void*)noalloc_kernel<1>(), (const void*)noalloc_kernel<2>(),
                           (const void*)noalloc_kernel<3>(), (const void*)noalloc_kernel<4>(),
                           (const void*)noalloc_kernel<6>(), (const void*)noalloc_kernel<8>(),
                           (const void*)k_update};
    for (const void* k : kerns)
        if ((e = cudaFuncGetAttributes(&fa, k)) != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
    return cudaSuccess;
}

cudaError_t noalloc_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev] && (e = noalloc_setup()) != cudaSuccess) return e;
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

template <int VPT>
cudaError_t noalloc_pass(const PassArgs& A0, int64_t rows, int nt, cudaStream_t s, int* grid_out) {
    constexpr int R = VPT >= 6 ? 1 : (VPT >= 3 ? 2 : 4);
    auto kern = noalloc_kernel<VPT>();
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    PassArgs A = A0;
    int64_t grid = std::max(1, per_sm) * (int64_t)sms;
    grid = std::min<int64_t>(grid, kNoAllocScratchFloats / A.n_sup);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, (rows + R - 1) / R));
    A.rows_per_cta = (rows + grid - 1) / grid;
    A.rows_per_cta = (A.rows_per_cta + R - 1) / R * R;
    grid = std::max<int64_t>(1, (rows + A.rows_per_cta - 1) / A.rows_per_cta);
    kern<<<(unsigned)grid, nt, 0, s>>>(A);
    *grid_out = (int)grid;
    // no error was pending before the call, so one seen here is this launch's
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) (void)cudaGetLastError();
    return e;
}

}  // namespace

lmosem_status run_model_rows(lmosem_ctx* c, const int64_t* ids, int64_t n, float* out) {
    if (n <= 0) return LMOSEM_OK;
    dim3 grid((c->n_sup + 255) / 256, (unsigned)std::min<int64_t>(n, 65535));
    const float* sc = c->fmt == LMOSEM_MODEL_FP32 ? nullptr : c->d_scale;
    LMOSEM_PROF_BEGIN(c);
    if (c->fmt == LMOSEM_MODEL_FP32)
        k_model_rows<float><<<grid, 256, 0, c->stream>>>((const float*)c->d_model, c->ld_model, sc,
                                                         c->d_rank, ids, n, c->n_sup, out);
    else if (c->fmt == LMOSEM_MODEL_FP16_SCALED)
        k_model_rows<__half><<<grid, 256, 0, c->stream>>>((const __half*)c->d_model, c->ld_model, sc,
                                                          c->d_rank, ids, n, c->n_sup, out);
    else
        k_model_rows<__nv_bfloat16><<<grid, 256, 0, c->stream>>>(
            (const __nv_bfloat16*)c->d_model, c->ld_model, sc, c->d_rank, ids, n, c->n_sup, out);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    return LMOSEM_OK;
}

}  // namespace lmosem

extern "C" lmosem_status lmosem_osem_subiter_noalloc(const float* d_rows, int64_t n_rows,
                                                     int32_t n_support, int64_t ld, float* d_f,
                                                     const double* d_sens_i, double acq_time,
                                                     void* stream) {
    using namespace lmosem;
    if (!d_rows || !d_f || !d_sens_i) return LMOSEM_EINVAL;
    if (n_rows < 1 || n_support < 1 || n_support > kNoAllocMaxSupport) return LMOSEM_EINVAL;
    if (ld < n_support || ld > kNoAllocMaxLd || ld % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(d_rows) & 15u) != 0)
        return LMOSEM_EINVAL;
    if (!(acq_time > 0.0) || !isfinite(acq_time)) return LMOSEM_EINVAL;
    // an error left by earlier work stays the caller's to read: run nothing
    if (cudaPeekAtLastError() != cudaSuccess) return LMOSEM_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return LMOSEM_ECUDA;

    // same column-vector shape as the context path (FP32 rows, 4 per vector)
    const int64_t nvec = ld / 4;
    const int opts[] = {1, 2, 3, 4, 6, kNoAllocMaxVpt};
    int vpt = kNoAllocMaxVpt;
    for (int v : opts)
        if ((nvec + v - 1) / v <= kMaxPassThreads) {
            vpt = v;
            break;
        }
    const int nt = (int)(((nvec + vpt - 1) / vpt + 31) / 32 * 32);
    PassArgs A;
    A.model = d_rows;
    A.ld_bytes = ld * 4;
    A.nvec = nvec;
    A.r0 = 0;
    A.r1 = n_rows;
    A.rows_per_cta = 0;
    A.f = d_f;
    A.scale = nullptr;
    A.weight = nullptr;
    A.n_sup = n_support;
    A.log_T = 0.0;
    A.bpart = scratch;
    A.llpart = nullptr;
    A.prefetch = 0;
    int grid = 0;
    cudaError_t e;
    switch (vpt) {
        case 1: e = noalloc_pass<1>(A, n_rows, nt, s, &grid); break;
        case 2: e = noalloc_pass<2>(A, n_rows, nt, s, &grid); break;
        case 3: e = noalloc_pass<3>(A, n_rows, nt, s, &grid); break;
        case 4: e = noalloc_pass<4>(A, n_rows, nt, s, &grid); break;
        case 6: e = noalloc_pass<6>(A, n_rows, nt, s, &grid); break;
        default: e = noalloc_pass<kNoAllocMaxVpt>(A, n_rows, nt, s, &grid); break;
    }
    if (e != cudaSuccess) return LMOSEM_ECUDA;
    k_update<<<(n_support + 31) / 32, 256, 0, s>>>(scratch, grid, n_support, d_f, d_sens_i, acq_time,
                                                   nullptr);
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return LMOSEM_ECUDA;
    }
    return LMOSEM_OK;
}
