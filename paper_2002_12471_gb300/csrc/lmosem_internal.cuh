// Internal declarations of the lmosem CUDA library (sm_103a only).
//
// Method: list-mode OS-LM-MLEM with attenuation and first-order in-plane
// scatter compensation (Rahman, Laforest, Jha, ISBI 2020, Sections 2.1-2.2).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lmosem.h"

namespace lmosem {

constexpr double kMec2Kev = 510.99895;
constexpr double kPi = 3.14159265358979323846;
constexpr float kLog2e = 1.4426950408889634f;
constexpr int kComptonNodes = 16385;  // nodes of the cos(psi) table on [-1, 1]

// Path-sum tile: TJ events x TN support pixels per CTA, MC scatter pixels
// staged per step, 256 threads each holding 8 events x 4 pixels.
constexpr int kTJ = 64;
constexpr int kTN = 128;
constexpr int kMC = 32;
constexpr int kBuildThreads = 256;

}  // namespace lmosem

struct lmosem_ctx {
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;

    // problem statement
    int nx = 0, ny = 0, npix = 0;
    double dpx = 0;
    int n_angles = 0, n_bins = 0;
    double angle0 = 0, bin_mm = 0, radius = 0, fwhm0 = 0, fwhm_slope = 0;
    double e0 = 0, fwhm_frac = 0, e_lo = 0, e_hi = 0;
    float k_sigma = 6.0f;
    float e_sigma = 6.0f;         // energy cut of the scatter terms (sigmas); <= 0: none
    int64_t table_budget = int64_t(4) << 30;

    int n_sup = 0, n_scat = 0, ld_w = 0;  // ld_w: support padded to kTN
    std::vector<int32_t> h_sup, h_scat;
    double kbar = 0;      // circle mean of the Klein-Nishina shape at E0
    double de0 = 0;       // energy-window mass of the photopeak

    // device: problem and attenuation tables
    float* d_mu = nullptr;        // npix
    int32_t* d_sup = nullptr;     // n_sup
    int32_t* d_scat = nullptr;    // n_scat
    float4* d_scat_geo = nullptr; // n_scat: (x_m, y_m, mu_m, pixel index as int bits)
    float2* d_trig = nullptr;     // n_angles: (cos, sin) theta_a
    float* d_l_edge = nullptr;    // n_angles x npix: mu(E0) integral pixel centre -> edge
    float* d_l_pair = nullptr;    // n_scat x n_sup: integral scatter centre <-> support centre
    float2* d_compton = nullptr;  // kComptonNodes: (sigma_KN(E')/sigma_KN(E0), window mass at E')
    float4* d_mpar = nullptr;     // n_angles x n_scat: (u_m, q_m, lq_m, cut_m)
    float4* d_ppar = nullptr;     // n_angles x ld_w:  (u_n, q_n, lp_n, D_u(n))
    float* d_du_m = nullptr;      // n_angles x n_scat: detector-extent mass D_u at m

    // sensitivity
    int sens_subsets = 0;
    double* d_sens = nullptr;     // sens_subsets x n_sup
    double* d_sens_angle = nullptr;  // n_angles x n_sup (per-angle partials)

    // model
    int fmt = -1;
    int64_t J = 0;
    int n_subsets = 0;
    int64_t ld_model = 0;         // row stride in elements
    void* d_model = nullptr;
    float* d_scale = nullptr;     // J row scales (scaled forms)
    float* d_stage = nullptr;     // FP32 staging rows for the scaled forms
    int64_t stage_rows = 0;
    int32_t* d_perm = nullptr;    // sorted row -> caller's event index
    int64_t* d_rank = nullptr;    // caller's event index -> sorted row
    float* d_u_s = nullptr;       // sorted positions
    float* d_e_s = nullptr;       // sorted energies
    int32_t* d_a_s = nullptr;     // sorted angles
    int n_real = 1;                                  // independent realisations in the model
    std::vector<int64_t> h_real_row0;                // n_real + 1
    std::vector<int64_t> h_angle_row0, h_angle_cnt;  // [r * n_angles + a] (sorted rows)
    std::vector<int64_t> h_subset_row0;              // [r * (n_subsets + 1) + i]
    int32_t* d_angle_row0 = nullptr;
    int32_t* d_angle_cnt = nullptr;
    int32_t* d_tile_prefix = nullptr;                // n_angles + 1 cumulative event tiles
    std::vector<int32_t> h_tile_prefix;
    // binned rows (the paper's binning experiment): per-row photon counts
    float* d_weight = nullptr;    // J counts (nullptr for list-mode events)
    double n_counts = 0.0;        // sum of the counts
    float* d_wtab = nullptr;      // scatter-weight planes (s, b, -lw) of one angle group
    float* d_wtab_all = nullptr;  // planes of every angle, indexed by angle: built with the
                                  // sensitivity when they fit the table budget, consumed (and
                                  // freed) by the next model build
    int64_t wtab_bytes = 0;

    // iteration scratch
    int pass_ctas = 0;            // capacity of the per-CTA partial buffers
    int pass_grid = 0;            // CTAs of the last pass (partials to reduce)
    float* d_bpart = nullptr;     // pass_ctas x n_sup
    double* d_llpart = nullptr;   // pass_ctas
    double* d_scalar = nullptr;   // small FP64 scratch
    unsigned long long* d_terms = nullptr;  // path terms of the last model build (path-sum kernels)
    bool terms_valid = false;
    int* d_status = nullptr;      // [0] = 1 after a bounded device wait ran out
    long long wait_budget = 2000000000LL;  // clock cycles per bounded wait
    int pass_variant = 0;         // 0 auto, 1 register pipeline, 2 bulk-copy ring, 3 cp.async ring,
                                  // 4 persistent cooperative launch (the automatic choice)
    int64_t* d_coop = nullptr;    // persistent form: subset offsets and two barrier words
    size_t coop_words = 0;
    // scatter surrogate
    float* d_surrogate = nullptr;             // LMOSEM_SURROGATE_PARAMS FP32 parameters
    float* d_line = nullptr;                  // surrogate inputs: [a][iu][is] mu(E0) integrated along the
                                              // detector line u_i from depth s_k to the detector
    int line_nu = 0, line_ns = 0;
    double line_u0 = 0, line_s0 = 0, line_h = 0;
    bool scatter_only = false;                // model build leaves the primary path out
    bool use_surrogate = false;               // model build takes the scatter part from the MLP
    int surrogate_kernel = 0;                 // inference: 0 auto (fused tcgen05), 1 product chain, 2 fused
    int prefetch_groups = 0;                  // register pass: groups prefetched into L2 ahead (-1 none, 0 auto)
    bool gemm_attrs = false;                  // shared-memory opt-in of the training products is set
    // exact check of a surrogate build: rows recomputed by the path sum
    double sur_tol = 1e-2;                    // rel-L2 above which the model is rebuilt exactly (0: never)
    int sur_check_rows = 512;                 // sampled rows
    bool sur_checked = false;                 // a surrogate build has been checked
    double sur_err = 0.0, sur_row_max = 0.0;  // rel-L2 of the sampled rows; largest per-row rel-L2
    bool sur_exact = false;                   // the check rebuilt the model with the exact path sum
    double sur_gate_tol = 0.0;                // energy gate: per-bin mean row error above which the
                                              // bin's rows (and every lower one) are exact (0: off)
    double sur_gate_bin = 5.0;                // energy bin width of the gate, keV
    double sur_cut = 0.0;                     // rows with E below this energy hold exact rows
    double sur_frac_exact = 0.0;              // fraction of the model's rows that are exact
    // batching form: per-realisation work words, partial slots, tiles, graph
    bool batch_model = false;
    int64_t* d_bsub_row0 = nullptr;           // n_real * (n_subsets + 1)
    int64_t* d_breal_row0 = nullptr;          // n_real + 1
    unsigned long long* d_bclaim = nullptr;   // n_real
    int* d_bdone = nullptr;                   // n_real + 1 (last: finished count)
    float* d_bpart_batch = nullptr;
    int64_t bpart_batch_floats = 0;
    int64_t batch_max_subset_rows = 0;
    int batch_chunk_rows = 0, batch_ctas_per_sm = 0;
    cudaGraphExec_t bgraph_exec = nullptr;
    const float* bgraph_f = nullptr;
    double bgraph_T = 0.0;
    int bgraph_iters = 0, bgraph_chunk = 0, bgraph_ctas = 0;
    int64_t bgraph_launches = 0;
    // one OSEM iteration captured as a CUDA graph (non-default streams)
    cudaGraphExec_t graph_exec = nullptr;
    const float* graph_f = nullptr;
    double graph_T = 0.0;
    int64_t graph_launches = 0;
    int ring_rows = 0, ring_stages = 0;  // ring shape (0: from the row size)

    // kernel timing (opts->profile)
    int profile = 0;              // 0 off, 1 every launch, 2 all but graph-replayed iterations
    bool capturing = false;       // a CUDA graph is being captured on the stream
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> prof_pool;
    cudaEvent_t prof_open = nullptr;
};

namespace lmosem {

lmosem_status fail(lmosem_ctx* c, lmosem_status st, const std::string& msg);
lmosem_status cuda_fail(lmosem_ctx* c, cudaError_t e, const char* what);

#define LMOSEM_CK(ctx, call)                                           \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::lmosem::cuda_fail(ctx, e_, #call); \
    } while (0)

// Every kernel launch is followed by LMOSEM_LAUNCHED(ctx, class); with
// profiling on, LMOSEM_PROF_BEGIN(ctx) precedes it.
void prof_begin(lmosem_ctx* c);
void prof_end(lmosem_ctx* c, int cls);

#define LMOSEM_PROF_BEGIN(ctx)                       \
    do {                                             \
        if ((ctx)->profile) ::lmosem::prof_begin(ctx); \
    } while (0)

#define LMOSEM_STR2(x) #x
#define LMOSEM_STR(x) LMOSEM_STR2(x)
#define LMOSEM_LAUNCHED(ctx, cls)                                              \
    do {                                                                       \
        (ctx)->launches++;                                                     \
        if ((ctx)->profile) ::lmosem::prof_end(ctx, cls);                      \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess)                                                 \
            return ::lmosem::cuda_fail(ctx, e_, "launch at " __FILE__ ":" LMOSEM_STR(__LINE__)); \
    } while (0)

// Device memory of a context is stream-ordered on the context's stream
// (cudaMallocAsync / cudaFreeAsync from the device's default pool, which keeps
// up to kPoolKeepBytes cached between calls): a buffer may be freed right
// after the launches that use it, and repeated builds reuse the pool's memory
// instead of paying a device-wide synchronising allocation each time.
constexpr uint64_t kPoolKeepBytes = uint64_t(16) << 30;

template <typename T>
lmosem_status dev_alloc(lmosem_ctx* c, T** p, size_t count) {
    if (*p) {
        cudaFreeAsync(*p, c->stream);
        *p = nullptr;
    }
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, LMOSEM_ENOMEM, "allocation of " + std::to_string(count * sizeof(T)) +
                                          " bytes failed: " + cudaGetErrorString(e));
    }
    return LMOSEM_OK;
}

template <typename T>
void dev_free(lmosem_ctx* c, T** p) {
    if (*p) cudaFreeAsync(*p, c->stream);
    *p = nullptr;
}

// Device buffers local to one call: allocated through the guard, freed
// (stream-ordered) when the guard goes out of scope, on every return path.
// Declare the guard after the pointers it owns.
class Scratch {
public:
    explicit Scratch(lmosem_ctx* c) : c_(c) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    ~Scratch() {
        for (void* p : owned_)
            if (p) cudaFreeAsync(p, c_->stream);
    }
    // the allocation itself is recorded, not the caller's pointer variable,
    // which may go out of scope before the Scratch does
    template <typename T>
    lmosem_status alloc(T** p, size_t count) {
        void* old = reinterpret_cast<void*>(*p);  // dev_alloc frees it
        for (void*& q : owned_)
            if (old && q == old) q = nullptr;
        lmosem_status st = dev_alloc(c_, p, count);
        if (st == LMOSEM_OK) owned_.push_back(reinterpret_cast<void*>(*p));
        return st;
    }

private:
    lmosem_ctx* c_;
    std::vector<void*> owned_;
};

// The sum v[0] + v[1] + ... + v[7], added in index order from 0, read with
// two 16-byte shared-memory loads (v: the per-warp partials of one row, 16-
// byte aligned; the slots of absent warps hold +0, and adding +0 leaves a
// sum's bits unchanged except that -0 becomes +0)
__device__ __forceinline__ float sum8_in_order(const float* v) {
    const float4 a = *reinterpret_cast<const float4*>(v);
    const float4 b = *reinterpret_cast<const float4*>(v + 4);
    float y = 0.0f;
    y += a.x;
    y += a.y;
    y += a.z;
    y += a.w;
    y += b.x;
    y += b.y;
    y += b.z;
    y += b.w;
    return y;
}

// ---- host entry points implemented in the other translation units
lmosem_status build_tables(lmosem_ctx* c);                      // siddon.cu
// h_offsets: n_real + 1 event offsets of the realisations (nullptr: one)
// EINVAL unless every event's angle, position and energy are in range (synchronises)
lmosem_status validate_events(lmosem_ctx* c, const int32_t* d_angle, const float* d_u, const float* d_e,
                              int64_t n);
// support.cu: the binned-OSEM support initialiser
lmosem_status run_binned_support(lmosem_ctx* c, const int32_t* d_angle, const float* d_u, int64_t n,
                                 int n_subsets, int n_iters, double threshold, int dilate,
                                 uint8_t* h_support, float* d_image);
lmosem_status sort_events(lmosem_ctx* c, const int32_t* d_angle, const float* d_u,
                          const float* d_e, int64_t n, int n_subsets,
                          const int64_t* h_offsets, int n_real);  // sort.cu
lmosem_status build_model_rows(lmosem_ctx* c);
// binned rows: model of every (angle, position bin, energy bin) row of the
// row map ([a][b][k] -> sorted row or -1) with energy bin edges e_edges
lmosem_status build_binned_rows(lmosem_ctx* c, const int32_t* d_rowmap, int n_ebins,
                                const double* e_edges);                  // model.cu
lmosem_status compute_sensitivity(lmosem_ctx* c, int n_subsets);  // sens.cu
// model.cu: every angle's scatter-weight planes into d_wtab_all and, in the
// same pass, the per-angle sensitivities (arithmetic of the sensitivity
// kernel: FP32 terms, FP64 every 32 terms); false from wtab_all_fits when
// the planes of all angles exceed the table budget
bool wtab_all_fits(const lmosem_ctx* c);
lmosem_status wtab_all_with_sens(lmosem_ctx* c, double* sens_angle, float w_const_sens, float de0);
lmosem_status run_iterations(lmosem_ctx* c, int n_iters, double T, float* d_f, double* d_ll);
lmosem_status run_loglik(lmosem_ctx* c, double T, const float* d_f, double* d_out);
lmosem_status run_init_image(lmosem_ctx* c, double T, float* d_f);
lmosem_status run_subset_totals(lmosem_ctx* c, double T, const float* d_f, double* d_out);
lmosem_status run_model_rows(lmosem_ctx* c, const int64_t* ids, int64_t n, float* out);
lmosem_status setup_pass(lmosem_ctx* c);
// the device status word (bounded waits that ran out), allocated once and zeroed
lmosem_status ensure_status(lmosem_ctx* c);
// ETIMEOUT (and the word cleared) if a bounded wait ran out since the last check
lmosem_status take_status(lmosem_ctx* c);                        // osem.cu
lmosem_status setup_batch(lmosem_ctx* c);                       // batch.cu
lmosem_status run_init_batch(lmosem_ctx* c, double T, float* d_f);
lmosem_status run_batch(lmosem_ctx* c, int n_iters, double T, float* d_f);
lmosem_status run_autotune_batch(lmosem_ctx* c, double T, const float* d_f, int32_t* h_choice);
// mlp.cu
lmosem_status run_surrogate_grad(lmosem_ctx* c, const float* blob, const float* feat, const float* targ,
                                 int64_t n, float* grad_out, double* h_loss);
lmosem_status run_surrogate_train(lmosem_ctx* c, const float* feat, const float* targ, const float* rel,
                                  int64_t n, int steps, int B, float lr, uint64_t seed, float floor_below,
                                  bool residual_fit, float magnitude_power, float* blob, double* h_loss_curve);
lmosem_status run_surrogate_infer(lmosem_ctx* c, const float* blob, const float* feat, int64_t n,
                                  float* out);
lmosem_status run_surrogate_samples(lmosem_ctx* c, float* feat, float* targ, float* rel);
lmosem_status build_model_surrogate(lmosem_ctx* c);
// model.cu: exact rows of an evenly spaced sample of the model's events
// against the rows the surrogate built (relative L2 over the sampled rows,
// and the largest per-row value); synchronises
lmosem_status judge_surrogate(lmosem_ctx* c, double* rel_err, double* row_max, std::vector<double>* row_sums,
                              std::vector<float>* row_e);
lmosem_status rebuild_rows_below(lmosem_ctx* c, double e_cut, int64_t* n_rebuilt);
std::vector<int64_t> judge_sample_rows(const lmosem_ctx* c);
lmosem_status build_surrogate_rows_above(lmosem_ctx* c, double e_cut, int64_t* n_built);
lmosem_status build_model_surrogate_rows(lmosem_ctx* c, const int64_t* d_rows, int64_t n);
// mlp_tc.cu: fused tcgen05 inference of M rows of BF16 inputs (M x 16)
lmosem_status forward_tc(lmosem_ctx* c, const float* blob, const __nv_bfloat16* w1,
                         const unsigned char* w234img, const __nv_bfloat16* X, float* y, int64_t M);
// mlp_tc.cu: C = A B^T on the tensor cores (tcgen05, BF16 operands with K
// contiguous, FP32 accumulation); epi 0: FP32 C (split z of K at
// C + z split_stride), 1: bias + ReLU to BF16, 2: ReLU mask of `mask` to BF16.
// K a multiple of 16, lda/ldb/ldc multiples of 8 elements.
struct GemmTcArgs {
    const __nv_bfloat16* A;
    int64_t lda;
    const __nv_bfloat16* B;
    int64_t ldb;
    void* C;
    int64_t ldc;
    int64_t split_stride;
    const float* bias;
    const __nv_bfloat16* mask;
    int64_t ldm;
    int64_t M;
    int N, K, k_per_split;
    int* status;
    long long budget;
};
lmosem_status gemm_tc(lmosem_ctx* c, int epi, const GemmTcArgs& G, int splits);
lmosem_status gemm_tc_setup(lmosem_ctx* c);  // once per context, before any stream capture
// hidden weights to the chunked operand layout of forward_tc (3 x 128 KB)
lmosem_status weights_img(lmosem_ctx* c, const __nv_bfloat16* w234, unsigned char* img);

// ---- device helpers shared by the CUDA translation units

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Pixel centres: the offset (i + 1/2 - n/2) is exact in FP32 and the scale
// is one rounded product (never fused into a later add), which the host
// reproduces for the scatter-pixel table.
__device__ __forceinline__ float pixel_x(int pix, int nx, float dpx) {
    return __fmul_rn((float)(pix % nx) + 0.5f - 0.5f * (float)nx, dpx);
}
__device__ __forceinline__ float pixel_y(int pix, int nx, int ny, float dpx) {
    return __fmul_rn((float)(pix / nx) + 0.5f - 0.5f * (float)ny, dpx);
}

// Linear interpolation of the cos(psi) table.
__device__ __forceinline__ float2 compton_lookup(const float2* tab, float c) {
    float x = (c + 1.0f) * (0.5f * (float)(kComptonNodes - 1));
    x = fminf(fmaxf(x, 0.0f), (float)(kComptonNodes - 1));
    int i = min((int)x, kComptonNodes - 2);
    float fr = x - (float)i;
    float2 a = __ldg(tab + i), b = __ldg(tab + i + 1);
    return make_float2(fmaf(fr, b.x - a.x, a.x), fmaf(fr, b.y - a.y, a.y));
}

// Geometry of one scatter path (n -> m at angle a) from the two pixel
// centres: cos of the deflection angle and 1/|p_m - p_n|.  Returns false
// when m == n.  Every mul-add is written out, so each kernel that forms a
// path gets the same bits whatever the compiler would have fused.
__device__ __forceinline__ bool path_geometry_xy(float xn, float yn, float xm, float ym, bool same,
                                                 float2 trig, float* cpsi, float* rinv) {
    if (same) return false;
    float vx = xm - xn;
    float vy = ym - yn;
    float ri = rsqrtf(fmaf(vx, vx, vy * vy));
    float c = fmaf(vx, trig.x, vy * trig.y) * ri;  // one contraction, fixed in the source
    *cpsi = fminf(fmaxf(c, -1.0f), 1.0f);
    *rinv = ri;
    return true;
}

// Compton kinematics at the photopeak: P = E'/E0 and the in-plane
// Klein-Nishina weight K(psi)/Kbar.
__device__ __forceinline__ void compton(float cpsi, float eps0, float inv_kbar, float* P, float* kt) {
    float inv_p = fmaf(eps0, 1.0f - cpsi, 1.0f);
    float p = __fdividef(1.0f, inv_p);  // inv_p in [1, 1 + 2 E0 / mc^2]
    float sin2 = fmaf(-cpsi, cpsi, 1.0f);
    *P = p;
    *kt = 0.5f * p * p * (p + inv_p - sin2) * inv_kbar;
}

}  // namespace lmosem
