// Batching form (row a10 of the hot path): OS-LM-MLEM for many independent
// list-mode data sets (noise realisations, paper Section 3: the study repeats
// the reconstruction over multiple noise realisations) of one object and
// scanner, all iterations of all realisations in one persistent launch.
//
// Every realisation r walks its own epochs e = t N_s + i (iteration t, subset
// i).  The rows of (r, subset i) are cut into chunks; a CTA claims a chunk of
// any realisation whose current epoch still has unclaimed chunks (one CAS on
// a 64-bit (epoch, next chunk) word), streams the rows (y_j, then b), and
// stores its partial b in the chunk's slot.  The CTA that completes the last
// chunk of (r, e) reduces the slots in chunk order (deterministic), applies
// the update of paper Eq. 7 to f_r and opens epoch e + 1.  A CTA that finds
// nothing to claim waits; the wait is bounded (status word, ETIMEOUT).
// Progress never depends on a waiting CTA: claimed chunks are processed by
// running CTAs without waiting, and the last one updates without waiting.
#include <math.h>

#include <algorithm>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kBatchThreads = 256;

struct BatchArgs {
    const float* model;
    int64_t ld;                    // row stride (floats)
    int64_t nvec;                  // float4 vectors per row holding the support
    int n_sup;
    int n_real, n_subsets, n_epochs;
    const int64_t* sub_row0;       // [r * (n_subsets + 1) + i]
    int chunk_rows;
    int max_chunks;                // partial slots per realisation
    float* f;                      // [r][n_sup]
    const double* sens;            // [i][n_sup]
    double T;
    unsigned long long* claim;     // [r]: epoch << 32 | next chunk
    int* done;                     // [r]: chunks finished in the current epoch
    int* finished;                 // realisations past their last epoch
    float* part;                   // [r][max_chunks][n_sup]
    int* status;                   // 1: a wait ran out
    long long wait_budget;
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int VPT>
__global__ void __launch_bounds__(kBatchThreads) k_batch(BatchArgs A) {
    constexpr int R = VPT >= 3 ? 2 : 4;
    static_assert(kBatchThreads == 256, "eight per-warp partials per row, every slot written");
    __shared__ __align__(16) float red[2][R][kBatchThreads / 32];
    __shared__ int s_r, s_e, s_c, s_last;
    const int NT = blockDim.x;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    int rot = blockIdx.x % A.n_real;
    long long idle_since = -1;

    while (true) {
        // ---- claim a chunk (thread 0)
        if (t == 0) {
            int got_r = -2;
            int n_fin = 0;
            for (int k = 0; k < A.n_real && got_r < 0; ++k) {
                const int r = (rot + k) % A.n_real;
                for (int tries = 0; tries < 64; ++tries) {
                    unsigned long long w = ld_relaxed_u64(A.claim + r);
                    const int e = (int)(w >> 32), c = (int)(w & 0xffffffffu);
                    if (e >= A.n_epochs) {
                        ++n_fin;
                        break;
                    }
                    const int i = e % A.n_subsets;
                    const int64_t rows = A.sub_row0[(size_t)r * (A.n_subsets + 1) + i + 1] -
                                         A.sub_row0[(size_t)r * (A.n_subsets + 1) + i];
                    const int nch = (int)std::max<int64_t>(1, (rows + A.chunk_rows - 1) / A.chunk_rows);
                    if (c >= nch) break;
                    if (atomicCAS(A.claim + r, w, w + 1ull) == w) {
                        got_r = r;
                        s_e = e;
                        s_c = c;
                        break;
                    }
                }
                if (got_r >= 0) rot = (r + 1) % A.n_real;
            }
            if (got_r < 0 && n_fin == A.n_real) got_r = -1;
            if (got_r == -2 && ld_relaxed_s32(A.finished) >= A.n_real) got_r = -1;
            if (got_r >= 0) __threadfence();  // see the image the epoch was opened with
            s_r = got_r;
        }
        __syncthreads();
        const int r = s_r;
        if (r == -1) break;
        if (r == -2) {
            // nothing claimable: wait (bounded) for an epoch to open
            bool give_up = false;
            if (t == 0) {
                long long now = clock64();
                if (idle_since < 0) idle_since = now;
                if (now - idle_since > A.wait_budget || ld_relaxed_s32(A.status) != 0) {
                    atomicExch(A.status, 1);
                    give_up = true;
                }
                __nanosleep(256);
            }
            if (__syncthreads_or(give_up)) break;
            continue;
        }
        idle_since = -1;
        const int e = s_e, ch = s_c, i = e % A.n_subsets;
        const int64_t sr0 = A.sub_row0[(size_t)r * (A.n_subsets + 1) + i];
        const int64_t sr1 = A.sub_row0[(size_t)r * (A.n_subsets + 1) + i + 1];
        const int64_t rb = std::min(sr1, sr0 + (int64_t)ch * A.chunk_rows);
        const int64_t re = std::min(sr1, rb + A.chunk_rows);
        const int nch = (int)std::max<int64_t>(1, (sr1 - sr0 + A.chunk_rows - 1) / A.chunk_rows);
        float* fr_g = A.f + (size_t)r * A.n_sup;

        // ---- stream the chunk's rows: y_j and b (register double-buffered)
        float fr[VPT][4], br[VPT][4];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int col0 = 4 * (t + NT * v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fr[v][q] = col0 + q < A.n_sup ? __ldcg(fr_g + col0 + q) : 0.0f;
                br[v][q] = 0.0f;
            }
        }
        auto load = [&](int64_t row, float4 (&dst)[R][VPT]) {
#pragma unroll
            for (int k = 0; k < R; ++k)
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    int64_t vec = t + (int64_t)NT * v;
                    dst[k][v] = (row + k < re && vec < A.nvec)
                                    ? __ldcs(reinterpret_cast<const float4*>(A.model + (row + k) * A.ld) + vec)
                                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
        };
        auto process = [&](int64_t row, const float4 (&P)[R][VPT], int rbuf) {
            float d[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                float s = 0.0f;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    s = fmaf(P[k][v].x, fr[v][0], s);
                    s = fmaf(P[k][v].y, fr[v][1], s);
                    s = fmaf(P[k][v].z, fr[v][2], s);
                    s = fmaf(P[k][v].w, fr[v][3], s);
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                d[k] = s;
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < R; ++k) red[rbuf][k][warp] = d[k];
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float y = sum8_in_order(red[rbuf][k]);
                const float inv = (row + k < re && y > 0.0f) ? 1.0f / y : 0.0f;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    br[v][0] = fmaf(P[k][v].x, inv, br[v][0]);
                    br[v][1] = fmaf(P[k][v].y, inv, br[v][1]);
                    br[v][2] = fmaf(P[k][v].z, inv, br[v][2]);
                    br[v][3] = fmaf(P[k][v].w, inv, br[v][3]);
                }
            }
        };
        {
            float4 P0[R][VPT], P1[R][VPT];
            if (rb < re) load(rb, P0);
            for (int64_t row = rb; row < re; row += 2 * R) {
                if (row + R < re) load(row + R, P1);
                process(row, P0, 0);
                if (row + R >= re) break;
                if (row + 2 * R < re) load(row + 2 * R, P0);
                process(row + R, P1, 1);
            }
        }
        float* slot = A.part + ((size_t)r * A.max_chunks + ch) * A.n_sup;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            int col0 = 4 * (t + NT * v);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (col0 + q < A.n_sup) __stcg(slot + col0 + q, br[v][q]);
        }
        __threadfence();
        __syncthreads();
        if (t == 0) s_last = atomicAdd(A.done + r, 1) == nch - 1;
        __syncthreads();
        if (s_last) {
            // ---- last chunk of (r, e): reduce the slots in order and update f_r
            __threadfence();
            const double* si = A.sens + (size_t)i * A.n_sup;
            const float* pr = A.part + (size_t)r * A.max_chunks * A.n_sup;
            for (int n = t; n < A.n_sup; n += NT) {
                float b = 0.0f;
                for (int k = 0; k < nch; ++k) b += __ldcg(pr + (size_t)k * A.n_sup + n);
                const double sd = si[n];
                const float ts = (float)(A.T * sd);
                __stcg(fr_g + n, sd > 0.0 ? __ldcg(fr_g + n) * b / ts : 0.0f);
            }
            __threadfence();
            __syncthreads();
            if (t == 0) {
                A.done[r] = 0;
                __threadfence();
                if (e + 1 >= A.n_epochs) atomicAdd(A.finished, 1);
                atomicExch(A.claim + r, (unsigned long long)(e + 1) << 32);
            }
        }
        __syncthreads();
    }
}

__global__ void k_init_batch(const double* __restrict__ s_total, int n_sup, const int64_t* __restrict__ row0,
                             int n_real, double T, float* __restrict__ f) {
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
    const int r = blockIdx.x;
    if (r >= n_real) return;
    const double J = (double)(row0[r + 1] - row0[r]);
    const float v = (float)(J / (T * sh[0]));
    for (int n = threadIdx.x; n < n_sup; n += blockDim.x) f[(size_t)r * n_sup + n] = v;
}

int batch_vpt(const lmosem_ctx* c) {
    int64_t nvec = c->ld_model / 4;
    const int opts[] = {1, 2, 3, 4, 6, 8};
    for (int v : opts)
        if ((nvec + v - 1) / v <= kBatchThreads) return v;
    return 8;
}

template <int VPT>
lmosem_status launch_batch_t(lmosem_ctx* c, const BatchArgs& A, int ctas_per_sm) {
    auto kern = k_batch<VPT>;
    int per_sm = 0, dev = 0, sms = 0;
    LMOSEM_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, 0));
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(per_sm, ctas_per_sm)) * sms;
    LMOSEM_PROF_BEGIN(c);
    kern<<<grid, kBatchThreads, 0, c->stream>>>(A);
    LMOSEM_LAUNCHED(c, LMOSEM_K_PASS);
    return LMOSEM_OK;
}

// enqueue one batched reconstruction: reset the work words, launch
lmosem_status enqueue_batch(lmosem_ctx* c, int n_iters, double T, float* d_f, int chunk_rows,
                            int ctas_per_sm) {
    LMOSEM_CK(c, cudaMemsetAsync(c->d_bclaim, 0, sizeof(unsigned long long) * c->n_real, c->stream));
    LMOSEM_CK(c, cudaMemsetAsync(c->d_bdone, 0, sizeof(int) * (c->n_real + 1), c->stream));
    BatchArgs A;
    A.model = reinterpret_cast<const float*>(c->d_model);
    A.ld = c->ld_model;
    A.nvec = c->ld_model / 4;
    A.n_sup = c->n_sup;
    A.n_real = c->n_real;
    A.n_subsets = c->n_subsets;
    A.n_epochs = n_iters * c->n_subsets;
    A.sub_row0 = c->d_bsub_row0;
    A.chunk_rows = chunk_rows;
    A.max_chunks = (int)((c->batch_max_subset_rows + chunk_rows - 1) / chunk_rows);
    if (A.max_chunks < 1) A.max_chunks = 1;
    A.f = d_f;
    A.sens = c->d_sens;
    A.T = T;
    A.claim = c->d_bclaim;
    A.done = c->d_bdone;
    A.finished = c->d_bdone + c->n_real;
    A.part = c->d_bpart_batch;
    A.status = c->d_status;
    A.wait_budget = c->wait_budget;
    switch (batch_vpt(c)) {
        case 1: return launch_batch_t<1>(c, A, ctas_per_sm);
        case 2: return launch_batch_t<2>(c, A, ctas_per_sm);
        case 3: return launch_batch_t<3>(c, A, ctas_per_sm);
        case 4: return launch_batch_t<4>(c, A, ctas_per_sm);
        case 6: return launch_batch_t<6>(c, A, ctas_per_sm);
        default: return launch_batch_t<8>(c, A, ctas_per_sm);
    }
}

// partial slots for the smallest chunk size any call may use
lmosem_status ensure_batch_buffers(lmosem_ctx* c, int chunk_rows) {
    const int64_t slots = std::max<int64_t>(1, (c->batch_max_subset_rows + chunk_rows - 1) / chunk_rows);
    const int64_t need = (int64_t)c->n_real * slots * c->n_sup;
    lmosem_status st;
    if (need > c->bpart_batch_floats) {
        if ((st = dev_alloc(c, &c->d_bpart_batch, (size_t)need))) return st;
        c->bpart_batch_floats = need;
    }
    return LMOSEM_OK;
}

}  // namespace

lmosem_status setup_batch(lmosem_ctx* c) {
    lmosem_status st;
    c->batch_max_subset_rows = 0;
    for (int r = 0; r < c->n_real; ++r)
        for (int i = 0; i < c->n_subsets; ++i) {
            size_t k = (size_t)r * (c->n_subsets + 1) + i;
            c->batch_max_subset_rows = std::max(c->batch_max_subset_rows,
                                                c->h_subset_row0[k + 1] - c->h_subset_row0[k]);
        }
    if ((st = dev_alloc(c, &c->d_bsub_row0, c->h_subset_row0.size()))) return st;
    if ((st = dev_alloc(c, &c->d_breal_row0, c->h_real_row0.size()))) return st;
    if ((st = dev_alloc(c, &c->d_bclaim, c->n_real))) return st;
    if ((st = dev_alloc(c, &c->d_bdone, c->n_real + 1))) return st;
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_bsub_row0, c->h_subset_row0.data(),
                                 c->h_subset_row0.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 c->stream));
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_breal_row0, c->h_real_row0.data(),
                                 c->h_real_row0.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));  // host vectors outlive the copies
    if (c->batch_chunk_rows <= 0) c->batch_chunk_rows = 512;
    if (c->batch_ctas_per_sm <= 0) c->batch_ctas_per_sm = 2;
    return ensure_batch_buffers(c, c->batch_chunk_rows);
}

lmosem_status run_init_batch(lmosem_ctx* c, double T, float* d_f) {
    LMOSEM_PROF_BEGIN(c);
    k_init_batch<<<c->n_real, 256, 0, c->stream>>>(c->d_sens + (size_t)c->sens_subsets * c->n_sup,
                                                   c->n_sup, c->d_breal_row0, c->n_real, T, d_f);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    return LMOSEM_OK;
}

// One persistent launch for all iterations, captured as a CUDA graph on a
// non-default stream (rebuilt when the image, T, the iteration count or the
// tiles change) and replayed.
lmosem_status run_batch(lmosem_ctx* c, int n_iters, double T, float* d_f) {
    lmosem_status st;
    if ((st = ensure_batch_buffers(c, c->batch_chunk_rows))) return st;
    const bool graphable = c->stream != nullptr && c->profile != 1;
    if (!graphable)
        return enqueue_batch(c, n_iters, T, d_f, c->batch_chunk_rows, c->batch_ctas_per_sm);
    if (!c->bgraph_exec || c->bgraph_f != d_f || c->bgraph_T != T || c->bgraph_iters != n_iters ||
        c->bgraph_chunk != c->batch_chunk_rows || c->bgraph_ctas != c->batch_ctas_per_sm) {
        if (c->bgraph_exec) cudaGraphExecDestroy(c->bgraph_exec);
        c->bgraph_exec = nullptr;
        const int64_t before = c->launches;
        LMOSEM_CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        st = enqueue_batch(c, n_iters, T, d_f, c->batch_chunk_rows, c->batch_ctas_per_sm);
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->bgraph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->bgraph_exec = nullptr;
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
        c->bgraph_launches = c->launches - before;
        c->launches = before;
        c->bgraph_f = d_f;
        c->bgraph_T = T;
        c->bgraph_iters = n_iters;
        c->bgraph_chunk = c->batch_chunk_rows;
        c->bgraph_ctas = c->batch_ctas_per_sm;
    }
    LMOSEM_PROF_BEGIN(c);
    LMOSEM_CK(c, cudaGraphLaunch(c->bgraph_exec, c->stream));
    c->launches += c->bgraph_launches - 1;
    LMOSEM_LAUNCHED(c, LMOSEM_K_PASS);
    return LMOSEM_OK;
}

// Autotuner: time one iteration of every (chunk rows, CTAs per SM)
// candidate on a scratch copy of the images and keep the fastest.
lmosem_status run_autotune_batch(lmosem_ctx* c, double T, const float* d_f, int32_t* h_choice) {
    lmosem_status st;
    const int chunks[] = {128, 256, 512, 1024, 2048};
    const int ctas[] = {1, 2, 3, 4};
    if ((st = ensure_batch_buffers(c, chunks[0]))) return st;
    float* scratch = nullptr;
    Scratch tmp(c);
    const size_t nimg = (size_t)c->n_real * c->n_sup;
    if ((st = tmp.alloc(&scratch, nimg))) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LMOSEM_CK(c, cudaEventCreate(&e0));
    LMOSEM_CK(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_ch = c->batch_chunk_rows, best_ct = c->batch_ctas_per_sm;
    const int saved_profile = c->profile;
    c->profile = 0;
    for (int rep = 0; rep < 2; ++rep) {  // first sweep warms up
        for (int ch : chunks)
            for (int ct : ctas) {
                LMOSEM_CK(c, cudaMemcpyAsync(scratch, d_f, nimg * sizeof(float), cudaMemcpyDeviceToDevice,
                                             c->stream));
                LMOSEM_CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
                LMOSEM_CK(c, cudaEventRecord(e0, c->stream));
                if ((st = enqueue_batch(c, 1, T, scratch, ch, ct))) {
                    c->profile = saved_profile;
                    return st;
                }
                LMOSEM_CK(c, cudaEventRecord(e1, c->stream));
                LMOSEM_CK(c, cudaEventSynchronize(e1));
                float ms = 0.0f;
                LMOSEM_CK(c, cudaEventElapsedTime(&ms, e0, e1));
                if (rep == 1 && ms < best) {
                    best = ms;
                    best_ch = ch;
                    best_ct = ct;
                }
            }
    }
    c->profile = saved_profile;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int h = 0;
    LMOSEM_CK(c, cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, LMOSEM_ETIMEOUT, "a bounded device wait ran out during autotuning");
    c->batch_chunk_rows = best_ch;
    c->batch_ctas_per_sm = best_ct;
    if (h_choice) {
        h_choice[0] = best_ch;
        h_choice[1] = best_ct;
    }
    return LMOSEM_OK;
}

}  // namespace lmosem
