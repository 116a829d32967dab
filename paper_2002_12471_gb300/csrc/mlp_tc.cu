// Scatter-surrogate inference on the 5th-generation tensor cores (tcgen05).
//
// One persistent CTA per SM takes tiles of 128 rows and runs the whole
// network on chip.  Roles:
//   * eight epilogue warps: read a layer's FP32 accumulator from TMEM
//     (tcgen05.ld; warp w reads lanes 32 (w % 4).. and columns of half w / 4),
//     add the bias, apply ReLU and write the next layer's BF16 input into
//     shared memory, 32 columns (one K chunk) at a time; the last hidden
//     layer's epilogue folds in the 256 -> 1 output layer;
//   * thread 0 (also an epilogue thread) issues the products: as soon as a
//     K chunk of the next layer's input is written and the matching chunk of
//     its weights has landed, the two K = 16 steps of that chunk go to the
//     tensor core as tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation,
//     M = 128, N = 256);
//   * one producer warp streams the weight chunks (16 KB each, pre-arranged
//     in global memory in the shared-memory operand layout) with
//     cp.async.bulk into eight slots guarded by full / empty mbarriers.
// Two 256-column accumulators alternate between layers, so the products of
// layer l + 1 run while the epilogue of layer l drains its accumulator, and
// the first layer of the next tile starts while the last epilogue of the
// current tile runs.  Every wait is bounded: a timeout (or the abort of
// another role) sets the status word; the CTA then waits (bounded again) for
// its products and copies in flight, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kH = 256, kInPad = 16, kTileM = 128;
constexpr int kEpiWarps = 8, kEpiThreads = kEpiWarps * 32, kThreads = kEpiThreads + 32;
constexpr int kChunks = 8, kChunkK = 32;
constexpr uint32_t kWChunkBytes = kH * kChunkK * 2;       // 16 KB
constexpr uint32_t kAChunkBytes = kTileM * kChunkK * 2;   // 8 KB
constexpr long long kDrainCycles = 1LL << 31;             // waits for in-flight work after an abort
constexpr int64_t kOffB1 = 256 * 6, kOffW2 = kOffB1 + 256, kOffB2 = kOffW2 + 256 * 256;
constexpr int64_t kLayerStride = 256 * 256 + 256;
constexpr int64_t kOffW5 = kOffW2 + 3 * kLayerStride, kOffB5 = kOffW5 + 256;

// Operand layouts (canonical K-major, no swizzle; core matrix = 8 rows x 16 B):
//  * K = 16 operands (inputs, first-layer weights): row group g of 8 rows at
//    g * 256 B, its two k groups 128 B apart (LBO 128, SBO 256);
//  * K = 256 operands (hidden activations, hidden weights) in 32-column
//    chunks: chunk c at c * R * 64 B, row group g at g * 512 B inside it, its
//    four k groups 128 B apart (LBO 128, SBO 512).  A chunk is contiguous, so
//    a weight chunk is one bulk copy.
__host__ __device__ constexpr uint32_t k16_offset(int r, int k) {
    return (uint32_t)((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__host__ __device__ constexpr uint32_t chunk_offset(int r, int k, int R) {
    return (uint32_t)((k >> 5) * (R * kChunkK * 2) + (r >> 3) * 512 + ((k & 31) >> 3) * 128 + (r & 7) * 16 +
                      (k & 7) * 2);
}

// shared memory (bytes)
constexpr uint32_t kSmW = 0;                                   // 8 weight chunks, 128 KB
constexpr uint32_t kSmA = kSmW + kChunks * kWChunkBytes;       // 128 x 256 activations, 64 KB
constexpr uint32_t kSmX = kSmA + kChunks * kAChunkBytes;       // 128 x 16 inputs
constexpr uint32_t kSmW1 = kSmX + kTileM * kInPad * 2;         // 256 x 16 first-layer weights
constexpr uint32_t kSmBias = kSmW1 + kH * kInPad * 2;          // 4 x 256 biases
constexpr uint32_t kSmW5 = kSmBias + 4 * kH * 4;               // output weights
constexpr uint32_t kSmYp = kSmW5 + kH * 4;                     // output partials of column half 1
constexpr uint32_t kSmBar = kSmYp + kTileM * 4;                // wfull[8] wempty[8] acc[2] drain
constexpr uint32_t kSmTmem = kSmBar + 19 * 8;
constexpr uint32_t kSmFlag = kSmTmem + 4;
constexpr uint32_t kSmBytes = kSmFlag + 12;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of sm_100 class devices; no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; gives up when the budget
// runs out or (if abort_flag) another role has aborted
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long budget,
                                         const volatile int* abort_flag) {
    if (bar_test(bar, parity)) return true;
    const long long t0 = clock64();
    for (int i = 0;; ++i) {
        if (bar_test(bar, parity)) return true;
        if ((abort_flag && *abort_flag) || clock64() - t0 > budget) return false;
        if (i > 32) __nanosleep(32);
    }
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// barrier 1 over the eight epilogue warps
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(kEpiThreads) : "memory"); }
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
        : "memory");
    return r != 0;
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const __nv_bfloat16* X;         // M x 16 scaled inputs (BF16)
    int64_t M;
    const __nv_bfloat16* w1;        // 256 x 16, row-major
    const unsigned char* w234img;   // 3 x 8 chunks x 16 KB: hidden weights in the operand layout
    const float* blob;              // biases, output layer
    float* y;                       // M outputs
    int* status;
    long long budget;
};

__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc(TcArgs A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* wfull = reinterpret_cast<uint64_t*>(sm + kSmBar);
    uint64_t* wempty = wfull + kChunks;
    uint64_t* accbar = wfull + 2 * kChunks;
    uint64_t* drain = accbar + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kSmTmem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kSmFlag);
    float* sb = reinterpret_cast<float*>(sm + kSmBias);
    float* sw5 = reinterpret_cast<float*>(sm + kSmW5);
    float* yp = reinterpret_cast<float*>(sm + kSmYp);
    const uint32_t base = su32(sm);

    // TMEM: two accumulators of 256 FP32 columns x 128 lanes
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(su32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2 * kChunks + 3; ++i) bar_init(wfull + i);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int i = tid; i < kH; i += kThreads) {
        sb[i] = A.blob[kOffB1 + i];
        for (int l = 0; l < 3; ++l) sb[(l + 1) * kH + i] = A.blob[kOffB2 + l * kLayerStride + i];
        sw5[i] = A.blob[kOffW5 + i];
    }
    for (int c = tid; c < kH * 2; c += kThreads)  // first-layer weights: 256 rows x 2 k groups
        cp16(base + kSmW1 + k16_offset(c >> 1, (c & 1) * 8), A.w1 + (c >> 1) * kInPad + (c & 1) * 8, true);
    cp_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const float b5 = A.blob[kOffB5];
    const uint32_t idesc = idesc_bf16(kTileM, kH);
    const int64_t ntiles = (A.M + kTileM - 1) / kTileM;

    uint32_t issued[kChunks];  // producer: copies issued per weight slot
#pragma unroll
    for (int c = 0; c < kChunks; ++c) issued[c] = 0;
    if (warp == kEpiWarps) {
        // ---------------- producer: hidden weight chunks, 3 layers per tile
        if (lane == 0) {
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
                for (int l = 0; l < 3 && ok; ++l)
                    for (int c = 0; c < kChunks; ++c) {
                        // the slot's previous chunk must have been consumed by its products
                        if (issued[c] > 0 && !bar_wait(&wempty[c], (issued[c] - 1) & 1u, A.budget, abort_flag)) {
                            ok = false;
                            break;
                        }
                        bulk_load(base + kSmW + c * kWChunkBytes,
                                  A.w234img + (size_t)l * kChunks * kWChunkBytes + (size_t)c * kWChunkBytes,
                                  kWChunkBytes, &wfull[c]);
                        ++issued[c];
                    }
            if (!ok) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps (thread 0 also issues the products)
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const bool issuer = tid == 0;
        uint32_t use = 0;  // weight-slot uses consumed (3 per tile)
        bool ok = true;

        auto load_x = [&](int64_t t) {  // 128 rows x 2 k groups, rows past M read as zeros
            const int64_t m0 = t * kTileM;
            const int r = tid >> 1, kg = tid & 1;
            const bool in = m0 + r < A.M;
            cp16(base + kSmX + k16_offset(r, kg * 8), A.X + (in ? (m0 + r) * kInPad + kg * 8 : 0), in);
        };
        auto issue_first = [&]() {  // layer 1 (K = 16) into accumulator 0
            fence_after();
            mma_bf16_tc(tmem, smem_desc(base + kSmX, 128, 256), smem_desc(base + kSmW1, 128, 256), idesc, 0u);
            mma_commit(&accbar[0]);
        };

        int64_t t = blockIdx.x;
        if (t < ntiles) {
            load_x(t);
            cp_wait_all();
            fence_async_smem();
            epi_sync();
            if (issuer) issue_first();
        }
        for (; t < ntiles && ok; t += gridDim.x) {
            const int64_t m0 = t * kTileM;
            const int64_t tn = t + gridDim.x;
            for (int l = 0; l < 4; ++l) {
                // layer l's accumulator is complete (layers alternate between the two)
                const bool done = bar_wait(&accbar[l & 1], (uint32_t)(l >> 1) & 1u, A.budget, abort_flag);
                if (epi_any(!done)) {
                    ok = false;
                    break;
                }
                fence_after();
                if (l == 1 && tn < ntiles) load_x(tn);  // the first layer's products have read X
                if (l == 3 && tn < ntiles) {            // next tile's first layer overlaps this epilogue
                    cp_wait_all();
                    fence_async_smem();
                    fence_before();
                    epi_sync();
                    if (issuer) issue_first();
                }
                const uint32_t acc = tmem + (uint32_t)(l & 1) * 256 + lane_off;
                const uint32_t nxt = tmem + (uint32_t)((l + 1) & 1) * 256;
                const float* bias = sb + l * kH;
                float ysum = 0.0f;
                for (int c = 0; c < kChunks; ++c) {
                    const int k0 = c * kChunkK + half * 16;
                    float v[16];
                    tmem_ld16(acc + (uint32_t)k0, v);
                    float b[16];
#pragma unroll
                    for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(b + j) =
                                                        *reinterpret_cast<const float4*>(bias + k0 + j);
                    if (l < 3) {
                        uint32_t pk[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(fmaxf(v[2 * e] + b[2 * e], 0.0f),
                                                                      fmaxf(v[2 * e + 1] + b[2 * e + 1], 0.0f));
                            pk[e] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        unsigned char* dst = sm + kSmA + chunk_offset(row, k0, kTileM);
                        *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *reinterpret_cast<uint4*>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        fence_async_smem();
                        fence_before();
                        epi_sync();  // chunk c of the next layer's input is written
                        if (issuer) {
                            if (!bar_wait(&wfull[c], use & 1u, A.budget, abort_flag)) {
                                *abort_flag = 1;
                            } else {
                                fence_after();
#pragma unroll
                                for (int s = 0; s < 2; ++s)
                                    mma_bf16_tc(nxt,
                                                smem_desc(base + kSmA + c * kAChunkBytes + s * 256, 128, 512),
                                                smem_desc(base + kSmW + c * kWChunkBytes + s * 256, 128, 512),
                                                idesc, (c | s) ? 1u : 0u);
                                mma_commit(&wempty[c]);
                                if (c == kChunks - 1) mma_commit(&accbar[(l + 1) & 1]);
                            }
                        }
                        __syncwarp();
                    } else {
                        float wv[16];
#pragma unroll
                        for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(wv + j) =
                                                            *reinterpret_cast<const float4*>(sw5 + k0 + j);
#pragma unroll
                        for (int j = 0; j < 16; ++j) ysum = fmaf(fmaxf(v[j] + b[j], 0.0f), wv[j], ysum);
                    }
                }
                if (l < 3) {
                    ++use;
                } else {
                    if (half == 1) yp[row] = ysum;
                    fence_before();
                    epi_sync();
                    if (half == 0 && m0 + row < A.M) A.y[m0 + row] = ysum + yp[row] + b5;
                }
            }
        }
        if (!ok) *abort_flag = 1;
        cp_wait_all();  // no input copy lands after the CTA has left
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {  // products in flight finish before TMEM is freed
            atomicExch(A.status, 1);
            mma_commit(drain);
            bar_wait(drain, 0u, kDrainCycles, nullptr);
        }
        if (warp == kEpiWarps && lane == 0)  // and the last weight copy of every slot lands
            for (int c = 0; c < kChunks; ++c)
                if (issued[c] > 0) bar_wait(&wfull[c], (issued[c] - 1) & 1u, kDrainCycles, nullptr);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
    }
}

}  // namespace

static_assert(kSmBytes <= 227 * 1024, "shared memory of the fused kernel");

lmosem_status take_status(lmosem_ctx* c) {
    if (!c->d_status) return LMOSEM_OK;
    int h = 0;
    LMOSEM_CK(c, cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (!h) return LMOSEM_OK;
    LMOSEM_CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    return fail(c, LMOSEM_ETIMEOUT, "a bounded device wait of the surrogate inference ran out");
}

// hidden weights (3 x 256 x 256, row-major [layer][out][in]) to the chunked
// operand layout the kernel copies from
__global__ void k_weights_img(const __nv_bfloat16* __restrict__ w234, unsigned char* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * kH * kH) return;
    const int l = i / (kH * kH), o = (i / kH) % kH, k = i % kH;
    *reinterpret_cast<__nv_bfloat16*>(img + (size_t)l * kChunks * kWChunkBytes + chunk_offset(o, k, kH)) = w234[i];
}

lmosem_status weights_img(lmosem_ctx* c, const __nv_bfloat16* w234, unsigned char* img) {
    LMOSEM_PROF_BEGIN(c);
    k_weights_img<<<(3 * kH * kH + 255) / 256, 256, 0, c->stream>>>(w234, img);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SURROGATE);
    return LMOSEM_OK;
}

lmosem_status forward_tc(lmosem_ctx* c, const float* blob, const __nv_bfloat16* w1,
                         const unsigned char* w234img, const __nv_bfloat16* X, float* y, int64_t M) {
    lmosem_status st;
    if ((st = ensure_status(c))) return st;
    int dev = 0, sms = 0;
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmBytes));
    TcArgs A;
    A.X = X;
    A.M = M;
    A.w1 = w1;
    A.w234img = w234img;
    A.blob = blob;
    A.y = y;
    A.status = c->d_status;
    A.budget = c->wait_budget;
    const int64_t ntiles = (M + kTileM - 1) / kTileM;
    const int grid = (int)std::min<int64_t>(ntiles, sms);
    LMOSEM_PROF_BEGIN(c);
    k_mlp_tc<<<grid, kThreads, kSmBytes, c->stream>>>(A);
    LMOSEM_LAUNCHED(c, LMOSEM_K_MLP);
    return LMOSEM_OK;
}

}  // namespace lmosem
