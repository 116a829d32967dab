// Scatter-surrogate inference on the 5th-generation tensor cores (tcgen05).
//
// One persistent CTA per SM (4 warps) takes tiles of 128 rows.  For every
// tile the whole network runs on chip: the layer inputs live in shared
// memory (BF16, K-major canonical layout without swizzle), every product
// D[128 x 256] = A[128 x K] W^T is issued by one thread as tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulator in 256 TMEM columns), and the
// four warps read the accumulator back with tcgen05.ld (thread t of warp w
// owns row 32 w + t), add the bias, apply ReLU and write the next layer's
// BF16 input; the last hidden layer's epilogue folds in the 256 -> 1 output
// layer.  The next layer's weights stream into shared memory (cp.async)
// while the current epilogue runs.  MMA completion is signalled through an
// mbarrier (tcgen05.commit); every wait on it is bounded and a timeout sets
// the status word, after which the CTA frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kH = 256, kInPad = 16, kTileM = 128, kThreads = 128;
constexpr long long kDrainCycles = 1LL << 31;   // wait for in-flight products after a timeout
constexpr int64_t kOffB1 = 256 * 6, kOffW2 = kOffB1 + 256, kOffB2 = kOffW2 + 256 * 256;
constexpr int64_t kLayerStride = 256 * 256 + 256;
constexpr int64_t kOffW5 = kOffW2 + 3 * kLayerStride, kOffB5 = kOffW5 + 256;

// canonical K-major layout (no swizzle): 8 x 16-byte core matrices; the k
// groups of a row group are adjacent (LBO = 128 B), row groups follow after
// all k groups (SBO = K / 8 * 128 B)
__host__ __device__ constexpr uint32_t kmajor_offset(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// smem layout of the kernel (bytes)
constexpr uint32_t kSmW1 = 0;                                   // 256 x 16
constexpr uint32_t kSmW = kSmW1 + 256 * kInPad * 2;             // 256 x 256
constexpr uint32_t kSmA = kSmW + 256 * kH * 2;                  // 128 x 256
constexpr uint32_t kSmX = kSmA + kTileM * kH * 2;               // 128 x 16
constexpr uint32_t kSmBias = kSmX + kTileM * kInPad * 2;        // 4 x 256 floats
constexpr uint32_t kSmW5 = kSmBias + 4 * kH * 4;                // 256 floats
constexpr uint32_t kSmBar = kSmW5 + kH * 4;                     // mbarrier (8 B)
constexpr uint32_t kSmTmem = kSmBar + 8;                        // TMEM address (4 B)
constexpr uint32_t kSmBytes = kSmTmem + 8;

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
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!bar_test(bar, parity)) {
        if (clock64() - t0 > budget) return false;
        __nanosleep(32);
    }
    return true;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const __nv_bfloat16* X;    // M x 16 scaled inputs (BF16)
    int64_t M;
    const __nv_bfloat16* w1;   // 256 x 16
    const __nv_bfloat16* w234; // 3 x 256 x 256
    const float* blob;         // biases, output layer
    float* y;                  // M outputs
    int* status;
    long long budget;
};

__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc(TcArgs A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSmBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kSmTmem);
    float* sb = reinterpret_cast<float*>(sm + kSmBias);
    float* sw5 = reinterpret_cast<float*>(sm + kSmW5);
    const uint32_t base = su32(sm);

    // TMEM: 256 FP32 columns x 128 lanes (one accumulator)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(su32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        bar_init(bar);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int i = tid; i < kH; i += kThreads) {
        sb[i] = A.blob[kOffB1 + i];
        for (int l = 0; l < 3; ++l) sb[(l + 1) * kH + i] = A.blob[kOffB2 + l * kLayerStride + i];
        sw5[i] = A.blob[kOffW5 + i];
    }
    // W1 once per CTA: 256 rows x 2 k groups
    for (int c = tid; c < 256 * 2; c += kThreads) {
        const int r = c >> 1, kg = c & 1;
        cp16(base + kSmW1 + kmajor_offset(r, kg * 8, kInPad), A.w1 + r * kInPad + kg * 8, true);
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const float b5 = A.blob[kOffB5];
    const uint32_t idesc = idesc_bf16(kTileM, kH);
    uint32_t phase = 0;
    bool ok = true;

    auto load_w = [&](int l) {  // W_{l+2}: 256 rows x 32 k groups
        const __nv_bfloat16* w = A.w234 + (int64_t)l * kH * kH;
        for (int c = tid; c < 256 * 32; c += kThreads) {
            const int r = c >> 5, kg = c & 31;
            cp16(base + kSmW + kmajor_offset(r, kg * 8, kH), w + r * kH + kg * 8, true);
        }
    };
    auto issue = [&](int layer) {  // thread 0: products of one layer, then commit
        if (layer == 0) {
            mma_bf16_tc(tmem, smem_desc(base + kSmX, 128, kInPad / 8 * 128),
                        smem_desc(base + kSmW1, 128, kInPad / 8 * 128), idesc, 0u);
        } else {
            for (int s = 0; s < kH / 16; ++s)
                mma_bf16_tc(tmem, smem_desc(base + kSmA + s * 256, 128, kH / 8 * 128),
                            smem_desc(base + kSmW + s * 256, 128, kH / 8 * 128), idesc, s > 0 ? 1u : 0u);
        }
        mma_commit(bar);
    };
    const int row = warp * 32 + (tid & 31);                      // this thread's TMEM lane
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);

    const int64_t ntiles = (A.M + kTileM - 1) / kTileM;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int64_t m0 = t * kTileM;
        // inputs: 128 rows x 2 k groups (rows past M read as zeros)
        for (int c = tid; c < kTileM * 2; c += kThreads) {
            const int r = c >> 1, kg = c & 1;
            const bool in = m0 + r < A.M;
            cp16(base + kSmX + kmajor_offset(r, kg * 8, kInPad), A.X + (in ? (m0 + r) * kInPad + kg * 8 : 0), in);
        }
        cp_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            issue(0);
        }
        for (int layer = 0; layer < 4; ++layer) {
            const bool done = bar_wait(bar, phase, A.budget);
            if (__syncthreads_or(!done)) {   // all threads agree; the phase stays pending
                ok = false;
                break;
            }
            phase ^= 1u;
            fence_after();
            if (layer < 3) load_w(layer);   // W buffer is free: the last products finished
            // epilogue: accumulator row -> bias, ReLU -> next input (or output)
            const float* bias = sb + layer * kH;
            float ysum = 0.0f;
            for (int c = 0; c < kH / 32; ++c) {
                float v[32];
                tmem_ld32(trow + c * 32, v);
                if (layer < 3) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int k = c * 32 + q * 8 + 2 * e;
                            __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(v[q * 8 + 2 * e] + bias[k], 0.0f),
                                                                     fmaxf(v[q * 8 + 2 * e + 1] + bias[k + 1], 0.0f));
                            pk[e] = *reinterpret_cast<uint32_t*>(&h);
                        }
                        *reinterpret_cast<uint4*>(sm + kSmA + kmajor_offset(row, c * 32 + q * 8, kH)) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) ysum = fmaf(fmaxf(v[i] + bias[c * 32 + i], 0.0f), sw5[c * 32 + i], ysum);
                }
            }
            if (layer == 3) {
                if (m0 + row < A.M) A.y[m0 + row] = ysum + b5;
                fence_before();
                __syncthreads();  // accumulator read before the next tile overwrites it
                break;
            }
            cp_wait_all();
            fence_async_smem();
            fence_before();
            __syncthreads();
            if (tid == 0) {
                fence_after();
                issue(layer + 1);
            }
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(A.status, 1);
        // the products of the pending phase still write TMEM: let them finish
        // (bounded again) before the columns are freed
        bar_wait(bar, phase, kDrainCycles);
    }
    cp_wait_all();  // no copy may land in shared memory after the CTA has left
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem) : "memory");
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

lmosem_status forward_tc(lmosem_ctx* c, const float* blob, const __nv_bfloat16* w1,
                         const __nv_bfloat16* w234, const __nv_bfloat16* X, float* y, int64_t M) {
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
    A.w234 = w234;
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
