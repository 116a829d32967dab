// Scatter-surrogate inference on the 5th-generation tensor cores (tcgen05).
//
// One persistent CTA per SM runs the whole network on chip for tiles of 128
// rows, two tiles at a time ("ping-pong"): each tile has its own 256-column
// FP32 accumulator in TMEM and its own BF16 activation buffer in shared
// memory, and while the epilogue drains one tile's accumulator the tensor
// core computes the other tile's layer.  Roles, handing work to each other
// through mbarriers only:
//   * producer warp: streams each tile's inputs (4 KB) and the hidden weights
//     (16 KB K chunks, pre-arranged in global memory in the shared-memory
//     operand layout) with cp.async.bulk, the weights through a ring of four
//     chunk slots in the order the products consume them;
//   * MMA warp: one thread issues every product as tcgen05.mma (kind::f16,
//     BF16 operands, FP32 accumulation, M = 128, N = 256), alternating
//     between the two tiles layer by layer;
//   * two epilogue groups of four warps, one per tile of the pair: read the
//     accumulator (warp w: TMEM lanes 32 (w % 4).., all 256 columns), add
//     the bias, apply ReLU, round to BF16 and write the next layer's input
//     in place; the last hidden layer's epilogue folds in the 256 -> 1 output
//     layer.
// Every wait is bounded: a timeout (or another role's abort) sets the status
// word; the CTA then waits (bounded again) for its products and copies in
// flight, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kH = 256, kInPad = 16, kTileM = 128;
constexpr int kGroupWarps = 4, kEpiWarps = 2 * kGroupWarps, kGroupThreads = kGroupWarps * 32;
constexpr int kProdWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1, kThreads = kEpiWarps * 32 + 64;
constexpr int kChunks = 8, kChunkK = 32, kSlots = 4;
constexpr uint32_t kWChunkBytes = kH * kChunkK * 2;       // 16 KB
constexpr uint32_t kAChunkBytes = kTileM * kChunkK * 2;   // 8 KB
constexpr uint32_t kABytes = kChunks * kAChunkBytes;      // 64 KB per tile
constexpr long long kDrainCycles = 1LL << 31;             // waits for in-flight work after an abort
constexpr int kBlobIn = 8;  // network inputs (first-layer columns in the blob)
constexpr int64_t kOffB1 = 256 * kBlobIn, kOffW2 = kOffB1 + 256, kOffB2 = kOffW2 + 256 * 256;
constexpr int64_t kLayerStride = 256 * 256 + 256;
constexpr int64_t kOffW5 = kOffW2 + 3 * kLayerStride, kOffB5 = kOffW5 + 256;
// the blob ends with the 28 baseline coefficients, mu and sigma
static_assert(kOffB5 + 1 + 28 + 2 == LMOSEM_SURROGATE_PARAMS, "parameter blob layout");

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
constexpr uint32_t kXTileBytes = kTileM * kInPad * 2;          // 4 KB
constexpr uint32_t kSmW = 0;                                   // weight ring, 4 x 16 KB
constexpr uint32_t kSmA = kSmW + kSlots * kWChunkBytes;        // 2 x (128 x 256) activations
constexpr uint32_t kSmX = kSmA + 2 * kABytes;                  // 2 input tiles of 128 x 16
constexpr uint32_t kSmW1 = kSmX + 2 * kXTileBytes;             // 256 x 16 first-layer weights
constexpr uint32_t kSmBias = kSmW1 + kH * kInPad * 2;          // 4 x 256 biases
constexpr uint32_t kSmW5 = kSmBias + 4 * kH * 4;               // output weights
// mbarriers: wfull[4] wempty[4] xfull[2] xempty[2] accfull[2] adone[2] drain
constexpr int kBars = 2 * kSlots + 9;
constexpr uint32_t kSmBar = kSmW5 + kH * 4;
constexpr uint32_t kSmTmem = kSmBar + kBars * 8;
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
__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(bar)) : "memory");
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
// OR over the four warps of epilogue group g (named barrier 1 + g)
__device__ __forceinline__ bool group_any(int g, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + g), "n"(kGroupThreads)
        : "memory");
    return r != 0;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane; the
// registers are valid after tmem_wait32 (which takes them as operands, so no
// use can be scheduled before the wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}
// (a0 + b0, a1 + b1) in one packed FP32x2 add
__device__ __forceinline__ uint64_t add2(uint32_t a0, uint32_t a1, float b0, float b1) {
    uint64_t d;
    asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%1, %2};\n\tmov.b64 b, {%3, %4};\n\t"
        "add.rn.f32x2 %0, a, b;\n\t}"
        : "=l"(d)
        : "r"(a0), "r"(a1), "f"(b0), "f"(b1));
    return d;
}
// BF16x2 of ReLU of the two halves (low half = first element)
__device__ __forceinline__ uint32_t relu_bf16x2(uint64_t v) {
    uint32_t d;
    asm("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tcvt.rn.relu.bf16x2.f32 %0, hi, lo;\n\t}"
        : "=r"(d)
        : "l"(v));
    return d;
}

struct TcArgs {
    const unsigned char* X;         // inputs, tile-major: 128-row tiles of 4 KB in the K = 16 operand layout
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
    uint64_t* wempty = wfull + kSlots;
    uint64_t* xfull = wempty + kSlots;
    uint64_t* xempty = xfull + 2;
    uint64_t* accfull = xempty + 2;
    uint64_t* adone = accfull + 2;   // epilogue of group g done with a layer (count 4 warps)
    uint64_t* drain = adone + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kSmTmem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kSmFlag);
    float* sb = reinterpret_cast<float*>(sm + kSmBias);
    float* sw5 = reinterpret_cast<float*>(sm + kSmW5);
    const uint32_t base = su32(sm);

    // TMEM: one accumulator of 256 FP32 columns x 128 lanes per tile of the pair
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(su32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kBars; ++i) bar_init(wfull + i, (adone <= wfull + i && wfull + i < drain) ? kGroupWarps : 1);
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
    // this CTA's tiles j = 0, 1, ... are blockIdx.x + j gridDim.x; tile j belongs to
    // group j % 2 as that group's tile j / 2; pairs p = (2p, 2p + 1)
    const int64_t nj = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t npairs = (nj + 1) / 2;
    auto tile_of = [&](int64_t j) { return (int64_t)blockIdx.x + j * gridDim.x; };

    // producer counters: weight chunks and input tiles issued (for the drain after an abort)
    uint32_t nw = 0, nx0 = 0, nx1 = 0;

    if (warp == kProdWarp) {
        // ---------------- producer: inputs of a pair, then its weight chunks in product order
        if (lane == 0) {
            bool ok = true;
            auto load_x = [&](int g, int64_t p) -> bool {
                if (2 * p + g >= nj) return true;
                uint32_t& n = g ? nx1 : nx0;  // == p
                if (n > 0 && !bar_wait(&xempty[g], (n - 1) & 1u, A.budget, abort_flag)) return false;
                bulk_load(base + kSmX + g * kXTileBytes, A.X + (size_t)tile_of(2 * p + g) * kXTileBytes,
                          kXTileBytes, &xfull[g]);
                ++n;
                return true;
            };
            ok = load_x(0, 0) && load_x(1, 0);
            for (int64_t p = 0; p < npairs && ok; ++p) {
                for (int l = 1; l < 4 && ok; ++l) {
                    for (int g = 0; g < 2 && ok; ++g) {
                        if (2 * p + g >= nj) continue;
                        for (int c = 0; c < kChunks; ++c) {
                            const uint32_t slot = nw % kSlots, u = nw / kSlots;
                            if (u > 0 && !bar_wait(&wempty[slot], (u - 1) & 1u, A.budget, abort_flag)) {
                                ok = false;
                                break;
                            }
                            bulk_load(base + kSmW + slot * kWChunkBytes,
                                      A.w234img + (size_t)(l - 1) * kChunks * kWChunkBytes +
                                          (size_t)c * kWChunkBytes,
                                      kWChunkBytes, &wfull[slot]);
                            ++nw;
                        }
                    }
                    // the pair's first-layer products have read their inputs: fetch the next pair's
                    if (l == 1 && ok) ok = load_x(0, p + 1) && load_x(1, p + 1);
                }
            }
            if (!ok) *abort_flag = 1;
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer: layer by layer, alternating between the pair's tiles
        if (lane == 0) {
            bool ok = true;
            uint32_t n = 0;  // weight chunks consumed
            for (int64_t p = 0; p < npairs && ok; ++p) {
                for (int l = 0; l < 4 && ok; ++l) {
                    for (int g = 0; g < 2 && ok; ++g) {
                        if (2 * p + g >= nj) continue;
                        const uint32_t d = tmem + (uint32_t)g * 256;
                        // the group's epilogue of the previous layer (for l = 0: of the last layer of its
                        // previous tile) has drained this accumulator and, for l >= 1, written the input;
                        // adone[g] completes 4 times per tile
                        if ((p > 0 || l > 0) &&
                            !bar_wait(&adone[g], (uint32_t)(l + 1) & 1u, A.budget, abort_flag)) {
                            ok = false;
                            break;
                        }
                        if (l == 0) {
                            if (!bar_wait(&xfull[g], (uint32_t)p & 1u, A.budget, abort_flag)) {
                                ok = false;
                                break;
                            }
                            fence_after();
                            mma_bf16_tc(d, smem_desc(base + kSmX + g * kXTileBytes, 128, 256),
                                        smem_desc(base + kSmW1, 128, 256), idesc, 0u);
                            mma_commit(&xempty[g]);
                        } else {
                            fence_after();
                            const uint32_t abase = base + kSmA + g * kABytes;
                            for (int c = 0; c < kChunks; ++c) {
                                const uint32_t slot = n % kSlots;
                                if (!bar_wait(&wfull[slot], (n / kSlots) & 1u, A.budget, abort_flag)) {
                                    ok = false;
                                    break;
                                }
                                fence_after();
#pragma unroll
                                for (int s2 = 0; s2 < 2; ++s2)
                                    mma_bf16_tc(d, smem_desc(abase + c * kAChunkBytes + s2 * 256, 128, 512),
                                                smem_desc(base + kSmW + slot * kWChunkBytes + s2 * 256, 128, 512),
                                                idesc, (c | s2) ? 1u : 0u);
                                mma_commit(&wempty[slot]);
                                ++n;
                            }
                            if (!ok) break;
                        }
                        mma_commit(&accfull[g]);
                    }
                }
            }
            if (!ok) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ---------------- epilogue group g = warp / 4: tiles j = g, g + 2, ...
        const int g = warp / kGroupWarps, quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t acc = tmem + (uint32_t)g * 256 + ((uint32_t)(quarter * 32) << 16);
        unsigned char* abuf = sm + kSmA + g * kABytes;
        bool ok = true;
        for (int64_t j = g; j < nj && ok; j += 2) {
            const int64_t m0 = tile_of(j) * kTileM;
            for (int l = 0; l < 4; ++l) {
                // accumulator g completes 4 times per tile: parity l & 1
                const bool done = bar_wait(&accfull[g], (uint32_t)l & 1u, A.budget, abort_flag);
                if (group_any(g, !done)) {
                    ok = false;
                    break;
                }
                fence_after();
                const float* bias = sb + l * kH;
                uint32_t ra[32], rb[32];
                float2 ydot = make_float2(0.0f, 0.0f);
                tmem_ld32(acc, ra);
#pragma unroll
                for (int c = 0; c < kChunks; ++c) {
                    uint32_t(&r)[32] = (c & 1) ? rb : ra;
                    uint32_t(&rn)[32] = (c & 1) ? ra : rb;
                    tmem_wait32(r);
                    if (c + 1 < kChunks) tmem_ld32(acc + (uint32_t)((c + 1) * kChunkK), rn);
                    if (l < 3) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {  // 8 columns: one 16-byte store
                            const float4 b0 = *reinterpret_cast<const float4*>(bias + c * kChunkK + q * 8);
                            const float4 b1 = *reinterpret_cast<const float4*>(bias + c * kChunkK + q * 8 + 4);
                            const uint32_t* v = r + q * 8;
                            *reinterpret_cast<uint4*>(abuf + chunk_offset(row, c * kChunkK + q * 8, kTileM)) =
                                make_uint4(relu_bf16x2(add2(v[0], v[1], b0.x, b0.y)),
                                           relu_bf16x2(add2(v[2], v[3], b0.z, b0.w)),
                                           relu_bf16x2(add2(v[4], v[5], b1.x, b1.y)),
                                           relu_bf16x2(add2(v[6], v[7], b1.z, b1.w)));
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            const float4 bb = *reinterpret_cast<const float4*>(bias + c * kChunkK + q);
                            const float4 ww = *reinterpret_cast<const float4*>(sw5 + c * kChunkK + q);
                            ydot.x = fmaf(fmaxf(__uint_as_float(r[q]) + bb.x, 0.0f), ww.x, ydot.x);
                            ydot.y = fmaf(fmaxf(__uint_as_float(r[q + 1]) + bb.y, 0.0f), ww.y, ydot.y);
                            ydot.x = fmaf(fmaxf(__uint_as_float(r[q + 2]) + bb.z, 0.0f), ww.z, ydot.x);
                            ydot.y = fmaf(fmaxf(__uint_as_float(r[q + 3]) + bb.w, 0.0f), ww.w, ydot.y);
                        }
                    }
                }
                if (l < 3) fence_async_smem();  // the next layer's input, for the tensor core
                fence_before();                 // accumulator reads ordered before its next products
                __syncwarp();
                if (lane == 0) bar_arrive(&adone[g]);
                if (l == 3 && m0 + row < A.M) A.y[m0 + row] = ydot.x + ydot.y + b5;
            }
        }
        if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) {
        if (warp == kMmaWarp && lane == 0) {  // products in flight finish before TMEM is freed
            mma_commit(drain);
            bar_wait(drain, 0u, kDrainCycles, nullptr);
        }
        if (warp == kProdWarp && lane == 0) {  // and the last copy of every slot lands
            for (uint32_t sl = 0; sl < (uint32_t)kSlots; ++sl) {
                const uint32_t u = nw / kSlots + (sl < nw % kSlots ? 1u : 0u);
                if (u > 0) bar_wait(&wfull[sl], (u - 1) & 1u, kDrainCycles, nullptr);
            }
            if (nx0 > 0) bar_wait(&xfull[0], (nx0 - 1) & 1u, kDrainCycles, nullptr);
            if (nx1 > 0) bar_wait(&xfull[1], (nx1 - 1) & 1u, kDrainCycles, nullptr);
        }
        if (tid == 0) atomicExch(A.status, 1);
    }
    fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
    }
}


// ---------------------------------------------------------------- training products
//
// C[M x N] = A[M x K] B[N x K]^T on the tensor cores: BF16 operands with K
// contiguous in global memory, FP32 accumulation in TMEM.  A CTA of four warps
// computes a 128 x BN tile.  K is staged in chunks of 32 by cp.async into the
// canonical K-major layout of the inference kernel (row group g at g * 512 B,
// k group at 128 B), kGemmStages chunk buffers, so copies run three chunks
// ahead of the tensor core; one thread issues the products (tcgen05.mma
// kind::f16, M = 128, N = BN, K = 16, two per chunk) and commits each chunk to
// an mbarrier that frees its buffer.  Epilogue: warp w reads TMEM lanes 32w..
// (its 32 rows of the tile), 32 columns at a time, and applies bias + ReLU,
// the ReLU mask of the layer input, or nothing (FP32).  gridDim.z splits K;
// split z writes its own FP32 slice of C.  Waits are bounded: a timeout sets
// the status word, the CTA drains its products and returns.
constexpr int kGemmRows = 128, kGemmChunk = 32, kGemmStages = 4;

__device__ __forceinline__ void cp_wait_upto(int n) {  // at most n of this thread's newest groups pending
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    }
}

template <int EPI, int BN>
__global__ void __launch_bounds__(128) k_gemm_tc(GemmTcArgs G) {
    constexpr uint32_t kAStage = kGemmRows * kGemmChunk * 2;  // 8 KB
    constexpr uint32_t kBStage = BN * kGemmChunk * 2;
    constexpr uint32_t kStage = kAStage + kBStage;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;             // TMEM columns (a power of two >= 32)
    constexpr int S = kGemmStages;
    extern __shared__ __align__(1024) unsigned char sm[];    // S chunk buffers
    __shared__ __align__(8) uint64_t bars[S + 1];             // chunk buffer free (S), all products done
    __shared__ uint32_t tslot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * kGemmRows;
    const int n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * G.k_per_split;
    const int ke = min(G.K, kb + G.k_per_split);
    const int nk = ke > kb ? (ke - kb + kGemmChunk - 1) / kGemmChunk : 0;
    const uint32_t base = su32(sm);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tslot)),
                     "n"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < S + 1; ++i) bar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tslot;
    const uint32_t idesc = idesc_bf16(kGemmRows, BN);

    auto load_chunk = [&](int c, int buf) {
        const int k0 = kb + c * kGemmChunk;
        const uint32_t a_s = base + (uint32_t)buf * kStage, b_s = a_s + kAStage;
        for (int p = tid; p < kGemmRows * 4; p += 128) {  // 16-byte pieces: row r, k group kg
            const int r = p >> 2, kg = p & 3, k = k0 + kg * 8;
            const bool ok = m0 + r < G.M && k < ke;
            cp16(a_s + (uint32_t)((r >> 3) * 512 + kg * 128 + (r & 7) * 16),
                 G.A + (ok ? (m0 + r) * G.lda + k : 0), ok);
        }
        for (int p = tid; p < BN * 4; p += 128) {
            const int r = p >> 2, kg = p & 3, k = k0 + kg * 8;
            const bool ok = n0 + r < G.N && k < ke;
            cp16(b_s + (uint32_t)((r >> 3) * 512 + kg * 128 + (r & 7) * 16),
                 G.B + (ok ? (int64_t)(n0 + r) * G.ldb + k : 0), ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    bool ok = true;
    int issued = 0;  // chunks whose copies were issued
    for (; issued < min(S - 1, nk); ++issued) load_chunk(issued, issued);
    for (int c = 0; c < nk; ++c) {
        const int buf = c % S;
        if (issued < nk) {
            // chunk `issued` goes to the buffer of chunk c - 1: its products must be done
            if (tid == 0) s_ok = c < 1 || bar_wait(&bars[(c - 1) % S], (uint32_t)((c - 1) / S) & 1u, G.budget, nullptr);
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
            load_chunk(issued, issued % S);
            ++issued;
        }
        cp_wait_upto(issued - c - 1);  // chunk c's copies (this thread's) have landed
        fence_async_smem();            // and are visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t a_s = base + (uint32_t)buf * kStage, b_s = a_s + kAStage;
            const int nmma = min(2, (ke - (kb + c * kGemmChunk) + 15) / 16);
            for (int s2 = 0; s2 < nmma; ++s2)
                mma_bf16_tc(tmem, smem_desc(a_s + s2 * 256, 128, 512), smem_desc(b_s + s2 * 256, 128, 512), idesc,
                            (c | s2) ? 1u : 0u);
            mma_commit(&bars[buf]);
        }
    }
    if (!ok) asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // no copy outlives the CTA
    if (tid == 0) {
        mma_commit(&bars[S]);  // every product issued so far
        s_ok = bar_wait(&bars[S], 0u, ok ? G.budget : kDrainCycles, nullptr) && ok;
        if (!s_ok) atomicExch(G.status, 1);
    }
    __syncthreads();
    fence_after();
    if (s_ok) {  // (an empty K split still writes its slice: zeros)
        const int row = warp * 32 + lane;
        const int64_t gr = m0 + row;
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            if (nk > 0) {
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
                tmem_wait32(r);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = 0u;
            }
            if (gr >= G.M) continue;
            const int col0 = n0 + c0;
            const int nv = min(32, G.N - col0);
            if constexpr (EPI == 0) {
                float* out = reinterpret_cast<float*>(G.C) + (int64_t)blockIdx.z * G.split_stride + gr * G.ldc + col0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nv) out[j] = __uint_as_float(r[j]);
            } else {
                __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(G.C) + gr * G.ldc + col0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (j >= nv) continue;
                    float v = __uint_as_float(r[j]);
                    if constexpr (EPI == 1) {
                        v = fmaxf(v + G.bias[col0 + j], 0.0f);
                    } else {
                        v = __bfloat162float(G.mask[gr * G.ldm + col0 + j]) > 0.0f ? v : 0.0f;
                    }
                    out[j] = __float2bfloat16_rn(v);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kCols) : "memory");
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
    return fail(c, LMOSEM_ETIMEOUT, "a bounded device wait ran out");
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
    // X: tile-major inputs (x_tile_index), rows padded to a multiple of 128
    lmosem_status st;
    if ((st = ensure_status(c))) return st;
    int dev = 0, sms = 0;
    LMOSEM_CK(c, cudaGetDevice(&dev));
    LMOSEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmBytes));
    TcArgs A;
    A.X = reinterpret_cast<const unsigned char*>(X);
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

// the products' shared-memory opt-in, once per context and before any
// stream capture (it is not a stream operation)
lmosem_status gemm_tc_setup(lmosem_ctx* c) {
    if (c->gemm_attrs) return LMOSEM_OK;
    const int s128 = kGemmStages * (kGemmRows + 128) * kGemmChunk * 2;
    const int s256 = kGemmStages * (kGemmRows + 256) * kGemmChunk * 2;
    LMOSEM_CK(c, cudaFuncSetAttribute(k_gemm_tc<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, s128));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_gemm_tc<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, s128));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_gemm_tc<2, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, s128));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_gemm_tc<0, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, s256));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_gemm_tc<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, s256));
    LMOSEM_CK(c, cudaFuncSetAttribute(k_gemm_tc<2, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, s256));
    c->gemm_attrs = true;
    return LMOSEM_OK;
}

lmosem_status gemm_tc(lmosem_ctx* c, int epi, const GemmTcArgs& G0, int splits) {
    lmosem_status st;
    if ((st = ensure_status(c))) return st;
    GemmTcArgs G = G0;
    G.status = c->d_status;
    G.budget = c->wait_budget;
    splits = std::max(1, splits);
    G.k_per_split = (G.K + splits - 1) / splits;
    G.k_per_split = (G.k_per_split + 15) / 16 * 16;
    const int bn = G.N <= 16 ? 16 : (G.N <= 128 ? 128 : 256);
    // 128-column tiles when the 128-row tiles alone leave SMs idle
    const int64_t mt = (G.M + kGemmRows - 1) / kGemmRows;
    const int bnu = (bn == 256 && mt < 152) ? 128 : bn;
    dim3 grid((unsigned)mt, (unsigned)((G.N + bnu - 1) / bnu), (unsigned)splits);
    const int smem = kGemmStages * (kGemmRows + bnu) * kGemmChunk * 2;  // the chunk buffers of A and B
    if (!c->gemm_attrs) return fail(c, LMOSEM_ESTATE, "gemm_tc_setup was not called");
    LMOSEM_PROF_BEGIN(c);
#define LMOSEM_GEMM_TC(E, BNV) k_gemm_tc<E, BNV><<<grid, 128, smem, c->stream>>>(G)
    if (bnu == 16) {
        if (epi == 0) LMOSEM_GEMM_TC(0, 16); else if (epi == 1) LMOSEM_GEMM_TC(1, 16); else LMOSEM_GEMM_TC(2, 16);
    } else if (bnu == 128) {
        if (epi == 0) LMOSEM_GEMM_TC(0, 128); else if (epi == 1) LMOSEM_GEMM_TC(1, 128); else LMOSEM_GEMM_TC(2, 128);
    } else {
        if (epi == 0) LMOSEM_GEMM_TC(0, 256); else if (epi == 1) LMOSEM_GEMM_TC(1, 256); else LMOSEM_GEMM_TC(2, 256);
    }
#undef LMOSEM_GEMM_TC
    LMOSEM_LAUNCHED(c, LMOSEM_K_MLP);
    return LMOSEM_OK;
}


}  // namespace lmosem
