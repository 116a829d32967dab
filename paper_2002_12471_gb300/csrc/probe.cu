// Throughput of the MUFU exponential (ex2.approx.ftz.f32) on this GPU.
//
// The path-sum kernel's terms each cost one ex2 and three FP32 FMAs, and the
// ex2 unit bounds it; its roofline divides by the rate this kernel measures.
// Every thread runs eight independent chains x <- ex2(x) - 1 (one MUFU and one
// FADD per step, the FADD on the FMA pipe), so the MUFU pipe, not latency or
// issue, sets the pace once enough warps are resident.
#include <cuda_runtime.h>

#include "lmosem_internal.cuh"

namespace lmosem {
namespace {

__global__ void k_ex2_rate(int64_t iters, float* sink) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = -0.125f * (float)(k + 1) - 1e-6f * (float)threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = ex2_approx(x[k]) - 1.0f;  // stays in (-1, 0]
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.0f) sink[blockIdx.x] = s;  // keeps the chains live; never taken
}

}  // namespace
}  // namespace lmosem

using namespace lmosem;

extern "C" lmosem_status lmosem_measure_ex2_rate(void* stream, int32_t ctas_per_sm, int32_t threads,
                                                 int64_t iters, double* h_per_second) {
    if (!h_per_second || ctas_per_sm < 1 || ctas_per_sm > 32 || threads < 32 || threads > 1024 ||
        threads % 32 || iters < 1 || iters > (int64_t(1) << 32))
        return LMOSEM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LMOSEM_ECUDA;
    const int grid = sms * ctas_per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (ok) {
        k_ex2_rate<<<grid, threads, 0, s>>>(iters, nullptr);  // warm-up (clocks up, module loaded)
        ok = cudaEventRecord(e0, s) == cudaSuccess;
    }
    if (ok) {
        k_ex2_rate<<<grid, threads, 0, s>>>(iters, nullptr);
        ok = cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!ok || !(ms > 0.0f)) return LMOSEM_ECUDA;
    *h_per_second = (double)grid * threads * 8.0 * (double)iters / (ms * 1e-3);
    return LMOSEM_OK;
}
