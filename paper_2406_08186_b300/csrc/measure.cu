// Measured denominators for rooflines that neither the HBM copy rate nor the
// tensor-core rate describes:
//   hw_measure_fp64  FP64 pipe throughput, for kernels bound by double-precision
//                    arithmetic (the complex128 coin, the complex128 series):
//                    every thread of a grid that fills the device runs
//                    independent chains of fused multiply-adds, enough to hide
//                    the pipe's latency; one operation per FMA (adds and
//                    multiplies take the same pipe slot).
//   hw_measure_l2    copy bandwidth of a working set that stays in L2, for
//                    kernels whose state fits in L2 (the complex64 coin on the
//                    2^20-vertex torus): one launch copies a 16 MB buffer into
//                    another many times over, 16-byte accesses, grid-stride.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double seed, double *sink)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + double(threadIdx.x + c);
    // x <- x * s + t with s just below one keeps every chain finite and away
    // from subnormals; the compiler cannot fold the loop
    const double s = 0.9999999999999998, t = 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], s, t);
    }
    double r = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r += a[c];
    if (r == -1.0) *sink = r;   // never true; keeps the chains live
}

__global__ void __launch_bounds__(512) k_l2_copy(const uint4 *__restrict__ a, uint4 *__restrict__ b, int64_t n, int reps)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = a[i];
}

}  // namespace

extern "C" hw_status hw_measure_l2(double *gbs, void *stream)
{
    hw_clear_error();
    if (!gbs) return hw_fail(HW_EINVAL, "gbs is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != HW_OK) return s;
    if ((s = hw_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count")) != HW_OK) return s;
    if ((s = hw_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_copy, 512, 0), "occupancy")) != HW_OK)
        return s;
    const int64_t n = (int64_t(16) << 20) / 16;   // 16 MB per buffer
    void *buf = nullptr;
    if ((s = hw_cuda(hw_malloc_async(&buf, size_t(2 * n * 16), st), "scratch")) != HW_OK) return s;
    uint4 *a = static_cast<uint4 *>(buf), *b = a + n;
    if ((s = hw_cuda(cudaMemsetAsync(buf, 0, size_t(2 * n * 16), st), "memset")) != HW_OK) {
        cudaFreeAsync(buf, st);
        return s;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sms * per_sm, reps = 200;
    k_l2_copy<<<grid, 512, 0, st>>>(a, b, n, 4);   // warm-up: both buffers into L2
    float best = 1e30f;
    for (int r = 0; r < 3 && s == HW_OK; ++r) {
        cudaEventRecord(e0, st);
        k_l2_copy<<<grid, 512, 0, st>>>(a, b, n, reps);
        cudaEventRecord(e1, st);
        s = hw_cuda(cudaEventSynchronize(e1), "L2 copy kernel");
        float ms = 0.0f;
        if (s == HW_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, st);
    if (s != HW_OK) return s;
    *gbs = 2.0 * double(n) * 16.0 * reps / (double(best) * 1e-3) / 1e9;
    return HW_OK;
}

extern "C" hw_status hw_measure_fp64(double *ops_per_s, void *stream)
{
    hw_clear_error();
    if (!ops_per_s) return hw_fail(HW_EINVAL, "ops_per_s is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != HW_OK) return s;
    if ((s = hw_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count")) != HW_OK) return s;
    if ((s = hw_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate, 256, 0), "occupancy")) != HW_OK)
        return s;
    const int grid = sms * per_sm;
    double *sink = nullptr;
    if ((s = hw_cuda(hw_malloc_async(reinterpret_cast<void **>(&sink), sizeof(double), st), "scratch")) != HW_OK)
        return s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 4096;
    k_fp64_rate<<<grid, 256, 0, st>>>(256, 1.0, sink);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3 && s == HW_OK; ++r) {
        cudaEventRecord(e0, st);
        k_fp64_rate<<<grid, 256, 0, st>>>(iters, 1.0 + r, sink);
        cudaEventRecord(e1, st);
        s = hw_cuda(cudaEventSynchronize(e1), "FP64 rate kernel");
        float ms = 0.0f;
        if (s == HW_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (s != HW_OK) return s;
    *ops_per_s = double(grid) * 256.0 * double(iters) * kChains / (double(best) * 1e-3);
    return HW_OK;
}
