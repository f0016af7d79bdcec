// Measured denominators for rooflines that neither the HBM copy rate nor the
// tensor-core rate describes:
//   hw_measure_fp64  FP64 pipe throughput, for kernels bound by double-precision
//                    arithmetic (the complex128 coin, the complex128 series):
//                    a grid that fills the device runs the inner loop of a
//                    register-blocked GEMM on shared-memory tiles; one
//                    operation per FMA (adds and multiplies take the same pipe
//                    slot).
//   hw_measure_l2    copy bandwidth of a working set that stays in L2, for
//                    kernels whose state fits in L2 (the complex64 coin on the
//                    2^20-vertex torus): one launch copies a 16 MB buffer into
//                    another many times over, 16-byte accesses, grid-stride.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

// The operands of the FMAs come from shared memory into a 4 x 4 register
// tile, as in a register-blocked GEMM: measured on B300, chains of FMAs on
// register-resident operands alone top out about 15% lower than this
// pattern, which reaches the rate a double-precision GEMM sustains.
__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double seed, double *sink)
{
    __shared__ double As[16][65];
    __shared__ double Bs[16][64];
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    for (int e = t; e < 16 * 64; e += 256) {
        As[e / 64][e % 64] = seed + 1e-3 * e;
        Bs[e / 64][e % 64] = 1.0 - 1e-9 * e;
    }
    __syncthreads();
    double acc[4][4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) r += acc[i][j];
    if (r == -1.0) *sink = r;   // never true; keeps the FMAs live
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
    const int iters = 512;   // x 16 x 16 FMAs per thread
    k_fp64_rate<<<grid, 256, 0, st>>>(32, 1.0, sink);   // warm-up
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
    *ops_per_s = double(grid) * 256.0 * double(iters) * 256.0 / (double(best) * 1e-3);
    return HW_OK;
}
