// Per-vertex probabilities and norms, accumulated in double precision.
//   coined (Sec. 3.2):  p_v = sum_{w in N(v)} |<v,w|psi>|^2
//   CTQW   (Sec. 3.1):  p_v = |<v|psi>|^2
// norm_b = sum over rows of |psi[row][b]|^2 by a fixed two-level reduction
// (per-CTA partials in scratch, then one pass over the partials), so that the
// result does not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace {

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

// coined: thread per (vertex, column), sequential over the vertex's arcs
template <typename R>
__global__ void k_prob_coined(const int32_t *__restrict__ row_ptr, int64_t n, int batch,
                              const void *psi_, double *__restrict__ prob)
{
    using V = typename Cx<R>::T;
    const V *__restrict__ psi = static_cast<const V *>(psi_);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * batch) return;
    int64_t rb;
    const int64_t v = (batch == 1) ? i : idx_div(i, batch, rb);
    const int b = (batch == 1) ? 0 : int(rb);
    double acc = 0.0;
    for (int a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
        const V p = psi[int64_t(a) * batch + b];
        acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
    }
    prob[i] = acc;
}

// CTQW: elementwise
template <typename R>
__global__ void k_prob_vertex(int64_t total, const void *psi_, double *__restrict__ prob)
{
    using V = typename Cx<R>::T;
    const V *__restrict__ psi = static_cast<const V *>(psi_);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const V p = psi[i];
        prob[i] = double(p.x) * double(p.x) + double(p.y) * double(p.y);
    }
}

constexpr int kNormThreads = 256;

// partial[blk*batch + b] = sum over rows [blk*chunk, (blk+1)*chunk) of |psi[row][b]|^2.
// Threads are laid out as (row lane r, column b) with batch <= 256 columns
// per pass; the per-column reduction over r runs in a fixed order.
template <typename R>
__global__ void __launch_bounds__(kNormThreads)
k_norm_partial(const void *psi_, int64_t rows, int batch, int64_t chunk, double *__restrict__ partial)
{
    using V = typename Cx<R>::T;
    __shared__ double red[kNormThreads];
    const V *__restrict__ psi = static_cast<const V *>(psi_);
    const int64_t r0 = int64_t(blockIdx.x) * chunk;
    const int64_t r1 = min(r0 + chunk, rows);
    for (int c0 = 0; c0 < batch; c0 += kNormThreads) {
        const int cols = min(kNormThreads, batch - c0);
        const int lanes = kNormThreads / cols;            // rows processed side by side
        const int t = threadIdx.x;
        const int r = t / cols, b = c0 + t % cols;
        double acc = 0.0;
        if (r < lanes) {
#pragma unroll 4
            for (int64_t row = r0 + r; row < r1; row += lanes) {
                const V p = psi[row * batch + b];
                acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
            }
        }
        red[t] = (r < lanes) ? acc : 0.0;
        __syncthreads();
        if (t < cols) {
            double s = 0.0;
            for (int k = 0; k < lanes; ++k) s += red[k * cols + t];
            partial[int64_t(blockIdx.x) * batch + c0 + t] = s;
        }
        __syncthreads();
    }
}

// one CTA per column: strided partial sums, then a fixed tree
__global__ void __launch_bounds__(kNormThreads)
k_norm_final(const double *__restrict__ partial, int nparts, int batch, double *__restrict__ norm)
{
    __shared__ double red[kNormThreads];
    const int b = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += kNormThreads) s += partial[int64_t(k) * batch + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kNormThreads / 2; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) norm[b] = red[0];
}

}  // namespace

// Partial count used by the norm reduction for `rows` rows.
static int norm_parts(int64_t rows)
{
    return int(std::max<int64_t>(1, std::min<int64_t>(1184, (rows + 4095) / 4096)));
}

hw_status launch_norm(hw_dtype dt, int batch, const void *psi, int64_t rows, double *partial,
                      double *norm, cudaStream_t st)
{
    const int parts = norm_parts(rows);
    const int64_t chunk = (rows + parts - 1) / parts;
    if (dt == HW_C128) k_norm_partial<double><<<parts, kNormThreads, 0, st>>>(psi, rows, batch, chunk, partial);
    else k_norm_partial<float><<<parts, kNormThreads, 0, st>>>(psi, rows, batch, chunk, partial);
    hw_status s = hw_cuda(cudaGetLastError(), "k_norm_partial launch");
    if (s != HW_OK) return s;
    k_norm_final<<<batch, kNormThreads, 0, st>>>(partial, parts, batch, norm);
    return hw_cuda(cudaGetLastError(), "k_norm_final launch");
}

size_t norm_scratch_bytes(int64_t rows, int batch)
{
    return sizeof(double) * size_t(norm_parts(rows)) * size_t(batch);
}

hw_status launch_probability(const hw_graph *g, int64_t n, hw_dtype dt, int batch, const void *psi,
                             double *prob, double *norm, cudaStream_t st)
{
    hw_status s = HW_OK;
    if (prob) {
        if (g) {
            const int64_t total = g->n * batch;
            const int64_t grid = std::max<int64_t>(1, (total + 255) / 256);
            if (dt == HW_C128) k_prob_coined<double><<<grid, 256, 0, st>>>(g->d_row_ptr, g->n, batch, psi, prob);
            else k_prob_coined<float><<<grid, 256, 0, st>>>(g->d_row_ptr, g->n, batch, psi, prob);
        } else {
            const int64_t total = n * batch;
            const int64_t grid = std::min<int64_t>(148 * 16, std::max<int64_t>(1, (total + 255) / 256));
            if (dt == HW_C128) k_prob_vertex<double><<<grid, 256, 0, st>>>(total, psi, prob);
            else k_prob_vertex<float><<<grid, 256, 0, st>>>(total, psi, prob);
        }
        if ((s = hw_cuda(cudaGetLastError(), "probability launch")) != HW_OK) return s;
    }
    if (norm) {
        const int64_t rows = g ? g->num_arcs : n;
        if (rows == 0) return hw_cuda(cudaMemsetAsync(norm, 0, sizeof(double) * batch, st), "memset norm");
        void *partial = nullptr;
        if ((s = hw_cuda(hw_malloc_async(&partial, norm_scratch_bytes(rows, batch), st),
                         "scratch allocation (norm partials)")) != HW_OK)
            return s;
        s = launch_norm(dt, batch, psi, rows, static_cast<double *>(partial), norm, st);
        cudaFreeAsync(partial, st);
    }
    return s;
}

// ---------------------------------------------------------------- search analysis
// The success probability of a search at sampled times (the paper's search
// use of simulate(range=...) and probability_distribution, Sec. 3, and the
// success probability / optimal running time of Sec. 5):
//   curve[r][b] = sum_{m in M} prob[r][m][b]   (marked ids ascending)
// and, per column b, the first sample r at which the curve is largest.
namespace {

__global__ void k_success_curve(const double *__restrict__ prob, int64_t R, int64_t n, int batch,
                                MarkedList mk, double *__restrict__ curve)
{
    const int64_t total = R * batch;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        int64_t b = 0;
        const int64_t r = (batch == 1) ? i : idx_div(i, batch, b);
        const double *row = prob + r * n * batch + b;
        double s = 0.0;
        for (int k = 0; k < mk.n; ++k) s += row[int64_t(marked_id(mk, k)) * batch];
        curve[i] = s;
    }
}

constexpr int kArgmaxThreads = 256;

// (value, sample) pairs: a pair with r < 0 holds nothing; otherwise the larger
// value wins and equal values go to the earlier sample.  NaN entries are
// skipped when the pairs are formed, so they never win.
__device__ __forceinline__ bool curve_better(double v, int64_t r, double bv, int64_t br)
{
    if (r < 0) return false;
    if (br < 0) return true;
    return v > bv || (v == bv && r < br);
}

// one CTA per column: strided scan, then a fixed tree over the threads
__global__ void __launch_bounds__(kArgmaxThreads)
k_curve_argmax(const double *__restrict__ curve, int64_t R, int batch, int64_t *__restrict__ argmax,
               double *__restrict__ maxv)
{
    __shared__ double sv[kArgmaxThreads];
    __shared__ int64_t sr[kArgmaxThreads];
    const int b = blockIdx.x;
    double bv = 0.0;
    int64_t br = -1;
    for (int64_t r = threadIdx.x; r < R; r += kArgmaxThreads) {
        const double v = curve[r * batch + b];
        if (v == v && curve_better(v, r, bv, br)) { bv = v; br = r; }
    }
    sv[threadIdx.x] = bv;
    sr[threadIdx.x] = br;
    __syncthreads();
    for (int o = kArgmaxThreads / 2; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o && curve_better(sv[threadIdx.x + o], sr[threadIdx.x + o], sv[threadIdx.x],
                                                 sr[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + o];
            sr[threadIdx.x] = sr[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (argmax) argmax[b] = sr[0];
        if (maxv) maxv[b] = sr[0] < 0 ? __longlong_as_double(0x7ff8000000000000LL) : sv[0];
    }
}

}  // namespace

extern "C" hw_status hw_success_curve(const double *prob, int64_t R, int64_t n, int32_t batch,
                                      const int32_t *marked, int32_t n_marked, double *curve_out,
                                      int64_t *argmax_out, double *max_out, void *stream)
{
    hw_clear_error();
    if (R < 0) return hw_fail(HW_EINVAL, "R must be >= 0");
    if (n < 1) return hw_fail(HW_EINVAL, "n must be >= 1");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (n_marked < 1 || !marked) return hw_fail(HW_EINVAL, "the success curve needs at least one marked vertex");
    if (R > 0 && !curve_out) return hw_fail(HW_EINVAL, "curve_out is NULL");
    if (R > 0 && !prob) return hw_fail(HW_EINVAL, "prob is NULL");
    if (((uintptr_t)prob | (uintptr_t)curve_out | (uintptr_t)argmax_out | (uintptr_t)max_out) % 8)
        return hw_fail(HW_EINVAL, "buffers must be 8-byte aligned");
    if (R > 0) {
        const char *p0 = reinterpret_cast<const char *>(prob);
        const char *c0 = reinterpret_cast<const char *>(curve_out);
        const size_t pb = sizeof(double) * size_t(R) * size_t(n) * size_t(batch);
        const size_t cb = sizeof(double) * size_t(R) * size_t(batch);
        if (p0 < c0 + cb && c0 < p0 + pb) return hw_fail(HW_EINVAL, "curve_out overlaps prob");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MarkedList mk;
    hw_status s = make_marked(marked, n_marked, n, st, &mk);
    if (s != HW_OK) return s;
    if (R > 0) {
        const int64_t total = R * batch;
        const int64_t grid = std::min<int64_t>(148 * 8, std::max<int64_t>(1, (total + 255) / 256));
        k_success_curve<<<grid, 256, 0, st>>>(prob, R, n, batch, mk, curve_out);
        s = hw_cuda(cudaGetLastError(), "k_success_curve launch");
    }
    if (s == HW_OK && (argmax_out || max_out)) {
        k_curve_argmax<<<batch, kArgmaxThreads, 0, st>>>(curve_out, R, batch, argmax_out, max_out);
        s = hw_cuda(cudaGetLastError(), "k_curve_argmax launch");
    }
    free_marked(mk, st);
    return s;
}

// ---------------------------------------------------------------- no allocation
// hw_probability for callers that cannot allocate device memory during a
// call: programs that run under a fixed, pre-reserved memory budget (a
// serving loop that must not hit out-of-memory halfway through a request),
// and platforms where the stream-ordered allocator is unavailable
// (cudaDevAttrMemoryPoolsSupported == 0, as under some virtualised or MPS
// setups).  The norm's per-CTA partials live in this file-scope device
// array instead of coming from the scratch pool.  Every device that loads the
// library holds the array until the process exits.
namespace {

constexpr int kNoAllocMaxParts = 1184;    // norm_parts() never exceeds this
constexpr int kNoAllocMaxBatch = 64;      // largest batch the array serves
static __device__ __align__(256) double g_norm_scratch[kNoAllocMaxParts * kNoAllocMaxBatch];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {};   // device address of g_norm_scratch, per device

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is resolved
// with cudaGetSymbolAddress, once per device, with that device current.
hw_status scratch_on_current_device(double **out)
{
    int dev = -1;
    hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != HW_OK) return s;
    if (dev < 0 || dev >= kMaxDevices) return hw_fail(HW_EUNSUPPORTED, "device index %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if ((s = hw_cuda(cudaGetSymbolAddress(&p, g_norm_scratch), "cudaGetSymbolAddress(g_norm_scratch)")) != HW_OK)
            return s;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return HW_OK;
}

}  // namespace

extern "C" hw_status hw_probability_noalloc(const hw_graph *g, int64_t n, hw_dtype dt, int32_t batch,
                                            const void *psi, double *prob_out, double *norm_out,
                                            void *stream)
{
    hw_clear_error();
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (!psi) return hw_fail(HW_EINVAL, "psi is NULL");
    if (!prob_out && !norm_out) return hw_fail(HW_EINVAL, "nothing to compute");
    if ((uintptr_t)psi % cplx_bytes(dt)) return hw_fail(HW_EINVAL, "psi misaligned");
    if (((uintptr_t)prob_out | (uintptr_t)norm_out) % 8) return hw_fail(HW_EINVAL, "outputs misaligned");
    if (norm_out && batch > kNoAllocMaxBatch)
        return hw_fail(HW_EINVAL, "hw_probability_noalloc: batch %d exceeds the built-in scratch limit of %d "
                       "states for the norm (use hw_probability)", batch, kNoAllocMaxBatch);
    if (g) {
        int dev = -1;
        hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        if (s != HW_OK) return s;
        if (dev != g->device) return hw_fail(HW_EINVAL, "graph lives on device %d, current is %d", g->device, dev);
        n = g->n;
    } else if (n < 1) {
        return hw_fail(HW_EINVAL, "n must be >= 1");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *scratch = nullptr;
    if (norm_out) {
        hw_status s = scratch_on_current_device(&scratch);
        if (s != HW_OK) return s;
    }
    if (prob_out) {
        hw_status s = launch_probability(g, n, dt, batch, psi, prob_out, nullptr, st);
        if (s != HW_OK) return s;
    }
    if (norm_out) {
        const int64_t rows = g ? g->num_arcs : n;
        if (rows == 0) return hw_cuda(cudaMemsetAsync(norm_out, 0, sizeof(double) * batch, st), "memset norm");
        // every partial the final pass reads is written by the first pass, so
        // nothing left in the array by an earlier call needs clearing
        return launch_norm(dt, batch, psi, rows, scratch, norm_out, st);
    }
    return HW_OK;
}
