// Continuous-time walk by the action of e^{-iH dt} on the state (Sec. 3.1),
// without forming U: each application splits dt into q = 2^s equal parts
// (e^{-iH dt} = (e^{-iH dt/q})^q) and sums the exponential series of each
// part to degree m, with (s, m) from the same rule as hw_ctqw_plan
// (||H dt/q|| <= 1/2, truncation < 2^-60).  A term is
//   t_k = (-i tau / k) H t_{k-1},  (H x)_v = -gamma sum_{w ~ v} x_w - [v in M] x_v,
// one CSR gather per vertex; the partial sum is accumulated in the same pass.
// Work per application: q*m sparse products of 2|E| + n entries, so large
// graphs that have no room for a dense n x n U stay cheap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace {

template <typename R> struct Cx3;
template <> struct Cx3<double> { using T = double2; };
template <> struct Cx3<float> { using T = float2; };

__device__ __forceinline__ int marked_index(const MarkedList &mk, int v)
{
    int lo = 0, hi = mk.n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int m = mk.dev ? mk.dev[mid] : mk.inl[mid];
        if (m == v) return mid;
        if (m < v) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// t_out = (-i tau/k) H t_in; acc = (first ? x + t_out : acc + t_out).
// Thread per (vertex, column); neighbours in sorted order.
template <typename R>
__global__ void k_ctqw_term(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ head, int64_t n,
                            int batch, MarkedList mk, double gamma, double coef, const void *x_,
                            const void *tin_, void *tout_, void *acc_, int first)
{
    using V = typename Cx3<R>::T;
    const V *__restrict__ x = static_cast<const V *>(x_);
    const V *__restrict__ tin = static_cast<const V *>(tin_);
    V *__restrict__ tout = static_cast<V *>(tout_);
    V *__restrict__ acc = static_cast<V *>(acc_);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    pdl_wait();   // t_in and acc come from the previous term
    if (i >= n * batch) {
        pdl_trigger();
        return;
    }
    const int64_t v = i / batch;
    const int b = int(i % batch);
    R sx = 0, sy = 0;
    for (int a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
        const V q = tin[int64_t(head[a]) * batch + b];
        sx += q.x;
        sy += q.y;
    }
    R hx = R(-gamma) * sx, hy = R(-gamma) * sy;
    if (mk.n && marked_index(mk, int(v)) >= 0) {
        const V q = tin[i];
        hx -= q.x;
        hy -= q.y;
    }
    // (-i c) (hx + i hy) = c hy - i c hx
    const R c = R(coef);
    V t;
    t.x = c * hy;
    t.y = -c * hx;
    tout[i] = t;
    const V base = first ? x[i] : acc[i];
    V o;
    o.x = base.x + t.x;
    o.y = base.y + t.y;
    acc[i] = o;
    pdl_trigger();
}

template <typename R>
hw_status launch_term(const hw_graph *g, int batch, const MarkedList &mk, double gamma, double coef, const void *x,
                      const void *tin, void *tout, void *acc, int first, cudaStream_t st)
{
    const int64_t total = g->n * batch;
    const int64_t grid = (total + 255) / 256;
    launch_pdl(k_ctqw_term<R>, dim3(unsigned(grid)), dim3(256), 0, st, (const int32_t *)g->d_row_ptr,
               (const int32_t *)g->d_head, g->n, batch, mk, gamma, coef, x, tin, tout, acc, first);
    return hw_cuda(cudaGetLastError(), "k_ctqw_term launch");
}

}  // namespace

extern "C" hw_status hw_ctqw_evolve_sparse(const hw_graph *g, double gamma, const int32_t *marked, int32_t n_marked,
                                           double time, hw_dtype dt, int32_t batch, int64_t steps,
                                           const void *psi_in, void *psi_out, double *record,
                                           const hw_opts *opts, void *stream)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (steps < 0) return hw_fail(HW_EINVAL, "steps must be >= 0");
    if (!psi_in || !psi_out) return hw_fail(HW_EINVAL, "NULL state");
    if (!std::isfinite(gamma) || !std::isfinite(time)) return hw_fail(HW_EINVAL, "gamma/time not finite");
    if (n_marked < 0 || (n_marked > 0 && !marked)) return hw_fail(HW_EINVAL, "bad marked list");
    const size_t esz = cplx_bytes(dt);
    if ((uintptr_t)psi_in % esz || (uintptr_t)psi_out % esz) return hw_fail(HW_EINVAL, "state misaligned");
    const int stride = opts ? opts->record_stride : 1;
    if (stride < 1) return hw_fail(HW_EINVAL, "record_stride must be >= 1");
    if (record && n_marked == 0) return hw_fail(HW_EINVAL, "record needs at least one marked vertex");
    const size_t bytes = size_t(g->n) * batch * esz;
    const char *ip = static_cast<const char *>(psi_in);
    const char *op = static_cast<const char *>(psi_out);
    if (ip != op && ip < op + bytes && op < ip + bytes)
        return hw_fail(HW_EINVAL, "psi_in and psi_out overlap without being equal");
    int dev = -1;
    hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != HW_OK) return s;
    if (dev != g->device) return hw_fail(HW_EINVAL, "graph lives on device %d, current is %d", g->device, dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (steps == 0) {
        if (ip != op) return hw_cuda(cudaMemcpyAsync(psi_out, psi_in, bytes, cudaMemcpyDeviceToDevice, st), "copy");
        return HW_OK;
    }
    int m_deg = 1, sq = 0;
    if ((s = hw_ctqw_plan(g, gamma, marked, n_marked, time, &m_deg, &sq)) != HW_OK) return s;
    if (opts && opts->taylor_degree > 0) m_deg = opts->taylor_degree;
    if (opts && opts->taylor_squarings >= 0) sq = opts->taylor_squarings;
    if (m_deg > 40 || sq > 30) return hw_fail(HW_EINVAL, "Taylor degree %d / splits 2^%d out of range", m_deg, sq);
    const int64_t parts = int64_t(1) << sq;
    const double tau = time / double(parts);
    MarkedList mk;
    if ((s = make_marked(marked, n_marked, g->n, st, &mk)) != HW_OK) return s;
    struct Rel { MarkedList &m; cudaStream_t st; ~Rel() { free_marked(m, st); } } rel{mk, st};
    const int64_t slots = record ? steps / stride : 0;
    void *mem = nullptr;
    const size_t rec_bytes = (slots && n_marked > 1) ? sizeof(double) * slots * n_marked * batch : 0;
    if ((s = hw_cuda(hw_malloc_async(&mem, 4 * bytes + rec_bytes + 64, st), "scratch allocation (ctqw buffers)")) != HW_OK)
        return s;
    struct Free { void *p; cudaStream_t st; ~Free() { cudaFreeAsync(p, st); } } fr{mem, st};
    char *b = static_cast<char *>(mem);
    void *X[2] = {b, b + bytes};
    void *T[2] = {b + 2 * bytes, b + 3 * bytes};
    double *rec_part = slots ? (n_marked == 1 ? record : reinterpret_cast<double *>(b + 4 * bytes)) : nullptr;
    if ((s = hw_cuda(cudaMemcpyAsync(X[0], psi_in, bytes, cudaMemcpyDeviceToDevice, st), "copy")) != HW_OK) return s;
    int cur = 0;
    for (int64_t w = 1; w <= steps; ++w) {
        for (int64_t r = 0; r < parts; ++r) {
            for (int k = 1; k <= m_deg; ++k) {
                const void *tin = (k == 1) ? X[cur] : T[(k - 1) % 2];
                const double coef = tau / double(k);
                s = (dt == HW_C128)
                        ? launch_term<double>(g, batch, mk, gamma, coef, X[cur], tin, T[k % 2], X[1 - cur], k == 1, st)
                        : launch_term<float>(g, batch, mk, gamma, coef, X[cur], tin, T[k % 2], X[1 - cur], k == 1, st);
                if (s != HW_OK) return s;
            }
            cur = 1 - cur;
        }
        if (slots && w % stride == 0) {
            s = launch_marked_prob(nullptr, dt, batch, X[cur], mk, rec_part + (w / stride - 1) * n_marked * batch, st);
            if (s != HW_OK) return s;
        }
    }
    if ((s = hw_cuda(cudaMemcpyAsync(psi_out, X[cur], bytes, cudaMemcpyDeviceToDevice, st), "copy")) != HW_OK)
        return s;
    if (slots && n_marked > 1) s = launch_record_finalize(rec_part, n_marked, slots, batch, record, st);
    return s;
}
