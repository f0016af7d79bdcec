// Continuous-time walk by the action of e^{-iH dt} on the state (Sec. 3.1),
// without forming U: each application splits dt into q = 2^s equal parts
// (e^{-iH dt} = (e^{-iH dt/q})^q) and sums the exponential series of each
// part to degree m, with (s, m) from the same rule as hw_ctqw_plan
// (||H dt/q|| <= 1/2, truncation < 2^-60).  A term is
//   t_k = (-i tau / k) H t_{k-1},  (H x)_v = -gamma sum_{w ~ v} W_vw x_w - [v in M] x_v,
// with W = A or a weighted Hermitian adjacency (hw_graph_csr_weighted),
// one CSR gather per vertex; the partial sum is accumulated in the same pass.
// Work per application: q*m sparse products of 2|E| + n entries, so large
// graphs that have no room for a dense n x n U stay cheap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "family.cuh"
#include "internal.h"
#include "sum4.cuh"

namespace {

template <typename R> struct Cx3;
template <> struct Cx3<double> { using T = double2; };
template <> struct Cx3<float> { using T = float2; };

__device__ __forceinline__ int marked_index(const MarkedList &mk, int v) { return marked_find(mk, v); }

// With s the sum of t_in over v's neighbours, (H t_in)_v = -gamma s - [v in M]
// t_in[v], and multiplying by -i c turns h = hx + i hy into c hy - i c hx:
//   t = (-(c gamma) s_y - c q_y, (c gamma) s_x + c q_x),  q = t_in[v] if v is
// marked, else 0.  Writes t_out[i] = t and acc[i] = (first ? x : acc)[i] + t.
template <typename R, typename V>
__device__ __forceinline__ void term_tail(R sx, R sy, const MarkedList &mk, int v, R cg, R c, const V *tin,
                                          const V *x, V *tout, V *acc, int64_t i, int first)
{
    V t;
    if (mk.n && marked_index(mk, v) >= 0) {
        const V q = tin[i];
        t.x = -fma(cg, sy, c * q.y);
        t.y = fma(cg, sx, c * q.x);
    } else {
        t.x = -(cg * sy);
        t.y = cg * sx;
    }
    tout[i] = t;
    const V base = first ? x[i] : acc[i];
    V o;
    o.x = base.x + t.x;
    o.y = base.y + t.y;
    acc[i] = o;
}

// t_out = (-i tau/k) H t_in; acc = (first ? x + t_out : acc + t_out).
// Thread per (vertex, column); neighbours in sorted order.  WT: 0 unweighted
// (the sum starts from the first neighbour), 1 real weights wr, 2 complex
// weights wr + i wi (the sum of w_a t_in[head a] by FMAs from zero).
template <typename R, int WT>
__global__ void k_ctqw_term(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ head,
                            const R *__restrict__ wr, const R *__restrict__ wi, int64_t n,
                            int batch, MarkedList mk, R cg, R coef, const void *x_,
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
    int64_t rb;
    const int64_t v = (batch == 1) ? i : idx_div(i, batch, rb);
    const int b = (batch == 1) ? 0 : int(rb);
    R sx = 0, sy = 0;
    int a = row_ptr[v];
    const int e = row_ptr[v + 1];
    if (WT == 0 && sizeof(R) == 8 && e - a >= 1 && e - a <= 4) {
        // complex128, up to four neighbours: their sum rounded once by integer
        // operations (sum4.cuh); larger degrees keep the double additions,
        // which measured faster there (the gathers, not the FP64 unit, bound them)
        double gx, gy;
        sum4::grouped_sum2(e - a, [&](int j) { return tin[int64_t(head[a + j]) * batch + b]; }, gx, gy);
        sx = R(gx);
        sy = R(gy);
    } else if constexpr (WT == 0) {
        if (a < e) {
            const V q = tin[int64_t(head[a]) * batch + b];
            sx = q.x;
            sy = q.y;
            ++a;
        }
        for (; a < e; ++a) {
            const V q = tin[int64_t(head[a]) * batch + b];
            sx += q.x;
            sy += q.y;
        }
    } else {
        for (; a < e; ++a) {
            const V q = tin[int64_t(head[a]) * batch + b];
            const R w = wr[a];
            sx = fma(w, q.x, sx);
            sy = fma(w, q.y, sy);
            if constexpr (WT == 2) {
                const R u = wi[a];
                sx = fma(-u, q.y, sx);
                sy = fma(u, q.x, sy);
            }
        }
    }
    term_tail<R, V>(sx, sy, mk, int(v), cg, coef, tin, x, tout, acc, i, first);
    pdl_trigger();
}

// The same term on a torus or hypercube: neighbour labels computed from v in
// ascending order (the order of the CSR row), so the sums are bit-identical
// to k_ctqw_term's, without the row_ptr and head reads.
template <typename R, int FAM>
__global__ void k_ctqw_term_fam(int64_t n, int batch, int L1, int L2, int grid2d, MarkedList mk, R cg, R coef,
                                const void *x_, const void *tin_, void *tout_, void *acc_, int first)
{
    using V = typename Cx3<R>::T;
    const V *__restrict__ x = static_cast<const V *>(x_);
    const V *__restrict__ tin = static_cast<const V *>(tin_);
    V *__restrict__ tout = static_cast<V *>(tout_);
    V *__restrict__ acc = static_cast<V *>(acc_);
    // torus, one column: a block row per torus row (grid2d), no division
    const uint32_t y2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = grid2d ? int64_t(blockIdx.y) * L2 + y2 : int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    pdl_wait();   // t_in and acc come from the previous term
    if (grid2d ? y2 >= uint32_t(L2) : i >= n * batch) {
        pdl_trigger();
        return;
    }
    int64_t rb;
    const int64_t v = (batch == 1) ? i : idx_div(i, batch, rb);
    const int b = (batch == 1) ? 0 : int(rb);
    R sx, sy;
    if constexpr (FAM == HW_GRAPH_TORUS) {
        int w[4];
        (grid2d ? TorusVertex(blockIdx.y, y2, n, L1, L2) : TorusVertex(v, n, L1, L2)).sorted(w);
        V q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) q[j] = tin[int64_t(w[j]) * batch + b];
        if constexpr (sizeof(R) == 8) {
            sum4::grouped_sum2(4, [&](int j) { return q[j]; }, sx, sy);
        } else {
            sx = q[0].x;
            sy = q[0].y;
#pragma unroll
            for (int j = 1; j < 4; ++j) {
                sx += q[j].x;
                sy += q[j].y;
            }
        }
    } else {
        CubeWalk cw(v, L1);   // L1 = k >= 1
        if (sizeof(R) == 8 && L1 <= 4) {
            // as the CSR kernel: up to four neighbours summed once by integer
            // operations; the walk yields them in the order grouped_sum2 asks for
            double gx, gy;
            sum4::grouped_sum2(L1, [&](int) { return tin[int64_t(uint32_t(v) ^ (1u << cw.next_bit())) * batch + b]; },
                               gx, gy);
            sx = R(gx);
            sy = R(gy);
        } else {
            const V q0 = tin[int64_t(uint32_t(v) ^ (1u << cw.next_bit())) * batch + b];
            sx = q0.x;
            sy = q0.y;
#pragma unroll 4
            for (int j = 1; j < L1; ++j) {
                const V q = tin[int64_t(uint32_t(v) ^ (1u << cw.next_bit())) * batch + b];
                sx += q.x;
                sy += q.y;
            }
        }
    }
    term_tail<R, V>(sx, sy, mk, int(v), cg, coef, tin, x, tout, acc, i, first);
    pdl_trigger();
}

template <typename R>
hw_status launch_term(const hw_graph *g, bool index_free, int batch, const MarkedList &mk, double gamma, double coef,
                      const void *x, const void *tin, void *tout, void *acc, int first, cudaStream_t st)
{
    // the constants in the kernel's precision, converted here once (a
    // conversion in the kernel would run per thread on the FP64 pipe)
    const R cg = R(coef * gamma), c = R(coef);
    const int64_t total = g->n * batch;
    const int64_t grid = (total + 255) / 256;
    const R *wr = nullptr, *wi = nullptr;
    if constexpr (sizeof(R) == 8) {
        wr = reinterpret_cast<const R *>(g->d_wre);
        wi = reinterpret_cast<const R *>(g->d_wim);
    } else {
        wr = reinterpret_cast<const R *>(g->d_wre_f);
        wi = reinterpret_cast<const R *>(g->d_wim_f);
    }
    if (g->weighted) {
        // weights are per arc of the CSR: the table path, no label arithmetic
        if (g->complex_weights)
            launch_pdl(k_ctqw_term<R, 2>, dim3(unsigned(grid)), dim3(256), 0, st, (const int32_t *)g->d_row_ptr,
                       (const int32_t *)g->d_head, wr, wi, g->n, batch, mk, cg, c, x, tin, tout, acc, first);
        else
            launch_pdl(k_ctqw_term<R, 1>, dim3(unsigned(grid)), dim3(256), 0, st, (const int32_t *)g->d_row_ptr,
                       (const int32_t *)g->d_head, wr, wi, g->n, batch, mk, cg, c, x, tin, tout, acc, first);
    } else if (index_free && g->kind == HW_GRAPH_TORUS)
    {
        const int L1 = int(g->dims[0]), L2 = int(g->dims[1]);
        const int g2 = (batch == 1 && L2 >= 128 && L1 <= 65535) ? 1 : 0;
        const dim3 gd = g2 ? dim3(unsigned((L2 + 255) / 256), unsigned(L1)) : dim3(unsigned(grid));
        launch_pdl(k_ctqw_term_fam<R, HW_GRAPH_TORUS>, gd, dim3(256), 0, st, g->n, batch, L1, L2, g2, mk, cg, c, x,
                   tin, tout, acc, first);
    }
    else if (index_free && g->kind == HW_GRAPH_HYPERCUBE)
        launch_pdl(k_ctqw_term_fam<R, HW_GRAPH_HYPERCUBE>, dim3(unsigned(grid)), dim3(256), 0, st, g->n, batch,
                   int(g->dims[0]), 0, 0, mk, cg, c, x, tin, tout, acc, first);
    else
        launch_pdl(k_ctqw_term<R, 0>, dim3(unsigned(grid)), dim3(256), 0, st, (const int32_t *)g->d_row_ptr,
                   (const int32_t *)g->d_head, wr, wi, g->n, batch, mk, cg, c, x, tin, tout, acc, first);
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
    if (opts && opts->addressing != 0 && opts->addressing != 1) return hw_fail(HW_EINVAL, "addressing must be 0 or 1");
    const bool index_free = !(opts && opts->addressing == 1);
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
                        ? launch_term<double>(g, index_free, batch, mk, gamma, coef, X[cur], tin, T[k % 2], X[1 - cur], k == 1, st)
                        : launch_term<float>(g, index_free, batch, mk, gamma, coef, X[cur], tin, T[k % 2], X[1 - cur], k == 1, st);
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
