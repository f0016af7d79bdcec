// Graph -> arc basis (Sec. 3.2): arcs sorted by tail then head, the flip-flop
// shift as a reversal table, and the vertex-block partition used by the
// fused coin+shift kernel.  Host code; the result is uploaded once per graph.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

hw_status hw_build_arcs_host(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             std::vector<int32_t> &rp, std::vector<int32_t> &head,
                             std::vector<int32_t> &rev, const double *w_re, const double *w_im,
                             std::vector<double> *wre_out, std::vector<double> *wim_out)
{
    if (n < 1) return hw_fail(HW_EINVAL, "n must be >= 1 (got %lld)", (long long)n);
    if (n >= (int64_t(1) << 31) - 1) return hw_fail(HW_EUNSUPPORTED, "n >= 2^31 - 1");
    if (!row_ptr) return hw_fail(HW_EINVAL, "row_ptr is NULL");
    if (row_ptr[0] != 0) return hw_fail(HW_EINVAL, "row_ptr[0] must be 0");
    for (int64_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return hw_fail(HW_EINVAL, "row_ptr decreases at %lld", (long long)v);
    const int64_t m = row_ptr[n];
    if (m >= (int64_t(1) << 31)) return hw_fail(HW_EUNSUPPORTED, "2|E| = %lld >= 2^31 arcs", (long long)m);
    if (m > 0 && !col_idx) return hw_fail(HW_EINVAL, "col_idx is NULL");

    rp.resize(n + 1);
    for (int64_t v = 0; v <= n; ++v) rp[v] = int32_t(row_ptr[v]);
    head.assign(col_idx, col_idx + m);
    if (w_re) {
        // weights travel with their columns through the row sort
        wre_out->assign(size_t(m), 0.0);
        if (w_im) wim_out->assign(size_t(m), 0.0);
        std::vector<std::pair<int32_t, int64_t>> row;
        for (int64_t v = 0; v < n; ++v) {
            row.clear();
            for (int64_t a = rp[v]; a < rp[v + 1]; ++a) row.emplace_back(col_idx[a], a);
            std::sort(row.begin(), row.end());
            for (size_t i = 0; i < row.size(); ++i) {
                const int64_t a = rp[v] + int64_t(i), src = row[i].second;
                if (!std::isfinite(w_re[src]) || (w_im && !std::isfinite(w_im[src])))
                    return hw_fail(HW_EINVAL, "weight of (%lld, %d) is not finite", (long long)v, row[i].first);
                (*wre_out)[a] = w_re[src];
                if (w_im) (*wim_out)[a] = w_im[src];
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) {
        int32_t *b = head.data() + rp[v], *e = head.data() + rp[v + 1];
        std::sort(b, e);
        for (int32_t *p = b; p < e; ++p) {
            if (*p < 0 || *p >= n)
                return hw_fail(HW_EINVAL, "column %d out of range in row %lld", *p, (long long)v);
            if (*p == v) return hw_fail(HW_EINVAL, "self-loop at vertex %lld", (long long)v);
            if (p > b && p[-1] == *p)
                return hw_fail(HW_EINVAL, "repeated entry (%lld, %d)", (long long)v, *p);
        }
    }
    rev.resize(m);
    for (int64_t v = 0; v < n; ++v) {
        for (int32_t a = rp[v]; a < rp[v + 1]; ++a) {
            const int32_t w = head[a];
            const int32_t *b = head.data() + rp[w], *e = head.data() + rp[w + 1];
            const int32_t *p = std::lower_bound(b, e, int32_t(v));
            if (p == e || *p != v)
                return hw_fail(HW_EINVAL, "not symmetric: (%lld, %d) has no (%d, %lld)",
                               (long long)v, w, w, (long long)v);
            rev[a] = int32_t(p - head.data());
        }
    }
    if (w_re) {
        // W must be Hermitian: arc (w, v) carries the conjugate of arc (v, w)'s weight
        for (int64_t v = 0; v < n; ++v)
            for (int32_t a = rp[v]; a < rp[v + 1]; ++a) {
                const int32_t b = rev[a];
                if ((*wre_out)[b] != (*wre_out)[a] || (w_im && (*wim_out)[b] != -(*wim_out)[a]))
                    return hw_fail(HW_EINVAL, "weights not Hermitian at (%lld, %d)", (long long)v, head[a]);
            }
    }
    return HW_OK;
}

void hw_partition_blocks(const std::vector<int32_t> &rp, int tile_arcs, int tile_verts,
                         std::vector<int32_t> &blk)
{
    const int64_t n = int64_t(rp.size()) - 1;
    blk.clear();
    blk.push_back(0);
    int64_t v0 = 0;
    while (v0 < n) {
        int64_t v = v0;
        // a vertex too large for a tile gets a block of its own
        if (rp[v + 1] - rp[v] > tile_arcs) {
            v = v0 + 1;
        } else {
            while (v < n && v - v0 < tile_verts && rp[v + 1] - rp[v0] <= tile_arcs) ++v;
        }
        blk.push_back(int32_t(v));
        v0 = v;
    }
}

// ---- recognised families (the Grid and Hypercube classes of Sec. 3.1, 3.2)
// Torus L1 x L2 (L1, L2 >= 3), v = x L2 + y: the sorted neighbours of vertex 0
// are 1, L2 - 1, L2, n - L2, which gives L2; every row is then compared with
// the four labels (x +- 1, y), (x, y +- 1) sorted.  Hypercube: n = 2^k, rows
// equal to the sorted v XOR 2^b.
static void torus_row(int64_t v, int64_t L1, int64_t L2, int32_t out[4])
{
    const int64_t x = v / L2, y = v % L2;
    out[0] = int32_t(((x + L1 - 1) % L1) * L2 + y);
    out[1] = int32_t(x * L2 + (y + L2 - 1) % L2);
    out[2] = int32_t(x * L2 + (y + 1) % L2);
    out[3] = int32_t(((x + 1) % L1) * L2 + y);
    std::sort(out, out + 4);
}

void hw_detect_family(int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &head,
                      int32_t *kind, int64_t dims[2])
{
    *kind = HW_GRAPH_GENERIC;
    dims[0] = dims[1] = 0;
    bool all4 = n >= 9, cube = n >= 2 && (n & (n - 1)) == 0;
    int k = 0;
    while (cube && (int64_t(1) << k) < n) ++k;
    for (int64_t v = 0; v < n && (all4 || cube); ++v) {
        const int32_t d = rp[v + 1] - rp[v];
        all4 = all4 && d == 4;
        cube = cube && d == k;
    }
    if (cube) {
        std::vector<int32_t> row(k);
        bool ok = true;
        for (int64_t v = 0; v < n && ok; ++v) {
            for (int b = 0; b < k; ++b) row[b] = int32_t(v ^ (int64_t(1) << b));
            std::sort(row.begin(), row.end());
            ok = std::equal(row.begin(), row.end(), head.begin() + rp[v]);
        }
        if (ok) {
            *kind = HW_GRAPH_HYPERCUBE;
            dims[0] = k;
            return;
        }
    }
    if (!all4) return;
    const int64_t L2 = head[2];
    if (L2 < 3 || n % L2 != 0 || n / L2 < 3) return;
    const int64_t L1 = n / L2;
    int32_t row[4];
    for (int64_t v = 0; v < n; ++v) {
        torus_row(v, L1, L2, row);
        if (!std::equal(row, row + 4, head.begin() + rp[v])) return;
    }
    *kind = HW_GRAPH_TORUS;
    dims[0] = L1;
    dims[1] = L2;
}

// persistent shift of the torus: arc (v, w) -> (w, u), u - w = w - v
static void torus_persistent(int64_t L1, int64_t L2, const std::vector<int32_t> &rp,
                             const std::vector<int32_t> &head, std::vector<int32_t> &pers)
{
    const int64_t n = L1 * L2;
    pers.resize(size_t(4 * n));
    for (int64_t v = 0; v < n; ++v) {
        const int64_t xv = v / L2, yv = v % L2;
        for (int32_t a = rp[v]; a < rp[v + 1]; ++a) {
            const int64_t w = head[a], xw = w / L2, yw = w % L2;
            const int64_t u = ((2 * xw - xv + L1) % L1) * L2 + (2 * yw - yv + L2) % L2;
            const int32_t *b = head.data() + rp[w], *e = head.data() + rp[w + 1];
            pers[a] = int32_t(std::lower_bound(b, e, int32_t(u)) - head.data());
        }
    }
}

extern "C" hw_status hw_graph_structure_host(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                             int32_t *kind, int64_t *dims)
{
    hw_clear_error();
    if (!kind) return hw_fail(HW_EINVAL, "kind is NULL");
    std::vector<int32_t> rp, head, rev;
    hw_status s = hw_build_arcs_host(n, row_ptr, col_idx, rp, head, rev, nullptr, nullptr, nullptr, nullptr);
    if (s != HW_OK) return s;
    int64_t d[2];
    hw_detect_family(n, rp, head, kind, d);
    if (dims) { dims[0] = d[0]; dims[1] = d[1]; }
    return HW_OK;
}

extern "C" hw_status hw_graph_structure(const hw_graph *g, int32_t *kind, int64_t *dims)
{
    hw_clear_error();
    if (!g || !kind) return hw_fail(HW_EINVAL, "graph or kind is NULL");
    *kind = g->kind;
    if (dims) { dims[0] = g->dims[0]; dims[1] = g->dims[1]; }
    return HW_OK;
}

static hw_status graph_build(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *w_re,
                             const double *w_im, void *stream, hw_graph **out)
{
    hw_clear_error();
    if (!out) return hw_fail(HW_EINVAL, "out is NULL");
    *out = nullptr;
    hw_graph *g = new (std::nothrow) hw_graph;
    if (!g) return hw_fail(HW_ENOMEM, "host allocation failed");
    std::vector<int32_t> head, rev;
    std::vector<double> wre, wim;
    hw_status s = hw_build_arcs_host(n, row_ptr, col_idx, g->h_row_ptr, head, rev, w_re, w_im, &wre, &wim);
    if (s != HW_OK) { delete g; return s; }
    g->weighted = w_re != nullptr;
    g->complex_weights = w_im != nullptr;
    if (g->weighted) {
        // row sums of |w| (the infinity norm of W) and the distinct |w| (the
        // tensor-core slicing test), both host-side
        g->h_rowabs.assign(size_t(n), 0.0);
        for (int64_t v = 0; v < n; ++v) {
            double r = 0.0;
            for (int32_t a = g->h_row_ptr[v]; a < g->h_row_ptr[v + 1]; ++a)
                r += g->complex_weights ? std::hypot(wre[a], wim[a]) : std::fabs(wre[a]);
            g->h_rowabs[v] = r;
            g->max_rowabs = std::max(g->max_rowabs, r);
        }
        if (!g->complex_weights) {
            for (double x : wre)
                if (x != 0.0) g->h_wabs.push_back(std::fabs(x));
            std::sort(g->h_wabs.begin(), g->h_wabs.end());
            g->h_wabs.erase(std::unique(g->h_wabs.begin(), g->h_wabs.end()), g->h_wabs.end());
        }
    }
    g->n = n;
    g->num_arcs = g->h_row_ptr[n];
    g->max_degree = 0;
    g->min_degree = INT32_MAX;
    for (int64_t v = 0; v < n; ++v) {
        int32_t d = g->h_row_ptr[v + 1] - g->h_row_ptr[v];
        g->max_degree = std::max(g->max_degree, d);
        g->min_degree = std::min(g->min_degree, d);
    }
    hw_partition_blocks(g->h_row_ptr, kTileArcs, kTileVerts, g->h_blk);
    g->nblk = int32_t(g->h_blk.size() - 1);

    std::vector<double> w(g->max_degree + 1, 0.0);
    for (int32_t d = 1; d <= g->max_degree; ++d) w[d] = 2.0 / double(d);
    std::vector<float> wf(w.size());
    for (size_t d = 0; d < w.size(); ++d) wf[d] = float(w[d]);
    std::vector<float> wre_f(wre.size()), wim_f(wim.size());
    for (size_t a = 0; a < wre.size(); ++a) wre_f[a] = float(wre[a]);
    for (size_t a = 0; a < wim.size(); ++a) wim_f[a] = float(wim[a]);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto fail = [&](hw_status e) { hw_graph_free(g); return e; };
    if ((s = hw_cuda(cudaGetDevice(&g->device), "cudaGetDevice")) != HW_OK) return fail(s);
    // edge-major reversal table of a regular graph (see hw_graph::d_revE)
    std::vector<int32_t> revE;
    const bool regular = n > 0 && g->min_degree == g->max_degree && g->max_degree >= 1;
    if (regular) {
        const int64_t d = g->max_degree;
        revE.resize(size_t(g->num_arcs));
        for (int64_t v = 0; v < n; ++v)
            for (int64_t j = 0; j < d; ++j) {
                const int64_t r = rev[size_t(v * d + j)];
                revE[size_t(j * n + v)] = int32_t((r % d) * n + r / d);
            }
    }
    hw_detect_family(n, g->h_row_ptr, head, &g->kind, g->dims);
    std::vector<int32_t> pers, persE;
    const bool torus = g->kind == HW_GRAPH_TORUS;
    if (torus) {
        torus_persistent(g->dims[0], g->dims[1], g->h_row_ptr, head, pers);
        persE.resize(pers.size());
        for (int64_t v = 0; v < n; ++v)
            for (int64_t j = 0; j < 4; ++j) {
                const int64_t r = pers[size_t(v * 4 + j)];
                persE[size_t(j * n + v)] = int32_t((r % 4) * n + r / 4);
            }
    }
    const size_t arcs_b = sizeof(int32_t) * std::max<int64_t>(g->num_arcs, 1);
    if (cudaMalloc(&g->d_row_ptr, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&g->d_head, arcs_b) != cudaSuccess ||
        cudaMalloc(&g->d_rev, arcs_b) != cudaSuccess ||
        (regular && cudaMalloc(&g->d_revE, arcs_b) != cudaSuccess) ||
        (torus && cudaMalloc(&g->d_pers, arcs_b) != cudaSuccess) ||
        (torus && cudaMalloc(&g->d_persE, arcs_b) != cudaSuccess) ||
        cudaMalloc(&g->d_blk, sizeof(int32_t) * g->h_blk.size()) != cudaSuccess ||
        cudaMalloc(&g->d_two_over_d, sizeof(double) * (g->max_degree + 1)) != cudaSuccess ||
        cudaMalloc(&g->d_two_over_d_f, sizeof(float) * (g->max_degree + 1)) != cudaSuccess ||
        (g->weighted && (cudaMalloc(&g->d_wre, sizeof(double) * std::max<int64_t>(g->num_arcs, 1)) != cudaSuccess ||
                         cudaMalloc(&g->d_wre_f, sizeof(float) * std::max<int64_t>(g->num_arcs, 1)) != cudaSuccess)) ||
        (g->complex_weights && (cudaMalloc(&g->d_wim, sizeof(double) * std::max<int64_t>(g->num_arcs, 1)) != cudaSuccess ||
                                cudaMalloc(&g->d_wim_f, sizeof(float) * std::max<int64_t>(g->num_arcs, 1)) != cudaSuccess)) ||
        cudaHostAlloc(&g->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&g->d_err, g->h_err, 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(hw_fail(HW_ENOMEM, "device allocation of the graph failed"));
    }
    if ((s = hw_cuda(cudaMemcpyAsync(g->d_row_ptr, g->h_row_ptr.data(), sizeof(int32_t) * (n + 1),
                                     cudaMemcpyHostToDevice, st), "upload row_ptr")) != HW_OK ||
        (s = hw_cuda(cudaMemcpyAsync(g->d_head, head.data(), sizeof(int32_t) * g->num_arcs,
                                     cudaMemcpyHostToDevice, st), "upload head")) != HW_OK ||
        (s = hw_cuda(cudaMemcpyAsync(g->d_rev, rev.data(), sizeof(int32_t) * g->num_arcs,
                                     cudaMemcpyHostToDevice, st), "upload rev")) != HW_OK ||
        (regular && (s = hw_cuda(cudaMemcpyAsync(g->d_revE, revE.data(), sizeof(int32_t) * g->num_arcs,
                                                 cudaMemcpyHostToDevice, st), "upload revE")) != HW_OK) ||
        (torus && (s = hw_cuda(cudaMemcpyAsync(g->d_pers, pers.data(), sizeof(int32_t) * g->num_arcs,
                                               cudaMemcpyHostToDevice, st), "upload pers")) != HW_OK) ||
        (torus && (s = hw_cuda(cudaMemcpyAsync(g->d_persE, persE.data(), sizeof(int32_t) * g->num_arcs,
                                               cudaMemcpyHostToDevice, st), "upload persE")) != HW_OK) ||
        (s = hw_cuda(cudaMemcpyAsync(g->d_blk, g->h_blk.data(), sizeof(int32_t) * g->h_blk.size(),
                                     cudaMemcpyHostToDevice, st), "upload blocks")) != HW_OK ||
        (s = hw_cuda(cudaMemcpyAsync(g->d_two_over_d, w.data(), sizeof(double) * w.size(),
                                     cudaMemcpyHostToDevice, st), "upload weights")) != HW_OK ||
        (s = hw_cuda(cudaMemcpyAsync(g->d_two_over_d_f, wf.data(), sizeof(float) * wf.size(),
                                     cudaMemcpyHostToDevice, st), "upload weights (float)")) != HW_OK ||
        (g->weighted && g->num_arcs &&
         ((s = hw_cuda(cudaMemcpyAsync(g->d_wre, wre.data(), sizeof(double) * g->num_arcs, cudaMemcpyHostToDevice, st),
                       "upload edge weights")) != HW_OK ||
          (s = hw_cuda(cudaMemcpyAsync(g->d_wre_f, wre_f.data(), sizeof(float) * g->num_arcs, cudaMemcpyHostToDevice, st),
                       "upload edge weights (float)")) != HW_OK)) ||
        (g->complex_weights && g->num_arcs &&
         ((s = hw_cuda(cudaMemcpyAsync(g->d_wim, wim.data(), sizeof(double) * g->num_arcs, cudaMemcpyHostToDevice, st),
                       "upload edge weights (imaginary)")) != HW_OK ||
          (s = hw_cuda(cudaMemcpyAsync(g->d_wim_f, wim_f.data(), sizeof(float) * g->num_arcs, cudaMemcpyHostToDevice, st),
                       "upload edge weights (imaginary, float)")) != HW_OK)) ||
        (s = hw_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) != HW_OK)
        return fail(s);
    *g->h_err = 0;
    *out = g;
    return HW_OK;
}

extern "C" hw_status hw_graph_csr(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                  void *stream, hw_graph **out)
{
    return graph_build(n, row_ptr, col_idx, nullptr, nullptr, stream, out);
}

extern "C" hw_status hw_graph_csr_weighted(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                           const double *w_re, const double *w_im, void *stream, hw_graph **out)
{
    if (!w_re) {
        hw_clear_error();
        return hw_fail(HW_EINVAL, "w_re is NULL (use hw_graph_csr for an unweighted graph)");
    }
    return graph_build(n, row_ptr, col_idx, w_re, w_im, stream, out);
}

extern "C" hw_status hw_graph_free(hw_graph *g)
{
    hw_clear_error();
    if (!g) return HW_OK;
    cudaFree(g->d_row_ptr);
    cudaFree(g->d_head);
    cudaFree(g->d_rev);
    cudaFree(g->d_revE);
    cudaFree(g->d_pers);
    cudaFree(g->d_persE);
    cudaFree(g->d_blk);
    cudaFree(g->d_two_over_d);
    cudaFree(g->d_two_over_d_f);
    cudaFree(g->d_wre);
    cudaFree(g->d_wim);
    cudaFree(g->d_wre_f);
    cudaFree(g->d_wim_f);
    if (g->h_err) cudaFreeHost(g->h_err);
    cudaGetLastError();
    delete g;
    return HW_OK;
}

extern "C" hw_status hw_graph_info(const hw_graph *g, int64_t *n, int64_t *num_arcs,
                                   const int32_t **d_row_ptr, const int32_t **d_head,
                                   const int32_t **d_rev)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (num_arcs) *num_arcs = g->num_arcs;
    if (d_row_ptr) *d_row_ptr = g->d_row_ptr;
    if (d_head) *d_head = g->d_head;
    if (d_rev) *d_rev = g->d_rev;
    return HW_OK;
}

extern "C" hw_status hw_graph_arcs_host(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                        int32_t *row_ptr_out, int32_t *head_out, int32_t *rev_out)
{
    hw_clear_error();
    std::vector<int32_t> rp, head, rev;
    hw_status s = hw_build_arcs_host(n, row_ptr, col_idx, rp, head, rev, nullptr, nullptr, nullptr, nullptr);
    if (s != HW_OK) return s;
    if (row_ptr_out) std::memcpy(row_ptr_out, rp.data(), sizeof(int32_t) * rp.size());
    if (head_out) std::memcpy(head_out, head.data(), sizeof(int32_t) * head.size());
    if (rev_out) std::memcpy(rev_out, rev.data(), sizeof(int32_t) * rev.size());
    return HW_OK;
}
