// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <utility>
#include <mutex>
#include <vector>

#include "hiperwalk_b300.h"

// Arc tile of the fused coin+shift kernel: a CTA owns whole vertices whose
// arcs fit in one tile; a vertex with more arcs than a tile gets a CTA alone.
constexpr int kTileArcs = 1024;
constexpr int kTileVerts = 1024;

struct hw_graph {
    int device = -1;
    int64_t n = 0;
    int64_t num_arcs = 0;
    int32_t max_degree = 0;
    int32_t min_degree = 0;
    int32_t nblk = 0;                // vertex blocks of the coin+shift kernel
    int32_t *d_row_ptr = nullptr;    // [n+1]
    int32_t *d_head = nullptr;       // [num_arcs]
    int32_t *d_rev = nullptr;        // [num_arcs]
    // regular graphs (degree d >= 1): the reversal table of the edge-major
    // layout E[j][v] = psi[v d + j]: revE[j n + v] = j' n + w where arc
    // v d + j = (v, w) reverses to w d + j'; nullptr otherwise
    int32_t *d_revE = nullptr;       // [num_arcs]
    // recognised family (hw_graph_kind) and its parameters: torus {L1, L2},
    // hypercube {k, 0}
    int32_t kind = HW_GRAPH_GENERIC;
    int64_t dims[2] = {0, 0};
    // tori: the persistent shift as arc tables, arc-major (pers[a]) and
    // edge-major (persE[j n + v]); nullptr otherwise
    int32_t *d_pers = nullptr;       // [num_arcs]
    int32_t *d_persE = nullptr;      // [num_arcs]
    // weighted adjacency W (hw_graph_csr_weighted), arc-aligned with d_head;
    // imaginary parts only for a complex Hermitian W
    bool weighted = false, complex_weights = false;
    double *d_wre = nullptr, *d_wim = nullptr;
    float *d_wre_f = nullptr, *d_wim_f = nullptr;
    std::vector<double> h_rowabs;    // sum over row v of |w|
    double max_rowabs = 0.0;
    std::vector<double> h_wabs;      // distinct nonzero |w| (real W)
    int32_t *d_blk = nullptr;        // [nblk+1] first vertex of each block
    double *d_two_over_d = nullptr;  // [max_degree+1], 2/d (0 for d = 0): the Grover weight
    float *d_two_over_d_f = nullptr; // the same rounded to float
    int *h_err = nullptr;            // zero-copy word: a kernel's bounded wait ran out of time
    int *d_err = nullptr;            // its device alias
    std::vector<int32_t> h_row_ptr;  // host copy for launch decisions
    std::vector<int32_t> h_blk;
    // autotuned launch shape of the batched kernel per (batch, dtype)
    mutable std::mutex tune_mu;
    mutable std::map<long long, int> tune_rows;
    // measured cost of a batch-1 coined walk (hw_coined_evolve, launch_mode 0)
    // per (dtype, shift): {fixed, per step} of the single launch, then of one
    // launch per step, in milliseconds
    mutable std::map<int, std::array<double, 4>> walk_cost;
};

// ---- errors (api.cpp)
hw_status hw_fail(hw_status s, const char *fmt, ...);
hw_status hw_cuda(cudaError_t e, const char *what);
// stream-ordered scratch from the library's per-device pool (free with cudaFreeAsync)
cudaError_t hw_malloc_async(void **p, size_t bytes, cudaStream_t st);
void hw_clear_error();

// ---- host graph construction (graph.cpp)
// Sorted rows, reversal table and block partition, all on the host.
// Sorted rows, reversal table and (w_re != NULL) the weights permuted with
// their columns and checked to be finite and Hermitian.
hw_status hw_build_arcs_host(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             std::vector<int32_t> &rp, std::vector<int32_t> &head,
                             std::vector<int32_t> &rev, const double *w_re, const double *w_im,
                             std::vector<double> *wre_out, std::vector<double> *wim_out);
void hw_partition_blocks(const std::vector<int32_t> &rp, int tile_arcs, int tile_verts,
                         std::vector<int32_t> &blk);
// family of a sorted arc basis (exact comparison of every row)
void hw_detect_family(int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &head,
                      int32_t *kind, int64_t dims[2]);

// ---- device launchers (coined.cu, prob.cu, ctqw.cu)
// Marked lists up to this length travel inside the kernel parameters (no
// upload, no host synchronisation); longer lists are uploaded once per call.
constexpr int kInlineMarked = 16;
struct MarkedList {
    const int32_t *dev;          // device array (sorted) when n > kInlineMarked, else nullptr
    int32_t n;
    int32_t inl[kInlineMarked];  // sorted ids when n <= kInlineMarked
};

#ifdef __CUDACC__
// Position of v in the marked list, or -1.  Inline ids are compared at
// constant indices (an unrolled scan stopping at the uniform count), so the
// list is read from the kernel's parameter bank: a computed index into a
// parameter array makes the compiler copy the whole list to local memory in
// every thread.
__device__ __forceinline__ int marked_find(const MarkedList &mk, int v)
{
    if (mk.dev) {
        int lo = 0, hi = mk.n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int m = __ldg(mk.dev + mid);
            if (m == v) return mid;
            if (m < v) lo = mid + 1; else hi = mid;
        }
        return -1;
    }
#pragma unroll
    for (int k = 0; k < kInlineMarked; ++k) {
        if (k >= mk.n) break;
        if (mk.inl[k] == v) return k;
    }
    return -1;
}

// the i-th marked id (0 <= i < n), by the same constant-index selection
__device__ __forceinline__ int marked_id(const MarkedList &mk, int i)
{
    if (mk.dev) return __ldg(mk.dev + i);
    int m = -1;
#pragma unroll
    for (int k = 0; k < kInlineMarked; ++k)
        if (k == i) m = mk.inl[k];
    return m;
}
#endif

enum { kShiftFlipFlop = 0, kShiftPersistent = 1 };

struct CoinedStep {
    const void *in;
    void *out;
    MarkedList marked;
    double *rec_part;        // [slots][n_marked] or nullptr
    int64_t rec_slot;        // slot receiving the marked probability of `in`, or -1
    int shift = kShiftFlipFlop;   // kShiftPersistent needs a torus (hw_graph::d_pers)
    bool index_free = false;      // edge-major path on a torus / hypercube: positions from labels
};
// the shift as an arc table: out[table[a]] = (C psi)[a]
inline const int32_t *shift_table(const hw_graph *g, int shift) { return shift == kShiftPersistent ? g->d_pers : g->d_rev; }
inline const int32_t *shift_table_em(const hw_graph *g, int shift) { return shift == kShiftPersistent ? g->d_persE : g->d_revE; }
// edge-major layout of regular graphs (see hw_graph::d_revE)
bool coined_em_supported(const hw_graph *g, hw_coin coin, hw_dtype dt);
hw_status launch_layout(const hw_graph *g, hw_dtype dt, const void *in, void *out, bool to_edge, cudaStream_t st);
hw_status launch_coined_step_em(const hw_graph *g, hw_dtype dt, hw_coin coin, const CoinedStep &s, cudaStream_t st);
hw_status launch_coined_step(const hw_graph *g, hw_dtype dt, hw_coin coin, const CoinedStep &s,
                             cudaStream_t st);
hw_status launch_coined_step_batched(const hw_graph *g, hw_dtype dt, hw_coin coin, int batch,
                                     const CoinedStep &s, int tile, cudaStream_t st);
// whole walks of small regular graphs in one thread-block cluster (coined_cluster.cu)
bool coined_cluster_supported(const hw_graph *g, hw_coin coin, hw_dtype dt);
bool coined_cluster_by_size(const hw_graph *g, hw_dtype dt);
hw_status launch_coined_cluster(const hw_graph *g, hw_dtype dt, const void *in, void *out, int64_t steps,
                                const MarkedList &mk, double *rec_part, int64_t stride, const int32_t *shift,
                                cudaStream_t st);
hw_status launch_marked_prob(const int32_t *row_ptr, hw_dtype dt, int batch, const void *psi,
                             const MarkedList &marked, double *dst, cudaStream_t st);
hw_status launch_record_finalize(const double *rec_part, int32_t n_marked, int64_t slots,
                                 int batch, double *record, cudaStream_t st);
hw_status launch_probability(const hw_graph *g, int64_t n, hw_dtype dt, int batch,
                             const void *psi, double *prob, double *norm, cudaStream_t st);

// Validated, sorted marked list; long lists get a device copy (stream-ordered
// allocation, released by free_marked on the same stream).
hw_status make_marked(const int32_t *marked, int32_t n_marked, int64_t n, cudaStream_t st,
                      MarkedList *out);
void free_marked(MarkedList &m, cudaStream_t st);

// tensor-core Taylor powers (gemm_tc.cu): Q_k = Q_{k-1} Y / k on tcgen05 from
// split-bf16 operands, accU += sign Q_k in double
// Y = off (times w[a] when w is not NULL) on every arc a of the CSR (row_ptr,
// col) plus diag on the marked vertices' diagonal: the sparse symmetric
// matrix whose powers are taken
struct SymSparse {
    const int32_t *row_ptr;
    const int32_t *col;
    const double *w;
    int n;
    double off;
    MarkedList mk;
    double diag;
};

struct TcPower;
bool tc_gemm_available();
hw_status tc_power_begin(const SymSparse &Y, const double *yvals, int nyvals, double theta, int mode, int tiles_mode,
                         cudaStream_t st, TcPower **out);
hw_status tc_power_step(TcPower *p, int k, double *accU, double sign);
// adds the last power to its sum and frees the state
hw_status tc_power_end(TcPower *p, cudaStream_t st, bool check);
// adds the last power while writing U = Re + i Im (complex64, n x n) from the
// lower triangles of Re and Im, and frees the state
hw_status tc_power_finish_c64(TcPower *p, const double *Re, const double *Im, void *U, cudaStream_t st);

// Programmatic dependent launch: consecutive steps of a loop overlap the next
// grid's launch with the current grid's tail.  A kernel launched this way
// reads the previous step's output only after pdl_wait(), which returns once
// the previous grid has completed and its writes are visible; pdl_trigger()
// lets the next grid be scheduled.
#ifdef __CUDACC__
// q = e / d, r = e - q d for non-negative indices: a 32-bit division when both
// fit in 32 bits (the usual case), the 64-bit one otherwise.  The 64-bit
// integer division is a long instruction sequence; in a thread-per-element
// kernel it can cost more than the element's own work.
__device__ __forceinline__ int64_t idx_div(int64_t e, int64_t d, int64_t &r)
{
    if (((uint64_t(e) | uint64_t(d)) >> 32) == 0) {
        const uint32_t q = uint32_t(e) / uint32_t(d);
        r = int64_t(uint32_t(e) - q * uint32_t(d));
        return int64_t(q);
    }
    const int64_t q = e / d;
    r = e - q * d;
    return q;
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

inline size_t cplx_bytes(hw_dtype dt) { return dt == HW_C128 ? 16 : 8; }
