/*
 * hiperwalk_b300.h -- C ABI of the B300 quantum-walk evolution library.
 *
 * The operations follow Motta, Bezerra, Santos, Portugal, "Hiperwalk:
 * Simulation of Quantum Walks with Heterogeneous High-Performance Computing"
 * (arXiv 2406.08186):
 *   Sec. 3.1  continuous-time walk: H = -gamma A - sum_{v in M} |v><v|,
 *             U(t) = e^{-iHt}, |psi(t)> = U(t)|psi(0)>, probability |<v|psi(t)>|^2
 *   Sec. 3.2  coined walk: U = S C, flip-flop shift S|v,w> = |w,v>, Grover coin
 *             C|v,w> = sum_{v' in N(v)} (2/d(v) - delta_{w,v'}) |v,v'>,
 *             |psi(t)> = U^t |psi(0)>, p_v(t) = sum_{w in N(v)} |<v,w|psi(t)>|^2;
 *             the basis is the arc list sorted by tail, then by head.
 *
 * General conventions (every entry point):
 *   - Every call returns an hw_status; on failure hw_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - Arguments are validated on the host before anything is launched; a
 *     call that fails validation launches nothing and writes nothing.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) of the CURRENT device, which
 *     must be the device the graph was created on.  Host pointers are read
 *     before the call returns; device buffers must stay alive until the
 *     stream has executed the work.
 *   - Device buffers (psi, U, record, prob) are allocated and owned by the
 *     caller; the library never frees them.  Complex numbers are interleaved
 *     (re, im): HW_C64 = 2 x float (8 bytes), HW_C128 = 2 x double (16 bytes).
 *     Device buffers must be aligned to their element size (16 bytes for
 *     HW_C128, 8 for HW_C64 and double).
 *   - Batched buffers are batch-innermost: element (i, b) is at i*batch + b.
 *   - No call waits without bound: device-side waits carry a time limit and
 *     report HW_ETIMEDOUT.
 *   - Host threads: calls may run concurrently from several threads, also on
 *     the same graph (its per-graph caches are locked), but a graph must not
 *     be freed while another call uses it, and one server (hw_server_*) is
 *     driven by one thread at a time.
 */
#ifndef HIPERWALK_B300_H
#define HIPERWALK_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HW_OK = 0,
    HW_EINVAL = -1,         /* invalid argument or graph */
    HW_ENOMEM = -2,         /* device or host allocation failed */
    HW_ECUDA = -3,          /* a CUDA runtime call or launch failed */
    HW_ETIMEDOUT = -4,      /* a device-side wait ran out of time */
    HW_EUNSUPPORTED = -5    /* valid request outside this build's limits */
} hw_status;

typedef enum { HW_C64 = 1, HW_C128 = 2 } hw_dtype;

/* Grover (Sec. 3.2) or Fourier: C[j][k] = omega^(jk)/sqrt(d), omega = e^{2 pi i/d},
 * j, k = positions of the vertex's arcs in basis order.  A marked vertex's coin
 * block is -I for both (the search oracle). */
typedef enum { HW_COIN_GROVER = 0, HW_COIN_FOURIER = 1 } hw_coin;

typedef struct hw_graph hw_graph;   /* opaque; owns the device CSR and index tables */

/* Optional knobs.  Pass NULL for defaults, or a struct set up by hw_opts_init. */
typedef struct hw_opts {
    int32_t record_stride;     /* coined/CTQW record: one entry every `stride` steps (>= 1, default 1) */
    int32_t taylor_degree;     /* hw_ctqw_expm: Taylor degree m (0 = chosen for < 2^-60 truncation) */
    int32_t taylor_squarings;  /* hw_ctqw_expm: squarings s (-1 = chosen so ||H dt||_1 / 2^s <= 1/2) */
    int32_t gemm_mode;         /* hw_ctqw_expm, HW_C64: tensor-core precision mode of the powers,
                                  0 = default (fp16 x 2), else as hw_gemm_tc's mode */
    int32_t u_symmetric;       /* hw_ctqw_evolve: 1 = U is complex symmetric (U^T = U, true for
                                  U from hw_ctqw_expm): the 64 x 64 blocks on and above the
                                  diagonal are copied once per call into device scratch
                                  (ceil(n/64) (ceil(n/64) + 1) / 2 blocks of 32 KB, contiguous),
                                  and each application reads every block once for both
                                  triangles (complex64, batch 1; other cases, and a call
                                  that cannot allocate that scratch, use the dense path) */
    int32_t tile;              /* batched Grover kernel launch shape: 0 = autotuned on the first
                                  call per (graph, dtype, batch), which then synchronises the
                                  stream once; 1..12 = register-row kernel with (rows held
                                  in registers, threads per CTA, vertices per warp) in
                                  {8,16} x {128,256} x {1,2,4}, row-major; 13, 14 = TMA-staged
                                  ring kernel with 2 or 1 CTAs per SM */
    int32_t addressing;        /* coined (edge-major path) and sparse-action CTQW on a graph that
                                  hw_graph_structure recognises as a torus or a hypercube:
                                  0 = default, neighbour and reversed-arc positions computed
                                  from the vertex label (no index table is read); 1 = read
                                  the reversal / head tables as for any other graph.  Both
                                  give bit-identical results. */
    int32_t shift;             /* coined walk's shift operator (Sec. 3.2): 0 = flip-flop
                                  S|v,w> = |w,v> (default); 1 = persistent, S|v,w> = |w,u> with
                                  u - w = w - v, the walker keeping its direction (graphs that
                                  hw_graph_structure recognises as a torus only, else HW_EINVAL) */
    int32_t launch_mode;       /* hw_coined_evolve, batch 1, Grover, regular graph of degree 2..8
                                  whose arcs fit the shared memory of one thread-block cluster
                                  (about 60000 arcs in complex128, 110000 in complex64): every
                                  step can run in one launch, the state held in that shared
                                  memory.  0 = default: the cheaper of the two paths for the
                                  call's step count, from their fixed and per-step costs
                                  measured on the first such call per (graph, dtype, shift),
                                  which then synchronises the stream once (under stream
                                  capture: one launch up to 16384 arcs in complex128, 24576 in
                                  complex64); 1 = one launch per step; 2 = one launch
                                  (HW_EUNSUPPORTED when the walk does not fit).  All give
                                  bit-identical results. */
    int32_t taylor_powers;     /* hw_ctqw_expm: how the powers Y^k / k! of Y = H time / 2^s are
                                  formed.  1 = dense n^3 products: FP64 GEMMs for HW_C128,
                                  the tensor cores (opts->gemm_mode) for HW_C64; 2 = sparse x
                                  dense products with the graph (row v of Y Q gathers the rows
                                  of v's neighbours; Y has d << n entries per row), in double
                                  for HW_C128 and in float for HW_C64; 0 = default: 2 for
                                  HW_C128, 1 for HW_C64.  The Taylor sum is in double and the
                                  squarings are dense FP64 GEMMs either way. */
    int32_t gemm_tiles;        /* hw_ctqw_expm, HW_C64 tensor-core powers: 0 = default (2 when
                                  the device runs thread-block clusters of two CTAs, else 1);
                                  1 = one CTA per 128 x 256 output tile; 2 = the two CTAs of a
                                  cluster share a 256 x 256 tile as one pair MMA (each loads
                                  its own A rows and half of the B rows). */
} hw_opts;

/* Fill `opts` with the defaults. */
void hw_opts_init(hw_opts *opts);

/*
 * hw_graph_csr -- build the arc basis of an undirected simple graph (Sec. 3.2).
 *   n        number of vertices (>= 1)
 *   row_ptr  HOST int64[n+1], row_ptr[0] = 0, non-decreasing
 *   col_idx  HOST int32[row_ptr[n]], the adjacency matrix's column indices, any
 *            order inside a row
 * The matrix must be the adjacency matrix of a simple undirected graph:
 * symmetric, 0/1, zero diagonal.  Degree-0 vertices are allowed (their arc
 * block is empty).  The library sorts each row (arc (v, w) then sits at
 * position row_ptr[v] + rank of w among v's neighbours), builds the
 * arc-reversal table rev[a] (the flip-flop shift as an index map:
 * S|v,w> = |w,v> sends arc a to arc rev[a]) and uploads both to the current
 * device.  The call synchronises `stream` before returning.
 *   *out     receives the graph handle, owned by the caller until hw_graph_free.
 * Errors: HW_EINVAL (self-loop, repeated entry, asymmetric, index out of
 * range, malformed row_ptr), HW_EUNSUPPORTED (2|E| >= 2^31), HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_graph_csr(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       void *stream, hw_graph **out);

/*
 * hw_graph_csr_weighted -- hw_graph_csr with a weighted adjacency W for the
 * continuous-time calls: H = -gamma W - sum_{m in M} |m><m| (Sec. 3.1 with A
 * generalised to edge weights).
 *   w_re     HOST double[row_ptr[n]], aligned with col_idx: W[v][col_idx[a]]
 *   w_im     HOST double[row_ptr[n]] or NULL.  NULL: W is real and must be
 *            symmetric, W[u][v] == W[v][u] exactly; else W = w_re + i w_im must
 *            be Hermitian, W[v][u] == conj(W[u][v]) exactly
 * Weights must be finite; a zero weight keeps its arc in the basis.  The
 * structure rules and the arc basis are those of hw_graph_csr.  Weighted
 * graphs serve hw_ctqw_plan, hw_ctqw_expm and hw_ctqw_evolve_sparse (real or
 * complex W; hw_ctqw_expm forms the U of a complex W by the sparse series on
 * the identity's columns); coined walks
 * and served jobs need an unweighted graph (HW_EINVAL / HW_EUNSUPPORTED).
 * Errors: as hw_graph_csr, plus HW_EINVAL for w_re NULL, a non-finite weight
 * or a W that is not symmetric / Hermitian.
 */
hw_status hw_graph_csr_weighted(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                const double *w_re, const double *w_im, void *stream, hw_graph **out);

/*
 * hw_graph_arcs_host -- the same arc basis as hw_graph_csr, computed on the
 * host only (no device is touched).  Same input rules and errors.
 *   row_ptr_out  HOST int32[n+1]           (may be NULL)
 *   head_out     HOST int32[row_ptr[n]]    heads, sorted inside each row (may be NULL)
 *   rev_out      HOST int32[row_ptr[n]]    reversal table (may be NULL)
 * Buffers are caller-owned.
 */
hw_status hw_graph_arcs_host(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             int32_t *row_ptr_out, int32_t *head_out, int32_t *rev_out);

/* Release the graph's device and host memory.  NULL is accepted.  The caller
 * must make sure no enqueued work still uses the graph. */
hw_status hw_graph_free(hw_graph *g);

/*
 * Read-only views of the graph (any output pointer may be NULL):
 *   n, num_arcs         vertex and arc counts
 *   d_row_ptr           DEVICE int32[n+1], first arc of each vertex
 *   d_head              DEVICE int32[num_arcs], head of each arc (sorted inside rows)
 *   d_rev               DEVICE int32[num_arcs], index of the reversed arc
 * The views live as long as the graph.
 */
hw_status hw_graph_info(const hw_graph *g, int64_t *n, int64_t *num_arcs,
                        const int32_t **d_row_ptr, const int32_t **d_head,
                        const int32_t **d_rev);

/*
 * Graph families whose arc basis the library recognises from the adjacency
 * alone (the Grid and Hypercube classes of Sec. 3.1 and 3.2, with their labels):
 *   HW_GRAPH_TORUS      dims = {L1, L2}, L1, L2 >= 3, n = L1 L2: vertex
 *                       v = x L2 + y is adjacent to ((x +- 1) mod L1, y) and
 *                       (x, (y +- 1) mod L2)
 *   HW_GRAPH_HYPERCUBE  dims = {k, 0}, k >= 1, n = 2^k: v is adjacent to
 *                       v XOR 2^b for b = 0..k-1
 *   HW_GRAPH_GENERIC    anything else (dims = {0, 0})
 * The test is exact (every row is compared with the family's neighbour list),
 * so a relabelled torus or hypercube is GENERIC.
 */
typedef enum { HW_GRAPH_GENERIC = 0, HW_GRAPH_TORUS = 1, HW_GRAPH_HYPERCUBE = 2 } hw_graph_kind;

/*
 * hw_graph_structure -- the family of a graph built by hw_graph_csr.
 *   kind   receives an hw_graph_kind
 *   dims   HOST int64[2], receives the family's parameters (may be NULL)
 * Errors: HW_EINVAL (NULL graph or kind).
 */
hw_status hw_graph_structure(const hw_graph *g, int32_t *kind, int64_t *dims);

/*
 * hw_graph_structure_host -- the same test on a host CSR (no device is
 * touched); input rules and errors as hw_graph_arcs_host.
 */
hw_status hw_graph_structure_host(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                  int32_t *kind, int64_t *dims);

/*
 * hw_coined_evolve -- |psi(t)> = (S C)^steps |psi(0)> (Sec. 3.2), coin first,
 * then the flip-flop shift, in every step.
 *   coin, marked     coin kind; HOST int32[n_marked] marked vertex ids (any order,
 *                    no repeats; n_marked = 0 allowed): their coin block is -I
 *   dt               HW_C128 or HW_C64 (amplitudes and coin arithmetic in that
 *                    precision; probabilities are always summed in double)
 *   batch            number of independent states sharing the graph (>= 1)
 *   psi_in           DEVICE [num_arcs][batch] initial states
 *   psi_out          DEVICE [num_arcs][batch] final states; may equal psi_in
 *                    (in place), must not overlap it otherwise
 *   record           DEVICE double[steps / stride][batch] or NULL: entry
 *                    (k-1, b) is the total probability on the marked vertices
 *                    of state b after step k*stride.  Needs n_marked >= 1.
 * Scratch: one state-sized buffer (and a small record buffer) is taken from
 * the stream-ordered allocator and returned on the same stream.
 * A device-side wait that runs out of time (the batched kernel's bounded
 * mbarrier waits) is reported as HW_ETIMEDOUT by the next call on the graph.
 * Errors: HW_EINVAL, HW_EUNSUPPORTED (Fourier coin on a vertex of degree > 4096),
 * HW_ENOMEM, HW_ECUDA, HW_ETIMEDOUT.
 */
hw_status hw_coined_evolve(const hw_graph *g, hw_coin coin, const int32_t *marked,
                           int32_t n_marked, hw_dtype dt, int32_t batch, int64_t steps,
                           const void *psi_in, void *psi_out, double *record,
                           const hw_opts *opts, void *stream);

/*
 * hw_coined_sample -- the states of a coined walk at sampled times: the
 * paper's simulate(range=(start, end, stride)) (Sec. 3.2, 4.2), which returns
 * |psi(k)> for k = start, start + stride, ... < end, k counting walk steps,
 * and its probability_distribution of each of them.
 *   start, end, stride  0 <= start <= end, stride >= 1; the call produces
 *                       R = ceil((end - start) / stride) samples (none when
 *                       end == start)
 *   psi_in              DEVICE [num_arcs][batch], the state at k = 0
 *   states_out          DEVICE [R][num_arcs][batch] or NULL; must not overlap psi_in
 *   prob_out            DEVICE double[R][n][batch] or NULL: per-vertex
 *                       probabilities of each sample (summed in double)
 *   coin, marked, dt, batch, opts as in hw_coined_evolve (no record)
 * Results equal hw_coined_evolve's for the same step counts.  Scratch: up to
 * four state-sized buffers from the stream-ordered allocator.
 * Errors: HW_EINVAL, HW_EUNSUPPORTED, HW_ENOMEM, HW_ECUDA, HW_ETIMEDOUT.
 */
hw_status hw_coined_sample(const hw_graph *g, hw_coin coin, const int32_t *marked, int32_t n_marked,
                           hw_dtype dt, int32_t batch, int64_t start, int64_t end, int64_t stride,
                           const void *psi_in, void *states_out, double *prob_out,
                           const hw_opts *opts, void *stream);

/*
 * hw_ctqw_expm -- U = e^{-i H time} with H = -gamma A - sum_{m in M} |m><m|
 * (Sec. 3.1), dense, by a truncated Taylor series with scaling and squaring:
 * U = (sum_{k<=m} (-i H time/2^s)^k / k!)^(2^s).
 *   U_out    DEVICE [n][n] row-major complex (dt), caller-owned
 *   dt       HW_C128: the powers (H time / 2^s)^k / k! in double precision,
 *            by default as sparse x dense products with the graph;
 *            HW_C64: by default the powers on the tensor cores from 16-bit
 *            slices of their operands (opts->gemm_mode, default fp16 x 2)
 *            with fp32 accumulation; opts->taylor_powers chooses the other
 *            form (dense FP64 GEMMs for HW_C128, sparse x dense products in
 *            float for HW_C64).  Taylor sums and squarings in double; U
 *            rounded to complex64 at the end for HW_C64.
 *   A graph with complex (Hermitian) weights has complex powers of H: U is
 *   then e^{-i H time} applied by hw_ctqw_evolve_sparse's series to all the
 *   columns of the identity at once (batch n), in dt's precision; scratch
 *   five n x n complex buffers.
 * Scratch: four or five n x n real buffers from the stream-ordered allocator.
 * On the tensor-core path the call synchronises `stream` before returning,
 * to report a device-side pipeline timeout of that kernel as HW_ETIMEDOUT.
 * Errors: HW_EINVAL, HW_EUNSUPPORTED (n > 32768), HW_ENOMEM, HW_ECUDA,
 * HW_ETIMEDOUT.
 */
hw_status hw_ctqw_expm(const hw_graph *g, double gamma, const int32_t *marked,
                       int32_t n_marked, double time, hw_dtype dt, void *U_out,
                       const hw_opts *opts, void *stream);

/*
 * hw_ctqw_plan -- the Taylor degree m and squaring count s that hw_ctqw_expm
 * uses by default: with nu = max_v (|gamma| d(v) + [v in M]) |time| (the
 * 1-norm of H time; H is symmetric), s = smallest with nu / 2^s <= 1/2 and
 * m = smallest with theta^(m+1)/(m+1)! < 2^-60, theta = nu / 2^s.  Host only.
 *   degree, squarings   HOST outputs (may be NULL)
 * Errors: HW_EINVAL.
 */
hw_status hw_ctqw_plan(const hw_graph *g, double gamma, const int32_t *marked, int32_t n_marked,
                       double time, int32_t *degree, int32_t *squarings);

/*
 * hw_ctqw_evolve -- psi_out = U^steps psi_in (Sec. 3.1: |psi(k dt)> = U(dt)^k |psi(0)>).
 *   U        DEVICE [n][n] row-major complex (dt), e.g. from hw_ctqw_expm
 *   psi_in   DEVICE [n][batch]; psi_out DEVICE [n][batch], may equal psi_in
 *   marked   HOST int32[n_marked]; record as in hw_coined_evolve
 *            (probability |<m|psi>|^2 summed over the marked vertices).
 * Errors: HW_EINVAL, HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_ctqw_evolve(const void *U, int64_t n, hw_dtype dt, int32_t batch, int64_t steps,
                         const void *psi_in, void *psi_out, const int32_t *marked,
                         int32_t n_marked, double *record, const hw_opts *opts, void *stream);

/*
 * hw_ctqw_sample -- U^k psi_in for k = start, start + stride, ... < end (the
 * paper's simulate(range=...) of a continuous-time walk, Sec. 3.1, 4.1),
 * k counting applications of U = e^{-iH dt}.
 *   U, n, dt, batch, opts  as in hw_ctqw_evolve
 *   start, end, stride     as in hw_coined_sample
 *   states_out             DEVICE [R][n][batch] or NULL; must not overlap psi_in
 *   prob_out               DEVICE double[R][n][batch] or NULL
 * Errors: HW_EINVAL, HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_ctqw_sample(const void *U, int64_t n, hw_dtype dt, int32_t batch, int64_t start, int64_t end,
                         int64_t stride, const void *psi_in, void *states_out, double *prob_out,
                         const hw_opts *opts, void *stream);

/*
 * hw_success_curve -- the success probability of a search at sampled times
 * and the sample where it peaks.  Sec. 3 provides search by walks with marked
 * vertices, evaluated with simulate(range=...) and probability_distribution
 * (Sec. 3.1, 3.2); Sec. 5 plans the success probability and the optimal
 * running time as outputs.  With prob_out of hw_coined_sample or
 * hw_ctqw_sample:
 *   curve[r][b] = sum_{m in M} prob[r][m][b]   (summed in double, ids ascending)
 *   argmax[b]   = the first r with the largest curve[r][b] (the optimal
 *                 running time is start + argmax * stride); NaN entries never
 *                 count; -1 when R = 0 or every entry is NaN
 *   max[b]      = curve[argmax[b]][b] (NaN when argmax[b] = -1)
 *   prob        DEVICE double[R][n][batch] (may be NULL when R = 0)
 *   R, n, batch samples (>= 0), vertices (>= 1), states per sample (>= 1)
 *   marked      HOST int32[n_marked], n_marked >= 1, ids in [0, n), no repeats
 *   curve_out   DEVICE double[R][batch], must not overlap prob (may be NULL when R = 0)
 *   argmax_out  DEVICE int64[batch] or NULL;  max_out DEVICE double[batch] or NULL
 * Buffers are caller-owned and 8-byte aligned.  Up to 16 marked ids travel
 * with the launch; longer lists are uploaded to stream-ordered scratch, which
 * synchronises the stream once.
 * Errors: HW_EINVAL, HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_success_curve(const double *prob, int64_t R, int64_t n, int32_t batch, const int32_t *marked,
                           int32_t n_marked, double *curve_out, int64_t *argmax_out, double *max_out,
                           void *stream);

/*
 * hw_probability -- per-vertex probabilities, summed in double precision.
 *   g != NULL: coined walk, p_v = sum_{w in N(v)} |<v,w|psi>|^2 (Sec. 3.2);
 *              psi is DEVICE [num_arcs][batch]; n is ignored.
 *   g == NULL: continuous-time walk, p_v = |<v|psi>|^2 (Sec. 3.1); psi is
 *              DEVICE [n][batch].
 *   prob_out  DEVICE double[n][batch] (may be NULL if only the norm is wanted)
 *   norm_out  DEVICE double[batch] or NULL: sum_v p_v per state
 * Errors: HW_EINVAL, HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_probability(const hw_graph *g, int64_t n, hw_dtype dt, int32_t batch,
                         const void *psi, double *prob_out, double *norm_out, void *stream);

/*
 * hw_probability_noalloc -- the same results as hw_probability, for callers
 * that cannot allocate device memory during a call: programs running under a
 * fixed, pre-reserved memory budget that must not meet out-of-memory halfway
 * through a request, and platforms without the stream-ordered allocator
 * (cudaDevAttrMemoryPoolsSupported == 0).  The paper has no counterpart; it
 * is a deployment variant of hw_probability.
 * It allocates nothing: the norm's partial sums use a static device array
 * built into the library (1184 x 64 doubles, about 0.6 MB, held on every
 * device that loads the library until the process exits).
 *   Arguments, layouts and results as hw_probability.
 *   Limit: batch <= 64 when norm_out != NULL (HW_EINVAL otherwise).
 * The array is device memory of the library's module: it is committed when
 * the module is loaded on a device, which with CUDA's lazy module loading
 * can be this entry point's first call there.  That first call also looks up
 * the array's device address (cudaGetSymbolAddress) with the device current.
 * So make one call per device at start-up, before the memory budget is
 * reserved and before any stream capture; later calls allocate nothing.  The
 * address is cached per device for the life of the process: resetting a
 * device (cudaDeviceReset) while the library is loaded is not supported.
 * All calls on a device share the one array, so calls whose work overlaps on
 * the GPU (different streams, no ordering) race on it and must be serialised
 * by the caller.
 * Errors: HW_EINVAL, HW_EUNSUPPORTED (device index >= 64), HW_ECUDA.
 */
hw_status hw_probability_noalloc(const hw_graph *g, int64_t n, hw_dtype dt, int32_t batch,
                                 const void *psi, double *prob_out, double *norm_out, void *stream);

/*
 * hw_gemm_tc -- C = A B^T on the tensor cores (tcgen05, 16-bit inputs, fp32
 * accumulation) with each fp32 operand split into 16-bit slices; `mode`:
 *   1 = bf16 x 1 (one product, ~2^-8),   2 = bf16 x 2 (3 products, ~2^-16),
 *   3 = bf16 x 3 (6 products, ~2^-24),   4 = fp16 x 2 (3 products, ~2^-22;
 *   each operand is first scaled by a power of two that puts its maximum in
 *   [1/2, 1], so errors are relative to the operand's largest entry).
 * This is the contraction behind the complex64 Taylor series of
 * hw_ctqw_expm (there A = Y^(k-1)/(k-1)!, B = Y, symmetric), exposed for tests
 * and measurement.
 *   A  DEVICE float[m][k] row-major;  B  DEVICE float[n][k] row-major
 *   C  DEVICE float[m][n] row-major, caller-owned
 * Scratch (slices, 3(m+n)k x 2 bytes) comes from the stream-ordered
 * allocator.  The call synchronises `stream` before returning, to report a
 * device-side pipeline timeout as HW_ETIMEDOUT.
 * A, B and C must be device memory of the current device (HW_EINVAL otherwise).
 * Errors: HW_EINVAL, HW_EUNSUPPORTED (not an sm_103 device), HW_ENOMEM,
 * HW_ECUDA, HW_ETIMEDOUT.
 */
hw_status hw_gemm_tc(int64_t m, int64_t n, int64_t k, const float *A, const float *B, float *C,
                     int32_t mode, void *stream);

/*
 * hw_ctqw_evolve_sparse -- psi_out = (e^{-iH time})^steps psi_in (Sec. 3.1)
 * without forming U: each application sums the exponential series of
 * H time/q on the CSR, q = 2^s parts, degree m, with (m, s) from
 * hw_ctqw_plan (opts may override).  Suited to graphs too large for a dense
 * U.  Arguments, layouts, record and errors as hw_ctqw_evolve, with the graph
 * and (gamma, marked) of hw_ctqw_expm.  Scratch: four state-sized buffers.
 */
hw_status hw_ctqw_evolve_sparse(const hw_graph *g, double gamma, const int32_t *marked, int32_t n_marked,
                                double time, hw_dtype dt, int32_t batch, int64_t steps,
                                const void *psi_in, void *psi_out, double *record,
                                const hw_opts *opts, void *stream);

/* ------------------------------------------------------------------ serving
 * Continuous batching of walk jobs on one GPU (no counterpart in the paper,
 * which evolves one walk per call).  Jobs wait in a queue until a slot and
 * device memory in the server's arena are free; every admitted job keeps its
 * states on the device, and each hw_server_run round advances every resident
 * job by K sub-steps (a coined step, or one series term of e^{-iH dt}) with
 * one multi-job kernel launch per sub-step, K launches replayed as one CUDA
 * graph.  CTQW jobs whose state and two series terms fit one CTA's shared
 * memory advance instead by whole walk steps in a kernel beside that graph,
 * between 1 and K steps per round, as many as keep its time close to the
 * graph's (measured on earlier rounds).  Each job starts from the uniform state over its basis (all arcs for
 * a coined walk, all vertices for a CTQW) and returns its probabilities
 * (Sec. 3.1 / 3.2, summed in double) and, with marked vertices, the total
 * marked probability after every step.  A job's result does not depend on
 * the other jobs in the mix.
 */
typedef enum { HW_JOB_COINED = 0, HW_JOB_CTQW = 1 } hw_job_kind;

typedef struct hw_job {
    const hw_graph *graph;   /* resident graph; coined jobs need a regular graph */
    int32_t kind;            /* hw_job_kind; coined jobs use the Grover coin */
    int32_t dt;              /* HW_C64 or HW_C128 */
    int64_t steps;           /* walk steps / applications of e^{-iH time} (>= 1) */
    const int32_t *marked;   /* HOST ids, copied at submit; 0..4 vertices */
    int32_t n_marked;
    int32_t reserved;
    double gamma;            /* CTQW: H = -gamma A - sum_m |m><m| */
    double time;             /* CTQW: time per application */
} hw_job;

typedef struct hw_server hw_server;

/*
 * hw_server_create -- reserve the device arena (arena_bytes, cudaMalloc once),
 * a pinned host arena for results (host_bytes), a job table of max_jobs
 * slots, and capture the K-launch graph (K = substeps_per_round).  The server
 * runs on a stream of its own; `stream` is unused (pass NULL).
 * Errors: HW_EINVAL, HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_server_create(int64_t arena_bytes, int32_t max_jobs, int32_t substeps_per_round,
                           int64_t host_bytes, void *stream, hw_server **out);

/* Queue a job; *job_id receives its id.  HW_ENOMEM if it could never fit the
 * arenas; HW_EUNSUPPORTED for a coined job on an irregular graph. */
hw_status hw_server_submit(hw_server *s, const hw_job *job, int64_t *job_id);

/*
 * One scheduling round: retire jobs whose last sub-step has run (their
 * results are produced and copied back asynchronously), release the memory
 * of retired jobs whose copies have completed, admit queued jobs first come
 * first served while a slot and arena memory are free, and launch K
 * sub-steps of all resident jobs.  Does not wait for the GPU, except for the
 * previous round's table upload.  *n_completed (may be NULL) receives the
 * number of jobs that became collectable in this round.
 */
hw_status hw_server_run(hw_server *s, int32_t *n_completed);

/* Ids of jobs that became collectable since the last poll (up to max_ids). */
hw_status hw_server_poll(hw_server *s, int64_t *ids, int32_t max_ids, int32_t *n_ids);

/*
 * Copy a finished job's results to HOST buffers and forget the job:
 *   prob      double[n] (n_prob must equal the graph's vertex count), or NULL
 *   record    double[steps] (needs a marked vertex), or NULL
 *   latency_s seconds from submit to the round that saw the results ready, or NULL
 */
hw_status hw_server_result(hw_server *s, int64_t job_id, double *prob, int64_t n_prob, double *record,
                           int64_t n_record, double *latency_s);

/* Occupancy counters (any output may be NULL). */
hw_status hw_server_stats(const hw_server *s, int64_t *queued, int64_t *resident, int64_t *arena_used,
                          int64_t *ticks);

/* Wait for the server's stream and free everything it holds. */
hw_status hw_server_destroy(hw_server *s);

/* Scratch buffers of every call come from a stream-ordered pool per device
   that keeps freed memory mapped for the next call.  This returns the pool's
   unused memory to the driver (HW_ECUDA on a driver error).  Call it only
   when no library call is in flight on any stream. */
hw_status hw_trim_scratch(void);

/* Message for the last failed call on this thread ("" if none). */
const char *hw_last_error(void);

/* Library version string. */
const char *hw_version(void);

/*
 * hw_measure_fp64 -- measured double-precision FMA throughput of the current
 * device, in operations per second (one FMA, add or multiply = one operation),
 * for the roofline of kernels bound by FP64 arithmetic.  Runs a grid of
 * independent FMA chains for a few milliseconds on `stream` and synchronises
 * it.  Errors: HW_EINVAL (NULL output), HW_ECUDA.
 */
hw_status hw_measure_fp64(double *ops_per_s, void *stream);

/*
 * hw_measure_l2 -- measured copy bandwidth (read + write bytes per second,
 * reported in GB/s) of a 32 MB working set that stays in the L2 cache, for the
 * roofline of kernels whose data fits in L2.  Synchronises `stream`.
 * Errors: HW_EINVAL (NULL output), HW_ENOMEM, HW_ECUDA.
 */
hw_status hw_measure_l2(double *gbs, void *stream);

/*
 * hw_check_device_wait -- the failure path of the device-side waits, for
 * tests.  Launches on `stream` one CTA that takes the bounded mbarrier wait
 * of the one-launch walks (hw_coined_evolve, launch_mode 2) on a barrier that
 * no copy completes: after the wait's budget (2 s) it gives up and sets g's
 * device error word, as a walk whose peer CTA never answers does.  The next
 * hw_coined_evolve on g then returns HW_ETIMEDOUT and clears the word; the
 * context stays usable.  The CTA occupies one SM for the budget.  Nothing
 * faults and nothing waits without a limit.
 * Errors: HW_EINVAL (NULL graph), HW_ECUDA.
 */
hw_status hw_check_device_wait(const hw_graph *g, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HIPERWALK_B300_H */
