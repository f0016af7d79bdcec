// Serving: continuous batching of walk jobs on one GPU.
//
// Jobs (a coined walk or a continuous-time walk on a resident graph, any
// step count, complex64 or complex128, up to 4 marked vertices) are queued by
// hw_server_submit and admitted as soon as a slot and device memory (a
// first-fit arena reserved at creation) are free.  Every resident job's
// buffers stay on the device; each scheduling round launches, as one CUDA
// graph, K sub-steps of a single multi-job kernel that advances every
// resident job by one sub-step (a coined walk step, or one Taylor term of
// e^{-iH dt}), reading a device job table and tile list, so jobs that join or
// leave between rounds never require re-capturing the graph.  Finished jobs
// are retired: probabilities (double sums) and the marked-probability record
// are produced on the device and copied to a pinned host arena; the caller
// collects them with hw_server_result.
//
// A continuous-time job whose three working vectors fit in one CTA's shared
// memory (complex64 up to 8192 vertices, complex128 up to 4096) is "local":
// a CTA of its own keeps the state and the series terms in shared memory and
// advances the job by whole walk steps, with block barriers between the
// Taylor terms instead of one launch per term.  These CTAs (k_serve_local,
// one launch per round) run on a second stream, beside the round's graph of
// k_serve_step sub-steps, L walk steps per round: L follows the measured
// times of the two branches, so that the local jobs (which advance whole
// steps) do not hold back the tiled CTQW jobs (which advance one term per
// sub-step) and are not held back by a round of idle sub-steps either.
//
// Each job's arithmetic depends only on its own data and a fixed per-vertex
// order, so its result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "cache_hints.cuh"
#include "family.cuh"
#include "internal.h"
#include "sum4.cuh"

namespace {

constexpr int kServeThreads = 256;
// CTQW tiles: 16 KiB of a job's four state-sized buffers each, one or two
// vertices per thread (a term's neighbour gathers are latency-bound, so small
// jobs need many CTAs)
constexpr int kTileVerticesC64 = 512, kTileVerticesC128 = 256;
constexpr int kServeTileArcs = 1024;  // coined tiles: whole vertices, at most this many arcs
constexpr int kMaxServeMarked = 4;
constexpr int kServeMaxDeg = 32;           // series degree bound (hw_ctqw_plan gives m <= 30)
// a CTQW job's coefficient tables: c_k and cg_k for k <= kServeMaxDeg, double then float
constexpr size_t kCoefBytes = ((2 * (kServeMaxDeg + 1) * (sizeof(double) + sizeof(float))) + 255) & ~size_t(255);
constexpr int kLocalBytes = 3 * 8192 * 8;  // shared memory of a local CTQW job: state and two terms
constexpr int kLocalThreads = 512;
constexpr int kLocalCtas = 64;             // local jobs advanced at once (each CTA takes one SM's memory)

struct SJob {
    const int32_t *row_ptr;
    const int32_t *head;
    const int32_t *rev;
    const int32_t *revE;     // coined: edge-major reversal table (states are edge-major while resident)
    void *X[2];              // state ping-pong
    void *T[2];              // CTQW series terms
    double *rec;             // [steps][n_marked] per-marked partials (nullptr if no marks)
    int64_t n;
    int64_t start_tick;
    int64_t total_subs;
    double two_over_d;
    float two_over_d_f;
    int32_t pad0;
    double gamma;
    double tau;
    // CTQW term k = 1..m: t_k = (-(cg_k) s_y - c_k q_y, cg_k s_x + c_k q_x) with
    // c_k = tau / k, cg_k = c_k gamma (s the neighbour sum of t_{k-1}, q its
    // own entry on a marked vertex), in both precisions: tables in the job's
    // device memory, written once at admission (the job table itself stays
    // small, since it is uploaded whenever the resident set changes)
    const double *cd, *cgd;
    const float *cf, *cgf;
    int32_t kind;            // 0 coined, 1 CTQW
    int32_t dt;              // HW_C64 / HW_C128
    int32_t d;               // coined: the graph's (regular) degree
    int32_t m;               // CTQW: series degree
    int32_t q;               // CTQW: parts per application
    int32_t n_marked;
    int32_t marked[kMaxServeMarked];
    int32_t local;           // CTQW job run by one CTA from shared memory
    int32_t fam;             // coined: hw_graph_kind of the graph (positions from labels when not generic)
    int32_t fdim0, fdim1;    // torus L1, L2 / hypercube k
};

struct Tile {
    int32_t job, v0, v1, pad;
};

template <typename R> struct CxS;
template <> struct CxS<double> { using T = double2; };
template <> struct CxS<float> { using T = float2; };

// the job's constants in the kernel's precision (no per-thread conversion)
__device__ __forceinline__ void term_coef(const SJob &J, int k, double &c, double &cg) { c = J.cd[k]; cg = J.cgd[k]; }
__device__ __forceinline__ void term_coef(const SJob &J, int k, float &c, float &cg) { c = J.cf[k]; cg = J.cgf[k]; }
__device__ __forceinline__ double grover_weight(const SJob &J, double) { return J.two_over_d; }
__device__ __forceinline__ float grover_weight(const SJob &J, float) { return J.two_over_d_f; }

__device__ __forceinline__ int job_marked(const SJob &J, int v)
{
    for (int i = 0; i < J.n_marked; ++i)
        if (J.marked[i] == v) return i;
    return -1;
}

// one Taylor term of a CTQW job for vertex v, sub-step index ls
template <typename R>
__device__ void serve_ctqw(const SJob &J, int64_t ls, int v)
{
    using V = typename CxS<R>::T;
    const int64_t per = int64_t(J.q) * J.m;
    int64_t rem, kk;
    const int64_t w = idx_div(ls, per, rem);
    const int64_t r = idx_div(rem, J.m, kk);
    const int k = int(kk) + 1;
    const int cur = int((w * J.q + r) & 1);
    const V *__restrict__ x = static_cast<const V *>(J.X[cur]);
    const V *__restrict__ tin = (k == 1) ? x : static_cast<const V *>(J.T[(k - 1) & 1]);
    V *__restrict__ tout = static_cast<V *>(J.T[k & 1]);
    V *__restrict__ acc = static_cast<V *>(J.X[1 - cur]);
    R sx = 0, sy = 0;
    const int a0 = J.row_ptr[v], a1 = J.row_ptr[v + 1];
#pragma unroll 4
    for (int a = a0; a < a1; ++a) {
        const V q = tin[J.head[a]];
        sx += q.x;
        sy += q.y;
    }
    R c, cg;
    term_coef(J, k, c, cg);
    const int mi = job_marked(J, v);
    V t;
    if (mi >= 0) {
        const V q = tin[v];
        t.x = -fma(cg, sy, c * q.y);
        t.y = fma(cg, sx, c * q.x);
    } else {
        t.x = -(cg * sy);
        t.y = cg * sx;
    }
    tout[v] = t;
    const V base = (k == 1) ? x[v] : acc[v];
    V o;
    o.x = base.x + t.x;
    o.y = base.y + t.y;
    acc[v] = o;
    if (mi >= 0 && J.rec && k == J.m && r == J.q - 1)
        J.rec[w * J.n_marked + mi] = double(o.x) * double(o.x) + double(o.y) * double(o.y);
}

// One coined step of the tile's vertices in the edge-major layout E[j][v]
// (thread per vertex, degree D known at compile time): the job's pointers and
// marked vertices are read once per tile, each thread loads its vertex's D
// arcs (D row segments across the warp) and reversal entries (none on a
// recognised torus or hypercube: positions from the label) before any
// arithmetic.  The Grover sum is the single-walk kernels': in arc order from
// arc 0 (complex128: integer group sums), one FMA per component.
template <typename R, int D>
__device__ void serve_coined_em(const SJob &Jg, int64_t w, int v0, int v1)
{
    using V = typename CxS<R>::T;
    const V *__restrict__ in = static_cast<const V *>(Jg.X[w & 1]);
    V *__restrict__ out = static_cast<V *>(Jg.X[(w + 1) & 1]);
    const int32_t *__restrict__ revE = Jg.revE;
    const int64_t n = Jg.n;
    const int nm = Jg.n_marked;
    int mk[kMaxServeMarked];
#pragma unroll
    for (int i = 0; i < kMaxServeMarked; ++i) mk[i] = (i < nm) ? Jg.marked[i] : -1;
    double *rec = Jg.rec;
    const R f = grover_weight(Jg, R(0));
    const bool torus = D == 4 && Jg.fam == HW_GRAPH_TORUS;   // uniform across the tile
    const bool cube = Jg.fam == HW_GRAPH_HYPERCUBE;
    for (int v = v0 + int(threadIdx.x); v < v1; v += blockDim.x) {
        V p[D];
        int r[D];
        if constexpr (D == 4) {
            if (torus) torus_targets<kAddrTorusFF>(TorusVertex(int64_t(v), n, Jg.fdim0, Jg.fdim1), n, r);
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            p[j] = in[j * n + v];
            if (!torus && !cube) r[j] = revE[j * n + v];
        }
        // hypercube: each output's position is computed where it is stored
        CubeWalk cw(v, D);
        int mi = -1;
#pragma unroll
        for (int i = 0; i < kMaxServeMarked; ++i)
            if (mk[i] == v) mi = i;
        if (mi >= 0) {
            if (rec && w >= 1) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < D; ++j) acc += double(p[j].x) * double(p[j].x) + double(p[j].y) * double(p[j].y);
                rec[(w - 1) * nm + mi] = acc;
            }
#pragma unroll
            for (int j = 0; j < D; ++j) {
                V c;
                c.x = -p[j].x;
                c.y = -p[j].y;
                out[cube ? cw.target(cw.next_bit(), n) : r[j]] = c;
            }
            continue;
        }
        R sx, sy;
        if constexpr (sizeof(R) == 8) {   // complex128: integer group sums (sum4.cuh)
            sum4::grouped_sum2_fixed<D>(p, sx, sy);
        } else {
            sx = p[0].x;
            sy = p[0].y;
#pragma unroll
            for (int j = 1; j < D; ++j) {
                sx += p[j].x;
                sy += p[j].y;
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V c;
            c.x = fma(f, sx, -p[j].x);
            c.y = fma(f, sy, -p[j].y);
            out[cube ? cw.target(cw.next_bit(), n) : r[j]] = c;
        }
    }
}

// The same for any degree: a pass for the sum and a pass for the outputs.
template <typename R>
__device__ void serve_coined_em_rt(const SJob &Jg, int64_t w, int v0, int v1)
{
    using V = typename CxS<R>::T;
    const V *__restrict__ in = static_cast<const V *>(Jg.X[w & 1]);
    V *__restrict__ out = static_cast<V *>(Jg.X[(w + 1) & 1]);
    const int32_t *__restrict__ revE = Jg.revE;
    // row j of vertex v at j n + v < 2|E| < 2^31 (the graph's limit): 32-bit indices
    const int n = int(Jg.n);
    const int d = Jg.d;
    const bool cube = Jg.fam == HW_GRAPH_HYPERCUBE;   // uniform across the tile
    const int nm = Jg.n_marked;
    int mk[kMaxServeMarked];
#pragma unroll
    for (int i = 0; i < kMaxServeMarked; ++i) mk[i] = (i < nm) ? Jg.marked[i] : -1;
    double *rec = Jg.rec;
    const R f = grover_weight(Jg, R(0));
    for (int v = v0 + int(threadIdx.x); v < v1; v += blockDim.x) {
        int mi = -1;
#pragma unroll
        for (int i = 0; i < kMaxServeMarked; ++i)
            if (mk[i] == v) mi = i;
        if (mi >= 0) {
            if (rec && w >= 1) {
                double acc = 0.0;
                for (int j = 0; j < d; ++j) {
                    const V p = in[j * n + v];
                    acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
                }
                rec[(w - 1) * nm + mi] = acc;
            }
            CubeWalk cw(v, d);
            for (int j = 0; j < d; ++j) {
                const V p = in[j * n + v];
                V c;
                c.x = -p.x;
                c.y = -p.y;
                out[cube ? cw.target(cw.next_bit(), n) : revE[j * n + v]] = c;
            }
            continue;
        }
        R sx, sy;
        if constexpr (sizeof(R) == 8) {   // complex128: integer group sums (sum4.cuh)
            // the rows are read again below: keep them in L2
            const uint64_t keep = l2_evict_last_policy();
            sum4::grouped_sum2(d, [&](int j) { return ld_keep(in + j * n + v, keep); }, sx, sy);
        } else {
            const V p0 = in[v];
            sx = p0.x;
            sy = p0.y;
#pragma unroll 4
            for (int j = 1; j < d; ++j) {
                const V p = in[j * n + v];
                sx += p.x;
                sy += p.y;
            }
        }
        CubeWalk cw(v, d);
        if constexpr (sizeof(R) == 8) {
            // complex128: the rows again, last first and as their last use,
            // with streaming stores (the plain path's k_coined_em_rt does the same)
#pragma unroll 4
            for (int j = d - 1; j >= 0; --j) {
                const V p = __ldcs(in + j * n + v);
                V c;
                c.x = fma(f, sx, -p.x);
                c.y = fma(f, sy, -p.y);
                __stcs(out + (cube ? cw.target(cw.prev_bit(), n) : revE[j * n + v]), c);
            }
        } else {
#pragma unroll 4
            for (int j = 0; j < d; ++j) {
                const V p = in[j * n + v];
                V c;
                c.x = fma(f, sx, -p.x);
                c.y = fma(f, sy, -p.y);
                out[cube ? cw.target(cw.next_bit(), n) : revE[j * n + v]] = c;
            }
        }
    }
}

// Hypercube degrees whose rows are held in registers (serve_coined_em<R, d>)
// rather than read twice: complex64 16..20, where the single-walk
// k_coined_em_cube was measured faster than the two-pass kernel, and
// complex128 9..12 (that kernel wins up to 16, but here every path shares one
// kernel's registers, and 13..16 complex128 rows push it into spills).
template <typename R> __device__ __forceinline__ bool serve_cube_regs(int d)
{
    return sizeof(R) == 8 ? (d >= 9 && d <= 12) : (d >= 16 && d <= 20);
}

template <typename R>
__device__ void serve_coined_cube(const SJob &J, int64_t w, int v0, int v1)
{
    if constexpr (sizeof(R) == 8) {
        switch (J.d) {
        case 9: serve_coined_em<R, 9>(J, w, v0, v1); break;
        case 10: serve_coined_em<R, 10>(J, w, v0, v1); break;
        case 11: serve_coined_em<R, 11>(J, w, v0, v1); break;
        default: serve_coined_em<R, 12>(J, w, v0, v1); break;
        }
    } else {
        switch (J.d) {
        case 16: serve_coined_em<R, 16>(J, w, v0, v1); break;
        case 17: serve_coined_em<R, 17>(J, w, v0, v1); break;
        case 18: serve_coined_em<R, 18>(J, w, v0, v1); break;
        case 19: serve_coined_em<R, 19>(J, w, v0, v1); break;
        default: serve_coined_em<R, 20>(J, w, v0, v1); break;
        }
    }
}

// Walk steps w0 .. w0 + ns - 1 (each q parts of m Taylor terms) of a local
// CTQW job: the state (acc) and the terms (T0, T1) live in shared memory for
// all of them.  The arithmetic of every term is serve_ctqw's, in the same
// order: t_1 is formed from the part's start state, and acc takes t_1, t_2,
// ... one at a time.
template <typename R>
__device__ void serve_ctqw_local(const SJob &J, int64_t w0, int ns, unsigned char *smem)
{
    using V = typename CxS<R>::T;
    const int n = int(J.n);
    V *acc = reinterpret_cast<V *>(smem);
    V *T0 = acc + n;
    V *T1 = T0 + n;
    const V *__restrict__ in = static_cast<const V *>(J.X[w0 & 1]);
    V *__restrict__ out = static_cast<V *>(J.X[(w0 + ns) & 1]);
    for (int v = threadIdx.x; v < n; v += blockDim.x) acc[v] = in[v];
    __syncthreads();
    for (int64_t w = w0; w < w0 + ns; ++w) {
        for (int r = 0; r < J.q; ++r) {
            for (int k = 1; k <= J.m; ++k) {
                const V *tin = (k == 1) ? acc : ((k & 1) ? T1 : T0);   // t_{k-1}
                V *tout = (k & 1) ? T0 : T1;                            // t_k
                R c, cg;
                term_coef(J, k, c, cg);
                for (int v = threadIdx.x; v < n; v += blockDim.x) {
                    R sx = 0, sy = 0;
                    for (int a = J.row_ptr[v]; a < J.row_ptr[v + 1]; ++a) {
                        const V q = tin[J.head[a]];
                        sx += q.x;
                        sy += q.y;
                    }
                    V t;
                    if (job_marked(J, v) >= 0) {
                        const V q = tin[v];
                        t.x = -fma(cg, sy, c * q.y);
                        t.y = fma(cg, sx, c * q.x);
                    } else {
                        t.x = -(cg * sy);
                        t.y = cg * sx;
                    }
                    tout[v] = t;
                    // acc takes t_{k-1} now (t_1 only once every gather of the
                    // start state is done, i.e. at k = 2) and t_m at the end
                    if (k >= 2) {
                        V o = acc[v];
                        const V tp = tin[v];
                        o.x = o.x + tp.x;
                        o.y = o.y + tp.y;
                        if (k == J.m) {
                            o.x = o.x + t.x;
                            o.y = o.y + t.y;
                        }
                        acc[v] = o;
                    }
                }
                __syncthreads();
                if (k == 1 && J.m == 1) {   // a single term: acc = x + t_1 after every gather
                    for (int v = threadIdx.x; v < n; v += blockDim.x) {
                        V o = acc[v];
                        o.x = o.x + T0[v].x;
                        o.y = o.y + T0[v].y;
                        acc[v] = o;
                    }
                    __syncthreads();
                }
            }
        }
        if (J.rec)
            for (int i = threadIdx.x; i < J.n_marked; i += blockDim.x) {
                const V o = acc[J.marked[i]];
                J.rec[w * J.n_marked + i] = double(o.x) * double(o.x) + double(o.y) * double(o.y);
            }
    }
    for (int v = threadIdx.x; v < n; v += blockDim.x) out[v] = acc[v];
}

// Up to L walk steps of every resident local CTQW job, a CTA per job;
// prog[slot] counts the steps a job has done (the host keeps the same count).
__global__ void __launch_bounds__(kLocalThreads, 1)
k_serve_local(const SJob *__restrict__ jobs, const int *__restrict__ local, const int *__restrict__ nlocal,
              int64_t *__restrict__ prog, int L)
{
    extern __shared__ __align__(16) unsigned char lsmem[];
    const int nl = *nlocal;
    for (int i = blockIdx.x; i < nl; i += gridDim.x) {
        const int slot = local[i];
        const SJob &J = jobs[slot];
        const int64_t w0 = prog[slot];
        const int64_t w1 = std::min<int64_t>(J.total_subs, w0 + L);
        if (w1 <= w0) continue;   // uniform over the CTA
        if (J.dt == HW_C128) serve_ctqw_local<double>(J, w0, int(w1 - w0), lsmem);
        else serve_ctqw_local<float>(J, w0, int(w1 - w0), lsmem);
        __syncthreads();   // every thread has read prog[slot]; the next job reuses the shared memory
        if (threadIdx.x == 0) prog[slot] = w1;
    }
}

// One sub-step of every resident job.  Tiles are (job, vertex range); the
// grid loops over them, so the launch shape never depends on the job mix.
__global__ void __launch_bounds__(kServeThreads)
k_serve_step(const SJob *__restrict__ jobs, const Tile *__restrict__ tiles, const int *__restrict__ ntiles,
             const int64_t *__restrict__ tick, int sub)
{
    const int nt = *ntiles;
    const int64_t now = *tick + sub;   // the tick advances once per round, after all its sub-steps
    pdl_trigger();
    pdl_wait();   // the previous sub-step's states
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SJob &J = jobs[tl.job];
        const int64_t local = now - J.start_tick;
        if (local < 0 || local >= J.total_subs) continue;   // uniform over the CTA
        if (J.kind == 0) {
            // coined, edge-major: unrolled for the common degrees and for the
            // hypercube degrees where rows held in registers beat two passes,
            // two passes otherwise
            const bool cube = J.fam == HW_GRAPH_HYPERCUBE;
            if (J.dt == HW_C128) {
                if (J.d == 3) serve_coined_em<double, 3>(J, local, tl.v0, tl.v1);
                else if (J.d == 4) serve_coined_em<double, 4>(J, local, tl.v0, tl.v1);
                else if (J.d == 8) serve_coined_em<double, 8>(J, local, tl.v0, tl.v1);
                else if (cube && serve_cube_regs<double>(J.d)) serve_coined_cube<double>(J, local, tl.v0, tl.v1);
                else serve_coined_em_rt<double>(J, local, tl.v0, tl.v1);
            } else {
                if (J.d == 3) serve_coined_em<float, 3>(J, local, tl.v0, tl.v1);
                else if (J.d == 4) serve_coined_em<float, 4>(J, local, tl.v0, tl.v1);
                else if (J.d == 8) serve_coined_em<float, 8>(J, local, tl.v0, tl.v1);
                else if (cube && serve_cube_regs<float>(J.d)) serve_coined_cube<float>(J, local, tl.v0, tl.v1);
                else serve_coined_em_rt<float>(J, local, tl.v0, tl.v1);
            }
        } else {
            for (int v = tl.v0 + threadIdx.x; v < tl.v1; v += blockDim.x) {
                if (J.dt == HW_C128) serve_ctqw<double>(J, local, v);
                else serve_ctqw<float>(J, local, v);
            }
        }
    }
}

__global__ void k_serve_tick(int64_t *tick, int K) { *tick += K; }

template <typename V>
__global__ void k_fill(V *x, int64_t count, double value)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        V v;
        v.x = decltype(v.x)(value);
        v.y = 0;
        x[i] = v;
    }
}

// record[w] = sum over marked of the partials, in marked order
__global__ void k_serve_record(const double *part, int n_marked, int64_t steps, double *record)
{
    const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (w >= steps) return;
    double s = 0.0;
    for (int i = 0; i < n_marked; ++i) s += part[w * n_marked + i];
    record[w] = s;
}

// First-fit allocator over one reserved region (device or pinned host).
class Arena {
public:
    void init(char *base, size_t size)
    {
        base_ = base;
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    char *alloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                live_[off] = bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(char *p)
    {
        if (!p) return;
        const size_t off = size_t(p - base_);
        auto lv = live_.find(off);
        if (lv == live_.end()) return;
        size_t len = lv->second;
        live_.erase(lv);
        used_ -= len;
        size_t start = off;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && nx->first == off + len) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

private:
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_, live_;
};

enum JobState { QUEUED, RESIDENT, RETIRING, DONE };

struct Job {
    int64_t id;
    hw_job spec;
    std::vector<int32_t> marked;
    JobState state = QUEUED;
    int slot = -1;
    char *dev = nullptr;        // arena block: states, terms, record partials, prob
    char *host = nullptr;       // pinned result block: prob, record
    int64_t n = 0, dim = 0;
    int64_t total_subs = 0;
    int64_t end_tick = 0;
    int32_t m = 1, q = 1;
    size_t dev_bytes = 0, host_bytes = 0;
    bool local = false;         // CTQW job run from shared memory by k_serve_local
    int64_t lprog = 0;          // local job: walk steps launched so far
    cudaEvent_t done_ev = nullptr;
    double t_submit = 0, t_done = 0;
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct hw_server {
    int device = -1;
    cudaStream_t st = nullptr;
    int max_jobs = 0;
    int K = 8;
    char *dev_base = nullptr;
    char *host_base = nullptr;
    Arena dev_arena, host_arena;
    SJob *d_jobs = nullptr, *h_jobs = nullptr;       // device table + pinned mirror
    char *h_coef = nullptr;                           // pinned staging of each slot's CTQW coefficients
    Tile *d_tiles = nullptr, *h_tiles = nullptr;
    int *d_ntiles = nullptr, *h_ntiles = nullptr;
    int *d_local = nullptr, *h_local = nullptr;       // slots of the resident local CTQW jobs
    int *d_nlocal = nullptr, *h_nlocal = nullptr;
    cudaStream_t st2 = nullptr;                       // the local CTQW jobs' branch of a round
    int64_t *d_lprog = nullptr;                       // steps done by the local job in each slot
    int L = 1;                                        // local steps per round
    static constexpr int kTimeSets = 8;               // rounds of branch timings in flight
    cudaEvent_t tev[kTimeSets][4] = {};               // graph start/end, local start/end
    bool tlocal[kTimeSets] = {};
    int64_t round_no = 0;
    int64_t *d_tick = nullptr;
    int64_t tick = 0;
    int max_tiles = 0;
    bool table_dirty = true;
    bool upload_pending = false;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    std::vector<int> free_slots;
    std::map<int64_t, Job> jobs;
    std::deque<int64_t> queue;
    std::vector<int64_t> resident;
    std::vector<int64_t> completed;   // not yet polled
    int64_t next_id = 1;
    cudaEvent_t upload_ev = nullptr;  // the pinned table mirror is free to rewrite after this
};

static hw_status server_capture(hw_server *s)
{
    cudaGraph_t g = nullptr;
    hw_status st = hw_cuda(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st != HW_OK) return st;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    const int smem = 0;
    st = hw_cuda(cudaFuncSetAttribute(k_serve_local, cudaFuncAttributeMaxDynamicSharedMemorySize, kLocalBytes),
                     "cudaFuncSetAttribute(k_serve_local)");
    if (st != HW_OK) {
        cudaStreamEndCapture(s->st, &g);
        if (g) cudaGraphDestroy(g);
        return st;
    }
    // the graph of a round: the K tiled sub-steps (chained by programmatic
    // dependent launch), then the tick; the local CTQW jobs run beside it
    // (hw_server_run)
    for (int k = 0; k < s->K; ++k)
        launch_pdl(k_serve_step, dim3(sms * 6), dim3(kServeThreads), smem, s->st, (const SJob *)s->d_jobs,
                   (const Tile *)s->d_tiles, (const int *)s->d_ntiles, (const int64_t *)s->d_tick, k);
    k_serve_tick<<<1, 1, 0, s->st>>>(s->d_tick, s->K);
    st = hw_cuda(cudaStreamEndCapture(s->st, &g), "end capture");
    if (st != HW_OK) return st;
    st = hw_cuda(cudaGraphInstantiate(&s->graph, g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    return st;
}

extern "C" hw_status hw_server_create(int64_t arena_bytes, int32_t max_jobs, int32_t substeps_per_round,
                                      int64_t host_bytes, void *stream, hw_server **out)
{
    hw_clear_error();
    if (!out) return hw_fail(HW_EINVAL, "out is NULL");
    *out = nullptr;
    if (arena_bytes < (1 << 20) || max_jobs < 1 || max_jobs > 65536 || substeps_per_round < 1 ||
        substeps_per_round > 1024 || host_bytes < (1 << 20))
        return hw_fail(HW_EINVAL, "bad server limits");
    (void)stream;
    hw_server *s = new (std::nothrow) hw_server;
    if (!s) return hw_fail(HW_ENOMEM, "host allocation failed");
    s->max_jobs = max_jobs;
    s->K = substeps_per_round;
    // Every full tile owns at least 15000 bytes of arena (two complex64 states
    // of a 1024-arc coined tile with degree <= 32 holds >= 993 arcs; four of a
    // 512-vertex complex64 or 256-vertex complex128 CTQW tile, 16 KiB) and each
    // job has at most one partial tile, so this bounds the tiles of any
    // resident set.
    s->max_tiles = int(std::min<int64_t>(int64_t(1) << 30, arena_bytes / 15000 + max_jobs));
    auto fail = [&](hw_status e) { hw_server_destroy(s); return e; };
    hw_status st;
    if ((st = hw_cuda(cudaGetDevice(&s->device), "cudaGetDevice")) != HW_OK) return fail(st);
    // the server runs on a stream of its own (graph capture needs a non-legacy stream)
    if ((st = hw_cuda(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking), "cudaStreamCreate")) != HW_OK)
        return fail(st);
    s->own_stream = true;
    if ((st = hw_cuda(cudaStreamCreateWithFlags(&s->st2, cudaStreamNonBlocking), "cudaStreamCreate")) != HW_OK)
        return fail(st);
    for (int r = 0; r < hw_server::kTimeSets; ++r)
        for (int e = 0; e < 4; ++e)
            if ((st = hw_cuda(cudaEventCreate(&s->tev[r][e]), "event")) != HW_OK) return fail(st);
    s->L = substeps_per_round;
    if ((st = hw_cuda(cudaMalloc(&s->dev_base, size_t(arena_bytes)), "cudaMalloc(serving arena)")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->host_base, size_t(host_bytes), cudaHostAllocDefault), "cudaHostAlloc(results)")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_jobs, sizeof(SJob) * max_jobs), "cudaMalloc(job table)")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->h_jobs, sizeof(SJob) * max_jobs, cudaHostAllocDefault), "cudaHostAlloc")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->h_coef, kCoefBytes * max_jobs, cudaHostAllocDefault), "cudaHostAlloc")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_tiles, sizeof(Tile) * s->max_tiles), "cudaMalloc(tiles)")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->h_tiles, sizeof(Tile) * s->max_tiles, cudaHostAllocDefault), "cudaHostAlloc")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_ntiles, sizeof(int)), "cudaMalloc")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->h_ntiles, sizeof(int), cudaHostAllocDefault), "cudaHostAlloc")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_tick, sizeof(int64_t)), "cudaMalloc")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_local, sizeof(int) * max_jobs), "cudaMalloc(local jobs)")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_lprog, sizeof(int64_t) * max_jobs), "cudaMalloc(local progress)")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->h_local, sizeof(int) * max_jobs, cudaHostAllocDefault), "cudaHostAlloc")) != HW_OK ||
        (st = hw_cuda(cudaMalloc(&s->d_nlocal, sizeof(int)), "cudaMalloc")) != HW_OK ||
        (st = hw_cuda(cudaHostAlloc(&s->h_nlocal, sizeof(int), cudaHostAllocDefault), "cudaHostAlloc")) != HW_OK ||
        (st = hw_cuda(cudaEventCreateWithFlags(&s->upload_ev, cudaEventDisableTiming), "event")) != HW_OK)
        return fail(st);
    s->dev_arena.init(s->dev_base, size_t(arena_bytes));
    s->host_arena.init(s->host_base, size_t(host_bytes));
    std::memset(s->h_jobs, 0, sizeof(SJob) * max_jobs);
    *s->h_ntiles = 0;
    *s->h_nlocal = 0;
    for (int i = max_jobs - 1; i >= 0; --i) s->free_slots.push_back(i);
    if ((st = hw_cuda(cudaMemsetAsync(s->d_tick, 0, sizeof(int64_t), s->st), "memset tick")) != HW_OK ||
        (st = hw_cuda(cudaMemsetAsync(s->d_ntiles, 0, sizeof(int), s->st), "memset")) != HW_OK ||
        (st = hw_cuda(cudaMemsetAsync(s->d_nlocal, 0, sizeof(int), s->st), "memset")) != HW_OK ||
        (st = server_capture(s)) != HW_OK)
        return fail(st);
    *out = s;
    return HW_OK;
}

extern "C" hw_status hw_server_destroy(hw_server *s)
{
    hw_clear_error();
    if (!s) return HW_OK;
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->st2) cudaStreamSynchronize(s->st2);
    for (auto &kv : s->jobs)
        if (kv.second.done_ev) cudaEventDestroy(kv.second.done_ev);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->upload_ev) cudaEventDestroy(s->upload_ev);
    cudaFree(s->dev_base);
    cudaFreeHost(s->host_base);
    cudaFree(s->d_jobs);
    cudaFreeHost(s->h_jobs);
    if (s->h_coef) cudaFreeHost(s->h_coef);
    cudaFree(s->d_tiles);
    cudaFreeHost(s->h_tiles);
    cudaFree(s->d_ntiles);
    cudaFreeHost(s->h_ntiles);
    cudaFree(s->d_tick);
    cudaFree(s->d_local);
    cudaFree(s->d_lprog);
    cudaFreeHost(s->h_local);
    cudaFree(s->d_nlocal);
    cudaFreeHost(s->h_nlocal);
    for (int r = 0; r < hw_server::kTimeSets; ++r)
        for (int e = 0; e < 4; ++e)
            if (s->tev[r][e]) cudaEventDestroy(s->tev[r][e]);
    if (s->st2) cudaStreamDestroy(s->st2);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    cudaGetLastError();
    delete s;
    return HW_OK;
}

extern "C" hw_status hw_server_submit(hw_server *s, const hw_job *job, int64_t *job_id)
{
    hw_clear_error();
    if (!s || !job || !job_id) return hw_fail(HW_EINVAL, "NULL argument");
    const hw_graph *g = job->graph;
    if (!g) return hw_fail(HW_EINVAL, "job has no graph");
    if (g->device != s->device) return hw_fail(HW_EINVAL, "graph and server live on different devices");
    if (job->kind != HW_JOB_COINED && job->kind != HW_JOB_CTQW) return hw_fail(HW_EINVAL, "unknown job kind");
    if (job->dt != HW_C64 && job->dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (job->steps < 1) return hw_fail(HW_EINVAL, "steps must be >= 1");
    if (job->n_marked < 0 || job->n_marked > kMaxServeMarked || (job->n_marked && !job->marked))
        return hw_fail(HW_EINVAL, "0..%d marked vertices", kMaxServeMarked);
    if (job->kind == HW_JOB_COINED && (!g->d_revE || g->min_degree != g->max_degree || g->max_degree < 1))
        return hw_fail(HW_EUNSUPPORTED, "served coined jobs need a regular graph");
    if (g->n >= (int64_t(1) << 30)) return hw_fail(HW_EUNSUPPORTED, "graph too large to serve");
    if (g->weighted) return hw_fail(HW_EUNSUPPORTED, "served jobs take unweighted graphs");
    Job J;
    J.id = s->next_id++;
    J.spec = *job;
    J.marked.assign(job->marked, job->marked + job->n_marked);
    std::sort(J.marked.begin(), J.marked.end());
    for (int i = 0; i < job->n_marked; ++i) {
        if (J.marked[i] < 0 || J.marked[i] >= g->n) return hw_fail(HW_EINVAL, "marked vertex out of range");
        if (i && J.marked[i] == J.marked[i - 1]) return hw_fail(HW_EINVAL, "marked vertex repeated");
    }
    J.spec.marked = nullptr;
    J.n = g->n;
    const size_t esz = cplx_bytes(hw_dtype(job->dt));
    if (job->kind == HW_JOB_COINED) {
        J.dim = g->num_arcs;
        J.total_subs = job->steps;
    } else {
        if (!std::isfinite(job->gamma) || !std::isfinite(job->time)) return hw_fail(HW_EINVAL, "gamma/time not finite");
        int m, sq;
        hw_status st = hw_ctqw_plan(g, job->gamma, J.marked.data(), job->n_marked, job->time, &m, &sq);
        if (st != HW_OK) return st;
        if (sq > 20) return hw_fail(HW_EUNSUPPORTED, "||H dt|| too large to serve");
        if (m > kServeMaxDeg) return hw_fail(HW_EUNSUPPORTED, "series degree %d above %d", m, kServeMaxDeg);
        J.m = m;
        J.q = 1 << sq;
        J.dim = g->n;
        J.local = 3 * size_t(g->n) * esz <= size_t(kLocalBytes);
        J.total_subs = J.local ? job->steps : job->steps * int64_t(J.q) * J.m;
    }
    const size_t state = (size_t(J.dim) * esz + 255) & ~size_t(255);
    const size_t rec = job->n_marked ? ((size_t(job->steps) * job->n_marked * 8 + 255) & ~size_t(255)) : 0;
    const size_t prob = (size_t(J.n) * 8 + 255) & ~size_t(255);
    J.dev_bytes = ((job->kind == HW_JOB_COINED || J.local) ? 2 : 4) * state + rec + prob +
                  ((size_t(job->steps) * 8 + 255) & ~size_t(255)) + (job->kind == HW_JOB_CTQW ? kCoefBytes : 0);
    J.host_bytes = prob + ((size_t(job->steps) * 8 + 255) & ~size_t(255));
    if (J.dev_bytes > s->dev_arena.size() || J.host_bytes > s->host_arena.size())
        return hw_fail(HW_ENOMEM, "job needs %zu device bytes; the serving arena holds %zu", J.dev_bytes,
                       s->dev_arena.size());
    J.t_submit = now_s();
    *job_id = J.id;
    s->queue.push_back(J.id);
    s->jobs.emplace(J.id, std::move(J));
    return HW_OK;
}

static hw_status rebuild_tiles(hw_server *s)
{
    int nt = 0, nl = 0;
    for (int64_t id : s->resident) {
        const Job &J = s->jobs[id];
        if (J.local) {
            s->h_local[nl++] = J.slot;
            continue;
        }
        // coined: a vertex per thread, and at least kServeTileArcs arcs per tile
        const int64_t step = (J.spec.kind == HW_JOB_COINED)
                                 ? std::max<int64_t>(kServeThreads, kServeTileArcs / J.spec.graph->max_degree)
                                 : (J.spec.dt == HW_C128 ? kTileVerticesC128 : kTileVerticesC64);
        for (int64_t v0 = 0; v0 < J.n; v0 += step) {
            if (nt >= s->max_tiles) return hw_fail(HW_EUNSUPPORTED, "tile list overflow (%d tiles)", nt);
            Tile t;
            t.job = J.slot;
            t.v0 = int32_t(v0);
            t.v1 = int32_t(std::min<int64_t>(J.n, v0 + step));
            t.pad = 0;
            s->h_tiles[nt++] = t;
        }
    }
    *s->h_ntiles = nt;
    *s->h_nlocal = nl;
    return HW_OK;
}

static hw_status admit(hw_server *s, Job &J)
{
    const hw_graph *g = J.spec.graph;
    const size_t esz = cplx_bytes(hw_dtype(J.spec.dt));
    char *dev = s->dev_arena.alloc(J.dev_bytes);
    if (!dev) return HW_ENOMEM;
    char *host = s->host_arena.alloc(J.host_bytes);
    if (!host) {
        s->dev_arena.release(dev);
        return HW_ENOMEM;
    }
    J.dev = dev;
    J.host = host;
    J.slot = s->free_slots.back();
    s->free_slots.pop_back();
    const size_t state = (size_t(J.dim) * esz + 255) & ~size_t(255);
    SJob &D = s->h_jobs[J.slot];
    std::memset(&D, 0, sizeof D);
    D.row_ptr = g->d_row_ptr;
    D.head = g->d_head;
    D.rev = g->d_rev;
    D.revE = g->d_revE;
    D.X[0] = dev;
    D.X[1] = dev + state;
    const int nstates = (J.spec.kind == HW_JOB_COINED || J.local) ? 2 : 4;
    if (nstates == 4) {
        D.T[0] = dev + 2 * state;
        D.T[1] = dev + 3 * state;
    }
    D.rec = J.spec.n_marked ? reinterpret_cast<double *>(dev + nstates * state) : nullptr;
    D.n = J.n;
    D.start_tick = s->tick;
    D.total_subs = J.total_subs;
    D.two_over_d = g->max_degree ? 2.0 / double(g->max_degree) : 0.0;
    D.two_over_d_f = float(D.two_over_d);
    D.gamma = J.spec.gamma;
    D.tau = J.spec.time / double(J.q);
    if (J.spec.kind == HW_JOB_CTQW) {
        // staged in the slot's pinned block: the slot is rewritten only by a
        // later admission, after this job's kernels (which follow the copy)
        char *cdev = dev + J.dev_bytes - kCoefBytes;
        char *ch = s->h_coef + kCoefBytes * size_t(J.slot);
        double *hd = reinterpret_cast<double *>(ch);
        float *hf = reinterpret_cast<float *>(ch + 2 * (kServeMaxDeg + 1) * sizeof(double));
        std::memset(ch, 0, kCoefBytes);
        for (int k = 1; k <= J.m && k <= kServeMaxDeg; ++k) {
            hd[k] = D.tau / double(k);
            hd[kServeMaxDeg + 1 + k] = hd[k] * D.gamma;
            hf[k] = float(hd[k]);
            hf[kServeMaxDeg + 1 + k] = float(hd[kServeMaxDeg + 1 + k]);
        }
        const hw_status cs = hw_cuda(cudaMemcpyAsync(cdev, ch, kCoefBytes, cudaMemcpyHostToDevice, s->st),
                                     "upload coefficients");
        if (cs != HW_OK) return cs;
        D.cd = reinterpret_cast<const double *>(cdev);
        D.cgd = D.cd + (kServeMaxDeg + 1);
        D.cf = reinterpret_cast<const float *>(cdev + 2 * (kServeMaxDeg + 1) * sizeof(double));
        D.cgf = D.cf + (kServeMaxDeg + 1);
    }
    D.kind = J.spec.kind;
    D.dt = J.spec.dt;
    D.d = g->max_degree;
    D.m = J.m;
    D.q = J.q;
    D.n_marked = J.spec.n_marked;
    for (int i = 0; i < J.spec.n_marked; ++i) D.marked[i] = J.marked[i];
    D.local = J.local ? 1 : 0;
    D.fam = g->kind;
    D.fdim0 = int32_t(g->dims[0]);
    D.fdim1 = int32_t(g->dims[1]);
    // uniform start over the basis: arcs (coined) or vertices (CTQW)
    const double amp = 1.0 / std::sqrt(double(J.dim));
    const int grid = int(std::min<int64_t>(148 * 16, (J.dim + 255) / 256));
    if (J.spec.dt == HW_C128) k_fill<double2><<<grid, 256, 0, s->st>>>(static_cast<double2 *>(D.X[0]), J.dim, amp);
    else k_fill<float2><<<grid, 256, 0, s->st>>>(static_cast<float2 *>(D.X[0]), J.dim, amp);
    J.end_tick = s->tick + J.total_subs;
    if (J.local) {
        J.lprog = 0;
        const hw_status ps = hw_cuda(cudaMemsetAsync(s->d_lprog + J.slot, 0, sizeof(int64_t), s->st), "memset progress");
        if (ps != HW_OK) return ps;
    }
    J.state = RESIDENT;
    s->resident.push_back(J.id);
    s->table_dirty = true;
    return hw_cuda(cudaGetLastError(), "k_fill launch");
}

static hw_status retire(hw_server *s, Job &J)
{
    const hw_graph *g = J.spec.graph;
    const SJob &D = s->h_jobs[J.slot];
    const hw_dtype dt = hw_dtype(J.spec.dt);
    const size_t esz = cplx_bytes(dt);
    const int nstates = (J.spec.kind == HW_JOB_COINED || J.local) ? 2 : 4;
    const size_t state = (size_t(J.dim) * esz + 255) & ~size_t(255);
    const size_t rec = J.spec.n_marked ? ((size_t(J.spec.steps) * J.spec.n_marked * 8 + 255) & ~size_t(255)) : 0;
    double *d_prob = reinterpret_cast<double *>(J.dev + nstates * state + rec);
    double *d_record = reinterpret_cast<double *>(J.dev + nstates * state + rec +
                                                  ((size_t(J.n) * 8 + 255) & ~size_t(255)));
    const int64_t final_parity = (J.spec.kind == HW_JOB_COINED || J.local) ? (J.spec.steps & 1)
                                                                            : ((J.spec.steps * J.q) & 1);
    const void *psi = D.X[final_parity];
    if (J.spec.kind == HW_JOB_COINED) {
        // back to the public arc order, into the other (free) state buffer
        hw_status ls = launch_layout(g, dt, psi, D.X[1 - final_parity], false, s->st);
        if (ls != HW_OK) return ls;
        psi = D.X[1 - final_parity];
    }
    hw_status st = launch_probability(J.spec.kind == HW_JOB_COINED ? g : nullptr, J.n, dt, 1, psi, d_prob, nullptr,
                                      s->st);
    if (st != HW_OK) return st;
    if (J.spec.n_marked) {
        if (J.spec.kind == HW_JOB_COINED) {
            MarkedList mk;
            std::memset(&mk, 0, sizeof mk);
            mk.n = J.spec.n_marked;
            for (int i = 0; i < mk.n; ++i) mk.inl[i] = J.marked[i];
            st = launch_marked_prob(g->d_row_ptr, dt, 1, psi, mk, D.rec + (J.spec.steps - 1) * mk.n, s->st);
            if (st != HW_OK) return st;
        }
        k_serve_record<<<int((J.spec.steps + 255) / 256), 256, 0, s->st>>>(D.rec, J.spec.n_marked, J.spec.steps,
                                                                          d_record);
        if ((st = hw_cuda(cudaGetLastError(), "k_serve_record")) != HW_OK) return st;
    }
    const size_t prob_b = (size_t(J.n) * 8 + 255) & ~size_t(255);
    if ((st = hw_cuda(cudaMemcpyAsync(J.host, d_prob, size_t(J.n) * 8, cudaMemcpyDeviceToHost, s->st), "D2H prob")) != HW_OK)
        return st;
    if (J.spec.n_marked &&
        (st = hw_cuda(cudaMemcpyAsync(J.host + prob_b, d_record, size_t(J.spec.steps) * 8, cudaMemcpyDeviceToHost, s->st),
                      "D2H record")) != HW_OK)
        return st;
    if ((st = hw_cuda(cudaEventCreateWithFlags(&J.done_ev, cudaEventDisableTiming), "event")) != HW_OK) return st;
    if ((st = hw_cuda(cudaEventRecord(J.done_ev, s->st), "event record")) != HW_OK) return st;
    J.state = RETIRING;
    return HW_OK;
}

// Local steps per round from the branch times of a finished round: the local
// branch should take about as long as the graph beside it.  With no tiled
// work the sub-steps are idle launches, and L stays at K.
static void pace_local(hw_server *s)
{
    if (*s->h_ntiles == 0) {
        s->L = s->K;
        return;
    }
    const int64_t r = s->round_no - hw_server::kTimeSets / 2;
    if (r < 0) return;
    const int set = int(r % hw_server::kTimeSets);
    if (!s->tlocal[set] || cudaEventQuery(s->tev[set][1]) != cudaSuccess ||
        cudaEventQuery(s->tev[set][3]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    float tg = 0.f, tl = 0.f;
    if (cudaEventElapsedTime(&tg, s->tev[set][0], s->tev[set][1]) != cudaSuccess ||
        cudaEventElapsedTime(&tl, s->tev[set][2], s->tev[set][3]) != cudaSuccess || tl <= 0.f) {
        cudaGetLastError();
        return;
    }
    const double want = double(s->L) * tg / tl;   // the L that matches the two branches
    if (tl > 1.25f * tg) s->L = std::max(1, int(want));
    else if (tl < 0.8f * tg) s->L = std::min(s->K, std::max(s->L + 1, int(want)));
}

// One round: the graph (K tiled sub-steps and the tick) on the server stream
// and, beside it on the second stream, L steps of every local CTQW job; the
// server stream then waits for both, so the next round's table updates and
// retirements follow them.  Branch times are recorded for pace_local.
static hw_status launch_round(hw_server *s)
{
    pace_local(s);
    const int set = int(s->round_no % hw_server::kTimeSets);
    cudaEvent_t *ev = s->tev[set];
    const bool local = *s->h_nlocal > 0;
    hw_status st;
    if ((st = hw_cuda(cudaEventRecord(ev[0], s->st), "event record")) != HW_OK) return st;
    if (local) {
        if ((st = hw_cuda(cudaStreamWaitEvent(s->st2, ev[0], 0), "stream wait")) != HW_OK ||
            (st = hw_cuda(cudaEventRecord(ev[2], s->st2), "event record")) != HW_OK)
            return st;
        k_serve_local<<<kLocalCtas, kLocalThreads, kLocalBytes, s->st2>>>(s->d_jobs, s->d_local, s->d_nlocal,
                                                                          s->d_lprog, s->L);
        if ((st = hw_cuda(cudaGetLastError(), "k_serve_local launch")) != HW_OK ||
            (st = hw_cuda(cudaEventRecord(ev[3], s->st2), "event record")) != HW_OK)
            return st;
    }
    if ((st = hw_cuda(cudaGraphLaunch(s->graph, s->st), "cudaGraphLaunch")) != HW_OK ||
        (st = hw_cuda(cudaEventRecord(ev[1], s->st), "event record")) != HW_OK)
        return st;
    if (local && (st = hw_cuda(cudaStreamWaitEvent(s->st, ev[3], 0), "stream wait")) != HW_OK) return st;
    s->tlocal[set] = local;
    ++s->round_no;
    s->tick += s->K;
    // the host's copy of every local job's progress (the kernel does the same)
    for (int64_t id : s->resident) {
        Job &J = s->jobs[id];
        if (J.local) J.lprog = std::min<int64_t>(J.spec.steps, J.lprog + s->L);
    }
    return HW_OK;
}

extern "C" hw_status hw_server_run(hw_server *s, int32_t *n_completed)
{
    hw_clear_error();
    if (!s) return hw_fail(HW_EINVAL, "server is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != s->device) return hw_fail(HW_EINVAL, "server lives on device %d, current is %d", s->device, dev);
    hw_status st;
    int32_t done = 0;
    // the pinned table mirror is rewritten below: the last upload must have read it
    if (s->upload_pending) {
        if ((st = hw_cuda(cudaEventSynchronize(s->upload_ev), "upload event")) != HW_OK) return st;
        s->upload_pending = false;
    }
    // 1. retire jobs whose last sub-step has been launched
    for (size_t i = 0; i < s->resident.size();) {
        Job &J = s->jobs[s->resident[i]];
        if (J.local ? J.lprog >= J.spec.steps : J.end_tick <= s->tick) {
            if ((st = retire(s, J)) != HW_OK) return st;
            s->free_slots.push_back(J.slot);
            s->resident.erase(s->resident.begin() + i);
            s->table_dirty = true;
        } else {
            ++i;
        }
    }
    // 2. finished copies: release memory, report
    for (auto &kv : s->jobs) {
        Job &J = kv.second;
        if (J.state != RETIRING) continue;
        const cudaError_t q = cudaEventQuery(J.done_ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return hw_cuda(q, "job completion");
        cudaEventDestroy(J.done_ev);
        J.done_ev = nullptr;
        s->dev_arena.release(J.dev);
        J.dev = nullptr;
        J.state = DONE;
        J.t_done = now_s();
        s->completed.push_back(J.id);
        ++done;
    }
    // 3. admit queued jobs while a slot and memory are free (first come, first served)
    while (!s->queue.empty() && !s->free_slots.empty()) {
        Job &J = s->jobs[s->queue.front()];
        st = admit(s, J);
        if (st == HW_ENOMEM) break;
        if (st != HW_OK) return st;
        s->queue.pop_front();
    }
    // 4. launch K sub-steps of every resident job
    if (!s->resident.empty()) {
        if (s->table_dirty) {
            if ((st = rebuild_tiles(s)) != HW_OK) return st;
            if ((st = hw_cuda(cudaMemcpyAsync(s->d_jobs, s->h_jobs, sizeof(SJob) * s->max_jobs, cudaMemcpyHostToDevice,
                                              s->st), "upload jobs")) != HW_OK ||
                (st = hw_cuda(cudaMemcpyAsync(s->d_tiles, s->h_tiles, sizeof(Tile) * std::max(1, *s->h_ntiles),
                                              cudaMemcpyHostToDevice, s->st), "upload tiles")) != HW_OK ||
                (st = hw_cuda(cudaMemcpyAsync(s->d_ntiles, s->h_ntiles, sizeof(int), cudaMemcpyHostToDevice, s->st),
                              "upload count")) != HW_OK ||
                (st = hw_cuda(cudaMemcpyAsync(s->d_local, s->h_local, sizeof(int) * std::max(1, *s->h_nlocal),
                                              cudaMemcpyHostToDevice, s->st), "upload local jobs")) != HW_OK ||
                (st = hw_cuda(cudaMemcpyAsync(s->d_nlocal, s->h_nlocal, sizeof(int), cudaMemcpyHostToDevice, s->st),
                              "upload count")) != HW_OK ||
                (st = hw_cuda(cudaEventRecord(s->upload_ev, s->st), "event record")) != HW_OK)
                return st;
            s->table_dirty = false;
            s->upload_pending = true;
        }
        if ((st = launch_round(s)) != HW_OK) return st;
    }
    if (n_completed) *n_completed = done;
    return HW_OK;
}

extern "C" hw_status hw_server_poll(hw_server *s, int64_t *ids, int32_t max_ids, int32_t *n_ids)
{
    hw_clear_error();
    if (!s || !n_ids || (max_ids > 0 && !ids)) return hw_fail(HW_EINVAL, "NULL argument");
    const int32_t n = int32_t(std::min<size_t>(size_t(std::max(max_ids, 0)), s->completed.size()));
    for (int32_t i = 0; i < n; ++i) ids[i] = s->completed[i];
    s->completed.erase(s->completed.begin(), s->completed.begin() + n);
    *n_ids = n;
    return HW_OK;
}

extern "C" hw_status hw_server_result(hw_server *s, int64_t job_id, double *prob, int64_t n_prob, double *record,
                                      int64_t n_record, double *latency_s)
{
    hw_clear_error();
    if (!s) return hw_fail(HW_EINVAL, "server is NULL");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return hw_fail(HW_EINVAL, "unknown job %lld", (long long)job_id);
    Job &J = it->second;
    if (J.state != DONE) return hw_fail(HW_EINVAL, "job %lld is not finished", (long long)job_id);
    if (prob && n_prob != J.n) return hw_fail(HW_EINVAL, "prob needs %lld entries", (long long)J.n);
    if (record && (n_record != J.spec.steps || !J.spec.n_marked))
        return hw_fail(HW_EINVAL, "record needs %lld entries and a marked vertex", (long long)J.spec.steps);
    const size_t prob_b = (size_t(J.n) * 8 + 255) & ~size_t(255);
    if (prob) std::memcpy(prob, J.host, size_t(J.n) * 8);
    if (record) std::memcpy(record, J.host + prob_b, size_t(J.spec.steps) * 8);
    if (latency_s) *latency_s = J.t_done - J.t_submit;
    s->host_arena.release(J.host);
    s->jobs.erase(it);
    return HW_OK;
}

extern "C" hw_status hw_server_stats(const hw_server *s, int64_t *queued, int64_t *resident, int64_t *arena_used,
                                     int64_t *ticks)
{
    hw_clear_error();
    if (!s) return hw_fail(HW_EINVAL, "server is NULL");
    if (queued) *queued = int64_t(s->queue.size());
    if (resident) {
        int64_t r = 0;
        for (const auto &kv : s->jobs) r += (kv.second.state == RESIDENT || kv.second.state == RETIRING);
        *resident = r;
    }
    if (arena_used) *arena_used = int64_t(s->dev_arena.used());
    if (ticks) *ticks = s->tick;
    return HW_OK;
}
