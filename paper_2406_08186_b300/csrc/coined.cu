// Fused coin + flip-flop shift for the coined quantum walk (Sec. 3.2):
//   psi'[rev[a]] = (C psi)[a],  C block-diagonal per vertex.
// Grover:   (C psi)_a = 2 m_v - psi_a,  m_v = mean of psi over v's arcs
// Fourier:  (C psi)_j = d^{-1/2} sum_k omega^{jk} psi_k, omega = e^{2 pi i/d}
// Marked vertex: (C psi)_a = -psi_a.
//
// One read and one scattered write of the state per arc plus the 4-byte
// reversal index: an HBM-bound stream.  A CTA owns a block of whole vertices
// (at most kTileArcs arcs), stages their arcs in shared memory with coalesced
// loads, forms the per-vertex coin in shared memory and scatters the results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "cache_hints.cuh"
#include "family.cuh"
#include "internal.h"
#include "sum4.cuh"

namespace {

constexpr int kThreads = 256;

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

template <typename V, typename R>
__device__ __forceinline__ V mkv(R x, R y) { V r; r.x = x; r.y = y; return r; }

// Fourier twiddles omega_d^r = (cos 2 pi r/d, sin 2 pi r/d) for d <= kTwMax,
// at c_tw[d*(d-1)/2 + r] (filled once from the host); larger d use sincospi.
constexpr int kTwMax = 32;
__constant__ double2 c_tw[kTwMax * (kTwMax + 1) / 2];
__constant__ float2 c_twf[kTwMax * (kTwMax + 1) / 2];   // the same rounded to float

__device__ __forceinline__ double2 tw_entry(int i, double) { return c_tw[i]; }
__device__ __forceinline__ float2 tw_entry(int i, float) { return c_twf[i]; }

__device__ __forceinline__ void twiddle(int r, int d, double *s, double *c)
{
    if (d <= kTwMax) {
        const double2 w = c_tw[d * (d - 1) / 2 + r];
        *c = w.x;
        *s = w.y;
    } else {
        sincospi(2.0 * double(r) / double(d), s, c);
    }
}
__device__ __forceinline__ void twiddle(int r, int d, float *s, float *c)
{
    if (d <= kTwMax) {
        const float2 w = c_twf[d * (d - 1) / 2 + r];
        *c = w.x;
        *s = w.y;
    } else {
        sincospif(2.0f * float(r) / float(d), s, c);
    }
}

// index of v in the sorted marked list, or -1
__device__ __forceinline__ int find_marked(const MarkedList &mk, int v) { return marked_find(mk, v); }

// the Grover weight 2/d in the kernel's precision, from the graph's tables
template <typename A> __device__ __forceinline__ double grover_w(const A &a, int d, double) { return a.two_over_d[d]; }
template <typename A> __device__ __forceinline__ float grover_w(const A &a, int d, float) { return __ldg(a.two_over_d_f + d); }

// deterministic block sum (fixed shuffle tree, then fixed order over warps)
template <typename T>
__device__ __forceinline__ T block_sum(T x, T *red)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = x;
    __syncthreads();
    T t = 0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

struct StepArgs {
    const double *two_over_d;
    const float *two_over_d_f;   // the same in float
    const int32_t *row_ptr;
    const int32_t *rev;
    const int32_t *blk;
    double *rec_part;
    const void *in;
    void *out;
    int64_t rec_slot;
    int32_t nblk;
    MarkedList mk;
};

// A vertex with more arcs than a tile: one CTA, two passes over global memory.
template <typename R, int COIN>
__device__ void heavy_vertex(const StepArgs &a, int v, int a0, int d)
{
    using V = typename Cx<R>::T;
    __shared__ R red_r[kThreads / 32];
    __shared__ double red_d[kThreads / 32];
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);
    const int mi = find_marked(a.mk, v);
    if (mi >= 0 && a.rec_part && a.rec_slot >= 0) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const V p = in[a0 + i];
            acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
        }
        acc = block_sum(acc, red_d);
        if (threadIdx.x == 0) a.rec_part[a.rec_slot * a.mk.n + mi] = acc;
    }
    if (mi >= 0) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const V p = in[a0 + i];
            out[a.rev[a0 + i]] = mkv<V, R>(-p.x, -p.y);
        }
        return;
    }
    if (COIN == HW_COIN_GROVER) {
        R sx = 0, sy = 0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const V p = in[a0 + i];
            sx += p.x;
            sy += p.y;
        }
        sx = block_sum(sx, red_r);
        sy = block_sum(sy, red_r);
        const R f = grover_w(a, d, R(0));
        const R mx = sx * f, my = sy * f;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const V p = in[a0 + i];
            out[a.rev[a0 + i]] = mkv<V, R>(mx - p.x, my - p.y);
        }
    } else {
        const R scale = R(1) / sqrt(R(d));
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            R cx = 0, cy = 0;
            for (int k = 0; k < d; ++k) {
                R s, c;
                twiddle(int((int64_t(j) * k) % d), d, &s, &c);
                const V p = in[a0 + k];
                cx += c * p.x - s * p.y;
                cy += c * p.y + s * p.x;
            }
            out[a.rev[a0 + j]] = mkv<V, R>(cx * scale, cy * scale);
        }
    }
}

template <typename R, int COIN>
__global__ void __launch_bounds__(kThreads) k_coined_step(StepArgs a)
{
    using V = typename Cx<R>::T;
    constexpr int kPer = kTileArcs / kThreads;   // arcs per thread
    __shared__ V s_psi[kTileArcs];
    __shared__ V s_coef[kTileVerts];          // Grover: 2 m_v (0 if marked); Fourier: (marked, 0)
    __shared__ int32_t s_rp[kTileVerts + 1];
    __shared__ uint16_t s_tail[kTileArcs];
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);

    for (int b = blockIdx.x; b < a.nblk; b += gridDim.x) {
        const int v0 = a.blk[b], v1 = a.blk[b + 1];
        const int nv = v1 - v0;
        for (int i = threadIdx.x; i <= nv; i += blockDim.x) s_rp[i] = a.row_ptr[v0 + i];
        __syncthreads();
        const int a0 = s_rp[0];
        const int na = s_rp[nv] - a0;
        if (na > kTileArcs) {              // block-uniform branch: one heavy vertex
            if (b == int(blockIdx.x)) pdl_wait();
            heavy_vertex<R, COIN>(a, v0, a0, na);
            __syncthreads();
            continue;
        }
        // all global loads of the tile first (state and reversal index)
        V p[kPer];
        int r[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * kThreads;
            if (i < na) r[k] = a.rev[a0 + i];
        }
        if (b == int(blockIdx.x)) pdl_wait();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * kThreads;
            if (i < na) {
                p[k] = in[a0 + i];
                s_psi[i] = p[k];
            }
        }
        __syncthreads();
        for (int lv = threadIdx.x; lv < nv; lv += blockDim.x) {
            const int s = s_rp[lv] - a0, e = s_rp[lv + 1] - a0;
            const int mi = find_marked(a.mk, v0 + lv);
            for (int j = s; j < e; ++j) s_tail[j] = uint16_t(lv);
            if (COIN == HW_COIN_GROVER) {
                R sx = 0, sy = 0;
                for (int j = s; j < e; ++j) { sx += s_psi[j].x; sy += s_psi[j].y; }
                const R f = (mi < 0) ? grover_w(a, e - s, R(0)) : R(0);
                s_coef[lv] = mkv<V, R>(sx * f, sy * f);
            } else {
                s_coef[lv] = mkv<V, R>(mi >= 0 ? R(1) : R(0), R(0));
            }
            if (mi >= 0 && a.rec_part && a.rec_slot >= 0) {
                double acc = 0.0;
                for (int j = s; j < e; ++j)
                    acc += double(s_psi[j].x) * double(s_psi[j].x) + double(s_psi[j].y) * double(s_psi[j].y);
                a.rec_part[a.rec_slot * a.mk.n + mi] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * kThreads;
            if (i >= na) break;
            const int lv = s_tail[i];
            V c;
            if (COIN == HW_COIN_GROVER) {
                const V m2 = s_coef[lv];
                c = mkv<V, R>(m2.x - p[k].x, m2.y - p[k].y);
            } else if (s_coef[lv].x != R(0)) {
                c = mkv<V, R>(-p[k].x, -p[k].y);
            } else {
                const int s = s_rp[lv] - a0, d = s_rp[lv + 1] - s_rp[lv], j = i - s;
                R cx = 0, cy = 0;
                for (int q = 0; q < d; ++q) {
                    R sn, cs;
                    twiddle((j * q) % d, d, &sn, &cs);
                    const V x = s_psi[s + q];
                    cx += cs * x.x - sn * x.y;
                    cy += cs * x.y + sn * x.x;
                }
                const R scale = R(1) / sqrt(R(d));
                c = mkv<V, R>(cx * scale, cy * scale);
            }
            out[r[k]] = c;
        }
        __syncthreads();
    }
    pdl_trigger();
}

// ---------------------------------------------------------------- regular
// Every vertex has the same degree D <= 8.  One thread owns one vertex and
// its D consecutive arcs: D vector loads of psi and one vector load of rev,
// the coin in registers, D scattered stores.  Thread-per-vertex keeps the
// floating-point instruction count per arc minimal, which matters for
// complex128: B300's FP64 pipe issues about one warp instruction every 16
// cycles per SM, so per-lane butterfly sums would make the step FP64-bound.
struct RegArgs {
    const int32_t *rev;
    double *rec_part;
    const void *in;
    void *out;
    int64_t rec_slot;
    int64_t n;
    double two_over_d;
    float two_over_d_f;     // the same weight rounded once on the host (no per-thread conversion)
    MarkedList mk;
};

template <typename R> __device__ __forceinline__ R grover_weight(const RegArgs &a);
template <> __device__ __forceinline__ float grover_weight<float>(const RegArgs &a) { return a.two_over_d_f; }

// Lane-group variant for complex64 (FP32 arithmetic is cheap; the limit is
// memory requests): a group of G = 2^ceil(log2 d) consecutive lanes owns one
// vertex, lane j < d holds arc d*v + j, so loads of psi and rev are fully
// coalesced; the Grover sum runs as an xor-shuffle tree inside the group.
template <typename R, int G, int COIN, int U>
__global__ void __launch_bounds__(kThreads) k_coined_lanes(RegArgs a, int d)
{
    using V = typename Cx<R>::T;
    constexpr int VPW = 32 / G;
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);
    const int lane = threadIdx.x & 31;
    const int j = lane & (G - 1);
    const int base = lane & ~(G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t vbase = warp * (VPW * U) + lane / G;
    const R f2 = grover_weight<R>(a);

    V p[U];
    int r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t v = vbase + u * VPW;
        r[u] = (v < a.n && j < d) ? __ldg(a.rev + v * d + j) : -1;   // constant table
    }
    pdl_wait();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t v = vbase + u * VPW;
        p[u] = (r[u] >= 0) ? in[v * d + j] : mkv<V, R>(R(0), R(0));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t v = vbase + u * VPW;
        const int mi = (v < a.n) ? find_marked(a.mk, int(v)) : -1;   // uniform in the group
        // warp-uniform test first, so warps without a marked vertex issue no FP64 work
        if (__any_sync(0xffffffffu, mi >= 0) && a.rec_part && a.rec_slot >= 0 && mi >= 0) {
            double acc = double(p[u].x) * double(p[u].x) + double(p[u].y) * double(p[u].y);
#pragma unroll
            for (int o = 1; o < G; o <<= 1) acc += __shfl_xor_sync(gmask, acc, o);
            if (j == 0) a.rec_part[a.rec_slot * a.mk.n + mi] = acc;
        }
        V c;
        if (COIN == HW_COIN_GROVER) {
            R sx = p[u].x, sy = p[u].y;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            const R f = (mi >= 0) ? R(0) : f2;
            c = mkv<V, R>(fma(f, sx, -p[u].x), fma(f, sy, -p[u].y));
        } else {
            R cx = 0, cy = 0;
            for (int k = 0; k < d; ++k) {
                const R qx = __shfl_sync(0xffffffffu, p[u].x, base + k);
                const R qy = __shfl_sync(0xffffffffu, p[u].y, base + k);
                R sn, cs;
                twiddle((j * k) % d, d, &sn, &cs);
                cx += cs * qx - sn * qy;
                cy += cs * qy + sn * qx;
            }
            const R scale = R(1) / sqrt(R(d));
            c = (mi >= 0) ? mkv<V, R>(-p[u].x, -p[u].y) : mkv<V, R>(cx * scale, cy * scale);
        }
        if (r[u] >= 0) out[r[u]] = c;
    }
    pdl_trigger();
}

// ---------------------------------------------------------------- batched
// States [num_arcs][batch] share the graph.  One warp per vertex: for each
// column the warp sums the vertex's rows (coalesced across the batch), then
// writes each coin output row to its reversed arc.
struct BatchArgs {
    const double *two_over_d;
    const float *two_over_d_f;   // the same in float
    const int32_t *row_ptr;
    const int32_t *rev;
    double *rec_part;
    const void *in;
    void *out;
    int64_t rec_slot;
    int32_t n;
    int32_t batch;
    int32_t verts_per_warp;
    MarkedList mk;
};

template <typename R, int COIN>
__global__ void __launch_bounds__(kThreads) k_coined_step_batched(BatchArgs a)
{
    using V = typename Cx<R>::T;
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int B = a.batch;
    const int64_t vbeg = warp * a.verts_per_warp;
    const int64_t vend = (vbeg + a.verts_per_warp < a.n) ? vbeg + a.verts_per_warp : int64_t(a.n);
    for (int64_t v = vbeg; v < vend; ++v) {
        const int s = a.row_ptr[v], e = a.row_ptr[v + 1], d = e - s;
        if (d == 0) continue;
        const int mi = find_marked(a.mk, int(v));
        for (int c = lane; c < B; c += 32) {
            if (mi >= 0) {
                double acc = 0.0;
                for (int j = s; j < e; ++j) {
                    const V p = in[int64_t(j) * B + c];
                    acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
                    out[int64_t(a.rev[j]) * B + c] = mkv<V, R>(-p.x, -p.y);
                }
                if (a.rec_part && a.rec_slot >= 0)
                    a.rec_part[(a.rec_slot * a.mk.n + mi) * B + c] = acc;
            } else if (COIN == HW_COIN_GROVER) {
                R sx = 0, sy = 0;
                for (int j = s; j < e; ++j) {
                    const V p = in[int64_t(j) * B + c];
                    sx += p.x;
                    sy += p.y;
                }
                const R f = grover_w(a, d, R(0));
                sx *= f;
                sy *= f;
                for (int j = s; j < e; ++j) {
                    const V p = in[int64_t(j) * B + c];
                    out[int64_t(a.rev[j]) * B + c] = mkv<V, R>(sx - p.x, sy - p.y);
                }
            } else {
                const R scale = R(1) / sqrt(R(d));
                for (int j = 0; j < d; ++j) {
                    R cx = 0, cy = 0;
                    for (int k = 0; k < d; ++k) {
                        R sn, cs;
                        twiddle(int((int64_t(j) * k) % d), d, &sn, &cs);
                        const V q = in[int64_t(s + k) * B + c];
                        cx += cs * q.x - sn * q.y;
                        cy += cs * q.y + sn * q.x;
                    }
                    out[int64_t(a.rev[s + j]) * B + c] = mkv<V, R>(cx * scale, cy * scale);
                }
            }
        }
    }
}


// Batched Grover step with rows held in registers.  The batch of a vertex's
// arc is one contiguous row (batch x 8 or 16 bytes); a warp owns a vertex,
// each lane a 16-byte (or 8-byte) slice of the row, so every row load and
// every row store to the reversed arc is one coalesced line.  Up to DREG rows
// stay in registers between the sum and the stores; larger vertices re-read.
struct RowsArgs {
    const double *two_over_d;
    const float *two_over_d_f;   // the same in float
    const int32_t *row_ptr;
    const int32_t *rev;
    double *rec_part;
    const void *in;
    void *out;
    int64_t rec_slot;
    int64_t n;
    int32_t batch;
    int32_t vpw;             // vertices per warp
    MarkedList mk;
};

template <typename R, int CPL> struct RowVec;
template <> struct RowVec<float, 2> {
    using T = float4;
    static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ float re(const T &v, int q) { return q ? v.z : v.x; }
    static __device__ __forceinline__ float im(const T &v, int q) { return q ? v.w : v.y; }
};
template <> struct RowVec<float, 1> {
    using T = float2;
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ float re(const T &v, int) { return v.x; }
    static __device__ __forceinline__ float im(const T &v, int) { return v.y; }
};
template <> struct RowVec<double, 1> {
    using T = double2;
    static __device__ __forceinline__ T zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ double re(const T &v, int) { return v.x; }
    static __device__ __forceinline__ double im(const T &v, int) { return v.y; }
};

// c = f * sum - p, componentwise (Grover), or -p (marked: f = 0 handled by caller)
__device__ __forceinline__ float4 grover_row(float f, const float4 &s, const float4 &p)
{
    return make_float4(fmaf(f, s.x, -p.x), fmaf(f, s.y, -p.y), fmaf(f, s.z, -p.z), fmaf(f, s.w, -p.w));
}
__device__ __forceinline__ float2 grover_row(float f, const float2 &s, const float2 &p)
{
    return make_float2(fmaf(f, s.x, -p.x), fmaf(f, s.y, -p.y));
}
__device__ __forceinline__ double2 grover_row(double f, const double2 &s, const double2 &p)
{
    return make_double2(fma(f, s.x, -p.x), fma(f, s.y, -p.y));
}
__device__ __forceinline__ void add_row(float4 &a, const float4 &b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }
__device__ __forceinline__ void add_row(float2 &a, const float2 &b) { a.x += b.x; a.y += b.y; }
__device__ __forceinline__ void add_row(double2 &a, const double2 &b) { a.x += b.x; a.y += b.y; }

template <typename R, int CPL, int DREG>
__global__ void __launch_bounds__(256) k_coined_rows(RowsArgs a)
{
    using RV = RowVec<R, CPL>;
    using T = typename RV::T;
    const T *__restrict__ in = static_cast<const T *>(a.in);
    T *__restrict__ out = static_cast<T *>(a.out);
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int B = a.batch;
    const int BV = B / CPL;                   // row length in vectors
    const int64_t v0 = gw * a.vpw;
    const int64_t v1 = (v0 + a.vpw < a.n) ? v0 + a.vpw : a.n;
    for (int64_t v = v0; v < v1; ++v) {
        const int s = a.row_ptr[v], e = a.row_ptr[v + 1], d = e - s;
        if (d == 0) continue;
        const int mi = find_marked(a.mk, int(v));
        const int rv = (lane < d) ? __ldg(a.rev + s + lane) : 0;
        const R f = (mi >= 0) ? R(0) : grover_w(a, d, R(0));
        for (int c0 = 0; c0 < BV; c0 += 32) {
            const int cv = c0 + lane;             // this lane's vector column
            const bool act = cv < BV;
            if (d <= DREG) {
                T p[DREG];
                T sum = RV::zero();
#pragma unroll
                for (int j = 0; j < DREG; ++j) {
                    if (j < d) {
                        p[j] = act ? in[int64_t(s + j) * BV + cv] : RV::zero();
                        add_row(sum, p[j]);
                    }
                }
                if (mi >= 0 && a.rec_part && a.rec_slot >= 0 && act) {
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        double acc = 0.0;
#pragma unroll
                        for (int j = 0; j < DREG; ++j)
                            if (j < d) {
                                const double x = RV::re(p[j], q), y = RV::im(p[j], q);
                                acc += x * x + y * y;
                            }
                        a.rec_part[(a.rec_slot * a.mk.n + mi) * B + cv * CPL + q] = acc;
                    }
                }
#pragma unroll
                for (int j = 0; j < DREG; ++j) {
                    if (j < d) {
                        const int r = __shfl_sync(0xffffffffu, rv, j);
                        if (act) out[int64_t(r) * BV + cv] = grover_row(f, sum, p[j]);
                    }
                }
            } else {
                T sum = RV::zero();
                double acc[CPL] = {};
                for (int j = 0; j < d; ++j) {
                    const T p = act ? in[int64_t(s + j) * BV + cv] : RV::zero();
                    add_row(sum, p);
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const double x = RV::re(p, q), y = RV::im(p, q);
                        acc[q] += x * x + y * y;
                    }
                }
                if (mi >= 0 && a.rec_part && a.rec_slot >= 0 && act)
#pragma unroll
                    for (int q = 0; q < CPL; ++q) a.rec_part[(a.rec_slot * a.mk.n + mi) * B + cv * CPL + q] = acc[q];
                for (int j = 0; j < d; ++j) {
                    const int r = (j < 32) ? __shfl_sync(0xffffffffu, rv, j) : __ldg(a.rev + s + j);
                    if (act) {
                        const T p = in[int64_t(s + j) * BV + cv];
                        out[int64_t(r) * BV + cv] = grover_row(f, sum, p);
                    }
                }
            }
        }
    }
}


// Batched Grover step with TMA bulk staging.  A vertex's batch rows are one
// contiguous block (d x rowbytes), so each warp streams its own consecutive
// vertices through a ring of kRingSlots shared-memory slots with
// cp.async.bulk (one mbarrier per slot), prefetching kRingSlots-1 vertices
// ahead while it sums and scatters the current one.  In-flight data occupies
// shared memory, not registers, so every SM keeps tens of KB of loads in
// flight.  Vertices whose rows do not fit a slot are read directly.
constexpr int kRingSlots = 3;
constexpr int kSlotBytes = 8192;
constexpr int kRingWarps = 4;
constexpr uint64_t kRingWaitNs = 2000000000ull;

struct RingArgs {
    const double *two_over_d;
    const float *two_over_d_f;   // the same in float
    const int32_t *row_ptr;
    const int32_t *rev;
    double *rec_part;
    const void *in;
    void *out;
    int *err;                // zero-copy host word: set on a wait timeout
    int64_t rec_slot;
    int64_t n;
    int64_t arcs;            // row_ptr[n]
    int32_t batch;
    int32_t rowbytes;
    MarkedList mk;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool ring_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 0) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > kRingWaitNs) return false;
        }
    }
}

// issued by one lane: stage the rows of the vertex with arc range [s, e) into
// a slot (or just arrive when they do not fit, or when in_range is false: the
// vertex is past the warp's range)
__device__ __forceinline__ void ring_issue(const RingArgs &a, bool in_range, int s, int e, uint32_t slot,
                                           uint32_t bar)
{
    uint32_t bytes = 0;
    const char *src = nullptr;
    if (in_range) {
        const int64_t b = int64_t(e - s) * a.rowbytes;
        if (b > 0 && b <= kSlotBytes) {
            bytes = uint32_t(b);
            src = static_cast<const char *>(a.in) + int64_t(s) * a.rowbytes;
        }
    }
    if (bytes) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(slot), "l"(src), "r"(bytes), "r"(bar) : "memory");
    } else {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    }
}

template <typename R, int CPL>
__global__ void __launch_bounds__(kRingWarps * 32) k_coined_ring(RingArgs a)
{
    using RV = RowVec<R, CPL>;
    using T = typename RV::T;
    extern __shared__ __align__(128) uint8_t ring_raw[];
    __shared__ __align__(8) uint64_t bars[kRingWarps][kRingSlots];
    __shared__ int rev_s[kRingWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *ring = ring_raw + warp * (kRingSlots * kSlotBytes);
    const uint32_t ring_s = smem_addr(ring);
    if (lane == 0) {
        for (int k = 0; k < kRingSlots; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[warp][k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t W = int64_t(gridDim.x) * kRingWarps;
    const int64_t w = int64_t(blockIdx.x) * kRingWarps + warp;
    const int64_t vbeg = a.n * w / W, vend = a.n * (w + 1) / W;
    const T *__restrict__ in = static_cast<const T *>(a.in);
    T *__restrict__ out = static_cast<T *>(a.out);
    const int BV = a.rowbytes / int(sizeof(T));       // 16-byte (or 8-byte) vectors per row
    const int B = a.batch;

    // rp[i] = row_ptr[v + i] for the current vertex v (a window over the
    // vertices being processed and staged; entries past n are not used), and
    // rev_c = the lane's reversal entry of v's block.  Both are loaded one
    // iteration ahead, so no iteration waits on a global load before its
    // stores: every fourth vertex's reversal entries and every 32nd vertex's
    // offsets miss the caches.
    constexpr int kAhead = kRingSlots - 1;   // vertices staged ahead of the current one
    int rp[kAhead + 2];
#pragma unroll
    for (int i = 0; i < kAhead + 2; ++i) rp[i] = a.row_ptr[vbeg + i <= a.n ? vbeg + i : a.n];
    int rev_c = (vbeg < vend && rp[0] + lane < rp[1]) ? __ldg(a.rev + rp[0] + lane) : 0;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kAhead; ++k)
            ring_issue(a, vbeg + k < vend, rp[k], rp[k + 1], ring_s + k * kSlotBytes, smem_addr(&bars[warp][k]));
    bool ok = true;
    int64_t waited = 0;     // slots consumed so far (phase bookkeeping for the drain)
    for (int64_t v = vbeg; v < vend && ok; ++v) {
        const int64_t k = v - vbeg;
        const int slot = int(k % kRingSlots);
        // keep kAhead vertices in flight: refill the slot freed last iteration
        if (lane == 0) {
            const int nxt = int((k + kAhead) % kRingSlots);
            ring_issue(a, v + kAhead < vend, rp[kAhead], rp[kAhead + 1], ring_s + nxt * kSlotBytes,
                       smem_addr(&bars[warp][nxt]));
        }
        const int s = rp[0], e = rp[1], d = e - s;
        rev_s[warp][lane] = rev_c;   // meaningful for lanes < d
        // the next iteration's window entry and reversal entries (its block starts at e)
#pragma unroll
        for (int i = 0; i < kAhead + 1; ++i) rp[i] = rp[i + 1];
        rp[kAhead + 1] = a.row_ptr[v + kAhead + 2 <= a.n ? v + kAhead + 2 : a.n];
        rev_c = (int64_t(e) + lane < a.arcs) ? __ldg(a.rev + e + lane) : 0;
        __syncwarp();
        if (!ring_wait(smem_addr(&bars[warp][slot]), uint32_t((k / kRingSlots) & 1))) {
            if (lane == 0) atomicExch(a.err, 1);
            ok = false;
            break;
        }
        waited = k + 1;
        if (d > 0) {
            const int mi = find_marked(a.mk, int(v));
            const bool staged = int64_t(d) * a.rowbytes <= kSlotBytes;
            const T *rows = staged ? reinterpret_cast<const T *>(ring + slot * kSlotBytes) : in + int64_t(s) * BV;
            if (mi >= 0) {
                // marked vertex (rare): -I coin, and its probability in double for the record.
                // Kept apart from the Grover loop so no FP64 work is issued for other vertices.
                for (int cv = lane; cv < BV; cv += 32) {
                    if (a.rec_part && a.rec_slot >= 0) {
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            double acc = 0.0;
                            for (int j = 0; j < d; ++j) {
                                const T p = rows[j * BV + cv];
                                const double x = RV::re(p, q), y = RV::im(p, q);
                                acc += x * x + y * y;
                            }
                            a.rec_part[(a.rec_slot * a.mk.n + mi) * B + cv * CPL + q] = acc;
                        }
                    }
                    for (int j = 0; j < d; ++j) {
                        const int r = (j < 32) ? rev_s[warp][j] : __ldg(a.rev + s + j);
                        out[int64_t(r) * BV + cv] = grover_row(R(0), RV::zero(), rows[j * BV + cv]);
                    }
                }
            } else {
                const R f = grover_w(a, d, R(0));
                for (int cv = lane; cv < BV; cv += 32) {
                    T sum = RV::zero();
                    for (int j = 0; j < d; ++j) add_row(sum, rows[j * BV + cv]);
                    for (int j = 0; j < d; ++j) {
                        const int r = (j < 32) ? rev_s[warp][j] : __ldg(a.rev + s + j);
                        out[int64_t(r) * BV + cv] = grover_row(f, sum, rows[j * BV + cv]);
                    }
                }
            }
        }
        // the slot is read; order those generic reads before the async refill
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // drain: wait (bounded) for every issued slot not consumed yet, so no bulk
    // copy is still writing this CTA's shared memory when it exits
    const int64_t issued = (vend - vbeg) + kRingSlots - 1;
    const int64_t last = ok ? issued : (waited + kRingSlots - 1 < issued ? waited + kRingSlots - 1 : issued);
    for (int64_t k = waited; k < last; ++k)
        if (!ring_wait(smem_addr(&bars[warp][int(k % kRingSlots)]), uint32_t((k / kRingSlots) & 1))) {
            if (lane == 0) atomicExch(a.err, 1);
            break;
        }
}

// -------------------------------------------------------- marked records
// dst[mi*batch + b] = sum over the arcs of marked[mi] of |psi|^2 (row_ptr != NULL),
// or |psi[marked[mi]]|^2 for a vertex-indexed state (row_ptr == NULL).
template <typename R>
__global__ void k_marked_prob(const int32_t *__restrict__ row_ptr, const void *psi_, MarkedList mk,
                              int batch, double *__restrict__ dst)
{
    using V = typename Cx<R>::T;
    const V *psi = static_cast<const V *>(psi_);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mk.n * batch) return;
    const int mi = i / batch, b = i % batch;
    const int v = marked_id(mk, mi);
    const int s = row_ptr ? row_ptr[v] : v;
    const int e = row_ptr ? row_ptr[v + 1] : v + 1;
    double acc = 0.0;
    for (int j = s; j < e; ++j) {
        const V p = psi[int64_t(j) * batch + b];
        acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
    }
    dst[i] = acc;
}

__global__ void k_record_finalize(const double *__restrict__ part, int n_marked, int64_t slots,
                                  int batch, double *__restrict__ record)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= slots * batch) return;
    const int64_t s = i / batch;
    const int b = int(i % batch);
    double acc = 0.0;
    for (int m = 0; m < n_marked; ++m) acc += part[(s * n_marked + m) * batch + b];
    record[i] = acc;
}

// ---- edge-major layout (regular graphs): E[j][v] = psi[v d + j]
// Arc j of every vertex forms a contiguous row, so a warp of consecutive
// vertices reads each of its rows as one 256/512-byte segment, and the
// reversal E'[revE[j n + v]] lands, for structured graphs (torus, hypercube),
// on consecutive vertices of one row as well: the shift writes whole sectors.
// hw_coined_evolve transposes in and out once per call.

struct EmArgs {
    const int32_t *revE;     // the shift as an edge-major table (table addressing)
    double *rec_part;
    const void *in;
    void *out;
    int64_t rec_slot;
    int64_t n;
    int32_t d;
    int32_t L1, L2;          // torus addressing: rows, columns
    int32_t grid2d;          // torus addressing: block row y = blockIdx.y is torus row x
    double two_over_d;
    float two_over_d_f;
    MarkedList mk;
};

template <typename R> __device__ __forceinline__ R em_weight(const EmArgs &a);
template <> __device__ __forceinline__ double em_weight<double>(const EmArgs &a) { return a.two_over_d; }
template <> __device__ __forceinline__ float em_weight<float>(const EmArgs &a) { return a.two_over_d_f; }

// thread per vertex, degree D known at compile time (the same arithmetic as
// the arc-major kernels: Grover sum in arc order from arc 0, one FMA per component)
template <typename R, int D, int COIN, int ADDR>
__global__ void __launch_bounds__(kThreads) k_coined_em(EmArgs a)
{
    using V = typename Cx<R>::T;
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);
    // 32-bit indices: every edge-major index j n + v is below the arc count < 2^31
    const int n = int(a.n);
    int v;
    bool live;
    V p[D];
    int r[D];
    if constexpr (ADDR == kAddrTable) {
        v = int(blockIdx.x * blockDim.x + threadIdx.x);
        live = v < n;
        if (live) {   // targets depend on the graph only: before the wait
#pragma unroll
            for (int j = 0; j < D; ++j) r[j] = __ldg(a.revE + j * n + v);
        }
    } else {
        static_assert(D == 4, "torus addressing is for degree 4");
        if (a.grid2d) {   // no division: the block row is the torus row
            const uint32_t y = blockIdx.x * blockDim.x + threadIdx.x;
            v = int(blockIdx.y) * a.L2 + int(y);
            live = y < uint32_t(a.L2);
            if (live) torus_targets<ADDR>(TorusVertex(blockIdx.y, y, n, a.L1, a.L2), n, r);
        } else {
            v = int(blockIdx.x * blockDim.x + threadIdx.x);
            live = v < n;
            if (live) torus_targets<ADDR>(TorusVertex(int64_t(v), n, a.L1, a.L2), n, r);
        }
    }
    pdl_wait();
    if (live) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            // complex128: each row is read once and the two state buffers do
            // not fit L2, so loads and stores stream (evict first); complex64
            // states stay in L2 from step to step and keep the default
            if constexpr (sizeof(R) == 8) p[j] = __ldcs(in + j * n + v);
            else p[j] = in[j * n + v];
        }
        const int mi = find_marked(a.mk, v);
        if (mi >= 0) {
            if (a.rec_part && a.rec_slot >= 0) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < D; ++j)
                    acc += double(p[j].x) * double(p[j].x) + double(p[j].y) * double(p[j].y);
                a.rec_part[a.rec_slot * a.mk.n + mi] = acc;
            }
#pragma unroll
            for (int j = 0; j < D; ++j) out[r[j]] = mkv<V, R>(-p[j].x, -p[j].y);
        } else if (COIN == HW_COIN_GROVER) {
            R sx, sy;
            if constexpr (D == 4 && sizeof(R) == 8) {
                // complex128, degree 4: each component's sum rounded once, by
                // integer operations (the FP64 unit bounds this kernel)
                sx = sum4::sum4_rn(p[0].x, p[1].x, p[2].x, p[3].x);
                sy = sum4::sum4_rn(p[0].y, p[1].y, p[2].y, p[3].y);
            } else {
                sx = p[0].x;
                sy = p[0].y;
#pragma unroll
                for (int j = 1; j < D; ++j) { sx += p[j].x; sy += p[j].y; }
            }
            const R f = em_weight<R>(a);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const V o = mkv<V, R>(fma(f, sx, -p[j].x), fma(f, sy, -p[j].y));
                if constexpr (sizeof(R) == 8) __stcs(out + r[j], o);
                else out[r[j]] = o;
            }
        } else {
            const R scale = R(1) / sqrt(R(D));
#pragma unroll
            for (int j = 0; j < D; ++j) {
                R cx = 0, cy = 0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const auto w = tw_entry(D * (D - 1) / 2 + (j * k) % D, R(0));
                    cx += w.x * p[k].x - w.y * p[k].y;
                    cy += w.x * p[k].y + w.y * p[k].x;
                }
                out[r[j]] = mkv<V, R>(cx * scale, cy * scale);
            }
        }
    }
    pdl_trigger();
}

// Grover, any degree: thread per vertex, a pass for the sum and a pass (rows
// read again, from L2) for the outputs; blocks of kRtThreads threads, half an
// SM's warp slots (64 registers a thread)
constexpr int kRtThreads = 128;
template <typename R, int ADDR>
__global__ void __launch_bounds__(kRtThreads, 2048 / kRtThreads / 2) k_coined_em_rt(EmArgs a)
{
    using V = typename Cx<R>::T;
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);
    // row j of vertex v at j n + v < 2|E| < 2^31 (the graph's limit): 32-bit indices
    const int v = int(blockIdx.x) * int(blockDim.x) + int(threadIdx.x);
    const int n = int(a.n);
    const int d = a.d;
    pdl_wait();
    if (v < n) {
        const int mi = find_marked(a.mk, v);
        if (mi >= 0) {
            if (a.rec_part && a.rec_slot >= 0) {
                double acc = 0.0;
                for (int j = 0; j < d; ++j) {
                    const V p = in[j * n + v];
                    acc += double(p.x) * double(p.x) + double(p.y) * double(p.y);
                }
                a.rec_part[a.rec_slot * a.mk.n + mi] = acc;
            }
            CubeWalk cw(v, d);
            for (int j = 0; j < d; ++j) {
                const V p = in[j * n + v];
                const int r = (ADDR == kAddrCube) ? cw.target(cw.next_bit(), n) : __ldg(a.revE + j * n + v);
                out[r] = mkv<V, R>(-p.x, -p.y);
            }
        } else {
            R sx, sy;
            if constexpr (sizeof(R) == 8) {
                // complex128: groups of four rows summed by integer operations
                // (sum4.cuh), the group sums added in double
                // first reads of the rows marked evict-last in L2: the second
                // pass reads them again
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
            const R f = em_weight<R>(a);
            // the rows again, last first: the rows read last by the sum are
            // the likeliest to be still in L2
            CubeWalk cw(v, d);
#pragma unroll 4
            for (int j = d - 1; j >= 0; --j) {
                // the rows' last use (evict first) and streaming stores, so
                // that L2 keeps the rows the other warps have still to re-read
                const V p = __ldcs(in + j * n + v);
                const int r = (ADDR == kAddrCube) ? cw.target(cw.prev_bit(), n) : __ldg(a.revE + j * n + v);
                __stcs(out + r, mkv<V, R>(fma(f, sx, -p.x), fma(f, sy, -p.y)));
            }
        }
    }
    pdl_trigger();
}

// Grover on a regular graph of degree K (K known at compile time): a thread
// per vertex loads its K rows into registers at once and writes the K
// outputs from them, so each row is read once (k_coined_em_rt reads the rows
// twice).  Hypercubes take the targets from the labels (kAddrCube), other
// graphs (and the tables' addressing of hypercubes) from revE; both give the
// same bits.  complex128 sums: grouped_sum2_fixed (groups of four, folded
// four at a time by the integer sum).
template <typename R, int K, int ADDR>
__global__ void __launch_bounds__(kThreads) k_coined_em_cube(EmArgs a)
{
    using V = typename Cx<R>::T;
    const V *__restrict__ in = static_cast<const V *>(a.in);
    V *__restrict__ out = static_cast<V *>(a.out);
    const int v = int(blockIdx.x) * int(blockDim.x) + int(threadIdx.x);
    const int n = int(a.n);   // K n < 2^31: the arc count fits the 32-bit device indices
    pdl_wait();
    if (v < n) {
        V p[K];
#pragma unroll
        for (int j = 0; j < K; ++j) p[j] = in[j * n + v];
        const int mi = find_marked(a.mk, v);
        CubeWalk cw(v, K);
        auto target = [&](int j) {
            return (ADDR == kAddrCube) ? cw.target(cw.next_bit(), n) : __ldg(a.revE + j * n + v);
        };
        if (mi >= 0) {
            if (a.rec_part && a.rec_slot >= 0) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < K; ++j) acc += double(p[j].x) * double(p[j].x) + double(p[j].y) * double(p[j].y);
                a.rec_part[a.rec_slot * a.mk.n + mi] = acc;
            }
#pragma unroll
            for (int j = 0; j < K; ++j) out[target(j)] = mkv<V, R>(-p[j].x, -p[j].y);
        } else {
            R sx, sy;
            if constexpr (sizeof(R) == 8) {
                sum4::grouped_sum2_fixed<K>(p, sx, sy);
            } else {
                sx = p[0].x;
                sy = p[0].y;
#pragma unroll
                for (int j = 1; j < K; ++j) {
                    sx += p[j].x;
                    sy += p[j].y;
                }
            }
            const R f = em_weight<R>(a);
#pragma unroll
            for (int j = 0; j < K; ++j) out[target(j)] = mkv<V, R>(fma(f, sx, -p[j].x), fma(f, sy, -p[j].y));
        }
    }
    pdl_trigger();
}

// arc-major [n][d] <-> edge-major [d][n]: element e of the source, read in order
template <typename V, bool TO_EDGE>
__global__ void k_layout(const V *__restrict__ in, V *__restrict__ out, int64_t n, int d)
{
    const int64_t total = n * d;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        if (TO_EDGE) {
            int64_t j;
            const int64_t v = idx_div(e, d, j);
            out[j * n + v] = in[e];
        } else {
            int64_t v;
            const int64_t j = idx_div(e, n, v);
            out[v * d + j] = in[e];
        }
    }
}

}  // namespace

template <typename R, int G, int COIN>
static void launch_lanes_g(const RegArgs &a, int d, cudaStream_t st)
{
    constexpr int U = 4;
    constexpr int VPW = 32 / G;
    const int64_t warps = (a.n + VPW * U - 1) / (VPW * U);
    const int64_t grid = (warps * 32 + kThreads - 1) / kThreads;
    launch_pdl(k_coined_lanes<R, G, COIN, U>, dim3(unsigned(grid)), dim3(kThreads), 0, st, a, d);
}

template <typename R, int COIN>
static void launch_lanes(int d, const RegArgs &a, cudaStream_t st)
{
    if (d <= 1) launch_lanes_g<R, 1, COIN>(a, d, st);
    else if (d <= 2) launch_lanes_g<R, 2, COIN>(a, d, st);
    else if (d <= 4) launch_lanes_g<R, 4, COIN>(a, d, st);
    else if (d <= 8) launch_lanes_g<R, 8, COIN>(a, d, st);
    else if (d <= 16) launch_lanes_g<R, 16, COIN>(a, d, st);
    else launch_lanes_g<R, 32, COIN>(a, d, st);
}

static hw_status upload_twiddles()
{
    // once per device (the constant bank is per device); the table is the same for all
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return HW_OK;
    std::vector<double2> tw(kTwMax * (kTwMax + 1) / 2);
    for (int d = 1; d <= kTwMax; ++d)
        for (int r = 0; r < d; ++r) {
            const double ang = 2.0 * 3.14159265358979323846 * double(r) / double(d);
            tw[d * (d - 1) / 2 + r] = make_double2(std::cos(ang), std::sin(ang));
        }
    std::vector<float2> twf(tw.size());
    for (size_t i = 0; i < tw.size(); ++i) twf[i] = make_float2(float(tw[i].x), float(tw[i].y));
    hw_status s = hw_cuda(cudaMemcpyToSymbol(c_tw, tw.data(), sizeof(double2) * tw.size()),
                          "cudaMemcpyToSymbol(twiddles)");
    if (s == HW_OK)
        s = hw_cuda(cudaMemcpyToSymbol(c_twf, twf.data(), sizeof(float2) * twf.size()),
                    "cudaMemcpyToSymbol(twiddles, float)");
    if (s == HW_OK) done.push_back(dev);
    return s;
}

hw_status launch_coined_step(const hw_graph *g, hw_dtype dt, hw_coin coin, const CoinedStep &s,
                             cudaStream_t st)
{
    if (coin == HW_COIN_FOURIER) {
        hw_status ts = upload_twiddles();
        if (ts != HW_OK) return ts;
    }
    const bool regular = g->min_degree == g->max_degree && g->max_degree >= 1;
    // complex64 regular graphs up to degree 32: lane groups (complex128
    // regular graphs always take the edge-major path)
    if (regular && dt == HW_C64 && g->max_degree <= 32) {
        const int d = g->max_degree;
        RegArgs r;
        r.rev = shift_table(g, s.shift);
        r.rec_part = s.rec_part;
        r.in = s.in;
        r.out = s.out;
        r.rec_slot = s.rec_slot;
        r.n = g->n;
        r.two_over_d = 2.0 / double(d);
        r.two_over_d_f = float(2.0 / double(d));
        r.mk = s.marked;
        if (coin == HW_COIN_GROVER) launch_lanes<float, HW_COIN_GROVER>(d, r, st);
        else launch_lanes<float, HW_COIN_FOURIER>(d, r, st);
        return hw_cuda(cudaGetLastError(), "k_coined_lanes launch");
    }
    StepArgs a;
    a.two_over_d = g->d_two_over_d;
    a.two_over_d_f = g->d_two_over_d_f;
    a.row_ptr = g->d_row_ptr;
    a.rev = shift_table(g, s.shift);
    a.blk = g->d_blk;
    a.nblk = g->nblk;
    a.mk = s.marked;
    a.rec_part = s.rec_part;
    a.rec_slot = s.rec_slot;
    a.in = s.in;
    a.out = s.out;
    const int grid = g->nblk;
    if (dt == HW_C128) {
        if (coin == HW_COIN_GROVER) launch_pdl(k_coined_step<double, HW_COIN_GROVER>, dim3(grid), dim3(kThreads), 0, st, a);
        else launch_pdl(k_coined_step<double, HW_COIN_FOURIER>, dim3(grid), dim3(kThreads), 0, st, a);
    } else {
        if (coin == HW_COIN_GROVER) launch_pdl(k_coined_step<float, HW_COIN_GROVER>, dim3(grid), dim3(kThreads), 0, st, a);
        else launch_pdl(k_coined_step<float, HW_COIN_FOURIER>, dim3(grid), dim3(kThreads), 0, st, a);
    }
    return hw_cuda(cudaGetLastError(), "k_coined_step launch");
}

// The edge-major path serves every regular graph except complex64 walks of
// degree 9..16, where full lane groups of the arc-major k_coined_lanes were
// measured faster than the two-pass k_coined_em_rt (2^16-vertex hypercube: 8.2
// vs 10.5 us per step), and the hypercube Q_16 is excepted from that: with
// index-free addressing it takes k_coined_em_cube (4.4 us), and through the
// table k_coined_em_rt, so that both addressings keep the same arithmetic.
// The two-pass kernel against the arc-major ones on the 2^20-vertex
// hypercube: 180 vs 409 us complex128, 89 vs 254 us complex64.
bool coined_em_supported(const hw_graph *g, hw_coin coin, hw_dtype dt)
{
    if (!g->d_revE || (coin == HW_COIN_FOURIER && g->max_degree > 8)) return false;
    if (g->kind == HW_GRAPH_HYPERCUBE && g->max_degree == 16) return true;
    return !(dt == HW_C64 && g->max_degree >= 9 && g->max_degree <= 16);
}

hw_status launch_layout(const hw_graph *g, hw_dtype dt, const void *in, void *out, bool to_edge, cudaStream_t st)
{
    const int64_t total = g->num_arcs;
    const int grid = int(std::min<int64_t>(148 * 16, (total + 255) / 256));
    const int d = g->max_degree;
    if (dt == HW_C128) {
        if (to_edge) k_layout<double2, true><<<grid, 256, 0, st>>>(static_cast<const double2 *>(in), static_cast<double2 *>(out), g->n, d);
        else k_layout<double2, false><<<grid, 256, 0, st>>>(static_cast<const double2 *>(in), static_cast<double2 *>(out), g->n, d);
    } else {
        if (to_edge) k_layout<float2, true><<<grid, 256, 0, st>>>(static_cast<const float2 *>(in), static_cast<float2 *>(out), g->n, d);
        else k_layout<float2, false><<<grid, 256, 0, st>>>(static_cast<const float2 *>(in), static_cast<float2 *>(out), g->n, d);
    }
    return hw_cuda(cudaGetLastError(), "k_layout launch");
}

// Which degrees take k_coined_em_cube (rows in registers) rather than the
// two-pass k_coined_em_rt, from per-step times on Q_12 .. Q_20:
// complex64 from degree 16 (Q_16 4.4 vs 7.9 us, Q_20 52.9 vs 68.8 us; the
// arc-major lane groups stay faster below 16), complex128 up to degree 16
// (Q_16 11.3 vs 14.5 us, 8.7 us with the folded group sums); above 16 the
// 80+ registers of complex128 rows leave too few warps per SM and the two
// passes win (Q_20 159 vs 165 us).
template <typename R> constexpr bool cube_regs_kernel(int d)
{
    return sizeof(R) == 8 ? (d >= 9 && d <= 16) : (d >= 16 && d <= 20);
}

template <typename R, int ADDR>
static void launch_cube(int d, dim3 grid, const EmArgs &a, cudaStream_t st)
{
    if constexpr (sizeof(R) == 8) {
        switch (d) {
        case 9: launch_pdl(k_coined_em_cube<R, 9, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 10: launch_pdl(k_coined_em_cube<R, 10, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 11: launch_pdl(k_coined_em_cube<R, 11, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 12: launch_pdl(k_coined_em_cube<R, 12, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 13: launch_pdl(k_coined_em_cube<R, 13, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 14: launch_pdl(k_coined_em_cube<R, 14, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 15: launch_pdl(k_coined_em_cube<R, 15, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        default: launch_pdl(k_coined_em_cube<R, 16, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        }
    } else {
        switch (d) {
        case 16: launch_pdl(k_coined_em_cube<R, 16, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 17: launch_pdl(k_coined_em_cube<R, 17, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 18: launch_pdl(k_coined_em_cube<R, 18, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        case 19: launch_pdl(k_coined_em_cube<R, 19, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        default: launch_pdl(k_coined_em_cube<R, 20, ADDR>, grid, dim3(kThreads), 0, st, a); break;
        }
    }
}

template <typename R, int COIN>
static void launch_em(int d, int addr, const EmArgs &a, cudaStream_t st)
{
    dim3 grid(unsigned((a.n + kThreads - 1) / kThreads));
    if (a.grid2d) grid = dim3(unsigned((a.L2 + kThreads - 1) / kThreads), unsigned(a.L1));
    switch (d) {
    case 1: launch_pdl(k_coined_em<R, 1, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    case 2: launch_pdl(k_coined_em<R, 2, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    case 3: launch_pdl(k_coined_em<R, 3, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    case 4:
        if (addr == kAddrTorusFF) launch_pdl(k_coined_em<R, 4, COIN, kAddrTorusFF>, grid, dim3(kThreads), 0, st, a);
        else if (addr == kAddrTorusPS) launch_pdl(k_coined_em<R, 4, COIN, kAddrTorusPS>, grid, dim3(kThreads), 0, st, a);
        else launch_pdl(k_coined_em<R, 4, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a);
        break;
    case 5: launch_pdl(k_coined_em<R, 5, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    case 6: launch_pdl(k_coined_em<R, 6, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    case 7: launch_pdl(k_coined_em<R, 7, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    case 8: launch_pdl(k_coined_em<R, 8, COIN, kAddrTable>, grid, dim3(kThreads), 0, st, a); break;
    default:   // Grover only
        if (cube_regs_kernel<R>(d) && addr == kAddrCube)
            launch_cube<R, kAddrCube>(d, grid, a, st);
        else if (cube_regs_kernel<R>(d))
            launch_cube<R, kAddrTable>(d, grid, a, st);
        else if (addr == kAddrCube)
            launch_pdl(k_coined_em_rt<R, kAddrCube>, dim3(unsigned((a.n + kRtThreads - 1) / kRtThreads)),
                       dim3(kRtThreads), 0, st, a);
        else
            launch_pdl(k_coined_em_rt<R, kAddrTable>, dim3(unsigned((a.n + kRtThreads - 1) / kRtThreads)),
                       dim3(kRtThreads), 0, st, a);
        break;
    }
}

hw_status launch_coined_step_em(const hw_graph *g, hw_dtype dt, hw_coin coin, const CoinedStep &s, cudaStream_t st)
{
    if (coin == HW_COIN_FOURIER) {
        hw_status ts = upload_twiddles();
        if (ts != HW_OK) return ts;
    }
    EmArgs a;
    a.revE = shift_table_em(g, s.shift);
    if (!a.revE) return hw_fail(HW_EINVAL, "the persistent shift needs a graph recognised as a torus");
    a.rec_part = s.rec_part;
    a.in = s.in;
    a.out = s.out;
    a.rec_slot = s.rec_slot;
    a.n = g->n;
    a.d = g->max_degree;
    a.L1 = int32_t(g->dims[0]);
    a.L2 = int32_t(g->dims[1]);
    a.grid2d = 0;
    a.two_over_d = 2.0 / double(g->max_degree);
    a.two_over_d_f = float(2.0 / double(g->max_degree));
    a.mk = s.marked;
    int addr = kAddrTable;
    if (s.index_free && g->kind == HW_GRAPH_TORUS) {
        addr = (s.shift == kShiftPersistent) ? kAddrTorusPS : kAddrTorusFF;
        // a block row per torus row when rows are long enough to fill blocks
        a.grid2d = (a.L2 >= kThreads / 2 && a.L1 <= 65535) ? 1 : 0;
    }
    else if (s.index_free && g->kind == HW_GRAPH_HYPERCUBE && a.d > 8)
        addr = kAddrCube;
    if (dt == HW_C128) {
        if (coin == HW_COIN_GROVER) launch_em<double, HW_COIN_GROVER>(a.d, addr, a, st);
        else launch_em<double, HW_COIN_FOURIER>(a.d, addr, a, st);
    } else {
        if (coin == HW_COIN_GROVER) launch_em<float, HW_COIN_GROVER>(a.d, addr, a, st);
        else launch_em<float, HW_COIN_FOURIER>(a.d, addr, a, st);
    }
    return hw_cuda(cudaGetLastError(), "k_coined_em launch");
}

// Launch shapes of the batched Grover kernel: (threads per CTA, vertices per
// warp, rows kept in registers).
constexpr int kNumRowShapes = 12;
constexpr int kRowShapes[kNumRowShapes][3] = {
    {128, 1, 8}, {128, 2, 8}, {128, 4, 8}, {256, 1, 8}, {256, 2, 8}, {256, 4, 8},
    {128, 1, 16}, {128, 2, 16}, {128, 4, 16}, {256, 1, 16}, {256, 2, 16}, {256, 4, 16}};

template <typename R, int CPL>
static void launch_rows(const RowsArgs &a, int shape, cudaStream_t st)
{
    const int threads = kRowShapes[shape][0];
    const int64_t warps = (a.n + a.vpw - 1) / a.vpw;
    const int64_t grid = (warps * 32 + threads - 1) / threads;
    if (kRowShapes[shape][2] == 8) k_coined_rows<R, CPL, 8><<<grid, threads, 0, st>>>(a);
    else k_coined_rows<R, CPL, 16><<<grid, threads, 0, st>>>(a);
}

constexpr int kNumShapes = kNumRowShapes + 2;   // + TMA ring with 2 or 1 CTAs per SM

template <typename R, int CPL>
static hw_status launch_ring(const RingArgs &a, int ctas_per_sm, cudaStream_t st)
{
    const int smem = kRingWarps * kRingSlots * kSlotBytes;
    cudaError_t e = cudaFuncSetAttribute(k_coined_ring<R, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_coined_ring)");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t warps_needed = (a.n + 3) / 4;   // at least 4 vertices per warp
    int64_t grid = int64_t(sms) * ctas_per_sm;
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, (warps_needed + kRingWarps - 1) / kRingWarps));
    k_coined_ring<R, CPL><<<grid, kRingWarps * 32, smem, st>>>(a);
    return HW_OK;
}

static void launch_rows_dt(hw_dtype dt, int batch, RowsArgs a, int shape, cudaStream_t st)
{
    a.vpw = kRowShapes[shape][1];
    if (dt == HW_C128) launch_rows<double, 1>(a, shape, st);
    else if (batch % 2 == 0) launch_rows<float, 2>(a, shape, st);
    else launch_rows<float, 1>(a, shape, st);
}

// ring staging needs 16-byte aligned rows that fit a slot
static bool ring_ok(hw_dtype dt, int batch, const void *in, const void *out)
{
    const int rowbytes = batch * int(cplx_bytes(dt));
    return rowbytes % 16 == 0 && rowbytes <= kSlotBytes && (uintptr_t(in) % 16) == 0 && (uintptr_t(out) % 16) == 0;
}

static hw_status launch_shape(const hw_graph *g, hw_dtype dt, int batch, const RowsArgs &a, int shape,
                              cudaStream_t st)
{
    if (shape < kNumRowShapes) {
        launch_rows_dt(dt, batch, a, shape, st);
        return HW_OK;
    }
    RingArgs r;
    r.two_over_d = a.two_over_d;
    r.two_over_d_f = a.two_over_d_f;
    r.row_ptr = a.row_ptr;
    r.rev = a.rev;
    r.rec_part = a.rec_part;
    r.in = a.in;
    r.out = a.out;
    r.err = g->d_err;
    r.rec_slot = a.rec_slot;
    r.n = a.n;
    r.arcs = g->num_arcs;
    r.batch = batch;
    r.rowbytes = batch * int(cplx_bytes(dt));
    r.mk = a.mk;
    const int per_sm = (shape == kNumRowShapes) ? 2 : 1;
    if (dt == HW_C128) return launch_ring<double, 1>(r, per_sm, st);
    return launch_ring<float, 2>(r, per_sm, st);
}

// Pick the fastest launch shape for (graph, dtype, batch) by timing each
// candidate on this call's own buffers (the outputs are rewritten by the
// real launch afterwards); the choice is cached on the graph.  Synchronises
// the stream once per new key.
static hw_status tune_rows(const hw_graph *g, hw_dtype dt, int batch, const RowsArgs &base, cudaStream_t st,
                           int *best)
{
    const long long key = (long long)batch * 4 + int(dt);
    {
        std::lock_guard<std::mutex> lock(g->tune_mu);
        auto it = g->tune_rows.find(key);
        if (it != g->tune_rows.end()) { *best = it->second; return HW_OK; }
    }
    RowsArgs a = base;
    a.rec_part = nullptr;
    cudaEvent_t e0, e1;
    hw_status s = hw_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    if (s != HW_OK) return s;
    if ((s = hw_cuda(cudaEventCreate(&e1), "cudaEventCreate")) != HW_OK) { cudaEventDestroy(e0); return s; }
    float best_ms = 1e30f;
    int pick = 4;
    const int shapes = ring_ok(dt, batch, base.in, base.out) ? kNumShapes : kNumRowShapes;
    for (int c = 0; c < shapes && s == HW_OK; ++c) {
        s = launch_shape(g, dt, batch, a, c, st);   // warm-up
        if (s != HW_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) launch_shape(g, dt, batch, a, c, st);
        cudaEventRecord(e1, st);
        s = hw_cuda(cudaEventSynchronize(e1), "autotune");
        float ms = 0.f;
        if (s == HW_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (s == HW_OK && ms < best_ms) { best_ms = ms; pick = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != HW_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g->tune_mu);
        g->tune_rows[key] = pick;
    }
    *best = pick;
    return HW_OK;
}

hw_status launch_coined_step_batched(const hw_graph *g, hw_dtype dt, hw_coin coin, int batch,
                                     const CoinedStep &s, int tile, cudaStream_t st)
{
    if (coin == HW_COIN_FOURIER) {
        hw_status ts = upload_twiddles();
        if (ts != HW_OK) return ts;
        BatchArgs a;
        a.two_over_d = g->d_two_over_d;
        a.two_over_d_f = g->d_two_over_d_f;
        a.row_ptr = g->d_row_ptr;
        a.rev = shift_table(g, s.shift);
        a.mk = s.marked;
        a.rec_part = s.rec_part;
        a.rec_slot = s.rec_slot;
        a.in = s.in;
        a.out = s.out;
        a.n = int32_t(g->n);
        a.batch = batch;
        a.verts_per_warp = 4;
        const int64_t warps = (g->n + a.verts_per_warp - 1) / a.verts_per_warp;
        const int64_t grid = (warps * 32 + kThreads - 1) / kThreads;
        if (dt == HW_C128) k_coined_step_batched<double, HW_COIN_FOURIER><<<grid, kThreads, 0, st>>>(a);
        else k_coined_step_batched<float, HW_COIN_FOURIER><<<grid, kThreads, 0, st>>>(a);
        return hw_cuda(cudaGetLastError(), "k_coined_step_batched launch");
    }
    RowsArgs a;
    a.two_over_d = g->d_two_over_d;
    a.two_over_d_f = g->d_two_over_d_f;
    a.row_ptr = g->d_row_ptr;
    a.rev = shift_table(g, s.shift);
    a.rec_part = s.rec_part;
    a.in = s.in;
    a.out = s.out;
    a.rec_slot = s.rec_slot;
    a.n = g->n;
    a.batch = batch;
    a.vpw = 1;
    a.mk = s.marked;
    int shape = tile - 1;
    if (tile <= 0) {
        hw_status ts = tune_rows(g, dt, batch, a, st, &shape);
        if (ts != HW_OK) return ts;
    }
    if (shape >= kNumRowShapes && !ring_ok(dt, batch, s.in, s.out)) shape = 9;
    hw_status ls = launch_shape(g, dt, batch, a, shape, st);
    if (ls != HW_OK) return ls;
    return hw_cuda(cudaGetLastError(), "batched coined launch");
}

hw_status launch_marked_prob(const int32_t *row_ptr, hw_dtype dt, int batch, const void *psi,
                             const MarkedList &mk, double *dst, cudaStream_t st)
{
    const int total = mk.n * batch;
    const int grid = (total + 127) / 128;
    if (dt == HW_C128) k_marked_prob<double><<<grid, 128, 0, st>>>(row_ptr, psi, mk, batch, dst);
    else k_marked_prob<float><<<grid, 128, 0, st>>>(row_ptr, psi, mk, batch, dst);
    return hw_cuda(cudaGetLastError(), "k_marked_prob launch");
}

hw_status launch_record_finalize(const double *rec_part, int32_t n_marked, int64_t slots, int batch,
                                 double *record, cudaStream_t st)
{
    const int64_t total = slots * batch;
    const int64_t grid = (total + 255) / 256;
    k_record_finalize<<<grid, 256, 0, st>>>(rec_part, n_marked, slots, batch, record);
    return hw_cuda(cudaGetLastError(), "k_record_finalize launch");
}
