// Continuous-time quantum walk (Sec. 3.1): H = -gamma A - sum_{m in M} |m><m|,
// U(t) = e^{-iHt}, |psi(k dt)> = U(dt)^k |psi(0)>.
//
// hw_ctqw_expm builds U(time) densely by scaling and squaring a truncated
// Taylor series.  With Y = H time / 2^s (real symmetric),
//   e^{-iY} = sum_{k<=m} (-i)^k Y^k / k!,
// so every power is real: Q_k = Y^k / k! = (Q_{k-1} Y) / k, and
//   Re U += Q_k for k = 0 mod 4,  -= for k = 2 mod 4,
//   Im U -= Q_k for k = 1 mod 4,  += for k = 3 mod 4.
// The accumulation runs in double in the GEMM epilogue.  Then s squarings
// U <- U^2 with U symmetric: Re' = Re Re - Im Im, Im' = X + X^T, X = Re Im.
//
// hw_ctqw_evolve applies U `steps` times (ping-pong) and records the
// probability on the marked vertices after each application.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "fpconv.cuh"
#include "internal.h"
#include "sum4.cuh"

namespace {

// ------------------------------------------------------------ FP64 GEMM
// C = A1 B1 (+ sigma A2 B2), row-major n x n, register-blocked SIMT DFMA.
constexpr int BM = 64, BN = 64, BK = 16;

enum { EPI_STORE = 0, EPI_TAYLOR = 1 };

struct GemmArgs {
    const double *A1, *B1, *A2, *B2;
    double sigma;
    int n;
    int epi;
    double *out;      // C (EPI_STORE) or Q_k (EPI_TAYLOR)
    double scale;     // C *= scale before the epilogue
    double *acc;      // EPI_TAYLOR: acc += sign * C
    double sign;
    int sym_out;      // C is symmetric (a product of commuting symmetric matrices): only the
                      // tiles on and above the diagonal are computed, each written to both places
};

__global__ void __launch_bounds__(256) k_dgemm(GemmArgs g)
{
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    const int n = g.n;
    const int t = threadIdx.x;
    const int ty = t / 16, tx = t % 16;
    int bi = blockIdx.y, bj = blockIdx.x;
    if (g.sym_out) {   // blockIdx.x numbers the upper tiles row by row
        const int nb = (n + BN - 1) / BN;
        int rem = blockIdx.x;
        bi = 0;
        while (rem >= nb - bi) {
            rem -= nb - bi;
            ++bi;
        }
        bj = bi + rem;
    }
    const int i0 = bi * BM, j0 = bj * BN;
    double acc[4][4] = {};
    for (int pass = 0; pass < (g.A2 ? 2 : 1); ++pass) {
        const double *A = pass ? g.A2 : g.A1;
        const double *B = pass ? g.B2 : g.B1;
        const double sg = pass ? g.sigma : 1.0;
        for (int k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = t + 256 * q;
                const int r = e / BK, c = e % BK;
                const int gi = i0 + r, gk = k0 + c;
                As[c][r] = (gi < n && gk < n) ? A[int64_t(gi) * n + gk] * sg : 0.0;
                const int rb = e / BN, cb = e % BN;
                const int gkb = k0 + rb, gj = j0 + cb;
                Bs[rb][cb] = (gkb < n && gj < n) ? B[int64_t(gkb) * n + gj] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
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
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = i0 + ty * 4 + i;
        if (gi >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = j0 + tx * 4 + j;
            if (gj >= n) continue;
            const int64_t o = int64_t(gi) * n + gj;
            const double c = acc[i][j] * g.scale;
            g.out[o] = c;
            if (g.epi == EPI_TAYLOR) g.acc[o] += g.sign * c;
            if (g.sym_out && bi != bj) {   // the mirror element (j, i) of a tile above the diagonal
                const int64_t mo = int64_t(gj) * n + gi;
                g.out[mo] = c;
                if (g.epi == EPI_TAYLOR) g.acc[mo] += g.sign * c;
            }
        }
    }
}

hw_status dgemm(const GemmArgs &a, cudaStream_t st)
{
    const int nb = (a.n + BN - 1) / BN;
    dim3 grid(nb, (a.n + BM - 1) / BM);
    if (a.sym_out) grid = dim3(unsigned(int64_t(nb) * (nb + 1) / 2), 1);
    k_dgemm<<<grid, 256, 0, st>>>(a);
    return hw_cuda(cudaGetLastError(), "k_dgemm launch");
}

// ------------------------------------------------------------ elementwise
// Y = tau * H: -gamma*tau (times the arc's weight for a weighted W) on every
// arc, -tau added on marked diagonals.
__global__ void k_scatter_y(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ head,
                            const double *__restrict__ w, int n, double off, double *__restrict__ Y)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int a = row_ptr[v]; a < row_ptr[v + 1]; ++a) Y[int64_t(v) * n + head[a]] = w ? off * w[a] : off;
}

__global__ void k_mark_diag(MarkedList mk, int n, double diag, double *__restrict__ Y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mk.n) return;
    const int m = marked_id(mk, i);
    Y[int64_t(m) * n + m] += diag;
}

// Re U = I, Im U = 0 on and below the diagonal (the rest is never read)
__global__ void k_init_lower(int n, double *__restrict__ re, double *__restrict__ im)
{
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int j = threadIdx.x; j <= i; j += blockDim.x) {
            re[int64_t(i) * n + j] = (i == j) ? 1.0 : 0.0;
            im[int64_t(i) * n + j] = 0.0;
        }
}

// Re U = I, Im U = -Y (the k = 0 and k = 1 terms); Q_1 = Y.
__global__ void k_taylor_init(int n, const double *__restrict__ Y, double *__restrict__ re,
                              double *__restrict__ im)
{
    const int64_t total = int64_t(n) * n;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int64_t j;
        const int64_t i = idx_div(e, n, j);
        re[e] = (i == j) ? 1.0 : 0.0;
        im[e] = -Y[e];
    }
}

// lower triangle -> upper triangle (the tensor-core series accumulates below the diagonal)
__global__ void k_mirror_lower(int n, double *__restrict__ x)
{
    const int64_t total = int64_t(n) * n;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int64_t j;
        const int64_t i = idx_div(e, n, j);
        if (j > i) x[e] = x[j * n + i];
    }
}

// Im' = X + X^T
__global__ void k_sym_add(int n, const double *__restrict__ X, double *__restrict__ out)
{
    const int64_t total = int64_t(n) * n;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int64_t j;
        const int64_t i = idx_div(e, n, j);
        out[e] = X[e] + X[j * n + i];
    }
}

__device__ __forceinline__ void pack1(double2 &u, double re, double im) { u = make_double2(re, im); }
__device__ __forceinline__ void pack1(float2 &u, double re, double im)
{
    u = make_float2(fpconv::f64_to_f32_rn(re), fpconv::f64_to_f32_rn(im));
}

template <typename V>
__global__ void k_pack_u(int64_t total, const double *__restrict__ re, const double *__restrict__ im,
                         V *__restrict__ U)
{
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        V u;
        pack1(u, re[e], im[e]);
        U[e] = u;
    }
}

// ------------------------------------------------------------ sparse Taylor powers
// Q_k = Y Q_{k-1} / k with Y = tau H: row v of Q_k combines the rows of v's
// neighbours w (weight -gamma tau W_vw) and, for a marked v, its own row
// (weight -tau).  Y has d << n entries per row, so this is a sparse x dense
// product: it runs as a gather of rows, not as an n^3 GEMM.  A thread owns one
// column c of a CTA's kSpRows rows, reads Q_{k-1}[w][c] for each neighbour
// (coalesced over the CTA's 256 columns), writes Q_k[v][c] and adds
// sign Q_k[v][c] to U's real or imaginary plane in double.  Blocks run row
// block by row block inside one 256-column slab before the next slab, so the
// rows gathered by the CTAs in flight (a slab is n x 256 values) stay in L2.
// complex128: Q in double, an unweighted row's neighbour sum in groups of
// four rounded once (sum4.cuh), the group sums added in order, then one
// multiply by -gamma tau / k; weighted
// rows take one FMA per neighbour.  complex64: Q in float, the sums and
// products in float, the accumulation into U in double.
constexpr int kSpRows = 8;       // rows per CTA
constexpr int kSpCols = 256;     // columns per CTA, one per thread
constexpr int kSpGather = 16;    // neighbour values held in registers at once

struct SparsePow {
    const int32_t *row_ptr, *head;
    const double *w;             // arc weights (weighted W) or nullptr
    const float *wf;             // the same in float
    int n;
    double off, diag;            // -gamma tau / k, -tau / k
    float offf, diagf;
    MarkedList mk;
    const void *Qp;              // Q_{k-1}, n x n
    void *Qn;                    // Q_k
    double *acc;                 // Re U or Im U, n x n
    int neg;                     // acc -= Q_k instead of +=
};

__device__ __forceinline__ double sp_weight(const SparsePow &a, int e, double) { return __ldg(a.w + e); }
__device__ __forceinline__ float sp_weight(const SparsePow &a, int e, float) { return __ldg(a.wf + e); }
__device__ __forceinline__ double sp_off(const SparsePow &a, double) { return a.off; }
__device__ __forceinline__ float sp_off(const SparsePow &a, float) { return a.offf; }
__device__ __forceinline__ double sp_diag(const SparsePow &a, double) { return a.diag; }
__device__ __forceinline__ float sp_diag(const SparsePow &a, float) { return a.diagf; }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return fpconv::f32_to_f64(x); }

// VEC adjacent columns per thread, moved as one vector
template <typename T, int VEC> struct SpVec;
template <> struct SpVec<double, 2> { using V = double2; };
template <> struct SpVec<float, 4> { using V = float4; };
template <> struct SpVec<float, 2> { using V = float2; };
template <> struct SpVec<double, 1> { using V = double; };
template <> struct SpVec<float, 1> { using V = float; };

template <typename T, int VEC>
__device__ __forceinline__ void sp_load(T (&x)[VEC], const T *p)
{
    const typename SpVec<T, VEC>::V v = *reinterpret_cast<const typename SpVec<T, VEC>::V *>(p);
    const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int k = 0; k < VEC; ++k) x[k] = e[k];
}

template <typename T, int VEC>
__device__ __forceinline__ void sp_store(T *p, const T (&x)[VEC])
{
    typename SpVec<T, VEC>::V v;
    T *e = reinterpret_cast<T *>(&v);
#pragma unroll
    for (int k = 0; k < VEC; ++k) e[k] = x[k];
    *reinterpret_cast<typename SpVec<T, VEC>::V *>(p) = v;
}

// neighbour sum of one column, terms x[0..deg) with deg <= kSpGather:
// complex128 unweighted in groups of four rounded once (sum4_rn, a short last
// group padded with -0), the group sums added in order; otherwise sequential
// from 0; constant indices, so that x stays in registers
template <typename T, bool WEIGHTED, int VEC>
__device__ __forceinline__ T sp_sum(const SparsePow &a, int e0, int deg, const T (&x)[kSpGather][VEC], int k)
{
    T sum = 0;
    if constexpr (WEIGHTED) {
#pragma unroll
        for (int j = 0; j < kSpGather; ++j)
            if (j < deg) sum = fma(sp_weight(a, e0 + j, T(0)), x[j][k], sum);
    } else if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int g0 = 0; g0 < kSpGather; g0 += 4) {
            if (g0 < deg) {
                const double q = sum4::sum4_rn(x[g0][k], g0 + 1 < deg ? x[g0 + 1][k] : -0.0,
                                               g0 + 2 < deg ? x[g0 + 2][k] : -0.0, g0 + 3 < deg ? x[g0 + 3][k] : -0.0);
                sum = (g0 == 0) ? q : sum + q;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < kSpGather; ++j)
            if (j < deg) sum += x[j][k];
    }
    return sum;
}

// the same sums for any degree, four neighbours at a time
template <typename T, bool WEIGHTED, int VEC>
__device__ __forceinline__ void sp_sum_long(const SparsePow &a, const T *Qp, int64_t n, int c0, int e0, int deg,
                                            T (&sum)[VEC])
{
#pragma unroll
    for (int k = 0; k < VEC; ++k) sum[k] = 0;
    for (int g0 = 0; g0 < deg; g0 += 4) {
        T x[4][VEC];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (g0 + u < deg) sp_load<T, VEC>(x[u], Qp + int64_t(__ldg(a.head + e0 + g0 + u)) * n + c0);
#pragma unroll
            for (int k = 0; k < VEC; ++k)
                if (g0 + u >= deg) x[u][k] = (sizeof(T) == 8 && !WEIGHTED) ? T(-0.0) : T(0);
        }
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            if constexpr (WEIGHTED) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (g0 + u < deg) sum[k] = fma(sp_weight(a, e0 + g0 + u, T(0)), x[u][k], sum[k]);
            } else if constexpr (sizeof(T) == 8) {
                const double q = sum4::sum4_rn(x[0][k], x[1][k], x[2][k], x[3][k]);
                sum[k] = (g0 == 0) ? q : sum[k] + q;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (g0 + u < deg) sum[k] += x[u][k];
            }
        }
    }
}

template <typename T, bool WEIGHTED, int VEC>
__global__ void __launch_bounds__(kSpCols) k_taylor_sparse(SparsePow a)
{
    const int c0 = (int(blockIdx.y) * kSpCols + int(threadIdx.x)) * VEC;
    if (c0 >= a.n) return;
    const T *__restrict__ Qp = static_cast<const T *>(a.Qp);
    T *__restrict__ Qn = static_cast<T *>(a.Qn);
    const int64_t n = a.n;
    const int v0 = int(blockIdx.x) * kSpRows;
    const int v1 = min(a.n, v0 + kSpRows);
    for (int v = v0; v < v1; ++v) {
        const int64_t e = int64_t(v) * n + c0;
        double u[VEC];   // U's plane, fetched before the gathers so its latency overlaps them
#pragma unroll
        for (int k = 0; k < VEC; k += (VEC > 1 ? 2 : 1)) {
            if constexpr (VEC > 1) {
                const double2 w2 = *reinterpret_cast<const double2 *>(a.acc + e + k);
                u[k] = w2.x;
                u[k + 1] = w2.y;
            } else {
                u[k] = a.acc[e + k];
            }
        }
        const int e0 = __ldg(a.row_ptr + v), deg = __ldg(a.row_ptr + v + 1) - e0;
        T sum[VEC];
        if (deg <= kSpGather) {
            T x[kSpGather][VEC];
#pragma unroll
            for (int j = 0; j < kSpGather; ++j)
                if (j < deg) sp_load<T, VEC>(x[j], Qp + int64_t(__ldg(a.head + e0 + j)) * n + c0);
#pragma unroll
            for (int k = 0; k < VEC; ++k) sum[k] = sp_sum<T, WEIGHTED, VEC>(a, e0, deg, x, k);
        } else {
            sp_sum_long<T, WEIGHTED, VEC>(a, Qp, n, c0, e0, deg, sum);
        }
        T q[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) q[k] = sp_off(a, T(0)) * sum[k];
        if (marked_find(a.mk, v) >= 0) {
            T own[VEC];
            sp_load<T, VEC>(own, Qp + e);
#pragma unroll
            for (int k = 0; k < VEC; ++k) q[k] = fma(sp_diag(a, T(0)), own[k], q[k]);
        }
        sp_store<T, VEC>(Qn + e, q);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const double qd = to_f64(q[k]);
            u[k] = a.neg ? u[k] - qd : u[k] + qd;
        }
#pragma unroll
        for (int k = 0; k < VEC; k += (VEC > 1 ? 2 : 1)) {
            if constexpr (VEC > 1) *reinterpret_cast<double2 *>(a.acc + e + k) = make_double2(u[k], u[k + 1]);
            else a.acc[e + k] = u[k];
        }
    }
}

// Re U = I, Im U = 0, Q_0 = I
template <typename T>
__global__ void k_taylor_identity(int n, double *__restrict__ re, double *__restrict__ im, T *__restrict__ q0)
{
    const int64_t total = int64_t(n) * n;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int64_t j;
        const int64_t i = idx_div(e, n, j);
        re[e] = (i == j) ? 1.0 : 0.0;
        im[e] = 0.0;
        q0[e] = (i == j) ? T(1) : T(0);
    }
}

int ew_grid(int64_t total) { return int(std::min<int64_t>(148 * 32, (total + 255) / 256)); }
int row_grid(int64_t rows) { return int(std::min<int64_t>(148 * 16, std::max<int64_t>(rows, 1))); }

// ------------------------------------------------------------ apply U
// y[i][b] = sum_j U[i][j] x[j][b].  One warp per row; lanes stride the
// columns (coalesced reads of U), x is staged in shared memory in chunks.
// A marked row also writes |y|^2 into the record partials.
constexpr int kApplyThreads = 256;
constexpr int kApplyChunk = 2048;   // columns of x staged per pass

template <typename R>
struct Cx2;
template <> struct Cx2<double> { using T = double2; };
template <> struct Cx2<float> { using T = float2; };

template <typename R, int BT>
__global__ void __launch_bounds__(kApplyThreads)
k_apply(const void *U_, const void *x_, void *y_, int n, int batch, MarkedList mk, double *rec_part,
        int64_t rec_slot)
{
    using V = typename Cx2<R>::T;
    extern __shared__ unsigned char smem_raw[];
    V *xs = reinterpret_cast<V *>(smem_raw);
    const V *__restrict__ U = static_cast<const V *>(U_);
    const V *__restrict__ x = static_cast<const V *>(x_);
    V *__restrict__ y = static_cast<V *>(y_);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (kApplyThreads / 32) + warp;
    pdl_wait();   // x is the previous application's output
    for (int b0 = 0; b0 < batch; b0 += BT) {
        const int nb = min(BT, batch - b0);
        R ax[BT], ay[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) { ax[b] = 0; ay[b] = 0; }
        for (int c0 = 0; c0 < n; c0 += kApplyChunk) {
            const int cn = min(kApplyChunk, n - c0);
            __syncthreads();
            for (int e = threadIdx.x; e < cn * nb; e += kApplyThreads) {
                const int j = e / nb, b = e % nb;
                xs[j * BT + b] = x[int64_t(c0 + j) * batch + b0 + b];
            }
            __syncthreads();
            if (i < n) {
                const V *Ui = U + int64_t(i) * n + c0;
                for (int j = lane; j < cn; j += 32) {
                    const V u = Ui[j];
#pragma unroll
                    for (int b = 0; b < BT; ++b) {
                        if (b < nb) {
                            const V q = xs[j * BT + b];
                            ax[b] = fma(u.x, q.x, fma(-u.y, q.y, ax[b]));
                            ay[b] = fma(u.x, q.y, fma(u.y, q.x, ay[b]));
                        }
                    }
                }
            }
        }
        if (i < n) {
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                R sx = ax[b], sy = ay[b];
                for (int o = 16; o > 0; o >>= 1) {
                    sx += __shfl_xor_sync(0xffffffffu, sx, o);
                    sy += __shfl_xor_sync(0xffffffffu, sy, o);
                }
                ax[b] = sx;
                ay[b] = sy;
            }
            if (lane < nb) {
                R ox = 0, oy = 0;
#pragma unroll
                for (int b = 0; b < BT; ++b)
                    if (b == lane) { ox = ax[b]; oy = ay[b]; }
                V o;
                o.x = ox;
                o.y = oy;
                y[int64_t(i) * batch + b0 + lane] = o;
                if (rec_part && rec_slot >= 0) {
                    // marked rows: |y|^2 into the partials [slot][mi][batch]
                    const int mi = marked_find(mk, int(i));
                    if (mi >= 0)
                        rec_part[(rec_slot * mk.n + mi) * batch + b0 + lane] =
                            double(ox) * double(ox) + double(oy) * double(oy);
                }
            }
        }
    }
    pdl_trigger();
}

template <typename R, int BT>
hw_status launch_apply_bt(const void *U, const void *x, void *y, int n, int batch, const MarkedList &mk,
                          double *rec_part, int64_t rec_slot, cudaStream_t st)
{
    using V = typename Cx2<R>::T;
    const int grid = (n + kApplyThreads / 32 - 1) / (kApplyThreads / 32);
    const size_t smem = sizeof(V) * kApplyChunk * BT;
    cudaError_t e = cudaFuncSetAttribute(k_apply<R, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_apply)");
    launch_pdl(k_apply<R, BT>, dim3(grid), dim3(kApplyThreads), smem, st, U, x, y, n, batch, mk, rec_part, rec_slot);
    return hw_cuda(cudaGetLastError(), "k_apply launch");
}

template <typename R>
hw_status launch_apply(const void *U, const void *x, void *y, int n, int batch, const MarkedList &mk,
                       double *rec_part, int64_t rec_slot, cudaStream_t st)
{
    if (batch == 1) return launch_apply_bt<R, 1>(U, x, y, n, batch, mk, rec_part, rec_slot, st);
    return launch_apply_bt<R, 4>(U, x, y, n, batch, mk, rec_part, rec_slot, st);
}

// ------------------------------------------------------------ apply U, complex128, three real products
// y = U x for one complex128 state with three real multiply-adds per element
// instead of four (the 3M form of a complex product): with U = A + iB and
// x = p + iq, P1 = A p, P2 = B q, P3 = (A + B)(p + q), and
// y = (P1 - P2) + i (P3 - P1 - P2).  S = A + B is formed once per call
// (k_sum_plane), p + q by the application that writes x.  The FP64 pipe bounds the
// four-product kernel, so a quarter of its work goes; the bytes read grow from
// 16 to 24 per element (U and S).
// Four warps (rows) per CTA and 1024 staged columns (24 KB), so that up to
// seven CTAs share an SM: n = 4096 gives 1024 CTAs, 6.9 per SM, and the SMs
// with one CTA more than the others wait 1/7 instead of 1/4 of the time
// (eight rows per CTA and 48 KB gave 3.5 per SM, four at most).
constexpr int k3mThreads = 128;
constexpr int k3mChunk = 1024;

// S[e] = Re U[e] + Im U[e] (also used for the start state's p + q)
__global__ void k_sum_plane(const double2 *__restrict__ U, double *__restrict__ S, int64_t count)
{
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < count; e += int64_t(gridDim.x) * blockDim.x) {
        const double2 u = U[e];
        S[e] = u.x + u.y;
    }
}

__global__ void __launch_bounds__(k3mThreads, 7)
k_apply_3m(const double2 *__restrict__ U, const double *__restrict__ S, const double2 *__restrict__ x,
           const double *__restrict__ xsum, double2 *__restrict__ y, double *__restrict__ ysum, int n,
           MarkedList mk, double *rec_part, int64_t rec_slot)
{
    extern __shared__ unsigned char smem_raw[];
    double2 *xs = reinterpret_cast<double2 *>(smem_raw);
    double *ss = reinterpret_cast<double *>(xs + k3mChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (k3mThreads / 32) + warp;
    pdl_wait();   // x is the previous application's output
    double p1 = 0, p2 = 0, p3 = 0;
    for (int c0 = 0; c0 < n; c0 += k3mChunk) {
        const int cn = min(k3mChunk, n - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < cn; j += k3mThreads) {
            xs[j] = x[c0 + j];
            ss[j] = xsum[c0 + j];
        }
        __syncthreads();
        if (i < n) {
            const double2 *Ui = U + int64_t(i) * n + c0;
            const double *Si = S + int64_t(i) * n + c0;
            // four columns per lane in flight (each lane still adds its
            // columns in increasing order)
            int j = lane;
            for (; j + 96 < cn; j += 128) {
                double2 u[4];
                double sv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u[q] = Ui[j + 32 * q];
                    sv[q] = Si[j + 32 * q];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double2 xq = xs[j + 32 * q];
                    p1 = fma(u[q].x, xq.x, p1);
                    p2 = fma(u[q].y, xq.y, p2);
                    p3 = fma(sv[q], ss[j + 32 * q], p3);
                }
            }
            for (; j < cn; j += 32) {
                const double2 u = Ui[j], q = xs[j];
                p1 = fma(u.x, q.x, p1);
                p2 = fma(u.y, q.y, p2);
                p3 = fma(Si[j], ss[j], p3);
            }
        }
    }
    if (i < n) {
        for (int o = 16; o > 0; o >>= 1) {
            p1 += __shfl_xor_sync(0xffffffffu, p1, o);
            p2 += __shfl_xor_sync(0xffffffffu, p2, o);
            p3 += __shfl_xor_sync(0xffffffffu, p3, o);
        }
        if (lane == 0) {
            const double ox = p1 - p2, oy = (p3 - p1) - p2;
            y[i] = make_double2(ox, oy);
            ysum[i] = ox + oy;   // the next application's p + q
            if (rec_part && rec_slot >= 0) {
                const int mi = marked_find(mk, i);
                if (mi >= 0) rec_part[rec_slot * mk.n + mi] = ox * ox + oy * oy;
            }
        }
    }
    pdl_trigger();
}

hw_status launch_apply_3m(const void *U, const double *S, const void *x, const double *xsum, void *y, double *ysum,
                          int n, const MarkedList &mk, double *rec_part, int64_t rec_slot, cudaStream_t st)
{
    const int grid = (n + k3mThreads / 32 - 1) / (k3mThreads / 32);
    const size_t smem = (sizeof(double2) + sizeof(double)) * k3mChunk;
    cudaError_t e = cudaFuncSetAttribute(k_apply_3m, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_apply_3m)");
    launch_pdl(k_apply_3m, dim3(grid), dim3(k3mThreads), smem, st, static_cast<const double2 *>(U), S,
               static_cast<const double2 *>(x), xsum, static_cast<double2 *>(y), ysum, n, mk, rec_part, rec_slot);
    return hw_cuda(cudaGetLastError(), "k_apply_3m launch");
}

// ------------------------------------------------------------ apply a symmetric U
// U = U^T (complex symmetric, complex64): every off-diagonal 64 x 64 block U_IJ
// (I < J) is read once and gives both y_I += U_IJ x_J and y_J += U_IJ^T x_I,
// so one application reads n^2/2 elements.  Before the first application the
// blocks on and above the diagonal are packed (k_sym_pack), each a contiguous
// 32 KB (zero past n), in the order the block pass walks them: packed, the
// 68 MB of n = 4096 stay in L2 from one application to the next, while read in
// place from the dense matrix (512-byte row pieces 32 KB apart) the same bytes
// came from DRAM every time.  Pass 1 (k_apply_sym) forms every block's row and
// column sums into per-block partials; pass 2 (k_apply_sym_reduce) adds a
// vertex's partials in a fixed order and writes y (and the record).
constexpr int kSymB = 64;
constexpr uint32_t kSymTileBytes = kSymB * kSymB * sizeof(float2);

// upper block b (row-major over the blocks on and above the diagonal) ->
// (I, J): I is the last row whose first block S(I) = I nb - I (I - 1) / 2 is
// at most b, estimated from the root of S(I) = b and then fixed exactly
__device__ __forceinline__ int64_t sym_row_start(int I, int nb)
{
    return int64_t(I) * nb - int64_t(I) * (I - 1) / 2;
}

__device__ __forceinline__ void sym_block_ij(int b, int nb, int &I, int &J)
{
    const float q = float(2 * nb + 1);
    int i = int((q - sqrtf(fmaxf(q * q - 8.f * float(b), 0.f))) * 0.5f);
    i = max(0, min(i, nb - 1));
    while (i > 0 && sym_row_start(i, nb) > b) --i;
    while (i + 1 < nb && sym_row_start(i + 1, nb) <= b) ++i;
    I = i;
    J = i + int(b - sym_row_start(i, nb));
}

// one CTA per upper block b (row-major over the upper triangle).  Within a
// packed row, columns 4g and 4g + 1 come first (positions 2g, 2g + 1), then
// columns 4g + 2 and 4g + 3 (positions 32 + 2g, 32 + 2g + 1): the block pass
// reads a row's column pairs as 16-byte vectors, 16 lanes side by side
__device__ __forceinline__ int sym_col_pos(int c) { return ((c & 2) << 4) + ((c >> 2) << 1) + (c & 1); }

__global__ void __launch_bounds__(256) k_sym_pack(const float2 *__restrict__ U, int n, int nb,
                                                  float2 *__restrict__ P)
{
    int I, J;
    sym_block_ij(int(blockIdx.x), nb, I, J);
    const int r0 = I * kSymB, c0 = J * kSymB;
    float2 *__restrict__ dst = P + int64_t(blockIdx.x) * kSymB * kSymB;
    for (int e = threadIdx.x; e < kSymB * kSymB; e += blockDim.x) {
        const int r = e / kSymB, c = e % kSymB;
        dst[r * kSymB + sym_col_pos(c)] =
            (r0 + r < n && c0 + c < n) ? U[int64_t(r0 + r) * n + c0 + c] : make_float2(0.f, 0.f);
    }
}

// The block pass, a persistent kernel: each CTA walks the packed blocks
// b = blockIdx.x, + gridDim.x, ... through two 32 KB stages, the next block
// arriving (one cp.async.bulk) while the current one is summed.  128 threads
// per block: half-warp h of warp w holds rows 16w + 8h .. 16w + 8h + 7, lane
// l of it columns 4l .. 4l + 3 (32 elements a thread, each read from shared
// memory once, as two 16-byte vectors per row, and used for both sums: its
// row's with x_J and its column's with x_I).  Row sums over the 16 lanes of a
// half-warp: a fixed halving butterfly.  Column sums: one halving step across
// the two half-warps, then the 4 warps added in order through shared memory.
constexpr int kSymStages = 2;
constexpr int kSymThreads = 128;
constexpr uint64_t kSymWaitNs = 2000000000ull;   // bounded stage waits (2 s)

__device__ __forceinline__ uint32_t sym_smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool sym_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
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
            else if (t - t0 > kSymWaitNs) return false;
        }
    }
}

// one thread: packed block b into the stage, completion on bar
__device__ __forceinline__ void sym_issue(const float2 *P, int b, uint32_t dst, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kSymTileBytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(P + int64_t(b) * kSymB * kSymB), "r"(kSymTileBytes), "r"(bar)
                 : "memory");
}

// acc += u x (complex, one rounding per fma: re then im)
__device__ __forceinline__ void cmac(float &re, float &im, float ux, float uy, float2 v)
{
    re = fmaf(ux, v.x, fmaf(-uy, v.y, re));
    im = fmaf(ux, v.y, fmaf(uy, v.x, im));
}

__global__ void __launch_bounds__(kSymThreads) k_apply_sym(const float2 *__restrict__ P, const void *x_, int n,
                                                           int nb, int nblocks, void *prow_, void *pcol_, int *err)
{
    extern __shared__ __align__(128) unsigned char sym_tma_smem[];
    // [stage][row * 32 + k]: float4 k < 16 holds columns 4k, 4k + 1; 16 + k columns 4k + 2, 4k + 3
    float4(*tile)[kSymB * kSymB / 2] = reinterpret_cast<float4(*)[kSymB * kSymB / 2]>(sym_tma_smem);
    __shared__ float4 cpart[kSymThreads / 32][32];   // [warp][lane]: two columns over the warp's 16 rows
    __shared__ __align__(8) uint64_t bars[kSymStages];
    __shared__ int failed;
    const float2 *__restrict__ x = static_cast<const float2 *>(x_);
    float *__restrict__ prow = static_cast<float *>(prow_);   // the complex partials as (re, im) floats
    float4 *__restrict__ pcol = static_cast<float4 *>(pcol_);  // two complex partials per float4
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const int hg = l >> 4, cg = l & 15;      // half-warp (8 rows) and column group (4 columns)
    const int rbase = 16 * w + 8 * hg;       // this thread's first row in the block
    if (t == 0) {
        failed = 0;
        for (int k = 0; k < kSymStages; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sym_smem_addr(&bars[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // U does not change between applications: the first blocks load before the wait
        for (int k = 0; k < kSymStages; ++k) {
            const int b = blockIdx.x + k * gridDim.x;
            if (b < nblocks) sym_issue(P, b, sym_smem_addr(&tile[k][0]), sym_smem_addr(&bars[k]));
        }
    }
    __syncthreads();
    pdl_wait();   // x is the previous application's output; the partials are free again
    const float2 zero = make_float2(0.f, 0.f);
    int k = 0;
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x, ++k) {
        const int stage = k % kSymStages;
        int I, J;
        sym_block_ij(b, nb, I, J);
        const int r0 = I * kSymB + rbase, c0 = J * kSymB + 4 * cg;
        // x_J at this thread's four columns, x_I at its eight rows (zero past
        // n, where the packed block is zero)
        float2 xj[4], xi[8];
        if ((J + 1) * kSymB <= n) {   // block inside n (uniform): no guards
#pragma unroll
            for (int j = 0; j < 4; ++j) xj[j] = __ldg(x + c0 + j);
#pragma unroll
            for (int i = 0; i < 8; ++i) xi[i] = __ldg(x + r0 + i);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) xj[j] = (c0 + j < n) ? __ldg(x + c0 + j) : zero;
#pragma unroll
            for (int i = 0; i < 8; ++i) xi[i] = (r0 + i < n) ? __ldg(x + r0 + i) : zero;
        }
        if (t == 0 && !sym_wait(sym_smem_addr(&bars[stage]), uint32_t((k / kSymStages) & 1))) {
            failed = 1;
            atomicExch(err, 1);
        }
        __syncthreads();
        if (failed) break;   // uniform: the stage never filled
        const float4 *sU = tile[stage];
        float rs[16];                       // rs[2i], rs[2i+1]: row rbase + i over the 4 columns (re, im)
        float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // column 4cg + j over the 8 rows
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 ua = sU[(rbase + i) * 32 + cg];        // columns 4cg, 4cg + 1
            const float4 ub = sU[(rbase + i) * 32 + 16 + cg];   // columns 4cg + 2, 4cg + 3
            float re = 0.f, im = 0.f;
            cmac(re, im, ua.x, ua.y, xj[0]);
            cmac(re, im, ua.z, ua.w, xj[1]);
            cmac(re, im, ub.x, ub.y, xj[2]);
            cmac(re, im, ub.z, ub.w, xj[3]);
            rs[2 * i] = re;
            rs[2 * i + 1] = im;
            cmac(cs[0], cs[1], ua.x, ua.y, xi[i]);
            cmac(cs[2], cs[3], ua.z, ua.w, xi[i]);
            cmac(cs[4], cs[5], ub.x, ub.y, xi[i]);
            cmac(cs[6], cs[7], ub.z, ub.w, xi[i]);
        }
        // rows: halving butterfly over the half-warp's 16 lanes; at offset o a
        // lane keeps the half of its values that its bit o selects and adds
        // the partner's copy of that half, so after offsets 8, 4, 2, 1 lane cg
        // holds value cg: row rbase + (cg >> 1), component cg & 1
#pragma unroll
        for (int h = 8, o = 8; h >= 1; h >>= 1, o >>= 1) {
            const bool up = (l & o) != 0;
#pragma unroll
            for (int q = 0; q < h; ++q) {
                const float keep = up ? rs[q + h] : rs[q];
                const float send = up ? rs[q] : rs[q + h];
                rs[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        prow[((int64_t(I) * nb + J) * kSymB + rbase + (cg >> 1)) * 2 + (cg & 1)] = rs[0];
        // columns: the two half-warps, then the warps; half-warp hg keeps
        // columns 4cg + 2hg and 4cg + 2hg + 1
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float keep = hg ? cs[q + 4] : cs[q];
            const float send = hg ? cs[q] : cs[q + 4];
            cs[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
        cpart[w][l] = make_float4(cs[0], cs[1], cs[2], cs[3]);
        __syncthreads();   // the stage and cpart are read and written
        if (t == 0) {
            const int bn = b + kSymStages * gridDim.x;
            // order the generic reads of the stage before the async-proxy refill
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (bn < nblocks) sym_issue(P, bn, sym_smem_addr(&tile[stage][0]), sym_smem_addr(&bars[stage]));
        }
        if (w == 0 && I != J) {   // column sums of the block, the 4 warps added in order
            float4 c = cpart[0][l];
#pragma unroll
            for (int v = 1; v < kSymThreads / 32; ++v) {
                const float4 d = cpart[v][l];
                c.x += d.x;
                c.y += d.y;
                c.z += d.z;
                c.w += d.w;
            }
            pcol[((int64_t(J) * nb + I) * kSymB) / 2 + 2 * cg + hg] = c;
        }
        // cpart is written again only after the next tile's barrier, which warp 0 reaches after reading it
    }
    // on a failed wait, wait (bounded) for every stage still in flight, so no
    // bulk copy writes this CTA's shared memory after it exits
    if (failed && t == 0) {
        for (int kk = k; kk < k + kSymStages; ++kk) {
            const int64_t bk = int64_t(blockIdx.x) + int64_t(kk) * gridDim.x;
            if (bk < nblocks) sym_wait(sym_smem_addr(&bars[kk % kSymStages]), uint32_t((kk / kSymStages) & 1));
        }
    }
    pdl_trigger();
}

// kSymSub threads per vertex: thread s adds the partials of blocks s,
// s + kSymSub, ... in order (four loads issued before their adds), then a
// fixed shuffle tree combines the kSymSub sums
constexpr int kSymSub = 16;

__global__ void __launch_bounds__(256) k_apply_sym_reduce(const void *prow_, const void *pcol_, int n, int nb,
                                                          void *y_, MarkedList mk, double *rec_part,
                                                          int64_t rec_slot)
{
    const float2 *__restrict__ prow = static_cast<const float2 *>(prow_);
    const float2 *__restrict__ pcol = static_cast<const float2 *>(pcol_);
    float2 *__restrict__ y = static_cast<float2 *>(y_);
    const int i = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / kSymSub);
    const int sub = threadIdx.x % kSymSub;
    pdl_wait();
    float sx = 0.f, sy = 0.f;
    if (i < n) {
        const int I = i / kSymB, r = i % kSymB;
        for (int K0 = sub; K0 < nb; K0 += 4 * kSymSub) {
            float2 p[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // block (I, K) for K >= I, its mirror (K, I) for K < I
                const int K = K0 + u * kSymSub;
                if (K < nb)
                    p[u] = (K >= I) ? prow[(int64_t(I) * nb + K) * kSymB + r] : pcol[(int64_t(I) * nb + K) * kSymB + r];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (K0 + u * kSymSub < nb) {
                    sx += p[u].x;
                    sy += p[u].y;
                }
            }
        }
    }
    for (int o = 1; o < kSymSub; o <<= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (i < n && sub == 0) {
        y[i] = make_float2(sx, sy);
        if (rec_part && rec_slot >= 0) {
            const int mi = marked_find(mk, int(i));
            if (mi >= 0) rec_part[rec_slot * mk.n + mi] = double(sx) * double(sx) + double(sy) * double(sy);
        }
    }
    pdl_trigger();
}

// the two passes of one application; P from k_sym_pack.  The block pass
// loads its first blocks before its dependency wait, which orders only the
// launch before it; so the first application after the pack (first = true)
// is launched without programmatic dependency, after the pack has completed.
hw_status launch_apply_sym(const float2 *P, const void *x, void *y, int n, void *prow, void *pcol,
                           const MarkedList &mk, double *rec_part, int64_t rec_slot, cudaStream_t st, int *err,
                           bool first)
{
    const int nb = (n + kSymB - 1) / kSymB;
    const int blocks = nb * (nb + 1) / 2;
    // resident CTAs per device (the shared-memory attribute is set per device too)
    static std::mutex mu;
    static std::map<int, int> grids;
    const size_t smem = size_t(kSymTileBytes) * kSymStages;
    int dev = 0, grid = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = grids.find(dev);
        if (it != grids.end()) {
            grid = it->second;
        } else {
            cudaError_t e = cudaFuncSetAttribute(k_apply_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_apply_sym)");
            int sms = 0, per = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_sym, kSymThreads, smem);
            if (e != cudaSuccess) return hw_cuda(e, "occupancy (k_apply_sym)");
            grid = grids[dev] = sms * std::max(per, 1);
        }
    }
    cudaError_t e;
    if (first) {
        k_apply_sym<<<std::min(grid, blocks), kSymThreads, smem, st>>>(P, x, n, nb, blocks, prow, pcol, err);
        e = cudaGetLastError();
    } else {
        e = launch_pdl(k_apply_sym, dim3(std::min(grid, blocks)), dim3(kSymThreads), smem, st, P, x, n, nb, blocks,
                       prow, pcol, err);
    }
    if (e != cudaSuccess) return hw_cuda(e, "k_apply_sym launch");
    e = launch_pdl(k_apply_sym_reduce, dim3(int((int64_t(n) * kSymSub + 255) / 256)), dim3(256), 0, st,
                   (const void *)prow, (const void *)pcol, n, nb, y, mk, rec_part, rec_slot);
    return hw_cuda(e, "k_apply_sym_reduce launch");
}

struct DevBuf {
    cudaStream_t st;
    void *p = nullptr;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    hw_status get(size_t bytes, const char *what)
    {
        return hw_cuda(hw_malloc_async(&p, std::max<size_t>(bytes, 16), st), what);
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
    ~DevBuf() { if (p) cudaFreeAsync(p, st); }
};

}  // namespace

// Taylor degree and squarings (exposed for tests through hw_ctqw_plan).
static void ctqw_plan(double norm1, int *m_out, int *s_out)
{
    int s = 0;
    while (norm1 / std::ldexp(1.0, s) > 0.5) ++s;
    const double theta = norm1 / std::ldexp(1.0, s);
    int m = 1;
    // smallest m with theta^(m+1)/(m+1)! < 2^-60
    double term = theta;   // theta^(m+1)/(m+1)! for m = 0
    while (m < 30) {
        term = term * theta / double(m + 1);
        if (term < std::ldexp(1.0, -60)) break;
        ++m;
    }
    *m_out = std::max(m, 1);
    *s_out = s;
}

extern "C" hw_status hw_ctqw_plan(const hw_graph *g, double gamma, const int32_t *marked,
                                  int32_t n_marked, double time, int32_t *degree, int32_t *squarings)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    // ||H||_1 = max over v of (gamma sum_w |W_vw| + [v in M]) (= gamma d_v + [v
    // in M] unweighted): the largest row of W, or a marked vertex's row,
    // whichever is larger (O(n_marked), no pass over the graph)
    auto row = [&](int64_t v) {
        return g->weighted ? g->h_rowabs[size_t(v)] : double(g->h_row_ptr[v + 1] - g->h_row_ptr[v]);
    };
    double norm1 = std::fabs(gamma) * (g->weighted ? g->max_rowabs : double(g->max_degree));
    for (int32_t i = 0; i < n_marked; ++i)
        if (marked && marked[i] >= 0 && marked[i] < g->n)
            norm1 = std::max(norm1, std::fabs(gamma) * row(marked[i]) + 1.0);
    norm1 *= std::fabs(time);
    int m, s;
    ctqw_plan(norm1, &m, &s);
    if (degree) *degree = m;
    if (squarings) *squarings = s;
    return HW_OK;
}

namespace {
// I[v][v] = 1 in a zeroed n x n complex matrix
template <typename V>
__global__ void k_unit_diagonal(V *__restrict__ I, int64_t n)
{
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) {
        V one;
        one.x = 1;
        one.y = 0;
        I[v * n + v] = one;
    }
}
}  // namespace

extern "C" hw_status hw_ctqw_expm(const hw_graph *g, double gamma, const int32_t *marked,
                                  int32_t n_marked, double time, hw_dtype dt, void *U_out,
                                  const hw_opts *opts, void *stream)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (!U_out) return hw_fail(HW_EINVAL, "U_out is NULL");
    if ((uintptr_t)U_out % cplx_bytes(dt)) return hw_fail(HW_EINVAL, "U_out misaligned");
    if (!std::isfinite(gamma) || !std::isfinite(time)) return hw_fail(HW_EINVAL, "gamma/time not finite");
    if (n_marked < 0 || (n_marked > 0 && !marked)) return hw_fail(HW_EINVAL, "bad marked list");
    if (g->n > 32768) return hw_fail(HW_EUNSUPPORTED, "dense U limited to n <= 32768 (n = %lld)", (long long)g->n);
    int dev = -1;
    hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != HW_OK) return s;
    if (dev != g->device) return hw_fail(HW_EINVAL, "graph lives on device %d, current is %d", g->device, dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (g->complex_weights) {
        // a complex Hermitian W: the powers of H are complex, so U is
        // e^{-iH time} applied by the sparse series to every column of the
        // identity at once (batch n; the [vertex][column] states are U row-major)
        const int64_t nn = g->n;
        const size_t bytes = size_t(nn) * size_t(nn) * cplx_bytes(dt);
        void *eye = nullptr;
        if ((s = hw_cuda(hw_malloc_async(&eye, bytes, st), "scratch allocation (identity)")) != HW_OK) return s;
        s = hw_cuda(cudaMemsetAsync(eye, 0, bytes, st), "clear the identity");
        if (s == HW_OK) {
            const unsigned grid = unsigned((nn + 255) / 256);
            if (dt == HW_C128) k_unit_diagonal<double2><<<grid, 256, 0, st>>>(static_cast<double2 *>(eye), nn);
            else k_unit_diagonal<float2><<<grid, 256, 0, st>>>(static_cast<float2 *>(eye), nn);
            s = hw_cuda(cudaGetLastError(), "k_unit_diagonal launch");
        }
        if (s == HW_OK)
            s = hw_ctqw_evolve_sparse(g, gamma, marked, n_marked, time, dt, int32_t(nn), 1, eye, U_out, nullptr, opts,
                                      stream);
        cudaFreeAsync(eye, st);
        return s;
    }
    const int n = int(g->n);
    MarkedList mk;
    if ((s = make_marked(marked, n_marked, g->n, st, &mk)) != HW_OK) return s;
    struct Rel { MarkedList &m; cudaStream_t st; ~Rel() { free_marked(m, st); } } rel{mk, st};

    int m_deg, sq;
    if ((s = hw_ctqw_plan(g, gamma, marked, n_marked, time, &m_deg, &sq)) != HW_OK) return s;
    if (opts && opts->taylor_degree > 0) m_deg = opts->taylor_degree;
    if (opts && opts->taylor_squarings >= 0) sq = opts->taylor_squarings;
    if (m_deg > 40 || sq > 60) return hw_fail(HW_EINVAL, "Taylor degree %d / squarings %d out of range", m_deg, sq);
    const int gmode = opts ? opts->gemm_mode : 0;
    if (gmode < 0 || gmode > 4) return hw_fail(HW_EINVAL, "gemm_mode must be 0..4");
    if (opts && (opts->gemm_tiles < 0 || opts->gemm_tiles > 2)) return hw_fail(HW_EINVAL, "gemm_tiles must be 0..2");
    const double tau = time / std::ldexp(1.0, sq);
    const int64_t nn = int64_t(n) * n;
    const size_t bytes = sizeof(double) * nn;

    const int powers = opts ? opts->taylor_powers : 0;
    if (powers < 0 || powers > 2) return hw_fail(HW_EINVAL, "taylor_powers must be 0, 1 or 2");
    // default: the measured faster form on the 4096-vertex hypercube search
    // (complex128: sparse x dense 4.9 ms against 697 ms of FP64 GEMMs;
    // complex64: tensor-core GEMMs on CTA pairs 1.24 ms against 1.60 ms sparse x dense)
    const bool sparse = powers == 2 || (powers == 0 && (dt == HW_C128 || !tc_gemm_available()));
    const bool use_tc = !sparse && (dt == HW_C64) && tc_gemm_available();
    DevBuf Y(st), Q(st), Qn(st), Re(st), Im(st), Qf(st), Qfn(st);
    if ((s = Re.get(bytes, "scratch allocation (ReU)")) != HW_OK || (s = Im.get(bytes, "scratch allocation (ImU)")) != HW_OK)
        return s;
    if ((!use_tc && !(sparse && dt == HW_C64)) || sq > 0) {
        // the FP64 powers (dense or sparse) and the squarings need two n x n
        // double work matrices, the dense FP64 powers also Y
        if ((s = Q.get(bytes, "scratch allocation (Q)")) != HW_OK || (s = Qn.get(bytes, "scratch allocation (Q)")) != HW_OK)
            return s;
    }
    bool packed = false;
    if (sparse) {
        // T2 + T3 as sparse x dense products: Q_0 = I, Q_k = Y Q_{k-1} / k for
        // k = 1..m, each added to Re / Im U with the sign of (-i)^k
        const bool c128 = dt == HW_C128;
        if (!c128 && ((s = Qf.get(sizeof(float) * nn, "scratch allocation (Q)")) != HW_OK ||
                      (s = Qfn.get(sizeof(float) * nn, "scratch allocation (Q)")) != HW_OK))
            return s;
        void *Qa = c128 ? Q.p : Qf.p, *Qb = c128 ? Qn.p : Qfn.p;
        if (c128) k_taylor_identity<double><<<ew_grid(nn), 256, 0, st>>>(n, Re.as<double>(), Im.as<double>(), static_cast<double *>(Qa));
        else k_taylor_identity<float><<<ew_grid(nn), 256, 0, st>>>(n, Re.as<double>(), Im.as<double>(), static_cast<float *>(Qa));
        if ((s = hw_cuda(cudaGetLastError(), "Taylor init")) != HW_OK) return s;
        // two adjacent columns per thread when every row starts on a pair boundary
        // (two floats, not four, for complex64: four held 116 registers, two CTAs per SM)
        const int vec = n % 2 == 0 ? 2 : 1;
        const dim3 grid((n + kSpRows - 1) / kSpRows, (n + kSpCols * vec - 1) / (kSpCols * vec));
        for (int k = 1; k <= m_deg; ++k) {
            SparsePow a;
            a.row_ptr = g->d_row_ptr;
            a.head = g->d_head;
            a.w = g->weighted ? g->d_wre : nullptr;
            a.wf = g->weighted ? g->d_wre_f : nullptr;
            a.n = n;
            a.off = -gamma * tau / double(k);
            a.diag = -tau / double(k);
            a.offf = float(a.off);
            a.diagf = float(a.diag);
            a.mk = mk;
            a.Qp = Qa;
            a.Qn = Qb;
            a.acc = (k % 2 == 0) ? Re.as<double>() : Im.as<double>();
            a.neg = (k % 4 == 0 || k % 4 == 3) ? 0 : 1;
            if (c128) {
                if (vec == 2) {
                    if (g->weighted) k_taylor_sparse<double, true, 2><<<grid, kSpCols, 0, st>>>(a);
                    else k_taylor_sparse<double, false, 2><<<grid, kSpCols, 0, st>>>(a);
                } else {
                    if (g->weighted) k_taylor_sparse<double, true, 1><<<grid, kSpCols, 0, st>>>(a);
                    else k_taylor_sparse<double, false, 1><<<grid, kSpCols, 0, st>>>(a);
                }
            } else {
                if (vec == 2) {
                    if (g->weighted) k_taylor_sparse<float, true, 2><<<grid, kSpCols, 0, st>>>(a);
                    else k_taylor_sparse<float, false, 2><<<grid, kSpCols, 0, st>>>(a);
                } else {
                    if (g->weighted) k_taylor_sparse<float, true, 1><<<grid, kSpCols, 0, st>>>(a);
                    else k_taylor_sparse<float, false, 1><<<grid, kSpCols, 0, st>>>(a);
                }
            }
            if ((s = hw_cuda(cudaGetLastError(), "k_taylor_sparse launch")) != HW_OK) return s;
            std::swap(Qa, Qb);
        }
    } else if (use_tc) {
        // complex64 path: powers on the tensor cores from 16-bit slices; the
        // series is summed below the diagonal only.
        // T1 + the k = 0, 1 terms: Re U = I, Im U = -Y = gamma tau A + tau sum_m |m><m|
        k_init_lower<<<row_grid(n), 256, 0, st>>>(n, Re.as<double>(), Im.as<double>());
        k_scatter_y<<<(n + 255) / 256, 256, 0, st>>>(g->d_row_ptr, g->d_head, g->d_wre, n, gamma * tau, Im.as<double>());
        if (mk.n) k_mark_diag<<<(mk.n + 127) / 128, 128, 0, st>>>(mk, n, tau, Im.as<double>());
        if ((s = hw_cuda(cudaGetLastError(), "Taylor init")) != HW_OK) return s;
        TcPower *tp = nullptr;
        // host-known magnitudes of Y's entries (edge weights gamma tau |w|,
        // marked diagonal tau) and ||Y||_inf
        std::vector<double> yvals;
        if (g->num_arcs && gamma != 0.0) {
            if (g->weighted)
                for (double wa : g->h_wabs) yvals.push_back(std::fabs(gamma * tau) * wa);
            else
                yvals.push_back(std::fabs(gamma * tau));
        }
        if (mk.n && tau != 0.0) yvals.push_back(std::fabs(tau));
        double theta = 0.0;
        {
            std::vector<char> is_m(n, 0);
            for (int32_t i = 0; i < n_marked; ++i) is_m[marked[i]] = 1;
            for (int v = 0; v < n; ++v) {
                const double rw = g->weighted ? g->h_rowabs[v] : double(g->h_row_ptr[v + 1] - g->h_row_ptr[v]);
                theta = std::max(theta, (std::fabs(gamma) * rw + (is_m[v] ? 1.0 : 0.0)) * std::fabs(tau));
            }
        }
        const SymSparse ys{g->d_row_ptr, g->d_head, g->d_wre, n, -gamma * tau, mk, -tau};
        if ((s = tc_power_begin(ys, yvals.data(), int(yvals.size()), theta, gmode, opts ? opts->gemm_tiles : 0, st,
                                &tp)) != HW_OK)
            return s;
        for (int k = 2; k <= m_deg && s == HW_OK; ++k) {
            double *accU = (k % 2 == 0) ? Re.as<double>() : Im.as<double>();
            const double sign = (k % 4 == 0 || k % 4 == 3) ? 1.0 : -1.0;
            s = tc_power_step(tp, k, accU, sign);
        }
        if (s != HW_OK) {
            tc_power_end(tp, st, false);
            return s;
        }
        if (sq == 0) {
            // last term, mirror and complex64 packing in one pass
            if ((s = tc_power_finish_c64(tp, Re.as<double>(), Im.as<double>(), U_out, st)) != HW_OK) return s;
            packed = true;
        } else {
            if ((s = tc_power_end(tp, st, true)) != HW_OK) return s;
            k_mirror_lower<<<ew_grid(nn), 256, 0, st>>>(n, Re.as<double>());
            k_mirror_lower<<<ew_grid(nn), 256, 0, st>>>(n, Im.as<double>());
            if ((s = hw_cuda(cudaGetLastError(), "mirror")) != HW_OK) return s;
        }
    } else {
        // T1: Y = tau H
        if ((s = Y.get(bytes, "scratch allocation (Y)")) != HW_OK) return s;
        if ((s = hw_cuda(cudaMemsetAsync(Y.p, 0, bytes, st), "memset Y")) != HW_OK) return s;
        k_scatter_y<<<(n + 255) / 256, 256, 0, st>>>(g->d_row_ptr, g->d_head, g->d_wre, n, -gamma * tau, Y.as<double>());
        if (mk.n) k_mark_diag<<<(mk.n + 127) / 128, 128, 0, st>>>(mk, n, -tau, Y.as<double>());
        k_taylor_init<<<ew_grid(nn), 256, 0, st>>>(n, Y.as<double>(), Re.as<double>(), Im.as<double>());
        if ((s = hw_cuda(cudaGetLastError(), "Taylor init")) != HW_OK) return s;
        // T2 + T3: Q_k = Q_{k-1} Y / k, accumulated into Re/Im U with the sign of (-i)^k
        double *Qk = Y.as<double>();   // Q_1 = Y
        double *dst = Q.as<double>();
        for (int k = 2; k <= m_deg; ++k) {
            GemmArgs a{};
            a.A1 = Qk;
            a.B1 = Y.as<double>();
            a.n = n;
            a.epi = EPI_TAYLOR;
            a.out = dst;
            a.scale = 1.0 / double(k);
            a.acc = (k % 2 == 0) ? Re.as<double>() : Im.as<double>();
            a.sign = (k % 4 == 0 || k % 4 == 3) ? 1.0 : -1.0;
            a.sym_out = 1;   // Q_k = Y^k / k! with Y real symmetric
            if ((s = dgemm(a, st)) != HW_OK) return s;
            Qk = dst;
            dst = (dst == Q.as<double>()) ? Qn.as<double>() : Q.as<double>();
        }
    }

    // T4: U <- U^2, sq times (FP64)
    for (int r = 0; r < sq; ++r) {
        GemmArgs a{};
        a.A1 = Re.as<double>(); a.B1 = Re.as<double>();
        a.A2 = Im.as<double>(); a.B2 = Im.as<double>();
        a.sigma = -1.0;
        a.n = n; a.epi = EPI_STORE; a.out = Q.as<double>(); a.scale = 1.0;
        a.sym_out = 1;   // Re^2 - Im^2 is symmetric for symmetric Re, Im
        if ((s = dgemm(a, st)) != HW_OK) return s;                     // Re Re - Im Im
        GemmArgs b{};
        b.A1 = Re.as<double>(); b.B1 = Im.as<double>();
        b.n = n; b.epi = EPI_STORE; b.out = Qn.as<double>(); b.scale = 1.0;
        if ((s = dgemm(b, st)) != HW_OK) return s;                     // X = Re Im
        k_sym_add<<<ew_grid(nn), 256, 0, st>>>(n, Qn.as<double>(), Im.as<double>());
        std::swap(Re.p, Q.p);
        if ((s = hw_cuda(cudaGetLastError(), "squaring")) != HW_OK) return s;
    }

    if (packed) return HW_OK;
    if (dt == HW_C128) k_pack_u<double2><<<ew_grid(nn), 256, 0, st>>>(nn, Re.as<double>(), Im.as<double>(), static_cast<double2 *>(U_out));
    else k_pack_u<float2><<<ew_grid(nn), 256, 0, st>>>(nn, Re.as<double>(), Im.as<double>(), static_cast<float2 *>(U_out));
    return hw_cuda(cudaGetLastError(), "pack U");
}

// Zero-copy word that the TMA-fed application sets when a bounded stage wait
// runs out of time; hw_ctqw_evolve reports it (HW_ETIMEDOUT) at its next call.
static int *g_apply_err_h = nullptr, *g_apply_err_d = nullptr;
static std::mutex g_apply_err_mu;

static hw_status apply_error_word(int **dev)
{
    std::lock_guard<std::mutex> lk(g_apply_err_mu);
    if (!g_apply_err_h) {
        if (cudaHostAlloc(&g_apply_err_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&g_apply_err_d, g_apply_err_h, 0) != cudaSuccess) {
            cudaGetLastError();
            g_apply_err_h = nullptr;
            return hw_fail(HW_ENOMEM, "host allocation of the error word failed");
        }
        *g_apply_err_h = 0;
    }
    *dev = g_apply_err_d;
    return HW_OK;
}

extern "C" hw_status hw_ctqw_evolve(const void *U, int64_t n, hw_dtype dt, int32_t batch, int64_t steps,
                                    const void *psi_in, void *psi_out, const int32_t *marked,
                                    int32_t n_marked, double *record, const hw_opts *opts, void *stream)
{
    hw_clear_error();
    if (g_apply_err_h && *reinterpret_cast<volatile int *>(g_apply_err_h)) {
        *g_apply_err_h = 0;
        return hw_fail(HW_ETIMEDOUT, "a device-side wait of an earlier hw_ctqw_evolve call ran out of time");
    }
    if (!U || !psi_in || !psi_out) return hw_fail(HW_EINVAL, "NULL buffer");
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (n < 1 || n > (int64_t(1) << 30)) return hw_fail(HW_EINVAL, "bad n");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (steps < 0) return hw_fail(HW_EINVAL, "steps must be >= 0");
    if (n_marked < 0 || (n_marked > 0 && !marked)) return hw_fail(HW_EINVAL, "bad marked list");
    const size_t esz = cplx_bytes(dt);
    if ((uintptr_t)U % esz || (uintptr_t)psi_in % esz || (uintptr_t)psi_out % esz)
        return hw_fail(HW_EINVAL, "buffers misaligned");
    const int stride = opts ? opts->record_stride : 1;
    if (stride < 1) return hw_fail(HW_EINVAL, "record_stride must be >= 1");
    if (record && n_marked == 0) return hw_fail(HW_EINVAL, "record needs at least one marked vertex");
    const size_t bytes = size_t(n) * batch * esz;
    const char *ip = static_cast<const char *>(psi_in);
    const char *op = static_cast<const char *>(psi_out);
    if (ip != op && ip < op + bytes && op < ip + bytes)
        return hw_fail(HW_EINVAL, "psi_in and psi_out overlap without being equal");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hw_status s;
    if (steps == 0) {
        if (ip != op) return hw_cuda(cudaMemcpyAsync(psi_out, psi_in, bytes, cudaMemcpyDeviceToDevice, st), "copy");
        return HW_OK;
    }
    MarkedList mk;
    if ((s = make_marked(marked, n_marked, n, st, &mk)) != HW_OK) return s;
    struct Rel { MarkedList &m; cudaStream_t st; ~Rel() { free_marked(m, st); } } rel{mk, st};
    const int64_t slots = record ? steps / stride : 0;
    // the symmetric path halves the bytes read; complex128 is bound by FP64
    // arithmetic, which both paths share, so it keeps the dense path
    bool sym = opts && opts->u_symmetric && batch == 1 && dt == HW_C64;
    const int nb = int((n + kSymB - 1) / kSymB);
    DevBuf tmp(st), recbuf(st), splane(st), packed(st);
    if (sym) {
        // the blocks on and above the diagonal, packed once for all applications;
        // without room for that copy (n^2 / 2 elements) the dense path runs
        const int64_t blocks = int64_t(nb) * (nb + 1) / 2;
        const hw_status ps = packed.get(size_t(blocks) * kSymTileBytes, "scratch allocation (packed blocks of U)");
        if (ps == HW_ENOMEM) {
            hw_clear_error();
            packed.p = nullptr;
            sym = false;
        } else if (ps != HW_OK) {
            return ps;
        } else {
            k_sym_pack<<<unsigned(blocks), 256, 0, st>>>(static_cast<const float2 *>(U), int(n), nb,
                                                          packed.as<float2>());
            if ((s = hw_cuda(cudaGetLastError(), "k_sym_pack launch")) != HW_OK) return s;
        }
    }
    int *derr = nullptr;
    if (sym && (s = apply_error_word(&derr)) != HW_OK) return s;
    const size_t part_bytes = sym ? size_t(nb) * nb * kSymB * esz : 0;   // one array of block partials
    // complex128, one state, dense U: the three-product form with S = Re U + Im U
    const bool three = !sym && dt == HW_C128 && batch == 1;
    if ((s = tmp.get(bytes + 2 * part_bytes + 256, "scratch allocation (state scratch)")) != HW_OK) return s;
    if (three) {
        // S, then Re x + Im x of the two state buffers
        if ((s = splane.get((size_t(n) * size_t(n) + 2 * size_t(n)) * sizeof(double),
                            "scratch allocation (Re U + Im U)")) != HW_OK)
            return s;
        const int64_t count = n * n;
        const int g = int(std::min<int64_t>(148 * 8, (count + 255) / 256));
        k_sum_plane<<<g, 256, 0, st>>>(static_cast<const double2 *>(U), splane.as<double>(), count);
        if ((s = hw_cuda(cudaGetLastError(), "k_sum_plane launch")) != HW_OK) return s;
    }
    double *xsum = three ? splane.as<double>() + n * n : nullptr, *ysum = three ? xsum + n : nullptr;
    void *prow = static_cast<char *>(tmp.p) + ((bytes + 255) & ~size_t(255));
    void *pcol = static_cast<char *>(prow) + part_bytes;
    double *rec_part = nullptr;
    if (slots) {
        if (n_marked == 1) {
            rec_part = record;
        } else {
            if ((s = recbuf.get(sizeof(double) * slots * n_marked * batch, "scratch allocation (record)")) != HW_OK)
                return s;
            rec_part = recbuf.as<double>();
        }
    }
    // same ping-pong schedule as the coined walk: the last step lands in psi_out
    void *P = psi_out, *T = tmp.p;
    const void *src = psi_in;
    if (ip == op && steps % 2 == 1) {
        if ((s = hw_cuda(cudaMemcpyAsync(T, psi_in, bytes, cudaMemcpyDeviceToDevice, st), "copy")) != HW_OK)
            return s;
        src = T;
    }
    if (three) {
        k_sum_plane<<<int((n + 255) / 256), 256, 0, st>>>(static_cast<const double2 *>(src), xsum, n);
        if ((s = hw_cuda(cudaGetLastError(), "k_sum_plane launch")) != HW_OK) return s;
    }
    for (int64_t k = 1; k <= steps; ++k) {
        void *dst = ((steps - k) % 2 == 0) ? P : T;
        const int64_t slot = (slots && k % stride == 0) ? k / stride - 1 : -1;
        if (sym)
            s = launch_apply_sym(packed.as<float2>(), src, dst, int(n), prow, pcol, mk, rec_part, slot, st, derr,
                                 k == 1);
        else if (three) {
            s = launch_apply_3m(U, splane.as<double>(), src, xsum, dst, ysum, int(n), mk, rec_part, slot, st);
            std::swap(xsum, ysum);
        }
        else
            s = (dt == HW_C128) ? launch_apply<double>(U, src, dst, int(n), batch, mk, rec_part, slot, st)
                                : launch_apply<float>(U, src, dst, int(n), batch, mk, rec_part, slot, st);
        if (s != HW_OK) return s;
        src = dst;
    }
    if (slots && n_marked > 1)
        if ((s = launch_record_finalize(rec_part, n_marked, slots, batch, record, st)) != HW_OK) return s;
    return HW_OK;
}

// Sampled CTQW (the paper's simulate(range=...)): U^t psi for t = start,
// start + stride, ... < end applications, each segment one hw_ctqw_evolve.
extern "C" hw_status hw_ctqw_sample(const void *U, int64_t n, hw_dtype dt, int32_t batch, int64_t start,
                                    int64_t end, int64_t stride, const void *psi_in, void *states_out,
                                    double *prob_out, const hw_opts *opts, void *stream)
{
    hw_clear_error();
    if (start < 0 || end < start || stride < 1) return hw_fail(HW_EINVAL, "need 0 <= start <= end and stride >= 1");
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (n < 1 || batch < 1) return hw_fail(HW_EINVAL, "bad n or batch");
    if (!U || !psi_in) return hw_fail(HW_EINVAL, "NULL buffer");
    const int64_t R = (end - start + stride - 1) / stride;
    if (R == 0) return HW_OK;
    const size_t bytes = size_t(n) * batch * cplx_bytes(dt);
    if (states_out) {
        const char *ip = static_cast<const char *>(psi_in);
        const char *op = static_cast<const char *>(states_out);
        if (ip < op + bytes * R && op < ip + bytes) return hw_fail(HW_EINVAL, "psi_in overlaps states_out");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf buf(st);
    hw_status s;
    if (!states_out && (s = buf.get(2 * bytes, "scratch allocation (samples)")) != HW_OK) return s;
    auto slot = [&](int64_t r) -> void * {
        return states_out ? static_cast<void *>(static_cast<char *>(states_out) + bytes * size_t(r))
                          : static_cast<void *>(buf.as<char>() + bytes * size_t(r & 1));
    };
    const void *src = psi_in;
    int64_t t = 0;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t tr = start + r * stride;
        if ((s = hw_ctqw_evolve(U, n, dt, batch, tr - t, src, slot(r), nullptr, 0, nullptr, opts, stream)) != HW_OK)
            return s;
        if (prob_out &&
            (s = launch_probability(nullptr, n, dt, batch, slot(r), prob_out + size_t(n) * batch * r, nullptr, st)) !=
                HW_OK)
            return s;
        src = slot(r);
        t = tr;
    }
    return HW_OK;
}
