// Tensor-core GEMM for the complex64 Taylor series of U = e^{-iHt}.
//
// C[m][n] = sum_k A[m][k] B[n][k] with fp32 operands split into 16-bit slices
// (x = x0 + x1 [+ x2], each slice the rounding of what the previous ones
// leave), multiplied on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, fp32 accumulator in tensor memory) and summed over the slice
// products that matter:
//   fp16 x 2 slices, 3 products (default): about 2^-22 of the matrix maximum;
//   bf16 x 3 slices, 6 products: about 2^-24; bf16 x 2: 2^-16; bf16 x 1: 2^-8.
// fp16 slices are taken of the operand times a power of two that puts its
// largest entry in [1/2, 1] (exact), so the 5-bit exponent never limits.  When
// every entry of B is exact in one slice (the Taylor step's Y = tau H of an
// unweighted graph, scaled by 1 / (gamma tau), has entries 0, 1 and 1/gamma),
// B keeps one slice and the products with its lower slices are dropped.
//
// Two forms.  The Taylor powers run on CTA pairs by default (k_tc_gemm_pair,
// below: 256 x 256 tiles, one pair MMA per K step, 64-element K blocks); the
// form described next, one CTA per tile, serves hw_gemm_tc and
// hw_opts.gemm_tiles = 1.
//
// Work is cut into 128 x 256 CTA tiles; persistent CTAs, one per SM, walk a
// list of tiles.  Each CTA loads its own A rows and all of its B rows with
// TMA into its own shared memory: the operands of a Taylor power (the previous
// power's slices and Y's) stay in L2, which serves the repeated B reads.  Per
// CTA, 14 warps (448 threads): warp 4 lane 0 streams K blocks (32 elements =
// one 64-byte swizzle row) of every slice into a shared-memory ring (up to 8
// stages, 216 KiB); warp 5 lane 0 issues the MMAs (M = 128, N = 256) into one
// of two 256-column TMEM accumulators and releases each stage with a
// tcgen05.commit on the stage's "empty" barrier; warps 0-3 and 6-9 drain the
// other accumulator (tcgen05.ld, warp w owns TMEM lanes of quadrant w % 4 =
// tile rows, warps 0-3 and 6-9 one half of the columns each) and run the
// epilogue of the previous tile:
//   EPI_STORE:  C = scale * acc (fp32)
//   EPI_TAYLOR: Q = scale * acc, written back as slices of qscale * Q (the
//               next power's A operand).
// The double-precision Taylor sum of the previous power (U += coef Q, lower
// triangle; the caller mirrors it) runs inside the next power's GEMM: warps
// 0-3 and 6-13 do it while the tensor cores work on the first tile (the
// previous power's slices are this GEMM's A operand, so they are mostly L2
// hits); the last power's term is added by k_finish_c64 while it packs the
// complex64 U, or by k_taylor_acc (tc_power_end).
// For a symmetric product (every Taylor power of the symmetric Y is
// symmetric) only cluster tiles that reach the upper triangle run, 128 x 128
// blocks below the diagonal are not written, and each off-diagonal block is
// also written to its mirror position with coalesced transposed stores.
// Every wait on an mbarrier is bounded; a timeout sets an error flag that the
// host reads, and the CTA still frees its tensor memory.  Before a CTA exits,
// its producer waits until every stage it filled has been released, so no
// copy or MMA is in flight when it leaves.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "fpconv.cuh"
#include "internal.h"

namespace {

constexpr int TM = 128, TN = 256, TK = 32;                // CTA tile; K block = one 64-byte swizzle row
constexpr int kATile = TM * TK * 2;                       // 8 KB per A slice
constexpr int kBTile = TN * TK * 2;                       // 16 KB per B slice
constexpr int kRingBytes = 216 * 1024;                    // shared-memory ring
constexpr int kMaxStages = 8;
constexpr int kSmemSlack = 2048;                          // alignment of the ring base + margin
constexpr int kAccWarps = 8;                              // warps 6..13: accumulation, then epilogues
constexpr int kThreads = 192 + 32 * kAccWarps;
constexpr int kTmemCols = 2 * TN;                         // two accumulators
constexpr int kEpiWarps = 12;                             // warps 0-3 and 6-13
constexpr uint64_t kWaitLimitNs = 2000000000ull;          // bounded mbarrier waits (2 s)

enum { FMT_BF16 = 0, FMT_F16 = 1 };
enum { EPI_STORE = 0, EPI_TAYLOR = 1 };

struct TcArgs {
    const int2 *tiles;       // tiles (P, Q): rows 128 P.. (CTA pairs: 256 P..), columns 256 Q..
    int m, n, k;
    int epi;
    int sym;                 // skip blocks below the diagonal, mirror the others
    float scale;             // acc multiplier (host-known part)
    const float *dscale;     // acc multiplier read on the device (or nullptr)
    float *C;                // EPI_STORE: [m][ldc]
    int ldc;
    void *Q[3];              // EPI_TAYLOR: output slices [m][ldq] of qscale * Q (na of them)
    int ldq;
    float qscale;
    const void *accQ[3];     // EPI_TAYLOR: slices of the previous power, added to accU by the
    double acc_coef;         // epilogue warps while the first tile multiplies (accU == nullptr: none)
    double *accU;
    int *err;                // set to 1 on a wait timeout
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true when the phase with this parity has completed; false after kWaitLimitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
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
            const uint64_t t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitLimitNs) return false;
        }
    }
}

// 2D tile load into this CTA's shared memory, completing on its mbarrier
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row
// groups 512 bytes apart (the layout TMA writes for a 32-wide 16-bit box).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr)
{
    uint64_t d = 0;
    d |= uint64_t((addr & 0x3FFFFu) >> 4);      // start address
    d |= uint64_t(1) << 16;                      // leading offset (unused when swizzled)
    d |= uint64_t(512 >> 4) << 32;               // stride offset between 8-row groups
    d |= uint64_t(1) << 46;                      // descriptor version
    d |= uint64_t(4) << 61;                      // 64-byte swizzle
    return d;
}

// The same for 128-byte rows (64 16-bit elements, 128-byte swizzle): 8-row
// groups 1024 bytes apart; the pair kernel's K blocks
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= uint64_t((addr & 0x3FFFFu) >> 4);      // start address
    d |= uint64_t(1) << 16;                      // leading offset (unused when swizzled)
    d |= uint64_t(1024 >> 4) << 32;              // stride offset between 8-row groups
    d |= uint64_t(1) << 46;                      // descriptor version
    d |= uint64_t(2) << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor: 16-bit A and B (bf16 = 1, fp16 = 0), fp32 accumulator,
// both K-major, M = TM, N = TN.
template <int FMT>
__device__ __forceinline__ constexpr uint32_t idesc()
{
    return (1u << 4) | (uint32_t(FMT == FMT_BF16 ? 1 : 0) << 7) | (uint32_t(FMT == FMT_BF16 ? 1 : 0) << 10) |
           (uint32_t(TN >> 3) << 17) | (uint32_t(TM >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void mma16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc<FMT>()), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// ---- CTA-pair forms (cta_group::2): the two CTAs of a cluster of 2 share
// one 256 x 256 tile; every tcgen05 instruction of the pair kernel takes the
// pair form.  Addresses of barriers are in the shared::cluster window: the
// CTA's own (a shared::cta address) or the peer's (mapa).

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// every thread of both CTAs: what each did before is visible to both after
__device__ __forceinline__ void pair_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// 2D tile load into this CTA's shared memory, its bytes counted on an
// mbarrier of either CTA of the pair (the leader's)
__device__ __forceinline__ void tma_load_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// M = 256 (128 rows from each CTA's shared memory, at the same offsets), N = TN
// (TN / 2 rows of B from each CTA); each CTA's TMEM receives its 128 rows
template <int FMT>
__device__ __forceinline__ constexpr uint32_t idesc_pair()
{
    return (1u << 4) | (uint32_t(FMT == FMT_BF16 ? 1 : 0) << 7) | (uint32_t(FMT == FMT_BF16 ? 1 : 0) << 10) |
           (uint32_t(TN >> 3) << 17) | (uint32_t((2 * TM) >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void mma16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc_pair<FMT>()), "r"(acc)
        : "memory");
}

// arrive on one mbarrier (either CTA) when the pair's earlier MMAs are done
__device__ __forceinline__ void mma_commit_pair(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16-bit slice storage
template <int FMT> struct Sl;
template <> struct Sl<FMT_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __bfloat162float(x); }
};
template <> struct Sl<FMT_F16> {
    using T = __half;
    static __device__ __forceinline__ T from(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __half2float(x); }
};

// x -> ns slices, x = s0 + s1 [+ s2] up to the last slice's rounding
template <int FMT>
__device__ __forceinline__ void split(float x, int ns, typename Sl<FMT>::T *s)
{
    using S = Sl<FMT>;
    s[0] = S::from(x);
    if (ns > 1) {
        const float r1 = x - S::to(s[0]);
        s[1] = S::from(r1);
        if (ns > 2) s[2] = S::from(r1 - S::to(s[1]));
    }
}

// T3 of the series: accU[i][j] += coef * Q[i][j] for j <= i (the lower
// triangle) over rows i = row0, row0 + rstride, ..., with Q given by its NA
// slices (of Q / coef up to sign); the slices are summed in fp32 (what the
// next power multiplies) and added in double.  The rows' elements are taken
// as one flat sequence, element e by thread e % nt, in batches of U elements
// per thread whose loads are all issued before their stores, so that each
// thread keeps U reads in flight whatever the rows' lengths.
template <int FMT, int NA>
__device__ __forceinline__ void acc_rows(int n, const void *q0, const void *q1, const void *q2, int ldq,
                                         double coef, double *__restrict__ accU, int row0, int rstride, int tid,
                                         int nt)
{
    using ST = typename Sl<FMT>::T;
    constexpr int U = 8;
    if (row0 >= n) return;
    // current row r (flat offset base of its first element) of this thread's walk
    int r = row0;
    int64_t base = 0;
    int64_t e = tid;
    while (true) {
        int64_t at_q[U], at_u[U];
        bool ok[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
            const int64_t et = e + int64_t(t) * nt;
            while (r < n && et >= base + r + 1) {   // past the end of row r
                base += r + 1;
                r += rstride;
            }
            ok[t] = r < n;
            const int64_t col = et - base;
            at_q[t] = int64_t(r) * ldq + col;
            at_u[t] = int64_t(r) * n + col;
        }
        float q[U];
        double x[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
            if (ok[t]) {
                q[t] = Sl<FMT>::to(static_cast<const ST *>(q0)[at_q[t]]);
                if (NA > 1) q[t] += Sl<FMT>::to(static_cast<const ST *>(q1)[at_q[t]]);
                if (NA > 2) q[t] += Sl<FMT>::to(static_cast<const ST *>(q2)[at_q[t]]);
                x[t] = accU[at_u[t]];
            }
        }
#pragma unroll
        for (int t = 0; t < U; ++t)
            if (ok[t]) accU[at_u[t]] = fma(coef, fpconv::f32_to_f64(q[t]), x[t]);
        if (!ok[U - 1]) break;
        e += int64_t(U) * nt;
    }
}

template <int FMT, int NA>
__global__ void __launch_bounds__(256) k_taylor_acc(int n, const void *q0, const void *q1, const void *q2,
                                                    int ldq, double coef, double *__restrict__ accU)
{
    acc_rows<FMT, NA>(n, q0, q1, q2, ldq, coef, accU, blockIdx.x, gridDim.x, threadIdx.x, blockDim.x);
}

// Epilogue of columns [cb, ce) of one 128 x 256 CTA tile whose accumulator is
// at TMEM column tacc, by a warp of lane quadrant quad (tile rows 32 quad..);
// Q is written as NA slices.
template <int FMT, int NA>
__device__ __forceinline__ void epilogue_tile(const TcArgs &a, int row0, int col0, uint32_t tacc, int quad, int lane,
                                              int cb, int ce)
{
    using S = Sl<FMT>;
    constexpr int na = NA;
    const float mult = a.scale * (a.dscale ? *a.dscale : 1.0f);
    const int row = row0 + quad * 32 + lane;    // tile row held by this thread
    const int rblk = row0 / 128;
    const bool c_vec = a.C && (a.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(a.C) % 16 == 0);
    for (int c0 = cb; c0 < ce; c0 += 16) {
        const int col0c = col0 + c0;
        const int cblk = col0c / 128;
        if (a.sym && cblk < rblk) continue;     // below the diagonal: written as the mirror of (cblk, rblk)
        uint32_t r[16];
        tmem_ld16(tacc + (uint32_t(quad * 32) << 16) + uint32_t(c0), r);
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]) * mult;
        if (a.epi == EPI_STORE) {
            if (row < a.m) {
                float *dst = a.C + int64_t(row) * a.ldc + col0c;
                if (c_vec && col0c + 16 <= a.n) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (col0c + q < a.n) dst[q] = v[q];
                }
            }
            continue;
        }
        // Taylor epilogue: slices of qscale * Q, written to both blocks of a
        // mirrored pair (the next power's A operand and the input of the
        // double-precision accumulation, k_taylor_acc)
        const bool mirror = a.sym && cblk != rblk;
        const bool in_row = row < a.m;
        const bool do_mirror = mirror && row < a.n;
        typename S::T sl[3][16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            typename S::T t3[3];
            split<FMT>(v[q] * a.qscale, na, t3);
            sl[0][q] = t3[0];
            sl[1][q] = t3[1];
            sl[2][q] = t3[2];
        }
        if (in_row) {
            const bool full = col0c + 16 <= a.n;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= na) break;
                typename S::T *qd = static_cast<typename S::T *>(a.Q[i]) + int64_t(row) * a.ldq + col0c;
                if (full) {
                    // 16 slice values = 32 contiguous bytes (ldq is a multiple of 64)
                    reinterpret_cast<uint4 *>(qd)[0] = *reinterpret_cast<const uint4 *>(&sl[i][0]);
                    reinterpret_cast<uint4 *>(qd)[1] = *reinterpret_cast<const uint4 *>(&sl[i][8]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (col0c + q < a.n) qd[q] = sl[i][q];
                }
            }
        }
        if (do_mirror) {
            // element (row, col) -> (col, row): consecutive lanes write consecutive columns
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int mrow = col0c + q;
                if (mrow >= a.m) continue;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    if (i < na) static_cast<typename S::T *>(a.Q[i])[int64_t(mrow) * a.ldq + row] = sl[i][q];
            }
        }
    }
}

// Ring geometry of a slice configuration: NA slices of A, NB of B per stage.
template <int NA, int NB>
struct Ring {
    static constexpr int kStageBytes = NA * kATile + NB * kBTile;
    static constexpr int kStages = (kRingBytes / kStageBytes < kMaxStages) ? kRingBytes / kStageBytes : kMaxStages;
};

// One K block of MMAs (TK / 16 steps x the slice products (i, j), i + j < NA,
// j < NB, smaller products first) from the stage whose descriptors start at
// dA (A slice 0) and dB (B slice 0).  Everything but the stage base is a
// compile-time constant, so the issuing thread spends a few instructions per
// MMA; acc0 = 0 starts the accumulator with the first product.
template <int FMT, int NA, int NB>
__device__ __forceinline__ void mma_block(uint32_t tacc, uint64_t dA, uint64_t dB, uint32_t acc0)
{
#pragma unroll
    for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
        for (int d = NA - 1; d >= 0; --d) {
#pragma unroll
            for (int i = d; i >= 0; --i) {
                const int j = d - i;
                if (j < NB) {
                    const uint64_t ad = dA + uint64_t((i * kATile) >> 4) + uint64_t(2 * kk);
                    const uint64_t bd = dB + uint64_t((j * kBTile) >> 4) + uint64_t(2 * kk);
                    const bool first = (kk == 0 && d == NA - 1 && i == d);
                    mma16<FMT>(tacc, ad, bd, first ? acc0 : 1u);
                }
            }
        }
    }
}

template <int FMT, int NA, int NB>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
          const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
          const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TcArgs a, int ntiles)
{
    constexpr int kStageBytes = Ring<NA, NB>::kStageBytes;
    constexpr int S = Ring<NA, NB>::kStages;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_tfull[2], bar_tempty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int timed_out;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cid = int(blockIdx.x), ncl = int(gridDim.x);
    const int nkb = (a.k + TK - 1) / TK;
    volatile int *tmo = &timed_out;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_tfull[b]), 1);
            mbar_init(smem_u32(&bar_tempty[b]), kEpiWarps);  // one arrival per epilogue warp
        }
        timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");   // visible to the async proxy
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 4) {
        if (lane == 0) {
            // producer: one TMA box per slice of the A tile (128 rows) and of
            // the B tile (256 rows) per K block
            const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
            const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};
            uint32_t g = 0, phase = 0;
            int s = 0;
            for (int t = cid; t < ntiles && !*tmo; t += ncl) {
                const int2 ct = a.tiles[t];
                const int rowA = ct.x * TM;
                const int rowB = ct.y * TN;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (g >= uint32_t(S) && !mbar_wait(smem_u32(&bar_empty[s]), phase ^ 1u)) {
                        *tmo = 1;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_full[s]);
                    mbar_expect_tx(full, uint32_t(kStageBytes));   // all bytes of the stage's boxes
                    const uint32_t st = base + uint32_t(s * kStageBytes);
#pragma unroll
                    for (int i = 0; i < NA; ++i) tma_load(st + uint32_t(i * kATile), mA[i], full, kb * TK, rowA);
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        tma_load(st + uint32_t(NA * kATile + j * kBTile), mB[j], full, kb * TK, rowB);
                    ++g;
                    if (++s == S) { s = 0; phase ^= 1u; }
                }
            }
            // drain: the last fill of every stage released by the MMAs
            for (uint32_t q = 0; q < uint32_t(S) && q < g; ++q) {
                const uint32_t last_use = (g - 1 - q) / uint32_t(S);
                if (!mbar_wait(smem_u32(&bar_empty[q]), last_use & 1u)) *tmo = 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: accumulator b = (local tile) & 1
            const uint64_t d0 = smem_desc_sw64(base);
            uint32_t phase = 0, li = 0;
            int s = 0;
            for (int t = cid; t < ntiles && !*tmo; t += ncl, ++li) {
                const int b = int(li & 1u);
                const uint32_t ub = li >> 1;
                if (ub > 0 && !mbar_wait(smem_u32(&bar_tempty[b]), (ub & 1u) ^ 1u)) {
                    *tmo = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tacc = tmem + uint32_t(b * TN);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(smem_u32(&bar_full[s]), phase)) {
                        *tmo = 1;
                        break;
                    }
                    const uint64_t dA = d0 + uint64_t((s * kStageBytes) >> 4);
                    mma_block<FMT, NA, NB>(tacc, dA, dA + uint64_t((NA * kATile) >> 4), kb > 0 ? 1u : 0u);
                    mma_commit(smem_u32(&bar_empty[s]));
                    if (++s == S) { s = 0; phase ^= 1u; }
                }
                mma_commit(smem_u32(&bar_tfull[b]));
            }
        }
    } else {
        // warps 0-3 and 6-13: first the previous power's accumulation (its
        // slices are this GEMM's A operand, so mostly L2 hits), rows spread
        // over all CTAs, while the tensor cores work on the first tile; then
        // the epilogues, warp w on TMEM lane quadrant w % 4 and a third of the
        // tile's columns (warps 0-3 the first, 6-9 the second, 10-13 the last)
        if (a.accU)
            acc_rows<FMT, NA>(a.n, a.accQ[0], a.accQ[1], a.accQ[2], a.ldq, a.acc_coef, a.accU, int(blockIdx.x),
                              int(gridDim.x), warp < 4 ? int(threadIdx.x) : int(threadIdx.x) - 64,
                              128 + 32 * kAccWarps);
        // the tile's 256 columns in three parts of 16-column chunks (6, 5, 5)
        const int quad = warp & 3, third = (warp < 4) ? 0 : (warp < 10 ? 1 : 2);
        const int cb = third == 0 ? 0 : (third == 1 ? 96 : 176), ce = third == 0 ? 96 : (third == 1 ? 176 : 256);
        uint32_t li = 0;
        for (int t = cid; t < ntiles; t += ncl, ++li) {
            const int b = int(li & 1u);
            if (!mbar_wait(smem_u32(&bar_tfull[b]), (li >> 1) & 1u)) {
                *tmo = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int2 ct = a.tiles[t];
            epilogue_tile<FMT, NA>(a, ct.x * TM, ct.y * TN, tmem + uint32_t(b * TN), quad, lane, cb, ce);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_tempty[b])) : "memory");
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (threadIdx.x == 0 && timed_out) atomicExch(a.err, 1);
}

// The same GEMM with 256 x 256 tiles, each computed by the two CTAs of a
// cluster as one pair MMA (M = 256): CTA r of the pair loads rows 128 r.. of
// the tile's A rows and rows 128 r.. of its B rows, so per unit of tensor work
// each CTA loads a quarter fewer bytes (A with two slices, B with one), and
// K blocks are 64 elements (whole 128-byte rows, 128-byte swizzle).  The even CTA
// (the leader) issues the MMAs; both CTAs' loads count on the leader's "full"
// barrier; the leader's commits arrive on the "empty" and "accumulator full"
// barriers of both CTAs (one commit each); both CTAs' epilogue warps arrive on
// the leader's "accumulator empty" barrier.  Tiles (P, Q) cover rows 256 P..,
// columns 256 Q..; everything else (ring, epilogues, accumulation, bounded
// waits, drain) is as in k_tc_gemm.
template <int FMT, int NA, int NB>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_gemm_pair(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
               const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
               const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TcArgs a,
               int ntiles)
{
    constexpr int TKP = 64;                                    // K block: one 128-byte swizzle row
    constexpr int kATileP = TM * TKP * 2;                      // 16 KB per A slice
    constexpr int kBHalf = (TN / 2) * TKP * 2;                 // TN / 2 rows of B per CTA: 16 KB
    constexpr int kStageBytes = NA * kATileP + NB * kBHalf;
    constexpr int S = (kRingBytes / kStageBytes < kMaxStages) ? kRingBytes / kStageBytes : kMaxStages;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_tfull[2], bar_tempty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int timed_out;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int pid = int(blockIdx.x) >> 1, npair = int(gridDim.x) >> 1;
    const int nkb = (a.k + TKP - 1) / TKP;
    volatile int *tmo = &timed_out;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_tfull[b]), 1);
            mbar_init(smem_u32(&bar_tempty[b]), 2 * kEpiWarps);   // epilogue warps of both CTAs
        }
        timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // both CTAs' barriers are initialised and their TMEM allocated before
    // either CTA signals the other
    pair_barrier();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 4) {
        if (lane == 0) {
            // producer (both CTAs): this CTA's A rows and half of the B rows
            const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
            const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};
            uint32_t g = 0, phase = 0;
            int s = 0;
            for (int t = pid; t < ntiles && !*tmo; t += npair) {
                const int2 ct = a.tiles[t];
                const int rowA = ct.x * 2 * TM + int(rank) * TM;
                const int rowB = ct.y * TN + int(rank) * (TN / 2);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (g >= uint32_t(S) && !mbar_wait(smem_u32(&bar_empty[s]), phase ^ 1u)) {
                        *tmo = 1;
                        break;
                    }
                    const uint32_t full_own = smem_u32(&bar_full[s]);
                    if (leader) mbar_expect_tx(full_own, uint32_t(2 * kStageBytes));   // both CTAs' boxes
                    const uint32_t full = leader ? full_own : peer_addr(full_own, 0);
                    const uint32_t st = base + uint32_t(s * kStageBytes);
#pragma unroll
                    for (int i = 0; i < NA; ++i) tma_load_pair(st + uint32_t(i * kATileP), mA[i], full, kb * TKP, rowA);
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        tma_load_pair(st + uint32_t(NA * kATileP + j * kBHalf), mB[j], full, kb * TKP, rowB);
                    ++g;
                    if (++s == S) { s = 0; phase ^= 1u; }
                }
            }
            // drain: the last fill of every stage released by the pair's MMAs
            for (uint32_t q = 0; q < uint32_t(S) && q < g; ++q) {
                const uint32_t last_use = (g - 1 - q) / uint32_t(S);
                if (!mbar_wait(smem_u32(&bar_empty[q]), last_use & 1u)) *tmo = 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0 && leader) {
            // MMA issuer (leader): accumulator b = (local tile) & 1, in both CTAs' TMEM
            const uint64_t d0 = smem_desc_sw128(base);
            uint32_t phase = 0, li = 0;
            int s = 0;
            for (int t = pid; t < ntiles && !*tmo; t += npair, ++li) {
                const int b = int(li & 1u);
                const uint32_t ub = li >> 1;
                if (ub > 0 && !mbar_wait(smem_u32(&bar_tempty[b]), (ub & 1u) ^ 1u)) {
                    *tmo = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tacc = tmem + uint32_t(b * TN);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(smem_u32(&bar_full[s]), phase)) {
                        *tmo = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t dA = d0 + uint64_t((s * kStageBytes) >> 4);
                    const uint64_t dB = dA + uint64_t((NA * kATileP) >> 4);
                    // K steps of 16 elements: 32 bytes further along the swizzled row
#pragma unroll
                    for (int kk = 0; kk < TKP / 16; ++kk) {
#pragma unroll
                        for (int d = NA - 1; d >= 0; --d) {
#pragma unroll
                            for (int i = d; i >= 0; --i) {
                                const int j = d - i;
                                if (j < NB) {
                                    const uint64_t ad = dA + uint64_t((i * kATileP) >> 4) + uint64_t(2 * kk);
                                    const uint64_t bd = dB + uint64_t((j * kBHalf) >> 4) + uint64_t(2 * kk);
                                    const bool first = (kk == 0 && d == NA - 1 && i == d);
                                    mma16_pair<FMT>(tacc, ad, bd, (first && kb == 0) ? 0u : 1u);
                                }
                            }
                        }
                    }
                    const uint32_t e = smem_u32(&bar_empty[s]);
                    mma_commit_pair(e);
                    mma_commit_pair(peer_addr(e, 1));
                    if (++s == S) { s = 0; phase ^= 1u; }
                }
                const uint32_t tf = smem_u32(&bar_tfull[b]);
                mma_commit_pair(tf);
                mma_commit_pair(peer_addr(tf, 1));
            }
        }
    } else {
        if (a.accU)
            acc_rows<FMT, NA>(a.n, a.accQ[0], a.accQ[1], a.accQ[2], a.ldq, a.acc_coef, a.accU, int(blockIdx.x),
                              int(gridDim.x), warp < 4 ? int(threadIdx.x) : int(threadIdx.x) - 64,
                              128 + 32 * kAccWarps);
        const int quad = warp & 3, third = (warp < 4) ? 0 : (warp < 10 ? 1 : 2);
        const int cb = third == 0 ? 0 : (third == 1 ? 96 : 176), ce = third == 0 ? 96 : (third == 1 ? 176 : 256);
        uint32_t li = 0;
        for (int t = pid; t < ntiles; t += npair, ++li) {
            const int b = int(li & 1u);
            if (!mbar_wait(smem_u32(&bar_tfull[b]), (li >> 1) & 1u)) {
                *tmo = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int2 ct = a.tiles[t];
            epilogue_tile<FMT, NA>(a, ct.x * 2 * TM + int(rank) * TM, ct.y * TN, tmem + uint32_t(b * TN), quad, lane,
                                   cb, ce);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                const uint32_t te = smem_u32(&bar_tempty[b]);
                if (leader)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(te) : "memory");
                else
                    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(peer_addr(te, 0))
                                 : "memory");
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // no CTA frees its TMEM or leaves while the pair's MMAs or the peer's
    // arrivals may still reach it
    pair_barrier();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (threadIdx.x == 0 && timed_out) atomicExch(a.err, 1);
}

// largest |x| of a matrix as float bits (non-negative floats order like their bits);
// blocks stride over rows, threads over columns
template <typename T>
__global__ void k_absmax(const T *__restrict__ x, int rows, int cols, int ldx, unsigned *out)
{
    float mx = 0.f;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const T *xr = x + int64_t(r) * ldx;
        for (int c = threadIdx.x; c < cols; c += blockDim.x) mx = fmaxf(mx, fabsf(float(xr[c])));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

// power-of-two scale that maps the maximum into [1/2, 1]; also stores 1/(sA sB)
__global__ void k_scales(const unsigned *mx, float *scale)
{
    float s[2];
    for (int i = 0; i < 2; ++i) {
        const float m = __uint_as_float(mx[i]);
        s[i] = (m > 0.f) ? exp2f(-ceilf(log2f(m))) : 1.f;
        scale[i] = s[i];
    }
    scale[2] = 1.f / (s[0] * s[1]);
}

// matrix -> ns slices of (scale * x) with row stride ld (columns >= cols
// untouched); blocks stride over rows, threads over columns
template <int FMT, typename T>
__global__ void k_split(const T *__restrict__ x, int rows, int cols, int ldx, int ns, int ld, const float *dscale,
                        double hscale, void *s0, void *s1, void *s2)
{
    using ST = typename Sl<FMT>::T;
    const double sc = dscale ? double(*dscale) : hscale;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const T *xr = x + int64_t(r) * ldx;
        ST *o0 = static_cast<ST *>(s0) + int64_t(r) * ld;
        ST *o1 = static_cast<ST *>(s1) + int64_t(r) * ld;
        ST *o2 = static_cast<ST *>(s2) + int64_t(r) * ld;
        for (int c = threadIdx.x; c < cols; c += blockDim.x) {
            const T x0 = xr[c];
            if (x0 == T(0)) {   // sparse Y: most entries are zero and so are their slices
                o0[c] = Sl<FMT>::from(0.0f);
                if (ns > 1) o1[c] = Sl<FMT>::from(0.0f);
                if (ns > 2) o2[c] = Sl<FMT>::from(0.0f);
                continue;
            }
            // the scale is applied and the first subtraction runs in T (double
            // for Y, so that fp64 inputs keep their low bits; float inputs are
            // scaled by powers of two, which is exact in float)
            const T xs = x0 * T(sc);
            const ST a0 = Sl<FMT>::from(float(xs));
            o0[c] = a0;
            if (ns > 1) {
                const T r1 = xs - T(Sl<FMT>::to(a0));
                const ST a1 = Sl<FMT>::from(float(r1));
                o1[c] = a1;
                if (ns > 2) o2[c] = Sl<FMT>::from(float(r1 - T(Sl<FMT>::to(a1))));
            }
        }
    }
}

// Slices of the sparse Y * scale written straight from the graph (the planes
// are zeroed first): the same arithmetic as k_split applies to each nonzero.
template <int FMT>
__device__ __forceinline__ void put_slices(double xs, int ns, int64_t at, void *s0, void *s1, void *s2)
{
    using ST = typename Sl<FMT>::T;
    const ST a0 = Sl<FMT>::from(float(xs));
    static_cast<ST *>(s0)[at] = a0;
    if (ns > 1) {
        const double r1 = xs - double(Sl<FMT>::to(a0));
        const ST a1 = Sl<FMT>::from(float(r1));
        static_cast<ST *>(s1)[at] = a1;
        if (ns > 2) static_cast<ST *>(s2)[at] = Sl<FMT>::from(float(r1 - double(Sl<FMT>::to(a1))));
    }
}

template <int FMT>
__global__ void k_scatter_slices(SymSparse Y, double sc, int ns, int ld, void *s0, void *s1, void *s2)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < Y.n) {
        const double xs = Y.off * sc;
        for (int a = Y.row_ptr[v]; a < Y.row_ptr[v + 1]; ++a)
            put_slices<FMT>(Y.w ? xs * Y.w[a] : xs, ns, int64_t(v) * ld + Y.col[a], s0, s1, s2);
    }
    if (v < Y.mk.n) {
        const int m = marked_id(Y.mk, v);
        put_slices<FMT>(Y.diag * sc, ns, int64_t(m) * ld + m, s0, s1, s2);
    }
}

// U[i][j] = (Re + i Im)[max(i,j)][min(i,j)] (+ coef * Q[i][j] on Re or Im: the
// last Taylor power, given by its slices) rounded to complex64.  A block takes
// a 32 x 32 tile (bi, bj) on or below the diagonal, reads it once (rows of Re,
// Im and Q into shared memory) and writes both U tiles (bi, bj) and (bj, bi),
// the second from the transposed shared copy, so every global access runs
// along a row and every element is read once.
template <int FMT, int NA>
__global__ void __launch_bounds__(256) k_finish_c64(int n, const double *__restrict__ re,
                                                    const double *__restrict__ im, const void *q0, const void *q1,
                                                    const void *q2, int ldq, double coef, int last_im,
                                                    float2 *__restrict__ U)
{
    using ST = typename Sl<FMT>::T;
    __shared__ double tr[32][33], ti[32][33];
    __shared__ float tq[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int gi = bi * 32 + r, gj = bj * 32 + tx;
        if (gi < n && gj < n && gj <= gi) {
            tr[r][tx] = re[int64_t(gi) * n + gj];
            ti[r][tx] = im[int64_t(gi) * n + gj];
            if (q0) {
                const int64_t at = int64_t(gi) * ldq + gj;
                float q = Sl<FMT>::to(static_cast<const ST *>(q0)[at]);
                if (NA > 1) q += Sl<FMT>::to(static_cast<const ST *>(q1)[at]);
                if (NA > 2) q += Sl<FMT>::to(static_cast<const ST *>(q2)[at]);
                tq[r][tx] = q;
            }
        }
    }
    __syncthreads();
    // the tile itself (on the diagonal, elements above it come from their mirror)
    for (int r = ty; r < 32; r += 8) {
        const int i = bi * 32 + r, j = bj * 32 + tx;
        if (i >= n || j >= n) continue;
        const bool flip = (bi == bj && tx > r);
        const int lr = flip ? tx : r, lc = flip ? r : tx;
        double x = tr[lr][lc], y = ti[lr][lc];
        if (q0) {
            if (last_im) y = fma(coef, fpconv::f32_to_f64(tq[lr][lc]), y);
            else x = fma(coef, fpconv::f32_to_f64(tq[lr][lc]), x);
        }
        U[int64_t(i) * n + j] = make_float2(fpconv::f64_to_f32_rn(x), fpconv::f64_to_f32_rn(y));
    }
    if (bi == bj) return;
    // the mirror tile (bj, bi): element (bj*32 + r, bi*32 + c) = tile element (c, r)
    for (int r = ty; r < 32; r += 8) {
        const int i = bj * 32 + r, j = bi * 32 + tx;
        if (i >= n || j >= n) continue;
        double x = tr[tx][r], y = ti[tx][r];
        if (q0) {
            if (last_im) y = fma(coef, fpconv::f32_to_f64(tq[tx][r]), y);
            else x = fma(coef, fpconv::f32_to_f64(tq[tx][r]), x);
        }
        U[int64_t(i) * n + j] = make_float2(fpconv::f64_to_f32_rn(x), fpconv::f64_to_f32_rn(y));
    }
}

// looked up once (a function-local static is initialised exactly once even
// when several host threads reach it together)
PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
        return nullptr;
    }();
    return fn;
}

// 2D 16-bit map over a [rows][cols] slice with row stride ld: box TK x box_rows
// with 64-byte swizzle, or (wide) 64 x box_rows with 128-byte swizzle
hw_status make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int ld, int fmt, int box_rows,
                   bool wide = false)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return hw_fail(HW_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
    cuuint32_t box[2] = {wide ? 64u : cuuint32_t(TK), cuuint32_t(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, fmt == FMT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     wide ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return hw_fail(HW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return HW_OK;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Slices {
    void *s[3] = {nullptr, nullptr, nullptr};
    CUtensorMap mapA[3];     // boxes of an A tile (128 rows x one K block)
    CUtensorMap mapB[3];     // boxes of a B tile (256 rows x one K block)
    CUtensorMap mapP[3];     // the pair kernel's boxes (128 rows x 64 columns, 128-byte swizzle)
};

// three slice planes of a rows x ld 16-bit matrix in one buffer, plus their maps
hw_status slices_make(Slices &S, uint16_t *buf, int rows, int cols, int ld, int fmt)
{
    for (int i = 0; i < 3; ++i) {
        S.s[i] = buf + size_t(i) * rows * ld;
        hw_status st = make_map(&S.mapA[i], S.s[i], rows, cols, ld, fmt, TM);
        if (st == HW_OK) st = make_map(&S.mapB[i], S.s[i], rows, cols, ld, fmt, TN);
        if (st == HW_OK) st = make_map(&S.mapP[i], S.s[i], rows, cols, ld, fmt, TM, true);
        if (st != HW_OK) return st;
    }
    return HW_OK;
}

// precision modes: (format, slices); the products are the slice pairs (i, j)
// with i + j < slices (3 for two slices, 6 for three)
struct Mode {
    int fmt, ns;
};
const Mode kModes[5] = {
    {FMT_F16, 2},    // 0: default = fp16 x 2
    {FMT_BF16, 1},   // 1: bf16 x 1
    {FMT_BF16, 2},   // 2: bf16 x 2
    {FMT_BF16, 3},   // 3: bf16 x 3
    {FMT_F16, 2},    // 4: fp16 x 2
};

// CTA tiles (P, Q) of 128 x 256, in groups of 8 x 4 (1024 x 1024 elements, so
// that the CTAs running at once share their A rows and B rows in L2); with
// sym only those holding a 128 x 128 block (r, c) with r <= c: row block P,
// column blocks 2Q, 2Q + 1
std::vector<int2> cta_tiles(int m, int n, bool sym)
{
    const int tp = (m + TM - 1) / TM, tq = (n + TN - 1) / TN;
    std::vector<int2> t;
    const int GP = 8, GQ = 4;
    for (int bp = 0; bp < tp; bp += GP)
        for (int bq = 0; bq < tq; bq += GQ)
            for (int p = bp; p < std::min(tp, bp + GP); ++p)
                for (int q = bq; q < std::min(tq, bq + GQ); ++q)
                    if (!sym || TM * p <= TN * q + TN - 1) t.push_back(make_int2(p, q));
    return t;
}

// pair tiles (P, Q) of 256 x 256, in groups of 4 x 4 (1024 x 1024 elements);
// with sym only those holding a 128 x 128 block (r, c) with r <= c, i.e. P <= Q
std::vector<int2> pair_tiles(int m, int n, bool sym)
{
    const int tp = (m + 2 * TM - 1) / (2 * TM), tq = (n + TN - 1) / TN;
    std::vector<int2> t;
    const int GP = 4, GQ = 4;
    for (int bp = 0; bp < tp; bp += GP)
        for (int bq = 0; bq < tq; bq += GQ)
            for (int p = bp; p < std::min(tp, bp + GP); ++p)
                for (int q = bq; q < std::min(tq, bq + GQ); ++q)
                    if (!sym || 2 * TM * p <= TN * q + TN - 1) t.push_back(make_int2(p, q));
    return t;
}

using TcKernel = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap,
                         const CUtensorMap, const CUtensorMap, TcArgs, int);

// dynamic shared memory of a configuration: its ring, no more, so that light
// kernels (the Taylor accumulation) can share the SM with the GEMM
int tc_smem_bytes(int na, int nb)
{
    const int stage = na * kATile + nb * kBTile;
    return std::min(kMaxStages, kRingBytes / stage) * stage + kSmemSlack;
}

TcKernel tc_kernel(int fmt, int na, int nb)
{
    if (fmt == FMT_F16) {
        if (na == 2 && nb == 2) return k_tc_gemm<FMT_F16, 2, 2>;
        if (na == 2 && nb == 1) return k_tc_gemm<FMT_F16, 2, 1>;
        return nullptr;
    }
    if (na == 1 && nb == 1) return k_tc_gemm<FMT_BF16, 1, 1>;
    if (na == 2 && nb == 2) return k_tc_gemm<FMT_BF16, 2, 2>;
    if (na == 2 && nb == 1) return k_tc_gemm<FMT_BF16, 2, 1>;
    if (na == 3 && nb == 3) return k_tc_gemm<FMT_BF16, 3, 3>;
    if (na == 3 && nb == 1) return k_tc_gemm<FMT_BF16, 3, 1>;
    return nullptr;
}

// A with na slices times B with nb slices (nb = na, or 1 when B is exact in one)
hw_status launch_tc(int fmt, int na, int nb, const Slices &A, const Slices &B, const TcArgs &a, int ntiles,
                    cudaStream_t st)
{
    static std::mutex mu;
    static std::map<std::pair<TcKernel, int>, int> max_ctas;   // (kernel, device) -> CTAs at once
    TcKernel kern = tc_kernel(fmt, na, nb);
    if (!kern) return hw_fail(HW_EINVAL, "no tensor-core kernel for %d x %d slices", na, nb);
    int dev = 0;
    cudaGetDevice(&dev);
    const int smem = tc_smem_bytes(na, nb);
    int nctas = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = max_ctas.find({kern, dev});
        if (it != max_ctas.end()) {
            nctas = it->second;
        } else {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_tc_gemm)");
            int sms = 148, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
            if (e != cudaSuccess) return hw_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_tc_gemm)");
            if (per_sm < 1) return hw_fail(HW_EUNSUPPORTED, "k_tc_gemm does not fit on an SM of this device");
            nctas = per_sm * sms;
            max_ctas[{kern, dev}] = nctas;
        }
    }
    // persistent: as many CTAs as run at once, each walking the tile list
    kern<<<std::min(ntiles, nctas), kThreads, smem, st>>>(A.mapA[0], A.mapA[1], A.mapA[2], B.mapB[0], B.mapB[1],
                                                          B.mapB[2], a, ntiles);
    return hw_cuda(cudaGetLastError(), "k_tc_gemm launch");
}

int tc_pair_smem_bytes(int na, int nb)
{
    const int stage = (na + nb) * TM * 64 * 2;   // 64-element K blocks, 128 rows of A and of B per slice
    return std::min(kMaxStages, kRingBytes / stage) * stage + kSmemSlack;
}

TcKernel tc_kernel_pair(int fmt, int na, int nb)
{
    if (fmt == FMT_F16) {
        if (na == 2 && nb == 2) return k_tc_gemm_pair<FMT_F16, 2, 2>;
        if (na == 2 && nb == 1) return k_tc_gemm_pair<FMT_F16, 2, 1>;
        return nullptr;
    }
    if (na == 1 && nb == 1) return k_tc_gemm_pair<FMT_BF16, 1, 1>;
    if (na == 2 && nb == 2) return k_tc_gemm_pair<FMT_BF16, 2, 2>;
    if (na == 2 && nb == 1) return k_tc_gemm_pair<FMT_BF16, 2, 1>;
    if (na == 3 && nb == 3) return k_tc_gemm_pair<FMT_BF16, 3, 3>;
    if (na == 3 && nb == 1) return k_tc_gemm_pair<FMT_BF16, 3, 1>;
    return nullptr;
}

cudaLaunchConfig_t pair_config(int ctas, int smem, cudaStream_t st, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// CTA pairs the device runs at once with this kernel (0: none), cached per (kernel, device)
int tc_pairs(int fmt, int na, int nb)
{
    static std::mutex mu;
    static std::map<std::pair<TcKernel, int>, int> pairs;
    TcKernel kern = tc_kernel_pair(fmt, na, nb);
    if (!kern) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
    std::lock_guard<std::mutex> lk(mu);
    auto it = pairs.find({kern, dev});
    if (it != pairs.end()) return it->second;
    const int smem = tc_pair_smem_bytes(na, nb);
    int nclusters = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess) {
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = pair_config(2, smem, nullptr, at);
        if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) nclusters = 0;
    }
    cudaGetLastError();
    pairs[{kern, dev}] = nclusters;
    return nclusters;
}

// the pair form: tiles from pair_tiles, B boxes of TN / 2 rows (the A maps' box)
hw_status launch_tc_pair(int fmt, int na, int nb, const Slices &A, const Slices &B, const TcArgs &a, int ntiles,
                         cudaStream_t st)
{
    TcKernel kern = tc_kernel_pair(fmt, na, nb);
    const int npairs = tc_pairs(fmt, na, nb);
    if (!kern || npairs < 1) return hw_fail(HW_EUNSUPPORTED, "no CTA-pair tensor-core kernel runs here");
    const int smem = tc_pair_smem_bytes(na, nb);
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = pair_config(2 * std::min(ntiles, npairs), smem, st, at);
    return hw_cuda(cudaLaunchKernelEx(&cfg, kern, A.mapP[0], A.mapP[1], A.mapP[2], B.mapP[0], B.mapP[1],
                                      B.mapP[2], a, ntiles),
                   "k_tc_gemm_pair launch");
}

int row_grid(int64_t rows) { return int(std::min<int64_t>(148 * 16, std::max<int64_t>(rows, 1))); }

hw_status read_err_flag(int *d_err, cudaStream_t st)
{
    int h = 0;
    hw_status s = hw_cuda(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read error flag");
    if (s == HW_OK) s = hw_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (s == HW_OK && h) s = hw_fail(HW_ETIMEDOUT, "tensor-core GEMM: a pipeline wait ran out of time");
    return s;
}

double pow2_scale(double maxabs)
{
    return maxabs > 0 ? std::ldexp(1.0, -int(std::ceil(std::log2(maxabs)))) : 1.0;
}

// true when x leaves nothing for a second slice: the remainder after the
// first slice rounds to zero, exactly as k_split computes it
bool one_slice(int fmt, double x)
{
    if (fmt == FMT_F16) {
        if (std::fabs(x) > 65504.0) return false;
        const __half s0 = __float2half_rn(float(x));
        return __half2float(__float2half_rn(float(x - double(__half2float(s0))))) == 0.0f;
    }
    const __nv_bfloat16 s0 = __float2bfloat16_rn(float(x));
    return __bfloat162float(__float2bfloat16_rn(float(x - double(__bfloat162float(s0))))) == 0.0f;
}

}  // namespace

struct TcPower {
    int n = 0, ld = 0;
    Mode md;
    int nb = 0;              // slices of Y as the B operand (1 when Y / y_unit is exact in one)
    void *mem = nullptr;     // Y slices, two Q slice buffers, tile list, error flag
    Slices Y, Q[2];
    int2 *d_tiles = nullptr;
    int ntiles = 0;
    bool pair = false;       // 256 x 256 tiles on CTA pairs (k_tc_gemm_pair)
    int cur = 0;
    int *err = nullptr;
    double sY = 1, s_prev = 1, theta = 0;
    cudaStream_t st = nullptr;
    // the power whose accumulation is still to do (the next GEMM's epilogue
    // warps do it, the last one a kernel of its own)
    double *pend_accU = nullptr;
    double pend_coef = 0;
    int pend_buf = -1;
};

bool tc_gemm_available()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encoder() != nullptr;
}

// Y: the n x n real symmetric matrix (double) whose powers are taken; yvals
// the magnitudes of its distinct nonzero entries and theta a bound on its
// infinity norm (all host-known).  Y is sliced at the scale 1 / min(yvals)
// when that makes every entry exact in one slice, else at the power of two
// that maps max(yvals) into [1/2, 1].
hw_status tc_power_begin(const SymSparse &Y, const double *yvals, int nyvals, double theta, int mode, int tiles_mode,
                         cudaStream_t st, TcPower **out)
{
    const int n = Y.n;
    *out = nullptr;
    if (mode < 0 || mode > 4) return hw_fail(HW_EINVAL, "gemm precision mode %d", mode);
    if (tiles_mode < 0 || tiles_mode > 2) return hw_fail(HW_EINVAL, "gemm_tiles must be 0..2");
    TcPower *p = new (std::nothrow) TcPower;
    if (!p) return hw_fail(HW_ENOMEM, "host allocation failed");
    p->n = n;
    p->md = kModes[mode];
    p->ld = round_up(n, 64);
    double ymax = 0.0, ymin = 0.0;
    for (int i = 0; i < nyvals; ++i) {
        ymax = std::max(ymax, yvals[i]);
        ymin = (ymin == 0.0) ? yvals[i] : std::min(ymin, yvals[i]);
    }
    bool exact = ymin > 0.0;
    for (int i = 0; i < nyvals && exact; ++i) exact = one_slice(p->md.fmt, yvals[i] * (1.0 / ymin));
    p->sY = exact ? 1.0 / ymin : pow2_scale(ymax);
    p->nb = exact ? 1 : p->md.ns;
    p->s_prev = p->sY;
    p->theta = theta;
    p->st = st;
    // pairs by default where the device co-schedules them
    const bool pairs_here = tc_pairs(p->md.fmt, p->md.ns, p->nb) > 0;
    if (tiles_mode == 2 && !pairs_here) {
        delete p;
        return hw_fail(HW_EUNSUPPORTED, "gemm_tiles = 2: this device runs no CTA pair of the kernel");
    }
    p->pair = tiles_mode == 2 || (tiles_mode == 0 && pairs_here);
    const std::vector<int2> tiles = p->pair ? pair_tiles(n, n, true) : cta_tiles(n, n, true);
    p->ntiles = int(tiles.size());
    const size_t one = size_t(n) * p->ld * 3;     // 16-bit elements per slice buffer (3 planes)
    const size_t tiles_b = sizeof(int2) * tiles.size();
    const size_t bytes = 3 * one * 2 + tiles_b + 256;
    hw_status s = hw_cuda(hw_malloc_async(&p->mem, bytes, st), "scratch allocation (tensor-core slices)");
    if (s != HW_OK) { delete p; return s; }
    uint16_t *b = static_cast<uint16_t *>(p->mem);
    p->d_tiles = reinterpret_cast<int2 *>(b + 3 * one);
    p->err = reinterpret_cast<int *>(reinterpret_cast<char *>(p->d_tiles) + tiles_b);
    const int fmt = p->md.fmt;
    if ((s = hw_cuda(cudaMemsetAsync(p->err, 0, sizeof(int), st), "memset flag")) != HW_OK ||
        (s = hw_cuda(cudaMemcpyAsync(p->d_tiles, tiles.data(), tiles_b, cudaMemcpyHostToDevice, st), "tiles")) != HW_OK ||
        (s = slices_make(p->Y, b, n, n, p->ld, fmt)) != HW_OK ||
        (s = slices_make(p->Q[0], b + one, n, n, p->ld, fmt)) != HW_OK ||
        (s = slices_make(p->Q[1], b + 2 * one, n, n, p->ld, fmt)) != HW_OK) {
        cudaFreeAsync(p->mem, st);
        delete p;
        return s;
    }
    // Y's slices: zero planes, then the nonzeros straight from the graph
    s = hw_cuda(cudaMemsetAsync(p->Y.s[0], 0, one * 2, st), "memset Y slices");
    if (s == HW_OK) {
        const int grid = (std::max(n, Y.mk.n) + 255) / 256;
        if (fmt == FMT_BF16)
            k_scatter_slices<FMT_BF16><<<grid, 256, 0, st>>>(Y, p->sY, p->md.ns, p->ld, p->Y.s[0], p->Y.s[1], p->Y.s[2]);
        else
            k_scatter_slices<FMT_F16><<<grid, 256, 0, st>>>(Y, p->sY, p->md.ns, p->ld, p->Y.s[0], p->Y.s[1], p->Y.s[2]);
        s = hw_cuda(cudaGetLastError(), "k_scatter_slices launch");
    }
    if (s != HW_OK) { cudaFreeAsync(p->mem, st); delete p; return s; }
    p->cur = -1;   // Q_1 = Y: the first step reads the Y slices as A
    *out = p;
    return HW_OK;
}

hw_status launch_acc(const TcPower *p, const Slices &Q, double coef, double *accU)
{
    const int grid = std::min(p->n, 4 * 148);
    if (p->md.fmt == FMT_F16)
        k_taylor_acc<FMT_F16, 2><<<grid, 256, 0, p->st>>>(p->n, Q.s[0], Q.s[1], Q.s[2], p->ld, coef, accU);
    else if (p->md.ns == 1)
        k_taylor_acc<FMT_BF16, 1><<<grid, 256, 0, p->st>>>(p->n, Q.s[0], Q.s[1], Q.s[2], p->ld, coef, accU);
    else if (p->md.ns == 2)
        k_taylor_acc<FMT_BF16, 2><<<grid, 256, 0, p->st>>>(p->n, Q.s[0], Q.s[1], Q.s[2], p->ld, coef, accU);
    else
        k_taylor_acc<FMT_BF16, 3><<<grid, 256, 0, p->st>>>(p->n, Q.s[0], Q.s[1], Q.s[2], p->ld, coef, accU);
    return hw_cuda(cudaGetLastError(), "k_taylor_acc launch");
}

// Q_k = Q_{k-1} Y / k (Y symmetric, so Y is its own K-major B operand; every
// Q_k is symmetric, so only the upper triangle's tiles run).  The same launch
// adds sign_{k-1} Q_{k-1} (its A operand) to accU_{k-1} in double below the
// diagonal; Q_k's own term is added by the next step or by tc_power_end.
hw_status tc_power_step(TcPower *p, int k, double *accU, double sign)
{
    const Slices &A = (p->cur < 0) ? p->Y : p->Q[p->cur];
    const int nxt = (p->cur == 0) ? 1 : 0;
    // bound on max |Q_k| <= ||Y||_inf^k / k!, hence the scale of Q_k's slices
    double bound = 1.0;
    for (int i = 1; i <= k; ++i) bound *= p->theta / double(i);
    const double s_k = pow2_scale(bound);
    TcArgs a{};
    a.tiles = p->d_tiles;
    a.m = a.n = a.k = p->n;
    a.epi = EPI_TAYLOR;
    a.sym = 1;
    a.scale = float(1.0 / (double(k) * p->s_prev * p->sY));
    a.dscale = nullptr;
    for (int i = 0; i < 3; ++i) a.Q[i] = p->Q[nxt].s[i];
    a.ldq = p->ld;
    a.qscale = float(s_k);
    a.err = p->err;
    if (p->pend_accU) {
        // the pending power is Q_{k-1}, this GEMM's A operand
        for (int i = 0; i < 3; ++i) a.accQ[i] = p->Q[p->pend_buf].s[i];
        a.acc_coef = p->pend_coef;
        a.accU = p->pend_accU;
    }
    hw_status s = p->pair ? launch_tc_pair(p->md.fmt, p->md.ns, p->nb, A, p->Y, a, p->ntiles, p->st)
                          : launch_tc(p->md.fmt, p->md.ns, p->nb, A, p->Y, a, p->ntiles, p->st);
    p->pend_accU = accU;
    p->pend_coef = sign / s_k;
    p->pend_buf = nxt;
    p->cur = nxt;
    p->s_prev = s_k;
    return s;
}

hw_status tc_power_end(TcPower *p, cudaStream_t st, bool check)
{
    if (!p) return HW_OK;
    hw_status s = HW_OK;
    if (check && p->pend_accU) s = launch_acc(p, p->Q[p->pend_buf], p->pend_coef, p->pend_accU);
    if (s == HW_OK && check) s = read_err_flag(p->err, st);
    cudaFreeAsync(p->mem, st);
    delete p;
    return s;
}

hw_status tc_power_finish_c64(TcPower *p, const double *Re, const double *Im, void *U, cudaStream_t st)
{
    const int n = p->n;
    const bool last = p->pend_accU != nullptr;
    const Slices &Q = p->Q[last ? p->pend_buf : 0];
    const void *q0 = last ? Q.s[0] : nullptr;
    const int last_im = (p->pend_accU == Im) ? 1 : 0;
    const dim3 grid((n + 31) / 32, (n + 31) / 32);   // blocks above the diagonal return at once
    float2 *u = static_cast<float2 *>(U);
    if (p->md.fmt == FMT_F16)
        k_finish_c64<FMT_F16, 2><<<grid, 256, 0, st>>>(n, Re, Im, q0, Q.s[1], Q.s[2], p->ld, p->pend_coef, last_im, u);
    else if (p->md.ns == 1)
        k_finish_c64<FMT_BF16, 1><<<grid, 256, 0, st>>>(n, Re, Im, q0, Q.s[1], Q.s[2], p->ld, p->pend_coef, last_im, u);
    else if (p->md.ns == 2)
        k_finish_c64<FMT_BF16, 2><<<grid, 256, 0, st>>>(n, Re, Im, q0, Q.s[1], Q.s[2], p->ld, p->pend_coef, last_im, u);
    else
        k_finish_c64<FMT_BF16, 3><<<grid, 256, 0, st>>>(n, Re, Im, q0, Q.s[1], Q.s[2], p->ld, p->pend_coef, last_im, u);
    hw_status s = hw_cuda(cudaGetLastError(), "k_finish_c64 launch");
    if (s == HW_OK) s = read_err_flag(p->err, st);
    cudaFreeAsync(p->mem, st);
    delete p;
    return s;
}

// ---------------------------------------------------------------- plain GEMM entry
extern "C" hw_status hw_gemm_tc(int64_t m, int64_t n, int64_t k, const float *A, const float *B, float *C,
                                int32_t mode, void *stream)
{
    hw_clear_error();
    if (m < 1 || n < 1 || k < 1 || m > (1 << 20) || n > (1 << 20) || k > (1 << 20))
        return hw_fail(HW_EINVAL, "bad GEMM shape");
    if (!A || !B || !C) return hw_fail(HW_EINVAL, "NULL operand");
    if (mode < 1 || mode > 4) return hw_fail(HW_EINVAL, "mode must be 1..4");
    if (!tc_gemm_available()) return hw_fail(HW_EUNSUPPORTED, "needs an sm_103 device");
    {
        // the operands must be memory of the current device (not host or peer memory)
        int dev = -1;
        hw_status ds = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        if (ds != HW_OK) return ds;
        const void *ptrs[3] = {A, B, C};
        for (const void *q : ptrs) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
                cudaGetLastError();
                return hw_fail(HW_EINVAL, "operand %p is not device memory", q);
            }
            if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
                return hw_fail(HW_EINVAL, "operand %p is not memory of the current device %d", q, dev);
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Mode &md = kModes[mode];
    const int ld = round_up(int(k), 64);
    const size_t sa = size_t(m) * ld * 3, sb = size_t(n) * ld * 3;
    const std::vector<int2> tiles = cta_tiles(int(m), int(n), false);
    const size_t tiles_b = sizeof(int2) * tiles.size();
    void *mem = nullptr;
    hw_status s = hw_cuda(hw_malloc_async(&mem, (sa + sb) * 2 + tiles_b + 256, st), "scratch allocation (slices)");
    if (s != HW_OK) return s;
    uint16_t *b = static_cast<uint16_t *>(mem);
    int2 *d_tiles = reinterpret_cast<int2 *>(b + sa + sb);
    char *tail = reinterpret_cast<char *>(d_tiles) + tiles_b;
    unsigned *d_max = reinterpret_cast<unsigned *>(tail);          // [2]
    float *d_scale = reinterpret_cast<float *>(tail + 16);         // [3]: sA, sB, 1/(sA sB)
    int *err = reinterpret_cast<int *>(tail + 64);
    Slices SA, SB;
    if ((s = hw_cuda(cudaMemsetAsync(tail, 0, 128, st), "memset")) == HW_OK &&
        (s = hw_cuda(cudaMemcpyAsync(d_tiles, tiles.data(), tiles_b, cudaMemcpyHostToDevice, st), "tiles")) == HW_OK &&
        (s = slices_make(SA, b, int(m), int(k), ld, md.fmt)) == HW_OK &&
        (s = slices_make(SB, b + sa, int(n), int(k), ld, md.fmt)) == HW_OK) {
        const float *dsA = nullptr, *dsB = nullptr, *dinv = nullptr;
        if (md.fmt == FMT_F16) {
            // fp16 slices are taken of the operand scaled to a maximum in [1/2, 1]
            k_absmax<float><<<row_grid(m), 256, 0, st>>>(A, int(m), int(k), int(k), d_max);
            k_absmax<float><<<row_grid(n), 256, 0, st>>>(B, int(n), int(k), int(k), d_max + 1);
            k_scales<<<1, 1, 0, st>>>(d_max, d_scale);
            dsA = d_scale;
            dsB = d_scale + 1;
            dinv = d_scale + 2;
        }
        if (md.fmt == FMT_BF16) {
            k_split<FMT_BF16, float><<<row_grid(m), 256, 0, st>>>(A, int(m), int(k), int(k), md.ns, ld, dsA, 1.0,
                                                                     SA.s[0], SA.s[1], SA.s[2]);
            k_split<FMT_BF16, float><<<row_grid(n), 256, 0, st>>>(B, int(n), int(k), int(k), md.ns, ld, dsB, 1.0,
                                                                     SB.s[0], SB.s[1], SB.s[2]);
        } else {
            k_split<FMT_F16, float><<<row_grid(m), 256, 0, st>>>(A, int(m), int(k), int(k), md.ns, ld, dsA, 1.0,
                                                                    SA.s[0], SA.s[1], SA.s[2]);
            k_split<FMT_F16, float><<<row_grid(n), 256, 0, st>>>(B, int(n), int(k), int(k), md.ns, ld, dsB, 1.0,
                                                                    SB.s[0], SB.s[1], SB.s[2]);
        }
        TcArgs a{};
        a.tiles = d_tiles;
        a.m = int(m);
        a.n = int(n);
        a.k = int(k);
        a.epi = EPI_STORE;
        a.sym = 0;
        a.scale = 1.0f;
        a.dscale = dinv;
        a.C = C;
        a.ldc = int(n);
        a.err = err;
        s = hw_cuda(cudaGetLastError(), "k_split launch");
        if (s == HW_OK) s = launch_tc(md.fmt, md.ns, md.ns, SA, SB, a, int(tiles.size()), st);
        if (s == HW_OK) s = read_err_flag(err, st);
    }
    cudaFreeAsync(mem, st);
    return s;
}
