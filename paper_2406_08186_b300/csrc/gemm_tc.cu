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
// largest entry in [1/2, 1] (exact), so the 5-bit exponent never limits.
//
// One CTA computes one 128 x 128 output tile with 4 warps: warp 0 lane 0
// streams the K blocks (64 elements = one 128-byte swizzle atom) of every
// slice of A and B with TMA into a shared-memory ring (2 to 6 stages,
// 192 KiB); warp 1 lane 0 issues the MMAs and releases stages with
// tcgen05.commit; after the last block all 4 warps drain the accumulator
// (tcgen05.ld, warp w owns TMEM lanes 32w..32w+31 = tile rows) and run the
// epilogue:
//   EPI_STORE:  C = scale * acc (fp32)
//   EPI_TAYLOR: Q = scale * acc, written back as slices of qscale * Q (the
//               next power's A operand) and added to the lower triangle of
//               Re/Im U in double (the caller mirrors it after the series).
// Tiles come from a host-built list in 8 x 8 supertile order, so CTAs that
// run together share operand blocks in L2.  For a symmetric product (every
// Taylor power of the symmetric Y is symmetric) only tiles with I <= J are
// computed and the mirror block is written from the same accumulator with
// coalesced transposed stores.
// Every wait on an mbarrier is bounded; a timeout sets an error flag that the
// host reads, and the CTA still frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr int TM = 128, TN = 128, TK = 64;
constexpr int kTileBytes = TM * TK * 2;                   // 16 KB per slice tile (A or B)
constexpr int kRingBytes = 192 * 1024;                    // shared-memory ring
constexpr int kMaxStages = 6;
constexpr int kSmemBytes = kRingBytes + 1024;             // + alignment slack
constexpr int kTmemCols = 128;                            // 128 lanes x 128 fp32 columns
constexpr uint64_t kWaitLimitNs = 2000000000ull;          // bounded mbarrier waits (2 s)

enum { FMT_BF16 = 0, FMT_F16 = 1 };
enum { EPI_STORE = 0, EPI_TAYLOR = 1 };

struct TcArgs {
    const int2 *tiles;       // (I, J) tile per CTA
    int m, n, k;
    int ns;                  // operand slices (1..3)
    int nprod;               // slice products
    int prod[6][2];          // (A slice, B slice), smallest first
    int stages;              // ring depth
    int epi;
    int sym;                 // mirror each off-diagonal tile to (J, I)
    float scale;             // acc multiplier (host-known part)
    const float *dscale;     // acc multiplier read on the device (or nullptr)
    float *C;                // EPI_STORE: [m][ldc]
    int ldc;
    void *Q[3];              // EPI_TAYLOR: output slices [m][ldq] of qscale * Q
    int ldq;
    float qscale;
    double *accU;            // EPI_TAYLOR: [m][ldu]
    int ldu;
    double sign;
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (the layout TMA writes for a 64-wide 16-bit box).
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

template <int FMT>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
          const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
          const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TcArgs a)
{
    using S = Sl<FMT>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int timed_out;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 tile = a.tiles[blockIdx.x];
    const int m0 = tile.x * TM, n0 = tile.y * TN;
    const int ns = a.ns;
    const int stage_bytes = 2 * ns * kTileBytes;
    const int nkb = (a.k + TK - 1) / TK;
    const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
    const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_done), 1);
        timed_out = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of every slice tile of A and B per K block
        const uint32_t bytes = uint32_t(stage_bytes);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % a.stages;
            const uint32_t use = uint32_t(kb / a.stages);
            if (kb >= a.stages && !mbar_wait(smem_u32(&bar_empty[s]), (use & 1u) ^ 1u)) {
                timed_out = 1;
                break;
            }
            const uint32_t full = smem_u32(&bar_full[s]);
            mbar_expect_tx(full, bytes);
            const uint32_t st = base + uint32_t(s * stage_bytes);
            for (int i = 0; i < ns; ++i) {
                tma_load_2d(st + uint32_t(i * kTileBytes), mA[i], full, kb * TK, m0);
                tma_load_2d(st + uint32_t((ns + i) * kTileBytes), mB[i], full, kb * TK, n0);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % a.stages;
            const uint32_t use = uint32_t(kb / a.stages);
            if (!mbar_wait(smem_u32(&bar_full[s]), use & 1u)) {
                timed_out = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + uint32_t(s * stage_bytes);
            for (int kk = 0; kk < TK / 16; ++kk) {
                for (int p = 0; p < a.nprod; ++p) {
                    const int i = a.prod[p][0], j = a.prod[p][1];
                    const uint64_t ad = smem_desc_sw128(st + uint32_t(i * kTileBytes)) + uint64_t(2 * kk);
                    const uint64_t bd = smem_desc_sw128(st + uint32_t((ns + j) * kTileBytes)) + uint64_t(2 * kk);
                    mma16<FMT>(tmem, ad, bd, (kb > 0 || kk > 0 || p > 0) ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&bar_empty[s]));
        }
        mma_commit(smem_u32(&bar_done));
    }
    __syncwarp();

    // epilogue: every warp drains its 32 TMEM lanes (tile rows)
    const bool done_ok = mbar_wait(smem_u32(&bar_done), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!done_ok) timed_out = 1;
    __syncthreads();
    if (!timed_out) {
        const float mult = a.scale * (a.dscale ? *a.dscale : 1.0f);
        const int rl = warp * 32 + lane;            // tile row held by this thread
        const int row = m0 + rl;
        const bool mirror = a.sym && tile.x != tile.y;
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]) * mult;
            const int col0 = n0 + c0;
            if (a.epi == EPI_STORE) {
                if (row < a.m) {
                    float *dst = a.C + int64_t(row) * a.ldc + col0;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (col0 + q < a.n) dst[q] = v[q];
                }
                continue;
            }
            // Taylor epilogue: slices of qscale * Q (both blocks of a mirrored
            // tile, the next power's A operand) and the double-precision sum,
            // which is kept in the lower triangle only (block (J, I), I <= J) and
            // mirrored once after the series.  The sum's stream uses evict-first
            // loads and stores so it does not push operand blocks out of L2, and
            // all of a chunk's loads are issued before its stores.
            const bool in_row = row < a.m;
            const bool do_mirror = mirror && row < a.n;
            double um[16];
            if (row < a.n) {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    um[q] = (col0 + q < a.m) ? __ldcs(a.accU + int64_t(col0 + q) * a.ldu + row) : 0.0;
            }
            typename S::T sl[3][16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                typename S::T t3[3];
                split<FMT>(v[q] * a.qscale, ns, t3);
                sl[0][q] = t3[0];
                sl[1][q] = t3[1];
                sl[2][q] = t3[2];
            }
            if (in_row) {
                const bool full = col0 + 16 <= a.n;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (i >= ns) break;
                    typename S::T *qd = static_cast<typename S::T *>(a.Q[i]) + int64_t(row) * a.ldq + col0;
                    if (full) {
                        // 16 slice values = 32 contiguous bytes (ldq is a multiple of 64)
                        reinterpret_cast<uint4 *>(qd)[0] = *reinterpret_cast<const uint4 *>(&sl[i][0]);
                        reinterpret_cast<uint4 *>(qd)[1] = *reinterpret_cast<const uint4 *>(&sl[i][8]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (col0 + q < a.n) qd[q] = sl[i][q];
                    }
                }
            }
            if (row < a.n) {
                // element (row, col) -> (col, row): consecutive lanes write consecutive columns
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int mrow = col0 + q;
                    if (mrow >= a.m) continue;
                    if (do_mirror) {
#pragma unroll
                        for (int i = 0; i < 3; ++i)
                            if (i < ns) static_cast<typename S::T *>(a.Q[i])[int64_t(mrow) * a.ldq + row] = sl[i][q];
                    }
                    __stcs(a.accU + int64_t(mrow) * a.ldu + row, um[q] + a.sign * double(v[q]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (threadIdx.x == 0 && timed_out) atomicExch(a.err, 1);
}

// largest |x| of a matrix as float bits (non-negative floats order like their bits)
template <typename T>
__global__ void k_absmax(const T *__restrict__ x, int rows, int cols, int ldx, unsigned *out)
{
    const int64_t total = int64_t(rows) * cols;
    float mx = 0.f;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x)
        mx = fmaxf(mx, fabsf(float(x[(e / cols) * ldx + e % cols])));
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

// matrix -> ns slices of (scale * x) with row stride ld (columns >= cols untouched)
template <int FMT, typename T>
__global__ void k_split(const T *__restrict__ x, int rows, int cols, int ldx, int ns, int ld, const float *dscale,
                        double hscale, void *s0, void *s1, void *s2)
{
    using ST = typename Sl<FMT>::T;
    const int64_t total = int64_t(rows) * cols;
    const double sc = dscale ? double(*dscale) : hscale;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        // the first subtraction runs in T (double for Y) so that fp64 inputs keep their low bits
        const T xs = T(double(x[i * ldx + j]) * sc);
        ST sl[3];
        sl[0] = Sl<FMT>::from(float(xs));
        if (ns > 1) {
            const T r1 = xs - T(Sl<FMT>::to(sl[0]));
            sl[1] = Sl<FMT>::from(float(r1));
            if (ns > 2) sl[2] = Sl<FMT>::from(float(r1 - T(Sl<FMT>::to(sl[1]))));
        }
        static_cast<ST *>(s0)[i * ld + j] = sl[0];
        if (ns > 1) static_cast<ST *>(s1)[i * ld + j] = sl[1];
        if (ns > 2) static_cast<ST *>(s2)[i * ld + j] = sl[2];
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2D 16-bit map over a [rows][cols] slice with row stride ld, box 64 x 128, 128B swizzle
hw_status make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int ld, int fmt)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return hw_fail(HW_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
    cuuint32_t box[2] = {TK, TM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, fmt == FMT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return hw_fail(HW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return HW_OK;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Slices {
    void *s[3] = {nullptr, nullptr, nullptr};
    CUtensorMap map[3];
};

// three slice planes of a rows x ld 16-bit matrix in one buffer, plus their maps
hw_status slices_make(Slices &S, uint16_t *buf, int rows, int cols, int ld, int fmt)
{
    for (int i = 0; i < 3; ++i) {
        S.s[i] = buf + size_t(i) * rows * ld;
        hw_status st = make_map(&S.map[i], S.s[i], rows, cols, ld, fmt);
        if (st != HW_OK) return st;
    }
    return HW_OK;
}

// precision modes: (format, slices, products smallest first)
struct Mode {
    int fmt, ns, nprod;
    int prod[6][2];
};
const Mode kModes[5] = {
    {FMT_F16, 2, 3, {{1, 0}, {0, 1}, {0, 0}}},                                   // 0: default = fp16 x 2
    {FMT_BF16, 1, 1, {{0, 0}}},                                                   // 1: bf16 x 1
    {FMT_BF16, 2, 3, {{1, 0}, {0, 1}, {0, 0}}},                                  // 2: bf16 x 2
    {FMT_BF16, 3, 6, {{1, 1}, {2, 0}, {0, 2}, {1, 0}, {0, 1}, {0, 0}}},          // 3: bf16 x 3
    {FMT_F16, 2, 3, {{1, 0}, {0, 1}, {0, 0}}},                                   // 4: fp16 x 2
};

void fill_mode(TcArgs &a, const Mode &md)
{
    a.ns = md.ns;
    a.nprod = md.nprod;
    std::memcpy(a.prod, md.prod, sizeof a.prod);
    a.stages = std::min(kMaxStages, kRingBytes / (2 * md.ns * kTileBytes));
}

// tiles in 8 x 8 supertile order; with sym only I <= J
std::vector<int2> tile_list(int tm, int tn, bool sym)
{
    std::vector<int2> t;
    const int G = 8;
    for (int bi = 0; bi < tm; bi += G)
        for (int bj = 0; bj < tn; bj += G)
            for (int i = bi; i < std::min(tm, bi + G); ++i)
                for (int j = bj; j < std::min(tn, bj + G); ++j)
                    if (!sym || i <= j) t.push_back(make_int2(i, j));
    return t;
}

hw_status launch_tc(int fmt, const Slices &A, const Slices &B, const TcArgs &a, int ntiles, cudaStream_t st)
{
    static int attr_dev[2] = {-1, -1};
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev[fmt] != dev) {
        cudaError_t e = cudaFuncSetAttribute(fmt == FMT_BF16 ? k_tc_gemm<FMT_BF16> : k_tc_gemm<FMT_F16>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_tc_gemm)");
        attr_dev[fmt] = dev;
    }
    if (fmt == FMT_BF16)
        k_tc_gemm<FMT_BF16><<<ntiles, 128, kSmemBytes, st>>>(A.map[0], A.map[1], A.map[2], B.map[0], B.map[1],
                                                             B.map[2], a);
    else
        k_tc_gemm<FMT_F16><<<ntiles, 128, kSmemBytes, st>>>(A.map[0], A.map[1], A.map[2], B.map[0], B.map[1],
                                                            B.map[2], a);
    return hw_cuda(cudaGetLastError(), "k_tc_gemm launch");
}

int ew_grid(int64_t total) { return int(std::min<int64_t>(148 * 32, (total + 255) / 256)); }

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

}  // namespace

struct TcPower {
    int n = 0, ld = 0;
    Mode md;
    void *mem = nullptr;     // Y slices, two Q slice buffers, tile list, error flag
    Slices Y, Q[2];
    int2 *d_tiles = nullptr;
    int ntiles = 0;
    int cur = 0;
    int *err = nullptr;
    double sY = 1, s_prev = 1, theta = 0;
};

bool tc_gemm_available()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encoder() != nullptr;
}

// Y: the n x n real symmetric matrix (double) whose powers are taken; maxY its
// largest |entry| and theta a bound on its infinity norm (host-known).
hw_status tc_power_begin(int n, const double *Y, double maxY, double theta, int mode, cudaStream_t st,
                         TcPower **out)
{
    *out = nullptr;
    if (mode < 0 || mode > 4) return hw_fail(HW_EINVAL, "gemm precision mode %d", mode);
    TcPower *p = new (std::nothrow) TcPower;
    if (!p) return hw_fail(HW_ENOMEM, "host allocation failed");
    p->n = n;
    p->md = kModes[mode];
    p->ld = round_up(n, 64);
    p->sY = pow2_scale(maxY);
    p->s_prev = p->sY;
    p->theta = theta;
    const int tm = (n + TM - 1) / TM;
    const std::vector<int2> tiles = tile_list(tm, tm, true);
    p->ntiles = int(tiles.size());
    const size_t one = size_t(n) * p->ld * 3;     // 16-bit elements per slice buffer (3 planes)
    const size_t tiles_b = sizeof(int2) * tiles.size();
    const size_t bytes = 3 * one * 2 + tiles_b + 256;
    hw_status s = hw_cuda(cudaMallocAsync(&p->mem, bytes, st), "cudaMallocAsync(tensor-core slices)");
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
    const int64_t nn = int64_t(n) * n;
    if (fmt == FMT_BF16)
        k_split<FMT_BF16, double><<<ew_grid(nn), 256, 0, st>>>(Y, n, n, n, p->md.ns, p->ld, nullptr, p->sY,
                                                               p->Y.s[0], p->Y.s[1], p->Y.s[2]);
    else
        k_split<FMT_F16, double><<<ew_grid(nn), 256, 0, st>>>(Y, n, n, n, p->md.ns, p->ld, nullptr, p->sY,
                                                              p->Y.s[0], p->Y.s[1], p->Y.s[2]);
    s = hw_cuda(cudaGetLastError(), "k_split launch");
    if (s != HW_OK) { cudaFreeAsync(p->mem, st); delete p; return s; }
    p->cur = -1;   // Q_1 = Y: the first step reads the Y slices as A
    *out = p;
    return HW_OK;
}

// Q_k = Q_{k-1} Y / k (Y symmetric, so Y is its own K-major B operand; every
// Q_k is symmetric, so only I <= J tiles run); accU += sign * Q_k in double.
hw_status tc_power_step(TcPower *p, int k, double *accU, double sign, cudaStream_t st)
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
    fill_mode(a, p->md);
    a.epi = EPI_TAYLOR;
    a.sym = 1;
    a.scale = float(1.0 / (double(k) * p->s_prev * p->sY));
    a.dscale = nullptr;
    for (int i = 0; i < 3; ++i) a.Q[i] = p->Q[nxt].s[i];
    a.ldq = p->ld;
    a.qscale = float(s_k);
    a.accU = accU;
    a.ldu = p->n;
    a.sign = sign;
    a.err = p->err;
    hw_status s = launch_tc(p->md.fmt, A, p->Y, a, p->ntiles, st);
    p->cur = nxt;
    p->s_prev = s_k;
    return s;
}

hw_status tc_power_end(TcPower *p, cudaStream_t st, bool check)
{
    if (!p) return HW_OK;
    hw_status s = check ? read_err_flag(p->err, st) : HW_OK;
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
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Mode &md = kModes[mode];
    const int ld = round_up(int(k), 64);
    const size_t sa = size_t(m) * ld * 3, sb = size_t(n) * ld * 3;
    const std::vector<int2> tiles = tile_list(int((m + TM - 1) / TM), int((n + TN - 1) / TN), false);
    const size_t tiles_b = sizeof(int2) * tiles.size();
    void *mem = nullptr;
    hw_status s = hw_cuda(cudaMallocAsync(&mem, (sa + sb) * 2 + tiles_b + 256, st), "cudaMallocAsync(slices)");
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
            k_absmax<float><<<ew_grid(m * k), 256, 0, st>>>(A, int(m), int(k), int(k), d_max);
            k_absmax<float><<<ew_grid(n * k), 256, 0, st>>>(B, int(n), int(k), int(k), d_max + 1);
            k_scales<<<1, 1, 0, st>>>(d_max, d_scale);
            dsA = d_scale;
            dsB = d_scale + 1;
            dinv = d_scale + 2;
        }
        if (md.fmt == FMT_BF16) {
            k_split<FMT_BF16, float><<<ew_grid(m * k), 256, 0, st>>>(A, int(m), int(k), int(k), md.ns, ld, dsA, 1.0,
                                                                     SA.s[0], SA.s[1], SA.s[2]);
            k_split<FMT_BF16, float><<<ew_grid(n * k), 256, 0, st>>>(B, int(n), int(k), int(k), md.ns, ld, dsB, 1.0,
                                                                     SB.s[0], SB.s[1], SB.s[2]);
        } else {
            k_split<FMT_F16, float><<<ew_grid(m * k), 256, 0, st>>>(A, int(m), int(k), int(k), md.ns, ld, dsA, 1.0,
                                                                    SA.s[0], SA.s[1], SA.s[2]);
            k_split<FMT_F16, float><<<ew_grid(n * k), 256, 0, st>>>(B, int(n), int(k), int(k), md.ns, ld, dsB, 1.0,
                                                                    SB.s[0], SB.s[1], SB.s[2]);
        }
        TcArgs a{};
        a.tiles = d_tiles;
        a.m = int(m);
        a.n = int(n);
        a.k = int(k);
        fill_mode(a, md);
        a.epi = EPI_STORE;
        a.sym = 0;
        a.scale = 1.0f;
        a.dscale = dinv;
        a.C = C;
        a.ldc = int(n);
        a.err = err;
        s = hw_cuda(cudaGetLastError(), "k_split launch");
        if (s == HW_OK) s = launch_tc(md.fmt, SA, SB, a, int(tiles.size()), st);
        if (s == HW_OK) s = read_err_flag(err, st);
    }
    cudaFreeAsync(mem, st);
    return s;
}
