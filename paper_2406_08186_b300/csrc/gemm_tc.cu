// Tensor-core GEMM for the complex64 Taylor series of U = e^{-iHt}.
//
// C[m][n] = sum_k A[m][k] B[n][k] with fp32 operands split into bf16 slices
// (x = x0 + x1 + x2, each slice the bf16 rounding of what the previous ones
// leave), multiplied on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, bf16 x bf16 -> fp32 accumulator in tensor memory) and summed
// over the slice products whose magnitude is at least 2^-16 of the leading
// one: 3 slices -> 6 products (about fp32 accuracy), 2 slices -> 3 products.
//
// One CTA computes one 128 x 128 output tile with 4 warps: warp 0 lane 0
// streams the K blocks (64 bf16 = one 128-byte swizzle atom) of every slice
// of A and B with TMA into a 2-stage shared-memory ring; warp 1 lane 0 issues
// the MMAs and releases stages with tcgen05.commit; after the last block all
// 4 warps drain the accumulator (tcgen05.ld, warp w owns TMEM lanes 32w..32w+31
// = tile rows) and run the epilogue:
//   EPI_STORE:  C = scale * acc (fp32)
//   EPI_TAYLOR: Q = scale * acc, written back as bf16 slices (the next power's
//               A operand), and accU += sign * Q in double (the Taylor sum).
// Every wait on an mbarrier is bounded; a timeout sets an error flag that the
// host reads, and the CTA still frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace {

constexpr int TM = 128, TN = 128, TK = 64;
constexpr int kStages = 2;
constexpr int kMaxSlices = 3;
constexpr int kTileBytes = TM * TK * 2;                   // 16 KB per slice tile (A or B)
constexpr int kStageBytes = 2 * kMaxSlices * kTileBytes;  // 96 KB
constexpr int kSmemBytes = kStages * kStageBytes + 1024;  // + alignment slack
constexpr int kTmemCols = 128;                            // 128 lanes x 128 fp32 columns
constexpr uint64_t kWaitLimitNs = 2000000000ull;           // bounded mbarrier waits (2 s)

enum { EPI_STORE = 0, EPI_TAYLOR = 1 };

struct TcArgs {
    int m, n, k;
    int nslices;
    int epi;
    float scale;
    float *C;            // EPI_STORE: [m][ldc]
    int ldc;
    __nv_bfloat16 *Q0, *Q1, *Q2;   // EPI_TAYLOR: output slices [m][ldq]
    int ldq;
    double *accU;        // EPI_TAYLOR: [m][ldu]
    int ldu;
    double sign;
    int *err;            // set to 1 on a wait timeout
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
// groups 1024 bytes apart (the layout TMA writes for a 64-wide bf16 box).
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

// Instruction descriptor: bf16 x bf16 -> fp32, both K-major, M = TM, N = TN.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TN >> 3) << 17) |
                            (uint32_t(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
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

// slice products (i, j): A slice i times B slice j, smallest first
__device__ __constant__ int c_prod3[6][2] = {{1, 1}, {2, 0}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
__device__ __constant__ int c_prod2[3][2] = {{1, 0}, {0, 1}, {0, 0}};

__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
          const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
          const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int timed_out;

    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int ns = a.nslices;
    const int nkb = (a.k + TK - 1) / TK;
    const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
    const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
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
        const uint32_t bytes = uint32_t(2 * ns * kTileBytes);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kStages;
            const uint32_t use = uint32_t(kb / kStages);
            if (kb >= kStages && !mbar_wait(smem_u32(&bar_empty[s]), (use & 1u) ^ 1u)) {
                timed_out = 1;
                break;
            }
            const uint32_t full = smem_u32(&bar_full[s]);
            mbar_expect_tx(full, bytes);
            const uint32_t st = base + uint32_t(s * kStageBytes);
            for (int i = 0; i < ns; ++i) {
                tma_load_2d(st + uint32_t(i * kTileBytes), mA[i], full, kb * TK, m0);
                tma_load_2d(st + uint32_t((kMaxSlices + i) * kTileBytes), mB[i], full, kb * TK, n0);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % kStages;
            const uint32_t use = uint32_t(kb / kStages);
            if (!mbar_wait(smem_u32(&bar_full[s]), use & 1u)) {
                timed_out = 1;
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + uint32_t(s * kStageBytes);
            const int np = (ns == 3) ? 6 : (ns == 2 ? 3 : 1);
            for (int kk = 0; kk < TK / 16; ++kk) {
                for (int p = 0; p < np; ++p) {
                    int i = 0, j = 0;
                    if (ns == 3) { i = c_prod3[p][0]; j = c_prod3[p][1]; }
                    else if (ns == 2) { i = c_prod2[p][0]; j = c_prod2[p][1]; }
                    const uint64_t ad = smem_desc_sw128(st + uint32_t(i * kTileBytes)) + uint64_t(2 * kk);
                    const uint64_t bd =
                        smem_desc_sw128(st + uint32_t((kMaxSlices + j) * kTileBytes)) + uint64_t(2 * kk);
                    mma_bf16(tmem, ad, bd, (kb > 0 || kk > 0 || p > 0) ? 1u : 0u);
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
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
            if (row >= a.m) continue;
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]) * a.scale;
            const int col0 = n0 + c0;
            if (a.epi == EPI_STORE) {
                float *dst = a.C + int64_t(row) * a.ldc + col0;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (col0 + q < a.n) dst[q] = v[q];
            } else {
                __nv_bfloat16 *q0 = a.Q0 + int64_t(row) * a.ldq + col0;
                __nv_bfloat16 *q1 = a.Q1 + int64_t(row) * a.ldq + col0;
                __nv_bfloat16 *q2 = a.Q2 + int64_t(row) * a.ldq + col0;
                double *u = a.accU + int64_t(row) * a.ldu + col0;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (col0 + q >= a.n) continue;
                    const __nv_bfloat16 h = __float2bfloat16_rn(v[q]);
                    const float r1 = v[q] - __bfloat162float(h);
                    const __nv_bfloat16 mdl = __float2bfloat16_rn(r1);
                    const float r2 = r1 - __bfloat162float(mdl);
                    q0[q] = h;
                    q1[q] = mdl;
                    if (a.Q2) q2[q] = __float2bfloat16_rn(r2);
                    u[q] += a.sign * double(v[q]);
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

// fp32 or fp64 matrix -> bf16 slices with row stride ld (columns >= cols untouched)
template <typename T>
__global__ void k_split(const T *__restrict__ x, int rows, int cols, int ldx, int ns, int ld,
                        __nv_bfloat16 *__restrict__ s0, __nv_bfloat16 *__restrict__ s1,
                        __nv_bfloat16 *__restrict__ s2)
{
    const int64_t total = int64_t(rows) * cols;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        T r = x[i * ldx + j];
        const __nv_bfloat16 h = __float2bfloat16_rn(float(r));
        r -= T(__bfloat162float(h));
        const __nv_bfloat16 mdl = __float2bfloat16_rn(float(r));
        r -= T(__bfloat162float(mdl));
        s0[i * ld + j] = h;
        s1[i * ld + j] = mdl;
        if (ns == 3) s2[i * ld + j] = __float2bfloat16_rn(float(r));
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

// 2D bf16 map over a [rows][cols] slice with row stride ld, box 64 x 128, 128B swizzle
hw_status make_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int rows, int cols, int ld)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return hw_fail(HW_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
    cuuint32_t box[2] = {TK, TM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return hw_fail(HW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return HW_OK;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Slices {
    __nv_bfloat16 *s[3] = {nullptr, nullptr, nullptr};
    CUtensorMap map[3];
};

// one buffer holding ns slices of a rows x ld bf16 matrix, plus their maps
hw_status slices_make(Slices &S, __nv_bfloat16 *buf, int rows, int cols, int ld, int ns)
{
    for (int i = 0; i < 3; ++i) {
        S.s[i] = (i < ns) ? buf + size_t(i) * rows * ld : nullptr;
        hw_status st = make_map(&S.map[i], S.s[i < ns ? i : 0], rows, cols, ld);
        if (st != HW_OK) return st;
    }
    return HW_OK;
}

hw_status launch_tc(const Slices &A, const Slices &B, const TcArgs &a, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return hw_cuda(e, "cudaFuncSetAttribute(k_tc_gemm)");
        attr_dev = dev;
    }
    dim3 grid((a.n + TN - 1) / TN, (a.m + TM - 1) / TM);
    k_tc_gemm<<<grid, 128, kSmemBytes, st>>>(A.map[0], A.map[1], A.map[2], B.map[0], B.map[1], B.map[2], a);
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

}  // namespace

struct TcPower {
    int n = 0, ns = 3, ld = 0;
    void *mem = nullptr;     // Y slices, then two Q slice buffers, then the error flag
    Slices Y, Q[2];
    int cur = 0;
    int *err = nullptr;
};

bool tc_gemm_available()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encoder() != nullptr;
}

// ---------------------------------------------------------------- Taylor powers
hw_status tc_power_begin(int n, const double *Y, int ns, cudaStream_t st, TcPower **out)
{
    *out = nullptr;
    TcPower *p = new (std::nothrow) TcPower;
    if (!p) return hw_fail(HW_ENOMEM, "host allocation failed");
    p->n = n;
    p->ns = ns;
    p->ld = round_up(n, 64);
    const size_t one = size_t(n) * p->ld * 3;     // elements per slice buffer (3 slices)
    const size_t bytes = 3 * one * sizeof(__nv_bfloat16) + 256;
    hw_status s = hw_cuda(cudaMallocAsync(&p->mem, bytes, st), "cudaMallocAsync(bf16 slices)");
    if (s != HW_OK) { delete p; return s; }
    __nv_bfloat16 *b = static_cast<__nv_bfloat16 *>(p->mem);
    p->err = reinterpret_cast<int *>(b + 3 * one);
    if ((s = hw_cuda(cudaMemsetAsync(p->err, 0, sizeof(int), st), "memset flag")) != HW_OK ||
        (s = slices_make(p->Y, b, n, n, p->ld, 3)) != HW_OK ||
        (s = slices_make(p->Q[0], b + one, n, n, p->ld, 3)) != HW_OK ||
        (s = slices_make(p->Q[1], b + 2 * one, n, n, p->ld, 3)) != HW_OK) {
        cudaFreeAsync(p->mem, st);
        delete p;
        return s;
    }
    const int64_t nn = int64_t(n) * n;
    k_split<double><<<ew_grid(nn), 256, 0, st>>>(Y, n, n, n, 3, p->ld, p->Y.s[0], p->Y.s[1], p->Y.s[2]);
    s = hw_cuda(cudaGetLastError(), "k_split launch");
    if (s != HW_OK) { cudaFreeAsync(p->mem, st); delete p; return s; }
    p->cur = -1;   // Q_1 = Y: the first step reads the Y slices as A
    *out = p;
    return HW_OK;
}

// Q_k = Q_{k-1} Y / k (Y symmetric, so Y is its own K-major B operand);
// accU += sign * Q_k in double.
hw_status tc_power_step(TcPower *p, int k, double *accU, double sign, cudaStream_t st)
{
    const Slices &A = (p->cur < 0) ? p->Y : p->Q[p->cur];
    const int nxt = (p->cur == 0) ? 1 : 0;
    TcArgs a{};
    a.m = a.n = a.k = p->n;
    a.nslices = p->ns;
    a.epi = EPI_TAYLOR;
    a.scale = float(1.0 / k);
    a.Q0 = p->Q[nxt].s[0];
    a.Q1 = p->Q[nxt].s[1];
    a.Q2 = p->Q[nxt].s[2];
    a.ldq = p->ld;
    a.accU = accU;
    a.ldu = p->n;
    a.sign = sign;
    a.err = p->err;
    hw_status s = launch_tc(A, p->Y, a, st);
    p->cur = nxt;
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
                                int32_t slices, void *stream)
{
    hw_clear_error();
    if (m < 1 || n < 1 || k < 1 || m > (1 << 20) || n > (1 << 20) || k > (1 << 20))
        return hw_fail(HW_EINVAL, "bad GEMM shape");
    if (!A || !B || !C) return hw_fail(HW_EINVAL, "NULL operand");
    if (slices != 1 && slices != 2 && slices != 3) return hw_fail(HW_EINVAL, "slices must be 1, 2 or 3");
    if (!tc_gemm_available()) return hw_fail(HW_EUNSUPPORTED, "needs an sm_103 device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ld = round_up(int(k), 64);
    const size_t sa = size_t(m) * ld * 3, sb = size_t(n) * ld * 3;
    void *mem = nullptr;
    hw_status s = hw_cuda(cudaMallocAsync(&mem, (sa + sb) * sizeof(__nv_bfloat16) + 256, st),
                          "cudaMallocAsync(slices)");
    if (s != HW_OK) return s;
    __nv_bfloat16 *b = static_cast<__nv_bfloat16 *>(mem);
    int *err = reinterpret_cast<int *>(b + sa + sb);
    Slices SA, SB;
    const int ns = slices;
    if ((s = hw_cuda(cudaMemsetAsync(err, 0, sizeof(int), st), "memset flag")) == HW_OK &&
        (s = slices_make(SA, b, int(m), int(k), ld, 3)) == HW_OK &&
        (s = slices_make(SB, b + sa, int(n), int(k), ld, 3)) == HW_OK) {
        k_split<float><<<ew_grid(m * k), 256, 0, st>>>(A, int(m), int(k), int(k), 3, ld, SA.s[0], SA.s[1], SA.s[2]);
        k_split<float><<<ew_grid(n * k), 256, 0, st>>>(B, int(n), int(k), int(k), 3, ld, SB.s[0], SB.s[1], SB.s[2]);
        TcArgs a{};
        a.m = int(m);
        a.n = int(n);
        a.k = int(k);
        a.nslices = ns;
        a.epi = EPI_STORE;
        a.scale = 1.0f;
        a.C = C;
        a.ldc = int(n);
        a.err = err;
        s = hw_cuda(cudaGetLastError(), "k_split launch");
        if (s == HW_OK) s = launch_tc(SA, SB, a, st);
        if (s == HW_OK) s = read_err_flag(err, st);
    }
    cudaFreeAsync(mem, st);
    return s;
}
