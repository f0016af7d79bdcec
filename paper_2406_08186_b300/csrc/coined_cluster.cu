// Whole coined walks of small regular graphs in one launch (Sec. 3.2,
// |psi(t)> = (S C)^t |psi(0)>).
//
// A walk on a few thousand vertices moves well under a megabyte per step, so
// one kernel launch per step leaves the GPU idle between launches.  Here one
// thread-block cluster of up to 16 CTAs keeps the whole state in the
// distributed shared memory of its CTAs and runs every step in one launch:
// CTA c owns a contiguous range of vertices and their arcs (arc-major, as in
// the basis), in two buffers at the same shared-memory offsets in every CTA.
// A step reads the owned arcs from the current buffer, applies the coin
// (Grover, -I on marked vertices) and stores each output at its shifted arc
// (reversal or persistent table) in the next buffer of the CTA that owns that
// arc, with st.shared::cluster; the hardware cluster barrier (release /
// acquire) then separates the steps, so no wait in this kernel is a software
// spin.  The state enters from and leaves to global memory once per call.
//
// The coin arithmetic is the edge-major kernels' (a sequential sum from arc
// 0, for complex128 degree 4 the integer four-term sum rounded once, then one
// FMA per component), so results are bit-identical to the per-step launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "sum4.cuh"

namespace {

constexpr int kMaxClusterCtas = 16;
constexpr int kMaxThreads = 1024;
constexpr int kSmemLimit = 200 * 1024;   // dynamic shared memory per CTA

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

struct ClusterArgs {
    const void *in;
    void *out;
    const int32_t *shift;     // arc-major shift table: out[shift[a]] = (C psi)[a]
    double *rec_part;         // [slots][n_marked] or nullptr
    int64_t steps;
    int64_t stride;           // record stride
    int32_t n;                // vertices
    int32_t vpc;              // vertices per CTA (the last CTAs may own fewer)
    double w;                 // 2/d
    float wf;
    MarkedList mk;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t cta_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// every thread of every CTA of the cluster: stores before it are visible to
// loads after it (release / acquire at cluster scope)
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// the shared::cluster address of shared-memory offset `addr` in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_peer(uint32_t addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

__device__ __forceinline__ void st_peer(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

template <typename R> __device__ __forceinline__ R weight(const ClusterArgs &a);
template <> __device__ __forceinline__ double weight<double>(const ClusterArgs &a) { return a.w; }
template <> __device__ __forceinline__ float weight<float>(const ClusterArgs &a) { return a.wf; }

// Shared memory of a CTA: buffer 0, buffer 1 (vpc D amplitudes each), then the
// packed target of every owned arc: (owner rank << 24) | arc index in the owner.
template <typename R, int D>
__global__ void __launch_bounds__(kMaxThreads) k_coined_cluster(ClusterArgs a)
{
    using V = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int cap = a.vpc * D;
    V *buf0 = reinterpret_cast<V *>(smem);
    V *buf1 = buf0 + cap;
    uint32_t *tgt = reinterpret_cast<uint32_t *>(buf1 + cap);
    const int rank = int(cta_rank());
    const int v0 = rank * a.vpc;
    const int nv = max(0, min(a.n, v0 + a.vpc) - v0);
    const int arcs = nv * D;
    const V *in = static_cast<const V *>(a.in);
    for (int i = threadIdx.x; i < arcs; i += blockDim.x) {
        const int t = __ldg(a.shift + v0 * D + i);   // global arc receiving arc v0 D + i
        const int r = (t / D) / a.vpc;
        tgt[i] = (uint32_t(r) << 24) | uint32_t(t - r * cap);
        buf0[i] = in[v0 * D + i];
    }
    // every CTA of the cluster is running and has its targets before any
    // peer stores into its buffers
    cluster_barrier();
    const uint32_t base0 = smem_addr(buf0), base1 = smem_addr(buf1);
    const R f = weight<R>(a);
    // two threads per vertex: thread 2i takes the real parts of vertex i's
    // arcs, thread 2i + 1 the imaginary parts (the two components of the
    // Grover coin are independent sums), so each step has twice the warps to
    // hide the shared-memory, FP64 and cluster-store latencies
    const int comp = threadIdx.x & 1;
    for (int64_t t = 1; t <= a.steps; ++t) {
        const R *cur = reinterpret_cast<const R *>((t & 1) ? buf0 : buf1);
        R *nxt = reinterpret_cast<R *>((t & 1) ? buf1 : buf0);
        const uint32_t nb = (t & 1) ? base1 : base0;
        for (int lv = threadIdx.x >> 1; lv < nv; lv += blockDim.x >> 1) {
            R p[D];
#pragma unroll
            for (int j = 0; j < D; ++j) p[j] = cur[2 * (lv * D + j) + comp];
            // a marked vertex's coin block is -I
            const bool marked = marked_find(a.mk, v0 + lv) >= 0;
            R sum = 0;
            if (!marked) {
                if constexpr (D == 4 && sizeof(R) == 8) {
                    sum = sum4::sum4_rn(p[0], p[1], p[2], p[3]);
                } else {
                    sum = p[0];
#pragma unroll
                    for (int j = 1; j < D; ++j) sum += p[j];
                }
            }
            // marked: fma(0, 0, -p) = -p, one FMA per output either way (a
            // select against a separate -p would negate every row on the FP64 pipe)
            const R fv = marked ? R(0) : f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const uint32_t g = tgt[lv * D + j];
                const R o = fma(fv, sum, -p[j]);
                const uint32_t e = (g & 0xFFFFFFu) * 2u + uint32_t(comp);
                // arcs owned by this CTA take a plain shared-memory store
                if ((g >> 24) == uint32_t(rank)) nxt[e] = o;
                else st_peer(peer_addr(nb + e * uint32_t(sizeof(R)), g >> 24), o);
            }
        }
        cluster_barrier();
        if (a.rec_part && t % a.stride == 0) {
            // marked probability after step t, from the owning CTA's buffer
            const V *now = (t & 1) ? buf1 : buf0;
            for (int i = threadIdx.x; i < a.mk.n; i += blockDim.x) {
                const int lv = marked_id(a.mk, i) - v0;
                if (lv < 0 || lv >= nv) continue;
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const V q = now[lv * D + j];
                    acc += double(q.x) * double(q.x) + double(q.y) * double(q.y);
                }
                a.rec_part[(t / a.stride - 1) * a.mk.n + i] = acc;
            }
        }
    }
    const V *fin = (a.steps & 1) ? buf1 : buf0;
    V *out = static_cast<V *>(a.out);
    for (int i = threadIdx.x; i < arcs; i += blockDim.x) out[v0 * D + i] = fin[i];
}

template <typename R, int D>
cudaError_t launch_one(const ClusterArgs &a, int ctas, int threads, size_t smem, cudaStream_t st)
{
    auto kern = k_coined_cluster<R, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess && ctas > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename R>
cudaError_t launch_deg(int d, const ClusterArgs &a, int ctas, int threads, size_t smem, cudaStream_t st)
{
    switch (d) {
    case 2: return launch_one<R, 2>(a, ctas, threads, smem, st);
    case 3: return launch_one<R, 3>(a, ctas, threads, smem, st);
    case 4: return launch_one<R, 4>(a, ctas, threads, smem, st);
    case 5: return launch_one<R, 5>(a, ctas, threads, smem, st);
    case 6: return launch_one<R, 6>(a, ctas, threads, smem, st);
    case 7: return launch_one<R, 7>(a, ctas, threads, smem, st);
    case 8: return launch_one<R, 8>(a, ctas, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// largest cluster size (16, else 8) this device runs for a kernel using `smem`
// bytes per CTA, cached per device and size class
std::mutex g_mu;

int cluster_ctas(size_t smem)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    static int cached[64][2] = {};   // [device][smem above 100 KB]: 0 = unknown, -1 = none
    if (dev < 0 || dev >= 64) return 0;
    const int cls = smem > 100 * 1024 ? 1 : 0;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cached[dev][cls] == 0) {
        int best = -1;
        const size_t probe = cls ? size_t(kSmemLimit) : size_t(100 * 1024);
        for (int c : {16, 8}) {
            auto kern = k_coined_cluster<double, 4>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(probe)) != cudaSuccess ||
                (c > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(256);
            cfg.dynamicSmemBytes = probe;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) {
                best = c;
                break;
            }
            cudaGetLastError();
        }
        cached[dev][cls] = best;
    }
    return cached[dev][cls] > 0 ? cached[dev][cls] : 0;
}

// arcs per CTA buffer and shared-memory bytes for a regular graph split over `ctas` CTAs
size_t cluster_smem(const hw_graph *g, hw_dtype dt, int ctas, int *vpc)
{
    const int d = g->max_degree;
    *vpc = int((g->n + ctas - 1) / ctas);
    return size_t(*vpc) * d * (2 * cplx_bytes(dt) + sizeof(uint32_t));
}

}  // namespace

bool coined_cluster_supported(const hw_graph *g, hw_coin coin, hw_dtype dt)
{
    if (coin != HW_COIN_GROVER || g->min_degree != g->max_degree || g->max_degree < 2 || g->max_degree > 8)
        return false;
    // the single launch pays off while a step is too small to fill the GPU.
    // Measured per walk step (one launch per step: 2.4 us whatever the size
    // below these limits): complex128 2.25 us on 16384 arcs, 4.8 us on 32000;
    // complex64 0.74 us on 16384, 3.3 us on 32000
    const int64_t limit = dt == HW_C128 ? 16384 : 24576;
    if (g->num_arcs > limit) return false;
    int vpc = 0;
    return cluster_smem(g, dt, kMaxClusterCtas, &vpc) <= size_t(kSmemLimit) &&
           cluster_ctas(cluster_smem(g, dt, kMaxClusterCtas, &vpc)) > 0;
}

hw_status launch_coined_cluster(const hw_graph *g, hw_dtype dt, const void *in, void *out, int64_t steps,
                                const MarkedList &mk, double *rec_part, int64_t stride, const int32_t *shift,
                                cudaStream_t st)
{
    int vpc = 0;
    const int ctas = cluster_ctas(cluster_smem(g, dt, kMaxClusterCtas, &vpc));
    if (ctas == 0) return hw_fail(HW_EUNSUPPORTED, "no thread-block cluster fits this graph");
    const size_t smem = cluster_smem(g, dt, ctas, &vpc);
    ClusterArgs a;
    a.in = in;
    a.out = out;
    a.shift = shift;
    a.rec_part = rec_part;
    a.steps = steps;
    a.stride = stride;
    a.n = int32_t(g->n);
    a.vpc = vpc;
    const double w = 2.0 / double(g->max_degree);
    a.w = w;
    a.wf = float(w);
    a.mk = mk;
    const int threads = std::min(kMaxThreads, std::max(32, (2 * vpc + 31) / 32 * 32));
    const cudaError_t e = (dt == HW_C128) ? launch_deg<double>(g->max_degree, a, ctas, threads, smem, st)
                                          : launch_deg<float>(g->max_degree, a, ctas, threads, smem, st);
    return hw_cuda(e, "k_coined_cluster launch");
}
