// Whole coined walks of small regular graphs in one launch (Sec. 3.2,
// |psi(t)> = (S C)^t |psi(0)>).
//
// A walk on a few thousand vertices moves well under a megabyte per step, so
// one kernel launch per step leaves the GPU idle between launches.  Here one
// thread-block cluster of up to 16 CTAs keeps the whole state in the
// distributed shared memory of its CTAs and runs every step in one launch:
// CTA c owns a contiguous range of vertices and their arcs (arc-major, as in
// the basis), in three buffers at the same shared-memory offsets in every
// CTA.  Step t reads the owned arcs from buffer (t-1) mod 3, applies the coin
// (Grover, -I on marked vertices) and stores each output at its shifted arc
// (reversal or persistent table) in buffer t mod 3 of the CTA that owns that
// arc: a plain shared-memory store when that is this CTA, else st.async,
// which also counts the bytes on the owner's mbarrier t mod 3.  A CTA then
// waits only for the bytes its own arcs receive from other CTAs (known from
// the table), not for the whole cluster.
//
// Why three buffers and no other handshake: a shift moves the walker from v
// to the head w of its arc, and the reverse arc (w, v) exists, so CTA c
// stores into CTA r exactly when r stores into c.  When c starts step t it
// has received r's outputs of step t-1, which r stores only after the CTA
// barrier that ends its step t-2, i.e. after r has read buffer (t-3) mod 3 =
// t mod 3 for the last time; and r cannot run ahead of c by more than one
// step, so each mbarrier only ever counts the bytes of one step.  Every wait
// is bounded (a timeout sets the graph's error word and ends the walk), and a
// hardware cluster barrier before exit keeps every CTA's shared memory alive
// while a peer may still address it.  The state enters from and leaves to
// global memory once per call.
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
    int *err;                 // set when a bounded wait runs out of time
};

constexpr uint64_t kWaitNs = 2000000000ull;   // bounded mbarrier waits (2 s)

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

// st.async: store to a peer CTA's shared memory and count the bytes on the
// peer's mbarrier (both addresses in the shared::cluster window)
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
                 "l"(__double_as_longlong(v)), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void st_async(uint32_t addr, float v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// the one local arrival of a phase, announcing the bytes peers will deliver
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase with this parity has completed (acquire at cluster
// scope: the peers' st.async data is visible after it); false after kWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 0) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitNs) return false;
        }
    }
}

template <typename R> __device__ __forceinline__ R weight(const ClusterArgs &a);
template <> __device__ __forceinline__ double weight<double>(const ClusterArgs &a) { return a.w; }
template <> __device__ __forceinline__ float weight<float>(const ClusterArgs &a) { return a.wf; }

// Shared memory of a CTA: buffers 0, 1, 2, each two planes (real parts,
// imaginary parts) of D rows of vpc values, arc position j of local vertex lv
// at row j, column lv; then the packed target of every owned arc, in the same
// [j][lv] order: (owner rank << 24) | (position in the owner's list) vpc +
// (local vertex in the owner); three mbarriers (static shared memory, same
// offset in every CTA).  A warp works on 32 consecutive vertices and one
// component, so its loads are one row segment, and where the shift keeps
// neighbours together (the torus and the hypercube) its stores are too.
template <typename R, int D>
__global__ void __launch_bounds__(kMaxThreads, 1) k_coined_cluster(ClusterArgs a)
{
    using V = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[3];
    __shared__ int s_local;
    const int vpc = a.vpc;
    const int plane = vpc * D;                 // values per component plane
    R *buf0 = reinterpret_cast<R *>(smem);     // buffer b starts at buf0 + 2 b plane
    uint32_t *tgt = reinterpret_cast<uint32_t *>(buf0 + 6 * plane);
    const int rank = int(cta_rank());
    const int v0 = rank * vpc;
    const int nv = max(0, min(a.n, v0 + vpc) - v0);
    const int arcs = nv * D;
    const V *in = static_cast<const V *>(a.in);
    const uint32_t bar0 = smem_addr(&bars[0]);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) mbar_init(bar0 + 8u * b, 1);
        // the initialised barriers are visible to the peers' st.async
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_local = 0;
    }
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < arcs; i += blockDim.x) {
        const int lv = i / D, j = i - lv * D;
        const int t = __ldg(a.shift + v0 * D + i);   // global arc receiving arc v0 D + i
        const int tw = t / D, r = tw / vpc;
        tgt[j * vpc + lv] = (uint32_t(r) << 24) | uint32_t((t - tw * D) * vpc + (tw - r * vpc));
        local += (r == rank);
        const V x = in[v0 * D + i];
        buf0[j * vpc + lv] = x.x;
        buf0[plane + j * vpc + lv] = x.y;
    }
    if (local) atomicAdd(&s_local, local);
    // every CTA of the cluster is running, has its targets and its barriers
    // before any peer stores into its buffers
    cluster_barrier();
    // the shift is a permutation, so as many owned arcs receive from this CTA
    // as owned arcs send to it; the rest arrive from peers, two components each
    const uint32_t in_bytes = uint32_t(arcs - s_local) * 2u * uint32_t(sizeof(R));
    const uint32_t base0 = smem_addr(buf0), bufbytes = uint32_t(2 * plane) * uint32_t(sizeof(R));
    const R f = weight<R>(a);
    // the two components of the Grover coin are independent sums: the first
    // half of the threads takes the real parts, the second the imaginary
    // parts (blockDim.x is a multiple of 64, so a warp holds one component),
    // which doubles the warps that hide the shared-memory, FP64 and
    // cluster-store latencies
    const int half = int(blockDim.x >> 1);
    const int comp = int(threadIdx.x) >= half ? 1 : 0;
    const int lane_v = int(threadIdx.x) - comp * half;
    int cb = 0, nb = 1;        // buffers read and written by step t
    uint32_t phase = 0;        // parity of each mbarrier's current phase
    for (int64_t t = 1; t <= a.steps; ++t) {
        const R *cur = buf0 + (2 * cb + comp) * plane;
        R *nxt = buf0 + 2 * nb * plane;
        const uint32_t nbase = base0 + uint32_t(nb) * bufbytes, bar = bar0 + 8u * uint32_t(nb);
        if (threadIdx.x == 0) mbar_expect(bar, in_bytes);
        for (int lv = lane_v; lv < nv; lv += half) {
            R p[D];
#pragma unroll
            for (int j = 0; j < D; ++j) p[j] = cur[j * vpc + lv];
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
                const uint32_t g = tgt[j * vpc + lv];
                const R o = fma(fv, sum, -p[j]);
                const uint32_t e = uint32_t(comp * plane) + (g & 0xFFFFFFu);
                const uint32_t r = g >> 24;
                // arcs owned by this CTA take a plain shared-memory store
                if (r == uint32_t(rank)) nxt[e] = o;
                else st_async(peer_addr(nbase + e * uint32_t(sizeof(R)), r), o, peer_addr(bar, r));
            }
        }
        const bool got = mbar_wait(bar, (phase >> nb) & 1u);
        phase ^= 1u << nb;
        // the local stores are visible, and every thread has read buffer cb
        if (__syncthreads_or(!got)) {
            if (threadIdx.x == 0) atomicExch(a.err, 1);
            break;
        }
        if (a.rec_part && t % a.stride == 0) {
            // marked probability after step t, from the owning CTA's buffer
            const R *now = buf0 + 2 * nb * plane;
            for (int i = threadIdx.x; i < a.mk.n; i += blockDim.x) {
                const int lv = marked_id(a.mk, i) - v0;
                if (lv < 0 || lv >= nv) continue;
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const double x = now[j * vpc + lv], y = now[plane + j * vpc + lv];
                    acc += x * x + y * y;
                }
                a.rec_part[(t / a.stride - 1) * a.mk.n + i] = acc;
            }
        }
        cb = nb;
        nb = (nb == 2) ? 0 : nb + 1;
    }
    const R *fin = buf0 + 2 * cb * plane;
    V *out = static_cast<V *>(a.out);
    for (int i = threadIdx.x; i < arcs; i += blockDim.x) {
        const int lv = i / D, j = i - lv * D;
        V x;
        x.x = fin[j * vpc + lv];
        x.y = fin[plane + j * vpc + lv];
        out[v0 * D + i] = x;
    }
    // no CTA leaves while a peer may still address its shared memory
    cluster_barrier();
}

// The walk's bounded wait on an mbarrier whose expected bytes no copy
// delivers: the wait gives up after kWaitNs and the kernel sets the error
// word, exactly as a walk whose peer never answers does (no copy is in
// flight, so the CTA may exit with the phase open).
__global__ void k_wait_check(int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        const uint32_t b = smem_addr(&bar);
        mbar_init(b, 1);
        mbar_expect(b, 16);
        if (!mbar_wait(b, 0)) atomicExch(err, 1);
    }
}

// the kernel attributes (shared-memory limit kSmemLimit, non-portable
// cluster size), set once per kernel and device: a walk of 100 steps takes
// about 90 us, and two driver calls per launch are a visible part of that
std::mutex g_attr_mu;

template <typename R, int D>
cudaError_t set_attributes_once()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return e != cudaSuccess ? e : cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (done[dev]) return cudaSuccess;
    auto kern = k_coined_cluster<R, D>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <typename R, int D>
cudaError_t launch_one(const ClusterArgs &a, int ctas, int threads, size_t smem, cudaStream_t st)
{
    auto kern = k_coined_cluster<R, D>;
    cudaError_t e = set_attributes_once<R, D>();
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
            // the attribute at the kernels' fixed limit (>= probe), as launches set it
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess ||
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
    return size_t(*vpc) * d * (3 * cplx_bytes(dt) + sizeof(uint32_t));
}

}  // namespace

bool coined_cluster_supported(const hw_graph *g, hw_coin coin, hw_dtype dt)
{
    if (coin != HW_COIN_GROVER || g->min_degree != g->max_degree || g->max_degree < 2 || g->max_degree > 8)
        return false;
    int vpc = 0;
    const size_t smem = cluster_smem(g, dt, kMaxClusterCtas, &vpc);
    return smem <= size_t(kSmemLimit) && cluster_ctas(smem) > 0;
}

// Whether the single launch pays off without a measurement of this graph:
// one launch per step costs about 2.4 us whatever the size below these
// limits, and the single launch (measured on tori, hypercubes, cycles and
// random regular graphs) costs about 0.35 us plus 0.7 ns (complex128) or
// 0.15 ns (complex64) per arc of a CTA plus 2 ns per arc it exchanges with
// another CTA, so it wins on every graph below these sizes but on some random
// regular graphs close to them
bool coined_cluster_by_size(const hw_graph *g, hw_dtype dt)
{
    return g->num_arcs <= (dt == HW_C128 ? 16384 : 24576);
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
    a.err = g->d_err;
    // two threads per vertex, a multiple of 64 so that each warp holds one component
    const int threads = std::min(kMaxThreads, std::max(64, (2 * vpc + 63) / 64 * 64));
    const cudaError_t e = (dt == HW_C128) ? launch_deg<double>(g->max_degree, a, ctas, threads, smem, st)
                                          : launch_deg<float>(g->max_degree, a, ctas, threads, smem, st);
    return hw_cuda(e, "k_coined_cluster launch");
}

extern "C" hw_status hw_check_device_wait(const hw_graph *g, void *stream)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    if (!g->d_err) return hw_fail(HW_EINVAL, "graph has no device error word");
    k_wait_check<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(g->d_err);
    return hw_cuda(cudaGetLastError(), "k_wait_check launch");
}
