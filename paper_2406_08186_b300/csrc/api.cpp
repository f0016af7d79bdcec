// Entry points of the C ABI: validation, scratch management and dispatch to
// the kernels.  Nothing here computes amplitudes; every step of a walk runs
// in the CUDA kernels of coined.cu, prob.cu and ctqw.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace {
thread_local std::string t_err;
}

hw_status hw_fail(hw_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

hw_status hw_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HW_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return hw_fail(HW_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return hw_fail(HW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void hw_clear_error() { t_err.clear(); }

// Scratch memory comes from one stream-ordered pool per device that keeps
// freed blocks mapped for the next call (the default pool returns them to the
// driver at every synchronisation, and mapping a few hundred MB again costs
// milliseconds).  hw_trim_scratch releases what is not in use.
namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t pool_of(int dev, cudaMemPool_t *out)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
    }
    g_pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}
}  // namespace

cudaError_t hw_malloc_async(void **p, size_t bytes, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (e == cudaSuccess) e = pool_of(dev, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    return e;
}

extern "C" hw_status hw_trim_scratch(void)
{
    hw_clear_error();
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto &kv : g_pools) {
        hw_status s = hw_cuda(cudaMemPoolTrimTo(kv.second, 0), "cudaMemPoolTrimTo");
        if (s != HW_OK) return s;
    }
    return HW_OK;
}

extern "C" const char *hw_last_error(void) { return t_err.c_str(); }

extern "C" const char *hw_version(void) { return "hiperwalk_b300 0.1 (sm_103a)"; }

extern "C" void hw_opts_init(hw_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->record_stride = 1;
    o->taylor_degree = 0;
    o->taylor_squarings = -1;
    o->gemm_mode = 0;
    o->tile = 0;
    o->u_symmetric = 0;
    o->addressing = 0;
    o->shift = 0;
    o->launch_mode = 0;
    o->taylor_powers = 0;
    o->gemm_tiles = 0;
}

hw_status make_marked(const int32_t *marked, int32_t n_marked, int64_t n, cudaStream_t st,
                      MarkedList *out)
{
    std::memset(out, 0, sizeof *out);
    if (n_marked == 0) return HW_OK;
    std::vector<int32_t> m(marked, marked + n_marked);
    std::sort(m.begin(), m.end());
    for (int32_t i = 0; i < n_marked; ++i) {
        if (m[i] < 0 || m[i] >= n) return hw_fail(HW_EINVAL, "marked vertex %d out of range", m[i]);
        if (i && m[i] == m[i - 1]) return hw_fail(HW_EINVAL, "marked vertex %d repeated", m[i]);
    }
    out->n = n_marked;
    if (n_marked <= kInlineMarked) {
        std::copy(m.begin(), m.end(), out->inl);
        return HW_OK;
    }
    int32_t *d = nullptr;
    hw_status s = hw_cuda(hw_malloc_async((void **)&d, sizeof(int32_t) * n_marked, st),
                          "scratch allocation (marked)");
    if (s != HW_OK) return s;
    // the host vector dies on return, so this copy must have completed by then
    s = hw_cuda(cudaMemcpyAsync(d, m.data(), sizeof(int32_t) * n_marked, cudaMemcpyHostToDevice, st),
                "upload marked");
    if (s == HW_OK) s = hw_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (s != HW_OK) { cudaFreeAsync(d, st); return s; }
    out->dev = d;
    return HW_OK;
}

void free_marked(MarkedList &m, cudaStream_t st)
{
    if (m.dev) cudaFreeAsync(const_cast<int32_t *>(m.dev), st);
    m.dev = nullptr;
}

static hw_status check_device(const hw_graph *g)
{
    int dev = -1;
    hw_status s = hw_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != HW_OK) return s;
    if (dev != g->device)
        return hw_fail(HW_EINVAL, "graph lives on device %d, current device is %d", g->device, dev);
    return HW_OK;
}

namespace {
// Scratch taken from the stream-ordered allocator; returned on the stream.
struct Scratch {
    cudaStream_t st;
    void *p = nullptr;
    explicit Scratch(cudaStream_t s) : st(s) {}
    hw_status get(size_t bytes, const char *what)
    {
        return hw_cuda(hw_malloc_async(&p, std::max<size_t>(bytes, 16), st), what);
    }
    ~Scratch() { if (p) cudaFreeAsync(p, st); }
};

// shift operator and addressing of a coined call (hw_opts.shift, .addressing)
hw_status coined_opts(const hw_graph *g, const hw_opts *opts, int *shift, bool *index_free)
{
    if (g->weighted)
        return hw_fail(HW_EINVAL, "coined walks take the adjacency of an unweighted graph (hw_graph_csr)");
    *shift = opts ? opts->shift : kShiftFlipFlop;
    const int addressing = opts ? opts->addressing : 0;
    if (*shift != kShiftFlipFlop && *shift != kShiftPersistent)
        return hw_fail(HW_EINVAL, "shift must be 0 (flip-flop) or 1 (persistent)");
    if (addressing != 0 && addressing != 1) return hw_fail(HW_EINVAL, "addressing must be 0 or 1");
    if (*shift == kShiftPersistent && g->kind != HW_GRAPH_TORUS)
        return hw_fail(HW_EINVAL, "the persistent shift needs a graph recognised as a torus");
    *index_free = addressing == 0;
    return HW_OK;
}
// Whether a batch-1 walk of `steps` steps that fits one thread-block cluster
// runs in one launch (hw_opts.launch_mode 0).  The choice rests on the
// measured fixed and per-step cost of both paths on this graph, dtype and
// shift: measured once, on the first such call (8 and 40 steps of each from
// psi_in into scratch, through hw_coined_evolve itself with launch_mode 2 and
// 1, which synchronises the stream once), then kept on the graph.  Under
// stream capture nothing can be timed and the size rule decides, as it does
// when the measurement cannot run (no memory for its scratch state).
hw_status choose_one_launch(const hw_graph *g, hw_coin coin, hw_dtype dt, const hw_opts *opts, int shift,
                            int64_t steps, const void *psi_in, size_t bytes, cudaStream_t st, bool *one)
{
    const int key = int(dt) * 4 + shift;
    std::array<double, 4> c{};
    bool known = false;
    {
        std::lock_guard<std::mutex> lock(g->tune_mu);
        auto it = g->walk_cost.find(key);
        if (it != g->walk_cost.end()) { c = it->second; known = true; }
    }
    if (!known) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            *one = coined_cluster_by_size(g, dt);
            return HW_OK;
        }
        Scratch out(st);
        hw_status s = out.get(bytes, "scratch allocation (launch choice)");
        if (s != HW_OK) {
            hw_clear_error();
            cudaGetLastError();
            *one = coined_cluster_by_size(g, dt);
            return HW_OK;
        }
        hw_opts o;
        if (opts) o = *opts; else hw_opts_init(&o);
        o.record_stride = 1;
        cudaEvent_t ev[5] = {};
        for (auto &e : ev)
            if (s == HW_OK) s = hw_cuda(cudaEventCreate(&e), "cudaEventCreate");
        float ms[4] = {};
        for (int m = 0; m < 2 && s == HW_OK; ++m) {
            o.launch_mode = (m == 0) ? 2 : 1;
            // a warm-up, then 8 and 40 steps between events
            s = hw_coined_evolve(g, coin, nullptr, 0, dt, 1, 8, psi_in, out.p, nullptr, &o, st);
            if (s == HW_OK) s = hw_cuda(cudaEventRecord(ev[0], st), "event record");
            if (s == HW_OK) s = hw_coined_evolve(g, coin, nullptr, 0, dt, 1, 8, psi_in, out.p, nullptr, &o, st);
            if (s == HW_OK) s = hw_cuda(cudaEventRecord(ev[1], st), "event record");
            if (s == HW_OK) s = hw_coined_evolve(g, coin, nullptr, 0, dt, 1, 40, psi_in, out.p, nullptr, &o, st);
            if (s == HW_OK) s = hw_cuda(cudaEventRecord(ev[2], st), "event record");
            if (s == HW_OK) s = hw_cuda(cudaEventSynchronize(ev[2]), "launch choice");
            if (s == HW_OK) {
                cudaEventElapsedTime(&ms[2 * m], ev[0], ev[1]);
                cudaEventElapsedTime(&ms[2 * m + 1], ev[1], ev[2]);
            }
        }
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (s != HW_OK) {
            // no measurement (e.g. no memory for the scratch state): the size
            // rule decides this call, and the next eligible call measures again
            hw_clear_error();
            cudaGetLastError();
            *one = coined_cluster_by_size(g, dt);
            return HW_OK;
        }
        for (int m = 0; m < 2; ++m) {
            const double per = std::max(0.0, (double(ms[2 * m + 1]) - double(ms[2 * m])) / 32.0);
            c[2 * m] = std::max(0.0, double(ms[2 * m]) - 8.0 * per);
            c[2 * m + 1] = per;
        }
        std::lock_guard<std::mutex> lock(g->tune_mu);
        g->walk_cost[key] = c;
    }
    *one = c[0] + c[1] * double(steps) <= c[2] + c[3] * double(steps);
    return HW_OK;
}

}  // namespace

extern "C" hw_status hw_coined_evolve(const hw_graph *g, hw_coin coin, const int32_t *marked,
                                      int32_t n_marked, hw_dtype dt, int32_t batch, int64_t steps,
                                      const void *psi_in, void *psi_out, double *record,
                                      const hw_opts *opts, void *stream)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    if (coin != HW_COIN_GROVER && coin != HW_COIN_FOURIER) return hw_fail(HW_EINVAL, "unknown coin");
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (steps < 0) return hw_fail(HW_EINVAL, "steps must be >= 0");
    if (n_marked < 0 || (n_marked > 0 && !marked)) return hw_fail(HW_EINVAL, "bad marked list");
    if (!psi_in || !psi_out) return hw_fail(HW_EINVAL, "psi_in/psi_out is NULL");
    const size_t esz = cplx_bytes(dt);
    if ((uintptr_t)psi_in % esz || (uintptr_t)psi_out % esz)
        return hw_fail(HW_EINVAL, "state buffers must be aligned to %zu bytes", esz);
    const int stride = opts ? opts->record_stride : 1;
    if (stride < 1) return hw_fail(HW_EINVAL, "record_stride must be >= 1");
    if (opts && (opts->tile < 0 || opts->tile > 14)) return hw_fail(HW_EINVAL, "tile must be 0..14");
    const int launch_mode = opts ? opts->launch_mode : 0;
    if (launch_mode < 0 || launch_mode > 2) return hw_fail(HW_EINVAL, "launch_mode must be 0, 1 or 2");
    int shift = kShiftFlipFlop;
    bool index_free = false;
    if (hw_status so = coined_opts(g, opts, &shift, &index_free); so != HW_OK) return so;
    if (record && n_marked == 0) return hw_fail(HW_EINVAL, "record needs at least one marked vertex");
    if (record && (uintptr_t)record % 8) return hw_fail(HW_EINVAL, "record must be 8-byte aligned");
    if (coin == HW_COIN_FOURIER && g->max_degree > 4096)
        return hw_fail(HW_EUNSUPPORTED, "Fourier coin limited to degree <= 4096 (max degree %d)",
                       g->max_degree);
    const size_t bytes = size_t(g->num_arcs) * batch * esz;
    const char *ip = static_cast<const char *>(psi_in);
    const char *op = static_cast<const char *>(psi_out);
    if (ip != op && ip < op + bytes && op < ip + bytes)
        return hw_fail(HW_EINVAL, "psi_in and psi_out overlap without being equal");
    hw_status s = check_device(g);
    if (s != HW_OK) return s;
    if (g->h_err && *reinterpret_cast<volatile int *>(g->h_err)) {
        *g->h_err = 0;
        return hw_fail(HW_ETIMEDOUT, "a device-side wait of an earlier call on this graph ran out of time");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    if (steps == 0 || g->num_arcs == 0) {
        if (ip != op && bytes)
            if ((s = hw_cuda(cudaMemcpyAsync(psi_out, psi_in, bytes, cudaMemcpyDeviceToDevice, st),
                             "copy")) != HW_OK)
                return s;
        if (record && steps >= stride) {
            // no arcs: every marked probability is zero
            if ((s = hw_cuda(cudaMemsetAsync(record, 0, sizeof(double) * (steps / stride) * batch, st),
                             "memset record")) != HW_OK)
                return s;
        }
        return HW_OK;
    }

    MarkedList mk;
    if ((s = make_marked(marked, n_marked, g->n, st, &mk)) != HW_OK) return s;
    struct FreeMarked {
        MarkedList &m; cudaStream_t st;
        ~FreeMarked() { free_marked(m, st); }
    } release_marked{mk, st};

    const int64_t slots = record ? steps / stride : 0;
    Scratch tmp(st), recbuf(st);
    double *rec_part = nullptr;
    if (slots) {
        if (n_marked == 1) {
            rec_part = record;  // one marked vertex: partials are the record itself
        } else {
            if ((s = recbuf.get(sizeof(double) * slots * n_marked * batch, "scratch allocation (record)")) != HW_OK)
                return s;
            rec_part = static_cast<double *>(recbuf.p);
        }
    }

    const bool fits = batch == 1 && launch_mode != 1 && coined_cluster_supported(g, coin, dt);
    if (launch_mode == 2 && !fits)
        return hw_fail(HW_EUNSUPPORTED, "launch_mode 2: the walk does not fit one thread-block cluster (batch 1, "
                                        "Grover, regular of degree 2..8, the arcs in the cluster's shared memory)");
    bool one_launch = fits && launch_mode == 2;
    if (fits && launch_mode == 0 &&
        (s = choose_one_launch(g, coin, dt, opts, shift, steps, psi_in, bytes, st, &one_launch)) != HW_OK)
        return s;
    if (one_launch) {
        // small regular graph: every step in one launch, the state held in
        // the shared memory of one thread-block cluster; the kernel records
        // the marked probability after every stride-th step itself
        if ((s = launch_coined_cluster(g, dt, psi_in, psi_out, steps, mk, rec_part, stride,
                                       shift_table(g, shift), st)) != HW_OK)
            return s;
        if (slots && n_marked > 1) return launch_record_finalize(rec_part, n_marked, slots, batch, record, st);
        return HW_OK;
    }
    if (batch == 1 && coined_em_supported(g, coin, dt)) {
        // regular graph: the steps run in the edge-major layout between two
        // scratch buffers; the state is transposed in and out once
        Scratch em(st);
        if ((s = em.get(2 * bytes, "scratch allocation (edge-major states)")) != HW_OK) return s;
        void *E[2] = {em.p, static_cast<char *>(em.p) + bytes};
        if ((s = launch_layout(g, dt, psi_in, E[0], true, st)) != HW_OK) return s;
        int cur = 0;
        for (int64_t k = 1; k <= steps; ++k) {
            CoinedStep cs;
            cs.in = E[cur];
            cs.out = E[1 - cur];
            cs.marked = mk;
            cs.rec_part = rec_part;
            cs.rec_slot = (slots && (k - 1) >= stride && (k - 1) % stride == 0) ? (k - 1) / stride - 1 : -1;
            cs.shift = shift;
            cs.index_free = index_free;
            if ((s = launch_coined_step_em(g, dt, coin, cs, st)) != HW_OK) return s;
            cur = 1 - cur;
        }
        if ((s = launch_layout(g, dt, E[cur], psi_out, false, st)) != HW_OK) return s;
    } else {
    if ((s = tmp.get(bytes, "scratch allocation (state scratch)")) != HW_OK) return s;
    // Ping-pong so that the last step lands in psi_out: step k (1-based) writes
    // psi_out when (steps - k) is even and the scratch otherwise.  In place
    // with an odd step count, step 1 would read and write psi_out, so it reads
    // a scratch copy of the input instead.
    void *P = psi_out, *T = tmp.p;
    const void *src = psi_in;
    if (ip == op && steps % 2 == 1) {
        if ((s = hw_cuda(cudaMemcpyAsync(T, psi_in, bytes, cudaMemcpyDeviceToDevice, st), "copy")) != HW_OK)
            return s;
        src = T;
    }
    for (int64_t k = 1; k <= steps; ++k) {
        void *dst = ((steps - k) % 2 == 0) ? P : T;
        CoinedStep cs;
        cs.in = src;
        cs.out = dst;
        cs.marked = mk;
        cs.rec_part = rec_part;
        cs.rec_slot = (slots && (k - 1) >= stride && (k - 1) % stride == 0) ? (k - 1) / stride - 1 : -1;
        cs.shift = shift;
        cs.index_free = index_free;
        s = (batch == 1) ? launch_coined_step(g, dt, coin, cs, st)
                         : launch_coined_step_batched(g, dt, coin, batch, cs, opts ? opts->tile : 0, st);
        if (s != HW_OK) return s;
        src = dst;
    }
    }
    if (slots && steps % stride == 0) {
        s = launch_marked_prob(g->d_row_ptr, dt, batch, psi_out, mk,
                               rec_part + (slots - 1) * n_marked * batch, st);
        if (s != HW_OK) return s;
    }
    if (slots && n_marked > 1) {
        if ((s = launch_record_finalize(rec_part, n_marked, slots, batch, record, st)) != HW_OK) return s;
    }
    return HW_OK;
}

// Sampled evolution (the paper's simulate(range=(start, end, stride))): the
// states after start, start + stride, ... < end walk steps.  On the
// edge-major path the state stays edge-major between samples and only each
// sample is transposed out; otherwise every segment is one hw_coined_evolve.
extern "C" hw_status hw_coined_sample(const hw_graph *g, hw_coin coin, const int32_t *marked, int32_t n_marked,
                                      hw_dtype dt, int32_t batch, int64_t start, int64_t end, int64_t stride,
                                      const void *psi_in, void *states_out, double *prob_out,
                                      const hw_opts *opts, void *stream)
{
    hw_clear_error();
    if (!g) return hw_fail(HW_EINVAL, "graph is NULL");
    if (start < 0 || end < start || stride < 1) return hw_fail(HW_EINVAL, "need 0 <= start <= end and stride >= 1");
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (!psi_in) return hw_fail(HW_EINVAL, "psi_in is NULL");
    int shift = kShiftFlipFlop;
    bool index_free = false;
    if (hw_status so = coined_opts(g, opts, &shift, &index_free); so != HW_OK) return so;
    const int64_t R = (end - start + stride - 1) / stride;
    if (R == 0) return HW_OK;
    const size_t esz = cplx_bytes(dt);
    const size_t bytes = size_t(g->num_arcs) * batch * esz;
    const size_t pbytes = size_t(g->n) * batch;   // doubles per probability sample
    if (states_out) {
        const char *ip = static_cast<const char *>(psi_in);
        const char *op = static_cast<const char *>(states_out);
        if (ip < op + bytes * R && op < ip + bytes) return hw_fail(HW_EINVAL, "psi_in overlaps states_out");
        if ((uintptr_t)states_out % esz) return hw_fail(HW_EINVAL, "states_out misaligned");
    }
    hw_status s = check_device(g);
    if (s != HW_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch buf(st);
    // where sample r goes when the caller keeps no states
    auto slot = [&](int64_t r) -> void * {
        return states_out ? static_cast<void *>(static_cast<char *>(states_out) + bytes * size_t(r))
                          : static_cast<void *>(static_cast<char *>(buf.p) + bytes * size_t(r & 1));
    };
    const bool em = batch == 1 && g->num_arcs > 0 && coined_em_supported(g, coin, dt);
    if ((s = buf.get((states_out ? 0 : 2 * bytes) + (em ? 2 * bytes : 0), "scratch allocation (samples)")) != HW_OK)
        return s;
    if (em) {
        if (coin != HW_COIN_GROVER && coin != HW_COIN_FOURIER) return hw_fail(HW_EINVAL, "unknown coin");
        MarkedList mk;
        if ((s = make_marked(marked, n_marked, g->n, st, &mk)) != HW_OK) return s;
        struct FreeMarked {
            MarkedList &m; cudaStream_t st;
            ~FreeMarked() { free_marked(m, st); }
        } release_marked{mk, st};
        char *eb = static_cast<char *>(buf.p) + (states_out ? 0 : 2 * bytes);
        void *E[2] = {eb, eb + bytes};
        if ((s = launch_layout(g, dt, psi_in, E[0], true, st)) != HW_OK) return s;
        int cur = 0;
        int64_t t = 0;
        for (int64_t r = 0; r < R; ++r) {
            for (const int64_t tr = start + r * stride; t < tr; ++t) {
                CoinedStep cs;
                cs.in = E[cur];
                cs.out = E[1 - cur];
                cs.marked = mk;
                cs.rec_part = nullptr;
                cs.rec_slot = -1;
                cs.shift = shift;
                cs.index_free = index_free;
                if ((s = launch_coined_step_em(g, dt, coin, cs, st)) != HW_OK) return s;
                cur = 1 - cur;
            }
            if ((s = launch_layout(g, dt, E[cur], slot(r), false, st)) != HW_OK) return s;
            if (prob_out && (s = launch_probability(g, g->n, dt, batch, slot(r), prob_out + pbytes * r, nullptr, st)) !=
                                HW_OK)
                return s;
        }
        return HW_OK;
    }
    const void *src = psi_in;
    int64_t t = 0;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t tr = start + r * stride;
        if ((s = hw_coined_evolve(g, coin, marked, n_marked, dt, batch, tr - t, src, slot(r), nullptr, opts,
                                  stream)) != HW_OK)
            return s;
        if (prob_out && (s = launch_probability(g, g->n, dt, batch, slot(r), prob_out + pbytes * r, nullptr, st)) !=
                            HW_OK)
            return s;
        src = slot(r);
        t = tr;
    }
    return HW_OK;
}

extern "C" hw_status hw_probability(const hw_graph *g, int64_t n, hw_dtype dt, int32_t batch,
                                    const void *psi, double *prob_out, double *norm_out, void *stream)
{
    hw_clear_error();
    if (dt != HW_C64 && dt != HW_C128) return hw_fail(HW_EINVAL, "unknown dtype");
    if (batch < 1) return hw_fail(HW_EINVAL, "batch must be >= 1");
    if (!psi) return hw_fail(HW_EINVAL, "psi is NULL");
    if (!prob_out && !norm_out) return hw_fail(HW_EINVAL, "nothing to compute");
    if ((uintptr_t)psi % cplx_bytes(dt)) return hw_fail(HW_EINVAL, "psi misaligned");
    if (((uintptr_t)prob_out | (uintptr_t)norm_out) % 8) return hw_fail(HW_EINVAL, "outputs misaligned");
    if (g) {
        hw_status s = check_device(g);
        if (s != HW_OK) return s;
        n = g->n;
    } else if (n < 1) {
        return hw_fail(HW_EINVAL, "n must be >= 1");
    }
    return launch_probability(g, n, dt, batch, psi, prob_out, norm_out, static_cast<cudaStream_t>(stream));
}
