"""Python binding of libhiperwalk_b300 (B300 quantum-walk evolution library).

Argument marshalling only: every function here forwards to the C ABI declared
in include/hiperwalk_b300.h, whose kernels do all the work.  Device buffers are
torch CUDA tensors (complex64 / complex128 / float64, contiguous); host inputs
are numpy arrays.  There is no CPU fallback: if the compiled library is
missing the first call raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhiperwalk_b300.so")

HW_OK, HW_EINVAL, HW_ENOMEM, HW_ECUDA, HW_ETIMEDOUT, HW_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
HW_C64, HW_C128 = 1, 2
HW_COIN_GROVER, HW_COIN_FOURIER = 0, 1
HW_JOB_COINED, HW_JOB_CTQW = 0, 1
HW_GRAPH_GENERIC, HW_GRAPH_TORUS, HW_GRAPH_HYPERCUBE = 0, 1, 2
HW_SHIFT_FLIPFLOP, HW_SHIFT_PERSISTENT = 0, 1

STATUS_NAMES = {0: "HW_OK", -1: "HW_EINVAL", -2: "HW_ENOMEM", -3: "HW_ECUDA",
                -4: "HW_ETIMEDOUT", -5: "HW_EUNSUPPORTED"}

# every entry point the header declares
EXPORTS = ("hw_opts_init", "hw_graph_csr", "hw_graph_arcs_host", "hw_graph_free", "hw_graph_info",
           "hw_coined_evolve", "hw_ctqw_plan", "hw_ctqw_expm", "hw_ctqw_evolve", "hw_probability",
           "hw_probability_noalloc", "hw_gemm_tc", "hw_ctqw_evolve_sparse",
           "hw_server_create", "hw_server_submit", "hw_server_run", "hw_server_poll",
           "hw_server_result", "hw_server_stats", "hw_server_destroy", "hw_trim_scratch", "hw_last_error",
           "hw_version", "hw_coined_sample", "hw_ctqw_sample", "hw_graph_structure",
           "hw_graph_structure_host", "hw_measure_fp64", "hw_measure_l2",
           "hw_graph_csr_weighted", "hw_success_curve", "hw_check_device_wait")


class HWError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.message = message


class hw_opts(ctypes.Structure):
    _fields_ = [("record_stride", ctypes.c_int32), ("taylor_degree", ctypes.c_int32),
                ("taylor_squarings", ctypes.c_int32), ("gemm_mode", ctypes.c_int32),
                ("u_symmetric", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("addressing", ctypes.c_int32), ("shift", ctypes.c_int32),
                ("launch_mode", ctypes.c_int32), ("taylor_powers", ctypes.c_int32),
                ("gemm_tiles", ctypes.c_int32)]


class hw_job(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("kind", ctypes.c_int32), ("dt", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("marked", ctypes.c_void_p), ("n_marked", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("gamma", ctypes.c_double), ("time", ctypes.c_double)]


_lib = None


def lib():
    """The loaded shared library (loaded on first use)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhiperwalk_b300.so is not built; run "
                              "`python -m paper_2406_08186_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        st = ctypes.c_int
        L.hw_opts_init.argtypes = [ctypes.POINTER(hw_opts)]
        L.hw_opts_init.restype = None
        L.hw_graph_csr.argtypes = [i64, P, P, P, ctypes.POINTER(P)]
        L.hw_graph_csr.restype = st
        L.hw_graph_csr_weighted.argtypes = [i64, P, P, P, P, P, ctypes.POINTER(P)]
        L.hw_graph_csr_weighted.restype = st
        L.hw_graph_arcs_host.argtypes = [i64, P, P, P, P, P]
        L.hw_graph_arcs_host.restype = st
        L.hw_graph_structure.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.hw_graph_structure.restype = st
        L.hw_graph_structure_host.argtypes = [i64, P, P, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.hw_graph_structure_host.restype = st
        L.hw_graph_free.argtypes = [P]
        L.hw_graph_free.restype = st
        L.hw_graph_info.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                    ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]
        L.hw_graph_info.restype = st
        L.hw_coined_evolve.argtypes = [P, st, P, i32, st, i32, i64, P, P, P, ctypes.POINTER(hw_opts), P]
        L.hw_coined_evolve.restype = st
        L.hw_ctqw_plan.argtypes = [P, d, P, i32, d, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.hw_ctqw_plan.restype = st
        L.hw_ctqw_expm.argtypes = [P, d, P, i32, d, st, P, ctypes.POINTER(hw_opts), P]
        L.hw_ctqw_expm.restype = st
        L.hw_ctqw_evolve.argtypes = [P, i64, st, i32, i64, P, P, P, i32, P, ctypes.POINTER(hw_opts), P]
        L.hw_ctqw_evolve.restype = st
        L.hw_coined_sample.argtypes = [P, st, P, i32, st, i32, i64, i64, i64, P, P, P, ctypes.POINTER(hw_opts), P]
        L.hw_coined_sample.restype = st
        L.hw_ctqw_sample.argtypes = [P, i64, st, i32, i64, i64, i64, P, P, P, ctypes.POINTER(hw_opts), P]
        L.hw_ctqw_sample.restype = st
        L.hw_success_curve.argtypes = [P, i64, i64, i32, P, i32, P, P, P, P]
        L.hw_success_curve.restype = st
        L.hw_probability.argtypes = [P, i64, st, i32, P, P, P, P]
        L.hw_probability.restype = st
        L.hw_probability_noalloc.argtypes = [P, i64, st, i32, P, P, P, P]
        L.hw_probability_noalloc.restype = st
        L.hw_gemm_tc.argtypes = [i64, i64, i64, P, P, P, i32, P]
        L.hw_gemm_tc.restype = st
        L.hw_ctqw_evolve_sparse.argtypes = [P, d, P, i32, d, st, i32, i64, P, P, P, ctypes.POINTER(hw_opts), P]
        L.hw_ctqw_evolve_sparse.restype = st
        L.hw_server_create.argtypes = [i64, i32, i32, i64, P, ctypes.POINTER(P)]
        L.hw_server_create.restype = st
        L.hw_server_submit.argtypes = [P, ctypes.POINTER(hw_job), ctypes.POINTER(i64)]
        L.hw_server_submit.restype = st
        L.hw_server_run.argtypes = [P, ctypes.POINTER(i32)]
        L.hw_server_run.restype = st
        L.hw_server_poll.argtypes = [P, P, i32, ctypes.POINTER(i32)]
        L.hw_server_poll.restype = st
        L.hw_server_result.argtypes = [P, i64, P, i64, P, i64, ctypes.POINTER(d)]
        L.hw_server_result.restype = st
        L.hw_server_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64)]
        L.hw_server_stats.restype = st
        L.hw_server_destroy.argtypes = [P]
        L.hw_server_destroy.restype = st
        L.hw_trim_scratch.argtypes = []
        L.hw_trim_scratch.restype = st
        L.hw_last_error.argtypes = []
        L.hw_last_error.restype = ctypes.c_char_p
        L.hw_measure_fp64.argtypes = [ctypes.POINTER(d), P]
        L.hw_measure_fp64.restype = st
        L.hw_measure_l2.argtypes = [ctypes.POINTER(d), P]
        L.hw_measure_l2.restype = st
        L.hw_check_device_wait.argtypes = [P, P]
        L.hw_check_device_wait.restype = st
        L.hw_version.argtypes = []
        L.hw_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int):
    if status != HW_OK:
        raise HWError(status, lib().hw_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


_CPLX = {HW_C64: "complex64", HW_C128: "complex128"}


def _dev(t, kind=None):
    """Device pointer of a contiguous CUDA tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if kind is not None and str(t.dtype).split(".")[-1] != kind:
        raise ValueError("expected dtype %s, got %s" % (kind, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _host_i32(a):
    if a is None:
        return None, 0
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.size


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, hw_opts):
        return ctypes.byref(opts)
    o = hw_opts_init()
    for k, v in dict(opts).items():
        setattr(o, k, v)
    return ctypes.byref(o)


def hw_opts_init() -> hw_opts:
    o = hw_opts()
    lib().hw_opts_init(ctypes.byref(o))
    return o


def hw_last_error() -> str:
    return lib().hw_last_error().decode()


def hw_trim_scratch():
    """Return the scratch pool's unused device memory to the driver."""
    _check(lib().hw_trim_scratch())


def hw_measure_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device (operations per second)."""
    r = ctypes.c_double()
    _check(lib().hw_measure_fp64(ctypes.byref(r), _stream(stream)))
    return r.value


def hw_measure_l2(stream=None) -> float:
    """Measured copy bandwidth (GB/s, read + write) of an L2-resident 32 MB working set."""
    r = ctypes.c_double()
    _check(lib().hw_measure_l2(ctypes.byref(r), _stream(stream)))
    return r.value


def hw_check_device_wait(g: Graph, stream=None):
    """Run the one-launch walk's bounded device wait on a barrier nothing completes (about 2 s);
    the next hw_coined_evolve on g reports HW_ETIMEDOUT."""
    _check(lib().hw_check_device_wait(g, _stream(stream)))


def hw_version() -> str:
    return lib().hw_version().decode()


class Graph:
    """Owner of an ``hw_graph`` handle (freed by ``free()`` or garbage collection)."""

    def __init__(self, handle, n, num_arcs):
        self.handle = handle
        self.n = n
        self.num_arcs = num_arcs

    def free(self):
        if self.handle is not None and _lib is not None:
            _lib.hw_graph_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if self.handle is None:
            raise ValueError("graph already freed")
        return self.handle


def hw_graph_csr(n: int, row_ptr, col_idx, stream=None) -> Graph:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().hw_graph_csr(int(n), rp.ctypes.data_as(ctypes.c_void_p),
                              ci.ctypes.data_as(ctypes.c_void_p), _stream(stream), ctypes.byref(h)))
    g = Graph(h, int(n), 0)
    g.num_arcs = hw_graph_info(g)["num_arcs"]
    return g


def hw_graph_csr_weighted(n: int, row_ptr, col_idx, weights, stream=None) -> Graph:
    """A graph whose CTQW Hamiltonian uses the weighted adjacency: ``weights`` is
    aligned with ``col_idx``, real (symmetric W) or complex (Hermitian W)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    w = np.asarray(weights)
    wre = np.ascontiguousarray(w.real, dtype=np.float64)
    wim = np.ascontiguousarray(w.imag, dtype=np.float64) if np.iscomplexobj(w) else None
    h = ctypes.c_void_p()
    _check(lib().hw_graph_csr_weighted(int(n), rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                                       wre.ctypes.data_as(ctypes.c_void_p),
                                       None if wim is None else wim.ctypes.data_as(ctypes.c_void_p),
                                       _stream(stream), ctypes.byref(h)))
    g = Graph(h, int(n), 0)
    g.num_arcs = hw_graph_info(g)["num_arcs"]
    return g


def hw_graph_arcs_host(n: int, row_ptr, col_idx):
    """(row_ptr int32[n+1], head int32[2E], rev int32[2E]) computed by the library on the host."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    m = int(rp[-1]) if rp.size else 0
    rp_out = np.zeros(int(n) + 1, dtype=np.int32)
    head = np.zeros(max(m, 0), dtype=np.int32)
    rev = np.zeros(max(m, 0), dtype=np.int32)
    _check(lib().hw_graph_arcs_host(int(n), rp.ctypes.data_as(ctypes.c_void_p),
                                    ci.ctypes.data_as(ctypes.c_void_p),
                                    rp_out.ctypes.data_as(ctypes.c_void_p),
                                    head.ctypes.data_as(ctypes.c_void_p),
                                    rev.ctypes.data_as(ctypes.c_void_p)))
    return rp_out, head, rev


def hw_graph_structure(g: Graph):
    """(kind, (a, b)): HW_GRAPH_TORUS with (L1, L2), HW_GRAPH_HYPERCUBE with (k, 0), else HW_GRAPH_GENERIC."""
    kind = ctypes.c_int32()
    dims = (ctypes.c_int64 * 2)()
    _check(lib().hw_graph_structure(g, ctypes.byref(kind), dims))
    return kind.value, (dims[0], dims[1])


def hw_graph_structure_host(n: int, row_ptr, col_idx):
    """hw_graph_structure's test on a host CSR (no device)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    kind = ctypes.c_int32()
    dims = (ctypes.c_int64 * 2)()
    _check(lib().hw_graph_structure_host(int(n), rp.ctypes.data_as(ctypes.c_void_p),
                                         ci.ctypes.data_as(ctypes.c_void_p), ctypes.byref(kind), dims))
    return kind.value, (dims[0], dims[1])


def hw_graph_free(g: Graph):
    g.free()


def hw_graph_info(g: Graph) -> dict:
    n, m = ctypes.c_int64(), ctypes.c_int64()
    rp, hd, rv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().hw_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(rp),
                               ctypes.byref(hd), ctypes.byref(rv)))
    return {"n": n.value, "num_arcs": m.value, "d_row_ptr": rp.value, "d_head": hd.value,
            "d_rev": rv.value}


def hw_coined_evolve(g: Graph, coin: int, marked, dt: int, batch: int, steps: int, psi_in, psi_out,
                     record=None, opts=None, stream=None):
    m, nm = _host_i32(marked)
    _check(lib().hw_coined_evolve(g, int(coin), None if m is None else m.ctypes.data_as(ctypes.c_void_p),
                                  nm, int(dt), int(batch), int(steps), _dev(psi_in, _CPLX[dt]),
                                  _dev(psi_out, _CPLX[dt]), _dev(record, "float64"), _opts(opts),
                                  _stream(stream)))


def hw_ctqw_plan(g: Graph, gamma: float, marked, time: float):
    """(Taylor degree, squarings) that hw_ctqw_expm chooses by default."""
    m, nm = _host_i32(marked)
    deg, sq = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().hw_ctqw_plan(g, float(gamma), None if m is None else m.ctypes.data_as(ctypes.c_void_p),
                              nm, float(time), ctypes.byref(deg), ctypes.byref(sq)))
    return deg.value, sq.value


def hw_ctqw_expm(g: Graph, gamma: float, marked, time: float, dt: int, U_out, opts=None, stream=None):
    m, nm = _host_i32(marked)
    _check(lib().hw_ctqw_expm(g, float(gamma), None if m is None else m.ctypes.data_as(ctypes.c_void_p),
                              nm, float(time), int(dt), _dev(U_out, _CPLX[dt]), _opts(opts),
                              _stream(stream)))


def hw_ctqw_evolve(U, n: int, dt: int, batch: int, steps: int, psi_in, psi_out, marked=None,
                   record=None, opts=None, stream=None):
    m, nm = _host_i32(marked)
    _check(lib().hw_ctqw_evolve(_dev(U, _CPLX[dt]), int(n), int(dt), int(batch), int(steps),
                                _dev(psi_in, _CPLX[dt]), _dev(psi_out, _CPLX[dt]),
                                None if m is None else m.ctypes.data_as(ctypes.c_void_p), nm,
                                _dev(record, "float64"), _opts(opts), _stream(stream)))


def hw_coined_sample(g: Graph, coin: int, marked, dt: int, batch: int, start: int, end: int, stride: int,
                     psi_in, states_out=None, prob_out=None, opts=None, stream=None):
    """States (and per-vertex probabilities) after start, start + stride, ... < end steps."""
    m, nm = _host_i32(marked)
    _check(lib().hw_coined_sample(g, int(coin), None if m is None else m.ctypes.data_as(ctypes.c_void_p), nm,
                                  int(dt), int(batch), int(start), int(end), int(stride), _dev(psi_in, _CPLX[dt]),
                                  _dev(states_out, _CPLX[dt]), _dev(prob_out, "float64"), _opts(opts),
                                  _stream(stream)))


def hw_ctqw_sample(U, n: int, dt: int, batch: int, start: int, end: int, stride: int, psi_in, states_out=None,
                   prob_out=None, opts=None, stream=None):
    """U^k psi_in for k = start, start + stride, ... < end (and their probabilities)."""
    _check(lib().hw_ctqw_sample(_dev(U, _CPLX[dt]), int(n), int(dt), int(batch), int(start), int(end),
                                int(stride), _dev(psi_in, _CPLX[dt]), _dev(states_out, _CPLX[dt]),
                                _dev(prob_out, "float64"), _opts(opts), _stream(stream)))


def sample_count(start: int, end: int, stride: int) -> int:
    """Number of samples of range(start, end, stride)."""
    return max(0, (end - start + stride - 1) // stride)


def hw_success_curve(prob, marked, curve_out, argmax_out=None, max_out=None, stream=None):
    """Success probability of a search per sample, curve[r][b] = sum over the
    marked vertices of prob[r][m][b], and the first sample where it peaks
    (device tensors: prob float64 [R][n] or [R][n][batch], curve_out float64
    [R] or [R][batch], argmax_out int64 [batch], max_out float64 [batch])."""
    R, n = int(prob.shape[0]), int(prob.shape[1])
    batch = int(prob.shape[2]) if prob.dim() == 3 else 1
    m, nm = _host_i32(marked)
    _check(lib().hw_success_curve(_dev(prob, "float64"), R, n, batch,
                                  None if m is None else m.ctypes.data_as(ctypes.c_void_p), nm,
                                  _dev(curve_out, "float64"), _dev(argmax_out, "int64"),
                                  _dev(max_out, "float64"), _stream(stream)))


def success_curve(prob, marked, stream=None):
    """(curve, sample index of the maximum, maximum) of a single-state search from
    its sampled probabilities prob [R][n] (a float64 CUDA tensor), computed by
    hw_success_curve; the two scalars are read back (the call synchronises)."""
    import torch
    curve = torch.empty(prob.shape[0], dtype=torch.float64, device=prob.device)
    k = torch.empty(1, dtype=torch.int64, device=prob.device)
    mx = torch.empty(1, dtype=torch.float64, device=prob.device)
    hw_success_curve(prob, marked, curve, k, mx, stream=stream)
    return curve, int(k.item()), float(mx.item())


def hw_probability(g, n: int, dt: int, batch: int, psi, prob_out=None, norm_out=None, stream=None):
    _check(lib().hw_probability(g, int(n), int(dt), int(batch), _dev(psi, _CPLX[dt]),
                                _dev(prob_out, "float64"), _dev(norm_out, "float64"), _stream(stream)))


def hw_probability_noalloc(g, n: int, dt: int, batch: int, psi, prob_out=None, norm_out=None,
                           stream=None):
    """hw_probability without device allocation (norm partials in a built-in array; batch <= 64)."""
    _check(lib().hw_probability_noalloc(g, int(n), int(dt), int(batch), _dev(psi, _CPLX[dt]),
                                        _dev(prob_out, "float64"), _dev(norm_out, "float64"),
                                        _stream(stream)))


HW_GEMM_BF16X1, HW_GEMM_BF16X2, HW_GEMM_BF16X3, HW_GEMM_F16X2 = 1, 2, 3, 4


def hw_gemm_tc(A, B, C, mode: int = HW_GEMM_F16X2, stream=None):
    """C = A @ B.T on the tensor cores from split 16-bit slices of fp32 operands (device float32 tensors)."""
    m, k = A.shape
    n = B.shape[0]
    _check(lib().hw_gemm_tc(int(m), int(n), int(k), _dev(A, "float32"), _dev(B, "float32"),
                            _dev(C, "float32"), int(mode), _stream(stream)))


def hw_ctqw_evolve_sparse(g: Graph, gamma: float, marked, time: float, dt: int, batch: int, steps: int,
                          psi_in, psi_out, record=None, opts=None, stream=None):
    m, nm = _host_i32(marked)
    _check(lib().hw_ctqw_evolve_sparse(g, float(gamma), None if m is None else m.ctypes.data_as(ctypes.c_void_p),
                                       nm, float(time), int(dt), int(batch), int(steps),
                                       _dev(psi_in, _CPLX[dt]), _dev(psi_out, _CPLX[dt]),
                                       _dev(record, "float64"), _opts(opts), _stream(stream)))


class Server:
    """Owner of an ``hw_server`` (continuous batching of walk jobs)."""

    def __init__(self, arena_bytes: int, max_jobs: int = 256, substeps: int = 8, host_bytes: int = 1 << 30):
        h = ctypes.c_void_p()
        _check(lib().hw_server_create(int(arena_bytes), int(max_jobs), int(substeps), int(host_bytes), None,
                                      ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    @property
    def _as_parameter_(self):
        return self.handle

    def submit(self, graph: Graph, kind: int, dt: int, steps: int, marked=(), gamma: float = 0.0,
               time: float = 0.0) -> int:
        m = np.ascontiguousarray(list(marked), dtype=np.int32)
        j = hw_job(graph.handle, int(kind), int(dt), int(steps),
                   m.ctypes.data_as(ctypes.c_void_p) if m.size else None, int(m.size), 0, float(gamma),
                   float(time))
        jid = ctypes.c_int64()
        _check(lib().hw_server_submit(self, ctypes.byref(j), ctypes.byref(jid)))
        self._keep[jid.value] = (graph, int(steps), int(m.size))
        return jid.value

    def run(self) -> int:
        n = ctypes.c_int32()
        _check(lib().hw_server_run(self, ctypes.byref(n)))
        return n.value

    def poll(self, max_ids: int = 4096):
        ids = np.zeros(max_ids, dtype=np.int64)
        n = ctypes.c_int32()
        _check(lib().hw_server_poll(self, ids.ctypes.data_as(ctypes.c_void_p), int(max_ids), ctypes.byref(n)))
        return [int(x) for x in ids[:n.value]]

    def result(self, job_id: int):
        graph, steps, nm = self._keep.pop(job_id)
        prob = np.empty(graph.n, dtype=np.float64)
        rec = np.empty(steps, dtype=np.float64) if nm else None
        lat = ctypes.c_double()
        _check(lib().hw_server_result(self, int(job_id), prob.ctypes.data_as(ctypes.c_void_p), prob.size,
                                      None if rec is None else rec.ctypes.data_as(ctypes.c_void_p),
                                      0 if rec is None else rec.size, ctypes.byref(lat)))
        return prob, rec, lat.value

    def stats(self):
        q, r, a, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().hw_server_stats(self, ctypes.byref(q), ctypes.byref(r), ctypes.byref(a), ctypes.byref(t)))
        return {"queued": q.value, "resident": r.value, "arena_used": a.value, "ticks": t.value}

    def drain(self):
        """Run rounds until every submitted job is collectable; returns their ids."""
        done = []
        while True:
            self.run()
            done += self.poll()
            st = self.stats()
            if st["queued"] == 0 and st["resident"] == 0:
                self.run()
                done += self.poll()
                return done

    def close(self):
        if self.handle is not None and _lib is not None:
            _lib.hw_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
