"""FP64 CPU oracle for quantum-walk evolution (TEST INFRASTRUCTURE ONLY).

A plain, slow restatement of the definitions in Motta et al., "Hiperwalk"
(arXiv 2406.08186): Sec. 3.1 (CTQW: H = -gamma A - sum_m |m><m|, U(t) = e^{-iHt},
with A optionally a weighted, Hermitian adjacency W,
probability |<v|psi>|^2) and Sec. 3.2 (coined walk: U = S C, flip-flop shift
S|v,w> = |w,v>, Grover coin, p_v = sum_w |<v,w|psi>|^2, arcs ordered by tail
then head).  The arithmetic lives in ``hw_oracle.c``; this module builds it
with gcc and wraps it with ctypes for numpy arrays.

Only the tests, the package smoke check and the bench's CPU-baseline leg may
use this module.  It shares no code with the CUDA library and imports nothing
from it; its inputs come from ``synth`` (seeded generators without method
arithmetic).

Readings where the paper is silent (stated here and in the design notes):
  * Fourier coin: C[j][k] = omega^(jk)/sqrt(d), omega = e^{+2 pi i/d}, with j, k
    the positions of the arcs inside the vertex's block (basis order).
  * Marked vertex in the coined walk: its coin block is -I.
  * One coined step applies the coin first, then the shift (U = S C).
  * Persistent shift (torus only): the walker keeps its direction of motion,
    arc (v, w) -> arc (w, u) with u - w = w - v on the torus's coordinates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt variant of the oracle (used by the mutation test, which plants
# mistakes in a copy of hw_oracle.c to show that the pins catch them).
_OVERRIDE = os.environ.get("HW_ORACLE_LIB_OVERRIDE")
_lib = None

GROVER, FOURIER = 0, 1


def build(force: bool = False) -> str:
    """Compile hw_oracle.c into liboracle.so (gcc, OpenMP, IEEE arithmetic)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-fcx-fortran-rules", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _OVERRIDE:
            lib = ctypes.CDLL(_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_threads.argtypes = [ctypes.c_int]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_build_arcs.argtypes = [i64, i64, P, P, P, P, P]
        lib.oracle_build_arcs.restype = ctypes.c_int
        lib.oracle_coin.argtypes = [i64, P, ctypes.c_int, P, P, P]
        lib.oracle_coin.restype = None
        lib.oracle_shift.argtypes = [i64, P, P, P, P]
        lib.oracle_shift.restype = None
        lib.oracle_shift_persistent_torus.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_shift_persistent_torus.restype = None
        lib.oracle_coined_evolve_persistent_torus.argtypes = [i64, i64, P, P, ctypes.c_int, P, P, i64, P]
        lib.oracle_coined_evolve_persistent_torus.restype = ctypes.c_int
        lib.oracle_prob_coined.argtypes = [i64, P, P, P]
        lib.oracle_prob_coined.restype = None
        lib.oracle_coined_evolve.argtypes = [i64, P, P, ctypes.c_int, P, P, i64, P]
        lib.oracle_coined_evolve.restype = ctypes.c_int
        lib.oracle_ctqw_evolve.argtypes = [i64, P, P, ctypes.c_double, P, ctypes.c_double, P, i64, P]
        lib.oracle_ctqw_evolve.restype = ctypes.c_int
        lib.oracle_ctqw_evolve_w.argtypes = [i64, P, P, ctypes.c_double, P, P, ctypes.c_double, P, i64, P]
        lib.oracle_ctqw_evolve_w.restype = ctypes.c_int
        lib.oracle_ctqw_columns_w.argtypes = [i64, P, P, ctypes.c_double, P, P, ctypes.c_double, P, i64, P]
        lib.oracle_ctqw_columns_w.restype = ctypes.c_int
        lib.oracle_arc_weights.argtypes = [i64, P, P, i64, P, P, P, P]
        lib.oracle_arc_weights.restype = ctypes.c_int
        lib.oracle_ctqw_columns.argtypes = [i64, P, P, ctypes.c_double, P, ctypes.c_double, P, i64, P]
        lib.oracle_ctqw_columns.restype = ctypes.c_int
        lib.oracle_ctqw_action.argtypes = [i64, P, P, ctypes.c_double, P, ctypes.c_double, P]
        lib.oracle_ctqw_action.restype = ctypes.c_int64
        lib.oracle_prob_vertex.argtypes = [i64, P, P]
        lib.oracle_prob_vertex.restype = None
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return _load().oracle_threads(n)


class Arcs:
    """The coined walk's computational basis for an undirected graph (Sec. 3.2)."""

    def __init__(self, n: int, eu: np.ndarray, ev: np.ndarray):
        eu = np.ascontiguousarray(eu, dtype=np.int64)
        ev = np.ascontiguousarray(ev, dtype=np.int64)
        self.n = int(n)
        self.row_ptr = np.zeros(self.n + 1, dtype=np.int64)
        self.head = np.zeros(2 * eu.size, dtype=np.int32)
        self.rev = np.zeros(2 * eu.size, dtype=np.int64)
        rc = _load().oracle_build_arcs(self.n, eu.size, _p(eu), _p(ev), _p(self.row_ptr),
                                       _p(self.head), _p(self.rev))
        if rc != 0:
            raise ValueError("invalid graph (oracle code %d)" % rc)

    @property
    def num_arcs(self) -> int:
        return int(self.row_ptr[-1])

    def tail(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))

    def weights(self, eu, ev, we) -> np.ndarray:
        """Arc weights in basis order from one value per edge {eu, ev}: arc (eu, ev)
        gets we, arc (ev, eu) its conjugate (a Hermitian weighted adjacency)."""
        eu = np.ascontiguousarray(eu, dtype=np.int64)
        ev = np.ascontiguousarray(ev, dtype=np.int64)
        we = np.ascontiguousarray(we, dtype=np.complex128)
        out = np.zeros(self.num_arcs, dtype=np.complex128)
        rc = _load().oracle_arc_weights(self.n, _p(self.row_ptr), _p(self.head), eu.size, _p(eu), _p(ev),
                                        _p(we), _p(out))
        if rc != 0:
            raise ValueError("edge without arc")
        return out

    def flags(self, marked) -> np.ndarray:
        f = np.zeros(self.n, dtype=np.uint8)
        if marked is not None and len(marked):
            f[np.asarray(marked, dtype=np.int64)] = 1
        return f


def coin(arcs: Arcs, psi: np.ndarray, coin_kind: int = GROVER, marked=None) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().oracle_coin(arcs.n, _p(arcs.row_ptr), coin_kind, _p(arcs.flags(marked)), _p(psi), _p(out))
    return out


def shift(arcs: Arcs, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().oracle_shift(arcs.n, _p(arcs.row_ptr), _p(arcs.head), _p(psi), _p(out))
    return out


def shift_persistent_torus(arcs: Arcs, L1: int, L2: int, psi: np.ndarray) -> np.ndarray:
    """The persistent shift of the L1 x L2 torus (vertex x*L2 + y): arc (v, w) -> (w, w + (w - v))."""
    assert arcs.n == L1 * L2
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().oracle_shift_persistent_torus(int(L1), int(L2), _p(arcs.row_ptr), _p(arcs.head), _p(psi), _p(out))
    return out


def coined_evolve(arcs: Arcs, psi0: np.ndarray, steps: int, coin_kind: int = GROVER,
                  marked=None, record: bool = False, persistent_torus=None):
    """(S C)^steps psi0; with ``record`` also the marked-vertex probability after each step.
    ``persistent_torus = (L1, L2)`` takes the torus's persistent shift for S instead of
    the flip-flop shift."""
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    rec = np.zeros(max(steps, 1), dtype=np.float64) if record else None
    flags = arcs.flags(marked) if marked is not None and len(marked) else None
    if persistent_torus is not None:
        L1, L2 = persistent_torus
        assert arcs.n == L1 * L2
        rc = _load().oracle_coined_evolve_persistent_torus(int(L1), int(L2), _p(arcs.row_ptr), _p(arcs.head),
                                                           coin_kind, _p(flags), _p(psi), int(steps), _p(rec))
    else:
        rc = _load().oracle_coined_evolve(arcs.n, _p(arcs.row_ptr), _p(arcs.head), coin_kind,
                                          _p(flags), _p(psi), int(steps), _p(rec))
    if rc != 0:
        raise MemoryError("oracle_coined_evolve")
    if record:
        return psi, (rec[:steps] if flags is not None else np.zeros(steps))
    return psi


def prob_coined(arcs: Arcs, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    p = np.empty(arcs.n, dtype=np.float64)
    _load().oracle_prob_coined(arcs.n, _p(arcs.row_ptr), _p(psi), _p(p))
    return p


def ctqw_evolve(arcs: Arcs, gamma: float, psi0: np.ndarray, dt: float, steps: int,
                marked=None, record: bool = False, weights=None):
    """U(dt)^steps psi0 with U = e^{-iH dt}, H = -gamma W - sum_m |m><m|; W = A, or the
    weighted adjacency whose arc weights (basis order, ``Arcs.weights``) are given."""
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    rec = np.zeros(max(steps, 1), dtype=np.float64) if record else None
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.complex128)
    rc = _load().oracle_ctqw_evolve_w(arcs.n, _p(arcs.row_ptr), _p(arcs.head), float(gamma),
                                      _p(arcs.flags(marked)), _p(w), float(dt), _p(psi), int(steps), _p(rec))
    if rc != 0:
        raise MemoryError("oracle_ctqw_evolve")
    return (psi, rec[:steps]) if record else psi


def ctqw_columns(arcs: Arcs, gamma: float, dt: float, cols, marked=None, weights=None) -> np.ndarray:
    """Columns U(dt)[:, j] for j in cols, returned as an [n, len(cols)] array."""
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty((cols.size, arcs.n), dtype=np.complex128)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.complex128)
    rc = _load().oracle_ctqw_columns_w(arcs.n, _p(arcs.row_ptr), _p(arcs.head), float(gamma),
                                       _p(arcs.flags(marked)), _p(w), float(dt), _p(cols), cols.size, _p(out))
    if rc != 0:
        raise MemoryError("oracle_ctqw_columns")
    return out.T.copy()


def ctqw_action(arcs: Arcs, gamma: float, dt: float, x: np.ndarray, marked=None) -> np.ndarray:
    y = np.array(x, dtype=np.complex128, copy=True)
    _load().oracle_ctqw_action(arcs.n, _p(arcs.row_ptr), _p(arcs.head), float(gamma),
                               _p(arcs.flags(marked)), float(dt), _p(y))
    return y


def prob_vertex(psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    p = np.empty(psi.size, dtype=np.float64)
    _load().oracle_prob_vertex(psi.size, _p(psi), _p(p))
    return p
