"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the quantum-walk method: it only draws
random numbers and lays out graphs and initial states.  Everything here is
deterministic given its seed.

Random numbers: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014).  Stream k of seed s
is ``mix(s + (k + 1) * 0x9E3779B97F4A7C15)``; doubles take the top 53 bits.
Gaussians use the Box-Muller transform in float64.

Graphs are returned as undirected edge lists ``(eu, ev)`` (int64, each edge
once, no self-loops, no duplicates) plus the vertex count.  ``adjacency_csr``
turns an edge list into the CSR of the symmetric 0/1 adjacency matrix with the
columns of each row in a scrambled (unsorted) order, which is the input form
the library accepts.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream of ``seed``."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def complex_gaussian(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` complex normals z = x + i y by Box-Muller, one pair of uniforms each."""
    u = uniform01(seed, 2 * count, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1 - u1 in (0, 1]
    th = 2.0 * math.pi * u2
    return r * np.cos(th) + 1j * (r * np.sin(th))


def seeded_vertex(seed: int, n: int) -> int:
    """First SplitMix64 output of ``seed`` reduced mod n (used for marked vertices)."""
    return int(splitmix64(seed, 1)[0] % np.uint64(n))


# ----------------------------------------------------------------------------- graphs

def torus(L: int):
    """L x L torus, vertex v = x*L + y, edges to (x+1 mod L, y) and (x, y+1 mod L)."""
    if L < 3:
        raise ValueError("torus needs L >= 3")
    v = np.arange(L * L, dtype=np.int64)
    x, y = v // L, v % L
    right = ((x + 1) % L) * L + y
    up = x * L + (y + 1) % L
    return L * L, np.concatenate([v, v]), np.concatenate([right, up])


def torus_rect(L1: int, L2: int):
    """L1 x L2 torus, vertex v = x*L2 + y, edges to (x+1 mod L1, y) and (x, y+1 mod L2)."""
    if L1 < 3 or L2 < 3:
        raise ValueError("torus needs L1, L2 >= 3")
    v = np.arange(L1 * L2, dtype=np.int64)
    x, y = v // L2, v % L2
    down = ((x + 1) % L1) * L2 + y
    right = x * L2 + (y + 1) % L2
    return L1 * L2, np.concatenate([v, v]), np.concatenate([down, right])


def cycle(N: int):
    if N < 3:
        raise ValueError("cycle needs N >= 3")
    v = np.arange(N, dtype=np.int64)
    return N, v, (v + 1) % N


def path(N: int):
    v = np.arange(N - 1, dtype=np.int64)
    return N, v, v + 1


def star(N: int):
    """Vertex 0 joined to 1..N-1."""
    leaves = np.arange(1, N, dtype=np.int64)
    return N, np.zeros_like(leaves), leaves


def hypercube(k: int):
    """Q_k: vertices 0..2^k-1, v ~ v xor 2^j."""
    N = 1 << k
    v = np.arange(N, dtype=np.int64)
    eu, ev = [], []
    for j in range(k):
        w = v ^ (1 << j)
        keep = v < w
        eu.append(v[keep])
        ev.append(w[keep])
    return N, np.concatenate(eu), np.concatenate(ev)


def complete(N: int):
    iu, iv = np.triu_indices(N, 1)
    return N, iu.astype(np.int64), iv.astype(np.int64)


def _pair_from_index(k: np.ndarray):
    """Pairs (u, v), u < v, listed column by column: k -> v = largest with v(v-1)/2 <= k."""
    v = np.floor((1.0 + np.sqrt(1.0 + 8.0 * k.astype(np.float64))) / 2.0).astype(np.int64)
    # exact integer correction of the float estimate
    v -= (v * (v - 1) // 2 > k).astype(np.int64)
    v += ((v + 1) * v // 2 <= k).astype(np.int64)
    u = k - v * (v - 1) // 2
    return u, v


def erdos_renyi(n: int, p: float, seed: int, drop_isolated: bool = True):
    """G(n, p) by geometric skipping over the n(n-1)/2 pairs (V. Batagelj, U. Brandes,
    "Efficient generation of large random networks", Phys. Rev. E 71, 2005).

    Skip lengths floor(log(1-r)/log(1-p)) are drawn in order from SplitMix64(seed).
    With ``drop_isolated`` the degree-0 vertices are removed and the rest relabelled
    in ascending order of their original labels.
    """
    total = n * (n - 1) // 2
    lq = math.log1p(-p)
    pos_chunks = []
    last = -1
    drawn = 0
    chunk = max(1024, int(total * p * 1.02) + 1024)
    while True:
        m = chunk
        r = uniform01(seed, m, drawn)
        drawn += m
        skip = np.floor(np.log1p(-r) / lq).astype(np.int64)
        pos = last + np.cumsum(skip + 1)
        inside = pos < total
        pos_chunks.append(pos[inside])
        if not inside.all():
            break
        last = int(pos[-1])
    k = np.concatenate(pos_chunks)
    eu, ev = _pair_from_index(k)
    if drop_isolated:
        deg = np.bincount(eu, minlength=n) + np.bincount(ev, minlength=n)
        keep = deg > 0
        relabel = np.cumsum(keep) - 1
        eu, ev = relabel[eu], relabel[ev]
        n = int(keep.sum())
    return n, eu.astype(np.int64), ev.astype(np.int64)


def random_regular(n: int, d: int, seed: int):
    """Random simple d-regular graph: a random pairing of the n*d stubs (stubs put in
    the order of SplitMix64(seed) keys), then random double-edge switches that remove
    every self-loop and repeated edge."""
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    stubs = stubs[np.argsort(splitmix64(seed, stubs.size), kind="stable")]
    eu = stubs[0::2].copy()
    ev = stubs[1::2].copy()
    m = eu.size
    draw = m + 1
    for _ in range(100000):
        a, b = np.minimum(eu, ev), np.maximum(eu, ev)
        key = a * n + b
        order = np.argsort(key, kind="stable")
        dup = np.zeros(m, bool)
        sk = key[order]
        dup[order[1:]] = sk[1:] == sk[:-1]
        bad = np.flatnonzero((eu == ev) | dup)
        if bad.size == 0:
            break
        for e in bad:
            f = int(splitmix64(seed, 1, draw)[0] % np.uint64(m))
            draw += 1
            if f == e:
                continue
            # switch (eu[e], ev[e]), (eu[f], ev[f]) -> (eu[e], eu[f]), (ev[e], ev[f])
            ev[e], eu[f] = eu[f], ev[e]
    else:  # pragma: no cover
        raise RuntimeError("switch repair did not converge")
    return n, eu, ev


# ----------------------------------------------------------------------------- inputs

def degrees(n: int, eu: np.ndarray, ev: np.ndarray) -> np.ndarray:
    return np.bincount(eu, minlength=n) + np.bincount(ev, minlength=n)


def adjacency_csr(n: int, eu: np.ndarray, ev: np.ndarray, scramble_seed: int | None = 7):
    """CSR (row_ptr int64[n+1], col int32[2E]) of the symmetric 0/1 adjacency matrix.

    Each row's columns come in a seeded scrambled order (the library accepts any
    column order); ``scramble_seed=None`` keeps the generation order.
    """
    tails = np.concatenate([eu, ev])
    heads = np.concatenate([ev, eu])
    order = _row_order(tails, scramble_seed)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(tails, minlength=n), out=row_ptr[1:])
    return row_ptr, heads[order].astype(np.int32)


def _row_order(tails: np.ndarray, scramble_seed):
    """Permutation grouping the entries by tail; inside a row, the order of the
    top 32 bits of SplitMix64(scramble_seed) draws (ties by position), or the
    given order when scramble_seed is None.  One sort of a packed 64-bit key
    (tails < 2^31)."""
    if scramble_seed is None:
        return np.argsort(tails, kind="stable")
    key = (tails.astype(np.uint64) << np.uint64(32)) | (splitmix64(scramble_seed, tails.size) >> np.uint64(32))
    return np.argsort(key, kind="stable")


def edge_weights(count: int, seed: int, complex_phase: bool = False) -> np.ndarray:
    """One weight per edge: modulus uniform in [0.25, 1.75) and, with
    ``complex_phase``, a phase uniform in [0, 2 pi) (SplitMix64 draws)."""
    r = 0.25 + 1.5 * uniform01(seed, count)
    if not complex_phase:
        return r.astype(np.float64)
    ph = 2 * np.pi * uniform01(seed, count, offset=count)
    return r * np.exp(1j * ph)


def weighted_csr(n: int, eu: np.ndarray, ev: np.ndarray, we: np.ndarray, scramble_seed: int | None = 7):
    """``adjacency_csr`` plus the weight of each entry: entry (eu, ev) holds we and
    entry (ev, eu) its conjugate, so the matrix is Hermitian (symmetric for real we).
    Returns (row_ptr, col, w) with w complex128 or float64 like ``we``."""
    tails = np.concatenate([eu, ev])
    heads = np.concatenate([ev, eu])
    vals = np.concatenate([we, np.conj(we)])
    order = _row_order(tails, scramble_seed)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(tails, minlength=n), out=row_ptr[1:])
    return row_ptr, heads[order].astype(np.int32), vals[order]


def arc_offsets(n: int, eu: np.ndarray, ev: np.ndarray) -> np.ndarray:
    """Start of each vertex's arc block in the tail-major arc order: a prefix sum of
    degrees, int64[n+1] (independent of how heads are ordered inside a block)."""
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(degrees(n, eu, ev), out=off[1:])
    return off


def state_on_vertex_arcs(offsets: np.ndarray, v: int) -> np.ndarray:
    """Equal real amplitudes on the arcs of vertex v, unit norm, complex128."""
    a0, a1 = int(offsets[v]), int(offsets[v + 1])
    psi = np.zeros(int(offsets[-1]), dtype=np.complex128)
    psi[a0:a1] = 1.0 / math.sqrt(a1 - a0)
    return psi


def uniform_state(dim: int) -> np.ndarray:
    return np.full(dim, 1.0 / math.sqrt(dim), dtype=np.complex128)


def gaussian_states(dim: int, batch: int, seed: int) -> np.ndarray:
    """``batch`` unit complex Gaussian states, shape [dim, batch] (batch innermost).

    Stream order is column-major: column b uses draws b*dim .. b*dim+dim-1.  Each
    column is normalised in float64.
    """
    out = np.empty((dim, batch), dtype=np.complex128)
    for b in range(batch):
        z = complex_gaussian(seed, dim, b * dim)
        out[:, b] = z / np.sqrt(np.sum(np.abs(z) ** 2))
    return out


def gaussian_states_device(dim: int, batch: int, seed: int, dtype=None, device="cuda"):
    """``gaussian_states`` drawn on a torch device: the same SplitMix64 streams
    (bit-exact 64-bit integer arithmetic), Box-Muller and per-column
    normalisation in float64 with the device's math functions, then cast to
    ``dtype`` (default complex128).  The device's log, sqrt, sin and cos and its
    summation order may differ from the host's in the last bit, so columns
    agree with ``gaussian_states`` to a few float64 ulps, not bit for bit.
    Returns a [dim, batch] tensor (batch innermost), one column drawn at a time."""
    import torch
    dtype = torch.complex128 if dtype is None else dtype
    out = torch.empty((dim, batch), dtype=dtype, device=device)
    golden = _as_i64(0x9E3779B97F4A7C15)
    m1, m2 = _as_i64(0xBF58476D1CE4E5B9), _as_i64(0x94D049BB133111EB)
    s0 = _as_i64(seed & 0xFFFFFFFFFFFFFFFF)

    def lsr(z, k):   # logical right shift of 64-bit patterns held in int64
        return (z >> k) & ((1 << (64 - k)) - 1)

    for b in range(batch):
        k = torch.arange(2 * b * dim + 1, 2 * (b + 1) * dim + 1, dtype=torch.int64, device=device)
        z = s0 + k * golden                      # wraps mod 2^64 like the uint64 form
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        u = lsr(z, 11).to(torch.float64) * (2.0 ** -53)
        u1, u2 = u[0::2], u[1::2]
        r = torch.sqrt(-2.0 * torch.log1p(-u1))
        th = 2.0 * math.pi * u2
        col = torch.complex(r * torch.cos(th), r * torch.sin(th))
        col = col / torch.sqrt(torch.sum(col.real * col.real + col.imag * col.imag))
        out[:, b] = col.to(dtype)
    return out


def _as_i64(x: int) -> int:
    """The int64 value with the bit pattern of the unsigned 64-bit x."""
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >= (1 << 63) else x


def random_state(dim: int, seed: int) -> np.ndarray:
    return gaussian_states(dim, 1, seed)[:, 0]
