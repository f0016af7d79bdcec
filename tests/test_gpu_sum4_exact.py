"""One complex128 Grover step on the GPU, bit for bit against exact rational
arithmetic (Sec. 3.2: on a vertex of degree d the coin is (2/d) J - I, so
output j is (2/d) S - psi_j with S the sum of the vertex's d amplitudes, and
the flip-flop shift moves it to the reversed arc).

The kernels form S from groups of four arcs.  A group's sum is the exact sum
rounded once to the nearest double (ties to even) when its nonzero addends are
normal and lie within 8 binades of the largest and the result is normal; else
the sequential double sum.  A sum of zeros is -0 only when every addend is -0,
and an exact cancellation of nonzero addends is +0.  Degree 4 is one group;
degree 12 folds its three group sums by the same four-term rule; degree 17
adds its five group sums in order in double.  The output is (2/d) S - psi_j
rounded once (one FMA).

The states mix signs, signed zeros, exact cancellations and exponent spreads
on both sides of 8 binades, so the integer exact path, the fallback and the
zero rules all occur.  Run through the one-launch cluster kernel and the
per-step kernel on the torus, the register kernel on Q_12 and the two-pass
kernel on Q_17 (sampled vertices)."""
import struct
from fractions import Fraction

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _efield(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0] >> 52 & 0x7FF


def _neg(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0] >> 63 == 1


PATHS = {"zeros": 0, "fallback": 0, "cancel": 0, "exact": 0}


def _sum4(xs):
    xs = [float(x) for x in xs]
    nz = [x for x in xs if x != 0.0]
    if not nz:
        PATHS["zeros"] += 1
        return -0.0 if all(_neg(x) for x in xs) else 0.0
    es = [_efield(x) for x in nz]
    seq = ((xs[0] + xs[1]) + xs[2]) + xs[3]
    if max(es) == 0x7FF or min(es) == 0 or max(es) - min(es) > 8:
        PATHS["fallback"] += 1
        return seq
    exact = sum((Fraction(x) for x in xs), Fraction(0))
    if exact == 0:
        PATHS["cancel"] += 1
        return 0.0
    r = float(exact)
    if abs(r) < 2.2250738585072014e-308 or abs(r) == float("inf"):
        PATHS["fallback"] += 1
        return seq
    PATHS["exact"] += 1
    return r


def _groups(p):
    out = []
    for j0 in range(0, len(p), 4):
        g = list(p[j0:j0 + 4]) + [-0.0] * (4 - len(p[j0:j0 + 4]))
        out.append(_sum4(g))
    return out


def _vertex_sum(p, fold):
    g = _groups(p)
    if len(g) == 1:
        return g[0]
    if fold:   # up to four group sums rounded once more by the four-term rule
        return _sum4(g + [-0.0] * (4 - len(g)))
    s = g[0]
    for x in g[1:]:
        s = s + x
    return s


def _fma(f, s, p):
    return float(Fraction(f) * Fraction(s) - Fraction(p))


def _state(num_arcs, d, seed):
    """Amplitudes per vertex block: a base exponent, a spread (0..20 binades),
    random signs and mantissas, about 8% signed zeros, some vertices whose
    first two arcs cancel exactly, some whose first four do, and some that
    hold only signed zeros."""
    rng = np.random.default_rng(seed)
    n = num_arcs // d
    comps = []
    for _ in range(2):
        base = rng.integers(-30, 1, size=n)
        spread = rng.choice([0, 2, 8, 9, 20], size=n)
        e = base[:, None] - rng.integers(0, 21, size=(n, d)) % (spread[:, None] + 1)
        m = 1.0 + rng.random((n, d))
        x = np.ldexp(m, e) * rng.choice([-1.0, 1.0], size=(n, d))
        z = rng.random((n, d)) < 0.08
        x[z] = np.where(rng.random(z.sum()) < 0.5, 0.0, -0.0)
        c = rng.random(n) < 0.1
        x[c, 1] = -x[c, 0]
        if d >= 4:   # some vertices cancel to zero exactly, some hold only signed zeros
            c = rng.random(n) < 0.05
            x[c, 3] = -x[c, 2]
            x[c, 1] = -x[c, 0]
            zv = rng.random(n) < 0.03
            x[zv] = np.where(rng.random((zv.sum(), d)) < 0.5, 0.0, -0.0)
        comps.append(x.reshape(-1))
    return comps[0] + 1j * comps[1]


def _sorted_heads(g):
    n, eu, ev = g
    tails = np.concatenate([eu, ev])
    heads = np.concatenate([ev, eu])
    order = np.lexsort((heads, tails))
    return heads[order]


CASES = [
    ("torus64_cluster", synth.torus(64), 2, False, None),
    ("torus64_per_step", synth.torus(64), 1, False, None),
    ("Q12", synth.hypercube(12), 0, True, None),
    ("Q17", synth.hypercube(17), 0, False, 1500),
]


@pytest.mark.parametrize("name,g,mode,fold,sample", CASES)
def test_one_step_bit_exact(hw, name, g, mode, fold, sample):
    import torch
    n = g[0]
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    d = G.num_arcs // n
    heads = _sorted_heads(g)
    psi = _state(G.num_arcs, d, seed=29 + d)
    x = torch.from_numpy(psi).to("cuda", torch.complex128)
    y = torch.empty_like(x)
    hw.hw_coined_evolve(G, 0, [], 2, 1, 1, x, y, opts={"launch_mode": mode})
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    G.free()
    f = 2.0 / d
    rng = np.random.default_rng(5)
    verts = range(n) if sample is None else sorted(rng.choice(n, size=sample, replace=False))
    hv = heads.reshape(n, d)
    for k in PATHS:
        PATHS[k] = 0
    for v in verts:
        for comp in (0, 1):
            p = [(psi[v * d + j].real if comp == 0 else psi[v * d + j].imag) for j in range(d)]
            S = _vertex_sum(p, fold)
            for j in range(d):
                w = int(hv[v, j])
                r = w * d + int(np.searchsorted(hv[w], v))
                want = _fma(f, S, p[j])
                have = got[r].real if comp == 0 else got[r].imag
                assert struct.pack("<d", have) == struct.pack("<d", want), (name, v, comp, j, have, want)
    # every rule of the sum was exercised
    assert min(PATHS.values()) > 0, PATHS
    assert PATHS["exact"] > PATHS["fallback"] > 0, PATHS
