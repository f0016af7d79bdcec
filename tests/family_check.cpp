// Checks the label arithmetic of the index-free kernels (family.cuh) on the
// host against brute force: for tori L1 x L2 and hypercubes Q_k, each
// vertex's neighbours are sorted by label, and the edge-major index of the
// flip-flop target (w, v) and of the persistent target (w, 2w - v) is found by
// searching w's sorted list; the hypercube walk is also checked in reverse.  The device intrinsics are given host
// definitions with the same meaning.  Prints "ok <count>" or the first
// mismatch; exits non-zero on a mismatch.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#define __device__
#define __forceinline__ inline
static inline int __popc(uint32_t x) { return __builtin_popcount(x); }
static inline int __clz(int x) { return x ? __builtin_clz(uint32_t(x)) : 32; }
static inline int __ffs(int x) { return __builtin_ffs(x); }

#include "family.cuh"

static long checked = 0;

static int pos_in(const std::vector<int> &row, int w)
{
    return int(std::find(row.begin(), row.end(), w) - row.begin());
}

static bool check_torus(int L1, int L2)
{
    const int n = L1 * L2;
    std::vector<std::vector<int>> nb(n);
    for (int v = 0; v < n; ++v) {
        const int x = v / L2, y = v % L2;
        nb[v] = {((x + L1 - 1) % L1) * L2 + y, x * L2 + (y + L2 - 1) % L2, x * L2 + (y + 1) % L2,
                 ((x + 1) % L1) * L2 + y};
        std::sort(nb[v].begin(), nb[v].end());
    }
    for (int v = 0; v < n; ++v) {
        int ff[4], ps[4], srt[4];
        torus_targets<kAddrTorusFF>(TorusVertex(int64_t(v), n, L1, L2), n, ff);
        // the coordinate form (launches with a block row per torus row)
        torus_targets<kAddrTorusPS>(TorusVertex(uint32_t(v / L2), uint32_t(v % L2), n, L1, L2), n, ps);
        TorusVertex(int64_t(v), n, L1, L2).sorted(srt);
        const int xv = v / L2, yv = v % L2;
        for (int j = 0; j < 4; ++j) {
            ++checked;
            const int w = nb[v][j], xw = w / L2, yw = w % L2;
            const int u = ((2 * xw - xv + 2 * L1) % L1) * L2 + (2 * yw - yv + 2 * L2) % L2;
            const int want_ff = pos_in(nb[w], v) * n + w, want_ps = pos_in(nb[w], u) * n + w;
            if (srt[j] != w || ff[j] != want_ff || ps[j] != want_ps) {
                std::printf("torus %dx%d v=%d j=%d: sorted %d/%d ff %d/%d ps %d/%d\n", L1, L2, v, j, srt[j], w,
                            ff[j], want_ff, ps[j], want_ps);
                return false;
            }
        }
    }
    return true;
}

static bool check_cube(int k)
{
    const int n = 1 << k;
    std::vector<std::vector<int>> nb(n);
    for (int v = 0; v < n; ++v) {
        for (int b = 0; b < k; ++b) nb[v].push_back(v ^ (1 << b));
        std::sort(nb[v].begin(), nb[v].end());
    }
    for (int v = 0; v < n; ++v) {
        CubeWalk cw(v, k);
        for (int j = 0; j < k; ++j) {
            ++checked;
            const int b = cw.next_bit();
            const int w = nb[v][j];
            const int want = pos_in(nb[w], v) * n + w;
            if ((v ^ (1 << b)) != w || cw.target(b, n) != want) {
                std::printf("cube k=%d v=%d j=%d: bit %d (w %d/%d) target %d/%d\n", k, v, j, b, v ^ (1 << b), w,
                            cw.target(b, n), want);
                return false;
            }
        }
        // the reverse walk visits the same positions from the last one down
        CubeWalk rw(v, k);
        for (int j = k - 1; j >= 0; --j) {
            ++checked;
            const int b = rw.prev_bit();
            if ((v ^ (1 << b)) != nb[v][j]) {
                std::printf("cube k=%d v=%d reverse position %d: bit %d (w %d/%d)\n", k, v, j, b, v ^ (1 << b),
                            nb[v][j]);
                return false;
            }
        }
    }
    return true;
}

int main()
{
    for (int L1 = 3; L1 <= 12; ++L1)
        for (int L2 = 3; L2 <= 12; ++L2)
            if (!check_torus(L1, L2)) return 1;
    if (!check_torus(64, 64) || !check_torus(3, 1000) || !check_torus(1000, 3) || !check_torus(31, 33)) return 1;
    for (int k = 1; k <= 16; ++k)
        if (!check_cube(k)) return 1;
    std::printf("ok %ld\n", checked);
    return 0;
}
