// Neighbour and arc positions of the two graph families that hw_graph_csr
// recognises (hw_graph_kind), computed from the vertex label instead of read
// from the head / reversal tables.  Arcs are sorted by head inside each
// vertex's block (Sec. 3.2), so "position" below is a rank among the vertex's
// neighbour labels.
//   torus L1 x L2 (L1, L2 >= 3):  v = x L2 + y, neighbours (x +- 1, y), (x, y +- 1)
//   hypercube Q_k:                v ~ v ^ 2^b, b = 0..k-1
#pragma once

#include <cstdint>

// Where the coin output of arc position j of vertex v goes in the edge-major
// layout (index j' n + w).  kAddrTable reads a table; the others compute it:
//   torus, flip-flop:   arc (v, w) -> (w, v)
//   torus, persistent:  arc (v, w) -> (w, w + (w - v))
//   hypercube:          arc (v, v ^ 2^b) -> (v ^ 2^b, v)
enum { kAddrTable = 0, kAddrTorusFF = 1, kAddrTorusPS = 2, kAddrCube = 3 };

// Position of direction dir (0 up = row x-1, 1 left = column y-1, 2 right,
// 3 down) in the sorted neighbour list of a torus vertex, from whether its row
// is the first (x0) or last (xl) and its column the first (y0) or last (yl).
// The position is the number of smaller neighbour labels, and each pairwise
// comparison is fixed by one flag when L1, L2 >= 3: up < left and up < right
// unless x0; left < down and right < down unless xl; up < down unless x0 or
// xl; left < right unless y0 or yl.
__device__ __forceinline__ int torus_rank(int dir, bool x0, bool xl, bool y0, bool yl)
{
    const int bu = !x0, bd = !xl, bud = !x0 && !xl, blr = !y0 && !yl;
    switch (dir) {
    case 0: return 2 * (1 - bu) + (1 - bud);
    case 1: return bu + (1 - blr) + (1 - bd);
    case 2: return bu + blr + (1 - bd);
    default: return bud + 2 * bd;
    }
}

struct TorusVertex {
    bool x0, xl, y0, yl;
    bool xs, xp, ys, yp;   // row is the second (x == 1) / the one before last; same for columns
    int w[4];              // neighbour labels by direction
    __device__ __forceinline__ TorusVertex(int64_t v, int64_t n, int L1, int L2)
    {
        const uint32_t x = uint32_t(v) / uint32_t(L2);
        init(x, uint32_t(v) - x * uint32_t(L2), n, L1, L2);
    }
    // from the coordinates (v = x L2 + y), e.g. a launch with a block row per torus row
    __device__ __forceinline__ TorusVertex(uint32_t x, uint32_t y, int64_t n, int L1, int L2) { init(x, y, n, L1, L2); }
    __device__ __forceinline__ void init(uint32_t x, uint32_t y, int64_t n, int L1, int L2)
    {
        x0 = x == 0;
        xl = x == uint32_t(L1 - 1);
        y0 = y == 0;
        yl = y == uint32_t(L2 - 1);
        xs = x == 1;
        xp = x == uint32_t(L1 - 2);
        ys = y == 1;
        yp = y == uint32_t(L2 - 2);
        const int sv = int(x * uint32_t(L2) + y), sn = int(n);
        w[0] = x0 ? sv + (sn - L2) : sv - L2;
        w[1] = y0 ? sv + (L2 - 1) : sv - 1;
        w[2] = yl ? sv - (L2 - 1) : sv + 1;
        w[3] = xl ? sv - (sn - L2) : sv + L2;
    }
    __device__ __forceinline__ int pos(int dir) const { return torus_rank(dir, x0, xl, y0, yl); }
    // position of direction dir2 in the list of the neighbour in direction k:
    // up is on row x - 1, down on x + 1, left on column y - 1, right on y + 1
    __device__ __forceinline__ int nbr_pos(int k, int dir2) const
    {
        switch (k) {
        case 0: return torus_rank(dir2, xs, x0, y0, yl);
        case 1: return torus_rank(dir2, x0, xl, ys, y0);
        case 2: return torus_rank(dir2, x0, xl, yl, yp);
        default: return torus_rank(dir2, xl, xp, y0, yl);
        }
    }
    // v and its neighbours are off the first and last rows and columns: the
    // ascending order is up, left, right, down everywhere around v
    __device__ __forceinline__ bool deep_interior() const { return !(x0 || xl || y0 || yl || xs || xp || ys || yp); }
    // neighbour labels in ascending order
    __device__ __forceinline__ void sorted(int s[4]) const
    {
        if (!(x0 || xl || y0 || yl)) {
#pragma unroll
            for (int j = 0; j < 4; ++j) s[j] = w[j];
            return;
        }
        int p[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = pos(k);
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] = (p[0] == j) ? w[0] : (p[1] == j) ? w[1] : (p[2] == j) ? w[2] : w[3];
    }
};

// r[j] for the four arc positions of torus vertex tv
template <int ADDR>
__device__ __forceinline__ void torus_targets(const TorusVertex &tv, int64_t n, int r[4])
{
    const int sn = int(n);
    if (tv.deep_interior()) {
        // positions up 0, left 1, right 2, down 3 at v and at every neighbour
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = ((ADDR == kAddrTorusFF) ? 3 - k : k) * sn + tv.w[k];
        return;
    }
    int p[4], t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        p[k] = tv.pos(k);
        // flip-flop: v is the neighbour's opposite direction; persistent: the
        // walker leaves the neighbour in direction k again
        t[k] = tv.nbr_pos(k, (ADDR == kAddrTorusFF) ? 3 - k : k) * sn + tv.w[k];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = (p[0] == j) ? t[0] : (p[1] == j) ? t[1] : (p[2] == j) ? t[2] : t[3];
}

// Hypercube Q_k: the sorted neighbours of v are v - 2^b for the set bits b of
// v, highest first, then v + 2^b for the clear bits, lowest first.  The walk
// visits the positions j = 0, 1, ...: next_bit() gives the bit of position j;
// target() the edge-major index of the reversed arc (w, v), w = v ^ 2^b, which
// sits in w's list at the number of set bits of w above b when bit b of w is
// set, else after w's popc(w) set bits at the number of clear bits of w below b.
struct CubeWalk {
    uint32_t v, set, clr;
    int pc, j;
    __device__ __forceinline__ CubeWalk(int64_t v_, int k)
    {
        v = uint32_t(v_);
        set = v;
        clr = ~v & ((1u << k) - 1u);
        pc = __popc(v);
        j = 0;
    }
    __device__ __forceinline__ int next_bit()
    {
        int b;
        if (j < pc) {
            b = 31 - __clz(set);
            set ^= 1u << b;
        } else {
            b = __ffs(clr) - 1;
            clr &= clr - 1u;
        }
        ++j;
        return b;
    }
    // the same positions from the last one down: position d - 1 first
    // (clear bits highest first, then set bits lowest first); a walk uses
    // either next_bit or prev_bit, not both
    __device__ __forceinline__ int prev_bit()
    {
        int b;
        if (clr) {
            b = 31 - __clz(clr);
            clr ^= 1u << b;
        } else {
            b = __ffs(set) - 1;
            set &= set - 1u;
        }
        return b;
    }
    __device__ __forceinline__ int target(int b, int64_t n) const
    {
        const int rpos = ((v >> b) & 1u) ? (pc - 1) + b - __popc(v & ((1u << b) - 1u)) : __popc(v >> (b + 1));
        return rpos * int(n) + int(v ^ (1u << b));
    }
};
