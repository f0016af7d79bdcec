/*
 * Oracle for quantum-walk evolution on graphs, after Motta, Bezerra, Santos,
 * Portugal, "Hiperwalk: Simulation of Quantum Walks with Heterogeneous
 * High-Performance Computing" (arXiv 2406.08186), Sec. 3.1 and Sec. 3.2.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 restatement of
 * the paper's definitions.  It is used by the tests, by the bench's CPU
 * baseline and by the package's smoke check; the product path never calls it.
 * It shares no code, header or table with the CUDA library.
 *
 * Conventions
 *   - complex amplitudes are C99 `double complex` (layout: re, im interleaved)
 *   - arcs (v, w) with tail v and head w are ordered by tail, then by head
 *     (Sec. 3.2, computational basis of the coined walk); row_ptr[v] is the
 *     index of the first arc with tail v
 *   - OpenMP only splits independent outer loops (vertices or arcs); every
 *     output element is computed by one thread in the order written here.
 *
 * Parity status: every function below is pinned by the tests in
 * tests/test_oracle_*.py (brute force, closed forms, invariants).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORACLE_GROVER = 0, ORACLE_FOURIER = 1 };

int oracle_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------ arcs */

typedef struct { int64_t tail, head; } arc_t;

static int arc_cmp(const void *pa, const void *pb)
{
    const arc_t *a = pa, *b = pb;
    if (a->tail != b->tail) return a->tail < b->tail ? -1 : 1;
    if (a->head != b->head) return a->head < b->head ? -1 : 1;
    return 0;
}

/* Position of arc (tail, head) in the sorted arc list, or -1 (bisection over
 * the whole list, compared lexicographically). */
static int64_t find_arc(const arc_t *arcs, int64_t num, int64_t tail, int64_t head)
{
    arc_t key = { tail, head };
    int64_t lo = 0, hi = num;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = arc_cmp(&arcs[mid], &key);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -1;
}

/*
 * Computational basis of the coined walk (Sec. 3.2): every undirected edge
 * {u, v} gives the two arcs (u, v) and (v, u); arcs are sorted by tail, then
 * head.  Outputs row_ptr[n+1], head[2E] and rev[2E], where rev[a] is the
 * position of the reversed arc, i.e. the index form of the flip-flop shift
 * S|v,w> = |w,v>.
 * Returns 0, or -1 (vertex id out of range), -2 (self-loop), -3 (repeated edge).
 */
int oracle_build_arcs(int64_t n, int64_t n_edges, const int64_t *eu, const int64_t *ev,
                      int64_t *row_ptr, int32_t *head, int64_t *rev)
{
    int64_t num = 2 * n_edges;
    arc_t *arcs = malloc(sizeof(arc_t) * (size_t)(num > 0 ? num : 1));
    if (!arcs) return -4;
    for (int64_t e = 0; e < n_edges; ++e) {
        if (eu[e] < 0 || eu[e] >= n || ev[e] < 0 || ev[e] >= n) { free(arcs); return -1; }
        if (eu[e] == ev[e]) { free(arcs); return -2; }
        arcs[2 * e].tail = eu[e];     arcs[2 * e].head = ev[e];
        arcs[2 * e + 1].tail = ev[e]; arcs[2 * e + 1].head = eu[e];
    }
    qsort(arcs, (size_t)num, sizeof(arc_t), arc_cmp);
    for (int64_t a = 1; a < num; ++a)
        if (arc_cmp(&arcs[a - 1], &arcs[a]) == 0) { free(arcs); return -3; }
    for (int64_t v = 0; v <= n; ++v) row_ptr[v] = 0;
    for (int64_t a = 0; a < num; ++a) row_ptr[arcs[a].tail + 1] += 1;
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    for (int64_t a = 0; a < num; ++a) {
        head[a] = (int32_t)arcs[a].head;
        rev[a] = find_arc(arcs, num, arcs[a].head, arcs[a].tail);
    }
    free(arcs);
    return 0;
}

/* ------------------------------------------------------------ coined walk */

/*
 * The coin C, block-diagonal with one d(v) x d(v) block per vertex (Sec. 3.2).
 * Inside the block of v, j and k index v's arcs in basis order.
 *   Grover  (Sec. 3.2):  C[j][k] = 2/d(v) - delta_jk
 *   Fourier:             C[j][k] = omega^(j*k) / sqrt(d(v)),  omega = exp(2 pi i / d(v))
 *   marked vertex (search oracle):  C[j][k] = -delta_jk
 * out = C psi, evaluated as the full row sum for every j (O(d^2) per vertex).
 */
void oracle_coin(int64_t n, const int64_t *row_ptr, int coin, const uint8_t *marked,
                 const cplx *psi, cplx *out)
{
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t v = 0; v < n; ++v) {
        int64_t s = row_ptr[v];
        int64_t d = row_ptr[v + 1] - s;
        for (int64_t j = 0; j < d; ++j) {
            cplx acc = 0.0;
            for (int64_t k = 0; k < d; ++k) {
                cplx c;
                if (marked && marked[v]) {
                    c = (j == k) ? -1.0 : 0.0;
                } else if (coin == ORACLE_GROVER) {
                    c = 2.0 / (double)d - ((j == k) ? 1.0 : 0.0);
                } else {
                    int64_t r = (j * k) % d;
                    double ang = 2.0 * M_PI * (double)r / (double)d;
                    c = (cos(ang) + I * sin(ang)) / sqrt((double)d);
                }
                acc += c * psi[s + k];
            }
            out[s + j] = acc;
        }
    }
}

/* Position of arc (tail, hd) inside tail's block, by bisection over its heads. */
static int64_t arc_in_row(const int64_t *row_ptr, const int32_t *head, int64_t tail, int64_t hd)
{
    int64_t lo = row_ptr[tail], hi = row_ptr[tail + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (head[mid] == hd) return mid;
        if (head[mid] < hd) lo = mid + 1; else hi = mid;
    }
    return -1;
}

/* Flip-flop shift S|v,w> = |w,v> (Sec. 3.2): the amplitude of arc (v, w) moves to
 * arc (w, v), located by searching head v in row w. */
void oracle_shift(int64_t n, const int64_t *row_ptr, const int32_t *head, const cplx *psi,
                  cplx *out)
{
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
            int64_t b = arc_in_row(row_ptr, head, head[a], v);
            out[b] = psi[a];
        }
    }
}

/* Persistent shift on the L1 x L2 torus (Sec. 3.2: the persistent shift that
 * the Grid class offers, where the walker keeps its direction): the amplitude
 * of arc (v, w) moves to arc (w, u), u being one more step from w in the
 * direction that led from v to w.  Vertex v = x L2 + y; the direction is the
 * difference of coordinates modulo L1 and L2 (L1, L2 >= 3, so it is one of
 * +-1 along exactly one axis). */
void oracle_shift_persistent_torus(int64_t L1, int64_t L2, const int64_t *row_ptr, const int32_t *head,
                                   const cplx *psi, cplx *out)
{
    int64_t n = L1 * L2;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t v = 0; v < n; ++v) {
        int64_t xv = v / L2, yv = v % L2;
        for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
            int64_t w = head[a];
            int64_t xw = w / L2, yw = w % L2;
            int64_t dx = (xw - xv + L1) % L1, dy = (yw - yv + L2) % L2;
            int64_t u = ((xw + dx) % L1) * L2 + (yw + dy) % L2;
            int64_t b = arc_in_row(row_ptr, head, w, u);
            out[b] = psi[a];
        }
    }
}

/* p_v = sum over arcs (v, w) of |<v,w|psi>|^2 (Sec. 3.2). */
void oracle_prob_coined(int64_t n, const int64_t *row_ptr, const cplx *psi, double *p)
{
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        double acc = 0.0;
        for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            acc += creal(psi[a]) * creal(psi[a]) + cimag(psi[a]) * cimag(psi[a]);
        p[v] = acc;
    }
}

static double marked_prob_coined(int64_t n, const int64_t *row_ptr, const uint8_t *marked,
                                 const cplx *psi)
{
    double acc = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        if (!marked[v]) continue;
        for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            acc += creal(psi[a]) * creal(psi[a]) + cimag(psi[a]) * cimag(psi[a]);
    }
    return acc;
}

/*
 * |psi(t)> = (S C)^t |psi(0)> (Sec. 3.2): each step applies the coin, then the
 * shift: the flip-flop shift when L1 == 0, else the persistent shift of the
 * L1 x L2 torus.  psi holds |psi(0)> on entry and |psi(steps)> on exit.  If
 * record is not NULL and marked is not NULL, record[t-1] receives the total
 * probability on the marked vertices after step t.  Returns 0 or -4 (out of
 * memory).
 */
static int coined_loop(int64_t n, const int64_t *row_ptr, const int32_t *head, int coin,
                       const uint8_t *marked, cplx *psi, int64_t steps, double *record,
                       int64_t L1, int64_t L2)
{
    int64_t num = row_ptr[n];
    cplx *tmp = malloc(sizeof(cplx) * (size_t)(num > 0 ? num : 1));
    if (!tmp) return -4;
    for (int64_t t = 1; t <= steps; ++t) {
        oracle_coin(n, row_ptr, coin, marked, psi, tmp);
        if (L1 == 0)
            oracle_shift(n, row_ptr, head, tmp, psi);
        else
            oracle_shift_persistent_torus(L1, L2, row_ptr, head, tmp, psi);
        if (record && marked) record[t - 1] = marked_prob_coined(n, row_ptr, marked, psi);
    }
    free(tmp);
    return 0;
}

int oracle_coined_evolve(int64_t n, const int64_t *row_ptr, const int32_t *head, int coin,
                         const uint8_t *marked, cplx *psi, int64_t steps, double *record)
{
    return coined_loop(n, row_ptr, head, coin, marked, psi, steps, record, 0, 0);
}

/* The same evolution with the persistent shift of the L1 x L2 torus. */
int oracle_coined_evolve_persistent_torus(int64_t L1, int64_t L2, const int64_t *row_ptr,
                                          const int32_t *head, int coin, const uint8_t *marked,
                                          cplx *psi, int64_t steps, double *record)
{
    return coined_loop(L1 * L2, row_ptr, head, coin, marked, psi, steps, record, L1, L2);
}

/* ------------------------------------------------------------ CTQW (Sec. 3.1) */

/* y = H x with H = -gamma W - sum_{m in M} |m><m| (Sec. 3.1, with the adjacency
 * A generalised to a weighted one): W = A when w is NULL, else row v of W holds
 * w[a] at column head[a] for each arc a of v (for a Hermitian W, arc (u, v)
 * carries the conjugate of arc (v, u)'s weight). */
static void ham_apply(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                      const uint8_t *marked, const cplx *w, const cplx *x, cplx *y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        cplx acc = 0.0;
        for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) acc += (w ? w[a] : 1.0) * x[head[a]];
        acc = -gamma * acc;
        if (marked && marked[v]) acc -= x[v];
        y[v] = acc;
    }
}

/*
 * psi <- exp(-i H dt) psi (Sec. 3.1, U(t) = e^{-iHt}) by the exponential series
 * sum_k (-i dt)^k H^k psi / k!.  To keep the series well conditioned, dt is cut
 * into q equal parts with ||H dt/q||_inf <= 1/2 (exact: e^{-iHdt} = (e^{-iHdt/q})^q);
 * each part sums terms until the latest one has max-abs below 1e-18.
 * work: 2n complex.  Returns the total number of series terms used.
 */
static int64_t ctqw_apply(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                          const uint8_t *marked, const cplx *w, double dt, cplx *psi, cplx *work)
{
    double hnorm = 0.0;                       /* max row sum of |H| */
    for (int64_t v = 0; v < n; ++v) {
        double rw = 0.0;
        for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) rw += w ? cabs(w[a]) : 1.0;
        double r = fabs(gamma) * rw;
        if (marked && marked[v]) r += 1.0;
        if (r > hnorm) hnorm = r;
    }
    int64_t q = (int64_t)ceil(hnorm * fabs(dt) / 0.5);
    if (q < 1) q = 1;
    double tau = dt / (double)q;
    cplx *term = work, *next = work + n;
    int64_t used = 0;
    for (int64_t r = 0; r < q; ++r) {
        memcpy(term, psi, sizeof(cplx) * (size_t)n);
        for (int k = 1; k <= 200; ++k) {
            ham_apply(n, row_ptr, head, gamma, marked, w, term, next);
            double mx = 0.0;
            cplx f = -I * tau / (double)k;
            for (int64_t v = 0; v < n; ++v) {
                next[v] *= f;
                psi[v] += next[v];
                double m = cabs(next[v]);
                if (m > mx) mx = m;
            }
            cplx *sw = term; term = next; next = sw;
            ++used;
            if (mx < 1e-18) break;
        }
        term = work; next = work + n;
    }
    return used;
}

/*
 * |psi(k dt)> = U(dt)^k |psi(0)>, k = 1..steps (Sec. 3.1).  psi: |psi(0)> in,
 * |psi(steps dt)> out.  record[k-1] (if not NULL) = total probability on the
 * marked vertices at time k dt.  Returns 0 or -4.
 */
int oracle_ctqw_evolve_w(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                         const uint8_t *marked, const cplx *w, double dt, cplx *psi, int64_t steps,
                         double *record)
{
    cplx *work = malloc(sizeof(cplx) * (size_t)(2 * (n > 0 ? n : 1)));
    if (!work) return -4;
    for (int64_t k = 1; k <= steps; ++k) {
        ctqw_apply(n, row_ptr, head, gamma, marked, w, dt, psi, work);
        if (record) {
            double acc = 0.0;
            for (int64_t v = 0; v < n; ++v)
                if (marked && marked[v]) acc += creal(psi[v]) * creal(psi[v]) + cimag(psi[v]) * cimag(psi[v]);
            record[k - 1] = acc;
        }
    }
    free(work);
    return 0;
}

int oracle_ctqw_evolve(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                       const uint8_t *marked, double dt, cplx *psi, int64_t steps,
                       double *record)
{
    return oracle_ctqw_evolve_w(n, row_ptr, head, gamma, marked, NULL, dt, psi, steps, record);
}

/* Columns U(dt) e_j of the evolution operator for the listed j (ncols of them):
 * out is row-major [ncols][n], out[c][i] = U[i][cols[c]].  w as in ham_apply.
 * Returns 0 or -4. */
int oracle_ctqw_columns_w(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                          const uint8_t *marked, const cplx *w, double dt, const int64_t *cols,
                          int64_t ncols, cplx *out)
{
    cplx *work = malloc(sizeof(cplx) * (size_t)(2 * (n > 0 ? n : 1)));
    if (!work) return -4;
    for (int64_t c = 0; c < ncols; ++c) {
        cplx *col = out + c * n;
        for (int64_t v = 0; v < n; ++v) col[v] = 0.0;
        col[cols[c]] = 1.0;
        ctqw_apply(n, row_ptr, head, gamma, marked, w, dt, col, work);
    }
    free(work);
    return 0;
}

int oracle_ctqw_columns(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                        const uint8_t *marked, double dt, const int64_t *cols, int64_t ncols,
                        cplx *out)
{
    return oracle_ctqw_columns_w(n, row_ptr, head, gamma, marked, NULL, dt, cols, ncols, out);
}

/* U(dt) x for one vector x (in place).  Returns the number of series terms. */
int64_t oracle_ctqw_action(int64_t n, const int64_t *row_ptr, const int32_t *head, double gamma,
                           const uint8_t *marked, double dt, cplx *x)
{
    cplx *work = malloc(sizeof(cplx) * (size_t)(2 * (n > 0 ? n : 1)));
    if (!work) return -4;
    int64_t used = ctqw_apply(n, row_ptr, head, gamma, marked, NULL, dt, x, work);
    free(work);
    return used;
}

/* Weights of the arcs of an edge list in basis order: edge e = {eu[e], ev[e]}
 * with value we[e] gives arc (eu, ev) the weight we[e] and arc (ev, eu) its
 * conjugate (a Hermitian W; a real we gives a symmetric one).  Arcs are found
 * by bisection in their rows.  Returns 0, or -1 when an edge has no arc. */
int oracle_arc_weights(int64_t n, const int64_t *row_ptr, const int32_t *head, int64_t n_edges,
                       const int64_t *eu, const int64_t *ev, const cplx *we, cplx *w_arc)
{
    (void)n;
    for (int64_t e = 0; e < n_edges; ++e) {
        int64_t a = arc_in_row(row_ptr, head, eu[e], ev[e]);
        int64_t b = arc_in_row(row_ptr, head, ev[e], eu[e]);
        if (a < 0 || b < 0) return -1;
        w_arc[a] = we[e];
        w_arc[b] = conj(we[e]);
    }
    return 0;
}

/* |<v|psi>|^2 (Sec. 3.1). */
void oracle_prob_vertex(int64_t n, const cplx *psi, double *p)
{
    for (int64_t v = 0; v < n; ++v)
        p[v] = creal(psi[v]) * creal(psi[v]) + cimag(psi[v]) * cimag(psi[v]);
}
