/*
 * Sequential CPU oracle of Fox / LazyFox overlapping community detection
 * (Garrels, Khodabakhsh, Renard, Baum: "LazyFox: Fast and parallelized
 * overlapping community detection in large graphs", arXiv 2210.03211).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no
 * code, header, table or helper with it.
 *
 * Plain, slow and sequential on purpose: every step is written the obvious
 * way, in the order the paper describes it, so that it can be checked against
 * the paper by eye.  FP64 throughout; build with -O2 -ffp-contract=off so
 * that no multiply-add is fused (the CUDA path evaluates the same expressions
 * with explicitly rounded operations, so the two agree bit for bit).
 *
 * Readings of passages the paper leaves open:
 *   - self-loops are dropped; nodes are the endpoints of the remaining edges
 *     (Preprocessing, "Remove Multi-Edges" / "Dense Node Labels");
 *   - node order: clustering coefficient descending compared as exact
 *     rationals, then degree descending, then dense id ascending (Node Order);
 *   - cc = correctly rounded sum of the rounded local CCs over all n nodes,
 *     divided by n (Heuristic Counting of Triangles, global cc);
 *   - the gain of a join or leave is, as the paper defines it (Node Changes:
 *     Joining / Leaving a Community), the improvement of \wcchat(P') over
 *     \wcchat(P), the sums of the per-node estimator over all memberships
 *     (\wcchat, sum equations): the moved community's members' terms after
 *     the move (new size, new internal edge count, and for x's neighbours
 *     their deg(y,C) changed by one) and x's own term, less the same
 *     community's terms before it, added with the correctly rounded sum
 *     (OG_GAIN_LITERAL, the default).  A departure kept as an option
 *     (OG_GAIN_MEANFIELD):
 *     the change of the community's mean-field score S(n, m, vol), every
 *     member given the mean internal degree 2m/n and mean total degree vol/n;
 *   - B(z) = C(z,2) for z >= 1, else 0;
 *   - "positive improvement" is strictly > 0; ties go to the lowest id;
 *   - a node may both leave and join in one step (leave applied first) and
 *     may end with no community;
 *   - communities with < 2 members are removed after every iteration,
 *     before the iteration's total is taken (Post-processing);
 *   - stop when (T_it - T_prev) / T_prev < threshold; if T_prev == 0, stop
 *     iff T_it == 0 (Stopping Criteria).
 *
 * Parity pins: see tests/test_oracle_*.py; whole runs on tiny graphs are
 * compared with an exact-rational brute force.  Whole runs on graphs beyond
 * brute-force size have no external reference (the paper prints no
 * intermediate values), so that part is "parity unpinned" beyond the
 * invariants, closed forms and brute-force checks in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_OK 0
#define OG_ERR_INVALID 1
#define OG_ERR_OOM 2
#define OG_ERR_STATE 6

/* decision rule of a move (see the readings above) */
#define OG_GAIN_LITERAL 0
#define OG_GAIN_MEANFIELD 1

typedef struct og_graph {
    int64_t n, m;          /* nodes, undirected simple edges */
    int32_t *labels;       /* dense id -> original id (ascending) */
    int64_t *off;          /* n+1 row offsets into adj */
    int32_t *adj;          /* 2m neighbours, each row ascending */
    int have_tri;
    int64_t *t;            /* triangles containing each node */
    int32_t *vt;           /* neighbours that share a triangle with the node */
    int32_t *order;        /* processing order (dense ids) */
    double cc;             /* global clustering coefficient */
    /* community state */
    int64_t ncomm;         /* community ids allocated: 0..ncomm-1 */
    int64_t *cn, *cm, *cvol; /* members, internal edges, sum of member degrees */
    int32_t **mem;         /* per node: ascending community ids */
    int32_t *nmem, *capmem;
    int32_t **kin;         /* per node, beside mem: deg(x,C) = |N(x) & C| of each membership */
    int32_t **cmem;        /* per community: ascending member ids (the same memberships) */
    int32_t *ncmem, *capcmem;
    int gain_rule;         /* OG_GAIN_LITERAL or OG_GAIN_MEANFIELD */
    /* last run */
    int32_t iterations;
    int32_t converged;
    double T0;
    double *T_hist;
    double *S_hist;        /* diagnostic: sum of the mean-field community scores per iteration */
    int64_t *joins_hist, *leaves_hist;
    int32_t hist_cap;
    int check_invariants;  /* recount aggregates after every batch */
    int invariant_failures;
    /* an inserted division replacing the initial clustering (Methods,
     * Initial Clustering): community c holds part_mem[part_off[c] .. part_off[c+1])
     * (dense ids); part_k < 0 = none */
    int64_t part_k;
    int64_t *part_off;
    int32_t *part_mem;
    /* diagnostic of the gain reading (off by default): during og_run, every
     * evaluated node's decision is also taken with the literal gains and the
     * two are compared; see og_set_literal_diagnostic */
    int literal_diag;
    int64_t diag[8];
} og_graph;

/* ------------------------------------------------------------------------ */
/* Correctly rounded sum (Shewchuk, "Adaptive Precision Floating-Point       */
/* Arithmetic and Fast Robust Geometric Predicates", 1997): keep a list of   */
/* non-overlapping partial sums, each addition done error-free with the      */
/* two-sum; at the end add the partials from the largest down and fix the    */
/* one case where the last rounding lands exactly half-way.                  */
/* ------------------------------------------------------------------------ */
double og_fsum(const double *x, int64_t count)
{
    int64_t cap = 64, np = 0;
    double *p = (double *)malloc((size_t)cap * sizeof(double));
    if (!p) return NAN;
    for (int64_t k = 0; k < count; ++k) {
        double v = x[k];
        int64_t i = 0;
        for (int64_t j = 0; j < np; ++j) {
            double y = p[j];
            if (fabs(v) < fabs(y)) { double tmp = v; v = y; y = tmp; }
            double hi = v + y;
            double lo = y - (hi - v);
            if (lo != 0.0) p[i++] = lo;
            v = hi;
        }
        if (i >= cap) {
            cap *= 2;
            double *q = (double *)realloc(p, (size_t)cap * sizeof(double));
            if (!q) { free(p); return NAN; }
            p = q;
        }
        p[i++] = v;
        np = i;
    }
    double hi = 0.0;
    if (np > 0) {
        int64_t k = np - 1;
        double lo = 0.0;
        hi = p[k];
        while (k > 0) {
            double a = hi;
            double b = p[--k];
            hi = a + b;
            double br = hi - a;
            lo = b - br;
            if (lo != 0.0) break;
        }
        if (k > 0 && ((lo < 0.0 && p[k - 1] < 0.0) || (lo > 0.0 && p[k - 1] > 0.0))) {
            double b = lo * 2.0;
            double a = hi + b;
            double br = a - hi;
            if (b == br) hi = a;
        }
    }
    free(p);
    return hi;
}

/* ------------------------------------------------------------------------ */
/* Preprocessing: remove multi-edges (and self-loops), dense node labels.    */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int32_t dense_id(const int32_t *labels, int64_t n, int32_t id)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (labels[mid] == id) return (int32_t)mid;
        if (labels[mid] < id) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

void og_destroy(og_graph *g);

og_graph *og_create(const int32_t *src, const int32_t *dst, int64_t num_edges, int *status)
{
    *status = OG_OK;
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    if (!g) { *status = OG_ERR_OOM; return NULL; }
    g->part_k = -1;
    g->gain_rule = OG_GAIN_LITERAL;
    for (int64_t e = 0; e < num_edges; ++e) {
        if (src[e] < 0 || dst[e] < 0) { *status = OG_ERR_INVALID; free(g); return NULL; }
    }
    /* each undirected pair once as (min, max); self-loops dropped */
    uint64_t *key = (uint64_t *)malloc((size_t)(num_edges > 0 ? num_edges : 1) * sizeof(uint64_t));
    int64_t k = 0;
    for (int64_t e = 0; e < num_edges; ++e) {
        uint32_t a = (uint32_t)src[e], b = (uint32_t)dst[e];
        if (a == b) continue;
        uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
        key[k++] = ((uint64_t)lo << 32) | hi;
    }
    qsort(key, (size_t)k, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t i = 0; i < k; ++i)
        if (i == 0 || key[i] != key[i - 1]) key[m++] = key[i];
    /* dense labels: the sorted distinct endpoint ids */
    int32_t *ids = (int32_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) {
        ids[2 * i] = (int32_t)(key[i] >> 32);
        ids[2 * i + 1] = (int32_t)(key[i] & 0xffffffffu);
    }
    qsort(ids, (size_t)(2 * m), sizeof(int32_t), cmp_i32);
    int64_t n = 0;
    for (int64_t i = 0; i < 2 * m; ++i)
        if (i == 0 || ids[i] != ids[i - 1]) ids[n++] = ids[i];
    g->n = n;
    g->m = m;
    g->labels = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    memcpy(g->labels, ids, (size_t)n * sizeof(int32_t));
    free(ids);
    /* symmetric adjacency with sorted rows */
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
    int32_t *eu = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) {
        eu[i] = dense_id(g->labels, n, (int32_t)(key[i] >> 32));
        ev[i] = dense_id(g->labels, n, (int32_t)(key[i] & 0xffffffffu));
        g->off[eu[i] + 1]++;
        g->off[ev[i] + 1]++;
    }
    for (int64_t x = 0; x < n; ++x) g->off[x + 1] += g->off[x];
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t x = 0; x < n; ++x) fill[x] = g->off[x];
    for (int64_t i = 0; i < m; ++i) {
        g->adj[fill[eu[i]]++] = ev[i];
        g->adj[fill[ev[i]]++] = eu[i];
    }
    for (int64_t x = 0; x < n; ++x)
        qsort(g->adj + g->off[x], (size_t)(g->off[x + 1] - g->off[x]), sizeof(int32_t), cmp_i32);
    free(fill); free(eu); free(ev); free(key);
    return g;
}

static int64_t deg(const og_graph *g, int64_t x) { return g->off[x + 1] - g->off[x]; }

static int64_t find_in_row(const og_graph *g, int64_t x, int32_t y)
{
    int64_t lo = g->off[x], hi = g->off[x + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->adj[mid] == y) return mid;
        if (g->adj[mid] < y) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int og_adjacent(const og_graph *g, int32_t x, int32_t y) { return find_in_row(g, x, y) >= 0; }

/* ------------------------------------------------------------------------ */
/* Triangles t(x,V) and triangle-forming neighbours vt(x,V).                  */
/* Each triangle u < v < w is met once, from the edge (u,v), as a common      */
/* neighbour w > v of u and v (sorted-row merge).  Its three edges are marked */
/* as lying on a triangle; vt(x) counts marked edges at x.                   */
/* ------------------------------------------------------------------------ */
int og_triangles(og_graph *g)
{
    int64_t n = g->n;
    free(g->t); free(g->vt);
    g->t = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    g->vt = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    uint8_t *mark = (uint8_t *)calloc((size_t)(2 * g->m > 0 ? 2 * g->m : 1), 1);
    if (!g->t || !g->vt || !mark) return OG_ERR_OOM;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t pv = g->off[u]; pv < g->off[u + 1]; ++pv) {
            int32_t v = g->adj[pv];
            if (v <= u) continue;
            int64_t i = g->off[u], iend = g->off[u + 1];
            int64_t j = g->off[v], jend = g->off[v + 1];
            while (i < iend && g->adj[i] <= v) ++i;
            while (j < jend && g->adj[j] <= v) ++j;
            while (i < iend && j < jend) {
                if (g->adj[i] < g->adj[j]) ++i;
                else if (g->adj[i] > g->adj[j]) ++j;
                else {
                    int32_t w = g->adj[i];
                    g->t[u]++; g->t[v]++; g->t[w]++;
                    mark[pv] = 1;   /* (u,v) */
                    mark[i] = 1;    /* (u,w) */
                    mark[j] = 1;    /* (v,w) */
                    ++i; ++j;
                }
            }
        }
    }
    for (int64_t u = 0; u < n; ++u)
        for (int64_t p = g->off[u]; p < g->off[u + 1]; ++p)
            if (g->adj[p] > u && mark[p]) { g->vt[u]++; g->vt[g->adj[p]]++; }
    free(mark);
    g->have_tri = 1;
    return OG_OK;
}

/* Triangle count of a single node by its definition (edges among its
 * neighbours), for sampled checks on graphs too large for og_triangles. */
int64_t og_node_triangles(const og_graph *g, int32_t x, int32_t *vt_out)
{
    int64_t tcount = 0;
    int32_t vtc = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
        int32_t y = g->adj[p];
        int64_t common = 0;
        int64_t i = g->off[x], iend = g->off[x + 1], j = g->off[y], jend = g->off[y + 1];
        while (i < iend && j < jend) {
            if (g->adj[i] < g->adj[j]) ++i;
            else if (g->adj[i] > g->adj[j]) ++j;
            else { ++common; ++i; ++j; }
        }
        tcount += common;
        if (common > 0) ++vtc;
    }
    if (vt_out) *vt_out = vtc;
    return tcount / 2;
}

/* ------------------------------------------------------------------------ */
/* Node order (decreasing CC, ties by decreasing degree) and global cc.       */
/* ------------------------------------------------------------------------ */
static const og_graph *g_sort_ctx;

static void cc_fraction(const og_graph *g, int64_t x, uint64_t *num, uint64_t *den)
{
    int64_t d = deg(g, x);
    if (d > 1) { *num = (uint64_t)g->t[x]; *den = (uint64_t)(d * (d - 1) / 2); }
    else { *num = 0; *den = 1; }
}

static int cmp_order(const void *a, const void *b)
{
    const og_graph *g = g_sort_ctx;
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    uint64_t nx, dx, ny, dy;
    cc_fraction(g, x, &nx, &dx);
    cc_fraction(g, y, &ny, &dy);
    unsigned __int128 lhs = (unsigned __int128)nx * dy;   /* CC(x) vs CC(y), exactly */
    unsigned __int128 rhs = (unsigned __int128)ny * dx;
    if (lhs != rhs) return lhs > rhs ? -1 : 1;
    int64_t degx = deg(g, x), degy = deg(g, y);
    if (degx != degy) return degx > degy ? -1 : 1;
    return (x > y) - (x < y);
}

double og_local_cc(const og_graph *g, int64_t x)
{
    int64_t d = deg(g, x);
    if (d <= 1) return 0.0;
    return (double)g->t[x] / (double)(d * (d - 1) / 2);
}

int og_order(og_graph *g)
{
    if (!g->have_tri) return OG_ERR_STATE;
    int64_t n = g->n;
    free(g->order);
    g->order = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t x = 0; x < n; ++x) g->order[x] = (int32_t)x;
    g_sort_ctx = g;
    qsort(g->order, (size_t)n, sizeof(int32_t), cmp_order);
    double *ccs = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t x = 0; x < n; ++x) ccs[x] = og_local_cc(g, x);
    g->cc = n > 0 ? og_fsum(ccs, n) / (double)n : 0.0;
    free(ccs);
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* The estimator.  B(z) = C(z,2) for z >= 1 (0 below), written 0.5*(z*(z-1)).*/
/* ------------------------------------------------------------------------ */
static double binom2(double z) { return z >= 1.0 ? 0.5 * (z * (z - 1.0)) : 0.0; }

/* \wcchat(x,C) for x in C with deg(x,C) = k, deg(x,V) = d, |C| = n and
 * m internal edges:  E[t(x,C)] / E[t(x,V)] * d / (|C \ {x}| + deg(x,V\C)),
 * E[t(x,C)] = C(k,2) p with p = 2m / (n(n-1)),  E[t(x,V)] = C(d,2) cc. */
double og_wcchat_node(int64_t k, int64_t d, int64_t n, int64_t m, double cc)
{
    if (n < 2) return 0.0;
    double nd = (double)n;
    double p = (2.0 * (double)m) / (nd * (nd - 1.0));
    double e_c = binom2((double)k) * p;
    double e_v = binom2((double)d) * cc;
    if (!(e_v > 0.0)) return 0.0;
    return (e_c / e_v) * ((double)d / ((nd - 1.0) + ((double)d - (double)k)));
}

/* Mean-field community score: n members, each with internal degree 2m/n and
 * total degree vol/n, put through the per-node estimator and summed. */
double og_community_score(int64_t n, int64_t m, int64_t vol, double cc)
{
    if (n < 2) return 0.0;
    double nd = (double)n;
    double din = (2.0 * (double)m) / nd;
    double dtot = (double)vol / nd;
    double p = (2.0 * (double)m) / (nd * (nd - 1.0));
    double e_c = binom2(din) * p;
    double e_v = binom2(dtot) * cc;
    if (!(e_v > 0.0)) return 0.0;
    return nd * ((e_c / e_v) * (dtot / ((nd - 1.0) + (dtot - din))));
}

/* The paper's exact WCC(x,C) (Methods, WCC), with C given as a sorted member
 * list; needs only the graph.  Used as a cross-check of the estimator. */
double og_exact_wcc(const og_graph *g, int32_t x, const int32_t *members, int64_t nm)
{
    /* in_c[y] for y in C via binary search on the sorted list */
    #define IN_C(y) (bsearch(&(y), members, (size_t)nm, sizeof(int32_t), cmp_i32) != NULL)
    int64_t t_xc = 0, t_xv = 0, vt_v = 0, vt_out = 0, c_minus_x = 0;
    for (int64_t i = 0; i < nm; ++i) if (members[i] != x) ++c_minus_x;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
        int32_t y = g->adj[p];
        int64_t common = 0, common_c = 0;
        int64_t i = g->off[x], iend = g->off[x + 1], j = g->off[y], jend = g->off[y + 1];
        while (i < iend && j < jend) {
            if (g->adj[i] < g->adj[j]) ++i;
            else if (g->adj[i] > g->adj[j]) ++j;
            else {
                int32_t w = g->adj[i];
                ++common;
                if (IN_C(y) && IN_C(w)) ++common_c;
                ++i; ++j;
            }
        }
        t_xv += common;
        t_xc += common_c;
        if (common > 0) { ++vt_v; if (!IN_C(y)) ++vt_out; }
    }
    #undef IN_C
    t_xv /= 2; t_xc /= 2;
    if (t_xv <= 0) return 0.0;
    return ((double)t_xc / (double)t_xv) * ((double)vt_v / (double)(c_minus_x + vt_out));
}

/* ------------------------------------------------------------------------ */
/* Community state.                                                          */
/* ------------------------------------------------------------------------ */
static int mem_has(const og_graph *g, int64_t y, int32_t c)
{
    return bsearch(&c, g->mem[y], (size_t)g->nmem[y], sizeof(int32_t), cmp_i32) != NULL;
}

/* insert v into the ascending list (*list, *cnt) of capacity *cap */
static void list_insert(int32_t **list, int32_t *cnt, int32_t *cap, int32_t v)
{
    if (*cnt == *cap) {
        *cap = *cap ? 2 * *cap : 4;
        *list = (int32_t *)realloc(*list, (size_t)*cap * sizeof(int32_t));
    }
    int32_t i = *cnt;
    while (i > 0 && (*list)[i - 1] > v) { (*list)[i] = (*list)[i - 1]; --i; }
    (*list)[i] = v;
    (*cnt)++;
}

static void list_remove(int32_t *list, int32_t *cnt, int32_t v)
{
    int32_t j = 0;
    for (int32_t i = 0; i < *cnt; ++i)
        if (list[i] != v) list[j++] = list[i];
    *cnt = j;
}

/* position of c in x's row, -1 if x is not a member */
static int32_t mem_slot(const og_graph *g, int64_t x, int32_t c)
{
    const int32_t *hit = (const int32_t *)bsearch(&c, g->mem[x], (size_t)g->nmem[x], sizeof(int32_t), cmp_i32);
    return hit ? (int32_t)(hit - g->mem[x]) : -1;
}

/* x becomes a member of c: c enters x's row (with deg(x,c) counted), x
 * enters c's member list, and every neighbour of x in c has one more
 * neighbour in c. */
static void mem_insert(og_graph *g, int64_t x, int32_t c)
{
    int32_t k = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
        int32_t y = g->adj[p];
        int32_t s = mem_slot(g, y, c);
        if (s >= 0) { g->kin[y][s]++; ++k; }
    }
    if (g->nmem[x] == g->capmem[x]) {
        g->capmem[x] = g->capmem[x] ? 2 * g->capmem[x] : 4;
        g->mem[x] = (int32_t *)realloc(g->mem[x], (size_t)g->capmem[x] * sizeof(int32_t));
        g->kin[x] = (int32_t *)realloc(g->kin[x], (size_t)g->capmem[x] * sizeof(int32_t));
    }
    int32_t i = g->nmem[x];
    while (i > 0 && g->mem[x][i - 1] > c) {
        g->mem[x][i] = g->mem[x][i - 1];
        g->kin[x][i] = g->kin[x][i - 1];
        --i;
    }
    g->mem[x][i] = c;
    g->kin[x][i] = k;
    g->nmem[x]++;
    list_insert(&g->cmem[c], &g->ncmem[c], &g->capcmem[c], (int32_t)x);
}

/* x stops being a member of c: the reverse of mem_insert */
static void mem_remove(og_graph *g, int64_t x, int32_t c)
{
    int32_t j = 0;
    for (int32_t i = 0; i < g->nmem[x]; ++i)
        if (g->mem[x][i] != c) { g->mem[x][j] = g->mem[x][i]; g->kin[x][j] = g->kin[x][i]; ++j; }
    g->nmem[x] = j;
    list_remove(g->cmem[c], &g->ncmem[c], (int32_t)x);
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
        int32_t y = g->adj[p];
        int32_t s = mem_slot(g, y, c);
        if (s >= 0) g->kin[y][s]--;
    }
}

/* |N(x) \cap C| in the current state */
static int64_t neighbours_in(const og_graph *g, int64_t x, int32_t c)
{
    int64_t k = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p)
        if (mem_has(g, g->adj[p], c)) ++k;
    return k;
}

static void free_state(og_graph *g)
{
    if (g->mem) for (int64_t x = 0; x < g->n; ++x) { free(g->mem[x]); free(g->kin[x]); }
    if (g->cmem) for (int64_t c = 0; c < g->ncomm; ++c) free(g->cmem[c]);
    free(g->mem); free(g->kin); free(g->nmem); free(g->capmem);
    g->kin = NULL;
    free(g->cmem); free(g->ncmem); free(g->capcmem);
    free(g->cn); free(g->cm); free(g->cvol);
    g->mem = NULL; g->nmem = g->capmem = NULL; g->cn = g->cm = g->cvol = NULL;
    g->cmem = NULL; g->ncmem = g->capcmem = NULL;
    g->ncomm = 0;
}

/* empty rows for n nodes and empty member lists for k communities */
static void alloc_state(og_graph *g, int64_t k)
{
    int64_t n = g->n;
    g->mem = (int32_t **)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t *));
    g->kin = (int32_t **)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t *));
    g->nmem = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    g->capmem = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    g->ncomm = k;
    g->cmem = (int32_t **)calloc((size_t)(k > 0 ? k : 1), sizeof(int32_t *));
    g->ncmem = (int32_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int32_t));
    g->capcmem = (int32_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int32_t));
    g->cn = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    g->cm = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    g->cvol = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
}

/* Initial clustering: walk the node order; a node not yet in a community
 * opens a new one (ids 0, 1, 2, ... in opening order) and every neighbour not
 * yet in a community joins it. */
int og_init_clustering(og_graph *g)
{
    if (!g->order) return OG_ERR_STATE;
    free_state(g);
    int64_t n = g->n;
    int32_t *comm = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t x = 0; x < n; ++x) comm[x] = -1;
    int32_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t x = g->order[i];
        if (comm[x] >= 0) continue;
        comm[x] = k;
        for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p)
            if (comm[g->adj[p]] < 0) comm[g->adj[p]] = k;
        ++k;
    }
    alloc_state(g, k);
    for (int64_t x = 0; x < n; ++x) {
        mem_insert(g, x, comm[x]);
        g->cn[comm[x]]++;
        g->cvol[comm[x]] += deg(g, x);
        for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p)
            if (g->adj[p] > x && comm[g->adj[p]] == comm[x]) g->cm[comm[x]]++;
    }
    free(comm);
    return OG_OK;
}

/* Initial state from an inserted division (Methods, Initial Clustering: an
 * existing division may replace the initial clustering step).  Community ids
 * are the division's indices, in its order; aggregates counted from scratch:
 * n_C members, m_C edges with both ends in C, vol_C the members' degrees. */
static int init_from_partition(og_graph *g)
{
    free_state(g);
    int64_t n = g->n, k = g->part_k;
    alloc_state(g, k);
    for (int64_t c = 0; c < k; ++c)
        for (int64_t i = g->part_off[c]; i < g->part_off[c + 1]; ++i) {
            int32_t x = g->part_mem[i];
            mem_insert(g, x, (int32_t)c);
            g->cn[c]++;
            g->cvol[c] += deg(g, x);
        }
    for (int64_t x = 0; x < n; ++x)
        for (int32_t j = 0; j < g->nmem[x]; ++j) {
            int32_t c = g->mem[x][j];
            for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p)
                if (g->adj[p] > x && mem_has(g, g->adj[p], c)) g->cm[c]++;
        }
    return OG_OK;
}

/* Insert a division: community c holds original ids members[off[c] ..
 * off[c+1]).  k < 0 removes it.  OG_ERR_INVALID for offsets that do not start
 * at 0 or decrease, ids not in the graph, or an id twice in one community. */
int og_set_partition(og_graph *g, const int64_t *off, const int32_t *members, int64_t k)
{
    free(g->part_off); free(g->part_mem);
    g->part_off = NULL; g->part_mem = NULL; g->part_k = -1;
    if (k < 0) return OG_OK;
    if (off[0] != 0) return OG_ERR_INVALID;
    for (int64_t c = 0; c < k; ++c)
        if (off[c + 1] < off[c]) return OG_ERR_INVALID;
    int64_t total = off[k];
    int64_t *po = (int64_t *)malloc((size_t)(k + 1) * sizeof(int64_t));
    int32_t *pm = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    for (int64_t c = 0; c <= k; ++c) po[c] = off[c];
    for (int64_t i = 0; i < total; ++i) {
        int32_t x = dense_id(g->labels, g->n, members[i]);
        if (x < 0) { free(po); free(pm); return OG_ERR_INVALID; }
        pm[i] = x;
    }
    for (int64_t c = 0; c < k; ++c) {   /* an id at most once per community */
        int64_t len = po[c + 1] - po[c];
        int32_t *tmp = (int32_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int32_t));
        memcpy(tmp, pm + po[c], (size_t)len * sizeof(int32_t));
        qsort(tmp, (size_t)len, sizeof(int32_t), cmp_i32);
        int dup = 0;
        for (int64_t i = 1; i < len; ++i) dup |= tmp[i] == tmp[i - 1];
        free(tmp);
        if (dup) { free(po); free(pm); return OG_ERR_INVALID; }
    }
    g->part_off = po;
    g->part_mem = pm;
    g->part_k = k;
    return OG_OK;
}

/* \wcchat(P): sum over every (node, community) membership of the per-node
 * estimator, added with the correctly rounded sum. */
double og_total(const og_graph *g)
{
    int64_t cnt = 0;
    for (int64_t x = 0; x < g->n; ++x) cnt += g->nmem[x];
    double *terms = (double *)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(double));
    int64_t i = 0;
    for (int64_t x = 0; x < g->n; ++x)
        for (int32_t j = 0; j < g->nmem[x]; ++j) {
            int32_t c = g->mem[x][j];
            terms[i++] = og_wcchat_node(neighbours_in(g, x, c), deg(g, x), g->cn[c], g->cm[c], g->cc);
        }
    double s = og_fsum(terms, cnt);
    free(terms);
    return s;
}

/* Diagnostic: sum of the mean-field community scores of live communities. */
double og_total_meanfield(const og_graph *g)
{
    double *terms = (double *)malloc((size_t)(g->ncomm > 0 ? g->ncomm : 1) * sizeof(double));
    for (int64_t c = 0; c < g->ncomm; ++c) terms[c] = og_community_score(g->cn[c], g->cm[c], g->cvol[c], g->cc);
    double s = og_fsum(terms, g->ncomm);
    free(terms);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Node changes (Joining / Leaving a Community; Algorithm 1 body).            */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t join, leave; int64_t kjoin, kleave; double gjoin, gleave; } og_action;

static og_action evaluate_node(const og_graph *g, int32_t x)
{
    og_action a = { -1, -1, 0, 0, 0.0, 0.0 };
    int64_t d = deg(g, x);
    /* every community met among the neighbours, once per neighbour */
    int64_t ne = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) ne += g->nmem[g->adj[p]];
    int64_t total = ne + g->nmem[x];
    int32_t *ent = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t e = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
        int32_t y = g->adj[p];
        for (int32_t j = 0; j < g->nmem[y]; ++j) ent[e++] = g->mem[y][j];
    }
    /* own communities take part even with no neighbour inside (k = 0) */
    for (int32_t j = 0; j < g->nmem[x]; ++j) ent[e++] = g->mem[x][j];
    qsort(ent, (size_t)total, sizeof(int32_t), cmp_i32);
    int64_t i = 0;
    while (i < total) {
        int32_t c = ent[i];
        int64_t run = 0;
        while (i < total && ent[i] == c) { ++run; ++i; }
        int own = mem_has(g, x, c);
        int64_t k = own ? run - 1 : run;   /* neighbours of x inside c */
        double before = og_community_score(g->cn[c], g->cm[c], g->cvol[c], g->cc);
        if (!own) {
            double after = og_community_score(g->cn[c] + 1, g->cm[c] + k, g->cvol[c] + d, g->cc);
            double gain = after - before;
            /* ascending c: a strictly larger gain is needed to replace, so ties keep the lowest id */
            if (gain > 0.0 && (a.join < 0 || gain > a.gjoin)) { a.join = c; a.kjoin = k; a.gjoin = gain; }
        } else {
            double after = og_community_score(g->cn[c] - 1, g->cm[c] - k, g->cvol[c] - d, g->cc);
            double gain = after - before;
            if (gain > 0.0 && (a.leave < 0 || gain > a.gleave)) { a.leave = c; a.kleave = k; a.gleave = gain; }
        }
    }
    free(ent);
    return a;
}

/* The paper's gain of a move (Joining / Leaving a Community): the change of
 * \wcchat(P) -- the sum of the per-node estimator over all memberships --
 * when x alone enters (joining != 0) or leaves community c and every other
 * membership stays: C's members see n_C, m_C and, for neighbours of x,
 * deg(y,C) change, and x's own term appears or disappears; no other term
 * changes.  The terms after the move and the negated terms before it are
 * added with the correctly rounded sum.  Costs O(sum of the members'
 * degrees) per candidate. */
static double literal_gain(const og_graph *g, int32_t x, int32_t c, int joining)
{
    int64_t d = deg(g, x);
    int64_t kx = neighbours_in(g, x, c);
    int64_t n0 = g->cn[c], m0 = g->cm[c];
    int64_t n1 = joining ? n0 + 1 : n0 - 1;
    int64_t m1 = joining ? m0 + kx : m0 - kx;
    double *terms = (double *)malloc((size_t)(2 * n0 + 2) * sizeof(double));
    int64_t t = 0;
    for (int32_t i = 0; i < g->ncmem[c]; ++i) {
        int64_t y = g->cmem[c][i];
        if (y == x) continue;
        int64_t ky = g->kin[y][mem_slot(g, y, c)];
        int64_t ky1 = ky;
        if (find_in_row(g, y, x) >= 0) ky1 += joining ? 1 : -1;
        terms[t++] = og_wcchat_node(ky1, deg(g, y), n1, m1, g->cc);
        terms[t++] = -og_wcchat_node(ky, deg(g, y), n0, m0, g->cc);
    }
    if (joining) terms[t++] = og_wcchat_node(kx, d, n1, m1, g->cc);
    else terms[t++] = -og_wcchat_node(kx, d, n0, m0, g->cc);
    double gain = og_fsum(terms, t);
    free(terms);
    return gain;
}

/* A node's decision with the paper's gains: the candidates are the
 * communities met among the neighbours that x is not in (joins) and x's own
 * communities (leaves); per kind the best strictly positive gain, ties to
 * the lowest id (Algorithm 1 body). */
static og_action evaluate_node_literal(const og_graph *g, int32_t x)
{
    og_action a = { -1, -1, 0, 0, 0.0, 0.0 };
    int64_t ne = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) ne += g->nmem[g->adj[p]];
    int64_t total = ne + g->nmem[x];
    int32_t *ent = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t e = 0;
    for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
        int32_t y = g->adj[p];
        for (int32_t j = 0; j < g->nmem[y]; ++j) ent[e++] = g->mem[y][j];
    }
    for (int32_t j = 0; j < g->nmem[x]; ++j) ent[e++] = g->mem[x][j];
    qsort(ent, (size_t)total, sizeof(int32_t), cmp_i32);
    for (int64_t i = 0; i < total; ) {
        int32_t c = ent[i];
        int64_t run = 0;
        while (i < total && ent[i] == c) { ++run; ++i; }
        int own = mem_has(g, x, c);
        int64_t k = own ? run - 1 : run;
        double gain = literal_gain(g, x, c, !own);
        if (!own) {
            if (gain > 0.0 && (a.join < 0 || gain > a.gjoin)) { a.join = c; a.kjoin = k; a.gjoin = gain; }
        } else {
            if (gain > 0.0 && (a.leave < 0 || gain > a.gleave)) { a.leave = c; a.kleave = k; a.gleave = gain; }
        }
    }
    free(ent);
    return a;
}

/* Apply one node's actions to the current partition, leave first.  Each
 * single move changes the community's internal edge count by the number of
 * edges between the node and the community's members at that moment. */
static void apply_actions(og_graph *g, int32_t x, og_action a)
{
    int64_t d = deg(g, x);
    if (a.leave >= 0) {
        mem_remove(g, x, a.leave);
        g->cn[a.leave] -= 1;
        g->cvol[a.leave] -= d;
        g->cm[a.leave] -= neighbours_in(g, x, a.leave);
    }
    if (a.join >= 0) {
        int64_t k = neighbours_in(g, x, a.join);
        mem_insert(g, x, a.join);
        g->cn[a.join] += 1;
        g->cvol[a.join] += d;
        g->cm[a.join] += k;
    }
}

/* Full recount of every community aggregate, of the member lists and of
 * each membership's deg(x,C) from the rows. */
static int recount_ok(const og_graph *g)
{
    int64_t k = g->ncomm;
    int64_t *n = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    int64_t *m2 = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    int64_t *vol = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    int ok = 1;
    for (int64_t x = 0; x < g->n; ++x)
        for (int32_t j = 0; j < g->nmem[x]; ++j) {
            int32_t c = g->mem[x][j];
            if (j > 0 && g->mem[x][j - 1] >= c) ok = 0;
            n[c]++;
            vol[c] += deg(g, x);
            int64_t kx = neighbours_in(g, x, c);
            m2[c] += kx;
            if (g->kin[x][j] != kx) ok = 0;
        }
    for (int64_t c = 0; c < k; ++c) {
        if (n[c] != g->cn[c] || vol[c] != g->cvol[c] || m2[c] != 2 * g->cm[c]) ok = 0;
        if (g->ncmem[c] != n[c]) ok = 0;
        for (int32_t i = 0; i < g->ncmem[c]; ++i)
            if ((i > 0 && g->cmem[c][i - 1] >= g->cmem[c][i]) || !mem_has(g, g->cmem[c][i], (int32_t)c)) ok = 0;
    }
    free(n); free(m2); free(vol);
    return ok;
}

/* Post-processing: drop communities with fewer than two members. */
static void prune(og_graph *g)
{
    for (int64_t x = 0; x < g->n; ++x) {
        int32_t j = 0;
        for (int32_t i = 0; i < g->nmem[x]; ++i)
            if (g->cn[g->mem[x][i]] >= 2) { g->mem[x][j] = g->mem[x][i]; g->kin[x][j] = g->kin[x][i]; ++j; }
        g->nmem[x] = j;
    }
    for (int64_t c = 0; c < g->ncomm; ++c)
        if (g->cn[c] < 2) { g->cn[c] = 0; g->cm[c] = 0; g->cvol[c] = 0; g->ncmem[c] = 0; }
}

/*
 * One LazyFox run (Algorithm 2; queue_size 1 is Fox, Algorithm 1).
 * Restarts from the initial clustering.  Iterations walk the node order in
 * queues of queue_size nodes (the last one may be shorter): every queued node
 * is evaluated against the partition as it stood when the queue was filled,
 * then all actions are applied.  After each iteration degenerate communities
 * are removed, \wcchat(P) is taken and compared with the previous one.
 * max_batches >= 0 stops after that many queues in total (for per-queue
 * comparisons; the iteration end runs only for completed iterations).
 */
int og_run(og_graph *g, int32_t queue_size, double threshold, int32_t max_iters, int64_t max_batches)
{
    if (queue_size < 1 || max_iters < 0) return OG_ERR_INVALID;
    int st = g->part_k >= 0 ? init_from_partition(g) : og_init_clustering(g);
    if (st) return st;
    free(g->T_hist); free(g->S_hist); free(g->joins_hist); free(g->leaves_hist);
    g->hist_cap = max_iters > 0 ? max_iters : 1;
    g->T_hist = (double *)calloc((size_t)g->hist_cap, sizeof(double));
    g->S_hist = (double *)calloc((size_t)g->hist_cap, sizeof(double));
    g->joins_hist = (int64_t *)calloc((size_t)g->hist_cap, sizeof(int64_t));
    g->leaves_hist = (int64_t *)calloc((size_t)g->hist_cap, sizeof(int64_t));
    g->iterations = 0;
    g->converged = 0;
    g->invariant_failures = 0;
    memset(g->diag, 0, sizeof(g->diag));
    g->T0 = og_total(g);
    double prev = g->T0;
    int64_t batches = 0;
    og_action *acts = (og_action *)malloc((size_t)queue_size * sizeof(og_action));
    for (int32_t it = 1; it <= max_iters; ++it) {
        int64_t joins = 0, leaves = 0;
        for (int64_t start = 0; start < g->n; start += queue_size) {
            if (max_batches >= 0 && batches >= max_batches) { free(acts); return OG_OK; }
            int64_t end = start + queue_size < g->n ? start + queue_size : g->n;
            for (int64_t i = start; i < end; ++i) {
                int32_t x = g->order[i];
                og_action lit = { -1, -1, 0, 0, 0.0, 0.0 }, mf = lit;
                if (g->gain_rule == OG_GAIN_LITERAL || g->literal_diag) lit = evaluate_node_literal(g, x);
                if (g->gain_rule == OG_GAIN_MEANFIELD || g->literal_diag) mf = evaluate_node(g, x);
                acts[i - start] = g->gain_rule == OG_GAIN_LITERAL ? lit : mf;
                if (g->literal_diag) {
                    /* same snapshot: nothing of this queue is applied yet */
                    int same_j = lit.join == mf.join, same_l = lit.leave == mf.leave;
                    g->diag[0]++;
                    g->diag[1] += same_j;
                    g->diag[2] += same_l;
                    g->diag[3] += same_j && same_l;
                    g->diag[4] += mf.join >= 0;
                    g->diag[5] += lit.join >= 0;
                    g->diag[6] += mf.leave >= 0;
                    g->diag[7] += lit.leave >= 0;
                }
            }
            for (int64_t i = start; i < end; ++i) {
                apply_actions(g, g->order[i], acts[i - start]);
                joins += acts[i - start].join >= 0;
                leaves += acts[i - start].leave >= 0;
            }
            ++batches;
            if (g->check_invariants && !recount_ok(g)) g->invariant_failures++;
        }
        prune(g);
        double T = og_total(g);
        g->T_hist[it - 1] = T;
        g->S_hist[it - 1] = og_total_meanfield(g);
        g->joins_hist[it - 1] = joins;
        g->leaves_hist[it - 1] = leaves;
        g->iterations = it;
        int stop;
        if (prev == 0.0) stop = (T == 0.0);
        else stop = ((T - prev) / prev) < threshold;
        prev = T;
        if (stop) { g->converged = 1; break; }
    }
    free(acts);
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Quality: F1-score of a detected cover against a reference cover (Methods,  */
/* Evaluation Criteria, F1-Score for Overlapping Communities): the mean over  */
/* detected communities C' of the best F1(C', C) over reference communities;  */
/* F1 = 2 (p r) / (p + r), p = |C ^ C'| / |C'|, r = |C ^ C'| / |C|; 0 when    */
/* they share no node.  Communities are sets of node ids.                      */
/* ------------------------------------------------------------------------ */
double og_f1_pair(int64_t k, int64_t a, int64_t b)
{
    if (k == 0) return 0.0;
    double p = (double)k / (double)a, r = (double)k / (double)b;
    return 2.0 * ((p * r) / (p + r));
}

int og_cover_f1(const int64_t *off_a, const int32_t *mem_a, int64_t ka, const int64_t *off_b,
                const int32_t *mem_b, int64_t kb, double *f1, int32_t *best)
{
    *f1 = 0.0;
    if (ka <= 0) return OG_OK;
    int64_t eb = kb > 0 ? off_b[kb] : 0;
    /* reference memberships sorted by node: (node << 32 | community) */
    uint64_t *pairs = (uint64_t *)malloc((size_t)(eb > 0 ? eb : 1) * sizeof(uint64_t));
    for (int64_t c = 0; c < kb; ++c)
        for (int64_t i = off_b[c]; i < off_b[c + 1]; ++i)
            pairs[i] = ((uint64_t)(uint32_t)mem_b[i] << 32) | (uint64_t)c;
    qsort(pairs, (size_t)eb, sizeof(uint64_t), cmp_u64);
    int64_t *cnt = (int64_t *)calloc((size_t)(kb > 0 ? kb : 1), sizeof(int64_t));
    int64_t *touched = (int64_t *)malloc((size_t)(eb > 0 ? eb : 1) * sizeof(int64_t));
    double *terms = (double *)malloc((size_t)ka * sizeof(double));
    for (int64_t c = 0; c < ka; ++c) {
        int64_t nt = 0;
        for (int64_t i = off_a[c]; i < off_a[c + 1]; ++i) {
            uint64_t key = (uint64_t)(uint32_t)mem_a[i] << 32;
            int64_t lo = 0, hi = eb;   /* first pair of the node */
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (pairs[mid] < key) lo = mid + 1; else hi = mid;
            }
            for (int64_t j = lo; j < eb && (pairs[j] >> 32) == (uint64_t)(uint32_t)mem_a[i]; ++j) {
                int64_t cb = (int64_t)(pairs[j] & 0xffffffffu);
                if (cnt[cb]++ == 0) touched[nt++] = cb;
            }
        }
        double m = 0.0;
        int32_t arg = -1;
        int64_t a = off_a[c + 1] - off_a[c];
        for (int64_t t = 0; t < nt; ++t) {
            int64_t cb = touched[t];
            double f = og_f1_pair(cnt[cb], a, off_b[cb + 1] - off_b[cb]);
            if (arg < 0 || f > m || (f == m && cb < arg)) {   /* ties: lowest reference index */
                m = f;
                arg = (int32_t)cb;
            }
            cnt[cb] = 0;
        }
        terms[c] = m;
        if (best) best[c] = arg;
    }
    *f1 = og_fsum(terms, ka) / (double)ka;
    free(pairs); free(cnt); free(touched); free(terms);
    return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Accessors for the tests.                                                  */
/* ------------------------------------------------------------------------ */
int og_prepare(og_graph *g)
{
    int st = og_triangles(g);
    if (st) return st;
    return og_order(g);
}

void og_sizes(const og_graph *g, int64_t *n, int64_t *m) { *n = g->n; *m = g->m; }

void og_get_csr(const og_graph *g, int64_t *off, int32_t *adj, int32_t *labels)
{
    if (off) memcpy(off, g->off, (size_t)(g->n + 1) * sizeof(int64_t));
    if (adj) memcpy(adj, g->adj, (size_t)(2 * g->m) * sizeof(int32_t));
    if (labels) memcpy(labels, g->labels, (size_t)g->n * sizeof(int32_t));
}

int og_get_node_stats(const og_graph *g, int64_t *t, int32_t *vt, double *cc)
{
    if (!g->have_tri) return OG_ERR_STATE;
    if (t) memcpy(t, g->t, (size_t)g->n * sizeof(int64_t));
    if (vt) memcpy(vt, g->vt, (size_t)g->n * sizeof(int32_t));
    if (cc) *cc = g->cc;
    return OG_OK;
}

int og_get_order(const og_graph *g, int32_t *order)
{
    if (!g->order) return OG_ERR_STATE;
    memcpy(order, g->order, (size_t)g->n * sizeof(int32_t));
    return OG_OK;
}

int64_t og_num_comm_ids(const og_graph *g) { return g->ncomm; }

int64_t og_num_memberships(const og_graph *g)
{
    int64_t c = 0;
    for (int64_t x = 0; x < g->n; ++x) c += g->nmem[x];
    return c;
}

/* memberships as CSR over dense node ids; aggregates for all community ids */
void og_get_state(const og_graph *g, int64_t *mem_off, int32_t *mem_ids,
                  int64_t *cn, int64_t *cm, int64_t *cvol)
{
    int64_t pos = 0;
    for (int64_t x = 0; x < g->n; ++x) {
        if (mem_off) mem_off[x] = pos;
        for (int32_t j = 0; j < g->nmem[x]; ++j) {
            if (mem_ids) mem_ids[pos] = g->mem[x][j];
            ++pos;
        }
    }
    if (mem_off) mem_off[g->n] = pos;
    for (int64_t c = 0; c < g->ncomm; ++c) {
        if (cn) cn[c] = g->cn[c];
        if (cm) cm[c] = g->cm[c];
        if (cvol) cvol[c] = g->cvol[c];
    }
}

void og_get_run(const og_graph *g, int32_t *iterations, int32_t *converged, double *T0,
                double *T_hist, int64_t *joins, int64_t *leaves, int32_t cap)
{
    *iterations = g->iterations;
    *converged = g->converged;
    *T0 = g->T0;
    for (int32_t i = 0; i < g->iterations && i < cap; ++i) {
        if (T_hist) T_hist[i] = g->T_hist[i];
        if (joins) joins[i] = g->joins_hist[i];
        if (leaves) leaves[i] = g->leaves_hist[i];
    }
}

/* Diagnostic history: the sum of the mean-field community scores after each
 * iteration of the last run (beside the literal totals that drive the stop). */
void og_get_meanfield_history(const og_graph *g, double *S_hist, int32_t cap)
{
    for (int32_t i = 0; i < g->iterations && i < cap; ++i) S_hist[i] = g->S_hist[i];
}

void og_set_check_invariants(og_graph *g, int on) { g->check_invariants = on; }
int og_invariant_failures(const og_graph *g) { return g->invariant_failures; }

/* Evaluate one node against the current state (no change), for tests. */
void og_evaluate(const og_graph *g, int32_t x, int32_t *join, int32_t *leave,
                 int64_t *kjoin, int64_t *kleave, double *gjoin, double *gleave)
{
    og_action a = evaluate_node(g, x);
    *join = a.join; *leave = a.leave; *kjoin = a.kjoin; *kleave = a.kleave;
    *gjoin = a.gjoin; *gleave = a.gleave;
}

/* Literal gain of x joining c (x not a member) or leaving it (a member). */
double og_literal_gain(const og_graph *g, int32_t x, int32_t c)
{
    return literal_gain(g, x, c, !mem_has(g, x, c));
}

void og_evaluate_literal(const og_graph *g, int32_t x, int32_t *join, int32_t *leave, double *gjoin,
                         double *gleave)
{
    og_action a = evaluate_node_literal(g, x);
    *join = a.join; *leave = a.leave; *gjoin = a.gjoin; *gleave = a.gleave;
}

/* Decision rule of the following runs: OG_GAIN_LITERAL (the paper's gain,
 * the default) or OG_GAIN_MEANFIELD (the mean-field departure). */
int og_set_gain_rule(og_graph *g, int rule)
{
    if (rule != OG_GAIN_LITERAL && rule != OG_GAIN_MEANFIELD) return OG_ERR_INVALID;
    g->gain_rule = rule;
    return OG_OK;
}
int og_get_gain_rule(const og_graph *g) { return g->gain_rule; }

/* on != 0: the following runs take every decision with both rules and count
 * agreement (the rule set by og_set_gain_rule decides).
 * Counts of the last run: evaluations, equal join decisions, equal leave
 * decisions, both equal, mean-field joins, literal joins, mean-field leaves,
 * literal leaves. */
void og_set_literal_diagnostic(og_graph *g, int on) { g->literal_diag = on; }
void og_get_literal_diagnostic(const og_graph *g, int64_t *out)
{
    for (int i = 0; i < 8; ++i) out[i] = g->diag[i];
}

double og_get_cc(const og_graph *g) { return g->cc; }

void og_destroy(og_graph *g)
{
    if (!g) return;
    free_state(g);
    free(g->part_off); free(g->part_mem);
    free(g->labels); free(g->off); free(g->adj); free(g->t); free(g->vt); free(g->order);
    free(g->T_hist); free(g->S_hist); free(g->joins_hist); free(g->leaves_hist);
    free(g);
}
