// Fox / LazyFox iterations on the GPU (Methods: Initial Clustering; Node
// Changes, Algorithm 1; Parallelism on Node Change Computations, Algorithm 2;
// Stopping Criteria; Post-processing):
//   a6  initial clustering: greedy non-overlapping decomposition in node order
//   a7  move evaluation of one queue: per-node community histogram in shared
//       memory, mean-field WCC-hat gains, best join / best leave
//   a8  bulk apply of one queue: membership rows and community aggregates,
//       with the exact internal-edge correction for nodes that move together
//   a9  iteration end: removal of degenerate communities, exact WCC-hat(P)
#include <algorithm>
#include <chrono>
#include <cmath>

#include "lf_internal.cuh"

namespace lf {
namespace {

constexpr int EV_WARPS = 8;
constexpr int EV_THREADS = EV_WARPS * 32;
constexpr int HW = 512;              // hash slots of one warp
constexpr int HB = EV_WARPS * HW;    // hash slots of a block (hub nodes)
constexpr int AP_THREADS = 256;
constexpr size_t EV_DYN_SMEM = (size_t)HB * 16;   // keys, counts, upper and lower screen bounds

struct RunArgs {
    const int64_t *off;
    const int32_t *adj;
    const int32_t *deg;
    const int32_t *order;
    const int32_t *pos;
    CommRec *comm;
    int32_t *mem;
    int32_t *nmem;
    int32_t K;
    int32_t qcap;
    int32_t *act;   // [join | leave | kjoin | kleave], qcap each
    DevScalars *ds;
    Readback *rbd;
    double cc;
    int64_t nbatches;
    int64_t nnodes;
    int32_t warp_max_deg;
    int32_t profile;   // count algorithmic bytes of the move evaluation
    int32_t debug;     // bounds-checked mode: every index read from device state is checked first
    // hubs: nodes of degree > huge_deg are evaluated one block each with a
    // hash table in global memory (hkeys/hvals/hub_ub/hub_lb at hub_toff[h]),
    // listed per queue: hub_pos[hub_qoff[b] .. hub_qoff[b+1]) are positions
    int32_t huge_deg;
    const int32_t *hub_pos;
    const int64_t *hub_qoff;
    const int64_t *hub_toff;
    const uint32_t *hub_tcap;
    uint32_t *hub_tcap_w;   // the same array, written by k_hub_caps
    int32_t *hkeys;
    uint32_t *hvals;
    float *hub_ub;
    float *hub_lb;
    const int32_t *hub_chunk_h;   // per-queue launches: hub and chunk of each block
    const int32_t *hub_chunk_c;
    const int32_t *hub_nch;
    uint32_t *hub_done;
    uint32_t *hub_ncand;
    int32_t *hub_lbj, *hub_lbl;
    uint32_t *hub_item_base, *hub_nitems, *hub_items_done;
    int32_t *hub_items;
    double *hub_item_g;
    int32_t *hub_item_ck;
    uint32_t *hub_qctr;   // per queue: items, next item to screen, next item to evaluate
    unsigned long long *qtimes;   // profile mode: time stamp after each queue (persistent kernel)
    int32_t screen;    // 1: rule candidates out with the FP32 bound first
    float cc32;        // cc rounded to float (screen)
    float delta;       // relative error bound of the screen (see score32)
    // a batch of graphs: per-graph cc (indexed by a community record's gid)
    // and per-graph exact sums; null for one graph
    const double *gcc;
    const float *gcc32;
    unsigned long long *gsacc;
    const int32_t *gid;
    // WCC-hat total: nodes of degree > TOT_CHUNK are counted in chunks
    const int32_t *tot_hubs;
    const int32_t *tot_chunk_hub;
    const int32_t *tot_first;
    int32_t *tot_cnt;
    uint32_t *tot_done;
    uint32_t *tot_next;
    int64_t tot_nchunks;
    // the paper's gain: deg(x,C) beside every membership, the member index of
    // the iteration (members at its start by community, and its joiners), the
    // per-community sums F(n-1), F(n), F(n+1), and the communities a queue's
    // moves touched (null under the mean-field rule)
    int32_t *kmem;
    const unsigned long long *cm_off;
    int32_t *cm_node;
    uint32_t *cm_cnt;   // entries used in each community's region (members at the start, then joiners)
    int32_t *jl_head, *jl_next, *jl_node;   // joiners beyond a region's capacity
    uint32_t *jl_count;
    float *litF;   // 8 per community: F(n-1), F(n+1), WCC-hat(C), 1/((n+1)n cc), 1/((n-1)(n-2) cc)
    int32_t *touched;
    uint32_t *ntouched;
    uint32_t *tstamp;
    // tables in global memory for nodes with more entries than a block's
    // shared table holds (bump-allocated per queue, lg_cap slots)
    int32_t *lg_keys;
    uint32_t *lg_vals;
    int32_t *lg_aux;
    float *lg_dv;
    unsigned long long lg_cap;
    int32_t lit_hub_deg;   // nodes of higher degree take the hub kernels (INT_MAX: none)
};

// ---------------------------------------------------------------------------
// a6: initial clustering.  A node opens a community iff no neighbour earlier
// in the order opened one (the lexicographically-first maximal independent
// set of the order); decided in rounds, each undecided node looking at its
// earlier neighbours.  Community id = number of openers before it in the
// order; every other node joins its earliest opening neighbour.
// ---------------------------------------------------------------------------
__global__ void k_mis_round(const int64_t *off, const int32_t *adj, const int32_t *pos, int64_t n,
                            int32_t *state, int32_t *undecided) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int und_count = 0;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        if (__ldcg(&state[x]) != 0) continue;
        const int32_t px = pos[x];
        bool seed = false, und = false;
        for (int64_t p = off[x] + lane; p < off[x + 1]; p += 32) {
            int32_t y = adj[p];
            if (pos[y] < px) {
                int32_t s = __ldcg(&state[y]);
                seed |= s == 1;
                und |= s == 0;
            }
        }
        seed = __any_sync(FULL, seed);
        und = __any_sync(FULL, und);
        if (lane == 0) {
            if (seed) state[x] = 2;
            else if (!und) state[x] = 1;
            else ++und_count;
        }
    }
    if (lane == 0 && und_count) atomicAdd(undecided, und_count);
}

__global__ void k_seed_flags(const int32_t *order, const int32_t *state, int64_t n, uint32_t *flag) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = state[order[p]] == 1 ? 1u : 0u;
}

__global__ void k_assign(const int64_t *off, const int32_t *adj, const int32_t *pos, const int32_t *state,
                         const uint32_t *cid, int64_t n, int32_t *comm_of) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        if (state[x] == 1) {
            if (lane == 0) comm_of[x] = (int32_t)cid[pos[x]];
            continue;
        }
        int32_t best = 0x7fffffff;
        for (int64_t p = off[x] + lane; p < off[x + 1]; p += 32) {
            int32_t y = adj[p];
            if (state[y] == 1) best = min(best, pos[y]);
        }
        best = __reduce_min_sync(FULL, best);
        if (lane == 0) comm_of[x] = best == 0x7fffffff ? 0 : (int32_t)cid[best];
    }
}

__global__ void k_init_rows(RunArgs a, const int32_t *comm_of, int64_t n) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = comm_of[x];
        a.mem[x * a.K] = c;
        a.nmem[x] = 1;
        if (a.gid) a.comm[c].gid = a.gid[x];   // every member is in the same graph
        atomicAdd(&a.comm[c].n, 1);
        atomicAdd(&a.comm[c].vol, (uint32_t)a.deg[x]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ds->maxcnt = n > 0 ? 1 : 0;
        a.ds->memberships = (unsigned long long)n;
    }
}

__device__ __forceinline__ bool row_has_c(const int32_t *row, int32_t cnt, int32_t c) {
    int lo = 0, hi = cnt - 1;   // rows are ascending
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = row[mid];
        if (v == c) return true;
        if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    return false;
}

// An inserted division as the initial state: entries x << 32 | c sorted
// ascending, so x's communities are a run of ascending ids.  Rows, member
// counts and degree sums here; internal edges in k_part_m2.
__global__ void k_part_rows(RunArgs a, const unsigned long long *keys, int64_t E, int32_t maxcnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        const int64_t x = (int64_t)(key >> 32);
        const int32_t c = (int32_t)(key & 0xffffffffull);
        int64_t lo = 0, hi = i;   // first entry of x's run
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(keys[mid] >> 32) < x) lo = mid + 1; else hi = mid;
        }
        a.mem[x * a.K + (i - lo)] = c;
        atomicAdd(&a.comm[c].n, 1);
        atomicAdd(&a.comm[c].vol, (uint32_t)a.deg[x]);
        if (i + 1 == E || (int64_t)(keys[i + 1] >> 32) != x) a.nmem[x] = (int32_t)(i - lo + 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ds->maxcnt = maxcnt;
        a.ds->memberships = (unsigned long long)E;
    }
}

// 2m_C of the inserted division: for each membership (x, C), the neighbours of
// x that are in C (one warp per membership).
__global__ void k_part_m2(RunArgs a, const unsigned long long *keys, int64_t E) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < E; i += warps) {
        const unsigned long long key = keys[i];
        const int64_t x = (int64_t)(key >> 32);
        const int32_t c = (int32_t)(key & 0xffffffffull);
        int cnt = 0;
        for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
            const int32_t y = a.adj[p];
            cnt += row_has_c(a.mem + (int64_t)y * a.K, a.nmem[y], c);
        }
        cnt = __reduce_add_sync(FULL, cnt);
        if (lane == 0 && cnt) atomicAdd(&a.comm[c].m2, (uint32_t)cnt);
    }
}

__global__ void k_init_m2(RunArgs a, const int32_t *comm_of, int64_t n) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const int32_t c = comm_of[x];
        int cnt = 0;
        for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) cnt += comm_of[a.adj[p]] == c;
        cnt = __reduce_add_sync(FULL, cnt);
        if (lane == 0 && cnt) atomicAdd(&a.comm[c].m2, (uint32_t)cnt);
    }
}

// ---------------------------------------------------------------------------
// a7: move evaluation.
// ---------------------------------------------------------------------------
struct Best {
    double g;
    int32_t c;
    int32_t k;
};

// (gain descending, id ascending); c < 0 = no action
__device__ __forceinline__ bool better(double g1, int32_t c1, double g2, int32_t c2) {
    if (c1 < 0) return false;
    if (c2 < 0) return true;
    return g1 > g2 || (g1 == g2 && c1 < c2);
}

__device__ __forceinline__ void warp_best(Best &b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double g2 = __shfl_down_sync(FULL, b.g, o);
        int32_t c2 = __shfl_down_sync(FULL, b.c, o);
        int32_t k2 = __shfl_down_sync(FULL, b.k, o);
        if (better(g2, c2, b.g, b.c)) {
            b.g = g2;
            b.c = c2;
            b.k = k2;
        }
    }
}

// Open-addressing insert (linear probing).  own: mark C as a community of the
// evaluated node; otherwise add `add` neighbours.  False if the table is full.
__device__ __forceinline__ bool ht_insert(int32_t *keys, uint32_t *vals, uint32_t hm, int32_t key,
                                          uint32_t add, bool own) {
    uint32_t h = hash32((uint32_t)key) & hm;
    for (uint32_t probe = 0; probe <= hm; ++probe) {
        int32_t prev = atomicCAS(&keys[h], EMPTY_KEY, key);
        if (prev == EMPTY_KEY || prev == key) {
            if (own) atomicOr(&vals[h], OWN_FLAG);
            else atomicAdd(&vals[h], add);
            return true;
        }
        h = (h + 1) & hm;
    }
    return false;
}

// Gain of joining (C not a community of x) or leaving (C one of x's
// communities): change of the community's mean-field score when x's d edges,
// k of them to C's members, enter or leave it.
__device__ __forceinline__ void eval_candidate(const RunArgs &a, int32_t C, uint32_t v, int32_t d, Best &bj,
                                               Best &bl) {
    const bool own = (v & OWN_FLAG) != 0;
    const int64_t k = (int64_t)(v & ~OWN_FLAG);
    const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
    const int64_t n = r.x, m2 = (uint32_t)r.y, vol = (uint32_t)r.z;
    const double cc = a.gcc ? a.gcc[r.w] : a.cc;   // the community's graph
    const double before = community_score(n, m2, vol, cc);
    if (own) {
        double g = __dsub_rn(community_score(n - 1, m2 - 2 * k, vol - d, cc), before);
        if (g > 0.0 && better(g, C, bl.g, bl.c)) bl = Best{g, C, (int32_t)k};
    } else {
        double g = __dsub_rn(community_score(n + 1, m2 + 2 * k, vol + d, cc), before);
        if (g > 0.0 && better(g, C, bj.g, bj.c)) bj = Best{g, C, (int32_t)k};
    }
}

// The same mean-field score in closed form.  With din = m2/n, D = vol/n and
// p = m2/(n(n-1)) the estimator collapses to
//     S = m2^2 (m2 - n) / (cc (n-1) (vol - n) (n(n-1) + vol - m2)),
// zero unless n >= 2, m2 > n (C(din,2) > 0) and vol > n (C(D,2) > 0).  Every
// factor is a non-negative integer below 2^32, converted from 32 bits (the
// 64-bit conversions are slow here); n(n-1) + vol - m2 is formed in float from
// non-negative parts (three roundings, no cancellation).  In all at most 15
// roundings: relative error < 20 x 2^-24.  It is only used to rule candidates
// out: the gain that decides is always the FP64 one.
__device__ __forceinline__ float score32(int64_t n, int64_t m2, int64_t vol, float cc32) {
    if (n < 2 || m2 <= n || vol <= n) return 0.f;
    const float a = __uint2float_rn((uint32_t)m2);
    const float b = __uint2float_rn((uint32_t)(m2 - n));
    const float c = __uint2float_rn((uint32_t)(n - 1));
    const float e = __uint2float_rn((uint32_t)(vol - n));
    const float f = __fadd_rn(__fmul_rn(__uint2float_rn((uint32_t)n), c), __uint2float_rn((uint32_t)(vol - m2)));
    return __fdiv_rn(__fmul_rn(__fmul_rn(a, a), b), __fmul_rn(__fmul_rn(__fmul_rn(c, e), f), cc32));
}

// FP32 gain and an upper bound on |FP64 gain - FP32 gain|:
// delta x (S_new + S_old) with delta covering the FP32 rounding, the FP64
// rounding of the estimator (which grows with m2 and vol through C(din,2) and
// D - din) and the two subtractions.
__device__ __forceinline__ void screen_gain_rec(const RunArgs &a, const int4 &r, uint32_t v, int32_t d, float &g,
                                               float &err) {
    const bool own = (v & OWN_FLAG) != 0;
    const int64_t k = (int64_t)(v & ~OWN_FLAG);
    const int64_t n = r.x, m2 = (uint32_t)r.y, vol = (uint32_t)r.z;
    const float cc32 = a.gcc32 ? a.gcc32[r.w] : a.cc32;
    const float so = score32(n, m2, vol, cc32);
    const float sn = own ? score32(n - 1, m2 - 2 * k, vol - d, cc32) : score32(n + 1, m2 + 2 * k, vol + d, cc32);
    if (!(isfinite(sn) && isfinite(so))) {   // out of float range: keep the candidate, bound nothing
        g = 0.f;
        err = INFINITY;
        return;
    }
    g = __fsub_rn(sn, so);
    err = __fmul_rn(a.delta, __fadd_rn(sn, so));
}

__device__ __forceinline__ float warp_max_f(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

// Pass 1 over candidate slots [lo, hi) (empty slots are skipped): the largest
// lower bound of a join gain and of a leave gain (per lane); each slot's
// upper and lower bounds are kept in ub[] and lb[].  Four record loads are
// issued before any of them is used.
__device__ __forceinline__ void screen_bounds(const RunArgs &a, const int32_t *keys, const uint32_t *vals,
                                              float *ub, float *lb, uint32_t lo, uint32_t hi, int32_t d, float &lbj,
                                              float &lbl) {
    const int lane = threadIdx.x & 31;
    for (uint32_t s0 = lo + lane; s0 < hi; s0 += 128) {
        int32_t C[4];
        uint32_t v[4];
        int4 r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t s = s0 + 32u * u;
            C[u] = s < hi ? keys[s] : EMPTY_KEY;
            v[u] = s < hi ? vals[s] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            r[u] = C[u] != EMPTY_KEY ? __ldcg(reinterpret_cast<const int4 *>(&a.comm[C[u]])) : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (C[u] == EMPTY_KEY) continue;
            float g, e;
            screen_gain_rec(a, r[u], v[u], d, g, e);
            const float l = __fsub_rn(g, e);
            const uint32_t s = s0 + 32u * u;
            ub[s] = __fadd_rn(g, e);
            lb[s] = l;
            if (v[u] & OWN_FLAG) lbl = fmaxf(lbl, l);
            else lbj = fmaxf(lbj, l);
        }
    }
}

// Survivors of the screen, per kind: their count and, when there is exactly
// one, which.  A lone survivor whose lower bound is positive is the best
// action of its kind without an FP64 evaluation: every other candidate's
// FP64 gain is strictly below its own, and its own is positive.
struct Survivors {
    int cj, cl;
    int32_t Cj, Cl;
    uint32_t vj, vl;
    float lbj, lbl;
};

__device__ __forceinline__ bool survives(float ub, uint32_t v, float lbj, float lbl) {
    return ub > 0.f && ub >= ((v & OWN_FLAG) ? lbl : lbj);
}

__device__ void count_survivors(const int32_t *keys, const uint32_t *vals, const float *ubs, const float *lbs,
                                uint32_t lo, uint32_t hi, float lbj, float lbl, Survivors &sv) {
    const int lane = threadIdx.x & 31;
    sv = Survivors{0, 0, -1, -1, 0u, 0u, 0.f, 0.f};
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t s = base + lane;
        bool sj = false, sl = false;
        int32_t C = EMPTY_KEY;
        uint32_t v = 0;
        float lb = 0.f;
        if (s < hi) {
            C = keys[s];
            if (C != EMPTY_KEY) {
                v = vals[s];
                if (survives(ubs[s], v, lbj, lbl)) {
                    lb = lbs[s];
                    if (v & OWN_FLAG) sl = true; else sj = true;
                }
            }
        }
        const unsigned mj = __ballot_sync(FULL, sj), ml = __ballot_sync(FULL, sl);
        if (mj) {
            const int src = __ffs(mj) - 1;
            const int32_t c1 = __shfl_sync(FULL, C, src);
            const uint32_t v1 = __shfl_sync(FULL, v, src);
            const float l1 = __shfl_sync(FULL, lb, src);
            if (sv.cj == 0) { sv.Cj = c1; sv.vj = v1; sv.lbj = l1; }
            sv.cj += __popc(mj);
        }
        if (ml) {
            const int src = __ffs(ml) - 1;
            const int32_t c1 = __shfl_sync(FULL, C, src);
            const uint32_t v1 = __shfl_sync(FULL, v, src);
            const float l1 = __shfl_sync(FULL, lb, src);
            if (sv.cl == 0) { sv.Cl = c1; sv.vl = v1; sv.lbl = l1; }
            sv.cl += __popc(ml);
        }
    }
}

// Pass 2 over table slots [lo, hi): candidates whose upper bound is positive
// and not below the best lower bound of their kind may be the best action;
// they are packed into the warp's buffer and evaluated in FP64 with full
// lanes.  Every candidate whose FP64 gain could be maximal and positive
// survives, so the choice equals an FP64 evaluation of all candidates.
__device__ void eval_survivors(const RunArgs &a, const int32_t *keys, const uint32_t *vals, const float *ubs,
                               uint32_t lo, uint32_t hi, int32_t d, float lbj, float lbl, bool do_j, bool do_l,
                               int32_t *bkey, uint32_t *bval, Best &bj, Best &bl) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    int nbuf = 0;
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t s = base + lane;
        bool surv = false;
        int32_t C = EMPTY_KEY;
        uint32_t v = 0;
        if (s < hi) {
            C = keys[s];
            if (C != EMPTY_KEY) {
                v = vals[s];
                const bool kind_ok = (v & OWN_FLAG) ? do_l : do_j;
                if (!kind_ok) surv = false;
                else if (a.screen) surv = survives(ubs[s], v, lbj, lbl);
                else surv = true;
            }
        }
        const unsigned mask = __ballot_sync(FULL, surv);
        const int cnt = __popc(mask);
        if (nbuf + cnt > 32) {
            if (lane < nbuf) eval_candidate(a, bkey[lane], bval[lane], d, bj, bl);
            __syncwarp();
            nbuf = 0;
        }
        if (surv) {
            const int p = nbuf + __popc(mask & lt);
            bkey[p] = C;
            bval[p] = v;
        }
        nbuf += cnt;
        __syncwarp();
    }
    if (lane < nbuf) eval_candidate(a, bkey[lane], bval[lane], d, bj, bl);
    __syncwarp();
}

__device__ __forceinline__ void write_action(const RunArgs &a, int i, const Best &bj, const Best &bl,
                                             unsigned long long serial) {
    a.act[i] = bj.c;
    a.act[a.qcap + i] = bl.c;
    a.act[2 * a.qcap + i] = bj.k;
    a.act[3 * a.qcap + i] = bl.k;
    (void)serial;
}

// One warp, one node: every membership of every neighbour goes into the
// warp's table; equal ids arriving in the same step are merged first with
// __match_any_sync, so each id costs one atomic per step.  `bound` (>= the
// number of distinct ids) keeps the table at most half full.
// Entry s of a membership row whose first eight entries are in r0, r1.
__device__ __forceinline__ int32_t row_entry(const int4 &r0, const int4 &r1, const int32_t *row, int s) {
    switch (s) {
    case 0: return r0.x;
    case 1: return r0.y;
    case 2: return r0.z;
    case 3: return r0.w;
    case 4: return r1.x;
    case 5: return r1.y;
    case 6: return r1.z;
    case 7: return r1.w;
    default: return __ldcg(row + s);
    }
}

// First eight entries of a row (rows are 16-byte aligned, K a multiple of 4).
__device__ __forceinline__ void row_head(const int32_t *row, int32_t cnt, int4 &r0, int4 &r1) {
    r0 = cnt > 0 ? __ldcg(reinterpret_cast<const int4 *>(row)) : make_int4(0, 0, 0, 0);
    r1 = cnt > 4 ? __ldcg(reinterpret_cast<const int4 *>(row) + 1) : make_int4(0, 0, 0, 0);
}

// Team of T warps (T in 1, 2, 4, 8) working on one node.  Teams of one
// block are numbered tm = warp / T; a team of the whole block synchronises with
// __syncthreads, a single warp with __syncwarp, others with named barrier 1+tm.
template <int T>
__device__ __forceinline__ void team_sync(int tm) {
    if constexpr (T == 1) {
        __syncwarp();
    } else if constexpr (T == EV_WARPS) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + tm), "r"(T * 32) : "memory");
    }
}

// Per-warp values a team exchanges through shared memory.
struct TeamScratch {
    long long part[EV_WARPS];
    float lbj[EV_WARPS], lbl[EV_WARPS];
    int cj[EV_WARPS], cl[EV_WARPS];
    int32_t Cj[EV_WARPS], Cl[EV_WARPS];
    uint32_t vj[EV_WARPS], vl[EV_WARPS];
    float ulj[EV_WARPS], ull[EV_WARPS];
    double bgj[EV_WARPS], bgl[EV_WARPS];
    int32_t bcj[EV_WARPS], bcl[EV_WARPS], bkj[EV_WARPS], bkl[EV_WARPS];
};

// Evaluate node x with a team of T warps.  `bound` (the number of
// (neighbour, community) entries plus x's own memberships) bounds the number
// of distinct ids; the team's table is sized to stay at most half full.  Warp
// w_in of the team takes adjacency chunks w_in, w_in + T, ... (its first chunk
// and the chunk's membership counts arrive in y0 / c0) and a contiguous slice
// of the table for the screen and the FP64 pass.
// Second half of a node's evaluation, on the filled table of H slots: compact
// the candidates, screen them in FP32, decide from the screen alone when one
// candidate of a kind provably wins, evaluate the rest in FP64, reduce over
// the team and record the actions.  bj / bl return the actions (team leader).
template <int T>
__device__ void decide_node(const RunArgs &a, int i, int32_t d, int32_t cx, uint32_t H, int32_t *keys,
                            uint32_t *vals, float *ubs, int32_t *bkey, uint32_t *bval, TeamScratch &ts, int tm,
                            int w_in, unsigned long long serial, unsigned long long pb, Best &bj_out,
                            Best &bl_out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int w0 = tm * T;
    // compact the occupied slots into a dense candidate list (ids into the
    // upper-bound area, counts into the lower-bound area; the table itself is
    // then free and holds the bounds)
    uint32_t ncand, lo, hi;
    int32_t *ck = reinterpret_cast<int32_t *>(ubs);
    uint32_t *cv = reinterpret_cast<uint32_t *>(ubs + HB);
    float *cub = reinterpret_cast<float *>(keys);
    float *clb = reinterpret_cast<float *>(vals);
    {
        const uint32_t slice = (H + T - 1) / T;
        const uint32_t tlo = min(H, (uint32_t)w_in * slice), thi = min(H, tlo + slice);
        uint32_t cnt = 0;
        for (uint32_t b0 = tlo; b0 < thi; b0 += 32) {
            const uint32_t s = b0 + lane;
            cnt += __popc(__ballot_sync(FULL, s < thi && keys[s] != EMPTY_KEY));
        }
        uint32_t offs = 0;
        ncand = cnt;
        if constexpr (T > 1) {
            if (lane == 0) ts.part[w] = cnt;
            team_sync<T>(tm);
            ncand = 0;
            for (int k = 0; k < T; ++k) {
                const uint32_t c = (uint32_t)ts.part[w0 + k];
                if (k < w_in) offs += c;
                ncand += c;
            }
        }
        const unsigned lt = lanemask_lt();
        for (uint32_t b0 = tlo; b0 < thi; b0 += 32) {
            const uint32_t s = b0 + lane;
            const bool occ = s < thi && keys[s] != EMPTY_KEY;
            const unsigned m = __ballot_sync(FULL, occ);
            if (occ) {
                const uint32_t q = offs + __popc(m & lt);
                ck[q] = keys[s];
                cv[q] = vals[s];
            }
            offs += __popc(m);
        }
        team_sync<T>(tm);
        const uint32_t dslice = (ncand + T - 1) / T;
        lo = min(ncand, (uint32_t)w_in * dslice);
        hi = min(ncand, lo + dslice);
    }
    Best bj{0.0, -1, 0}, bl{0.0, -1, 0};
    float lbj = -INFINITY, lbl = -INFINITY;
    bool do_j = true, do_l = true;
    Best uj{0.0, -1, 0}, ul{0.0, -1, 0};   // decided by the screen alone
    if (a.screen) {
        screen_bounds(a, ck, cv, cub, clb, lo, hi, d, lbj, lbl);
        lbj = warp_max_f(lbj);
        lbl = warp_max_f(lbl);
        if constexpr (T > 1) {
            if (lane == 0) {
                ts.lbj[w] = lbj;
                ts.lbl[w] = lbl;
            }
            team_sync<T>(tm);
            for (int k = 0; k < T; ++k) {
                lbj = fmaxf(lbj, ts.lbj[w0 + k]);
                lbl = fmaxf(lbl, ts.lbl[w0 + k]);
            }
        } else {
            __syncwarp();
        }
        Survivors sv;
        count_survivors(ck, cv, cub, clb, lo, hi, lbj, lbl, sv);
        if constexpr (T > 1) {
            if (lane == 0) {
                ts.cj[w] = sv.cj; ts.Cj[w] = sv.Cj; ts.vj[w] = sv.vj; ts.ulj[w] = sv.lbj;
                ts.cl[w] = sv.cl; ts.Cl[w] = sv.Cl; ts.vl[w] = sv.vl; ts.ull[w] = sv.lbl;
            }
            team_sync<T>(tm);
            sv = Survivors{0, 0, -1, -1, 0u, 0u, 0.f, 0.f};
            for (int k = 0; k < T; ++k) {
                const int q = w0 + k;
                if (ts.cj[q] > 0 && sv.cj == 0) { sv.Cj = ts.Cj[q]; sv.vj = ts.vj[q]; sv.lbj = ts.ulj[q]; }
                if (ts.cl[q] > 0 && sv.cl == 0) { sv.Cl = ts.Cl[q]; sv.vl = ts.vl[q]; sv.lbl = ts.ull[q]; }
                sv.cj += ts.cj[q];
                sv.cl += ts.cl[q];
            }
        }
        do_j = sv.cj > 1 || (sv.cj == 1 && !(sv.lbj > 0.f));
        do_l = sv.cl > 1 || (sv.cl == 1 && !(sv.lbl > 0.f));
        if (sv.cj == 1 && !do_j) uj = Best{INFINITY, sv.Cj, (int32_t)(sv.vj & ~OWN_FLAG)};
        if (sv.cl == 1 && !do_l) ul = Best{INFINITY, sv.Cl, (int32_t)(sv.vl & ~OWN_FLAG)};
        if (sv.cj == 0) do_j = false;
        if (sv.cl == 0) do_l = false;
    }
    if (do_j || do_l) eval_survivors(a, ck, cv, cub, lo, hi, d, lbj, lbl, do_j, do_l, bkey, bval, bj, bl);
    if (a.profile && lane == 0) pb += 16ull * (unsigned long long)(hi - lo);
    warp_best(bj);
    warp_best(bl);
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if (lane == 0) atomicAdd(&a.ds->prof_bytes, pb + (w_in == 0 ? 44ull + 4ull * (unsigned long long)cx : 0ull));
    }
    if constexpr (T > 1) {
        if (lane == 0) {
            ts.bgj[w] = bj.g; ts.bcj[w] = bj.c; ts.bkj[w] = bj.k;
            ts.bgl[w] = bl.g; ts.bcl[w] = bl.c; ts.bkl[w] = bl.k;
        }
        team_sync<T>(tm);
        if (w_in == 0 && lane == 0) {
            for (int k = 1; k < T; ++k) {
                const int q = w0 + k;
                if (better(ts.bgj[q], ts.bcj[q], bj.g, bj.c)) bj = Best{ts.bgj[q], ts.bcj[q], ts.bkj[q]};
                if (better(ts.bgl[q], ts.bcl[q], bl.g, bl.c)) bl = Best{ts.bgl[q], ts.bcl[q], ts.bkl[q]};
            }
        }
    }
    if (w_in == 0 && lane == 0) {
        if (uj.c >= 0) bj = uj;
        if (ul.c >= 0) bl = ul;
        write_action(a, i, bj, bl, serial);
    }
    bj_out = bj;
    bl_out = bl;
    team_sync<T>(tm);
}

// Histogram of one warp step: the (neighbour, membership) pairs of the
// warp's 32 neighbours laid end to end and taken 32 per round, so rounds
// follow the pairs' count rather than the longest row.  A lane finds its
// pair's neighbour by a binary search over the warp's prefix sums
// (shuffles), takes the community from that neighbour's row head in
// registers (or from memory past eight), and equal ids of a round are merged
// with __match_any_sync before one insert.
// keep(C): whether this pass counts C; insert(C, count): count C (one lane per
// distinct C of a round).
template <typename Keep, typename Insert>
__device__ __forceinline__ void fill_flat_with(const RunArgs &a, int32_t y, int32_t cy, const int4 &r0, const int4 &r1,
                                               Keep keep, Insert insert) {
    const int lane = threadIdx.x & 31;
    int incl = cy;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int tot = __shfl_sync(FULL, incl, 31);
    const int excl = incl - cy;
    for (int e0 = 0; e0 < tot; e0 += 32) {
        const int e = e0 + lane;
        int j = 0;   // last lane whose pairs start at or before e
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int ex = __shfl_sync(FULL, excl, j + step);
            if (ex <= e) j += step;
        }
        const int k = e - __shfl_sync(FULL, excl, j);
        const int32_t v0 = __shfl_sync(FULL, r0.x, j), v1 = __shfl_sync(FULL, r0.y, j);
        const int32_t v2 = __shfl_sync(FULL, r0.z, j), v3 = __shfl_sync(FULL, r0.w, j);
        const int32_t v4 = __shfl_sync(FULL, r1.x, j), v5 = __shfl_sync(FULL, r1.y, j);
        const int32_t v6 = __shfl_sync(FULL, r1.z, j), v7 = __shfl_sync(FULL, r1.w, j);
        const int32_t yj = __shfl_sync(FULL, y, j);
        int32_t C = -2 - lane;
        if (e < tot) {
            C = k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : k == 3 ? v3 : k == 4 ? v4 : k == 5 ? v5 : k == 6 ? v6 : v7;
            if (k >= 8) C = __ldcg(&a.mem[(int64_t)yj * a.K + k]);
            if (!keep(C)) C = -2 - lane;
        }
        const unsigned mask = __match_any_sync(FULL, C);
        if (C >= 0 && lane == __ffs(mask) - 1) insert(C, (uint32_t)__popc(mask));
    }
}

__device__ __forceinline__ void fill_flat(const RunArgs &a, int32_t *keys, uint32_t *vals, uint32_t hm, int32_t y,
                                          int32_t cy, const int4 &r0, const int4 &r1) {
    fill_flat_with(a, y, cy, r0, r1, [](int32_t) { return true; },
                   [&](int32_t C, uint32_t c) { ht_insert(keys, vals, hm, C, c, false); });
}

template <int T>
__device__ void eval_team(const RunArgs &a, int i, int32_t x, int32_t d, int64_t beg, int64_t end, int64_t bound,
                          int32_t y0, int32_t c0, int32_t *keys, uint32_t *vals, float *ubs, int32_t *bkey,
                          uint32_t *bval, TeamScratch &ts, int tm, int w_in, unsigned long long serial) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tl = w_in * 32 + lane;
    constexpr int NT = T * 32;
    const int w0 = tm * T;   // first warp of the team
    uint32_t H = 32;
    while ((int64_t)H < 2 * bound) H <<= 1;
    const uint32_t hm = H - 1;
    for (uint32_t s = tl; s < H; s += NT) {
        keys[s] = EMPTY_KEY;
        vals[s] = 0u;
    }
    team_sync<T>(tm);
    const int32_t cx = __ldcg(&a.nmem[x]);
    const int32_t *rowx = a.mem + (int64_t)x * a.K;
    for (int j = tl; j < cx; j += NT) ht_insert(keys, vals, hm, __ldcg(&rowx[j]), 0u, true);
    team_sync<T>(tm);
    unsigned long long pb = 0;
    const int64_t first = beg + w_in * 32;
    for (int64_t p0 = first; p0 < end; p0 += NT) {
        const int64_t p = p0 + lane;
        int32_t y = 0, cy = 0;
        if (p0 == first) {
            y = y0;
            cy = c0;
        } else if (p < end) {
            y = a.adj[p];
            cy = __ldcg(&a.nmem[y]);
        }
        if (p < end) pb += 8ull + 4ull * (unsigned long long)cy;
        const int32_t *rowy = a.mem + (int64_t)y * a.K;
        int4 r0, r1;
        row_head(rowy, cy, r0, r1);
        fill_flat(a, keys, vals, hm, y, cy, r0, r1);
    }
    team_sync<T>(tm);
    Best bj, bl;
    decide_node<T>(a, i, d, cx, H, keys, vals, ubs, bkey, bval, ts, tm, w_in, serial, pb, bj, bl);
}

__device__ __forceinline__ uint32_t part_of(int32_t C, int P) {
    return hash32((uint32_t)C ^ 0x9e3779b9u) % (uint32_t)P;
}

struct BlockScratch {
    double gj[EV_WARPS], gl[EV_WARPS];
    int32_t cj[EV_WARPS], cl[EV_WARPS], kj[EV_WARPS], kl[EV_WARPS];
    float lbj[EV_WARPS], lbl[EV_WARPS];
    int overflow;
};

// One block, one node (high degree).  The ids are split into P parts by a
// hash and each part is counted in the block's table in its own pass; if a
// pass overflows the table, P doubles and the evaluation restarts.
__device__ void eval_block(const RunArgs &a, int i, int32_t x, int64_t bound, int32_t *keys, uint32_t *vals,
                           float *ubs, int32_t *bkey, uint32_t *bval, BlockScratch &bs, unsigned long long serial,
                           float *lbs = nullptr, uint32_t hcap = HB) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t d = a.deg[x];
    const int32_t cx = __ldcg(&a.nmem[x]);
    const int32_t *rowx = a.mem + (int64_t)x * a.K;
    const int64_t beg = a.off[x], end = a.off[x + 1];
    if (!lbs) lbs = ubs + HB;
    int P = bound <= hcap / 2 ? 1 : (int)((bound + hcap / 4 - 1) / (hcap / 4));
    Best bj, bl;
    unsigned long long pb = 0;
    for (;;) {
        bj = Best{0.0, -1, 0};
        bl = Best{0.0, -1, 0};
        pb = 0;
        // running best lower bounds over the parts seen so far
        float lbj = -INFINITY, lbl = -INFINITY;
        uint32_t H = hcap;
        if (P == 1) {
            H = 32;
            while ((int64_t)H < 2 * bound) H <<= 1;
        }
        const uint32_t hm = H - 1;
        bool overflow = false;
        for (int part = 0; part < P; ++part) {
            for (uint32_t s = threadIdx.x; s < H; s += EV_THREADS) {
                keys[s] = EMPTY_KEY;
                vals[s] = 0u;
            }
            if (threadIdx.x == 0) bs.overflow = 0;
            __syncthreads();
            for (int j = threadIdx.x; j < cx; j += EV_THREADS) {
                int32_t C = __ldcg(&rowx[j]);
                if (P == 1 || part_of(C, P) == (uint32_t)part)
                    if (!ht_insert(keys, vals, hm, C, 0u, true)) bs.overflow = 1;
            }
            __syncthreads();
            for (int64_t p0 = beg + w * 32; p0 < end; p0 += EV_THREADS) {
                const int64_t p = p0 + lane;
                int32_t y = 0, cy = 0;
                if (p < end) {
                    y = a.adj[p];
                    cy = __ldcg(&a.nmem[y]);
                    if (part == 0) pb += 8ull + 4ull * (unsigned long long)cy;
                }
                const int32_t *rowy = a.mem + (int64_t)y * a.K;
                int4 r0, r1;
                row_head(rowy, cy, r0, r1);
                fill_flat_with(
                    a, y, cy, r0, r1, [&](int32_t C) { return P == 1 || part_of(C, P) == (uint32_t)part; },
                    [&](int32_t C, uint32_t c) {
                        if (!ht_insert(keys, vals, hm, C, c, false)) bs.overflow = 1;
                    });
            }
            __syncthreads();
            if (bs.overflow) {
                overflow = true;
                __syncthreads();
                break;
            }
            // each warp owns a contiguous slice of the table
            const uint32_t slice = (H + EV_WARPS - 1) / EV_WARPS;
            const uint32_t lo = min(H, (uint32_t)w * slice), hi = min(H, lo + slice);
            if (a.screen) {
                float wj = lbj, wl = lbl;
                screen_bounds(a, keys, vals, ubs, lbs, lo, hi, d, wj, wl);
                wj = warp_max_f(wj);
                wl = warp_max_f(wl);
                if (lane == 0) {
                    bs.lbj[w] = wj;
                    bs.lbl[w] = wl;
                }
                __syncthreads();
                for (int ww = 0; ww < EV_WARPS; ++ww) {
                    lbj = fmaxf(lbj, bs.lbj[ww]);
                    lbl = fmaxf(lbl, bs.lbl[ww]);
                }
            }
            eval_survivors(a, keys, vals, ubs, lo, hi, d, lbj, lbl, true, true, bkey, bval, bj, bl);
            if (a.profile)
                for (uint32_t s = lo + lane; s < hi; s += 32) pb += keys[s] != EMPTY_KEY ? 16ull : 0ull;
            __syncthreads();
        }
        if (!overflow) break;
        if (P >= (1 << 20)) {   // cannot happen for a hash of distinct ids; report instead of looping
            if (threadIdx.x == 0) atomicOr(&a.ds->err, DERR_CHECK);
            break;
        }
        P *= 2;
    }
    warp_best(bj);
    warp_best(bl);
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if (lane == 0) atomicAdd(&a.ds->prof_bytes, pb + (w == 0 ? 44ull + 4ull * (unsigned long long)cx : 0ull));
    }
    if (lane == 0) {
        bs.gj[w] = bj.g; bs.cj[w] = bj.c; bs.kj[w] = bj.k;
        bs.gl[w] = bl.g; bs.cl[w] = bl.c; bs.kl[w] = bl.k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Best fj{0.0, -1, 0}, fl{0.0, -1, 0};
        for (int ww = 0; ww < EV_WARPS; ++ww) {
            if (better(bs.gj[ww], bs.cj[ww], fj.g, fj.c)) fj = Best{bs.gj[ww], bs.cj[ww], bs.kj[ww]};
            if (better(bs.gl[ww], bs.cl[ww], fl.g, fl.c)) fl = Best{bs.gl[ww], bs.cl[ww], bs.kl[ww]};
        }
        write_action(a, i, fj, fl, serial);
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned long long queue_serial(const RunArgs &a, int64_t bidx) {
    return (unsigned long long)__ldcg(&a.ds->iter) * (unsigned long long)a.nbatches + (unsigned long long)bidx + 1ull;
}

// The hubs of queue b, one block each (block-strided), each with its own
// hash table in global memory sized for (d+1) x K entries when the run was
// planned: one pass over the neighbours however many distinct communities
// they bring.
__device__ void eval_huge(const RunArgs &a, int64_t bstart, int64_t b, unsigned long long serial, int32_t *bkey,
                          uint32_t *bval, BlockScratch &bs) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ long long s_entries[EV_WARPS];
    if (!a.hub_qoff) return;
    for (int64_t h = a.hub_qoff[b] + blockIdx.x; h < a.hub_qoff[b + 1]; h += gridDim.x) {
        const int64_t p = a.hub_pos[h];
        const int32_t x = a.order[p];
        const int64_t beg = a.off[x], end = a.off[x + 1];
        long long e = 0;
        for (int64_t q = beg + threadIdx.x; q < end; q += EV_THREADS) e += __ldcg(&a.nmem[a.adj[q]]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
        if (lane == 0) s_entries[w] = e;
        __syncthreads();
        long long entries = __ldcg(&a.nmem[x]);
        for (int k = 0; k < EV_WARPS; ++k) entries += s_entries[k];
        __syncthreads();
        const int64_t t0 = a.hub_toff[h];
        const uint32_t cap = a.hub_tcap[h];
        eval_block(a, (int)(p - bstart), x, entries, a.hkeys + t0, a.hvals + t0, a.hub_ub + t0, bkey, bval, bs, serial,
                   a.hub_lb + t0, cap);
        for (uint32_t s = threadIdx.x; s < cap; s += EV_THREADS) {   // tables are left clean between uses
            a.hkeys[t0 + s] = EMPTY_KEY;
            a.hvals[t0 + s] = 0u;
        }
        __syncthreads();
    }
}

// Count `add` for key in a shared table, giving up after `probes` slots (the
// caller then counts it elsewhere).
__device__ __forceinline__ bool st_insert_bounded(int32_t *keys, uint32_t *vals, uint32_t hm, int32_t key,
                                                  uint32_t add, int probes) {
    uint32_t h = hash32((uint32_t)key) & hm;
    for (int probe = 0; probe < probes; ++probe) {
        const int32_t prev = atomicCAS(&keys[h], EMPTY_KEY, key);
        if (prev == EMPTY_KEY || prev == key) {
            atomicAdd(&vals[h], add);
            return true;
        }
        h = (h + 1) & hm;
    }
    return false;
}

// Insert into a hub's global table; a new id also gets its slot appended to
// the hub's list of occupied slots.  False if the table is full.
__device__ __forceinline__ bool hub_insert(int32_t *keys, uint32_t *vals, uint32_t hm, int32_t key, uint32_t add,
                                           bool own, int32_t *list, uint32_t *ncand) {
    uint32_t h = hash32((uint32_t)key) & hm;
    for (uint32_t probe = 0; probe <= hm; ++probe) {
        const int32_t prev = atomicCAS(&keys[h], EMPTY_KEY, key);
        if (prev == EMPTY_KEY || prev == key) {
            if (own) atomicOr(&vals[h], OWN_FLAG);
            else atomicAdd(&vals[h], add);
            if (prev == EMPTY_KEY) list[atomicAdd(ncand, 1u)] = (int32_t)h;
            return true;
        }
        h = (h + 1) & hm;
    }
    return false;
}

// Table size of every hub for this iteration: twice a bound on its entries,
// own row + one possible join + sum over neighbours of (row length + one
// possible join), as a power of two; never above the planned worst case.
// Dense tables keep the random accesses of the fill and the compaction in
// fewer sectors than the worst-case size would.
__global__ void __launch_bounds__(EV_THREADS) k_hub_caps(RunArgs a, const uint32_t *wcap, int64_t nhubs) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nhubs; h += warps) {
        const int32_t x = a.order[a.hub_pos[h]];
        const int64_t beg = a.off[x], end = a.off[x + 1];
        unsigned long long e = 0;
        for (int64_t p = beg + lane; p < end; p += 32) e += 1ull + (unsigned long long)__ldcg(&a.nmem[a.adj[p]]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
        if (lane == 0) {
            e += 1ull + (unsigned long long)__ldcg(&a.nmem[x]);
            unsigned long long cap = 32;
            while (cap < 2ull * e) cap <<= 1;
            a.hub_tcap_w[h] = (uint32_t)min(cap, (unsigned long long)wcap[h]);
        }
    }
}

// Hubs with more than HUGE_BIG_NCAND candidates: items of HUGE_CAND_CHUNK
// candidates.  k_huge_screen moves an item's candidates out of the table
// (ids and counts into dense arrays in the upper- and lower-bound areas, the
// slots cleared), computes their FP32 upper bounds and raises the hub's best
// lower bounds; k_huge_eval evaluates the survivors in FP64 and the block
// finishing a hub's last item records the best actions.
constexpr uint32_t HUGE_BIG_NCAND = 8192;
constexpr uint32_t HUGE_CAND_CHUNK = 4096;

__device__ __forceinline__ int32_t f2ord(float f) {
    const int32_t b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int32_t k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

struct HubItem {
    int h, j;
    int64_t t0;
    uint32_t cap, lo, hi;
};

__device__ __forceinline__ HubItem hub_item(const RunArgs &a, uint32_t it) {
    HubItem r;
    r.h = a.hub_items[2 * it];
    r.j = a.hub_items[2 * it + 1];
    r.t0 = a.hub_toff[r.h];
    r.cap = a.hub_tcap[r.h];
    const uint32_t ncand = __ldcg(&a.hub_ncand[r.h]);
    r.lo = (uint32_t)r.j * HUGE_CAND_CHUNK;
    r.hi = min(ncand, r.lo + HUGE_CAND_CHUNK);
    return r;
}

__global__ void __launch_bounds__(EV_THREADS) k_huge_screen(RunArgs a, int64_t bidx) {
    __shared__ uint32_t s_it;
    __shared__ float s_lbj[EV_WARPS], s_lbl[EV_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *qc = a.hub_qctr + 3 * bidx;
    const uint32_t count = __ldcg(&qc[0]);
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(&qc[1], 1u);
        __syncthreads();
        const uint32_t it = s_it;
        __syncthreads();
        if (it >= count) break;
        const HubItem I = hub_item(a, it);
        int32_t *keys = a.hkeys + I.t0;
        uint32_t *vals = a.hvals + I.t0;
        const int32_t *list = reinterpret_cast<const int32_t *>(a.hub_lb + I.t0);
        int32_t *ck = reinterpret_cast<int32_t *>(a.hub_ub + I.t0);
        float *cub = a.hub_ub + I.t0 + I.cap / 2;
        uint32_t *cv = reinterpret_cast<uint32_t *>(a.hub_lb + I.t0) + I.cap / 2;
        const int32_t x = a.order[a.hub_pos[I.h]];
        const int32_t d = a.deg[x];
        float lbj = -INFINITY, lbl = -INFINITY;
        unsigned long long pb = 0;
        constexpr int U = 4;   // candidates per thread and step, their loads issued together
        for (uint32_t k0 = I.lo + threadIdx.x; k0 < I.hi; k0 += U * EV_THREADS) {
            int32_t sl[U], C[U];
            uint32_t v[U];
            int4 r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t k = k0 + u * EV_THREADS;
                sl[u] = k < I.hi ? __ldcg(&list[k]) : -1;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                C[u] = sl[u] >= 0 ? __ldcg(&keys[sl[u]]) : EMPTY_KEY;
                v[u] = sl[u] >= 0 ? __ldcg(&vals[sl[u]]) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                r[u] = (a.screen && sl[u] >= 0) ? __ldcg(reinterpret_cast<const int4 *>(&a.comm[C[u]]))
                                                 : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (sl[u] < 0) continue;
                const uint32_t k = k0 + u * EV_THREADS;
                keys[sl[u]] = EMPTY_KEY;
                vals[sl[u]] = 0u;
                ck[k] = C[u];
                cv[k] = v[u];
                float ub = INFINITY;
                if (a.screen) {
                    float g, e;
                    screen_gain_rec(a, r[u], v[u], d, g, e);
                    ub = __fadd_rn(g, e);
                    const float l = __fsub_rn(g, e);
                    if (v[u] & OWN_FLAG) lbl = fmaxf(lbl, l); else lbj = fmaxf(lbj, l);
                }
                cub[k] = ub;
                pb += 16ull;
            }
        }
        lbj = warp_max_f(lbj);
        lbl = warp_max_f(lbl);
        if (lane == 0) {
            s_lbj[w] = lbj;
            s_lbl[w] = lbl;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < EV_WARPS; ++k) {
                lbj = fmaxf(lbj, s_lbj[k]);
                lbl = fmaxf(lbl, s_lbl[k]);
            }
            atomicMax(&a.hub_lbj[I.h], f2ord(lbj));
            atomicMax(&a.hub_lbl[I.h], f2ord(lbl));
        }
        if (a.profile) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
            if (lane == 0 && pb) atomicAdd(&a.ds->prof_bytes, pb);
        }
    }
}

__global__ void __launch_bounds__(EV_THREADS) k_huge_eval(RunArgs a, int64_t bstart, int64_t bidx) {
    __shared__ uint32_t s_it;
    __shared__ unsigned s_last;
    __shared__ BlockScratch bs;
    __shared__ int32_t bkey[EV_WARPS][32];
    __shared__ uint32_t bval[EV_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *qc = a.hub_qctr + 3 * bidx;
    const uint32_t count = __ldcg(&qc[0]);
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(&qc[2], 1u);
        __syncthreads();
        const uint32_t it = s_it;
        __syncthreads();
        if (it >= count) break;
        const HubItem I = hub_item(a, it);
        const int32_t *ck = reinterpret_cast<const int32_t *>(a.hub_ub + I.t0);
        const float *cub = a.hub_ub + I.t0 + I.cap / 2;
        const uint32_t *cv = reinterpret_cast<const uint32_t *>(a.hub_lb + I.t0) + I.cap / 2;
        const int64_t p = a.hub_pos[I.h];
        const int32_t x = a.order[p];
        const int32_t d = a.deg[x];
        const float lbj = ord2f(__ldcg(&a.hub_lbj[I.h])), lbl = ord2f(__ldcg(&a.hub_lbl[I.h]));
        const uint32_t n = I.hi - I.lo, slice = (n + EV_WARPS - 1) / EV_WARPS;
        const uint32_t lo = min(I.hi, I.lo + (uint32_t)w * slice), hi = min(I.hi, lo + slice);
        Best bj{0.0, -1, 0}, bl{0.0, -1, 0};
        eval_survivors(a, ck, cv, cub, lo, hi, d, lbj, lbl, true, true, bkey[w], bval[w], bj, bl);
        warp_best(bj);
        warp_best(bl);
        if (lane == 0) {
            bs.gj[w] = bj.g; bs.cj[w] = bj.c; bs.kj[w] = bj.k;
            bs.gl[w] = bl.g; bs.cl[w] = bl.c; bs.kl[w] = bl.k;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Best fj{0.0, -1, 0}, fl{0.0, -1, 0};
            for (int ww = 0; ww < EV_WARPS; ++ww) {
                if (better(bs.gj[ww], bs.cj[ww], fj.g, fj.c)) fj = Best{bs.gj[ww], bs.cj[ww], bs.kj[ww]};
                if (better(bs.gl[ww], bs.cl[ww], fl.g, fl.c)) fl = Best{bs.gl[ww], bs.cl[ww], bs.kl[ww]};
            }
            a.hub_item_g[2 * it] = fj.g;
            a.hub_item_g[2 * it + 1] = fl.g;
            a.hub_item_ck[4 * it] = fj.c;
            a.hub_item_ck[4 * it + 1] = fj.k;
            a.hub_item_ck[4 * it + 2] = fl.c;
            a.hub_item_ck[4 * it + 3] = fl.k;
            __threadfence();
            s_last = atomicAdd(&a.hub_items_done[I.h], 1u) == a.hub_nitems[I.h] - 1;
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {   // every item of the hub is in: its best actions
            __threadfence();
            const uint32_t base = a.hub_item_base[I.h], ni = a.hub_nitems[I.h];
            Best fj{0.0, -1, 0}, fl{0.0, -1, 0};
            for (uint32_t k = base; k < base + ni; ++k) {
                const double gj = __ldcg(&a.hub_item_g[2 * k]), gl = __ldcg(&a.hub_item_g[2 * k + 1]);
                const int32_t cj = __ldcg(&a.hub_item_ck[4 * k]), kj = __ldcg(&a.hub_item_ck[4 * k + 1]);
                const int32_t cl = __ldcg(&a.hub_item_ck[4 * k + 2]), kl = __ldcg(&a.hub_item_ck[4 * k + 3]);
                if (better(gj, cj, fj.g, fj.c)) fj = Best{gj, cj, kj};
                if (better(gl, cl, fl.g, fl.c)) fl = Best{gl, cl, kl};
            }
            write_action(a, (int)(p - bstart), fj, fl, queue_serial(a, bidx));
            if (a.profile) atomicAdd(&a.ds->prof_bytes, 44ull + 4ull * (unsigned long long)__ldcg(&a.nmem[x]));
            a.hub_items_done[I.h] = 0u;
            a.hub_ncand[I.h] = 0u;
            a.hub_lbj[I.h] = f2ord(-INFINITY);
            a.hub_lbl[I.h] = f2ord(-INFINITY);
        }
        __syncthreads();
    }
}

// Per-queue launches: one block per chunk of HUGE_CHUNK neighbours of a hub.
// Each block adds its neighbours' memberships to the hub's table in global
// memory (the first chunk also the hub's own row); the block that finishes
// the hub's last chunk screens and evaluates the candidates, records the
// actions and clears the table.
constexpr int HUGE_CHUNK = 1024;
constexpr int HUGE_ROUNDS = HUGE_CHUNK / EV_THREADS;   // neighbours per thread
constexpr uint32_t HUGE_SH = 8192;   // shared-memory table of a chunk block (keys and counts: 64 KiB)

__device__ void huge_decide(const RunArgs &a, int i, int32_t d, int32_t cx, const int32_t *keys, const uint32_t *vals,
                            float *ubs, float *lbs, uint32_t H, int32_t *bkey, uint32_t *bval, BlockScratch &bs,
                            unsigned long long serial) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t slice = (H + EV_WARPS - 1) / EV_WARPS;
    const uint32_t lo = min(H, (uint32_t)w * slice), hi = min(H, lo + slice);
    float lbj = -INFINITY, lbl = -INFINITY;
    if (a.screen) {
        float wj = lbj, wl = lbl;
        screen_bounds(a, keys, vals, ubs, lbs, lo, hi, d, wj, wl);
        wj = warp_max_f(wj);
        wl = warp_max_f(wl);
        if (lane == 0) {
            bs.lbj[w] = wj;
            bs.lbl[w] = wl;
        }
        __syncthreads();
        for (int ww = 0; ww < EV_WARPS; ++ww) {
            lbj = fmaxf(lbj, bs.lbj[ww]);
            lbl = fmaxf(lbl, bs.lbl[ww]);
        }
    }
    Best bj{0.0, -1, 0}, bl{0.0, -1, 0};
    eval_survivors(a, keys, vals, ubs, lo, hi, d, lbj, lbl, true, true, bkey, bval, bj, bl);
    if (a.profile) {
        unsigned long long pb = 0;
        for (uint32_t s = lo + lane; s < hi; s += 32) pb += keys[s] != EMPTY_KEY ? 16ull : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if (lane == 0) atomicAdd(&a.ds->prof_bytes, pb + (w == 0 ? 44ull + 4ull * (unsigned long long)cx : 0ull));
    }
    warp_best(bj);
    warp_best(bl);
    if (lane == 0) {
        bs.gj[w] = bj.g; bs.cj[w] = bj.c; bs.kj[w] = bj.k;
        bs.gl[w] = bl.g; bs.cl[w] = bl.c; bs.kl[w] = bl.k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Best fj{0.0, -1, 0}, fl{0.0, -1, 0};
        for (int ww = 0; ww < EV_WARPS; ++ww) {
            if (better(bs.gj[ww], bs.cj[ww], fj.g, fj.c)) fj = Best{bs.gj[ww], bs.cj[ww], bs.kj[ww]};
            if (better(bs.gl[ww], bs.cl[ww], fl.g, fl.c)) fl = Best{bs.gl[ww], bs.cl[ww], bs.kl[ww]};
        }
        write_action(a, i, fj, fl, serial);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(EV_THREADS) k_huge_chunks(RunArgs a, int64_t bstart, int64_t bidx, int64_t cbase) {
    extern __shared__ int32_t hs_dyn[];   // HUGE_SH keys, HUGE_SH counts
    __shared__ BlockScratch bs;
    __shared__ int32_t bkey[EV_WARPS][32];
    __shared__ uint32_t bval[EV_WARPS][32];
    __shared__ unsigned s_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t ch = cbase + blockIdx.x;
    const int h = a.hub_chunk_h[ch];
    const int c = a.hub_chunk_c[ch];
    const int64_t p = a.hub_pos[h];
    const int32_t x = a.order[p];
    const int64_t t0 = a.hub_toff[h];
    const uint32_t cap = a.hub_tcap[h], hm = cap - 1;
    int32_t *keys = a.hkeys + t0;
    uint32_t *vals = a.hvals + t0;
    int32_t *list = reinterpret_cast<int32_t *>(a.hub_lb + t0);   // occupied slots, in order of arrival
    const int32_t cx = __ldcg(&a.nmem[x]);
    const int64_t beg = a.off[x] + (int64_t)c * HUGE_CHUNK;
    const int64_t end = min(a.off[x + 1], beg + HUGE_CHUNK);
    bool bad = false;
    if (c == 0) {
        const int32_t *rowx = a.mem + (int64_t)x * a.K;
        for (int j = threadIdx.x; j < cx; j += EV_THREADS)
            if (!hub_insert(keys, vals, hm, __ldcg(&rowx[j]), 0u, true, list, &a.hub_ncand[h])) bad = true;
    }
    // the chunk's memberships are first counted in a shared table, then each
    // distinct id goes to the hub's table once (entries the shared table
    // cannot take go there directly)
    // the shared table is sized for this chunk's entries (twice, pow2, at most HUGE_SH)
    __shared__ unsigned s_ent[EV_WARPS];
    int32_t ys[HUGE_ROUNDS], cys[HUGE_ROUNDS];
    unsigned ent = 0;
#pragma unroll
    for (int r = 0; r < HUGE_ROUNDS; ++r) {
        const int64_t q = beg + r * EV_THREADS + w * 32 + lane;
        ys[r] = q < end ? a.adj[q] : 0;
    }
#pragma unroll
    for (int r = 0; r < HUGE_ROUNDS; ++r) {
        const int64_t q = beg + r * EV_THREADS + w * 32 + lane;
        cys[r] = q < end ? __ldcg(&a.nmem[ys[r]]) : 0;
        ent += (unsigned)cys[r];
    }
    ent = __reduce_add_sync(FULL, ent);
    if (lane == 0) s_ent[w] = ent;
    __syncthreads();
    ent = 0;
    for (int k = 0; k < EV_WARPS; ++k) ent += s_ent[k];
    uint32_t SH = 256;
    while (SH < 2u * ent && SH < HUGE_SH) SH <<= 1;
    int32_t *skeys = hs_dyn;
    uint32_t *svals = reinterpret_cast<uint32_t *>(hs_dyn + HUGE_SH);
    for (uint32_t sl = threadIdx.x; sl < SH; sl += EV_THREADS) {
        skeys[sl] = EMPTY_KEY;
        svals[sl] = 0u;
    }
    __syncthreads();
    unsigned long long pb = 0;
#pragma unroll
    for (int r = 0; r < HUGE_ROUNDS; ++r) {
        const int32_t y = ys[r], cy = cys[r];
        if (beg + r * EV_THREADS + w * 32 + lane < end) pb += 8ull + 4ull * (unsigned long long)cy;
        const int32_t *rowy = a.mem + (int64_t)y * a.K;
        int4 r0, r1;
        row_head(rowy, cy, r0, r1);
        fill_flat_with(a, y, cy, r0, r1, [](int32_t) { return true; }, [&](int32_t C, uint32_t c) {
            if (!st_insert_bounded(skeys, svals, SH - 1, C, c, 32))
                if (!hub_insert(keys, vals, hm, C, c, false, list, &a.hub_ncand[h])) bad = true;
        });
    }
    __syncthreads();
    for (uint32_t s0 = threadIdx.x; s0 < SH; s0 += 4 * EV_THREADS) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t sl = s0 + u * EV_THREADS;
            const int32_t C = sl < SH ? skeys[sl] : EMPTY_KEY;
            if (C != EMPTY_KEY)
                if (!hub_insert(keys, vals, hm, C, svals[sl], false, list, &a.hub_ncand[h])) bad = true;
        }
    }
    if (bad) atomicOr(&a.ds->err, DERR_CHECK);   // the planned table bounds every entry: cannot happen
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if (lane == 0 && pb) atomicAdd(&a.ds->prof_bytes, pb);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.hub_done[h], 1u) == (unsigned)(a.hub_nch[h] - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();   // every chunk's insertions are visible from here on
    const uint32_t ncand = __ldcg(&a.hub_ncand[h]);
    if (ncand > HUGE_BIG_NCAND) {   // screened and evaluated by k_huge_screen / k_huge_eval
        if (threadIdx.x == 0) {
            const uint32_t ni = (ncand + HUGE_CAND_CHUNK - 1) / HUGE_CAND_CHUNK;
            const uint32_t base = atomicAdd(&a.hub_qctr[3 * bidx], ni);
            a.hub_item_base[h] = base;
            a.hub_nitems[h] = ni;
            a.hub_done[h] = 0u;
            for (uint32_t j = 0; j < ni; ++j) {
                a.hub_items[2 * (base + j)] = h;
                a.hub_items[2 * (base + j) + 1] = (int32_t)j;
            }
        }
        return;
    }
    // dense candidates: ids into the upper-bound area, counts over the slot
    // list; the table is cleared as it is read and then holds the bounds
    int32_t *ck = reinterpret_cast<int32_t *>(a.hub_ub + t0);
    uint32_t *cv = reinterpret_cast<uint32_t *>(list);
    for (uint32_t k = threadIdx.x; k < ncand; k += EV_THREADS) {
        const int32_t sl = __ldcg(&list[k]);
        ck[k] = __ldcg(&keys[sl]);
        cv[k] = __ldcg(&vals[sl]);
        keys[sl] = EMPTY_KEY;
        vals[sl] = 0u;
    }
    __syncthreads();
    huge_decide(a, (int)(p - bstart), a.deg[x], cx, ck, cv, reinterpret_cast<float *>(keys),
                reinterpret_cast<float *>(vals), ncand, bkey[w], bval[w], bs, queue_serial(a, bidx));
    for (uint32_t k = threadIdx.x; k < ncand; k += EV_THREADS) {   // the bounds' slots back to empty
        keys[k] = EMPTY_KEY;
        vals[k] = 0u;
    }
    if (threadIdx.x == 0) {
        a.hub_done[h] = 0u;
        a.hub_ncand[h] = 0u;
    }
}

struct EvalShared {
    int32_t hub[EV_WARPS];
    long long hub_bound[EV_WARPS];
    int nhub;
    BlockScratch bs;
    TeamScratch ts;
    int32_t bkey[EV_WARPS][32];
    uint32_t bval[EV_WARPS][32];
};

// Static data of a team's next node, fetched ahead of time (the node order,
// degrees, offsets and adjacency never change during a run); y0 is this
// warp's first adjacency chunk (chunk w_in of the node).
struct NodePrefetch {
    int32_t x, d, y0, valid;
    int64_t beg, end;
};

__device__ __forceinline__ void prefetch_node(const RunArgs &a, int64_t bstart, int32_t blen, int i, int w_in,
                                              NodePrefetch &pf) {
    const int lane = threadIdx.x & 31;
    pf.valid = 0;
    if (i >= blen) return;
    pf.x = a.order[bstart + i];
    pf.d = a.deg[pf.x];
    pf.beg = a.off[pf.x];
    pf.end = a.off[pf.x + 1];
    const int64_t p = pf.beg + w_in * 32 + lane;
    pf.y0 = p < pf.end ? a.adj[p] : 0;
    pf.valid = 1;
}

// One block evaluates queue nodes base .. base + EV_WARPS/T - 1, one team of T
// warps per node; nodes too large for a team's table are done afterwards by
// the whole block (with several passes over hash parts if needed).
template <int T>
__device__ void eval_group(const RunArgs &a, int64_t bstart, int32_t blen, int base, unsigned long long serial,
                           int32_t *s_keys, uint32_t *s_vals, float *s_ub, EvalShared &es,
                           const NodePrefetch *pf = nullptr) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tm = w / T, w_in = w % T;
    if (threadIdx.x == 0) es.nhub = 0;
    __syncthreads();
    const int i = base + tm;
    bool mine = i < blen;
    int32_t x = 0, d = 0;
    if (mine) {
        const bool have = pf && pf->valid;
        x = have ? pf->x : a.order[bstart + i];
        d = have ? pf->d : a.deg[x];
        mine = d <= a.huge_deg;   // hubs are evaluated by eval_huge
    }
    if (mine) {
        const bool have = pf && pf->valid;
        const int64_t beg = have ? pf->beg : a.off[x], end = have ? pf->end : a.off[x + 1];
        // exact number of entries the histogram will receive
        int32_t y0 = 0, c0 = 0;
        long long entries = 0;
        const int64_t first = beg + w_in * 32;
        for (int64_t p0 = first; p0 < end; p0 += T * 32) {
            const int64_t p = p0 + lane;
            int32_t y = 0, cy = 0;
            if (p < end) {
                y = (have && p0 == first) ? pf->y0 : a.adj[p];
                cy = __ldcg(&a.nmem[y]);
            }
            if (p0 == first) {
                y0 = y;
                c0 = cy;
            }
            entries += cy;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) entries += __shfl_xor_sync(FULL, entries, o);
        if constexpr (T > 1) {
            if (lane == 0) es.ts.part[w] = entries;
            team_sync<T>(tm);
            entries = 0;
            for (int k = 0; k < T; ++k) entries += es.ts.part[tm * T + k];
            team_sync<T>(tm);   // part[] is rewritten by the team's next node only after this
        }
        entries += __ldcg(&a.nmem[x]);
        if (d <= a.warp_max_deg && entries <= (long long)T * HW / 2) {
            eval_team<T>(a, i, x, d, beg, end, entries, y0, c0, s_keys + tm * T * HW, s_vals + tm * T * HW,
                         s_ub + tm * T * HW, es.bkey[w], es.bval[w], es.ts, tm, w_in, serial);
        } else if (w_in == 0 && lane == 0) {
            const int h = atomicAdd(&es.nhub, 1);
            es.hub[h] = i;
            es.hub_bound[h] = entries;
        }
    }
    __syncthreads();
    const int nh = es.nhub;
    for (int h = 0; h < nh; ++h) {
        const int ih = es.hub[h];
        const int32_t x = a.order[bstart + ih];
        eval_block(a, ih, x, (int64_t)es.hub_bound[h], s_keys, s_vals, s_ub, es.bkey[w], es.bval[w], es.bs, serial);
    }
    __syncthreads();
}

// Large queues: a resident grid whose warps take the queue's nodes one at a
// time from a counter, so that no warp waits at a block-wide barrier for the
// others' nodes.  Nodes whose histogram does not fit a warp's table are
// listed (position and entry count) for k_eval_blocks; hubs are left to
// k_huge_chunks.
__global__ void __launch_bounds__(EV_THREADS) k_eval_dyn(RunArgs a, int64_t bstart, int32_t blen, int64_t bidx,
                                                         uint32_t *ctr, int32_t *list, long long *lbound) {
    extern __shared__ int32_t ev_dyn[];   // per warp: HW keys, HW counts, HW upper and HW lower bounds
    __shared__ TeamScratch ts;
    __shared__ int32_t bkey[EV_WARPS][32];
    __shared__ uint32_t bval[EV_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *keys = ev_dyn + w * HW;
    uint32_t *vals = reinterpret_cast<uint32_t *>(ev_dyn + HB) + w * HW;
    float *ubs = reinterpret_cast<float *>(ev_dyn + 2 * HB) + w * HW;
    const unsigned long long serial = queue_serial(a, bidx);
    for (;;) {
        int i = 0;
        if (lane == 0) i = (int)atomicAdd(&ctr[0], 1u);
        i = __shfl_sync(FULL, i, 0);
        if (i >= blen) break;
        const int32_t x = a.order[bstart + i];
        const int32_t d = a.deg[x];
        if (d > a.huge_deg) continue;   // evaluated by k_huge_chunks
        const int64_t beg = a.off[x], end = a.off[x + 1];
        int32_t y0 = 0, c0 = 0;
        long long entries = 0;
        for (int64_t p0 = beg; p0 < end; p0 += 32) {
            const int64_t p = p0 + lane;
            int32_t y = 0, cy = 0;
            if (p < end) {
                y = a.adj[p];
                cy = __ldcg(&a.nmem[y]);
            }
            if (p0 == beg) {
                y0 = y;
                c0 = cy;
            }
            entries += cy;
        }
        entries = __reduce_add_sync(FULL, (unsigned)entries);
        entries += __ldcg(&a.nmem[x]);
        if (d <= a.warp_max_deg && entries <= HW / 2) {
            eval_team<1>(a, i, x, d, beg, end, entries, y0, c0, keys, vals, ubs, bkey[w], bval[w], ts, w, 0, serial);
        } else if (lane == 0) {
            const uint32_t k = atomicAdd(&ctr[1], 1u);
            list[k] = i;
            lbound[k] = entries;
        }
    }
}

// Teams of T warps take listed nodes (queue position and entry count) from a
// counter; a node whose entries exceed the team's table goes on to the next
// list.  in_ctr: [count, next]; out_ctr: [count].
template <int T>
__global__ void __launch_bounds__(EV_THREADS, 3) k_eval_tdyn(RunArgs a, int64_t bstart, int64_t bidx, uint32_t *in_ctr,
                                                          const int32_t *in_list, const long long *in_bound,
                                                          uint32_t *out_ctr, int32_t *out_list,
                                                          long long *out_bound) {
    extern __shared__ int32_t ev_dyn[];
    __shared__ TeamScratch ts;
    __shared__ int32_t bkey[EV_WARPS][32];
    __shared__ uint32_t bval[EV_WARPS][32];
    __shared__ uint32_t s_k[EV_WARPS / T];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tm = w / T, w_in = w % T;
    int32_t *keys = ev_dyn + tm * T * HW;
    uint32_t *vals = reinterpret_cast<uint32_t *>(ev_dyn + HB) + tm * T * HW;
    float *ubs = reinterpret_cast<float *>(ev_dyn + 2 * HB) + tm * T * HW;
    const uint32_t count = __ldcg(&in_ctr[0]);
    const unsigned long long serial = queue_serial(a, bidx);
    for (;;) {
        if (w_in == 0 && lane == 0) s_k[tm] = atomicAdd(&in_ctr[1], 1u);
        team_sync<T>(tm);
        const uint32_t k = s_k[tm];
        team_sync<T>(tm);   // the slot is rewritten only after every warp of the team has read it
        if (k >= count) break;
        const int i = in_list[k];
        const long long entries = in_bound[k];
        const int32_t x = a.order[bstart + i];
        const int32_t d = a.deg[x];
        if (entries > (long long)T * HW / 2) {
            if (w_in == 0 && lane == 0) {
                const uint32_t o = atomicAdd(&out_ctr[0], 1u);
                out_list[o] = i;
                out_bound[o] = entries;
            }
            continue;
        }
        const int64_t beg = a.off[x], end = a.off[x + 1];
        const int64_t p = beg + w_in * 32 + lane;
        const int32_t y0 = p < end ? a.adj[p] : 0;
        const int32_t c0 = p < end ? __ldcg(&a.nmem[y0]) : 0;
        eval_team<T>(a, i, x, d, beg, end, entries, y0, c0, keys, vals, ubs, bkey[w], bval[w], ts, tm, w_in, serial);
    }
}

// The nodes k_eval_dyn listed, one block each (shared-memory table, several
// passes over hash parts when it does not fit).
__global__ void __launch_bounds__(EV_THREADS) k_eval_blocks(RunArgs a, int64_t bstart, int64_t bidx,
                                                            const uint32_t *cnt, const int32_t *list,
                                                            const long long *lbound) {
    extern __shared__ int32_t ev_dyn[];
    __shared__ BlockScratch bs;
    __shared__ int32_t bkey[EV_WARPS][32];
    __shared__ uint32_t bval[EV_WARPS][32];
    const int w = threadIdx.x >> 5;
    const uint32_t count = __ldcg(cnt);
    const unsigned long long serial = queue_serial(a, bidx);
    for (uint32_t k = blockIdx.x; k < count; k += gridDim.x) {
        const int i = list[k];
        const int32_t x = a.order[bstart + i];
        eval_block(a, i, x, (int64_t)lbound[k], ev_dyn, reinterpret_cast<uint32_t *>(ev_dyn + HB),
                   reinterpret_cast<float *>(ev_dyn + 2 * HB), bkey[w], bval[w], bs, serial);
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel of the stream finishes;
// it reads only static data (node order, degrees, adjacency) before
// pdl_wait, which returns once the previous kernel has completed and its
// writes are visible.  pdl_trigger lets the next kernel be scheduled early.
// Both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <int T>
__global__ void __launch_bounds__(EV_THREADS, 3) k_eval(RunArgs a, int64_t bstart, int32_t blen, int64_t bidx) {
    extern __shared__ int32_t ev_dyn[];   // HB keys, HB counts, HB upper and HB lower screen bounds
    __shared__ EvalShared es;
    // the team's node and its first adjacency chunk: static, read before the wait
    const int w = threadIdx.x >> 5;
    NodePrefetch pf;
    prefetch_node(a, bstart, blen, (int)(blockIdx.x * (EV_WARPS / T)) + w / T, w % T, pf);
    pdl_trigger();
    pdl_wait();
    eval_group<T>(a, bstart, blen, blockIdx.x * (EV_WARPS / T), queue_serial(a, bidx), ev_dyn,
                  reinterpret_cast<uint32_t *>(ev_dyn + HB), reinterpret_cast<float *>(ev_dyn + 2 * HB), es, &pf);
}

// ---------------------------------------------------------------------------
// a8: bulk apply of one queue.  For a joiner x of C (k = |N(x) & C| before the
// queue), the internal edge sum 2m_C grows by 2k + (joiner neighbours of x
// also joining C) - 2 (neighbours of x leaving C); for a leaver it shrinks by
// 2k - (neighbours of x also leaving C).  Summed over the queue this is the
// exact change of 2m_C; the neighbour scan is needed only when another action
// of the same queue targets C.  Integer atomics: order-independent.
// ---------------------------------------------------------------------------
__device__ void apply_node(const RunArgs &a, int64_t bstart, int32_t blen, int64_t i, unsigned long long serial,
                           unsigned long long &nj, unsigned long long &nl) {
    const int lane = threadIdx.x & 31;
    const int32_t j = __ldcg(&a.act[i]), l = __ldcg(&a.act[a.qcap + i]);
    if (j < 0 && l < 0) {
        if (a.profile && lane == 0) atomicAdd(&a.ds->prof_bytes, 8ull);
        return;
    }
    const int32_t x = a.order[bstart + i];
    // neighbours acting on the same community in this queue (static adjacency
    // and positions; only in-queue neighbours' actions are read)
    (void)serial;
    const bool need_j = j >= 0;
    const bool need_l = l >= 0;
    int jj = 0, jl = 0, ll = 0;
    if (need_j || need_l) {
        for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
            const int32_t y = a.adj[p];
            const int64_t py = a.pos[y];
            if (py >= bstart && py < bstart + blen) {
                const int64_t iy = py - bstart;
                const int32_t aj = __ldcg(&a.act[iy]), al = __ldcg(&a.act[a.qcap + iy]);
                if (need_j) {
                    jj += aj == j;
                    jl += al == j;
                }
                if (need_l) ll += al == l;
            }
        }
        jj = __reduce_add_sync(FULL, jj);
        jl = __reduce_add_sync(FULL, jl);
        ll = __reduce_add_sync(FULL, ll);
    }
    const int32_t d = a.deg[x];
    int32_t *row = a.mem + (int64_t)x * a.K;
    const int32_t c = __ldcg(&a.nmem[x]);
    int32_t c_new = c;
    if (c <= 32) {
        // whole row in one coalesced load; leave l, insert j, keep ascending order
        const int32_t v = lane < c ? __ldcg(&row[lane]) : 0;
        const bool keep = lane < c && v != l;
        const unsigned km = __ballot_sync(FULL, keep);
        const unsigned lt = lanemask_lt();
        const int kept = __popc(km);
        int ins = kept;   // slot of j among the kept entries
        if (j >= 0) ins = __popc(__ballot_sync(FULL, keep && v < j));
        if (j >= 0 && kept >= a.K) {
            if (lane == 0) atomicOr(&a.ds->err, DERR_CAPACITY);
        } else {
            if (keep) {
                const int dst = __popc(km & lt);
                row[dst + ((j >= 0 && dst >= ins) ? 1 : 0)] = v;
            }
            if (j >= 0 && lane == 0) row[ins] = j;
            c_new = kept + (j >= 0 ? 1 : 0);
        }
    } else if (lane == 0) {
        int32_t cc = c;
        if (l >= 0) {
            int32_t o = 0;
            for (int32_t s = 0; s < cc; ++s) {
                const int32_t v = __ldcg(&row[s]);
                if (v != l) row[o++] = v;
            }
            cc = o;
        }
        if (j >= 0) {
            if (cc >= a.K) {
                atomicOr(&a.ds->err, DERR_CAPACITY);
            } else {
                int32_t s = cc;
                while (s > 0) {
                    const int32_t v = __ldcg(&row[s - 1]);
                    if (v <= j) break;
                    row[s] = v;
                    --s;
                }
                row[s] = j;
                ++cc;
            }
        }
        c_new = cc;
    }
    if (lane == 0) {
        if (l >= 0) {
            const int32_t kl = __ldcg(&a.act[3 * a.qcap + i]);
            atomicAdd(&a.comm[l].n, -1);
            atomicAdd(&a.comm[l].vol, (uint32_t)(-d));
            atomicAdd(&a.comm[l].m2, (uint32_t)(-2 * kl + ll));
            ++nl;
        }
        if (j >= 0) {
            const int32_t kj = __ldcg(&a.act[2 * a.qcap + i]);
            atomicAdd(&a.comm[j].n, 1);
            atomicAdd(&a.comm[j].vol, (uint32_t)d);
            atomicAdd(&a.comm[j].m2, (uint32_t)(2 * kj + jj - 2 * jl));
            ++nj;
        }
        a.nmem[x] = c_new;
        if (a.profile) {
            const unsigned long long nb_scan = (need_j || need_l) ? 16ull * (unsigned long long)(a.off[x + 1] - a.off[x]) : 0ull;
            atomicAdd(&a.ds->prof_bytes, 24ull + 4ull * (unsigned long long)c + 12ull * ((j >= 0) + (l >= 0)) + nb_scan);
        }
    }
}

__device__ __forceinline__ void flush_counts(const RunArgs &a, unsigned long long nj, unsigned long long nl) {
    __shared__ unsigned long long s_j, s_l;
    if (threadIdx.x == 0) {
        s_j = 0;
        s_l = 0;
    }
    __syncthreads();
    if (nj) atomicAdd(&s_j, nj);
    if (nl) atomicAdd(&s_l, nl);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_j) atomicAdd(&a.ds->joins, s_j);
        if (s_l) atomicAdd(&a.ds->leaves, s_l);
    }
}

__global__ void __launch_bounds__(AP_THREADS) k_apply(RunArgs a, int64_t bstart, int32_t blen, int64_t bidx) {
    pdl_trigger();
    pdl_wait();   // the queue's actions come from the kernel before
    const unsigned long long serial = queue_serial(a, bidx);
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long nj = 0, nl = 0;
    if (i < blen) apply_node(a, bstart, blen, i, serial, nj, nl);
    flush_counts(a, nj, nl);
}

// ---------------------------------------------------------------------------
// a7/a8 with the paper's gain.  The gain of x joining (leaving) C is the
// change of WCC-hat(P) (Node Changes: Joining / Leaving a Community, with
// the WCC-hat sum equations): C's members' terms after the move -- new size
// and internal edge count, and for x's neighbours deg(y,C) one higher (lower)
// -- and x's own term, less C's terms before it, summed exactly and rounded
// once.  With deg(y,C) kept per membership (kmem, beside the rows) and the
// members of C reachable through a per-iteration index (the members at the
// iteration's start, cm_off/cm_node, plus a list of the iteration's joiners),
// the exact value costs a pass over C.  It is only needed near ties: every
// candidate first gets a bracket from per-community sums.  Writing
//     g_y(nu) = C(k_y,2) d_y / (C(d_y,2) (nu - 1 + d_y - k_y)),
// a member's estimator at size nu and internal edges m is (2m/(nu(nu-1))/cc)
// g_y(nu), so in real arithmetic
//   join:  gain = p'/cc [F(n+1) + sum_{y in N(x)&C} h+_y + g_x(n+1)] - p/cc F(n)
//   leave: gain = p'/cc [F(n-1) - g_x(n-1) + sum_{y in N(x)&C} h-_y] - p/cc F(n)
// with F(nu) = sum_{y in C} g_y(nu) (litF: the three sums per community and
// the factors p/cc F(n), 1/((n+1) n cc), 1/((n-1)(n-2) cc), kept current
// after every queue for the communities it touched), p, p' the
// densities before and after, and h+_y = g_y(n+1; k_y+1) - g_y(n+1; k_y),
// h-_y = g_y(n-1; k_y-1) - g_y(n-1; k_y) in closed forms free of
// cancellation.  Every term is non-negative except the h-.  The F sums are
// taken in FP64 and stored, with the factors, as floats; the corrections and
// g_x are FP32 and summed in FP32; the bracket itself is evaluated in FP32
// (GB300's FP64 pipe is the scarce one).  The exact value of the rounded
// terms and the computed value both lie within
//   E = (1.5e-6 + (n + k + 64) 2.3e-16) M + (k + 16) 1.2e-7 p'/cc (|sum h| + g_x)
// of the real one (M: the same expression with every term's magnitude; the
// FP64 sums are at most 2n + k + 40 roundings of non-negative terms, the
// float path about ten roundings of 2^-24 on terms bounded by M (1.5e-6 is
// 25 of them), a correction about ten roundings plus one per addition --
// every count taken about twice over).  Per kind, candidates whose upper end cannot reach
// the best lower end (or 0) are dropped; one surviving candidate with a
// positive lower end is the answer; otherwise the survivors' gains are
// computed exactly (a signed integer superaccumulator over C's members) and
// compared.  The margin also covers one rounding of the compared values, so
// a dropped candidate can neither win nor tie.
// ---------------------------------------------------------------------------
constexpr int LW = 512;                            // table slots of one warp
constexpr int LB_SLOTS = EV_WARPS * LW;            // table slots of a block
constexpr uint32_t SURV_FLAG = 0x40000000u;        // candidate survives the bracket test
constexpr uint32_t CNT_MASK = 0x3fffffffu;
constexpr size_t LIT_SMEM = (size_t)LB_SLOTS * 16 + (size_t)EV_WARPS * SACC_CHUNKS * 8;
constexpr int LIT_PART_ENTRIES = 1024;             // entries per pass of a multi-pass node

// Signed exact accumulation: like sacc_add, with negative values added as
// negated digits (64-bit words wrap, so each word holds a signed sum).
__device__ __forceinline__ void ssacc_add(unsigned long long *acc, double v) {
    if (v == 0.0) return;
    const bool neg = v < 0.0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    unsigned long long mant = b & 0xfffffffffffffull;
    int p;
    if (e == 0) {
        p = 0;
    } else {
        mant |= 1ull << 52;
        p = (int)e - 1;
    }
    const int c = p >> 5, sh = p & 31;
    const unsigned long long lo = mant << sh;
    const unsigned long long hi = sh ? (mant >> (64 - sh)) : 0ull;
    const unsigned long long d[3] = {lo & 0xffffffffull, lo >> 32, hi};
#pragma unroll
    for (int t = 0; t < 3; ++t)
        if (d[t]) atomicAdd(&acc[c + t], neg ? (unsigned long long)(-(long long)d[t]) : d[t]);
}

// The double nearest (ties to even) to the non-negative value held in 32-bit
// digits dg (bit 0 = 2^-1074).
__device__ inline double round_digits(const uint32_t *dg) {
    int top = -1;
    for (int i = SACC_CHUNKS - 1; i >= 0; --i)
        if (dg[i]) {
            top = i;
            break;
        }
    if (top < 0) return 0.0;
    int P = 32 * top + (31 - __clz((int)dg[top]));
    auto bit = [&](int q) -> unsigned long long {
        return q < 0 ? 0ull : (unsigned long long)((dg[q >> 5] >> (q & 31)) & 1u);
    };
    if (P <= 52) {
        unsigned long long v = 0;
        for (int q = P; q >= 0; --q) v = (v << 1) | bit(q);
        return __longlong_as_double((long long)v);
    }
    unsigned long long mant = 0;
    for (int q = P; q >= P - 52; --q) mant = (mant << 1) | bit(q);
    const int r = P - 53;
    const bool round_bit = bit(r) != 0;
    bool sticky = false;
    for (int i = 0; i < (r >> 5) && !sticky; ++i) sticky = dg[i] != 0u;
    if (!sticky && (r & 31)) sticky = (dg[r >> 5] & ((1u << (r & 31)) - 1u)) != 0u;
    if (round_bit && (sticky || (mant & 1ull))) ++mant;
    if (mant == (1ull << 53)) {
        mant >>= 1;
        ++P;
    }
    const long long biased = (long long)P - 51;
    if (biased >= 2047) return __longlong_as_double(0x7ff0000000000000ll);
    return __longlong_as_double((long long)(((unsigned long long)biased << 52) | (mant & 0xfffffffffffffull)));
}

// Round the signed accumulated value to the nearest double and clear the
// accumulator.  One thread.
__device__ inline double ssacc_round_and_clear(unsigned long long *acc) {
    uint32_t dg[SACC_CHUNKS];
    long long carry = 0;
    for (int i = 0; i < SACC_CHUNKS; ++i) {
        const long long v = (long long)acc[i] + carry;
        acc[i] = 0ull;
        const uint32_t low = (uint32_t)(unsigned long long)v;
        dg[i] = low;
        carry = (v - (long long)low) / 4294967296ll;   // exact: v - low is a multiple of 2^32
    }
    const bool neg = carry < 0;   // the value is (digits) - 2^(32 * SACC_CHUNKS)
    if (neg) {
        unsigned long long c = 1;
        for (int i = 0; i < SACC_CHUNKS; ++i) {
            const unsigned long long t = (unsigned long long)(uint32_t)~dg[i] + c;
            dg[i] = (uint32_t)t;
            c = t >> 32;
        }
    }
    const double r = round_digits(dg);
    return neg ? -r : r;
}

// Bounds-checked mode (lf_options.debug_checks): a value read from device
// state that is out of its range sets DERR_CHECK and the access is skipped
// (never a trap; the call then fails with a message).
__device__ __forceinline__ bool dbg_ok(const RunArgs &a, bool ok) {
    if (!a.debug || ok) return true;
    atomicOr(&a.ds->err, DERR_CHECK);
    return false;
}

// Position of C in a row of cnt ascending ids, -1 if absent.
__device__ __forceinline__ int row_find(const int32_t *row, int32_t cnt, int32_t C) {
    int lo = 0, hi = cnt - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = __ldcg(&row[mid]);
        if (v == C) return mid;
        if (v < C) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// y in the ascending adjacency list adj[beg, end)?
__device__ __forceinline__ bool adj_has(const int32_t *adj, int64_t beg, int64_t end, int32_t y) {
    int64_t lo = beg, hi = end - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = adj[mid];
        if (v == y) return true;
        if (v < y) lo = mid + 1;
        else hi = mid - 1;
    }
    return false;
}

// g_y(nu) = C(k,2) d / (C(d,2) (nu - 1 + d - k)): a member's estimator
// without the factor (2m / (nu (nu - 1))) / cc.  Zero where the estimator is
// (k < 2, or d < 2 so that E[t(x,V)] = 0).
__device__ __forceinline__ double lit_g(int64_t k, int64_t d, int64_t nu) {
    if (k < 2 || d < 2) return 0.0;
    const int64_t den = nu - 1 + d - k;
    if (den <= 0) return 0.0;
    const double bk = 0.5 * ((double)k * (double)(k - 1));
    const double bd = 0.5 * ((double)d * (double)(d - 1));
    return (bk * (double)d) / (bd * (double)den);
}

// The neighbours' corrections:
//   h+ = g(n+1; k+1) - g(n+1; k) = d (k D + C(k,2)) / (C(d,2) D (D-1)), D = n + d - k
//        (a neighbour y of a joining x; y is not x, so k <= d - 1 and D - 1 >= n >= 1),
//   h- = g(n-1; k-1) - g(n-1; k) = -d (C(k-1,2) + (k-1)(D+1)) / (C(d,2) D (D+1)),
//        D = n - 2 + d - k (used only when n - 1 >= 2, so D >= 1),
// and x's own g, in FP32 (about ten roundings each, relative error
// < 16 x 2^-24; a sum of k of them adds k roundings): used only in the
// bracket, whose bound E carries a term for them.
__device__ __forceinline__ float lit_h_join32(int64_t k, int64_t d, int64_t n) {
    if (d < 2 || k < 1) return 0.f;
    const float D = (float)(n + d - k), kf = (float)k, df = (float)d;
    const float bk = 0.5f * (kf * (kf - 1.f));
    const float bd = 0.5f * (df * (df - 1.f));
    return (df * (kf * D + bk)) / (bd * (D * (D - 1.f)));
}

__device__ __forceinline__ float lit_h_leave32(int64_t k, int64_t d, int64_t n) {
    if (d < 2 || k < 2 || n < 3) return 0.f;
    const float D = (float)(n - 2 + d - k), kf = (float)k, df = (float)d;
    const float bk1 = 0.5f * ((kf - 1.f) * (kf - 2.f));
    const float bd = 0.5f * (df * (df - 1.f));
    return -(df * (bk1 + (kf - 1.f) * (D + 1.f))) / (bd * (D * (D + 1.f)));
}

__device__ __forceinline__ float lit_g32(int64_t k, int64_t d, int64_t nu) {
    if (k < 2 || d < 2) return 0.f;
    const int64_t den = nu - 1 + d - k;
    if (den <= 0) return 0.f;
    const float kf = (float)k, df = (float)d;
    return (0.5f * (kf * (kf - 1.f)) * df) / (0.5f * (df * (df - 1.f)) * (float)den);
}

// Bracket of one candidate: FP64 value X of the expression above and a bound
// E on its distance from the exactly summed, once rounded gain.
__device__ __forceinline__ void lit_screen(const RunArgs &a, int32_t C, uint32_t v, int32_t d, float Hs, float &X,
                                           float &E) {
    // per community (k_lit_fsum, rounded to float): F(n-1), F(n+1),
    // WCC-hat(C) = p/cc F(n), 1/((n+1) n cc), 1/((n-1)(n-2) cc)
    const bool own = (v & OWN_FLAG) != 0;
    const int64_t k = (int64_t)(v & CNT_MASK);
    const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
    const int64_t n = r.x;
    const float m2 = (float)(uint32_t)r.y;
    const float *fp = a.litF + 8 * (int64_t)C;
    const float4 f = __ldcg(reinterpret_cast<const float4 *>(fp));
    float A, S1, Sm, Eh;
    if (!own) {
        A = (m2 + 2.f * (float)k) * f.w;
        const float gx = lit_g32(k, d, n + 1);
        S1 = (f.y + Hs) + gx;
        Sm = S1;
        Eh = Hs + gx;
    } else {
        A = (m2 - 2.f * (float)k) * __ldcg(&fp[4]);
        const float gx = A != 0.f ? lit_g32(k, d, n - 1) : 0.f;
        S1 = (f.x - gx) + Hs;
        Sm = (f.x + gx) - Hs;
        Eh = gx - Hs;
    }
    X = A * S1 - f.z;
    const float M = A * Sm + f.z;
    E = (1.5e-6f + ((float)(n + k) + 64.f) * 2.3e-16f) * M + ((float)k + 16.f) * 1.2e-7f * (A * Eh) + 1e-30f;
    if (!isfinite(X) || !isfinite(E)) {   // out of float range: only the exact sum can decide
        X = 0.f;
        E = INFINITY;
    }
}

// The (neighbour, membership) entries of neighbours [qb, qe) of one warp:
// 32 neighbours at a time, their entries laid end to end over the lanes
// (lane e of a round takes entry e, found by a shuffle search over the
// prefix sums of the neighbours' membership counts), so a warp's work does
// not depend on how the entries spread over its neighbours.  fn(C, ky, dy,
// n): the community, deg(y,C), deg(y) and C's size before the queue.
// Every lane of the warp must call this with the same range.
template <typename Fn>
__device__ __forceinline__ void lit_warp_entries(const RunArgs &a, int64_t qb, int64_t qe, unsigned long long &pb,
                                                 bool count_bytes, Fn &&fn) {
    const int lane = threadIdx.x & 31;
    for (int64_t q0 = qb; q0 < qe; q0 += 32) {
        const int64_t q = q0 + lane;
        int32_t y = 0, cy = 0, dy = 0;
        if (q < qe) {
            y = a.adj[q];
            if (dbg_ok(a, y >= 0 && y < a.nnodes)) {
                cy = __ldcg(&a.nmem[y]);
                if (!dbg_ok(a, cy >= 0 && cy <= a.K)) cy = 0;
                dy = a.deg[y];
                if (count_bytes) pb += 12ull + 8ull * (unsigned long long)cy;
            }
        }
        int inc = cy;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            int j = 0;   // first lane whose inclusive prefix exceeds e
#pragma unroll
            for (int b = 16; b > 0; b >>= 1)
                if (__shfl_sync(FULL, inc, j + b - 1) <= e) j += b;
            const int32_t yj = __shfl_sync(FULL, y, j);
            const int32_t first = __shfl_sync(FULL, inc - cy, j);
            const int32_t dj = __shfl_sync(FULL, dy, j);
            if (e < total) {
                const int64_t rb = (int64_t)yj * a.K + (e - first);
                const int32_t C = __ldcg(&a.mem[rb]);
                const int32_t ky = __ldcg(&a.kmem[rb]);
                if (dbg_ok(a, C >= 0 && C < a.nnodes)) fn(C, (int64_t)ky, (int64_t)dj, (int64_t)__ldcg(&a.comm[C].n));
            }
        }
    }
}

// Every entry of C's member index -- the members at the iteration's start
// and its joiners since, in C's region and, past its capacity, in C's list --
// handed to f, entry t to thread `tid` of `nthreads` when t % nthreads == tid.
// Entries of nodes that left C since are included (f checks the row).
template <typename F>
__device__ __forceinline__ void lit_members(const RunArgs &a, int32_t C, int tid, int nthreads, F &&f) {
    const int64_t b0 = (int64_t)a.cm_off[C], cap = (int64_t)a.cm_off[C + 1] - b0;
    const int64_t used = (int64_t)__ldcg(&a.cm_cnt[C]);
    const int64_t b1 = b0 + (used < cap ? used : cap);
    for (int64_t p = b0 + tid; p < b1; p += nthreads) f(__ldcg(&a.cm_node[p]));
    if (used > cap) {
        int idx = 0;
        for (int32_t e = __ldcg(&a.jl_head[C]); e >= 0; e = __ldcg(&a.jl_next[e]), ++idx)
            if (idx % nthreads == tid) f(__ldcg(&a.jl_node[e]));
    }
}

// Whether y is a neighbour of x (adjacency [xb, xe), ascending): without a
// fence a binary search in global memory; with one (fence[j] = adj[xb + j
// step], nf entries, in shared memory) the search first finds the segment
// between two fence entries, then searches only that segment.
__device__ __forceinline__ bool adj_has_fenced(const int32_t *adj, int64_t xb, int64_t xe, const int32_t *fence,
                                               int nf, int64_t step, int32_t y) {
    if (!fence) return adj_has(adj, xb, xe, y);
    int lo = 0, hi = nf;   // the last j with fence[j] <= y
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fence[mid] <= y) lo = mid;
        else hi = mid;
    }
    if (fence[lo] > y) return false;
    const int64_t b = xb + (int64_t)lo * step;
    return adj_has(adj, b, min(xe, b + step), y);
}

// The exact gain of x joining (own = false) or leaving C: every member's term
// after and before, x's own term, added into a signed superaccumulator (acc:
// the warp's, zero on entry and on exit).  One warp (tid, nthreads = lane,
// 32), or a whole block (threadIdx.x, blockDim.x; each warp adds into its own
// accumulator, acc + warp x SACC_CHUNKS, and the words are summed before the
// one rounding).
__device__ double lit_exact_gain(const RunArgs &a, int32_t x, int32_t d, int32_t C, bool own, int64_t k,
                                 unsigned long long *acc, const int32_t *fence = nullptr, int nf = 0,
                                 int64_t step = 0, bool block = false, double *s_g = nullptr) {
    const int lane = threadIdx.x & 31;
    const int tid = block ? (int)threadIdx.x : lane, nthreads = block ? (int)blockDim.x : 32;
    unsigned long long *wacc = block ? acc + (threadIdx.x >> 5) * SACC_CHUNKS : acc;
    const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
    const int64_t n0 = r.x;
    const uint32_t m20 = (uint32_t)r.y;
    const double cc = a.gcc ? a.gcc[r.w] : a.cc;
    const int64_t n1 = own ? n0 - 1 : n0 + 1;
    const uint32_t m21 = own ? m20 - (uint32_t)(2 * k) : m20 + (uint32_t)(2 * k);
    const int64_t xb = a.off[x], xe = a.off[x + 1];
    auto member = [&](int32_t y) {
        if (y == x) return;
        if (!dbg_ok(a, y >= 0 && y < a.nnodes)) return;
        const int32_t cy = __ldcg(&a.nmem[y]);
        if (!dbg_ok(a, cy >= 0 && cy <= a.K)) return;
        const int s = row_find(a.mem + (int64_t)y * a.K, cy, C);
        if (s < 0) return;   // left C earlier in this iteration
        const int64_t ky = __ldcg(&a.kmem[(int64_t)y * a.K + s]);
        const int64_t dy = a.deg[y];
        if (!dbg_ok(a, ky >= 0 && ky <= dy)) return;
        const int64_t k1 = adj_has_fenced(a.adj, xb, xe, fence, nf, step, y) ? (own ? ky - 1 : ky + 1) : ky;
        ssacc_add(wacc, wcchat_member(k1, dy, n1, m21, cc));
        ssacc_add(wacc, -wcchat_member(ky, dy, n0, m20, cc));
    };
    lit_members(a, C, tid, nthreads, member);
    if (tid == 0) ssacc_add(wacc, own ? -wcchat_member(k, d, n0, m20, cc) : wcchat_member(k, d, n1, m21, cc));
    if (!block) {
        __syncwarp();
        double g = 0.0;
        if (lane == 0) g = ssacc_round_and_clear(acc);
        __syncwarp();
        return __shfl_sync(FULL, g, 0);
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    for (int c = threadIdx.x; c < SACC_CHUNKS; c += blockDim.x) {
        unsigned long long t = acc[c];
        for (int w2 = 1; w2 < nw; ++w2) {
            t += acc[w2 * SACC_CHUNKS + c];   // words wrap: the sum of the warps' signed sums
            acc[w2 * SACC_CHUNKS + c] = 0ull;
        }
        acc[c] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *s_g = ssacc_round_and_clear(acc);
    __syncthreads();
    const double g = *s_g;
    __syncthreads();
    return g;
}

// Per-warp values a literal team exchanges.
struct LitScratch {
    float lbj[EV_WARPS], lbl[EV_WARPS];
    int cj[EV_WARPS], cl[EV_WARPS];
    int32_t sCj[EV_WARPS], sCl[EV_WARPS], skj[EV_WARPS], skl[EV_WARPS];
    float sLj[EV_WARPS], sLl[EV_WARPS];
    double bgj[EV_WARPS], bgl[EV_WARPS];
    int32_t bcj[EV_WARPS], bcl[EV_WARPS], bkj[EV_WARPS], bkl[EV_WARPS];
    int flag[EV_WARPS];
    long long part[EV_WARPS];
};

struct LitNode {
    int32_t x, d, cx;
    int64_t beg, end;
};

// Open-addressing insert of one neighbour entry: the slot of key (claimed if
// new) with its count raised by one, or -1 if the table is full.
__device__ __forceinline__ int lit_insert(int32_t *keys, uint32_t *vals, uint32_t hm, int32_t key) {
    uint32_t h = hash32((uint32_t)key) & hm;
    for (uint32_t probe = 0; probe <= hm; ++probe) {
        const int32_t prev = atomicCAS(&keys[h], EMPTY_KEY, key);
        if (prev == EMPTY_KEY || prev == key) {
            atomicAdd(&vals[h], 1u);
            return (int)h;
        }
        h = (h + 1) & hm;
    }
    return -1;
}

// One pass over the node's candidates of part p (of P): the table gets x's
// own communities (own flag), then every neighbour membership (y, C) adds
// one to C's count and its correction h(y) (by C's size before the queue and
// whether C is x's own) to C's sum (dv); then each candidate's bracket:
// dv <- X, aux <- E (as a float rounded up).  Per lane: the largest lower
// ends of the two kinds.  Returns false (team-wide) if the table overflowed.
template <int T>
__device__ bool lit_pass(const RunArgs &a, const LitNode &ln, int P, int p, int32_t *keys, uint32_t *vals,
                         int32_t *aux, float *dv, uint32_t H, LitScratch &ls, int tm, int w_in, float &lbj,
                         float &lbl, unsigned long long &pb, bool count_bytes) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tl = w_in * 32 + lane;
    constexpr int NT = T * 32;
    const uint32_t hm = H - 1;
    float *hs = reinterpret_cast<float *>(aux);   // corrections, then (as bits) the bound E
    for (uint32_t s = tl; s < H; s += NT) {
        keys[s] = EMPTY_KEY;
        vals[s] = 0u;
        hs[s] = 0.f;
    }
    team_sync<T>(tm);
    bool ok = true;
    const int32_t *rowx = a.mem + (int64_t)ln.x * a.K;
    for (int j = tl; j < ln.cx; j += NT) {
        const int32_t C = __ldcg(&rowx[j]);
        if (P == 1 || (int)part_of(C, P) == p) ok &= ht_insert(keys, vals, hm, C, 0u, true);
    }
    team_sync<T>(tm);
    {   // each warp of the team takes a contiguous share of the neighbours
        const int64_t deg = ln.end - ln.beg, per = (deg + T - 1) / T;
        const int64_t qb = ln.beg + min(deg, (int64_t)w_in * per), qe = ln.beg + min(deg, (int64_t)(w_in + 1) * per);
        lit_warp_entries(a, qb, qe, pb, count_bytes, [&](int32_t C, int64_t ky, int64_t dy, int64_t n) {
            if (P > 1 && (int)part_of(C, P) != p) return;
            if (!dbg_ok(a, ky >= 0 && ky <= dy)) return;
            const int slot = lit_insert(keys, vals, hm, C);
            if (slot < 0) {
                ok = false;
                return;
            }
            const float h = (vals[slot] & OWN_FLAG) ? lit_h_leave32(ky, dy, n) : lit_h_join32(ky, dy, n);
            if (h != 0.f) atomicAdd(&hs[slot], h);
        });
    }
    // a full table: the whole team starts over with more parts
    if constexpr (T > 1) {
        const bool all = __all_sync(FULL, ok);
        if (lane == 0) ls.flag[w] = all ? 1 : 0;
        team_sync<T>(tm);
        for (int k2 = 0; k2 < T; ++k2) ok &= ls.flag[tm * T + k2] != 0;
        team_sync<T>(tm);
    } else {
        ok = __all_sync(FULL, ok);
    }
    if (!ok) return false;
    for (uint32_t s = tl; s < H; s += NT) {
        const int32_t C = keys[s];
        if (C == EMPTY_KEY) continue;
        const uint32_t v = vals[s];
        float X, E;
        lit_screen(a, C, v, ln.d, hs[s], X, E);
        dv[s] = X;
        aux[s] = __float_as_int(E);
        const float L = X - E;
        if (v & OWN_FLAG) lbl = fmaxf(lbl, L);
        else lbj = fmaxf(lbj, L);
        if (count_bytes) {
            pb += 40ull;
            atomicAdd(&a.ds->prof_cands, 1ull);
        }
    }
    team_sync<T>(tm);
    return true;
}

// The largest value of a team (through ls.lbj/lbl slots of its warps).
template <int T>
__device__ __forceinline__ void team_max2(LitScratch &ls, int tm, float &x1, float &x2) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x1 = warp_max_f(x1);
    x2 = warp_max_f(x2);
    if constexpr (T > 1) {
        if (lane == 0) {
            ls.lbj[w] = x1;
            ls.lbl[w] = x2;
        }
        team_sync<T>(tm);
        for (int k2 = 0; k2 < T; ++k2) {
            x1 = fmaxf(x1, ls.lbj[tm * T + k2]);
            x2 = fmaxf(x2, ls.lbl[tm * T + k2]);
        }
        team_sync<T>(tm);
    }
}

// Mark the survivors of the bracket test in the table (SURV_FLAG) and count
// them per kind; for a lone survivor, its id, count and lower end.
template <int T>
__device__ void lit_mark(const RunArgs &a, int32_t *keys, uint32_t *vals, const int32_t *aux, const float *dv,
                         uint32_t H, float lbj, float lbl, LitScratch &ls, int tm, int w_in, int &cj, int &cl,
                         int32_t &Cj, int32_t &Cl, int32_t &kj, int32_t &kl, float &Lj, float &Ll) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int nj = 0, nl = 0;
    int32_t fCj = -1, fCl = -1, fkj = 0, fkl = 0;
    float fLj = 0.f, fLl = 0.f;
    for (uint32_t b0 = (uint32_t)w_in * 32; b0 < H; b0 += T * 32) {
        const uint32_t s = b0 + lane;
        bool sj = false, sl = false;
        int32_t C = EMPTY_KEY;
        uint32_t v = 0;
        float L = 0.f;
        if (s < H) {
            C = keys[s];
            if (C != EMPTY_KEY) {
                v = vals[s];
                const float X = dv[s], E = __int_as_float(aux[s]);
                const float U = X + E;
                L = X - E;
                const bool own = (v & OWN_FLAG) != 0;
                const bool surv = !a.screen || (U > 0.f && U >= (own ? lbl : lbj));
                if (surv) {
                    vals[s] = v | SURV_FLAG;
                    if (own) sl = true;
                    else sj = true;
                } else if (v & SURV_FLAG) {
                    vals[s] = v & ~SURV_FLAG;
                }
            }
        }
        const unsigned mj = __ballot_sync(FULL, sj), ml = __ballot_sync(FULL, sl);
        if (mj) {
            const int src = __ffs(mj) - 1;
            const int32_t c1 = __shfl_sync(FULL, C, src);
            const uint32_t v1 = __shfl_sync(FULL, v, src);
            const float l1 = __shfl_sync(FULL, L, src);
            if (nj == 0) {
                fCj = c1;
                fkj = (int32_t)(v1 & CNT_MASK);
                fLj = l1;
            }
            nj += __popc(mj);
        }
        if (ml) {
            const int src = __ffs(ml) - 1;
            const int32_t c1 = __shfl_sync(FULL, C, src);
            const uint32_t v1 = __shfl_sync(FULL, v, src);
            const float l1 = __shfl_sync(FULL, L, src);
            if (nl == 0) {
                fCl = c1;
                fkl = (int32_t)(v1 & CNT_MASK);
                fLl = l1;
            }
            nl += __popc(ml);
        }
    }
    if constexpr (T > 1) {
        if (lane == 0) {
            ls.cj[w] = nj; ls.cl[w] = nl;
            ls.sCj[w] = fCj; ls.sCl[w] = fCl; ls.skj[w] = fkj; ls.skl[w] = fkl;
            ls.sLj[w] = fLj; ls.sLl[w] = fLl;
        }
        team_sync<T>(tm);
        nj = nl = 0;
        for (int k2 = 0; k2 < T; ++k2) {
            const int q = tm * T + k2;
            if (ls.cj[q] > 0 && nj == 0) { fCj = ls.sCj[q]; fkj = ls.skj[q]; fLj = ls.sLj[q]; }
            if (ls.cl[q] > 0 && nl == 0) { fCl = ls.sCl[q]; fkl = ls.skl[q]; fLl = ls.sLl[q]; }
            nj += ls.cj[q];
            nl += ls.cl[q];
        }
        team_sync<T>(tm);
    }
    cj += nj;
    cl += nl;
    if (Cj < 0 && fCj >= 0) { Cj = fCj; kj = fkj; Lj = fLj; }
    if (Cl < 0 && fCl >= 0) { Cl = fCl; kl = fkl; Ll = fLl; }
}

// Exact gains of the marked survivors of the kinds still open; each warp of
// the team takes its slots' survivors one at a time.
template <int T>
__device__ void lit_exact_survivors(const RunArgs &a, const LitNode &ln, const int32_t *keys, const uint32_t *vals,
                                    uint32_t H, bool do_j, bool do_l, unsigned long long *acc, int w_in, Best &bj,
                                    Best &bl) {
    const int lane = threadIdx.x & 31;
    for (uint32_t b0 = (uint32_t)w_in * 32; b0 < H; b0 += T * 32) {
        const uint32_t s = b0 + lane;
        bool want = false;
        int32_t C = EMPTY_KEY;
        uint32_t v = 0;
        if (s < H) {
            C = keys[s];
            if (C != EMPTY_KEY) {
                v = vals[s];
                want = (v & SURV_FLAG) && ((v & OWN_FLAG) ? do_l : do_j);
            }
        }
        unsigned m = __ballot_sync(FULL, want);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const int32_t c1 = __shfl_sync(FULL, C, src);
            const uint32_t v1 = __shfl_sync(FULL, v, src);
            const bool own = (v1 & OWN_FLAG) != 0;
            const int64_t k = (int64_t)(v1 & CNT_MASK);
            const double g = lit_exact_gain(a, ln.x, ln.d, c1, own, k, acc);
            if (a.profile && lane == 0) atomicAdd(&a.ds->prof_exact, 1ull);
            if (g > 0.0) {
                Best &b = own ? bl : bj;
                if (better(g, c1, b.g, b.c)) b = Best{g, c1, (int32_t)k};
            }
        }
    }
}

// A node's decision with the paper's gain, by a team of T warps over a table
// of H slots (P parts of the candidates, one pass each).  False if a part
// overflowed the table (the caller retries with more parts).
template <int T>
__device__ bool lit_eval_node(const RunArgs &a, int i, const LitNode &ln, int P, int32_t *keys, uint32_t *vals,
                              int32_t *aux, float *dv, uint32_t H, LitScratch &ls, unsigned long long *acc,
                              int tm, int w_in) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long pb = 0;
    float lbj = -INFINITY, lbl = -INFINITY;
    for (int p = 0; p < P; ++p)
        if (!lit_pass<T>(a, ln, P, p, keys, vals, aux, dv, H, ls, tm, w_in, lbj, lbl, pb, a.profile != 0))
            return false;
    team_max2<T>(ls, tm, lbj, lbl);
    int cj = 0, cl = 0;
    int32_t Cj = -1, Cl = -1, kj = 0, kl = 0;
    float Lj = 0.f, Ll = 0.f;
    for (int p = 0; p < P; ++p) {
        if (P > 1 && !lit_pass<T>(a, ln, P, p, keys, vals, aux, dv, H, ls, tm, w_in, lbj, lbl, pb, false))
            return false;
        lit_mark<T>(a, keys, vals, aux, dv, H, lbj, lbl, ls, tm, w_in, cj, cl, Cj, Cl, kj, kl, Lj, Ll);
    }
    Best bj{0.0, -1, 0}, bl{0.0, -1, 0};
    bool do_j = cj > 0, do_l = cl > 0;
    if (a.screen && cj == 1 && Lj > 0.f) {
        bj = Best{INFINITY, Cj, kj};
        do_j = false;
    }
    if (a.screen && cl == 1 && Ll > 0.f) {
        bl = Best{INFINITY, Cl, kl};
        do_l = false;
    }
    if (do_j || do_l) {
        for (int p = 0; p < P; ++p) {
            if (P > 1) {
                float d1 = -INFINITY, d2 = -INFINITY;
                if (!lit_pass<T>(a, ln, P, p, keys, vals, aux, dv, H, ls, tm, w_in, d1, d2, pb, false)) return false;
                int c1 = 0, c2 = 0;
                int32_t e1 = -1, e2 = -1, e3 = 0, e4 = 0;
                float e5 = 0.f, e6 = 0.f;
                lit_mark<T>(a, keys, vals, aux, dv, H, lbj, lbl, ls, tm, w_in, c1, c2, e1, e2, e3, e4, e5, e6);
            }
            lit_exact_survivors<T>(a, ln, keys, vals, H, do_j, do_l, acc, w_in, bj, bl);
            team_sync<T>(tm);
        }
        if constexpr (T > 1) {
            if (lane == 0) {
                ls.bgj[w] = bj.g; ls.bcj[w] = bj.c; ls.bkj[w] = bj.k;
                ls.bgl[w] = bl.g; ls.bcl[w] = bl.c; ls.bkl[w] = bl.k;
            }
            team_sync<T>(tm);
            if (w_in == 0) {
                for (int k2 = 1; k2 < T; ++k2) {
                    const int q = tm * T + k2;
                    if (better(ls.bgj[q], ls.bcj[q], bj.g, bj.c)) bj = Best{ls.bgj[q], ls.bcj[q], ls.bkj[q]};
                    if (better(ls.bgl[q], ls.bcl[q], bl.g, bl.c)) bl = Best{ls.bgl[q], ls.bcl[q], ls.bkl[q]};
                }
            }
            team_sync<T>(tm);
        }
    }
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if (lane == 0) atomicAdd(&a.ds->prof_bytes, pb + (w_in == 0 ? 44ull + 8ull * (unsigned long long)ln.cx : 0ull));
    }
    if (w_in == 0 && lane == 0) write_action(a, i, bj, bl, 0ull);
    team_sync<T>(tm);
    return true;
}

__device__ __forceinline__ void lit_smem(double *base, float *&dv, int32_t *&keys, uint32_t *&vals, int32_t *&aux,
                                         unsigned long long *&acc) {
    dv = reinterpret_cast<float *>(base);
    keys = reinterpret_cast<int32_t *>(dv + LB_SLOTS);
    vals = reinterpret_cast<uint32_t *>(keys + LB_SLOTS);
    aux = reinterpret_cast<int32_t *>(vals + LB_SLOTS);
    acc = reinterpret_cast<unsigned long long *>(aux + LB_SLOTS);
}

// Teams of T warps, one queued node each.  A node whose entries (own rows
// plus its neighbours' rows) could fill more than half of the team's table
// is listed for k_lit_big.  Counters: over[0] = listed nodes, over[1] = next.
template <int T>
__global__ void __launch_bounds__(EV_THREADS, 2) k_lit_eval(RunArgs a, int64_t bstart, int32_t blen, uint32_t *over,
                                                           int32_t *over_list) {
    extern __shared__ double lit_dyn[];
    __shared__ LitScratch ls;
    float *dv;
    int32_t *keys, *aux;
    uint32_t *vals;
    unsigned long long *acc;
    lit_smem(lit_dyn, dv, keys, vals, aux, acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = lane; c < SACC_CHUNKS; c += 32) acc[w * SACC_CHUNKS + c] = 0ull;
    pdl_trigger();
    pdl_wait();
    const int tm = w / T, w_in = w % T;
    const int i = (int)blockIdx.x * (EV_WARPS / T) + tm;
    if (i >= blen) return;   // the whole team leaves together
    LitNode ln;
    ln.x = a.order[bstart + i];
    ln.beg = a.off[ln.x];
    ln.end = a.off[ln.x + 1];
    ln.d = (int32_t)(ln.end - ln.beg);
    if (ln.d > a.lit_hub_deg) return;   // the hub kernels decide it
    ln.cx = __ldcg(&a.nmem[ln.x]);
    long long bound = w_in == 0 && lane == 0 ? ln.cx : 0;
    for (int64_t q = ln.beg + w_in * 32 + lane; q < ln.end; q += T * 32) bound += __ldcg(&a.nmem[a.adj[q]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(FULL, bound, o);
    if constexpr (T > 1) {
        if (lane == 0) ls.part[w] = bound;
        team_sync<T>(tm);
        bound = 0;
        for (int k2 = 0; k2 < T; ++k2) bound += ls.part[tm * T + k2];
        team_sync<T>(tm);
    }
    uint32_t H = 32;
    while ((long long)H < 2 * bound) H <<= 1;
    if (H > (uint32_t)(T * LW)) {
        if (w_in == 0 && lane == 0) {
            const uint32_t slot = atomicAdd(&over[0], 1u);
            over_list[slot] = i;
        }
        return;
    }
    const int base = tm * T * LW;
    if (!lit_eval_node<T>(a, i, ln, 1, keys + base, vals + base, aux + base, dv + base, H, ls, acc + w * SACC_CHUNKS,
                          tm, w_in)) {
        if (w_in == 0 && lane == 0) atomicOr(&a.ds->err, DERR_CHECK);   // cannot happen: H >= 2 x entries
    }
}

// Listed nodes, one block each, over the block's whole table in as many
// parts as needed (a part that overflows doubles the parts).
__global__ void __launch_bounds__(EV_THREADS, 3) k_lit_big(RunArgs a, int64_t bstart, uint32_t *over,
                                                          const int32_t *over_list, unsigned long long *used) {
    extern __shared__ double lit_dyn[];
    __shared__ LitScratch ls;
    __shared__ int s_i;
    __shared__ long long s_base;
    float *dv;
    int32_t *keys, *aux;
    uint32_t *vals;
    unsigned long long *acc;
    lit_smem(lit_dyn, dv, keys, vals, aux, acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = lane; c < SACC_CHUNKS; c += 32) acc[w * SACC_CHUNKS + c] = 0ull;
    pdl_trigger();
    pdl_wait();
    const uint32_t count = __ldcg(&over[0]);
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(&over[1], 1u);
            s_i = t < count ? over_list[t] : -1;
        }
        __syncthreads();
        const int i = s_i;
        __syncthreads();
        if (i < 0) break;
        LitNode ln;
        ln.x = a.order[bstart + i];
        ln.beg = a.off[ln.x];
        ln.end = a.off[ln.x + 1];
        ln.d = (int32_t)(ln.end - ln.beg);
        ln.cx = __ldcg(&a.nmem[ln.x]);
        long long bound = threadIdx.x == 0 ? ln.cx : 0;
        for (int64_t q = ln.beg + threadIdx.x; q < ln.end; q += EV_THREADS) bound += __ldcg(&a.nmem[a.adj[q]]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(FULL, bound, o);
        if (lane == 0) ls.part[w] = bound;
        __syncthreads();
        bound = 0;
        for (int k2 = 0; k2 < EV_WARPS; ++k2) bound += ls.part[k2];
        __syncthreads();
        if (2 * bound > LB_SLOTS) {   // a table of its own in global memory, if the queue's area has room
            unsigned long long H = 32;
            while ((long long)H < 2 * bound) H <<= 1;
            if (threadIdx.x == 0) {
                const unsigned long long base = atomicAdd(used, H);
                s_base = base + H <= a.lg_cap ? (long long)base : -1ll;
            }
            __syncthreads();
            const long long base = s_base;
            __syncthreads();
            if (base >= 0) {
                lit_eval_node<EV_WARPS>(a, i, ln, 1, a.lg_keys + base, a.lg_vals + base, a.lg_aux + base,
                                        a.lg_dv + base, (uint32_t)H, ls, acc + w * SACC_CHUNKS, 0, w);
                continue;
            }
        }
        int P = (int)((bound + LIT_PART_ENTRIES - 1) / LIT_PART_ENTRIES);
        uint32_t Hs = (uint32_t)LB_SLOTS;
        if (P < 1 || 2 * bound <= LB_SLOTS) {   // one pass over a table of pow2 >= 2 x entries
            P = 1;
            Hs = 32;
            while ((long long)Hs < 2 * bound) Hs <<= 1;
        }
        while (!lit_eval_node<EV_WARPS>(a, i, ln, P, keys, vals, aux, dv, Hs, ls, acc + w * SACC_CHUNKS, 0, w)) {
            Hs = (uint32_t)LB_SLOTS;
            P *= 2;
            if (P > (1 << 22)) {   // cannot happen for < 2^31 entries; leave an error, not a loop
                if (threadIdx.x == 0) atomicOr(&a.ds->err, DERR_CHECK);
                break;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Hubs under the paper's gain: a queued node of degree > LIT_HUB_DEG is
// evaluated by many blocks over one table in global memory (planned per
// queue for the worst case, pow2 >= 2 (d+1) K slots): k_lh_fill (one block per
// 1024 neighbours: counts, own flags, FP32 corrections), k_lh_bound (one
// block per 4096 slots: brackets, the hub's best lower ends by an
// order-preserving integer max), k_lh_mark (one block per 4096 slots:
// survivors listed, slots cleared) and k_lh_decide (one block per hub: a lone
// survivor with a positive lower end, or the survivors' exact sums; those of
// large communities by the whole block, with the hub's adjacency searched
// through a fence in shared memory).  Team and block kernels skip these nodes.
// ---------------------------------------------------------------------------
constexpr int LIT_HUB_DEG = 1024;
constexpr int LH_CHUNK = 1024;       // neighbours per fill block
constexpr int LH_SLOTS = 4096;       // table slots per bracket / mark block

struct LitHubPlan {
    const int32_t *pos;       // per hub: its position in the queue
    const int64_t *toff;      // per hub: first slot of its table
    const uint32_t *tcap;     // per hub: table slots
    const int64_t *soff;      // per hub: first entry of its survivor list (tcap/2 entries)
    const int32_t *fh, *fc;   // fill items of every queue: hub, chunk
    const int32_t *sh, *sr;   // slot items of every queue: hub, range
    const int32_t *nsr;       // per hub: its slot items (worst case)
    uint32_t *heff;           // per hub: table slots used in this queue
    int32_t *lb;              // per hub: best lower ends (join, leave), order-preserving
    uint32_t *ns;             // per hub: survivors listed
    int32_t *sv_c;            // survivor lists: community, count word, lower end
    uint32_t *sv_v;
    float *sv_l;
    int32_t *keys;            // tables: keys, counts, FP32 corrections (then E), X
    uint32_t *vals;
    float *hs;
    float *dv;
};

// Each hub's table size for this queue: pow2 >= 2 (own row + neighbours'
// rows), at least LH_SLOTS, at most the planned worst case (one block per hub).
__global__ void __launch_bounds__(256) k_lh_size(RunArgs a, LitHubPlan hp, int64_t bstart, int64_t h0, int64_t nh) {
    __shared__ long long part[8];
    const int64_t h = h0 + blockIdx.x;
    if (blockIdx.x >= nh) return;
    const int32_t x = a.order[bstart + hp.pos[h]];
    long long b = threadIdx.x == 0 ? __ldcg(&a.nmem[x]) : 0;
    for (int64_t q = a.off[x] + threadIdx.x; q < a.off[x + 1]; q += blockDim.x) b += __ldcg(&a.nmem[a.adj[q]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(FULL, b, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k2 = 0; k2 < (int)(blockDim.x >> 5); ++k2) t += part[k2];
        unsigned long long H = LH_SLOTS;
        while ((long long)H < 2 * t && H < hp.tcap[h]) H <<= 1;
        hp.heff[h] = (uint32_t)H;
    }
}

__global__ void __launch_bounds__(256) k_lh_fill(RunArgs a, LitHubPlan hp, int64_t bstart, int64_t first) {
    const int64_t it = first + blockIdx.x;
    const int h = hp.fh[it], c = hp.fc[it];
    const int32_t x = a.order[bstart + hp.pos[h]];
    const int64_t beg = a.off[x], end = a.off[x + 1];
    const int64_t t0 = hp.toff[h];
    const uint32_t hm = __ldcg(&hp.heff[h]) - 1;
    int32_t *keys = hp.keys + t0;
    uint32_t *vals = hp.vals + t0;
    float *hs = hp.hs + t0;
    const int32_t cx = __ldcg(&a.nmem[x]);
    const int32_t *rowx = a.mem + (int64_t)x * a.K;
    if (c == 0)
        for (int j = threadIdx.x; j < cx; j += blockDim.x)
            if (!ht_insert(keys, vals, hm, __ldcg(&rowx[j]), 0u, true)) atomicOr(&a.ds->err, DERR_CHECK);
    unsigned long long pb = 0;
    const int64_t cb = beg + (int64_t)c * LH_CHUNK, ce = min(end, cb + LH_CHUNK);
    {   // each warp takes a contiguous eighth of the chunk
        const int64_t per = (ce - cb + 7) / 8, w = threadIdx.x >> 5;
        const int64_t qb = min(ce, cb + w * per), qe = min(ce, cb + (w + 1) * per);
        lit_warp_entries(a, qb, qe, pb, a.profile != 0, [&](int32_t C, int64_t ky, int64_t dy, int64_t n) {
            if (!dbg_ok(a, ky >= 0 && ky <= dy)) return;
            const int slot = lit_insert(keys, vals, hm, C);
            if (slot < 0) {   // cannot happen: the table holds 2 (d+1) K slots
                atomicOr(&a.ds->err, DERR_CHECK);
                return;
            }
            const float hv = row_find(rowx, cx, C) >= 0 ? lit_h_leave32(ky, dy, n) : lit_h_join32(ky, dy, n);
            if (hv != 0.f) atomicAdd(&hs[slot], hv);
        });
    }
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if ((threadIdx.x & 31) == 0 && pb) atomicAdd(&a.ds->prof_bytes, pb);
    }
}

__global__ void __launch_bounds__(256) k_lh_bound(RunArgs a, LitHubPlan hp, int64_t bstart, int64_t first) {
    __shared__ float red[2][8];
    const int64_t it = first + blockIdx.x;
    const int h = hp.sh[it], r = hp.sr[it];
    const int32_t x = a.order[bstart + hp.pos[h]];
    const int32_t d = (int32_t)(a.off[x + 1] - a.off[x]);
    const int64_t t0 = hp.toff[h];
    const uint32_t lo = (uint32_t)r * LH_SLOTS, hi = min(__ldcg(&hp.heff[h]), lo + LH_SLOTS);
    if (lo >= hi) return;   // beyond this queue's table
    float lbj = -INFINITY, lbl = -INFINITY;
    unsigned long long nc = 0;
    for (uint32_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
        const int32_t C = hp.keys[t0 + s];
        if (C == EMPTY_KEY) continue;
        const uint32_t v = hp.vals[t0 + s];
        float X, E;
        lit_screen(a, C, v, d, hp.hs[t0 + s], X, E);
        hp.dv[t0 + s] = X;
        hp.hs[t0 + s] = E;
        const float L = X - E;
        if (v & OWN_FLAG) lbl = fmaxf(lbl, L);
        else lbj = fmaxf(lbj, L);
        ++nc;
    }
    lbj = warp_max_f(lbj);
    lbl = warp_max_f(lbl);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = lbj;
        red[1][w] = lbl;
    }
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nc += __shfl_down_sync(FULL, nc, o);
        if (lane == 0 && nc) {
            atomicAdd(&a.ds->prof_cands, nc);
            atomicAdd(&a.ds->prof_bytes, 40ull * nc);
        }
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        float m = -INFINITY;
        for (int k2 = 0; k2 < (int)(blockDim.x >> 5); ++k2) m = fmaxf(m, red[threadIdx.x][k2]);
        if (m > -INFINITY) atomicMax(&hp.lb[2 * h + threadIdx.x], f2ord(m));
    }
}

constexpr int LH_FENCE = 2048;        // fence entries of a hub's adjacency (exact sums)
constexpr int64_t LH_BLOCK_MEMBERS = 256;   // survivors of larger communities are summed by the whole block

// Survivors of a hub's bracket test listed (one block per 4096 slots), the
// table left clean for the hub's next queue.
__global__ void __launch_bounds__(256, 4) k_lh_mark(RunArgs a, LitHubPlan hp, int64_t bstart, int64_t first) {
    const int64_t it = first + blockIdx.x;
    const int h = hp.sh[it], r = hp.sr[it];
    const int64_t t0 = hp.toff[h], so = hp.soff[h];
    const float lbj = ord2f(__ldcg(&hp.lb[2 * h])), lbl = ord2f(__ldcg(&hp.lb[2 * h + 1]));
    const uint32_t heff = __ldcg(&hp.heff[h]);
    const uint32_t lo = (uint32_t)r * LH_SLOTS, hi = min(heff, lo + LH_SLOTS);
    if (lo >= hi) return;   // beyond this queue's table
    for (uint32_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
        const int32_t C = hp.keys[t0 + s];
        if (C == EMPTY_KEY) continue;
        const uint32_t v = hp.vals[t0 + s];
        const float X = hp.dv[t0 + s], E = hp.hs[t0 + s];
        const float U = X + E;
        const bool own = (v & OWN_FLAG) != 0;
        if (!a.screen || (U > 0.f && U >= (own ? lbl : lbj))) {
            const uint32_t e = atomicAdd(&hp.ns[h], 1u);
            hp.sv_c[so + e] = C;
            hp.sv_v[so + e] = v;
            hp.sv_l[so + e] = X - E;
        }
        hp.keys[t0 + s] = EMPTY_KEY;   // the table is left clean for the hub's next queue
        hp.vals[t0 + s] = 0u;
        hp.hs[t0 + s] = 0.f;
    }
}

// A hub's decision from its listed survivors (one block per hub of the
// queue): a lone survivor with a positive lower end wins; otherwise the
// survivors' gains are summed exactly and compared.
__global__ void __launch_bounds__(256) k_lh_decide(RunArgs a, LitHubPlan hp, int64_t bstart, int64_t h0, int64_t nh) {
    __shared__ unsigned long long acc_s[8 * SACC_CHUNKS];
    __shared__ int32_t fence[LH_FENCE];
    __shared__ double s_g;
    __shared__ double bg[2][8];
    __shared__ int32_t bc[2][8], bk[2][8];
    if (blockIdx.x >= nh) return;
    const int64_t h = h0 + blockIdx.x;
    const int32_t i = hp.pos[h];
    const int32_t x = a.order[bstart + i];
    const int32_t d = (int32_t)(a.off[x + 1] - a.off[x]);
    const int64_t so = hp.soff[h];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t ns = __ldcg(&hp.ns[h]);
    int cj = 0, cl = 0;
    int32_t Cj = -1, Cl = -1, kj = 0, kl = 0;
    float Lj = 0.f, Ll = 0.f;
    for (uint32_t e = 0; e < ns; ++e) {   // every thread reads the (short) list
        const uint32_t v = __ldcg(&hp.sv_v[so + e]);
        const int32_t C = __ldcg(&hp.sv_c[so + e]);
        const float L = __ldcg(&hp.sv_l[so + e]);
        if (v & OWN_FLAG) {
            if (cl++ == 0) { Cl = C; kl = (int32_t)(v & CNT_MASK); Ll = L; }
        } else {
            if (cj++ == 0) { Cj = C; kj = (int32_t)(v & CNT_MASK); Lj = L; }
        }
    }
    Best bj{0.0, -1, 0}, bl{0.0, -1, 0};
    bool do_j = cj > 0, do_l = cl > 0;
    if (a.screen && cj == 1 && Lj > 0.f) {
        bj = Best{INFINITY, Cj, kj};
        do_j = false;
    }
    if (a.screen && cl == 1 && Ll > 0.f) {
        bl = Best{INFINITY, Cl, kl};
        do_l = false;
    }
    if (do_j || do_l) {
        unsigned long long *acc = acc_s + w * SACC_CHUNKS;
        for (int c2 = lane; c2 < SACC_CHUNKS; c2 += 32) acc[c2] = 0ull;
        // every step-th entry of x's adjacency, for the neighbour tests of the member passes
        const int64_t xb = a.off[x];
        const int64_t step = ((int64_t)d + LH_FENCE - 1) / LH_FENCE;
        const int nf = (int)(((int64_t)d + step - 1) / step);
        for (int j = threadIdx.x; j < nf; j += blockDim.x) fence[j] = a.adj[xb + (int64_t)j * step];
        __syncthreads();
        // survivors of large communities: one at a time, the whole block over the members
        for (uint32_t e = 0; e < ns; ++e) {
            const uint32_t v = __ldcg(&hp.sv_v[so + e]);
            const bool own = (v & OWN_FLAG) != 0;
            if (own ? !do_l : !do_j) continue;
            const int32_t C = __ldcg(&hp.sv_c[so + e]);
            if ((int64_t)__ldcg(&a.comm[C].n) <= LH_BLOCK_MEMBERS) continue;
            const int64_t k = (int64_t)(v & CNT_MASK);
            const double g = lit_exact_gain(a, x, d, C, own, k, acc_s, fence, nf, step, true, &s_g);
            if (a.profile && threadIdx.x == 0) atomicAdd(&a.ds->prof_exact, 1ull);
            if (g > 0.0) {
                Best &b = own ? bl : bj;
                if (better(g, C, b.g, b.c)) b = Best{g, C, (int32_t)k};
            }
        }
        // the others: a warp each
        for (uint32_t e = w; e < ns; e += blockDim.x >> 5) {
            const uint32_t v = __ldcg(&hp.sv_v[so + e]);
            const bool own = (v & OWN_FLAG) != 0;
            if (own ? !do_l : !do_j) continue;
            const int32_t C = __ldcg(&hp.sv_c[so + e]);
            if ((int64_t)__ldcg(&a.comm[C].n) > LH_BLOCK_MEMBERS) continue;
            const int64_t k = (int64_t)(v & CNT_MASK);
            const double g = lit_exact_gain(a, x, d, C, own, k, acc, fence, nf, step);
            if (a.profile && lane == 0) atomicAdd(&a.ds->prof_exact, 1ull);
            if (g > 0.0) {
                Best &b = own ? bl : bj;
                if (better(g, C, b.g, b.c)) b = Best{g, C, (int32_t)k};
            }
        }
        if (lane == 0) {
            bg[0][w] = bj.g; bc[0][w] = bj.c; bk[0][w] = bj.k;
            bg[1][w] = bl.g; bc[1][w] = bl.c; bk[1][w] = bl.k;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k2 = 1; k2 < (int)(blockDim.x >> 5); ++k2) {
                if (better(bg[0][k2], bc[0][k2], bj.g, bj.c)) bj = Best{bg[0][k2], bc[0][k2], bk[0][k2]};
                if (better(bg[1][k2], bc[1][k2], bl.g, bl.c)) bl = Best{bg[1][k2], bc[1][k2], bk[1][k2]};
            }
    }
    if (threadIdx.x == 0) {
        write_action(a, i, bj, bl, 0ull);
        if (a.profile) atomicAdd(&a.ds->prof_bytes, 44ull + 8ull * (unsigned long long)__ldcg(&a.nmem[x]));
        hp.ns[h] = 0u;   // ready for the hub's next queue
        hp.lb[2 * h] = f2ord(-INFINITY);
        hp.lb[2 * h + 1] = f2ord(-INFINITY);
    }
}

// Apply of one queue under the paper's gain: as apply_node (rows, n_C,
// vol_C, 2m_C with the same in-queue corrections), and in addition each
// membership's deg(x,C) moves with the row, a joiner's starts at its count
// before the queue (k_lit_kupd adds the queue's other moves), the joiner is
// appended to C's list of this iteration's joiners, and every community a
// move touches is listed once for k_lit_fsum.
__device__ void lit_apply_node(const RunArgs &a, int64_t bstart, int32_t blen, int64_t i, uint32_t serial,
                               unsigned long long &nj, unsigned long long &nl) {
    const int lane = threadIdx.x & 31;
    const int32_t j = __ldcg(&a.act[i]), l = __ldcg(&a.act[a.qcap + i]);
    if (j < 0 && l < 0) return;
    if (!dbg_ok(a, j < a.nnodes && l < a.nnodes && (j < 0 || j != l))) return;
    const int32_t x = a.order[bstart + i];
    int jj = 0, jl = 0, ll = 0;
    for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
        const int32_t y = a.adj[p];
        const int64_t py = a.pos[y];
        if (py >= bstart && py < bstart + blen) {
            const int64_t iy = py - bstart;
            const int32_t aj = __ldcg(&a.act[iy]), al = __ldcg(&a.act[a.qcap + iy]);
            if (j >= 0) {
                jj += aj == j;
                jl += al == j;
            }
            if (l >= 0) ll += al == l;
        }
    }
    jj = __reduce_add_sync(FULL, jj);
    jl = __reduce_add_sync(FULL, jl);
    ll = __reduce_add_sync(FULL, ll);
    const int32_t d = a.deg[x];
    const int32_t kjoin = __ldcg(&a.act[2 * a.qcap + i]);
    int32_t *row = a.mem + (int64_t)x * a.K;
    int32_t *krow = a.kmem + (int64_t)x * a.K;
    const int32_t c = __ldcg(&a.nmem[x]);
    if (!dbg_ok(a, c >= 0 && c <= a.K && (j < 0 || (kjoin >= 0 && kjoin <= d)))) return;
    int32_t c_new = c;
    if (lane == 0) {
        int32_t cc2 = c;
        if (l >= 0) {
            int32_t o = 0;
            for (int32_t s = 0; s < cc2; ++s) {
                const int32_t v = __ldcg(&row[s]);
                if (v != l) {
                    krow[o] = __ldcg(&krow[s]);
                    row[o++] = v;
                }
            }
            cc2 = o;
        }
        if (j >= 0) {
            if (cc2 >= a.K) {
                atomicOr(&a.ds->err, DERR_CAPACITY);
            } else {
                int32_t s = cc2;
                while (s > 0) {
                    const int32_t v = __ldcg(&row[s - 1]);
                    if (v <= j) break;
                    row[s] = v;
                    krow[s] = __ldcg(&krow[s - 1]);
                    --s;
                }
                row[s] = j;
                krow[s] = kjoin;
                ++cc2;
            }
        }
        c_new = cc2;
        if (l >= 0) {
            const int32_t kl = __ldcg(&a.act[3 * a.qcap + i]);
            atomicAdd(&a.comm[l].n, -1);
            atomicAdd(&a.comm[l].vol, (uint32_t)(-d));
            atomicAdd(&a.comm[l].m2, (uint32_t)(-2 * kl + ll));
            ++nl;
            if (atomicExch(&a.tstamp[l], serial) != serial) a.touched[atomicAdd(a.ntouched, 1u)] = l;
        }
        if (j >= 0) {
            atomicAdd(&a.comm[j].n, 1);
            atomicAdd(&a.comm[j].vol, (uint32_t)d);
            atomicAdd(&a.comm[j].m2, (uint32_t)(2 * kjoin + jj - 2 * jl));
            ++nj;
            const unsigned long long slot = atomicAdd(&a.cm_cnt[j], 1u);
            if ((long long)slot < (long long)(a.cm_off[j + 1] - a.cm_off[j])) {
                a.cm_node[a.cm_off[j] + slot] = x;
            } else {
                const int32_t e = (int32_t)atomicAdd(a.jl_count, 1u);
                a.jl_node[e] = x;
                a.jl_next[e] = atomicExch(&a.jl_head[j], e);
            }
            if (atomicExch(&a.tstamp[j], serial) != serial) a.touched[atomicAdd(a.ntouched, 1u)] = j;
        }
        a.nmem[x] = c_new;
    }
}

__global__ void __launch_bounds__(AP_THREADS) k_lit_apply(RunArgs a, int64_t bstart, int32_t blen, int64_t bidx) {
    pdl_trigger();
    pdl_wait();
    const uint32_t serial = (uint32_t)queue_serial(a, bidx);
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long nj = 0, nl = 0;
    if (i < blen) lit_apply_node(a, bstart, blen, i, serial, nj, nl);
    flush_counts(a, nj, nl);
}

// Every neighbour y of a node that joined (left) C and is in C after the
// queue has one more (fewer) neighbour in C.  Summed over the queue this
// turns each membership's count before the queue into its count after it,
// for stayers and joiners alike (leavers' memberships are gone).
__global__ void __launch_bounds__(AP_THREADS) k_lit_kupd(RunArgs a, int64_t bstart, int32_t blen) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= blen) return;
    const int32_t j = __ldcg(&a.act[i]), l = __ldcg(&a.act[a.qcap + i]);
    if (j < 0 && l < 0) return;
    const int32_t x = a.order[bstart + i];
    for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
        const int32_t y = a.adj[p];
        const int32_t cy = __ldcg(&a.nmem[y]);
        const int32_t *row = a.mem + (int64_t)y * a.K;
        if (j >= 0) {
            const int s = row_find(row, cy, j);
            if (s >= 0) {
                const int32_t was = atomicAdd(&a.kmem[(int64_t)y * a.K + s], 1);
                dbg_ok(a, was >= 0 && was < a.deg[y]);
            }
        }
        if (l >= 0) {
            const int s = row_find(row, cy, l);
            if (s >= 0) {
                const int32_t was = atomicAdd(&a.kmem[(int64_t)y * a.K + s], -1);
                dbg_ok(a, was >= 1);
            }
        }
    }
}

// F(n-1), F(n), F(n+1) of communities: list[0 .. *count) (or every id below
// ncount when list is null).  Blocks take eight entries at a time: each warp
// sums a community of up to LIT_FSUM_WARP members alone, larger ones are then
// summed by the whole block, one after the other.
constexpr int LIT_FSUM_WARP = 512;

__device__ __forceinline__ void lit_fsum_member(const RunArgs &a, int32_t C, int64_t n, int32_t y, double &f0,
                                                double &f1, double &f2) {
    if (!dbg_ok(a, y >= 0 && y < a.nnodes)) return;
    const int32_t cy = __ldcg(&a.nmem[y]);
    if (!dbg_ok(a, cy >= 0 && cy <= a.K)) return;
    const int s = row_find(a.mem + (int64_t)y * a.K, cy, C);
    if (s < 0) return;   // left C earlier in this iteration
    const int64_t ky = __ldcg(&a.kmem[(int64_t)y * a.K + s]);
    const int64_t dy = a.deg[y];
    if (!dbg_ok(a, ky >= 0 && ky <= dy)) return;
    f0 += lit_g(ky, dy, n - 1);
    f1 += lit_g(ky, dy, n);
    f2 += lit_g(ky, dy, n + 1);
}

// The per-community values of the bracket from the member sums (rounded
// to float; the bound E allows for it).
__device__ __forceinline__ void lit_fsum_store(const RunArgs &a, int32_t C, double f0, double f1, double f2) {
    const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
    const int64_t n = r.x;
    const double m2 = (double)(uint32_t)r.y;
    const double cc = a.gcc ? a.gcc[r.w] : a.cc;
    const bool on = cc > 0.0 && n >= 1;
    float *f = a.litF + 8 * (int64_t)C;
    f[0] = (float)f0;
    f[1] = (float)f2;
    f[2] = on && n >= 2 ? (float)(((m2 / ((double)n * (double)(n - 1))) / cc) * f1) : 0.f;
    f[3] = on ? (float)((1.0 / ((double)(n + 1) * (double)n)) / cc) : 0.f;
    f[4] = on && n - 1 >= 2 ? (float)((1.0 / ((double)(n - 1) * (double)(n - 2))) / cc) : 0.f;
}

__global__ void __launch_bounds__(256) k_lit_fsum(RunArgs a, const int32_t *list, const uint32_t *count,
                                                  int64_t ncount) {
    __shared__ double red[3][8];
    __shared__ int32_t big[8];
    __shared__ int nbig;
    const int64_t total = list ? (int64_t)__ldcg(count) : ncount;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t0 = (int64_t)blockIdx.x * 8; t0 < total; t0 += (int64_t)gridDim.x * 8) {
        if (threadIdx.x == 0) nbig = 0;
        __syncthreads();
        const int64_t t = t0 + w;
        if (t < total) {
            const int32_t C = list ? __ldcg(&list[t]) : (int32_t)t;
            const int64_t n = __ldcg(&a.comm[C].n);
            if (n > LIT_FSUM_WARP) {
                if (lane == 0) big[atomicAdd(&nbig, 1)] = C;
            } else {
                double f0 = 0.0, f1 = 0.0, f2 = 0.0;
                if (n > 0)
                    lit_members(a, C, lane, 32, [&](int32_t y) { lit_fsum_member(a, C, n, y, f0, f1, f2); });
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    f0 += __shfl_xor_sync(FULL, f0, o);
                    f1 += __shfl_xor_sync(FULL, f1, o);
                    f2 += __shfl_xor_sync(FULL, f2, o);
                }
                if (lane == 0) lit_fsum_store(a, C, f0, f1, f2);
            }
        }
        __syncthreads();
        for (int b = 0; b < nbig; ++b) {
            const int32_t C = big[b];
            const int64_t n = __ldcg(&a.comm[C].n);
            double f0 = 0.0, f1 = 0.0, f2 = 0.0;
            lit_members(a, C, threadIdx.x, blockDim.x, [&](int32_t y) { lit_fsum_member(a, C, n, y, f0, f1, f2); });
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                f0 += __shfl_xor_sync(FULL, f0, o);
                f1 += __shfl_xor_sync(FULL, f1, o);
                f2 += __shfl_xor_sync(FULL, f2, o);
            }
            if (lane == 0) {
                red[0][w] = f0;
                red[1][w] = f1;
                red[2][w] = f2;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double sum[3] = {0.0, 0.0, 0.0};
                for (int k2 = 0; k2 < (int)(blockDim.x >> 5); ++k2)
                    for (int t2 = 0; t2 < 3; ++t2) sum[t2] += red[t2][k2];
                lit_fsum_store(a, C, sum[0], sum[1], sum[2]);
            }
            __syncthreads();
        }
    }
}

// deg(x,C) of every membership, counted over x's neighbours (a warp per node).
__global__ void k_lit_kinit(RunArgs a, int64_t n) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const int32_t cx = a.nmem[x];
        const int32_t *row = a.mem + x * a.K;
        for (int32_t s = 0; s < cx; ++s) {
            const int32_t C = row[s];
            int cnt = 0;
            for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
                const int32_t y = a.adj[p];
                cnt += row_find(a.mem + (int64_t)y * a.K, a.nmem[y], C) >= 0;
            }
            cnt = __reduce_add_sync(FULL, cnt);
            if (lane == 0) a.kmem[x * a.K + s] = cnt;
        }
    }
}

// Member index at an iteration's start: members per community, then (after
// a scan into cm_off) every node listed under each of its communities.
__global__ void k_lit_count(RunArgs a, int64_t n, uint32_t *cnt) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t cx = a.nmem[x];
        const int32_t *row = a.mem + x * a.K;
        for (int32_t s = 0; s < cx; ++s) atomicAdd(&cnt[row[s]], 1u);
    }
}

// Region capacity of each community: its members at the start plus room
// for 3 n + 32 joiners (more joiners go to the community's list).
__global__ void k_lit_caps(const uint32_t *cnt, int64_t nc, unsigned long long *cap) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        cap[c] = 4ull * cnt[c] + 32ull;
}

__global__ void k_lit_fill(RunArgs a, int64_t n, unsigned long long *cursor, int32_t *cm_node) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t cx = a.nmem[x];
        const int32_t *row = a.mem + x * a.K;
        for (int32_t s = 0; s < cx; ++s) cm_node[atomicAdd(&cursor[row[s]], 1ull)] = (int32_t)x;
    }
}

// ---------------------------------------------------------------------------
// Persistent queue loop: one cooperative launch runs queues first ..
// first+count-1 of an iteration: evaluate (blocks take groups of EV_WARPS
// nodes), grid barrier, apply (warps take nodes), grid barrier.  Every
// barrier wait is bounded; a wait that runs out sets DERR_TIMEOUT and the
// kernel returns (the other blocks then run out at their next wait).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier on per-block epoch flags (flags[0 .. nblocks-1]) and one
// release flag (flags[nblocks]).  The block's threads meet at __syncthreads;
// thread 0 publishes the arrival with a release store of the barrier's epoch
// (the release orders every write the block made before the __syncthreads).
//   mode 0 (flat): warp 0 of every block polls all arrival flags.
//   mode 1 (central): warp 0 of block 0 polls the arrival flags and then
//     publishes the epoch in the release flag, which the other blocks poll
//     (one line, with a short back-off).
// Polling uses relaxed loads; an acquire fence after the wait orders the
// block's later reads after the other blocks' writes.  No read-modify-write
// on a shared counter.  The wait is bounded: when it runs out (or another
// block reported a timeout) DERR_TIMEOUT is set and false returned.
__device__ bool grid_sync(unsigned *flags, unsigned nblocks, unsigned epoch, long long spin_limit, DevScalars *ds,
                          int *s_ok, int mode) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) st_release_u32(flags + blockIdx.x, epoch);
        int ok = 1;
        long long it = 0;
        const bool gather = mode == 0 || blockIdx.x == 0;
        for (;;) {
            bool done = true;
            if (gather) {
                for (unsigned b = lane; b < nblocks; b += 32)
                    done = done && (int)(ld_relaxed_u32(flags + b) - epoch) >= 0;
            } else {
                done = (int)(ld_relaxed_u32(flags + nblocks) - epoch) >= 0;
            }
            if (__all_sync(FULL, done)) break;
            ++it;
            if (it > spin_limit ||
                ((it & 255) == 0 && (*((volatile int *)&ds->err) & DERR_TIMEOUT))) {
                ok = 0;
                break;
            }
            if (!gather) __nanosleep(32);
        }
        if (mode == 1 && blockIdx.x == 0 && lane == 0 && ok) st_release_u32(flags + nblocks, epoch);
        fence_acq_rel_gpu();
        if (lane == 0) {
            if (!ok) atomicOr(&ds->err, DERR_TIMEOUT);
            *s_ok = ok;
        }
        __syncwarp();
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Fused warp path of the persistent kernel, for queues that fit in one round
// (one warp per node).  All of a node's independent loads go out together:
// its neighbours' membership counts, positions and row heads, and its own
// count and row head.  The warp keeps the node's state in registers across
// the grid barrier and applies its own action from them: in-queue
// neighbours are recognised from the positions already loaded, the row is
// rewritten from the registers.  Nodes with more than 32 neighbours or more
// than 8 memberships take the general path.
// ---------------------------------------------------------------------------
struct WarpNode {
    int64_t beg, end;
    int32_t x, d, cx;
    int32_t py0;       // this lane's first-chunk neighbour's position in the order (-1: none)
    int4 rx0, rx1;     // own row head
    int32_t j, l, kj, kl;
    int valid, fused;
};

__device__ void eval_fused(const RunArgs &a, int64_t bstart, int32_t blen, int i, const NodePrefetch &pf,
                           WarpNode &wn, int32_t *keys, uint32_t *vals, float *ubs, EvalShared &es,
                           unsigned long long serial) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    wn.valid = i < blen;
    wn.fused = 0;
    wn.j = wn.l = -1;
    if (!wn.valid) return;
    const bool have = pf.valid != 0;
    const int32_t x = have ? pf.x : a.order[bstart + i];
    const int32_t d = have ? pf.d : a.deg[x];
    if (d > a.huge_deg) return;   // evaluated by eval_huge; applied by the general path
    const int64_t beg = have ? pf.beg : a.off[x], end = have ? pf.end : a.off[x + 1];
    wn.x = x;
    wn.d = d;
    wn.beg = beg;
    wn.end = end;
    const bool on = beg + lane < end;
    const int32_t y0 = have ? pf.y0 : (on ? a.adj[beg + lane] : 0);
    // one round of independent loads
    const int32_t *rowx = a.mem + (int64_t)x * a.K;
    const int32_t *rowy = a.mem + (int64_t)y0 * a.K;
    const int32_t cy0 = on ? __ldcg(&a.nmem[y0]) : 0;
    wn.py0 = on ? a.pos[y0] : -1;
    const int32_t cx = __ldcg(&a.nmem[x]);
    wn.rx0 = __ldcg(reinterpret_cast<const int4 *>(rowx));
    wn.rx1 = a.K >= 8 ? __ldcg(reinterpret_cast<const int4 *>(rowx) + 1) : make_int4(0, 0, 0, 0);
    const int4 ry0 = on ? __ldcg(reinterpret_cast<const int4 *>(rowy)) : make_int4(0, 0, 0, 0);
    const int4 ry1 = (on && a.K >= 8) ? __ldcg(reinterpret_cast<const int4 *>(rowy) + 1) : make_int4(0, 0, 0, 0);
    wn.cx = cx;
    long long entries = cy0;
    for (int64_t p0 = beg + 32; p0 < end; p0 += 32) {   // nodes above 32 neighbours: count the rest
        const int64_t p = p0 + lane;
        if (p < end) entries += __ldcg(&a.nmem[a.adj[p]]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) entries += __shfl_xor_sync(FULL, entries, o);
    entries += cx;
    if (d > a.warp_max_deg || entries > HW / 2) {   // the whole block evaluates it afterwards
        if (lane == 0) {
            const int h = atomicAdd(&es.nhub, 1);
            es.hub[h] = i;
            es.hub_bound[h] = entries;
        }
        return;
    }
    if (d > 32 || cx > 8) {   // general one-warp path (reloads what it needs)
        eval_team<1>(a, i, x, d, beg, end, entries, y0, cy0, keys, vals, ubs, es.bkey[w], es.bval[w], es.ts, w, 0,
                     serial);
        return;
    }
    uint32_t H = 32;
    while ((int64_t)H < 2 * entries) H <<= 1;
    const uint32_t hm = H - 1;
    for (uint32_t s = lane; s < H; s += 32) {
        keys[s] = EMPTY_KEY;
        vals[s] = 0u;
    }
    __syncwarp();
    if (lane < cx) ht_insert(keys, vals, hm, row_entry(wn.rx0, wn.rx1, rowx, lane), 0u, true);
    __syncwarp();
    const int32_t cmax = __reduce_max_sync(FULL, cy0);
    for (int s = 0; s < cmax; ++s) {
        int32_t C = s < cy0 ? row_entry(ry0, ry1, rowy, s) : -2 - lane;
        unsigned mask = __match_any_sync(FULL, C);
        if (C >= 0 && lane == __ffs(mask) - 1) ht_insert(keys, vals, hm, C, (uint32_t)__popc(mask), false);
    }
    unsigned long long pb = on ? 8ull + 4ull * (unsigned long long)cy0 : 0ull;
    __syncwarp();
    Best bj, bl;
    decide_node<1>(a, i, d, cx, H, keys, vals, ubs, es.bkey[w], es.bval[w], es.ts, w, 0, serial, pb, bj, bl);
    wn.j = __shfl_sync(FULL, bj.c, 0);
    wn.kj = __shfl_sync(FULL, bj.k, 0);
    wn.l = __shfl_sync(FULL, bl.c, 0);
    wn.kl = __shfl_sync(FULL, bl.k, 0);
    wn.fused = 1;
}

__device__ void apply_fused(const RunArgs &a, int64_t bstart, int32_t blen, int i, const WarpNode &wn,
                            unsigned long long serial, unsigned long long &nj, unsigned long long &nl) {
    if (!wn.valid) return;
    if (!wn.fused) {
        apply_node(a, bstart, blen, i, serial, nj, nl);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int32_t j = wn.j, l = wn.l;
    if (j < 0 && l < 0) {
        if (a.profile && lane == 0) atomicAdd(&a.ds->prof_bytes, 8ull);
        return;
    }
    int jj = 0, jl = 0, ll = 0;
    if (wn.py0 >= bstart && wn.py0 < bstart + blen) {
        const int64_t iy = wn.py0 - bstart;
        const int32_t aj = __ldcg(&a.act[iy]), al = __ldcg(&a.act[a.qcap + iy]);
        jj = j >= 0 && aj == j;
        jl = j >= 0 && al == j;
        ll = l >= 0 && al == l;
    }
    jj = __reduce_add_sync(FULL, jj);
    jl = __reduce_add_sync(FULL, jl);
    ll = __reduce_add_sync(FULL, ll);
    // new row from the registers: leave l, insert j, ascending
    int32_t *row = a.mem + (int64_t)wn.x * a.K;
    const int32_t c = wn.cx;
    const int32_t v = lane < c ? row_entry(wn.rx0, wn.rx1, row, lane) : 0;
    const bool keep = lane < c && v != l;
    const unsigned km = __ballot_sync(FULL, keep);
    const int kept = __popc(km);
    int ins = kept;
    if (j >= 0) ins = __popc(__ballot_sync(FULL, keep && v < j));
    int32_t c_new = c;
    if (j >= 0 && kept >= a.K) {
        if (lane == 0) atomicOr(&a.ds->err, DERR_CAPACITY);
    } else {
        if (keep) {
            const int dst = __popc(km & lanemask_lt());
            row[dst + ((j >= 0 && dst >= ins) ? 1 : 0)] = v;
        }
        if (j >= 0 && lane == 0) row[ins] = j;
        c_new = kept + (j >= 0 ? 1 : 0);
    }
    if (lane == 0) {
        if (l >= 0) {
            atomicAdd(&a.comm[l].n, -1);
            atomicAdd(&a.comm[l].vol, (uint32_t)(-wn.d));
            atomicAdd(&a.comm[l].m2, (uint32_t)(-2 * wn.kl + ll));
            ++nl;
        }
        if (j >= 0) {
            atomicAdd(&a.comm[j].n, 1);
            atomicAdd(&a.comm[j].vol, (uint32_t)wn.d);
            atomicAdd(&a.comm[j].m2, (uint32_t)(2 * wn.kj + jj - 2 * jl));
            ++nj;
        }
        a.nmem[wn.x] = c_new;
        if (a.profile)
            atomicAdd(&a.ds->prof_bytes, 24ull + 4ull * (unsigned long long)c + 12ull * ((j >= 0) + (l >= 0)) +
                                             16ull * (unsigned long long)wn.d);
    }
}

template <int T>
__global__ void __launch_bounds__(EV_THREADS, 2) k_iterate(RunArgs a, int64_t q, int64_t first, int64_t count,
                                                           long long spin_limit, int inject_stall, unsigned *flags,
                                                           unsigned epoch, int bar_mode) {
    extern __shared__ int32_t ev_dyn[];
    __shared__ EvalShared es;
    __shared__ int s_ok;
    int32_t *s_keys = ev_dyn;
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(ev_dyn + HB);
    float *s_ub = reinterpret_cast<float *>(ev_dyn + 2 * HB);
    constexpr int TEAMS = EV_WARPS / T;
    const int64_t n = a.nnodes;
    const unsigned nblocks = gridDim.x;
    const int64_t warps = (int64_t)gridDim.x * EV_WARPS;
    const int64_t teams = (int64_t)gridDim.x * TEAMS;
    const int w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * EV_WARPS + w;
    unsigned long long nj = 0, nl = 0;
    if (inject_stall && blockIdx.x == 0) return;   // test hook: a block that never arrives
    NodePrefetch pf;
    pf.valid = 0;
    if (a.qtimes && blockIdx.x == 0 && threadIdx.x == 0) a.qtimes[0] = global_ns();
    if constexpr (T == 1) {
        if (q <= warps) {   // every queue in one round: fused evaluate + apply per warp
            WarpNode wn;
            for (int64_t b = first; b < first + count; ++b) {
                const int64_t bstart = b * q;
                const int32_t blen = (int32_t)min(q, n - bstart);
                const unsigned long long serial = queue_serial(a, b);
                eval_huge(a, bstart, b, serial, es.bkey[w], es.bval[w], es.bs);
                if (threadIdx.x == 0) es.nhub = 0;
                __syncthreads();
                eval_fused(a, bstart, blen, (int)gw, pf, wn, s_keys + w * HW, s_vals + w * HW, s_ub + w * HW, es,
                           serial);
                __syncthreads();
                const int nh = es.nhub;
                for (int h = 0; h < nh; ++h) {
                    const int ih = es.hub[h];
                    eval_block(a, ih, a.order[bstart + ih], (int64_t)es.hub_bound[h], s_keys, s_vals, s_ub, es.bkey[w],
                               es.bval[w], es.bs, serial);
                }
                if (!grid_sync(flags, nblocks, ++epoch, spin_limit, a.ds, &s_ok, bar_mode)) return;
                if (b + 1 < first + count) {
                    const int64_t nstart = (b + 1) * q;
                    prefetch_node(a, nstart, (int32_t)min(q, n - nstart), (int)gw, 0, pf);
                } else {
                    pf.valid = 0;
                }
                apply_fused(a, bstart, blen, (int)gw, wn, serial, nj, nl);
                if (!grid_sync(flags, nblocks, ++epoch, spin_limit, a.ds, &s_ok, bar_mode)) return;
                if (a.qtimes && blockIdx.x == 0 && threadIdx.x == 0) a.qtimes[b - first + 1] = global_ns();
            }
            flush_counts(a, nj, nl);
            return;
        }
    }
    for (int64_t b = first; b < first + count; ++b) {
        const int64_t bstart = b * q;
        const int32_t blen = (int32_t)min(q, n - bstart);
        const unsigned long long serial = queue_serial(a, b);
        const int64_t base0 = (int64_t)blockIdx.x * TEAMS;
        eval_huge(a, bstart, b, serial, es.bkey[w], es.bval[w], es.bs);
        for (int64_t base = base0; base < blen; base += teams)
            eval_group<T>(a, bstart, blen, (int)base, serial, s_keys, s_vals, s_ub, es, base == base0 ? &pf : nullptr);
        if (!grid_sync(flags, nblocks, ++epoch, spin_limit, a.ds, &s_ok, bar_mode)) return;
        // the next queue's first node of this team: its static data loads while
        // this queue is applied and the barrier completes
        if (b + 1 < first + count) {
            const int64_t nstart = (b + 1) * q;
            prefetch_node(a, nstart, (int32_t)min(q, n - nstart), (int)(base0 + w / T), w % T, pf);
        } else {
            pf.valid = 0;
        }
        for (int64_t i = gw; i < blen; i += warps) apply_node(a, bstart, blen, i, serial, nj, nl);
        if (!grid_sync(flags, nblocks, ++epoch, spin_limit, a.ds, &s_ok, bar_mode)) return;
        if (a.qtimes && blockIdx.x == 0 && threadIdx.x == 0) a.qtimes[b - first + 1] = global_ns();
    }
    flush_counts(a, nj, nl);
}

// ---------------------------------------------------------------------------
// a9: iteration end.
// ---------------------------------------------------------------------------
// Communities with fewer than two members are removed (their last member
// loses the membership).  Whether a row sees a community's count before or
// after its reset, the count is < 2 either way, so one kernel does both.
__global__ void k_prune(RunArgs a, int64_t n, int64_t ncomm) {
    int32_t mc = 0;
    unsigned long long memb = 0, live = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n + ncomm;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < n) {
            int32_t *row = a.mem + idx * a.K;
            const int32_t c = a.nmem[idx];
            int32_t o = 0;
            for (int32_t s = 0; s < c; ++s) {
                int32_t C = row[s];
                if (__ldcg(&a.comm[C].n) >= 2) {
                    if (a.kmem) a.kmem[idx * a.K + o] = a.kmem[idx * a.K + s];
                    row[o++] = C;
                }
            }
            if (o != c) a.nmem[idx] = o;
            mc = max(mc, o);
            memb += (unsigned long long)o;
        } else {
            const int64_t C = idx - n;
            const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
            if (r.x < 2) {
                if (r.x != 0 || r.y != 0 || r.z != 0) *reinterpret_cast<int4 *>(&a.comm[C]) = make_int4(0, 0, 0, 0);
            } else {
                ++live;
            }
        }
    }
    mc = __reduce_max_sync(FULL, mc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        memb += __shfl_down_sync(FULL, memb, o);
        live += __shfl_down_sync(FULL, live, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mc) atomicMax(&a.ds->maxcnt, mc);
        if (memb) atomicAdd(&a.ds->memberships, memb);
        if (live) atomicAdd(&a.ds->live_comms, live);
    }
}

__device__ __forceinline__ bool row_has(const int32_t *row, int32_t c, int32_t C) {
    int lo = 0, hi = c - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int32_t v = row[mid];
        if (v == C) return true;
        if (v < C) lo = mid + 1; else hi = mid - 1;
    }
    return false;
}

// WCC-hat(P) = sum over memberships (x, C) of WCC-hat(x, C), with
// deg(x, C) read from the membership's count under the paper's gain (kept
// exact through every apply), else counted over x's neighbours; exact sum, so the total does not
// depend on the order of the additions.  Warps take runs of node ids from a
// counter; a node of degree > TOT_CHUNK is counted in chunks of TOT_CHUNK
// neighbours taken from a second counter, each chunk adding its counts to the
// node's counters in global memory, and the warp that finishes the node's
// last chunk evaluates its memberships (and clears the counters).
constexpr int TOT_WARPS = 8;
constexpr int TOT_ROW = 64;      // own rows up to this length are counted in one pass
constexpr int TOT_CHUNK = 1024;  // neighbours per work unit of a high-degree node
constexpr int TOT_BATCH = 32;    // node ids per grab

// Own row of at most four communities held in registers: each lane counts
// its neighbours' memberships against them (rows ascending, -1 past the end),
// four neighbours per step with their loads issued together.
__device__ __forceinline__ void tot_match(int32_t C, const int4 &rx, int &k0, int &k1, int &k2, int &k3) {
    k0 += C == rx.x;
    k1 += C == rx.y;
    k2 += C == rx.z;
    k3 += C == rx.w;
}

__device__ __forceinline__ void tot_count4(const RunArgs &a, int64_t pb, int64_t pe, const int4 &rx, int &k0, int &k1,
                                           int &k2, int &k3) {
    const int lane = threadIdx.x & 31;
    constexpr int U = 4;
    for (int64_t p0 = pb; p0 < pe; p0 += 32 * U) {
        int32_t y[U], cy[U];
        int4 r[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t p = p0 + j * 32 + lane;
            y[j] = p < pe ? a.adj[p] : -1;
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            cy[j] = y[j] >= 0 ? __ldcg(&a.nmem[y[j]]) : 0;
            r[j] = y[j] >= 0 ? __ldcg(reinterpret_cast<const int4 *>(a.mem + (int64_t)y[j] * a.K))
                             : make_int4(-1, -1, -1, -1);
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (cy[j] > 0) tot_match(r[j].x, rx, k0, k1, k2, k3);
            if (cy[j] > 1) tot_match(r[j].y, rx, k0, k1, k2, k3);
            if (cy[j] > 2) tot_match(r[j].z, rx, k0, k1, k2, k3);
            if (cy[j] > 3) tot_match(r[j].w, rx, k0, k1, k2, k3);
            for (int32_t s = 4; s < cy[j]; ++s)
                tot_match(__ldcg(&a.mem[(int64_t)y[j] * a.K + s]), rx, k0, k1, k2, k3);
        }
    }
}

// Counts of the c <= TOT_ROW communities in row_s (ascending, shared) among
// neighbours [pb, pe), added to cnt_s.
__device__ __forceinline__ void tot_count_smem(const RunArgs &a, int64_t pb, int64_t pe, const int32_t *row_s, int c,
                                               int32_t *cnt_s) {
    const int lane = threadIdx.x & 31;
    const int32_t lo = row_s[0], hi = row_s[c - 1];
    for (int64_t p = pb + lane; p < pe; p += 32) {
        const int32_t y = a.adj[p];
        const int32_t cy = __ldcg(&a.nmem[y]);
        const int32_t *ry = a.mem + (int64_t)y * a.K;
        for (int32_t s = 0; s < cy; ++s) {
            const int32_t C = __ldcg(&ry[s]);
            if (C < lo) continue;
            if (C > hi) break;
            int l = 0, h = c - 1;
            while (l <= h) {
                const int mid = (l + h) >> 1;
                const int32_t v = row_s[mid];
                if (v == C) {
                    atomicAdd(&cnt_s[mid], 1);
                    break;
                }
                if (v < C) l = mid + 1; else h = mid - 1;
            }
        }
    }
}

__device__ __forceinline__ void tot_member(const RunArgs &a, unsigned long long *acc, int32_t C, int64_t k,
                                           int32_t d) {
    const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
    if (a.gsacc)   // a batch: the sum of the community's graph
        sacc_add(a.gsacc + (int64_t)r.w * SACC_CHUNKS, wcchat_member(k, d, r.x, (uint32_t)r.y, a.gcc[r.w]));
    else
        sacc_add(acc, wcchat_member(k, d, r.x, (uint32_t)r.y, a.cc));
}

// Memberships waiting for their FP64 term, per warp: evaluated 32 at a time so
// that the (slow) double-precision pipe runs with every lane busy.
struct TotBuf {
    int32_t *C, *k, *d;
    int n;
};

__device__ __forceinline__ void tot_flush(const RunArgs &a, unsigned long long *acc, TotBuf &b) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < b.n) tot_member(a, acc, b.C[lane], b.k[lane], b.d[lane]);
    __syncwarp();
    b.n = 0;
}

// Warp-collective: lanes with `has` queue (C, k, d).
__device__ __forceinline__ void tot_push(const RunArgs &a, unsigned long long *acc, TotBuf &b, bool has, int32_t C,
                                         int32_t k, int32_t d) {
    const unsigned m = __ballot_sync(FULL, has);
    const int cnt = __popc(m);
    if (cnt == 0) return;
    if (b.n + cnt > 32) tot_flush(a, acc, b);
    if (has) {
        const int s = b.n + __popc(m & lanemask_lt());
        b.C[s] = C;
        b.k[s] = k;
        b.d[s] = d;
    }
    b.n += cnt;
}

// deg(x, C) for x's memberships over neighbours [pb, pe).  whole: add the
// node's terms to acc; otherwise add the counts to the node's global counters
// `gcnt`.
__device__ void tot_node(const RunArgs &a, int32_t x, int64_t pb, int64_t pe, bool whole, int32_t *gcnt,
                         unsigned long long *acc, TotBuf &buf, int32_t *row_s, int32_t *cnt_s) {
    const int lane = threadIdx.x & 31;
    const int32_t c = __ldcg(&a.nmem[x]);
    const int32_t d = a.deg[x];
    const int32_t *row = a.mem + (int64_t)x * a.K;
    if (c <= 4) {
        int4 rx = __ldcg(reinterpret_cast<const int4 *>(row));
        if (c < 2) rx.y = -3;
        if (c < 3) rx.z = -3;
        if (c < 4) rx.w = -3;
        int k0 = 0, k1 = 0, k2 = 0, k3 = 0;
        tot_count4(a, pb, pe, rx, k0, k1, k2, k3);
        k0 = __reduce_add_sync(FULL, k0);
        k1 = __reduce_add_sync(FULL, k1);
        k2 = __reduce_add_sync(FULL, k2);
        k3 = __reduce_add_sync(FULL, k3);
        const int k = lane == 0 ? k0 : lane == 1 ? k1 : lane == 2 ? k2 : k3;
        const int32_t C = lane == 0 ? rx.x : lane == 1 ? rx.y : lane == 2 ? rx.z : rx.w;
        if (whole) tot_push(a, acc, buf, lane < c, C, k, d);
        else if (lane < c && k) atomicAdd(&gcnt[lane], k);
    } else if (c <= TOT_ROW) {
        for (int j = lane; j < c; j += 32) {
            row_s[j] = __ldcg(&row[j]);
            cnt_s[j] = 0;
        }
        __syncwarp();
        tot_count_smem(a, pb, pe, row_s, c, cnt_s);
        __syncwarp();
        for (int j0 = 0; j0 < c; j0 += 32) {
            const int j = j0 + lane;
            const int32_t C = j < c ? row_s[j] : 0, k = j < c ? cnt_s[j] : 0;
            if (whole) tot_push(a, acc, buf, j < c, C, k, d);
            else if (j < c && k) atomicAdd(&gcnt[j], k);
        }
        __syncwarp();
    } else {
        for (int32_t s = 0; s < c; ++s) {
            const int32_t C = __ldcg(&row[s]);
            int cnt = 0;
            for (int64_t p = pb + lane; p < pe; p += 32) {
                const int32_t y = a.adj[p];
                cnt += row_has(a.mem + (int64_t)y * a.K, __ldcg(&a.nmem[y]), C);
            }
            cnt = __reduce_add_sync(FULL, cnt);
            if (whole) tot_push(a, acc, buf, lane == 0, C, cnt, d);
            else if (lane == 0 && cnt) atomicAdd(&gcnt[s], cnt);
        }
    }
}

__global__ void __launch_bounds__(TOT_WARPS * 32) k_total(RunArgs a, int64_t n) {
    __shared__ unsigned long long acc[SACC_CHUNKS];
    __shared__ int32_t s_row[TOT_WARPS][TOT_ROW];
    __shared__ int32_t s_cnt[TOT_WARPS][TOT_ROW];
    __shared__ int32_t s_buf[TOT_WARPS][3][32];
    for (int s = threadIdx.x; s < SACC_CHUNKS; s += blockDim.x) acc[s] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *row_s = s_row[w], *cnt_s = s_cnt[w];
    TotBuf buf{s_buf[w][0], s_buf[w][1], s_buf[w][2], 0};
    if (a.kmem) {   // the paper's gain keeps deg(x, C) of every membership: no recount
        for (;;) {
            long long b0 = 0;
            if (lane == 0) b0 = (long long)atomicAdd(&a.tot_next[0], 1u) * 32;
            b0 = __shfl_sync(FULL, b0, 0);
            if (b0 >= n) break;
            const int64_t x = b0 + lane;   // a node per lane
            int32_t c = 0, d = 0;
            if (x < n) {
                c = __ldcg(&a.nmem[x]);
                if (!dbg_ok(a, c >= 0 && c <= a.K)) c = 0;
                d = a.deg[x];
            }
            const int cmax = __reduce_max_sync(FULL, c);
            for (int s = 0; s < cmax; ++s) {
                int32_t C = 0, k = 0;
                bool has = s < c;
                if (has) {
                    C = __ldcg(&a.mem[x * a.K + s]);
                    k = __ldcg(&a.kmem[x * a.K + s]);
                    has = dbg_ok(a, C >= 0 && C < a.nnodes && k >= 0 && k <= d);
                }
                tot_push(a, acc, buf, has, C, k, d);
            }
        }
        if (buf.n > 0) tot_flush(a, acc, buf);
        __syncthreads();
        for (int s = threadIdx.x; s < SACC_CHUNKS; s += blockDim.x)
            if (acc[s]) atomicAdd(&a.ds->sacc[s], acc[s]);
        return;
    }
    // nodes of degree <= TOT_CHUNK, whole
    for (;;) {
        long long b0 = 0;
        if (lane == 0) b0 = (long long)atomicAdd(&a.tot_next[0], 1u) * TOT_BATCH;
        b0 = __shfl_sync(FULL, b0, 0);
        if (b0 >= n) break;
        const int64_t bend = min(n, (int64_t)b0 + TOT_BATCH);
        for (int64_t x = b0; x < bend; ++x) {
            if (__ldcg(&a.nmem[x]) == 0) continue;
            const int64_t pb = a.off[x], pe = a.off[x + 1];
            if (pe - pb > TOT_CHUNK) continue;
            tot_node(a, (int32_t)x, pb, pe, true, nullptr, acc, buf, row_s, cnt_s);
        }
    }
    // chunks of the larger nodes
    for (;;) {
        long long ch = 0;
        if (lane == 0) ch = (long long)atomicAdd(&a.tot_next[1], 1u);
        ch = __shfl_sync(FULL, ch, 0);
        if (ch >= a.tot_nchunks) break;
        const int h = a.tot_chunk_hub[ch];
        const int32_t x = a.tot_hubs[h];
        const int nch = a.tot_first[h + 1] - a.tot_first[h];
        const int64_t pb = a.off[x] + (int64_t)(ch - a.tot_first[h]) * TOT_CHUNK;
        const int64_t pe = min(a.off[x + 1], pb + TOT_CHUNK);
        int32_t *gcnt = a.tot_cnt + (int64_t)h * a.K;
        const int32_t c = __ldcg(&a.nmem[x]);
        if (c > 0) tot_node(a, x, pb, pe, false, gcnt, acc, buf, row_s, cnt_s);
        __threadfence();
        unsigned old = 0;
        if (lane == 0) old = atomicAdd(&a.tot_done[h], 1u);
        old = __shfl_sync(FULL, old, 0);
        if (old == (unsigned)(nch - 1)) {   // last chunk of x: its counts are complete
            __threadfence();
            const int32_t d = a.deg[x];
            const int32_t *row = a.mem + (int64_t)x * a.K;
            for (int j0 = 0; j0 < c; j0 += 32) {
                const int j = j0 + lane;
                const int32_t C = j < c ? __ldcg(&row[j]) : 0, k = j < c ? atomicExch(&gcnt[j], 0) : 0;
                tot_push(a, acc, buf, j < c, C, k, d);
            }
            if (lane == 0) a.tot_done[h] = 0u;
        }
    }
    if (buf.n > 0) tot_flush(a, acc, buf);
    __syncthreads();
    for (int s = threadIdx.x; s < SACC_CHUNKS; s += blockDim.x)
        if (acc[s]) atomicAdd(&a.ds->sacc[s], acc[s]);
}

// Per-graph totals of a batch (one thread per graph); the shared counters
// are finalised by k_finalize as for one graph.
__global__ void k_finalize_batch(unsigned long long *gsacc, int64_t G, double *gT) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += (int64_t)gridDim.x * blockDim.x)
        gT[i] = sacc_round_and_clear(gsacc + i * SACC_CHUNKS);
}

__global__ void k_finalize(DevScalars *ds, Readback *rbd, int advance) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double T = sacc_round_and_clear(ds->sacc);
    ds->total = T;
    rbd->total = T;
    rbd->joins = ds->joins;
    rbd->leaves = ds->leaves;
    rbd->live_comms = ds->live_comms;
    rbd->memberships = ds->memberships;
    rbd->maxcnt = ds->maxcnt;
    rbd->err = ds->err;
    ds->kb = ds->maxcnt + 1;
    ds->joins = 0;
    ds->leaves = 0;
    ds->live_comms = 0;
    ds->memberships = 0;
    ds->maxcnt = 0;
    if (advance) ds->iter += 1;
}

__global__ void k_regrow(const int32_t *mem, const int32_t *nmem, int64_t n, int32_t K, int32_t *mem2,
                         int32_t K2, const int32_t *kmem, int32_t *kmem2) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = nmem[x];
        for (int32_t s = 0; s < c; ++s) mem2[x * K2 + s] = mem[x * K + s];
        if (kmem)
            for (int32_t s = 0; s < c; ++s) kmem2[x * K2 + s] = kmem[x * K + s];
    }
}

RunArgs make_args(lf_graph *g, Readback *rbd) {
    RunArgs a;
    a.off = g->off;
    a.adj = g->adj;
    a.deg = g->deg;
    a.order = g->order;
    a.pos = g->pos;
    a.comm = g->comm;
    a.mem = g->mem;
    a.nmem = g->nmem;
    a.K = g->K;
    a.qcap = g->qcap;
    a.act = g->act;
    a.ds = g->ds;
    a.rbd = rbd;
    a.cc = g->cc;
    a.nbatches = 0;
    a.nnodes = g->n;
    a.warp_max_deg = g->warp_max_degree > 0 ? g->warp_max_degree : 0x7fffffff;
    a.profile = g->profile;
    a.debug = g->debug_checks;
    a.qtimes = g->qtimes;
    a.huge_deg = g->hub_qoff ? g->hub_degree : 0x7fffffff;
    a.hub_pos = g->hub_pos;
    a.hub_qoff = g->hub_qoff;
    a.hub_toff = g->hub_toff;
    a.hub_tcap = g->hub_tcap;
    a.hub_tcap_w = g->hub_tcap;
    a.hkeys = g->hub_scratch;
    a.hvals = reinterpret_cast<uint32_t *>(g->hub_scratch + g->hub_slots);
    a.hub_ub = reinterpret_cast<float *>(g->hub_scratch + 2 * g->hub_slots);
    a.hub_lb = reinterpret_cast<float *>(g->hub_scratch + 3 * g->hub_slots);
    a.hub_chunk_h = g->hub_chunk_h;
    a.hub_chunk_c = g->hub_chunk_c;
    a.hub_nch = g->hub_nch;
    a.hub_done = g->hub_done;
    a.hub_ncand = g->hub_ncand;
    a.hub_lbj = g->hub_lbj;
    a.hub_lbl = g->hub_lbl;
    a.hub_item_base = g->hub_item_base;
    a.hub_nitems = g->hub_nitems;
    a.hub_items_done = g->hub_items_done;
    a.hub_items = g->hub_items;
    a.hub_item_g = g->hub_item_g;
    a.hub_item_ck = g->hub_item_ck;
    a.hub_qctr = g->hub_qctr;
    // FP32 screen: cc must be a normal float with room to spare; delta bounds
    // 15 FP32 roundings (20 ulp) and the FP32 subtraction, the FP64 estimator's error u (m2 + 3 vol +
    // 17) with m2, vol <= 2m, the two gain subtractions, and a 2% margin.
    a.screen = (g->cc >= 1e-30 && g->screen) ? 1 : 0;
    a.cc32 = (float)g->cc;
    const double u64 = 1.1102230246251565e-16, u32 = 5.960464477539063e-08;
    a.delta = (float)(1.02 * (21.0 * u32 + u64 * (200.0 + 8.0 * (double)g->m) + 2.0 * u64) + 1e-9);
    a.gcc = g->ngraphs > 0 ? g->gcc : nullptr;
    a.gcc32 = g->ngraphs > 0 ? g->gcc32 : nullptr;
    a.gsacc = g->ngraphs > 0 ? g->gsacc : nullptr;
    a.gid = g->ngraphs > 0 ? g->gid : nullptr;
    if (g->ngraphs > 0) {
        a.order = g->qorder ? g->qorder : g->order;   // the queue schedule of the active graphs
        a.pos = g->qpos ? g->qpos : g->pos;
        a.screen = g->screen ? 1 : 0;                 // per graph: cc32 = 0 keeps every candidate
    }
    a.tot_hubs = g->tot_hubs;
    a.tot_chunk_hub = g->tot_chunk_hub;
    a.tot_first = g->tot_first;
    a.tot_cnt = g->tot_cnt;
    a.tot_done = g->tot_done;
    a.tot_next = g->tot_next;
    a.tot_nchunks = g->tot_nchunks;
    const bool lit = g->gain_rule == LF_GAIN_LITERAL;
    a.kmem = lit ? g->kmem : nullptr;
    a.cm_off = g->cm_off;
    a.cm_node = g->cm_node;
    a.cm_cnt = g->cm_cnt;
    a.jl_head = g->jl_head;
    a.jl_next = g->jl_next;
    a.jl_node = g->jl_node;
    a.jl_count = g->lit_misc;
    a.litF = g->litF;
    a.touched = g->touched;
    a.ntouched = g->lit_ctr;
    a.tstamp = g->tstamp;
    a.lg_cap = g->lg_cap;
    a.lg_dv = static_cast<float *>(g->lg_area);
    a.lg_keys = reinterpret_cast<int32_t *>(a.lg_dv + g->lg_cap);
    a.lg_vals = reinterpret_cast<uint32_t *>(a.lg_keys + g->lg_cap);
    a.lg_aux = reinterpret_cast<int32_t *>(a.lg_vals + g->lg_cap);
    a.lit_hub_deg = g->lh_n > 0 ? LIT_HUB_DEG : 0x7fffffff;
    if (lit) a.screen = g->screen ? 1 : 0;   // brackets need no FP32 range condition
    return a;
}

Readback *device_readback(lf_graph *g) {
    // the device-side Readback sits right after the DevScalars block
    return reinterpret_cast<Readback *>(g->ds + 1);
}

// Timing events: inside a stream capture they must be external event nodes,
// otherwise the capture keeps only the ordering and records nothing.
void record_event(lf_graph *g, cudaEvent_t e, bool capturing) {
    if (capturing) LF_CUDA(cudaEventRecordWithFlags(e, g->stream, cudaEventRecordExternal));
    else LF_CUDA(cudaEventRecord(e, g->stream));
}

int num_sms() {
    int dev = 0, sms = 0;
    LF_CUDA(cudaGetDevice(&dev));
    LF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, sms);
}

// Resident blocks per SM of a kernel at a launch shape (at least 1).
template <typename K>
int blocks_per_sm(K kernel, int threads, size_t smem) {
    int v = 0;
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem));
    return std::max(1, v);
}

// Queue b: positions [start, start + len) of the order the kernels read (the
// batch schedule when there is one).
void queue_bounds(const lf_graph *g, int64_t q, int64_t b, int64_t &start, int32_t &len) {
    if (!g->sched.empty()) {
        start = g->sched[(size_t)b];
        len = (int32_t)(g->sched[(size_t)b + 1] - start);
    } else {
        start = b * q;
        len = (int32_t)std::min<int64_t>(q, g->n - start);
    }
}

int64_t num_queues(const lf_graph *g, int64_t q) {
    if (!g->sched.empty()) return (int64_t)g->sched.size() - 1;
    return g->n > 0 ? (g->n + q - 1) / q : 0;
}

int64_t max_queue(const lf_graph *g, int64_t q) {
    if (g->sched.empty()) return q;
    int64_t m = 1;
    for (size_t b = 0; b + 1 < g->sched.size(); ++b) m = std::max(m, g->sched[b + 1] - g->sched[b]);
    return m;
}

// Warps per node: as many as keep q x T warps within about 16 per SM, so that
// small queues spread each node's loads over more warps.
int choose_team(lf_graph *g, int64_t q) {
    if (g->warps_per_node == 1 || g->warps_per_node == 2 || g->warps_per_node == 4 || g->warps_per_node == 8)
        return g->warps_per_node;
    const int64_t target = (int64_t)num_sms() * 16;
    int T = EV_WARPS;
    while (T > 1 && q * T > target) T >>= 1;
    return T;
}

// Launch with programmatic stream serialisation (see pdl_wait).
template <typename... P, typename... A>
void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LF_CUDA(cudaLaunchKernelEx(&cfg, k, args...));
}

template <int T>
void launch_eval(lf_graph *g, const RunArgs &a, int64_t bstart, int32_t blen, int64_t b) {
    constexpr int teams = EV_WARPS / T;
    launch_pdl(k_eval<T>, (unsigned)((blen + teams - 1) / teams), EV_THREADS, EV_DYN_SMEM, g->stream, a, bstart,
               blen, b);
}

void set_eval_attrs() {
    LF_CUDA(cudaFuncSetAttribute(k_eval<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_eval<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_eval<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_eval<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_eval_dyn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_eval_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_eval_tdyn<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_huge_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(HUGE_SH * 8)));
    LF_CUDA(cudaFuncSetAttribute(k_lit_eval<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LIT_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_lit_eval<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LIT_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_lit_eval<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LIT_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_lit_eval<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LIT_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_lit_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LIT_SMEM));
}

void drop_graph(lf_graph *g) {
    if (g->iter_exec) {
        cudaGraphExecDestroy(g->iter_exec);
        g->iter_exec = nullptr;
    }
}

// Queues at least this large are evaluated by k_eval_dyn (one warp per node,
// nodes handed out by a counter) and k_eval_blocks.
constexpr int64_t DYN_MIN_Q = 4096;

bool use_dyn(lf_graph *g, int64_t q) { return q >= DYN_MIN_Q && choose_team(g, q) == 1; }

void ensure_side(lf_graph *g) {
    if (g->side) return;
    LF_CUDA(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
    LF_CUDA(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
    LF_CUDA(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
}

// Four counters per queue: next node, list-1 count, list-1 next, list-2
// count; two lists of up to q entries (positions, then entry counts).
void ensure_dyn(lf_graph *g, int64_t q, int64_t nb) {
    if (g->dyn_ctr_cap < 4 * nb) {
        if (g->dyn_ctr) dfree(g, g->dyn_ctr);
        g->dyn_ctr = dalloc_n<uint32_t>(g, 4 * nb);
        g->dyn_ctr_cap = 4 * nb;
        drop_graph(g);
    }
    if (g->dyn_list_cap < q) {
        if (g->dyn_list) dfree(g, g->dyn_list);
        if (g->dyn_bound) dfree(g, g->dyn_bound);
        g->dyn_list = dalloc_n<int32_t>(g, 2 * q);
        g->dyn_bound = dalloc_n<long long>(g, 2 * q);
        g->dyn_list_cap = q;
        drop_graph(g);
    }
}

void launch_batches(lf_graph *g, const RunArgs &a, int64_t q, int64_t first, int64_t count,
                    bool capturing = false) {
    const bool sched = !g->sched.empty();
    const int T0 = choose_team(g, q);
    const bool any_dyn = sched ? use_dyn(g, max_queue(g, q)) : use_dyn(g, q);
    const int64_t nhubs = g->hub_qoff_host.empty() ? 0 : g->hub_qoff_host.back();
    if (nhubs > 0 && first == 0) {
        k_hub_caps<<<grid_for(nhubs * 32, EV_THREADS, 4096), EV_THREADS, 0, g->stream>>>(a, g->hub_wcap, nhubs);
        ++g->launches;
    }
    int dyn_grid = 0, blk_grid = 0;
    if (any_dyn) {
        // computed once (function-local statics: thread-safe, as the serving workers need)
        static const int per_sm = blocks_per_sm(k_eval_dyn, EV_THREADS, EV_DYN_SMEM);
        static const int per_sm_blk = blocks_per_sm(k_eval_blocks, EV_THREADS, EV_DYN_SMEM);
        dyn_grid = num_sms() * std::max(1, per_sm);
        blk_grid = num_sms() * std::max(1, per_sm_blk);
        LF_CUDA(cudaMemsetAsync(g->dyn_ctr + 4 * first, 0, (size_t)(4 * count) * sizeof(uint32_t), g->stream));
    }
    if (any_dyn || nhubs > 0) ensure_side(g);

    const bool prof = g->profile && (int64_t)g->prof_ev.size() >= 2 * (first + count);
    for (int64_t b = first; b < first + count; ++b) {
        int64_t bstart;
        int32_t blen;
        queue_bounds(g, q, b, bstart, blen);
        const int T = sched ? choose_team(g, blen) : T0;
        const bool dyn = sched ? (blen >= DYN_MIN_Q && T == 1) : any_dyn;
        if (prof) record_event(g, g->prof_ev[2 * b], capturing);
        const int64_t nch =
            g->hub_cqoff_host.empty() ? 0 : g->hub_cqoff_host[(size_t)b + 1] - g->hub_cqoff_host[(size_t)b];
        const bool fork = nch > 0;   // hub chunks on the second stream, beside the other evaluations
        if (fork) {
            LF_CUDA(cudaEventRecord(g->ev_fork, g->stream));
            LF_CUDA(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        }
        if (nch > 0) {
            cudaStream_t hs = fork ? g->side : g->stream;
            const bool big = !g->hub_qbig.empty() && g->hub_qbig[(size_t)b];
            if (big) LF_CUDA(cudaMemsetAsync(g->hub_qctr + 3 * b, 0, 3 * sizeof(uint32_t), hs));
            k_huge_chunks<<<(unsigned)nch, EV_THREADS, (size_t)HUGE_SH * 8, hs>>>(a, bstart, b,
                                                                                g->hub_cqoff_host[(size_t)b]);
            ++g->launches;
            if (big) {
                k_huge_screen<<<(unsigned)(6 * num_sms()), EV_THREADS, 0, hs>>>(a, b);
                k_huge_eval<<<(unsigned)(3 * num_sms()), EV_THREADS, 0, hs>>>(a, bstart, b);
                g->launches += 2;
            }
        }
        if (fork) LF_CUDA(cudaEventRecord(g->ev_join, g->side));
        if (dyn) {
            uint32_t *ctr = g->dyn_ctr + 4 * b;
            const int64_t L = g->dyn_list_cap;
            const unsigned grid = (unsigned)std::min<int64_t>(dyn_grid, (blen + EV_WARPS - 1) / EV_WARPS);
            k_eval_dyn<<<grid, EV_THREADS, EV_DYN_SMEM, g->stream>>>(a, bstart, blen, b, ctr, g->dyn_list,
                                                                      g->dyn_bound);
            k_eval_tdyn<4><<<(unsigned)blk_grid, EV_THREADS, EV_DYN_SMEM, g->stream>>>(
                a, bstart, b, ctr + 1, g->dyn_list, g->dyn_bound, ctr + 3, g->dyn_list + L, g->dyn_bound + L);
            k_eval_blocks<<<(unsigned)blk_grid, EV_THREADS, EV_DYN_SMEM, g->stream>>>(a, bstart, b, ctr + 3,
                                                                                     g->dyn_list + L,
                                                                                     g->dyn_bound + L);
            g->launches += 3;
            if (fork) LF_CUDA(cudaStreamWaitEvent(g->stream, g->ev_join, 0));
        } else {
            switch (T) {
            case 1: launch_eval<1>(g, a, bstart, blen, b); break;
            case 2: launch_eval<2>(g, a, bstart, blen, b); break;
            case 4: launch_eval<4>(g, a, bstart, blen, b); break;
            default: launch_eval<8>(g, a, bstart, blen, b); break;
            }
            ++g->launches;
            if (fork) LF_CUDA(cudaStreamWaitEvent(g->stream, g->ev_join, 0));
        }
        if (prof) record_event(g, g->prof_ev[2 * b + 1], capturing);
        launch_pdl(k_apply, grid_for((int64_t)blen * 32, AP_THREADS, 1 << 30), AP_THREADS, 0, g->stream, a, bstart,
                   blen, b);
        ++g->launches;
    }
    LF_LAUNCHED();
}

void free_lit_hub_plan(lf_graph *g) {
    for (int32_t **pp : {&g->lh_pos, &g->lh_nsr, &g->lh_fh, &g->lh_fc, &g->lh_sh, &g->lh_sr, &g->lh_svc})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    for (int64_t **pp : {&g->lh_toff, &g->lh_soff})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    for (uint32_t **pp : {&g->lh_tcap, &g->lh_ns, &g->lh_svv, &g->lh_heff})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    if (g->lh_lb) dfree(g, g->lh_lb);
    if (g->lh_svl) dfree(g, g->lh_svl);
    if (g->lh_tab) dfree(g, g->lh_tab);
    g->lh_lb = nullptr;
    g->lh_svl = nullptr;
    g->lh_tab = nullptr;
    g->lh_tab_cap = 0;
    g->lh_n = 0;
    g->lh_fq.clear();
    g->lh_sq.clear();
    g->lh_hq.clear();
    g->lh_plan_q = g->lh_plan_sched = -1;
    g->lh_plan_K = 0;
}

// The hubs of every queue (degree > LIT_HUB_DEG): worst-case tables of
// pow2 >= 2 (d+1) K slots (K bounds every row), fill items of LH_CHUNK
// neighbours, slot items of LH_SLOTS slots.  Queues run one after the other,
// so their tables and survivor lists share one area.
void build_lit_hub_plan(lf_graph *g, int64_t q, int64_t nb) {
    if (g->lh_plan_q == q && g->lh_plan_K == g->K && g->lh_plan_sched == g->sched_version) return;
    free_lit_hub_plan(g);
    drop_graph(g);
    g->lh_plan_q = q;
    g->lh_plan_K = g->K;
    g->lh_plan_sched = g->sched_version;
    g->lh_fq.assign((size_t)nb + 1, 0);
    g->lh_sq.assign((size_t)nb + 1, 0);
    g->lh_hq.assign((size_t)nb + 1, 0);
    if (g->n == 0 || g->max_deg <= LIT_HUB_DEG) return;
    const int64_t len = g->sched.empty() ? g->n : g->sched.back();
    std::vector<int32_t> order((size_t)std::max<int64_t>(len, 1)), deg((size_t)g->n);
    if (len > 0)
        LF_CUDA(cudaMemcpyAsync(order.data(), g->sched.empty() ? g->order : g->qorder, (size_t)len * 4,
                                cudaMemcpyDeviceToHost, g->stream));
    LF_CUDA(cudaMemcpyAsync(deg.data(), g->deg, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream));
    LF_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<int32_t> pos, nsr, fh, fc, sh, sr;
    std::vector<int64_t> toff, soff;
    std::vector<uint32_t> tcap;
    int64_t area = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t qs;
        int32_t ql;
        queue_bounds(g, q, b, qs, ql);
        int64_t used = 0;
        for (int64_t p = qs; p < qs + ql; ++p) {
            const int32_t d = deg[(size_t)order[(size_t)p]];
            if (d <= LIT_HUB_DEG) continue;
            uint64_t cap = LH_SLOTS;
            while (cap < 2ull * (uint64_t)(d + 1) * (uint64_t)g->K) cap <<= 1;
            const int32_t h = (int32_t)pos.size();
            pos.push_back((int32_t)(p - qs));
            toff.push_back(used);
            soff.push_back(used / 2);
            tcap.push_back((uint32_t)cap);
            const int32_t nf = (d + LH_CHUNK - 1) / LH_CHUNK, ns = (int32_t)(cap / LH_SLOTS);
            nsr.push_back(ns);
            for (int32_t c = 0; c < nf; ++c) {
                fh.push_back(h);
                fc.push_back(c);
            }
            for (int32_t r = 0; r < ns; ++r) {
                sh.push_back(h);
                sr.push_back(r);
            }
            used += (int64_t)cap;
        }
        g->lh_fq[(size_t)b + 1] = (int64_t)fh.size();
        g->lh_sq[(size_t)b + 1] = (int64_t)sh.size();
        g->lh_hq[(size_t)b + 1] = (int64_t)pos.size();
        area = std::max(area, used);
    }
    const int64_t H = (int64_t)pos.size();
    g->lh_n = H;
    if (H == 0) return;
    auto up = [&](auto *&dst, const auto &v) {
        using E = typename std::decay<decltype(v[0])>::type;
        dst = dalloc_n<E>(g, (int64_t)v.size());
        LF_CUDA(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice, g->stream));
    };
    up(g->lh_pos, pos);
    up(g->lh_nsr, nsr);
    up(g->lh_fh, fh);
    up(g->lh_fc, fc);
    up(g->lh_sh, sh);
    up(g->lh_sr, sr);
    up(g->lh_toff, toff);
    up(g->lh_soff, soff);
    up(g->lh_tcap, tcap);
    g->lh_heff = dalloc_n<uint32_t>(g, H);
    g->lh_ns = dalloc_n<uint32_t>(g, H);
    LF_CUDA(cudaMemsetAsync(g->lh_ns, 0, (size_t)H * 4, g->stream));
    {
        // best lower ends start at -inf (order-preserving: -inf's bits ^ 0x7fffffff)
        const int32_t ninf = (int32_t)(0xff800000u ^ 0x7fffffffu);
        std::vector<int32_t> lb((size_t)(2 * H), ninf);
        up(g->lh_lb, lb);
    }
    g->lh_tab_cap = area;
    g->lh_tab = dalloc(g, (size_t)area * 16);
    // keys empty, counts and corrections zero (the X area needs no start value)
    char *t = static_cast<char *>(g->lh_tab);
    LF_CUDA(cudaMemsetAsync(t + (size_t)area * 4, 0xff, (size_t)area * 4, g->stream));
    LF_CUDA(cudaMemsetAsync(t + (size_t)area * 8, 0, (size_t)area * 8, g->stream));
    g->lh_svc = dalloc_n<int32_t>(g, area / 2);
    g->lh_svv = dalloc_n<uint32_t>(g, area / 2);
    g->lh_svl = dalloc_n<float>(g, area / 2);
    LF_CUDA(cudaStreamSynchronize(g->stream));
}

LitHubPlan lit_hub_plan(lf_graph *g) {
    LitHubPlan hp;
    hp.pos = g->lh_pos;
    hp.toff = g->lh_toff;
    hp.tcap = g->lh_tcap;
    hp.soff = g->lh_soff;
    hp.fh = g->lh_fh;
    hp.fc = g->lh_fc;
    hp.sh = g->lh_sh;
    hp.sr = g->lh_sr;
    hp.nsr = g->lh_nsr;
    hp.heff = g->lh_heff;
    hp.lb = g->lh_lb;
    hp.ns = g->lh_ns;
    hp.sv_c = g->lh_svc;
    hp.sv_v = g->lh_svv;
    hp.sv_l = g->lh_svl;
    const int64_t cap = g->lh_tab_cap;
    hp.dv = static_cast<float *>(g->lh_tab);
    hp.keys = reinterpret_cast<int32_t *>(hp.dv + cap);
    hp.vals = reinterpret_cast<uint32_t *>(hp.keys + cap);
    hp.hs = reinterpret_cast<float *>(hp.vals + cap);
    return hp;
}

// Per-queue launches under the paper's gain: teams evaluate the queue's nodes
// (k_lit_eval), blocks take the nodes too large for a team (k_lit_big), then
// the apply, the neighbours' deg(y,C) updates and the touched communities'
// sums.
void launch_batches_lit(lf_graph *g, const RunArgs &a, int64_t q, int64_t first, int64_t count,
                        bool capturing = false) {
    const bool sched = !g->sched.empty();
    const int T0 = choose_team(g, q);
    static const int per_sm_big = blocks_per_sm(k_lit_big, EV_THREADS, LIT_SMEM);
    const unsigned big_grid = (unsigned)(num_sms() * std::max(1, per_sm_big));
    LF_CUDA(cudaMemsetAsync(g->lit_ctr + 3 * first, 0, (size_t)(3 * count) * sizeof(uint32_t), g->stream));
    LF_CUDA(cudaMemsetAsync(g->lit_used + first, 0, (size_t)count * sizeof(unsigned long long), g->stream));
    const bool prof = g->profile && (int64_t)g->prof_ev.size() >= 2 * (first + count);
    for (int64_t b = first; b < first + count; ++b) {
        int64_t bstart;
        int32_t blen;
        queue_bounds(g, q, b, bstart, blen);
        const int T = sched ? choose_team(g, blen) : T0;
        const int teams = EV_WARPS / T;
        uint32_t *ctr = g->lit_ctr + 3 * b;
        RunArgs ab = a;
        ab.ntouched = ctr + 2;
        if (prof) record_event(g, g->prof_ev[2 * b], capturing);
        const unsigned grid = (unsigned)((blen + teams - 1) / teams);
        switch (T) {
        case 1: launch_pdl(k_lit_eval<1>, grid, EV_THREADS, LIT_SMEM, g->stream, ab, bstart, blen, ctr, g->lit_over); break;
        case 2: launch_pdl(k_lit_eval<2>, grid, EV_THREADS, LIT_SMEM, g->stream, ab, bstart, blen, ctr, g->lit_over); break;
        case 4: launch_pdl(k_lit_eval<4>, grid, EV_THREADS, LIT_SMEM, g->stream, ab, bstart, blen, ctr, g->lit_over); break;
        default: launch_pdl(k_lit_eval<8>, grid, EV_THREADS, LIT_SMEM, g->stream, ab, bstart, blen, ctr, g->lit_over); break;
        }
        launch_pdl(k_lit_big, std::min<unsigned>(big_grid, (unsigned)blen), EV_THREADS, LIT_SMEM, g->stream, ab,
                   bstart, ctr, (const int32_t *)g->lit_over, g->lit_used + b);
        const int64_t f0 = g->lh_fq.empty() ? 0 : g->lh_fq[(size_t)b];
        const int64_t nf = g->lh_fq.empty() ? 0 : g->lh_fq[(size_t)b + 1] - f0;
        if (nf > 0) {
            const LitHubPlan hp = lit_hub_plan(g);
            const int64_t s0 = g->lh_sq[(size_t)b], nsl = g->lh_sq[(size_t)b + 1] - s0;
            const int64_t h0 = g->lh_hq[(size_t)b], nh = g->lh_hq[(size_t)b + 1] - h0;
            k_lh_size<<<(unsigned)nh, 256, 0, g->stream>>>(ab, hp, bstart, h0, nh);
            k_lh_fill<<<(unsigned)nf, 256, 0, g->stream>>>(ab, hp, bstart, f0);
            k_lh_bound<<<(unsigned)nsl, 256, 0, g->stream>>>(ab, hp, bstart, s0);
            k_lh_mark<<<(unsigned)nsl, 256, 0, g->stream>>>(ab, hp, bstart, s0);
            k_lh_decide<<<(unsigned)nh, 256, 0, g->stream>>>(ab, hp, bstart, h0, nh);
            g->launches += 5;
        }
        if (prof) record_event(g, g->prof_ev[2 * b + 1], capturing);
        const unsigned ag = grid_for((int64_t)blen * 32, AP_THREADS, 1 << 30);
        launch_pdl(k_lit_apply, ag, AP_THREADS, 0, g->stream, ab, bstart, blen, b);
        k_lit_kupd<<<ag, AP_THREADS, 0, g->stream>>>(ab, bstart, blen);
        k_lit_fsum<<<(unsigned)std::min<int64_t>((2 * (int64_t)blen + 7) / 8, 8 * (int64_t)num_sms()), 256, 0,
                     g->stream>>>(ab, g->touched, ctr + 2, 0);
        g->launches += 5;
    }
    LF_LAUNCHED();
}

// Arrays of the paper's gain for queues of up to q nodes and nb queues.
void ensure_lit(lf_graph *g, int64_t q, int64_t nb) {
    const int64_t n = std::max<int64_t>(g->n, 1);
    if (!g->litF) {
        g->litF = dalloc_n<float>(g, 8 * n);
        g->cm_off = dalloc_n<unsigned long long>(g, n + 1);
        g->cm_cur = dalloc_n<unsigned long long>(g, n + 1);
        g->jl_head = dalloc_n<int32_t>(g, n);
        g->jl_next = dalloc_n<int32_t>(g, n);
        g->jl_node = dalloc_n<int32_t>(g, n);
        g->tstamp = dalloc_n<uint32_t>(g, n);
        g->lit_misc = dalloc_n<uint32_t>(g, 4);
        g->cm_cnt = dalloc_n<uint32_t>(g, n);
    }
    if (g->cm_cap < (4 * (int64_t)g->K + 32) * n) {   // regions: 4 (members) + 32 per community
        if (g->cm_node) dfree(g, g->cm_node);
        g->cm_cap = (4 * (int64_t)g->K + 32) * n;
        g->cm_node = dalloc_n<int32_t>(g, g->cm_cap);
        drop_graph(g);
    }
    if (g->lit_qcap < q) {
        if (g->lit_over) dfree(g, g->lit_over);
        if (g->touched) dfree(g, g->touched);
        g->lit_qcap = q;
        g->lit_over = dalloc_n<int32_t>(g, q);
        g->touched = dalloc_n<int32_t>(g, 2 * q);
        drop_graph(g);
    }
    if (g->lit_ctr_cap < 3 * nb) {
        if (g->lit_ctr) dfree(g, g->lit_ctr);
        if (g->lit_used) dfree(g, g->lit_used);
        g->lit_ctr_cap = 3 * nb;
        g->lit_ctr = dalloc_n<uint32_t>(g, 3 * nb);
        g->lit_used = dalloc_n<unsigned long long>(g, nb);
        drop_graph(g);
    }
    build_lit_hub_plan(g, q, nb);
    // global tables: per queue, every node whose entries can exceed half a
    // block's table gets pow2 >= 2 (d+1) K slots (K bounds every row, so
    // (d+1) K bounds its entries); queues run one after the other and share
    // the area, sized for the largest queue
    if (g->lg_plan_q != q || g->lg_plan_K != g->K || g->lg_plan_sched != g->sched_version) {
        g->lg_plan_q = q;
        g->lg_plan_K = g->K;
        g->lg_plan_sched = g->sched_version;
        unsigned long long cap = 0;
        if (g->n > 0 && (long long)(g->max_deg + 1) * g->K * 2 > LB_SLOTS) {
            const int64_t len = g->sched.empty() ? g->n : g->sched.back();
            std::vector<int32_t> order((size_t)std::max<int64_t>(len, 1)), deg((size_t)g->n);
            if (len > 0)
                LF_CUDA(cudaMemcpyAsync(order.data(), g->sched.empty() ? g->order : g->qorder, (size_t)len * 4,
                                        cudaMemcpyDeviceToHost, g->stream));
            LF_CUDA(cudaMemcpyAsync(deg.data(), g->deg, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream));
            LF_CUDA(cudaStreamSynchronize(g->stream));
            for (int64_t b = 0; b < nb; ++b) {
                int64_t qs;
                int32_t ql;
                queue_bounds(g, q, b, qs, ql);
                unsigned long long used = 0;
                for (int64_t p2 = qs; p2 < qs + ql; ++p2) {
                    const unsigned long long e = (unsigned long long)(deg[(size_t)order[(size_t)p2]] + 1) * g->K;
                    if (2 * e <= (unsigned long long)LB_SLOTS) continue;
                    unsigned long long H = 32;
                    while (H < 2 * e) H <<= 1;
                    used += H;
                }
                cap = std::max(cap, used);
            }
        }
        // the area is a reservation for the worst case; past 32 MiB + 64 bytes
        // per edge a node that finds no room takes the multi-pass shared path
        cap = std::min<unsigned long long>(cap, ((32ull << 20) + 64ull * (unsigned long long)g->m) / 16);
        if (cap != g->lg_cap) {
            if (g->lg_area) dfree(g, g->lg_area);
            g->lg_area = cap ? dalloc(g, (size_t)cap * 16) : nullptr;
            g->lg_cap = cap;
            drop_graph(g);
        }
    }
}

// Start of an iteration under the paper's gain: the member index (members
// by community), no joiners yet, and every community's sums.
void lit_iteration_start(lf_graph *g, const RunArgs &a) {
    const int64_t n = g->n, nc = g->ncomm;
    if (n == 0 || nc == 0) return;
    cudaStream_t st = g->stream;
    LF_CUDA(cudaMemsetAsync(g->cm_cnt, 0, (size_t)nc * 4, st));
    k_lit_count<<<grid_for(n, 256, 1 << 16), 256, 0, st>>>(a, n, g->cm_cnt);
    k_lit_caps<<<grid_for(nc, 256, 1 << 16), 256, 0, st>>>(g->cm_cnt, nc, g->cm_cur);
    LF_LAUNCHED();
    scan_exclusive<unsigned long long>(g, g->cm_cur, g->cm_off, nc, g->cm_off + nc);
    LF_CUDA(cudaMemcpyAsync(g->cm_cur, g->cm_off, (size_t)nc * 8, cudaMemcpyDeviceToDevice, st));
    k_lit_fill<<<grid_for(n, 256, 1 << 16), 256, 0, st>>>(a, n, g->cm_cur, g->cm_node);
    LF_CUDA(cudaMemsetAsync(g->jl_head, 0xff, (size_t)nc * 4, st));
    LF_CUDA(cudaMemsetAsync(g->lit_misc, 0, 4 * sizeof(uint32_t), st));
    // touched-list stamps are queue serials of this iteration (a batch's queue
    // count changes between iterations, so serials of different iterations
    // may coincide): clear them
    LF_CUDA(cudaMemsetAsync(g->tstamp, 0, (size_t)n * 4, st));
    k_lit_fsum<<<(unsigned)std::min<int64_t>((nc + 7) / 8, 16 * (int64_t)num_sms()), 256, 0, st>>>(a, nullptr, nullptr,
                                                                                                   nc);
    g->launches += 4;
    LF_LAUNCHED();
}

// Queue order of a batch: segments (source position in the graph-by-graph
// order, destination, length) copied one warp each.
__global__ void k_gather_order(const int32_t *order, const long long *seg, int64_t nseg, int32_t *qorder,
                               int32_t *qpos) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nseg; s += warps) {
        const long long src = seg[3 * s], dst = seg[3 * s + 1], len = seg[3 * s + 2];
        for (long long i = lane; i < len; i += 32) {
            const int32_t x = order[src + i];
            qorder[dst + i] = x;
            qpos[x] = (int32_t)(dst + i);
        }
    }
}

// The queues of a batch iteration: queue j holds the j-th q nodes (in node
// order) of every active graph, graph by graph.  Graphs do not interact, so
// each graph sees exactly the queues it would have alone.
void build_schedule(lf_graph *g, int64_t q, const std::vector<char> &active) {
    const int64_t G = g->ngraphs;
    int64_t J = 0;
    for (int64_t i = 0; i < G; ++i)
        if (active[(size_t)i]) J = std::max(J, (g->gnoff[(size_t)i + 1] - g->gnoff[(size_t)i] + q - 1) / q);
    std::vector<long long> seg;
    std::vector<int64_t> sched(1, 0);
    int64_t cur = 0;
    for (int64_t j = 0; j < J; ++j) {
        for (int64_t i = 0; i < G; ++i) {
            if (!active[(size_t)i]) continue;
            const int64_t ni = g->gnoff[(size_t)i + 1] - g->gnoff[(size_t)i];
            const int64_t len = std::min(q, ni - j * q);
            if (len <= 0) continue;
            seg.push_back(g->gnoff[(size_t)i] + j * q);
            seg.push_back(cur);
            seg.push_back(len);
            cur += len;
        }
        sched.push_back(cur);
    }
    if (!g->qorder) {
        g->qorder = dalloc_n<int32_t>(g, std::max<int64_t>(g->n, 1));
        g->qpos = dalloc_n<int32_t>(g, std::max<int64_t>(g->n, 1));
    }
    // nodes of stopped graphs are in no queue (position -1)
    LF_CUDA(cudaMemsetAsync(g->qpos, 0xff, (size_t)std::max<int64_t>(g->n, 1) * 4, g->stream));
    const int64_t nseg = (int64_t)seg.size() / 3;
    if (nseg > 0) {
        long long *d = dalloc_n<long long>(g, 3 * nseg);
        LF_CUDA(cudaMemcpyAsync(d, seg.data(), (size_t)(3 * nseg) * 8, cudaMemcpyHostToDevice, g->stream));
        k_gather_order<<<grid_for(nseg * 32, 256, 1 << 16), 256, 0, g->stream>>>(g->order, d, nseg, g->qorder,
                                                                                   g->qpos);
        ++g->launches;
        LF_LAUNCHED();
        LF_CUDA(cudaStreamSynchronize(g->stream));
        dfree(g, d);
    }
    g->sched = sched;
    ++g->sched_version;
}

// The WCC-hat total on a resident grid (work is handed out by counters).
void launch_total(lf_graph *g, const RunArgs &a) {
    static const int per_sm = blocks_per_sm(k_total, TOT_WARPS * 32, 0);
    LF_CUDA(cudaMemsetAsync(g->tot_next, 0, 2 * sizeof(uint32_t), g->stream));
    k_total<<<num_sms() * std::max(1, per_sm), TOT_WARPS * 32, 0, g->stream>>>(a, g->n);
    ++g->launches;
}

void launch_iteration_end(lf_graph *g, const RunArgs &a) {
    const int64_t n = g->n;
    k_prune<<<grid_for(n + g->ncomm, 256, 1 << 16), 256, 0, g->stream>>>(a, n, g->ncomm); ++g->launches;
    launch_total(g, a);
    k_finalize<<<1, 32, 0, g->stream>>>(g->ds, device_readback(g), 1); ++g->launches;
    LF_LAUNCHED();
    LF_CUDA(cudaMemcpyAsync(g->rb, device_readback(g), sizeof(Readback), cudaMemcpyDeviceToHost, g->stream));
    if (g->ngraphs > 0) {
        k_finalize_batch<<<grid_for(g->ngraphs, 256, 1024), 256, 0, g->stream>>>(g->gsacc, g->ngraphs, g->gT);
        ++g->launches;
        LF_LAUNCHED();
        LF_CUDA(cudaMemcpyAsync(g->gT_host, g->gT, (size_t)g->ngraphs * 8, cudaMemcpyDeviceToHost, g->stream));
    }
}

void ensure_capacity(lf_graph *g, int64_t q) {
    const int64_t n = g->n;
    if (!g->comm) {
        g->comm = dalloc_n<CommRec>(g, n);
        g->nmem = dalloc_n<int32_t>(g, n);
        g->K = std::max(4, (g->member_slots + 3) / 4 * 4);   // rows start on 16-byte boundaries
        g->mem = dalloc_n<int32_t>(g, n * g->K);
    }
    if (g->gain_rule == LF_GAIN_LITERAL && !g->kmem) g->kmem = dalloc_n<int32_t>(g, n * g->K);
    if (g->qcap < q) {
        if (g->act) dfree(g, g->act);
        g->qcap = (int32_t)q;
        g->act = dalloc_n<int32_t>(g, 4 * q);
        drop_graph(g);
    }
}

void grow_rows(lf_graph *g, int32_t need) {
    int32_t K2 = g->K;
    while (K2 < need) K2 *= 2;
    if (K2 == g->K) return;
    int32_t *mem2 = dalloc_n<int32_t>(g, g->n * K2);
    int32_t *kmem2 = g->kmem ? dalloc_n<int32_t>(g, g->n * K2) : nullptr;
    k_regrow<<<grid_for(g->n, 256, 1 << 16), 256, 0, g->stream>>>(g->mem, g->nmem, g->n, g->K, mem2, K2, g->kmem,
                                                                   kmem2); ++g->launches;
    LF_LAUNCHED();
    dfree(g, g->mem);
    g->mem = mem2;
    if (g->kmem) {
        dfree(g, g->kmem);
        g->kmem = kmem2;
    }
    g->K = K2;
    drop_graph(g);
}

double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float t = 0.f;
    LF_CUDA(cudaEventElapsedTime(&t, a, b));
    return (double)t;
}

template <int T>
const void *iterate_kernel() {
    return (const void *)k_iterate<T>;
}

const void *iterate_kernel_for(int T) {
    switch (T) {
    case 1: return iterate_kernel<1>();
    case 2: return iterate_kernel<2>();
    case 4: return iterate_kernel<4>();
    default: return iterate_kernel<8>();
    }
}

// Blocks of the persistent queue kernel that can be resident at once.
int persistent_grid_max(lf_graph *g, int T) {
    int per_sm = 0;
    const void *k = iterate_kernel_for(T);
    LF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DYN_SMEM));
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, EV_THREADS, EV_DYN_SMEM));
    (void)g;
    return std::max(1, per_sm) * num_sms();
}

// One cooperative launch runs queues first .. first+count-1.
void launch_persistent(lf_graph *g, RunArgs a, int64_t q, int64_t first, int64_t count, int grid_max, int T,
                       cudaEvent_t e0, cudaEvent_t e1) {
    if (count <= 0) return;
    const int64_t teams = EV_WARPS / T;
    const int64_t want = (q + teams - 1) / teams;
    unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, grid_max));
    long long spin = (long long)g->barrier_timeout_ms * 4000ll;   // >= ~250 ns per poll of the flags
    int inject = g->inject_stall;
    unsigned *flags = g->bar_flags;
    unsigned epoch = g->bar_epoch;
    g->bar_epoch += (unsigned)(2 * count);
    int bar_mode = g->barrier_mode;
    void *args[] = {&a, &q, &first, &count, &spin, &inject, &flags, &epoch, &bar_mode};
    if (e0) LF_CUDA(cudaEventRecord(e0, g->stream));
    LF_CUDA(cudaLaunchCooperativeKernel(iterate_kernel_for(T), dim3(grid), dim3(EV_THREADS), args, EV_DYN_SMEM,
                                        g->stream));
    ++g->launches;
    if (e1) LF_CUDA(cudaEventRecord(e1, g->stream));
}

void free_hub_plan(lf_graph *g) {
    if (g->hub_pos) dfree(g, g->hub_pos);
    if (g->hub_qoff) dfree(g, g->hub_qoff);
    if (g->hub_toff) dfree(g, g->hub_toff);
    if (g->hub_tcap) dfree(g, g->hub_tcap);
    if (g->hub_wcap) dfree(g, g->hub_wcap);
    g->hub_wcap = nullptr;
    if (g->hub_scratch) dfree(g, g->hub_scratch);
    if (g->hub_chunk_h) dfree(g, g->hub_chunk_h);
    if (g->hub_chunk_c) dfree(g, g->hub_chunk_c);
    if (g->hub_nch) dfree(g, g->hub_nch);
    if (g->hub_done) dfree(g, g->hub_done);
    if (g->hub_ncand) dfree(g, g->hub_ncand);
    g->hub_chunk_h = g->hub_chunk_c = g->hub_nch = nullptr;
    g->hub_done = g->hub_ncand = nullptr;
    for (int32_t **pp : {&g->hub_lbj, &g->hub_lbl, &g->hub_items, &g->hub_item_ck})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    for (uint32_t **pp : {&g->hub_item_base, &g->hub_nitems, &g->hub_items_done, &g->hub_qctr})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    if (g->hub_item_g) dfree(g, g->hub_item_g);
    g->hub_item_g = nullptr;
    g->hub_items_cap = 0;
    g->hub_qbig.clear();
    g->hub_cqoff_host.clear();
    g->hub_pos = nullptr;
    g->hub_qoff = nullptr;
    g->hub_toff = nullptr;
    g->hub_tcap = nullptr;
    g->hub_scratch = nullptr;
    g->hub_slots = 0;
    g->hub_qoff_host.clear();
    g->hub_plan_q = 0;
    g->hub_plan_K = 0;
}

// Static per-run plan of the hubs (degree > hub_degree): their positions per
// queue and a table of pow2 >= 2 (d+1) K slots each (K bounds every row, so
// (d+1) K bounds the entries).  Queues run one after the other, so the
// tables of every queue share one scratch area.
void build_hub_plan(lf_graph *g, int64_t q) {
    if (g->hub_plan_q == q && g->hub_plan_K == g->K && g->hub_plan_sched == g->sched_version &&
        g->hub_plan_deg == g->hub_degree)
        return;
    free_hub_plan(g);
    g->hub_plan_q = q;
    g->hub_plan_K = g->K;
    g->hub_plan_deg = g->hub_degree;
    g->hub_plan_sched = g->sched_version;
    const int64_t n = g->n;
    if (n == 0 || g->max_deg <= g->hub_degree) return;
    const int64_t len = g->sched.empty() ? n : g->sched.back();   // positions in the order the kernels read
    std::vector<int32_t> order((size_t)std::max<int64_t>(len, 1)), deg((size_t)n);
    if (len > 0)
        LF_CUDA(cudaMemcpyAsync(order.data(), g->sched.empty() ? g->order : g->qorder, (size_t)len * 4,
                                cudaMemcpyDeviceToHost, g->stream));
    LF_CUDA(cudaMemcpyAsync(deg.data(), g->deg, (size_t)n * 4, cudaMemcpyDeviceToHost, g->stream));
    LF_CUDA(cudaStreamSynchronize(g->stream));
    const int64_t nb = num_queues(g, q);
    std::vector<int32_t> pos, nch, chunk_h, chunk_c;
    std::vector<int64_t> qoff((size_t)nb + 1, 0), cqoff((size_t)nb + 1, 0), toff;
    std::vector<uint32_t> tcap;
    std::vector<char> qbig((size_t)nb, 0);
    int64_t slots = 0, items_cap = 0;
    for (int64_t b = 0; b < nb; ++b) {
        qoff[(size_t)b] = (int64_t)pos.size();
        cqoff[(size_t)b] = (int64_t)chunk_h.size();
        int64_t used = 0, items = 0;
        int64_t qs;
        int32_t ql;
        queue_bounds(g, q, b, qs, ql);
        for (int64_t p = qs; p < qs + ql; ++p) {
            const int32_t d = deg[(size_t)order[(size_t)p]];
            if (d <= g->hub_degree) continue;
            uint64_t cap = 32;
            while (cap < 2ull * (uint64_t)(d + 1) * (uint64_t)g->K) cap <<= 1;
            const int32_t c = (d + HUGE_CHUNK - 1) / HUGE_CHUNK;
            for (int32_t k = 0; k < c; ++k) {
                chunk_h.push_back((int32_t)pos.size());
                chunk_c.push_back(k);
            }
            pos.push_back((int32_t)p);
            nch.push_back(c);
            toff.push_back(used);
            tcap.push_back((uint32_t)cap);
            used += (int64_t)cap;
            if (cap / 2 > HUGE_BIG_NCAND) {   // candidates <= cap / 2
                qbig[(size_t)b] = 1;
                items += (int64_t)((cap / 2 + HUGE_CAND_CHUNK - 1) / HUGE_CAND_CHUNK);
            }
        }
        slots = std::max(slots, used);
        items_cap = std::max(items_cap, items);
    }
    g->hub_qbig = qbig;
    qoff[(size_t)nb] = (int64_t)pos.size();
    cqoff[(size_t)nb] = (int64_t)chunk_h.size();
    g->hub_qoff_host = qoff;
    g->hub_cqoff_host = cqoff;
    if (pos.empty()) return;
    const int64_t NC = (int64_t)chunk_h.size();
    g->hub_chunk_h = dalloc_n<int32_t>(g, NC);
    g->hub_chunk_c = dalloc_n<int32_t>(g, NC);
    LF_CUDA(cudaMemcpyAsync(g->hub_chunk_h, chunk_h.data(), (size_t)NC * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->hub_chunk_c, chunk_c.data(), (size_t)NC * 4, cudaMemcpyHostToDevice, g->stream));
    const int64_t H = (int64_t)pos.size();
    g->hub_pos = dalloc_n<int32_t>(g, H);
    g->hub_qoff = dalloc_n<int64_t>(g, nb + 1);
    g->hub_toff = dalloc_n<int64_t>(g, H);
    g->hub_tcap = dalloc_n<uint32_t>(g, H);
    g->hub_scratch = dalloc_n<int32_t>(g, 4 * slots);
    g->hub_slots = slots;
    g->hub_nch = dalloc_n<int32_t>(g, H);
    g->hub_done = dalloc_n<uint32_t>(g, H);
    g->hub_ncand = dalloc_n<uint32_t>(g, H);
    LF_CUDA(cudaMemcpyAsync(g->hub_nch, nch.data(), (size_t)H * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemsetAsync(g->hub_done, 0, (size_t)H * 4, g->stream));
    LF_CUDA(cudaMemsetAsync(g->hub_ncand, 0, (size_t)H * 4, g->stream));
    g->hub_lbj = dalloc_n<int32_t>(g, H);
    g->hub_lbl = dalloc_n<int32_t>(g, H);
    g->hub_item_base = dalloc_n<uint32_t>(g, H);
    g->hub_nitems = dalloc_n<uint32_t>(g, H);
    g->hub_items_done = dalloc_n<uint32_t>(g, H);
    {
        const int32_t neg_inf_ord = (int32_t)(0xff800000u ^ 0x7fffffffu);   // -inf, order-preserving
        std::vector<int32_t> ninf((size_t)H, neg_inf_ord);
        LF_CUDA(cudaMemcpyAsync(g->hub_lbj, ninf.data(), (size_t)H * 4, cudaMemcpyHostToDevice, g->stream));
        LF_CUDA(cudaMemcpyAsync(g->hub_lbl, ninf.data(), (size_t)H * 4, cudaMemcpyHostToDevice, g->stream));
        LF_CUDA(cudaStreamSynchronize(g->stream));
    }
    LF_CUDA(cudaMemsetAsync(g->hub_items_done, 0, (size_t)H * 4, g->stream));
    g->hub_qctr = dalloc_n<uint32_t>(g, 3 * nb);
    LF_CUDA(cudaMemsetAsync(g->hub_qctr, 0, (size_t)(3 * nb) * 4, g->stream));
    g->hub_items_cap = std::max<int64_t>(1, items_cap);
    g->hub_items = dalloc_n<int32_t>(g, 2 * g->hub_items_cap);
    g->hub_item_g = dalloc_n<double>(g, 2 * g->hub_items_cap);
    g->hub_item_ck = dalloc_n<int32_t>(g, 4 * g->hub_items_cap);
    // tables start clean (keys empty, counts zero) and are left clean after each use
    LF_CUDA(cudaMemsetAsync(g->hub_scratch, 0xff, (size_t)slots * 4, g->stream));
    LF_CUDA(cudaMemsetAsync(g->hub_scratch + slots, 0, (size_t)slots * 4, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->hub_pos, pos.data(), (size_t)H * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->hub_qoff, qoff.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->hub_toff, toff.data(), (size_t)H * 8, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->hub_tcap, tcap.data(), (size_t)H * 4, cudaMemcpyHostToDevice, g->stream));
    g->hub_wcap = dalloc_n<uint32_t>(g, H);
    LF_CUDA(cudaMemcpyAsync(g->hub_wcap, tcap.data(), (size_t)H * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaStreamSynchronize(g->stream));
}

void free_total_plan(lf_graph *g) {
    for (int32_t **p : {&g->tot_hubs, &g->tot_chunk_hub, &g->tot_first, &g->tot_cnt})
        if (*p) {
            dfree(g, *p);
            *p = nullptr;
        }
    if (g->tot_done) dfree(g, g->tot_done);
    if (g->tot_next) dfree(g, g->tot_next);
    g->tot_done = g->tot_next = nullptr;
    g->tot_nh = g->tot_nchunks = 0;
    g->tot_plan_K = 0;
}

// Nodes of degree > TOT_CHUNK for the WCC-hat total, largest first, with one
// chunk per TOT_CHUNK neighbours, and their zeroed counters (K per node).
void build_total_plan(lf_graph *g) {
    if (g->tot_next && g->tot_plan_K == g->K) return;
    free_total_plan(g);
    g->tot_plan_K = g->K;
    g->tot_next = dalloc_n<uint32_t>(g, 2);
    const int64_t n = g->n;
    if (n == 0 || g->max_deg <= TOT_CHUNK) return;
    std::vector<int32_t> deg((size_t)n);
    LF_CUDA(cudaMemcpyAsync(deg.data(), g->deg, (size_t)n * 4, cudaMemcpyDeviceToHost, g->stream));
    LF_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<int32_t> hubs;
    for (int64_t x = 0; x < n; ++x)
        if (deg[(size_t)x] > TOT_CHUNK) hubs.push_back((int32_t)x);
    std::stable_sort(hubs.begin(), hubs.end(),
                     [&](int32_t u, int32_t v) { return deg[(size_t)u] > deg[(size_t)v]; });
    std::vector<int32_t> first(hubs.size() + 1, 0), chunk_hub;
    for (size_t h = 0; h < hubs.size(); ++h) {
        const int32_t nch = (deg[(size_t)hubs[h]] + TOT_CHUNK - 1) / TOT_CHUNK;
        first[h + 1] = first[h] + nch;
        for (int32_t c = 0; c < nch; ++c) chunk_hub.push_back((int32_t)h);
    }
    const int64_t nh = (int64_t)hubs.size(), nc = (int64_t)chunk_hub.size();
    g->tot_nh = nh;
    g->tot_nchunks = nc;
    g->tot_hubs = dalloc_n<int32_t>(g, nh);
    g->tot_first = dalloc_n<int32_t>(g, nh + 1);
    g->tot_chunk_hub = dalloc_n<int32_t>(g, nc);
    g->tot_cnt = dalloc_n<int32_t>(g, nh * g->K);
    g->tot_done = dalloc_n<uint32_t>(g, nh);
    LF_CUDA(cudaMemcpyAsync(g->tot_hubs, hubs.data(), (size_t)nh * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->tot_first, first.data(), (size_t)(nh + 1) * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemcpyAsync(g->tot_chunk_hub, chunk_hub.data(), (size_t)nc * 4, cudaMemcpyHostToDevice, g->stream));
    LF_CUDA(cudaMemsetAsync(g->tot_cnt, 0, (size_t)(nh * g->K) * 4, g->stream));
    LF_CUDA(cudaMemsetAsync(g->tot_done, 0, (size_t)nh * 4, g->stream));
    LF_CUDA(cudaStreamSynchronize(g->stream));
}

}  // namespace

void free_run_state(lf_graph *g) {
    drop_graph(g);
    free_hub_plan(g);
    free_total_plan(g);
    if (g->side) {
        cudaStreamSynchronize(g->side);
        cudaStreamDestroy(g->side);
        cudaEventDestroy(g->ev_fork);
        cudaEventDestroy(g->ev_join);
        g->side = nullptr;
        g->ev_fork = g->ev_join = nullptr;
    }
    if (g->dyn_ctr) dfree(g, g->dyn_ctr);
    if (g->dyn_list) dfree(g, g->dyn_list);
    if (g->dyn_bound) dfree(g, g->dyn_bound);
    g->dyn_ctr = nullptr;
    g->dyn_list = nullptr;
    g->dyn_bound = nullptr;
    g->dyn_ctr_cap = g->dyn_list_cap = 0;
    if (g->qtimes) dfree(g, g->qtimes);
    g->qtimes = nullptr;
    if (g->bar_flags) dfree(g, g->bar_flags);
    g->bar_flags = nullptr;
    g->bar_flags_cap = 0;
    for (auto e : g->prof_ev) cudaEventDestroy(e);
    g->prof_ev.clear();
    for (int32_t **pp : {&g->kmem, &g->cm_node, &g->jl_head, &g->jl_next, &g->jl_node, &g->lit_over, &g->touched})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    for (unsigned long long **pp : {&g->cm_off, &g->cm_cur})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    free_lit_hub_plan(g);
    if (g->lit_used) dfree(g, g->lit_used);
    g->lit_used = nullptr;
    if (g->lg_area) dfree(g, g->lg_area);
    g->lg_area = nullptr;
    g->lg_cap = 0;
    g->lg_plan_q = g->lg_plan_sched = -1;
    g->lg_plan_K = 0;
    for (uint32_t **pp : {&g->lit_misc, &g->tstamp, &g->lit_ctr, &g->cm_cnt})
        if (*pp) {
            dfree(g, *pp);
            *pp = nullptr;
        }
    if (g->litF) dfree(g, g->litF);
    g->litF = nullptr;
    g->cm_cap = g->lit_ctr_cap = g->lit_qcap = 0;
    if (g->act) dfree(g, g->act);
    if (g->mem) dfree(g, g->mem);
    if (g->nmem) dfree(g, g->nmem);
    if (g->comm) dfree(g, g->comm);
    g->act = g->mem = g->nmem = nullptr;
    g->comm = nullptr;
    g->qcap = 0;
    g->K = 0;
}

void run_impl(lf_graph *g, int32_t q_in, double thr, int32_t max_iters, int64_t max_batches, lf_run_stats *stats) {
    if (q_in < 1) fail(LF_ERR_INVALID, "queue_size must be >= 1 (got %d)", q_in);
    if (max_iters < 0) fail(LF_ERR_INVALID, "max_iters must be >= 0 (got %d)", max_iters);
    if (std::isnan(thr)) fail(LF_ERR_INVALID, "wcc_threshold is NaN");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = g->stream;
    const int64_t n = g->n;
    const bool batch = g->ngraphs > 0;
    if (batch && max_batches >= 0) fail(LF_ERR_INVALID, "lf_run_partial is not available for a batch of graphs");
    int64_t q = std::max<int64_t>(1, std::min<int64_t>(q_in, std::max<int64_t>(n, 1)));
    std::vector<char> gactive;
    if (batch) {   // every graph with nodes starts active; queues from the schedule
        const int64_t G = g->ngraphs;
        int64_t nmax = 1;
        gactive.assign((size_t)G, 0);
        for (int64_t i = 0; i < G; ++i) {
            const int64_t ni = g->gnoff[(size_t)i + 1] - g->gnoff[(size_t)i];
            gactive[(size_t)i] = ni > 0;
            nmax = std::max(nmax, ni);
        }
        q = std::max<int64_t>(1, std::min<int64_t>(q_in, nmax));
        if (!g->gT_host) LF_CUDA(cudaMallocHost(&g->gT_host, (size_t)G * 8));
        LF_CUDA(cudaMemsetAsync(g->gsacc, 0, (size_t)(G * SACC_CHUNKS) * 8, g->stream));
        g->g_iters.assign((size_t)G, 0);
        g->g_conv.assign((size_t)G, 0);
        g->g_T0.assign((size_t)G, 0.0);
        g->g_hist.assign((size_t)G, std::vector<double>());
        g->sched.clear();
        if (n > 0) build_schedule(g, q, gactive);
    }
    ensure_capacity(g, batch ? max_queue(g, q) : q);
    set_eval_attrs();
    cudaEvent_t ev[3];
    for (auto &e : ev) LF_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]);
        }
    } eg{ev};
    LF_CUDA(cudaEventRecord(ev[0], st));
    // reset run state
    LF_CUDA(cudaMemsetAsync(g->comm, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(CommRec), st));
    LF_CUDA(cudaMemsetAsync(g->nmem, 0, (size_t)std::max<int64_t>(n, 1) * 4, st));
    LF_CUDA(cudaMemsetAsync(g->ds->sacc, 0, sizeof(g->ds->sacc), st));
    {
        DevScalars z{};
        // zero the run counters (the fields from `joins` up to `max_id`)
        const size_t o = offsetof(DevScalars, joins);
        LF_CUDA(cudaMemcpyAsync(reinterpret_cast<char *>(g->ds) + o, reinterpret_cast<char *>(&z) + o,
                                offsetof(DevScalars, max_id) - o, cudaMemcpyHostToDevice, st));
        LF_CUDA(cudaMemsetAsync(&g->ds->bar_count, 0, sizeof(unsigned), st));
        LF_CUDA(cudaStreamSynchronize(st));
    }
    build_total_plan(g);
    RunArgs a = make_args(g, device_readback(g));
    const unsigned long long launches0 = g->launches;
    const int64_t nb_all = n > 0 ? (n + q - 1) / q : 0;
    if (g->profile && (int64_t)g->prof_ev.size() < 2 * nb_all) {
        drop_graph(g);   // a captured graph would not record the new events
        while ((int64_t)g->prof_ev.size() < 2 * nb_all) {
            cudaEvent_t e;
            LF_CUDA(cudaEventCreate(&e));
            g->prof_ev.push_back(e);
        }
    }
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    double qpct[4] = {0, 0, 0, 0};
    if (g->profile && nb_all > 0) {
        if (g->qtimes) dfree(g, g->qtimes);
        g->qtimes = dalloc_n<unsigned long long>(g, nb_all + 1);
    }

    // ---- a6: initial clustering, or an inserted division
    int64_t k0 = 0;
    if (n > 0 && g->part_k >= 0) {
        if (g->part_maxcnt + 1 > g->K) {
            grow_rows(g, g->part_maxcnt + 1);
            a = make_args(g, device_readback(g));
        }
        const int64_t E = (int64_t)g->part_mem.size();
        if (E > 0) {
            std::vector<unsigned long long> hk((size_t)E);
            for (int64_t c = 0; c < g->part_k; ++c)
                for (int64_t i = g->part_off[(size_t)c]; i < g->part_off[(size_t)c + 1]; ++i)
                    hk[(size_t)i] = ((unsigned long long)g->part_mem[(size_t)i] << 32) | (unsigned long long)c;
            unsigned long long *keys = dalloc_n<unsigned long long>(g, E);
            LF_CUDA(cudaMemcpyAsync(keys, hk.data(), (size_t)E * 8, cudaMemcpyHostToDevice, st));
            std::vector<int> shifts;
            const int bc = bits_for((unsigned long long)std::max<int64_t>(g->part_k - 1, 0));
            const int bx = bits_for((unsigned long long)(n - 1));
            for (int b = 0; b < bc; b += 8) shifts.push_back(b);
            for (int b = 0; b < bx; b += 8) shifts.push_back(32 + b);
            radix_sort(g, keys, nullptr, E, shifts);
            k_part_rows<<<grid_for(E, 256, 1 << 16), 256, 0, st>>>(a, keys, E, g->part_maxcnt); ++g->launches;
            k_part_m2<<<grid_for(E * 32, 256, 1 << 16), 256, 0, st>>>(a, keys, E); ++g->launches;
            LF_LAUNCHED();
            LF_CUDA(cudaStreamSynchronize(st));
            dfree(g, keys);
        }
        k0 = g->part_k;
    } else if (n > 0) {
        int32_t *state = dalloc_n<int32_t>(g, n);
        int32_t *und = dalloc_n<int32_t>(g, 1);
        LF_CUDA(cudaMemsetAsync(state, 0, (size_t)n * 4, st));
        for (int round = 0;; ++round) {
            LF_CUDA(cudaMemsetAsync(und, 0, 4, st));
            k_mis_round<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(g->off, g->adj, g->pos, n, state, und); ++g->launches;
            LF_LAUNCHED();
            int32_t left = 0;
            LF_CUDA(cudaMemcpyAsync(&left, und, 4, cudaMemcpyDeviceToHost, st));
            LF_CUDA(cudaStreamSynchronize(st));
            if (left == 0) break;
            if (round > n + 2) fail(LF_ERR_CUDA, "initial clustering did not converge");
        }
        uint32_t *flag = dalloc_n<uint32_t>(g, n + 1);
        k_seed_flags<<<grid_for(n, 256, 1 << 16), 256, 0, st>>>(g->order, state, n, flag); ++g->launches;
        LF_LAUNCHED();
        scan_exclusive<uint32_t>(g, flag, flag, n, flag + n);
        uint32_t kk = 0;
        LF_CUDA(cudaMemcpyAsync(&kk, flag + n, 4, cudaMemcpyDeviceToHost, st));
        int32_t *comm_of = dalloc_n<int32_t>(g, n);
        k_assign<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(g->off, g->adj, g->pos, state, flag, n, comm_of); ++g->launches;
        k_init_rows<<<grid_for(n, 256, 1 << 16), 256, 0, st>>>(a, comm_of, n); ++g->launches;
        k_init_m2<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(a, comm_of, n); ++g->launches;
        LF_LAUNCHED();
        LF_CUDA(cudaStreamSynchronize(st));
        k0 = kk;
        dfree(g, comm_of);
        dfree(g, flag);
        dfree(g, und);
        dfree(g, state);
    }
    g->ncomm = k0;
    const bool lit = g->gain_rule == LF_GAIN_LITERAL;
    if (lit && n > 0) {   // deg(x,C) of every membership of the starting state
        ensure_lit(g, batch ? max_queue(g, q) : q, num_queues(g, q));
        a = make_args(g, device_readback(g));
        k_lit_kinit<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(a, n); ++g->launches;
        LF_LAUNCHED();
    }
    launch_total(g, a);
    k_finalize<<<1, 32, 0, st>>>(g->ds, device_readback(g), 0); ++g->launches;
    LF_LAUNCHED();
    LF_CUDA(cudaMemcpyAsync(g->rb, device_readback(g), sizeof(Readback), cudaMemcpyDeviceToHost, st));
    if (batch) {   // every graph's T0
        k_finalize_batch<<<grid_for(g->ngraphs, 256, 1024), 256, 0, st>>>(g->gsacc, g->ngraphs, g->gT);
        ++g->launches;
        LF_LAUNCHED();
        LF_CUDA(cudaMemcpyAsync(g->gT_host, g->gT, (size_t)g->ngraphs * 8, cudaMemcpyDeviceToHost, st));
    }
    LF_CUDA(cudaEventRecord(ev[1], st));
    LF_CUDA(cudaStreamSynchronize(st));
    const double T0 = g->rb->total;
    int32_t maxcnt = g->rb->maxcnt;
    g->ran = true;
    std::vector<double> gprev;
    if (batch) {
        gprev.assign(g->gT_host, g->gT_host + g->ngraphs);
        g->g_T0 = gprev;
    }

    int64_t nb = num_queues(g, q);
    if (batch && !lit) ensure_dyn(g, max_queue(g, q), nb);
    else if (!lit && use_dyn(g, q)) ensure_dyn(g, q, nb);
    // measured on GB300: the persistent loop wins for small queues (grid
    // barriers over few blocks), launches per queue for large ones
    const bool persistent = !batch && !lit && (g->per_queue == 0 || (g->per_queue < 0 && q <= 256));
    const int team = choose_team(g, q);
    const int grid_max = persistent ? persistent_grid_max(g, team) : 0;
    if (persistent) {
        if (g->bar_flags_cap < grid_max + 1) {
            if (g->bar_flags) dfree(g, g->bar_flags);
            g->bar_flags = dalloc_n<unsigned>(g, grid_max + 1);
            g->bar_flags_cap = grid_max + 1;
        }
        LF_CUDA(cudaMemsetAsync(g->bar_flags, 0, (size_t)(grid_max + 1) * sizeof(unsigned), st));
        g->bar_epoch = 0;
    }
    cudaEvent_t pev[2] = {nullptr, nullptr};
    if (persistent && g->profile)
        for (auto &e : pev) LF_CUDA(cudaEventCreate(&e));
    struct PevGuard {
        cudaEvent_t *e;
        ~PevGuard() {
            for (int i = 0; i < 2; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } pg{pev};
    int32_t iters = 0, converged = 0;
    int64_t batches = 0;
    double prev = T0;
    unsigned long long last_live = (unsigned long long)k0, last_memb = (unsigned long long)n;
    for (int32_t it = 1; it <= max_iters; ++it) {
        if (batch) {   // graphs that stopped leave the queues
            if (std::find(gactive.begin(), gactive.end(), (char)1) == gactive.end()) break;
            if (it > 1) {
                build_schedule(g, q, gactive);
                nb = num_queues(g, q);
                if (!lit) ensure_dyn(g, max_queue(g, q), nb);
            }
        }
        if (maxcnt + 1 > g->K) grow_rows(g, maxcnt + 1);
        if (!lit) build_hub_plan(g, q);
        build_total_plan(g);
        if (lit) ensure_lit(g, batch ? max_queue(g, q) : q, nb);
        a = make_args(g, device_readback(g));
        a.nbatches = nb;
        if (lit) lit_iteration_start(g, a);
        const bool partial = max_batches >= 0 && batches + nb > max_batches;
        if (partial) {
            if (persistent) launch_persistent(g, a, q, 0, max_batches - batches, grid_max, team, nullptr, nullptr);
            else if (lit) launch_batches_lit(g, a, q, 0, max_batches - batches);
            else launch_batches(g, a, q, 0, max_batches - batches);
            batches = max_batches;
            LF_CUDA(cudaStreamSynchronize(st));
            int32_t err = 0;
            LF_CUDA(cudaMemcpy(&err, &g->ds->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (err & DERR_TIMEOUT) fail(LF_ERR_TIMEOUT, "a grid-barrier wait ran out (limit %d ms)", g->barrier_timeout_ms);
            break;
        }
        if (persistent) {
            launch_persistent(g, a, q, 0, nb, grid_max, team, pev[0], pev[1]);
            launch_iteration_end(g, a);
        } else if (g->use_graphs > 0 && max_batches < 0) {
            if (!g->iter_exec || g->graph_q != q || g->graph_K != g->K || g->graph_sched != g->sched_version ||
                g->graph_wpn != g->warps_per_node || g->graph_wmd != g->warp_max_degree ||
                g->graph_hdeg != g->hub_degree) {
                drop_graph(g);
                cudaGraph_t graph;
                const unsigned long long before = g->launches;
                LF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                try {
                    if (lit) launch_batches_lit(g, a, q, 0, nb, true);
                    else launch_batches(g, a, q, 0, nb, true);
                    launch_iteration_end(g, a);
                } catch (...) {
                    cudaGraph_t tmp;
                    cudaStreamEndCapture(st, &tmp);
                    if (tmp) cudaGraphDestroy(tmp);
                    throw;
                }
                LF_CUDA(cudaStreamEndCapture(st, &graph));
                g->graph_kernels = g->launches - before;
                g->launches = before;
                cudaError_t e = cudaGraphInstantiate(&g->iter_exec, graph, 0);
                cudaGraphDestroy(graph);
                LF_CUDA(e);
                g->graph_q = (int32_t)q;
                g->graph_K = g->K;
                g->graph_sched = g->sched_version;
                g->graph_wpn = g->warps_per_node;
                g->graph_wmd = g->warp_max_degree;
                g->graph_hdeg = g->hub_degree;
            }
            LF_CUDA(cudaGraphLaunch(g->iter_exec, st));
            g->launches += g->graph_kernels;
        } else {
            if (lit) launch_batches_lit(g, a, q, 0, nb);
            else launch_batches(g, a, q, 0, nb);
            launch_iteration_end(g, a);
        }
        batches += nb;
        LF_CUDA(cudaStreamSynchronize(st));
        if (g->profile && persistent) {
            prof_ms += elapsed_ms(pev[0], pev[1]);
            prof_launches += 1;
            if (g->qtimes && nb > 0) {
                std::vector<unsigned long long> t((size_t)nb + 1);
                LF_CUDA(cudaMemcpy(t.data(), g->qtimes, (size_t)(nb + 1) * 8, cudaMemcpyDeviceToHost));
                std::vector<double> dt((size_t)nb);
                for (int64_t b = 0; b < nb; ++b) dt[(size_t)b] = 1e-3 * (double)(t[(size_t)b + 1] - t[(size_t)b]);
                std::sort(dt.begin(), dt.end());
                const double fr[3] = {0.5, 0.9, 0.99};
                for (int k = 0; k < 3; ++k) qpct[k] = dt[(size_t)std::min<int64_t>(nb - 1, (int64_t)(fr[k] * nb))];
                qpct[3] = dt.back();
            }
        } else if (g->profile) {
            for (int64_t b = 0; b < nb && !std::isnan(prof_ms); ++b) {
                float t = 0.f;
                if (cudaEventElapsedTime(&t, g->prof_ev[2 * b], g->prof_ev[2 * b + 1]) == cudaSuccess) {
                    prof_ms += (double)t;
                } else {
                    cudaGetLastError();   // timing unavailable for this launch mode: report NaN
                    prof_ms = std::nan("");
                }
            }
            prof_launches += nb;
        }
        const Readback rb = *g->rb;
        if (rb.err & DERR_TIMEOUT) fail(LF_ERR_TIMEOUT, "a grid-barrier wait ran out (limit %d ms)", g->barrier_timeout_ms);
        if (rb.err & DERR_CAPACITY) fail(LF_ERR_CAPACITY, "membership row overflow (internal bound violated)");
        if (rb.err & DERR_CHECK)
            fail(LF_ERR_CUDA, "a device-side consistency check failed (bounds-checked mode or table partitioning)");
        iters = it;
        maxcnt = rb.maxcnt;
        last_live = rb.live_comms;
        last_memb = rb.memberships;
        if (stats && stats->history_cap >= it) {
            if (stats->wcc_history) stats->wcc_history[it - 1] = rb.total;
            if (stats->joins_history) stats->joins_history[it - 1] = (int64_t)rb.joins;
            if (stats->leaves_history) stats->leaves_history[it - 1] = (int64_t)rb.leaves;
        }
        if (batch) {   // each graph's own stopping test
            for (int64_t i = 0; i < g->ngraphs; ++i) {
                if (!gactive[(size_t)i]) continue;
                const double Ti = g->gT_host[i], Pi = gprev[(size_t)i];
                g->g_hist[(size_t)i].push_back(Ti);
                g->g_iters[(size_t)i] = it;
                const bool stop_i = Pi == 0.0 ? (Ti == 0.0) : ((Ti - Pi) / Pi) < thr;
                gprev[(size_t)i] = Ti;
                if (stop_i) {
                    gactive[(size_t)i] = 0;
                    g->g_conv[(size_t)i] = 1;
                }
            }
            continue;
        }
        const double T = rb.total;
        if (g->it_cb) {   // the caller may read the communities of this iteration
            g->in_callback = true;
            int halt = 0;
            try {
                halt = g->it_cb(g, it, T, g->it_ctx);
            } catch (...) {
                g->in_callback = false;
                throw;
            }
            g->in_callback = false;
            if (halt) break;
        }
        bool stop;
        if (prev == 0.0) stop = (T == 0.0);
        else stop = ((T - prev) / prev) < thr;
        prev = T;
        if (stop) {
            converged = 1;
            break;
        }
    }
    LF_CUDA(cudaEventRecord(ev[2], st));
    LF_CUDA(cudaStreamSynchronize(st));
    if (batch) {   // converged when every graph did
        converged = 1;
        for (int64_t i = 0; i < g->ngraphs; ++i)
            if (g->gnoff[(size_t)i + 1] > g->gnoff[(size_t)i] && !g->g_conv[(size_t)i]) converged = 0;
    }
    if (stats) {
        stats->iterations = iters;
        stats->converged = converged;
        stats->num_batches = batches;
        stats->wcc_initial = T0;
        stats->num_communities = (int64_t)last_live;
        stats->num_memberships = (int64_t)last_memb;
        stats->ms_init = elapsed_ms(ev[0], ev[1]);
        stats->ms_iterations = elapsed_ms(ev[1], ev[2]);
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats->num_launches = (int64_t)(g->launches - launches0);
        stats->prof_move_launches = prof_launches;
        stats->prof_move_ms = prof_ms;
        unsigned long long pbytes = 0, pc[2] = {0, 0};
        if (g->profile) {
            LF_CUDA(cudaMemcpy(&pbytes, &g->ds->prof_bytes, 8, cudaMemcpyDeviceToHost));
            LF_CUDA(cudaMemcpy(pc, &g->ds->prof_cands, 16, cudaMemcpyDeviceToHost));
        }
        stats->prof_move_bytes = (int64_t)pbytes;
        stats->prof_candidates = (int64_t)pc[0];
        stats->prof_exact = (int64_t)pc[1];
        for (int k = 0; k < 4; ++k) stats->prof_queue_us[k] = qpct[k];
    }
}

}  // namespace lf
