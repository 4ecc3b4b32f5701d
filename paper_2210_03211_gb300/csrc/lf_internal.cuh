// Internal declarations of the LazyFox GB300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lazyfox.h"

namespace lf {

// ---------------------------------------------------------------------------
// Errors: internal code throws lf::Error; every ABI entry point catches it.
// ---------------------------------------------------------------------------
struct Error {
    lf_status status;
};

void set_error(lf_status st, const char *fmt, ...);
[[noreturn]] void fail(lf_status st, const char *fmt, ...);

#define LF_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            ::lf::fail(LF_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                       cudaGetErrorString(e_));                                            \
    } while (0)

#define LF_LAUNCHED() LF_CUDA(cudaGetLastError())

constexpr unsigned FULL = 0xffffffffu;
constexpr int32_t EMPTY_KEY = -1;
constexpr uint32_t OWN_FLAG = 0x80000000u;
constexpr int SACC_CHUNKS = 68;   // 32-bit digits, bit 0 = 2^-1074

// Device error bits (DevScalars::err).
constexpr int32_t DERR_CAPACITY = 1;    // a membership row overflowed
constexpr int32_t DERR_CHECK = 2;       // a consistency check failed
constexpr int32_t DERR_TIMEOUT = 4;     // a bounded grid-barrier wait ran out

// Community aggregate record: members, 2 x internal edges (sum of internal
// degrees), sum of member degrees.  16 bytes: one vector load per candidate.
struct __align__(16) CommRec {
    int32_t n;
    uint32_t m2;
    uint32_t vol;
    int32_t gid;   // graph of the community in a batch of graphs (0 for one graph)
};

// Small device-resident scalars of one graph.
struct DevScalars {
    unsigned long long sacc[SACC_CHUNKS];   // superaccumulator (exact sum)
    double total;                           // last rounded exact sum
    double cc;                              // global clustering coefficient
    unsigned long long joins, leaves;       // actions applied in this iteration
    unsigned long long num_tri;             // triangle count
    unsigned long long merge_bytes;         // triangle merge-stream bytes
    unsigned long long live_comms;          // communities with n >= 2 after pruning
    unsigned long long memberships;         // sum of row counts after pruning
    unsigned long long prof_bytes;          // profile mode: move-evaluation algorithmic bytes
    unsigned long long prof_cands;          // profile mode, paper's gain: candidates bracketed
    unsigned long long prof_exact;          // profile mode, paper's gain: candidates summed exactly
    int32_t maxcnt;                         // max memberships of a node (after pruning)
    int32_t kb;                             // bound on memberships during an iteration
    int32_t err;                            // DERR_* bits
    int32_t iter;                           // iteration counter (stamps)
    int32_t undecided;                      // MIS rounds
    int32_t bad_runs;                       // order fix-up
    int32_t count32;
    int32_t max_id;
    int32_t neg_id;
    unsigned bar_count;                     // grid barrier: arrivals
    unsigned bar_gen;                       // grid barrier: generation
    int32_t pad;
};

// What the host reads back after each iteration (pinned).
struct Readback {
    double total;
    unsigned long long joins, leaves, live_comms, memberships;
    int32_t maxcnt;
    int32_t err;
};

}  // namespace lf

// ---------------------------------------------------------------------------
// The graph handle.
// ---------------------------------------------------------------------------
struct lf_graph {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lf_alloc_fn alloc_cb = nullptr;
    lf_free_fn free_cb = nullptr;
    void *alloc_ctx = nullptr;
    int32_t member_slots = 4;
    int32_t warp_max_degree = 0;
    int32_t use_graphs = 1;
    int32_t profile = 0;
    int32_t screen = 1;                            // FP32 candidate screen in the move evaluation
    int32_t per_queue = -1;                        // 1: launches per queue, 0: persistent loop, -1: by queue size
    int32_t barrier_timeout_ms = 2000;
    int32_t inject_stall = 0;
    int32_t barrier_mode = 0;                      // grid barrier: 0 flat flags, 1 central release flag
    int32_t warps_per_node = 0;                    // team size of the move evaluation (0: by queue size)
    int32_t hub_degree = 384;                      // above it a node takes the hub path
    int32_t gain_rule = LF_GAIN_LITERAL;           // decision rule of the move evaluation (paper's gain)
    int32_t debug_checks = 0;                      // bounds-checked kernels
    unsigned long long launches = 0;               // kernels launched (host count)
    std::vector<std::pair<void *, size_t>> live;   // outstanding allocations

    // graph
    int64_t n = 0, m = 0;
    int32_t *labels = nullptr;   // n
    int64_t *off = nullptr;      // n+1
    int32_t *adj = nullptr;      // 2m
    int32_t *deg = nullptr;      // n
    int64_t *ooff = nullptr;     // n+1
    int32_t *oadj = nullptr;     // m
    int32_t *odeg = nullptr;     // n
    long long *tri = nullptr;    // n  t(x,V)
    int32_t *vt = nullptr;       // n
    int32_t *order = nullptr;    // n
    int32_t *pos = nullptr;      // n  position in the order
    int32_t max_deg = 0;
    double cc = 0.0;
    lf::DevScalars *ds = nullptr;
    lf::Readback *rb = nullptr;  // pinned host
    lf_create_stats cstats{};

    // run state
    bool ran = false;
    int64_t ncomm = 0;            // community ids 0..ncomm-1
    // inserted division (dense ids), replacing the initial clustering; part_k < 0 = none
    int64_t part_k = -1;
    std::vector<int64_t> part_off;
    std::vector<int32_t> part_mem;
    int32_t part_maxcnt = 0;      // most communities of one node in it
    lf_iteration_fn it_cb = nullptr;
    void *it_ctx = nullptr;
    bool in_callback = false;
    // a batch of independent graphs held as one disjoint union (ngraphs > 0):
    // graph i's nodes are the dense ids [gnoff[i], gnoff[i+1]), its original
    // ids were shifted by gbase[i]; per-graph cc, WCC-hat sums and stop tests
    int64_t ngraphs = 0;
    std::vector<int64_t> gnoff, gbase;
    int32_t *gid = nullptr;                 // graph of each node
    double *gcc = nullptr;                  // per-graph cc
    float *gcc32 = nullptr;                 // per-graph cc rounded to float
    unsigned long long *gsacc = nullptr;    // per-graph exact sums (SACC_CHUNKS words each)
    double *gT = nullptr;                   // per-graph WCC-hat(P) of the last iteration end
    double *gT_host = nullptr;              // its pinned host copy
    std::vector<double> gcc_host;
    std::vector<int32_t> g_iters, g_conv;   // per graph: iterations run, converged
    std::vector<double> g_T0;
    std::vector<std::vector<double>> g_hist;
    // queue schedule of a batch: queue b holds qorder[sched[b] .. sched[b+1])
    int32_t *qorder = nullptr;
    int32_t *qpos = nullptr;                // position of every node in qorder (-1: not queued)
    std::vector<int64_t> sched;
    int64_t sched_version = 0, graph_sched = -1, hub_plan_sched = -1;
    int32_t graph_wpn = -1, graph_wmd = -1, graph_hdeg = -1;   // launch shape of the captured iteration
    lf::CommRec *comm = nullptr;  // n records (ncomm used)
    unsigned long long *stamp = nullptr;  // n words
    int32_t K = 0;                // row capacity
    int32_t *mem = nullptr;       // n*K
    int32_t *nmem = nullptr;      // n
    int32_t qcap = 0;             // queue capacity of the action arrays
    int32_t *act = nullptr;       // 4*qcap: join, leave, kjoin, kleave
    cudaGraphExec_t iter_exec = nullptr;
    int32_t graph_q = 0, graph_K = 0;
    unsigned long long graph_kernels = 0;          // kernel nodes of iter_exec
    std::vector<cudaEvent_t> prof_ev;              // profile mode: 2 per queue
    unsigned *bar_flags = nullptr;                 // grid barrier: one epoch flag per block
    int bar_flags_cap = 0;
    unsigned bar_epoch = 0;
    unsigned long long *qtimes = nullptr;          // profile mode: per-queue time stamps
    // hubs evaluated with global-memory tables (plan for queue size hub_plan_q, row capacity hub_plan_K)
    int32_t *hub_pos = nullptr;
    int64_t *hub_qoff = nullptr;
    int64_t *hub_toff = nullptr;
    uint32_t *hub_tcap = nullptr;      // table size used this iteration (<= hub_wcap)
    uint32_t *hub_wcap = nullptr;      // table size planned for the worst case, (d+1) K entries
    int32_t *hub_scratch = nullptr;
    int64_t hub_slots = 0;
    std::vector<int64_t> hub_qoff_host;
    // chunks of HUGE_CHUNK neighbours per hub: (hub, chunk) pairs listed per
    // queue, chunks per hub, chunks finished per hub (zero between queues)
    int32_t *hub_chunk_h = nullptr;
    int32_t *hub_chunk_c = nullptr;
    int32_t *hub_nch = nullptr;
    uint32_t *hub_done = nullptr;
    uint32_t *hub_ncand = nullptr;      // distinct ids in each hub's table, listed in its lower-bound area
    // hubs with many candidates are screened and evaluated by several blocks:
    // per hub the best lower bounds (order-preserving ints), its items and
    // items finished; per item (hub, chunk) and its best actions
    int32_t *hub_lbj = nullptr, *hub_lbl = nullptr;
    uint32_t *hub_item_base = nullptr, *hub_nitems = nullptr, *hub_items_done = nullptr;
    int32_t *hub_items = nullptr;       // 2 per item
    double *hub_item_g = nullptr;       // 2 per item (join, leave)
    int32_t *hub_item_ck = nullptr;     // 4 per item (join id, join k, leave id, leave k)
    int64_t hub_items_cap = 0;
    uint32_t *hub_qctr = nullptr;       // 3 per queue: items, next to screen, next to evaluate
    std::vector<char> hub_qbig;         // per queue: may hold a hub with more than HUGE_BIG_NCAND candidates
    std::vector<int64_t> hub_cqoff_host;
    int64_t hub_plan_q = 0;
    int32_t hub_plan_K = 0;
    int32_t hub_plan_deg = 0;
    // nodes of degree > TOT_CHUNK in the WCC-hat total, counted in chunks of
    // neighbours (plan for row capacity tot_plan_K)
    int32_t *tot_hubs = nullptr;        // node ids, degree descending
    int32_t *tot_chunk_hub = nullptr;   // hub index of each chunk
    int32_t *tot_first = nullptr;       // first chunk of each hub (tot_nh + 1 entries)
    int32_t *tot_cnt = nullptr;         // tot_nh x tot_plan_K counts, zero between launches
    uint32_t *tot_done = nullptr;       // chunks finished per hub, zero between launches
    uint32_t *tot_next = nullptr;       // work counters: node runs, chunks
    int64_t tot_nh = 0, tot_nchunks = 0;
    int32_t tot_plan_K = 0;
    // large queues: per-queue counters (next node, overflow count), overflow
    // list (queue positions) and their histogram bounds
    uint32_t *dyn_ctr = nullptr;
    int64_t dyn_ctr_cap = 0;
    int32_t *dyn_list = nullptr;
    long long *dyn_bound = nullptr;
    int64_t dyn_list_cap = 0;
    // the paper's gain (gain_rule == LF_GAIN_LITERAL): deg(x,C) beside each
    // membership, the member index of the current iteration (members at its
    // start, by community; its joiners as per-community lists), per-community
    // sums F(n-1), F(n), F(n+1), per-queue counters (overflow count, overflow
    // next, touched count), the overflow list, the touched list and stamps
    int32_t *kmem = nullptr;              // n*K
    unsigned long long *cm_off = nullptr; // n+1
    unsigned long long *cm_cur = nullptr; // n+1
    int32_t *cm_node = nullptr;           // regions of (4 members + 32) entries per community
    uint32_t *cm_cnt = nullptr;           // n: entries used per region
    int64_t cm_cap = 0;
    int32_t *jl_head = nullptr, *jl_next = nullptr, *jl_node = nullptr;   // n each
    uint32_t *lit_misc = nullptr;         // [0]: joiners listed in this iteration
    float *litF = nullptr;                // 8n: F(n-1), F(n+1), WCC-hat(C), 1/((n+1)n cc), 1/((n-1)(n-2) cc)
    uint32_t *tstamp = nullptr;           // n
    uint32_t *lit_ctr = nullptr;          // 3 per queue
    int64_t lit_ctr_cap = 0;
    int32_t *lit_over = nullptr;          // qcap
    int32_t *touched = nullptr;           // 2 qcap
    int64_t lit_qcap = 0;
    unsigned long long *lit_used = nullptr;   // per queue: global table slots handed out
    void *lg_area = nullptr;              // global tables: lg_cap slots of 16 bytes
    unsigned long long lg_cap = 0;
    int64_t lg_plan_q = -1, lg_plan_sched = -1;
    int32_t lg_plan_K = 0;
    // hubs under the paper's gain: per hub its queue position, table offset
    // and size, survivor-list offset, slot items, best lower ends, counters;
    // fill items and slot items of all queues (offsets per queue on the host);
    // the tables and survivor lists shared by the queues
    int64_t lh_plan_q = -1, lh_plan_sched = -1;
    int32_t lh_plan_K = 0;
    int64_t lh_n = 0;
    std::vector<int64_t> lh_fq, lh_sq, lh_hq;
    uint32_t *lh_heff = nullptr;
    int32_t *lh_pos = nullptr, *lh_nsr = nullptr, *lh_fh = nullptr, *lh_fc = nullptr, *lh_sh = nullptr,
            *lh_sr = nullptr, *lh_svc = nullptr;
    int64_t *lh_toff = nullptr, *lh_soff = nullptr;
    uint32_t *lh_tcap = nullptr, *lh_ns = nullptr, *lh_svv = nullptr;
    int32_t *lh_lb = nullptr;
    float *lh_svl = nullptr;
    void *lh_tab = nullptr;               // tables: 16 bytes per slot
    int64_t lh_tab_cap = 0;
    // second stream: hub chunks run beside the other evaluation kernels of a queue
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace lf {

// memory
void *dalloc(lf_graph *g, size_t bytes);
void dfree(lf_graph *g, void *p);
template <typename T>
T *dalloc_n(lf_graph *g, int64_t count) {
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    return static_cast<T *>(dalloc(g, bytes));
}

// primitives (lf_prims.cu)
template <typename T>
void scan_exclusive(lf_graph *g, const T *in, T *out, int64_t count, T *d_total);
void radix_sort(lf_graph *g, unsigned long long *keys, uint32_t *vals, int64_t count,
                const std::vector<int> &shifts);
int bits_for(unsigned long long max_value);   // bits needed to hold max_value

// run (lf_run.cu)
void run_impl(lf_graph *g, int32_t q, double thr, int32_t max_iters, int64_t max_batches,
              lf_run_stats *stats);
void free_run_state(lf_graph *g);

inline unsigned grid_for(int64_t work, int per_block, int64_t cap = 1 << 20) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// ---------------------------------------------------------------------------
// Device helpers shared by the kernels.
// ---------------------------------------------------------------------------

// C(z,2) for z >= 1, else 0 -- written 0.5*(z*(z-1)) with each operation
// rounded once (no fused multiply-add anywhere in the score functions).
__device__ __forceinline__ double binom2(double z) {
    return z >= 1.0 ? __dmul_rn(0.5, __dmul_rn(z, __dsub_rn(z, 1.0))) : 0.0;
}

// WCC-hat(x,C) of a member x with deg(x,C) = k, deg(x,V) = d, in a community
// with n members and m2 = 2 x (internal edges):
//   E[t(x,C)] / E[t(x,V)] * d / (|C \ {x}| + deg(x, V \ C)),
//   E[t(x,C)] = C(k,2) p, p = m2 / (n (n-1)),  E[t(x,V)] = C(d,2) cc.
// (Heuristic Counting of Triangles; zero when n < 2 or E[t(x,V)] = 0.)
__device__ __forceinline__ double wcchat_member(int64_t k, int64_t d, int64_t n, uint32_t m2,
                                                double cc) {
    if (n < 2) return 0.0;
    double nd = (double)n;
    double p = __ddiv_rn((double)m2, __dmul_rn(nd, __dsub_rn(nd, 1.0)));
    double ec = __dmul_rn(binom2((double)k), p);
    double ev = __dmul_rn(binom2((double)d), cc);
    if (!(ev > 0.0)) return 0.0;
    double dd = (double)d;
    return __dmul_rn(__ddiv_rn(ec, ev),
                     __ddiv_rn(dd, __dadd_rn(__dsub_rn(nd, 1.0), __dsub_rn(dd, (double)k))));
}

// Mean-field community score: every member given the mean internal degree
// m2/n and the mean total degree vol/n, put through WCC-hat and summed
// (n copies).  The gain of a join or leave is the change of this score.
__device__ __forceinline__ double community_score(int64_t n, int64_t m2, int64_t vol, double cc) {
    if (n < 2) return 0.0;
    // all three fit in 32 bits (n < 2^31, m2 and vol < 2^32): exact conversions
    const double nd = __uint2double_rn((uint32_t)n);
    const double md = __uint2double_rn((uint32_t)m2);
    const double vd = __uint2double_rn((uint32_t)vol);
    double din = __ddiv_rn(md, nd);
    double dt = __ddiv_rn(vd, nd);
    double p = __ddiv_rn(md, __dmul_rn(nd, __dsub_rn(nd, 1.0)));
    double ec = __dmul_rn(binom2(din), p);
    double ev = __dmul_rn(binom2(dt), cc);
    if (!(ev > 0.0)) return 0.0;
    return __dmul_rn(nd, __dmul_rn(__ddiv_rn(ec, ev),
                                   __ddiv_rn(dt, __dadd_rn(__dsub_rn(nd, 1.0), __dsub_rn(dt, din)))));
}

// Add a finite, non-negative double exactly into a fixed-point accumulator of
// 32-bit digits held in 64-bit words (bit 0 = 2^-1074).  Integer atomics, so
// the result does not depend on the order of the additions.  Each word can
// take 2^31 additions before it could overflow.
__device__ __forceinline__ void sacc_add(unsigned long long *acc, double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (b == 0ull) return;
    unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    unsigned long long mant = b & 0xfffffffffffffull;
    int p;
    if (e == 0) {
        p = 0;
    } else {
        mant |= 1ull << 52;
        p = (int)e - 1;
    }
    int c = p >> 5, sh = p & 31;
    unsigned long long lo = mant << sh;
    unsigned long long hi = sh ? (mant >> (64 - sh)) : 0ull;
    unsigned long long d0 = lo & 0xffffffffull, d1 = lo >> 32;
    if (d0) atomicAdd(&acc[c], d0);
    if (d1) atomicAdd(&acc[c + 1], d1);
    if (hi) atomicAdd(&acc[c + 2], hi);
}

// Round the accumulated exact value to the nearest double (ties to even) and
// clear the accumulator.  One thread.
__device__ inline double sacc_round_and_clear(unsigned long long *acc) {
    uint32_t dg[SACC_CHUNKS];
    unsigned long long carry = 0;
    for (int i = 0; i < SACC_CHUNKS; ++i) {
        unsigned long long v = acc[i] + carry;
        acc[i] = 0ull;
        dg[i] = (uint32_t)(v & 0xffffffffull);
        carry = v >> 32;
    }
    int top = -1;
    for (int i = SACC_CHUNKS - 1; i >= 0; --i)
        if (dg[i]) { top = i; break; }
    if (top < 0) return 0.0;
    int P = 32 * top + (31 - __clz((int)dg[top]));   // index of the leading bit
    auto bit = [&](int q) -> unsigned long long {
        return q < 0 ? 0ull : (unsigned long long)((dg[q >> 5] >> (q & 31)) & 1u);
    };
    if (P <= 52) {   // fewer than 54 significant bits: exact (subnormal or smallest binade)
        unsigned long long v = 0;
        for (int q = P; q >= 0; --q) v = (v << 1) | bit(q);
        return __longlong_as_double((long long)v);
    }
    unsigned long long mant = 0;
    for (int q = P; q >= P - 52; --q) mant = (mant << 1) | bit(q);
    int r = P - 53;                        // round bit position (>= 0)
    bool round_bit = bit(r) != 0;
    bool sticky = false;
    for (int i = 0; i < (r >> 5) && !sticky; ++i) sticky = dg[i] != 0u;
    if (!sticky && (r & 31)) sticky = (dg[r >> 5] & ((1u << (r & 31)) - 1u)) != 0u;
    if (round_bit && (sticky || (mant & 1ull))) ++mant;
    if (mant == (1ull << 53)) {
        mant >>= 1;
        ++P;
    }
    long long biased = (long long)P - 51;
    if (biased >= 2047) return __longlong_as_double(0x7ff0000000000000ll);
    unsigned long long bits = ((unsigned long long)biased << 52) | (mant & 0xfffffffffffffull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

}  // namespace lf
