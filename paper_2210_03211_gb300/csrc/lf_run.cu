// Fox / LazyFox iterations on the GPU (Methods: Initial Clustering; Node
// Changes, Algorithm 1; Parallelism on Node Change Computations, Algorithm 2;
// Stopping Criteria; Post-processing):
//   a6  initial clustering: greedy non-overlapping decomposition in node order
//   a7  move evaluation of one queue: per-node community histogram in shared
//       memory, mean-field WCC-hat gains, best join / best leave
//   a8  bulk apply of one queue: membership rows and community aggregates,
//       with the exact internal-edge correction for nodes that move together
//   a9  iteration end: removal of degenerate communities, exact WCC-hat(P)
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

struct RunArgs {
    const int64_t *off;
    const int32_t *adj;
    const int32_t *deg;
    const int32_t *order;
    const int32_t *pos;
    CommRec *comm;
    unsigned long long *stamp;
    int32_t *mem;
    int32_t *nmem;
    int32_t K;
    int32_t qcap;
    int32_t *act;   // [join | leave | kjoin | kleave], qcap each
    DevScalars *ds;
    Readback *rbd;
    double cc;
    int64_t nbatches;
    int32_t warp_max_deg;
    int32_t profile;   // count algorithmic bytes of the move evaluation
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
        atomicAdd(&a.comm[c].n, 1);
        atomicAdd(&a.comm[c].vol, (uint32_t)a.deg[x]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ds->maxcnt = n > 0 ? 1 : 0;
        a.ds->memberships = (unsigned long long)n;
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
    const double before = community_score(n, m2, vol, a.cc);
    if (own) {
        double g = __dsub_rn(community_score(n - 1, m2 - 2 * k, vol - d, a.cc), before);
        if (g > 0.0 && better(g, C, bl.g, bl.c)) bl = Best{g, C, (int32_t)k};
    } else {
        double g = __dsub_rn(community_score(n + 1, m2 + 2 * k, vol + d, a.cc), before);
        if (g > 0.0 && better(g, C, bj.g, bj.c)) bj = Best{g, C, (int32_t)k};
    }
}

// Saturating "how many actions of this queue target C" counter, tagged with
// the queue's serial number so that it never needs clearing.
__device__ __forceinline__ void stamp_add(unsigned long long *w, unsigned long long serial) {
    unsigned long long old = *((volatile unsigned long long *)w), assumed;
    do {
        assumed = old;
        unsigned long long c = (assumed >> 2) == serial ? (assumed & 3ull) : 0ull;
        unsigned long long nw = (serial << 2) | (c >= 2ull ? 2ull : c + 1ull);
        if (nw == assumed) return;
        old = atomicCAS(w, assumed, nw);
    } while (old != assumed);
}

__device__ __forceinline__ bool stamp_multi(const unsigned long long *w, unsigned long long serial) {
    unsigned long long v = __ldcg(w);
    return (v >> 2) == serial && (v & 3ull) >= 2ull;
}

__device__ __forceinline__ void write_action(const RunArgs &a, int i, const Best &bj, const Best &bl,
                                             unsigned long long serial) {
    a.act[i] = bj.c;
    a.act[a.qcap + i] = bl.c;
    a.act[2 * a.qcap + i] = bj.k;
    a.act[3 * a.qcap + i] = bl.k;
    if (bj.c >= 0) stamp_add(a.stamp + bj.c, serial);
    if (bl.c >= 0) stamp_add(a.stamp + bl.c, serial);
}

// One warp, one node: every membership of every neighbour goes into the
// warp's table; equal ids arriving in the same step are merged first with
// __match_any_sync, so each id costs one atomic per step.  `bound` (>= the
// number of distinct ids) keeps the table at most half full.
__device__ void eval_warp(const RunArgs &a, int i, int32_t x, int32_t d, int64_t bound, int32_t *keys,
                          uint32_t *vals, unsigned long long serial) {
    const int lane = threadIdx.x & 31;
    uint32_t H = 32;
    while ((int64_t)H < 2 * bound) H <<= 1;
    const uint32_t hm = H - 1;
    for (uint32_t s = lane; s < H; s += 32) {
        keys[s] = EMPTY_KEY;
        vals[s] = 0u;
    }
    __syncwarp();
    const int32_t cx = a.nmem[x];
    const int32_t *rowx = a.mem + (int64_t)x * a.K;
    for (int j = lane; j < cx; j += 32) ht_insert(keys, vals, hm, rowx[j], 0u, true);
    __syncwarp();
    const int64_t beg = a.off[x], end = a.off[x + 1];
    unsigned long long pb = 0;
    for (int64_t p0 = beg; p0 < end; p0 += 32) {
        const int64_t p = p0 + lane;
        int32_t y = 0, cy = 0;
        if (p < end) {
            y = a.adj[p];
            cy = a.nmem[y];
            pb += 8ull + 4ull * (unsigned long long)cy;
        }
        const int32_t cmax = __reduce_max_sync(FULL, cy);
        const int32_t *rowy = a.mem + (int64_t)y * a.K;
        for (int s = 0; s < cmax; ++s) {
            int32_t C = s < cy ? rowy[s] : -2 - lane;
            unsigned mask = __match_any_sync(FULL, C);
            if (C >= 0 && lane == __ffs(mask) - 1) ht_insert(keys, vals, hm, C, (uint32_t)__popc(mask), false);
        }
    }
    __syncwarp();
    Best bj{0.0, -1, 0}, bl{0.0, -1, 0};
    for (uint32_t s = lane; s < H; s += 32) {
        int32_t C = keys[s];
        if (C != EMPTY_KEY) {
            eval_candidate(a, C, vals[s], d, bj, bl);
            pb += 16ull;
        }
    }
    warp_best(bj);
    warp_best(bl);
    if (a.profile) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pb += __shfl_down_sync(FULL, pb, o);
        if (lane == 0) atomicAdd(&a.ds->prof_bytes, pb + 44ull + 4ull * (unsigned long long)cx);
    }
    if (lane == 0) write_action(a, i, bj, bl, serial);
    __syncwarp();
}

__device__ __forceinline__ uint32_t part_of(int32_t C, int P) {
    return hash32((uint32_t)C ^ 0x9e3779b9u) % (uint32_t)P;
}

struct BlockScratch {
    double gj[EV_WARPS], gl[EV_WARPS];
    int32_t cj[EV_WARPS], cl[EV_WARPS], kj[EV_WARPS], kl[EV_WARPS];
    int overflow;
};

// One block, one node (high degree).  The ids are split into P parts by a
// hash and each part is counted in the block's table in its own pass; if a
// pass overflows the table, P doubles and the evaluation restarts.
__device__ void eval_block(const RunArgs &a, int i, int32_t x, int64_t bound, int32_t *keys, uint32_t *vals,
                           BlockScratch &bs, unsigned long long serial) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t d = a.deg[x];
    const int32_t cx = a.nmem[x];
    const int32_t *rowx = a.mem + (int64_t)x * a.K;
    const int64_t beg = a.off[x], end = a.off[x + 1];
    int P = bound <= HB / 2 ? 1 : (int)((bound + HB / 4 - 1) / (HB / 4));
    Best bj, bl;
    unsigned long long pb = 0;
    for (;;) {
        bj = Best{0.0, -1, 0};
        bl = Best{0.0, -1, 0};
        pb = 0;
        uint32_t H = HB;
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
                int32_t C = rowx[j];
                if (P == 1 || part_of(C, P) == (uint32_t)part)
                    if (!ht_insert(keys, vals, hm, C, 0u, true)) bs.overflow = 1;
            }
            __syncthreads();
            for (int64_t p0 = beg + w * 32; p0 < end; p0 += EV_THREADS) {
                const int64_t p = p0 + lane;
                int32_t y = 0, cy = 0;
                if (p < end) {
                    y = a.adj[p];
                    cy = a.nmem[y];
                    if (part == 0) pb += 8ull + 4ull * (unsigned long long)cy;
                }
                const int32_t cmax = __reduce_max_sync(FULL, cy);
                const int32_t *rowy = a.mem + (int64_t)y * a.K;
                for (int s = 0; s < cmax; ++s) {
                    int32_t C = s < cy ? rowy[s] : -1;
                    if (C >= 0 && P > 1 && part_of(C, P) != (uint32_t)part) C = -1;
                    if (C < 0) C = -2 - lane;
                    unsigned mask = __match_any_sync(FULL, C);
                    if (C >= 0 && lane == __ffs(mask) - 1)
                        if (!ht_insert(keys, vals, hm, C, (uint32_t)__popc(mask), false)) bs.overflow = 1;
                }
            }
            __syncthreads();
            if (bs.overflow) {
                overflow = true;
                __syncthreads();
                break;
            }
            for (uint32_t s = threadIdx.x; s < H; s += EV_THREADS) {
                int32_t C = keys[s];
                if (C != EMPTY_KEY) {
                    eval_candidate(a, C, vals[s], d, bj, bl);
                    pb += 16ull;
                }
            }
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

__global__ void __launch_bounds__(EV_THREADS) k_eval(RunArgs a, int64_t bstart, int32_t blen, int64_t bidx) {
    __shared__ int32_t s_keys[HB];
    __shared__ uint32_t s_vals[HB];
    __shared__ int32_t s_hub[EV_WARPS];
    __shared__ int s_nhub;
    __shared__ BlockScratch bs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_nhub = 0;
    __syncthreads();
    const int32_t kb = __ldcg(&a.ds->kb);
    const unsigned long long serial = (unsigned long long)__ldcg(&a.ds->iter) * (unsigned long long)a.nbatches +
                                      (unsigned long long)bidx + 1ull;
    const int i = blockIdx.x * EV_WARPS + w;
    if (i < blen) {
        const int32_t x = a.order[bstart + i];
        const int32_t d = a.deg[x];
        const int64_t bound = (int64_t)(d + 1) * kb;
        if (d <= a.warp_max_deg && bound <= HW / 2) {
            eval_warp(a, i, x, d, bound, s_keys + w * HW, s_vals + w * HW, serial);
        } else if (lane == 0) {
            s_hub[atomicAdd(&s_nhub, 1)] = i;
        }
    }
    __syncthreads();
    const int nh = s_nhub;
    for (int h = 0; h < nh; ++h) {
        const int ih = s_hub[h];
        const int32_t x = a.order[bstart + ih];
        eval_block(a, ih, x, (int64_t)(a.deg[x] + 1) * kb, s_keys, s_vals, bs, serial);
    }
}

// ---------------------------------------------------------------------------
// a8: bulk apply of one queue.  For a joiner x of C (k = |N(x) & C| before the
// queue), the internal edge sum 2m_C grows by 2k + (joiner neighbours of x
// also joining C) - 2 (neighbours of x leaving C); for a leaver it shrinks by
// 2k - (neighbours of x also leaving C).  Summed over the queue this is the
// exact change of 2m_C; the neighbour scan is needed only when another action
// of the same queue targets C.  Integer atomics: order-independent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(AP_THREADS) k_apply(RunArgs a, int64_t bstart, int32_t blen, int64_t bidx) {
    __shared__ unsigned long long s_j, s_l;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_j = 0;
        s_l = 0;
    }
    __syncthreads();
    const unsigned long long serial = (unsigned long long)__ldcg(&a.ds->iter) * (unsigned long long)a.nbatches +
                                      (unsigned long long)bidx + 1ull;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i < blen) {
        const int32_t j = a.act[i], l = a.act[a.qcap + i];
        if (j >= 0 || l >= 0) {
            const int32_t x = a.order[bstart + i];
            const bool nj = j >= 0 && stamp_multi(a.stamp + j, serial);
            const bool nl = l >= 0 && stamp_multi(a.stamp + l, serial);
            int jj = 0, jl = 0, ll = 0;
            if (nj || nl) {
                for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
                    const int32_t y = a.adj[p];
                    const int64_t py = a.pos[y];
                    if (py >= bstart && py < bstart + blen) {
                        const int64_t iy = py - bstart;
                        const int32_t aj = a.act[iy], al = a.act[a.qcap + iy];
                        if (nj) {
                            jj += aj == j;
                            jl += al == j;
                        }
                        if (nl) ll += al == l;
                    }
                }
                jj = __reduce_add_sync(FULL, jj);
                jl = __reduce_add_sync(FULL, jl);
                ll = __reduce_add_sync(FULL, ll);
            }
            if (lane == 0) {
                const int32_t d = a.deg[x];
                int32_t *row = a.mem + (int64_t)x * a.K;
                int32_t c = a.nmem[x];
                if (l >= 0) {
                    const int32_t kl = a.act[3 * a.qcap + i];
                    atomicAdd(&a.comm[l].n, -1);
                    atomicAdd(&a.comm[l].vol, (uint32_t)(-d));
                    atomicAdd(&a.comm[l].m2, (uint32_t)(-2 * kl + ll));
                    int32_t o = 0;
                    for (int32_t s = 0; s < c; ++s)
                        if (row[s] != l) row[o++] = row[s];
                    c = o;
                    atomicAdd(&s_l, 1ull);
                }
                if (j >= 0) {
                    const int32_t kj = a.act[2 * a.qcap + i];
                    atomicAdd(&a.comm[j].n, 1);
                    atomicAdd(&a.comm[j].vol, (uint32_t)d);
                    atomicAdd(&a.comm[j].m2, (uint32_t)(2 * kj + jj - 2 * jl));
                    if (c >= a.K) {
                        atomicOr(&a.ds->err, DERR_CAPACITY);
                    } else {
                        int32_t s = c;
                        while (s > 0 && row[s - 1] > j) {
                            row[s] = row[s - 1];
                            --s;
                        }
                        row[s] = j;
                        ++c;
                    }
                    atomicAdd(&s_j, 1ull);
                }
                a.nmem[x] = c;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_j) atomicAdd(&a.ds->joins, s_j);
        if (s_l) atomicAdd(&a.ds->leaves, s_l);
    }
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
                if (__ldcg(&a.comm[C].n) >= 2) row[o++] = C;
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
// deg(x, C) counted over x's neighbours; exact sum, so the total does not
// depend on the order of the additions.
__global__ void k_total(RunArgs a, int64_t n) {
    __shared__ unsigned long long acc[SACC_CHUNKS];
    for (int s = threadIdx.x; s < SACC_CHUNKS; s += blockDim.x) acc[s] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const int32_t c = a.nmem[x];
        if (c == 0) continue;
        const int32_t d = a.deg[x];
        const int32_t *row = a.mem + x * a.K;
        for (int32_t s = 0; s < c; ++s) {
            const int32_t C = row[s];
            int cnt = 0;
            for (int64_t p = a.off[x] + lane; p < a.off[x + 1]; p += 32) {
                const int32_t y = a.adj[p];
                cnt += row_has(a.mem + (int64_t)y * a.K, a.nmem[y], C);
            }
            cnt = __reduce_add_sync(FULL, cnt);
            if (lane == 0) {
                const int4 r = __ldcg(reinterpret_cast<const int4 *>(&a.comm[C]));
                sacc_add(acc, wcchat_member(cnt, d, r.x, (uint32_t)r.y, a.cc));
            }
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < SACC_CHUNKS; s += blockDim.x)
        if (acc[s]) atomicAdd(&a.ds->sacc[s], acc[s]);
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
                         int32_t K2) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = nmem[x];
        for (int32_t s = 0; s < c; ++s) mem2[x * K2 + s] = mem[x * K + s];
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
    a.stamp = g->stamp;
    a.mem = g->mem;
    a.nmem = g->nmem;
    a.K = g->K;
    a.qcap = g->qcap;
    a.act = g->act;
    a.ds = g->ds;
    a.rbd = rbd;
    a.cc = g->cc;
    a.nbatches = 0;
    a.warp_max_deg = g->warp_max_degree > 0 ? g->warp_max_degree : 0x7fffffff;
    a.profile = g->profile;
    return a;
}

Readback *device_readback(lf_graph *g) {
    // the device-side Readback sits right after the DevScalars block
    return reinterpret_cast<Readback *>(g->ds + 1);
}

void launch_batches(lf_graph *g, const RunArgs &a, int64_t q, int64_t first, int64_t count) {
    const bool prof = g->profile && (int64_t)g->prof_ev.size() >= 2 * (first + count);
    for (int64_t b = first; b < first + count; ++b) {
        const int64_t bstart = b * q;
        const int32_t blen = (int32_t)std::min<int64_t>(q, g->n - bstart);
        if (prof) LF_CUDA(cudaEventRecord(g->prof_ev[2 * b], g->stream));
        k_eval<<<(unsigned)((blen + EV_WARPS - 1) / EV_WARPS), EV_THREADS, 0, g->stream>>>(a, bstart, blen, b); ++g->launches;
        if (prof) LF_CUDA(cudaEventRecord(g->prof_ev[2 * b + 1], g->stream));
        k_apply<<<grid_for((int64_t)blen * 32, AP_THREADS, 1 << 30), AP_THREADS, 0, g->stream>>>(a, bstart, blen, b); ++g->launches;
    }
    LF_LAUNCHED();
}

void launch_iteration_end(lf_graph *g, const RunArgs &a) {
    const int64_t n = g->n;
    k_prune<<<grid_for(n + g->ncomm, 256, 1 << 16), 256, 0, g->stream>>>(a, n, g->ncomm); ++g->launches;
    k_total<<<grid_for(n * 32, 256, 1 << 16), 256, 0, g->stream>>>(a, n); ++g->launches;
    k_finalize<<<1, 32, 0, g->stream>>>(g->ds, device_readback(g), 1); ++g->launches;
    LF_LAUNCHED();
    LF_CUDA(cudaMemcpyAsync(g->rb, device_readback(g), sizeof(Readback), cudaMemcpyDeviceToHost, g->stream));
}

void drop_graph(lf_graph *g) {
    if (g->iter_exec) {
        cudaGraphExecDestroy(g->iter_exec);
        g->iter_exec = nullptr;
    }
}

void ensure_capacity(lf_graph *g, int64_t q) {
    const int64_t n = g->n;
    if (!g->comm) {
        g->comm = dalloc_n<CommRec>(g, n);
        g->stamp = dalloc_n<unsigned long long>(g, n);
        g->nmem = dalloc_n<int32_t>(g, n);
        g->K = std::max(2, g->member_slots);
        g->mem = dalloc_n<int32_t>(g, n * g->K);
    }
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
    k_regrow<<<grid_for(g->n, 256, 1 << 16), 256, 0, g->stream>>>(g->mem, g->nmem, g->n, g->K, mem2, K2); ++g->launches;
    LF_LAUNCHED();
    dfree(g, g->mem);
    g->mem = mem2;
    g->K = K2;
    drop_graph(g);
}

double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float t = 0.f;
    LF_CUDA(cudaEventElapsedTime(&t, a, b));
    return (double)t;
}

}  // namespace

void free_run_state(lf_graph *g) {
    drop_graph(g);
    for (auto e : g->prof_ev) cudaEventDestroy(e);
    g->prof_ev.clear();
    if (g->act) dfree(g, g->act);
    if (g->mem) dfree(g, g->mem);
    if (g->nmem) dfree(g, g->nmem);
    if (g->stamp) dfree(g, g->stamp);
    if (g->comm) dfree(g, g->comm);
    g->act = g->mem = g->nmem = nullptr;
    g->stamp = nullptr;
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
    const int64_t q = std::max<int64_t>(1, std::min<int64_t>(q_in, std::max<int64_t>(n, 1)));
    ensure_capacity(g, q);
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
    LF_CUDA(cudaMemsetAsync(g->stamp, 0, (size_t)std::max<int64_t>(n, 1) * 8, st));
    LF_CUDA(cudaMemsetAsync(g->nmem, 0, (size_t)std::max<int64_t>(n, 1) * 4, st));
    LF_CUDA(cudaMemsetAsync(g->ds->sacc, 0, sizeof(g->ds->sacc), st));
    {
        DevScalars z{};
        // zero the run counters (the fields from `joins` up to `max_id`)
        const size_t o = offsetof(DevScalars, joins);
        LF_CUDA(cudaMemcpyAsync(reinterpret_cast<char *>(g->ds) + o, reinterpret_cast<char *>(&z) + o,
                                offsetof(DevScalars, max_id) - o, cudaMemcpyHostToDevice, st));
        LF_CUDA(cudaStreamSynchronize(st));
    }
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

    // ---- a6: initial clustering
    int64_t k0 = 0;
    if (n > 0) {
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
    k_total<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(a, n); ++g->launches;
    k_finalize<<<1, 32, 0, st>>>(g->ds, device_readback(g), 0); ++g->launches;
    LF_LAUNCHED();
    LF_CUDA(cudaMemcpyAsync(g->rb, device_readback(g), sizeof(Readback), cudaMemcpyDeviceToHost, st));
    LF_CUDA(cudaEventRecord(ev[1], st));
    LF_CUDA(cudaStreamSynchronize(st));
    const double T0 = g->rb->total;
    int32_t maxcnt = g->rb->maxcnt;
    g->ran = true;

    const int64_t nb = n > 0 ? (n + q - 1) / q : 0;
    int32_t iters = 0, converged = 0;
    int64_t batches = 0;
    double prev = T0;
    unsigned long long last_live = (unsigned long long)k0, last_memb = (unsigned long long)n;
    for (int32_t it = 1; it <= max_iters; ++it) {
        if (maxcnt + 1 > g->K) grow_rows(g, maxcnt + 1);
        a = make_args(g, device_readback(g));
        a.nbatches = nb;
        const bool partial = max_batches >= 0 && batches + nb > max_batches;
        if (partial) {
            launch_batches(g, a, q, 0, max_batches - batches);
            batches = max_batches;
            LF_CUDA(cudaStreamSynchronize(st));
            break;
        }
        if (g->use_graphs > 0 && max_batches < 0) {
            if (!g->iter_exec || g->graph_q != q || g->graph_K != g->K) {
                drop_graph(g);
                cudaGraph_t graph;
                const unsigned long long before = g->launches;
                LF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                try {
                    launch_batches(g, a, q, 0, nb);
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
            }
            LF_CUDA(cudaGraphLaunch(g->iter_exec, st));
            g->launches += g->graph_kernels;
        } else {
            launch_batches(g, a, q, 0, nb);
            launch_iteration_end(g, a);
        }
        batches += nb;
        LF_CUDA(cudaStreamSynchronize(st));
        if (g->profile) {
            for (int64_t b = 0; b < nb; ++b) prof_ms += elapsed_ms(g->prof_ev[2 * b], g->prof_ev[2 * b + 1]);
            prof_launches += nb;
        }
        const Readback rb = *g->rb;
        if (rb.err & DERR_CAPACITY) fail(LF_ERR_CAPACITY, "membership row overflow (internal bound violated)");
        if (rb.err & DERR_CHECK) fail(LF_ERR_CUDA, "device consistency check failed (histogram partitioning)");
        iters = it;
        maxcnt = rb.maxcnt;
        last_live = rb.live_comms;
        last_memb = rb.memberships;
        if (stats && stats->history_cap >= it) {
            if (stats->wcc_history) stats->wcc_history[it - 1] = rb.total;
            if (stats->joins_history) stats->joins_history[it - 1] = (int64_t)rb.joins;
            if (stats->leaves_history) stats->leaves_history[it - 1] = (int64_t)rb.leaves;
        }
        const double T = rb.total;
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
        stats->prof_eval_launches = prof_launches;
        stats->prof_eval_ms = prof_ms;
        unsigned long long pbytes = 0;
        if (g->profile) {
            LF_CUDA(cudaMemcpy(&pbytes, &g->ds->prof_bytes, 8, cudaMemcpyDeviceToHost));
        }
        stats->prof_eval_bytes = (int64_t)pbytes;
    }
}

}  // namespace lf
