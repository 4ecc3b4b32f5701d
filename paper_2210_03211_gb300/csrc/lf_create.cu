// One-time preprocessing of a graph (Methods, Preprocessing; Methods, WCC;
// Heuristic Counting of Triangles):
//   a1  self-loop and multi-edge removal, dense relabel, symmetric CSR
//   a2  degree-ordered orientation N+(u)
//   a3  triangle counts t(x,V) and the marks of edges that lie on a triangle
//   a4  vt(x,V) from the edge marks
//   a5  local CC, node order (exact rational compare), global cc
#include <cstring>
#include <mutex>

#include <algorithm>

#include "lf_internal.cuh"

namespace lf {
namespace {

constexpr int TRI_WARP_MAX = 128;       // out-degree handled by one warp
constexpr int TRI_MID_MAX = 2048;       // out-degree handled by one 256-thread block
constexpr int TRI_MID_THREADS = 256;
constexpr int TRI_BLOCK_LIST = 16384;   // out-neighbour list held in shared memory by one big block
constexpr int TRI_BLOCK_THREADS = 1024;

// ---- a1 --------------------------------------------------------------------
__global__ void k_id_range(const int32_t *src, const int32_t *dst, int64_t E, DevScalars *ds,
                           unsigned long long *nonloops) {
    int32_t mx = -1, neg = 0;
    unsigned long long nl = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[e], b = dst[e];
        neg |= (a < 0) | (b < 0);
        if (a != b) {
            mx = max(mx, max(a, b));
            ++nl;
        }
    }
    mx = __reduce_max_sync(FULL, mx);
    neg = __reduce_or_sync(FULL, neg);
    unsigned long long nls = nl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nls += __shfl_down_sync(FULL, nls, o);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&ds->max_id, mx);
        if (neg) atomicOr(&ds->neg_id, 1);
        if (nls) atomicAdd(nonloops, nls);
    }
}

__global__ void k_mark_ids(const int32_t *src, const int32_t *dst, int64_t E, uint32_t *bm) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t a = (uint32_t)src[e], b = (uint32_t)dst[e];
        if (a == b) continue;
        atomicOr(&bm[a >> 5], 1u << (a & 31));
        atomicOr(&bm[b >> 5], 1u << (b & 31));
    }
}

__global__ void k_word_popc(const uint32_t *bm, int64_t nwords, uint32_t *cnt) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x)
        cnt[w] = __popc(bm[w]);
}

__global__ void k_labels(const uint32_t *bm, const uint32_t *wb, int64_t nwords, int32_t *labels) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = bm[w];
        uint32_t o = wb[w];
        while (b) {
            int bit = __ffs(b) - 1;
            labels[o++] = (int32_t)(w * 32 + bit);
            b &= b - 1;
        }
    }
}

__device__ __forceinline__ uint32_t id_rank(const uint32_t *bm, const uint32_t *wb, uint32_t id) {
    uint32_t w = id >> 5;
    return wb[w] + __popc(bm[w] & ((1u << (id & 31)) - 1u));
}

// Both directions of every non-loop pair as (row << 32 | col); the slot of a
// warp's keys comes from one atomic, so the output order is arbitrary -- the
// radix sort that follows fixes it.
__global__ void k_make_keys(const int32_t *src, const int32_t *dst, int64_t E, const uint32_t *bm,
                            const uint32_t *wb, unsigned long long *keys, unsigned long long *cursor) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < E; e0 += stride) {
        int64_t e = e0 + lane;
        bool ok = false;
        uint32_t ra = 0, rb = 0;
        if (e < E) {
            uint32_t a = (uint32_t)src[e], b = (uint32_t)dst[e];
            if (a != b) {
                ok = true;
                ra = id_rank(bm, wb, a);
                rb = id_rank(bm, wb, b);
            }
        }
        unsigned mask = __ballot_sync(FULL, ok);
        unsigned long long base = 0;
        if (lane == 0 && mask) base = atomicAdd(cursor, 2ull * __popc(mask));
        base = __shfl_sync(FULL, base, 0);
        if (ok) {
            unsigned long long p = base + 2ull * __popc(mask & lanemask_lt());
            keys[p] = ((unsigned long long)ra << 32) | rb;
            keys[p + 1] = ((unsigned long long)rb << 32) | ra;
        }
    }
}

__global__ void k_unique_flags(const unsigned long long *keys, int64_t count, uint32_t *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_unique_compact(const unsigned long long *keys, int64_t count, const uint32_t *flag,
                                 const uint32_t *idx, int32_t *adj, int64_t *off) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        unsigned long long k = keys[i];
        uint32_t j = idx[i];
        adj[j] = (int32_t)(k & 0xffffffffull);
        uint32_t row = (uint32_t)(k >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != row) off[row] = (int64_t)j;
    }
}

__global__ void k_degrees(const int64_t *off, int64_t n, int64_t total, int64_t *off_last, int32_t *deg,
                          DevScalars *ds) {
    int32_t mx = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        int64_t hi = (x + 1 < n) ? off[x + 1] : total;
        int32_t d = (int32_t)(hi - off[x]);
        deg[x] = d;
        mx = max(mx, d);
    }
    mx = __reduce_max_sync(FULL, mx);
    if ((threadIdx.x & 31) == 0) atomicMax(&ds->count32, mx);
    if (blockIdx.x == 0 && threadIdx.x == 0) *off_last = total;
}

// ---- a2 --------------------------------------------------------------------
__device__ __forceinline__ bool ranks_above(int32_t dv, int32_t v, int32_t du, int32_t u) {
    return dv > du || (dv == du && v > u);
}

__global__ void k_out_degree(const int64_t *off, const int32_t *adj, const int32_t *deg, int64_t n,
                             int64_t *odeg) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        int32_t du = deg[u];
        int cnt = 0;
        for (int64_t p = off[u] + lane; p < off[u + 1]; p += 32) {
            int32_t v = adj[p];
            cnt += ranks_above(deg[v], v, du, (int32_t)u);
        }
        cnt = __reduce_add_sync(FULL, cnt);
        if (lane == 0) odeg[u] = cnt;
    }
}

__global__ void k_orient_fill(const int64_t *off, const int32_t *adj, const int32_t *deg, int64_t n,
                              const int64_t *ooff, int32_t *oadj) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        int32_t du = deg[u];
        int64_t out = ooff[u];
        for (int64_t p0 = off[u]; p0 < off[u + 1]; p0 += 32) {
            int64_t p = p0 + lane;
            int32_t v = 0;
            bool keep = false;
            if (p < off[u + 1]) {
                v = adj[p];
                keep = ranks_above(deg[v], v, du, (int32_t)u);
            }
            unsigned mask = __ballot_sync(FULL, keep);
            if (keep) oadj[out + __popc(mask & lanemask_lt())] = v;
            out += __popc(mask);
        }
    }
}

// ---- a3 --------------------------------------------------------------------
__device__ __forceinline__ int find_sorted(const int32_t *list, int len, int32_t key) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int32_t v = list[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Triangles, credited without per-triangle global atomics.  For a node u,
// every w in N+(v) for v in N+(u) that is also in N+(u) closes the triangle
// (u, v, w) with rank u < v < w, met exactly once.  Credits: t[v] and t[w]
// through one counter per position of N+(u) (a single global atomic per
// position at the end), t[u] as their common total.  Edge marks: v->w when
// found, u->v and u->w from the counters.
//
// The work of a node is flattened: the lists N+(v) are laid end to end
// (prefix sums of their lengths in shared memory) and consumed 32 elements
// per lane group whatever the v boundaries, so short lists leave no lanes
// idle; each lane issues TRI_UNROLL independent loads before it uses any.
// Membership in N+(u) goes through a shared-memory hash table of the ids.

constexpr int TRI_UNROLL = 4;
constexpr int TW_HASH = 2 * TRI_WARP_MAX;   // slots of a warp's table (load <= 1/2)
constexpr int TM_HASH = 2 * TRI_MID_MAX;    // slots of a block's table

template <int HS, typename IdxT>
__device__ __forceinline__ int tri_lookup(const int32_t *hk, const IdxT *hp, int32_t w) {
    uint32_t h = hash32((uint32_t)w) & (HS - 1);
    for (int probe = 0; probe < HS; ++probe) {
        const int32_t k = hk[h];
        if (k == w) return (int)hp[h];
        if (k == -1) return -1;
        h = (h + 1) & (HS - 1);
    }
    return -1;
}

template <int HS, typename IdxT>
__device__ __forceinline__ void tri_insert(int32_t *hk, IdxT *hp, int32_t v, int k) {
    uint32_t h = hash32((uint32_t)v) & (HS - 1);
    while (atomicCAS(&hk[h], -1, v) != -1) h = (h + 1) & (HS - 1);
    hp[h] = (IdxT)k;
}

// Elements [e_begin, e_end) of a node's flattened stream, walked by one warp
// from position p (pre[p] <= e_begin).  Returns this lane's triangle count.
template <int HS, typename IdxT>
__device__ __forceinline__ int tri_stream(int e_begin, int e_end, int p, const int32_t *pre, const long long *base,
                                          const int32_t *__restrict__ oadj, int32_t lo_id, int32_t hi_id,
                                          const int32_t *hk, const IdxT *hp, int *cnt, uint8_t *sup, int lane) {
    int tu = 0;
    for (int e0 = e_begin; e0 < e_end; e0 += 32 * TRI_UNROLL) {
        int pp[TRI_UNROLL];
        long long at[TRI_UNROLL];
        int32_t x[TRI_UNROLL];
#pragma unroll
        for (int j = 0; j < TRI_UNROLL; ++j) {
            const int e = e0 + j * 32 + lane;
            pp[j] = -1;
            at[j] = 0;
            x[j] = 0;
            if (e < e_end) {
                while (pre[p + 1] <= e) ++p;
                at[j] = base[p] + (e - pre[p]);
                pp[j] = p;
                x[j] = oadj[at[j]];
            }
        }
#pragma unroll
        for (int j = 0; j < TRI_UNROLL; ++j) {
            if (pp[j] >= 0 && x[j] >= lo_id && x[j] <= hi_id) {
                const int idx = tri_lookup<HS, IdxT>(hk, hp, x[j]);
                if (idx >= 0) {
                    atomicAdd(&cnt[idx], 1);
                    atomicAdd(&cnt[pp[j]], 1);
                    sup[at[j]] = 1;
                    ++tu;
                }
            }
        }
        p = __shfl_sync(FULL, p, 31);   // lane 31 holds the furthest position
    }
    return tu;
}

// One warp per node u with 2 <= d+(u) <= TRI_WARP_MAX.
__global__ void __launch_bounds__(256) k_tri_warp(const int64_t *ooff, const int32_t *__restrict__ oadj, int64_t n,
                                                  unsigned long long *tri, uint8_t *sup, DevScalars *ds) {
    __shared__ long long s_base[8][TRI_WARP_MAX];
    __shared__ int32_t s_list[8][TRI_WARP_MAX];
    __shared__ int32_t s_pre[8][TRI_WARP_MAX + 1];
    __shared__ int32_t s_cnt[8][TRI_WARP_MAX];
    __shared__ int32_t s_hk[8][TW_HASH];
    __shared__ uint8_t s_hp[8][TW_HASH];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *list = s_list[w], *pre = s_pre[w], *cnt = s_cnt[w], *hk = s_hk[w];
    long long *base = s_base[w];
    uint8_t *hp = s_hp[w];
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long found = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t s = ooff[u];
        const int du = (int)(ooff[u + 1] - s);
        if (du < 2 || du > TRI_WARP_MAX) continue;
        for (int k = lane; k < TW_HASH; k += 32) hk[k] = -1;
        int carry = 0;
        for (int k0 = 0; k0 < du; k0 += 32) {
            const int k = k0 + lane;
            int len = 0;
            if (k < du) {
                const int32_t v = oadj[s + k];
                const int64_t b = ooff[v];
                list[k] = v;
                base[k] = b;
                len = (int)(ooff[v + 1] - b);
                cnt[k] = 0;
            }
            int x = len;   // inclusive warp scan of the lengths
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            if (k < du) pre[k + 1] = carry + x;
            carry += __shfl_sync(FULL, x, 31);
        }
        if (lane == 0) pre[0] = 0;
        __syncwarp();
        for (int k = lane; k < du; k += 32) tri_insert<TW_HASH, uint8_t>(hk, hp, list[k], k);
        __syncwarp();
        int tu = tri_stream<TW_HASH, uint8_t>(0, pre[du], 0, pre, base, oadj, list[0], list[du - 1], hk, hp, cnt,
                                              sup, lane);
        __syncwarp();
        for (int k = lane; k < du; k += 32) {
            const int c = cnt[k];
            if (c > 0) {
                atomicAdd(&tri[list[k]], (unsigned long long)c);
                sup[s + k] = 1;
            }
        }
        tu = __reduce_add_sync(FULL, tu);
        if (lane == 0 && tu > 0) atomicAdd(&tri[u], (unsigned long long)tu);
        found += (unsigned long long)tu;
        __syncwarp();
    }
    if (lane == 0 && found) atomicAdd(&ds->num_tri, found);
}

// One 256-thread block per node with TRI_WARP_MAX < d+(u) <= TRI_MID_MAX: the
// stream is cut into one contiguous range per warp.
__global__ void __launch_bounds__(TRI_MID_THREADS) k_tri_mid(const int64_t *ooff, const int32_t *__restrict__ oadj,
                                                             const int32_t *mids, const uint32_t *nmid,
                                                             unsigned long long *tri, uint8_t *sup, DevScalars *ds) {
    extern __shared__ long long mid_dyn[];
    long long *base = mid_dyn;                                            // TRI_MID_MAX
    int32_t *hk = reinterpret_cast<int32_t *>(mid_dyn + TRI_MID_MAX);     // TM_HASH
    int32_t *list = hk + TM_HASH;                                         // TRI_MID_MAX
    int32_t *pre = list + TRI_MID_MAX;                                    // TRI_MID_MAX + 1
    int32_t *cnt = pre + TRI_MID_MAX + 1;                                 // TRI_MID_MAX
    uint16_t *hp = reinterpret_cast<uint16_t *>(cnt + TRI_MID_MAX);       // TM_HASH
    __shared__ int32_t s_part[TRI_MID_THREADS / 32];
    __shared__ unsigned long long s_tu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = TRI_MID_THREADS / 32;
    constexpr int PER = TRI_MID_MAX / TRI_MID_THREADS;
    for (uint32_t h = blockIdx.x; h < *nmid; h += gridDim.x) {
        const int32_t u = mids[h];
        const int64_t s = ooff[u];
        const int du = (int)(ooff[u + 1] - s);
        if (threadIdx.x == 0) s_tu = 0;
        for (int k = threadIdx.x; k < TM_HASH; k += TRI_MID_THREADS) hk[k] = -1;
        // lengths: thread t owns entries t*PER .. t*PER+PER-1, then a block scan
        int lens[PER];
        int sum = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int k = threadIdx.x * PER + j;
            lens[j] = 0;
            if (k < du) {
                const int32_t v = oadj[s + k];
                const int64_t b = ooff[v];
                list[k] = v;
                base[k] = b;
                lens[j] = (int)(ooff[v + 1] - b);
                cnt[k] = 0;
            }
            sum += lens[j];
        }
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_part[w] = x;
        __syncthreads();
        int run = x - sum;
        for (int k = 0; k < w; ++k) run += s_part[k];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int k = threadIdx.x * PER + j;
            if (k < du) pre[k] = run;
            run += lens[j];
        }
        if (threadIdx.x == TRI_MID_THREADS - 1) pre[du] = run;
        for (int k = threadIdx.x; k < du; k += TRI_MID_THREADS) tri_insert<TM_HASH, uint16_t>(hk, hp, list[k], k);
        __syncthreads();
        const int total = pre[du];
        const int eb = (int)((long long)total * w / NW), ee = (int)((long long)total * (w + 1) / NW);
        int tu = 0;
        if (eb < ee) {
            // first position whose range holds eb (pre is ascending, pre[du] > eb)
            int lo = 0, hi = du - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (pre[mid + 1] <= eb) lo = mid + 1; else hi = mid;
            }
            tu = tri_stream<TM_HASH, uint16_t>(eb, ee, lo, pre, base, oadj, list[0], list[du - 1], hk, hp, cnt, sup,
                                               lane);
        }
        tu = __reduce_add_sync(FULL, tu);
        if (lane == 0 && tu) atomicAdd(&s_tu, (unsigned long long)tu);
        __syncthreads();
        for (int k = threadIdx.x; k < du; k += TRI_MID_THREADS) {
            const int c = cnt[k];
            if (c > 0) {
                atomicAdd(&tri[list[k]], (unsigned long long)c);
                sup[s + k] = 1;
            }
        }
        if (threadIdx.x == 0 && s_tu) {
            atomicAdd(&tri[u], s_tu);
            atomicAdd(&ds->num_tri, s_tu);
        }
        __syncthreads();
    }
}

constexpr size_t TRI_MID_SMEM = (size_t)TRI_MID_MAX * 8 + (size_t)TM_HASH * 4 + (size_t)(3 * TRI_MID_MAX + 1) * 4 +
                                (size_t)TM_HASH * 2;

// One block per node with d+(u) > TRI_MID_MAX; warps take the v's.  When the
// list does not fit in shared memory, the look-ups go to global memory and
// the credits are made per triangle.
__global__ void __launch_bounds__(TRI_BLOCK_THREADS) k_tri_block(const int64_t *ooff, const int32_t *oadj,
                                                                 const int32_t *bigs_end, const uint32_t *nbig,
                                                                 unsigned long long *tri, uint8_t *sup,
                                                                 DevScalars *ds) {
    extern __shared__ int32_t dyn[];
    __shared__ unsigned long long s_tu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t h = blockIdx.x; h < *nbig; h += gridDim.x) {
        const int32_t u = bigs_end[-1 - (int64_t)h];
        const int64_t s = ooff[u];
        const int du = (int)(ooff[u + 1] - s);
        const bool in_smem = du <= TRI_BLOCK_LIST;
        int32_t *list = dyn;
        int32_t *top = dyn + TRI_BLOCK_LIST;
        uint8_t *mid = reinterpret_cast<uint8_t *>(dyn + 2 * TRI_BLOCK_LIST);
        if (threadIdx.x == 0) s_tu = 0;
        if (in_smem)
            for (int i = threadIdx.x; i < du; i += blockDim.x) {
                list[i] = oadj[s + i];
                top[i] = 0;
                mid[i] = 0;
            }
        __syncthreads();
        const int32_t *L = in_smem ? list : oadj + s;
        const int32_t lo_id = L[0], hi_id = L[du - 1];
        unsigned long long tu = 0;
        for (int p = w; p < du; p += nw) {
            const int32_t v = L[p];
            const int64_t sv = ooff[v];
            const int dv = (int)(ooff[v + 1] - sv);
            int c = 0;
            for (int j = lane; j < dv; j += 32) {
                int32_t x = oadj[sv + j];
                if (x < lo_id || x > hi_id) continue;
                int idx = find_sorted(L, du, x);
                if (idx >= 0) {
                    sup[sv + j] = 1;
                    ++c;
                    if (in_smem) {
                        atomicAdd(&top[idx], 1);
                    } else {
                        atomicAdd(&tri[x], 1ull);
                        sup[s + idx] = 1;
                    }
                }
            }
            c = __reduce_add_sync(FULL, c);
            if (c > 0 && lane == 0) {
                atomicAdd(&tri[v], (unsigned long long)c);
                if (in_smem) mid[p] = 1; else sup[s + p] = 1;
            }
            tu += (unsigned long long)c;
        }
        if (lane == 0 && tu) atomicAdd(&s_tu, tu);
        __syncthreads();
        if (in_smem)
            for (int i = threadIdx.x; i < du; i += blockDim.x) {
                int cnt = top[i];
                if (cnt > 0) atomicAdd(&tri[list[i]], (unsigned long long)cnt);
                if (cnt > 0 || mid[i]) sup[s + i] = 1;
            }
        if (threadIdx.x == 0 && s_tu) {
            atomicAdd(&tri[u], s_tu);
            atomicAdd(&ds->num_tri, s_tu);
        }
        __syncthreads();
    }
}

// Nodes for the block kernels: mid-size ones from the front of `hubs`
// (count nh[0]), big ones from the back (count nh[1]); n entries hold both.
__global__ void k_select_hubs(const int64_t *ooff, int64_t n, int32_t *hubs, uint32_t *nh) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t du = ooff[u + 1] - ooff[u];
        if (du > TRI_MID_MAX) hubs[n - 1 - atomicAdd(&nh[1], 1u)] = (int32_t)u;
        else if (du > TRI_WARP_MAX) hubs[atomicAdd(&nh[0], 1u)] = (int32_t)u;
    }
}

constexpr size_t TRI_BIG_SMEM = (size_t)TRI_BLOCK_LIST * 9;

void set_triangle_attrs() {
    LF_CUDA(cudaFuncSetAttribute(k_tri_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRI_BIG_SMEM));
    LF_CUDA(cudaFuncSetAttribute(k_tri_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRI_MID_SMEM));
}

// Triangle counts and support marks of an oriented graph with n > 0 nodes.
// `hubs` holds n ints of scratch and `nh` two counters that start at zero.
// Returns the number of kernels launched.
int launch_triangles(const int64_t *ooff, const int32_t *oadj, int64_t n, int32_t *hubs, uint32_t *nh,
                     unsigned long long *tri, uint8_t *sup, DevScalars *ds, cudaStream_t st) {
    const int sms = 152;
    k_select_hubs<<<grid_for(n, 256, 8192), 256, 0, st>>>(ooff, n, hubs, nh);
    LF_LAUNCHED();
    k_tri_warp<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(ooff, oadj, n, tri, sup, ds);
    LF_LAUNCHED();
    k_tri_mid<<<sms * 8, TRI_MID_THREADS, TRI_MID_SMEM, st>>>(ooff, oadj, hubs, nh, tri, sup, ds);
    LF_LAUNCHED();
    k_tri_block<<<2 * sms, TRI_BLOCK_THREADS, TRI_BIG_SMEM, st>>>(ooff, oadj, hubs + n, nh + 1, tri, sup, ds);
    LF_LAUNCHED();
    return 4;
}


// ---- a3, main path: triangles by their middle vertex ------------------------
// A triangle u < v < w (rank order) is found at v: for every in-neighbour u of
// v (u -> v), the list N+(u) is streamed and each w in it probed against
// N+(v).  The elements read are sum over u of d+(u)^2, against sum over v of
// d-(v) d+(v) when triangles are found at u, several times fewer on
// power-law graphs, whose middle-rank nodes have long out-lists.
// Credits of a triangle (u, v, w): t[w] and the mark v->w through one counter
// per position of N+(v); t[u] and the mark u->v through one counter per
// in-neighbour; t[v] as the common total; the mark u->w where w is met.
// The streams of all in-neighbours are laid end to end, as above.
//
// Most stream elements are not in N+(v).  Each is first tested against a
// one-bit-per-slot filter of N+(v) (one shared load); the few that pass are
// queued per warp and looked up 32 at a time in the exact set, so the costly
// path runs on full warps.

constexpr int TV_WARP_DPLUS = 128;   // |N+(v)| hashed by one warp
constexpr int TV_WARP_DEG = 1024;    // deg(v) walked by one warp
constexpr int TV_ROUND = 64;         // entries of N(v) compacted per warp round
constexpr int TV_ITEM = 512;         // entries of N(v) per block item
constexpr int TV_BLOCK_DPLUS = 1024; // |N+(v)| hashed by one block
constexpr int TV_THREADS = 256;
constexpr int TV_WHASH = 2 * TV_WARP_DPLUS;   // slots: buckets of four ids, at most half full
constexpr int TV_BHASH = 2 * TV_BLOCK_DPLUS;
constexpr int TV_WBITS_LOG = 11;     // filter bits per warp table (>= 16 per id)
constexpr int TV_BBITS_LOG = 14;     // filter bits per block table
constexpr int TV_QUEUE = 64;         // queued candidates per warp

__device__ __forceinline__ uint32_t tv_mix(int32_t w) { return (uint32_t)w * 0x9E3779B1u; }   // Knuth

// Set of ids with their positions: buckets of four slots read as one 16-byte
// shared load, multiplicative hashing on the bucket index, linear probing
// over buckets.  At most half full, so a lookup nearly always reads one
// bucket.
template <int SLOTS, typename IdxT>
struct TvBuckets {
    static constexpr int NB = SLOTS / 4;
    static constexpr int SHIFT = 32 - __builtin_ctz(NB);
    int32_t *hk;   // SLOTS ids, -1 = empty; 16-byte aligned
    IdxT *hp;      // SLOTS positions
    __device__ __forceinline__ static uint32_t bucket(int32_t w) { return tv_mix(w) >> SHIFT; }
    __device__ __forceinline__ void insert(int32_t v, int k) const {
        uint32_t b = bucket(v);
        for (;;) {
#pragma unroll
            for (int sl = 0; sl < 4; ++sl)
                if (atomicCAS(&hk[4 * b + sl], -1, v) == -1) {
                    hp[4 * b + sl] = (IdxT)k;
                    return;
                }
            b = (b + 1) & (NB - 1);
        }
    }
    __device__ __forceinline__ int find(int32_t w) const {
        uint32_t b = bucket(w);
        for (int probe = 0; probe < NB; ++probe) {
            const int4 q = reinterpret_cast<const int4 *>(hk)[b];
            const int sl = q.x == w ? 0 : q.y == w ? 1 : q.z == w ? 2 : q.w == w ? 3 : -1;
            if (sl >= 0) return (int)hp[4 * b + sl];
            if (q.w == -1) return -1;   // slots fill in order, so a free last slot ends the chain
            b = (b + 1) & (NB - 1);
        }
        return -1;
    }
};
using TvHash8 = TvBuckets<TV_WHASH, uint8_t>;
using TvHash16 = TvBuckets<TV_BHASH, uint16_t>;

struct TvSorted {  // N+(v) as a sorted list, in shared or global memory
    const int32_t *list;
    int len;
    __device__ __forceinline__ int find(int32_t w) const {
        int lo = 0, hi = len - 1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int32_t x = list[mid];
            if (x == w) return mid;
            if (x < w) lo = mid + 1; else hi = mid - 1;
        }
        return -1;
    }
};

template <int LOGB>
__device__ __forceinline__ void tv_filter_add(uint32_t *bits, int32_t w) {
    const uint32_t h = tv_mix(w) >> (32 - LOGB);
    atomicOr(&bits[h >> 5], 1u << (h & 31));
}

template <int LOGB>
__device__ __forceinline__ bool tv_filter_has(const uint32_t *bits, int32_t w) {
    const uint32_t h = tv_mix(w) >> (32 - LOGB);
    return (bits[h >> 5] >> (h & 31)) & 1u;
}

// Shared arrays of one round: compacted in-neighbours u; ooff[u], turned into
// ooff[u] - pre[u] once the prefix sums pre of d+(u) are known, so that stream
// element e of position p sits at oadj[shift[p] + e]; triangles per u; and the
// stream index at which v appears in N+(u).
template <typename Idx>
struct TvRound {
    int32_t *ul;
    Idx *shift;   // int32_t when the oriented CSR has fewer than 2^31 entries
    int32_t *pre;
    int32_t *hits;
    int32_t *vrel;
};

struct TvQueue {   // one warp's candidates: id, stream index, position
    int32_t *x;
    int32_t *e;
    int32_t *p;
};

// Elements [e_begin, e_end) of a round's stream, walked by one warp from
// position p (pre[p] <= e_begin).  LOCAL: per-position counters of N+(v) in
// `cnt`; otherwise t[w] and the mark v->w are written directly.  Returns this
// lane's triangle count.
template <bool LOCAL, int LOGB, typename Idx, typename Set>
__device__ __forceinline__ int tv_stream(int e_begin, int e_end, int p, const TvRound<Idx> &r,
                                         const int32_t *__restrict__ oadj, int32_t v, int64_t vs,
                                         const uint32_t *bits, const Set &set, const TvQueue &q, int *cnt,
                                         unsigned long long *tri, uint8_t *sup, int lane) {
    int tv = 0, qn = 0;
    const unsigned lt = lanemask_lt();
    // lanes below `count` take the last `count` queue entries
    auto drain = [&](int count) {
        __syncwarp();
        if (lane < count) {
            const int k = qn - count + lane;
            const int32_t x = q.x[k];
            const int pp = q.p[k];
            const int idx = set.find(x);
            if (idx >= 0) {
                if (LOCAL) {
                    atomicAdd(&cnt[idx], 1);
                } else {
                    atomicAdd(&tri[x], 1ull);
                    sup[vs + idx] = 1;
                }
                atomicAdd(&r.hits[pp], 1);
                sup[r.shift[pp] + (Idx)q.e[k]] = 1;
                ++tv;
            }
        }
        qn -= count;
        __syncwarp();
    };
    for (int e0 = e_begin; e0 < e_end; e0 += 32 * TRI_UNROLL) {
        int pp[TRI_UNROLL];
        int32_t x[TRI_UNROLL];
        if (e0 + 32 * TRI_UNROLL <= e_end) {   // full steps: no bound checks
#pragma unroll
            for (int j = 0; j < TRI_UNROLL; ++j) {
                const int e = e0 + j * 32 + lane;
                while (r.pre[p + 1] <= e) ++p;
                pp[j] = p;
                x[j] = oadj[r.shift[p] + (Idx)e];
            }
        } else {
#pragma unroll
            for (int j = 0; j < TRI_UNROLL; ++j) {
                const int e = e0 + j * 32 + lane;
                pp[j] = -1;
                x[j] = 0;
                if (e < e_end) {
                    while (r.pre[p + 1] <= e) ++p;
                    pp[j] = p;
                    x[j] = oadj[r.shift[p] + (Idx)e];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TRI_UNROLL; ++j) {
            const int e = e0 + j * 32 + lane;
            bool cand = false;
            if (pp[j] >= 0) {
                if (x[j] == v) r.vrel[pp[j]] = e;
                cand = tv_filter_has<LOGB>(bits, x[j]);
            }
            const unsigned m = __ballot_sync(FULL, cand);
            if (cand) {
                const int k = qn + __popc(m & lt);
                q.x[k] = x[j];
                q.e[k] = e;
                q.p[k] = pp[j];
            }
            qn += __popc(m);
            if (qn >= 32) drain(32);
        }
        p = __shfl_sync(FULL, p, 31);   // lane 31 holds the furthest position
    }
    if (qn > 0) drain(qn);
    __syncwarp();   // every vrel and hits write seen by the warp's readers
    return tv;
}

// The in-neighbours u of v with d+(u) >= 2 among C entries of N(v) a lane
// holds (entries j0 + c * 32): loads first, then the warp ballots.  Returns
// the entries kept by this warp (written from slot `at` on); lengths go to
// pre[slot + 1].
template <int C, typename Idx>
__device__ __forceinline__ int tv_compact(const int32_t *adj, const int32_t *deg, const int64_t *ooff, int64_t as,
                                          int j0, int jend, int32_t dv, int32_t v, int at, const TvRound<Idx> &r,
                                          int lane) {
    int32_t u[C], du[C];
    long long b[C];
    int len[C];
    bool keep[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int j = j0 + c * 32;
        u[c] = j < jend ? adj[as + j] : -1;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) du[c] = u[c] >= 0 ? deg[u[c]] : 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        b[c] = 0;
        len[c] = 0;
        if (u[c] >= 0 && ranks_above(dv, v, du[c], u[c])) {
            b[c] = ooff[u[c]];
            len[c] = (int)(ooff[u[c] + 1] - b[c]);
        }
        keep[c] = len[c] >= 2;
    }
    int kept = 0;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const unsigned mask = __ballot_sync(FULL, keep[c]);
        if (keep[c]) {
            const int slot = at + kept + __popc(mask & lt);
            r.ul[slot] = u[c];
            r.shift[slot] = (Idx)b[c];
            r.pre[slot + 1] = len[c];
            r.hits[slot] = 0;
        }
        kept += __popc(mask);
    }
    return kept;
}

// One warp per node v with 1 <= d+(v) <= TV_WARP_DPLUS and deg(v) <= TV_WARP_DEG.
// A resident grid; each warp takes runs of TV_WARP_BATCH node ids from a
// counter, so that a block is not held by one long node while its other warps
// idle.
constexpr int TV_WARP_BATCH = 64;

template <typename Idx>
__global__ void __launch_bounds__(256, 5) k_tv_warp(const int64_t *off, const int32_t *adj, const int32_t *deg,
                                                    const int64_t *ooff, const int32_t *__restrict__ oadj,
                                                    int64_t n, uint32_t *next, unsigned long long *tri, uint8_t *sup,
                                                    DevScalars *ds) {
    __shared__ Idx s_shift[8][TV_ROUND];
    __shared__ int32_t s_ul[8][TV_ROUND];
    __shared__ int32_t s_pre[8][TV_ROUND + 1];
    __shared__ int32_t s_hits[8][TV_ROUND];
    __shared__ int32_t s_vrel[8][TV_ROUND];
    __shared__ int32_t s_cnt[8][TV_WARP_DPLUS];
    __shared__ __align__(16) int32_t s_hk[8][TV_WHASH];
    __shared__ uint8_t s_hp[8][TV_WHASH];
    __shared__ uint32_t s_bits[8][(1 << TV_WBITS_LOG) / 32];
    __shared__ int32_t s_q[8][3][TV_QUEUE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TvRound<Idx> r{s_ul[w], s_shift[w], s_pre[w], s_hits[w], s_vrel[w]};
    const TvQueue q{s_q[w][0], s_q[w][1], s_q[w][2]};
    int32_t *cnt = s_cnt[w], *hk = s_hk[w];
    uint32_t *bits = s_bits[w];
    const TvHash8 set{hk, s_hp[w]};
    unsigned long long found = 0;
    int64_t vv = 0, vend = 0;
    for (;;) {
        if (vv == vend) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = (unsigned long long)atomicAdd(next, 1u) * TV_WARP_BATCH;
            b0 = __shfl_sync(FULL, b0, 0);
            if ((int64_t)b0 >= n) break;
            vv = (int64_t)b0;
            vend = min(n, vv + TV_WARP_BATCH);
        }
        const int32_t v = (int32_t)(vv++);
        const int64_t vs = ooff[v];
        const int dpv = (int)(ooff[v + 1] - vs);
        const int64_t as = off[v];
        const int dv = (int)(off[v + 1] - as);
        if (dpv < 1 || dpv > TV_WARP_DPLUS || dv > TV_WARP_DEG || dv == dpv) continue;
        for (int k = lane; k < TV_WHASH; k += 32) hk[k] = -1;
        for (int k = lane; k < (1 << TV_WBITS_LOG) / 32; k += 32) bits[k] = 0;
        __syncwarp();
        for (int k = lane; k < dpv; k += 32) {
            const int32_t x = oadj[vs + k];
            set.insert(x, k);
            tv_filter_add<TV_WBITS_LOG>(bits, x);
            cnt[k] = 0;
        }
        int tv = 0;
        for (int r0 = 0; r0 < dv; r0 += TV_ROUND) {
            const int nk = tv_compact<TV_ROUND / 32>(adj, deg, ooff, as, r0 + lane, min(dv, r0 + TV_ROUND), dv, v, 0,
                                                     r, lane);
            if (nk == 0) continue;
            __syncwarp();
            int carry = 0;
            for (int k0 = 0; k0 < nk; k0 += 32) {   // prefix sums of the lengths, in place
                const int k = k0 + lane;
                int x = k < nk ? r.pre[k + 1] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += y;
                }
                if (k < nk) r.pre[k + 1] = carry + x;
                carry += __shfl_sync(FULL, x, 31);
            }
            if (lane == 0) r.pre[0] = 0;
            __syncwarp();
            for (int k = lane; k < nk; k += 32) r.shift[k] -= (Idx)r.pre[k];
            __syncwarp();
            tv += tv_stream<true, TV_WBITS_LOG>(0, r.pre[nk], 0, r, oadj, v, vs, bits, set, q, cnt, tri, sup, lane);
            for (int k = lane; k < nk; k += 32) {
                const int h = r.hits[k];
                if (h > 0) {
                    atomicAdd(&tri[r.ul[k]], (unsigned long long)h);
                    sup[r.shift[k] + (Idx)r.vrel[k]] = 1;
                }
            }
            __syncwarp();
        }
        for (int k = lane; k < dpv; k += 32) {
            const int c = cnt[k];
            if (c > 0) {
                atomicAdd(&tri[oadj[vs + k]], (unsigned long long)c);
                sup[vs + k] = 1;
            }
        }
        tv = __reduce_add_sync(FULL, tv);
        if (lane == 0 && tv > 0) atomicAdd(&tri[v], (unsigned long long)tv);
        found += (unsigned long long)tv;
        __syncwarp();
    }
    if (lane == 0 && found) atomicAdd(&ds->num_tri, found);
}

// Block items: (v, a run of TV_ITEM entries of N(v)), for the nodes the warp
// kernel leaves.  BIG = false: |N+(v)| <= TV_BLOCK_DPLUS, hashed, counters in
// shared memory.  BIG = true: N+(v) sorted in shared memory (global beyond
// TRI_BLOCK_LIST ids), t[w] and v->w written per triangle.  Items are taken
// from a counter, so long and short ones balance across the blocks.
constexpr int TV_NW = TV_THREADS / 32;
constexpr size_t tv_round_smem(size_t idx_bytes) {
    return (size_t)TV_ITEM * idx_bytes + (size_t)(4 * TV_ITEM + 4) * 4 + (size_t)TV_NW * 3 * TV_QUEUE * 4 +
           ((size_t)1 << TV_BBITS_LOG) / 8;
}
constexpr size_t tv_items_smem(bool big, size_t idx_bytes) {
    return tv_round_smem(idx_bytes) +
           (big ? (size_t)TRI_BLOCK_LIST * 4 : (size_t)TV_BHASH * 6 + (size_t)TV_BLOCK_DPLUS * 4);
}

template <bool BIG, typename Idx>
__global__ void __launch_bounds__(TV_THREADS) k_tv_items(const int64_t *off, const int32_t *adj, const int32_t *deg,
                                                         const int64_t *ooff, const int32_t *__restrict__ oadj,
                                                         const unsigned long long *items, const uint32_t *nitems,
                                                         uint32_t *next, unsigned long long *tri, uint8_t *sup,
                                                         DevScalars *ds) {
    extern __shared__ int4 tv_dyn[];
    Idx *shift = reinterpret_cast<Idx *>(tv_dyn);                            // TV_ITEM
    int32_t *ul = reinterpret_cast<int32_t *>(shift + TV_ITEM);             // TV_ITEM
    int32_t *pre = ul + TV_ITEM;                                             // TV_ITEM + 1 (+3 padding)
    int32_t *hits = pre + TV_ITEM + 4;                                       // TV_ITEM
    int32_t *vrel = hits + TV_ITEM;                                          // TV_ITEM
    int32_t *qbuf = vrel + TV_ITEM;                                          // TV_NW * 3 * TV_QUEUE
    uint32_t *bits = reinterpret_cast<uint32_t *>(qbuf + TV_NW * 3 * TV_QUEUE);   // 2^TV_BBITS_LOG bits
    int32_t *hk = reinterpret_cast<int32_t *>(bits + (1 << TV_BBITS_LOG) / 32);  // TV_BHASH, 16-byte aligned
    int32_t *cnt = hk + TV_BHASH;                                            // TV_BLOCK_DPLUS
    uint16_t *hp = reinterpret_cast<uint16_t *>(cnt + TV_BLOCK_DPLUS);      // TV_BHASH
    int32_t *slist = hk;                                                     // BIG: TRI_BLOCK_LIST ids
    __shared__ int32_t s_part[TV_NW];
    __shared__ uint32_t s_item;
    __shared__ unsigned long long s_tv;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TvRound<Idx> r{ul, shift, pre, hits, vrel};
    const TvQueue q{qbuf + w * 3 * TV_QUEUE, qbuf + w * 3 * TV_QUEUE + TV_QUEUE, qbuf + w * 3 * TV_QUEUE + 2 * TV_QUEUE};
    const uint32_t count = *nitems;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(next, 1u);
            s_tv = 0;
        }
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= count) break;
        const unsigned long long item = BIG ? items[-1 - (int64_t)it] : items[it];
        const int32_t v = (int32_t)(item >> 32);
        const int chunk = (int)(item & 0xffffffffu);
        const int64_t vs = ooff[v];
        const int dpv = (int)(ooff[v + 1] - vs);
        const int64_t as = off[v];
        const int dv = (int)(off[v + 1] - as);
        const int32_t *glist = oadj + vs;
        // membership structures of N+(v): the filter, and the exact set
        for (int k = threadIdx.x; k < (1 << TV_BBITS_LOG) / 32; k += TV_THREADS) bits[k] = 0;
        if (!BIG)
            for (int k = threadIdx.x; k < TV_BHASH; k += TV_THREADS) hk[k] = -1;
        __syncthreads();
        for (int k = threadIdx.x; k < dpv; k += TV_THREADS) {
            const int32_t x = glist[k];
            tv_filter_add<TV_BBITS_LOG>(bits, x);
            if (!BIG) {
                TvHash16{hk, hp}.insert(x, k);
                cnt[k] = 0;
            } else if (dpv <= TRI_BLOCK_LIST) {
                slist[k] = x;
            }
        }
        // compaction of this item's in-neighbours: each warp takes a run of
        // TV_ITEM / TV_NW entries
        constexpr int RUN = TV_ITEM / TV_NW;
        const int j0 = chunk * TV_ITEM + w * RUN;
        const int jend = min(dv, chunk * TV_ITEM + TV_ITEM);
        {
            // count first, so that the warps' slots can be placed
            int32_t u[RUN / 32];
            bool keep[RUN / 32];
            long long b[RUN / 32];
            int len[RUN / 32];
            int wk = 0;
#pragma unroll
            for (int c = 0; c < RUN / 32; ++c) {
                const int j = j0 + c * 32 + lane;
                u[c] = j < jend ? adj[as + j] : -1;
            }
#pragma unroll
            for (int c = 0; c < RUN / 32; ++c) {
                keep[c] = false;
                b[c] = 0;
                len[c] = 0;
                if (u[c] >= 0 && ranks_above(dv, v, deg[u[c]], u[c])) {
                    b[c] = ooff[u[c]];
                    len[c] = (int)(ooff[u[c] + 1] - b[c]);
                    keep[c] = len[c] >= 2;
                }
                wk += __popc(__ballot_sync(FULL, keep[c]));
            }
            if (lane == 0) s_part[w] = wk;
            __syncthreads();
            int at = 0;
            for (int k = 0; k < w; ++k) at += s_part[k];
            const unsigned lt = lanemask_lt();
#pragma unroll
            for (int c = 0; c < RUN / 32; ++c) {
                const unsigned mask = __ballot_sync(FULL, keep[c]);
                if (keep[c]) {
                    const int slot = at + __popc(mask & lt);
                    ul[slot] = u[c];
                    shift[slot] = (Idx)b[c];
                    pre[slot + 1] = len[c];
                    hits[slot] = 0;
                }
                at += __popc(mask);
            }
        }
        int nk = 0;
        for (int k = 0; k < TV_NW; ++k) nk += s_part[k];
        __syncthreads();
        if (nk > 0) {
            // prefix sums of the lengths: thread t owns entries PER t .. PER t + PER - 1
            constexpr int PER = TV_ITEM / TV_THREADS;
            int lens[PER];
            int sum = 0;
#pragma unroll
            for (int c = 0; c < PER; ++c) {
                const int k = threadIdx.x * PER + c;
                lens[c] = k < nk ? pre[k + 1] : 0;
                sum += lens[c];
            }
            int x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            __syncthreads();   // every length read before any prefix is written
            if (lane == 31) s_part[w] = x;
            __syncthreads();
            int run = x - sum;
            for (int k = 0; k < w; ++k) run += s_part[k];
#pragma unroll
            for (int c = 0; c < PER; ++c) {
                const int k = threadIdx.x * PER + c;
                if (k < nk) pre[k] = run;
                run += lens[c];
            }
            if (threadIdx.x == TV_THREADS - 1) pre[nk] = run;
            __syncthreads();
            for (int k = threadIdx.x; k < nk; k += TV_THREADS) shift[k] -= (Idx)pre[k];
            __syncthreads();
            const int total = pre[nk];
            const int eb = (int)((long long)total * w / TV_NW), ee = (int)((long long)total * (w + 1) / TV_NW);
            int tv = 0;
            if (eb < ee) {
                int lo = 0, hi = nk - 1;   // first position whose range holds eb
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[mid + 1] <= eb) lo = mid + 1; else hi = mid;
                }
                if (!BIG)
                    tv = tv_stream<true, TV_BBITS_LOG>(eb, ee, lo, r, oadj, v, vs, bits, TvHash16{hk, hp}, q, cnt,
                                                       tri, sup, lane);
                else
                    tv = tv_stream<false, TV_BBITS_LOG>(eb, ee, lo, r, oadj, v, vs, bits,
                                                        TvSorted{dpv <= TRI_BLOCK_LIST ? slist : glist, dpv}, q, cnt,
                                                        tri, sup, lane);
            }
            tv = __reduce_add_sync(FULL, tv);
            if (lane == 0 && tv) atomicAdd(&s_tv, (unsigned long long)tv);
            __syncthreads();
            for (int k = threadIdx.x; k < nk; k += TV_THREADS) {
                const int h = hits[k];
                if (h > 0) {
                    atomicAdd(&tri[ul[k]], (unsigned long long)h);
                    sup[shift[k] + (Idx)vrel[k]] = 1;
                }
            }
        }
        if (!BIG)
            for (int k = threadIdx.x; k < dpv; k += TV_THREADS) {
                const int c = cnt[k];
                if (c > 0) {
                    atomicAdd(&tri[glist[k]], (unsigned long long)c);
                    sup[vs + k] = 1;
                }
            }
        if (threadIdx.x == 0 && s_tv) {
            atomicAdd(&tri[v], s_tv);
            atomicAdd(&ds->num_tri, s_tv);
        }
        __syncthreads();
    }
}

// Items for the block kernels: hashed ones from the front (count cnt[0]), big
// ones from the back (count cnt[1]); `cap` entries hold both.
__global__ void k_tv_plan(const int64_t *off, const int64_t *ooff, int64_t n, unsigned long long *items, int64_t cap,
                          uint32_t *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dpv = ooff[v + 1] - ooff[v];
        const int64_t dv = off[v + 1] - off[v];
        if (dpv < 1 || dv == dpv) continue;
        if (dpv <= TV_WARP_DPLUS && dv <= TV_WARP_DEG) continue;
        const uint32_t nch = (uint32_t)((dv + TV_ITEM - 1) / TV_ITEM);
        if (dpv <= TV_BLOCK_DPLUS) {
            const uint32_t at = atomicAdd(&cnt[0], nch);
            for (uint32_t c = 0; c < nch; ++c) items[at + c] = ((unsigned long long)v << 32) | c;
        } else {
            const uint32_t at = atomicAdd(&cnt[1], nch);
            for (uint32_t c = 0; c < nch; ++c) items[cap - 1 - (int64_t)(at + c)] = ((unsigned long long)v << 32) | c;
        }
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    LF_CUDA(cudaGetDevice(&dev));
    LF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms > 0 ? sms : 1;
}

// Triangles of the oriented graph by their middle vertex.  `cnt` holds five
// counters that start at zero.  Returns the number of kernels launched.
template <typename Idx>
int launch_tv(const int64_t *off, const int32_t *adj, const int32_t *deg, const int64_t *ooff, const int32_t *oadj,
              int64_t n, unsigned long long *items, int64_t cap, uint32_t *cnt, unsigned long long *tri,
              uint8_t *sup, DevScalars *ds, cudaStream_t st) {
    constexpr size_t hs = tv_items_smem(false, sizeof(Idx)), bs = tv_items_smem(true, sizeof(Idx));
    LF_CUDA(cudaFuncSetAttribute(k_tv_items<false, Idx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs));
    LF_CUDA(cudaFuncSetAttribute(k_tv_items<true, Idx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs));
    int per_sm = 0;
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tv_warp<Idx>, 256, 0));
    const int sms = sm_count();
    k_tv_plan<<<grid_for(n, 256, 8192), 256, 0, st>>>(off, ooff, n, items, cap, cnt);
    LF_LAUNCHED();
    k_tv_items<false, Idx><<<sms * 5, TV_THREADS, hs, st>>>(off, adj, deg, ooff, oadj, items, cnt, cnt + 2, tri, sup,
                                                            ds);
    LF_LAUNCHED();
    k_tv_items<true, Idx><<<sms * 2, TV_THREADS, bs, st>>>(off, adj, deg, ooff, oadj, items + cap, cnt + 1, cnt + 3,
                                                           tri, sup, ds);
    LF_LAUNCHED();
    k_tv_warp<Idx><<<sms * std::max(1, per_sm), 256, 0, st>>>(off, adj, deg, ooff, oadj, n, cnt + 4, tri, sup, ds);
    LF_LAUNCHED();
    return 4;
}

// Capacity of the item array: nodes with deg > TV_WARP_DEG or d+ > TV_WARP_DPLUS
// number at most 2m / (TV_WARP_DPLUS + 1), plus one item per TV_ITEM entries.
int64_t tv_item_cap(int64_t m) { return 2 * m / (TV_WARP_DPLUS + 1) + 2 * m / TV_ITEM + 2; }

// ---- a4 --------------------------------------------------------------------
__global__ void k_vt(const int64_t *ooff, const int32_t *oadj, const uint8_t *sup, int64_t n, int32_t *vt,
                     DevScalars *ds) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mb = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t s = ooff[u], e = ooff[u + 1];
        const int64_t du = e - s;
        int cnt = 0;
        for (int64_t p = s + lane; p < e; p += 32) {
            int32_t v = oadj[p];
            mb += 4ull * (unsigned long long)(du + (ooff[v + 1] - ooff[v]));
            if (sup[p]) {
                ++cnt;
                atomicAdd(&vt[v], 1);
            }
        }
        cnt = __reduce_add_sync(FULL, cnt);
        if (lane == 0 && cnt) atomicAdd(&vt[u], cnt);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb += __shfl_down_sync(FULL, mb, o);
    if (lane == 0 && mb) atomicAdd(&ds->merge_bytes, mb);
}

// ---- a5 --------------------------------------------------------------------
__device__ __forceinline__ void cc_fraction(long long t, int32_t d, unsigned long long &num,
                                            unsigned long long &den) {
    if (d > 1) {
        num = (unsigned long long)t;
        den = (unsigned long long)d * (unsigned long long)(d - 1) / 2ull;
    } else {
        num = 0;
        den = 1;
    }
}

__device__ __forceinline__ double local_cc(long long t, int32_t d) {
    if (d <= 1) return 0.0;
    long long c2 = (long long)d * (long long)(d - 1) / 2;
    return __ddiv_rn((double)t, (double)c2);
}

// 128-bit compare of a*b against c*e.
__device__ __forceinline__ int cmp_prod(unsigned long long a, unsigned long long b, unsigned long long c,
                                        unsigned long long e) {
    unsigned long long h1 = __umul64hi(a, b), l1 = a * b;
    unsigned long long h2 = __umul64hi(c, e), l2 = c * e;
    if (h1 != h2) return h1 < h2 ? -1 : 1;
    if (l1 != l2) return l1 < l2 ? -1 : 1;
    return 0;
}

// true when x must come before y in the node order
__device__ bool order_before(const unsigned long long *tri, const int32_t *deg, int32_t x, int32_t y) {
    unsigned long long nx, dx, ny, dy;
    cc_fraction((long long)tri[x], deg[x], nx, dx);
    cc_fraction((long long)tri[y], deg[y], ny, dy);
    int c = cmp_prod(nx, dy, ny, dx);
    if (c != 0) return c > 0;
    if (deg[x] != deg[y]) return deg[x] > deg[y];
    return x < y;
}

__global__ void k_order_keys_deg(const int32_t *deg, int64_t n, int32_t max_deg, unsigned long long *keys,
                                 uint32_t *vals) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        keys[x] = (unsigned long long)(max_deg - deg[x]);
        vals[x] = (uint32_t)x;
    }
}

constexpr unsigned long long ONE_BITS = 0x3ff0000000000000ull;   // bits of 1.0

__global__ void k_order_keys_cc(const unsigned long long *tri, const int32_t *deg, int64_t n,
                                const uint32_t *vals, unsigned long long *keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = (int32_t)vals[i];
        double c = local_cc((long long)tri[x], deg[x]);
        keys[i] = ONE_BITS - (unsigned long long)__double_as_longlong(c);   // descending CC
    }
}

// Equal rounded CC but different exact rationals: RN is monotone, so such
// nodes are adjacent in the sorted order; their run needs the exact compare.
__global__ void k_order_check(const unsigned long long *keys, const uint32_t *vals,
                              const unsigned long long *tri, const int32_t *deg, int64_t n, DevScalars *ds) {
    for (int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (keys[i] != keys[i - 1]) continue;
        int32_t a = (int32_t)vals[i - 1], b = (int32_t)vals[i];
        unsigned long long na, da, nb, db;
        cc_fraction((long long)tri[a], deg[a], na, da);
        cc_fraction((long long)tri[b], deg[b], nb, db);
        if (cmp_prod(na, db, nb, da) != 0) atomicAdd(&ds->bad_runs, 1);
    }
}

// Rare path, one thread: insertion-sort every run of equal rounded CC that
// holds distinct rationals with the exact comparator.
__global__ void k_order_fix(const unsigned long long *keys, uint32_t *vals, const unsigned long long *tri,
                            const int32_t *deg, int64_t n) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t i = 0;
    while (i < n) {
        int64_t j = i + 1;
        while (j < n && keys[j] == keys[i]) ++j;
        if (j - i > 1) {
            for (int64_t a = i + 1; a < j; ++a) {
                uint32_t v = vals[a];
                int64_t b = a - 1;
                while (b >= i && order_before(tri, deg, (int32_t)v, (int32_t)vals[b])) {
                    vals[b + 1] = vals[b];
                    --b;
                }
                vals[b + 1] = v;
            }
        }
        i = j;
    }
}

__global__ void k_positions(const uint32_t *vals, int64_t n, int32_t *order, int32_t *pos) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = (int32_t)vals[i];
        order[i] = x;
        pos[x] = (int32_t)i;
    }
}

__global__ void k_cc_sum(const unsigned long long *tri, const int32_t *deg, int64_t n, DevScalars *ds) {
    __shared__ unsigned long long acc[SACC_CHUNKS];
    for (int i = threadIdx.x; i < SACC_CHUNKS; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        sacc_add(acc, local_cc((long long)tri[x], deg[x]));
    __syncthreads();
    for (int i = threadIdx.x; i < SACC_CHUNKS; i += blockDim.x)
        if (acc[i]) atomicAdd(&ds->sacc[i], acc[i]);
}

__global__ void k_cc_final(DevScalars *ds, int64_t n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = sacc_round_and_clear(ds->sacc);
    ds->cc = n > 0 ? __ddiv_rn(s, (double)n) : 0.0;
}

// ---- batches of graphs -----------------------------------------------------
// Graph of each node: its dense id falls in [gnoff[i], gnoff[i+1]).
__global__ void k_fill_gid(const int64_t *gnoff, int64_t G, int64_t n, int32_t *gid) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = G - 1;   // last i with gnoff[i] <= x
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (gnoff[mid] <= x) lo = mid; else hi = mid - 1;
        }
        gid[x] = (int32_t)lo;
    }
}

__global__ void k_gid_keys(const uint32_t *vals, const int32_t *gid, int64_t n, unsigned long long *keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (unsigned long long)gid[vals[i]];
}

// cc of every graph of a batch: RN(exact sum of RN(CC_i) over its nodes) / n_i.
__global__ void k_cc_sum_batch(const unsigned long long *tri, const int32_t *deg, const int32_t *gid, int64_t n,
                               unsigned long long *gsacc) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        sacc_add(gsacc + (int64_t)gid[x] * SACC_CHUNKS, local_cc((long long)tri[x], deg[x]));
}

__global__ void k_cc_final_batch(unsigned long long *gsacc, const int64_t *gnoff, int64_t G, double *gcc,
                                 float *gcc32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ni = gnoff[i + 1] - gnoff[i];
        const double s = sacc_round_and_clear(gsacc + i * SACC_CHUNKS);
        const double c = ni > 0 ? __ddiv_rn(s, (double)ni) : 0.0;
        gcc[i] = c;
        gcc32[i] = c >= 1e-30 ? (float)c : 0.f;   // 0 turns the FP32 screen off for the graph
    }
}

template <typename T>
T read_scalar(lf_graph *g, const T *dptr) {
    T v;
    LF_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, g->stream));
    LF_CUDA(cudaStreamSynchronize(g->stream));
    return v;
}

struct PhaseTimer {
    lf_graph *g;
    cudaEvent_t ev[6];
    int used = 0;
    explicit PhaseTimer(lf_graph *gg) : g(gg) {
        for (auto &e : ev) LF_CUDA(cudaEventCreate(&e));
    }
    ~PhaseTimer() {
        for (auto &e : ev) cudaEventDestroy(e);
    }
    void mark() { LF_CUDA(cudaEventRecord(ev[used++], g->stream)); }
    double ms(int a, int b) {
        float t = 0.f;
        LF_CUDA(cudaEventElapsedTime(&t, ev[a], ev[b]));
        return (double)t;
    }
};

}  // namespace

void build_graph(lf_graph *g, const int32_t *src, const int32_t *dst, int64_t E, bool on_device) {
    cudaStream_t st = g->stream;
    DevScalars *ds = g->ds;
    PhaseTimer pt(g);
    pt.mark();   // 0
    const int32_t *dsrc = src, *ddst = dst;
    int32_t *own_src = nullptr, *own_dst = nullptr;
    if (E > 0 && !on_device) {
        own_src = dalloc_n<int32_t>(g, E);
        own_dst = dalloc_n<int32_t>(g, E);
        LF_CUDA(cudaMemcpyAsync(own_src, src, (size_t)E * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LF_CUDA(cudaMemcpyAsync(own_dst, dst, (size_t)E * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        dsrc = own_src;
        ddst = own_dst;
    }
    unsigned long long *tmp64 = dalloc_n<unsigned long long>(g, 4);
    LF_CUDA(cudaMemsetAsync(tmp64, 0, 4 * sizeof(unsigned long long), st));
    int32_t minus1 = -1;
    LF_CUDA(cudaMemcpyAsync(&ds->max_id, &minus1, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    unsigned long long nonloops = 0;
    int32_t max_id = -1, neg = 0;
    if (E > 0) {
        k_id_range<<<grid_for(E, 256, 4096), 256, 0, st>>>(dsrc, ddst, E, ds, tmp64); ++g->launches;
        LF_LAUNCHED();
        nonloops = read_scalar(g, tmp64);
        max_id = read_scalar(g, &ds->max_id);
        neg = read_scalar(g, &ds->neg_id);
    }
    if (neg) fail(LF_ERR_INVALID, "edge list holds a negative node id");
    if (nonloops >= (1ull << 31)) fail(LF_ERR_CAPACITY, "more than 2^31-1 edges");

    int64_t n = 0, two_m = 0;
    if (nonloops > 0) {
        // dense labels from a bitmap over the id range: rank = set bits below the id
        int64_t nwords = ((int64_t)max_id >> 5) + 1;
        uint32_t *bm = dalloc_n<uint32_t>(g, nwords);
        uint32_t *wb = dalloc_n<uint32_t>(g, nwords + 1);
        LF_CUDA(cudaMemsetAsync(bm, 0, (size_t)nwords * 4, st));
        k_mark_ids<<<grid_for(E, 256, 4096), 256, 0, st>>>(dsrc, ddst, E, bm); ++g->launches;
        LF_LAUNCHED();
        k_word_popc<<<grid_for(nwords, 256, 4096), 256, 0, st>>>(bm, nwords, wb); ++g->launches;
        LF_LAUNCHED();
        scan_exclusive<uint32_t>(g, wb, wb, nwords, wb + nwords);
        n = read_scalar(g, wb + nwords);
        g->n = n;
        g->labels = dalloc_n<int32_t>(g, n);
        k_labels<<<grid_for(nwords, 256, 4096), 256, 0, st>>>(bm, wb, nwords, g->labels); ++g->launches;
        LF_LAUNCHED();
        // both directions of every pair, sorted by (row, col), duplicates dropped
        int64_t nkeys = 2 * (int64_t)nonloops;
        unsigned long long *keys = dalloc_n<unsigned long long>(g, nkeys);
        LF_CUDA(cudaMemsetAsync(tmp64, 0, sizeof(unsigned long long), st));
        k_make_keys<<<grid_for(E, 256, 4096), 256, 0, st>>>(dsrc, ddst, E, bm, wb, keys, tmp64); ++g->launches;
        LF_LAUNCHED();
        dfree(g, wb);
        dfree(g, bm);
        if (own_src) { dfree(g, own_src); dfree(g, own_dst); own_src = own_dst = nullptr; }
        std::vector<int> shifts;
        int b = bits_for((unsigned long long)(n - 1));
        for (int s = 0; s < b; s += 8) shifts.push_back(s);
        for (int s = 0; s < b; s += 8) shifts.push_back(32 + s);
        radix_sort(g, keys, nullptr, nkeys, shifts);
        uint32_t *flag = dalloc_n<uint32_t>(g, nkeys + 1);
        uint32_t *idx = dalloc_n<uint32_t>(g, nkeys + 1);
        k_unique_flags<<<grid_for(nkeys, 256, 8192), 256, 0, st>>>(keys, nkeys, flag); ++g->launches;
        LF_LAUNCHED();
        scan_exclusive<uint32_t>(g, flag, idx, nkeys, idx + nkeys);
        two_m = read_scalar(g, idx + nkeys);
        g->m = two_m / 2;
        g->adj = dalloc_n<int32_t>(g, two_m);
        g->off = dalloc_n<int64_t>(g, n + 1);
        k_unique_compact<<<grid_for(nkeys, 256, 8192), 256, 0, st>>>(keys, nkeys, flag, idx, g->adj, g->off); ++g->launches;
        LF_LAUNCHED();
        dfree(g, idx);
        dfree(g, flag);
        dfree(g, keys);
        g->deg = dalloc_n<int32_t>(g, n);
        LF_CUDA(cudaMemsetAsync(&ds->count32, 0, sizeof(int32_t), st));
        k_degrees<<<grid_for(n, 256, 8192), 256, 0, st>>>(g->off, n, two_m, g->off + n, g->deg, ds); ++g->launches;
        LF_LAUNCHED();
        g->max_deg = read_scalar(g, &ds->count32);
    } else {
        g->n = 0;
        g->m = 0;
        g->labels = dalloc_n<int32_t>(g, 1);
        g->off = dalloc_n<int64_t>(g, 1);
        g->adj = dalloc_n<int32_t>(g, 1);
        g->deg = dalloc_n<int32_t>(g, 1);
        LF_CUDA(cudaMemsetAsync(g->off, 0, sizeof(int64_t), st));
    }
    if (own_src) { dfree(g, own_src); dfree(g, own_dst); }
    pt.mark();   // 1

    // ---- a2: orientation
    const int64_t m = g->m;
    g->ooff = dalloc_n<int64_t>(g, n + 1);
    g->oadj = dalloc_n<int32_t>(g, m);
    if (n > 0) {
        int64_t *odeg = dalloc_n<int64_t>(g, n);
        k_out_degree<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(g->off, g->adj, g->deg, n, odeg); ++g->launches;
        LF_LAUNCHED();
        scan_exclusive<int64_t>(g, odeg, g->ooff, n, g->ooff + n);
        dfree(g, odeg);
        k_orient_fill<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(g->off, g->adj, g->deg, n, g->ooff, g->oadj); ++g->launches;
        LF_LAUNCHED();
    } else {
        LF_CUDA(cudaMemsetAsync(g->ooff, 0, sizeof(int64_t), st));
    }
    pt.mark();   // 2

    // ---- a3: triangles
    g->tri = reinterpret_cast<long long *>(dalloc_n<unsigned long long>(g, n));
    g->vt = dalloc_n<int32_t>(g, n);
    uint8_t *sup = dalloc_n<uint8_t>(g, m);
    LF_CUDA(cudaMemsetAsync(g->tri, 0, (size_t)(n > 0 ? n : 1) * 8, st));
    LF_CUDA(cudaMemsetAsync(g->vt, 0, (size_t)(n > 0 ? n : 1) * 4, st));
    LF_CUDA(cudaMemsetAsync(sup, 0, (size_t)(m > 0 ? m : 1), st));
    unsigned long long *utri = reinterpret_cast<unsigned long long *>(g->tri);
    if (n > 0) {
        const int64_t cap = tv_item_cap(m);
        unsigned long long *items = dalloc_n<unsigned long long>(g, cap);
        // [0..1] item counts, [2..3] item counters, [4] node-run counter
        uint32_t *cnt = reinterpret_cast<uint32_t *>(tmp64);
        LF_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(uint32_t), st));
        if (m < (int64_t)INT32_MAX)
            g->launches += launch_tv<int32_t>(g->off, g->adj, g->deg, g->ooff, g->oadj, n, items, cap, cnt, utri, sup,
                                              ds, st);
        else
            g->launches += launch_tv<long long>(g->off, g->adj, g->deg, g->ooff, g->oadj, n, items, cap, cnt, utri,
                                                sup, ds, st);
        dfree(g, items);
    }
    pt.mark();   // 3
    if (n > 0) {
        k_vt<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(g->ooff, g->oadj, sup, n, g->vt, ds); ++g->launches;
        LF_LAUNCHED();
    }
    dfree(g, sup);
    pt.mark();   // 4

    // ---- a5: order and cc
    g->order = dalloc_n<int32_t>(g, n);
    g->pos = dalloc_n<int32_t>(g, n);
    int64_t *gnoff_d = nullptr;
    if (g->ngraphs > 0) {   // a batch: the graph of every node, from the shifted label ranges
        const int64_t G = g->ngraphs;
        std::vector<int32_t> lab((size_t)n);
        if (n > 0) LF_CUDA(cudaMemcpyAsync(lab.data(), g->labels, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
        LF_CUDA(cudaStreamSynchronize(st));
        g->gnoff.assign((size_t)G + 1, n);
        for (int64_t i = 0; i < G; ++i)
            g->gnoff[(size_t)i] = std::lower_bound(lab.begin(), lab.end(), (int32_t)g->gbase[(size_t)i]) - lab.begin();
        gnoff_d = dalloc_n<int64_t>(g, G + 1);
        LF_CUDA(cudaMemcpyAsync(gnoff_d, g->gnoff.data(), (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, st));
        g->gid = dalloc_n<int32_t>(g, std::max<int64_t>(n, 1));
        if (n > 0) {
            k_fill_gid<<<grid_for(n, 256, 8192), 256, 0, st>>>(gnoff_d, G, n, g->gid); ++g->launches;
            LF_LAUNCHED();
        }
        g->gcc = dalloc_n<double>(g, G);
        g->gcc32 = dalloc_n<float>(g, G);
        g->gT = dalloc_n<double>(g, G);
        g->gsacc = dalloc_n<unsigned long long>(g, G * SACC_CHUNKS);
        LF_CUDA(cudaMemsetAsync(g->gsacc, 0, (size_t)(G * SACC_CHUNKS) * 8, st));
    }
    if (n > 0) {
        unsigned long long *keys = dalloc_n<unsigned long long>(g, n);
        uint32_t *vals = dalloc_n<uint32_t>(g, n);
        k_order_keys_deg<<<grid_for(n, 256, 8192), 256, 0, st>>>(g->deg, n, g->max_deg, keys, vals); ++g->launches;
        LF_LAUNCHED();
        std::vector<int> sh;
        for (int s = 0; s < bits_for((unsigned long long)g->max_deg); s += 8) sh.push_back(s);
        radix_sort(g, keys, vals, n, sh);
        k_order_keys_cc<<<grid_for(n, 256, 8192), 256, 0, st>>>(utri, g->deg, n, vals, keys); ++g->launches;
        LF_LAUNCHED();
        sh.clear();
        for (int s = 0; s < 62; s += 8) sh.push_back(s);
        radix_sort(g, keys, vals, n, sh);
        LF_CUDA(cudaMemsetAsync(&ds->bad_runs, 0, sizeof(int32_t), st));
        k_order_check<<<grid_for(n, 256, 8192), 256, 0, st>>>(keys, vals, utri, g->deg, n, ds); ++g->launches;
        LF_LAUNCHED();
        if (read_scalar(g, &ds->bad_runs) > 0) {
            k_order_fix<<<1, 1, 0, st>>>(keys, vals, utri, g->deg, n); ++g->launches;
            LF_LAUNCHED();
        }
        if (g->ngraphs > 0) {   // graph by graph: a stable pass on the graph index keeps each graph's order
            k_gid_keys<<<grid_for(n, 256, 8192), 256, 0, st>>>(vals, g->gid, n, keys); ++g->launches;
            LF_LAUNCHED();
            std::vector<int> gs;
            for (int s = 0; s < bits_for((unsigned long long)(g->ngraphs - 1)); s += 8) gs.push_back(s);
            radix_sort(g, keys, vals, n, gs);
        }
        k_positions<<<grid_for(n, 256, 8192), 256, 0, st>>>(vals, n, g->order, g->pos); ++g->launches;
        LF_LAUNCHED();
        dfree(g, vals);
        dfree(g, keys);
        if (g->ngraphs > 0) {
            k_cc_sum_batch<<<grid_for(n, 256, 8192), 256, 0, st>>>(utri, g->deg, g->gid, n, g->gsacc); ++g->launches;
        } else {
            k_cc_sum<<<grid_for(n, 256, 1024), 256, 0, st>>>(utri, g->deg, n, ds); ++g->launches;
        }
        LF_LAUNCHED();
    }
    if (g->ngraphs > 0) {
        k_cc_final_batch<<<grid_for(g->ngraphs, 256, 1024), 256, 0, st>>>(g->gsacc, gnoff_d, g->ngraphs, g->gcc,
                                                                          g->gcc32); ++g->launches;
        LF_LAUNCHED();
        g->gcc_host.assign((size_t)g->ngraphs, 0.0);
        LF_CUDA(cudaMemcpyAsync(g->gcc_host.data(), g->gcc, (size_t)g->ngraphs * 8, cudaMemcpyDeviceToHost, st));
        LF_CUDA(cudaStreamSynchronize(st));
        dfree(g, gnoff_d);
    }
    k_cc_final<<<1, 32, 0, st>>>(ds, n); ++g->launches;
    LF_LAUNCHED();
    pt.mark();   // 5
    dfree(g, tmp64);
    LF_CUDA(cudaStreamSynchronize(st));
    g->cc = read_scalar(g, &ds->cc);
    lf_create_stats &cs = g->cstats;
    cs.num_nodes = n;
    cs.num_edges = g->m;
    cs.num_triangles = (int64_t)read_scalar(g, &ds->num_tri);
    cs.merge_bytes = (int64_t)read_scalar(g, &ds->merge_bytes);
    cs.ms_csr = pt.ms(0, 1);
    cs.ms_orient = pt.ms(1, 2);
    cs.ms_triangles = pt.ms(2, 3);
    cs.ms_vt = pt.ms(3, 4);
    cs.ms_order = pt.ms(4, 5);
    cs.num_launches = (int64_t)g->launches;
}

// ---------------------------------------------------------------------------
// Triangle counts without any allocation.
//
// For callers that cannot allocate device memory at the time of the call
// (device memory owned entirely by another allocator, or a latency-critical
// loop where an allocation could stall or fail): the same triangle kernels as
// lf_graph_create, with their working memory (edge marks, hub list, counters)
// taken from one array reserved statically in this library.  Every GPU that
// loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;   // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
bool g_noalloc_attrs[NOALLOC_MAX_DEVICES] = {};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the array on the current device (the host-side symbol is
// only a stand-in), looked up on every call with that device current (so a
// device reset between calls does not leave a stale address); the kernels'
// shared-memory limits are raised once per device.
unsigned char *noalloc_scratch() {
    int dev = 0;
    LF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(LF_ERR_CAPACITY, "device %d beyond %d", dev, NOALLOC_MAX_DEVICES);
    void *p = nullptr;
    LF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_attrs[dev]) {
        set_triangle_attrs();
        g_noalloc_attrs[dev] = true;
    }
    return static_cast<unsigned char *>(p);
}

// The oriented CSR must be well formed before the counting kernels index
// the array with it: offsets from 0 to m, non-decreasing, ids in [0, n).
// Any violation sets *bad.
__global__ void k_noalloc_check(const int64_t *ooff, const int32_t *oadj, int64_t n, int64_t m, int32_t *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0 && (ooff[0] != 0 || ooff[n] != m)) atomicOr(bad, 1);
    for (int64_t x = i0; x < n; x += stride)
        if (ooff[x + 1] < ooff[x]) atomicOr(bad, 1);
    for (int64_t e = i0; e < m; e += stride)
        if (oadj[e] < 0 || (int64_t)oadj[e] >= n) atomicOr(bad, 1);
}

}  // namespace

size_t noalloc_scratch_needed(int64_t n, int64_t m) {
    return round256(sizeof(DevScalars)) + 256 + round256((size_t)n * sizeof(int32_t)) + round256((size_t)m);
}

void triangles_noalloc(const int64_t *ooff, const int32_t *oadj, int64_t n, int64_t m, int64_t *t, int32_t *vt,
                       cudaStream_t st) {
    if (n < 0 || m < 0) fail(LF_ERR_INVALID, "negative size (n=%lld, m=%lld)", (long long)n, (long long)m);
    const size_t need = noalloc_scratch_needed(n, m);
    if (need > NOALLOC_SCRATCH_BYTES)
        fail(LF_ERR_CAPACITY,
             "graph too large for the static scratch: needs %zu bytes (m + 4n + %zu), limit %zu bytes (16 MiB)", need,
             round256(sizeof(DevScalars)) + 256, NOALLOC_SCRATCH_BYTES);
    if (n > 0 && (!ooff || !t || !vt)) fail(LF_ERR_INVALID, "NULL device pointer");
    if (m > 0 && !oadj) fail(LF_ERR_INVALID, "NULL device pointer");
    unsigned char *base = noalloc_scratch();
    DevScalars *ds = reinterpret_cast<DevScalars *>(base);
    uint32_t *nh = reinterpret_cast<uint32_t *>(base + round256(sizeof(DevScalars)));
    int32_t *hubs = reinterpret_cast<int32_t *>(base + round256(sizeof(DevScalars)) + 256);
    uint8_t *sup = base + round256(sizeof(DevScalars)) + 256 + round256((size_t)n * sizeof(int32_t));
    // the array keeps the previous call's contents: clear what must start at zero
    LF_CUDA(cudaMemsetAsync(ds, 0, sizeof(DevScalars), st));
    LF_CUDA(cudaMemsetAsync(nh, 0, 2 * sizeof(uint32_t), st));
    if (m > 0) LF_CUDA(cudaMemsetAsync(sup, 0, (size_t)m, st));
    if (n == 0) return;
    // validate the input first (its flag is a word of the array; the host
    // waits for it: a malformed CSR is rejected before anything indexes with it)
    k_noalloc_check<<<grid_for(std::max(n, m), 256, 1 << 14), 256, 0, st>>>(ooff, oadj, n, m, &ds->err);
    LF_LAUNCHED();
    int32_t bad = 0;
    LF_CUDA(cudaMemcpyAsync(&bad, &ds->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LF_CUDA(cudaStreamSynchronize(st));
    if (bad)
        fail(LF_ERR_INVALID, "malformed oriented CSR: offsets must run from 0 to num_edges without decreasing "
                             "and every neighbour id must lie in [0, num_nodes)");
    LF_CUDA(cudaMemsetAsync(t, 0, (size_t)n * sizeof(int64_t), st));
    LF_CUDA(cudaMemsetAsync(vt, 0, (size_t)n * sizeof(int32_t), st));
    unsigned long long *utri = reinterpret_cast<unsigned long long *>(t);
    launch_triangles(ooff, oadj, n, hubs, nh, utri, sup, ds, st);
    k_vt<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(ooff, oadj, sup, n, vt, ds);
    LF_LAUNCHED();
}

}  // namespace lf

extern "C" lf_status lf_triangles_noalloc(const int64_t *oriented_offsets, const int32_t *out_neighbours,
                                          int64_t num_nodes, int64_t num_edges, int64_t *t, int32_t *vt,
                                          void *stream) {
    try {
        lf::triangles_noalloc(oriented_offsets, out_neighbours, num_nodes, num_edges, t, vt,
                              static_cast<cudaStream_t>(stream));
        return LF_OK;
    } catch (const lf::Error &e) {
        return e.status;
    } catch (...) {
        lf::set_error(LF_ERR_CUDA, "unexpected internal error");
        return LF_ERR_CUDA;
    }
}
