// One-time preprocessing of a graph (Methods, Preprocessing; Methods, WCC;
// Heuristic Counting of Triangles):
//   a1  self-loop and multi-edge removal, dense relabel, symmetric CSR
//   a2  degree-ordered orientation N+(u)
//   a3  triangle counts t(x,V) and the marks of edges that lie on a triangle
//   a4  vt(x,V) from the edge marks
//   a5  local CC, node order (exact rational compare), global cc
#include <cstring>
#include <mutex>

#include "lf_internal.cuh"

namespace lf {
namespace {

constexpr int TRI_WARP_MAX = 64;        // out-degree handled by one warp
constexpr int TRI_BLOCK_LIST = 16384;   // out-neighbour list held in shared memory by one block
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

// One warp per node u with 2 <= d+(u) <= TRI_WARP_MAX.  For every v in N+(u)
// the warp streams N+(v) and looks each w up in N+(u) (kept in shared
// memory): w found means triangle (u, v, w) with rank u < v < w, met exactly
// once.  Credits: t[u] += |N+(u) & N+(v)| summed over v, t[v] += that count
// per v (one atomic per oriented edge), t[w] accumulated per position of w
// in N+(u) (one atomic per oriented edge).  Edge marks: v->w directly,
// u->v and u->w from the per-position counters.
__global__ void __launch_bounds__(256) k_tri_warp(const int64_t *ooff, const int32_t *oadj, int64_t n,
                                                  unsigned long long *tri, uint8_t *sup, DevScalars *ds) {
    __shared__ int32_t s_list[8][TRI_WARP_MAX];
    __shared__ int32_t s_top[8][TRI_WARP_MAX];
    __shared__ int32_t s_mid[8][TRI_WARP_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *list = s_list[w], *top = s_top[w], *mid = s_mid[w];
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long found = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t s = ooff[u];
        const int du = (int)(ooff[u + 1] - s);
        if (du < 2 || du > TRI_WARP_MAX) continue;
        for (int i = lane; i < du; i += 32) {
            list[i] = oadj[s + i];
            top[i] = 0;
            mid[i] = 0;
        }
        __syncwarp();
        const int32_t lo_id = list[0], hi_id = list[du - 1];
        unsigned long long tu = 0;
        for (int p = 0; p < du; ++p) {
            const int32_t v = list[p];
            const int64_t sv = ooff[v];
            const int dv = (int)(ooff[v + 1] - sv);
            int c = 0;
            for (int j = lane; j < dv; j += 32) {
                int32_t x = oadj[sv + j];
                if (x < lo_id || x > hi_id) continue;
                int idx = find_sorted(list, du, x);
                if (idx >= 0) {
                    atomicAdd(&top[idx], 1);
                    sup[sv + j] = 1;
                    ++c;
                }
            }
            c = __reduce_add_sync(FULL, c);
            if (c > 0 && lane == 0) {
                atomicAdd(&tri[v], (unsigned long long)c);
                mid[p] = 1;
            }
            tu += (unsigned long long)c;
        }
        __syncwarp();
        for (int i = lane; i < du; i += 32) {
            int cnt = top[i];
            if (cnt > 0) atomicAdd(&tri[list[i]], (unsigned long long)cnt);
            if (cnt > 0 || mid[i]) sup[s + i] = 1;
        }
        if (lane == 0 && tu > 0) atomicAdd(&tri[u], tu);
        found += tu;
        __syncwarp();
    }
    if (lane == 0 && found) atomicAdd(&ds->num_tri, found);
}

// One block per node with d+(u) > TRI_WARP_MAX; warps take the v's.  When the
// list does not fit in shared memory, the look-ups go to global memory and
// the credits are made per triangle.
__global__ void __launch_bounds__(TRI_BLOCK_THREADS) k_tri_block(const int64_t *ooff, const int32_t *oadj,
                                                                 const int32_t *hubs, const uint32_t *nhubs,
                                                                 unsigned long long *tri, uint8_t *sup,
                                                                 DevScalars *ds) {
    extern __shared__ int32_t dyn[];
    __shared__ unsigned long long s_tu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t h = blockIdx.x; h < *nhubs; h += gridDim.x) {
        const int32_t u = hubs[h];
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

__global__ void k_select_hubs(const int64_t *ooff, int64_t n, int32_t *hubs, uint32_t *nhubs) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        if (ooff[u + 1] - ooff[u] > TRI_WARP_MAX) hubs[atomicAdd(nhubs, 1u)] = (int32_t)u;
}

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
    unsigned long long *tmp64 = dalloc_n<unsigned long long>(g, 2);
    LF_CUDA(cudaMemsetAsync(tmp64, 0, 2 * sizeof(unsigned long long), st));
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
        int32_t *hubs = dalloc_n<int32_t>(g, n);
        uint32_t *nh = reinterpret_cast<uint32_t *>(tmp64);
        LF_CUDA(cudaMemsetAsync(nh, 0, sizeof(uint32_t), st));
        k_select_hubs<<<grid_for(n, 256, 8192), 256, 0, st>>>(g->ooff, n, hubs, nh); ++g->launches;
        LF_LAUNCHED();
        k_tri_warp<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(g->ooff, g->oadj, n, utri, sup, ds); ++g->launches;
        LF_LAUNCHED();
        const size_t smem = (size_t)TRI_BLOCK_LIST * 9;
        LF_CUDA(cudaFuncSetAttribute(k_tri_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tri_block<<<304, TRI_BLOCK_THREADS, smem, st>>>(g->ooff, g->oadj, hubs, nh, utri, sup, ds); ++g->launches;
        LF_LAUNCHED();
        dfree(g, hubs);
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
        k_positions<<<grid_for(n, 256, 8192), 256, 0, st>>>(vals, n, g->order, g->pos); ++g->launches;
        LF_LAUNCHED();
        dfree(g, vals);
        dfree(g, keys);
        k_cc_sum<<<grid_for(n, 256, 1024), 256, 0, st>>>(utri, g->deg, n, ds); ++g->launches;
        LF_LAUNCHED();
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
unsigned char *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the array on the current device (the host-side symbol is
// only a stand-in), looked up once per device with that device current.
unsigned char *noalloc_scratch() {
    int dev = 0;
    LF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(LF_ERR_CAPACITY, "device %d beyond %d", dev, NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        LF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        LF_CUDA(cudaFuncSetAttribute(k_tri_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)TRI_BLOCK_LIST * 9)));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    return g_noalloc_ptr[dev];
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
    LF_CUDA(cudaMemsetAsync(nh, 0, sizeof(uint32_t), st));
    if (m > 0) LF_CUDA(cudaMemsetAsync(sup, 0, (size_t)m, st));
    if (n == 0) return;
    LF_CUDA(cudaMemsetAsync(t, 0, (size_t)n * sizeof(int64_t), st));
    LF_CUDA(cudaMemsetAsync(vt, 0, (size_t)n * sizeof(int32_t), st));
    unsigned long long *utri = reinterpret_cast<unsigned long long *>(t);
    k_select_hubs<<<grid_for(n, 256, 8192), 256, 0, st>>>(ooff, n, hubs, nh);
    LF_LAUNCHED();
    k_tri_warp<<<grid_for(n * 32, 256, 1 << 16), 256, 0, st>>>(ooff, oadj, n, utri, sup, ds);
    LF_LAUNCHED();
    k_tri_block<<<304, TRI_BLOCK_THREADS, (size_t)TRI_BLOCK_LIST * 9, st>>>(ooff, oadj, hubs, nh, utri, sup, ds);
    LF_LAUNCHED();
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
