// C ABI entry points, error plumbing, device memory, and result extraction.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "lf_internal.cuh"

namespace lf {

void build_graph(lf_graph *g, const int32_t *src, const int32_t *dst, int64_t E, bool on_device);

namespace {
thread_local std::string g_last_error;
}

void set_error(lf_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    (void)st;
    g_last_error = buf;
}

[[noreturn]] void fail(lf_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    throw Error{st};
}

void *dalloc(lf_graph *g, size_t bytes) {
    void *p = nullptr;
    if (g->alloc_cb) {
        p = g->alloc_cb(bytes, (void *)g->stream, g->alloc_ctx);
        if (!p) fail(LF_ERR_OOM, "device allocation of %zu bytes failed (callback)", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, g->stream);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(LF_ERR_OOM, "cudaMallocAsync of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    g->live.emplace_back(p, bytes);
    return p;
}

// Frees only what this handle holds: a pointer already freed (a member left
// dangling when the allocation that was to replace it failed) is ignored.
void dfree(lf_graph *g, void *p) {
    if (!p) return;
    size_t bytes = 0;
    bool held = false;
    for (size_t i = 0; i < g->live.size(); ++i)
        if (g->live[i].first == p) {
            bytes = g->live[i].second;
            g->live[i] = g->live.back();
            g->live.pop_back();
            held = true;
            break;
        }
    if (!held) return;
    if (g->free_cb) g->free_cb(p, bytes, (void *)g->stream, g->alloc_ctx);
    else cudaFreeAsync(p, g->stream);
}

namespace {

struct CommKeyArgs {
    const int32_t *mem;
    const int32_t *nmem;
    int32_t K;
};

__global__ void k_member_counts(const int32_t *nmem, int64_t n, int64_t *cnt) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        cnt[x] = nmem[x];
}

__global__ void k_member_keys(CommKeyArgs a, int64_t n, const int64_t *moff, unsigned long long *keys) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = a.nmem[x];
        for (int32_t s = 0; s < c; ++s)
            keys[moff[x] + s] = ((unsigned long long)(uint32_t)a.mem[x * a.K + s] << 32) | (uint32_t)x;
    }
}

__global__ void k_live_flags(const CommRec *comm, int64_t ncomm, uint32_t *flag) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncomm; c += (int64_t)gridDim.x * blockDim.x)
        flag[c] = comm[c].n >= 1 ? 1u : 0u;
}

__global__ void k_comm_output(const unsigned long long *keys, int64_t M, const uint32_t *rank, const int32_t *labels,
                              int64_t *offsets, int32_t *members, int64_t L) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const uint32_t C = (uint32_t)(k >> 32);
        members[i] = labels[(uint32_t)(k & 0xffffffffull)];
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != C) offsets[rank[C]] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) offsets[L] = M;
}

template <typename T>
void d2h(lf_graph *g, T *host, const T *dev, int64_t count) {
    if (count <= 0 || !host) return;
    LF_CUDA(cudaMemcpyAsync(host, dev, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost, g->stream));
}

}  // namespace
}  // namespace lf

using namespace lf;

namespace {

template <typename F>
lf_status call_guarded(F &&fn) {
    try {
        fn();
        return LF_OK;
    } catch (const lf::Error &e) {
        return e.status;
    } catch (const std::bad_alloc &) {
        lf::set_error(LF_ERR_OOM, "host allocation failed");
        return LF_ERR_OOM;
    } catch (...) {
        lf::set_error(LF_ERR_CUDA, "unexpected internal error");
        return LF_ERR_CUDA;
    }
}

void release_all(lf_graph *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);   // no kernel may still use what is freed
    free_run_state(g);
    while (!g->live.empty()) dfree(g, g->live.back().first);
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->rb) cudaFreeHost(g->rb);
    g->rb = nullptr;
    if (g->gT_host) cudaFreeHost(g->gT_host);
    g->gT_host = nullptr;
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    g->stream = nullptr;
}

// After a run that failed part way (an allocation that returned NULL, a
// CUDA error, a device-side timeout), the run state may be half built: wait
// for the stream, drop all of it, and let the next run start from scratch.
void abandon_run(lf_graph *g) {
    if (g->stream) cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    try {
        free_run_state(g);
    } catch (...) {
    }
    g->ran = false;
}

template <typename F>
lf_status run_guarded(lf_graph *g, F &&fn) {
    const lf_status st = call_guarded(fn);
    if (st != LF_OK) abandon_run(g);
    return st;
}

}  // namespace

extern "C" {

const char *lf_last_error(void) {
    static thread_local std::string copy;
    copy = lf::g_last_error;
    return copy.c_str();
}

namespace {
// Shared by lf_graph_create and lf_batch_create: the handle, its options and
// stream, then the preprocessing.  batch_base: for a batch, the id shift of
// every graph (ngraphs + 1 entries), else empty.
lf_status create_handle(const int32_t *src, const int32_t *dst, int64_t num_edges, const lf_options *opt,
                        const std::vector<int64_t> &batch_base, lf_graph **out) {
    *out = nullptr;
    lf_graph *g = nullptr;
    lf_status st = call_guarded([&] {
        if (num_edges < 0) fail(LF_ERR_INVALID, "num_edges < 0");
        if (num_edges > 0 && (!src || !dst)) fail(LF_ERR_INVALID, "src/dst is NULL");
        if (num_edges >= (1ll << 31)) fail(LF_ERR_CAPACITY, "more than 2^31-1 input edges");
        g = new lf_graph();
        if (!batch_base.empty()) {
            g->ngraphs = (int64_t)batch_base.size() - 1;
            g->gbase = batch_base;
        }
        if (opt) {
            g->stream = static_cast<cudaStream_t>(opt->stream);
            g->alloc_cb = opt->alloc;
            g->free_cb = opt->free;
            g->alloc_ctx = opt->alloc_ctx;
            if (opt->member_slots > 0) g->member_slots = opt->member_slots;
            g->warp_max_degree = opt->warp_max_degree;
            g->use_graphs = opt->use_graphs < 0 ? 0 : 1;
            g->profile = opt->profile == 1 ? 1 : 0;
            g->screen = opt->exhaustive_fp64 == 1 ? 0 : 1;
            g->per_queue = opt->per_queue_launches == 1 ? 1 : (opt->per_queue_launches == 2 ? 0 : -1);
            if (opt->barrier_timeout_ms > 0) g->barrier_timeout_ms = opt->barrier_timeout_ms;
            g->inject_stall = opt->inject_barrier_stall == 1 ? 1 : 0;
            g->barrier_mode = opt->barrier_mode == 1 ? 1 : 0;
            g->warps_per_node = opt->warps_per_node;
            if (opt->hub_degree > 0) g->hub_degree = opt->hub_degree;
            if (opt->gain_rule != 0 && opt->gain_rule != LF_GAIN_LITERAL && opt->gain_rule != LF_GAIN_MEANFIELD)
                fail(LF_ERR_INVALID, "unknown gain_rule %d", opt->gain_rule);
            if (opt->gain_rule != 0) g->gain_rule = opt->gain_rule;
            g->debug_checks = opt->debug_checks == 1 ? 1 : 0;
            if ((g->alloc_cb == nullptr) != (g->free_cb == nullptr))
                fail(LF_ERR_INVALID, "alloc and free callbacks must be set together");
        }
        int dev_count = 0;
        if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
            cudaGetLastError();
            fail(LF_ERR_CUDA, "no CUDA device available");
        }
        if (!g->stream) {
            LF_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
            g->own_stream = true;
        }
        LF_CUDA(cudaMallocHost(&g->rb, sizeof(lf::Readback)));
        std::memset(g->rb, 0, sizeof(lf::Readback));
        g->ds = static_cast<lf::DevScalars *>(dalloc(g, sizeof(lf::DevScalars) + sizeof(lf::Readback)));
        LF_CUDA(cudaMemsetAsync(g->ds, 0, sizeof(lf::DevScalars) + sizeof(lf::Readback), g->stream));
        build_graph(g, src, dst, num_edges, batch_base.empty() && opt && opt->edges_on_device);
    });
    if (st != LF_OK) {
        if (g) {
            try { release_all(g); } catch (...) {}
            delete g;
        }
        return st;
    }
    *out = g;
    return LF_OK;
}
}  // namespace

lf_status lf_graph_create(const int32_t *src, const int32_t *dst, int64_t num_edges, const lf_options *opt,
                          lf_graph **out) {
    if (!out) {
        set_error(LF_ERR_INVALID, "out is NULL");
        return LF_ERR_INVALID;
    }
    return create_handle(src, dst, num_edges, opt, std::vector<int64_t>(), out);
}

lf_status lf_batch_create(const int32_t *src, const int32_t *dst, const int64_t *edge_offsets, int64_t num_graphs,
                          const lf_options *opt, lf_graph **out) {
    if (!out) {
        set_error(LF_ERR_INVALID, "out is NULL");
        return LF_ERR_INVALID;
    }
    *out = nullptr;
    std::vector<int32_t> s2, d2;
    std::vector<int64_t> base;
    lf_status st = call_guarded([&] {
        if (num_graphs < 1) fail(LF_ERR_INVALID, "num_graphs must be >= 1");
        if (!edge_offsets) fail(LF_ERR_INVALID, "edge_offsets is NULL");
        if (edge_offsets[0] != 0) fail(LF_ERR_INVALID, "edge_offsets[0] must be 0");
        for (int64_t i = 0; i < num_graphs; ++i)
            if (edge_offsets[i + 1] < edge_offsets[i]) fail(LF_ERR_INVALID, "edge_offsets decrease at graph %lld", (long long)i);
        const int64_t E = edge_offsets[num_graphs];
        if (E > 0 && (!src || !dst)) fail(LF_ERR_INVALID, "src/dst is NULL");
        if (E >= (1ll << 31)) fail(LF_ERR_CAPACITY, "more than 2^31-1 input edges");
        // each graph's ids shifted past the previous graphs' largest id: one
        // disjoint union whose dense ids keep the graphs apart and in order
        base.assign((size_t)num_graphs + 1, 0);
        for (int64_t i = 0; i < num_graphs; ++i) {
            int64_t mx = -1;
            for (int64_t e = edge_offsets[i]; e < edge_offsets[i + 1]; ++e) {
                if (src[e] < 0 || dst[e] < 0) fail(LF_ERR_INVALID, "negative node id in graph %lld", (long long)i);
                mx = std::max<int64_t>(mx, std::max(src[e], dst[e]));
            }
            base[(size_t)i + 1] = base[(size_t)i] + mx + 1;
            if (base[(size_t)i + 1] >= (1ll << 31)) fail(LF_ERR_CAPACITY, "shifted node ids exceed 2^31-1");
        }
        s2.resize((size_t)E);
        d2.resize((size_t)E);
        for (int64_t i = 0; i < num_graphs; ++i)
            for (int64_t e = edge_offsets[i]; e < edge_offsets[i + 1]; ++e) {
                s2[(size_t)e] = (int32_t)(src[e] + base[(size_t)i]);
                d2[(size_t)e] = (int32_t)(dst[e] + base[(size_t)i]);
            }
    });
    if (st != LF_OK) return st;
    lf_options o{};
    if (opt) o = *opt;
    o.edges_on_device = 0;
    return create_handle(s2.data(), d2.data(), (int64_t)s2.size(), &o, base, out);
}

lf_status lf_batch_get_info(lf_graph *g, int64_t *num_graphs, int64_t *node_offsets, int32_t *iterations,
                            int32_t *converged, double *wcc_initial, double *wcc_final, double *cc) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (g->ngraphs == 0) {
        set_error(LF_ERR_STATE, "not a batch");
        return LF_ERR_STATE;
    }
    const int64_t G = g->ngraphs;
    if (num_graphs) *num_graphs = G;
    if (node_offsets)
        for (int64_t i = 0; i <= G; ++i) node_offsets[i] = g->gnoff[(size_t)i];
    if (cc)
        for (int64_t i = 0; i < G; ++i) cc[i] = g->gcc_host[(size_t)i];
    const bool ran = g->ran && (int64_t)g->g_iters.size() == G;
    for (int64_t i = 0; i < G; ++i) {
        if (iterations) iterations[i] = ran ? g->g_iters[(size_t)i] : 0;
        if (converged) converged[i] = ran ? g->g_conv[(size_t)i] : 0;
        if (wcc_initial) wcc_initial[i] = ran ? g->g_T0[(size_t)i] : 0.0;
        if (wcc_final)
            wcc_final[i] = !ran ? 0.0 : (g->g_hist[(size_t)i].empty() ? g->g_T0[(size_t)i] : g->g_hist[(size_t)i].back());
    }
    return LF_OK;
}

lf_status lf_batch_get_history(lf_graph *g, int64_t graph, double *wcc, int32_t cap, int32_t *count) {
    if (!g || g->ngraphs == 0 || graph < 0 || graph >= g->ngraphs) {
        set_error(LF_ERR_INVALID, "not a batch, or graph index out of range");
        return LF_ERR_INVALID;
    }
    if (!g->ran || (int64_t)g->g_hist.size() != g->ngraphs) {
        set_error(LF_ERR_STATE, "no run yet");
        return LF_ERR_STATE;
    }
    const auto &h = g->g_hist[(size_t)graph];
    if (count) *count = (int32_t)h.size();
    if (wcc)
        for (int32_t i = 0; i < cap && i < (int32_t)h.size(); ++i) wcc[i] = h[(size_t)i];
    return LF_OK;
}

lf_status lf_batch_get_communities(lf_graph *g, int64_t *graph_offsets, int64_t *offsets, int64_t offsets_cap,
                                   int32_t *members, int64_t members_cap, int64_t *num_communities,
                                   int64_t *num_members) {
    if (!g || g->ngraphs == 0) {
        set_error(LF_ERR_INVALID, "not a batch");
        return LF_ERR_INVALID;
    }
    int64_t nc = 0, nm = 0;
    lf_status st = lf_get_communities(g, offsets, offsets_cap, members, members_cap, &nc, &nm);
    if (num_communities) *num_communities = nc;
    if (num_members) *num_members = nm;
    if (st != LF_OK || !offsets || !members) return st;
    // community ids follow the graph-by-graph node order, so each graph's
    // communities are one run; members back to the graph's own ids
    const int64_t G = g->ngraphs;
    int64_t gi = 0;
    if (graph_offsets) graph_offsets[0] = 0;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t first = offsets[c], last = offsets[c + 1];
        const int32_t id0 = last > first ? members[first] : 0;
        const int64_t gc = (int64_t)(std::upper_bound(g->gbase.begin(), g->gbase.end(), (int64_t)id0) - g->gbase.begin()) - 1;
        while (gi < gc) {
            ++gi;
            if (graph_offsets) graph_offsets[gi] = c;
        }
        for (int64_t i = first; i < last; ++i) members[i] = (int32_t)(members[i] - g->gbase[(size_t)gc]);
    }
    while (gi < G) {
        ++gi;
        if (graph_offsets) graph_offsets[gi] = nc;
    }
    return LF_OK;
}

void lf_graph_destroy(lf_graph *g) {
    if (!g) return;
    try {
        release_all(g);
    } catch (...) {
    }
    delete g;
}

lf_status lf_run(lf_graph *g, int32_t queue_size, double wcc_threshold, int32_t max_iters, lf_run_stats *stats) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (g->in_callback) {
        set_error(LF_ERR_STATE, "lf_run inside an iteration callback");
        return LF_ERR_STATE;
    }
    return run_guarded(g, [&] { run_impl(g, queue_size, wcc_threshold, max_iters, -1, stats); });
}

lf_status lf_set_partition(lf_graph *g, const int64_t *offsets, const int32_t *members, int64_t num_communities) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (g->in_callback) {
        set_error(LF_ERR_STATE, "lf_set_partition inside an iteration callback");
        return LF_ERR_STATE;
    }
    if (g->ngraphs > 0) {
        set_error(LF_ERR_STATE, "lf_set_partition on a batch of graphs");
        return LF_ERR_STATE;
    }
    return call_guarded([&] {
        if (num_communities < 0) {
            g->part_k = -1;
            g->part_off.clear();
            g->part_mem.clear();
            g->part_maxcnt = 0;
            return;
        }
        if (!offsets) lf::fail(LF_ERR_INVALID, "offsets is NULL");
        if (num_communities > g->n)
            lf::fail(LF_ERR_CAPACITY, "%lld communities for %lld nodes", (long long)num_communities, (long long)g->n);
        if (offsets[0] != 0) lf::fail(LF_ERR_INVALID, "offsets[0] = %lld, not 0", (long long)offsets[0]);
        for (int64_t c = 0; c < num_communities; ++c)
            if (offsets[c + 1] < offsets[c]) lf::fail(LF_ERR_INVALID, "offsets decrease at community %lld", (long long)c);
        const int64_t total = offsets[num_communities];
        if (total > 0 && !members) lf::fail(LF_ERR_INVALID, "members is NULL");
        // original ids -> dense ids through the (ascending) label table
        std::vector<int32_t> labels((size_t)g->n);
        if (g->n > 0) {
            LF_CUDA(cudaMemcpyAsync(labels.data(), g->labels, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream));
            LF_CUDA(cudaStreamSynchronize(g->stream));
        }
        std::vector<int32_t> dense((size_t)total), cnt((size_t)g->n, 0);
        for (int64_t i = 0; i < total; ++i) {
            const auto it = std::lower_bound(labels.begin(), labels.end(), members[i]);
            if (it == labels.end() || *it != members[i])
                lf::fail(LF_ERR_INVALID, "id %d is not a node of the graph", members[i]);
            dense[(size_t)i] = (int32_t)(it - labels.begin());
        }
        int32_t maxcnt = 0;
        for (int64_t c = 0; c < num_communities; ++c) {
            std::vector<int32_t> row(dense.begin() + offsets[c], dense.begin() + offsets[c + 1]);
            std::sort(row.begin(), row.end());
            if (std::adjacent_find(row.begin(), row.end()) != row.end())
                lf::fail(LF_ERR_INVALID, "a node appears twice in community %lld", (long long)c);
            for (int32_t x : row) maxcnt = std::max(maxcnt, ++cnt[(size_t)x]);
        }
        g->part_off.assign(offsets, offsets + num_communities + 1);
        g->part_mem = std::move(dense);
        g->part_k = num_communities;
        g->part_maxcnt = maxcnt;
    });
}

lf_status lf_autotune(lf_graph *g, int32_t queue_size, int32_t trial_iters, lf_tune_result *result) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (g->in_callback) {
        set_error(LF_ERR_STATE, "lf_autotune inside an iteration callback");
        return LF_ERR_STATE;
    }
    if (trial_iters < 1 || queue_size < 1) {
        set_error(LF_ERR_INVALID, "queue_size and trial_iters must be >= 1");
        return LF_ERR_INVALID;
    }
    return run_guarded(g, [&] {
        const int32_t teams[4] = {0, 1, 2, 4};
        const int32_t limits[3] = {0, 96, 192};
        const int32_t hubs[2] = {384, 128};
        const int32_t keep_t = g->warps_per_node, keep_l = g->warp_max_degree, keep_h = g->hub_degree;
        lf_iteration_fn keep_cb = g->it_cb;
        g->it_cb = nullptr;   // trials run without the caller's callback
        double best = 0.0, dflt = 0.0;
        int32_t bt = keep_t, bl = keep_l, bh = keep_h, trials = 0;
        cudaEvent_t e0, e1;
        LF_CUDA(cudaEventCreate(&e0));
        LF_CUDA(cudaEventCreate(&e1));
        // under the paper's gain only the team size shapes the launches (the
        // degree thresholds belong to the mean-field kernels)
        const bool lit = g->gain_rule == LF_GAIN_LITERAL;
        const int nh = lit ? 1 : 2, nl = lit ? 1 : 3;
        try {
            for (int ih = 0; ih < nh; ++ih)
            for (int32_t T : teams)
                for (int il = 0; il < nl; ++il) {
                    const int32_t H = lit ? keep_h : hubs[ih], L = lit ? keep_l : limits[il];
                    g->warps_per_node = T;
                    g->warp_max_degree = L;
                    g->hub_degree = H;
                    LF_CUDA(cudaEventRecord(e0, g->stream));
                    run_impl(g, queue_size, -INFINITY, trial_iters, -1, nullptr);
                    LF_CUDA(cudaEventRecord(e1, g->stream));
                    LF_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    LF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (T == 0 && (lit || (L == 0 && H == 384))) dflt = ms;
                    if (trials == 0 || ms < best) {
                        best = ms;
                        bt = T;
                        bl = L;
                        bh = H;
                    }
                    ++trials;
                }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            g->warps_per_node = keep_t;
            g->warp_max_degree = keep_l;
            g->hub_degree = keep_h;
            g->it_cb = keep_cb;
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        g->warps_per_node = bt;
        g->warp_max_degree = bl;
        g->hub_degree = bh;
        g->it_cb = keep_cb;
        if (result) {
            result->warps_per_node = bt;
            result->warp_max_degree = bl;
            result->trials = trials;
            result->hub_degree = bh;
            result->best_ms = best;
            result->default_ms = dflt;
        }
    });
}

lf_status lf_set_iteration_callback(lf_graph *g, lf_iteration_fn cb, void *ctx) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    g->it_cb = cb;
    g->it_ctx = ctx;
    return LF_OK;
}

lf_status lf_run_partial(lf_graph *g, int32_t queue_size, double wcc_threshold, int32_t max_iters,
                         int64_t max_batches, lf_run_stats *stats) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (g->in_callback) {
        set_error(LF_ERR_STATE, "lf_run inside an iteration callback");
        return LF_ERR_STATE;
    }
    return run_guarded(g, [&] { run_impl(g, queue_size, wcc_threshold, max_iters, max_batches, stats); });
}

lf_status lf_get_sizes(lf_graph *g, int64_t *num_nodes, int64_t *num_edges) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (num_nodes) *num_nodes = g->n;
    if (num_edges) *num_edges = g->m;
    return LF_OK;
}

lf_status lf_get_create_stats(lf_graph *g, lf_create_stats *stats) {
    if (!g || !stats) {
        set_error(LF_ERR_INVALID, "NULL argument");
        return LF_ERR_INVALID;
    }
    *stats = g->cstats;
    return LF_OK;
}

lf_status lf_get_node_stats(lf_graph *g, int64_t *t, int32_t *vt, double *cc_global) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    return call_guarded([&] {
        d2h(g, reinterpret_cast<long long *>(t), g->tri, g->n);
        d2h(g, vt, g->vt, g->n);
        LF_CUDA(cudaStreamSynchronize(g->stream));
        if (cc_global) *cc_global = g->cc;
    });
}

lf_status lf_get_csr(lf_graph *g, int64_t *offsets, int32_t *neighbours, int32_t *labels) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    return call_guarded([&] {
        d2h(g, offsets, g->off, g->n + 1);
        d2h(g, neighbours, g->adj, 2 * g->m);
        d2h(g, labels, g->labels, g->n);
        LF_CUDA(cudaStreamSynchronize(g->stream));
    });
}

lf_status lf_get_oriented(lf_graph *g, int64_t *offsets, int32_t *out_neighbours) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    return call_guarded([&] {
        d2h(g, offsets, g->ooff, g->n + 1);
        d2h(g, out_neighbours, g->oadj, g->m);
        LF_CUDA(cudaStreamSynchronize(g->stream));
    });
}

lf_status lf_get_order(lf_graph *g, int32_t *order) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    return call_guarded([&] {
        d2h(g, order, g->order, g->n);
        LF_CUDA(cudaStreamSynchronize(g->stream));
    });
}

lf_status lf_get_state(lf_graph *g, int64_t *mem_offsets, int32_t *mem_ids, int64_t *comm_n, int64_t *comm_m,
                       int64_t *comm_vol, int64_t *num_memberships, int64_t *num_comm_ids) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (!g->ran) {
        set_error(LF_ERR_STATE, "no run yet");
        return LF_ERR_STATE;
    }
    return call_guarded([&] {
        const int64_t n = g->n;
        std::vector<int32_t> cnt((size_t)n);
        std::vector<int32_t> rows((size_t)(n * g->K));
        std::vector<lf::CommRec> rec((size_t)g->ncomm);
        d2h(g, cnt.data(), g->nmem, n);
        d2h(g, rows.data(), g->mem, n * g->K);
        d2h(g, rec.data(), g->comm, g->ncomm);
        LF_CUDA(cudaStreamSynchronize(g->stream));
        int64_t total = 0;
        for (int64_t x = 0; x < n; ++x) {
            if (mem_offsets) mem_offsets[x] = total;
            for (int32_t s = 0; s < cnt[x]; ++s) {
                if (mem_ids) mem_ids[total] = rows[(size_t)(x * g->K + s)];
                ++total;
            }
        }
        if (mem_offsets) mem_offsets[n] = total;
        for (int64_t c = 0; c < g->ncomm; ++c) {
            if (comm_n) comm_n[c] = rec[c].n;
            if (comm_m) comm_m[c] = rec[c].m2 / 2;
            if (comm_vol) comm_vol[c] = rec[c].vol;
        }
        if (num_memberships) *num_memberships = total;
        if (num_comm_ids) *num_comm_ids = g->ncomm;
    });
}

lf_status lf_get_communities(lf_graph *g, int64_t *offsets, int64_t offsets_cap, int32_t *members,
                             int64_t members_cap, int64_t *num_communities, int64_t *num_members) {
    if (!g) {
        set_error(LF_ERR_INVALID, "graph is NULL");
        return LF_ERR_INVALID;
    }
    if (!g->ran) {
        set_error(LF_ERR_STATE, "no run yet");
        return LF_ERR_STATE;
    }
    return call_guarded([&] {
        cudaStream_t st = g->stream;
        const int64_t n = g->n, nc = g->ncomm;
        // memberships as (community << 32 | node), sorted: communities ascending, members ascending
        int64_t *moff = dalloc_n<int64_t>(g, n + 1);
        k_member_counts<<<grid_for(n, 256, 1 << 16), 256, 0, st>>>(g->nmem, n, moff); ++g->launches;
        LF_LAUNCHED();
        scan_exclusive<int64_t>(g, moff, moff, n, moff + n);
        uint32_t *rank = dalloc_n<uint32_t>(g, nc + 1);
        k_live_flags<<<grid_for(nc, 256, 1 << 16), 256, 0, st>>>(g->comm, nc, rank); ++g->launches;
        LF_LAUNCHED();
        scan_exclusive<uint32_t>(g, rank, rank, nc, rank + nc);
        int64_t M = 0;
        uint32_t L = 0;
        LF_CUDA(cudaMemcpyAsync(&M, moff + n, 8, cudaMemcpyDeviceToHost, st));
        LF_CUDA(cudaMemcpyAsync(&L, rank + nc, 4, cudaMemcpyDeviceToHost, st));
        LF_CUDA(cudaStreamSynchronize(st));
        if (num_communities) *num_communities = (int64_t)L;
        if (num_members) *num_members = M;
        const bool want = offsets && members;
        if (want && (offsets_cap < (int64_t)L + 1 || members_cap < M)) {
            dfree(g, rank);
            dfree(g, moff);
            fail(LF_ERR_CAPACITY, "output buffers too small: need %lld offsets and %lld members",
                 (long long)L + 1, (long long)M);
        }
        if (want) {
            unsigned long long *keys = dalloc_n<unsigned long long>(g, M);
            CommKeyArgs ka{g->mem, g->nmem, g->K};
            k_member_keys<<<grid_for(n, 256, 1 << 16), 256, 0, st>>>(ka, n, moff, keys); ++g->launches;
            LF_LAUNCHED();
            std::vector<int> sh;
            const int bx = bits_for((unsigned long long)(n > 0 ? n - 1 : 0));
            const int bc = bits_for((unsigned long long)(nc > 0 ? nc - 1 : 0));
            for (int s = 0; s < bx; s += 8) sh.push_back(s);
            for (int s = 0; s < bc; s += 8) sh.push_back(32 + s);
            radix_sort(g, keys, nullptr, M, sh);
            int64_t *d_off = dalloc_n<int64_t>(g, (int64_t)L + 1);
            int32_t *d_mem = dalloc_n<int32_t>(g, M);
            k_comm_output<<<grid_for(M, 256, 1 << 16), 256, 0, st>>>(keys, M, rank, g->labels, d_off, d_mem, L); ++g->launches;
            LF_LAUNCHED();
            d2h(g, offsets, d_off, (int64_t)L + 1);
            d2h(g, members, d_mem, M);
            LF_CUDA(cudaStreamSynchronize(st));
            dfree(g, d_mem);
            dfree(g, d_off);
            dfree(g, keys);
        }
        dfree(g, rank);
        dfree(g, moff);
    });
}

}  // extern "C"
