/*
 * lazyfox.h -- C ABI of the GB300 (sm_103a) implementation of Fox / LazyFox
 * overlapping community detection (Garrels, Khodabakhsh, Renard, Baum,
 * "LazyFox: Fast and parallelized overlapping community detection in large
 * graphs", arXiv 2210.03211).
 *
 * Every step of the method runs in this library's own CUDA kernels on one
 * GPU; there is no CPU fallback.  Plain C types only.  No exception crosses
 * the boundary: every call returns an lf_status and, on failure, leaves a
 * message for lf_last_error() (thread-local).
 *
 * Conventions
 *  - Pointers marked "host" are read or written by the call before it returns;
 *    the library keeps no reference to them.  Pointers marked "device" are
 *    CUDA device pointers, used in order on the graph's stream.
 *  - A graph handle owns all device state of one graph.  One handle must not
 *    be used by two threads at the same time; distinct handles are
 *    independent.
 *  - All work of a handle is ordered on one CUDA stream (lf_options.stream,
 *    or a stream the library creates).  Calls that return host data
 *    synchronise that stream.
 *  - Node ids in the input are non-negative int32; the library relabels them
 *    densely (0..n-1, increasing with the original id) and reports results in
 *    original ids.
 *  - Community ids are assigned by the initial clustering (0, 1, 2, ... in
 *    the order the communities are opened) and never reused during a run.
 */
#ifndef LAZYFOX_H
#define LAZYFOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LF_OK = 0,
    LF_ERR_INVALID = 1,   /* bad argument or malformed input */
    LF_ERR_OOM = 2,       /* an allocation failed (device or callback) */
    LF_ERR_CUDA = 3,      /* a CUDA runtime call or a kernel failed */
    LF_ERR_CAPACITY = 4,  /* a size exceeds a documented limit, or an output buffer is too small */
    LF_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    LF_ERR_STATE = 6      /* call out of order (e.g. results before any run) */
} lf_status;

typedef struct lf_graph lf_graph;   /* opaque; owns all device state of one graph */

/* Device memory callbacks: alloc returns a device pointer (NULL on failure)
 * usable on `stream`; free releases it.  Used instead of cudaMallocAsync when
 * set, e.g. to route the library's memory through PyTorch's caching
 * allocator. */
typedef void *(*lf_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lf_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct lf_options {
    void *stream;            /* cudaStream_t to run on; NULL: the library creates one */
    lf_alloc_fn alloc;       /* NULL: cudaMallocAsync on the stream */
    lf_free_fn free;
    void *alloc_ctx;
    int32_t edges_on_device; /* 1: src/dst of lf_graph_create are device pointers */
    int32_t member_slots;    /* initial per-node membership capacity (0: default 4); grows as needed */
    int32_t warp_max_degree; /* 0: default; smaller values send more nodes to the block-wide
                                kernels (tuning and tests) */
    int32_t use_graphs;      /* per-queue launch mode only: 0 (default) captures each
                                iteration in a CUDA graph, -1 launches kernels directly */
    int32_t profile;         /* 1: time every launch that processes queues with CUDA events
                                and count its algorithmic bytes (lf_run_stats.prof_*) */
    int32_t exhaustive_fp64; /* 1: evaluate every candidate gain in FP64 (no FP32 screen);
                                the chosen actions are the same either way */
    int32_t per_queue_launches; /* 1: kernel launches per queue (evaluate, apply), an
                                iteration captured in a CUDA graph; 2: one persistent
                                cooperative kernel per iteration runs every queue
                                (evaluate, grid barrier, apply, grid barrier); 0 (default):
                                persistent for queues of at most 256 nodes, else per queue */
    int32_t barrier_timeout_ms; /* bound on one grid-barrier wait (0: 2000 ms); a wait that
                                runs out ends the call with LF_ERR_TIMEOUT */
    int32_t inject_barrier_stall; /* test hook: 1 makes one block of the persistent kernel
                                skip its barriers, so that the bounded waits run out */
    int32_t barrier_mode;    /* persistent kernel's grid barrier: 0 (default) every block
                                polls all arrival flags; 1 block 0 gathers them and
                                publishes one release flag */
    int32_t warps_per_node;  /* warps that evaluate one node together: 1, 2, 4 or 8; 0 (default)
                                picks by queue size (more warps per node for small queues) */
    int32_t hub_degree;      /* nodes of higher degree are evaluated with a table in global
                                memory, in blocks of their own (per-queue launches: on a second
                                stream); 0 (default) = 384 */
    int32_t gain_rule;       /* decision rule of a move (LF_GAIN_*); 0 (default): LF_GAIN_LITERAL */
    int32_t debug_checks;    /* 1: bounds-checked mode -- the move evaluation, apply, community
                                sums and total of LF_GAIN_LITERAL check every node id, community id,
                                row count and deg(x,C) they read from device state before using it; a value
                                out of range is skipped and the run fails with LF_ERR_CUDA and a
                                message (no kernel traps).  Slower; for tests and debugging */
} lf_options;

/* lf_options.gain_rule.  LF_GAIN_LITERAL is the paper's gain (Methods, Node
 * Changes: Joining / Leaving a Community): the improvement of WCC-hat(P') over
 * WCC-hat(P), the sums of the per-node estimator over all memberships, i.e.
 * the changed community's members' terms (new size and internal edge count,
 * and for the node's neighbours deg(y,C) changed by one) and the node's own
 * term, summed exactly and rounded once.  LF_GAIN_MEANFIELD is a departure
 * kept as an option: the change of the community's mean-field score, every
 * member given the mean internal degree 2m/n and mean degree vol/n. */
#define LF_GAIN_LITERAL 1
#define LF_GAIN_MEANFIELD 2

/* Per-run statistics.  The history pointers are optional caller buffers with
 * `history_cap` entries each (NULL to skip). */
typedef struct lf_run_stats {
    int32_t iterations;      /* iterations completed */
    int32_t converged;       /* 1 if the relative-change test stopped the run */
    int64_t num_batches;     /* queues processed in total */
    double wcc_initial;      /* WCC-hat(P) of the initial clustering */
    int64_t num_communities; /* live communities after the run */
    int64_t num_memberships; /* (node, community) pairs after the run */
    double ms_total;         /* wall time of the call */
    double ms_init;          /* initial clustering and its total (device time) */
    double ms_iterations;    /* all iterations (device time) */
    int32_t history_cap;
    double *wcc_history;     /* WCC-hat(P) after iterations 1..iterations */
    int64_t *joins_history;  /* join actions applied per iteration */
    int64_t *leaves_history; /* leave actions applied per iteration */
    int64_t num_launches;    /* kernels launched by the call */
    int64_t prof_move_launches; /* profile mode: launches that process queues (the move
                                evaluation kernel in per-queue mode, the persistent queue
                                kernel otherwise) */
    double prof_move_ms;     /* profile mode: their summed device time */
    int64_t prof_move_bytes; /* profile mode: their algorithmic bytes.  LF_GAIN_LITERAL
                                (evaluation kernels of a queue): per node 44 + 8|M(x)| (its
                                offsets, count and actions, its row with deg(x,C)), per
                                neighbour y 12 + 8|M(y)| (id, count, degree, row with
                                deg(y,C)), 40 per distinct candidate community (its 16-byte
                                record, its size read with the entries, 20 bytes of member
                                sums).  LF_GAIN_MEANFIELD evaluation: per node 28 + 4|M(x)|,
                                per neighbour y 8 + 4|M(y)|, 16 per distinct candidate
                                community, 16 for the actions; apply (persistent kernel): 8
                                per node, and per moving node 24 + 4|M(x)| + 12 per action,
                                plus 16 per neighbour when the neighbour scan runs */
    double prof_queue_us[4]; /* profile mode, persistent kernel: p50, p90, p99 and max of the
                                time per queue (evaluate + apply + barriers), last iteration */
    int64_t prof_candidates; /* profile mode, LF_GAIN_LITERAL: candidate (node, community) pairs
                                bracketed */
    int64_t prof_exact;      /* profile mode, LF_GAIN_LITERAL: of these, the ones whose gain was
                                summed exactly (the bracket could not decide) */
} lf_run_stats;

/* Device times of the phases of lf_graph_create. */
typedef struct lf_create_stats {
    int64_t num_nodes;
    int64_t num_edges;       /* undirected simple edges m */
    int64_t num_triangles;
    double ms_csr;           /* self-loop/duplicate removal, relabel, symmetric CSR */
    double ms_orient;        /* degree-ordered orientation */
    double ms_triangles;     /* triangle kernels: t(x,V) and the edge marks */
    double ms_vt;            /* vt(x,V) */
    double ms_order;         /* local CC, node order, global cc */
    int64_t merge_bytes;     /* sum over oriented edges u->v of 4*(d+(u) + d+(v)) */
    int64_t num_launches;    /* kernels launched by lf_graph_create */
} lf_create_stats;

/*
 * lf_graph_create -- build a graph from an undirected, unweighted edge list
 * (Methods, Input Data) and run the one-time preprocessing (Methods,
 * Preprocessing; Methods, WCC; Heuristic Counting of Triangles):
 *   - remove self-loops and repeated pairs ("Remove Multi-Edges");
 *   - relabel endpoint ids densely in increasing order ("Dense Node Labels");
 *     the nodes are the endpoints of the remaining edges;
 *   - build the symmetric CSR (ascending rows) and the degree-ordered
 *     orientation N+(u) = {v in N(u) : (deg v, v) > (deg u, u)};
 *   - count t(x,V), the triangles containing x, and vt(x,V), the neighbours
 *     of x that share at least one triangle with x;
 *   - compute the local clustering coefficients CC(i) = t_i / C(d_i,2)
 *     (0 if d_i <= 1), the node order (CC descending, compared exactly as
 *     rationals; then degree descending; then dense id ascending) and the
 *     global cc: the correctly rounded sum of the rounded local CCs over all
 *     n nodes, divided by n ("Node Order"; global cc).
 * src, dst : num_edges ids each; host memory, or device memory if
 *            opt->edges_on_device.  Ids must be >= 0 (else LF_ERR_INVALID).
 * num_edges: >= 0; 0 gives an empty graph (n = 0).
 * opt      : may be NULL (defaults).  Copied; its stream and callbacks must
 *            stay valid until lf_graph_destroy.
 * out      : receives the new handle (NULL on failure).
 * Limits   : fewer than 2^31 simple edges (LF_ERR_CAPACITY).
 */
lf_status lf_graph_create(const int32_t *src, const int32_t *dst, int64_t num_edges,
                          const lf_options *opt, lf_graph **out);

/*
 * lf_run -- Fox / LazyFox community detection (Methods: Initial Clustering,
 * Node Changes with Algorithm 1, Parallelism on Node Change Computations
 * with Algorithm 2, Stopping Criteria, Post-processing).  Always restarts
 * from the initial clustering:
 *   - initial clustering: walk the node order; a node not yet in a community
 *     opens a new one and its unassigned neighbours join it;
 *   - each iteration walks the node order in queues of queue_size nodes (the
 *     last may be shorter).  Every queued node x is evaluated against the
 *     partition as it stood when the queue was filled: for each community C
 *     adjacent to x (x not in C) the gain of joining, for each community of x
 *     the gain of leaving, both as the change of the community's mean-field
 *     WCC-hat score; the best strictly positive gain of each kind is chosen
 *     (lowest community id on ties).  Then all chosen actions of the queue are
 *     applied (leave before join).  queue_size 1 is Fox;
 *   - after each iteration, communities with fewer than two members are
 *     removed and WCC-hat(P), the sum of WCC-hat(x,C) over all memberships, is
 *     taken; the run stops when (T_it - T_prev) / T_prev < wcc_threshold (if
 *     T_prev == 0: when T_it == 0) or after max_iters iterations.
 * queue_size   : >= 1 (else LF_ERR_INVALID).
 * wcc_threshold: relative-change threshold; -INFINITY never stops early.
 * max_iters    : >= 0 (0 runs only the initial clustering).
 * stats        : optional (NULL); filled on return.
 * Errors       : LF_ERR_CAPACITY if a queue of queue_size nodes cannot be
 *                held (queue_size is clamped to n internally, so this only
 *                happens when device memory runs out), LF_ERR_CUDA, LF_ERR_OOM.
 */
lf_status lf_run(lf_graph *g, int32_t queue_size, double wcc_threshold, int32_t max_iters,
                 lf_run_stats *stats);

/*
 * lf_get_communities -- the communities of the last run: live communities in
 * ascending id, members ascending, as original node ids (Post-processing: no
 * post-processing beyond removing degenerate communities).  After a run with
 * max_iters = 0 the initial clustering is returned (singletons included).
 * offsets: host, num_communities + 1 entries (member ranges).
 * members: host, num_members entries.
 * Passing NULL buffers (or caps that are too small) only reports the sizes in
 * *num_communities and *num_members; too-small non-NULL buffers also return
 * LF_ERR_CAPACITY.  LF_ERR_STATE before the first lf_run.
 */
lf_status lf_get_communities(lf_graph *g, int64_t *offsets, int64_t offsets_cap,
                             int32_t *members, int64_t members_cap,
                             int64_t *num_communities, int64_t *num_members);

/*
 * lf_get_node_stats -- per-node triangle counts t(x,V) (int64, n entries),
 * vt(x,V) (int32, n entries) and the global cc (Methods, WCC; Heuristic
 * Counting of Triangles), indexed by dense id.  Any pointer may be NULL.
 * Host buffers.
 */
lf_status lf_get_node_stats(lf_graph *g, int64_t *t, int32_t *vt, double *cc_global);

/* Sizes of the graph: nodes n, undirected simple edges m. */
lf_status lf_get_sizes(lf_graph *g, int64_t *num_nodes, int64_t *num_edges);

/* Device times of lf_graph_create's phases (see lf_create_stats). */
lf_status lf_get_create_stats(lf_graph *g, lf_create_stats *stats);

/*
 * Inspection hooks (host buffers, dense ids).  They expose intermediate
 * results of the preprocessing and of a run for parity tests and tooling.
 *  lf_get_csr      : offsets (n+1), neighbours (2m), labels (n: dense -> original id).
 *  lf_get_oriented : offsets (n+1) and out-neighbours (m) of the orientation.
 *  lf_get_order    : the node order (n dense ids).
 *  lf_get_state    : memberships as CSR over dense ids (mem_offsets n+1,
 *                    mem_ids as counted by *num_memberships, each row
 *                    ascending) and, for every community id ever used
 *                    (*num_comm_ids of them), members n_C, internal edges m_C
 *                    and the sum of member degrees vol_C.  NULL buffers: sizes
 *                    only.  LF_ERR_STATE before the first run.
 */
lf_status lf_get_csr(lf_graph *g, int64_t *offsets, int32_t *neighbours, int32_t *labels);
lf_status lf_get_oriented(lf_graph *g, int64_t *offsets, int32_t *out_neighbours);
lf_status lf_get_order(lf_graph *g, int32_t *order);
lf_status lf_get_state(lf_graph *g, int64_t *mem_offsets, int32_t *mem_ids,
                       int64_t *comm_n, int64_t *comm_m, int64_t *comm_vol,
                       int64_t *num_memberships, int64_t *num_comm_ids);

/*
 * lf_set_partition -- insert an existing division that replaces the initial
 * clustering of the following lf_run calls (Methods, Initial Clustering: an
 * existing division can be inserted instead of the greedy clustering).
 * Community c (0 <= c < num_communities) holds the original node ids
 * members[offsets[c] .. offsets[c+1]); communities may overlap; community ids
 * in the run are the indices c, so ties between communities are broken in
 * the given order.  Passing the communities that lf_get_communities returned
 * after iteration k of a run, and running again, continues that run exactly
 * (the same totals, moves and communities as one longer run).
 * offsets: host, num_communities + 1 entries, offsets[0] = 0, non-decreasing.
 * members: host, offsets[num_communities] entries; copied.
 * num_communities < 0 (pointers ignored) removes the division: lf_run goes back
 * to the initial clustering.
 * Errors: LF_ERR_INVALID for bad offsets, an id that is not a node of the graph
 *         or an id twice in one community; LF_ERR_CAPACITY for more
 *         communities than nodes.  On error the previous division is kept.
 */
lf_status lf_set_partition(lf_graph *g, const int64_t *offsets, const int32_t *members,
                           int64_t num_communities);

/*
 * lf_set_iteration_callback -- cb(g, iteration, wcc, ctx) is called by lf_run
 * after every iteration, once the iteration's pruning and WCC-hat(P) total
 * (wcc) are done and before the stopping test.  Inside it lf_get_communities
 * and the other getters may be called on g (to save the intermediate
 * communities, as the paper does after each iteration on Friendster); lf_run
 * and lf_set_partition may not.  A nonzero return ends the run after this
 * iteration (stats->converged stays 0).  cb = NULL removes it.  Host code,
 * called on the thread that called lf_run.
 */
typedef int (*lf_iteration_fn)(lf_graph *g, int32_t iteration, double wcc, void *ctx);
lf_status lf_set_iteration_callback(lf_graph *g, lf_iteration_fn cb, void *ctx);

/*
 * lf_batch_create -- many independent graphs in one handle, run together:
 * every kernel launch of lf_run covers all of them (the paper runs one
 * graph at a time).  Graph i is the edge
 * list src/dst[edge_offsets[i] .. edge_offsets[i+1]) with its own ids (>= 0);
 * each graph is treated exactly as lf_graph_create + lf_run would treat it
 * alone: its own node order, global clustering coefficient cc, initial
 * clustering, queues of queue_size of its nodes, WCC-hat(P) and stopping test
 * (a graph that stops leaves the later queues).  Internally the graphs form
 * one disjoint union (ids shifted per graph; queue j holds the j-th
 * queue_size nodes of every active graph).
 * src, dst    : host, edge_offsets[num_graphs] entries each.
 * edge_offsets: host, num_graphs + 1 entries, [0] = 0, non-decreasing.
 * Errors: LF_ERR_INVALID (bad offsets, negative ids), LF_ERR_CAPACITY (the
 *         shifted ids or the edges exceed 2^31-1), LF_ERR_CUDA, LF_ERR_OOM.
 * The handle takes lf_run (not lf_run_partial or lf_set_partition), the
 * getters of one graph (over the union), and the lf_batch_get_* calls.
 */
lf_status lf_batch_create(const int32_t *src, const int32_t *dst, const int64_t *edge_offsets,
                          int64_t num_graphs, const lf_options *opt, lf_graph **out);

/*
 * lf_batch_get_info -- per graph of a batch (host arrays, any may be NULL):
 * node_offsets (num_graphs + 1: graph i's nodes are the union's dense ids
 * [node_offsets[i], node_offsets[i+1])), iterations run, converged (1/0),
 * WCC-hat(P) after the initial clustering and at the end, and cc.
 * LF_ERR_STATE if g is not a batch.
 */
lf_status lf_batch_get_info(lf_graph *g, int64_t *num_graphs, int64_t *node_offsets, int32_t *iterations,
                            int32_t *converged, double *wcc_initial, double *wcc_final, double *cc);

/* WCC-hat(P) after each iteration of one graph of a batch: *count values, at
 * most cap written to wcc. */
lf_status lf_batch_get_history(lf_graph *g, int64_t graph, double *wcc, int32_t cap, int32_t *count);

/*
 * lf_batch_get_communities -- lf_get_communities of a batch, with the members
 * in their own graph's ids and graph_offsets (num_graphs + 1 entries; may be
 * NULL) telling which communities belong to which graph: graph i's are
 * [graph_offsets[i], graph_offsets[i+1]).  Size queries as in
 * lf_get_communities.
 */
lf_status lf_batch_get_communities(lf_graph *g, int64_t *graph_offsets, int64_t *offsets, int64_t offsets_cap,
                                   int32_t *members, int64_t members_cap, int64_t *num_communities,
                                   int64_t *num_members);

/*
 * lf_autotune -- choose the launch shape of g's later runs by timing short
 * runs: warps per evaluated node (1, 2, 4 or the automatic choice) and the
 * degree above which a node is evaluated by a whole block instead of warps
 * (no limit, 96 or 192) and the degree above which it takes the hub path
 * (384 or 128) -- 24 shapes under LF_GAIN_MEANFIELD; under LF_GAIN_LITERAL
 * only the warps per node (4 shapes; the degree limits belong to the
 * mean-field kernels).  Every candidate computes the same result (the shape
 * changes only which threads do the work), so the choice affects speed only.
 * queue_size: the queue size the later runs will use; trial_iters (>= 1)
 * iterations per trial.  result (may be NULL): the chosen shape, its time and
 * the time of the default shape.  The state of g afterwards is that of the
 * last trial (run lf_run again for a result).
 */
typedef struct lf_tune_result {
    int32_t warps_per_node;    /* 0 = automatic */
    int32_t warp_max_degree;   /* 0 = no limit */
    int32_t trials;
    int32_t hub_degree;        /* degree above which a node takes the hub path */
    double best_ms;            /* device time of the chosen shape's trial */
    double default_ms;         /* device time of the default shape's trial */
} lf_tune_result;
lf_status lf_autotune(lf_graph *g, int32_t queue_size, int32_t trial_iters, lf_tune_result *result);

/*
 * Serving -- a request loop with continuous batching (not in the paper).  Jobs (one graph each, with its queue
 * size, threshold and iteration limit) are submitted at any time; up to
 * max_active worker threads admit them in arrival order while the device
 * memory estimated for the admitted jobs (from their edge counts) stays
 * within hbm_budget_bytes (a job larger than the budget runs alone), keep each
 * job's graph and community state resident on the device for its whole run,
 * and run the jobs side by side on their own streams, so their iterations
 * overlap on the device.  A job's communities are those lf_graph_create +
 * lf_run + lf_get_communities give for it alone.
 *   lf_server_create : opt may be NULL (defaults below).
 *   lf_server_submit : copies the edge list; *job_id identifies the job.
 *   lf_server_wait   : blocks until the job finished (timeout_s < 0: no limit,
 *                      else LF_ERR_TIMEOUT when it runs out); returns the job's
 *                      own status, with its result in *res (may be NULL).
 *   lf_server_get_communities: as lf_get_communities, for a finished job.
 *   lf_server_release: forgets a finished job's result.
 *   lf_server_destroy: drops the jobs not yet admitted (they finish with
 *                      LF_ERR_STATE), waits for the running ones and for the
 *                      threads inside lf_server_wait to return, frees
 *                      everything.  No call on the same server may start once
 *                      it has begun.
 * Times in lf_job_result are milliseconds since the server was created.
 */
typedef struct lf_server lf_server;
typedef struct lf_server_options {
    int64_t hbm_budget_bytes;   /* <= 0: half of the device memory free at creation */
    int32_t max_active;         /* jobs resident and running at once; < 1: 4 */
    int32_t pad;
} lf_server_options;
typedef struct lf_job_result {
    int32_t status;             /* lf_status of the job */
    int32_t iterations;
    int32_t converged;
    int32_t pad;
    double wcc_initial, wcc_final;
    int64_t num_nodes, num_edges, num_communities;
    int64_t est_bytes;          /* device memory the admission reserved for it */
    double t_submit_ms, t_admit_ms, t_done_ms;
} lf_job_result;
lf_status lf_server_create(const lf_server_options *opt, lf_server **out);
lf_status lf_server_submit(lf_server *s, const int32_t *src, const int32_t *dst, int64_t num_edges,
                           int32_t queue_size, double wcc_threshold, int32_t max_iters, int64_t *job_id);
lf_status lf_server_wait(lf_server *s, int64_t job_id, double timeout_s, lf_job_result *res);
lf_status lf_server_get_communities(lf_server *s, int64_t job_id, int64_t *offsets, int64_t offsets_cap,
                                    int32_t *members, int64_t members_cap, int64_t *num_communities,
                                    int64_t *num_members);
lf_status lf_server_release(lf_server *s, int64_t job_id);
void lf_server_destroy(lf_server *s);

/*
 * lf_cover_f1 -- F1-score of a detected cover against a reference cover
 * (Methods, Evaluation Criteria, F1-Score for Overlapping Communities): the
 * mean over detected communities C' of the largest F1(C', C) over reference
 * communities C, F1 = 2 (p r) / (p + r) with p = |C & C'| / |C'| and
 * r = |C & C'| / |C| (0 when they share no node), rounded operation by
 * operation in double precision; the mean is the correctly rounded sum
 * divided by the number of detected communities (0 for none).  Not
 * symmetric: the paper scores LazyFox's communities against Fox's or a
 * ground truth.  Computed on the GPU.
 * det_*, ref_*: host CSR covers (offsets num+1 entries from 0, members
 *               node ids >= 0, no community empty, no id twice in one).
 * best        : host, num_det entries or NULL: index of each detected
 *               community's best reference community (lowest on ties; -1
 *               when it shares no node with any).
 * stream      : cudaStream_t or NULL (a stream of the call's own).
 */
lf_status lf_cover_f1(const int64_t *det_offsets, const int32_t *det_members, int64_t num_det,
                      const int64_t *ref_offsets, const int32_t *ref_members, int64_t num_ref,
                      double *f1, int32_t *best, void *stream);

/*
 * lf_run_partial -- lf_run that stops after max_batches queues in total
 * (iteration ends run only for completed iterations), for per-queue parity
 * checks.  max_batches < 0 behaves like lf_run.
 */
lf_status lf_run_partial(lf_graph *g, int32_t queue_size, double wcc_threshold, int32_t max_iters,
                         int64_t max_batches, lf_run_stats *stats);

/*
 * lf_triangles_noalloc -- t(x,V) and vt(x,V) for callers that cannot allocate
 * device memory when they call: for example a program whose device memory is
 * owned entirely by another allocator, or a latency-critical loop in which an
 * allocation could stall or fail.  It runs the same triangle kernels as
 * lf_graph_create but allocates nothing: the kernels' working memory (edge
 * marks, hub list, counters) comes from one array of 16 MiB reserved
 * statically in this library, which every GPU that loads the library holds
 * until the process exits.  The paper has no counterpart of this call.
 * oriented_offsets: device, num_nodes+1 int64 offsets of a degree-ordered
 *                   orientation (as returned by lf_get_oriented): out-rows
 *                   ascending, every undirected edge exactly once;
 * out_neighbours  : device, num_edges int32;
 * t, vt           : device outputs, num_nodes each (overwritten);
 * stream          : cudaStream_t the work is queued on (NULL: legacy default).
 * Limit: num_edges + 4 num_nodes + ~1 KiB must fit in the 16 MiB array, else
 * LF_ERR_CAPACITY (nothing is launched).  The input is checked on the device
 * first (offsets from 0 to num_edges, non-decreasing, neighbour ids in
 * [0, num_nodes)); the call waits for that check (one 4-byte read) and
 * returns LF_ERR_INVALID for a malformed CSR without launching the counting.
 * Otherwise it returns when the counting is queued; results are ready when
 * the stream reaches them.  Because of that wait the call cannot be captured
 * in a CUDA graph.
 * Every call looks the array's device address up (with the call's device
 * current; the first call on a device also raises the kernels' shared-memory
 * limits).  Every call uses
 * the same array, which keeps the previous call's contents (the call clears
 * what must start at zero): calls whose work overlaps on a GPU race with each
 * other and must be ordered by the caller (e.g. one stream).
 */
lf_status lf_triangles_noalloc(const int64_t *oriented_offsets, const int32_t *out_neighbours,
                               int64_t num_nodes, int64_t num_edges, int64_t *t, int32_t *vt, void *stream);

/* Release every device buffer and the handle (NULL is a no-op). */
void lf_graph_destroy(lf_graph *g);

/* Message of the last failed call on this thread ("" if none). */
const char *lf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
