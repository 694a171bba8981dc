/*
 * gbbc.h - C ABI of libgbbc.so: exact Brandes betweenness centrality on one
 * GB300 (sm_103a), undirected graphs (unweighted, or with integer edge
 * weights: bc_graph_create_weighted), the whole graph in HBM.
 *
 * The problem statement follows Sec. II of the paper: the input is a graph
 * with N vertices and M edges and a set of sources (Algorithm 1's input);
 * the output is BC[v] = sum over sources s != v of delta_s(v) (Eq. 1, Eq. 2).
 * BC counts ordered pairs (s, t): no factor 1/2 for undirected graphs, and no
 * rescaling when only k < n sources are used.
 *
 * Conventions for every call
 *  - Every call returns a gbbc_status; nothing throws across this boundary.
 *    Output buffers are left untouched when the status is not GBBC_OK.
 *  - Pointers may point to host memory or to CUDA device memory of the
 *    current device; the library tells them apart with
 *    cudaPointerGetAttributes.  The caller owns all buffers it passes in;
 *    the library copies inputs before returning and owns all device memory
 *    it allocates (released by bc_graph_destroy into the library's pool,
 *    which bc_release_memory empties).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it; a call may synchronize it internally, and may run
 *    batches on streams of its own (joined back to `stream` before it
 *    returns).  One handle must not be used from two host threads at once,
 *    and calls on one handle are ordered on the stream given to them.
 *  - Device-side failures (queue capacity, sigma width, a bounded device
 *    wait that gave up) are detected by the library and reported as status
 *    codes; no kernel traps.
 *
 * Graph format: CSR with int32 row_ptr[n+1] and int32 col[nnz]; the graph
 * must be symmetric (undirected), with no self-loops and no duplicate
 * entries (a duplicate would count a path twice); rows need not be sorted
 * unless validation is on.  nnz < 2^31.
 */
#ifndef GBBC_H
#define GBBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbbc_graph gbbc_graph; /* opaque handle */

typedef enum gbbc_status {
    GBBC_OK = 0,
    GBBC_ERR_INVALID = 1,  /* bad argument or graph (see bc_last_error_detail) */
    GBBC_ERR_OOM = 2,      /* device allocation failed or mem_limit_bytes hit */
    GBBC_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    GBBC_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    GBBC_ERR_CAPACITY = 5, /* an internal queue or the sigma format overflowed */
    GBBC_ERR_STATE = 6     /* call not valid in the handle's current state */
} gbbc_status;

/* Direction policy of the forward phase (per level: top-down push from the
 * frontier or bottom-up pull into unvisited vertices). */
enum gbbc_policy {
    GBBC_POLICY_AUTO = 0,    /* learned policy if loaded, else threshold rule */
    GBBC_POLICY_BEAMER = 1,  /* threshold rule (Beamer, Asanovic, Patterson, SC'12) */
    GBBC_POLICY_LEARNED = 2, /* MLP loaded by bc_policy_load (error if none) */
    GBBC_POLICY_PUSH = 3,    /* always top-down */
    GBBC_POLICY_PULL = 4     /* bottom-up from level 1 on */
};

enum gbbc_flags {
    GBBC_KEEP_STATE = 1u << 0, /* keep per-source dist/sigma of the last
                                  bc_compute for bc_read_source_state */
    GBBC_TRACE = 1u << 1,      /* record per-level features and CUDA-event
                                  times (bc_get_trace, bc_get_profile) */
    GBBC_TRACE_BOTH = 1u << 2, /* with GBBC_TRACE: time both directions at
                                  every forward level (the step is run top-down,
                                  undone, then run bottom-up); results are
                                  unchanged, only slower */
    GBBC_DEVICE_LOOP = 1u << 3, /* grid schedule: run the level loop on the
                                  device, in one persistent cooperative launch
                                  per call (see GBBC_SCHEDULE_GRID); same bits */
    GBBC_SYNC_BACKWARD = 1u << 4 /* bc_compute_partitioned: level-synchronous
                                  backward over the whole graph instead of the
                                  asynchronous per-part backward; same bits */
};

typedef struct gbbc_options {
    uint32_t struct_size;  /* sizeof(gbbc_options); set by bc_options_init */
    int32_t batch_width;   /* sources per bitset word: 0 = automatic (64, or
                              tuned; see autotuning), 1 = plain
                              one-source-at-a-time kernels (with
                              GBBC_SCHEDULE_BLOCK: one source per thread
                              block, many blocks at once), 32 or 64 */
    int32_t policy;        /* enum gbbc_policy */
    int32_t validate;      /* 1: check CSR symmetry, sorted rows, no loops or
                              duplicates on the device at create time */
    int64_t timeout_spins; /* bound on any device-side wait, in polls of the
                              waited-for word (a poll takes about 0.1 us):
                              a grid barrier of the persistent grid schedule
                              that waits longer gives up, every block of the
                              launch returns, and the call fails with
                              GBBC_ERR_TIMEOUT (the handle's BC is then
                              undefined until bc_reset); 0 = default, 10^8 */
    uint32_t flags;        /* enum gbbc_flags */
    int32_t heavy_degree;  /* rows longer than this are split into chunk
                              tasks of 1024 entries, a thread block each;
                              0 = automatic: 1024, or tuned (see autotuning) */
    int64_t mem_limit_bytes; /* 0 = no limit; else allocations beyond this
                                many bytes fail with GBBC_ERR_OOM */
    int32_t schedule;      /* enum gbbc_schedule */
    int32_t streams;       /* batches the grid schedule runs at once, each on
                              its own stream and slot (BC summed exactly at
                              the end of the call): 0 = auto (8, fewer when
                              memory is short), 1 = one at a time, at most
                              16; tracing and kept state run one at a time */
} gbbc_options;

/* How batches are mapped to the GPU. */
enum gbbc_schedule {
    GBBC_SCHEDULE_AUTO = 0,  /* graphs above 65,536 vertices with average
                                degree at most 12 and a BFS eccentricity of at
                                least 64 (from a vertex of the largest row) run
                                pair when their sources in the call number at
                                most 8 per SM; batches of other graphs above 65,536
                                vertices with average degree above 6 run grid;
                                for the rest, block when the batches fill the
                                GPU, else the first call times some batches in
                                both modes (results kept) and the faster mode
                                is kept for the handle */
    GBBC_SCHEDULE_GRID = 1,  /* batches on the whole GPU.  By default the host
                                drives the level loop: a kernel per level
                                step, a counter read-back per level, up to
                                `streams` batches at once (8 by default) on
                                their own streams and host threads.  With
                                GBBC_DEVICE_LOOP (or when the autotuner picks
                                it) one persistent cooperative launch per call
                                runs the loop on the device instead: up to
                                `streams` batches in flight, each one level
                                step per tick, the ticks separated by
                                grid-wide barriers bounded by timeout_spins.
                                Tracing and kept state use the host loop */
    GBBC_SCHEDULE_BLOCK = 2, /* one thread-block cluster (1 to 8 blocks) per
                                batch, many batches at once, one persistent
                                launch per call; the level loop runs on the
                                device (cluster barriers only).  With
                                batch_width 1: each thread block runs whole
                                sources from the call's list, one at a time,
                                on per-block arrays of 28n bytes (as many
                                blocks as fit in half the free memory and
                                mem_limit_bytes, at most the resident count);
                                BC bits equal the other paths'; kept state and
                                tracing use the one-source-at-a-time kernels.
                                A source whose counts reach 2^64 adds nothing
                                and the call fails with GBBC_ERR_CAPACITY
                                after the other sources were added */
    GBBC_SCHEDULE_PAIR = 3   /* the weighted graphs' kernel with all weights
                                1: one block per batch of ceil(k / resident
                                blocks) sources (at most 64), work items
                                (vertex, source) pairs,
                                for graphs whose sources rarely share a BFS
                                level (high diameter); one launch per call.
                                BC agrees with the other schedules to
                                rounding, bit for bit while path counts stay
                                below 2^64 */
};

/*
 * Autotuning.  When batch_width and heavy_degree are both left automatic,
 * a handle's first call with at least 2560 sources on one graph of the grid
 * schedule (above 65,536 vertices, average degree above 6, or the grid
 * schedule chosen) times five launch configurations on spread blocks of 64
 * of its sources (width 64 with heavy-row thresholds 1024, 512, 2048; width
 * 32; the persistent kernel) and keeps the fastest for the handle
 * (bc_get_stats: batch_width, tuned_heavy_degree, tuned_device_loop); the
 * default (width 64, threshold 1024, host loop) stays unless another is more
 * than 3% faster.  The trial sources are part of the call's work; BC does
 * not depend on the configuration.
 */

/* Fill *opt with defaults (auto width, auto policy, no validation). */
void bc_options_init(gbbc_options* opt);

/*
 * Create a handle from one CSR graph (copied to the device).
 * n >= 0 vertices, nnz entries; row_ptr[n+1], col[nnz] (host or device).
 * opt may be NULL (defaults).  *out receives the handle.
 * Errors: GBBC_ERR_INVALID (n < 0, nnz out of range, row_ptr[0] != 0,
 * row_ptr[n] != nnz, or a failed validation), GBBC_ERR_OOM, GBBC_ERR_CUDA.
 */
gbbc_status bc_graph_create(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                            const gbbc_options* opt, void* stream, gbbc_graph** out);

/*
 * Create a handle over `count` independent graphs held as one disjoint union
 * (graph i's vertex v becomes offset_i + v).  n[i], nnz[i], row_ptr[i],
 * col[i] describe graph i (host arrays of pointers; the pointed-to CSR arrays
 * may be host or device).  BC of the union restricted to graph i equals BC
 * of graph i, because no path leaves a component.
 */
gbbc_status bc_graph_create_multi(int32_t count, const int32_t* n, const int64_t* nnz,
                                  const int32_t* const* row_ptr, const int32_t* const* col,
                                  const gbbc_options* opt, void* stream, gbbc_graph** out);

/*
 * Run Brandes' forward and backward phases for the k sources (vertex ids of
 * the whole handle, host or device int32[k]) and ADD their dependencies into
 * the handle's BC vector (Eq. 2: BC[v] += delta_s(v) for v != s).
 * Duplicated sources are counted with multiplicity.  BC accumulates across
 * calls until bc_reset.  Sources are packed into batches of the batch width
 * in list order; for a fixed list, width and policy the result is
 * bit-for-bit reproducible.
 * Errors: GBBC_ERR_INVALID (k < 0, a source outside [0, n)),
 * GBBC_ERR_CAPACITY, GBBC_ERR_TIMEOUT, GBBC_ERR_OOM, GBBC_ERR_CUDA.
 */
gbbc_status bc_compute(gbbc_graph* g, const int32_t* sources, int64_t k, void* stream);

/* bc_compute for a multi-graph handle: source j is vertex local_src[j] of
 * graph graph_id[j] (host or device arrays of k entries).  Sources of one
 * graph are batched together. */
gbbc_status bc_compute_multi(gbbc_graph* g, const int32_t* graph_id, const int32_t* local_src, int64_t k,
                             void* stream);

/*
 * Copy the accumulated BC into bc_out (host or device double[]): the whole
 * vector (n of the handle) when graph_id == -1, else graph graph_id's n
 * entries.  Synchronizes `stream`.
 */
gbbc_status bc_read(gbbc_graph* g, double* bc_out, int32_t graph_id, void* stream);

/*
 * The accumulated BC in its exact internal form: 128-bit unsigned fixed
 * point in units of 2^-64, as (low 64 bits, high 64 bits) pairs, 2 * n
 * uint64 values (host or device).  Sums of these integers are exact and
 * independent of order, so partial results computed on different GPUs (or
 * calls) over disjoint source sets add up to bit-identical totals; round
 * the sum to FP64 once, at the end.  graph_id as in bc_read.
 */
gbbc_status bc_read_fixed(gbbc_graph* g, uint64_t* out, int32_t graph_id, void* stream);

/*
 * Add a BC vector in the exact internal form (2 * n uint64 values as
 * bc_read_fixed gives them; host or device) into the handle's accumulated
 * BC: the whole vector when graph_id == -1, else graph graph_id's entries.
 * The adds are 128-bit integer adds with carry, exact and independent of
 * order, so partial results over disjoint source sets (computed by other
 * GPUs or other handles of the same graph, Eq. 2 being a sum over sources)
 * combine into exactly the bits one handle over all the sources holds;
 * bc_read then rounds the total to FP64 once.  Enqueued on `stream` and
 * synchronised before returning.
 * Errors: GBBC_ERR_INVALID (NULL partial, bad graph_id), GBBC_ERR_OOM (a
 * host partial needs a device staging buffer), GBBC_ERR_CUDA.
 */
gbbc_status bc_add_fixed(gbbc_graph* g, const uint64_t* partial, int32_t graph_id, void* stream);

/*
 * Per-source state of the last bc_compute, for sources in that call when
 * GBBC_KEEP_STATE was set: dist (int32[n], -1 unreachable), sigma (uint64[n],
 * number of shortest paths mod 2^64), overflow (uint8[n], 1 iff the true
 * count is >= 2^64).  source_index is the position in that call's list.
 * Any of the three pointers may be NULL.  Host or device buffers.
 * Errors: GBBC_ERR_STATE (no kept state), GBBC_ERR_INVALID (index).
 */
gbbc_status bc_read_source_state(gbbc_graph* g, int64_t source_index, int32_t* dist, uint64_t* sigma,
                                 uint8_t* overflow);

/* Zero the accumulated BC (kept state is dropped). */
gbbc_status bc_reset(gbbc_graph* g);

/* Synchronize the handle's last stream and return any deferred device error. */
gbbc_status bc_sync(gbbc_graph* g);

/* Release all device memory of the handle.  NULL is ignored. */
void bc_graph_destroy(gbbc_graph* g);

/* Static string naming a status code. */
const char* bc_status_string(gbbc_status s);

/* Copy a NUL-terminated description of the handle's last error into buf.
 * With g == NULL: the last failed bc_graph_create* call on this thread. */
gbbc_status bc_last_error_detail(const gbbc_graph* g, char* buf, size_t len);

/* Counters of the handle's work so far. */
typedef struct gbbc_stats {
    int64_t sources;        /* sources processed */
    int64_t batches;        /* batches run */
    int64_t levels_fwd;     /* forward levels summed over batches */
    int64_t levels_push;    /* forward levels run top-down */
    int64_t levels_pull;    /* forward levels run bottom-up */
    int64_t wide_batches;   /* batches that needed the wide sigma format */
    int64_t kernel_launches;/* kernels launched by the library */
    int64_t device_bytes;   /* device memory held by the handle */
    int32_t batch_width;    /* width in use */
    int32_t policy;         /* policy in use */
    int32_t schedule;       /* schedule of the last call (after autotuning;
                               0 when it mixed both) */
    int32_t block_slots;    /* concurrent batches of the block schedule */
    int64_t persist_launches; /* launches of the persistent grid-schedule kernel */
    double persist_ms;      /* their summed duration (CUDA events recorded on
                               the launch stream around each launch) */
    int32_t persist_slots;  /* batches in flight in the last such launch */
    int32_t persist_blocks; /* its cooperative grid */
    int32_t tuned_heavy_degree; /* heavy-row threshold the autotuner chose (0:
                               not tuned); batch_width holds its width */
    int32_t tuned_device_loop;  /* 1 when it chose the persistent kernel */
} gbbc_stats;

gbbc_status bc_get_stats(const gbbc_graph* g, gbbc_stats* out);

/*
 * Per-level trace (GBBC_TRACE): one record per forward step of every batch,
 * appended until bc_clear_trace.  A step at level l discovers level l+1.
 * "lanes" count (vertex, source) pairs; times are CUDA-event milliseconds on
 * the compute stream (-1 when not measured).
 */
typedef struct gbbc_level_trace {
    int32_t batch;              /* batch index since the handle was created */
    int32_t level;              /* l */
    int32_t direction;          /* step run: 0 top-down push, 1 bottom-up pull */
    int32_t active_lanes;       /* sources whose frontier is not empty */
    int64_t n_range;            /* vertices of the batch's graph */
    int64_t nnz_range;          /* CSR entries of the batch's graph */
    int64_t frontier_vertices;  /* vertices at level l in some lane */
    int64_t frontier_edges;     /* sum of their degrees */
    int64_t frontier_lanes;     /* (vertex, lane) pairs at level l */
    int64_t visited_lanes;      /* (vertex, lane) pairs at levels <= l */
    int64_t visited_lane_edges; /* sum of degree over those pairs */
    int64_t max_degree;         /* largest degree in the graph */
    int64_t next_vertices;      /* vertices at level l+1 in some lane */
    int64_t next_edges;         /* sum of their degrees */
    int64_t scanned_edges;      /* CSR entries read by a bottom-up step */
    float ms_push;              /* top-down discovery time */
    float ms_pull;              /* bottom-up discovery time */
    float ms_gather;            /* sigma gather of level l+1 */
    float ms_backward;          /* backward step of level l+1 */
    float features[6];          /* direction-policy features of this step:
                                   log-scaled frontier popcount, frontier edge
                                   sum, unvisited (vertex, lane) pairs, level,
                                   degree mean, degree max (see bc_policy_eval) */
} gbbc_level_trace;

/* Copy up to max records into out; *count receives the number available. */
gbbc_status bc_get_trace(const gbbc_graph* g, gbbc_level_trace* out, int64_t max, int64_t* count);
gbbc_status bc_clear_trace(gbbc_graph* g);

/*
 * Per-step-kind profile (GBBC_TRACE): CUDA-event time and algorithmic bytes
 * summed over all launches since the last bc_clear_trace.  Kinds: "push",
 * "pull", "gather", "backward", "init".  Algorithmic bytes follow a
 * compulsory-traffic model: each CSR row, mask word, sigma and coefficient
 * the step needs is counted once per step.
 */
typedef struct gbbc_kernel_profile {
    char name[32];
    int64_t launches;  /* steps of this kind (each is one warp-per-row and one
                          block-per-row kernel, two plus a filter for pull) */
    double ms;         /* summed CUDA-event time */
    double bytes;      /* summed algorithmic bytes */
} gbbc_kernel_profile;

gbbc_status bc_get_profile(const gbbc_graph* g, gbbc_kernel_profile* out, int32_t max, int32_t* count);

/*
 * Learned direction policy.  A multilayer perceptron 6 -> 32 -> 32 -> K
 * (ReLU hidden layers) with FP32 parameters laid out as W1[32][6], b1[32],
 * W2[32][32], b2[32], W3[K][32], b3[K].  For the direction head K = 2
 * (logits of top-down push and bottom-up pull; the larger wins).  Its inputs
 * are the six features of gbbc_level_trace.features.  The network only
 * chooses the schedule: BC, dist and sigma do not depend on it.  The paper
 * has no learned component; its nearest analogue is choosing the CPU:GPU
 * split from measured run times (Sec. V-D).
 *
 * bc_mlp_* run on the device: params, x (n x 6, row-major), target, weight,
 * out, grad, loss pointers are DEVICE memory (FP32); they synchronize the
 * stream before returning.
 */
int64_t bc_mlp_param_count(int32_t k_out);  /* -1 if k_out is not 1 or 2 */

/* out[n][k_out] = network(x) in FP32. */
gbbc_status bc_mlp_forward(const float* params, int32_t k_out, const float* x, int64_t n, float* out, void* stream);

/*
 * Loss and its gradient over n samples (full batch).  loss_kind 0: softmax
 * cross-entropy with target[i] the class index (k_out = 2); loss_kind 1:
 * squared error against target[i] (k_out = 1).  Sample i is weighted by
 * weight[i] / sum(weight) (weight may be NULL: equal weights).  grad has
 * bc_mlp_param_count(k_out) entries; *loss_out (device, may be NULL) gets
 * the loss.  Sums over samples run in sample order: deterministic.
 */
gbbc_status bc_mlp_loss_grad(const float* params, int32_t k_out, const float* x, const float* target,
                             const float* weight, int64_t n, int32_t loss_kind, float* grad, float* loss_out,
                             void* stream);

/* One Adam step (Kingma and Ba, ICLR 2015) with bias correction at step t >= 1. */
gbbc_status bc_mlp_adam_step(float* params, const float* grad, float* m, float* v, int64_t count, float lr,
                             float beta1, float beta2, float eps, int32_t t, void* stream);

/* epochs of full-batch Adam (beta 0.9/0.999, eps 1e-8) from the given params;
 * loss_history (device, may be NULL) receives the loss before each step. */
gbbc_status bc_mlp_train(float* params, int32_t k_out, const float* x, const float* target, const float* weight,
                         int64_t n, int32_t loss_kind, int32_t epochs, float lr, float* loss_history, void* stream);

/* The level loop's inference path on n feature vectors: FP16 weights, FP32
 * sums.  logits[n][2] and choice[n] (0 push, 1 pull) may be NULL. */
gbbc_status bc_policy_eval(const float* params, const float* x, int64_t n, float* logits, int32_t* choice,
                           void* stream);

/* Load a direction network (FP32 params, host or device, bytes =
 * bc_mlp_param_count(2) * 4) into the handle; GBBC_POLICY_AUTO then uses it
 * and GBBC_POLICY_LEARNED requires it.  params == NULL unloads it. */
gbbc_status bc_policy_load(gbbc_graph* g, const float* params, size_t bytes);

/*
 * bc_graph_create_weighted - a weighted graph: as bc_graph_create, plus
 * weight[nnz] (host or device, copied), the positive integer length of each
 * CSR entry's edge, in [1, GBBC_MAX_WEIGHT]; both entries of an edge must
 * carry the same weight (checked when opt->validate is set).  Shortest paths
 * are then those of least total weight (the SSSP case of the paper's forward
 * phase, Sec. IV-C) and bc_compute adds Eq. 2's dependencies along them.
 * The weighted path runs 64 sources per batch on one CTA each (batch_width 1
 * is rejected; 32 runs as 64), ignores the direction policy, grouping and
 * tracing, and keeps per-source state under GBBC_KEEP_STATE (distances as
 * int32).  A shortest-path count reaching 2^64 fails bc_compute with
 * GBBC_ERR_CAPACITY (no wide format here).  GBBC_ERR_INVALID also when
 * max weight * (n - 1) may exceed the int32 distance range.
 */
#define GBBC_MAX_WEIGHT 64
gbbc_status bc_graph_create_weighted(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                                     const int32_t* weight, const gbbc_options* opt, void* stream,
                                     gbbc_graph** out);

/*
 * bc_release_memory - the library takes device memory from one pool per
 * device and keeps what destroyed handles free (so the next handle's
 * allocations are immediate).  This returns the unused part of device's pool
 * (-1: the current device) to the driver.  Synchronises the device.
 */
gbbc_status bc_release_memory(int32_t device);

/*
 * Learned source grouping.  A network of the same shape with K = 1 output
 * scores each source from six features (bc_source_features: log-scaled
 * degree of s, sum and maximum of its neighbours' degrees, and the size,
 * mean degree and maximum degree of its graph); it is trained to predict the
 * source's mean BFS distance.  With weights loaded, bc_compute orders each
 * graph's sources by score (stable) before packing them into words, so that
 * sources whose levels line up share a word (and isolated sources fill words
 * of their own).  The order changes the batches, never the BC bits.  It is
 * not applied when GBBC_KEEP_STATE is set (kept state follows list order).
 */
gbbc_status bc_source_features(gbbc_graph* g, const int32_t* sources, int64_t k, float* out /* k x 6 */,
                               void* stream);
/* bytes = bc_mlp_param_count(1) * 4 FP32 params (host or device); NULL unloads. */
gbbc_status bc_grouping_load(gbbc_graph* g, const float* params, size_t bytes);
/* The loaded network's score of each source (the key bc_compute sorts by);
 * GBBC_ERR_STATE when no grouping weights are loaded. */
gbbc_status bc_grouping_scores(gbbc_graph* g, const int32_t* sources, int64_t k, float* out, void* stream);

/*
 * The partitioned method (Sec. IV and Sec. V-A).  The paper splits a graph
 * too large for one device into a CPU part and a GPU part; here the P parts
 * live on one GPU, and the method reaches exactly the results of
 * bc_compute.  A border edge joins two parts; its end points are border
 * nodes.
 *
 * bc_partition: part[v] in [0, P) for each of the handle's n vertices (host
 * or device int32), or part == NULL for P contiguous ranges of vertex ids.
 * Builds, once, the intra-part graph (border edges removed), the border
 * edges, the border nodes of every part (by part, then vertex id), and the
 * border matrices (Sec. IV-B): BM_p[i][j] = length of a shortest path from
 * border node i to border node j of part p inside p (-1: none), and
 * sigmaM_p[i][j] = the number of such paths (Sec. V-A), by BFS inside the
 * part from every border node.  Single-graph, unweighted handles only;
 * 1 <= P <= 32.
 * Errors: GBBC_ERR_INVALID (weighted or multi-graph handle, P, part values),
 * GBBC_ERR_OOM (the border matrices, sum of |B_p|^2 entries, do not fit).
 */
gbbc_status bc_partition(gbbc_graph* g, const int32_t* part, int32_t P, void* stream);

typedef struct gbbc_partition_info {
    int32_t parts;             /* P (0: not partitioned) */
    int64_t border_nodes;      /* over all parts */
    int64_t border_edges;      /* CSR entries joining two parts */
    int64_t intra_entries;     /* CSR entries inside parts */
    int64_t matrix_entries;    /* sum over parts of |B_p|^2 */
    int64_t refinement_sweeps; /* Steps 2-5 sweeps of the last bc_compute_partitioned */
    int64_t backward_waits;    /* waits of one part for another in the asynchronous
                                  backward phases of that call */
} gbbc_partition_info;

gbbc_status bc_partition_info(const gbbc_graph* g, gbbc_partition_info* out);

/* Part p's border-node count (*nodes = |B_p|, host), border nodes
 * (int32[|B_p|], sorted vertex ids), BM (int32, row-major |B_p| x |B_p|),
 * sigmaM mod 2^64 (uint64) and its overflow flags (uint8: 1 when the count
 * is >= 2^64); any pointer may be NULL; host or device buffers.
 * Errors: GBBC_ERR_STATE (no partition), GBBC_ERR_INVALID. */
gbbc_status bc_read_border_matrix(gbbc_graph* g, int32_t p, int64_t* nodes, int32_t* border, int32_t* bm,
                                  uint64_t* sigma_m, uint8_t* overflow);

/*
 * bc_compute by the partitioned method (after bc_partition), per batch of
 * 64 sources in list order:
 *   Step 1     BFS with sigma from each source inside its part (Sec. IV-C);
 *   Steps 2-5  the border nodes' distances refined over the border edges
 *              (Steps 2, 4) and the border matrices (Steps 3, 5), in sweeps
 *              over all parts until no distance changes;
 *   sigma      of every border node b: the paths that stay in the source's
 *              part (Step 1's count, when Step 1 found the final distance)
 *              plus, for each border node b' of b's part, the paths whose
 *              last border edge enters at b' (the sum of sigma over the
 *              border neighbours of b' one level up) times sigmaM[b'][b]
 *              when BM[b'][b] closes the distance (Sec. V-A);
 *   Step 6     relaxation: BFS inside every part from the source and from
 *              the border nodes entering at their refined distances with
 *              those counts, giving every vertex its distance and sigma;
 * then the asynchronous backward phase (Sec. V-B, Eq. 2): each part walks
 * its own levels, deepest first, on its own group of blocks of one
 * cooperative launch, and waits for another part only at a level where one
 * of its border nodes has a successor in that part one level deeper, until
 * that part has finished the deeper level (every wait bounded by
 * timeout_spins: GBBC_ERR_TIMEOUT, the handle's BC then undefined until
 * bc_reset); with GBBC_SYNC_BACKWARD the backward runs level-synchronously
 * over the whole graph instead.  At most 32 parts.  dist and sigma (mod
 * 2^64, with the overflow flag) equal bc_compute's bit for bit, and so does
 * BC while counts stay below 2^64 (beyond, the wide counts are products
 * rounded to 64-bit mantissas: BC agrees to rounding).  GBBC_KEEP_STATE
 * keeps per-source state as for bc_compute.  Sources are not reordered and
 * the grid schedule's host loop runs each step.
 * Errors: GBBC_ERR_STATE (no partition), GBBC_ERR_INVALID, GBBC_ERR_CAPACITY,
 * GBBC_ERR_OOM, GBBC_ERR_CUDA.
 */
gbbc_status bc_compute_partitioned(gbbc_graph* g, const int32_t* sources, int64_t k, void* stream);

/*
 * bc_compute_noalloc - BC of one small graph with no memory allocation.
 * The paper has no counterpart; this entry point exists for callers that
 * must not allocate memory themselves (code running under a pool allocator
 * that owns the whole device, plug-in hosts whose allocator may not be
 * bypassed, real-time loops that cannot afford cudaMalloc's implicit
 * synchronisation).  It calls no cudaMalloc/cudaFree and no allocating
 * library routine, creates no handle and keeps nothing on the caller's
 * stack beyond a few words (worker threads of plug-in hosts often have
 * small stacks).
 *
 * Working state lives in one static device array of the library, sized for
 * GBBC_NOALLOC_MAX_VERTICES vertices (about 48 MiB); every GPU that loads
 * libgbbc.so holds it until the process exits.  All calls share it, so the
 * work of two calls must never overlap on the GPU: the library serialises
 * calls on one device with a host lock held for the whole call, and a call
 * returns only after its work on `stream` has finished.  The array keeps the
 * previous call's contents; each call and each batch clears what must start
 * at zero.  The first call on a device looks up the array's device address
 * with cudaGetSymbolAddress (once per device, with that device current).
 * The call synchronises `stream` and copies between pageable host memory
 * and the device, so it must not be called while `stream` (or the legacy
 * default stream) is being captured into a CUDA graph.
 *
 * Inputs: n <= GBBC_NOALLOC_MAX_VERTICES vertices; row_ptr[n+1], col[nnz]
 * and bc_out[n] in DEVICE memory; sources[k] in HOST memory, each in [0, n).
 * The CSR must be symmetric with sorted rows and no self-loops or duplicate
 * entries, and row_ptr[0] = 0, row_ptr[n] = nnz: every call checks this on
 * the device (in the static array) before any other kernel reads col.
 * The dependencies of the k sources are ADDED into bc_out (zero it first for
 * plain BC), in 64-source batches, always expanding top-down.
 * Errors: GBBC_ERR_CAPACITY when n exceeds GBBC_NOALLOC_MAX_VERTICES or a
 * shortest-path count reaches 2^64 (bc_out is then left unchanged),
 * GBBC_ERR_INVALID for bad arguments, a CSR that fails the check, or
 * pointers in the wrong memory, GBBC_ERR_CUDA.
 */
#define GBBC_NOALLOC_MAX_VERTICES 16384
gbbc_status bc_compute_noalloc(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                               const int32_t* sources, int64_t k, double* bc_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GBBC_H */
