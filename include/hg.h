/*
 * hg.h - C ABI of the GB300 deterministic hypergraph coarsening and
 * label-propagation library (Mt-KaHyPar's deterministic multilevel path,
 * arXiv 2303.17679).
 *
 * The library holds a level hierarchy H_0 (the input) ... H_L in device
 * memory and offers the per-level operations of Algorithm 1: one
 * deterministic clustering + contraction step, the seeded initial partition,
 * projection, and deterministic lambda-1 label propagation with the objective.
 *
 * Conventions for every entry point:
 *  - Return value: HG_OK (0) on success, HG_STOP (1) where documented, a
 *    negative HG_ERR_* code otherwise.  No C++ exception crosses the ABI.
 *  - Integer types: node, net and block ids, node and net weights are int32;
 *    pin offsets are int32 (so fewer than 2^31 pins); objectives, block
 *    weights and move counts are int64.
 *  - Memory: "host" pointers are ordinary CPU memory, "device" pointers are
 *    CUDA global memory of the device current at hg_create.  The caller owns
 *    every pointer it passes and keeps it valid for the duration of the call;
 *    the library copies what it keeps.  The handle owns all device memory of
 *    the hierarchy and frees it in hg_destroy.
 *  - Streams: all work is issued on the stream given to hg_create, in
 *    stream order.  Entry points that return host scalars synchronize that
 *    stream before returning.  One handle must not be used from two host
 *    threads at once.
 *  - Errors: HG_ERR_INVALID for malformed arguments (nothing is changed),
 *    HG_ERR_UNSUPPORTED for sizes outside the supported range, HG_ERR_OOM
 *    when device memory runs out, HG_ERR_CUDA for a CUDA error (sticky: the
 *    handle then only accepts hg_destroy and the query calls), HG_ERR_TIMEOUT
 *    when a bounded device-side wait gave up, HG_ERR_STATE for calls out of
 *    order (for example refining a level that does not exist).
 *  - Determinism: for the same inputs and options every output is bit-identical
 *    from run to run, whatever the launch configuration (Sec. 11).
 */
#ifndef HG_H
#define HG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HG_OK 0
#define HG_STOP 1
#define HG_ERR_INVALID (-1)
#define HG_ERR_UNSUPPORTED (-2)
#define HG_ERR_OOM (-3)
#define HG_ERR_CUDA (-4)
#define HG_ERR_TIMEOUT (-5)
#define HG_ERR_STATE (-6)

#define HG_MEM_HOST 0
#define HG_MEM_DEVICE 1

#define HG_MAX_K 64

typedef struct hg_t hg_t;

/* Options fixed for the lifetime of a handle. */
typedef struct {
  /* Seed of every hashed decision: sub-round of a node (Sec. 11, synchronous
   * local moving in sub-rounds) and the order of the initial partition. */
  uint64_t seed;
  /* S: number of sub-rounds of one clustering round and of one label-
   * propagation pass (Sec. 11).  1 <= S <= 256.  Default 16. */
  int32_t subrounds;
  /* T: nets with more than T pins are skipped by the rating function but kept
   * everywhere else.  2 <= T <= 2^20.  Default 1000. */
  int32_t rating_max_net_size;
  /* f in the contraction limit f*k and in c_max = ceil(c(V) / (f*k))
   * (Sec. 4.1, "Contraction Limit"; the paper uses 160).  Default 160. */
  int32_t contraction_limit_factor;
  /* Number of bits kept of the identical-net fingerprint (0 = all 64).  A
   * test knob: fewer bits force fingerprint collisions, which the exact pin
   * comparison must resolve; results do not change, only the work. */
  int32_t fingerprint_bits;
  /* Optional device allocator (for example a framework's caching allocator).
   * Both NULL: stream-ordered allocations (cudaMallocFromPoolAsync /
   * cudaFreeAsync) from the library's own memory pool of the device, which
   * keeps freed blocks for later handles (hg_trim_memory returns them to the
   * driver); the device's default pool is not touched. */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  /* Launch mapping, the autotuner's knobs (0 = built-in default).  Results
   * never depend on them: every mapping computes the same integer sums and
   * the same picks.  A rated node with D = min(W(u), n) distinct-candidate
   * bound (W(u) = pins of its rated nets) goes to the first team whose bound
   * holds: one warp (rate_warp_max_d, <= 256, default 256), four warps
   * (rate_pair_max_d, <= 1024, default 1024), eight warps (rate_quad_max_d,
   * <= 2048, default 2048), sixteen warps (rate_block_max_d, <= 4096,
   * default 4096), else the grid-split path.  In label propagation, nodes
   * with more than lp_block_min_deg incident nets (default 64, <= 2^20) are
   * evaluated by a block of sixteen warps, the others by one warp. */
  int32_t rate_warp_max_d;
  int32_t rate_pair_max_d;
  int32_t rate_quad_max_d;
  int32_t rate_block_max_d;
  int32_t lp_block_min_deg;
  /* 1: wait for the device by sleeping on a blocking-sync event instead of
   * spinning (frees the host core while waiting, at a few microseconds of
   * wake-up latency per wait; the executor sets it for its jobs).  0 (default):
   * spin. */
  int32_t blocking_sync;
  /* Graph path (Sec. 10): 0 (default) = a level whose nets all have exactly
   * two pins is kept as a graph with one adjacency array (the other endpoint
   * and the edge weight of every incidence); its rating reads neighbours
   * directly (no per-net deduplication is needed), and its label propagation
   * computes g(u, t) = w(u, V_t) - w(u, V_Pi(u)) from the neighbours' blocks
   * without pin counts.  Contraction keeps a graph a graph.  1 = always use
   * the hypergraph path.  Results are identical either way. */
  int32_t graph_path;
  /* 1: hg_partition first detects communities (hg_detect_communities) and
   * keeps every contraction inside a community.  0 (default): off. */
  int32_t community_detection;
} hg_options;

/* Per-phase device time (milliseconds, from CUDA events) and work counters,
 * accumulated since hg_create or the last hg_reset_stats.  Phases are only
 * timed when hg_enable_timing(h, 1) was called. */
typedef struct {
  double ms_transpose;  /* incidence build (a1) */
  double ms_rating;     /* heavy-edge rating of all sub-rounds (a3) */
  double ms_approve;    /* cluster approval of all sub-rounds (a4) */
  double ms_contract;   /* map, remap, identical nets, compaction (a5-a8) */
  double ms_project;    /* projection (a9) */
  double ms_phi;        /* pin counts, connectivity sets, block weights (a10) */
  double ms_lp_gain;    /* label-propagation best moves (a11) */
  double ms_lp_select;  /* move gathering or bucketing and prefix selection (a12) */
  double ms_lp_apply;   /* move application (a13) */
  double ms_objective;  /* objective (a14) */
  double ms_initial;    /* host initial partition incl. copies */
  int64_t launches;     /* kernels launched */
  int64_t rating_launches;
  int64_t rating_pin_visits;  /* pins read by the rating kernels */
  int64_t rating_nodes;       /* nodes rated */
  int64_t rating_incidences;  /* incident nets read by the rating kernels */
  int64_t lp_incidences;      /* incident nets read by the gain kernels */
  int64_t lp_nodes;           /* nodes evaluated by the gain kernels */
  int64_t lp_gain_launches;
  double ms_rating_kernels;   /* sum of rating kernel durations (timing on) */
  double ms_lp_gain_kernels;  /* best-move kernel duration (timing flag 2; inside a captured
                                 pass the two parallel branches count once) */
  double ms_rating_refresh;   /* per-sub-round refresh of the deduplicated pin clusters */
  double ms_rating_class[8];  /* rating kernel time per node class (timing flag 2) */
  int64_t rating_visits_class[8]; /* pin visits per node class */
  double ms_lp_select_kernels; /* bucketing and pair selection duration (timing flag 2) */
  double ms_lp_apply_kernels;  /* move application duration (timing flag 2) */
  int64_t lp_moved_incidences; /* incident nets of the moved nodes */
  int64_t lp_passes;           /* label-propagation passes run */
  int64_t timing_failures;     /* kernel-timing event pairs that could not be read */
  double ms_communities;       /* community detection (timing flag 1) */
  int64_t louvain_levels;      /* Louvain levels aggregated */
  int64_t louvain_rounds;      /* local-moving rounds */
  int64_t louvain_moves;       /* vertex moves of the local moving */
} hg_stats;

/* Fills *opt with the defaults listed above (seed 1). */
void hg_default_options(hg_options* opt);

/* Creates a handle holding level 0 = the input hypergraph H = (V, E, c, w)
 * of Sec. 2 in net-major CSR: the pins of net e are
 * pins[net_offsets[e] .. net_offsets[e+1]).
 *   n, m          nodes and nets, n >= 1, m >= 0
 *   net_offsets   m+1 entries, net_offsets[0] = 0, non-decreasing
 *   pins          net_offsets[m] entries in [0, n); no node twice in a net;
 *                 nets may not be empty
 *   net_weights   m entries > 0, or NULL for all 1
 *   node_weights  n entries > 0, or NULL for all 1
 *   mem           HG_MEM_HOST or HG_MEM_DEVICE: where the four arrays live
 *   opt           options, or NULL for the defaults
 *   cuda_stream   cudaStream_t to issue all work on (NULL = legacy default)
 * Builds the incident-net lists I(u) on the device (a1).  Rejects with
 * HG_ERR_INVALID: bad sizes or offsets, pins out of range, repeated pins in
 * a net, empty nets, weights <= 0, total node or net weight >= 2^31
 * (host inputs: up to 65,536 pins checked on the host; up to 4,194,304
 * pins offsets and weights on the host and pins on the device after the
 * upload; larger host inputs and all device inputs on the device right after
 * the upload).  *out is NULL on failure. */
int hg_create(int32_t n, int32_t m, const int32_t* net_offsets, const int32_t* pins,
              const int32_t* net_weights, const int32_t* node_weights, int32_t mem,
              const hg_options* opt, void* cuda_stream, hg_t** out);

/* One deterministic clustering + contraction step (Sec. 4.1, Sec. 4.2,
 * Sec. 11 "Deterministic Clustering for Coarsening") on the coarsest level
 * built so far, producing a new resident level.  k (2..64) sets the
 * contraction limit f*k and c_max = ceil(c(V) / (f*k)).
 * Returns HG_STOP without building a level when the coarsest level has at
 * most f*k nodes, or when the previous step shrank the node count by less
 * than 1 % (that level is kept).  On HG_OK the out-parameters (each may be
 * NULL) receive the new level's index and sizes. */
int hg_coarsen_level(hg_t* h, int32_t k, int32_t* out_level, int32_t* out_n, int32_t* out_m,
                     int64_t* out_p);

/* 1 in *out_graph when the level runs on the graph path (see
 * hg_options.graph_path), else 0. */
int hg_level_is_graph(const hg_t* h, int32_t level, int32_t* out_graph);

/* Number of levels held (1 + coarsening steps done) and the sizes of one. */
int hg_num_levels(const hg_t* h, int32_t* out_levels);
int hg_level_info(const hg_t* h, int32_t level, int32_t* out_n, int32_t* out_m, int64_t* out_p);

/* Seeded initial partition of a level (the paper's portfolio of Sec. 5 is
 * replaced by one deterministic rule): nodes in order of
 * (mix64(seed ^ 2^63 ^ u), u), each to the lightest block so far, ties to the
 * smaller block id; mix64 = the SplitMix64 output function.  Computed on the
 * host from the level's node weights.  part: device, n_level int32, written. */
int hg_initial_partition(hg_t* h, int32_t level, int32_t k, int32_t* part);

/* Projection Pi_l[u] = Pi_{l+1}[map(u)] from level coarse_level (>= 1) to
 * coarse_level - 1 (Algorithm 1, uncoarsening).  Both device int32 arrays;
 * coarse_part has n_{coarse_level} entries, fine_part n_{coarse_level-1}. */
int hg_project(hg_t* h, int32_t coarse_level, const int32_t* coarse_part, int32_t* fine_part);

/* Deterministic lambda-1 label propagation on one level (Sec. 11
 * "Deterministic Label Propagation Refinement", gain of Sec. 6): up to
 * max_passes passes of S sub-rounds; each node of a sub-round proposes its
 * best positive-gain move from the sub-round's starting state; per block pair
 * the moves are ordered by (gain desc, id asc) and the last feasible prefix
 * pair on the merge path is applied, with per-pair slack
 * floor(max(0, L_max - c(V_i)) / (k-1)) and
 * L_max = floor(ceil(c(V)/k) * (10^6 + eps_ppm) / 10^6) (Sec. 2).  A pass
 * that applies no move ends the call.
 *   part           device, n_level int32 in [0, k), read and updated in place
 *   out_objective  host, may be NULL: f_{lambda-1} after refinement
 *   out_moves      host, may be NULL: moves applied
 * k in 2..64, eps_ppm >= 0, max_passes >= 0.  Synchronizes the stream. */
int hg_lp_refine(hg_t* h, int32_t level, int32_t k, int32_t eps_ppm, int32_t max_passes,
                 int32_t* part, int64_t* out_objective, int64_t* out_moves);

/* Connectivity objective f_{lambda-1} = sum over nets of (lambda(e)-1) w(e)
 * (Sec. 2) of a partition (device int32, n_level entries in [0, k)) into
 * *out (host).  k in 1..64.  Synchronizes the stream. */
int hg_objective(hg_t* h, int32_t level, int32_t k, const int32_t* part, int64_t* out);

/* Pin counts Phi(e, V_i) (host m x k int32, may be NULL), connectivity sets
 * Lambda(e) as bit masks (host m uint64, may be NULL) and block weights c(V_i)
 * (host k int64, may be NULL) of a partition (device) - for inspection. */
int hg_pin_counts(hg_t* h, int32_t level, int32_t k, const int32_t* part, int32_t* phi,
                  uint64_t* lambda, int64_t* block_weights);

/* Exact gains of a move sequence (Sec. 6.3, "The Parallel Gain Recalculation
 * Algorithm", Algorithm 4).  Move i moves node move_nodes[i] from its block
 * in `part` to move_targets[i]; the moves are taken in index order and every
 * node moves at most once.  gains[i] = the objective decrease (Sec. 2) that
 * move i causes after moves 0 .. i-1, so the gains sum to
 * f(part) - f(part after all moves).  Computed per net over the nets of the
 * moved nodes; `part` is not changed.
 *   level         a level held by the handle
 *   k             2..64; part has n_level device int32 entries in [0, k)
 *   num_moves     0..n_level
 *   move_nodes, move_targets  device, num_moves int32 each
 *   gains         device, num_moves int64, written
 * HG_ERR_INVALID for a node moved twice, a node or target out of range, a
 * target equal to the node's block, or a block id in `part` out of range
 * (checked on the device; the handle stays usable).  Synchronizes the stream. */
int hg_recalculate_gains(hg_t* h, int32_t level, int32_t k, const int32_t* part,
                         int32_t num_moves, const int32_t* move_nodes,
                         const int32_t* move_targets, int64_t* gains);

/* Gain table (Sec. 6.2, "The Gain Table"): benefit b(u) = w of the nets of
 * u in which u is the only pin of its block, penalty p(u, V_i) = w of the
 * nets of u without a pin in V_i; the gain of Sec. 6 is b(u) - p(u, V_t).
 *   part      device, n_level int32 in [0, k) (k in 2..64)
 *   benefit   device, n_level int64, written
 *   penalty   device, n_level x k int64 (row per node), written
 * HG_ERR_INVALID for a block id out of range.  Synchronizes the stream. */
int hg_gain_table(hg_t* h, int32_t level, int32_t k, const int32_t* part, int64_t* benefit,
                  int64_t* penalty);

/* Moves move_nodes[i] to move_targets[i] for all i at once (every node at
 * most once, each target in [0, k) and not the node's block), updating
 * `part` in place and the gain table (benefit, penalty: the table of `part`
 * on entry, as hg_gain_table writes it) with the update rules of Sec. 6.2
 * applied concurrently; afterwards the benefits of the moved nodes are
 * recomputed (Sec. 6.2, "Benefit Peculiarities"), so the table equals
 * hg_gain_table of the new partition.  Same arguments and errors as
 * hg_gain_table plus those of hg_recalculate_gains for the moves (nothing
 * is changed when the moves are bad).  Synchronizes the stream. */
int hg_gain_table_move(hg_t* h, int32_t level, int32_t k, int32_t* part, int32_t num_moves,
                       const int32_t* move_nodes, const int32_t* move_targets, int64_t* benefit,
                       int64_t* penalty);

/* The connectivity objective (for every net, its weight times the number of
 * blocks its pins lie in minus one, summed over the nets) and the weight of
 * every block, for a partition of a hypergraph that the caller holds in
 * device memory, with no handle and without allocating device memory.  The
 * paper has no counterpart.  It serves callers that cannot allocate: a
 * serving loop in which a cudaMalloc/cudaFree would synchronize the device
 * and stall the other streams, a process that reserved all device memory up
 * front, or code running inside an hg_options.dev_alloc callback, which must
 * not re-enter the allocator.
 *   n, m, p       nodes (>= 1), nets (>= 0), pins (0 <= p < 2^31)
 *   net_offsets   device, m+1 int32 entries in [0, p], non-decreasing
 *   pins          device, p int32 entries in [0, n) (NULL when p == 0)
 *   net_weights   device, m int32 entries, or NULL for all 1
 *   node_weights  device, n int32 entries, or NULL for all 1
 *   k             1..64
 *   part          device, n int32 entries in [0, k)
 *   cuda_stream   cudaStream_t to run on (NULL = legacy default stream)
 *   out_objective host, written; an empty net counts 0
 *   out_block_weights host, k int64 entries written, or NULL
 * Scratch: a fixed 9,248-byte device array inside the library (1024 block
 * partials, 64 block-weight counters, a finished-block counter, a status word
 * and a result record), enough for any n, m and p since the grid is capped
 * at 1024 blocks.  Every GPU that loads the library holds it until the
 * process exits.  Returns HG_ERR_UNSUPPORTED for k > 64 (the scratch holds
 * 64 block-weight counters), HG_ERR_INVALID for other bad sizes or NULL
 * pointers (checked on the host, nothing launched) and for offsets, pins or
 * block ids out of range (checked on the device; the call then returns
 * after the kernel without writing the outputs), HG_ERR_CUDA / HG_ERR_OOM for
 * a CUDA error (also when the kernel did not complete).  Synchronizes the
 * stream.
 * The first call on a device loads the library's device code there; make it
 * before any stream capture begins.  The scratch is shared by all calls on a
 * device and keeps the last call's contents (each call clears what must
 * start at zero): calls that overlap in time on one device (from two host
 * threads, or on two streams) race and must be serialized by the caller. */
int hg_objective_noalloc(int32_t n, int32_t m, int64_t p, const int32_t* net_offsets,
                         const int32_t* pins, const int32_t* net_weights,
                         const int32_t* node_weights, int32_t k, const int32_t* part,
                         void* cuda_stream, int64_t* out_objective, int64_t* out_block_weights);

/* Community detection (Sec. 4, "Community-Aware Coarsening"; Sec. 11,
 * "Deterministic Louvain Method") on level 0, before any coarsening; the
 * communities then restrict every later clustering step: a node only joins
 * a cluster of its own community, and coarse nodes inherit it.
 * The hypergraph is turned into its bipartite graph (a vertex per node and
 * per net, an edge {v, n + e} of weight floor(w(e) * 2^20 / |e|) per pin) and
 * the Louvain method maximises its modularity: per level up to 5 rounds of S
 * synchronous sub-rounds (vertex i in sub-round
 * mix64(seed ^ 2^62 ^ level<<32 ^ (round+1)<<48 ^ i) mod S), every vertex of
 * a sub-round moving to the neighbouring cluster with the largest modularity
 * gain (exact 128-bit integer comparison, ties to the smaller id) when that
 * beats staying; a round moving fewer than 1 % of the vertices ends a level,
 * a level without moves ends the method; clusters are then aggregated into
 * the next level's vertices (numbered by the rank of the cluster id).  The
 * community of a node is its vertex in the last level.
 *   out_communities  host, may be NULL: number of distinct communities
 * HG_ERR_STATE once a level has been coarsened.  Synchronizes the stream. */
int hg_detect_communities(hg_t* h, int32_t* out_communities);

/* Copies the community of every node of a level (host, n_level int32).
 * HG_ERR_STATE when no communities were detected. */
int hg_get_communities(const hg_t* h, int32_t level, int32_t* comm);

/* The whole deterministic multilevel path (Algorithm 1 without FM and
 * flows): with hg_options.community_detection, communities first; then
 * coarsen until HG_STOP, initial partition of the coarsest level,
 * label propagation on it, then project and refine level by level down to
 * level 0.  part: device, n_0 int32, written.  Levels already built are
 * reused; the handle keeps all levels afterwards. */
int hg_partition(hg_t* h, int32_t k, int32_t eps_ppm, int32_t max_passes, int32_t* part,
                 int64_t* out_objective);

/* ------------------------------------------------------------------
 * Executor: many partition jobs on one GPU (batching and serving).
 * The paper has no counterpart; it runs whole jobs of Algorithm 1 (as
 * hg_partition) concurrently.  Each of `slots` host threads owns a
 * non-blocking CUDA stream on the device current at hg_exec_create and runs
 * one job at a time: hg_create from the job's host CSR, hg_partition, the
 * partition copied to job.part_out, hg_destroy.  A job's results are those of
 * the same plain calls: every step is deterministic and a handle touches no
 * state outside itself.  Jobs start in submission order when a slot is free
 * and the estimated device bytes of the running jobs plus the next one fit
 * mem_budget_bytes (0: 80 % of the device memory free at creation); a job
 * whose estimate exceeds the whole budget starts once nothing else runs.
 * The kernels of jobs on different slots overlap on the device.  The CUDA
 * runtime maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8
 * by default), and streams that share a queue serialise each other's
 * dependent launches: set it to 32 (or at least the slot count) in the
 * environment before the process creates its CUDA context.
 * ------------------------------------------------------------------ */
typedef struct hg_exec_t hg_exec_t;

typedef struct {
  int32_t n, m;                 /* as hg_create */
  const int32_t* net_offsets;   /* host, m+1; read at submission and while the job runs */
  const int32_t* pins;          /* host, net_offsets[m] */
  const int32_t* net_weights;   /* host, m, or NULL for all 1 */
  const int32_t* node_weights;  /* host, n, or NULL for all 1 */
  int32_t k, eps_ppm, max_passes; /* as hg_partition; k in 2..64 */
  int32_t* part_out;            /* host, n int32, written when the job finishes */
  int64_t tag;                  /* returned with the result */
} hg_job;

typedef struct {
  int64_t ticket, tag;
  int32_t status;               /* HG_OK or the first error of the job's calls */
  int32_t levels;               /* levels of the job's hierarchy */
  int64_t objective;            /* f_{lambda-1} of part_out (as hg_partition) */
  int64_t level_pins;           /* sum of the pins of all levels */
  int64_t est_bytes;            /* device-memory estimate used for admission */
  int64_t t_submit_ns, t_start_ns, t_end_ns; /* hg_exec_now_ns clock */
} hg_job_result;

/* slots in 1..256; mem_budget_bytes >= 0; opt as hg_create (NULL: defaults). */
int hg_exec_create(int32_t slots, int64_t mem_budget_bytes, const hg_options* opt,
                   hg_exec_t** out);
/* Queues a job; the caller keeps the job's host arrays valid and part_out
 * untouched until its result has been returned by hg_exec_wait.  Rejects bad
 * sizes and NULL pointers with HG_ERR_INVALID (the CSR itself is checked by
 * hg_create when the job runs; its status is then in the result). */
int hg_exec_submit(hg_exec_t* ex, const hg_job* job, int64_t* out_ticket);
/* Returns up to max_results finished jobs (in completion order) in out and
 * their number in *out_count.  Waits until at least one is available, at
 * most timeout_ms (negative: no limit); returns at once with *out_count = 0
 * when no job is queued, running or unreturned. */
int hg_exec_wait(hg_exec_t* ex, int32_t max_results, int32_t timeout_ms, hg_job_result* out,
                 int32_t* out_count);
/* Jobs queued and running now (either pointer may be NULL). */
int hg_exec_pending(hg_exec_t* ex, int32_t* out_queued, int32_t* out_running);
/* Monotonic clock of the result timestamps, in nanoseconds. */
int64_t hg_exec_now_ns(void);
/* Runs every queued job to completion, then frees the executor.  Safe on
 * NULL.  Results not yet returned are dropped. */
int hg_exec_destroy(hg_exec_t* ex);

/* Copies a level to the host in canonical form.  Any pointer may be NULL.
 *   offsets (m+1), pins (p), net_weights (m), node_weights (n);
 *   map (n): coarse node of every node in level+1 (only for levels that have
 *   been coarsened; HG_ERR_STATE otherwise when map != NULL);
 *   rep (n): representative of every node in the clustering that produced
 *   level+1 (same condition). */
int hg_get_level(const hg_t* h, int32_t level, int32_t* offsets, int32_t* pins,
                 int32_t* net_weights, int32_t* node_weights, int32_t* map, int32_t* rep);

/* Copies the incident-net lists of a level to the host: offsets (n+1) and
 * nets (p).  The order of nets inside one list is unspecified. */
int hg_get_incidence(const hg_t* h, int32_t level, int32_t* offsets, int32_t* nets);

/* Drops every level above `level` (keeps 0..level) so coarsening can be
 * redone, e.g. with another k. */
int hg_truncate(hg_t* h, int32_t level);

/* Statistics (see hg_stats). */
int hg_enable_timing(hg_t* h, int32_t on);
int hg_get_stats(hg_t* h, hg_stats* out);
int hg_reset_stats(hg_t* h);

/* Returns the device memory cached in the library's own pool of the current
 * device (blocks freed by destroyed handles, kept for reuse) to the driver.
 * The paper has no counterpart.  Memory of live handles is not affected. */
int hg_trim_memory(void);

/* Frees everything the handle owns.  Safe on NULL and after any error.
 * Its blocks go back to the library's pool (see hg_options.dev_alloc). */
int hg_destroy(hg_t* h);

/* Measures the shared-memory atomic-add rate of the current device (the
 * ceiling of the rating's table updates, Sec. 4.1): conflict-free 32-bit and
 * 64-bit atomic adds over every SM, timed with CUDA events on cuda_stream;
 * writes operations per second.  The paper has no counterpart.
 * Synchronizes the stream. */
int hg_calibrate_smem_atomics(void* cuda_stream, double* out_u32_per_s, double* out_u64_per_s);

/* Static description of a status code. */
const char* hg_strerror(int status);

/* Library version string. */
const char* hg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HG_H */
