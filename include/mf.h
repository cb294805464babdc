/*
 * libmf — maximum flow / minimum cut on one GB300 GPU (sm_103a) by the
 * synchronous parallel push-relabel algorithm of Baumstark, Blelloch and Shun,
 * "Efficient Implementation of a Synchronous Parallel Push-Relabel Algorithm"
 * (arXiv:1507.01926), Section 3, Section 3.1, Algorithms 1 and 2.
 *
 * Problem (Section 2): a directed graph with integer capacities c >= 0, a
 * source s and a sink t; find a maximum flow f, its value |f|, and the minimal
 * source side S_min of a minimum cut (the vertices reachable from s in the
 * residual graph G_f of any maximum flow; unique).
 *
 * Graph format ("paired slots", the inline-reverse adjacency arrays of Section
 * 4.2): a CSR over n vertices whose m entries ("slots") are directed arcs.
 * Slot a lies in the row of its tail, head[a] is its head, cap[a] >= 0 its
 * capacity, and rev[a] is the slot of the opposite direction (head[a] ->
 * tail(a)), so that rev[rev[a]] == a and rev[a] != a. An input arc (u,v,c)
 * with no partner is stored as the pair (u->v, c) / (v->u, 0); antiparallel
 * input arcs (u,v,c1), (v,u,c2) may share one pair (c1 / c2). Residual
 * capacities of a pair always sum to cap[a] + cap[rev[a]], which must not
 * exceed INT32_MAX. mf_build_csr produces this format from an arc list.
 *
 * Arithmetic is exact integer: int32 residual capacities, int64 excesses and
 * flow value. Per-slot flow is f(a) = max(0, cap[a] - residual[a]).
 *
 * Ownership: every input array belongs to the caller and is only read during
 * the call (the library copies what it needs). Output arrays are allocated by
 * the caller, except those of mf_build_csr (freed with mf_free_csr).
 *
 * Errors: every int-returning call returns MF_OK (0), MF_PENDING (1, only
 * mf_poll) or a negative MF_ERR_* code; mf_last_error() then describes the
 * last failure of the calling thread. Calls on one mf_graph must not overlap;
 * different graphs may be used from different threads.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MF_OK 0
#define MF_PENDING 1
#define MF_ERR_INVALID_ARG (-1)  /* bad size, index out of range, null pointer, negative capacity */
#define MF_ERR_BAD_PAIRING (-2)  /* rev[rev[a]] != a, rev[a] == a, or head[rev[a]] != tail(a) */
#define MF_ERR_S_EQ_T (-3)       /* source equals sink */
#define MF_ERR_CAP_OVERFLOW (-4) /* cap[a] + cap[rev[a]] > INT32_MAX */
#define MF_ERR_OOM (-5)          /* device or host allocation failed */
#define MF_ERR_OVER_BUDGET (-6)  /* instance larger than the service's device-memory budget */
#define MF_ERR_ITER_LIMIT (-7)   /* round limit (mf_options.max_rounds) reached */
#define MF_ERR_TIMEOUT (-8)      /* a device-side wait exceeded mf_options.timeout_ms */
#define MF_ERR_CUDA (-9)         /* a CUDA runtime call failed */
#define MF_ERR_INTERNAL (-10)    /* a self-check of the solver failed */
#define MF_ERR_TOO_LARGE (-11)   /* n or m beyond the int32 limits of the device layout */
#define MF_ERR_UNKNOWN_TICKET (-12)

/* Tuning and safety limits. Fill with mf_default_options, then override. */
typedef struct mf_options {
  /* Global relabeling runs when gr_freq * work > gr_alpha * n + m, work being
   * the sum of (out-degree + work_beta) over relabels since the last one
   * (Algorithm 1; defaults 0.5, 6, 12 from the paper). */
  double gr_freq;
  int32_t gr_alpha;
  int32_t work_beta;
  /* Degree bins of the discharge and BFS kernels: a vertex of degree
   * <= bin_thread is handled by one thread, <= bin_warp by one warp, larger
   * by a whole CTA. bin_thread <= 8, or <= 16 with kernel_variant 4 (the
   * BFS hands vertices of degree 9..16 to a warp either way). */
  int32_t bin_thread;
  int32_t bin_warp;
  /* Persistent-kernel shape: threads per CTA (multiple of 32, 64..512) and
   * CTAs per SM (0 = as many as fit). */
  int32_t block_threads;
  int32_t blocks_per_sm;
  /* Safety limits: maximum push-relabel rounds per phase (0 = 2,000,000)
   * and the longest device-side wait before MF_ERR_TIMEOUT. */
  int64_t max_rounds;
  int32_t timeout_ms;
  /* 1: stop after the maximum preflow (no per-arc flow; the cut is the set
   * reachable from s and from every vertex holding excess, which equals
   * S_min). */
  int32_t cut_only;
  /* CUDA device ordinal the graph lives on. */
  int32_t device;
  /* Additional global-relabel trigger (0 = off; default 2): relabel when the
   * time spent in rounds since the last global relabel exceeds gr_time_ratio
   * times the time that relabel took. On a GPU a round costs about as much as
   * a few BFS levels whatever its size, so the work-based trigger alone lets
   * a few trapped vertices climb to n one round at a time. */
  double gr_time_ratio;
  /* Register budget of the persistent kernel: 0 = up to 128 registers per
   * thread, 1 = 85 (CTAs of <= 256 threads), 2 = 64 (<= 256 threads),
   * 3 = 64 (<= 512 threads), 4 = up to 255 (<= 256 threads, one CTA per SM)
   * with a thread path for degrees up to 16 (bin_thread <= 16). Fewer
   * registers keep more warps resident; variant 4 lets one thread discharge
   * a vertex of degree 9..16 that would otherwise take a whole warp. */
  int32_t kernel_variant;
  /* 1: run the simple synchronous rounds of Section 3 instead of the improved
   * discharge of Section 3.1: each round pushes along admissible arcs with the
   * round-start labels, then relabels every vertex still holding excess once.
   * No arc is contested and nothing is read while it changes, so every solve of
   * a graph gives the same per-arc flow: a single graph runs without the
   * time-based relabel trigger (gr_time_ratio is taken as 0), and in a batch or
   * service union with instance_relabel every instance keeps a relabel schedule
   * of its own (work and round counts only), so its per-arc flow is the same
   * alone and packed with any other instances. More rounds than the default. */
  int32_t simple_rounds;
  /* 1: capture a solve's launch sequence (control-block reset, the persistent
   * kernel, the status read-back) into a CUDA graph on the first solve and
   * replay it on later solves of the same graph with the same outputs (a
   * changed output set, option or stream captures anew). Needs a stream
   * other than the legacy default stream; on that stream the sequence is
   * launched directly. mf_stats.solve_ms then times the whole replay. */
  int32_t use_graph;
  /* On graphs whose vertices other than s and t all have at most bin_thread
   * slots, a CTA that adds at most K vertices to the next working set or BFS
   * frontier keeps them in its shared memory and discharges or expands them
   * itself in the next round or level, instead of appending them to the list
   * in device memory (saves the list-space atomic, the list writes and the
   * list reads of a round); a CTA with more appends them all, and appended
   * entries are spread evenly over all CTAs. 0: off (always append);
   * 1 (default): K = block_threads / 2; 32 <= K <= 512: that K, at most
   * block_threads. While thread 0 of a CTA waits at the grid barrier before
   * such a round or level, its other threads load the row offsets and arc
   * heads of their kept vertices and pull the rest of their data into L2.
   * No effect with simple_rounds. Results are the same for every setting. */
  int32_t local_lists;
  /* Global relabels and cut BFS: with local_lists active, a CTA expands the
   * vertices it reached itself for up to bfs_hops levels per grid barrier
   * (label-correcting: a label found too early is lowered later; the labels
   * at the end are the exact BFS distances either way). 1: one level per
   * barrier, as Algorithm 2. Default 8; range [1, 64]. */
  int32_t bfs_hops;
  /* Gap relabeling every gap_every rounds (0 = off, the default): when no
   * vertex has some label g below n, every vertex with a label between g and
   * n cannot reach the sink and gets label n (Section 2.1's gap heuristic,
   * which the paper's parallel code leaves out). Single-instance graphs with
   * the improved rounds only (no effect on batches and simple_rounds). */
  int32_t gap_every;
  /* Direction-optimizing BFS: a level of a level-synchronous BFS (bfs_hops
   * 1 or the CTA-local lists not active) whose frontier holds more than
   * n / bfs_pull vertices runs bottom-up: every vertex not reached yet scans
   * its own arcs for one into the frontier and stops at the first. Same
   * labels. Default 50; 0 = always top-down. */
  int32_t bfs_pull;
  /* Serving: most requests a lane packs into one persistent launch (0 = as
   * many as are queued and fit the budget, the default). */
  int32_t union_max_requests;
  /* Batches and service unions: 1 (default) = every instance keeps its own
   * global-relabel schedule, as if it were solved alone: it asks for a
   * relabel when its relabel work since its last one exceeds
   * (gr_alpha * n_k + m_k) / gr_freq for its own n_k and m_k, or (with
   * gr_time_ratio > 0) when it has run more than gr_time_ratio times the
   * depth (largest label) of its last relabel in rounds since; a relabel then
   * covers the instances that asked, and the others keep their working sets.
   * The first relabel of a phase and the one that confirms its end cover every
   * instance. 0 = one schedule for the whole union (the single-graph rules on
   * its totals), every relabel covering every instance. Same values and cuts;
   * with simple_rounds, 1 makes every instance's per-arc flow independent of
   * the other instances it is packed with. */
  int32_t instance_relabel;
} mf_options;

/* Counters of the last solve. Arc scans count every slot examined by a
 * discharge pass (a relabel pass of the simple rounds) or a BFS expansion,
 * slots with zero residual included; scans_discharge_residual counts the
 * discharge scans of slots with positive residual. */
typedef struct mf_stats {
  int64_t rounds;           /* push-relabel rounds, both phases */
  int64_t rounds_phase1;
  int64_t global_relabels;  /* BFS relabels, both phases */
  int64_t bfs_levels;       /* BFS levels over all BFS runs */
  int64_t scans_discharge;
  int64_t scans_bfs;
  int64_t pushes;
  int64_t relabels;
  int64_t visits_discharge; /* working-set entries discharged */
  int64_t visits_bfs;       /* frontier entries expanded */
  double solve_ms;          /* device time of the whole solve (CUDA events) */
  double preflow_ms;        /* device time to the maximum preflow */
  double relabel_ms;        /* time in global relabels (BFS + working-set rebuild) */
  double discharge_ms;      /* time in push-relabel rounds */
  int64_t rounds_by_size[4]; /* rounds whose working set had <1K, <16K, <256K, more vertices */
  /* CTA 0's view of where round and BFS-level time goes (ms): its own work,
   * the list flush and reductions, and the wait at the grid barrier */
  double round_work_ms, round_tail_ms, round_wait_ms, level_work_ms, level_wait_ms;
  int32_t grid_blocks;      /* persistent-kernel CTAs */
  int32_t block_threads;
  int64_t gap_lifted;       /* vertices lifted to label n by gap relabeling */
  int64_t scans_discharge_residual;
  int64_t global_relabels_partial; /* of global_relabels, those that covered only some instances */
} mf_stats;

typedef struct mf_graph mf_graph;
typedef struct mf_batch mf_batch;
typedef struct mf_service mf_service;
typedef int64_t mf_ticket;

/* Paired-slot CSR produced by mf_build_csr (arrays malloc'd by the library). */
typedef struct mf_csr {
  int32_t n;
  int64_t m;            /* slots */
  int64_t *row_offsets; /* n + 1 */
  int32_t *head;        /* m */
  int32_t *cap;         /* m */
  int64_t *rev;         /* m */
  int64_t *arc_slot;    /* m_in: slot holding input arc i, -1 for a dropped self-loop */
  int64_t dropped_self_loops;
} mf_csr;

/* Host description of one instance (arrays in host memory). */
typedef struct mf_graph_desc {
  int32_t n;
  int64_t m;
  const int64_t *row_offsets;
  const int32_t *head;
  const int32_t *cap;
  const int64_t *rev;
  int32_t s, t;
} mf_graph_desc;

/* Fills *opt with the defaults documented at each field. */
void mf_default_options(mf_options *opt);

/* Sizes in bytes of mf_options and mf_stats as this library was built, so
 * that a binding can check its copies of the two structs (either pointer
 * nullable). No counterpart in the paper. */
void mf_struct_sizes(int32_t *options_bytes, int32_t *stats_bytes);

/* Last error message of the calling thread ("" if none). */
const char *mf_last_error(void);

/*
 * Builds the paired-slot CSR from an input arc list (tail[i] -> head[i],
 * capacity cap[i] >= 0, 0 <= m_in). Self-loops are dropped (counted in
 * dropped_self_loops, arc_slot = -1). For every unordered vertex pair the k-th
 * input arc u->v is paired with the k-th input arc v->u (input order); unpaired
 * arcs get a reverse slot of capacity 0. Rows are sorted by head, ties in
 * input order. Returns MF_ERR_CAP_OVERFLOW if a pair's capacities sum beyond
 * INT32_MAX, MF_ERR_TOO_LARGE if the slots exceed INT32_MAX.
 */
int mf_build_csr(int32_t n, int64_t m_in, const int32_t *tail, const int32_t *head, const int32_t *cap,
                 mf_csr *out);
void mf_free_csr(mf_csr *csr);

/*
 * Copies a paired-slot CSR (host arrays, format above) to the device of
 * opt->device and validates it there. n >= 2, 0 <= m < 2^31, 0 <= s, t < n,
 * s != t. opt may be NULL (defaults). On success *out owns device memory
 * until mf_destroy_graph.
 */
int mf_create_graph(int32_t n, int64_t m, const int64_t *row_offsets, const int32_t *head, const int32_t *cap,
                    const int64_t *rev, int32_t s, int32_t t, const mf_options *opt, mf_graph **out);

/* Same, from arrays already in device memory of opt->device, read on `stream`
 * (a cudaStream_t; NULL = legacy default stream). */
int mf_create_graph_device(int32_t n, int64_t m, const int64_t *d_row_offsets, const int32_t *d_head,
                           const int32_t *d_cap, const int64_t *d_rev, int32_t s, int32_t t, const mf_options *opt,
                           void *stream, mf_graph **out);

/*
 * Solves max flow on g (Algorithms 1 and 2 for the maximum preflow, then the
 * preflow becomes a flow by returning excess to s; Section 2.1). Outputs in
 * host memory, each nullable: *flow_value = |f|; arc_flow[a] (m entries) =
 * flow on slot a; cut_bits (ceil(n/32) words) has bit v%32 of word v/32 set
 * iff v is in S_min. With opt.cut_only, arc_flow must be NULL.
 * May be called repeatedly; each call starts from the input capacities.
 */
int mf_solve(mf_graph *g, int64_t *flow_value, int32_t *arc_flow, uint32_t *cut_bits);

/* Same with outputs in device memory, enqueued on `stream` (cudaStream_t);
 * returns after the solve finished (it reads the status word back). */
int mf_solve_device(mf_graph *g, void *stream, int64_t *d_flow_value, int32_t *d_arc_flow, uint32_t *d_cut_bits);

/* Tracing: solves g like mf_solve (no outputs) and records, for each of the
 * first `capacity` push-relabel rounds of both phases, the working-set size
 * (live[k]) and whether a global relabel ran right before the round
 * (relabel_before[k] = 1), and for each of the first `level_capacity` BFS
 * levels (grid barriers of a BFS: Algorithm 2 and the cut) its frontier size
 * (level_sizes[k]). round_ns[k] and level_ns[k] (nullable; same capacities)
 * receive the duration of round / level k in ns as CTA 0 sees it, from its
 * start to the end of the grid barrier that closes it (%globaltimer; clipped
 * to INT32_MAX), so that the time of a solve can be split by working-set
 * size. *rounds and *levels (nullable) = totals (may exceed the capacities).
 * Host arrays, nullable when their capacity is 0. */
int mf_solve_trace(mf_graph *g, int32_t *live, int32_t *relabel_before, int64_t capacity, int64_t *rounds,
                   int32_t *level_sizes, int64_t level_capacity, int64_t *levels, int32_t *round_ns,
                   int32_t *level_ns);

/* Counters of the last solve on g. */
int mf_get_stats(const mf_graph *g, mf_stats *out);

/*
 * Inspection for tests: initialises phase 1 (Algorithm 1 initialisation),
 * runs the global relabel and then at most `rounds` push-relabel rounds of
 * phase 1; when final_relabel != 0 runs one more global relabel after them.
 * Copies the state out (host arrays, each nullable): residual[m] per slot,
 * label[n] (the source's label reads n, the sink's 0), excess[n]. Returns MF_OK
 * or MF_PENDING-free error codes; *rounds_done (nullable) = rounds run.
 */
int mf_run_rounds(mf_graph *g, int64_t rounds, int32_t final_relabel, int32_t *residual, int32_t *label,
                  int64_t *excess, int64_t *rounds_done);

void mf_destroy_graph(mf_graph *g);

/*
 * Batched solving: `count` independent instances (host descriptions, copied)
 * packed into one device graph (instance-offset CSR) and solved by one
 * persistent launch; every instance keeps its own n, s, t and label cap, and
 * takes part in a round only while it has active vertices. values[i] = flow
 * value of instance i; arc_flows[i] / cut_bits[i] (each entry nullable, and the
 * pointer arrays themselves nullable) as for mf_solve, in instance-local
 * numbering. The union must stay below 2^30 vertices and 2^31 slots.
 */
int mf_batch_create(int32_t count, const mf_graph_desc *descs, const mf_options *opt, mf_batch **out);
int mf_batch_solve(mf_batch *b, int64_t *values, int32_t **arc_flows, uint32_t **cut_bits);
int mf_batch_get_stats(const mf_batch *b, mf_stats *out);
void mf_batch_destroy(mf_batch *b);

/*
 * Autotuning (no counterpart in the paper, which fixes freq 0.5, alpha 6 and
 * beta 12 for a CPU). mf_autotune times solves of g under candidate options
 * and keeps the fastest: coordinate descent over gr_time_ratio {0, 1, 2, 4},
 * gr_freq {0.25, 0.5, 1, 2}, bin_thread {2, 4, 8, 16}, bin_warp {128, 1024, 8192},
 * the launch shape (threads per CTA, CTAs per SM) {(256, 2), (512, 1),
 * (128, 4), (256, 1)}, kernel_variant {0..4} (and variant 4 with
 * bin_thread 16), local_lists {0, 1}, bfs_hops {1, 4, 8, 16} (these two
 * only on graphs where they act) and bfs_pull {0, 20, 50, 200},
 * starting from g's current options; candidates that are invalid together or
 * do not fit the GPU are skipped. A candidate's time is the median device time of spec->reps solves
 * (maximum flow value only, no per-arc outputs); spec->sweeps passes over the
 * coordinates at most (fewer when a pass changes nothing); no new candidate
 * starts once the solves took spec->time_budget_ms (0 = no limit). spec may
 * be NULL (3 reps, 1 sweep, no limit). Every candidate must reproduce the flow
 * values of the starting options, else MF_ERR_INTERNAL. On success g keeps the
 * best options; *best and *best_ms (nullable) receive them and their median
 * time. A solve error of a candidate is returned as is (g keeps the best
 * options found before it).
 *
 * mf_set_options replaces the options of an existing graph (validated, the
 * launch shape recomputed; opt->device must be the graph's device).
 * mf_batch_set_options and mf_batch_autotune do the same for a batch (the
 * values of all its instances are checked).
 */
typedef struct mf_tune_spec {
  int32_t reps;           /* solves per candidate, 1..99 */
  int32_t sweeps;         /* passes over the coordinates, 1..9 */
  double time_budget_ms;  /* device time after which no new candidate starts; 0 = no limit */
} mf_tune_spec;

int mf_set_options(mf_graph *g, const mf_options *opt);
int mf_autotune(mf_graph *g, const mf_tune_spec *spec, mf_options *best, double *best_ms);
int mf_batch_set_options(mf_batch *b, const mf_options *opt);
int mf_batch_autotune(mf_batch *b, const mf_tune_spec *spec, mf_options *best, double *best_ms);

/*
 * Serving with continuous batching. mf_service_create starts worker lanes on
 * opt->device (each lane: a host thread, a CUDA stream and one CTA of
 * opt->block_threads threads on every SM for its persistent launches; as many
 * lanes as such CTAs fit an SM, at most 8 and at most opt->blocks_per_sm when
 * that is set). mf_submit copies the instance (host arrays, paired-slot CSR)
 * and returns a ticket at once; MF_ERR_OVER_BUDGET if the instance alone would
 * exceed device_budget_bytes (its estimated device footprint is 77 bytes per
 * vertex + 32 bytes per slot). A free lane admits queued requests in arrival
 * order, at most its share of the queue (queue length / lanes, rounded up),
 * while the resident footprint stays within the budget, and solves each
 * admitted group in one persistent launch. With instance_relabel (the default) every
 * request goes through its own phases inside the launch and is complete as soon
 * as its own results are written: the kernel flags it in mapped host memory,
 * the lane copies its outputs while the rest of the group is still solving,
 * and mf_wait / mf_poll see it done at once. A request that arrives while
 * others are solving starts on the next free lane; a group's device memory is
 * released when its launch ends.
 * mf_poll returns MF_PENDING until the ticket's result is ready, then the
 * result (outputs as for mf_solve, each nullable; the solve's error code if it
 * failed) and forgets the ticket. mf_wait blocks until the ticket is done
 * (timeout_ms < 0: no limit; MF_PENDING on timeout) without consuming it, and
 * reports the time from submission to completion. Unknown tickets give
 * MF_ERR_UNKNOWN_TICKET. mf_service_destroy waits for running solves and drops
 * queued requests.
 */
int mf_service_create(size_t device_budget_bytes, const mf_options *opt, mf_service **out);
/* The options mf_service_create uses when opt is NULL: mf_default_options
 * with block_threads 128, i.e. four lanes on a GB300 (with 256 threads two
 * lanes fit; on the serving stream four lanes halved the median latency of the
 * small requests at the same throughput). */
void mf_service_default_options(mf_options *o);
int mf_submit(mf_service *svc, const mf_graph_desc *g, mf_ticket *out);
int mf_poll(mf_service *svc, mf_ticket ticket, int64_t *flow_value, int32_t *arc_flow, uint32_t *cut_bits);
int mf_wait(mf_service *svc, mf_ticket ticket, int32_t timeout_ms, double *latency_ms);
void mf_service_destroy(mf_service *svc);

/*
 * Solve without allocating: for callers that cannot call cudaMalloc (code
 * running inside another runtime's memory pool or under a fixed memory
 * budget, plug-ins that must leave the CUDA allocator alone, services that
 * commit all device memory at start-up). The paper has no counterpart; this is
 * a deployment variant of mf_solve_device.
 *
 * Inputs are device pointers of the current device in the paired-slot format
 * with int32 offsets: d_row[n + 1], d_head[m], d_cap[m], d_rev[m]; they are
 * validated as in mf_create_graph. Outputs are device pointers: d_value (one
 * int64, required), d_flow[m] and d_cut[ceil(n/32)] (nullable). Work is
 * enqueued on `stream` (a cudaStream_t); the call returns when the solve is
 * done. All working state lives in one static device scratch area of 32 MiB
 * that every GPU loading the library holds until the process exits; a graph
 * needing more (about 56 bytes per vertex + 8 per slot) is rejected with
 * MF_ERR_TOO_LARGE before any work. The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine. Every call looks up the scratch
 * area's device address (cudaGetSymbolAddress). With lazy module loading (the
 * CUDA default) the first call on a device loads the library's device code
 * there, and that commits the 32 MiB area: make that first call at start-up,
 * before the rest of device memory is committed and before any stream capture.
 * Every call on a device uses the same scratch area and re-initialises it;
 * calls whose work overlaps on the GPU race.
 */
int mf_solve_noalloc(int32_t n, int32_t m, const int32_t *d_row, const int32_t *d_head, const int32_t *d_cap,
                     const int32_t *d_rev, int32_t s, int32_t t, int64_t *d_value, int32_t *d_flow,
                     uint32_t *d_cut, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */
