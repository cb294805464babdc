// Device-side data model of the solver (shared by the kernels and the host
// launch code). Everything is plain integer state resident in HBM.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace mf {

// Vertices per tile of a multi-instance graph (Dev::tiles).
constexpr int TILE_VERTICES = 4096;

// Sentinel label of a vertex not yet reached by a BFS; a source-role vertex
// carries UNV + 1 during a BFS so that it is never discovered.
constexpr int UNV = 0x3fffffff;

// What the persistent kernel does.
enum Mode : int {
  MODE_SOLVE = 0,   // phase 1, phase 2 (unless cut_only), cut, outputs
  MODE_ROUNDS = 1,  // phase 1 for at most stop_rounds rounds (+ optional final BFS relabel), no outputs
};

// Control block in device memory, zeroed before every launch.
struct Ctl {
  unsigned long long bar;  // grid barrier arrivals (monotone)
  int err;             // 0 or an MF_ERR_* code
  int err_where;       // which wait or check failed
  int cnt[4];          // list sizes of generations g % 4
  int lcnt[4];         // entries of generation g % 4 kept in the CTAs' shared memory (all CTAs together)
  long long work[3];   // per-round relabel work, by round % 3
  int gr_req[2];       // time-based relabel request, by round parity
  long long value;     // flow value (excess of the sink after phase 1)
  long long leftover;  // vertices still holding excess after phase 2
  // statistics
  long long rounds, rounds_phase1, grs, levels;
  long long scans_dis, scans_bfs, pushes, relabels;
  long long visits_dis, visits_bfs;
  unsigned long long t_gr, t_dis;            // ns in global relabels / rounds (CTA 0's view)
  unsigned long long t_rwork, t_rtail, t_rwait;  // rounds, CTA 0: own discharge work, list flush + sums, barrier wait
  unsigned long long t_lwork, t_lwait;       // BFS levels, CTA 0: own expansion work, barrier wait
  long long rounds_by_size[4];               // rounds with <1K, <16K, <256K, more list entries
  unsigned long long t_start, t_preflow, t_end;  // %globaltimer, ns
  int stopped_round;   // MODE_ROUNDS: rounds run
  int gap;             // gap relabeling: smallest label without a vertex (INT_MAX: none found yet)
  long long gap_lifted;  // vertices lifted to the label cap by gap relabeling
  long long scans_res;   // discharge scans of slots with positive residual
  long long grs_partial;  // global relabels that covered only some instances
  int due_any[3];         // some instance asked for a global relabel in round rnd (by rnd % 3; multi-instance)
  int carry_n;            // working-set entries carried over a partial global relabel
  int ph2_started;        // unions: a relabel ended the preflow of some instances (they need a relabel from s)
  int cut_pending;        // unions: a relabel ended the flow phase of some instances (they need their cut)
  int done_cnt;           // unions: instances whose results are written
  long long bad_index;    // builds with MF_CHECK_BOUNDS: the first gather index found outside its array
};
// the kernel reads cnt as one int4 and gr_req as one int2
static_assert(offsetof(Ctl, cnt) % 16 == 0 && offsetof(Ctl, lcnt) % 16 == 0 && offsetof(Ctl, gr_req) % 8 == 0,
              "Ctl layout");

// Relabel schedule of one instance of a multi-instance graph: each instance
// gets its own global relabels, when the relabel work since its last one
// exceeds its own threshold (Algorithm 1's rule with its own n and m), or when
// it has run more rounds since its last one than gr_time_ratio times that
// relabel's depth (its largest finite label).
struct InstState {
  long long thr;   // (alpha n_k + m_k) / freq
  int last;        // round index of its last global relabel
  int depth;       // largest finite label its last global relabel found
  int due;         // 1: asked for a global relabel
  int ph;          // its phase: 1 preflow (toward t), 2 flow (excess back to s), 3 cut pending, 4 done
  int act;         // working-set entries its last global relabel found
  int pad;
};
static_assert(sizeof(InstState) == 32, "instance state layout");
// The relabel work of instance k since its last global relabel lives apart, at
// Dev::inst_work[k * INST_WORK_STRIDE] (one 64-byte line each): it takes an
// atomic add from every relabeling warp, and the state above is read by every
// visit, which must not queue behind those atomics.
constexpr int INST_WORK_STRIDE = 8;

// Per-vertex record (addedExcess: excess received while the vertex is in the
// working set).
struct __align__(32) VRec {
  int lab0, stamp0, lab1, stamp1;
  long long exc, added;
};
static_assert(sizeof(VRec) == 32, "one sector per vertex");

// Device view of one (possibly multi-instance) graph.
//
// Vertex state, one 32-byte sector per vertex (VRec): two slots by round
// parity, each {label, active-round stamp}, and the excess pair {excess,
// addedExcess}. The slot a round reads, the slot it writes and the excess a
// push adds to share the sector that the gather of a neighbour's label
// brings into L2. Round r
// reads the label of every vertex from slot r & 1 and a discharged vertex
// writes d' into slot (r + 1) & 1; a vertex is in the working set of round r
// iff its stamp in slot r & 1 equals r. A BFS works on its own label array
// blab; both slots hold the same labels at phase ends.
struct Dev {
  int n;        // vertices (all instances)
  int m;        // slots (all instances)
  int n_cap;    // label cap when vinst == nullptr (single instance)
  const int2 *__restrict__ vinst;  // per vertex {label cap = its instance's n, its instance}, or nullptr
  const int *__restrict__ row;   // n + 1 slot offsets
  const int *__restrict__ head;  // m
  const int *__restrict__ rev;   // m
  const int *__restrict__ cap;   // m, input capacities (= initial residuals)
  int2 *rr;          // m: {residual of the slot, residual of its reverse slot}
  VRec *vs;          // n vertex records (above)
  unsigned long long *blab;  // n: BFS words {label, flags} (dense, so that BFS gathers stay in L2); the rebuild
                             // copies the labels into both label slots
  int bfs_hops;      // BFS levels a CTA may expand per grid barrier (1: one level per barrier)
  int gap_every;     // gap relabeling every this many rounds (0: off; single instance, improved rounds only)
  int bfs_pull;      // bottom-up BFS levels when the frontier exceeds n / bfs_pull vertices (0: never)
  int *hist;         // n + 1 label counts for gap relabeling (zero between uses), or nullptr
  int *list[3];      // vertex lists, generation g uses list[g % 3]
  const int *src;    // sources (phase 1), one per instance
  const int *snk;    // sinks (phase 1), one per instance
  int ninst;
  // multi-instance graphs (nullptr otherwise): runs of at most TILE_VERTICES
  // vertices of one instance {first vertex, end, instance, 0}, the first vertex
  // of every instance (ninst + 1 entries), and per instance the number of the
  // last partial global relabel that covers it
  const int4 *tiles;
  int ntiles;
  const int *voff;
  int *live;
  int inst_relabel;         // 1: per-instance relabel schedule (InstState), partial relabels carry the rest over
  InstState *inst;          // per instance
  long long *inst_work;     // per instance, INST_WORK_STRIDE apart
  const int *inst_marcs;    // per instance: slots with positive capacity
  int *carry;               // n: working-set entries of the instances a partial relabel does not cover
  int *gseed, *gblock;      // per instance: the seed and the blocker of its next global relabel (t and s in the
                            // preflow, s and t in the flow phase)
  unsigned *out_cutw;       // per-instance cut bitmaps, instance k's from word cwoff[k] (nullable)
  const long long *cwoff;
  volatile unsigned *done_flag;  // per instance, in mapped host memory (nullable): 1 once its results are written
  int union_phases;         // 1: every instance goes through its own phases, cut and outputs (service lanes, which
                            // hand each request its results as soon as they are written)
  double gr_alpha, gr_freq; // Algorithm 1's constants, for the per-instance thresholds
  Ctl *ctl;
  // options
  int bin_thread;
  int bin_warp;
  int beta;
  long long gr_threshold;  // global relabel when work since the last one exceeds this
  double gr_time_ratio;    // also when time since the last one exceeds this times its duration (0 = off)
  long long max_rounds;
  unsigned long long timeout_ns;
  int mode;
  long long stop_rounds;
  int final_gr;
  int cut_only;
  int simple;              // 1: the simple synchronous rounds of Section 3 (push pass, then one relabel)
  int cta_vertices;        // 0: no vertex other than a source or sink has more than bin_warp slots, so no
                           //    discharge needs a whole CTA (the CTA-wide check is skipped)
  int keep_local;          // a CTA that stages at most this many entries of a list generation keeps them in
                           // its shared memory for the phase that consumes the generation instead of
                           // appending them to the list in global memory (0: always append). Set only when
                           // every vertex other than a source or sink is thread-sized (one thread per vertex)
  // per-round trace (nullable): trace[k] = {list entries of round k, 1 if a global relabel ran just before}
  int2 *trace;
  int *trace_ns;          // nullable: ns of round k (CTA 0: from its start to the end of its grid barrier)
  long long trace_cap;
  int *trace_lv;          // nullable: frontier size of every BFS level, in order
  int *trace_lv_ns;       // nullable: ns of every BFS level (CTA 0, to the end of its grid barrier)
  long long trace_lv_cap;
  // outputs (device pointers, each nullable)
  long long *out_value;   // per instance
  int *out_flow;          // m
  unsigned *out_cut;      // ceil(n / 32)
};

}  // namespace mf
