// Internal declarations shared by the host-side translation units.
#pragma once
#include <cuda_runtime.h>

#include "mf.h"
#include "mf_device.cuh"

struct mf_graph {
  int device = 0;
  int n = 0;
  long long m = 0;
  int s = 0, t = 0;
  int ninst = 1;
  int n_cap = 0;               // label cap of a single instance (n)
  long long n_total_for_gr = 0;  // n in the relabel threshold alpha * n + m
  long long m_arcs = 0;        // slots with positive capacity
  long long max_degree = 0;    // largest slot count of a vertex that is not a source or a sink
  mf_options opt{};
  mf_stats stats{};
  int grid = 0, block = 0;
  // device state
  int *row = nullptr, *head = nullptr, *rev = nullptr, *cap = nullptr;
  int2 *rr = nullptr;
  mf::VRec *vs = nullptr;      // per-vertex labels, stamps and excess
  unsigned long long *blab = nullptr;
  int *list[3] = {nullptr, nullptr, nullptr};
  int *src = nullptr, *snk = nullptr;
  int2 *vinst = nullptr;       // multi-instance graphs: per vertex {label cap, instance}
  mf::InstState *inst = nullptr;  // multi-instance graphs: per-instance relabel schedule
  long long *inst_work = nullptr;  // multi-instance graphs: per-instance relabel work (INST_WORK_STRIDE apart)
  int *inst_marcs = nullptr;   // multi-instance graphs: positive-capacity slots per instance
  int *carry = nullptr;        // multi-instance graphs: carried working-set entries (n)
  int *gseed = nullptr, *gblocker = nullptr;  // multi-instance graphs: per-instance relabel seed and blocker
  long long *cwoff = nullptr;  // multi-instance graphs: first word of every instance's cut bitmap, ninst + 1
  unsigned *d_cutw = nullptr;  // multi-instance graphs: the instances' cut bitmaps, each from a word boundary
  int4 *tiles = nullptr;       // multi-instance graphs: vertex runs of one instance (mf::Dev::tiles)
  int ntiles = 0;
  int *voff = nullptr;         // multi-instance graphs: first vertex of every instance, ninst + 1 entries
  int *live = nullptr;         // multi-instance graphs: per-instance relabel flags
  int *hist = nullptr;         // label counts for gap relabeling (allocated on first use)
  mf::Ctl *ctl = nullptr;
  long long *d_value = nullptr;
  int *d_flow = nullptr;
  unsigned *d_cut = nullptr;
  mf::Ctl *h_ctl = nullptr;    // pinned
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // service lanes: device memory comes from this pool, allocated and freed in stream order on `stream`
  // (no device-wide synchronisation), and h_ctl / ev0 / ev1 belong to the lane
  cudaMemPool_t pool = nullptr;
  bool lane_host = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // captured launch sequence (mf_options.use_graph) and what it was captured for
  cudaGraphExec_t gexec = nullptr;
  mf::Dev gdev{};
  cudaStream_t gstream = nullptr;
  int ggrid = 0, gblock = 0, gvariant = -1;
};

namespace mf {
// What a service lane lends to every union it solves: its memory pool and its
// pinned control-block copy and timing events.
struct LaneHost {
  cudaMemPool_t pool;
  Ctl *h_ctl;
  cudaEvent_t ev0, ev1;
  cudaStream_t copy;       // copies of finished requests' results while the kernel runs
  unsigned *h_done;        // mapped host memory: per-instance done flags the kernel sets
  unsigned *d_done;        // their device address
  int done_cap;            // flags available
};

int fail(int code, const char *fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char *what);
int alloc_state(mf_graph *g);
int galloc(mf_graph *g, void **p, size_t bytes, const char *what);
void gfree(mf_graph *g, void *p);
int validate_on_device(mf_graph *g, const long long *row64, const long long *rev64, cudaStream_t st);
int launch_config(mf_graph *g);
int check_options(const mf_options *o);
Dev make_dev(const mf_graph *g);
long long relabel_threshold(const mf_options &o, long long n, long long m_arcs);
int device_status(const Ctl &c);
int run_kernel(mf_graph *g, Dev &D, cudaStream_t st);
int launch_kernel(mf_graph *g, Dev &D, cudaStream_t st);
int finish_kernel(mf_graph *g);
int keep_local_limit(const mf_options &o, long long max_degree, int block_threads);
int solver_variants();
int solver_variant_max_threads(int variant);
int solver_variant_max_bin_thread(int variant);
int solver_occupancy(int block_threads, int *blocks_per_sm, int variant, bool multi);
cudaError_t launch_solver(const Dev &D, int grid, int block, cudaStream_t stream, int variant);
int set_options(mf_graph *g, const mf_options *o);
int autotune(mf_graph *g, const mf_tune_spec *spec, mf_options *best, double *best_ms);
}  // namespace mf
