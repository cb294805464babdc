// Host side of the C-ABI (include/mf.h): graph objects, validation on the
// device, launch of the persistent solver, error reporting.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "mf.h"
#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

const char *last_error() { return g_err.c_str(); }  // calling thread's message

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(MF_ERR_OOM, "%s: out of device memory", what);
  }
  return fail(MF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ validation

enum : unsigned {
  V_ROW = 1u,        // row offsets not monotone / wrong ends
  V_HEAD = 2u,       // head out of range
  V_REV = 4u,        // rev out of range or rev[a] == a
  V_CAP = 8u,        // negative capacity
  V_PAIR = 16u,      // rev[rev[a]] != a
  V_TAIL = 32u,      // head[rev[a]] != tail(a)
  V_OVERFLOW = 64u,  // cap[a] + cap[rev[a]] > INT32_MAX
};

__global__ void k_check_rows(int n, long long m, const long long *row64, int *row32, unsigned *flags) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v <= n; v += (long long)gridDim.x * blockDim.x) {
    const long long x = row64[v];
    bool bad = x < 0 || x > m;
    if (v == 0 && x != 0) bad = true;
    if (v == n && x != m) bad = true;
    if (v < n && x > row64[v + 1]) bad = true;
    if (bad) atomicOr(flags, V_ROW);
    row32[v] = (int)(bad ? 0 : x);
  }
}

__global__ void k_check_slots(int n, long long m, const int *head, const int *cap, const long long *rev64,
                              int *rev32, unsigned *flags) {
  unsigned f = 0;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m; a += (long long)gridDim.x * blockDim.x) {
    const int h = head[a];
    if (h < 0 || h >= n) f |= V_HEAD;
    if (cap[a] < 0) f |= V_CAP;
    const long long r = rev64[a];
    if (r < 0 || r >= m || r == a) {
      f |= V_REV;
      rev32[a] = (int)a;
    } else {
      rev32[a] = (int)r;
    }
  }
  if (f) atomicOr(flags, f);
}

// Pairing checks, one warp per vertex v (the row gives every slot's tail, so
// no search is needed): rev[rev[a]] = a, head[rev[a]] = v, and the pair's
// capacities fit int32; counts the slots with positive capacity.
__global__ void k_check_pairs(int n, const int *row, const int *head, const int *cap, const int *rev, unsigned *flags,
                              unsigned long long *m_arcs) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  unsigned f = 0;
  unsigned long long cnt = 0;
  for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int b = row[v], e = row[v + 1];
    for (int a = b + lane; a < e; a += 32) {
      const int ra = rev[a];
      if (rev[ra] != a) f |= V_PAIR;
      if (head[ra] != (int)v) f |= V_TAIL;
      if ((long long)cap[a] + (long long)cap[ra] > 2147483647LL) f |= V_OVERFLOW;
      if (cap[a] > 0) cnt++;
    }
  }
  f = __reduce_or_sync(0xffffffffu, f);
  cnt = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
  if (lane == 0) {
    if (f) atomicOr(flags, f);
    if (cnt) atomicAdd(m_arcs, cnt);
  }
}

// Largest out-degree (slots) of a vertex other than s and t.
__global__ void k_max_degree(int n, const int *row, int s, int t, unsigned *out) {
  unsigned mx = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (v != s && v != t) mx = max(mx, (unsigned)(row[v + 1] - row[v]));
  if (mx) atomicMax(out, mx);
}

static int flags_to_status(unsigned f) {
  if (f & (V_ROW | V_HEAD | V_REV | V_CAP)) {
    return fail(MF_ERR_INVALID_ARG, "invalid graph:%s%s%s%s", (f & V_ROW) ? " row_offsets not a valid CSR;" : "",
                (f & V_HEAD) ? " head out of range;" : "", (f & V_REV) ? " rev out of range or rev[a]==a;" : "",
                (f & V_CAP) ? " negative capacity;" : "");
  }
  if (f & (V_PAIR | V_TAIL))
    return fail(MF_ERR_BAD_PAIRING, "bad reverse pairing:%s%s", (f & V_PAIR) ? " rev[rev[a]] != a;" : "",
                (f & V_TAIL) ? " head[rev[a]] != tail(a);" : "");
  if (f & V_OVERFLOW) return fail(MF_ERR_CAP_OVERFLOW, "cap[a] + cap[rev[a]] exceeds INT32_MAX");
  return MF_OK;
}

// ------------------------------------------------------------------ graph

// Device memory of a graph: cudaMalloc, or for a service lane's union the
// lane's pool in stream order (cudaFree would wait for the other lanes' work).
int galloc(mf_graph *g, void **p, size_t bytes, const char *what) {
  if (!bytes) bytes = 16;
  const cudaError_t e = g->pool ? cudaMallocFromPoolAsync(p, bytes, g->pool, g->stream) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  return MF_OK;
}

void gfree(mf_graph *g, void *p) {
  if (!p) return;
  if (g->pool)
    cudaFreeAsync(p, g->stream);
  else
    cudaFree(p);
}

static void free_graph_buffers(mf_graph *g) {
  void *ps[] = {g->row, g->head, g->rev, g->cap, g->rr, g->vs, g->blab, g->list[0], g->list[1], g->list[2],
                g->src, g->snk, g->ctl, g->d_value, g->d_flow, g->d_cut, g->vinst, g->hist,
                g->tiles, g->voff, g->live, g->cwoff, g->d_cutw, g->inst, g->inst_work, g->inst_marcs, g->carry,
                g->gseed, g->gblocker};
  for (void *p : ps) gfree(g, p);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (!g->lane_host) {
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
  }
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
}

static int dalloc(mf_graph *g, void **p, size_t bytes, const char *what) { return galloc(g, p, bytes, what); }

#define TRY(x)               \
  do {                       \
    int _rc = (x);           \
    if (_rc != MF_OK) {      \
      mf_destroy_graph(g);   \
      return _rc;            \
    }                        \
  } while (0)

#define TRYC(x, what)                       \
  do {                                      \
    cudaError_t _e = (x);                   \
    if (_e != cudaSuccess) {                \
      int _rc = cuda_fail(_e, what);        \
      mf_destroy_graph(g);                  \
      return _rc;                           \
    }                                       \
  } while (0)

int alloc_state(mf_graph *g) {
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  int rc;
  if ((rc = dalloc(g, (void **)&g->row, (n + 1) * 4, "cudaMalloc row"))) return rc;
  if ((rc = dalloc(g, (void **)&g->head, m * 4, "cudaMalloc head"))) return rc;
  if ((rc = dalloc(g, (void **)&g->rev, m * 4, "cudaMalloc rev"))) return rc;
  if ((rc = dalloc(g, (void **)&g->cap, m * 4, "cudaMalloc cap"))) return rc;
  if ((rc = dalloc(g, (void **)&g->rr, m * 8, "cudaMalloc residuals"))) return rc;
  if ((rc = dalloc(g, (void **)&g->vs, n * sizeof(VRec), "cudaMalloc vertex state"))) return rc;
  if ((rc = dalloc(g, (void **)&g->blab, n * 8, "cudaMalloc BFS labels"))) return rc;
  for (int k = 0; k < 3; k++)
    if ((rc = dalloc(g, (void **)&g->list[k], n * 4, "cudaMalloc list"))) return rc;
  if ((rc = dalloc(g, (void **)&g->src, (size_t)g->ninst * 4, "cudaMalloc sources"))) return rc;
  if ((rc = dalloc(g, (void **)&g->snk, (size_t)g->ninst * 4, "cudaMalloc sinks"))) return rc;
  if ((rc = dalloc(g, (void **)&g->ctl, sizeof(Ctl), "cudaMalloc control block"))) return rc;
  if ((rc = dalloc(g, (void **)&g->d_value, (size_t)g->ninst * 8, "cudaMalloc value"))) return rc;
  if (g->lane_host) return MF_OK;  // pinned control-block copy and events come from the service lane
  cudaError_t e = cudaMallocHost((void **)&g->h_ctl, sizeof(Ctl));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
  if ((e = cudaEventCreate(&g->ev0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&g->ev1)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  return MF_OK;
}

// Validates the copied CSR (row64/rev64 in device memory) and fills the
// int32 device arrays; computes m_arcs.
int validate_on_device(mf_graph *g, const long long *row64, const long long *rev64, cudaStream_t st) {
  unsigned *flags = nullptr;
  unsigned long long *marcs = nullptr;
  int arc = galloc(g, (void **)&flags, 16, "cudaMalloc flags");
  if (arc) return arc;
  cudaError_t e;
  marcs = reinterpret_cast<unsigned long long *>(flags) + 1;
  cudaMemsetAsync(flags, 0, 16, st);
  const int T = 256;
  const int Gn = (int)((g->n + 1 + T - 1) / T < 65535 * 16 ? (g->n + 1 + T - 1) / T : 65535 * 16);
  const long long gm = (g->m + T - 1) / T;
  const int Gm = (int)(gm < 1 ? 1 : (gm < 65535LL * 16 ? gm : 65535LL * 16));
  k_check_rows<<<Gn, T, 0, st>>>(g->n, g->m, row64, g->row, flags);
  k_check_slots<<<Gm, T, 0, st>>>(g->n, g->m, g->head, g->cap, rev64, g->rev, flags);
  unsigned h[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(h, flags, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    gfree(g, flags);
    return cuda_fail(e, "graph validation");
  }
  if (h[0] == 0 && g->m > 0) {
    const long long gw = ((long long)g->n * 32 + T - 1) / T;  // one warp per vertex
    const int Gw = (int)(gw < 65535LL * 16 ? gw : 65535LL * 16);
    k_check_pairs<<<Gw, T, 0, st>>>(g->n, g->row, g->head, g->cap, g->rev, flags, marcs);
    k_max_degree<<<Gn, T, 0, st>>>(g->n, g->row, g->s, g->t, flags + 1);
    e = cudaMemcpyAsync(h, flags, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      gfree(g, flags);
      return cuda_fail(e, "graph validation");
    }
  }
  gfree(g, flags);
  g->m_arcs = (long long)((unsigned long long)h[2] | ((unsigned long long)h[3] << 32));
  g->max_degree = h[1];
  return flags_to_status(h[0]);
}

int launch_config(mf_graph *g) {
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (!prop.cooperativeLaunch) return fail(MF_ERR_CUDA, "device %d lacks cooperative launch", g->device);
  int bps = 0;
  if (solver_occupancy(g->opt.block_threads, &bps, g->opt.kernel_variant, g->vinst != nullptr) || bps < 1)
    return fail(MF_ERR_CUDA, "solver kernel does not fit %d threads per CTA", g->opt.block_threads);
  if (g->opt.blocks_per_sm > 0 && g->opt.blocks_per_sm < bps) bps = g->opt.blocks_per_sm;
  g->grid = bps * prop.multiProcessorCount;
  g->block = g->opt.block_threads;
  return MF_OK;
}

int check_options(const mf_options *o) {
  if (o->block_threads < 64 || o->block_threads > 512 || o->block_threads % 32)
    return fail(MF_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [64, 512]");
  if (o->bin_thread < 0 || o->bin_thread > 16) return fail(MF_ERR_INVALID_ARG, "bin_thread must be in [0, 16]");
  if (o->bin_warp < o->bin_thread) return fail(MF_ERR_INVALID_ARG, "bin_warp must be >= bin_thread");
  if (!(o->gr_freq > 0)) return fail(MF_ERR_INVALID_ARG, "gr_freq must be > 0");
  if (o->gr_alpha < 0 || o->work_beta < 0) return fail(MF_ERR_INVALID_ARG, "gr_alpha, work_beta must be >= 0");
  if (o->timeout_ms <= 0) return fail(MF_ERR_INVALID_ARG, "timeout_ms must be > 0");
  if (o->max_rounds < 0) return fail(MF_ERR_INVALID_ARG, "max_rounds must be >= 0");
  if (!(o->gr_time_ratio >= 0)) return fail(MF_ERR_INVALID_ARG, "gr_time_ratio must be >= 0");
  if (o->use_graph != 0 && o->use_graph != 1) return fail(MF_ERR_INVALID_ARG, "use_graph must be 0 or 1");
  if (o->bfs_hops < 1 || o->bfs_hops > 64) return fail(MF_ERR_INVALID_ARG, "bfs_hops must be in [1, 64]");
  if (o->gap_every < 0) return fail(MF_ERR_INVALID_ARG, "gap_every must be >= 0");
  if (o->bfs_pull < 0) return fail(MF_ERR_INVALID_ARG, "bfs_pull must be >= 0");
  if (o->union_max_requests < 0) return fail(MF_ERR_INVALID_ARG, "union_max_requests must be >= 0");
  if (o->instance_relabel != 0 && o->instance_relabel != 1)
    return fail(MF_ERR_INVALID_ARG, "instance_relabel must be 0 or 1");
  if (o->local_lists < 0 || (o->local_lists > 1 && o->local_lists < 32) || o->local_lists > 512)
    return fail(MF_ERR_INVALID_ARG, "local_lists must be 0, 1 or in [32, 512]");
  if (o->kernel_variant < 0 || o->kernel_variant >= solver_variants())
    return fail(MF_ERR_INVALID_ARG, "kernel_variant must be in [0, %d)", solver_variants());
  if (o->block_threads > solver_variant_max_threads(o->kernel_variant))
    return fail(MF_ERR_INVALID_ARG, "kernel_variant %d takes at most %d threads per CTA", o->kernel_variant,
                solver_variant_max_threads(o->kernel_variant));
  if (o->bin_thread > solver_variant_max_bin_thread(o->kernel_variant))
    return fail(MF_ERR_INVALID_ARG, "kernel_variant %d takes bin_thread <= %d", o->kernel_variant,
                solver_variant_max_bin_thread(o->kernel_variant));
  return MF_OK;
}

// Relabel work after which a global relabel runs: (alpha n + m) / freq, m
// counting the slots with positive capacity (Algorithm 1), clamped to int64.
long long relabel_threshold(const mf_options &o, long long n, long long m_arcs) {
  const double thr = ((double)o.gr_alpha * (double)n + (double)m_arcs) / o.gr_freq;
  return thr > 9.0e18 ? (long long)9e18 : (long long)thr;
}

Dev make_dev(const mf_graph *g) {
  Dev D;
  memset(&D, 0, sizeof(D));
  D.n = g->n;
  D.m = (int)g->m;
  D.n_cap = g->n_cap;
  D.vinst = g->vinst;
  D.row = g->row;
  D.head = g->head;
  D.rev = g->rev;
  D.cap = g->cap;
  D.rr = g->rr;
  D.vs = g->vs;
  D.blab = g->blab;
  for (int k = 0; k < 3; k++) D.list[k] = g->list[k];
  D.src = g->src;
  D.snk = g->snk;
  D.ninst = g->ninst;
  D.tiles = g->tiles;
  D.ntiles = g->ntiles;
  D.voff = g->voff;
  D.live = g->live;
  D.inst = g->inst;
  D.inst_work = g->inst_work;
  D.inst_marcs = g->inst_marcs;
  D.carry = g->carry;
  D.gseed = g->gseed;
  D.gblock = g->gblocker;
  D.cwoff = g->cwoff;
  D.inst_relabel = (g->inst && g->opt.instance_relabel) ? 1 : 0;
  D.gr_alpha = (double)g->opt.gr_alpha;
  D.gr_freq = g->opt.gr_freq;
  D.ctl = g->ctl;
  D.bin_thread = g->opt.bin_thread;
  D.bin_warp = g->opt.bin_warp;
  D.beta = g->opt.work_beta;
  D.gr_threshold = relabel_threshold(g->opt, g->n_total_for_gr, g->m_arcs);
  D.max_rounds = g->opt.max_rounds > 0 ? g->opt.max_rounds : 2000000LL;
  D.simple = g->opt.simple_rounds ? 1 : 0;
  D.cta_vertices = g->max_degree > (long long)g->opt.bin_warp ? 1 : 0;
  D.keep_local = keep_local_limit(g->opt, g->max_degree, g->block);
  D.bfs_hops = D.keep_local > 0 ? g->opt.bfs_hops : 1;
  D.gap_every = (g->ninst == 1 && !D.simple && g->hist) ? g->opt.gap_every : 0;
  D.bfs_pull = g->opt.bfs_pull;
  D.hist = g->hist;
  // the time-based trigger of a single graph depends on measured times; a union's per-instance trigger
  // counts rounds and labels, so it stays deterministic with simple_rounds
  D.gr_time_ratio = (D.simple && !D.inst_relabel) ? 0.0 : g->opt.gr_time_ratio;
  D.timeout_ns = (unsigned long long)g->opt.timeout_ms * 1000000ULL;
  D.mode = MODE_SOLVE;
  D.cut_only = g->opt.cut_only;
  return D;
}

// The launch sequence of one solve: control-block reset, the persistent
// kernel (between two timing events when `timed`), the read-back of the
// control block.
static cudaError_t enqueue_solve(mf_graph *g, const Dev &D, cudaStream_t st, bool timed) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), st)) != cudaSuccess) return e;
  if (timed && (e = cudaEventRecord(g->ev0, st)) != cudaSuccess) return e;
  if ((e = launch_solver(D, g->grid, g->block, st, g->opt.kernel_variant)) != cudaSuccess) return e;
  if (timed && (e = cudaEventRecord(g->ev1, st)) != cudaSuccess) return e;
  return cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
}

// Captures the launch sequence for (D, st, launch shape) into g->gexec unless
// the current capture already matches.
static int ensure_graph(mf_graph *g, const Dev &D, cudaStream_t st) {
  if (g->gexec && g->gstream == st && g->ggrid == g->grid && g->gblock == g->block &&
      g->gvariant == g->opt.kernel_variant && memcmp(&g->gdev, &D, sizeof(Dev)) == 0)
    return MF_OK;
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  const cudaError_t le = enqueue_solve(g, D, st, false);  // events of a capture are not recorded
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(st, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(le != cudaSuccess ? le : e, "capture of the solve launch sequence");
  }
  e = cudaGraphInstantiate(&g->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->gexec = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  g->gdev = D;
  g->gstream = st;
  g->ggrid = g->grid;
  g->gblock = g->block;
  g->gvariant = g->opt.kernel_variant;
  return MF_OK;
}

// Runs the persistent kernel once with D; fills g->h_ctl and g->stats.
int run_kernel(mf_graph *g, Dev &D, cudaStream_t st) {
  const int rc = launch_kernel(g, D, st);
  if (rc) return rc;
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "solver");
  return finish_kernel(g);
}

// Enqueues one solve with D on st (see run_kernel); returns without waiting.
int launch_kernel(mf_graph *g, Dev &D, cudaStream_t st) {
  cudaError_t e;
  if (g->opt.gap_every > 0 && g->ninst == 1 && !g->opt.simple_rounds && !g->hist) {
    // label counts for gap relabeling, zeroed by the kernel before use
    if ((e = cudaMalloc((void **)&g->hist, ((size_t)g->n_cap + 1) * sizeof(int))) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc label counts");
    D.hist = g->hist;
    D.gap_every = g->opt.gap_every;
  }
  if (g->opt.use_graph && st != nullptr) {
    const int rc = ensure_graph(g, D, st);
    if (rc) return rc;
    // the timing events bracket the whole replay (reset, kernel, read-back)
    e = cudaEventRecord(g->ev0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(g->gexec, st);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev1, st);
  } else {
    e = enqueue_solve(g, D, st, true);
  }
  return e == cudaSuccess ? MF_OK : cuda_fail(e, "solver launch");
}

// After a launch finished: statistics and status from the control block.
int finish_kernel(mf_graph *g) {
  const Ctl &c = *g->h_ctl;
  float ms = 0;
  cudaEventElapsedTime(&ms, g->ev0, g->ev1);
  mf_stats &s = g->stats;
  s.rounds = c.rounds;
  s.rounds_phase1 = c.rounds_phase1;
  s.global_relabels = c.grs;
  s.bfs_levels = c.levels;
  s.scans_discharge = c.scans_dis;
  s.scans_bfs = c.scans_bfs;
  s.pushes = c.pushes;
  s.relabels = c.relabels;
  s.visits_discharge = c.visits_dis;
  s.visits_bfs = c.visits_bfs;
  s.solve_ms = ms;
  s.relabel_ms = (double)c.t_gr * 1e-6;
  s.discharge_ms = (double)c.t_dis * 1e-6;
  for (int i = 0; i < 4; i++) s.rounds_by_size[i] = c.rounds_by_size[i];
  s.round_work_ms = (double)c.t_rwork * 1e-6;
  s.round_tail_ms = (double)c.t_rtail * 1e-6;
  s.round_wait_ms = (double)c.t_rwait * 1e-6;
  s.level_work_ms = (double)c.t_lwork * 1e-6;
  s.level_wait_ms = (double)c.t_lwait * 1e-6;
  s.preflow_ms = c.t_preflow > c.t_start ? (double)(c.t_preflow - c.t_start) * 1e-6 : 0.0;
  s.grid_blocks = g->grid;
  s.block_threads = g->block;
  s.gap_lifted = c.gap_lifted;
  s.scans_discharge_residual = c.scans_res;
  s.global_relabels_partial = c.grs_partial;
  return device_status(c);
}

// Status of a finished launch from its control block: MF_OK, or the error the
// kernel recorded with the site (err_where) that recorded it.
int device_status(const Ctl &c) {
  if (!c.err) return MF_OK;
  static const char *where[] = {"init barrier", "saturation barrier", "relabel BFS", "working-set rebuild",
                                "discharge barrier", "apply barrier", "cut BFS (preflow)", "excess check",
                                "phase-2 excess check", "cut BFS", "round limit", "list capacity",
                                "settle barrier", "gap relabeling"};
  if (c.err == MF_ERR_INTERNAL && c.err_where >= 1000)  // a build with gather checks (MF_CHECK_BOUNDS)
    return fail(MF_ERR_INTERNAL, "gather index %lld out of bounds at mf_solver.cuh line %d", c.bad_index,
                c.err_where - 1000);
  const char *w = (c.err_where >= 0 && c.err_where <= 13) ? where[c.err_where] : "?";
  if (c.err == MF_ERR_TIMEOUT) return fail(MF_ERR_TIMEOUT, "device wait timed out (%s)", w);
  if (c.err == MF_ERR_ITER_LIMIT) return fail(MF_ERR_ITER_LIMIT, "round limit reached (%lld rounds)", c.rounds);
  if (c.err == MF_ERR_INTERNAL && c.err_where == 8)
    return fail(MF_ERR_INTERNAL, "self-check failed: %lld vertices kept excess", c.leftover);
  if (c.err == MF_ERR_INTERNAL) return fail(MF_ERR_INTERNAL, "self-check failed (%s)", w);
  return fail(c.err, "device error %d (%s)", c.err, w);
}

}  // namespace mf

using namespace mf;

extern "C" {

void mf_default_options(mf_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->gr_freq = 0.5;
  o->gr_alpha = 6;
  o->work_beta = 12;
  o->bin_thread = 8;
  o->bin_warp = 1024;
  o->block_threads = 256;
  o->blocks_per_sm = 0;
  o->max_rounds = 0;
  o->timeout_ms = 5000;
  o->cut_only = 0;
  o->device = 0;
  o->gr_time_ratio = 2.0;
  o->local_lists = 1;
  o->bfs_hops = 8;
  o->bfs_pull = 50;
  o->instance_relabel = 1;
}

void mf_service_default_options(mf_options *o) {
  if (!o) return;
  mf_default_options(o);
  // lanes of 128-thread CTAs: four lanes' persistent launches fit the SMs together (two with 256 threads),
  // so a request that arrives while others are solving finds a free lane sooner
  o->block_threads = 128;
}

const char *mf_last_error(void) { return last_error(); }

void mf_struct_sizes(int32_t *options_bytes, int32_t *stats_bytes) {
  if (options_bytes) *options_bytes = (int32_t)sizeof(mf_options);
  if (stats_bytes) *stats_bytes = (int32_t)sizeof(mf_stats);
}

static int create_common(int32_t n, int64_t m, int32_t s, int32_t t, const mf_options *opt, mf_graph **out,
                         mf_graph **gp) {
  clear_error();
  if (!out) return fail(MF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 2) return fail(MF_ERR_INVALID_ARG, "n must be >= 2");
  if (n > UNV - 4) return fail(MF_ERR_TOO_LARGE, "n exceeds the label range (%d)", UNV - 4);
  if (m < 0) return fail(MF_ERR_INVALID_ARG, "m must be >= 0");
  if (m > 2147483647LL - 1) return fail(MF_ERR_TOO_LARGE, "m exceeds INT32_MAX slots");
  if (s < 0 || s >= n || t < 0 || t >= n) return fail(MF_ERR_INVALID_ARG, "s or t out of range");
  if (s == t) return fail(MF_ERR_S_EQ_T, "source equals sink");
  mf_options o;
  if (opt)
    o = *opt;
  else
    mf_default_options(&o);
  int rc = check_options(&o);
  if (rc) return rc;
  cudaError_t e = cudaSetDevice(o.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  mf_graph *g = new mf_graph();
  g->opt = o;
  g->device = o.device;
  g->n = n;
  g->m = m;
  g->s = s;
  g->t = t;
  g->ninst = 1;
  g->n_cap = n;
  g->n_total_for_gr = n;
  *gp = g;
  return MF_OK;
}

int mf_create_graph(int32_t n, int64_t m, const int64_t *row_offsets, const int32_t *head, const int32_t *cap,
                    const int64_t *rev, int32_t s, int32_t t, const mf_options *opt, mf_graph **out) {
  mf_graph *g = nullptr;
  int rc = create_common(n, m, s, t, opt, out, &g);
  if (rc) return rc;
  if (!row_offsets || (m > 0 && (!head || !cap || !rev))) {
    delete g;
    return fail(MF_ERR_INVALID_ARG, "NULL array");
  }
  TRYC(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking), "cudaStreamCreate");
  g->own_stream = true;
  TRY(alloc_state(g));
  long long *row64 = nullptr, *rev64 = nullptr;
  TRYC(cudaMalloc((void **)&row64, ((size_t)n + 1) * 8), "cudaMalloc staging");
  cudaError_t e = cudaMalloc((void **)&rev64, (size_t)(m > 0 ? m : 1) * 8);
  if (e != cudaSuccess) {
    cudaFree(row64);
    TRYC(e, "cudaMalloc staging");
  }
  e = cudaMemcpyAsync(row64, row_offsets, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(rev64, rev, (size_t)m * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->head, head, (size_t)m * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->cap, cap, (size_t)m * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->src, &g->s, 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->snk, &g->t, 4, cudaMemcpyHostToDevice, g->stream);
  if (e != cudaSuccess) {
    cudaFree(row64);
    cudaFree(rev64);
    TRYC(e, "host-to-device copy");
  }
  rc = validate_on_device(g, row64, rev64, g->stream);
  cudaFree(row64);
  cudaFree(rev64);
  TRY(rc);
  TRY(launch_config(g));
  *out = g;
  return MF_OK;
}

int mf_create_graph_device(int32_t n, int64_t m, const int64_t *d_row_offsets, const int32_t *d_head,
                           const int32_t *d_cap, const int64_t *d_rev, int32_t s, int32_t t, const mf_options *opt,
                           void *stream, mf_graph **out) {
  mf_graph *g = nullptr;
  int rc = create_common(n, m, s, t, opt, out, &g);
  if (rc) return rc;
  if (!d_row_offsets || (m > 0 && (!d_head || !d_cap || !d_rev))) {
    delete g;
    return fail(MF_ERR_INVALID_ARG, "NULL array");
  }
  g->stream = (cudaStream_t)stream;
  g->own_stream = false;
  TRY(alloc_state(g));
  cudaError_t e = cudaSuccess;
  if (m > 0) e = cudaMemcpyAsync(g->head, d_head, (size_t)m * 4, cudaMemcpyDeviceToDevice, g->stream);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->cap, d_cap, (size_t)m * 4, cudaMemcpyDeviceToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->src, &g->s, 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->snk, &g->t, 4, cudaMemcpyHostToDevice, g->stream);
  TRYC(e, "device copy");
  TRY(validate_on_device(g, (const long long *)d_row_offsets, (const long long *)d_rev, g->stream));
  TRY(launch_config(g));
  *out = g;
  return MF_OK;
}

void mf_destroy_graph(mf_graph *g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  free_graph_buffers(g);
  delete g;
}

static int solve_into(mf_graph *g, cudaStream_t st, int64_t *d_value, int32_t *d_flow, uint32_t *d_cut) {
  if (g->opt.cut_only && d_flow) return fail(MF_ERR_INVALID_ARG, "cut_only solves produce no per-arc flow");
  Dev D = make_dev(g);
  D.out_value = d_value ? reinterpret_cast<long long *>(d_value) : g->d_value;
  D.out_flow = d_flow;
  D.out_cut = d_cut;
  return run_kernel(g, D, st);
}

int mf_solve(mf_graph *g, int64_t *flow_value, int32_t *arc_flow, uint32_t *cut_bits) {
  clear_error();
  if (!g) return fail(MF_ERR_INVALID_ARG, "graph is NULL");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (arc_flow && !g->d_flow) {
    e = cudaMalloc((void **)&g->d_flow, (size_t)(g->m > 0 ? g->m : 1) * 4);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc flow output");
  }
  const size_t words = ((size_t)g->n + 31) / 32;
  if (cut_bits && !g->d_cut) {
    e = cudaMalloc((void **)&g->d_cut, words * 4);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc cut output");
  }
  int rc = solve_into(g, g->stream, nullptr, arc_flow ? g->d_flow : nullptr, cut_bits ? g->d_cut : nullptr);
  if (rc) return rc;
  if (flow_value) *flow_value = g->h_ctl->value;
  if (arc_flow && g->m > 0) e = cudaMemcpyAsync(arc_flow, g->d_flow, (size_t)g->m * 4, cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess && cut_bits) e = cudaMemcpyAsync(cut_bits, g->d_cut, words * 4, cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy of the outputs");
  return MF_OK;
}

int mf_solve_device(mf_graph *g, void *stream, int64_t *d_flow_value, int32_t *d_arc_flow, uint32_t *d_cut_bits) {
  clear_error();
  if (!g) return fail(MF_ERR_INVALID_ARG, "graph is NULL");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return solve_into(g, (cudaStream_t)stream, d_flow_value, d_arc_flow, d_cut_bits);
}

int mf_solve_trace(mf_graph *g, int32_t *live, int32_t *relabel_before, int64_t capacity, int64_t *rounds,
                   int32_t *level_sizes, int64_t level_capacity, int64_t *levels, int32_t *round_ns,
                   int32_t *level_ns) {
  clear_error();
  if (!g || capacity < 0 || (capacity > 0 && (!live || !relabel_before)) || level_capacity < 0 ||
      (level_capacity > 0 && !level_sizes))
    return fail(MF_ERR_INVALID_ARG, "bad arguments");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  int2 *tr = nullptr;
  int *trn = nullptr, *tl = nullptr, *tln = nullptr;
  auto release = [&]() {
    if (tr) cudaFree(tr);
    if (trn) cudaFree(trn);
    if (tl) cudaFree(tl);
    if (tln) cudaFree(tln);
  };
  if ((capacity > 0 && (e = cudaMalloc((void **)&tr, (size_t)capacity * sizeof(int2))) != cudaSuccess) ||
      (capacity > 0 && round_ns && (e = cudaMalloc((void **)&trn, (size_t)capacity * sizeof(int))) != cudaSuccess) ||
      (level_capacity > 0 && (e = cudaMalloc((void **)&tl, (size_t)level_capacity * sizeof(int))) != cudaSuccess) ||
      (level_capacity > 0 && level_ns &&
       (e = cudaMalloc((void **)&tln, (size_t)level_capacity * sizeof(int))) != cudaSuccess)) {
    release();
    return cuda_fail(e, "cudaMalloc trace");
  }
  Dev D = make_dev(g);
  D.out_value = g->d_value;
  D.trace = tr;
  D.trace_ns = trn;
  D.trace_cap = capacity;
  D.trace_lv = tl;
  D.trace_lv_ns = tln;
  D.trace_lv_cap = level_capacity;
  int rc = run_kernel(g, D, g->stream);
  if (rc == MF_OK && level_capacity > 0) {
    const long long nl = g->h_ctl->levels < level_capacity ? g->h_ctl->levels : level_capacity;
    e = cudaMemcpy(level_sizes, tl, (size_t)nl * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && tln) e = cudaMemcpy(level_ns, tln, (size_t)nl * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "trace copy");
  }
  if (levels && rc == MF_OK) *levels = g->h_ctl->levels;
  if (rc == MF_OK && capacity > 0) {
    const long long nr = g->h_ctl->rounds < capacity ? g->h_ctl->rounds : capacity;
    int2 *h = (int2 *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int2));
    if (!h) {
      rc = fail(MF_ERR_OOM, "host allocation");
    } else {
      e = cudaMemcpy(h, tr, (size_t)nr * sizeof(int2), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && trn) e = cudaMemcpy(round_ns, trn, (size_t)nr * sizeof(int), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) rc = cuda_fail(e, "trace copy");
      for (long long k = 0; k < nr && rc == MF_OK; k++) {
        live[k] = h[k].x;
        relabel_before[k] = h[k].y;
      }
      free(h);
    }
  }
  if (rounds && rc == MF_OK) *rounds = g->h_ctl->rounds;
  release();
  return rc;
}

int mf_get_stats(const mf_graph *g, mf_stats *out) {
  clear_error();
  if (!g || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *out = g->stats;
  return MF_OK;
}

int mf_run_rounds(mf_graph *g, int64_t rounds, int32_t final_relabel, int32_t *residual, int32_t *label,
                  int64_t *excess, int64_t *rounds_done) {
  clear_error();
  if (!g) return fail(MF_ERR_INVALID_ARG, "graph is NULL");
  if (rounds < 0) return fail(MF_ERR_INVALID_ARG, "rounds must be >= 0");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  Dev D = make_dev(g);
  D.mode = MODE_ROUNDS;
  D.stop_rounds = rounds;
  D.final_gr = final_relabel ? 1 : 0;
  int rc = run_kernel(g, D, g->stream);
  if (rc) return rc;
  if (rounds_done) *rounds_done = g->h_ctl->stopped_round;
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  if (residual && m > 0) {
    int2 *tmp = (int2 *)malloc(m * sizeof(int2));
    if (!tmp) return fail(MF_ERR_OOM, "host allocation");
    e = cudaMemcpyAsync(tmp, g->rr, m * sizeof(int2), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    for (size_t a = 0; a < m && e == cudaSuccess; a++) residual[a] = tmp[a].x;
    free(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "state copy");
  }
  if (label) {
    e = cudaMemcpy2DAsync(label, sizeof(int), g->vs, sizeof(VRec), sizeof(int), n, cudaMemcpyDeviceToHost,
                          g->stream);  // the label half of every slot-0 entry
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state copy");
    for (size_t v = 0; v < n; v++)
      if (label[v] > g->n) label[v] = g->n;
  }
  if (excess) {
    e = cudaMemcpy2DAsync(excess, 8, &g->vs->exc, sizeof(VRec), 8, n, cudaMemcpyDeviceToHost,
                          g->stream);  // the excess of every record
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state copy");
  }
  return MF_OK;
}

}  // extern "C"
