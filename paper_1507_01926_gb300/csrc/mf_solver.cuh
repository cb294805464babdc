#pragma once
// The persistent solver kernel (instantiated by mf_kernels_s0.cu / _s1.cu for
// single graphs and by mf_kernels_m0.cu / _m1.cu for batches and service
// unions, units that compile in parallel; mf_solver.cu holds the launch code).
//
// Synchronous parallel push-relabel (arXiv:1507.01926, Section 3.1 and
// Algorithm 1) with parallel global relabeling (Section 3, Algorithm 2) as one
// persistent cooperative kernel for sm_103a.
//
// One launch runs a whole solve: initialisation and source saturation,
// phase 1 (rounds of discharge, a BFS global relabel whenever the relabel work
// since the last one exceeds the threshold), phase 2 (the same rounds toward
// s return the excess that cannot reach t), the cut BFS from s and the
// outputs. Phases are separated by a grid barrier whose waits are bounded in
// time (MF_ERR_TIMEOUT instead of a hang). A round needs one barrier: the
// label a vertex computes in round r goes to the other parity slot, and the
// merge steps of Algorithm 1 (d := d', e += addedExcess) for round r run
// during round r + 1, where they touch nothing that round reads.
//
// Data model (mf_device.cuh): CSR of paired slots with an inline copy of the
// reverse residual (int2 rr[a] = {res[a], res[rev[a]]}: the residual of an
// arc's reverse is kept next to the arc, as in the paper's layout, Section 4.2),
// per-vertex {label, active stamp} slots by round parity, int64 excess.
// Vertex lists are plain arrays filled by warp-aggregated atomics; a list is
// consumed in tiles of blockDim entries that are binned in shared memory by
// degree (thread / warp / CTA per vertex).
//
// Readings of the listing that the kernel follows (Algorithm 1):
//  * the activity test of a neighbour w (a test of its excess) is membership
//    of w in the current working set, kept as a round stamp;
//  * pushes use the local excess of the discharging vertex;
//  * excess received by a vertex of the working set goes to its addedExcess
//    (atomic), excess received by any other vertex is added to its excess
//    directly (atomic; nobody reads it during the round);
//  * the next working set holds every vertex that received excess (not the
//    sink) plus every discharged vertex left with excess and d' < n; a vertex
//    whose label reached n is skipped when its turn comes; excess pushed into
//    the sink accumulates into e(sink), which is the flow value;
//  * arcs of one vertex are scanned in CSR order; a warp or CTA reproduces
//    that order with an exclusive prefix sum of the pushable residuals;
//  * the source keeps label n + 1 internally (equivalent to n: no label
//    reaches n + 2, and relabels start from n);
//  * after every global relabel the working set is rebuilt from all vertices
//    with excess and 0 < d < n, and a phase ends only when a rebuild right
//    after a global relabel finds no active vertex.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "mf.h"
#include "mf_device.cuh"

namespace cg = cooperative_groups;

namespace mf {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KT = 8;           // largest degree handled by one thread (register-cached arcs)
constexpr int MAX_BLOCK = 512;  // largest CTA
constexpr int MAX_WARPS = MAX_BLOCK / 32;

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add64(unsigned long long *p, unsigned long long x) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(x) : "memory");
}

__device__ __forceinline__ int vol_read(const int *p) { return *(const volatile int *)p; }

// Index checks of the gathers (a build with MF_CHECK_BOUNDS, for tests): an
// index outside its array is recorded in the error word (MF_ERR_INTERNAL, the
// solver source line in err_where and the index in bad_index, first one wins)
// and replaced by 0, so the access stays inside the array and the solve ends
// at its next grid barrier; no trap. Without MF_CHECK_BOUNDS the macros are the
// index itself.
#ifdef MF_CHECK_BOUNDS
static __device__ __noinline__ long long mf_bad_index(const Dev &D, long long i, int line) {
  if (atomicCAS(&D.ctl->err, 0, MF_ERR_INTERNAL) == 0) {
    atomicExch(&D.ctl->err_where, 1000 + line);
    atomicExch(reinterpret_cast<unsigned long long *>(&D.ctl->bad_index), (unsigned long long)i);
  }
  return 0;
}
#define MF_CHECKED(D, i, lim) \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(lim)) ? (i)                     \
                                                                              : (decltype((i) + 0))mf_bad_index(D, (i), __LINE__))
#define MF_SLOT(D, a) MF_CHECKED(D, a, (D).m)
#define MF_VTX(D, v) MF_CHECKED(D, v, (D).n)
#define MF_ROW(D, v) MF_CHECKED(D, v, (D).n + 1)
#else
#define MF_SLOT(D, a) (a)
#define MF_VTX(D, v) (v)
#define MF_ROW(D, v) (v)
#endif

// label slot p / active stamp slot p of v
__device__ __forceinline__ int *lab_ptr(const Dev &D, int v, int p) { return reinterpret_cast<int *>(D.vs + MF_VTX(D, v)) + 2 * p; }
__device__ __forceinline__ int *act_ptr(const Dev &D, int v, int p) { return lab_ptr(D, v, p) + 1; }
// {label, stamp} of v in slot p
__device__ __forceinline__ int2 load_slot(const Dev &D, int p, int v) {
  return __ldcg(reinterpret_cast<const int2 *>(D.vs + MF_VTX(D, v)) + p);
}

__device__ __forceinline__ int cap_of(const Dev &D, int v) { return D.vinst ? __ldg(&D.vinst[v]).x : D.n_cap; }
// {label cap, instance} of v (instance -1 for a single-instance graph). The
// solver is compiled twice: MULTI for batches and service unions (per-vertex
// label caps and the per-instance relabel schedules), and without for single
// graphs, which then carry none of that code or its registers.
template <bool MULTI>
__device__ __forceinline__ int2 vinst_of(const Dev &D, int v) {
  if (MULTI) return __ldg(&D.vinst[v]);
  return make_int2(D.n_cap, -1);
}

// excess and addedExcess of v share one 16-byte entry
__device__ __forceinline__ long long *exc_ptr(const Dev &D, int v) { return &D.vs[MF_VTX(D, v)].exc; }
__device__ __forceinline__ long long *add_ptr(const Dev &D, int v) { return &D.vs[MF_VTX(D, v)].added; }
__device__ __forceinline__ longlong2 load_ea(const Dev &D, int v) {
  return __ldcg(reinterpret_cast<const longlong2 *>(&D.vs[MF_VTX(D, v)].exc));
}

__device__ __forceinline__ void set_err(const Dev &D, int code, int where) {
  if (atomicCAS(&D.ctl->err, 0, code) == 0) atomicExch(&D.ctl->err_where, where);
}

__device__ __forceinline__ long long take_added(const Dev &D, int v) {
  return (long long)atomicExch(reinterpret_cast<unsigned long long *>(add_ptr(D, v)), 0ULL);
}

__device__ __forceinline__ void atomic_add64(long long *p, long long x) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)x);
}

// Win rule of Section 3.1 for two active neighbours, on the labels at the
// start of the round: v owns the pair iff d(v) = d(w) + 1, or d(v) < d(w) - 1,
// or d(v) = d(w) and v < w. Exactly one of v, w wins.
__device__ __forceinline__ bool wins(int dv, int dw, int v, int w) {
  return (dv == dw + 1) || (dv < dw - 1) || (dv == dw && v < w);
}

// Push delta along slot a (reverse slot ra): res[a] -= delta, res[ra] += delta,
// with the inline reverse copies updated alike. Each slot is one 64-bit word
// {res, rres}; the win rule gives every pair a single pusher per round and the
// pair sums stay within int32, so the packed adds never carry between halves.
__device__ __forceinline__ void push_res(const Dev &D, int a, int ra, int delta) {
  unsigned long long d64 = (unsigned long long)(unsigned)delta;
  atomicAdd(reinterpret_cast<unsigned long long *>(&D.rr[MF_SLOT(D, a)]), (d64 << 32) - d64);
  atomicAdd(reinterpret_cast<unsigned long long *>(&D.rr[MF_SLOT(D, ra)]), d64 - (d64 << 32));
}

__device__ __forceinline__ int *list_of(const Dev &D, int gen) { return D.list[gen % 3]; }

// Appends one value per calling thread to the list of generation gen with one
// atomic per converged group of lanes. Lists hold at most n entries (every
// list holds distinct vertices); an overflow would be a solver bug and is
// reported as MF_ERR_INTERNAL instead of being written.
__device__ __forceinline__ void append(const Dev &D, int gen, int val) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&D.ctl->cnt[gen & 3], (int)g.size());
  base = g.shfl(base, 0);
  const int idx = base + (int)g.thread_rank();
  if (idx < D.n)
    list_of(D, gen)[idx] = val;
  else
    set_err(D, MF_ERR_INTERNAL, 11);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

__device__ __forceinline__ int warp_min(int x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = min(x, __shfl_xor_sync(FULL, x, o));
  return x;
}

__device__ __forceinline__ long long warp_incl_scan(long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

constexpr int QCAP = 2048;  // per-CTA staging of list appends

// Control words as they stood at the last grid barrier, read once by thread 0
// and shared with the CTA: the error word, the list sizes, the per-round
// relabel work and the time-based relabel requests.
struct Snap {
  int err;
  int cnt[4];
  int lcnt[4];
  long long work[3];
  int gr_req[2];
  int due_any[3];
  int ph2_started, cut_pending;
};

struct Shared {
  unsigned long long bars;  // grid barriers passed by this CTA
  Snap snap;
  int pick;
  int flag;
  int qn;                   // staged appends (may exceed QCAP; the excess went straight to the list)
  int qbase;
  int qk;                   // staged entries to publish to the list in global memory
  int lk;                   // staged entries to keep in shared memory
  long long wsum;
  int imin[MAX_WARPS];
  long long lsum[MAX_WARPS];
  int lqn[3];               // kept entries of list generation g, in lq[g % 3]
  int qbuf[QCAP];
  int qrow[MAX_BLOCK];      // BFS staging: row[v] of qbuf[i] (i < MAX_BLOCK) when known (qdeg[i] >= 0)
  int qdeg[MAX_BLOCK];      // BFS staging: degree of qbuf[i] (i < MAX_BLOCK), -1 when unknown
  int lq[3][MAX_BLOCK];
  // read-only data of the vertex thread t handles first in the next round or
  // BFS level, loaded while thread 0 waits at the grid barrier (pv[t] = -1:
  // none). Row offsets and heads never change, so an entry is valid for its
  // vertex whenever it is read.
  int pv[MAX_BLOCK];
  int pbeg[MAX_BLOCK];
  int pdeg[MAX_BLOCK];
  int phead[KT][MAX_BLOCK];
};

// Stages one append to the list of generation gen in shared memory; phase_end
// publishes the CTA's staged entries with one global atomic.
__device__ __forceinline__ void qpush(const Dev &D, Shared &sh, int gen, int val) {
  const int i = atomicAdd(&sh.qn, 1);
  if (i < QCAP) {
    sh.qbuf[i] = val;
    if (i < MAX_BLOCK) sh.qdeg[i] = -1;
  } else {
    append(D, gen, val);
  }
}

// qpush with the row offsets of the staged vertex (BFS: read while the vertex
// was offered its label, so that an expansion inside the CTA starts at its arcs).
__device__ __forceinline__ void qpush_row(const Dev &D, Shared &sh, int gen, int val, int beg, int deg) {
  const int i = atomicAdd(&sh.qn, 1);
  if (i < QCAP) {
    sh.qbuf[i] = val;
    if (i < MAX_BLOCK) {
      sh.qrow[i] = beg;
      sh.qdeg[i] = deg;
    }
  } else {
    append(D, gen, val);
  }
}

// Entries of a list that one CTA takes per sweep: a whole block when the list
// fills the grid; otherwise the list is spread evenly over all CTAs in warp
// multiples, so that a short list loads every SM's memory pipeline a little
// instead of a few SMs heavily.
__device__ __forceinline__ int sweep_chunk(int total) {
  const int per = (int)(((long long)total + gridDim.x - 1) / gridDim.x);
  const int w = (per + 31) & ~31;
  return w < (int)blockDim.x ? w : (int)blockDim.x;
}

// All threads of the CTA call this at the end of a phase that staged entries of
// list generation gen, and adds the CTA's sum of `work` to *work_dst
// (nullable). At most D.keep_local staged entries stay in the CTA's shared
// memory (lq[gen % 3]; their number is added to lcnt), more are published to
// the list in global memory with one atomic for the space. Every generation is
// staged by exactly one phase. Two CTA barriers; the next phase starts after a
// grid barrier, which begins with a CTA barrier.
static __device__ void phase_end(const Dev &D, Shared &sh, int gen, long long work, long long *work_dst) {
  const long long w = warp_sum(work);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(reinterpret_cast<unsigned long long *>(&sh.wsum), (unsigned long long)w);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int k = min(sh.qn, QCAP);
    const bool keep = sh.qn <= D.keep_local;  // keep_local <= MAX_BLOCK < QCAP: nothing overflowed
    sh.qk = keep ? 0 : k;
    sh.lk = keep ? k : 0;
    sh.lqn[gen % 3] = keep ? k : 0;
    if (!keep && k > 0) sh.qbase = atomicAdd(&D.ctl->cnt[gen & 3], k);
    if (keep && k > 0) atomicAdd(&D.ctl->lcnt[gen & 3], k);
    if (work_dst && sh.wsum) atomic_add64(work_dst, sh.wsum);
    sh.qn = 0;
    sh.wsum = 0;
  }
  __syncthreads();
  const int k = sh.qk;
  if (k > 0) {
    const int base = sh.qbase;
    int *L = list_of(D, gen);
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const int idx = base + i;
      if (idx < D.n)
        L[idx] = sh.qbuf[i];
      else
        set_err(D, MF_ERR_INTERNAL, 11);
    }
  }
  int *lq = sh.lq[gen % 3];
  for (int i = threadIdx.x; i < sh.lk; i += blockDim.x) lq[i] = sh.qbuf[i];
}

// Block-wide sum of a 64-bit value (all threads call; result valid in all).
static __device__ long long block_sum(long long x, Shared &sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  x = warp_sum(x);
  __syncthreads();
  if (lane == 0) sh.lsum[wid] = x;
  __syncthreads();
  long long t = 0;
  for (int i = 0; i < nw; i++) t += sh.lsum[i];
  __syncthreads();
  return t;
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// What the phase after a grid barrier is, for the prefetch in the barrier
// window.
enum PfKind : int { PF_NONE = 0, PF_ROUND = 1, PF_LEVEL = 2 };

// Runs on every thread between its CTA's arrival at a grid barrier and the
// barrier's completion. The next phase hands thread t its CTA's kept entry t
// of generation `next` (a round: then entry t - n of the kept entries of
// generation `prev`, prev >= 0, whose merge step it does): load that vertex's
// row offsets and arc heads into shared memory (they never change) and pull
// what the phase reads and updates (residual pairs, reverse-slot indices,
// vertex records, neighbours' records or BFS labels) into L2. Loads of mutable
// data would be stale, a prefetch into L2 is not.
__device__ __forceinline__ void prefetch_next(const Dev &D, Shared &sh, int kind, int next, int prev) {
  const int t = threadIdx.x;
  sh.pv[t] = -1;
  if (kind == PF_NONE) return;
  const int nl = sh.lqn[next % 3];
  if (t < nl) {
    const int v = sh.lq[next % 3][t];
    const int beg = __ldg(&D.row[MF_ROW(D, v)]);
    const int deg = __ldg(&D.row[MF_ROW(D, v + 1)]) - beg;
    if (deg > KT) return;
    int h[KT];
#pragma unroll
    for (int i = 0; i < KT; i++) h[i] = i < deg ? __ldg(&D.head[MF_SLOT(D, beg + i)]) : 0;
    if (deg > 0) {
      prefetch_l2(&D.rr[MF_SLOT(D, beg)]);
      prefetch_l2(&D.rr[MF_SLOT(D, beg + deg - 1)]);
    }
    if (kind == PF_ROUND) {
      prefetch_l2(&D.vs[MF_VTX(D, v)]);
      if (deg > 0) {
        prefetch_l2(&D.rev[MF_SLOT(D, beg)]);
        prefetch_l2(&D.rev[MF_SLOT(D, beg + deg - 1)]);
      }
#pragma unroll
      for (int i = 0; i < KT; i++)
        if (i < deg) prefetch_l2(&D.vs[MF_VTX(D, h[i])]);
    } else {
#pragma unroll
      for (int i = 0; i < KT; i++)
        if (i < deg) prefetch_l2(&D.blab[MF_VTX(D, h[i])]);
    }
#pragma unroll
    for (int i = 0; i < KT; i++) sh.phead[i][t] = h[i];
    sh.pbeg[t] = beg;
    sh.pdeg[t] = deg;
    sh.pv[t] = v;
  } else if (kind == PF_ROUND && prev >= 0 && t - nl < sh.lqn[prev % 3]) {
    prefetch_l2(&D.vs[MF_VTX(D, sh.lq[prev % 3][t - nl])]);
  }
}

// Grid barrier on a monotone 64-bit arrival counter: CTA k's b-th arrival is
// complete when the counter reaches b * gridDim.x. The CTA barrier orders the
// CTA's writes before thread 0's release add, and thread 0's acquire load
// before the CTA barrier that releases the other threads. While thread 0
// waits, every thread runs the prefetch for the next phase (`pf`, see
// prefetch_next). Every wait is bounded by D.timeout_ns; on expiry the error
// word is set and all CTAs leave at their next barrier.
static __device__ bool grid_sync(const Dev &D, Shared &sh, int where, int pf = PF_NONE, int next = 0, int prev = -1) {
  __syncthreads();
  unsigned long long *c = reinterpret_cast<unsigned long long *>(&D.ctl->bar);
  if (threadIdx.x == 0) red_release_add64(c, 1ULL);
  if (pf != PF_NONE) prefetch_next(D, sh, pf, next, prev);
  if (threadIdx.x == 0) {
    const unsigned long long target = (sh.bars + 1) * (unsigned long long)gridDim.x;
    if (ld_acquire64(c) < target) {
      const unsigned long long t0 = gtimer();
      unsigned spins = 0;
      while (ld_acquire64(c) < target) {
        if ((++spins & 31u) == 0 && gtimer() - t0 > D.timeout_ns) {
          set_err(D, MF_ERR_TIMEOUT, where);
          break;
        }
        __nanosleep(20);
      }
    }
    sh.bars++;
    // one round trip for every control word the next phase reads
    const Ctl *cw = D.ctl;
    const int err = vol_read(&cw->err);
    const int4 k = __ldcg(reinterpret_cast<const int4 *>(cw->cnt));
    const int4 lk = __ldcg(reinterpret_cast<const int4 *>(cw->lcnt));
    const long long w0 = __ldcg(&cw->work[0]), w1 = __ldcg(&cw->work[1]), w2 = __ldcg(&cw->work[2]);
    const int2 q = __ldcg(reinterpret_cast<const int2 *>(cw->gr_req));
    const int d0 = vol_read(&cw->due_any[0]), d1 = vol_read(&cw->due_any[1]), d2 = vol_read(&cw->due_any[2]);
    const int p2 = vol_read(&cw->ph2_started), cp = vol_read(&cw->cut_pending);
    sh.snap.err = err;
    sh.snap.cnt[0] = k.x;
    sh.snap.cnt[1] = k.y;
    sh.snap.cnt[2] = k.z;
    sh.snap.cnt[3] = k.w;
    sh.snap.lcnt[0] = lk.x;
    sh.snap.lcnt[1] = lk.y;
    sh.snap.lcnt[2] = lk.z;
    sh.snap.lcnt[3] = lk.w;
    sh.snap.work[0] = w0;
    sh.snap.work[1] = w1;
    sh.snap.work[2] = w2;
    sh.snap.gr_req[0] = q.x;
    sh.snap.gr_req[1] = q.y;
    sh.snap.due_any[0] = d0;
    sh.snap.due_any[1] = d1;
    sh.snap.due_any[2] = d2;
    sh.snap.ph2_started = p2;
    sh.snap.cut_pending = cp;
  }
  __syncthreads();
  return sh.snap.err == 0;
}

// Size of the list of generation gen in global memory as of the last grid
// barrier.
__device__ __forceinline__ int list_count(const Dev &D, const Shared &sh, int gen) {
  return min(sh.snap.cnt[gen & 3], D.n);
}

// Entries of generation gen in global memory and in all CTAs' shared memory.
__device__ __forceinline__ long long gen_total(const Dev &D, const Shared &sh, int gen) {
  return (long long)list_count(D, sh, gen) + sh.snap.lcnt[gen & 3];
}

// The items one CTA handles in a phase: its kept entries of up to two
// generations (a, then b), then its share of the concatenation of two lists in
// global memory (ga[0, na), then gb[0, nb)), spread over all CTAs in chunks of
// `per` entries. Items are taken blockDim at a time; every thread of the CTA
// runs the same number of sweeps.
struct Sweep {
  const int *la, *lb, *ga, *gb;
  int nla, nlb, na, nb;
  int per;     // global chunk size (0: no global entries)
  int gitems;  // global items of this CTA (whole chunks; the last may run past na + nb)
  int items;   // all items of this CTA
};

__device__ __forceinline__ Sweep make_sweep(const int *la, int nla, const int *lb, int nlb, const int *ga, int na,
                                            const int *gb, int nb) {
  Sweep w{la, lb, ga, gb, nla, nlb, na, nb, 0, 0, 0};
  const int total = na + nb;
  if (total > 0) {
    w.per = sweep_chunk(total);
    const int chunks = (total + w.per - 1) / w.per;
    const int mine = (int)blockIdx.x < chunks ? (chunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    w.gitems = mine * w.per;
  }
  w.items = nla + nlb + w.gitems;
  return w;
}

// Item `it` of the CTA: returns 1 (and the vertex) for an entry of the first
// generation, 2 for one of the second, 0 for none.
__device__ __forceinline__ int sweep_item(const Sweep &w, int it, int &v) {
  if (it < w.nla) {
    v = w.la[it];
    return 1;
  }
  it -= w.nla;
  if (it < w.nlb) {
    v = w.lb[it];
    return 2;
  }
  it -= w.nlb;
  if (it >= w.gitems) return 0;
  const int c = it / w.per;
  const long long idx = ((long long)blockIdx.x + (long long)c * gridDim.x) * w.per + (it - c * w.per);
  if (idx < w.na) {
    v = __ldcg(&w.ga[idx]);
    return 1;
  }
  if (idx < (long long)w.na + w.nb) {
    v = __ldcg(&w.gb[idx - w.na]);
    return 2;
  }
  return 0;
}

// Per-thread counters, summed over the grid at the end of a launch. scans_dis
// counts every slot a discharge pass (or a relabel pass of the simple rounds)
// examines, zero residuals included; scans_res those of them with positive
// residual. 32 bits per thread keep them out of the way of the solver's
// registers: one thread would need 2^32 events of one kind in one launch to
// wrap, billions of times its share of any solve.
struct TStat {
  unsigned scans_dis = 0, scans_res = 0, scans_bfs = 0, pushes = 0, relabels = 0, visits_dis = 0, visits_bfs = 0;
};

// ------------------------------------------------------------------ partial relabels
//
// A multi-instance graph (batch or service union) shares rounds and global
// relabels among its instances. Vertices, labels and arcs of one instance never
// touch another's, and an instance without an active vertex has no excess to
// move: a global relabel leaves it as it is. So a relabel taken while some
// vertex is active covers only the instances of the working set ("live"
// instances, flagged with the relabel's number `epoch` in D.live); the first
// relabel of a phase and the one that confirms the end of a phase cover every
// instance. The vertex loops of such a relabel walk the static tiles of the
// live instances (D.tiles: runs of vertices of one instance).

struct Sel {
  bool on;    // cover only the instances whose D.live entry equals epoch
  int epoch;
};

// Runs f(v, valid) for every vertex the relabel covers, in sweeps that are
// uniform across the CTA (valid = false on the lanes past the end of a run,
// so warp collectives inside f see every lane).
template <typename F>
__device__ __forceinline__ void for_covered(const Dev &D, const Sel &S, F f) {
  if (!S.on) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < D.n; b += stride) {
      const long long v = b + threadIdx.x;
      f(v < D.n ? (int)v : 0, v < D.n);
    }
    return;
  }
  for (int k = blockIdx.x; k < D.ntiles; k += gridDim.x) {
    const int4 T = __ldg(&D.tiles[k]);
    if (__ldcg(&D.live[T.z]) != S.epoch) continue;  // uniform in the CTA
    for (int b = T.x; b < T.y; b += blockDim.x) {
      const int v = b + (int)threadIdx.x;
      f(v < T.y ? v : T.x, v < T.y);
    }
  }
}

// Relabel schedule of instance k, checked at a visit of one of its vertices in
// round rnd (one lane per instance and warp): with gr_time_ratio > 0 the
// instance asks for a global relabel once it has run more than gr_time_ratio
// times the depth of its last relabel in rounds since (the work rule is checked
// where the work is added, inst_add_work). Reads only words that change at
// relabels.
__device__ __forceinline__ void inst_check(const Dev &D, int k, int rnd) {
  if (!(D.gr_time_ratio > 0)) return;
  InstState *I = D.inst + k;
  const int2 ld = __ldcg(reinterpret_cast<const int2 *>(&I->last));  // {last, depth}
  if ((double)(rnd - ld.x) > D.gr_time_ratio * (double)max(ld.y, 1) && !__ldcg(&I->due)) {
    I->due = 1;
    D.ctl->due_any[rnd % 3] = 1;  // by round, like the relabel work: a CTA still reading the last round's
  }                               // control words must not see this round's requests
}

// Adds relabel work w to instance k in round rnd; the add that takes the
// instance's work past its threshold (alpha n_k + m_k) / freq (Algorithm 1's
// rule on the instance's own n and m) asks for a global relabel. Exactly one
// add crosses, whatever the order of the atomics.
__device__ __forceinline__ void inst_add_one(const Dev &D, int k, long long w, int rnd) {
  InstState *I = D.inst + k;
  const long long thr = __ldcg(&I->thr);
  const long long old = (long long)atomicAdd(
      reinterpret_cast<unsigned long long *>(&D.inst_work[(size_t)k * INST_WORK_STRIDE]), (unsigned long long)w);
  if (old <= thr && old + w > thr) {
    I->due = 1;
    D.ctl->due_any[rnd % 3] = 1;
  }
}

// inst_add_one for the lanes of a warp with work w > 0, lanes with work for the
// same instance combined into one atomic. All lanes of the warp call.
__device__ __forceinline__ void inst_add_work(const Dev &D, int k, long long w, int rnd) {
  if (!__ballot_sync(FULL, w > 0)) return;
  if (w > 0) {
    cg::coalesced_group g = cg::coalesced_threads();
    cg::coalesced_group part = cg::labeled_partition(g, k);
    const long long sum = cg::reduce(part, w, cg::plus<long long>());
    if (part.thread_rank() == 0) inst_add_one(D, k, sum, rnd);
  }
}

// Carries one working-set entry over a partial relabel (D.carry, one atomic
// per converged group of lanes).
__device__ __forceinline__ void carry_push(const Dev &D, int v) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&D.ctl->carry_n, (int)g.size());
  base = g.shfl(base, 0);
  const int idx = base + (int)g.thread_rank();
  if (idx < D.n)
    D.carry[idx] = v;
  else
    set_err(D, MF_ERR_INTERNAL, 11);
}

// Merge step of the previous round for vertex u of its working set, as the
// next round (stamp r, labels in slot p = r & 1) would do it: unless u is in
// that round's working set, carry its label into slot p ^ 1 and fold its
// addedExcess into its excess.
__device__ __forceinline__ void merge_prev(const Dev &D, int u, int r) {
  const int p = r & 1;
  const int2 y = load_slot(D, p, u);
  if (y.y != r) {
    *lab_ptr(D, u, p ^ 1) = y.x;
    const long long ad = take_added(D, u);
    if (ad) atomic_add64(exc_ptr(D, u), ad);
  }
}

// Share of its relabel schedule instance k has used up by round rnd (1 = due):
// the larger of its relabel work against its threshold and its rounds since
// its last relabel against gr_time_ratio times that relabel's depth.
__device__ __forceinline__ double inst_progress(const Dev &D, int k, int rnd) {
  const InstState *I = D.inst + k;
  double p = (double)__ldcg(&D.inst_work[(size_t)k * INST_WORK_STRIDE]) / (double)max(__ldcg(&I->thr), 1LL);
  if (D.gr_time_ratio > 0)
    p = fmax(p, (double)(rnd - __ldcg(&I->last)) / (D.gr_time_ratio * (double)max(__ldcg(&I->depth), 1)));
  return p;
}

// First step of a partial global relabel before the round with stamp r and
// index rnd (working set: list generation gen; previous working set: gen - 1
// when prev_valid): the instances that asked for a relabel, and with them
// (except in the simple rounds, whose instances keep schedules of their own so
// that their flows do not depend on the mix) the instances that relabeled
// vertices since their last relabel and have used up at least half of their
// schedule (so that relabels of many instances coincide), are flagged
// with `epoch` in D.live; the working-set entries of the others are saved in
// D.carry, and the merge step of the previous round is done now for their
// vertices (the relabel rebuilds the flagged instances, whose lists the BFS
// overwrites). Two grid barriers.
static __device__ __noinline__ bool partial_prep(const Dev &D, Shared &sh, int r, int gen, bool prev_valid, int epoch,
                                                 int rnd) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  for (int k = tid; k < D.ninst; k += nthr)
    if (__ldcg(&D.inst[k].due) ||
        (!D.simple && __ldcg(&D.inst_work[(size_t)k * INST_WORK_STRIDE]) > 0 && inst_progress(D, k, rnd) >= 0.5))
      D.live[k] = epoch;
  if (tid == 0) D.ctl->carry_n = 0;
  if (!grid_sync(D, sh, 2)) return false;
  auto kept = [&](int v) { return __ldcg(&D.live[__ldg(&D.vinst[v]).y]) != epoch; };
  if (prev_valid) {
    const int cnt = list_count(D, sh, gen - 1);
    const int *L = list_of(D, gen + 2);
    for (int i = tid; i < cnt; i += nthr) {
      const int u = __ldcg(&L[i]);
      if (kept(u)) merge_prev(D, u, r);
    }
    const int *lq = sh.lq[(gen + 2) % 3];
    for (int i = threadIdx.x; i < sh.lqn[(gen + 2) % 3]; i += blockDim.x)
      if (kept(lq[i])) merge_prev(D, lq[i], r);
  }
  {
    const int cnt = list_count(D, sh, gen);
    const int *L = list_of(D, gen);
    for (int i = tid; i < cnt; i += nthr) {
      const int v = __ldcg(&L[i]);
      if (kept(v)) carry_push(D, v);
    }
    const int *lq = sh.lq[gen % 3];
    for (int i = threadIdx.x; i < sh.lqn[gen % 3]; i += blockDim.x)
      if (kept(lq[i])) carry_push(D, lq[i]);
  }
  return grid_sync(D, sh, 2);
}

// ------------------------------------------------------------------ discharge
//
// Algorithm 1, inner loop, for one vertex v of the working set of round r
// (labels read from slot p = r & 1): with the local excess ex and d' = d(v),
// repeat passes over the residual arcs in order:
//   admissible  <=> d'(v) = d(w) + 1 (old label of w);
//   w active and v loses the win rule and the arc is admissible => skip the
//     arc and end the discharge after this pass;
//   otherwise push min(res, ex) along an admissible arc;
//   relabel candidate: d(w) + 1 over arcs still residual with d(w) >= d'(v).
// After a pass: stop when ex = 0 or an arc was skipped; else d' := candidate
// minimum (starting at n), work += deg + beta, stop when d' = n.

struct RoundCtx {
  int r;     // round stamp
  int p;     // r & 1
  int next;  // list generation receiving the next working set
  int rnd;   // round index of the phase sequence (relabel schedules of multi-instance graphs)
};

// Excess delta reaches w (not the sink). Returns true when w must join the
// next working set through this call (first discovery this round).
__device__ __forceinline__ bool deliver(const Dev &D, const RoundCtx &R, int w, bool w_active, long long delta) {
  atomic_add64(w_active ? add_ptr(D, w) : exc_ptr(D, w), delta);
  return atomicExch(act_ptr(D, w, R.p ^ 1), R.r + 1) != R.r + 1;
}

__device__ __forceinline__ void finish_vertex(const Dev &D, Shared &sh, const RoundCtx &R, int v, int dp,
                                              long long ex, int cap_v) {
  *lab_ptr(D, v, R.p ^ 1) = dp;
  *exc_ptr(D, v) = ex;
  if (ex > 0 && dp < cap_v) {
    if (atomicExch(act_ptr(D, v, R.p ^ 1), R.r + 1) != R.r + 1) qpush(D, sh, R.next, v);
  }
}

// Sink deliveries of one lane are summed in `to_sink`; lanes that delivered
// to the same sink combine into one atomic.
__device__ __forceinline__ void flush_sink(const Dev &D, int sink, long long to_sink) {
  if (sink < 0) return;
  cg::coalesced_group g = cg::coalesced_threads();
  cg::coalesced_group part = cg::labeled_partition(g, sink);
  const long long sum = cg::reduce(part, to_sink, cg::plus<long long>());
  if (part.thread_rank() == 0) atomic_add64(exc_ptr(D, sink), sum);
}

// A vertex in the working set of round r whose label has reached the cap (it
// was discovered while it relabeled to n): carry its label into the next slot
// and fold its addedExcess into its excess.
__device__ __forceinline__ void retire_dead(const Dev &D, const RoundCtx &R, int v, int dv) {
  *lab_ptr(D, v, R.p ^ 1) = dv;
  const long long ad = take_added(D, v);
  if (ad) *exc_ptr(D, v) = __ldcg(exc_ptr(D, v)) + ad;
}

// One thread, deg <= KTD: arcs cached in registers for all passes. With
// `pre`, the heads were loaded during the last grid barrier (prefetch_next)
// and dv is not known yet: the vertex record, the residuals and all
// neighbours' label slots are read in one round trip, then a vertex whose
// label reached the cap is retired.
template <int KTD>
__device__ __forceinline__ void discharge_thread(const Dev &D, Shared &sh, const RoundCtx &R, int v, int beg,
                                                 int deg, int dv, int cap_v, TStat &st, long long &work, bool pre) {
  int wv[KTD], rs[KTD], dw[KTD], rv[KTD];
  unsigned act = 0;
  // excess: own value plus what neighbours delivered so far; exactly that
  // delivered amount is taken out of addedExcess at the end (later deliveries stay)
  // (simple rounds: only the round-start excess; deliveries are folded in after the pushes)
  longlong2 ea;
  if (pre) {
    const int2 own = load_slot(D, R.p, v);
    ea = load_ea(D, v);
#pragma unroll
    for (int i = 0; i < KTD; i++) {
      wv[i] = (i < KT && i < deg) ? sh.phead[i < KT ? i : 0][threadIdx.x] : 0;
      rs[i] = 0;
      dw[i] = 0;
      rv[i] = 0;
      if (i < deg) {
        rs[i] = __ldcg(&D.rr[MF_SLOT(D, beg + i)]).x;
        rv[i] = __ldg(&D.rev[MF_SLOT(D, beg + i)]);
        const int2 x = load_slot(D, R.p, wv[i]);
        dw[i] = x.x;
        if (x.y == R.r) act |= 1u << i;
      }
    }
    dv = own.x;
    if (dv >= cap_v) {
      retire_dead(D, R, v, dv);
      return;
    }
    st.visits_dis++;
#pragma unroll
    for (int i = 0; i < KTD; i++)
      if (rs[i] <= 0) act &= ~(1u << i);
  } else {
    ea = load_ea(D, v);
#pragma unroll
    for (int i = 0; i < KTD; i++) {
      wv[i] = 0;
      rs[i] = 0;
      dw[i] = 0;
      rv[i] = 0;
      if (i < deg) {
        wv[i] = __ldg(&D.head[MF_SLOT(D, beg + i)]);
        rs[i] = __ldcg(&D.rr[MF_SLOT(D, beg + i)]).x;
        rv[i] = __ldg(&D.rev[MF_SLOT(D, beg + i)]);
      }
    }
#pragma unroll
    for (int i = 0; i < KTD; i++)
      if (rs[i] > 0) {
        const int2 x = load_slot(D, R.p, wv[i]);
        dw[i] = x.x;
        if (x.y == R.r) act |= 1u << i;
      }
  }
  const long long got = D.simple ? 0 : ea.y;
  long long ex = ea.x + got;
  int dp = dv;
  long long to_sink = 0;
  int sink = -1;
  // Discovery test-and-set results are collected per arc and read only after
  // the discharge, so the atomics of several pushes are in flight together.
  unsigned tested = 0;
  int prev_stamp[KTD];
#pragma unroll
  for (int i = 0; i < KTD; i++) prev_stamp[i] = R.r + 1;
  for (;;) {
    int newl = cap_v;
    bool skipped = false;
#pragma unroll
    for (int i = 0; i < KTD; i++) {
      if (i < deg && ex > 0) st.scans_dis++;
      if (i < deg && ex > 0 && rs[i] > 0) {
        st.scans_res++;
        const bool adm = (dp == dw[i] + 1);
        if (adm && !D.simple && ((act >> i) & 1u) && !wins(dv, dw[i], v, wv[i])) {
          skipped = true;
        } else {
          if (adm) {
            const long long delta = rs[i] < ex ? (long long)rs[i] : ex;
            push_res(D, beg + i, rv[i], (int)delta);
            rs[i] -= (int)delta;
            ex -= delta;
            st.pushes++;
            if (dw[i] == 0) {
              to_sink += delta;
              sink = wv[i];
            } else {
              atomic_add64((act >> i) & 1u ? add_ptr(D, wv[i]) : exc_ptr(D, wv[i]), delta);
              if (!((tested >> i) & 1u)) {
                tested |= 1u << i;
                prev_stamp[i] = atomicExch(act_ptr(D, wv[i], R.p ^ 1), R.r + 1);
              }
            }
          }
          if (rs[i] > 0 && dw[i] >= dp) newl = min(newl, dw[i] + 1);
        }
      }
    }
    if (ex == 0 || skipped || D.simple) break;
    dp = newl;
    st.relabels++;
    work += deg + D.beta;
    if (dp >= cap_v) break;
  }
  if (got) atomic_add64(add_ptr(D, v), -got);
  if (D.simple)
    *exc_ptr(D, v) = ex;  // label and re-activation: relabel_phase
  else
    finish_vertex(D, sh, R, v, dp, ex, cap_v);
#pragma unroll
  for (int i = 0; i < KTD; i++)
    if (prev_stamp[i] != R.r + 1) qpush(D, sh, R.next, wv[i]);
  flush_sink(D, sink, to_sink);
}

// One warp (all 32 lanes call), arcs in chunks of 32.
static __device__ void discharge_warp(const Dev &D, Shared &sh, const RoundCtx &R, int v, int dv, int cap_v, TStat &st,
                               long long &work) {
  const int lane = threadIdx.x & 31;
  const int beg = __ldg(&D.row[MF_ROW(D, v)]);
  const int deg = __ldg(&D.row[MF_ROW(D, v + 1)]) - beg;
  long long ex = 0;
  if (lane == 0) ex = __ldcg(exc_ptr(D, v)) + (D.simple ? 0 : take_added(D, v));
  ex = __shfl_sync(FULL, ex, 0);
  int dp = dv;
  long long to_sink = 0;
  int sink = -1;
  for (;;) {
    int newl = cap_v;
    bool skipped = false;
    for (int c = 0; c < deg && ex > 0; c += 32) {
      const int i = c + lane;
      int w = 0, rs = 0, dw = 0;
      bool wact = false;
      if (i < deg) {
        w = __ldg(&D.head[MF_SLOT(D, beg + i)]);
        rs = __ldcg(&D.rr[MF_SLOT(D, beg + i)]).x;
        if (rs > 0) {
          const int2 x = load_slot(D, R.p, w);
          dw = x.x;
          wact = x.y == R.r;
        }
      }
      const bool resid = rs > 0;
      const bool adm = resid && dp == dw + 1;
      const bool skip = adm && !D.simple && wact && !wins(dv, dw, v, w);
      const bool pushable = adm && !skip;
      const long long pr = pushable ? (long long)rs : 0;
      const long long incl = warp_incl_scan(pr, lane);
      const long long excl = incl - pr;
      const long long total = __shfl_sync(FULL, incl, 31);
      long long delta = 0;
      if (pushable && excl < ex) delta = min((long long)rs, ex - excl);
      st.scans_dis += (i < deg ? 1 : 0);
      st.scans_res += (resid ? 1 : 0);
      bool found = false;
      if (delta > 0) {
        push_res(D, beg + i, __ldg(&D.rev[MF_SLOT(D, beg + i)]), (int)delta);
        rs -= (int)delta;
        st.pushes++;
        if (dw == 0) {
          to_sink += delta;
          sink = w;
        } else {
          found = deliver(D, R, w, wact, delta);
        }
      }
      if (found) qpush(D, sh, R.next, w);
      if (resid && !skip && rs > 0 && dw >= dp) newl = min(newl, dw + 1);
      skipped |= (__ballot_sync(FULL, skip) != 0);
      ex = total >= ex ? 0 : ex - total;
    }
    newl = warp_min(newl);
    if (ex == 0 || skipped || D.simple) break;
    dp = newl;
    if (lane == 0) {
      st.relabels++;
      work += deg + D.beta;
    }
    if (dp >= cap_v) break;
  }
  if (lane == 0) {
    if (D.simple)
      *exc_ptr(D, v) = ex;
    else
      finish_vertex(D, sh, R, v, dp, ex, cap_v);
  }
  __syncwarp();
  if (sink >= 0) flush_sink(D, sink, to_sink);
  __syncwarp();
}

// One CTA (all threads call), arcs in chunks of blockDim.
static __device__ void discharge_block(const Dev &D, const RoundCtx &R, int v, int dv, int cap_v, TStat &st,
                                long long &work, Shared &sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int beg = __ldg(&D.row[MF_ROW(D, v)]);
  const int deg = __ldg(&D.row[MF_ROW(D, v + 1)]) - beg;
  __syncthreads();
  if (threadIdx.x == 0) sh.lsum[0] = __ldcg(exc_ptr(D, v)) + (D.simple ? 0 : take_added(D, v));
  __syncthreads();
  long long ex = sh.lsum[0];
  int dp = dv;
  long long to_sink = 0;
  int sink = -1;
  for (;;) {
    int newl = cap_v;
    int skipped = 0;
    for (int c = 0; c < deg && ex > 0; c += blockDim.x) {
      const int i = c + threadIdx.x;
      int w = 0, rs = 0, dw = 0;
      bool wact = false;
      if (i < deg) {
        w = __ldg(&D.head[MF_SLOT(D, beg + i)]);
        rs = __ldcg(&D.rr[MF_SLOT(D, beg + i)]).x;
        if (rs > 0) {
          const int2 x = load_slot(D, R.p, w);
          dw = x.x;
          wact = x.y == R.r;
        }
      }
      const bool resid = rs > 0;
      const bool adm = resid && dp == dw + 1;
      const bool skip = adm && !D.simple && wact && !wins(dv, dw, v, w);
      const bool pushable = adm && !skip;
      const long long pr = pushable ? (long long)rs : 0;
      const long long incl_w = warp_incl_scan(pr, lane);
      __syncthreads();  // previous chunk finished reading sh
      if (lane == 31) sh.lsum[wid] = incl_w;
      if (threadIdx.x == 0) sh.flag = 0;
      __syncthreads();
      long long wbase = 0, total = 0;
      for (int k = 0; k < nw; k++) {
        long long s = sh.lsum[k];
        if (k < wid) wbase += s;
        total += s;
      }
      const long long excl = wbase + incl_w - pr;
      long long delta = 0;
      if (pushable && excl < ex) delta = min((long long)rs, ex - excl);
      st.scans_dis += (i < deg ? 1 : 0);
      st.scans_res += (resid ? 1 : 0);
      bool found = false;
      if (delta > 0) {
        push_res(D, beg + i, __ldg(&D.rev[MF_SLOT(D, beg + i)]), (int)delta);
        rs -= (int)delta;
        st.pushes++;
        if (dw == 0) {
          to_sink += delta;
          sink = w;
        } else {
          found = deliver(D, R, w, wact, delta);
        }
      }
      if (found) qpush(D, sh, R.next, w);
      if (resid && !skip && rs > 0 && dw >= dp) newl = min(newl, dw + 1);
      if (skip) sh.flag = 1;
      __syncthreads();
      skipped |= sh.flag;
      ex = total >= ex ? 0 : ex - total;
    }
    // block min of newl
    int wm = warp_min(newl);
    __syncthreads();
    if (lane == 0) sh.imin[wid] = wm;
    __syncthreads();
    newl = cap_v;
    for (int k = 0; k < nw; k++) newl = min(newl, sh.imin[k]);
    if (ex == 0 || skipped || D.simple) break;
    dp = newl;
    if (threadIdx.x == 0) {
      st.relabels++;
      work += deg + D.beta;
    }
    if (dp >= cap_v) break;
  }
  if (threadIdx.x == 0) {
    if (D.simple)
      *exc_ptr(D, v) = ex;
    else
      finish_vertex(D, sh, R, v, dp, ex, cap_v);
  }
  if (sink >= 0) flush_sink(D, sink, to_sink);
  __syncthreads();
}


// One round over a combined index space: entries [0, count) are the working
// set of this round (list generation gen), discharged; entries [count, count +
// cp) are the previous working set, whose members that are not in this one get
// the merge step of the previous round (label carried into the next slot,
// addedExcess folded into the excess). Both kinds run side by side on
// different threads. Discoveries go to generation gen + 1.
template <int KTD, bool MULTI>
__device__ void round_phase(const Dev &D, Shared &sh, int r, int gen, bool prev_valid, long long rnd, TStat &st,
                            unsigned long long &t_phase0) {
  const RoundCtx R{r, r & 1, gen + 1, (int)rnd};
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.ctl->cnt[(gen + 2) & 3] = 0;
    D.ctl->lcnt[(gen + 2) & 3] = 0;
    D.ctl->work[(rnd + 1) % 3] = 0;
    D.ctl->due_any[(rnd + 1) % 3] = 0;
  }
  // this round's working set (generation gen) and the previous one (gen - 1 = gen + 2 mod 3)
  const Sweep sw = make_sweep(sh.lq[gen % 3], sh.lqn[gen % 3], sh.lq[(gen + 2) % 3], prev_valid ? sh.lqn[(gen + 2) % 3] : 0,
                              list_of(D, gen), list_count(D, sh, gen), list_of(D, gen + 2),
                              prev_valid ? list_count(D, sh, gen - 1) : 0);
  const int lane = threadIdx.x & 31;
  long long work = 0;
  for (int off = 0; off < sw.items; off += blockDim.x) {
    int x = -1;
    const int kind = sweep_item(sw, off + (int)threadIdx.x, x);
    int v = -1, beg = 0, deg = 0, cls = 0, dv = 0, cap_v = 0, k = -1;
    if (kind == 1 && sh.pv[threadIdx.x] == x && sh.pdeg[threadIdx.x] <= D.bin_thread) {
      v = x;  // thread-sized, row and heads loaded during the last grid barrier
      const int2 vi = vinst_of<MULTI>(D, v);
      cap_v = vi.x;
      k = vi.y;
      beg = sh.pbeg[threadIdx.x];
      deg = sh.pdeg[threadIdx.x];
      cls = 4;
    } else if (kind == 1) {
      v = x;
      // label and row offsets in one round trip (the offsets are unused when the label is at the cap)
      const int b0 = __ldg(&D.row[MF_ROW(D, v)]), b1 = __ldg(&D.row[MF_ROW(D, v + 1)]);
      dv = __ldcg(lab_ptr(D, v, R.p));
      const int2 vi = vinst_of<MULTI>(D, v);
      cap_v = vi.x;
      if (dv >= cap_v) {
        retire_dead(D, R, v, dv);
        v = -1;
      } else {
        k = vi.y;
        beg = b0;
        deg = b1 - b0;
        cls = deg <= D.bin_thread ? 1 : (deg <= D.bin_warp ? 2 : 3);
        st.visits_dis++;
      }
    } else if (kind == 2) {
      const int u = x;
      const int2 y = load_slot(D, R.p, u);
      if (y.y != r) {  // not in this working set
        *lab_ptr(D, u, R.p ^ 1) = y.x;
        const long long ad = take_added(D, u);
        if (ad) atomic_add64(exc_ptr(D, u), ad);  // the excess of a non-member may receive pushes now
      }
    }
    if (MULTI && D.inst_relabel) {  // relabel schedule of the instances visited, one lane per instance
      const unsigned grp = __match_any_sync(FULL, k);
      if (k >= 0 && lane == __ffs(grp) - 1) inst_check(D, k, R.rnd);
    }
    for (bool any = D.cta_vertices && __syncthreads_or(cls == 3); any;) {  // CTA per vertex
      if (threadIdx.x == 0) sh.pick = -1;
      __syncthreads();
      if (cls == 3) sh.pick = threadIdx.x;
      __syncthreads();
      const int pt = sh.pick;
      if (pt < 0) break;
      if (threadIdx.x == pt) {
        cls = 0;
        sh.imin[0] = v;
        sh.imin[1] = dv;
        sh.imin[2] = cap_v;
        sh.imin[3] = k;
      }
      __syncthreads();
      const int bv = sh.imin[0], bdv = sh.imin[1], bcap = sh.imin[2], bk = sh.imin[3];
      const long long w0 = work;  // the block path accumulates its work in thread 0
      discharge_block(D, R, bv, bdv, bcap, st, work, sh);
      if (MULTI && D.inst_relabel && threadIdx.x == 0 && work > w0) inst_add_one(D, bk, work - w0, R.rnd);
    }
    for (;;) {  // warp per vertex
      const unsigned mm = __ballot_sync(FULL, cls == 2);
      if (!mm) break;
      const int leader = __ffs(mm) - 1;
      const int pv = __shfl_sync(FULL, v, leader);
      const int pdv = __shfl_sync(FULL, dv, leader);
      const int pcap = __shfl_sync(FULL, cap_v, leader);
      const int pk = __shfl_sync(FULL, k, leader);
      if (lane == leader) cls = 0;
      const long long w0 = work;  // the warp path accumulates its work in lane 0
      discharge_warp(D, sh, R, pv, pdv, pcap, st, work);
      if (MULTI && D.inst_relabel && lane == 0 && work > w0) inst_add_one(D, pk, work - w0, R.rnd);
    }
    long long wt = 0;
    if (cls == 1 || cls == 4) {
      const long long w0 = work;
      discharge_thread<KTD>(D, sh, R, v, beg, deg, dv, cap_v, st, work, cls == 4);
      wt = work - w0;
    }
    __syncwarp();
    if (MULTI && D.inst_relabel) inst_add_work(D, k, wt, R.rnd);
  }
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  const unsigned long long t1 = timer ? gtimer() : 0;
  phase_end(D, sh, R.next, work, &D.ctl->work[rnd % 3]);
  if (timer) {
    const unsigned long long t2 = gtimer();
    D.ctl->t_rwork += t1 - t_phase0;
    D.ctl->t_rtail += t2 - t1;
    t_phase0 = t2;
  }
}

// Simple synchronous rounds (Section 3, steps 2-3): after all pushes of the
// round, every vertex of the working set still holding excess relabels once,
// d := 1 + min{d(w) : (v,w) residual} with the round-start labels, capped at
// n; the new label goes to the next slot and the vertex re-enters the working
// set when it is below n. Vertices without excess keep their label.
template <bool MULTI>
__device__ void relabel_phase(const Dev &D, Shared &sh, int r, int gen, long long rnd, TStat &st) {
  const RoundCtx R{r, r & 1, gen + 1, (int)rnd};
  const Sweep sw = make_sweep(sh.lq[gen % 3], sh.lqn[gen % 3], nullptr, 0, list_of(D, gen), list_count(D, sh, gen),
                              nullptr, 0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long work = 0;
  for (int off = 0; off < sw.items; off += blockDim.x) {
    int x = -1;
    int v = -1, beg = 0, deg = 0, cls = 0, cap_v = 0, k = -1;
    if (sweep_item(sw, off + (int)threadIdx.x, x) == 1) {
      v = x;
      const int dv = __ldcg(lab_ptr(D, v, R.p));
      const int2 vi = vinst_of<MULTI>(D, v);
      cap_v = vi.x;
      k = vi.y;
      // Section 3 step 4 for this vertex: the excess it received this round joins its excess now
      const long long ex_own = __ldcg(exc_ptr(D, v));
      const long long ad = dv >= cap_v ? 0 : take_added(D, v);
      if (ad) *exc_ptr(D, v) = ex_own + ad;
      if (dv >= cap_v) {
        v = -1;  // retired in the push step
      } else if (ex_own == 0) {
        *lab_ptr(D, v, R.p ^ 1) = dv;
        v = -1;
      } else {
        beg = __ldg(&D.row[MF_ROW(D, v)]);
        deg = __ldg(&D.row[MF_ROW(D, v + 1)]) - beg;
        cls = deg <= D.bin_thread ? 1 : (deg <= D.bin_warp ? 2 : 3);
      }
    }
    int newl = INT_MAX;
    for (bool any = D.cta_vertices && __syncthreads_or(cls == 3); any;) {  // CTA per vertex
      if (threadIdx.x == 0) sh.pick = -1;
      __syncthreads();
      if (cls == 3) sh.pick = threadIdx.x;
      __syncthreads();
      const int pt = sh.pick;
      if (pt < 0) break;
      if (threadIdx.x == pt) {
        cls = 0;
        sh.imin[0] = v;
      }
      __syncthreads();
      const int bv = sh.imin[0];
      const int b = __ldg(&D.row[MF_ROW(D, bv)]), e = __ldg(&D.row[MF_ROW(D, bv + 1)]);
      int m = INT_MAX;
      for (int a = b + threadIdx.x; a < e; a += blockDim.x) {
        st.scans_dis++;
        if (__ldcg(&D.rr[MF_SLOT(D, a)]).x > 0) {
          st.scans_res++;
          m = min(m, __ldcg(lab_ptr(D, __ldg(&D.head[MF_SLOT(D, a)]), R.p)) + 1);
        }
      }
      m = warp_min(m);
      __syncthreads();
      if (lane == 0) sh.imin[wid] = m;
      __syncthreads();
      if (threadIdx.x == pt)
        for (int k = 0; k < nw; k++) newl = min(newl, sh.imin[k]);
      __syncthreads();
    }
    for (;;) {  // warp per vertex
      const unsigned mm = __ballot_sync(FULL, cls == 2);
      if (!mm) break;
      const int leader = __ffs(mm) - 1;
      const int pv = __shfl_sync(FULL, v, leader);
      const int b = __ldg(&D.row[MF_ROW(D, pv)]), e = __ldg(&D.row[MF_ROW(D, pv + 1)]);
      int m = INT_MAX;
      for (int a = b + lane; a < e; a += 32) {
        st.scans_dis++;
        if (__ldcg(&D.rr[MF_SLOT(D, a)]).x > 0) {
          st.scans_res++;
          m = min(m, __ldcg(lab_ptr(D, __ldg(&D.head[MF_SLOT(D, a)]), R.p)) + 1);
        }
      }
      m = warp_min(m);
      if (lane == leader) {
        cls = 0;
        newl = m;
      }
    }
    if (cls == 1) {
      for (int a = beg; a < beg + deg; a++) {
        st.scans_dis++;
        if (__ldcg(&D.rr[MF_SLOT(D, a)]).x > 0) {
          st.scans_res++;
          newl = min(newl, __ldcg(lab_ptr(D, __ldg(&D.head[MF_SLOT(D, a)]), R.p)) + 1);
        }
      }
    }
    long long wt = 0;
    if (v >= 0) {
      newl = min(newl, cap_v);
      *lab_ptr(D, v, R.p ^ 1) = newl;
      st.relabels++;
      wt = deg + D.beta;
      work += wt;
      if (newl < cap_v && atomicExch(act_ptr(D, v, R.p ^ 1), r + 1) != r + 1) qpush(D, sh, R.next, v);
    }
    __syncwarp();
    if (MULTI && D.inst_relabel) inst_add_work(D, k, wt, R.rnd);
  }
  phase_end(D, sh, R.next, work, &D.ctl->work[rnd % 3]);
}

// ------------------------------------------------------------------ BFS
//
// BFS (Algorithm 2) from the seeds, on 64-bit words blab[v] = {label (high
// half), flags (low half)}: bit 0 = v is queued for expansion, bit 1 = v is a
// blocker (never entered). A queued vertex v is expanded with its current
// label l, read while its queued bit is cleared (one atomic); through slot
// a = (v -> w) it offers w the label l + 1 when the tested residual is positive
// (reverse BFS for the global relabel: res[rev[a]] = c_f(w, v); forward BFS
// for the cut: res[a] = c_f(v, w)) with atomicMin(blab[w], {l + 1, queued}).
// The offer lowers w's label iff l + 1 is smaller; w joins the next list iff
// it was not queued already (a queued w is expanded later with its newest
// label). Expanding the list level by level with a grid barrier between
// levels gives every vertex its BFS distance the first time, as Algorithm 2
// does. With D.bfs_hops > 1 a CTA also expands the few vertices it reached
// itself right away, up to bfs_hops levels per grid barrier: a label found
// that way can be too large and is lowered by a later offer, which queues the
// vertex again. Either way the words settle when no vertex is queued, and then
// every label is the exact distance: each label is the length of a path, and
// every arc out of an expanded vertex was offered with that vertex's final
// label.

constexpr unsigned long long BQ = 1ULL;  // queued
constexpr unsigned long long BB = 2ULL;  // blocker

__device__ __forceinline__ unsigned long long bword(int label, unsigned long long flags) {
  return ((unsigned long long)(unsigned)label << 32) | flags;
}

// Expansion start: clears v's queued bit and returns its label.
__device__ __forceinline__ int bfs_take(const Dev &D, int v) {
  return (int)(atomicAnd(D.blab + MF_VTX(D, v), ~BQ) >> 32);
}

// Offers label l to w; true when w must join the next list.
__device__ __forceinline__ bool bfs_offer(const Dev &D, int w, int l) {
  const unsigned long long c = bword(l, BQ);
  const unsigned long long old = atomicMin(D.blab + MF_VTX(D, w), c);
  return old > c && !(old & BQ);
}

__device__ __forceinline__ void bfs_arc(const Dev &D, Shared &sh, int a, int l, bool reverse, int next) {
  const int w = __ldg(&D.head[MF_SLOT(D, a)]);
  const int2 x = __ldcg(&D.rr[MF_SLOT(D, a)]);
  const int cf = reverse ? x.y : x.x;
  if (cf > 0 && bfs_offer(D, w, l)) qpush(D, sh, next, w);
}

// One thread, deg <= KTD, loads issued together (with `pre`, deg <= KT and the
// heads were loaded during the last grid barrier).
template <int KTD>
__device__ __forceinline__ void bfs_thread(const Dev &D, Shared &sh, int beg, int deg, int l, bool reverse, int next,
                                           bool pre) {
  int w[KTD], cf[KTD];
  bool got[KTD];
#pragma unroll
  for (int i = 0; i < KTD; i++) {
    w[i] = 0;
    cf[i] = 0;
    if (i < deg) {
      w[i] = (pre && i < KT) ? sh.phead[i < KT ? i : 0][threadIdx.x] : __ldg(&D.head[MF_SLOT(D, beg + i)]);
      const int2 x = __ldcg(&D.rr[MF_SLOT(D, beg + i)]);
      cf[i] = reverse ? x.y : x.x;
    }
  }
  if (D.bfs_hops > 1) {
    // all offers and the offered vertices' row offsets in flight together
    int rb[KTD], re[KTD];
#pragma unroll
    for (int i = 0; i < KTD; i++) {
      got[i] = cf[i] > 0 && bfs_offer(D, w[i], l);
      rb[i] = cf[i] > 0 ? __ldg(&D.row[MF_ROW(D, w[i])]) : 0;
      re[i] = cf[i] > 0 ? __ldg(&D.row[MF_ROW(D, w[i] + 1)]) : 0;
    }
#pragma unroll
    for (int i = 0; i < KTD; i++)
      if (got[i]) qpush_row(D, sh, next, w[i], rb[i], re[i] - rb[i]);
    return;
  }
  // all offers first (in flight together), then the appends
#pragma unroll
  for (int i = 0; i < KTD; i++) got[i] = cf[i] > 0 && bfs_offer(D, w[i], l);
#pragma unroll
  for (int i = 0; i < KTD; i++)
    if (got[i]) qpush(D, sh, next, w[i]);
}

// One BFS level: expands the list of generation gen into generation gen + 1,
// then (D.bfs_hops > 1) up to bfs_hops - 1 more levels of the vertices this
// CTA reached itself, while they fit one per thread.
template <int KTD>
__device__ void bfs_level(const Dev &D, Shared &sh, int gen, bool reverse, TStat &st) {
  const int next = gen + 1;
  const Sweep sw = make_sweep(sh.lq[gen % 3], sh.lqn[gen % 3], nullptr, 0, list_of(D, gen), list_count(D, sh, gen),
                              nullptr, 0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.ctl->cnt[(gen + 2) & 3] = 0;
    D.ctl->lcnt[(gen + 2) & 3] = 0;
  }
  const int lane = threadIdx.x & 31;
  for (int off = 0; off < sw.items; off += blockDim.x) {
    int v = -1;
    if (sweep_item(sw, off + (int)threadIdx.x, v) != 1) v = -1;
    int beg = 0, deg = 0, cls = 0, l = 0;
    const bool pre = v >= 0 && sh.pv[threadIdx.x] == v;  // row and heads loaded during the last grid barrier
    if (v >= 0) {
      l = bfs_take(D, v) + 1;
      if (pre) {
        beg = sh.pbeg[threadIdx.x];
        deg = sh.pdeg[threadIdx.x];
      } else {
        beg = __ldg(&D.row[MF_ROW(D, v)]);
        deg = __ldg(&D.row[MF_ROW(D, v + 1)]) - beg;
      }
      cls = deg <= KTD ? 1 : (deg <= D.bin_warp ? 2 : 3);
      st.scans_bfs += deg;
      st.visits_bfs++;
    }
    for (bool any = __syncthreads_or(cls == 3); any;) {
      if (threadIdx.x == 0) sh.pick = -1;
      __syncthreads();
      if (cls == 3) sh.pick = threadIdx.x;
      __syncthreads();
      const int pt = sh.pick;
      if (pt < 0) break;
      if (threadIdx.x == pt) {
        cls = 0;
        sh.imin[0] = v;
        sh.imin[1] = l;
      }
      __syncthreads();
      const int pv = sh.imin[0], pl = sh.imin[1];
      const int b = __ldg(&D.row[MF_ROW(D, pv)]), e = __ldg(&D.row[MF_ROW(D, pv + 1)]);
      for (int a = b + threadIdx.x; a < e; a += blockDim.x) bfs_arc(D, sh, a, pl, reverse, next);
      __syncthreads();
    }
    for (;;) {
      const unsigned mm = __ballot_sync(FULL, cls == 2);
      if (!mm) break;
      const int leader = __ffs(mm) - 1;
      const int pv = __shfl_sync(FULL, v, leader);
      const int pl = __shfl_sync(FULL, l, leader);
      if (lane == leader) cls = 0;
      const int b = __ldg(&D.row[MF_ROW(D, pv)]), e = __ldg(&D.row[MF_ROW(D, pv + 1)]);
      for (int a = b + lane; a < e; a += 32) bfs_arc(D, sh, a, pl, reverse, next);
      __syncwarp();
    }
    if (cls == 1) bfs_thread<KTD>(D, sh, beg, deg, l, reverse, next, pre);
    __syncwarp();
  }
  // more levels inside the CTA (only on graphs whose vertices are all
  // thread-sized; staged entries are taken out of the staging buffer)
  for (int hop = 1; hop < D.bfs_hops; hop++) {
    __syncthreads();  // staging of the previous level complete
    const int k = sh.qn;
    if (k == 0 || k > (int)blockDim.x) break;
    const int v = (int)threadIdx.x < k ? sh.qbuf[threadIdx.x] : -1;
    int beg = v >= 0 ? sh.qrow[threadIdx.x] : 0;
    int deg = v >= 0 ? sh.qdeg[threadIdx.x] : 0;
    __syncthreads();  // every thread has read qn and its entry
    if (threadIdx.x == 0) sh.qn = 0;
    __syncthreads();
    if (v >= 0) {
      if (deg < 0) {
        beg = __ldg(&D.row[MF_ROW(D, v)]);
        deg = __ldg(&D.row[MF_ROW(D, v + 1)]) - beg;
      }
      if (deg > KT) {
        qpush(D, sh, next, v);  // still queued: the next level's sweep expands it
      } else {
        const int l = bfs_take(D, v) + 1;
        st.scans_bfs += deg;
        st.visits_bfs++;
        bfs_thread<KT>(D, sh, beg, deg, l, reverse, next, false);
      }
    }
  }
  phase_end(D, sh, next, 0, nullptr);
}

// One bottom-up level (direction-optimizing BFS, Beamer, Asanovic and Patterson
// 2012) for a level-synchronous BFS whose frontier is large: every vertex w not
// reached yet looks for a residual arc to a vertex labelled `depth` and takes
// depth + 1 at the first one, instead of the frontier offering labels along all
// its arcs. Same labels as the top-down level: w is reached at depth + 1 iff
// such an arc exists. Slot a of w's row is (w -> v); the reverse BFS (global
// relabel) needs c_f(w, v) = res[a], the forward BFS (cut) c_f(v, w) =
// res[rev[a]]. Thread per vertex up to 32 slots, warp per vertex above.
static __device__ void bfs_pull_level(const Dev &D, Shared &sh, int gen, int depth, bool reverse, TStat &st,
                               const Sel &S) {
  const int next = gen + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.ctl->cnt[(gen + 2) & 3] = 0;
    D.ctl->lcnt[(gen + 2) & 3] = 0;
  }
  const int lane = threadIdx.x & 31;
  for_covered(D, S, [&](int wv, bool valid) {
    const int w = valid ? wv : -1;
    int beg = 0, deg = 0;
    bool open = false;
    if (w >= 0) {
      const unsigned long long x = __ldcg(D.blab + MF_VTX(D, w));
      open = (int)(x >> 32) == UNV && !(x & BB);
      if (open) {
        beg = __ldg(&D.row[MF_ROW(D, w)]);
        deg = __ldg(&D.row[MF_ROW(D, w + 1)]) - beg;
        open = deg > 0;
      }
    }
    if (open && deg <= 32) {  // thread per vertex, stop at the first arc into the level
      for (int i = 0; i < deg; i++) {
        st.scans_bfs++;
        const int2 r = __ldcg(&D.rr[MF_SLOT(D, beg + i)]);
        if ((reverse ? r.x : r.y) <= 0) continue;
        const unsigned long long y = __ldcg(D.blab + MF_VTX(D, __ldg(&D.head[MF_SLOT(D, beg + i)])));
        if ((int)(y >> 32) == depth && !(y & BB)) {
          D.blab[MF_VTX(D, w)] = bword(depth + 1, BQ);
          st.visits_bfs++;
          qpush(D, sh, next, w);
          break;
        }
      }
      open = false;
    }
    for (;;) {  // warp per vertex
      const unsigned mm = __ballot_sync(FULL, open);
      if (!mm) break;
      const int leader = __ffs(mm) - 1;
      const int pw = __shfl_sync(FULL, w, leader);
      const int pb = __shfl_sync(FULL, beg, leader);
      const int pd = __shfl_sync(FULL, deg, leader);
      if (lane == leader) open = false;
      for (int c = 0; c < pd; c += 32) {
        bool hit = false;
        if (c + lane < pd) {
          st.scans_bfs++;
          const int a = pb + c + lane;
          const int2 r = __ldcg(&D.rr[MF_SLOT(D, a)]);
          if ((reverse ? r.x : r.y) > 0) {
            const unsigned long long y = __ldcg(D.blab + MF_VTX(D, __ldg(&D.head[MF_SLOT(D, a)])));
            hit = (int)(y >> 32) == depth && !(y & BB);
          }
        }
        if (__ballot_sync(FULL, hit)) {
          if (lane == 0) {
            D.blab[MF_VTX(D, pw)] = bword(depth + 1, BQ);
            st.visits_bfs++;
            qpush(D, sh, next, pw);
          }
          break;
        }
      }
      __syncwarp();
    }
  });
  phase_end(D, sh, next, 0, nullptr);
}

// CTA 0 thread 0 after the grid barrier that ends a BFS level which started at
// t0 and whose own expansion ended at t1 (%globaltimer): counters and trace.
__device__ __forceinline__ void level_done(const Dev &D, unsigned long long t0, unsigned long long t1) {
  const unsigned long long t2 = gtimer();
  const long long k = D.ctl->levels++;
  if (D.trace_lv_ns && k < D.trace_lv_cap) D.trace_lv_ns[k] = (int)min(t2 - t0, (unsigned long long)INT_MAX);
  D.ctl->t_lwork += t1 - t0;
  D.ctl->t_lwait += t2 - t1;
}

// Level 0 of a BFS from one seed with many arcs (slots [b, e)), the seed
// labelled 0 and not queued (generation gen is empty): the whole grid offers
// label 1 along its arcs, one arc per thread, into generation gen + 1. Ends
// with a grid barrier.
static __device__ __noinline__ bool bfs_wide_level(const Dev &D, Shared &sh, int gen, int b, int e, bool reverse,
                                                   TStat &st, int where) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  const unsigned long long t0 = timer ? gtimer() : 0;
  if (timer) {
    D.ctl->cnt[(gen + 2) & 3] = 0;
    D.ctl->lcnt[(gen + 2) & 3] = 0;
    const long long k = D.ctl->levels;
    if (D.trace_lv && k < D.trace_lv_cap) D.trace_lv[k] = 1;
    st.visits_bfs++;
  }
  for (int a = b + tid; a < e; a += nthr) {
    bfs_arc(D, sh, a, 1, reverse, gen + 1);
    st.scans_bfs++;
  }
  phase_end(D, sh, gen + 1, 0, nullptr);
  const unsigned long long t1 = timer ? gtimer() : 0;
  if (!grid_sync(D, sh, where, PF_LEVEL, gen + 1)) return false;
  if (timer) level_done(D, t0, t1);
  return true;
}

// BFS from `seeds` (label 0) over blab. `blockers` are never entered. With
// `excess_seeds`, every vertex holding excess whose label lies in [1, cap] is
// a seed as well (cut from the maximum preflow). Returns false on error. On
// return the last list generation (gen) is empty and no vertex is queued.
// With S.on only the live instances take part (seeds, blockers and labels of
// the others are left as they are; no arc leads into them).
template <int KTD>
__device__ bool bfs(const Dev &D, Shared &sh, const int *seeds, const int *blockers, int nterm, bool reverse,
                    bool excess_seeds, int &gen, TStat &st, int where, const Sel &S = Sel{false, 0}) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int next = gen + 1;
  // phase A: every label to UNV (excess-holding non-terminals become seeds)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.ctl->cnt[(gen + 2) & 3] = 0;
    D.ctl->lcnt[(gen + 2) & 3] = 0;
  }
  for_covered(D, S, [&](int v, bool valid) {
    if (!valid) return;
    unsigned long long x = bword(UNV, 0);
    if (excess_seeds) {
      const int d = __ldcg(lab_ptr(D, v, 0));
      if (d >= 1 && d <= cap_of(D, v) && __ldcg(exc_ptr(D, v)) > 0) {
        x = bword(0, BQ);
        qpush(D, sh, next, v);
      }
    }
    D.blab[MF_VTX(D, v)] = x;
  });
  phase_end(D, sh, next, 0, nullptr);
  if (!grid_sync(D, sh, where)) return false;
  // phase B: terminals (seeds join generation gen + 1 as well)
  // (seeds and blockers are read through L2: a union's per-instance seeds change during the launch)
  // A lone seed with more arcs than a CTA has threads (the sink or the source of a single graph) is not
  // queued: its level is expanded below by the whole grid, one arc per thread, instead of by one CTA.
  int wide_b = 0, wide_e = 0;
  if (nterm == 1 && !excess_seeds && !S.on) {
    const int s0 = __ldcg(&seeds[0]);
    const int b = __ldg(&D.row[MF_ROW(D, s0)]), e = __ldg(&D.row[MF_ROW(D, s0 + 1)]);
    if (e - b > (int)blockDim.x) {
      wide_b = b;
      wide_e = e;
    }
  }
  const bool wide = wide_e > wide_b;  // the same in every thread
  for (int i = tid; i < nterm; i += nthr) {
    if (S.on && __ldcg(&D.live[i]) != S.epoch) continue;
    D.blab[MF_VTX(D, __ldcg(&seeds[i]))] = bword(0, wide ? 0 : BQ);
    if (blockers) D.blab[MF_VTX(D, __ldcg(&blockers[i]))] = bword(0, BB);
  }
  if (blockIdx.x == 0 && !wide)
    for (int i = threadIdx.x; i < nterm; i += blockDim.x)
      if (!S.on || __ldcg(&D.live[i]) == S.epoch) append(D, next, __ldcg(&seeds[i]));
  if (!grid_sync(D, sh, where)) return false;
  gen++;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  int depth0 = 0;
  if (wide) {
    if (!bfs_wide_level(D, sh, gen, wide_b, wide_e, reverse, st, where)) return false;
    gen++;
    depth0 = 1;
  }
  for (int depth = depth0;; depth++) {
    const long long fcount = gen_total(D, sh, gen);
    if (fcount == 0) break;
    if (timer && D.trace_lv) {
      const long long k = D.ctl->levels;
      if (k < D.trace_lv_cap) D.trace_lv[k] = (int)fcount;
    }
    const unsigned long long t0 = timer ? gtimer() : 0;
    // bottom-up when the frontier holds more than n / bfs_pull vertices (only for level-synchronous
    // BFS, where every frontier vertex carries the label `depth`)
    if (D.bfs_pull > 0 && D.bfs_hops == 1 && fcount * D.bfs_pull > D.n)
      bfs_pull_level(D, sh, gen, depth, reverse, st, S);
    else
      bfs_level<KTD>(D, sh, gen, reverse, st);
    const unsigned long long t1 = timer ? gtimer() : 0;
    if (!grid_sync(D, sh, where, PF_LEVEL, gen + 1)) return false;
    gen++;
    if (timer) level_done(D, t0, t1);
  }
  return true;
}

// Label of v after a BFS: its distance, cap for an unreached vertex, cap + 1
// for a blocker.
__device__ __forceinline__ int bfs_label(unsigned long long x, int cap) {
  if (x & BB) return cap + 1;
  const int l = (int)(x >> 32);
  return l >= UNV ? cap : l;
}

// Global relabel (Algorithm 2 from the sinks, never entering the sources),
// then the working set is rebuilt for round r: labels left at UNV become the
// cap n, sources n + 1, both label slots get the result, addedExcess is folded
// into the excess, and every vertex with excess and 0 < d < n is stamped
// active. Result: list generation gen.
template <int KTD, bool MULTI>
__device__ bool global_relabel(const Dev &D, Shared &sh, const int *sinks, const int *sources, int r, int &gen,
                               TStat &st, const Sel &S, int rnd = 0, bool carried = false) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  if (MULTI && D.inst_relabel) {  // relabel schedule of the covered instances starts over
    for (int k = tid; k < D.ninst; k += nthr)
      if (!S.on || __ldcg(&D.live[k]) == S.epoch) {
        InstState *I = D.inst + k;
        D.inst_work[(size_t)k * INST_WORK_STRIDE] = 0;
        I->last = rnd;
        I->depth = 0;
        I->due = 0;
        I->act = 0;
      }
  }
  if (!bfs<KTD>(D, sh, sinks, sources, D.ninst, true, false, gen, st, 2, S)) return false;
  const int next = gen + 1;
  const int p = r & 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.ctl->cnt[(gen + 2) & 3] = 0;
    D.ctl->lcnt[(gen + 2) & 3] = 0;
    D.ctl->grs++;
  }
  for_covered(D, S, [&](int v, bool valid) {
    int depth = -1, k = -1;
    bool active = false;
    if (valid) {
      const int2 vi = vinst_of<MULTI>(D, v);
      const int c = vi.x;
      k = vi.y;
      const int d = bfs_label(__ldcg(D.blab + MF_VTX(D, v)), c);
      *lab_ptr(D, v, 0) = d;
      *lab_ptr(D, v, 1) = d;
      const longlong2 ea = load_ea(D, v);
      long long ev = ea.x;
      const long long ad = ea.y;
      if (ad) {
        ev += ad;
        *exc_ptr(D, v) = ev;
        *add_ptr(D, v) = 0;
      }
      if (d > 0 && d < c && ev > 0) {
        *act_ptr(D, v, p) = r;
        qpush(D, sh, next, v);
        active = true;
      }
      if (d < c) depth = d;
    }
    if (MULTI && D.inst_relabel) {  // every covered instance: its depth (largest finite label), its active vertices
      const int kk = depth >= 0 ? k : -1;
      const unsigned grp = __match_any_sync(FULL, kk);
      const int dmax = __reduce_max_sync(grp, depth);
      if (kk >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(&D.inst[kk].depth, dmax);
      const int ka = active ? k : -1;
      const unsigned ga = __match_any_sync(FULL, ka);
      if (ka >= 0 && (threadIdx.x & 31) == __ffs(ga) - 1) atomicAdd(&D.inst[ka].act, __popc(ga));
    }
  });
  if (carried) {  // working-set entries of the instances this relabel did not cover (partial_prep)
    const int cn = min(__ldcg(&D.ctl->carry_n), D.n);
    for (int i = tid; i < cn; i += nthr) {
      const int v = __ldcg(&D.carry[i]);
      *act_ptr(D, v, p) = r;
      qpush(D, sh, next, v);
    }
  }
  phase_end(D, sh, next, 0, nullptr);
  if (!grid_sync(D, sh, 3, PF_ROUND, next)) return false;
  gen++;
  return true;
}

// Gap relabeling (Section 2.1 names the heuristic; the paper's parallel code
// leaves it out). Between two rounds, with the labels the next round reads in
// slot p: if no vertex has label g (0 < g < cap) while some have larger
// labels below the cap, none of those can reach the sink: a residual path
// from such a vertex passes labels that drop by at most one per arc (valid
// labels), so it would pass label g. They get the cap in both slots, which
// keeps the labels valid. Three grid barriers: count labels, find the
// smallest empty label, lift. Single-instance graphs only (one label range).
static __device__ bool gap_relabel(const Dev &D, Shared &sh, int p) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int cap = D.n_cap;
  if (tid == 0) D.ctl->gap = INT_MAX;
  for (int v = tid; v < D.n; v += nthr) {
    const int d = __ldcg(lab_ptr(D, v, p));
    if (d >= 1 && d < cap) atomicAdd(&D.hist[d], 1);
  }
  if (!grid_sync(D, sh, 13)) return false;
  for (int k = 1 + tid; k < cap; k += nthr)
    if (__ldcg(&D.hist[k]) == 0) {
      atomicMin(&D.ctl->gap, k);
      break;  // this thread's later k are larger
    }
  if (!grid_sync(D, sh, 13)) return false;
  const int g = vol_read(&D.ctl->gap);
  long long lifted = 0;
  if (g < cap)
    for (int v = tid; v < D.n; v += nthr) {
      const int d = __ldcg(lab_ptr(D, v, p));
      if (d > g && d < cap) {
        *lab_ptr(D, v, 0) = cap;
        *lab_ptr(D, v, 1) = cap;
        lifted++;
      }
    }
  for (int k = tid; k <= cap; k += nthr) D.hist[k] = 0;
  lifted = block_sum(lifted, sh);
  if (threadIdx.x == 0 && lifted) atomic_add64(&D.ctl->gap_lifted, lifted);
  return grid_sync(D, sh, 13);
}

// Ends a MODE_ROUNDS run between rounds: every vertex gets its current label
// (slot p) in both slots and its addedExcess folded into its excess.
static __device__ bool settle(const Dev &D, Shared &sh, int p) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  for (int v = tid; v < D.n; v += nthr) {
    const int d = __ldcg(lab_ptr(D, v, p));
    *lab_ptr(D, v, p ^ 1) = d;
    const long long ad = __ldcg(add_ptr(D, v));
    if (ad) {
      *exc_ptr(D, v) = __ldcg(exc_ptr(D, v)) + ad;
      *add_ptr(D, v) = 0;
    }
  }
  return grid_sync(D, sh, 12);
}

// Rounds of Algorithm 1 toward `sinks` until no vertex is active right after a
// global relabel (or, in MODE_ROUNDS, until stop_rounds rounds ran).
template <int KTD, bool MULTI>
__device__ bool run_phase(const Dev &D, Shared &sh, const int *sinks, const int *sources, int &r, int &gen,
                          long long &rnd, bool phase1, TStat &st, int &epoch) {
  long long since_gr = LLONG_MAX;
  bool fresh = false, time_req = false, prev_valid = false;
  // Multi-instance graphs with per-instance relabel schedules: an instance asks for a global relabel
  // (InstState); a relabel then covers the instances that asked and carries the working sets of the others
  // over. The first relabel of a phase and the one confirming its end (an empty working set) cover every
  // instance.
  const bool per_inst = MULTI && D.inst_relabel != 0;
  bool full_next = true;   // the next global relabel covers every instance
  bool last_full = false;  // the last global relabel covered every instance
  long long rounds = 0;
  unsigned long long last_gr_ns = 0, last_gr_end = 0;  // meaningful in CTA 0 thread 0 only
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  for (;;) {
    // requests of the round just finished (rnd - 1), read at its grid barrier
    const bool partial = per_inst && !full_next && !fresh && sh.snap.due_any[(rnd + 2) % 3] != 0;
    if (per_inst ? (full_next || partial) : (since_gr > D.gr_threshold || time_req)) {
      const unsigned long long t0 = timer ? gtimer() : 0;
      Sel S{false, 0};
      if (partial) {
        S = Sel{true, ++epoch};
        if (timer) D.ctl->grs_partial++;
        if (!partial_prep(D, sh, r, gen, prev_valid, S.epoch, (int)rnd)) return false;
        r += 2;  // fresh stamps, same label slot: the carried entries keep the labels of slot r & 1
      } else {
        r++;  // fresh stamp: marks of the discarded working set are stale
      }
      if (!global_relabel<KTD, MULTI>(D, sh, sinks, sources, r, gen, st, S, (int)rnd, partial)) return false;
      last_full = !partial;
      full_next = false;
      if (timer) {
        last_gr_end = gtimer();
        last_gr_ns = last_gr_end - t0;
        D.ctl->t_gr += last_gr_ns;
      }
      since_gr = 0;
      fresh = true;
      time_req = false;
      prev_valid = false;
    }
    const long long count = gen_total(D, sh, gen);
    if (count == 0) {
      if (fresh && last_full) break;
      since_gr = LLONG_MAX;  // confirm with a relabel of every instance
      full_next = true;
      continue;
    }
    if (D.mode == MODE_ROUNDS && rounds >= D.stop_rounds) break;
    if (rounds >= D.max_rounds) {
      set_err(D, MF_ERR_ITER_LIMIT, 10);
      return false;
    }
    unsigned long long t0 = 0;
    if (timer) {
      D.ctl->rounds_by_size[count < 1024 ? 0 : count < 16384 ? 1 : count < 262144 ? 2 : 3]++;
      if (D.trace && rnd < D.trace_cap) D.trace[rnd] = make_int2((int)count, fresh ? 1 : 0);
      t0 = gtimer();
      D.ctl->gr_req[rnd & 1] =
          D.gr_time_ratio > 0 && (double)(t0 - last_gr_end) > D.gr_time_ratio * (double)last_gr_ns;
    }
    fresh = false;
    unsigned long long tp = t0;
    round_phase<KTD, MULTI>(D, sh, r, gen, prev_valid, rnd, st, tp);
    if (!grid_sync(D, sh, 4, D.simple ? PF_NONE : PF_ROUND, gen + 1, gen)) return false;
    if (D.simple) {
      relabel_phase<MULTI>(D, sh, r, gen, rnd, st);
      if (!grid_sync(D, sh, 4)) return false;
    }
    if (timer) {
      const unsigned long long t3 = gtimer();
      D.ctl->t_dis += t3 - t0;
      D.ctl->t_rwait += t3 - tp;
      if (D.trace_ns && rnd < D.trace_cap) D.trace_ns[rnd] = (int)min(t3 - t0, (unsigned long long)INT_MAX);
    }
    since_gr += sh.snap.work[rnd % 3];
    time_req = sh.snap.gr_req[rnd & 1] != 0;
    r++;
    gen++;
    rnd++;
    rounds++;
    prev_valid = true;
    if (timer) {
      D.ctl->rounds++;
      if (phase1) D.ctl->rounds_phase1++;
    }
    if (D.gap_every > 0 && rounds % D.gap_every == 0 && !gap_relabel(D, sh, r & 1)) return false;
  }
  if (D.mode == MODE_ROUNDS) {
    if (timer) D.ctl->stopped_round = (int)rounds;
    if (D.final_gr) {
      r++;
      if (!global_relabel<KTD, MULTI>(D, sh, sinks, sources, r, gen, st, Sel{false, 0})) return false;
    } else if (!fresh) {
      if (!settle(D, sh, r & 1)) return false;
    }
  }
  return true;
}

// ------------------------------------------------------------------ unions
//
// Batches and service unions with per-instance relabel schedules: every
// instance goes through its own phases inside the one launch, as it would
// solved alone: the preflow (rounds toward its t), the flow phase (its excess
// back to its s), then its cut BFS and its outputs, after which its results
// are final (and, with D.done_flag, announced to the host while the others
// go on). An instance's phase ends when a global relabel covering it finds no
// active vertex of it, as a phase of a single graph ends (reading 9). Every
// global relabel here covers a set of flagged instances (partial_prep): the
// ones that asked for one, or every instance not done yet when the working
// set is empty, and carries the working sets of the others over.

// Instance k's value is final once its preflow ended: the excess of its sink.
// Transitions after a relabel that covered the instances flagged `epoch`: one
// without active vertices ends its phase (preflow: value recorded, next relabel
// from s, blocking t; flow: cut pending). Ends with a grid barrier.
static __device__ __noinline__ bool union_transitions(const Dev &D, Shared &sh, int epoch, int gen) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  if (tid == 0) {
    D.ctl->ph2_started = 0;
    D.ctl->cut_pending = 0;
  }
  if (!grid_sync(D, sh, 3)) return false;
  for (int k = tid; k < D.ninst; k += nthr) {
    if (__ldcg(&D.live[k]) != epoch) continue;
    InstState *I = D.inst + k;
    if (__ldcg(&I->act) != 0) continue;
    const int ph = __ldcg(&I->ph);
    if (ph == 1) {
      const long long val = __ldcg(exc_ptr(D, D.snk[k]));
      if (D.out_value) D.out_value[k] = val;
      if (k == 0) D.ctl->value = val;
      I->ph = 2;
      D.gseed[k] = D.src[k];
      D.gblock[k] = D.snk[k];
      I->due = 1;
      D.ctl->ph2_started = 1;
    } else if (ph == 2) {
      I->ph = 3;
      D.ctl->cut_pending = 1;
    }
  }
  return grid_sync(D, sh, 3, PF_ROUND, gen);
}

// Cut and outputs of the instances whose flow phase ended (phase 3): BFS from
// their sources over residual arcs (S_min), their cut bitmaps (word-aligned per
// instance), their per-slot flows, a check that none of their vertices other
// than s and t kept excess, then phase 4 and the host's flag. Runs right after
// a global relabel; the working set of the other instances (list generation
// gen, which the BFS's lists overwrite) is saved in D.carry and comes back as
// the next generation, stamps unchanged.
template <int KTD>
__device__ __noinline__ bool union_cut(const Dev &D, Shared &sh, int &gen, TStat &st, int &epoch) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const Sel S{true, ++epoch};
  for (int k = tid; k < D.ninst; k += nthr)
    if (__ldcg(&D.inst[k].ph) == 3) D.live[k] = S.epoch;
  if (tid == 0) D.ctl->carry_n = 0;
  if (!grid_sync(D, sh, 9)) return false;
  {
    const int cnt = list_count(D, sh, gen);
    const int *L = list_of(D, gen);
    for (int i = tid; i < cnt; i += nthr) carry_push(D, __ldcg(&L[i]));
    const int *lq = sh.lq[gen % 3];
    for (int i = threadIdx.x; i < sh.lqn[gen % 3]; i += blockDim.x) carry_push(D, lq[i]);
  }
  if (!grid_sync(D, sh, 9)) return false;
  if (!bfs<KTD>(D, sh, D.src, nullptr, D.ninst, false, false, gen, st, 9, S)) return false;
  long long left = 0;
  for (int t = blockIdx.x; t < D.ntiles; t += gridDim.x) {
    const int4 T = __ldg(&D.tiles[t]);
    if (__ldcg(&D.live[T.z]) != S.epoch) continue;  // uniform in the CTA
    const int k = T.z, V = __ldg(&D.voff[k]);
    if (D.out_cutw) {  // bit v of instance k at bit (v - V) of its run; tiles start at multiples of 32 in it
      const int words = (T.y - T.x + 31) >> 5;
      unsigned *out = D.out_cutw + D.cwoff[k] + ((T.x - V) >> 5);
      for (int w = threadIdx.x; w < words; w += blockDim.x) {
        unsigned bits = 0;
        for (int j = 0; j < 32; j++) {
          const int v = T.x + 32 * w + j;
          if (v < T.y && (int)(__ldcg(D.blab + MF_VTX(D, v)) >> 32) != UNV) bits |= 1u << j;
        }
        out[w] = bits;
      }
    }
    if (D.out_flow) {
      const int a0 = __ldg(&D.row[MF_ROW(D, T.x)]), a1 = __ldg(&D.row[MF_ROW(D, T.y)]);
      for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
        const int f = __ldg(&D.cap[MF_SLOT(D, a)]) - __ldcg(&D.rr[MF_SLOT(D, a)]).x;
        D.out_flow[a] = f > 0 ? f : 0;
      }
    }
    for (int v = T.x + threadIdx.x; v < T.y; v += blockDim.x)
      if (v != D.src[k] && v != D.snk[k] && __ldcg(exc_ptr(D, v)) != 0) left++;
  }
  left = block_sum(left, sh);
  if (threadIdx.x == 0 && left) {
    atomic_add64(&D.ctl->leftover, left);
    set_err(D, MF_ERR_INTERNAL, 8);
  }
  {  // the saved working set becomes the next generation (the BFS left generation gen empty)
    const int next = gen + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      D.ctl->cnt[(gen + 2) & 3] = 0;
      D.ctl->lcnt[(gen + 2) & 3] = 0;
    }
    const int cn = min(__ldcg(&D.ctl->carry_n), D.n);
    for (int i = tid; i < cn; i += nthr) qpush(D, sh, next, __ldcg(&D.carry[i]));
    phase_end(D, sh, next, 0, nullptr);
  }
  if (!grid_sync(D, sh, 9)) return false;
  gen++;
  for (int k = tid; k < D.ninst; k += nthr) {
    if (__ldcg(&D.live[k]) != S.epoch) continue;
    D.inst[k].ph = 4;
    atomicAdd(&D.ctl->done_cnt, 1);
    if (D.done_flag) {
      __threadfence_system();  // the outputs before the flag, for the host and its copies
      D.done_flag[k] = 1u;
    }
  }
  return grid_sync(D, sh, 9, PF_ROUND, gen);
}

// Instances whose working set ran empty without a relabel of theirs (between
// rounds; the next round has index rnd and working set generation gen): flag
// the instances present in the working set; every other instance not finished
// asks for a relabel, under the request flag of the round just finished.
static __device__ __noinline__ bool union_presence(const Dev &D, Shared &sh, int gen, int rnd) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int cnt = list_count(D, sh, gen);
  const int *L = list_of(D, gen);
  const int mark = -2 - rnd;  // never a relabel epoch (those are positive)
  for (int i = tid; i < cnt; i += nthr) D.live[__ldg(&D.vinst[__ldcg(&L[i])]).y] = mark;
  for (int i = threadIdx.x; i < sh.lqn[gen % 3]; i += blockDim.x) D.live[__ldg(&D.vinst[sh.lq[gen % 3][i]]).y] = mark;
  if (!grid_sync(D, sh, 4)) return false;
  for (int k = tid; k < D.ninst; k += nthr) {
    InstState *I = D.inst + k;
    const int ph = __ldcg(&I->ph);
    if ((ph == 1 || ph == 2) && __ldcg(&D.live[k]) != mark && !__ldcg(&I->due)) {
      I->due = 1;
      D.ctl->due_any[(rnd + 2) % 3] = 1;  // read at the next barrier
    }
  }
  return grid_sync(D, sh, 4, PF_ROUND, gen);
}

// The whole solve of a union with per-instance phases (see above).
template <int KTD>
__device__ bool run_union(const Dev &D, Shared &sh, int &r, int &gen, long long &rnd, TStat &st, int &epoch) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  bool fresh = false, prev_valid = false, full_next = true, pending = false;
  long long rounds = 0;
  unsigned long long last_gr_end = 0;  // CTA 0 thread 0
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  for (;;) {
    // instances whose working set ran empty without a relabel of theirs: every 16 rounds, flag the
    // instances present in the working set; the others, not finished, ask for a relabel
    if (!fresh && rounds > 0 && rounds % 16 == 0 && !full_next && !pending && !union_presence(D, sh, gen, (int)rnd))
      return false;
    const bool partial = !full_next && (pending || (!fresh && sh.snap.due_any[(rnd + 2) % 3] != 0));
    if (full_next || partial) {
      const unsigned long long t0 = timer ? gtimer() : 0;
      const int ep = ++epoch;
      if (timer && partial) D.ctl->grs_partial++;
      if (full_next)  // cover every instance not finished: flag them as asking
        for (int k = tid; k < D.ninst; k += nthr)
          if (__ldcg(&D.inst[k].ph) <= 2) D.inst[k].due = 1;
      if (full_next && !grid_sync(D, sh, 2)) return false;
      if (!partial_prep(D, sh, r, gen, prev_valid, ep, (int)rnd)) return false;
      r += 2;  // fresh stamps, same label slot for the carried entries
      if (!global_relabel<KTD, true>(D, sh, D.gseed, D.gblock, r, gen, st, Sel{true, ep}, (int)rnd, true))
        return false;
      if (!union_transitions(D, sh, ep, gen)) return false;
      if (sh.snap.cut_pending && !union_cut<KTD>(D, sh, gen, st, epoch)) return false;
      pending = sh.snap.ph2_started != 0;
      if (timer) {
        last_gr_end = gtimer();
        D.ctl->t_gr += last_gr_end - t0;
      }
      full_next = false;
      fresh = true;
      prev_valid = false;
    }
    const long long count = gen_total(D, sh, gen);
    if (count == 0) {
      if (vol_read(&D.ctl->done_cnt) >= D.ninst) break;  // every CTA reads the same: written before a barrier
      if (!pending) full_next = true;  // confirm the instances not finished (or start their next phase)
      fresh = false;
      continue;
    }
    if (rounds >= 2 * D.max_rounds) {
      set_err(D, MF_ERR_ITER_LIMIT, 10);
      return false;
    }
    unsigned long long t0 = 0;
    if (timer) {
      D.ctl->rounds_by_size[count < 1024 ? 0 : count < 16384 ? 1 : count < 262144 ? 2 : 3]++;
      if (D.trace && rnd < D.trace_cap) D.trace[rnd] = make_int2((int)count, fresh ? 1 : 0);
      t0 = gtimer();
    }
    fresh = false;
    unsigned long long tp = t0;
    round_phase<KTD, true>(D, sh, r, gen, prev_valid, rnd, st, tp);
    if (!grid_sync(D, sh, 4, D.simple ? PF_NONE : PF_ROUND, gen + 1, gen)) return false;
    if (D.simple) {
      relabel_phase<true>(D, sh, r, gen, rnd, st);
      if (!grid_sync(D, sh, 4)) return false;
    }
    if (timer) {
      const unsigned long long t3 = gtimer();
      D.ctl->t_dis += t3 - t0;
      D.ctl->t_rwait += t3 - tp;
      if (D.trace_ns && rnd < D.trace_cap) D.trace_ns[rnd] = (int)min(t3 - t0, (unsigned long long)INT_MAX);
    }
    r++;
    gen++;
    rnd++;
    rounds++;
    prev_valid = true;
    if (timer) D.ctl->rounds++;
  }
  return true;
}

// ------------------------------------------------------------------ kernel

template <int KTD, bool MULTI>
__device__ __forceinline__ void solve_body(const Dev &D) {
  __shared__ Shared sh;
  if (threadIdx.x == 0) {
    sh.bars = 0;
    sh.qn = 0;
    sh.wsum = 0;
    sh.lqn[0] = sh.lqn[1] = sh.lqn[2] = 0;
  }
  sh.pv[threadIdx.x] = -1;
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  TStat st;
  if (tid == 0) D.ctl->t_start = gtimer();

  // Initialisation (Algorithm 1): residuals from the capacities, labels 0,
  // excess 0, no stamps.
  for (int a = tid; a < D.m; a += nthr) D.rr[MF_SLOT(D, a)] = make_int2(__ldg(&D.cap[MF_SLOT(D, a)]), __ldg(&D.cap[MF_SLOT(D, __ldg(&D.rev[MF_SLOT(D, a)]))]));
  for (int v = tid; v < D.n; v += nthr) {
    reinterpret_cast<int4 *>(D.vs + MF_VTX(D, v))[0] = make_int4(0, -1, 0, -1);
    reinterpret_cast<longlong2 *>(D.vs + MF_VTX(D, v))[1] = make_longlong2(0, 0);
  }
  if (D.gap_every > 0)
    for (int k = tid; k <= D.n_cap; k += nthr) D.hist[k] = 0;
  if (MULTI && D.live)
    for (int k = tid; k < D.ninst; k += nthr) D.live[k] = 0;
  if (MULTI && D.inst)
    for (int k = tid; k < D.ninst; k += nthr) {
      const double thr = (D.gr_alpha * (double)(__ldg(&D.voff[k + 1]) - __ldg(&D.voff[k])) +
                          (double)__ldg(&D.inst_marcs[k])) / D.gr_freq;
      D.inst[k] = InstState{thr > 9.0e18 ? (long long)9e18 : (long long)thr, 0, 0, 0, 1, 0, 0};
      D.inst_work[(size_t)k * INST_WORK_STRIDE] = 0;
      if (D.gseed) {
        D.gseed[k] = D.snk[k];
        D.gblock[k] = D.src[k];
      }
    }
  bool ok = grid_sync(D, sh, 0);
  // Saturate every arc out of each source (self-loops excluded).
  if (ok) {
    for (int k = 0; k < D.ninst; k++) {
      const int s = D.src[k];
      const int b = __ldg(&D.row[MF_ROW(D, s)]), e = __ldg(&D.row[MF_ROW(D, s + 1)]);
      for (int a = b + tid; a < e; a += nthr) {
        const int c = __ldg(&D.cap[MF_SLOT(D, a)]);
        const int w = __ldg(&D.head[MF_SLOT(D, a)]);
        if (c <= 0 || w == s) continue;
        const int ra = __ldg(&D.rev[MF_SLOT(D, a)]);
        const int cr = __ldg(&D.cap[MF_SLOT(D, ra)]);
        D.rr[MF_SLOT(D, a)] = make_int2(0, cr + c);
        D.rr[MF_SLOT(D, ra)] = make_int2(cr + c, 0);
        atomic_add64(exc_ptr(D, w), c);
      }
    }
    ok = grid_sync(D, sh, 1);
  }
  int r = 0, gen = 0, epoch = 0;
  long long rnd = 0;
  // unions with per-instance schedules: every instance's phases, cut and outputs inside run_union
  const bool per_instance = MULTI && D.union_phases && D.inst_relabel && D.mode == MODE_SOLVE && !D.cut_only && D.gseed;
  if (ok && per_instance) {
    ok = run_union<KTD>(D, sh, r, gen, rnd, st, epoch);
    if (tid == 0) D.ctl->t_preflow = gtimer();
  }
  if (!per_instance && ok) ok = run_phase<KTD, MULTI>(D, sh, D.snk, D.src, r, gen, rnd, true, st, epoch);
  if (!per_instance && ok && D.mode == MODE_SOLVE) {
    if (tid == 0) D.ctl->t_preflow = gtimer();
    for (int k = tid; k < D.ninst; k += nthr) {
      const long long val = __ldcg(exc_ptr(D, D.snk[k]));
      if (D.out_value) D.out_value[k] = val;
      if (k == 0) D.ctl->value = val;
    }
    if (D.cut_only) {
      // S_min from the maximum preflow: reachable from s and every excess vertex.
      ok = bfs<KTD>(D, sh, D.src, nullptr, D.ninst, false, true, gen, st, 6);
    } else {
      // Phase 2: return the excess that cannot reach t to s (s plays the sink).
      ok = run_phase<KTD, MULTI>(D, sh, D.src, D.snk, r, gen, rnd, false, st, epoch);
      if (ok) {
        long long left = 0;
        for (int v = tid; v < D.n; v += nthr) {
          const int d = __ldcg(lab_ptr(D, v, 0));
          if (d >= 1 && d <= cap_of(D, v) && __ldcg(exc_ptr(D, v)) != 0) left++;
        }
        left = block_sum(left, sh);
        if (threadIdx.x == 0 && left) atomic_add64(&D.ctl->leftover, left);
        ok = grid_sync(D, sh, 7);
        if (ok && __ldcg(&D.ctl->leftover) != 0) {
          set_err(D, MF_ERR_INTERNAL, 8);
          ok = false;
        }
      }
      // Cut: BFS from s over arcs with positive residual.
      if (ok) ok = bfs<KTD>(D, sh, D.src, nullptr, D.ninst, false, false, gen, st, 9);
    }
    if (ok) {
      if (D.out_cut) {
        const int words = (D.n + 31) >> 5;
        for (int wd = tid; wd < words; wd += nthr) {
          unsigned bits = 0;
          for (int j = 0; j < 32; j++) {
            const int v = wd * 32 + j;
            if (v < D.n && (int)(__ldcg(D.blab + MF_VTX(D, v)) >> 32) != UNV) bits |= 1u << j;
          }
          D.out_cut[wd] = bits;
        }
      }
      if (D.out_flow)
        for (int a = tid; a < D.m; a += nthr) {
          const int f = __ldg(&D.cap[MF_SLOT(D, a)]) - __ldcg(&D.rr[MF_SLOT(D, a)]).x;
          D.out_flow[a] = f > 0 ? f : 0;
        }
    }
  }
  // statistics
  long long x;
  x = block_sum((long long)st.scans_dis, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->scans_dis, x);
  x = block_sum((long long)st.scans_res, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->scans_res, x);
  x = block_sum((long long)st.scans_bfs, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->scans_bfs, x);
  x = block_sum((long long)st.pushes, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->pushes, x);
  x = block_sum((long long)st.relabels, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->relabels, x);
  x = block_sum((long long)st.visits_dis, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->visits_dis, x);
  x = block_sum((long long)st.visits_bfs, sh);
  if (threadIdx.x == 0 && x) atomic_add64(&D.ctl->visits_bfs, x);
  if (tid == 0) D.ctl->t_end = gtimer();
}

// Register-budget variants of the same kernel: __launch_bounds__(MAXT, MINB)
// caps registers at 65536 / (MAXT * MINB) so that more warps stay resident.
// KTD is the largest degree a single thread discharges (arcs cached in
// registers); 16 needs the register budget of one 256-thread CTA per SM.
template <int MAXT, int MINB, int KTD, bool MULTI>
__global__ void __launch_bounds__(MAXT, MINB) solve_kernel(Dev D) {
  solve_body<KTD, MULTI>(D);
}

}  // namespace mf

