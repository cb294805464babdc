// Batched solving (mf_batch_*): many independent instances packed into one
// device graph (instance-offset CSR: instance k's vertices start at V_k and
// its slots at M_k) and solved by one launch of the persistent kernel. Every
// vertex carries its instance's label cap n_k; every instance has its own
// source and sink; phases, rounds and global relabels are shared, and an
// instance whose vertices are all inactive simply takes no part in a round.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "mf.h"
#include "mf_internal.h"

using namespace mf;

struct mf_batch {
  mf_graph *g = nullptr;  // the packed union
  int count = 0;
  std::vector<int> n, s, t;
  std::vector<long long> m, voff, moff;
  std::vector<long long> cwoff;  // first word of every instance's cut bitmap in g->d_cutw (count + 1)
};

namespace mf {

// Runs f(k) for every instance k on the host cores: contiguous runs of
// instances of about equal slot counts (moff = first slot of each instance,
// M = all slots), one thread per run.
template <typename F>
static void parallel_instances(int count, const std::vector<long long> &moff, long long M, F f) {
  unsigned nt = std::thread::hardware_concurrency();
  nt = nt == 0 ? 1 : (nt > 64 ? 64 : nt);
  if (count < 2 * (int)nt || M < (1LL << 20)) nt = 1;
  if (nt == 1) {
    for (int k = 0; k < count; k++) f(k);
    return;
  }
  std::vector<std::thread> th;
  int k0 = 0;
  for (unsigned j = 0; j < nt && k0 < count; j++) {
    const long long target = M * (long long)(j + 1) / (long long)nt;
    int k1 = k0 + 1;
    while (k1 < count && (j + 1 == nt || moff[(size_t)k1] < target)) k1++;
    th.emplace_back([=, &f] {
      for (int k = k0; k < k1; k++) f(k);
    });
    k0 = k1;
  }
  for (int k = k0; k < count; k++) f(k);
  for (auto &t : th) t.join();
}

// Packs `count` host descriptions into one union CSR on the device of opt.
int create_union(int32_t count, const mf_graph_desc *descs, const mf_options *opt, cudaStream_t stream,
                 mf_batch *b, const LaneHost *lane) {
  long long N = 0, M = 0;
  b->count = count;
  for (int k = 0; k < count; k++) {
    const mf_graph_desc &d = descs[k];
    if (d.n < 2) return fail(MF_ERR_INVALID_ARG, "instance %d: n must be >= 2", k);
    if (d.m < 0) return fail(MF_ERR_INVALID_ARG, "instance %d: m must be >= 0", k);
    if (!d.row_offsets || (d.m > 0 && (!d.head || !d.cap || !d.rev)))
      return fail(MF_ERR_INVALID_ARG, "instance %d: NULL array", k);
    if (d.s < 0 || d.s >= d.n || d.t < 0 || d.t >= d.n) return fail(MF_ERR_INVALID_ARG, "instance %d: s or t out of range", k);
    if (d.s == d.t) return fail(MF_ERR_S_EQ_T, "instance %d: source equals sink", k);
    b->n.push_back(d.n);
    b->s.push_back(d.s);
    b->t.push_back(d.t);
    b->m.push_back(d.m);
    b->voff.push_back(N);
    b->moff.push_back(M);
    N += d.n;
    M += d.m;
  }
  if (N > UNV - 4) return fail(MF_ERR_TOO_LARGE, "batch has %lld vertices, beyond the label range", N);
  if (M > 2147483646LL) return fail(MF_ERR_TOO_LARGE, "batch has %lld slots, beyond INT32_MAX", M);
  // host packing with per-instance range checks (offsets must not leak across instances), spread over the
  // host cores by instance (each instance writes its own ranges)
  std::vector<long long> row((size_t)N + 1), rev((size_t)(M > 0 ? M : 1));
  std::vector<int> head((size_t)(M > 0 ? M : 1)), cap((size_t)(M > 0 ? M : 1)), src(count), snk(count);
  std::vector<int2> vinst((size_t)N);       // {label cap, instance} per vertex
  std::vector<int> marcs((size_t)count, 0);  // slots with positive capacity per instance
  std::vector<int> bad(count, 0);  // 1: row offsets, 2: not monotone, 3: head, 4: rev
  std::vector<long long> maxdeg_inst(count, 0);
  parallel_instances(count, b->moff, M, [&](int k) {
    const mf_graph_desc &d = descs[k];
    const long long V = b->voff[k], S = b->moff[k];
    if (d.row_offsets[0] != 0 || d.row_offsets[d.n] != d.m) {
      bad[k] = 1;
      return;
    }
    long long md = 0;
    for (int v = 0; v < d.n; v++) {
      if (d.row_offsets[v] > d.row_offsets[v + 1]) {
        bad[k] = 2;
        return;
      }
      row[(size_t)(V + v)] = S + d.row_offsets[v];
      vinst[(size_t)(V + v)] = make_int2(d.n, k);
      if (v != d.s && v != d.t) md = std::max(md, (long long)(d.row_offsets[v + 1] - d.row_offsets[v]));
    }
    for (long long a = 0; a < d.m; a++) {
      if (d.head[a] < 0 || d.head[a] >= d.n) {
        bad[k] = 3;
        return;
      }
      if (d.rev[a] < 0 || d.rev[a] >= d.m) {
        bad[k] = 4;
        return;
      }
      head[(size_t)(S + a)] = (int)(V + d.head[a]);
      rev[(size_t)(S + a)] = S + d.rev[a];
      cap[(size_t)(S + a)] = d.cap[a];
      if (d.cap[a] > 0) marcs[(size_t)k]++;
    }
    src[k] = (int)(V + d.s);
    snk[k] = (int)(V + d.t);
    maxdeg_inst[k] = md;
  });
  for (int k = 0; k < count; k++) {
    static const char *what[] = {"", "row_offsets must run from 0 to m", "row_offsets not monotone",
                                 "head out of range", "rev out of range"};
    if (bad[k]) return fail(MF_ERR_INVALID_ARG, "instance %d: %s", k, what[bad[k]]);
  }
  row[(size_t)N] = M;

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
  b->g = g;
  g->opt = o;
  g->device = o.device;
  g->n = (int)N;
  g->m = M;
  g->s = src[0];
  g->t = snk[0];
  g->ninst = count;
  g->n_cap = 0;
  g->n_total_for_gr = N;
  if (stream) {
    g->stream = stream;
    g->own_stream = false;
  } else {
    if ((e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    g->own_stream = true;
  }
  if (lane) {
    g->pool = lane->pool;
    g->lane_host = true;
    g->h_ctl = lane->h_ctl;
    g->ev0 = lane->ev0;
    g->ev1 = lane->ev1;
  }
  if ((rc = alloc_state(g))) return rc;
  if ((rc = galloc(g, (void **)&g->vinst, (size_t)N * sizeof(int2), "cudaMalloc vertex instances"))) return rc;
  if ((rc = galloc(g, (void **)&g->inst, (size_t)count * sizeof(InstState), "cudaMalloc instance state"))) return rc;
  if ((rc = galloc(g, (void **)&g->inst_work, (size_t)count * INST_WORK_STRIDE * 8, "cudaMalloc instance work")))
    return rc;
  if ((rc = galloc(g, (void **)&g->inst_marcs, (size_t)count * 4, "cudaMalloc instance arcs"))) return rc;
  if ((rc = galloc(g, (void **)&g->carry, (size_t)N * 4, "cudaMalloc carried entries"))) return rc;
  if ((rc = galloc(g, (void **)&g->gseed, (size_t)count * 4, "cudaMalloc relabel seeds"))) return rc;
  if ((rc = galloc(g, (void **)&g->gblocker, (size_t)count * 4, "cudaMalloc relabel blockers"))) return rc;
  // instance vertex offsets and tiles (runs of at most TILE_VERTICES vertices of one instance) for the
  // global relabels that cover only some instances
  std::vector<int> voff((size_t)count + 1);
  std::vector<int4> tiles;
  for (int k = 0; k < count; k++) {
    const int V = (int)b->voff[(size_t)k], nk = descs[k].n;
    voff[(size_t)k] = V;
    for (int a = 0; a < nk; a += TILE_VERTICES) tiles.push_back(make_int4(V + a, V + std::min(nk, a + TILE_VERTICES), k, 0));
  }
  voff[(size_t)count] = (int)N;
  g->ntiles = (int)tiles.size();
  b->cwoff.assign((size_t)count + 1, 0);
  for (int k = 0; k < count; k++) b->cwoff[(size_t)k + 1] = b->cwoff[(size_t)k] + (descs[k].n + 31) / 32;
  if ((rc = galloc(g, (void **)&g->voff, voff.size() * 4, "cudaMalloc instance offsets"))) return rc;
  if ((rc = galloc(g, (void **)&g->tiles, tiles.size() * sizeof(int4), "cudaMalloc tiles"))) return rc;
  if ((rc = galloc(g, (void **)&g->live, (size_t)count * 4, "cudaMalloc instance flags"))) return rc;
  if ((rc = galloc(g, (void **)&g->cwoff, b->cwoff.size() * 8, "cudaMalloc cut offsets"))) return rc;
  long long *row64 = nullptr, *rev64 = nullptr;
  if ((rc = galloc(g, (void **)&row64, ((size_t)N + 1) * 8, "cudaMalloc staging"))) return rc;
  if ((rc = galloc(g, (void **)&rev64, (size_t)(M > 0 ? M : 1) * 8, "cudaMalloc staging"))) {
    gfree(g, row64);
    return rc;
  }
  e = cudaMemcpyAsync(row64, row.data(), ((size_t)N + 1) * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(rev64, rev.data(), (size_t)M * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(g->head, head.data(), (size_t)M * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(g->cap, cap.data(), (size_t)M * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->vinst, vinst.data(), (size_t)N * sizeof(int2), cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->inst_marcs, marcs.data(), (size_t)count * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->src, src.data(), (size_t)count * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->snk, snk.data(), (size_t)count * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->voff, voff.data(), voff.size() * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->cwoff, b->cwoff.data(), b->cwoff.size() * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);  // host vectors go out of scope below
  if (e != cudaSuccess) {
    gfree(g, row64);
    gfree(g, rev64);
    return cuda_fail(e, "host-to-device copy");
  }
  rc = validate_on_device(g, row64, rev64, g->stream);
  gfree(g, row64);
  gfree(g, rev64);
  if (rc) return rc;
  long long maxdeg = 0;  // over all instances, sources and sinks excluded
  for (int k = 0; k < count; k++) maxdeg = std::max(maxdeg, maxdeg_inst[(size_t)k]);
  g->max_degree = maxdeg;
  return launch_config(g);
}

// Copies each instance's part of the union's cut bitmap (bit u of word u / 32)
// to its own run of words starting at word cwoff[k] of `out`, bit v of
// instance k at bit v of its run (words past the instance's n_k bits zero).
__global__ void k_split_cut(const unsigned *cut, long long words, const int *voff, const long long *cwoff, int count,
                            unsigned *out) {
  const long long total = cwoff[count];
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = count;  // cwoff[lo] <= w < cwoff[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (cwoff[mid] <= w) lo = mid; else hi = mid;
    }
    const long long j = w - cwoff[lo];
    const long long left = (long long)(voff[lo + 1] - voff[lo]) - 32 * j;  // >= 1
    const long long u = (long long)voff[lo] + 32 * j;                       // union bit of the word's first bit
    const long long q = u >> 5;
    const int r = (int)(u & 31);
    unsigned x = cut[q] >> r;
    if (r && q + 1 < words) x |= cut[q + 1] << (32 - r);
    if (left < 32) x &= (1u << left) - 1u;
    out[w] = x;
  }
}

// True when the kernel can run every instance's phases, cut and outputs itself
// (per-instance relabel schedules, full solves), writing each instance's cut
// bitmap straight into its word-aligned run of g->d_cutw. Service lanes use it
// to hand out results early; mf_batch_solve, which returns all results at once,
// keeps the phases shared (fewer global relabels).
static bool per_instance_possible(const mf_graph *g) { return g->inst && g->opt.instance_relabel && !g->opt.cut_only; }

// Device outputs of a union solve and the Dev that writes them (per_instance:
// the kernel runs every instance's phases and outputs on its own).
static int prepare_union(mf_batch *b, bool want_flow, bool want_cut, bool per_instance, Dev &D) {
  mf_graph *g = b->g;
  int rc;
  if (want_flow && !g->d_flow && (rc = galloc(g, (void **)&g->d_flow, (size_t)g->m * 4, "cudaMalloc flow output")))
    return rc;
  const size_t words = ((size_t)g->n + 31) / 32;
  if (want_cut && !per_instance && !g->d_cut &&
      (rc = galloc(g, (void **)&g->d_cut, words * 4, "cudaMalloc cut output")))
    return rc;
  if (want_cut && !g->d_cutw &&
      (rc = galloc(g, (void **)&g->d_cutw, (size_t)b->cwoff[(size_t)b->count] * 4, "cudaMalloc cut outputs")))
    return rc;
  D = make_dev(g);
  D.out_value = g->d_value;
  D.out_flow = want_flow ? g->d_flow : nullptr;
  D.union_phases = per_instance ? 1 : 0;
  if (per_instance)
    D.out_cutw = want_cut ? g->d_cutw : nullptr;
  else
    D.out_cut = want_cut ? g->d_cut : nullptr;
  return MF_OK;
}

// Copies instance k's outputs (value, its slice of the per-slot flow, its cut
// bitmap) to host memory on stream st (enqueued only).
static cudaError_t copy_instance(mf_batch *b, int k, cudaStream_t st, int64_t *value, int32_t *flow, uint32_t *cut) {
  mf_graph *g = b->g;
  cudaError_t e = cudaSuccess;
  if (value) e = cudaMemcpyAsync(value, g->d_value + k, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && flow && b->m[(size_t)k] > 0)
    e = cudaMemcpyAsync(flow, g->d_flow + b->moff[(size_t)k], (size_t)b->m[(size_t)k] * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && cut)
    e = cudaMemcpyAsync(cut, g->d_cutw + b->cwoff[(size_t)k],
                        (size_t)(b->cwoff[(size_t)k + 1] - b->cwoff[(size_t)k]) * 4, cudaMemcpyDeviceToHost, st);
  return e;
}

// Solves the packed union and copies the outputs of every instance to its host
// arrays: values, the instance's slice of the per-slot flow, and its cut
// bitmap (split on the device, or written per instance by the kernel).
int solve_union(mf_batch *b, int64_t *values, int32_t **arc_flows, uint32_t **cut_bits) {
  mf_graph *g = b->g;
  bool want_flow = false, want_cut = false;
  for (int k = 0; k < b->count; k++) {
    if (arc_flows && arc_flows[k]) want_flow = true;
    if (cut_bits && cut_bits[k]) want_cut = true;
  }
  if (g->opt.cut_only && want_flow) return fail(MF_ERR_INVALID_ARG, "cut_only solves produce no per-arc flow");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  Dev D;
  int rc = prepare_union(b, want_flow, want_cut, false, D);
  if (rc) return rc;
  rc = run_kernel(g, D, g->stream);
  if (rc) return rc;
  if (want_cut) {
    const size_t words = ((size_t)g->n + 31) / 32;
    const long long total = b->cwoff[(size_t)b->count];
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    k_split_cut<<<blocks > 0 ? blocks : 1, 256, 0, g->stream>>>(g->d_cut, (long long)words, g->voff, g->cwoff,
                                                              b->count, g->d_cutw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cut split");
  }
  std::vector<long long> vals((size_t)b->count);
  for (int k = 0; k < b->count && e == cudaSuccess; k++)
    e = copy_instance(b, k, g->stream, nullptr, want_flow ? arc_flows[k] : nullptr, want_cut ? cut_bits[k] : nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(vals.data(), g->d_value, (size_t)b->count * 8, cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy of the outputs");
  if (values)
    for (int k = 0; k < b->count; k++) values[k] = vals[(size_t)k];
  return MF_OK;
}

// Service lanes: solves the union like solve_union, but hands every instance
// its results as soon as the kernel has written them (its done flag in the
// lane's mapped host memory), while the other instances are still being
// solved: their outputs are copied on the lane's copy stream, then
// on_done(k, MF_OK) runs. When the kernel has finished, instances without a
// result get the launch's error (on_done(k, rc)). Returns the launch's status.
int solve_union_streaming(mf_batch *b, const LaneHost &lane, int64_t *values, int32_t **arc_flows,
                          uint32_t **cut_bits, void (*on_done)(void *ctx, int k, int rc), void *ctx) {
  mf_graph *g = b->g;
  if (!per_instance_possible(g) || b->count > lane.done_cap) {
    const int rc = solve_union(b, values, arc_flows, cut_bits);
    for (int k = 0; k < b->count; k++) on_done(ctx, k, rc);
    return rc;
  }
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  Dev D;
  int rc = prepare_union(b, true, true, true, D);
  if (rc) return rc;
  memset(lane.h_done, 0, (size_t)b->count * sizeof(unsigned));
  D.done_flag = lane.d_done;
  rc = launch_kernel(g, D, g->stream);
  if (rc) return rc;
  std::vector<char> given((size_t)b->count, 0);
  int left = b->count;
  auto deliver_ready = [&]() -> cudaError_t {
    std::vector<int> ready;
    for (int k = 0; k < b->count; k++)
      if (!given[(size_t)k] && ((volatile unsigned *)lane.h_done)[k]) ready.push_back(k);
    if (ready.empty()) return cudaSuccess;
    cudaError_t ce = cudaSuccess;
    for (int k : ready)
      if (ce == cudaSuccess) ce = copy_instance(b, k, lane.copy, values + k, arc_flows[k], cut_bits[k]);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(lane.copy);
    if (ce != cudaSuccess) return ce;
    for (int k : ready) {
      given[(size_t)k] = 1;
      left--;
      on_done(ctx, k, MF_OK);
    }
    return cudaSuccess;
  };
  for (;;) {
    const cudaError_t q = cudaStreamQuery(g->stream);
    if ((e = deliver_ready()) != cudaSuccess) break;
    if (q != cudaErrorNotReady) {
      e = q;
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  rc = e == cudaSuccess ? finish_kernel(g) : cuda_fail(e, "solver");
  if (rc == MF_OK && left > 0) {  // the kernel finished without flagging some instance: copy them all now
    for (int k = 0; k < b->count && e == cudaSuccess; k++)
      if (!given[(size_t)k]) e = copy_instance(b, k, lane.copy, values + k, arc_flows[k], cut_bits[k]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lane.copy);
    if (e != cudaSuccess) rc = cuda_fail(e, "device-to-host copy of the outputs");
  }
  for (int k = 0; k < b->count; k++)
    if (!given[(size_t)k]) on_done(ctx, k, rc);
  return rc;
}

mf_batch *new_batch() { return new mf_batch(); }

void destroy_union(mf_batch *b) {
  if (!b) return;
  if (b->g) mf_destroy_graph(b->g);
  delete b;
}

}  // namespace mf

extern "C" {

int mf_batch_create(int32_t count, const mf_graph_desc *descs, const mf_options *opt, mf_batch **out) {
  clear_error();
  if (!out) return fail(MF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !descs) return fail(MF_ERR_INVALID_ARG, "count must be >= 1 with descriptions");
  mf_batch *b = new mf_batch();
  int rc = create_union(count, descs, opt, nullptr, b, nullptr);
  if (rc) {
    destroy_union(b);
    return rc;
  }
  *out = b;
  return MF_OK;
}

int mf_batch_solve(mf_batch *b, int64_t *values, int32_t **arc_flows, uint32_t **cut_bits) {
  clear_error();
  if (!b || !b->g) return fail(MF_ERR_INVALID_ARG, "batch is NULL");
  return solve_union(b, values, arc_flows, cut_bits);
}

int mf_batch_get_stats(const mf_batch *b, mf_stats *out) {
  clear_error();
  if (!b || !b->g || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  *out = b->g->stats;
  return MF_OK;
}

void mf_batch_destroy(mf_batch *b) { destroy_union(b); }

int mf_batch_set_options(mf_batch *b, const mf_options *opt) {
  clear_error();
  if (!b || !b->g || !opt) return fail(MF_ERR_INVALID_ARG, "null batch or options");
  return set_options(b->g, opt);
}

int mf_batch_autotune(mf_batch *b, const mf_tune_spec *spec, mf_options *best, double *best_ms) {
  clear_error();
  if (!b || !b->g) return fail(MF_ERR_INVALID_ARG, "null batch");
  return autotune(b->g, spec, best, best_ms);
}

}  // extern "C"
