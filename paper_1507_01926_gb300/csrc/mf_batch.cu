// Batched solving (mf_batch_*): many independent instances packed into one
// device graph (instance-offset CSR: instance k's vertices start at V_k and
// its slots at M_k) and solved by one launch of the persistent kernel. Every
// vertex carries its instance's label cap n_k; every instance has its own
// source and sink; phases, rounds and global relabels are shared, and an
// instance whose vertices are all inactive simply takes no part in a round.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mf.h"
#include "mf_internal.h"

using namespace mf;

struct mf_batch {
  mf_graph *g = nullptr;  // the packed union
  int count = 0;
  std::vector<int> n, s, t;
  std::vector<long long> m, voff, moff;
};

namespace mf {

// Packs `count` host descriptions into one union CSR on the device of opt.
int create_union(int32_t count, const mf_graph_desc *descs, const mf_options *opt, cudaStream_t stream,
                 mf_batch *b) {
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
  // host packing with per-instance range checks (offsets must not leak across instances)
  std::vector<long long> row((size_t)N + 1), rev((size_t)(M > 0 ? M : 1));
  std::vector<int> head((size_t)(M > 0 ? M : 1)), cap((size_t)(M > 0 ? M : 1)), ncap((size_t)N), src(count), snk(count);
  for (int k = 0; k < count; k++) {
    const mf_graph_desc &d = descs[k];
    const long long V = b->voff[k], S = b->moff[k];
    if (d.row_offsets[0] != 0 || d.row_offsets[d.n] != d.m)
      return fail(MF_ERR_INVALID_ARG, "instance %d: row_offsets must run from 0 to m", k);
    for (int v = 0; v < d.n; v++) {
      if (d.row_offsets[v] > d.row_offsets[v + 1]) return fail(MF_ERR_INVALID_ARG, "instance %d: row_offsets not monotone", k);
      row[(size_t)(V + v)] = S + d.row_offsets[v];
      ncap[(size_t)(V + v)] = d.n;
    }
    for (long long a = 0; a < d.m; a++) {
      if (d.head[a] < 0 || d.head[a] >= d.n) return fail(MF_ERR_INVALID_ARG, "instance %d: head out of range", k);
      if (d.rev[a] < 0 || d.rev[a] >= d.m) return fail(MF_ERR_INVALID_ARG, "instance %d: rev out of range", k);
      head[(size_t)(S + a)] = (int)(V + d.head[a]);
      rev[(size_t)(S + a)] = S + d.rev[a];
      cap[(size_t)(S + a)] = d.cap[a];
    }
    src[k] = (int)(V + d.s);
    snk[k] = (int)(V + d.t);
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
  if ((rc = alloc_state(g))) return rc;
  if ((e = cudaMalloc((void **)&g->ncap, (size_t)N * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc label caps");
  long long *row64 = nullptr, *rev64 = nullptr;
  if ((e = cudaMalloc((void **)&row64, ((size_t)N + 1) * 8)) != cudaSuccess) return cuda_fail(e, "cudaMalloc staging");
  if ((e = cudaMalloc((void **)&rev64, (size_t)(M > 0 ? M : 1) * 8)) != cudaSuccess) {
    cudaFree(row64);
    return cuda_fail(e, "cudaMalloc staging");
  }
  e = cudaMemcpyAsync(row64, row.data(), ((size_t)N + 1) * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(rev64, rev.data(), (size_t)M * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(g->head, head.data(), (size_t)M * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(g->cap, cap.data(), (size_t)M * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->ncap, ncap.data(), (size_t)N * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->src, src.data(), (size_t)count * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->snk, snk.data(), (size_t)count * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);  // host vectors go out of scope below
  if (e != cudaSuccess) {
    cudaFree(row64);
    cudaFree(rev64);
    return cuda_fail(e, "host-to-device copy");
  }
  rc = validate_on_device(g, row64, rev64, g->stream);
  cudaFree(row64);
  cudaFree(rev64);
  if (rc) return rc;
  long long maxdeg = 0;  // over all instances, sources and sinks excluded
  for (int k = 0; k < count; k++) {
    const mf_graph_desc &d = descs[k];
    for (int v = 0; v < d.n; v++)
      if (v != d.s && v != d.t) maxdeg = std::max(maxdeg, (long long)(d.row_offsets[v + 1] - d.row_offsets[v]));
  }
  g->max_degree = maxdeg;
  return launch_config(g);
}

// Solves the packed union and splits the outputs per instance (host arrays).
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
  if (want_flow && !g->d_flow && (e = cudaMalloc((void **)&g->d_flow, (size_t)(g->m > 0 ? g->m : 1) * 4)) != cudaSuccess)
    return cuda_fail(e, "cudaMalloc flow output");
  const size_t words = ((size_t)g->n + 31) / 32;
  if (want_cut && !g->d_cut && (e = cudaMalloc((void **)&g->d_cut, words * 4)) != cudaSuccess)
    return cuda_fail(e, "cudaMalloc cut output");
  Dev D = make_dev(g);
  D.out_value = g->d_value;
  D.out_flow = want_flow ? g->d_flow : nullptr;
  D.out_cut = want_cut ? g->d_cut : nullptr;
  int rc = run_kernel(g, D, g->stream);
  if (rc) return rc;
  std::vector<long long> vals((size_t)b->count);
  e = cudaMemcpyAsync(vals.data(), g->d_value, (size_t)b->count * 8, cudaMemcpyDeviceToHost, g->stream);
  std::vector<int> flow;
  std::vector<unsigned> cut;
  if (e == cudaSuccess && want_flow) {
    flow.resize((size_t)g->m);
    e = cudaMemcpyAsync(flow.data(), g->d_flow, (size_t)g->m * 4, cudaMemcpyDeviceToHost, g->stream);
  }
  if (e == cudaSuccess && want_cut) {
    cut.resize(words);
    e = cudaMemcpyAsync(cut.data(), g->d_cut, words * 4, cudaMemcpyDeviceToHost, g->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy of the outputs");
  for (int k = 0; k < b->count; k++) {
    if (values) values[k] = vals[(size_t)k];
    if (want_flow && arc_flows[k] && b->m[(size_t)k] > 0)
      memcpy(arc_flows[k], flow.data() + b->moff[(size_t)k], (size_t)b->m[(size_t)k] * 4);
    if (want_cut && cut_bits[k]) {
      const long long V = b->voff[(size_t)k];
      const int nk = b->n[(size_t)k];
      uint32_t *out = cut_bits[k];
      memset(out, 0, ((size_t)nk + 31) / 32 * 4);
      for (int v = 0; v < nk; v++) {
        const long long u = V + v;
        if ((cut[(size_t)(u >> 5)] >> (u & 31)) & 1u) out[v >> 5] |= 1u << (v & 31);
      }
    }
  }
  return MF_OK;
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
  int rc = create_union(count, descs, opt, nullptr, b);
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
