// Autotuner: chooses the solver options of one graph or batch by timing
// solves of it.
//
// The paper fixes its global-relabel constants (Algorithm 1: freq 0.5,
// alpha 6, beta 12, taken from hi_pr) for a 40-core CPU. On the GPU the
// relabel trigger, the degree bins of the discharge and BFS kernels, the
// persistent kernel's launch shape, the CTA-local lists and the BFS levels per
// grid barrier trade off differently for each graph
// family (a 3D grid runs ~45,000 short rounds, a power-law graph a few
// hundred wide ones), so they are measured: coordinate descent over a fixed
// table of candidates, each candidate timed by the median device time of a
// few solves. Every candidate must reproduce the flow values of the starting
// options (the value is unique), which makes each tuning run a self-check.
#include <algorithm>
#include <cstring>
#include <vector>

#include "mf.h"
#include "mf_internal.h"

namespace mf {
namespace {

// One solve with the current options (outputs off except the values);
// *ms = device time of the kernel.
int timed_solve(mf_graph *g, double *ms, std::vector<long long> *values) {
  Dev D = make_dev(g);
  D.out_value = g->d_value;
  int rc = run_kernel(g, D, g->stream);
  if (rc) return rc;
  values->assign((size_t)g->ninst, 0);
  cudaError_t e = cudaMemcpyAsync(values->data(), g->d_value, (size_t)g->ninst * 8, cudaMemcpyDeviceToHost,
                                  g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy of the flow values");
  *ms = g->stats.solve_ms;
  return MF_OK;
}

// Median device time of `reps` solves; adds their time to *spent.
int measure(mf_graph *g, int reps, double *median_ms, std::vector<long long> *values, double *spent) {
  std::vector<double> t;
  for (int i = 0; i < reps; i++) {
    double ms = 0;
    const int rc = timed_solve(g, &ms, values);
    if (rc) return rc;
    t.push_back(ms);
    *spent += ms;
  }
  std::sort(t.begin(), t.end());
  *median_ms = t[t.size() / 2];
  return MF_OK;
}

enum Coord { GR_TIME_RATIO, GR_FREQ, BIN_THREAD, BIN_WARP, SHAPE, VARIANT, LOCAL, HOPS, PULL, NCOORD };

const double kTimeRatio[] = {0.0, 1.0, 2.0, 4.0};
const double kFreq[] = {0.25, 0.5, 1.0, 2.0};
const int kBinThread[] = {2, 4, 8, 16};
const int kBinWarp[] = {128, 1024, 8192};
const int kShape[][2] = {{256, 2}, {512, 1}, {128, 4}, {256, 1}, {64, 4}};  // threads per CTA, CTAs per SM
// kernel_variant, with the bin_thread it is tried with (-1: unchanged); variant
// 4's 16-slot thread path is tried together with bin_thread 16, which no other
// variant accepts (one coordinate at a time could not reach the pair)
const int kVariant[][2] = {{0, -1}, {1, -1}, {2, -1}, {3, -1}, {4, -1}, {4, 16}};
const int kLocal[] = {0, 1};            // CTA-local lists off / on (K = block_threads / 2)
const int kHops[] = {1, 4, 8, 16};      // BFS levels per grid barrier
const int kPull[] = {0, 20, 50, 200};    // bottom-up BFS levels above n / bfs_pull frontier vertices

int candidates(Coord c) {
  switch (c) {
    case GR_TIME_RATIO: return 4;
    case GR_FREQ: return 4;
    case BIN_THREAD: return 4;
    case BIN_WARP: return 3;
    case SHAPE: return 5;
    case VARIANT: return 6;
    case LOCAL: return 2;
    case HOPS: return 4;
    case PULL: return 4;
    default: return 0;
  }
}

mf_options with(const mf_options &o, Coord c, int k) {
  mf_options x = o;
  switch (c) {
    case GR_TIME_RATIO: x.gr_time_ratio = kTimeRatio[k]; break;
    case GR_FREQ: x.gr_freq = kFreq[k]; break;
    case BIN_THREAD: x.bin_thread = kBinThread[k]; break;
    case BIN_WARP: x.bin_warp = kBinWarp[k]; break;
    case SHAPE:
      x.block_threads = kShape[k][0];
      x.blocks_per_sm = kShape[k][1];
      break;
    case VARIANT:
      x.kernel_variant = kVariant[k][0];
      if (kVariant[k][1] >= 0) x.bin_thread = kVariant[k][1];
      break;
    case LOCAL: x.local_lists = kLocal[k]; break;
    case HOPS: x.bfs_hops = kHops[k]; break;
    case PULL: x.bfs_pull = kPull[k]; break;
    default: break;
  }
  return x;
}

bool same(const mf_options &a, const mf_options &b) { return memcmp(&a, &b, sizeof(mf_options)) == 0; }

}  // namespace

// Replaces the options of g (validated; the launch shape is recomputed). On
// failure g keeps its options.
int set_options(mf_graph *g, const mf_options *o) {
  int rc = check_options(o);
  if (rc) return rc;
  if (o->device != g->device)
    return fail(MF_ERR_INVALID_ARG, "options name device %d, the graph lives on device %d", o->device, g->device);
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const mf_options old = g->opt;
  g->opt = *o;
  if ((rc = launch_config(g))) {
    g->opt = old;
    launch_config(g);
    return rc;
  }
  return MF_OK;
}

int autotune(mf_graph *g, const mf_tune_spec *spec, mf_options *best, double *best_ms) {
  const int reps = spec ? spec->reps : 3;
  const int sweeps = spec ? spec->sweeps : 1;
  const double budget = spec ? spec->time_budget_ms : 0.0;
  if (reps < 1 || reps > 99 || sweeps < 1 || sweeps > 9 || !(budget >= 0))
    return fail(MF_ERR_INVALID_ARG, "tuning needs 1 <= reps <= 99, 1 <= sweeps <= 9, time_budget_ms >= 0");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  mf_options cur = g->opt;
  double cur_ms = 0, spent = 0;
  std::vector<long long> ref, vals;
  int rc = measure(g, reps, &cur_ms, &ref, &spent);
  if (rc) return rc;
  for (int sw = 0; sw < sweeps; sw++) {
    bool moved = false;
    for (int c = 0; c < NCOORD; c++) {
      for (int k = 0; k < candidates((Coord)c); k++) {
        if (budget > 0 && spent >= budget) goto done;
        const mf_options o = with(cur, (Coord)c, k);
        if (same(o, cur)) continue;
        // the local lists and BFS hops act only on graphs whose vertices are all thread-sized
        if ((c == LOCAL || c == HOPS) && keep_local_limit(o, g->max_degree, o.block_threads) == 0 &&
            keep_local_limit(cur, g->max_degree, cur.block_threads) == 0)
          continue;
        if (set_options(g, &o)) {  // an invalid combination or a shape that does not fit: skip it
          clear_error();
          continue;
        }
        double ms = 0;
        if ((rc = measure(g, reps, &ms, &vals, &spent))) {
          set_options(g, &cur);
          return rc;
        }
        if (vals != ref) {
          set_options(g, &cur);
          return fail(MF_ERR_INTERNAL, "a tuning candidate changed a flow value (solver self-check)");
        }
        if (ms < cur_ms) {
          cur = o;
          cur_ms = ms;
          moved = true;
        }
      }
      if ((rc = set_options(g, &cur))) return rc;
    }
    if (!moved) break;
  }
done:
  if ((rc = set_options(g, &cur))) return rc;
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return MF_OK;
}

}  // namespace mf

using namespace mf;

extern "C" {

int mf_set_options(mf_graph *g, const mf_options *opt) {
  clear_error();
  if (!g || !opt) return fail(MF_ERR_INVALID_ARG, "null graph or options");
  return set_options(g, opt);
}

int mf_autotune(mf_graph *g, const mf_tune_spec *spec, mf_options *best, double *best_ms) {
  clear_error();
  if (!g) return fail(MF_ERR_INVALID_ARG, "null graph");
  return autotune(g, spec, best, best_ms);
}

}  // extern "C"
