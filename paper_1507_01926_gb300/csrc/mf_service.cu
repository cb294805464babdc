// Serving (mf_service_*, mf_submit, mf_poll, mf_wait): continuous batching of
// max-flow requests on one GPU.
//
// Requests are copied at submission and queued. Worker lanes (host threads,
// each with its own CUDA stream and a share of the SMs for its persistent
// launches) admit queued requests in arrival order while their estimated
// device footprint fits the memory budget, pack them into one instance-offset
// union (mf_batch machinery) and solve it. A request that arrives while other
// requests are on the GPU is admitted by the next free lane as soon as memory
// allows, so its solve overlaps with the ones already running. Results stay
// with the service until mf_poll hands them out.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mf.h"
#include "mf_internal.h"

using namespace mf;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  mf_ticket id = 0;
  int n = 0, s = 0, t = 0;
  long long m = 0;
  std::vector<int64_t> row, rev;
  std::vector<int32_t> head, cap;
  size_t bytes = 0;
  Clock::time_point t_submit, t_done;
  bool done = false;
  int rc = MF_OK;
  std::string err;
  int64_t value = 0;
  std::vector<int32_t> flow;
  std::vector<uint32_t> cut;
};

// Device bytes one request occupies while resident (vertex state, slot
// arrays, staging during creation, outputs).
size_t footprint(long long n, long long m) { return (size_t)(77 * n + 32 * m + 65536); }

}  // namespace

struct mf_service {
  size_t budget = 0;
  mf_options opt{};
  int lanes = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  cudaMemPool_t pool = nullptr;  // device memory of the lanes' unions (stream-ordered)
  std::deque<Request *> pending;
  std::unordered_map<mf_ticket, Request *> tickets;
  size_t in_use = 0;
  long long resident_n = 0, resident_m = 0;
  mf_ticket next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace mf {
int create_union(int32_t count, const mf_graph_desc *descs, const mf_options *opt, cudaStream_t stream,
                 mf_batch *b, const LaneHost *lane);
int solve_union(mf_batch *b, int64_t *values, int32_t **arc_flows, uint32_t **cut_bits);
int solve_union_streaming(mf_batch *b, const LaneHost &lane, int64_t *values, int32_t **arc_flows,
                          uint32_t **cut_bits, void (*on_done)(void *ctx, int k, int rc), void *ctx);
mf_batch *new_batch();
void destroy_union(mf_batch *b);
const char *last_error();
}  // namespace mf

namespace {
// A lane's view of the requests of the union it is solving.
struct LaneUnion {
  mf_service *svc;
  std::vector<Request *> *batch;
  std::vector<int64_t> *values;
};

// Completes request k of the lane's union (its outputs are in place): called as
// soon as the kernel has written them, while the rest of the union may still
// be solving.
void lane_on_done(void *ctx, int k, int rc) {
  LaneUnion *u = static_cast<LaneUnion *>(ctx);
  Request *r = (*u->batch)[(size_t)k];
  const std::string err = rc ? std::string(last_error()) : std::string();
  {
    std::lock_guard<std::mutex> lk(u->svc->mu);
    r->value = (*u->values)[(size_t)k];
    r->rc = rc;
    r->err = err;
    r->done = true;
    r->t_done = Clock::now();
    // the instance itself is no longer needed
    std::vector<int64_t>().swap(r->row);
    std::vector<int64_t>().swap(r->rev);
    std::vector<int32_t>().swap(r->head);
    std::vector<int32_t>().swap(r->cap);
  }
  u->svc->cv_done.notify_all();
}
}  // namespace

static void lane_main(mf_service *svc, int lane) {
  mf_options o = svc->opt;
  cudaSetDevice(o.device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  LaneHost lh{svc->pool, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
  cudaMallocHost((void **)&lh.h_ctl, sizeof(Ctl));
  cudaEventCreate(&lh.ev0);
  cudaEventCreate(&lh.ev1);
  cudaStreamCreateWithFlags(&lh.copy, cudaStreamNonBlocking);
  // done flags the kernel sets per instance, read by this thread while the kernel runs (unions of more
  // instances than this are solved without early delivery)
  const int kDoneCap = 1 << 16;
  if (cudaHostAlloc((void **)&lh.h_done, kDoneCap * sizeof(unsigned), cudaHostAllocMapped) == cudaSuccess &&
      cudaHostGetDevicePointer((void **)&lh.d_done, lh.h_done, 0) == cudaSuccess)
    lh.done_cap = kDoneCap;
  else
    cudaGetLastError();
  for (;;) {
    std::vector<Request *> batch;
    size_t bytes = 0;
    long long adm_n = 0, adm_m = 0;  // the admitted requests' sizes (a request may be handed out and freed by
                                     // mf_poll while the rest of its union is still being solved)
    {
      std::unique_lock<std::mutex> lk(svc->mu);
      svc->cv_work.wait(lk, [&] {
        return svc->stop ||
               (!svc->pending.empty() && svc->in_use + svc->pending.front()->bytes <= svc->budget);
      });
      if (svc->stop) break;
      long long nn = 0, mm = 0;
      // a lane takes its share of the queue (the rest is left to the other lanes, which run beside it), so
      // that a burst is spread over all lanes instead of filling one lane's launch
      const size_t share = (svc->pending.size() + (size_t)svc->lanes - 1) / (size_t)svc->lanes;
      while (!svc->pending.empty()) {
        if (o.union_max_requests > 0 && (int)batch.size() >= o.union_max_requests) break;
        if (batch.size() >= share) break;
        Request *r = svc->pending.front();
        if (svc->in_use + bytes + r->bytes > svc->budget) break;
        if (svc->resident_n + nn + r->n > UNV - 4 || svc->resident_m + mm + r->m > 2147483646LL) break;
        bytes += r->bytes;
        nn += r->n;
        mm += r->m;
        batch.push_back(r);
        svc->pending.pop_front();
      }
      svc->in_use += bytes;
      svc->resident_n += nn;
      svc->resident_m += mm;
      adm_n = nn;
      adm_m = mm;
      if (!svc->pending.empty()) svc->cv_work.notify_one();  // another lane may take the rest
    }
    std::vector<mf_graph_desc> descs(batch.size());
    for (size_t i = 0; i < batch.size(); i++) {
      Request *r = batch[i];
      descs[i] = mf_graph_desc{r->n, r->m, r->row.data(), r->head.data(), r->cap.data(), r->rev.data(), r->s, r->t};
      r->flow.resize((size_t)r->m);
      r->cut.resize(((size_t)r->n + 31) / 32);
    }
    std::vector<int64_t> values(batch.size(), 0);
    std::vector<int32_t *> fl(batch.size());
    std::vector<uint32_t *> cu(batch.size());
    for (size_t i = 0; i < batch.size(); i++) {
      fl[i] = batch[i]->flow.data();
      cu[i] = batch[i]->cut.data();
    }
    mf_batch *b = new_batch();
    LaneUnion u{svc, &batch, &values};
    int rc = (lh.h_ctl && lh.ev0 && lh.ev1 && lh.copy)
                 ? create_union((int32_t)batch.size(), descs.data(), &o, stream, b, &lh)
                 : fail(MF_ERR_CUDA, "service lane set-up failed");
    if (rc == MF_OK)  // every request completes as soon as its own results are written
      solve_union_streaming(b, lh, values.data(), fl.data(), cu.data(), lane_on_done, &u);
    else
      for (size_t i = 0; i < batch.size(); i++) lane_on_done(&u, (int)i, rc);
    destroy_union(b);
    {  // every request of the union is done (and may be gone): only the admitted totals are used here
      std::lock_guard<std::mutex> lk(svc->mu);
      svc->in_use -= bytes;
      svc->resident_n -= adm_n;
      svc->resident_m -= adm_m;
    }
    svc->cv_work.notify_all();
  }
  if (stream) cudaStreamSynchronize(stream);
  if (lh.h_ctl) cudaFreeHost(lh.h_ctl);
  if (lh.ev0) cudaEventDestroy(lh.ev0);
  if (lh.ev1) cudaEventDestroy(lh.ev1);
  if (lh.copy) cudaStreamDestroy(lh.copy);
  if (lh.h_done) cudaFreeHost(lh.h_done);
  if (stream) cudaStreamDestroy(stream);
}

extern "C" {

int mf_service_create(size_t device_budget_bytes, const mf_options *opt, mf_service **out) {
  clear_error();
  if (!out) return fail(MF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (device_budget_bytes < (1u << 20)) return fail(MF_ERR_INVALID_ARG, "budget must be at least 1 MiB");
  mf_options o;
  if (opt)
    o = *opt;
  else
    mf_service_default_options(&o);
  int rc = check_options(&o);
  if (rc) return rc;
  cudaError_t e = cudaSetDevice(o.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  int bps = 0;
  if (solver_occupancy(o.block_threads, &bps, o.kernel_variant, true) || bps < 1)
    return fail(MF_ERR_CUDA, "solver kernel does not fit %d threads per CTA", o.block_threads);
  mf_service *svc = new mf_service();
  svc->budget = device_budget_bytes;
  // one stream-ordered pool for the lanes' unions: freeing a finished union does not wait for the other
  // lanes' kernels (cudaFree would), and freed memory stays in the pool for the next union
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = o.device;
  if ((e = cudaMemPoolCreate(&svc->pool, &props)) != cudaSuccess) {
    delete svc;
    return cuda_fail(e, "cudaMemPoolCreate");
  }
  unsigned long long keep = ~0ULL;
  cudaMemPoolSetAttribute(svc->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  // one lane per CTA slot of an SM (at most 8): a lane's launch takes one CTA per SM, so the lanes'
  // persistent kernels are resident together and the requests of different lanes overlap on the device
  if (o.blocks_per_sm > 0 && o.blocks_per_sm < bps) bps = o.blocks_per_sm;
  svc->lanes = bps < 8 ? bps : 8;
  o.blocks_per_sm = 1;
  svc->opt = o;
  for (int k = 0; k < svc->lanes; k++) svc->workers.emplace_back(lane_main, svc, k);
  *out = svc;
  return MF_OK;
}

int mf_submit(mf_service *svc, const mf_graph_desc *g, mf_ticket *out) {
  clear_error();
  if (!svc || !g || !out) return fail(MF_ERR_INVALID_ARG, "NULL argument");
  if (g->n < 2 || g->m < 0) return fail(MF_ERR_INVALID_ARG, "n must be >= 2 and m >= 0");
  if (!g->row_offsets || (g->m > 0 && (!g->head || !g->cap || !g->rev))) return fail(MF_ERR_INVALID_ARG, "NULL array");
  if (g->s < 0 || g->s >= g->n || g->t < 0 || g->t >= g->n) return fail(MF_ERR_INVALID_ARG, "s or t out of range");
  if (g->s == g->t) return fail(MF_ERR_S_EQ_T, "source equals sink");
  const size_t bytes = footprint(g->n, g->m);
  if (bytes > svc->budget)
    return fail(MF_ERR_OVER_BUDGET, "instance needs about %zu bytes, budget is %zu", bytes, svc->budget);
  Request *r = new Request();
  r->n = g->n;
  r->m = g->m;
  r->s = g->s;
  r->t = g->t;
  r->bytes = bytes;
  r->row.assign(g->row_offsets, g->row_offsets + g->n + 1);
  r->head.assign(g->head, g->head + g->m);
  r->cap.assign(g->cap, g->cap + g->m);
  r->rev.assign(g->rev, g->rev + g->m);
  {
    std::lock_guard<std::mutex> lk(svc->mu);
    r->id = svc->next_id++;
    r->t_submit = Clock::now();
    svc->tickets[r->id] = r;
    svc->pending.push_back(r);
  }
  svc->cv_work.notify_one();
  *out = r->id;
  return MF_OK;
}

int mf_wait(mf_service *svc, mf_ticket ticket, int32_t timeout_ms, double *latency_ms) {
  clear_error();
  if (!svc) return fail(MF_ERR_INVALID_ARG, "service is NULL");
  std::unique_lock<std::mutex> lk(svc->mu);
  auto it = svc->tickets.find(ticket);
  if (it == svc->tickets.end()) return fail(MF_ERR_UNKNOWN_TICKET, "unknown ticket %lld", (long long)ticket);
  Request *r = it->second;
  if (timeout_ms < 0)
    svc->cv_done.wait(lk, [&] { return r->done; });
  else if (!svc->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
    return MF_PENDING;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return MF_OK;
}

int mf_poll(mf_service *svc, mf_ticket ticket, int64_t *flow_value, int32_t *arc_flow, uint32_t *cut_bits) {
  clear_error();
  if (!svc) return fail(MF_ERR_INVALID_ARG, "service is NULL");
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lk(svc->mu);
    auto it = svc->tickets.find(ticket);
    if (it == svc->tickets.end()) return fail(MF_ERR_UNKNOWN_TICKET, "unknown ticket %lld", (long long)ticket);
    r = it->second;
    if (!r->done) return MF_PENDING;
    svc->tickets.erase(it);
  }
  int rc = r->rc;
  if (rc == MF_OK) {
    if (flow_value) *flow_value = r->value;
    if (arc_flow && r->m > 0) memcpy(arc_flow, r->flow.data(), (size_t)r->m * 4);
    if (cut_bits) memcpy(cut_bits, r->cut.data(), r->cut.size() * 4);
  } else {
    fail(rc, "%s", r->err.c_str());
  }
  delete r;
  return rc;
}

void mf_service_destroy(mf_service *svc) {
  if (!svc) return;
  {
    std::lock_guard<std::mutex> lk(svc->mu);
    svc->stop = true;
  }
  svc->cv_work.notify_all();
  for (auto &t : svc->workers) t.join();
  for (auto &kv : svc->tickets) delete kv.second;
  if (svc->pool) cudaMemPoolDestroy(svc->pool);
  delete svc;
}

}  // extern "C"
