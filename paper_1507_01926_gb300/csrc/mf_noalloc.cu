// mf_solve_noalloc: a max-flow solve that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside another runtime's
// memory pool or under a strict memory budget, plug-ins that must leave the
// CUDA allocator alone, or services that have pre-committed all device memory
// at start-up. They hold the graph and
// the outputs in device memory already; what the solve needs beyond that
// (residuals, labels, excesses, vertex lists, the control block) is placed
// in one fixed scratch area that the library declares statically, so the call
// itself never allocates.
//
// The scratch area is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES
// (32 MiB); every GPU that loads the library holds it until the process exits.
// All calls on a device share it and it keeps the last call's contents: every
// call re-initialises what must start at zero, and calls whose work overlaps on
// the GPU (different streams or host threads at the same time) race on it.
#include <cuda_runtime.h>
#include <string.h>

#include "mf.h"
#include "mf_internal.h"

namespace mf {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch layout for n vertices and m slots (offsets from the start).
struct Layout {
  size_t ctl, flags, term, rr, vs, blab, list0, list1, list2, total;
};

Layout layout(long long n, long long m) {
  Layout L;
  size_t o = 0;
  L.ctl = o;
  o = align256(o + sizeof(Ctl));
  L.flags = o;
  o = align256(o + 16);
  L.term = o;
  o = align256(o + 8);
  L.rr = o;
  o = align256(o + 8 * (size_t)m);
  L.vs = o;
  o = align256(o + sizeof(VRec) * (size_t)n);
  L.blab = o;
  o = align256(o + 8 * (size_t)n);
  L.list0 = o;
  o = align256(o + 4 * (size_t)n);
  L.list1 = o;
  o = align256(o + 4 * (size_t)n);
  L.list2 = o;
  o = align256(o + 4 * (size_t)n);
  L.total = o;
  return L;
}

// The scratch array's device address on the current device. Looked up on
// every call (no allocation once the module is loaded, and cheap): an address
// kept from an earlier call would be stale after cudaDeviceReset or a new
// primary context, which load the module, and the array with it, anew.
int scratch_base(unsigned char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch area");
  *out = static_cast<unsigned char *>(p);
  return MF_OK;
}

enum : unsigned { N_ROW = 1u, N_HEAD = 2u, N_REV = 4u, N_CAP = 8u, N_PAIR = 16u, N_TAIL = 32u, N_OVERFLOW = 64u };

__global__ void k_noalloc_rows(int n, int m, const int *row, unsigned *flags) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
    const int x = row[v];
    bool bad = x < 0 || x > m || (v == 0 && x != 0) || (v == n && x != m) || (v < n && x > row[v + 1]);
    if (bad) atomicOr(flags, N_ROW);
  }
}

__global__ void k_noalloc_maxdeg(int n, const int *row, int s, int t, unsigned *out) {
  unsigned mx = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (v != s && v != t) mx = max(mx, (unsigned)(row[v + 1] - row[v]));
  if (mx) atomicMax(out, mx);
}

__global__ void k_noalloc_slots(int n, int m, const int *row, const int *head, const int *cap, const int *rev,
                                unsigned *flags, unsigned long long *m_arcs) {
  unsigned f = 0;
  unsigned long long cnt = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) {
    const int h = head[a], ra = rev[a], c = cap[a];
    if (h < 0 || h >= n) f |= N_HEAD;
    if (c < 0) f |= N_CAP;
    if (ra < 0 || ra >= m || ra == a) {
      f |= N_REV;
      continue;
    }
    int lo = 0, hi = n;  // tail(a): row[lo] <= a < row[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (row[mid] <= a) lo = mid; else hi = mid;
    }
    if (rev[ra] != a) f |= N_PAIR;
    if (head[ra] != lo) f |= N_TAIL;
    if ((long long)c + (long long)cap[ra] > 2147483647LL) f |= N_OVERFLOW;
    if (c > 0) cnt++;
  }
  if (f) atomicOr(flags, f);
  if (cnt) atomicAdd(m_arcs, cnt);
}

int read_flags(unsigned char *dev_flags, cudaStream_t st, unsigned *f, unsigned long long *marcs,
               unsigned *maxdeg) {
  unsigned h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(h, dev_flags, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "graph validation");
  *f = h[0];
  *maxdeg = h[1];
  *marcs = (unsigned long long)h[2] | ((unsigned long long)h[3] << 32);
  return MF_OK;
}

}  // namespace
}  // namespace mf

using namespace mf;

extern "C" int mf_solve_noalloc(int32_t n, int32_t m, const int32_t *d_row, const int32_t *d_head,
                                const int32_t *d_cap, const int32_t *d_rev, int32_t s, int32_t t, int64_t *d_value,
                                int32_t *d_flow, uint32_t *d_cut, void *stream) {
  clear_error();
  if (n < 2 || m < 0) return fail(MF_ERR_INVALID_ARG, "n must be >= 2 and m >= 0");
  if (!d_row || (m > 0 && (!d_head || !d_cap || !d_rev)) || !d_value) return fail(MF_ERR_INVALID_ARG, "NULL array");
  if (s < 0 || s >= n || t < 0 || t >= n) return fail(MF_ERR_INVALID_ARG, "s or t out of range");
  if (s == t) return fail(MF_ERR_S_EQ_T, "source equals sink");
  const Layout L = layout(n, m);
  if (L.total > NOALLOC_SCRATCH_BYTES)
    return fail(MF_ERR_TOO_LARGE,
                "graph needs %zu bytes of scratch (about 56 per vertex + 8 per slot); the fixed area holds %zu",
                L.total, NOALLOC_SCRATCH_BYTES);
  unsigned char *base = nullptr;
  int rc = scratch_base(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  mf_options o;
  mf_default_options(&o);
  cudaError_t e = cudaGetDevice(&o.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

  // validation (flags and the positive-arc count live in the scratch area)
  unsigned char *flags = base + L.flags;
  if ((e = cudaMemsetAsync(flags, 0, 16, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int T = 256;
  k_noalloc_rows<<<(n + 1 + T - 1) / T < 4096 ? (n + 1 + T - 1) / T : 4096, T, 0, st>>>(n, m, d_row,
                                                                                      (unsigned *)flags);
  unsigned f = 0, maxdeg = 0;
  unsigned long long marcs = 0;
  if ((rc = read_flags(flags, st, &f, &marcs, &maxdeg))) return rc;
  if (!f && m > 0) {
    k_noalloc_slots<<<(m + T - 1) / T < 4096 ? (m + T - 1) / T : 4096, T, 0, st>>>(
        n, m, d_row, d_head, d_cap, d_rev, (unsigned *)flags, (unsigned long long *)(flags + 8));
    k_noalloc_maxdeg<<<(n + T - 1) / T < 4096 ? (n + T - 1) / T : 4096, T, 0, st>>>(n, d_row, s, t,
                                                                                   (unsigned *)flags + 1);
    if ((rc = read_flags(flags, st, &f, &marcs, &maxdeg))) return rc;
  }
  if (f & (N_ROW | N_HEAD | N_REV | N_CAP))
    return fail(MF_ERR_INVALID_ARG, "invalid graph (flags 0x%x): row offsets, head, rev or capacity", f);
  if (f & (N_PAIR | N_TAIL)) return fail(MF_ERR_BAD_PAIRING, "bad reverse pairing (flags 0x%x)", f);
  if (f & N_OVERFLOW) return fail(MF_ERR_CAP_OVERFLOW, "cap[a] + cap[rev[a]] exceeds INT32_MAX");

  // launch shape from the device, as for mf_create_graph
  int bps = 0, sms = 0;
  if (solver_occupancy(o.block_threads, &bps, o.kernel_variant, false) || bps < 1)
    return fail(MF_ERR_CUDA, "solver kernel does not fit");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device)) != cudaSuccess)
    return cuda_fail(e, "cudaDeviceGetAttribute");

  Dev D;
  memset(&D, 0, sizeof(D));
  D.n = n;
  D.m = m;
  D.n_cap = n;
  D.vinst = nullptr;
  D.row = d_row;
  D.head = d_head;
  D.rev = d_rev;
  D.cap = d_cap;
  D.rr = reinterpret_cast<int2 *>(base + L.rr);
  D.vs = reinterpret_cast<VRec *>(base + L.vs);
  D.blab = reinterpret_cast<unsigned long long *>(base + L.blab);
  D.bfs_hops = 1;
  D.list[0] = reinterpret_cast<int *>(base + L.list0);
  D.list[1] = reinterpret_cast<int *>(base + L.list1);
  D.list[2] = reinterpret_cast<int *>(base + L.list2);
  int *term = reinterpret_cast<int *>(base + L.term);
  D.src = term;
  D.snk = term + 1;
  D.ninst = 1;
  D.ctl = reinterpret_cast<Ctl *>(base + L.ctl);
  D.bin_thread = o.bin_thread;
  D.bin_warp = o.bin_warp;
  D.beta = o.work_beta;
  D.gr_threshold = relabel_threshold(o, n, (long long)marcs);
  D.gr_time_ratio = o.gr_time_ratio;
  D.max_rounds = 2000000LL;
  D.timeout_ns = (unsigned long long)o.timeout_ms * 1000000ULL;
  D.mode = MODE_SOLVE;
  D.cta_vertices = maxdeg > (unsigned)o.bin_warp ? 1 : 0;
  D.out_value = reinterpret_cast<long long *>(d_value);
  D.out_flow = d_flow;
  D.out_cut = d_cut;

  const int st_terms[2] = {s, t};
  if ((e = cudaMemcpyAsync(term, st_terms, sizeof(st_terms), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync");
  if ((e = cudaMemsetAsync(D.ctl, 0, sizeof(Ctl), st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if ((e = launch_solver(D, bps * sms, o.block_threads, st, o.kernel_variant)) != cudaSuccess)
    return cuda_fail(e, "cooperative launch of the solver");
  Ctl c;
  e = cudaMemcpyAsync(&c, D.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "solver");
  return device_status(c);
}
