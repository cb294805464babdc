// CSR builder with reverse-slot pairing (mf_build_csr in include/mf.h).
//
// The paired-slot layout is the adjacency-array representation in which each
// edge also holds the residual capacity of its reverse (arXiv:1507.01926,
// Section 4.2). Steps, all O(m + n) with stable counting sorts:
//   1. drop self-loops;
//   2. group the arcs by unordered vertex pair {u, v}, input order kept;
//   3. in each group pair the k-th arc u->v with the k-th arc v->u; every
//      other arc gets a partner slot of capacity 0;
//   4. emit the pairs in order of their first input arc, two slots each, and
//      sort the slots into rows by (tail, head), ties in emission order.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "mf.h"

namespace mf {
int fail(int code, const char *fmt, ...);
void clear_error();
}  // namespace mf

using namespace mf;

namespace {

// Stable counting sort of idx[] by key(idx) in [0, nkeys).
template <class Key>
void counting_sort(std::vector<long long> &idx, long long nkeys, Key key) {
  std::vector<long long> cnt((size_t)nkeys + 1, 0);
  for (long long i : idx) cnt[(size_t)key(i) + 1]++;
  for (long long k = 0; k < nkeys; k++) cnt[(size_t)k + 1] += cnt[(size_t)k];
  std::vector<long long> out(idx.size());
  for (long long i : idx) out[(size_t)cnt[(size_t)key(i)]++] = i;
  idx.swap(out);
}

}  // namespace

extern "C" {

int mf_build_csr(int32_t n, int64_t m_in, const int32_t *tail, const int32_t *head, const int32_t *cap,
                 mf_csr *out) {
  clear_error();
  if (!out) return fail(MF_ERR_INVALID_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  if (n < 1) return fail(MF_ERR_INVALID_ARG, "n must be >= 1");
  if (m_in < 0) return fail(MF_ERR_INVALID_ARG, "m_in must be >= 0");
  if (m_in > 0 && (!tail || !head || !cap)) return fail(MF_ERR_INVALID_ARG, "NULL array");
  for (int64_t i = 0; i < m_in; i++) {
    if (tail[i] < 0 || tail[i] >= n || head[i] < 0 || head[i] >= n)
      return fail(MF_ERR_INVALID_ARG, "arc %lld has an endpoint out of range", (long long)i);
    if (cap[i] < 0) return fail(MF_ERR_INVALID_ARG, "arc %lld has a negative capacity", (long long)i);
  }
  // 1-2: non-loop arcs grouped by (min endpoint, max endpoint), input order kept
  std::vector<long long> idx;
  idx.reserve((size_t)m_in);
  long long loops = 0;
  for (int64_t i = 0; i < m_in; i++) {
    if (tail[i] == head[i])
      loops++;
    else
      idx.push_back(i);
  }
  auto lo = [&](long long i) { return (long long)(tail[i] < head[i] ? tail[i] : head[i]); };
  auto hi = [&](long long i) { return (long long)(tail[i] < head[i] ? head[i] : tail[i]); };
  counting_sort(idx, n, hi);
  counting_sort(idx, n, lo);
  // 3: partner of each arc (-1 = none)
  std::vector<long long> partner((size_t)m_in, -1);
  for (size_t g0 = 0; g0 < idx.size();) {
    size_t g1 = g0;
    while (g1 < idx.size() && lo(idx[g1]) == lo(idx[g0]) && hi(idx[g1]) == hi(idx[g0])) g1++;
    size_t f = g0, b = g0;  // next unpaired forward (tail = lo) / backward arc
    for (;;) {
      while (f < g1 && tail[idx[f]] != lo(idx[f])) f++;
      while (b < g1 && tail[idx[b]] == lo(idx[b])) b++;
      if (f >= g1 || b >= g1) break;
      partner[(size_t)idx[f]] = idx[b];
      partner[(size_t)idx[b]] = idx[f];
      f++;
      b++;
    }
    g0 = g1;
  }
  // 4: emit pairs in order of first input arc
  long long npairs = 0;
  for (int64_t i = 0; i < m_in; i++)
    if (tail[i] != head[i] && (partner[(size_t)i] < 0 || partner[(size_t)i] > i)) npairs++;
  const long long m = 2 * npairs;
  if (m > 2147483646LL) return fail(MF_ERR_TOO_LARGE, "%lld slots exceed INT32_MAX", m);
  // slot s: tail stail[s], head shead[s], cap scap[s], partner slot s ^ 1, input arc sarc[s] (-1 none)
  std::vector<int32_t> stail((size_t)m), shead((size_t)m), scap((size_t)m);
  std::vector<long long> sarc((size_t)m);
  long long k = 0;
  for (int64_t i = 0; i < m_in; i++) {
    if (tail[i] == head[i]) continue;
    const long long p = partner[(size_t)i];
    if (p >= 0 && p < i) continue;
    const long long c1 = cap[i], c2 = p >= 0 ? cap[p] : 0;
    if (c1 + c2 > 2147483647LL)
      return fail(MF_ERR_CAP_OVERFLOW, "arcs %lld and %lld: capacities sum beyond INT32_MAX", (long long)i, p);
    stail[(size_t)k] = tail[i];
    shead[(size_t)k] = head[i];
    scap[(size_t)k] = (int32_t)c1;
    sarc[(size_t)k] = i;
    stail[(size_t)k + 1] = head[i];
    shead[(size_t)k + 1] = tail[i];
    scap[(size_t)k + 1] = (int32_t)c2;
    sarc[(size_t)k + 1] = p;
    k += 2;
  }
  std::vector<long long> order((size_t)m);
  for (long long s = 0; s < m; s++) order[(size_t)s] = s;
  counting_sort(order, n, [&](long long s) { return (long long)shead[(size_t)s]; });
  counting_sort(order, n, [&](long long s) { return (long long)stail[(size_t)s]; });
  std::vector<long long> pos((size_t)m);
  for (long long j = 0; j < m; j++) pos[(size_t)order[(size_t)j]] = j;

  out->row_offsets = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  out->head = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  out->cap = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  out->rev = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
  out->arc_slot = (int64_t *)malloc((size_t)(m_in > 0 ? m_in : 1) * sizeof(int64_t));
  if (!out->row_offsets || !out->head || !out->cap || !out->rev || !out->arc_slot) {
    mf_free_csr(out);
    return fail(MF_ERR_OOM, "host allocation failed");
  }
  out->n = n;
  out->m = m;
  out->dropped_self_loops = loops;
  for (int32_t v = 0; v <= n; v++) out->row_offsets[v] = 0;
  for (long long s = 0; s < m; s++) out->row_offsets[stail[(size_t)s] + 1]++;
  for (int32_t v = 0; v < n; v++) out->row_offsets[v + 1] += out->row_offsets[v];
  for (int64_t i = 0; i < m_in; i++) out->arc_slot[i] = -1;
  for (long long j = 0; j < m; j++) {
    const long long s = order[(size_t)j];
    out->head[j] = shead[(size_t)s];
    out->cap[j] = scap[(size_t)s];
    out->rev[j] = pos[(size_t)(s ^ 1)];
    if (sarc[(size_t)s] >= 0) out->arc_slot[sarc[(size_t)s]] = j;
  }
  return MF_OK;
}

void mf_free_csr(mf_csr *c) {
  if (!c) return;
  free(c->row_offsets);
  free(c->head);
  free(c->cap);
  free(c->rev);
  free(c->arc_slot);
  memset(c, 0, sizeof(*c));
}

}  // extern "C"
