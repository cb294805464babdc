/*
 * CPU oracle for maximum flow / minimum cut. TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the bench's CPU-baseline leg call it; the GPU
 * solver never does. It shares no code with the GPU path.
 *
 * Source: Baumstark, Blelloch and Shun, "Efficient Implementation of a
 * Synchronous Parallel Push-Relabel Algorithm" (arXiv:1507.01926).
 *   - problem, residual graph, max-flow/min-cut:            Section 2, Eqs. (1)-(2)
 *   - push-relabel (labels, admissible arcs, push, relabel,
 *     active vertices), global relabeling, FIFO order,
 *     maximum preflow then flow decomposition:               Section 2.1
 *   - global-relabel schedule (freq 0.5, alpha 6 => about
 *     every 12n + 2m arc scans), work = deg + 12 per relabel: Section 3 (footnote), Algorithm 1
 *   - global relabel as reverse BFS from the sink:           Section 3, Algorithm 2
 *
 * The oracle is the plain sequential FIFO form of push-relabel with global
 * relabeling. Its results are compared with the GPU solver only where they
 * are unique: the maximum flow value and the minimal source-side minimum cut
 * (the set of vertices reachable from s in the residual graph of any maximum
 * flow, Section 2). Per-arc flows are checked by invariants.
 *
 * Representation (textbook, deliberately different from the solver's): every
 * input arc i = (u, v, c) becomes arc 2i (u -> v, residual c) and arc 2i+1
 * (v -> u, residual 0); the reverse of arc a is a ^ 1. Residuals and excesses
 * are int64.
 *
 * Other routines: Edmonds-Karp (shortest augmenting paths), brute-force cut
 * enumeration, exact BFS sink distances in a given residual graph, and a flow
 * checker. Each is written out from its definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EWORK (-3)     /* work limit reached before the maximum preflow */
#define ORC_EIDENT (-4)    /* internal: the two cut computations disagree */
#define ORC_EPHASE2 (-5)   /* internal: excess left after flow reconstruction */
#define ORC_ECHECK (-6)    /* checked mode: an invariant of push-relabel failed */

typedef struct {
  int32_t n;
  int64_t m;      /* input arcs */
  int64_t *off;   /* n+1: arcs of vertex v are adj[off[v] .. off[v+1]) */
  int64_t *adj;   /* arc ids grouped by tail, input order kept */
  int32_t *to;    /* 2m: head of arc a */
  int64_t *res;   /* 2m: residual capacity of arc a */
  int64_t *e;     /* n: excess */
  int32_t *d;     /* n: distance label */
  int64_t *cur;   /* n: current-arc position in adj */
  int32_t *queue; /* n: FIFO ring */
  uint8_t *inq;   /* n */
  /* statistics */
  int64_t scans, pushes, relabels, grs, work_limit;
  /* checked mode (orc_maxflow_checked): input capacities, and what failed */
  const int32_t *cap_in;
  int check;           /* 0 off, 1 check, 2 check with the planted relabel mistake */
  int64_t checks;      /* invariant checks run */
  int32_t check_s;     /* the source s of the instance (its excess may be negative) */
  int64_t bad;         /* 0, or 1 + the failed invariant (see check_state) */
} orc_graph;

static void orc_free(orc_graph *g) {
  free(g->off);
  free(g->adj);
  free(g->to);
  free(g->res);
  free(g->e);
  free(g->d);
  free(g->cur);
  free(g->queue);
  free(g->inq);
  memset(g, 0, sizeof(*g));
}

static int orc_init(orc_graph *g, int32_t n, int64_t m, const int32_t *tail, const int32_t *head,
                    const int32_t *cap) {
  memset(g, 0, sizeof(*g));
  if (n < 2 || m < 0) return ORC_EINVAL;
  for (int64_t i = 0; i < m; i++)
    if (tail[i] < 0 || tail[i] >= n || head[i] < 0 || head[i] >= n || cap[i] < 0) return ORC_EINVAL;
  g->n = n;
  g->m = m;
  g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  g->adj = (int64_t *)malloc((size_t)(2 * m + 1) * sizeof(int64_t));
  g->to = (int32_t *)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
  g->res = (int64_t *)malloc((size_t)(2 * m + 1) * sizeof(int64_t));
  g->e = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  g->d = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  g->cur = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  g->queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  g->inq = (uint8_t *)calloc((size_t)n, 1);
  if (!g->off || !g->adj || !g->to || !g->res || !g->e || !g->d || !g->cur || !g->queue || !g->inq) {
    orc_free(g);
    return ORC_ENOMEM;
  }
  for (int64_t i = 0; i < m; i++) {
    g->to[2 * i] = head[i];
    g->res[2 * i] = cap[i];
    g->to[2 * i + 1] = tail[i];
    g->res[2 * i + 1] = 0;
    g->off[tail[i] + 1]++;
    g->off[head[i] + 1]++;
  }
  for (int32_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
  int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!fill) {
    orc_free(g);
    return ORC_ENOMEM;
  }
  memcpy(fill, g->off, (size_t)n * sizeof(int64_t));
  for (int64_t a = 0; a < 2 * m; a++) {
    int32_t from = g->to[a ^ 1];
    g->adj[fill[from]++] = a;
  }
  free(fill);
  return ORC_OK;
}

/* Global relabeling (Section 2.1; Algorithm 2): d(v) := exact distance from v
 * to snk in the residual graph, found by BFS from snk over the reverse
 * residual graph. src is never labelled (keeps d = n), unreachable vertices
 * keep d = n. Vertex w is discovered from v through arc a = (v -> w) when the
 * opposite arc a^1 = (w -> v) has residual capacity. */
static void global_relabel(orc_graph *g, int32_t src, int32_t snk) {
  int32_t n = g->n;
  for (int32_t v = 0; v < n; v++) g->d[v] = n;
  g->d[snk] = 0;
  int64_t qh = 0, qt = 0;
  g->queue[qt++] = snk;
  while (qh < qt) {
    int32_t v = g->queue[qh++];
    for (int64_t k = g->off[v]; k < g->off[v + 1]; k++) {
      int64_t a = g->adj[k];
      int32_t w = g->to[a];
      g->scans++;
      if (w == src || w == snk || g->d[w] != n) continue;
      if (g->res[a ^ 1] > 0) {
        g->d[w] = g->d[v] + 1;
        g->queue[qt++] = w;
      }
    }
  }
  g->grs++;
}

/* Relabel (Section 2.1): d(v) := 1 + min{ d(w) : (v,w) residual }, at most n.
 * check == 2 plants a mistake (one more than that) for the checker's own test. */
static void relabel(orc_graph *g, int32_t v) {
  int32_t n = g->n;
  int64_t best = n;
  for (int64_t k = g->off[v]; k < g->off[v + 1]; k++) {
    int64_t a = g->adj[k];
    g->scans++;
    if (g->res[a] > 0 && (int64_t)g->d[g->to[a]] + 1 < best) best = (int64_t)g->d[g->to[a]] + 1;
  }
  if (g->check == 2 && best < n) best++;
  g->d[v] = (int32_t)best;
  g->relabels++;
}

/* Checked mode: the invariants of a push-relabel phase toward snk (Section
 * 2.1) on the current state. Returns 0, or the number of the first failure:
 *   1: a residual is negative;
 *   2: an arc pair does not keep its capacity (res[a] + res[a^1] = cap);
 *   3: a vertex other than s holds negative excess;
 *   4: an excess differs from the net inflow implied by the residuals;
 *   5: a label is not valid: d(u) > d(w) + 1 for a residual arc (u, w) with
 *      u other than src (the paper's validity condition for distance labels). */
static int check_state(orc_graph *g, int32_t s, int32_t src) {
  const int32_t n = g->n;
  g->checks++;
  int64_t *net = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  if (!net) return 0;
  int fail = 0;
  for (int64_t i = 0; i < g->m && !fail; i++) {
    const int64_t f = g->res[2 * i + 1], r = g->res[2 * i];
    if (r < 0 || f < 0) fail = 1;
    else if (r + f != (int64_t)g->cap_in[i]) fail = 2;
    else {
      net[g->to[2 * i]] += f;      /* head receives f */
      net[g->to[2 * i + 1]] -= f;  /* tail sends f */
    }
  }
  for (int32_t v = 0; v < n && !fail; v++) {
    if (v != s && g->e[v] < 0) fail = 3;
    else if (g->e[v] != net[v]) fail = 4;
  }
  for (int64_t a = 0; a < 2 * g->m && !fail; a++) {
    const int32_t u = g->to[a ^ 1], w = g->to[a];
    if (u != src && g->res[a] > 0 && (int64_t)g->d[u] > (int64_t)g->d[w] + 1) fail = 5;
  }
  free(net);
  return fail;
}

/*
 * One push-relabel phase in FIFO order with global relabeling, moving excess
 * toward snk (Section 2.1). Vertices src and snk are never active. A vertex is
 * active when e > 0 and d < n; the phase ends when none is (a maximum preflow
 * for phase 1). Global relabeling runs first and then whenever the work since
 * the last one exceeds 12n + 2m, work being deg(v) + 12 per relabel
 * (Section 3 footnote; Algorithm 1 constants freq = 1/2, alpha = 6, beta = 12).
 */
static int pr_phase(orc_graph *g, int32_t src, int32_t snk) {
  int32_t n = g->n;
  int64_t thr = 12LL * n + 2LL * g->m;
  int64_t work = INT64_MAX; /* global relabel before the first discharge */
  int64_t qh = 0, qcount = 0;
  for (;;) {
    if (work > thr) {
      global_relabel(g, src, snk);
      if (g->check) {
        const int f = check_state(g, g->check_s, src);
        if (f) {
          g->bad = f;
          return ORC_ECHECK;
        }
      }
      work = 0;
      qh = 0;
      qcount = 0;
      memset(g->inq, 0, (size_t)n);
      for (int32_t v = 0; v < n; v++) {
        g->cur[v] = g->off[v];
        if (v != src && v != snk && g->e[v] > 0 && g->d[v] < n) {
          g->queue[(qh + qcount++) % n] = v;
          g->inq[v] = 1;
        }
      }
    }
    if (qcount == 0) break;
    if (g->work_limit > 0 && g->scans > g->work_limit) return ORC_EWORK;
    int32_t v = g->queue[qh];
    qh = (qh + 1) % n;
    qcount--;
    g->inq[v] = 0;
    if (g->d[v] >= n || g->e[v] == 0) continue;
    /* discharge v: push along admissible arcs (d(v) = d(w) + 1, residual > 0)
     * from the current arc on; relabel when the arc list is exhausted. */
    while (g->e[v] > 0) {
      if (g->cur[v] == g->off[v + 1]) {
        relabel(g, v);
        if (g->check) {  /* after every relabel as well */
          const int f = check_state(g, g->check_s, src);
          if (f) {
            g->bad = f;
            return ORC_ECHECK;
          }
        }
        work += (g->off[v + 1] - g->off[v]) + 12;
        g->cur[v] = g->off[v];
        if (g->d[v] >= n) break;
        continue;
      }
      int64_t a = g->adj[g->cur[v]];
      int32_t w = g->to[a];
      g->scans++;
      if (g->res[a] > 0 && g->d[v] == g->d[w] + 1) {
        int64_t delta = g->e[v] < g->res[a] ? g->e[v] : g->res[a];
        g->res[a] -= delta;
        g->res[a ^ 1] += delta;
        g->e[v] -= delta;
        g->e[w] += delta;
        g->pushes++;
        if (w != src && w != snk && !g->inq[w]) {
          g->queue[(qh + qcount++) % n] = w;
          g->inq[w] = 1;
        }
        if (g->res[a] == 0) g->cur[v]++;
      } else {
        g->cur[v]++;
      }
    }
    if (g->check) {  /* after every discharge */
      const int f = check_state(g, g->check_s, src);
      if (f) {
        g->bad = f;
        return ORC_ECHECK;
      }
    }
  }
  return ORC_OK;
}

/* Vertices reachable in the residual graph from the marked seeds (mark[] in/out). */
static void residual_reach(orc_graph *g, uint8_t *mark) {
  int64_t qh = 0, qt = 0;
  for (int32_t v = 0; v < g->n; v++)
    if (mark[v]) g->queue[qt++] = v;
  while (qh < qt) {
    int32_t v = g->queue[qh++];
    for (int64_t k = g->off[v]; k < g->off[v + 1]; k++) {
      int64_t a = g->adj[k];
      int32_t w = g->to[a];
      if (g->res[a] > 0 && !mark[w]) {
        mark[w] = 1;
        g->queue[qt++] = w;
      }
    }
  }
}

/*
 * Maximum flow by two-phase FIFO push-relabel.
 *   phase 1: maximum preflow (initial saturation of all arcs out of s, then
 *            pr_phase toward t). The flow value is e(t).
 *   phase 2: the preflow becomes a flow by returning every remaining excess to
 *            s, with the same pr_phase run toward s (t plays the never-active
 *            end). Section 2.1 names a greedy decomposition for this step;
 *            any method that returns the excess gives a maximum flow.
 *   cut:     minimal source side S_min = vertices reachable from s in the
 *            residual graph of the flow (Section 2). It is also computed a
 *            second way, from the maximum preflow, as the set reachable from
 *            s and from every vertex still holding excess; the two must agree.
 *
 * flow_out[i] (nullable, m entries) = flow on input arc i; cut_out[v]
 * (nullable, n entries) = 1 iff v in S_min; stats (nullable, 8 entries) =
 * {arc scans, pushes, relabels, global relabels, phase-1 arc scans, phase-1
 * pushes, phase-1 relabels, phase-1 global relabels}. work_limit > 0 stops
 * phase 1 after about that many arc scans and returns ORC_EWORK (used to time
 * a bounded sample). Returns the flow value (>= 0) or a negative error.
 */
static int64_t maxflow_impl(int32_t n, int64_t m, const int32_t *tail, const int32_t *head, const int32_t *cap,
                            int32_t s, int32_t t, int64_t work_limit, int64_t *flow_out, uint8_t *cut_out,
                            int64_t *stats, int check, int64_t *check_out) {
  if (s < 0 || s >= n || t < 0 || t >= n || s == t) return ORC_EINVAL;
  orc_graph g;
  int rc = orc_init(&g, n, m, tail, head, cap);
  if (rc) return rc;
  g.work_limit = work_limit;
  g.cap_in = cap;
  g.check = check;
  g.check_s = s;
  /* initialization: d = 0 except d(s) = n; saturate every arc out of s */
  for (int32_t v = 0; v < n; v++) g.d[v] = 0;
  g.d[s] = n;
  for (int64_t k = g.off[s]; k < g.off[s + 1]; k++) {
    int64_t a = g.adj[k];
    int64_t c = g.res[a];
    if (c <= 0) continue;
    g.res[a] = 0;
    g.res[a ^ 1] += c;
    g.e[g.to[a]] += c;
    g.e[s] -= c;
  }
  rc = pr_phase(&g, s, t);
  int64_t p1[4] = {g.scans, g.pushes, g.relabels, g.grs};
  if (rc) {
    if (stats) {
      int64_t st[8] = {g.scans, g.pushes, g.relabels, g.grs, p1[0], p1[1], p1[2], p1[3]};
      memcpy(stats, st, sizeof(st));
    }
    if (check_out) {
      check_out[0] = g.checks;
      check_out[1] = g.bad;
    }
    orc_free(&g);
    return rc;
  }
  int64_t value = g.e[t];

  /* second cut computation, from the maximum preflow */
  uint8_t *r = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *smin = (uint8_t *)calloc((size_t)n, 1);
  if (!r || !smin) {
    free(r);
    free(smin);
    orc_free(&g);
    return ORC_ENOMEM;
  }
  r[s] = 1;
  for (int32_t v = 0; v < n; v++)
    if (v != s && v != t && g.e[v] > 0) r[v] = 1;
  residual_reach(&g, r);

  /* phase 2 */
  g.work_limit = 0;
  rc = pr_phase(&g, t, s);
  for (int32_t v = 0; v < n && rc == ORC_OK; v++)
    if (v != s && v != t && g.e[v] != 0) rc = ORC_EPHASE2;
  if (rc == ORC_OK) {
    smin[s] = 1;
    residual_reach(&g, smin);
    if (memcmp(r, smin, (size_t)n) != 0) rc = ORC_EIDENT;
  }
  if (rc == ORC_OK) {
    if (flow_out)
      for (int64_t i = 0; i < m; i++) flow_out[i] = g.res[2 * i + 1];
    if (cut_out) memcpy(cut_out, smin, (size_t)n);
  }
  if (stats) {
    int64_t st[8] = {g.scans, g.pushes, g.relabels, g.grs, p1[0], p1[1], p1[2], p1[3]};
    memcpy(stats, st, sizeof(st));
  }
  if (check_out) {
    check_out[0] = g.checks;
    check_out[1] = g.bad;
  }
  free(r);
  free(smin);
  orc_free(&g);
  return rc == ORC_OK ? value : rc;
}

int64_t orc_maxflow(int32_t n, int64_t m, const int32_t *tail, const int32_t *head, const int32_t *cap, int32_t s,
                    int32_t t, int64_t work_limit, int64_t *flow_out, uint8_t *cut_out, int64_t *stats) {
  return maxflow_impl(n, m, tail, head, cap, s, t, work_limit, flow_out, cut_out, stats, 0, NULL);
}

/*
 * orc_maxflow in checked mode: after every global relabel, relabel and
 * discharge of both phases the state is checked (check_state: residual bounds, pair
 * capacities, excess = net inflow, label validity). plant = 1 plants a
 * mistake in relabel (one too high), so that a test can see the checker
 * catch it. check_out (2 entries) = {checks run, 0 or 1 + failed invariant}.
 * Returns as orc_maxflow, or ORC_ECHECK when an invariant failed.
 */
int64_t orc_maxflow_checked(int32_t n, int64_t m, const int32_t *tail, const int32_t *head, const int32_t *cap,
                            int32_t s, int32_t t, int32_t plant, int64_t *flow_out, uint8_t *cut_out,
                            int64_t *stats, int64_t *check_out) {
  return maxflow_impl(n, m, tail, head, cap, s, t, 0, flow_out, cut_out, stats, plant ? 2 : 1, check_out);
}

/*
 * Edmonds-Karp: repeatedly augment along a shortest residual s-t path found by
 * BFS until none is left (Ford-Fulkerson, Section 2). cut_out (nullable) =
 * vertices reachable from s in the final residual graph. Returns the value.
 */
int64_t orc_edmonds_karp(int32_t n, int64_t m, const int32_t *tail, const int32_t *head, const int32_t *cap,
                         int32_t s, int32_t t, uint8_t *cut_out) {
  if (s < 0 || s >= n || t < 0 || t >= n || s == t) return ORC_EINVAL;
  orc_graph g;
  int rc = orc_init(&g, n, m, tail, head, cap);
  if (rc) return rc;
  int64_t *pred = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!pred) {
    orc_free(&g);
    return ORC_ENOMEM;
  }
  int64_t value = 0;
  for (;;) {
    for (int32_t v = 0; v < n; v++) pred[v] = -1;
    pred[s] = -2;
    int64_t qh = 0, qt = 0;
    g.queue[qt++] = s;
    while (qh < qt && pred[t] == -1) {
      int32_t v = g.queue[qh++];
      for (int64_t k = g.off[v]; k < g.off[v + 1]; k++) {
        int64_t a = g.adj[k];
        int32_t w = g.to[a];
        if (g.res[a] > 0 && pred[w] == -1) {
          pred[w] = a;
          g.queue[qt++] = w;
        }
      }
    }
    if (pred[t] == -1) break;
    int64_t b = INT64_MAX;
    for (int32_t v = t; v != s; v = g.to[pred[v] ^ 1])
      if (g.res[pred[v]] < b) b = g.res[pred[v]];
    for (int32_t v = t; v != s; v = g.to[pred[v] ^ 1]) {
      g.res[pred[v]] -= b;
      g.res[pred[v] ^ 1] += b;
    }
    value += b;
  }
  if (cut_out) {
    memset(cut_out, 0, (size_t)n);
    cut_out[s] = 1;
    residual_reach(&g, cut_out);
  }
  free(pred);
  orc_free(&g);
  return value;
}

/*
 * Minimum cut by enumeration of every source side S (s in S, t not in S) over
 * n <= 22 vertices: cap(S) = sum of capacities of arcs leaving S. Returns the
 * minimum; smin_out (nullable) = intersection of all minimising S, which is
 * the minimal source side (minimum cuts are closed under intersection).
 */
int64_t orc_bruteforce_cut(int32_t n, int64_t m, const int32_t *tail, const int32_t *head, const int32_t *cap,
                           int32_t s, int32_t t, uint8_t *smin_out) {
  if (n < 2 || n > 22 || s < 0 || s >= n || t < 0 || t >= n || s == t) return ORC_EINVAL;
  int32_t others[22];
  int k = 0;
  for (int32_t v = 0; v < n; v++)
    if (v != s && v != t) others[k++] = v;
  int64_t best = INT64_MAX;
  uint32_t inter = 0;
  for (uint64_t mask = 0; mask < (1ULL << k); mask++) {
    uint32_t side = 1u << s;
    for (int j = 0; j < k; j++)
      if (mask >> j & 1) side |= 1u << others[j];
    int64_t c = 0;
    for (int64_t i = 0; i < m; i++)
      if ((side >> tail[i] & 1) && !(side >> head[i] & 1)) c += cap[i];
    if (c < best) {
      best = c;
      inter = side;
    } else if (c == best) {
      inter &= side;
    }
  }
  if (smin_out)
    for (int32_t v = 0; v < n; v++) smin_out[v] = (uint8_t)(inter >> v & 1);
  return best;
}

/*
 * Exact labels of a global relabel (Section 3; Algorithm 2) for a given
 * residual graph, given as its list of residual arcs (rtail[k] -> rhead[k],
 * each with positive residual capacity): d(t) = 0; d(v) = length of a
 * shortest residual path from v to t whose vertices other than v avoid s;
 * d(s) = n; d(v) = n when no such path exists.
 */
int orc_sink_distances(int32_t n, int64_t k, const int32_t *rtail, const int32_t *rhead, int32_t s, int32_t t,
                       int32_t *d_out) {
  if (n < 2 || k < 0 || s < 0 || s >= n || t < 0 || t >= n || s == t) return ORC_EINVAL;
  int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *in = (int32_t *)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!off || !in || !q) {
    free(off);
    free(in);
    free(q);
    return ORC_ENOMEM;
  }
  for (int64_t i = 0; i < k; i++) {
    if (rtail[i] < 0 || rtail[i] >= n || rhead[i] < 0 || rhead[i] >= n) {
      free(off);
      free(in);
      free(q);
      return ORC_EINVAL;
    }
    off[rhead[i] + 1]++;
  }
  for (int32_t v = 0; v < n; v++) off[v + 1] += off[v];
  int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!fill) {
    free(off);
    free(in);
    free(q);
    return ORC_ENOMEM;
  }
  memcpy(fill, off, (size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < k; i++) in[fill[rhead[i]]++] = rtail[i];
  free(fill);
  for (int32_t v = 0; v < n; v++) d_out[v] = n;
  d_out[t] = 0;
  int64_t qh = 0, qt = 0;
  q[qt++] = t;
  while (qh < qt) {
    int32_t v = q[qh++];
    for (int64_t j = off[v]; j < off[v + 1]; j++) {
      int32_t u = in[j];
      if (u == s || u == t || d_out[u] != n) continue;
      d_out[u] = d_out[v] + 1;
      q[qt++] = u;
    }
  }
  free(off);
  free(in);
  free(q);
  return ORC_OK;
}

/*
 * Checks a claimed maximum flow against the definitions of Section 2:
 *   bit 0: some 0 <= f(a) <= c(a) fails
 *   bit 1: conservation fails at some v not in {s, t} (Eq. 1)
 *   bit 2: net outflow of s != value
 *   bit 3: net inflow of t != value
 *   bit 4: a residual s-t path exists (the flow is not maximum)
 *   bit 5: cut invalid (s not in S, or t in S)
 *   bit 6: capacity of the cut (S, V\S) != value
 *   bit 7: S is not the set reachable from s in the residual graph
 * cut (nullable) gives S (1 = source side); bits 5-7 are checked only with it.
 * Returns 0 when every check passes, a negative error for bad arguments.
 */
int orc_check_flow(int32_t n, int64_t m, const int32_t *tail, const int32_t *head, const int32_t *cap, int32_t s,
                   int32_t t, const int64_t *flow, int64_t value, const uint8_t *cut) {
  orc_graph g;
  int rc = orc_init(&g, n, m, tail, head, cap);
  if (rc) return rc;
  int bad = 0;
  for (int64_t i = 0; i < m; i++) {
    if (flow[i] < 0 || flow[i] > cap[i]) bad |= 1;
    g.e[head[i]] += flow[i];
    g.e[tail[i]] -= flow[i];
    g.res[2 * i] = (int64_t)cap[i] - flow[i];
    g.res[2 * i + 1] = flow[i];
  }
  for (int32_t v = 0; v < n; v++)
    if (v != s && v != t && g.e[v] != 0) bad |= 2;
  if (-g.e[s] != value) bad |= 4;
  if (g.e[t] != value) bad |= 8;
  uint8_t *r = (uint8_t *)calloc((size_t)n, 1);
  if (!r) {
    orc_free(&g);
    return ORC_ENOMEM;
  }
  r[s] = 1;
  if (!(bad & 1)) {
    residual_reach(&g, r);
    if (r[t]) bad |= 16;
  }
  if (cut) {
    if (!cut[s] || cut[t]) bad |= 32;
    int64_t c = 0;
    for (int64_t i = 0; i < m; i++)
      if (cut[tail[i]] && !cut[head[i]]) c += cap[i];
    if (c != value) bad |= 64;
    if (!(bad & 1) && memcmp(r, cut, (size_t)n) != 0) bad |= 128;
  }
  free(r);
  orc_free(&g);
  return bad;
}
