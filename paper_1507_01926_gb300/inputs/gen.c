/*
 * Seeded synthetic max-flow instances (input arc lists).
 *
 * This module holds structure and random numbers only: it builds the vertex
 * numbering, the arc lists and the capacities of the workload families, and
 * nothing of the max-flow method. Both the CPU oracle and the GPU solver take
 * its output as their input.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used in its counter form:
 * draw i of a stream with key k is mix(k + (i + 1) * golden_gamma), so every
 * draw can be taken independently and in any order. U[a,b] maps a 64-bit draw
 * to [a,b] by the multiply-high method (Lemire 2019) without the rejection
 * step; its bias is below (b-a+1)/2^64. logU[a,b] = floor(exp(U(ln a,
 * ln(b+1)))) clamped to [a,b].
 *
 * Every graph is a list of directed arcs (tail, head, cap) with int32
 * capacities >= 1. Vertex ids are 0..n-1; s and t are given with the list.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw i (0-based) of the SplitMix64 sequence whose state starts at key. */
static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN_GAMMA); }

/* Independent stream `stream` of a seed. */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed * GOLDEN_GAMMA + stream * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL);
}

static inline int64_t unif(uint64_t x, int64_t a, int64_t b) {
  uint64_t r = (uint64_t)(b - a + 1);
  return a + (int64_t)(((unsigned __int128)x * r) >> 64);
}

static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static inline int64_t logunif(uint64_t x, int64_t a, int64_t b) {
  double la = log((double)a), lb = log((double)(b + 1));
  int64_t k = (int64_t)floor(exp(la + u01(x) * (lb - la)));
  if (k < a) k = a;
  if (k > b) k = b;
  return k;
}

typedef struct {
  int32_t n, s, t;
  int64_t m;
  int32_t *tail, *head, *cap;
} mfg_arcs;

void mfg_free(mfg_arcs *g) {
  if (!g) return;
  free(g->tail);
  free(g->head);
  free(g->cap);
  g->tail = g->head = g->cap = NULL;
  g->m = 0;
}

static int alloc_arcs(mfg_arcs *g, int64_t m) {
  g->m = m;
  size_t b = (size_t)(m > 0 ? m : 1) * sizeof(int32_t);
  g->tail = (int32_t *)malloc(b);
  g->head = (int32_t *)malloc(b);
  g->cap = (int32_t *)malloc(b);
  if (!g->tail || !g->head || !g->cap) {
    mfg_free(g);
    return -1;
  }
  return 0;
}

/* Exposed single draws, for parameters sampled on the Python side. */
uint64_t mfg_draw(uint64_t seed, uint64_t stream, uint64_t i) { return draw(stream_key(seed, stream), i); }
int64_t mfg_unif(uint64_t seed, uint64_t stream, uint64_t i, int64_t a, int64_t b) {
  return unif(draw(stream_key(seed, stream), i), a, b);
}
int64_t mfg_logunif(uint64_t seed, uint64_t stream, uint64_t i, int64_t a, int64_t b) {
  return logunif(draw(stream_key(seed, stream), i), a, b);
}
double mfg_u01(uint64_t seed, uint64_t stream, uint64_t i) { return u01(draw(stream_key(seed, stream), i)); }

/*
 * 2D 4-connected H x W grid (vision-style). Pixel p = y*W + x; s = H*W,
 * t = H*W + 1. Every pixel has an arc to each existing neighbour in the order
 * (-x, +x, -y, +y), capacity U[nlo,nhi] per direction. Then every pixel gets
 * a terminal arc: s->p with probability 1/2, else p->t, capacity U[tlo,thi].
 */
int mfg_grid2d(int32_t H, int32_t W, uint64_t seed, int32_t nlo, int32_t nhi, int32_t tlo, int32_t thi,
               mfg_arcs *out) {
  if (H < 1 || W < 1 || (int64_t)H * W > 2000000000LL) return -1;
  int64_t np = (int64_t)H * W;
  int64_t mg = 2LL * H * (W - 1) + 2LL * W * (H - 1);
  memset(out, 0, sizeof(*out));
  if (alloc_arcs(out, mg + np)) return -2;
  out->n = (int32_t)(np + 2);
  out->s = (int32_t)np;
  out->t = (int32_t)np + 1;
  uint64_t kc = stream_key(seed, 1), kt = stream_key(seed, 2);
  int64_t k = 0;
  for (int32_t y = 0; y < H; y++)
    for (int32_t x = 0; x < W; x++) {
      int64_t p = (int64_t)y * W + x;
      const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
      for (int d = 0; d < 4; d++) {
        int32_t xx = x + dx[d], yy = y + dy[d];
        if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
        out->tail[k] = (int32_t)p;
        out->head[k] = (int32_t)((int64_t)yy * W + xx);
        out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)p * 4 + d), nlo, nhi);
        k++;
      }
    }
  for (int64_t p = 0; p < np; p++) {
    int src = (draw(kt, 2 * (uint64_t)p) >> 63) != 0;
    int32_t c = (int32_t)unif(draw(kt, 2 * (uint64_t)p + 1), tlo, thi);
    out->tail[k] = src ? out->s : (int32_t)p;
    out->head[k] = src ? (int32_t)p : out->t;
    out->cap[k] = c;
    k++;
  }
  out->m = k;
  return 0;
}

/*
 * 3D 6-connected X x Y x Z grid. Voxel p = (z*Y + y)*X + x; s = XYZ,
 * t = XYZ + 1. Neighbour arcs in the order (-x,+x,-y,+y,-z,+z) with capacity
 * U[clo,chi] per direction; s->p for every voxel of face z=0 and p->t for every
 * voxel of face z=Z-1, both at capacity tcap.
 */
int mfg_grid3d(int32_t X, int32_t Y, int32_t Z, uint64_t seed, int32_t clo, int32_t chi, int32_t tcap,
               mfg_arcs *out) {
  if (X < 1 || Y < 1 || Z < 2) return -1;
  int64_t np = (int64_t)X * Y * Z;
  if (np > 2000000000LL) return -1;
  int64_t mg = 2LL * ((int64_t)(X - 1) * Y * Z + (int64_t)X * (Y - 1) * Z + (int64_t)X * Y * (Z - 1));
  int64_t face = (int64_t)X * Y;
  memset(out, 0, sizeof(*out));
  if (alloc_arcs(out, mg + 2 * face)) return -2;
  out->n = (int32_t)(np + 2);
  out->s = (int32_t)np;
  out->t = (int32_t)np + 1;
  uint64_t kc = stream_key(seed, 1);
  int64_t k = 0;
  for (int32_t z = 0; z < Z; z++)
    for (int32_t y = 0; y < Y; y++)
      for (int32_t x = 0; x < X; x++) {
        int64_t p = ((int64_t)z * Y + y) * X + x;
        const int dx[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0}, dz[6] = {0, 0, 0, 0, -1, 1};
        for (int d = 0; d < 6; d++) {
          int32_t xx = x + dx[d], yy = y + dy[d], zz = z + dz[d];
          if (xx < 0 || xx >= X || yy < 0 || yy >= Y || zz < 0 || zz >= Z) continue;
          out->tail[k] = (int32_t)p;
          out->head[k] = (int32_t)(((int64_t)zz * Y + yy) * X + xx);
          out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)p * 6 + d), clo, chi);
          k++;
        }
      }
  for (int64_t p = 0; p < face; p++) {
    out->tail[k] = out->s;
    out->head[k] = (int32_t)p;
    out->cap[k] = tcap;
    k++;
  }
  for (int64_t p = np - face; p < np; p++) {
    out->tail[k] = (int32_t)p;
    out->head[k] = out->t;
    out->cap[k] = tcap;
    k++;
  }
  out->m = k;
  return 0;
}

/* LSD radix sort of 64-bit keys (used for R-MAT de-duplication). */
static int radix_sort_u64(uint64_t *a, int64_t n, int key_bits) {
  uint64_t *tmp = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
  if (!tmp) return -1;
  int64_t cnt[1 << 11];
  uint64_t *src = a, *dst = tmp;
  for (int shift = 0; shift < key_bits; shift += 11) {
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < n; i++) cnt[(src[i] >> shift) & 2047]++;
    int64_t sum = 0;
    for (int b = 0; b < 2048; b++) {
      int64_t c = cnt[b];
      cnt[b] = sum;
      sum += c;
    }
    for (int64_t i = 0; i < n; i++) dst[cnt[(src[i] >> shift) & 2047]++] = src[i];
    uint64_t *sw = src;
    src = dst;
    dst = sw;
  }
  if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
  free(tmp);
  return 0;
}

/*
 * R-MAT power-law graph (Chakrabarti, Zhan and Faloutsos 2004) with 2^scale
 * vertices and edge_factor * 2^scale draws. Each draw descends `scale` levels;
 * at each level the quadrant is picked with probabilities (pa, pb, pc, pd)
 * given in hundredths (a digit of a base-100 expansion of 64-bit draws, so the
 * choice is exact integer arithmetic). Quadrant b sets the head bit, c the
 * tail bit, d both. No noise. Self-loops and duplicate (tail, head) pairs are
 * dropped; arcs come out sorted by (tail, head) and arc k gets capacity
 * U[clo,chi] from draw k. s = the vertex of largest out-degree, t = the vertex
 * of largest in-degree among the others (lowest id on ties).
 */
int mfg_rmat(int32_t scale, int32_t edge_factor, uint64_t seed, int32_t pa, int32_t pb, int32_t pc,
             int32_t clo, int32_t chi, mfg_arcs *out) {
  if (scale < 2 || scale > 30 || edge_factor < 1) return -1;
  if (pa < 0 || pb < 0 || pc < 0 || pa + pb + pc > 100) return -1;
  int64_t nv = 1LL << scale;
  int64_t nd = nv * edge_factor;
  memset(out, 0, sizeof(*out));
  uint64_t *keys = (uint64_t *)malloc((size_t)nd * sizeof(uint64_t));
  if (!keys) return -2;
  uint64_t ke = stream_key(seed, 1);
  int per_draw = 9; /* base-100 digits taken from one 64-bit draw (100^9 < 2^64) */
  int nper = (scale + per_draw - 1) / per_draw;
  const int tab = pa + pb, tabc = pa + pb + pc;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nd; i++) {
    uint64_t u = 0, v = 0;
    int lvl = 0;
    for (int j = 0; j < nper && lvl < scale; j++) {
      uint64_t x = draw(ke, (uint64_t)i * nper + j);
      for (int q = 0; q < per_draw && lvl < scale; q++, lvl++) {
        uint64_t x100 = x / 100;
        int dgt = (int)(x - x100 * 100);
        x = x100;
        /* quadrant a: (0,0); b: head bit; c: tail bit; d: both */
        uint64_t ub = (uint64_t)(dgt >= tab);
        uint64_t vb = (uint64_t)((dgt >= pa) & (dgt < tab)) | (uint64_t)(dgt >= tabc);
        u = (u << 1) | ub;
        v = (v << 1) | vb;
      }
    }
    keys[i] = (u << scale) | v;
  }
  if (radix_sort_u64(keys, nd, 2 * scale)) {
    free(keys);
    return -2;
  }
  int64_t m = 0;
  uint64_t mask = (uint64_t)nv - 1;
  for (int64_t i = 0; i < nd; i++) {
    uint64_t kk = keys[i];
    if (((kk >> scale) & mask) == (kk & mask)) continue;
    if (m > 0 && keys[m - 1] == kk) continue;
    keys[m++] = kk;
  }
  if (alloc_arcs(out, m)) {
    free(keys);
    return -2;
  }
  int64_t *od = (int64_t *)calloc((size_t)nv, sizeof(int64_t));
  int64_t *id = (int64_t *)calloc((size_t)nv, sizeof(int64_t));
  if (!od || !id) {
    free(keys);
    free(od);
    free(id);
    mfg_free(out);
    return -2;
  }
  uint64_t kc = stream_key(seed, 2);
  for (int64_t k = 0; k < m; k++) {
    int32_t u = (int32_t)((keys[k] >> scale) & mask), v = (int32_t)(keys[k] & mask);
    out->tail[k] = u;
    out->head[k] = v;
    out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)k), clo, chi);
    od[u]++;
    id[v]++;
  }
  int64_t s = 0, t = -1;
  for (int64_t v = 1; v < nv; v++)
    if (od[v] > od[s]) s = v;
  for (int64_t v = 0; v < nv; v++) {
    if (v == s) continue;
    if (t < 0 || id[v] > id[t]) t = v;
  }
  out->n = (int32_t)nv;
  out->s = (int32_t)s;
  out->t = (int32_t)t;
  free(keys);
  free(od);
  free(id);
  return 0;
}

/*
 * Layered random graph (the rlg family): L layers of W vertices. Vertex
 * (l, j) = l*W + j; s = L*W, t = L*W + 1. Every vertex of a layer l < L-1 has
 * 4 arcs to uniformly drawn vertices of layer l+1 (repeats kept); every vertex
 * has 1 arc to a uniformly drawn other vertex of its own layer (none when
 * W = 1). Capacities U[clo,chi]. s -> every vertex of layer 0 and every vertex
 * of layer L-1 -> t at capacity tcap.
 */
int mfg_layered(int32_t L, int32_t W, uint64_t seed, int32_t clo, int32_t chi, int32_t tcap, mfg_arcs *out) {
  if (L < 2 || W < 1) return -1;
  int64_t np = (int64_t)L * W;
  if (np > 2000000000LL) return -1;
  int64_t m = 4LL * (L - 1) * W + (W > 1 ? np : 0) + 2LL * W;
  memset(out, 0, sizeof(*out));
  if (alloc_arcs(out, m)) return -2;
  out->n = (int32_t)(np + 2);
  out->s = (int32_t)np;
  out->t = (int32_t)np + 1;
  uint64_t kh = stream_key(seed, 1), kc = stream_key(seed, 2);
  int64_t k = 0;
  for (int64_t p = 0; p < np; p++) {
    int64_t l = p / W, j = p % W;
    if (l < L - 1)
      for (int r = 0; r < 4; r++) {
        out->tail[k] = (int32_t)p;
        out->head[k] = (int32_t)((l + 1) * W + unif(draw(kh, (uint64_t)p * 5 + r), 0, W - 1));
        out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)p * 5 + r), clo, chi);
        k++;
      }
    if (W > 1) {
      int64_t q = unif(draw(kh, (uint64_t)p * 5 + 4), 0, W - 2);
      if (q >= j) q++;
      out->tail[k] = (int32_t)p;
      out->head[k] = (int32_t)(l * W + q);
      out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)p * 5 + 4), clo, chi);
      k++;
    }
  }
  for (int64_t j = 0; j < W; j++) {
    out->tail[k] = out->s;
    out->head[k] = (int32_t)j;
    out->cap[k] = tcap;
    k++;
  }
  for (int64_t j = 0; j < W; j++) {
    out->tail[k] = (int32_t)((int64_t)(L - 1) * W + j);
    out->head[k] = out->t;
    out->cap[k] = tcap;
    k++;
  }
  out->m = k;
  return 0;
}

/*
 * Multi-frame grid (video-style): F frames of a side x side 4-connected grid,
 * pixel (f, y, x) = (f*side + y)*side + x; s = F*side^2, t = s + 1. In-frame
 * neighbour arcs as in mfg_grid2d with capacity U[nlo,nhi]; pixel p of frame
 * f < F-1 has an arc to pixel perm_f(p) of frame f+1 (perm_f a uniform random
 * permutation, Fisher-Yates) with capacity U[flo,fhi]; terminal arcs by the
 * 2D-grid rule (s->p or p->t with probability 1/2 each, capacity U[tlo,thi]).
 */
int mfg_multiframe(int32_t F, int32_t side, uint64_t seed, int32_t nlo, int32_t nhi, int32_t flo, int32_t fhi,
                   int32_t tlo, int32_t thi, mfg_arcs *out) {
  if (F < 1 || side < 1) return -1;
  int64_t fp = (int64_t)side * side, np = fp * F;
  if (np > 2000000000LL) return -1;
  int64_t mg = (2LL * side * (side - 1) * 2) * F + fp * (F - 1) + np;
  memset(out, 0, sizeof(*out));
  if (alloc_arcs(out, mg)) return -2;
  out->n = (int32_t)(np + 2);
  out->s = (int32_t)np;
  out->t = (int32_t)np + 1;
  uint64_t kc = stream_key(seed, 1), kt = stream_key(seed, 2), kp = stream_key(seed, 3), kf = stream_key(seed, 4);
  int32_t *perm = (int32_t *)malloc((size_t)fp * sizeof(int32_t));
  if (!perm) {
    mfg_free(out);
    return -2;
  }
  int64_t k = 0;
  for (int32_t f = 0; f < F; f++) {
    for (int32_t y = 0; y < side; y++)
      for (int32_t x = 0; x < side; x++) {
        int64_t p = ((int64_t)f * side + y) * side + x;
        const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
        for (int d = 0; d < 4; d++) {
          int32_t xx = x + dx[d], yy = y + dy[d];
          if (xx < 0 || xx >= side || yy < 0 || yy >= side) continue;
          out->tail[k] = (int32_t)p;
          out->head[k] = (int32_t)(((int64_t)f * side + yy) * side + xx);
          out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)p * 4 + d), nlo, nhi);
          k++;
        }
      }
    if (f + 1 < F) {
      for (int64_t i = 0; i < fp; i++) perm[i] = (int32_t)i;
      for (int64_t i = fp - 1; i > 0; i--) {
        int64_t j = unif(draw(kp, (uint64_t)f * (uint64_t)fp + (uint64_t)i), 0, i);
        int32_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
      }
      for (int64_t i = 0; i < fp; i++) {
        int64_t p = (int64_t)f * fp + i;
        out->tail[k] = (int32_t)p;
        out->head[k] = (int32_t)((int64_t)(f + 1) * fp + perm[i]);
        out->cap[k] = (int32_t)unif(draw(kf, (uint64_t)p), flo, fhi);
        k++;
      }
    }
  }
  free(perm);
  for (int64_t p = 0; p < np; p++) {
    int src = (draw(kt, 2 * (uint64_t)p) >> 63) != 0;
    int32_t c = (int32_t)unif(draw(kt, 2 * (uint64_t)p + 1), tlo, thi);
    out->tail[k] = src ? out->s : (int32_t)p;
    out->head[k] = src ? (int32_t)p : out->t;
    out->cap[k] = c;
    k++;
  }
  out->m = k;
  return 0;
}

/*
 * Uniform random directed multigraph for tests: m arcs with tail and head
 * uniform over 0..n-1 (self-loops redrawn unless allow_loops), capacities
 * U[clo,chi]; s = 0, t = n-1. With dense != 0 and m = 0 every ordered pair
 * (u,v), u != v, gets an arc with probability 1/2 instead.
 */
int mfg_random(int32_t n, int64_t m, uint64_t seed, int32_t clo, int32_t chi, int32_t allow_loops, mfg_arcs *out) {
  if (n < 2 || m < 0) return -1;
  memset(out, 0, sizeof(*out));
  if (alloc_arcs(out, m)) return -2;
  out->n = n;
  out->s = 0;
  out->t = n - 1;
  uint64_t ka = stream_key(seed, 1), kc = stream_key(seed, 2);
  for (int64_t k = 0; k < m; k++) {
    uint64_t j = 0;
    int32_t u, v;
    do {
      u = (int32_t)unif(draw(ka, (uint64_t)k * 64 + 2 * j), 0, n - 1);
      v = (int32_t)unif(draw(ka, (uint64_t)k * 64 + 2 * j + 1), 0, n - 1);
      j++;
    } while (!allow_loops && u == v && j < 32);
    if (!allow_loops && u == v) v = (u + 1) % n;
    out->tail[k] = u;
    out->head[k] = v;
    out->cap[k] = (int32_t)unif(draw(kc, (uint64_t)k), clo, chi);
  }
  return 0;
}
