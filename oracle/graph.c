/*
 * Oracle: the p-computer on general sparse graphs.  TEST INFRASTRUCTURE
 * ONLY (see oracle.h).
 *
 * Algorithms S1 and S2 take weights, biases and a colormap.  Graph colouring
 * (Methods, "Graph Coloring of 3D Cubic Spin Glass Instances") partitions the
 * p-bits into independent sets that are updated in parallel; the paper
 * colours with DSATUR (Brelaz 1979), needs 2 to 4 colours for lattices with
 * missing spins or embeddings, and one more colour for the replicated DT-SQA
 * network when the number of replicas is odd.  This file restates that on
 * an arbitrary graph in CSR form: DSATUR, the graph-coloured Gibbs sweep
 * (Eqs. synapse and neuron), the energy (Eq. ising_energy), APT with replica
 * exchange, ICM and minimum-energy tracking (Algorithm S2) and DT-SQA on the
 * replicated network (Eq. S.3, Algorithm S1).  The randomness contract is in
 * oracle.h.
 */
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"
#include "oracle_internal.h"

#define G_MAX_COLOURS 32

/* ---------------- graph checks and DSATUR ---------------- */

static int find_edge(const int32_t *rp, const int32_t *col, int v, int u) {
  for (int q = rp[v]; q < rp[v + 1]; ++q)
    if (col[q] == u) return q;
  return -1;
}

int or_graph_check(int n, const int32_t *rp, const int32_t *col, const int8_t *w) {
  if (n < 1 || !rp || rp[0] != 0) return -1;
  for (int v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) return -1;
  for (int v = 0; v < n; ++v)
    for (int q = rp[v]; q < rp[v + 1]; ++q) {
      int u = col[q];
      if (u < 0 || u >= n || u == v) return -1;
      if (w && w[q] == 0) return -1;
      for (int q2 = rp[v]; q2 < q; ++q2)
        if (col[q2] == u) return -1;   /* repeated neighbour */
      int back = find_edge(rp, col, u, v);
      if (back < 0) return -1;         /* not symmetric */
      if (w && w[back] != w[q]) return -1;
    }
  return 0;
}

/* Number of distinct colours among the coloured neighbours of v: a
 * neighbour counts when no earlier neighbour has its colour. */
static int saturation(const int32_t *rp, const int32_t *col, const int32_t *colour, int v) {
  int s = 0;
  for (int q = rp[v]; q < rp[v + 1]; ++q) {
    int c = colour[col[q]];
    if (c < 0) continue;
    int first = 1;
    for (int q2 = rp[v]; q2 < q && first; ++q2) first = colour[col[q2]] != c;
    s += first;
  }
  return s;
}

int or_dsatur(int n, const int32_t *rp, const int32_t *col, int32_t *colour, int *n_colours) {
  if (or_graph_check(n, rp, col, NULL)) return -1;
  for (int v = 0; v < n; ++v) colour[v] = -1;
  int C = 0;
  for (int step = 0; step < n; ++step) {
    int best = -1, bs = -1, bd = -1;
    for (int v = 0; v < n; ++v) {
      if (colour[v] >= 0) continue;
      int s = saturation(rp, col, colour, v);
      int d = 0;   /* degree in the uncoloured subgraph */
      for (int q = rp[v]; q < rp[v + 1]; ++q) d += colour[col[q]] < 0;
      if (s > bs || (s == bs && d > bd)) { best = v; bs = s; bd = d; }
    }
    /* the smallest colour that no neighbour of `best` has */
    int c = 0;
    for (;; ++c) {
      int used = 0;
      for (int q = rp[best]; q < rp[best + 1] && !used; ++q) used = colour[col[q]] == c;
      if (!used) break;
    }
    colour[best] = c;
    if (c + 1 > C) C = c + 1;
  }
  if (C > G_MAX_COLOURS) return -1;
  if (n_colours) *n_colours = C;
  return 0;
}

static int colour_count(int n, const int32_t *rp, const int32_t *col, const int32_t *colour) {
  int C = 0;
  for (int v = 0; v < n; ++v) {
    if (colour[v] < 0 || colour[v] >= G_MAX_COLOURS) return -1;
    if (colour[v] + 1 > C) C = colour[v] + 1;
    for (int q = rp[v]; q < rp[v + 1]; ++q)
      if (colour[col[q]] == colour[v]) return -1;   /* not a proper colouring */
  }
  return C;
}

/* Replicated network of Algorithm S1: slice k of v takes
 * (colour[v] + f(k)) mod C' with f(k) = k & 1, and f(P-1) = 2 for odd P.
 * Neighbouring slices differ in f by 1 or 2 (mod C' >= 3 for odd P), and
 * within a slice the shift keeps the base colouring proper. */
static int sqa_colour_of(int c, int k, int P, int Cp) {
  int f = (P & 1) && k == P - 1 ? 2 : (k & 1);
  return (c + f) % Cp;
}

int or_graph_sqa_colouring(int n, const int32_t *colour, int P, int32_t *out, int *n_colours) {
  if (n < 1 || P < 2) return -1;
  int C = 0;
  for (int v = 0; v < n; ++v) {
    if (colour[v] < 0 || colour[v] >= G_MAX_COLOURS) return -1;
    if (colour[v] + 1 > C) C = colour[v] + 1;
  }
  int Cp = C > ((P & 1) ? 3 : 2) ? C : ((P & 1) ? 3 : 2);
  for (int k = 0; k < P; ++k)
    for (int v = 0; v < n; ++v) out[(size_t)k * n + v] = sqa_colour_of(colour[v], k, P, Cp);
  if (n_colours) *n_colours = Cp;
  return 0;
}

/* ---------------- field and energy ---------------- */

/* Eq. synapse on a graph: I_v = h_v + sum_u w_vu s_u. */
static int64_t g_field(const int32_t *rp, const int32_t *col, const int8_t *w, const int8_t *h,
                       const int8_t *s, int v) {
  int64_t I = h ? h[v] : 0;
  for (int q = rp[v]; q < rp[v + 1]; ++q) I += (int64_t)w[q] * s[col[q]];
  return I;
}

static int64_t g_energy(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                        const int8_t *h, const int8_t *s) {
  int64_t E = 0;
  for (int v = 0; v < n; ++v) {
    for (int q = rp[v]; q < rp[v + 1]; ++q)
      if (col[q] > v) E -= (int64_t)w[q] * s[v] * s[col[q]];
    if (h) E -= (int64_t)h[v] * s[v];
  }
  return E;
}

int or_graph_energy(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                    const int8_t *h, const int8_t *spin, int64_t *E_out) {
  if (or_graph_check(n, rp, col, w)) return -1;
  *E_out = g_energy(n, rp, col, w, h, spin);
  return 0;
}

static int64_t g_field_bound(int n, const int32_t *rp, const int8_t *w, const int8_t *h) {
  int64_t m = 0;
  for (int v = 0; v < n; ++v) {
    int64_t s = h ? llabs((long long)h[v]) : 0;
    for (int q = rp[v]; q < rp[v + 1]; ++q) s += llabs((long long)w[q]);
    if (s > m) m = s;
  }
  return m;
}

/* Colour-local indices: j(v) = #{u < v : colour[u] = colour[v]}. */
static void colour_local(int n, const int32_t *colour, int32_t *j) {
  int cnt[G_MAX_COLOURS] = {0};
  for (int v = 0; v < n; ++v) j[v] = cnt[colour[v]]++;
}

/* ---------------- APT on graphs ---------------- */
typedef struct {
  int n, C;
  int32_t *rp, *col, *colour, *cidx;
  int8_t *w, *h;            /* h NULL when every bias is 0 */
  int T, A, B;
  double *beta;
  int64_t Imax;
  uint32_t **tab;           /* [T][2 Imax + 1] */
  int32_t *rid;             /* per slot b = r*A + a: 32 a + r */
  int8_t *spin, *tmp;       /* [B][n], [n] */
  int64_t *E;
  uint32_t ent;
  int64_t best_E, best_sweep, hit_sweep, target;
  int32_t best_buf;
  int8_t *best_spin;
  int64_t *att, *acc;
  int64_t icm[3];
  int32_t *queue;
  uint8_t *inC;
} g_entry;

struct or_gapt {
  int n;
  g_entry *e;
  uint64_t seed;
  int joint;
  int64_t sweeps_done, swaps_done;
};

static void g_entry_free(g_entry *e) {
  if (e->tab)
    for (int t = 0; t < e->T; ++t) free(e->tab[t]);
  free(e->tab);
  free(e->rp); free(e->col); free(e->colour); free(e->cidx); free(e->w); free(e->h);
  free(e->beta); free(e->rid); free(e->spin); free(e->tmp); free(e->E); free(e->best_spin);
  free(e->att); free(e->acc); free(e->queue); free(e->inC);
}

void or_gapt_destroy(or_gapt *g) {
  if (!g) return;
  for (int i = 0; i < g->n; ++i) g_entry_free(&g->e[i]);
  free(g->e);
  free(g);
}

/* Random initial state of slot b (Algorithm S2): +1 iff the init half-word
 * is below 2^15. */
static void g_init_slot(const g_entry *e, int b, uint64_t seed) {
  for (int v = 0; v < e->n; ++v) {
    const int j = e->cidx[v];
    uint32_t ctr[4] = {(uint32_t)j, 0u,
                       ((uint32_t)e->colour[v] << 16) | (uint32_t)(e->rid[b] >> 3),
                       (e->ent << 8) | OR_TAG_G_INIT};
    uint32_t x[4];
    or_philox(ctr, seed, x);
    e->spin[(size_t)b * e->n + v] = (or_half(x, e->rid[b] & 7) < 0x8000u) ? 1 : -1;
  }
}

/* One sweep in the order of the colormap: every vertex of colour 0 in every
 * slot, then colour 1, ...; each update solves Eq. synapse for I_v and
 * Eq. neuron through the threshold of the slot's temperature. */
static void g_sweep(g_entry *e, uint64_t seed, uint32_t s) {
  for (int c = 0; c < e->C; ++c)
    for (int b = 0; b < e->B; ++b) {
      int8_t *sb = e->spin + (size_t)b * e->n;
      const uint32_t *T = e->tab[b / e->A];
      for (int v = 0; v < e->n; ++v) {
        if (e->colour[v] != c) continue;
        int64_t I = g_field(e->rp, e->col, e->w, e->h, sb, v);
        const int j = e->cidx[v];
        uint32_t u = or_uniform32(seed, (uint32_t)j, s,
                                  ((uint32_t)c << 16) | (uint32_t)(e->rid[b] >> 3), e->ent,
                                  OR_TAG_G_SWEEP, OR_TAG_G_REFINE, e->rid[b] & 7);
        sb[v] = (u < T[I + e->Imax]) ? 1 : -1;
      }
    }
}

int or_gapt_create(or_gapt **out, int n_prob, const int32_t *n_vert, const int32_t *rp,
                   const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
                   const int32_t *n_temps, const double *betas, int n_labels, uint64_t seed,
                   uint32_t entry0) {
  *out = NULL;
  if (n_prob < 1 || !(n_labels == 1 || n_labels == 2 || n_labels == 4)) return -1;
  or_gapt *g = (or_gapt *)calloc(1, sizeof(or_gapt));
  if (!g) return -2;
  g->n = n_prob;
  g->seed = seed;
  g->e = (g_entry *)calloc((size_t)n_prob, sizeof(g_entry));
  if (!g->e) { free(g); return -2; }
  size_t voff = 0, eoff = 0, roff = 0, boff = 0;
  for (int i = 0; i < n_prob; ++i) {
    g_entry *e = &g->e[i];
    const int n = n_vert[i];
    const int32_t *rpi = rp + roff;
    if (n < 1 || or_graph_check(n, rpi, col + eoff, w + eoff)) { or_gapt_destroy(g); return -1; }
    const int m = rpi[n];
    e->n = n;
    e->rp = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    memcpy(e->rp, rpi, sizeof(int32_t) * (n + 1));
    e->col = (int32_t *)malloc(sizeof(int32_t) * (m ? m : 1));
    e->w = (int8_t *)malloc((size_t)(m ? m : 1));
    memcpy(e->col, col + eoff, sizeof(int32_t) * m);
    memcpy(e->w, w + eoff, (size_t)m);
    if (h) {
      int any = 0;
      for (int v = 0; v < n; ++v) any |= h[voff + v] != 0;
      if (any) {
        e->h = (int8_t *)malloc((size_t)n);
        memcpy(e->h, h + voff, (size_t)n);
      }
    }
    e->colour = (int32_t *)malloc(sizeof(int32_t) * n);
    if (colour) {
      memcpy(e->colour, colour + voff, sizeof(int32_t) * n);
      e->C = colour_count(n, e->rp, e->col, e->colour);
    } else if (or_dsatur(n, e->rp, e->col, e->colour, &e->C)) {
      e->C = -1;
    }
    if (e->C < 1) { or_gapt_destroy(g); return -1; }
    e->cidx = (int32_t *)malloc(sizeof(int32_t) * n);
    colour_local(n, e->colour, e->cidx);
    e->T = n_temps[i];
    e->A = n_labels;
    e->B = e->T * e->A;
    if (e->T < 1 || e->T > 32) { or_gapt_destroy(g); return -1; }
    e->ent = entry0 + (uint32_t)i;
    e->beta = (double *)malloc(sizeof(double) * e->T);
    memcpy(e->beta, betas + boff, sizeof(double) * e->T);
    for (int t = 1; t < e->T; ++t)
      if (!(e->beta[t] > e->beta[t - 1])) { or_gapt_destroy(g); return -1; }
    e->Imax = g_field_bound(n, e->rp, e->w, e->h);
    e->tab = (uint32_t **)calloc((size_t)e->T, sizeof(uint32_t *));
    for (int t = 0; t < e->T; ++t) {
      e->tab[t] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(2 * e->Imax + 1));
      for (int64_t I = -e->Imax; I <= e->Imax; ++I)
        e->tab[t][I + e->Imax] = or_pbit_threshold(e->beta[t], I);
    }
    e->rid = (int32_t *)malloc(sizeof(int32_t) * e->B);
    for (int b = 0; b < e->B; ++b) e->rid[b] = 32 * (b % e->A) + b / e->A;
    e->spin = (int8_t *)malloc((size_t)e->B * n);
    e->tmp = (int8_t *)malloc((size_t)n);
    e->E = (int64_t *)malloc(sizeof(int64_t) * e->B);
    e->best_spin = (int8_t *)calloc((size_t)n, 1);
    e->att = (int64_t *)calloc((size_t)(e->T > 1 ? e->T - 1 : 1) * e->A, sizeof(int64_t));
    e->acc = (int64_t *)calloc((size_t)(e->T > 1 ? e->T - 1 : 1) * e->A, sizeof(int64_t));
    e->queue = (int32_t *)malloc(sizeof(int32_t) * n);
    e->inC = (uint8_t *)malloc((size_t)n);
    e->best_E = INT64_MAX;
    e->best_sweep = -1;
    e->best_buf = -1;
    e->hit_sweep = -1;
    e->target = INT64_MIN;
    for (int b = 0; b < e->B; ++b) {
      g_init_slot(e, b, seed);
      e->E[b] = g_energy(n, e->rp, e->col, e->w, e->h, e->spin + (size_t)b * n);
    }
    voff += (size_t)n;
    eoff += (size_t)m;
    roff += (size_t)n + 1;
    boff += (size_t)e->T;
  }
  *out = g;
  return 0;
}

/* Minimum-energy tracking as in the lattice path: lowest slot on ties,
 * strict improvement only. */
static void g_best_update(g_entry *e, int64_t sweeps) {
  int bmin = 0;
  for (int b = 1; b < e->B; ++b)
    if (e->E[b] < e->E[bmin]) bmin = b;
  if (e->E[bmin] < e->best_E) {
    e->best_E = e->E[bmin];
    e->best_sweep = sweeps;
    e->best_buf = bmin;
    memcpy(e->best_spin, e->spin + (size_t)bmin * e->n, (size_t)e->n);
  }
  if (e->hit_sweep < 0 && e->best_E <= e->target) e->hit_sweep = sweeps;
}

/* ICMop (Algorithm S2) on two configurations; x = the pair's Philox block.
 * The k-th vertex with q = s^a s^b = -1 in canonical order (colour 0 by
 * increasing v, then colour 1, ...), k = floor(x0 n_minus / 2^32), seeds the
 * cluster = its connected component of {q = -1} in the graph.  A cluster of
 * more than half of the n spins flips one whole replica (x1 bit 0: 0 -> a);
 * otherwise the cluster flips in both replicas.  With h = 0 either move keeps
 * E_a + E_b.  Returns 0 (no mismatch), 1 (cluster) or 2 (whole replica). */
static int g_icm_core(int n, const int32_t *rp, const int32_t *col, const int32_t *colour, int C,
                      int8_t *sa, int8_t *sb, const uint32_t x[4], int32_t *queue, uint8_t *inC,
                      int64_t *size_out) {
  int64_t nminus = 0;
  for (int v = 0; v < n; ++v) nminus += sa[v] != sb[v];
  *size_out = 0;
  if (nminus == 0) return 0;
  int64_t k = (int64_t)(((uint64_t)x[0] * (uint64_t)nminus) >> 32);
  int seed_v = -1;
  int64_t cnt = 0;
  for (int c = 0; c < C && seed_v < 0; ++c)
    for (int v = 0; v < n; ++v) {
      if (colour[v] != c || sa[v] == sb[v]) continue;
      if (cnt == k) { seed_v = v; break; }
      ++cnt;
    }
  memset(inC, 0, (size_t)n);
  int head = 0, tail = 0;
  queue[tail++] = seed_v;
  inC[seed_v] = 1;
  while (head < tail) {
    int v = queue[head++];
    for (int q = rp[v]; q < rp[v + 1]; ++q) {
      int u = col[q];
      if (inC[u] || sa[u] == sb[u]) continue;
      inC[u] = 1;
      queue[tail++] = u;
    }
  }
  *size_out = tail;
  if (2 * (int64_t)tail > (int64_t)n) {
    int8_t *sf = (x[1] & 1u) ? sb : sa;
    for (int v = 0; v < n; ++v) sf[v] = (int8_t)-sf[v];
    return 2;
  }
  for (int q = 0; q < tail; ++q) {
    int v = queue[q];
    sa[v] = (int8_t)-sa[v];
    sb[v] = (int8_t)-sb[v];
  }
  return 1;
}

/* ICMop on slots (ba, bb) of temperature r at attempt t, pair p. */
static void g_icm_op(g_entry *e, uint64_t seed, int ba, int bb, uint32_t r, uint32_t t, uint32_t p) {
  const int n = e->n;
  int8_t *sa = e->spin + (size_t)ba * n, *sb = e->spin + (size_t)bb * n;
  uint32_t ctr[4] = {r, t, p, (e->ent << 8) | OR_TAG_G_ICM}, x[4];
  or_philox(ctr, seed, x);
  int64_t size;
  int br = g_icm_core(n, e->rp, e->col, e->colour, e->C, sa, sb, x, e->queue, e->inC, &size);
  e->icm[br]++;
  if (br == 0) return;
  e->E[ba] = g_energy(n, e->rp, e->col, e->w, e->h, sa);
  e->E[bb] = g_energy(n, e->rp, e->col, e->w, e->h, sb);
}

int or_gicm_apply(int n, const int32_t *rp, const int32_t *col, const int32_t *colour, int8_t *sa,
                  int8_t *sb, uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, uint32_t p,
                  int64_t *cluster_size) {
  if (or_graph_check(n, rp, col, NULL)) return -1;
  int C = colour_count(n, rp, col, colour);
  if (C < 1) return -1;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * n);
  uint8_t *inC = (uint8_t *)malloc((size_t)n);
  uint32_t ctr[4] = {r, t, p, (entry << 8) | OR_TAG_G_ICM}, x[4];
  or_philox(ctr, seed, x);
  int br = g_icm_core(n, rp, col, colour, C, sa, sb, x, queue, inC, cluster_size);
  free(queue);
  free(inC);
  return br;
}

/* Pairs of labels at temperature r: (0,1) with two labels; with four, the
 * matching m = floor(3 x2 / 2^32) of pair 0's ICM block picks
 * (0,1)(2,3), (0,2)(1,3) or (0,3)(1,2). */
static void g_icm_matching(const g_entry *e, uint64_t seed, uint32_t r, uint32_t t, int q[4]) {
  static const int M[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
  int m = 0;
  if (e->A == 4) {
    uint32_t ctr[4] = {r, t, 0u, (e->ent << 8) | OR_TAG_G_ICM}, x[4];
    or_philox(ctr, seed, x);
    m = (int)(((uint64_t)x[2] * 3u) >> 32);
  }
  for (int i = 0; i < 4; ++i) q[i] = M[m][i];
}

static void g_swap_states(g_entry *e, int sA, int sB) {
  const int n = e->n;
  int8_t *pA = e->spin + (size_t)sA * n, *pB = e->spin + (size_t)sB * n;
  memcpy(e->tmp, pA, (size_t)n);
  memcpy(pA, pB, (size_t)n);
  memcpy(pB, e->tmp, (size_t)n);
  int64_t te = e->E[sA];
  e->E[sA] = e->E[sB];
  e->E[sB] = te;
}

/* Replica exchange at attempt t: even t pairs (0,1),(2,3),..., odd t pairs
 * (1,2),(3,4),...; accept with min(1, exp(dbeta dE)), per label or (joint)
 * once per pair with the labels' summed dE. */
static void g_swap_step(g_entry *e, uint64_t seed, uint32_t t, int joint) {
  for (int r = (int)(t & 1u); r + 1 < e->T; r += 2) {
    const double db = e->beta[r + 1] - e->beta[r];
    if (joint) {
      int64_t dE = 0;
      for (int a = 0; a < e->A; ++a) dE += e->E[(r + 1) * e->A + a] - e->E[r * e->A + a];
      uint32_t ctr[4] = {(uint32_t)r, t, 0u, (e->ent << 8) | OR_TAG_G_SWAP}, x[4];
      or_philox(ctr, seed, x);
      int accept = (dE >= 0) || (x[0] < or_swap_threshold(db, dE));
      for (int a = 0; a < e->A; ++a) {
        e->att[r * e->A + a]++;
        if (accept) {
          g_swap_states(e, r * e->A + a, (r + 1) * e->A + a);
          e->acc[r * e->A + a]++;
        }
      }
      continue;
    }
    for (int a = 0; a < e->A; ++a) {
      const int sA = r * e->A + a, sB = (r + 1) * e->A + a;
      int64_t dE = e->E[sB] - e->E[sA];
      uint32_t ctr[4] = {(uint32_t)r, t, (uint32_t)a, (e->ent << 8) | OR_TAG_G_SWAP}, x[4];
      or_philox(ctr, seed, x);
      int accept = (dE >= 0) || (x[0] < or_swap_threshold(db, dE));
      e->att[r * e->A + a]++;
      if (accept) {
        g_swap_states(e, sA, sB);
        e->acc[r * e->A + a]++;
      }
    }
  }
}

/* Algorithm S2 main loop: per attempt, sweeps_per_swap sweeps, energies,
 * best tracking, ICM on every temperature (then best tracking again), the
 * replica exchange. */
int or_gapt_run(or_gapt *g, int64_t n_swaps, int sweeps_per_swap, int icm, int threads) {
  if (!g || n_swaps < 0 || sweeps_per_swap < 1) return -1;
  for (int i = 0; i < g->n; ++i) {
    if (icm && g->e[i].A != 2 && g->e[i].A != 4) return -1;
    if (icm && g->e[i].h) return -1; /* the whole-replica flip needs h = 0 */
  }
  int64_t s0 = g->sweeps_done, t0 = g->swaps_done;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < g->n; ++i) {
    g_entry *e = &g->e[i];
    int64_t s = s0;
    for (int64_t k = 0; k < n_swaps; ++k) {
      uint32_t t = (uint32_t)(t0 + k);
      for (int q = 0; q < sweeps_per_swap; ++q, ++s) g_sweep(e, g->seed, (uint32_t)s);
      for (int b = 0; b < e->B; ++b)
        e->E[b] = g_energy(e->n, e->rp, e->col, e->w, e->h, e->spin + (size_t)b * e->n);
      g_best_update(e, s);
      if (icm) {
        for (int r = 0; r < e->T; ++r) {
          int q[4];
          g_icm_matching(e, g->seed, (uint32_t)r, t, q);
          for (int p = 0; p < e->A / 2; ++p)
            g_icm_op(e, g->seed, r * e->A + q[2 * p], r * e->A + q[2 * p + 1], (uint32_t)r, t,
                     (uint32_t)p);
        }
        g_best_update(e, s);
      }
      g_swap_step(e, g->seed, t, g->joint);
    }
  }
  (void)threads;
  g->sweeps_done += n_swaps * sweeps_per_swap;
  g->swaps_done += n_swaps;
  return 0;
}

int or_gapt_set_joint_swap(or_gapt *g, int joint) {
  if (!g) return -1;
  g->joint = joint != 0;
  return 0;
}

int or_gapt_set_target(or_gapt *g, int prob, int64_t e_target) {
  if (!g || prob < 0 || prob >= g->n) return -1;
  g_entry *e = &g->e[prob];
  e->target = e_target;
  e->hit_sweep = -1;
  if (e->best_E <= e_target) e->hit_sweep = e->best_sweep;
  return 0;
}

int or_gapt_state(const or_gapt *g, int prob, int8_t *spins, int64_t *energies, int32_t *colour) {
  if (!g || prob < 0 || prob >= g->n) return -1;
  const g_entry *e = &g->e[prob];
  if (spins) memcpy(spins, e->spin, (size_t)e->B * e->n);
  if (energies) memcpy(energies, e->E, sizeof(int64_t) * e->B);
  if (colour) memcpy(colour, e->colour, sizeof(int32_t) * e->n);
  return 0;
}

int or_gapt_best(const or_gapt *g, int prob, int64_t *E, int64_t *sweep, int32_t *buf,
                 int64_t *hit_sweep, int8_t *spins) {
  if (!g || prob < 0 || prob >= g->n) return -1;
  const g_entry *e = &g->e[prob];
  if (E) *E = e->best_E;
  if (sweep) *sweep = e->best_sweep;
  if (buf) *buf = e->best_buf;
  if (hit_sweep) *hit_sweep = e->hit_sweep;
  if (spins) memcpy(spins, e->best_spin, (size_t)e->n);
  return 0;
}

int or_gapt_stats(const or_gapt *g, int prob, int64_t *att, int64_t *acc, int64_t *icm) {
  if (!g || prob < 0 || prob >= g->n) return -1;
  const g_entry *e = &g->e[prob];
  size_t np = (size_t)(e->T > 1 ? e->T - 1 : 0) * e->A;
  if (att) memcpy(att, e->att, sizeof(int64_t) * np);
  if (acc) memcpy(acc, e->acc, sizeof(int64_t) * np);
  if (icm) memcpy(icm, e->icm, sizeof(e->icm));
  return 0;
}

/* ---------------- DT-SQA on graphs (Eq. S.3, Algorithm S1) ---------------- */
/* P slices of the graph, each with the full weights and biases; slice k is
 * coupled to slices k-1 and k+1 (periodic) by J_perp at the same vertex.
 * beta_eff = 1/(P T), J_perp in Q16.16 as in the lattice path.  The
 * replicated network is coloured from the colormap (rule in oracle.h) and
 * swept colour by colour. */
static void gsqa_run(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                     const int8_t *h, const int32_t *rcol, int Cp, const int32_t *ridx, int P,
                     double T, int n_sweeps, const double *gamma, uint32_t run, uint64_t seed,
                     int64_t Imax, int64_t *E_out, int8_t *spins_out) {
  int8_t *s = (int8_t *)malloc((size_t)P * n);
  uint32_t *tab = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)(2 * Imax + 1));
  double beta_eff = 1.0 / ((double)P * T);
  for (int k = 0; k < P; ++k)
    for (int v = 0; v < n; ++v) {
      const size_t kv = (size_t)k * n + v;
      const int j = ridx[kv];
      uint32_t ctr[4] = {(uint32_t)j, 0u, (uint32_t)rcol[kv], ((run >> 3) << 8) | OR_TAG_GS_INIT};
      uint32_t x[4];
      or_philox(ctr, seed, x);
      s[kv] = (or_half(x, (int)(run & 7u)) < 0x8000u) ? 1 : -1;
    }
  for (int sw = 0; sw < n_sweeps; ++sw) {
    int32_t jq = or_jperp_q(gamma[sw], P, T);
    for (int nn = 0; nn < 3; ++nn)
      for (int64_t I = -Imax; I <= Imax; ++I)
        tab[(size_t)nn * (2 * Imax + 1) + (I + Imax)] =
            or_sqa_threshold(beta_eff, I, jq, 2 * nn - 2);
    for (int c = 0; c < Cp; ++c)
      for (int k = 0; k < P; ++k) {
        int8_t *sk = s + (size_t)k * n;
        const int8_t *sdn = s + (size_t)((k + P - 1) % P) * n;
        const int8_t *sup = s + (size_t)((k + 1) % P) * n;
        for (int v = 0; v < n; ++v) {
          const size_t kv = (size_t)k * n + v;
          if (rcol[kv] != c) continue;
          int64_t I = g_field(rp, col, w, h, sk, v);
          int nb = sdn[v] + sup[v];
          const int j = ridx[kv];
          uint32_t u = or_uniform32(seed, (uint32_t)j, (uint32_t)sw, (uint32_t)c, run >> 3,
                                    OR_TAG_GS_SWEEP, OR_TAG_GS_REFINE, (int)(run & 7u));
          uint32_t thr = tab[(size_t)((nb + 2) / 2) * (2 * Imax + 1) + (I + Imax)];
          sk[v] = (u < thr) ? 1 : -1;
        }
      }
  }
  for (int k = 0; k < P; ++k) E_out[k] = g_energy(n, rp, col, w, h, s + (size_t)k * n);
  if (spins_out) memcpy(spins_out, s, (size_t)P * n);
  free(s);
  free(tab);
}

int or_gsqa_anneal(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                   const int8_t *h, const int32_t *colour, int P, double T, int n_sweeps,
                   const double *gamma, int R, uint32_t run0, uint64_t seed, int64_t *E_out,
                   int8_t *spins_out, int threads) {
  if (P < 2 || !(T > 0) || n_sweeps < 0 || R < 1) return -1;
  if (or_graph_check(n, rp, col, w)) return -1;
  for (int i = 0; i < n_sweeps; ++i)
    if (!(gamma[i] > 0)) return -1;
  int32_t *base = (int32_t *)malloc(sizeof(int32_t) * n);
  int C = -1;
  if (colour) {
    memcpy(base, colour, sizeof(int32_t) * n);
    C = colour_count(n, rp, col, base);
  } else if (or_dsatur(n, rp, col, base, &C)) {
    C = -1;
  }
  if (C < 1) { free(base); return -1; }
  int32_t *rcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * n);
  int32_t *ridx = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * n);
  int Cp = 0;
  or_graph_sqa_colouring(n, base, P, rcol, &Cp);
  /* class-local index of (v, k): classes ordered by k, then v */
  int cnt[G_MAX_COLOURS] = {0};
  for (int k = 0; k < P; ++k)
    for (int v = 0; v < n; ++v) ridx[(size_t)k * n + v] = cnt[rcol[(size_t)k * n + v]]++;
  int64_t Imax = g_field_bound(n, rp, w, h);
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int r = 0; r < R; ++r)
    gsqa_run(n, rp, col, w, h, rcol, Cp, ridx, P, T, n_sweeps, gamma, run0 + (uint32_t)r, seed,
             Imax, E_out + (size_t)r * P, spins_out ? spins_out + (size_t)r * P * n : NULL);
  (void)threads;
  free(base); free(rcol); free(ridx);
  return 0;
}

/* ---------------- adaptive ladder on graphs ---------------- */
/* Algorithm S2's preprocessing (Methods, "APT details") on a graph: n_chains
 * chains sweep `sweeps` times at beta_t, warm-started from the previous
 * step; sigma_E is the square root of the chains' mean unbiased variance of
 * their last `tail` post-sweep energies; beta_{t+1} = beta_t + alpha /
 * sigma_E; stop at the first beta with sigma_E < tol. */
int or_graph_adaptive_ladder(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                             const int8_t *h, const int32_t *colour, uint32_t entry, uint64_t seed,
                             double beta0, double alpha, int n_chains, int sweeps, int tail,
                             double tol, int max_len, double *beta_out, double *sigma_out,
                             int *len_out) {
  if (n_chains < 1 || n_chains > 128 || sweeps < 1 || tail < 2 || tail > sweeps || max_len < 1 ||
      !(beta0 > 0))
    return -1;
  double b1 = 1.0;
  or_gapt *g = NULL;
  int32_t nv = n, T = 1;
  /* one problem with one "temperature" per chain is built through the APT
     set-up only for its graph checks, colouring and colour-local indices */
  int rc = or_gapt_create(&g, 1, &nv, rp, col, w, h, colour, &T, &b1, 1, seed, entry);
  if (rc) return rc;
  g_entry *e = &g->e[0];
  const int64_t Imax = e->Imax;
  int8_t *spin = (int8_t *)malloc((size_t)n_chains * n);
  int64_t *sE = (int64_t *)malloc(sizeof(int64_t) * n_chains);
  int64_t *sE2 = (int64_t *)malloc(sizeof(int64_t) * n_chains);
  uint32_t *tab = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(2 * Imax + 1));
  for (int b = 0; b < n_chains; ++b)
    for (int v = 0; v < n; ++v) {
      const int j = e->cidx[v];
      uint32_t ctr[4] = {(uint32_t)j, 0u, ((uint32_t)e->colour[v] << 16) | (uint32_t)(b >> 3),
                         (entry << 8) | OR_TAG_GL_INIT};
      uint32_t x[4];
      or_philox(ctr, seed, x);
      spin[(size_t)b * n + v] = (or_half(x, b & 7) < 0x8000u) ? 1 : -1;
    }
  double beta = beta0;
  int len = 0, status = 1;
  uint32_t s = 0;
  while (len < max_len) {
    for (int64_t I = -Imax; I <= Imax; ++I) tab[I + Imax] = or_pbit_threshold(beta, I);
    memset(sE, 0, sizeof(int64_t) * n_chains);
    memset(sE2, 0, sizeof(int64_t) * n_chains);
    for (int k = 0; k < sweeps; ++k, ++s) {
      for (int c = 0; c < e->C; ++c)
        for (int b = 0; b < n_chains; ++b) {
          int8_t *sb = spin + (size_t)b * n;
          for (int v = 0; v < n; ++v) {
            if (e->colour[v] != c) continue;
            int64_t I = g_field(e->rp, e->col, e->w, e->h, sb, v);
            uint32_t u = or_uniform32(seed, (uint32_t)e->cidx[v], s,
                                      ((uint32_t)c << 16) | (uint32_t)(b >> 3), entry,
                                      OR_TAG_GL_SWEEP, OR_TAG_GL_REFINE, b & 7);
            sb[v] = (u < tab[I + Imax]) ? 1 : -1;
          }
        }
      if (k >= sweeps - tail)
        for (int b = 0; b < n_chains; ++b) {
          int64_t E = g_energy(n, e->rp, e->col, e->w, e->h, spin + (size_t)b * n);
          sE[b] += E;
          sE2[b] += E * E;
        }
    }
    double mean_var = 0.0;
    for (int b = 0; b < n_chains; ++b) {
      int64_t num = (int64_t)tail * sE2[b] - sE[b] * sE[b];
      mean_var += (double)num / ((double)tail * (double)(tail - 1));
    }
    mean_var /= (double)n_chains;
    double sigma = sqrt(mean_var);
    beta_out[len] = beta;
    if (sigma_out) sigma_out[len] = sigma;
    ++len;
    if (sigma < tol) { status = 0; break; }
    beta = beta + alpha / sigma;
  }
  *len_out = len;
  free(spin); free(sE); free(sE2); free(tab);
  or_gapt_destroy(g);
  return status;
}
