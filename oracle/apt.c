/*
 * Oracle: p-bit Gibbs sweeps, adaptive parallel tempering with replica
 * exchange and isoenergetic cluster moves, the adaptive beta ladder and the
 * pilot-run histograms.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Replicas live in slots (temperature r, ICM label a), slot index
 * r * A + a.  An accepted swap exchanges the p-bit states of the two slots
 * (Algorithm S2, "swap the p-bit states").  Random numbers are keyed by the
 * slot's replica id  rid(r, a) = a * Tp + r  with Tp = 8 * ceil(T / 8), so
 * the eight replicas of one Philox call are eight temperatures of one label.
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

/* ---------------- shared sampler pieces ---------------- */

/* Threshold table of one temperature over I in [-Imax, Imax]. */
static uint32_t *make_table(double beta, int64_t Imax) {
  uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(2 * Imax + 1));
  if (!t) return NULL;
  for (int64_t I = -Imax; I <= Imax; ++I) t[I + Imax] = or_pbit_threshold(beta, I);
  return t;
}

/* Random initial state (Algorithm S2 "Initialize all replicas to random
 * states"): +1 iff the init half-word is below 2^15. */
static void init_spins(const or_lat *L, int B, const int32_t *rid, int8_t *spin, uint64_t seed,
                       uint32_t ent, uint32_t tag) {
  for (int b = 0; b < B; ++b) {
    const int id = rid ? rid[b] : b;
    for (int lin = 0; lin < L->N; ++lin) {
      int c = or_colour(L, lin);
      uint32_t ctr[4] = {(uint32_t)(lin >> 1), 0u, ((uint32_t)c << 16) | (uint32_t)(id >> 3),
                         (ent << 8) | tag};
      uint32_t x[4];
      or_philox(ctr, seed, x);
      spin[(size_t)b * L->N + lin] = (or_half(x, id & 7) < 0x8000u) ? 1 : -1;
    }
  }
}

/* One Monte Carlo sweep (every spin of every buffer updated once) in the
 * graph-coloured order of Algorithm S2's p-computer: all colour-0 sites,
 * then all colour-1 sites.  Each update solves Eq. synapse for I and
 * Eq. neuron through the threshold of the buffer's temperature. */
static void gibbs_sweep(const or_lat *L, const int8_t *J, const int8_t *h, int64_t Imax,
                        int B, const int32_t *rid, int8_t *spin, const int32_t *temp_of,
                        uint32_t *const *tab, uint64_t seed, uint32_t ent, uint32_t s,
                        uint32_t tag_main, uint32_t tag_ref) {
  for (int c = 0; c < 2; ++c) {
    for (int b = 0; b < B; ++b) {
      int8_t *sb = spin + (size_t)b * L->N;
      const uint32_t *T = tab[temp_of[b]];
      const int id = rid ? rid[b] : b;
      for (int lin = 0; lin < L->N; ++lin) {
        if (or_colour(L, lin) != c) continue;
        int64_t I = or_field(L, J, h, sb, lin);
        uint32_t u = or_uniform32(seed, (uint32_t)(lin >> 1), s,
                                  ((uint32_t)c << 16) | (uint32_t)(id >> 3), ent, tag_main,
                                  tag_ref, id & 7);
        sb[lin] = (u < T[I + Imax]) ? 1 : -1;
      }
    }
  }
}

/* ---------------- APT ---------------- */
typedef struct {
  or_lat L;
  int8_t *J, *h;
  int T, A, B;
  double *beta;
  int64_t Imax;
  uint32_t **tab;
  int32_t *temp_of, *rid;   /* per slot: temperature r, replica id a*Tp + r */
  int8_t *spin;
  int8_t *tmp;
  int64_t *E;
  uint32_t ent;
  int64_t best_E, best_sweep, hit_sweep, target;
  int32_t best_buf;
  int8_t *best_spin;
  int64_t *att, *acc;
  int64_t icm[3];
  int32_t *queue;
  uint8_t *inC;
} apt_entry;

struct or_apt {
  int n;
  apt_entry *e;
  uint64_t seed;
  int joint;   /* 1: one swap decision per temperature pair for all labels */
  int icm_big;  /* 1 (default): the big-cluster branch of ICMop is on */
  int icm_seed; /* 0 (default): uniform mismatch site; 1: uniform cluster */
  int64_t sweeps_done, swaps_done;
};

static void entry_free(apt_entry *e) {
  if (e->tab)
    for (int t = 0; t < e->T; ++t) free(e->tab[t]);
  free(e->tab);
  free(e->J); free(e->h); free(e->beta); free(e->temp_of); free(e->rid); free(e->tmp);
  free(e->spin); free(e->E); free(e->best_spin); free(e->att); free(e->acc);
  free(e->queue); free(e->inC);
  or_lat_free(&e->L);
}

void or_apt_destroy(or_apt *a) {
  if (!a) return;
  for (int i = 0; i < a->n; ++i) entry_free(&a->e[i]);
  free(a->e);
  free(a);
}

int or_apt_create(or_apt **out, int n_inst, const int32_t *dims, const uint8_t *periodic,
                  const uint8_t *present, const int8_t *J, const int8_t *h, const int32_t *n_temps,
                  const double *betas, int n_labels, uint64_t seed, uint32_t entry0) {
  *out = NULL;
  if (n_inst < 1 || !(n_labels == 1 || n_labels == 2 || n_labels == 4)) return -1;
  or_apt *a = (or_apt *)calloc(1, sizeof(or_apt));
  if (!a) return -2;
  a->n = n_inst;
  a->seed = seed;
  a->icm_big = 1;
  a->icm_seed = 0;
  a->e = (apt_entry *)calloc((size_t)n_inst, sizeof(apt_entry));
  if (!a->e) { free(a); return -2; }
  size_t joff = 0, boff = 0;
  for (int i = 0; i < n_inst; ++i) {
    apt_entry *e = &a->e[i];
    int rc = or_lat_init(&e->L, dims + 3 * i, periodic ? periodic + 3 * i : NULL);
    if (!rc) rc = or_lat_set_present(&e->L, present ? present + joff : NULL);
    if (rc) { or_apt_destroy(a); return rc; }
    int N = e->L.N;
    e->T = n_temps[i];
    e->A = n_labels;
    e->B = e->T * e->A;
    if (e->T < 1) { or_apt_destroy(a); return -1; }
    e->ent = entry0 + (uint32_t)i;
    e->J = (int8_t *)malloc((size_t)3 * N);
    memcpy(e->J, J + 3 * joff, (size_t)3 * N);
    if (h) {
      e->h = (int8_t *)malloc((size_t)N);
      memcpy(e->h, h + joff, (size_t)N);
    }
    e->beta = (double *)malloc(sizeof(double) * e->T);
    memcpy(e->beta, betas + boff, sizeof(double) * e->T);
    for (int t = 1; t < e->T; ++t)
      if (!(e->beta[t] > e->beta[t - 1])) { or_apt_destroy(a); return -1; }
    e->Imax = or_field_bound(&e->L, e->J, e->h);
    e->tab = (uint32_t **)calloc((size_t)e->T, sizeof(uint32_t *));
    for (int t = 0; t < e->T; ++t) e->tab[t] = make_table(e->beta[t], e->Imax);
    e->temp_of = (int32_t *)malloc(sizeof(int32_t) * e->B);
    e->rid = (int32_t *)malloc(sizeof(int32_t) * e->B);
    e->tmp = (int8_t *)malloc((size_t)N);
    const int Tp = 8 * ((e->T + 7) / 8);
    for (int b = 0; b < e->B; ++b) {
      e->temp_of[b] = b / e->A;                      /* slot b = (r, a) = (b / A, b % A) */
      e->rid[b] = (b % e->A) * Tp + b / e->A;
    }
    e->spin = (int8_t *)malloc((size_t)e->B * N);
    e->E = (int64_t *)malloc(sizeof(int64_t) * e->B);
    e->best_spin = (int8_t *)calloc((size_t)N, 1);
    e->att = (int64_t *)calloc((size_t)(e->T > 1 ? e->T - 1 : 1) * e->A, sizeof(int64_t));
    e->acc = (int64_t *)calloc((size_t)(e->T > 1 ? e->T - 1 : 1) * e->A, sizeof(int64_t));
    e->queue = (int32_t *)malloc(sizeof(int32_t) * N);
    e->inC = (uint8_t *)malloc((size_t)N);
    e->best_E = INT64_MAX;
    e->best_sweep = -1;
    e->best_buf = -1;
    e->hit_sweep = -1;
    e->target = INT64_MIN;
    init_spins(&e->L, e->B, e->rid, e->spin, seed, e->ent, OR_TAG_APT_INIT);
    for (int b = 0; b < e->B; ++b)
      e->E[b] = or_energy_lat(&e->L, e->J, e->h, e->spin + (size_t)b * N);
    joff += (size_t)N;
    boff += (size_t)e->T;
  }
  *out = a;
  return 0;
}

/* Minimum-energy selection (Algorithm S2 output; the paper keeps the
 * minimum-energy replica at every swap): lowest buffer index on ties, strict
 * improvement only. */
static void best_update(apt_entry *e, int64_t sweeps) {
  int bmin = 0;
  for (int b = 1; b < e->B; ++b)
    if (e->E[b] < e->E[bmin]) bmin = b;
  if (e->E[bmin] < e->best_E) {
    e->best_E = e->E[bmin];
    e->best_sweep = sweeps;
    e->best_buf = bmin;
    memcpy(e->best_spin, e->spin + (size_t)bmin * e->L.N, (size_t)e->L.N);
  }
  if (e->hit_sweep < 0 && e->best_E <= e->target) e->hit_sweep = sweeps;
}

/* Flood of the mismatch component of `seed_site` into queue[0 .. size-1]
 * (breadth first over lattice adjacency); marks inC. */
static int64_t icm_component(const or_lat *L, const int8_t *sa, const int8_t *sb, int seed_site,
                             int32_t *queue, uint8_t *inC) {
  int head = 0, tail = 0;
  queue[tail++] = seed_site;
  inC[seed_site] = 1;
  while (head < tail) {
    int v = queue[head++];
    for (int dir = 0; dir < 6; ++dir) {
      int n = L->nb[6 * v + dir];
      if (n < 0 || inC[n] || sa[n] == sb[n]) continue;
      inC[n] = 1;
      queue[tail++] = n;
    }
  }
  return tail;
}

static int icm_mismatch(const or_lat *L, const int8_t *sa, const int8_t *sb, int lin) {
  return sa[lin] != sb[lin] && !(L->vac && L->vac[lin]);
}

/* Number of choices of the seed rule: the mismatch sites (seed_rule 0) or
 * the mismatch clusters (seed_rule 1). */
static int64_t icm_choices(const or_lat *L, const int8_t *sa, const int8_t *sb, int seed_rule,
                           int32_t *queue, uint8_t *inC) {
  const int N = L->N;
  int64_t n = 0;
  if (seed_rule == 0) {
    for (int lin = 0; lin < N; ++lin) n += icm_mismatch(L, sa, sb, lin);
    return n;
  }
  memset(inC, 0, (size_t)N);
  for (int lin = 0; lin < N; ++lin)
    if (icm_mismatch(L, sa, sb, lin) && !inC[lin]) {
      icm_component(L, sa, sb, lin, queue, inC);
      ++n;
    }
  return n;
}

/* ICMop with the seed choice k in [0, n_choices) given: the seed is the
 * k-th mismatch site in canonical order (colour 0 by increasing lin, then
 * colour 1) under seed_rule 0, or the first site, in that order, of the
 * k-th cluster met in that order under seed_rule 1.  The seed's cluster C
 * is flipped in both replicas; with big_rule set and 2|C| larger than the
 * spins present, one whole replica (flip_b: the second, else the first)
 * is flipped instead.  Returns 1 (cluster) or 2 (whole replica). */
static int icm_apply_choice(const or_lat *L, int8_t *sa, int8_t *sb, int64_t k, int flip_b, int big_rule,
                            int seed_rule, int32_t *queue, uint8_t *inC, int64_t *size_out) {
  const int N = L->N;
  int seed_site = -1;
  int64_t cnt = 0;
  memset(inC, 0, (size_t)N);
  for (int c = 0; c < 2 && seed_site < 0; ++c)
    for (int lin = 0; lin < N; ++lin) {
      if (or_colour(L, lin) != c || !icm_mismatch(L, sa, sb, lin)) continue;
      if (seed_rule == 1) {
        if (inC[lin]) continue;               /* a cluster met before */
        if (cnt == k) { seed_site = lin; break; }
        icm_component(L, sa, sb, lin, queue, inC);
      } else if (cnt == k) {
        seed_site = lin;
        break;
      }
      ++cnt;
    }
  memset(inC, 0, (size_t)N);
  const int64_t size = icm_component(L, sa, sb, seed_site, queue, inC);
  *size_out = size;
  if (big_rule && 2 * size > (int64_t)L->nreal) {   /* more than half of the spins present */
    int8_t *sf = flip_b ? sb : sa;
    for (int lin = 0; lin < N; ++lin) sf[lin] = (int8_t)-sf[lin];
    return 2;
  }
  for (int64_t q = 0; q < size; ++q) {
    int v = queue[q];
    sa[v] = (int8_t)-sa[v];
    sb[v] = (int8_t)-sb[v];
  }
  return 1;
}

/* Core of ICMop on two configurations; x = the pair's Philox block.
 * The choice is k = floor(x0 n / 2^32) of the n choices of the seed rule,
 * and bit 0 of x1 picks the replica of a whole-replica flip.  Returns 0 (no
 * mismatch), 1 (cluster flipped in both) or 2 (one whole replica flipped);
 * *size = cluster size. */
static int icm_core(const or_lat *L, int8_t *sa, int8_t *sb, const uint32_t x[4], int big_rule, int seed_rule,
                    int32_t *queue, uint8_t *inC, int64_t *size_out) {
  *size_out = 0;
  const int64_t n = icm_choices(L, sa, sb, seed_rule, queue, inC);
  if (n == 0) return 0;
  const int64_t k = (int64_t)(((uint64_t)x[0] * (uint64_t)n) >> 32);
  return icm_apply_choice(L, sa, sb, k, (int)(x[1] & 1u), big_rule, seed_rule, queue, inC, size_out);
}

/* ICMop of Algorithm S2 on buffers (ba, bb) at attempt t, temperature r:
 * overlap q_i = s_i^a s_i^b; the seed (a uniform mismatch site, or the
 * first site of a uniform mismatch cluster) starts the cluster = its
 * connected component of {q = -1} on the lattice graph, flipped in both
 * replicas, or, when it holds more than half of all spins and the
 * big-cluster rule is on, one whole replica is flipped instead. */
static void icm_op(apt_entry *e, uint64_t seed, int ba, int bb, uint32_t r, uint32_t t, uint32_t p,
                   int big_rule, int seed_rule) {
  int N = e->L.N;
  int8_t *sa = e->spin + (size_t)ba * N, *sb = e->spin + (size_t)bb * N;
  uint32_t ctr[4] = {r, t, p, (e->ent << 8) | OR_TAG_ICM}, x[4];
  or_philox(ctr, seed, x);
  int64_t size;
  int br = icm_core(&e->L, sa, sb, x, big_rule, seed_rule, e->queue, e->inC, &size);
  e->icm[br]++;
  if (br == 0) return;
  e->E[ba] = or_energy_lat(&e->L, e->J, e->h, sa);
  e->E[bb] = or_energy_lat(&e->L, e->J, e->h, sb);
}

int or_icm_apply(const int32_t dims[3], const uint8_t periodic[3], int8_t *sa, int8_t *sb,
                 uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, uint32_t p,
                 int64_t *cluster_size) {
  return or_icm_apply_rules(dims, periodic, sa, sb, seed, entry, r, t, p, 1, 0, cluster_size);
}

int or_icm_apply_rules(const int32_t dims[3], const uint8_t periodic[3], int8_t *sa, int8_t *sb,
                       uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, uint32_t p, int big_rule,
                       int seed_rule, int64_t *cluster_size) {
  or_lat L;
  int rc = or_lat_init(&L, dims, periodic);
  if (rc) return rc;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * L.N);
  uint8_t *inC = (uint8_t *)malloc((size_t)L.N);
  uint32_t ctr[4] = {r, t, p, (entry << 8) | OR_TAG_ICM}, x[4];
  or_philox(ctr, seed, x);
  int br = icm_core(&L, sa, sb, x, big_rule != 0, seed_rule != 0, queue, inC, cluster_size);
  free(queue); free(inC);
  or_lat_free(&L);
  return br;
}

int or_icm_choice(const int32_t dims[3], const uint8_t periodic[3], int8_t *sa, int8_t *sb, int64_t k,
                  int flip_b, int big_rule, int seed_rule, int64_t *n_choices, int64_t *cluster_size) {
  or_lat L;
  int rc = or_lat_init(&L, dims, periodic);
  if (rc) return rc;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * L.N);
  uint8_t *inC = (uint8_t *)malloc((size_t)L.N);
  const int64_t n = icm_choices(&L, sa, sb, seed_rule != 0, queue, inC);
  *n_choices = n;
  *cluster_size = 0;
  int br = 0;
  if (n > 0 && k >= 0 && k < n)
    br = icm_apply_choice(&L, sa, sb, k, flip_b != 0, big_rule != 0, seed_rule != 0, queue, inC, cluster_size);
  else if (n > 0)
    br = -1;
  free(queue); free(inC);
  or_lat_free(&L);
  return br;
}

/* Random partition of the ICM labels of temperature r into pairs at attempt
 * t (Algorithm S2 "Randomly partition ICM replicas into pairs"; Methods: two
 * randomly chosen pairs per temperature with 4 labels).  Two labels form
 * the one pair (0, 1).  Four labels have three perfect matchings,
 * m = floor(3 x2 / 2^32) with x = the Philox block of pair 0's ICM draw:
 * m = 0: (0,1)(2,3); m = 1: (0,2)(1,3); m = 2: (0,3)(1,2). */
static int icm_matching(uint64_t seed, uint32_t ent, uint32_t r, uint32_t t, int A, int pairs[4]) {
  static const int M[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
  int m = 0;
  if (A == 4) {
    uint32_t ctr[4] = {r, t, 0u, (ent << 8) | OR_TAG_ICM}, x[4];
    or_philox(ctr, seed, x);
    m = (int)(((uint64_t)x[2] * 3u) >> 32);
  }
  for (int q = 0; q < 4; ++q) pairs[q] = M[m][q];
  return m;
}

int or_icm_pairing(uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, int n_labels,
                   int32_t *pairs) {
  if (!pairs || !(n_labels == 2 || n_labels == 4)) return -1;
  int q[4];
  int m = icm_matching(seed, entry, r, t, n_labels, q);
  for (int i = 0; i < (n_labels == 4 ? 4 : 2); ++i) pairs[i] = q[i];
  return m;
}

/* Replica exchange at attempt t (0-based): even t pairs (0,1),(2,3),...
 * (the paper's odd-numbered attempt), odd t pairs (1,2),(3,4),...; within
 * each pair every label decides on its own with
 * p_swap = min(1, exp(dbeta dE)), dE = E_{r+1} - E_r, dbeta = b_{r+1}-b_r. */
static void swap_states(apt_entry *e, int sA, int sB) {
  const int N = e->L.N;
  int8_t *pA = e->spin + (size_t)sA * N, *pB = e->spin + (size_t)sB * N;
  memcpy(e->tmp, pA, (size_t)N);
  memcpy(pA, pB, (size_t)N);
  memcpy(pB, e->tmp, (size_t)N);
  int64_t te = e->E[sA];
  e->E[sA] = e->E[sB];
  e->E[sB] = te;
}

static void swap_step(apt_entry *e, uint64_t seed, uint32_t t, int joint) {
  for (int r = (int)(t & 1u); r + 1 < e->T; r += 2) {
    if (joint) {
      /* Algorithm S2 read literally: one decision swaps all iso-temperature
       * replicas of the pair; the move exchanges A states at once, so its
       * Metropolis ratio is the product exp(dbeta sum_a dE_a) */
      int64_t dE = 0;
      for (int a = 0; a < e->A; ++a) dE += e->E[(r + 1) * e->A + a] - e->E[r * e->A + a];
      uint32_t ctr[4] = {(uint32_t)r, t, 0u, (e->ent << 8) | OR_TAG_SWAP}, x[4];
      or_philox(ctr, seed, x);
      int accept = (dE >= 0) || (x[0] < or_swap_threshold(e->beta[r + 1] - e->beta[r], dE));
      for (int a = 0; a < e->A; ++a) {
        e->att[r * e->A + a]++;
        if (accept) {
          swap_states(e, r * e->A + a, (r + 1) * e->A + a);
          e->acc[r * e->A + a]++;
        }
      }
      continue;
    }
    for (int a = 0; a < e->A; ++a) {
      const int sA = r * e->A + a, sB = (r + 1) * e->A + a;
      int64_t dE = e->E[sB] - e->E[sA];
      uint32_t ctr[4] = {(uint32_t)r, t, (uint32_t)a, (e->ent << 8) | OR_TAG_SWAP}, x[4];
      or_philox(ctr, seed, x);
      int accept = (dE >= 0) || (x[0] < or_swap_threshold(e->beta[r + 1] - e->beta[r], dE));
      e->att[r * e->A + a]++;
      if (accept) {
        /* swap the p-bit states (and energies) of the two replicas */
        swap_states(e, sA, sB);
        e->acc[r * e->A + a]++;
      }
    }
  }
}

int or_apt_run(or_apt *a, int64_t n_swaps, int sweeps_per_swap, int icm, int threads) {
  if (!a || n_swaps < 0 || sweeps_per_swap < 1) return -1;
  for (int i = 0; i < a->n; ++i) {
    if (icm && a->e[i].A != 2 && a->e[i].A != 4) return -1;
    if (icm && a->e[i].h) return -1; /* whole-replica flip needs h = 0 */
  }
  int64_t s0 = a->sweeps_done, t0 = a->swaps_done;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < a->n; ++i) {
    apt_entry *e = &a->e[i];
    int64_t s = s0;
    for (int64_t k = 0; k < n_swaps; ++k) {
      uint32_t t = (uint32_t)(t0 + k);
      for (int q = 0; q < sweeps_per_swap; ++q, ++s)
        gibbs_sweep(&e->L, e->J, e->h, e->Imax, e->B, e->rid, e->spin, e->temp_of, e->tab, a->seed,
                    e->ent, (uint32_t)s, OR_TAG_APT_SWEEP, OR_TAG_APT_REFINE);
      for (int b = 0; b < e->B; ++b)
        e->E[b] = or_energy_lat(&e->L, e->J, e->h, e->spin + (size_t)b * e->L.N);
      best_update(e, s);
      if (icm) {
        for (int r = 0; r < e->T; ++r) {
          int q[4];
          icm_matching(a->seed, e->ent, (uint32_t)r, t, e->A, q);
          for (int p = 0; p < e->A / 2; ++p)
            icm_op(e, a->seed, r * e->A + q[2 * p], r * e->A + q[2 * p + 1], (uint32_t)r, t, (uint32_t)p,
                   a->icm_big, a->icm_seed);
        }
        best_update(e, s);
      }
      swap_step(e, a->seed, t, a->joint);
    }
  }
  (void)threads;
  a->sweeps_done += n_swaps * sweeps_per_swap;
  a->swaps_done += n_swaps;
  return 0;
}

int or_apt_set_joint_swap(or_apt *a, int joint) {
  if (!a) return -1;
  a->joint = joint != 0;
  return 0;
}

int or_apt_set_icm_rules(or_apt *a, int big_cluster_rule, int cluster_seed) {
  if (!a) return -1;
  a->icm_big = big_cluster_rule != 0;
  a->icm_seed = cluster_seed != 0;
  return 0;
}

int or_apt_set_target(or_apt *a, int inst, int64_t e_target) {
  if (!a || inst < 0 || inst >= a->n) return -1;
  a->e[inst].target = e_target;
  a->e[inst].hit_sweep = -1;
  if (a->e[inst].best_E <= e_target) a->e[inst].hit_sweep = a->e[inst].best_sweep;
  return 0;
}

int or_apt_state(const or_apt *a, int inst, int8_t *spins, int64_t *energies, int32_t *temp_of) {
  if (!a || inst < 0 || inst >= a->n) return -1;
  const apt_entry *e = &a->e[inst];
  if (spins) memcpy(spins, e->spin, (size_t)e->B * e->L.N);
  if (energies) memcpy(energies, e->E, sizeof(int64_t) * e->B);
  if (temp_of) memcpy(temp_of, e->temp_of, sizeof(int32_t) * e->B);
  return 0;
}

int or_apt_best(const or_apt *a, int inst, int64_t *E, int64_t *sweep, int32_t *buf,
                int64_t *hit_sweep, int8_t *spins) {
  if (!a || inst < 0 || inst >= a->n) return -1;
  const apt_entry *e = &a->e[inst];
  if (E) *E = e->best_E;
  if (sweep) *sweep = e->best_sweep;
  if (buf) *buf = e->best_buf;
  if (hit_sweep) *hit_sweep = e->hit_sweep;
  if (spins) memcpy(spins, e->best_spin, (size_t)e->L.N);
  return 0;
}

int or_apt_stats(const or_apt *a, int inst, int64_t *att, int64_t *acc, int64_t *icm) {
  if (!a || inst < 0 || inst >= a->n) return -1;
  const apt_entry *e = &a->e[inst];
  size_t np = (size_t)(e->T > 1 ? e->T - 1 : 0) * e->A;
  if (att) memcpy(att, e->att, sizeof(int64_t) * np);
  if (acc) memcpy(acc, e->acc, sizeof(int64_t) * np);
  if (icm) memcpy(icm, e->icm, sizeof(e->icm));
  return 0;
}

int64_t or_apt_sweeps(const or_apt *a) { return a ? a->sweeps_done : -1; }

/* ---------------- adaptive ladder ---------------- */
/* Preprocessing of Algorithm S2 (Methods, "APT details"): n_chains chains
 * run `sweeps` sweeps at beta_t, warm-started from the previous step's
 * states; each chain's energy variance comes from its last `tail`
 * post-sweep energies; sigma_E is the square root of the chains' mean
 * variance; beta_{t+1} = beta_t + alpha / sigma_E; stop at the first beta
 * whose sigma_E < tol. */
int or_adaptive_ladder(const int32_t dims[3], const uint8_t periodic[3], const int8_t *J,
                       const int8_t *h, uint32_t entry, uint64_t seed, double beta0,
                       double alpha, int n_chains, int sweeps, int tail, double tol,
                       int max_len, double *beta_out, double *sigma_out, int *len_out) {
  if (n_chains < 1 || sweeps < 1 || tail < 2 || tail > sweeps || max_len < 1 || !(beta0 > 0))
    return -1;
  or_lat L;
  int rc = or_lat_init(&L, dims, periodic);
  if (rc) return rc;
  int N = L.N;
  int64_t Imax = or_field_bound(&L, J, h);
  int8_t *spin = (int8_t *)malloc((size_t)n_chains * N);
  int32_t *temp_of = (int32_t *)calloc((size_t)n_chains, sizeof(int32_t));
  int64_t *sE = (int64_t *)malloc(sizeof(int64_t) * n_chains);
  int64_t *sE2 = (int64_t *)malloc(sizeof(int64_t) * n_chains);
  init_spins(&L, n_chains, NULL, spin, seed, entry, OR_TAG_LAD_INIT);
  double beta = beta0;
  int len = 0, status = 1;
  uint32_t s = 0;
  while (len < max_len) {
    uint32_t *tab = make_table(beta, Imax);
    memset(sE, 0, sizeof(int64_t) * n_chains);
    memset(sE2, 0, sizeof(int64_t) * n_chains);
    for (int k = 0; k < sweeps; ++k, ++s) {
      gibbs_sweep(&L, J, h, Imax, n_chains, NULL, spin, temp_of, &tab, seed, entry, s,
                  OR_TAG_LAD_SWEEP, OR_TAG_LAD_REFINE);
      if (k >= sweeps - tail) {
        for (int b = 0; b < n_chains; ++b) {
          int64_t E = or_energy_lat(&L, J, h, spin + (size_t)b * N);
          sE[b] += E;
          sE2[b] += E * E;
        }
      }
    }
    free(tab);
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
  free(spin); free(temp_of); free(sE); free(sE2);
  or_lat_free(&L);
  return status;
}

/* ---------------- pilot histograms ---------------- */
int or_pilot_hist(const int32_t dims[3], const uint8_t periodic[3], const int8_t *J,
                  const int8_t *h, uint32_t entry, uint64_t seed, int n_beta,
                  const double *betas, int chains_per_beta, int sweeps, int burn,
                  int n_bins, int64_t *counts) {
  if (n_beta < 1 || chains_per_beta < 1 || sweeps < 1 || burn < 0 || burn >= sweeps ||
      n_bins < 1)
    return -1;
  or_lat L;
  int rc = or_lat_init(&L, dims, periodic);
  if (rc) return rc;
  int N = L.N, B = n_beta * chains_per_beta;
  int64_t Imax = or_field_bound(&L, J, h);
  int8_t *spin = (int8_t *)malloc((size_t)B * N);
  int32_t *temp_of = (int32_t *)malloc(sizeof(int32_t) * B);
  uint32_t **tab = (uint32_t **)malloc(sizeof(uint32_t *) * n_beta);
  for (int b = 0; b < B; ++b) temp_of[b] = b / chains_per_beta;
  for (int t = 0; t < n_beta; ++t) tab[t] = make_table(betas[t], Imax);
  memset(counts, 0, sizeof(int64_t) * (size_t)n_beta * n_bins);
  init_spins(&L, B, NULL, spin, seed, entry, OR_TAG_PIL_INIT);
  int64_t span = 3 * (int64_t)N;
  for (int s = 0; s < sweeps; ++s) {
    gibbs_sweep(&L, J, h, Imax, B, NULL, spin, temp_of, tab, seed, entry, (uint32_t)s,
                OR_TAG_PIL_SWEEP, OR_TAG_PIL_REFINE);
    if (s < burn) continue;
    for (int b = 0; b < B; ++b) {
      int64_t E = or_energy_lat(&L, J, h, spin + (size_t)b * N);
      int64_t num = (E + span) * n_bins;
      int64_t bin = num < 0 ? 0 : num / span;
      if (bin > n_bins - 1) bin = n_bins - 1;
      counts[(size_t)temp_of[b] * n_bins + bin]++;
    }
  }
  for (int t = 0; t < n_beta; ++t) free(tab[t]);
  free(tab); free(spin); free(temp_of);
  or_lat_free(&L);
  return 0;
}
