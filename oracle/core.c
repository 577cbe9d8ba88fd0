/*
 * Oracle core: Philox4x32-10, acceptance thresholds, lattice geometry and
 * the Ising energy.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "oracle_internal.h"

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  One round maps (c0,c1,c2,c3) under key (k0,k1)
 * to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the
 * key is bumped by the Weyl constants between rounds. */
void or_philox(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox_many(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out) {
  for (int64_t i = 0; i < n; ++i) or_philox(ctr + 4 * i, seed, out + 4 * i);
}

uint32_t or_half(const uint32_t x[4], int i) {
  return (x[i >> 1] >> (16 * (i & 1))) & 0xffffu;
}

uint32_t or_uniform32(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t ent,
                      uint32_t tag_main, uint32_t tag_ref, int i) {
  uint32_t ctr[4], xm[4], xr[4];
  ctr[0] = c0; ctr[1] = c1; ctr[2] = c2; ctr[3] = (ent << 8) | tag_main;
  or_philox(ctr, seed, xm);
  ctr[3] = (ent << 8) | tag_ref;
  or_philox(ctr, seed, xr);
  return (or_half(xm, i) << 16) | or_half(xr, i);
}

/* floor(2^32 p) clamped to [0, 2^32-1] for p in [0, 1]. */
static uint32_t prob_to_threshold(double p) {
  double t = floor(ldexp(p, 32));
  if (!(t > 0.0)) return 0u;
  if (t >= 4294967295.0) return 0xffffffffu;
  return (uint32_t)t;
}

/* Eq. neuron: sigma = sgn(tanh(beta I) - r), r ~ U[-1,1], so
 * P(sigma = +1) = (1 + tanh(beta I))/2 = 1/(1 + exp(-2 beta I)). */
uint32_t or_pbit_threshold(double beta, int64_t I) {
  double p = 1.0 / (1.0 + exp(-2.0 * beta * (double)I));
  return prob_to_threshold(p);
}

/* Replica exchange: p_swap = min(1, exp(dbeta dE)); the threshold is used
 * only when dbeta dE < 0. */
uint32_t or_swap_threshold(double dbeta, int64_t dE) {
  double p = exp(dbeta * (double)dE);
  if (p >= 1.0) return 0xffffffffu;
  return prob_to_threshold(p);
}

/* Eq. S.3 with the temperature T of a P-slice Trotter decomposition:
 * J_perp = -(P T / 2) ln tanh(Gamma / (P T)), held in Q16.16. */
int32_t or_jperp_q(double gamma, int P, double T) {
  double pt = (double)P * T;
  double jp = -0.5 * pt * log(tanh(gamma / pt));
  return (int32_t)llround(jp * 65536.0);
}

/* Slice-spin update of DT-SQA: local field I (intra-slice, full J) plus
 * J_perp * n with n = s_{k-1} + s_{k+1}; beta_eff = 1/(P T). */
uint32_t or_sqa_threshold(double beta_eff, int64_t I, int32_t jq, int n) {
  double h = (double)I + ldexp((double)jq, -16) * (double)n;
  double p = 1.0 / (1.0 + exp(-2.0 * beta_eff * h));
  return prob_to_threshold(p);
}

/* ------------------------------------------------------------------------ */
int or_lat_init(or_lat *L, const int32_t dims[3], const uint8_t periodic[3]) {
  memset(L, 0, sizeof(*L));
  L->vac = NULL;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1 || dims[a] > 4096) return -1;
    L->L[a] = dims[a];
    L->per[a] = periodic ? (periodic[a] != 0) : 1;
    /* a periodic axis must have even length >= 2 so that (x+y+z)&1 is a
       proper 2-colouring and no site is bonded to itself */
    if (L->per[a] && (dims[a] < 2 || (dims[a] & 1))) return -1;
  }
  L->N = dims[0] * dims[1] * dims[2];
  if (L->N > (1 << 24)) return -1;
  L->nreal = L->N;
  L->nb = (int32_t *)malloc(sizeof(int32_t) * 6 * (size_t)L->N);
  if (!L->nb) return -2;
  for (int lin = 0; lin < L->N; ++lin) {
    int x = lin % L->L[0], y = (lin / L->L[0]) % L->L[1], z = lin / (L->L[0] * L->L[1]);
    int c[3] = {x, y, z};
    for (int a = 0; a < 3; ++a) {
      for (int s = 0; s < 2; ++s) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[a] += s ? -1 : 1;
        int ok = 1;
        if (cc[a] < 0 || cc[a] >= L->L[a]) {
          if (L->per[a]) cc[a] = (cc[a] + L->L[a]) % L->L[a];
          else ok = 0;
        }
        L->nb[6 * lin + 2 * a + s] = ok ? cc[0] + L->L[0] * (cc[1] + L->L[1] * cc[2]) : -1;
      }
    }
  }
  return 0;
}

int or_lat_set_present(or_lat *L, const uint8_t *present) {
  if (!present) return 0;
  L->vac = (uint8_t *)calloc((size_t)L->N, 1);
  if (!L->vac) return -2;
  L->nreal = 0;
  for (int lin = 0; lin < L->N; ++lin) {
    L->vac[lin] = present[lin] ? 0 : 1;
    L->nreal += present[lin] ? 1 : 0;
  }
  /* a bond exists only between two present sites */
  for (int lin = 0; lin < L->N; ++lin)
    for (int d = 0; d < 6; ++d) {
      int n = L->nb[6 * lin + d];
      if (n >= 0 && (L->vac[lin] || L->vac[n])) L->nb[6 * lin + d] = -1;
    }
  return 0;
}

void or_lat_free(or_lat *L) {
  free(L->nb);
  L->nb = NULL;
  free(L->vac);
  L->vac = NULL;
}

int or_colour(const or_lat *L, int lin) {
  int x = lin % L->L[0], y = (lin / L->L[0]) % L->L[1], z = lin / (L->L[0] * L->L[1]);
  return (x + y + z) & 1;
}

/* Coupling on the bond from lin along direction dir (0:+x 1:-x 2:+y 3:-y
 * 4:+z 5:-z); forward bonds are stored at the site, backward ones at the
 * neighbour.  0 if the bond does not exist. */
int or_coupling(const or_lat *L, const int8_t *J, int lin, int dir) {
  int n = L->nb[6 * lin + dir];
  if (n < 0) return 0;
  int a = dir >> 1;
  return (dir & 1) ? J[3 * n + a] : J[3 * lin + a];
}

/* Eq. synapse: I_i = sum_j J_ij s_j + h_i. */
int64_t or_field(const or_lat *L, const int8_t *J, const int8_t *h, const int8_t *s, int lin) {
  int64_t I = (h && !(L->vac && L->vac[lin])) ? h[lin] : 0;
  for (int dir = 0; dir < 6; ++dir) {
    int n = L->nb[6 * lin + dir];
    if (n >= 0) I += (int64_t)or_coupling(L, J, lin, dir) * s[n];
  }
  return I;
}

/* Eq. ising_energy: E = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i, each bond
 * counted once as the forward bond of its lower endpoint along its axis. */
int64_t or_energy_lat(const or_lat *L, const int8_t *J, const int8_t *h, const int8_t *s) {
  int64_t E = 0;
  for (int lin = 0; lin < L->N; ++lin) {
    for (int a = 0; a < 3; ++a) {
      int n = L->nb[6 * lin + 2 * a];
      if (n >= 0) E -= (int64_t)J[3 * lin + a] * s[lin] * s[n];
    }
    if (h && !(L->vac && L->vac[lin])) E -= (int64_t)h[lin] * s[lin];
  }
  return E;
}

int or_energy(const int32_t dims[3], const uint8_t periodic[3], const uint8_t *present, const int8_t *J,
              const int8_t *h, const int8_t *spin, int64_t *E_out) {
  or_lat L;
  int rc = or_lat_init(&L, dims, periodic);
  if (rc) return rc;
  if ((rc = or_lat_set_present(&L, present))) { or_lat_free(&L); return rc; }
  *E_out = or_energy_lat(&L, J, h, spin);
  or_lat_free(&L);
  return 0;
}

int64_t or_field_bound(const or_lat *L, const int8_t *J, const int8_t *h) {
  int64_t m = 0;
  for (int lin = 0; lin < L->N; ++lin) {
    int64_t s = h ? llabs((long long)h[lin]) : 0;
    for (int dir = 0; dir < 6; ++dir) s += llabs((long long)or_coupling(L, J, lin, dir));
    if (s > m) m = s;
  }
  return m;
}
