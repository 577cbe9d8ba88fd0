/*
 * Oracle: discrete-time simulated quantum annealing (Suzuki-Trotter
 * mapping of Eq. S.3, Algorithm S1).  TEST INFRASTRUCTURE ONLY (oracle.h).
 *
 * The classical (d+1)-dimensional system has P slices of the 3D lattice,
 * each with the full couplings J, and a ferromagnetic coupling J_perp
 * between the same site of neighbouring slices (periodic in the slice
 * index).  Spins are sampled from exp(-H_C / (P T)):
 *   H_C = -sum_k [ sum_<ij> J_ij s_ik s_jk + J_perp sum_i s_ik s_i,k+1 ],
 *   J_perp(Gamma) = -(P T / 2) ln tanh(Gamma / (P T)),
 * which is Eq. S.3 (J_par = J/P, beta J_perp = -1/2 ln tanh(beta Gamma/P))
 * multiplied through by P.  J_perp is held in Q16.16 fixed point.
 *
 * 4D colouring: c = (x + y + z + k) & 1.  For slice k the half-word index
 * is m = k >> 1 (block m >> 3, nibble m & 7), and the update uniform of
 * site (lin, k) at sweep s uses counters
 *   (lin, s, (c << 16) | (m >> 3), (run << 8) | TAG)  half (m & 7).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"
#include "oracle_internal.h"

static void sqa_run(const or_lat *L, const int8_t *J, int P, double T, int n_sweeps,
                    const double *gamma, uint32_t run, uint64_t seed, int64_t Imax,
                    int64_t *E_out, int8_t *spins_out) {
  int N = L->N;
  int8_t *s = (int8_t *)malloc((size_t)P * N);
  uint32_t *tab = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)(2 * Imax + 1));
  double beta_eff = 1.0 / ((double)P * T);
  /* Algorithm S1: initialise all spins in all replicas to random states */
  for (int k = 0; k < P; ++k)
    for (int lin = 0; lin < N; ++lin) {
      int c = (or_colour(L, lin) + k) & 1, m = k >> 1;
      uint32_t ctr[4] = {(uint32_t)lin, 0u, ((uint32_t)c << 16) | (uint32_t)(m >> 3),
                         (run << 8) | OR_TAG_SQA_INIT};
      uint32_t x[4];
      or_philox(ctr, seed, x);
      s[(size_t)k * N + lin] = (or_half(x, m & 7) < 0x8000u) ? 1 : -1;
    }
  for (int sw = 0; sw < n_sweeps; ++sw) {
    /* transverse field from the schedule -> transverse coupling */
    int32_t jq = or_jperp_q(gamma[sw], P, T);
    for (int nn = 0; nn < 3; ++nn)
      for (int64_t I = -Imax; I <= Imax; ++I)
        tab[(size_t)nn * (2 * Imax + 1) + (I + Imax)] =
            or_sqa_threshold(beta_eff, I, jq, 2 * nn - 2);
    for (int c = 0; c < 2; ++c)
      for (int k = 0; k < P; ++k) {
        int8_t *sk = s + (size_t)k * N;
        const int8_t *sdn = s + (size_t)((k + P - 1) % P) * N;
        const int8_t *sup = s + (size_t)((k + 1) % P) * N;
        int m = k >> 1;
        for (int lin = 0; lin < N; ++lin) {
          if (((or_colour(L, lin) + k) & 1) != c) continue;
          int64_t I = or_field(L, J, NULL, sk, lin);
          int n = sdn[lin] + sup[lin];
          uint32_t u = or_uniform32(seed, (uint32_t)lin, (uint32_t)sw,
                                    ((uint32_t)c << 16) | (uint32_t)(m >> 3), run,
                                    OR_TAG_SQA_SWEEP, OR_TAG_SQA_REFINE, m & 7);
          uint32_t thr = tab[(size_t)((n + 2) / 2) * (2 * Imax + 1) + (I + Imax)];
          sk[lin] = (u < thr) ? 1 : -1;
        }
      }
  }
  /* Algorithm S1: compute the (classical) energy of each replica */
  for (int k = 0; k < P; ++k) E_out[k] = or_energy_lat(L, J, NULL, s + (size_t)k * N);
  if (spins_out) memcpy(spins_out, s, (size_t)P * N);
  free(s);
  free(tab);
}

int or_sqa_anneal(const int32_t dims[3], const uint8_t periodic[3], const uint8_t *present, const int8_t *J,
                  int P, double T, int n_sweeps, const double *gamma, int R,
                  uint32_t run0, uint64_t seed, int64_t *E_out, int8_t *spins_out,
                  int threads) {
  if (P < 2 || (P & 1) || !(T > 0) || n_sweeps < 0 || R < 1) return -1;
  for (int i = 0; i < n_sweeps; ++i)
    if (!(gamma[i] > 0)) return -1;
  or_lat L;
  int rc = or_lat_init(&L, dims, periodic);
  if (!rc) rc = or_lat_set_present(&L, present);
  if (rc) { or_lat_free(&L); return rc; }
  int64_t Imax = or_field_bound(&L, J, NULL);
  int N = L.N;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int r = 0; r < R; ++r)
    sqa_run(&L, J, P, T, n_sweeps, gamma, run0 + (uint32_t)r, seed, Imax,
            E_out + (size_t)r * P, spins_out ? spins_out + (size_t)r * P * N : NULL);
  (void)threads;
  or_lat_free(&L);
  return 0;
}
