/*
 * CPU oracle for the probabilistic-computer Monte Carlo of arXiv 2503.10302.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct C that restates
 * the paper's method step by step (p-bit / Gibbs updates, Eqs. synapse and
 * neuron; the Edwards-Anderson energy, Eqs. EAmodel and ising_energy; the
 * replica-exchange rule of Sec. "Comparison with Adaptive Parallel
 * Tempering"; ICMop and the adaptive beta ladder of Algorithm S2; DT-SQA of
 * Eq. S.3 and Algorithm S1).  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * All functions return 0 on success and a negative value on invalid input.
 *
 * Randomness contract (both implementations follow it; each has its own
 * Philox4x32-10 written from Salmon et al., SC'11):
 *   key  = (seed & 0xffffffff, seed >> 32)
 *   half v_i of a Philox output block x[0..3], i in 0..7:
 *        (x[i >> 1] >> (16 * (i & 1))) & 0xffff
 *   sampler replica id b of problem entry e: group g = b >> 3, nibble
 *   i = b & 7 (APT: the replica in slot (temperature r, label a) has id
 *   a * Tp + r, Tp = 8 ceil(T/8); ladder and pilot chains: id = chain).
 *   A site lin of colour c = (x+y+z)&1 has colour-local index j = lin >> 1.
 *   update uniform u (32 bits) at sweep s:
 *        hi = v_i(Philox((j, s, (c<<16)|g, (e<<8)|TAG_MAIN)))
 *        lo = v_i(Philox((j, s, (c<<16)|g, (e<<8)|TAG_REFINE)))
 *        u  = (hi << 16) | lo;   sigma <- +1 iff u < T(beta, I)
 *   initial spin: +1 iff v_i(Philox((j, 0, (c<<16)|g, (e<<8)|TAG_INIT))) < 0x8000
 */
#ifndef PCOMP_ORACLE_H
#define PCOMP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_TAG_APT_INIT = 1, OR_TAG_APT_SWEEP = 2, OR_TAG_APT_REFINE = 3,
  OR_TAG_SWAP = 4, OR_TAG_ICM = 5,
  OR_TAG_LAD_INIT = 6, OR_TAG_LAD_SWEEP = 7, OR_TAG_LAD_REFINE = 8,
  OR_TAG_PIL_INIT = 9, OR_TAG_PIL_SWEEP = 10, OR_TAG_PIL_REFINE = 11,
  OR_TAG_SQA_INIT = 12, OR_TAG_SQA_SWEEP = 13, OR_TAG_SQA_REFINE = 14,
  /* general sparse graphs (graph.c) */
  OR_TAG_G_INIT = 15, OR_TAG_G_SWEEP = 16, OR_TAG_G_REFINE = 17, OR_TAG_G_SWAP = 18,
  OR_TAG_G_ICM = 19, OR_TAG_GS_INIT = 20, OR_TAG_GS_SWEEP = 21, OR_TAG_GS_REFINE = 22,
  OR_TAG_GL_INIT = 23, OR_TAG_GL_SWEEP = 24, OR_TAG_GL_REFINE = 25
};

/* Philox4x32-10 on one counter. */
void or_philox(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]);
/* n counters [n][4] -> n blocks [n][4]. */
void or_philox_many(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out);

/* Acceptance thresholds (uint32, compared with a uniform 32-bit u). */
uint32_t or_pbit_threshold(double beta, int64_t I);   /* floor(2^32 / (1+exp(-2 beta I))) */
uint32_t or_swap_threshold(double dbeta, int64_t dE); /* floor(2^32 exp(dbeta dE)), dE < 0 */
int32_t  or_jperp_q(double gamma, int P, double T);   /* round(2^16 J_perp) */
uint32_t or_sqa_threshold(double beta_eff, int64_t I, int32_t jq, int n);

/* Energy E = -sum_bonds J s s - sum h s of one configuration (int64). */
/* present [N] (nullable): 0 marks a vacancy (missing spin) with no bonds;
 * the same convention holds for or_apt_create and or_sqa_anneal. */
int or_energy(const int32_t dims[3], const uint8_t periodic[3], const uint8_t *present, const int8_t *J,
              const int8_t *h, const int8_t *spin, int64_t *E_out);

/* ---------------- adaptive parallel tempering (Algorithm S2) ---------------- */
typedef struct or_apt or_apt;
/* n_inst problems; dims/periodic [n][3]; J concatenated [sum N][3];
   h concatenated [sum N] or NULL; n_temps[n]; betas concatenated. */
int or_apt_create(or_apt **out, int n_inst, const int32_t *dims, const uint8_t *periodic,
                  const uint8_t *present,
                  const int8_t *J, const int8_t *h, const int32_t *n_temps,
                  const double *betas, int n_labels, uint64_t seed, uint32_t entry0);
void or_apt_destroy(or_apt *a);
/* n_swaps swap attempts, each preceded by sweeps_per_swap sweeps.
   icm: 0 off, 1 on.  threads: OpenMP threads over problems (<=0: default). */
int or_apt_run(or_apt *a, int64_t n_swaps, int sweeps_per_swap, int icm, int threads);
/* Swap rule: 0 (default) = each label decides on its own (Methods); 1 = one
 * decision per temperature pair swaps all labels, accepted with
 * min(1, exp(dbeta sum_a dE_a)) (Algorithm S2 read literally). */
int or_apt_set_joint_swap(or_apt *a, int joint);
/* ICMop rules of later runs (Algorithm S2 ICMop): big_cluster_rule 1
 * (default) flips one whole replica when the cluster holds more than half
 * of the spins present, 0 always flips the cluster in both replicas;
 * cluster_seed 0 (default) seeds the cluster at a uniformly chosen mismatch
 * site, 1 picks one of the mismatch clusters uniformly ("randomly pick one
 * cluster"), k = floor(x0 n_clusters / 2^32), clusters ordered by their first
 * site in canonical order. */
int or_apt_set_icm_rules(or_apt *a, int big_cluster_rule, int cluster_seed);
int or_apt_set_target(or_apt *a, int inst, int64_t e_target);
/* spins [B][N] in slot order (slot r*A + a: temperature r, label a);
   energies [B]; temperature index of each slot [B] (= slot / A). */
int or_apt_state(const or_apt *a, int inst, int8_t *spins, int64_t *energies, int32_t *temp_of);
/* best energy, sweep count when found, buffer, target hit sweep (-1: never). */
int or_apt_best(const or_apt *a, int inst, int64_t *E, int64_t *sweep, int32_t *buf,
                int64_t *hit_sweep, int8_t *spins /* nullable [N] */);
/* swap attempts / accepts [n_temps-1][n_labels]; icm counters [3]:
   empty overlap, cluster flips, whole-replica flips. */
int or_apt_stats(const or_apt *a, int inst, int64_t *att, int64_t *acc, int64_t *icm);
int64_t or_apt_sweeps(const or_apt *a);
/* One ICMop on two configurations (ctr = (r, t, p, (entry<<8)|TAG_ICM));
   returns 0 no overlap mismatch, 1 cluster flipped in both, 2 one whole
   replica flipped; *cluster_size = size of the grown cluster. */
/* Pairs of ICM labels at temperature r, attempt t (Algorithm S2 "Randomly
 * partition ICM replicas into pairs"): pairs[0..1], pairs[2..3] (4 labels)
 * or pairs[0..1] = (0, 1) (2 labels).  Returns the matching index 0..2. */
int or_icm_pairing(uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, int n_labels,
                   int32_t *pairs);
int or_icm_apply(const int32_t dims[3], const uint8_t periodic[3], int8_t *sa, int8_t *sb,
                 uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, uint32_t p,
                 int64_t *cluster_size);
/* As or_icm_apply under the rules of or_apt_set_icm_rules. */
int or_icm_apply_rules(const int32_t dims[3], const uint8_t periodic[3], int8_t *sa, int8_t *sb,
                       uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, uint32_t p, int big_rule,
                       int seed_rule, int64_t *cluster_size);
/* ICMop with its random choices given: seed choice k in [0, n_choices)
 * (mismatch site or cluster, by seed_rule) and flip_b (whole-replica flip
 * of the second replica).  *n_choices receives the number of choices
 * (0: nothing moves).  Returns 0 (no mismatch), 1 (cluster), 2 (whole
 * replica) or -1 (k out of range).  Used to enumerate transition matrices. */
int or_icm_choice(const int32_t dims[3], const uint8_t periodic[3], int8_t *sa, int8_t *sb, int64_t k,
                  int flip_b, int big_rule, int seed_rule, int64_t *n_choices, int64_t *cluster_size);

/* ---------------- adaptive beta ladder (Algorithm S2 preprocessing) --------- */
/* beta_out/sigma_out have room for max_len; *len_out = ladder length;
   returns 1 (not 0) if max_len was reached before sigma_E < tol. */
int or_adaptive_ladder(const int32_t dims[3], const uint8_t periodic[3], const int8_t *J,
                       const int8_t *h, uint32_t entry, uint64_t seed, double beta0,
                       double alpha, int n_chains, int sweeps, int tail, double tol,
                       int max_len, double *beta_out, double *sigma_out, int *len_out);

/* ---------------- pilot-run energy histograms ---------------- */
/* counts [n_beta][n_bins]: post-sweep energies of sweeps burn..sweeps-1 of
   chains_per_beta chains at each beta; bin = floor(n_bins (E+3N)/(3N)),
   clamped to [0, n_bins-1] (E/N over [-3, 0]). */
int or_pilot_hist(const int32_t dims[3], const uint8_t periodic[3], const int8_t *J,
                  const int8_t *h, uint32_t entry, uint64_t seed, int n_beta,
                  const double *betas, int chains_per_beta, int sweeps, int burn,
                  int n_bins, int64_t *counts);

/* ---------------- DT-SQA (Eq. S.3, Algorithm S1) ---------------- */
/* R runs (global ids run0..run0+R-1) of P slices; E_out [R][P] final classical
   slice energies; spins_out [R][P][N] or NULL. */
int or_sqa_anneal(const int32_t dims[3], const uint8_t periodic[3], const uint8_t *present, const int8_t *J,
                  int P, double T, int n_sweeps, const double *gamma, int R,
                  uint32_t run0, uint64_t seed, int64_t *E_out, int8_t *spins_out,
                  int threads);

/* ---------------- general sparse graphs (graph.c) ---------------- */
/* A graph of n p-bits is given in CSR form: the neighbours of v are
 * col[rp[v] .. rp[v+1]-1] with integer weights w (J_vu, nonzero), listed in
 * both directions with equal weights, no self-loops, no repeats; biases h
 * [n] or NULL.  Couplings are integers: fixed-point weights with f
 * fractional bits are passed as integers with beta scaled by 2^-f.
 *
 * Colour classes: a proper colouring colour[v] in [0, C) (C <= 32); the
 * colour-local index of v is j(v) = #{u < v : colour[u] = colour[v]}; the
 * canonical vertex order is colour 0 by increasing v, then colour 1, ...
 *
 * Randomness (APT on graphs): replica in slot (temperature r, label a) has
 * id b = 32 a + r (T <= 32), group g = b >> 3 and half i = b & 7, as the
 * lattice path's replica groups; vertex v of colour c (colour-local index j)
 * at sweep s uses
 *   hi = v_i(Philox((j, s, (c << 16) | g, (e << 8) | TAG_G_SWEEP)))
 *   lo = the same half of the TAG_G_REFINE block;  +1 iff (hi<<16|lo) < T.
 * Initial spin: +1 iff v_i(Philox((j, 0, (c<<16)|g, (e<<8)|TAG_G_INIT))) < 2^15.
 * Swap of pair (r, r+1), label a, attempt t: word 0 of P(r, t, a, (e<<8)|TAG_G_SWAP).
 * ICM of pair p at temperature r, attempt t: P(r, t, p, (e<<8)|TAG_G_ICM),
 * words as in the lattice path (seed k, whole-replica bit, 4-label matching).
 *
 * DT-SQA on graphs: slice k of vertex v has colour (colour[v] + f(k)) mod C'
 * with f(k) = k & 1, except f(P-1) = 2 when P is odd; C' = max(C, 2) for
 * even P and max(C, 3) for odd P.  A class is ordered by k, then v; (v, k)
 * of class c with class-local index j in run q uses
 *   v_{q&7}(Philox((j, s, c, ((q >> 3) << 8) | TAG_GS_SWEEP / TAG_GS_REFINE))),
 * so one call serves 8 consecutive runs. */

/* 0 if (rp, col, w) is a valid symmetric graph as above; -1 otherwise. */
int or_graph_check(int n, const int32_t *rp, const int32_t *col, const int8_t *w);
/* DSATUR (Brelaz 1979): repeatedly colour the uncoloured vertex of largest
 * saturation (distinct colours among its coloured neighbours), ties by the
 * largest degree in the uncoloured subgraph, then the smallest index, with
 * the smallest colour absent from its neighbours.  *n_colours = C. */
int or_dsatur(int n, const int32_t *rp, const int32_t *col, int32_t *colour, int *n_colours);
/* Colours [P][n] of the replicated DT-SQA network (rule above); *n_colours = C'. */
int or_graph_sqa_colouring(int n, const int32_t *colour, int P, int32_t *out, int *n_colours);
/* E = -sum_{u<v} w_uv s_u s_v - sum_v h_v s_v. */
int or_graph_energy(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                    const int8_t *h, const int8_t *spin, int64_t *E_out);

typedef struct or_gapt or_gapt;
/* n_prob graphs; n_vert[i]; rp concatenated ([n_i + 1] each, local
 * offsets), col/w concatenated (local vertex ids), h concatenated or NULL,
 * colour concatenated or NULL (DSATUR); n_temps[i] <= 32; betas
 * concatenated; n_labels in {1, 2, 4}. */
int or_gapt_create(or_gapt **out, int n_prob, const int32_t *n_vert, const int32_t *rp,
                   const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
                   const int32_t *n_temps, const double *betas, int n_labels, uint64_t seed,
                   uint32_t entry0);
void or_gapt_destroy(or_gapt *g);
int or_gapt_run(or_gapt *g, int64_t n_swaps, int sweeps_per_swap, int icm, int threads);
int or_gapt_set_joint_swap(or_gapt *g, int joint);
int or_gapt_set_target(or_gapt *g, int prob, int64_t e_target);
/* spins [B][n] and energies [B] in slot order r*A + a; colours [n] used. */
int or_gapt_state(const or_gapt *g, int prob, int8_t *spins, int64_t *energies, int32_t *colour);
int or_gapt_best(const or_gapt *g, int prob, int64_t *E, int64_t *sweep, int32_t *buf,
                 int64_t *hit_sweep, int8_t *spins);
int or_gapt_stats(const or_gapt *g, int prob, int64_t *att, int64_t *acc, int64_t *icm);

/* One ICMop on two configurations of a coloured graph (ctr = (r, t, p,
 * (entry<<8)|TAG_G_ICM)); returns 0 / 1 / 2 as or_icm_apply. */
int or_gicm_apply(int n, const int32_t *rp, const int32_t *col, const int32_t *colour, int8_t *sa,
                  int8_t *sb, uint64_t seed, uint32_t entry, uint32_t r, uint32_t t, uint32_t p,
                  int64_t *cluster_size);

/* Adaptive beta ladder on a graph (Algorithm S2 preprocessing, as
 * or_adaptive_ladder): chain b (< 128) draws like APT replica id b with the
 * TAG_GL_* tags, the sweep counter running on across beta steps.  colour
 * NULL -> DSATUR.  Returns 1 if max_len was reached before sigma_E < tol. */
int or_graph_adaptive_ladder(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                             const int8_t *h, const int32_t *colour, uint32_t entry, uint64_t seed,
                             double beta0, double alpha, int n_chains, int sweeps, int tail,
                             double tol, int max_len, double *beta_out, double *sigma_out,
                             int *len_out);

/* R runs of P slices on a graph; colour NULL -> DSATUR; E_out [R][P]
 * classical slice energies (with h); spins_out [R][P][n] or NULL. */
int or_gsqa_anneal(int n, const int32_t *rp, const int32_t *col, const int8_t *w,
                   const int8_t *h, const int32_t *colour, int P, double T, int n_sweeps,
                   const double *gamma, int R, uint32_t run0, uint64_t seed, int64_t *E_out,
                   int8_t *spins_out, int threads);

#ifdef __cplusplus
}
#endif
#endif
