/*
 * pcomp: GB300 (sm_103a) probabilistic-computer Monte Carlo for 3D +-J
 * Edwards-Anderson spin glasses, after arXiv 2503.10302 ("Pushing the
 * Boundary of Quantum Advantage in Hard Combinatorial Optimization with
 * Probabilistic Computers").
 *
 * C ABI.  Plain pointers and sizes only.  Unless a name ends in _dev, every
 * pointer argument is a HOST pointer owned by the caller; the library never
 * keeps a caller pointer after a call returns.  Device memory behind a
 * context is owned by the context and freed by pc_destroy.  *_dev calls
 * take DEVICE pointers owned by the caller, valid on the context's device,
 * and enqueue work on the context's stream without synchronising.
 *
 * Every int-returning call returns PC_OK (0) or a negative PC_E* code and
 * sets a thread-local message readable with pc_last_error().  No call
 * aborts the process.  Kernels contain no unbounded waits.
 *
 * Lattices: dims = (Lx, Ly, Lz), site lin = x + Lx*(y + Ly*z), all three
 * axes periodic, every dimension even, 2 <= Lx <= 16, Ly, Lz >= 2,
 * N = Lx*Ly*Lz <= 4096.  Couplings J are int8 [N][3]: the forward bond of
 * site lin along +x, +y, +z, each in {-1, +1} (Eq. EAmodel).  No field
 * (h = 0) on this path.
 *
 * Randomness contract (shared with the CPU oracle, which has its own
 * code): Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed;
 * every draw is a counter (c0, c1, c2, c3) whose 8 16-bit halves feed 8
 * spins of one "group" of 8 replicas (or 8 Trotter slices); a spin's
 * 32-bit uniform is (main half << 16) | (refine half).  A lattice spin
 * update draws the counter (j, sweep, (colour << 16) | group,
 * (entry << 8) | tag) with j = lin >> 1 the site's index within its
 * checkerboard colour; a swap of pair (r, r+1), label a at attempt t draws
 * (r, t, a, (entry << 8) | 4) and an ICM move of pair p at temperature r
 * draws (r, t, p, (entry << 8) | 5).
 */
#ifndef PCOMP_H
#define PCOMP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PC_OK 0
#define PC_EINVAL (-1)   /* bad argument / unsupported shape */
#define PC_ENOMEM (-2)   /* host or device allocation failed */
#define PC_ECUDA (-3)    /* CUDA runtime error (message has the detail) */
#define PC_ESTATE (-4)   /* call out of order (e.g. run before load) */
#define PC_EDEVICE (-5)  /* a kernel reported a failed device-side check */

typedef struct pc_ctx pc_ctx;

/* Context on CUDA device `device` with Philox seed `seed`.  All launches go
 * to the context's stream (a new non-blocking stream unless pc_set_stream
 * names another). */
int pc_create(pc_ctx **out, int device, uint64_t seed);
void pc_destroy(pc_ctx *ctx);
const char *pc_last_error(void);
/* Use `stream` (a cudaStream_t, or NULL for the legacy default stream). */
int pc_set_stream(pc_ctx *ctx, void *stream);
int pc_synchronize(pc_ctx *ctx);
int pc_device_sm_count(pc_ctx *ctx, int *sms);

/* Device Philox4x32-10 on n host counters [n][4] -> host out [n][4] (the
 * generator of the randomness contract; used to check it on the GPU). */
int pc_philox(pc_ctx *ctx, int64_t n, const uint32_t *ctr, uint32_t *out);

/* ------------------------------------------------------------------------
 * Thresholds (host functions; the CUDA kernels read these tables).
 * Eq. neuron gives P(s = +1) = (1 + tanh(beta I)) / 2 = 1/(1 + e^{-2 beta I});
 * the threshold is floor(2^32 P) clamped to 2^32 - 1 and a spin becomes +1
 * iff its 32-bit uniform is below it.
 * ---------------------------------------------------------------------- */
uint32_t pc_pbit_threshold(double beta, int I);
/* Replica exchange (Sec. "Comparison with Adaptive Parallel Tempering"):
 * p_swap = min(1, exp(dbeta dE)); threshold floor(2^32 exp(dbeta dE)) for
 * dbeta dE < 0. */
uint32_t pc_swap_threshold(double dbeta, int64_t dE);
/* Eq. S.3 multiplied by P: J_perp = -(P T / 2) ln tanh(Gamma / (P T)),
 * returned in Q16.16 (round to nearest). */
int32_t pc_jperp_q(double gamma, int P, double T);

/* ------------------------------------------------------------------------
 * Adaptive parallel tempering with isoenergetic cluster moves
 * (Algorithm S2; Methods "APT details").
 * ---------------------------------------------------------------------- */
/* Load a batch of n_inst problems: dims [n][3], J concatenated [sum N][3],
 * n_temps [n], betas concatenated (strictly increasing per problem),
 * n_labels in {1, 2, 4} replicas per temperature (ICM needs 2 or 4; the
 * paper uses 4), n_temps <= 32 and 8 * ceil(n_temps / 8) * n_labels <= 128
 * (above 64 the problem runs as two CTAs, see pc_apt_set_split).  Problem i uses entry id entry0 + i in its
 * Philox counters.  Builds the p-bit and swap tables, draws the random
 * initial state (Algorithm S2 "Initialize all replicas to random states")
 * and resets counters, best energies and statistics.  Replaces any batch
 * loaded before. */
int pc_apt_load(pc_ctx *ctx, int n_inst, const int32_t *dims, const int8_t *J,
                const int32_t *n_temps, const double *betas, int n_labels, uint32_t entry0);
/* As pc_apt_load with boundary conditions per axis and vacancies:
 * periodic [n][3] (host, nonzero = periodic, NULL = all periodic) and
 * present [sum N] (host, 0 = vacancy / missing spin, NULL = none).
 *   - An open axis has no bonds across its ends (the paper's instances are
 *     open in x and y, Methods); its forward couplings J[3 s + axis] at the
 *     far end are ignored.
 *   - A vacancy has no bonds; it takes no part in ICM (never mismatched),
 *     its spin in the returned states is meaningless, and the ICM
 *     big-cluster rule compares with half of the spins present.  An odd
 *     length on an open axis is a lattice padded to even length with a
 *     vacant end layer.
 *   - Lengths stay even on every axis (checkerboard layout).
 *   - Sites on an open face or next to a vacancy see a local field over
 *     their present bonds, odd I included; energies sum the present bonds. */
int pc_apt_load_bc(pc_ctx *ctx, int n_inst, const int32_t *dims, const uint8_t *periodic,
                   const uint8_t *present, const int8_t *J, const int32_t *n_temps,
                   const double *betas, int n_labels, uint32_t entry0);
/* n_swaps swap attempts; each = sweeps_per_swap checkerboard sweeps of all
 * replicas, replica energies, best-energy update, (icm != 0) one ICMop per
 * pair of labels of every temperature (two labels: the pair (0, 1); four:
 * two pairs of a random perfect matching, Algorithm S2 "randomly partition
 * ICM replicas into pairs") and a second best update, then the
 * neighbour swaps of that attempt's parity.  Resumable: state, counters and
 * statistics carry over between calls.  Enqueued on the context stream. */
int pc_apt_run(pc_ctx *ctx, int64_t n_swaps, int sweeps_per_swap, int icm);
/* Swap rule of later pc_apt_run calls.  joint = 0 (default, Methods: swaps
 * only between equal labels): every label of a temperature pair decides on
 * its own.  joint = 1 (Algorithm S2 read literally, "swap the p-bit states
 * of all corresponding iso-temperature replicas"): one decision per pair
 * moves all labels, accepted with min(1, exp(dbeta sum_a dE_a)) from word 0
 * of the label-0 swap draw. */
int pc_apt_set_joint_swap(pc_ctx *ctx, int joint);
/* ICMop rules of later pc_apt_run calls (Algorithm S2 ICMop).
 * big_cluster_rule 1 (default): a cluster holding more than half of the
 * spins present flips one whole replica instead ("greater than half");
 * 0: every cluster flips in both replicas, which makes the move an exact
 * symmetric proposal on pairs of states.  cluster_seed 0 (default): the
 * cluster grows from a uniformly chosen mismatch site (the Houdayer
 * choice); 1: one of the mismatch clusters is chosen uniformly ("randomly
 * pick one cluster"), the k-th in the order of their first sites (colour 0
 * by lin, then colour 1), k = floor(x0 n_clusters / 2^32) with x0 word 0 of
 * the pair's ICM draw. */
int pc_apt_set_icm_rules(pc_ctx *ctx, int big_cluster_rule, int cluster_seed);
/* Placement of each problem: one CTA, or a cluster of two CTAs that split
 * its temperatures (rank 0 the hotter half: the ladder's first, lowest-beta
 * temperatures).  The two CTAs exchange the
 * boundary swap and the best-energy candidates through distributed shared
 * memory; results are identical either way.  A problem with more than 64
 * replicas (e.g. 32 temperatures x 4 labels) always splits and needs at
 * least 9 temperatures in every problem of the batch.  pref: 0 (default)
 * also splits when the batch fills at most half the SMs; 1 splits only when
 * needed; 2 splits whenever every problem has at least 9 temperatures; 3
 * splits, problem by problem, those that need it and those (with at least 9
 * temperatures) whose work N x replicas exceeds the batch's mean work per
 * SM, and runs the others as one CTA each, in a second launch on a second
 * stream beside the first (for a batch whose largest problems would
 * otherwise set its time).  pc_apt_is_split reports the current placement:
 * 0 one CTA per problem, 1 every problem split, 2 some problems split. */
int pc_apt_set_split(pc_ctx *ctx, int pref);
int pc_apt_is_split(pc_ctx *ctx, int *split);
/* Autotuner of the fused kernel's launch shape (the paper batches many
 * instances per chip, Sec. "Architecture-based scaling improvement and
 * massive parallelism"): times trial_swaps attempts (with or without ICM)
 * of every candidate on a scratch copy of the loaded batch (the loaded
 * chains do not move) and keeps the fastest for later pc_apt_run calls.
 * Candidates: the placement (one CTA per problem, or two-CTA clusters that
 * split the temperatures, where every problem has at least 9), for two-CTA
 * clusters the split point (the colder CTA takes the groups of 8
 * temperatures above the first split_groups of each label; 0 = half), threads
 * per CTA (256, 320, 384, 448, 512), and the split of those threads over
 * sites and replica groups (nch chunks of threads, each sweeping
 * ceil(groups / nch) groups of its sites; 0 = a cost model's choice, or 1, 2,
 * 4), and the per-problem placement of preference 3 where it differs from
 * both others.  Returns the choice in *tpb, *nch, *split (0 = one CTA per
 * problem, 1 = two-CTA clusters, 2 = clusters for some problems) and
 * *split_groups; any may be NULL.  Results do not depend on the shape:
 * randomness is keyed by slot and site. */
int pc_apt_autotune(pc_ctx *ctx, int trial_swaps, int icm, int *tpb, int *nch, int *split,
                    int *split_groups);
/* Set the launch shape directly: tpb threads per CTA (a multiple of 64 in
 * [64, 512]), nch thread chunks (0, 1, 2, 4 or 8; applied where it fits,
 * else the cost model decides), split_pref (0 .. 3) as pc_apt_set_split, and
 * split_groups (0 .. 3) the temperature groups per label of the hotter CTA of
 * a split problem (0: half; clamped to leave the colder CTA one). */
int pc_apt_set_launch(pc_ctx *ctx, int tpb, int nch, int split_pref, int split_groups);
/* Set the threads per CTA directly (multiple of 64 in [64, 512]). */
int pc_apt_set_block_threads(pc_ctx *ctx, int tpb);
/* Checkpoint / resume: pc_apt_save writes the batch's dynamic state
 * (replica spins, energies, best energies and states, hit sweeps, targets,
 * statistics, counters) to a file; pc_apt_restore reads it back into a
 * context on which the same batch (shapes, ladders' sizes, entry ids, seed)
 * was loaded.  Counter-based randomness makes the resumed chains identical
 * to uninterrupted ones. */
int pc_apt_save(pc_ctx *ctx, const char *path);
int pc_apt_restore(pc_ctx *ctx, const char *path);
/* Sweeps and swap attempts done since pc_apt_load. */
int pc_apt_progress(pc_ctx *ctx, int64_t *sweeps, int64_t *swaps);
/* Target energy for time-to-target: the first sweep count at which the
 * best energy is <= e_target is recorded as the hit sweep. */
int pc_apt_set_target(pc_ctx *ctx, int inst, int64_t e_target);
/* Replica spins [B][N] int8 +-1 (slot order, lin order), energies [B],
 * temperature index of each slot [B]; any output may be NULL.
 * B = n_temps * n_labels; slot b is temperature b / n_labels with label
 * b % n_labels (accepted swaps exchange the replicas' states). */
int pc_apt_get_state(pc_ctx *ctx, int inst, int8_t *spins, int64_t *energies, int32_t *temp_of);
/* Best energy seen at a measurement point, the sweep count then, the
 * slot, the hit sweep (-1 if the target was never reached), and the
 * best state [N] (nullable). */
int pc_apt_get_best(pc_ctx *ctx, int inst, int64_t *E, int64_t *sweep, int32_t *buf,
                    int64_t *hit_sweep, int8_t *spins);
/* Best energies [n_inst] and hit sweeps [n_inst] of all problems. */
int pc_apt_get_best_all(pc_ctx *ctx, int64_t *E, int64_t *hit_sweep);
/* Swap attempts / accepts [n_temps-1][n_labels]; icm [3] = (empty
 * overlap, cluster flips, whole-replica flips). */
int pc_apt_get_stats(pc_ctx *ctx, int inst, int64_t *att, int64_t *acc, int64_t *icm);
/* The tables the kernels use: p-bit thresholds [n_temps][7] for I = 2c - 6,
 * c = 0..6, and the swap table of pair (r, r+1): entry k = threshold for
 * dE = -2k, k = 0..len-1 (entries past len are 0). */
int pc_apt_get_pbit_table(pc_ctx *ctx, int inst, uint32_t *out);
int pc_apt_get_swap_table(pc_ctx *ctx, int inst, int pair, uint32_t *out, int max_len, int *len);

/* ------------------------------------------------------------------------
 * Discrete-time simulated quantum annealing (Eq. S.3, Algorithm S1).
 * ---------------------------------------------------------------------- */
/* One instance (dims, J) with P Trotter slices (P a multiple of 16,
 * N * P <= 262144), temperature T and the transverse-field schedule
 * gamma[n_sweeps] (all > 0).  Builds J_perp (Q16.16) and the per-sweep
 * threshold tables and uploads everything. */
int pc_sqa_setup(pc_ctx *ctx, const int32_t *dims, const int8_t *J, int P, double T,
                 int n_sweeps, const double *gamma);
/* As pc_sqa_setup with per-axis boundary conditions and vacancies:
 * periodic [3] (host, nonzero = periodic, NULL = all periodic), present [N]
 * (host, 0 = vacancy, NULL = none), as for pc_apt_load_bc.  Slice energies
 * sum the present bonds. */
int pc_sqa_setup_bc(pc_ctx *ctx, const int32_t *dims, const uint8_t *periodic, const uint8_t *present,
                    const int8_t *J, int P, double T, int n_sweeps, const double *gamma);
/* Bytes pc_sqa_setup copies host -> device for N sites and n_sweeps sweeps:
 * the 16-bit coupling word of every site and the 40 threshold words of every
 * sweep (host function). */
int64_t pc_sqa_upload_bytes(int N, int n_sweeps);
/* Threshold table of sweep s: out[3][7] for n = s_{k-1} + s_{k+1} in
 * {-2, 0, 2} and intra-slice field I = 2c - 6; *jq = J_perp in Q16.16. */
int pc_sqa_get_table(pc_ctx *ctx, int sweep, uint32_t *out, int32_t *jq);
/* Anneal R independent runs (global run ids run0 .. run0+R-1) from random
 * states through the whole schedule.  Outputs (host, nullable): E_out
 * [R][P] final classical slice energies (full J, no J_perp term), spins_out
 * [R][P][N] final slice spins (lin order). */
int pc_sqa_run(pc_ctx *ctx, int R, uint32_t run0, int64_t *E_out, int8_t *spins_out);
/* Device-buffer variant: E_dev [R][P] int32 and best_dev [R][2] int32
 * (minimum slice energy, its slice index; lowest index on ties). */
int pc_sqa_run_dev(pc_ctx *ctx, int R, uint32_t run0, int32_t *E_dev, int32_t *best_dev);
/* As pc_sqa_run_dev, plus the replica-direction correlation of each run's
 * final state (Supplementary Fig. S17, C_r = (1/N) sum_i s_{i,0} s_{i,r}):
 * corr_dev [R][P] int32 (device, caller-owned) receives N * C_r, i.e.
 * sum over sites of s(site, slice 0) * s(site, slice r), r = 0..P-1 (r = 0
 * gives N).  PC_EINVAL if corr_dev is NULL with R > 0. */
int pc_sqa_run_corr_dev(pc_ctx *ctx, int R, uint32_t run0, int32_t *E_dev, int32_t *best_dev,
                        int32_t *corr_dev);
/* Self-test of the bounded waits of the time-sliced anneal schedule: runs
 * two runs from their second chunk, so that no wait for a previous chunk
 * can succeed; every wait gives up after 50 ms.  *status receives the
 * status the host then reports (PC_EDEVICE when the waits gave up as they
 * must); the context stays usable.  Needs a prior pc_sqa_setup with at
 * least 2 sweeps. */
int pc_sqa_selftest_wait(pc_ctx *ctx, int *status);
/* One call from host data to host results: setup + run + copy back. */
int pc_sqa_anneal(pc_ctx *ctx, const int32_t *dims, const int8_t *J, int P, double T,
                  int n_sweeps, const double *gamma, int R, uint32_t run0, int64_t *E_out);

/* The DT-SQA anneal without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * code whose device memory is all owned by another allocator (a framework's
 * caching allocator or a fixed arena) or code that must not allocate on a
 * latency-critical path.  It runs the same kernel as pc_sqa_run_dev with the
 * same results, but keeps its scratch (packed couplings and per-sweep
 * threshold tables) in a static device array of about 1.57 MiB that every
 * GPU loading this library holds until the process exits.
 *   device, stream   CUDA device and stream (NULL: legacy default stream).
 *   seed             Philox key.
 *   dims, J, P, T, n_sweeps, gamma   as pc_sqa_setup (host pointers).
 *   R, run0          as pc_sqa_run_dev.
 *   E_dev [R][P], best_dev [R][2] (nullable)   caller-owned device buffers.
 * Limits: n_sweeps <= 10240, N <= 4096 (else PC_EINVAL with a message).
 * No cudaMalloc, cudaFree or other allocating call is made.  The first call
 * on a device looks up the array's device address (under a host lock, so
 * concurrent first calls are safe).  Host data reaches the device as kernel
 * parameters of staging launches on `stream`, not as copies from host
 * memory.  All calls share the one array and leave it
 * holding the last call's tables, so calls that overlap on the GPU (e.g. on
 * two streams) race; issue them in one stream or serialise them. */
int pc_sqa_anneal_noalloc(int device, void *stream, uint64_t seed, const int32_t *dims,
                          const int8_t *J, int P, double T, int n_sweeps, const double *gamma,
                          int R, uint32_t run0, int32_t *E_dev, int32_t *best_dev);

/* ------------------------------------------------------------------------
 * Adaptive beta ladder (Algorithm S2 preprocessing; Methods: beta_0 = 0.5,
 * alpha = 1.25, 100 chains, 10^4 sweeps, variance from the last 10^3).
 * ---------------------------------------------------------------------- */
/* For each of n_inst instances (dims [n][3], J concatenated, Philox entry
 * entry0 + i): n_chains chains sweep `sweeps` times at beta_t (warm start),
 * sigma_E = sqrt(mean over chains of the unbiased variance of the last
 * `tail` post-sweep energies), beta_{t+1} = beta_t + alpha / sigma_E, until
 * sigma_E < tol.  Outputs [n][max_len] betas and sigmas, len [n], and
 * converged [n] (0 if max_len was reached first). */
int pc_adaptive_ladder(pc_ctx *ctx, int n_inst, const int32_t *dims, const int8_t *J,
                       uint32_t entry0, double beta0, double alpha, int n_chains, int sweeps,
                       int tail, double tol, int max_len, double *beta_out, double *sigma_out,
                       int32_t *len_out, int32_t *converged_out);
/* Piecewise-linear resampling of a ladder to n points in normalised index,
 * endpoints kept (host). */
int pc_resample_ladder(const double *beta, int len, int n, double *out);

/* ------------------------------------------------------------------------
 * Learned ladder: pilot histograms, features and the MLP predictor.
 * ---------------------------------------------------------------------- */
/* Energy histograms of a short pilot run: for each instance, n_beta
 * temperatures x chains_per_beta chains, post-sweep energies of sweeps
 * burn..sweeps-1, bin = floor(n_bins (E + 3N) / (3N)) clamped to
 * [0, n_bins-1].  counts [n][n_beta][n_bins]. */
int pc_pilot_hist(pc_ctx *ctx, int n_inst, const int32_t *dims, const int8_t *J,
                  uint32_t entry0, int n_beta, const double *betas, int chains_per_beta,
                  int sweeps, int burn, int n_bins, int64_t *counts);
/* [cbrt(N)/16, fraction of J > 0, fraction of frustrated plaquettes]. */
int pc_instance_features(const int32_t *dims, const int8_t *J, double *out3);

/* ------------------------------------------------------------------------
 * General sparse graphs.  Algorithms S1 and S2 take weights, biases and a
 * colormap; the Methods ("Graph Coloring of 3D Cubic Spin Glass Instances")
 * colour the p-bits with DSATUR, need 2 to 4 colours when spins are missing
 * or instances are embedded, and one more colour for the replicated DT-SQA
 * network when the number of replicas is odd.
 *
 * A graph of n p-bits is CSR on the host: the neighbours of v are
 * col[row_ptr[v] .. row_ptr[v+1]-1] (0-based, row_ptr[0] = 0) with int8
 * weights w (J_vu, nonzero, equal in both directions, each pair listed once
 * per direction, no self-loops); biases h [n] int8 or NULL.  Weights are
 * integers: fixed-point weights with f fractional bits are passed as
 * integers with beta scaled by 2^-f.  Limits: degree <= 1023, |h_v| +
 * sum_u |w_vu| <= 127, at most 32 colours.  A colormap colour [n] (values
 * 0..C-1, proper) may be given; NULL colours the graph with DSATUR.
 * Energies are E = -sum_{u<v} w_uv s_u s_v - sum_v h_v s_v (Eq. ising_energy).
 * ---------------------------------------------------------------------- */
/* DSATUR (Brelaz 1979): repeatedly colour the uncoloured vertex of largest
 * saturation (distinct colours among its coloured neighbours), ties by the
 * largest degree among uncoloured neighbours, then the smallest index, with
 * the smallest colour free at its neighbours.  colour [n] host output,
 * *n_colours = C.  PC_EINVAL for a malformed graph or more than 32 colours. */
int pc_graph_dsatur(int n, const int32_t *row_ptr, const int32_t *col, int32_t *colour,
                    int *n_colours);
/* Load n_prob APT problems on graphs (Algorithm S2): n_vert [n_prob];
 * row_ptr concatenated ([n_i + 1] each, local offsets), col and w
 * concatenated (local vertex ids), h concatenated or NULL, colour
 * concatenated or NULL (DSATUR per problem); n_temps [n_prob] <= 32, betas
 * concatenated (strictly increasing), n_labels in {1, 2, 4}.  Slot (r, a)
 * = temperature r, label a; replica id 32 a + r in the counters of problem
 * entry entry0 + i.  Shared memory holds a problem: 4 ((2 Imax + 1) 32 +
 * n (A + 2)) bytes must fit the device's per-block limit.  Draws the random
 * initial states and computes their energies; replaces any graph batch
 * loaded before (the lattice APT batch is separate). */
int pc_gapt_load(pc_ctx *ctx, int n_prob, const int32_t *n_vert, const int32_t *row_ptr,
                 const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
                 const int32_t *n_temps, const double *betas, int n_labels, uint32_t entry0);
/* n_swaps attempts, each: sweeps_per_swap sweeps (colour class by colour
 * class), energies, best tracking, ICM on every temperature when icm != 0
 * (n_labels 2 or 4, all h = 0) followed by best tracking, and the replica
 * exchange of pairs (r, r+1), r = t mod 2, t mod 2 + 2, ...  Resumable. */
int pc_gapt_run(pc_ctx *ctx, int64_t n_swaps, int sweeps_per_swap, int icm);
/* 0 (default): each label decides its swap; 1: one decision per pair with
 * the labels' summed dE (as pc_apt_set_joint_swap). */
int pc_gapt_set_joint_swap(pc_ctx *ctx, int joint);
/* Best-energy target of problem `prob` (time to target). */
int pc_gapt_set_target(pc_ctx *ctx, int prob, int64_t e_target);
/* Energies [n_temps * n_labels] in slot order r * n_labels + a. */
int pc_gapt_get_energies(pc_ctx *ctx, int prob, int64_t *E);
/* Spins [n_temps * n_labels][n] (+-1) in slot order, original vertex order. */
int pc_gapt_get_spins(pc_ctx *ctx, int prob, int8_t *spins);
/* The colormap in use [n] (given or DSATUR). */
int pc_gapt_get_colours(pc_ctx *ctx, int prob, int32_t *colour);
/* Best energy so far, sweep count when found, slot, target hit sweep (-1:
 * not yet), best state [n] (nullable; zeros before the first run). */
int pc_gapt_get_best(pc_ctx *ctx, int prob, int64_t *E, int64_t *sweep, int32_t *slot,
                     int64_t *hit_sweep, int8_t *spins);
/* Swap attempts / accepts [n_temps-1][n_labels]; icm [3] as pc_apt_get_stats. */
int pc_gapt_get_stats(pc_ctx *ctx, int prob, int64_t *att, int64_t *acc, int64_t *icm);
/* Adaptive beta ladder on graphs (Algorithm S2 preprocessing, as
 * pc_adaptive_ladder): for each of n_prob graphs (arrays as pc_gapt_load,
 * Philox entry entry0 + i) n_chains <= 128 chains sweep `sweeps` times at
 * beta_t (warm start), sigma_E = sqrt(mean over chains of the unbiased
 * variance of the last `tail` post-sweep energies), beta_{t+1} = beta_t +
 * alpha / sigma_E, until sigma_E < tol.  Chain b draws as APT replica id b
 * with the ladder's own counter tags.  Outputs [n_prob][max_len] betas and
 * sigmas (sigma_out nullable), len [n_prob], converged [n_prob] (nullable;
 * 0 if max_len was reached first).  Leaves any loaded graph batch alone. */
int pc_graph_adaptive_ladder(pc_ctx *ctx, int n_prob, const int32_t *n_vert, const int32_t *row_ptr,
                             const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
                             uint32_t entry0, double beta0, double alpha, int n_chains, int sweeps,
                             int tail, double tol, int max_len, double *beta_out, double *sigma_out,
                             int32_t *len_out, int32_t *converged_out);
/* DT-SQA on a graph (Eq. S.3, Algorithm S1): R runs (ids run0 ..) of P >= 2
 * slices at temperature T under gamma[n_sweeps] (all > 0).  The replicated
 * network takes colour (colour[v] + f(k)) mod C' for slice k, f(k) = k & 1
 * except f(P-1) = 2 for odd P, C' = max(C, 2) (even P) or max(C, 3) (odd P).
 * E_out [R][P] classical slice energies (biases included); spins_out
 * [R][P][n] or NULL.  A run group's P n words of state live in shared
 * memory: in one CTA when they fit, else split by slices over a cluster of
 * 2, 4 or 8 CTAs (P n 4 bytes / 8 must fit one CTA).  run0 is a multiple of
 * 8 (one Philox call serves runs 8g .. 8g+7). */
int pc_gsqa_anneal(pc_ctx *ctx, int n, const int32_t *row_ptr, const int32_t *col,
                   const int8_t *w, const int8_t *h, const int32_t *colour, int P, double T,
                   int n_sweeps, const double *gamma, int R, uint32_t run0, int64_t *E_out,
                   int8_t *spins_out);

/* Judge of beta ladders by their swap-acceptance profile.  For each of
 * n_inst periodic lattices (dims [n][3], J concatenated) with the ladder
 * betas [n][n_temps] (strictly increasing), runs the first probe_attempts
 * APT attempts (one sweep, ICM when n_labels >= 2, the swaps; Algorithm S2)
 * on a scratch batch whose problem i draws with entry entry0 + i, exactly as
 * a pc_apt_load of that ladder followed by pc_apt_run would (the loaded APT
 * batch is not touched).  acc_out [n][n_temps-1] (nullable) receives each
 * pair's acceptance pooled over the labels, accepts / attempts (-1 for a
 * pair the probe never attempted); pass_out [n] is 1 iff every attempted
 * pair reaches acc_floor, i.e. accepts >= acc_floor * attempts in double.
 * The adaptive procedure spaces temperatures so that dbeta sigma_E = alpha,
 * a flat acceptance of erfc(alpha / 2) for Gaussian energies (about 0.38 at
 * the paper's alpha = 1.25; Supplementary "Temperature profile and swap
 * acceptance rate in APT": flat except the last pairs); erfc(1.25 alpha) =
 * 0.027, the acceptance of a gap 2.5 times the adaptive one, is the floor
 * the library's tools use. */
int pc_ladder_judge(pc_ctx *ctx, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
                    int n_temps, const double *betas, int n_labels, int probe_attempts, double acc_floor,
                    double *acc_out, int32_t *pass_out);

/* MLP 259 -> 256 -> 256 -> 256 -> 32 (ReLU hidden), head
 * beta_k = beta_min + sum_{m<=k} softplus(o_m), loss = mean (beta - y)^2
 * + gap_weight * mean_{k>=1} ((softplus(o_k) - d_k) / d_k)^2 with d_k =
 * y_k - y_{k-1} the target's gaps (gap_weight 0 unless set), fp32 on the
 * GPU, Adam.  W[l] is [out][in] row-major, b[l] is [out]. */
typedef struct pc_mlp pc_mlp;
int pc_mlp_create(pc_ctx *ctx, pc_mlp **out, const float *const *W, const float *const *b,
                  float beta_min);
/* Frees the network; it may be called after its context was destroyed
 * (every other pc_mlp_* call needs the context alive). */
void pc_mlp_destroy(pc_mlp *m);
/* X [batch][259] -> beta [batch][32] (host). */
int pc_mlp_forward(pc_mlp *m, int batch, const float *X, float *beta);
/* Loss and gradients without updating (host outputs, [out][in] / [out]). */
int pc_mlp_grads(pc_mlp *m, int batch, const float *X, const float *Y, float *loss,
                 float *const *gW, float *const *gb);
/* One Adam step (lr, b1 = 0.9, b2 = 0.999, eps = 1e-8) on a minibatch;
 * *loss = loss before the step (nullable). */
int pc_mlp_train_step(pc_mlp *m, int batch, const float *X, const float *Y, float lr,
                      float *loss);
/* Device-buffer training step: X_dev [batch][259], Y_dev [batch][32]. */
int pc_mlp_train_step_dev(pc_mlp *m, int batch, const float *X_dev, const float *Y_dev,
                          float lr, float *loss_dev);
int pc_mlp_get_params(pc_mlp *m, float *const *W, float *const *b);
/* Weight of the relative-gap term of later training steps and gradients
 * (>= 0).  A pair's swap acceptance depends on its gap, and the squared
 * error of the cumulative ladder alone barely penalises gap errors that
 * cancel between neighbours. */
int pc_mlp_set_gap_weight(pc_mlp *m, float w);
/* Weights file of the network: the bytes "PCMLP001", the five layer widths
 * (int32), beta_min (fp32), then W[l] and b[l] of each layer (fp32,
 * little-endian).  pc_mlp_load creates a network on ctx from such a file
 * (PC_EINVAL if the file is missing, truncated or of another shape). */
int pc_mlp_save(pc_mlp *m, const char *path);
int pc_mlp_load(pc_ctx *ctx, const char *path, pc_mlp **out);

/* Learned beta ladder: the network above in place of the adaptive
 * procedure of Algorithm S2's preprocessing (Methods "APT details"), with
 * that procedure kept as judge and fallback.  The paper has no learned
 * component; it observes that ladders of one size are nearly identical
 * across instances (Fig. S12), which makes them predictable from cheap
 * features.  Options: */
typedef struct {
  const double *pilot_betas;  /* [4] pilot temperatures, those the network was trained with */
  int pilot_chains;           /* chains per pilot temperature (4 * pilot_chains <= 64) */
  int pilot_sweeps;           /* pilot sweeps; energies of sweeps >= pilot_burn are counted */
  int pilot_burn;
  int probe_attempts;         /* judge's APT attempts; 0: no judge and no fallback */
  int probe_labels;           /* labels per temperature of the probe (1, 2 or 4) */
  double acc_floor;           /* least pooled swap acceptance of every pair (pc_ladder_judge) */
  double beta0, alpha;        /* fallback: pc_adaptive_ladder with these settings, */
  int n_chains, sweeps, tail; /* resampled to 32 points (pc_resample_ladder) */
  double tol;
  int max_len;
} pc_learned_opts;
/* For each of n_inst periodic lattices (dims [n][3], J concatenated; the
 * instance i draws with entry entry0 + i), all on the device:
 *   1. pilot histograms as pc_pilot_hist (4 temperatures, 64 bins);
 *   2. features: cbrt(N)/16, the fraction of J > 0, the fraction of
 *      frustrated plaquettes, and each pilot temperature's histogram divided
 *      by its total (fp32);
 *   3. the network m (created on ctx) gives 32 betas;
 *   4. ladder k becomes max(b_0, 0), then max(b_k, beta_{k-1} + 1e-6), in
 *      double, so that it is strictly increasing;
 *   5. with probe_attempts > 0, pc_ladder_judge of these ladders
 *      (probe_labels, probe_attempts, acc_floor; acc_out [n][31] nullable);
 *   6. every rejected instance falls back to pc_adaptive_ladder (same entry
 *      id) resampled to 32 points, and fallback_out [n] (nullable) is 1.
 * beta_out [n][32] receives the ladders (host); ready_s [n] (nullable) the
 * seconds (host clock) from the call's start until each instance's ladder
 * was final: after the judge, or after its fallback. */
int pc_learned_ladder(pc_ctx *ctx, pc_mlp *m, int n_inst, const int32_t *dims, const int8_t *J,
                      uint32_t entry0, const pc_learned_opts *opt, double *beta_out, double *acc_out,
                      int32_t *fallback_out, double *ready_s);
/* Steps 1 and 2 alone (the pilot fields of opt): the network's inputs
 * X_out [n][259] fp32 (host), as pc_learned_ladder computes them; used to
 * build training sets. */
int pc_learned_features(pc_ctx *ctx, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
                        const pc_learned_opts *opt, float *X_out);


#ifdef __cplusplus
}
#endif
#endif
