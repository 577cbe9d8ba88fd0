// Device-side description of p-computer problems on general sparse graphs
// (Algorithms S1 and S2 with weights, biases and a colormap), shared by the
// host layer (graph_api.cpp) and the kernels (graph.cu).
//
// Vertices are renumbered colour-major: class c holds the vertices of colour
// c in increasing original index, at new indices off[c] .. off[c+1]-1, so the
// colour-local index of new vertex p is p - off[c] and the canonical ICM
// order is increasing p.
//
//   vinfo[p] = {start, deg | kl << 10 | (h & 0xFF) << 20}
//     start: first adjacency entry; deg: neighbours; kl: neighbours of a
//     lower colour (they come first: adjacency is sorted by new index);
//     h: the bias, int8.
//   adj[e]   = (o << 8) | (w & 0xFF): weight int8 and o = the byte offset of
//     neighbour u's first spin word (4 A u in APT with A labels, 4 u in
//     DT-SQA).
//   spins    : word [p][a] holds label a's bit for 32 temperatures (lane r =
//     temperature r, bit set = spin +1); unused temperatures stay 0.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace pc {

constexpr int kGMaxColours = 32;
constexpr int kGMaxDeg = 1023;
constexpr int kGMaxImax = 127;
constexpr int kGThreads = 512;
// counter tags of the APT and adaptive-ladder draws on graphs
constexpr uint32_t kTagGInit = 15, kTagGSweep = 16, kTagGRefine = 17;
constexpr uint32_t kTagGLInit = 23, kTagGLSweep = 24, kTagGLRefine = 25;
constexpr int kGWarps = kGThreads / 32;

struct GProbDev {
  int n, C, T, A, Imax, m;
  uint32_t ent;                 // problem entry of the counters
  uint32_t vbase;               // first vertex in vinfo / spins ([n][A] words from vbase * A)
  uint32_t abase;               // first adjacency entry
  uint32_t thbase;              // first word of the [32][2 Imax + 1] p-bit table
  uint32_t swbase;              // first (offset, length) pair in swapidx
  uint32_t bestbase;            // first word of the best-state bits
  uint32_t statbase;            // first counter: att[T-1][A], acc[T-1][A], icm[3]
  int off[kGMaxColours + 1];
};

struct GAptArgs {
  const GProbDev *prob;
  const int2 *vinfo;
  const uint32_t *adj;
  const uint32_t *pbit;         // [32][2 Imax + 1] per problem (zero rows for r >= T)
  const uint32_t *swaptab;      // thresholds by |dE| (entry 0: always accepted)
  const uint32_t *swapidx;      // per pair: offset, length
  uint32_t *spins;              // [n][A] words per problem
  int32_t *E;                   // [n_prob][4][32]
  uint32_t *best_bits;          // [ceil(n/32)] words per problem
  long long *best;              // [n_prob][4]: E, sweep, slot, hit sweep
  const long long *target;      // [n_prob]
  unsigned long long *stats;    // counters per problem
  uint32_t k0, k1;
  uint32_t sweep0, swap0;       // counters of the first sweep / attempt of this launch
  int n_swaps, spp, icm, joint;
  // counter tags of the initial-state and sweep draws
  uint32_t tag_init, tag_sweep, tag_refine;
  // adaptive-ladder mode (ladder != 0): no ICM, best tracking or swaps; the
  // energies of attempts t >= window_from accumulate into sum1 / sum2
  // ([n_prob][128], slot 32 a + r); problems with active[i] == 0 are skipped
  int ladder, window_from;
  long long *sum1, *sum2;
  const int *active;
};

struct GSqaArgs {
  int n, P, Cp, S, Imax, R, m;  // vertices, slices, colours, sweeps, field bound, runs, adjacency entries
  uint32_t run0, k0, k1;
  const int2 *vinfo;            // as above
  const uint32_t *adj;
  const uint32_t *cls;          // [P n]: class-major list of (k << 20) | p
  const int *cls_off;           // [Cp + 1]
  const uint32_t *table;        // [S][3][2 Imax + 1]
  long long *E;                 // [R][P]
  uint32_t *spins;              // [ceil(R/32)][P][n] words (nullable)
  int CS;                       // CTAs per run group (cluster size; 1: one CTA holds all slices)
  const int *cls_rank;          // [Cp][CS + 1]: class-list offsets of each CTA's slices (CS > 1)
};

// m < 0: vertex table and adjacency read from global memory; m >= 0: staged
// in shared memory as well (m adjacency entries).
size_t gapt_smem_bytes(int n, int A, int Imax, int m);
// Imax: the batch's largest field bound (selects the bit-plane count).
int gapt_launch(const GAptArgs &a, int n_prob, int A, int Imax, bool staged, size_t smem, bool init,
                cudaStream_t st);
size_t gsqa_smem_bytes(int n, int P, int Imax, int m, int CS);
// staged: vertex table and adjacency in shared memory (m >= 0 in gsqa_smem_bytes)
int gsqa_launch(const GSqaArgs &a, bool staged, size_t smem, cudaStream_t st);

}  // namespace pc
