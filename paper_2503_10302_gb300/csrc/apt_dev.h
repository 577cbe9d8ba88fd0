// Device-side descriptors of the adaptive-parallel-tempering kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace pc {

enum : int { APT_MODE_APT = 0, APT_MODE_LADDER = 1, APT_MODE_PILOT = 2, APT_MODE_ENERGY = 3 };

// One problem (lattice + replicas) of a batch; offsets index the batch-wide
// arrays of AptArgs.
struct AptProbDev {
  int Lx, Ly, Lz, N;
  uint32_t mhx, mLy;      // ceil(2^32 / (Lx/2)), ceil(2^32 / Ly)
  uint32_t mLy2;          // ceil(2^32 / (Ly/2))
  uint32_t open;          // bit a < 3: axis a open (no wrap-around bonds); bit 3: vacancies
  int nbonds;             // bonds present (3N when every axis is periodic)
  int nreal;              // spins present (N without vacancies)
  int T, Tp, A, B;        // temperatures, padded temperatures 8*ceil(T/8), labels,
                          // buffers (APT: A * Tp; ladder / pilot: chains)
  uint32_t ent;           // Philox entry id
  uint32_t spin_off;      // words: [G][2][N/2]
  uint32_t jneg_off;      // [2][N/2] per (colour, j): bits 0-5 coupling signs, 8-13 missing bonds
  uint32_t pbit_off;      // words: [T][16] p-bit thresholds, index I + 6 for I = -6..6
  uint32_t swapidx_off;   // words: [T-1][2] (offset, length) of each pair's swap table
  uint32_t buf_off;       // per-buffer arrays (temp_of, buf_of, E, sums)
  uint32_t best_off;      // bytes: best state [N] in lin order
  uint32_t stat_off;      // int64: att [(T-1)A], acc [(T-1)A], icm [3]
  uint32_t hist_off;      // int64: [T][n_bins]
};

struct AptArgs {
  const AptProbDev *prob;
  const int *cta_prob, *cta_g0, *cta_gc, *cta_nch;
  uint32_t *spins;
  const uint16_t *jneg;
  const uint32_t *pbit, *swaptab, *swapidx;
  int32_t *temp_of, *buf_of, *E;
  int64_t *best_E, *best_sweep, *hit_sweep;
  const int64_t *target;
  int32_t *best_buf;
  int8_t *best_spins;
  int8_t *best_spins2;    // best-state candidates of rank 1 (split problems), same layout
  int64_t *stats;
  int64_t *sum1, *sum2;   // ladder: per-buffer sums of E and E^2
  int64_t *hist;          // pilot histograms
  int n_bins;
  int mode, n_iter, spp, icm;
  int joint_swap;         // 1: one swap decision per temperature pair for all labels
  int icm_big;            // 1: ICM flips one whole replica when the cluster holds more than half
  int icm_seed;           // 0: ICM seeds at a uniform mismatch site; 1: at a uniform cluster
  int prio;               // host side only: launch priority of a cluster launch (0: default)
  int stage_swt;          // split problems keep the first swap-table entries in shared memory
  int split;              // 1: every problem runs as a cluster of two CTAs (by temperature)
  int64_t *ctr;           // [2]: sweeps and swap attempts done before this launch
  int64_t window_from;
  uint32_t tag_init, tag_main, tag_ref;
  uint32_t k0, k1;
};

size_t apt_smem_bytes(int N, int Gc, int nwarps, int mode, int icm, int T, int n_bins, int stage_swt);
int apt_launch(const AptArgs &a, int n_cta, int tpb, size_t smem, cudaStream_t st);
int apt_init_launch(const AptArgs &a, int n_prob, int max_words, cudaStream_t st);
// ctr[0] += sweeps, ctr[1] += swaps (stream-ordered after a launch).
int apt_advance_launch(int64_t *ctr, int64_t sweeps, int64_t swaps, cudaStream_t st);

// Learned-ladder steps (learned.cu): features [n_inst][ldx] fp32 of a pilot
// batch (instance features, then the normalised histograms of its n_beta
// temperatures), and strictly increasing double ladders from fp32 ones.
int learned_features_launch(const AptProbDev *prob, int n_inst, const uint16_t *jneg, const int64_t *hist,
                            int n_beta, int n_bins, float *X, int ldx, cudaStream_t st);
int ladder_monotone_launch(int n, int len, const float *b, double gap, double *out, cudaStream_t st);

}  // namespace pc
