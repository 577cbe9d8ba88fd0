// Host-side declarations shared by the C-ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcomp.h"

namespace pc {

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
// Status of the exception being handled (call inside a catch block only):
// PC_ENOMEM for failed host allocations, PC_EINVAL otherwise.  Every C-ABI
// entry point ends in a handler that calls it, so no exception leaves the
// library.
int fail_exception();

#define PC_CUDA_TRY(call)                                                          \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ::pc::fail(PC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------- lattice
struct Lattice {
  int L[3];
  int N;
};
// jneg byte of every site: bit d set iff the coupling on direction d
// (0:+x 1:-x 2:+y 3:-y 4:+z 5:-z) is -1.
std::vector<uint8_t> pack_jneg(const Lattice &lat, const int8_t *J);
// Per site (lin order): bits 0-5 coupling signs as pack_jneg for the bonds
// present, bits 8-13 the absent bonds, bit 15 a vacancy.  A bond is absent
// across the ends of an open axis (per[a] = 0) and next to a vacancy
// (present[s] = 0, a missing spin; present may be NULL).  *nbonds and
// *nreal receive the bonds and spins present.
std::vector<uint16_t> pack_jn16(const Lattice &lat, const uint8_t per[3], const uint8_t *present,
                                const int8_t *J, int *nbonds, int *nreal);
int check_lattice(const int32_t *dims, const int8_t *J, Lattice *out);
uint32_t recip32(uint32_t d);   // ceil(2^32 / d)
uint32_t sqa_threshold(double beta_eff, int I, int32_t jq, int n);

// ---------------------------------------------------------------- DT-SQA
constexpr int kSqaTab = 40;   // threshold words per sweep: [3 m][13 I] (+1 pad)
struct SqaArgs {
  int Lx, Ly, Lz, N, P, NB, S;
  uint32_t mLx, mLy;       // reciprocals of Lx and Ly
  uint32_t run0, k0, k1;
  const uint16_t *jneg;    // [N] pack_jn16 words
  int nbonds;              // bonds present (3N with periodic axes)
  const uint32_t *table;   // [S][40]: index I + 6 + 13 m (I = -6..6, m = 0..2)
  int32_t *E;              // [R][P]
  int32_t *best;           // [R][2] (nullable)
  int8_t *spins;           // [R][P][N] (nullable)
  int32_t *corr;           // [R][P] sum_s s(s,0) s(s,k) (nullable)
  // persistent time-sliced schedule (state == nullptr: one CTA per run)
  uint32_t *state;         // [R][2][NB][N] run states between chunks
  int *done, *queue, *err; // [R] chunks done per run; work counter; error flag
  int R, K, n_items;       // runs, sweeps per chunk, R * chunks
  int first_item;          // first queue item (0; the wait self-test skips chunk 0)
  uint64_t wait_ns;        // limit of one wait for a previous chunk
};
size_t sqa_smem_bytes(int N, int P);
int sqa_launch(const SqaArgs &a, int R, cudaStream_t st);

// ---------------------------------------------------------------- MLP (mlp.cu)
pc_ctx *mlp_context(pc_mlp *m);
// The network's device input buffer [batch][259], grown as needed.
int mlp_input(pc_mlp *m, int batch, float **X_dev);
// Forward pass of the input buffer; *beta_dev receives [batch][32] fp32
// ladders on the device, valid until the next call on m.
int mlp_forward_input(pc_mlp *m, int batch, const float **beta_dev);

// ---------------------------------------------------------------- Philox check
int philox_launch(const uint32_t *ctr, uint32_t *out, int64_t n, uint32_t k0, uint32_t k1,
                  cudaStream_t st);

}  // namespace pc
