// Device building blocks shared by the sweep kernels: the counter-based
// generator, the 8-spin acceptance decision and lattice index helpers.
#pragma once
#include <cstdint>

namespace pcdev {

// Counter tags of the randomness contract (each draw site has its own).
enum : uint32_t {
  TAG_APT_INIT = 1, TAG_APT_SWEEP = 2, TAG_APT_REFINE = 3, TAG_SWAP = 4, TAG_ICM = 5,
  TAG_LAD_INIT = 6, TAG_LAD_SWEEP = 7, TAG_LAD_REFINE = 8,
  TAG_PIL_INIT = 9, TAG_PIL_SWEEP = 10, TAG_PIL_REFINE = 11,
  TAG_SQA_INIT = 12, TAG_SQA_SWEEP = 13, TAG_SQA_REFINE = 14
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Per round the two
// 32x32->64 products of (c0, c2) by the multipliers are mixed with (c1, c3)
// and the round key; the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ k0;
    c2 = hi0 ^ c3 ^ k1;
    c1 = lo1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t word_of(const uint4 &x, int w) {
  return w == 0 ? x.x : (w == 1 ? x.y : (w == 2 ? x.z : x.w));
}

// Half-word i of a Philox block placed in the high 16 bits (low bits 0).
__device__ __forceinline__ uint32_t half_hi(const uint4 &x, int i) {
  const uint32_t w = word_of(x, i >> 1);
  return (i & 1) ? (w & 0xFFFF0000u) : (w << 16);
}
__device__ __forceinline__ uint32_t half_lo(const uint4 &x, int i) {
  const uint32_t w = word_of(x, i >> 1);
  return (i & 1) ? (w >> 16) : (w & 0xFFFFu);
}

// Eq. neuron for 8 spins at once.  Spin i (nibble i) becomes +1 iff its
// 32-bit uniform u_i = (main half i << 16) | (refine half i) is below its
// threshold.  Thresholds come from a shared-memory table indexed by the byte
// i/2 of De (even i) or Do (odd i); `Th` holds the table with the low 16
// bits cleared.  The main half decides unless it equals the top half of the
// threshold (probability 2^-16); then `tie` is set and the caller settles
// those nibbles exactly with refine8.
__device__ __forceinline__ uint32_t lut_index(uint32_t De, uint32_t Do, int i) {
  return (((i & 1) ? Do : De) >> (8 * (i >> 1))) & 0x1Fu;
}

__device__ __forceinline__ uint32_t decide8(const uint4 &x, uint32_t De, uint32_t Do,
                                            const uint32_t *Th, bool &tie) {
  uint32_t w = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t v = half_hi(x, i), th = Th[lut_index(De, Do, i)];
    w |= (v < th) ? (1u << (4 * i)) : 0u;
    tie |= (v == th);
  }
  return w;
}

// Exact settlement of the tied nibbles with the refine block y; T is the
// full 32-bit table.
static __device__ __noinline__ uint32_t refine8(uint32_t w, uint4 x, uint4 y, uint32_t De, uint32_t Do,
                                         const uint32_t *T) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t t = T[lut_index(De, Do, i)];
    const uint32_t v = half_hi(x, i);
    if (v == (t & 0xFFFF0000u)) {
      const uint32_t u = v | half_lo(y, i);
      w = (u < t) ? (w | (1u << (4 * i))) : (w & ~(1u << (4 * i)));
    }
  }
  return w;
}

// Exact n / d for n < 2^16, 2 <= d < 2^16 via a 32-bit reciprocal
// m = ceil(2^32/d); d = 1 has no 32-bit reciprocal and is passed as m = 0.
__device__ __forceinline__ uint32_t fdiv(uint32_t n, uint32_t m) { return m ? __umulhi(n, m) : n; }

__device__ __forceinline__ uint32_t nib_mask(uint32_t bit) { return bit * 0x11111111u; }

}  // namespace pcdev
