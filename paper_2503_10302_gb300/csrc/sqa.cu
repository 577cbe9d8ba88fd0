// Discrete-time simulated quantum annealing (Suzuki-Trotter mapping, Eq. S.3;
// Algorithm S1) as one persistent CTA per independent run.
//
// Layout.  A run is the (d+1)-dimensional lattice of P slices of the 3D
// lattice.  Its 4D checkerboard colour is c = (x + y + z + k) & 1, so at a
// 3D site s of parity q the slices of colour c are k = 2m + (c ^ q).  Eight
// consecutive m of one (colour, site) share a 32-bit word, one spin per
// nibble (bit 0 = spin +1), block b = m >> 3.  Shared memory holds
// W[c][s][b] for the whole run (N * P / 2 bytes; the NB words of a site are
// contiguous, so they move as one vector access).  With this packing
//  - the six spatial neighbours of a word are the words of the other colour
//    at the neighbouring sites with the SAME block: nibble-aligned, and the
//    coupling J (common to all slices) is one mask per direction;
//  - the two imaginary-time neighbours are the other colour's word at the
//    same site and that word shifted by one nibble (carry from block b +- 1).
// So one word yields 8 nibble-packed satisfied-bond counts (0..6) and 8
// time-neighbour counts (0..2) with a handful of 32-bit ops, and one
// Philox4x32-10 call supplies the 8 16-bit uniforms.
#include <cuda_runtime.h>

#include <mutex>

#include "device.cuh"
#include "internal.h"

// Build-time tuning knobs of the anneal kernel (defaults are the tuned
// values): keep one site's constants in registers across sweeps, unroll the
// loop over slice blocks, CTAs per SM the register budget is sized for.
#ifndef PC_SQA_HOIST
#define PC_SQA_HOIST 1
#endif
#ifndef PC_SQA_UNROLL
#define PC_SQA_UNROLL 1
#endif
#ifndef PC_SQA_MINB
#define PC_SQA_MINB 1
#endif
#ifndef PC_SQA_TPB
#define PC_SQA_TPB 512
#endif

namespace {
using namespace pcdev;

// Site coordinates of a 3D site index.
struct Site {
  int s, x, y, z, q;
  uint32_t jb;
};

__device__ __forceinline__ Site site_of(const pc::SqaArgs &a, int s, const uint16_t *jn) {
  Site t;
  t.s = s;
  const int r = (int)fdiv((uint32_t)s, a.mLx);   // s / Lx
  t.x = s - r * a.Lx;
  t.z = (int)fdiv((uint32_t)r, a.mLy);           // r / Ly
  t.y = r - t.z * a.Ly;
  t.q = (t.x + t.y + t.z) & 1;
  t.jb = jn[s];
  return t;
}

// Neighbour of site t along direction d (0:+x 1:-x 2:+y 3:-y 4:+z 5:-z),
// periodic boundaries.
__device__ __forceinline__ int neighbour(const pc::SqaArgs &a, const Site &t, int d) {
  const int LxLy = a.Lx * a.Ly;
  switch (d) {
    case 0: return (t.x + 1 == a.Lx) ? t.s - (a.Lx - 1) : t.s + 1;
    case 1: return (t.x == 0) ? t.s + (a.Lx - 1) : t.s - 1;
    case 2: return (t.y + 1 == a.Ly) ? t.s - (a.Ly - 1) * a.Lx : t.s + a.Lx;
    case 3: return (t.y == 0) ? t.s + (a.Ly - 1) * a.Lx : t.s - a.Lx;
    case 4: return (t.z + 1 == a.Lz) ? t.s - (a.Lz - 1) * LxLy : t.s + LxLy;
    default: return (t.z == 0) ? t.s + (a.Lz - 1) * LxLy : t.s - LxLy;
  }
}

// Nibble-packed counts, per block, of satisfied terms J_d s_nbr = +1 over
// the spatial bonds present (Eq. synapse with I = 2C - deg).  XOR with the
// all-nibbles mask turns a neighbour spin into J_d s_nbr for J_d = -1.
template <int NB>
__device__ __forceinline__ void spatial_counts(const pc::SqaArgs &a, const uint32_t *Wo,
                                               const Site &t, uint32_t (&C)[NB]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) C[b] = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if ((t.jb >> (8 + d)) & 1u) continue;   // absent bond (open axis)
    const int n = neighbour(a, t, d);
    const uint32_t m = nib_mask((t.jb >> d) & 1u);
#pragma unroll
    for (int b = 0; b < NB; ++b) C[b] += Wo[(size_t)n * NB + b] ^ m;
  }
}

// Per-site constants of the sweep: neighbour indices and the coupling
// signs.  With s_nbr in {0,1} per nibble, J s_nbr "satisfied" is s_nbr for
// J = +1 and 1 - s_nbr for J = -1, so the packed count of satisfied terms is
// C = K + sum_d eps_d W_d with eps_d = +-1 and K = 0x11111111 * #(J = -1):
// six multiply-adds per word.
struct SiteK {
  int nb[6];
  int eps[6];        // +-1, 0 for an absent bond
  uint32_t K;
  uint32_t kb;       // absent bonds k: 2k in every byte (threshold index I + 6 = 2C + k)
  int q;
};

__device__ __forceinline__ SiteK site_consts(const pc::SqaArgs &a, int s, const uint16_t *jn) {
  const Site t = site_of(a, s, jn);
  SiteK k;
  k.q = t.q;
  int nneg = 0, nmiss = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    k.nb[d] = neighbour(a, t, d);
    const int neg = (t.jb >> d) & 1, miss = (t.jb >> (8 + d)) & 1;
    k.eps[d] = miss ? 0 : 1 - 2 * neg;
    nneg += miss ? 0 : neg;
    nmiss += miss;
  }
  k.K = 0x11111111u * (uint32_t)nneg;
  k.kb = 0x01010101u * (uint32_t)(2 * nmiss);
  return k;
}

// Threshold tables in static shared memory, so that a byte of a packed
// index word is directly an address offset: [2 sweeps][40 entries], entry
// I + 6 + 13 m for in-slice field I = -6..6 and time count m = 0..2;
// top halves (Th, 16-bit, 2-byte steps) and full values (Tf).
__shared__ __align__(16) uint16_t s_Th[2][pc::kSqaTab];
__shared__ __align__(16) uint32_t s_Tf[2][pc::kSqaTab];

// Eq. neuron for the 8 nibbles of one word.  Byte k of Dlo / Dhi is the
// byte offset of the threshold of nibble 2k / 2k+1 in s_Th (index * 2 plus
// 80 for the odd sweep's buffer).  The main half v decides against the top
// half t of the threshold: d = v - t is negative iff v < t, and d = 0 is a
// tie, which the main half cannot decide.
__device__ __forceinline__ uint32_t decide_word(const uint4 &x, uint32_t Dlo, uint32_t Dhi, bool &tie) {
  uint32_t w = 0;
  uint32_t tp = 1u;   // product of the differences (mod 2^32): 0 when some half equals its threshold
  const char *base = reinterpret_cast<const char *>(&s_Th[0][0]);
#pragma unroll
  for (int i = 7; i >= 0; --i) {
    const uint32_t off = __byte_perm((i & 1) ? Dhi : Dlo, 0u, 0x4440u + (uint32_t)(i >> 1));
    const uint32_t th = *reinterpret_cast<const uint16_t *>(base + off);
    const uint32_t xw = word_of(x, i >> 1);
    const uint32_t v = (i & 1) ? (xw >> 16) : (xw & 0xFFFFu);
    const uint32_t d = v - th;   // both below 2^16: bit 31 set iff v < th
    // the top 4 bits of d enter w as its new nibble 0, so after the loop
    // bit 3 of nibble i is the sign of half i's difference
    w = __funnelshift_l(d, w, 4);
    tp *= d;
  }
  // a zero product flags a tie; a product that merely wraps to 0 only sends
  // the word through settle_ties, which rechecks every half exactly
  tie |= (tp == 0);
  return (w >> 3) & 0x11111111u;
}

__device__ __noinline__ uint32_t settle_ties(uint32_t w, uint4 x, uint4 y, uint32_t Dlo, uint32_t Dhi) {
  const char *base = reinterpret_cast<const char *>(&s_Tf[0][0]);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t off = __byte_perm((i & 1) ? Dhi : Dlo, 0u, 0x4440u + (uint32_t)(i >> 1));
    const uint32_t t = *reinterpret_cast<const uint32_t *>(base + 2 * off);
    const uint32_t v = half_hi(x, i);
    if (v == (t & 0xFFFF0000u)) {
      const uint32_t u = v | half_lo(y, i);
      w = (u < t) ? (w | (1u << (4 * i))) : (w & ~(1u << (4 * i)));
    }
  }
  return w;
}

// NB consecutive words as one vector access (NB = 1, 2, 4, 8; else scalar).
template <int NB>
__device__ __forceinline__ void load_words(const uint32_t *p, uint32_t (&v)[NB]) {
  if constexpr (NB % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NB; q += 4) {
      const uint4 t = *reinterpret_cast<const uint4 *>(p + q);
      v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
    }
  } else if constexpr (NB % 2 == 0) {
#pragma unroll
    for (int q = 0; q < NB; q += 2) {
      const uint2 t = *reinterpret_cast<const uint2 *>(p + q);
      v[q] = t.x; v[q + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NB; ++q) v[q] = p[q];
  }
}
template <int NB>
__device__ __forceinline__ void store_words(uint32_t *p, const uint32_t (&v)[NB]) {
  if constexpr (NB % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NB; q += 4)
      *reinterpret_cast<uint4 *>(p + q) = make_uint4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  } else if constexpr (NB % 2 == 0) {
#pragma unroll
    for (int q = 0; q < NB; q += 2) *reinterpret_cast<uint2 *>(p + q) = make_uint2(v[q], v[q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < NB; ++q) p[q] = v[q];
  }
}

// All NB words of one (site, colour) in one sweep.
template <int NB>
__device__ __forceinline__ void update_site(const pc::SqaArgs &a, const uint32_t *Wo, uint32_t *Wc,
                                            int s, const SiteK &k, int c, uint32_t sw,
                                            uint32_t boff, uint32_t ent) {
  const int e = c ^ k.q;   // slice parity of this word's nibbles
  const uint32_t c2 = (uint32_t)c << 16;
  uint32_t O[NB], C[NB], w[NB];
  load_words<NB>(Wo + (size_t)s * NB, O);
#pragma unroll
  for (int b = 0; b < NB; ++b) C[b] = k.K;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    uint32_t Nw[NB];
    load_words<NB>(Wo + (size_t)k.nb[d] * NB, Nw);
#pragma unroll
    for (int b = 0; b < NB; ++b) C[b] += (uint32_t)k.eps[d] * Nw[b];
  }
  // time neighbours k-1, k+1 of word b: the other colour's word and that
  // word shifted by one nibble (funnel shift through the adjacent block);
  // byte offsets 2 (2C + k + 13 m) + 80 (odd sweep): at most 156
  const uint32_t kb = k.kb + boff;
  auto offsets = [&](int b, uint32_t &Dlo, uint32_t &Dhi) {
    const int bp = (b + 1 == NB) ? 0 : b + 1, bm = (b == 0) ? NB - 1 : b - 1;
    const uint32_t lo = e ? O[b] : O[bm];
    const uint32_t hi = e ? O[bp] : O[b];
    const uint32_t M = O[b] + __funnelshift_r(lo, hi, e ? 4u : 28u);
    Dlo = ((C[b] & 0x0F0F0F0Fu) << 2) + (M & 0x0F0F0F0Fu) * 26u + kb;
    Dhi = (((C[b] >> 4) & 0x0F0F0F0Fu) << 2) + ((M >> 4) & 0x0F0F0F0Fu) * 26u + kb;
  };
  // up to 4 words, the decisions form one branch-free block and ties
  // (probability 2^-16 per spin) are settled after it; with more words the
  // register budget settles each word's ties at once
  uint32_t tmask = 0u;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    uint32_t Dlo, Dhi;
    offsets(b, Dlo, Dhi);
    const uint4 x = philox((uint32_t)s, sw, c2 | (uint32_t)b, (ent << 8) | TAG_SQA_SWEEP, a.k0, a.k1);
    bool tie = false;
    w[b] = decide_word(x, Dlo, Dhi, tie);
    if constexpr (NB <= 4) {
      tmask |= tie ? (1u << b) : 0u;
    } else if (tie) {
      const uint4 y = philox((uint32_t)s, sw, c2 | (uint32_t)b, (ent << 8) | TAG_SQA_REFINE, a.k0, a.k1);
      w[b] = settle_ties(w[b], x, y, Dlo, Dhi);
    }
  }
  if (NB <= 4 && tmask) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!((tmask >> b) & 1u)) continue;
      uint32_t Dlo, Dhi;
      offsets(b, Dlo, Dhi);
      const uint4 x = philox((uint32_t)s, sw, c2 | (uint32_t)b, (ent << 8) | TAG_SQA_SWEEP, a.k0, a.k1);
      const uint4 y = philox((uint32_t)s, sw, c2 | (uint32_t)b, (ent << 8) | TAG_SQA_REFINE, a.k0, a.k1);
      w[b] = settle_ties(w[b], x, y, Dlo, Dhi);
    }
  }
  store_words<NB>(Wc + (size_t)s * NB, w);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *flag >= want (acquire); false after limit_ns.
__device__ __forceinline__ bool wait_at_least(const int *flag, int want, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (;;) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= want) return true;
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(256);
  }
}

// Anneal of sweeps [s0, s1) of one run.  s0 == 0 draws the random initial
// state, otherwise the state comes from the run's slot in global memory;
// s1 == S computes the final slice energies, otherwise the state goes back.
template <int NB>
__device__ __forceinline__ void anneal_span(const pc::SqaArgs &a, uint32_t *W, int32_t *Eacc,
                                            const uint16_t *jn, const SiteK &kh, bool hoist,
                                            int run, int s0, int s1) {
  const int N = a.N, P = a.P;
  const uint32_t ent = a.run0 + (uint32_t)run;
  const int tid = threadIdx.x, nt = blockDim.x;
  uint32_t *gstate = a.state ? a.state + (size_t)run * 2 * NB * N : nullptr;
  if (s0 == 0) {
    // Algorithm S1: all spins of all slices start random (+1 iff half < 2^15)
    for (int idx = tid; idx < 2 * NB * N; idx += nt) {
      const int b = idx % NB, cs = idx / NB, s = cs % N, c = cs / N;   // W[c][s][b]
      const uint4 x = philox((uint32_t)s, 0u, ((uint32_t)c << 16) | (uint32_t)b,
                             (ent << 8) | TAG_SQA_INIT, a.k0, a.k1);
      uint32_t w = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) w |= (half_lo(x, i) < 0x8000u) ? (1u << (4 * i)) : 0u;
      W[idx] = w;
    }
  } else {
    for (int idx = tid; idx < 2 * NB * N; idx += nt) W[idx] = __ldcg(gstate + idx);
  }
  for (int e = tid; e < pc::kSqaTab; e += nt) {   // small runs have fewer threads than entries
    const uint32_t t = s0 < a.S ? a.table[(size_t)s0 * pc::kSqaTab + e] : 0u;
    s_Tf[s0 & 1][e] = t;
    s_Th[s0 & 1][e] = (uint16_t)(t >> 16);
  }
  __syncthreads();

  for (int sw = s0; sw < s1; ++sw) {
    // the transverse coupling of this sweep lives in its threshold table;
    // prefetch the next sweep's table into the other buffer
    if (sw + 1 < a.S)
      for (int e = tid; e < pc::kSqaTab; e += nt) {
        const uint32_t t = a.table[(size_t)(sw + 1) * pc::kSqaTab + e];
        s_Tf[(sw + 1) & 1][e] = t;
        s_Th[(sw + 1) & 1][e] = (uint16_t)(t >> 16);
      }
    const uint32_t boff = (sw & 1) ? 0x50505050u : 0u;   // 80 bytes: the odd sweep's table
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const uint32_t *Wo = W + (1 - c) * NB * N;
      uint32_t *Wc = W + c * NB * N;
      if (hoist) {
        if (tid < N) update_site<NB>(a, Wo, Wc, tid, kh, c, (uint32_t)sw, boff, ent);
      } else {
        for (int s = tid; s < N; s += nt) {
          const SiteK k = site_consts(a, s, jn);
          update_site<NB>(a, Wo, Wc, s, k, c, (uint32_t)sw, boff, ent);
        }
      }
      __syncthreads();
    }
  }

  if (s1 < a.S) {
    for (int idx = tid; idx < 2 * NB * N; idx += nt) __stcg(gstate + idx, W[idx]);
    return;
  }
  // Algorithm S1: classical energy of every slice (full J, no J_perp).  Each
  // bond has one endpoint with 3D parity 1, so E_k = nbonds - 2 sum_{q(s)=1} sat.
  for (int k = tid; k < P; k += nt) Eacc[k] = 0;
  __syncthreads();
  for (int c = 0; c < 2; ++c) {
    const uint32_t *Wo = W + (1 - c) * NB * N;
    const uint32_t *Wc = W + c * NB * N;
    for (int s = tid; s < N; s += nt) {
      const Site t = site_of(a, s, jn);
      if (!t.q) continue;
      const int e = c ^ 1;
      uint32_t C[NB];
      spatial_counts<NB>(a, Wo, t, C);
      const int deg = 6 - __popc((t.jb >> 8) & 0x3Fu);
      for (int b = 0; b < NB; ++b) {
        const uint32_t w = Wc[(size_t)s * NB + b];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int ci = (C[b] >> (4 * i)) & 0xF;
          const int sat = ((w >> (4 * i)) & 1u) ? ci : deg - ci;
          atomicAdd(&Eacc[2 * (8 * b + i) + e], sat);
        }
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < P; k += nt) {
    Eacc[k] = a.nbonds - 2 * Eacc[k];
    a.E[(size_t)run * P + k] = Eacc[k];
  }
  __syncthreads();
  if (a.best && tid == 0) {
    int kb = 0;
    for (int k = 1; k < P; ++k)
      if (Eacc[k] < Eacc[kb]) kb = k;
    a.best[2 * run] = Eacc[kb];
    a.best[2 * run + 1] = kb;
  }
  if (a.corr) {
    // replica-direction correlation (Fig. S17): sum over sites of
    // s(s,0) s(s,k) = 2 #agree - N.  Slice k of site s is nibble (k>>1)&7 of
    // word W[(k&1) ^ q(s)][s][k>>4].  Eacc is reused once the best slice
    // has been read from it.
    __syncthreads();
    for (int k = tid; k < P; k += nt) Eacc[k] = 0;
    __syncthreads();
    for (int s = tid; s < N; s += nt) {
      const int r = (int)fdiv((uint32_t)s, a.mLx), x = s - r * a.Lx;
      const int z = (int)fdiv((uint32_t)r, a.mLy), y = r - z * a.Ly;
      const int q = (x + y + z) & 1;
      const uint32_t s0 = W[(size_t)q * NB * N + (size_t)s * NB] & 1u;   // slice 0
      const uint32_t flip = s0 ? 0u : 0x11111111u;
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < NB; ++b) {
          const uint32_t agree = (W[(size_t)c * NB * N + (size_t)s * NB + b] ^ flip) & 0x11111111u;
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if ((agree >> (4 * i)) & 1u) atomicAdd(&Eacc[2 * (8 * b + i) + (c ^ q)], 1);
        }
    }
    __syncthreads();
    for (int k = tid; k < P; k += nt) a.corr[(size_t)run * P + k] = 2 * Eacc[k] - N;
    __syncthreads();
  }
  if (a.spins) {
    for (int idx = tid; idx < 2 * NB * N; idx += nt) {
      const int b = idx % NB, cs = idx / NB, s = cs % N, c = cs / N;   // W[c][s][b]
      const int r = (int)fdiv((uint32_t)s, a.mLx), x = s - r * a.Lx;
      const int z = (int)fdiv((uint32_t)r, a.mLy), y = r - z * a.Ly;
      const int e = c ^ ((x + y + z) & 1);
      const uint32_t w = W[idx];
      for (int i = 0; i < 8; ++i) {
        const int k = 2 * (8 * b + i) + e;
        a.spins[((size_t)run * P + k) * N + s] = ((w >> (4 * i)) & 1u) ? 1 : -1;
      }
    }
  }
  __syncthreads();
}

// PERSIST = false: one CTA per run, the whole schedule.  PERSIST = true: a
// persistent grid pulls (chunk, run) items in chunk-major order from a
// queue; chunk k of a run waits (bounded) until chunk k-1 of that run has
// stored its state.  Time-slicing the runs keeps every SM busy when the
// number of runs is not a multiple of the number of SMs.
template <int NB, bool PERSIST>
__global__ void __launch_bounds__(PC_SQA_TPB, PC_SQA_MINB) sqa_kernel(const pc::SqaArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_item;
  const int N = a.N, P = a.P;
  uint32_t *W = smem;                                       // [2][NB][N]
  int32_t *Eacc = reinterpret_cast<int32_t *>(W + 2 * NB * N);   // [P]
  uint16_t *jn = reinterpret_cast<uint16_t *>(Eacc + P);    // [N]
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N; i += nt) jn[i] = a.jneg[i];
  __syncthreads();
  // one site per thread (N <= blockDim): its constants stay in registers
  const bool hoist = PC_SQA_HOIST && N <= nt;
  SiteK kh;
  if (hoist && tid < N) kh = site_consts(a, tid, jn);
  if constexpr (!PERSIST) {
    anneal_span<NB>(a, W, Eacc, jn, kh, hoist, blockIdx.x, 0, a.S);
  } else {
    for (;;) {
      if (tid == 0) s_item = atomicAdd(a.queue, 1) + a.first_item;
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= a.n_items) break;
      const int chunk = item / a.R, run = item - chunk * a.R;
      const int s0 = chunk * a.K, s1 = min(a.S, s0 + a.K);
      if (chunk > 0) {
        if (tid == 0 && !wait_at_least(a.done + run, chunk, a.wait_ns)) atomicExch(a.err, 1);
        __syncthreads();
      }
      anneal_span<NB>(a, W, Eacc, jn, kh, hoist, run, s0, s1);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.done + run), "r"(chunk + 1) : "memory");
      }
    }
  }
}

__global__ void philox_kernel(const uint32_t *ctr, uint32_t *out, int64_t n, uint32_t k0,
                              uint32_t k1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 x = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
  out[4 * i] = x.x;
  out[4 * i + 1] = x.y;
  out[4 * i + 2] = x.z;
  out[4 * i + 3] = x.w;
}

template <int NB>
int launch_nb(const pc::SqaArgs &a, int R, cudaStream_t st) {
  const size_t smem = pc::sqa_smem_bytes(a.N, a.P);
  int tpb = ((a.N + 31) / 32) * 32;
  if (tpb > PC_SQA_TPB) tpb = PC_SQA_TPB;
  if (!a.state) {
    PC_CUDA_TRY(cudaFuncSetAttribute(sqa_kernel<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    sqa_kernel<NB, false><<<R, tpb, smem, st>>>(a);
  } else {
    PC_CUDA_TRY(cudaFuncSetAttribute(sqa_kernel<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    PC_CUDA_TRY(cudaGetDevice(&dev));
    PC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sqa_kernel<NB, true>, tpb, smem));
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    if (grid > a.n_items) grid = a.n_items;
    sqa_kernel<NB, true><<<grid, tpb, smem, st>>>(a);
  }
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

}  // namespace

namespace pc {

size_t sqa_smem_bytes(int N, int P) {
  const int NB = P / 16;
  return (size_t)2 * NB * N * 4 + (size_t)P * 4 + (size_t)N * 2;
}

int sqa_launch(const SqaArgs &a, int R, cudaStream_t st) {
  switch (a.NB) {
    case 1: return launch_nb<1>(a, R, st);
    case 2: return launch_nb<2>(a, R, st);
    case 3: return launch_nb<3>(a, R, st);
    case 4: return launch_nb<4>(a, R, st);
    case 5: return launch_nb<5>(a, R, st);
    case 6: return launch_nb<6>(a, R, st);
    case 7: return launch_nb<7>(a, R, st);
    case 8: return launch_nb<8>(a, R, st);
    default: return fail(PC_EINVAL, "P must be 16 * k with 1 <= k <= 8");
  }
}

int philox_launch(const uint32_t *ctr, uint32_t *out, int64_t n, uint32_t k0, uint32_t k1,
                  cudaStream_t st) {
  if (n <= 0) return PC_OK;
  const int tpb = 256;
  philox_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(ctr, out, n, k0, k1);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

}  // namespace pc

// ---------------------------------------------------------------------------
// DT-SQA entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running under a memory manager
// that owns every device allocation (a framework's caching allocator or a
// fixed arena), or code that must not allocate on a latency-critical path.
// pc_sqa_anneal_noalloc runs the same anneal kernel as pc_sqa_run_dev but
// keeps its scratch (the packed couplings and the per-sweep threshold
// tables) in the file-scope device array below instead of in
// library-allocated buffers.  Every GPU that loads this library keeps this
// array (about 1.57 MiB) until the process exits.
namespace {

constexpr int kNoallocMaxSweeps = 10240;
constexpr int kNoallocJnegBytes = 8192;   // N <= 4096 sites, 16-bit coupling words
constexpr size_t kNoallocTableBytes = (size_t)kNoallocMaxSweeps * pc::kSqaTab * 4;
constexpr size_t kNoallocBytes = kNoallocJnegBytes + kNoallocTableBytes;

static __device__ __align__(256) unsigned char g_sqa_noalloc_scratch[kNoallocBytes];

// Host data reaches the scratch array as kernel parameters, which the
// launch copies by value: no host buffer has to outlive the call and no
// pageable copy is issued.  One chunk carries 12 KiB (a host stack buffer).
constexpr int kStageWords = 3072;
struct StageChunk {
  uint32_t off;                 // destination offset in 32-bit words
  uint32_t n;                   // words carried (<= kStageWords)
  uint32_t w[kStageWords];
};

__global__ void noalloc_stage_kernel(uint32_t *dst, const __grid_constant__ StageChunk c) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c.n; i += gridDim.x * blockDim.x)
    dst[c.off + i] = c.w[i];
}

int stage_words(uint32_t *dst, StageChunk &c, cudaStream_t st) {
  if (c.n == 0) return PC_OK;
  noalloc_stage_kernel<<<8, 512, 0, st>>>(dst, c);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

// Device address of the scratch array, looked up once per device (with that
// device current) under a lock, so that host threads making their first
// calls at the same time do not race.  The symbol's name is a host-side
// stand-in, never a device address, so only this pointer is handed to
// kernels.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_lock;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

int noalloc_scratch(int device, unsigned char **out) {
  if (device < 0 || device >= kMaxDevices) return pc::fail(PC_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_lock);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sqa_noalloc_scratch);
    if (e != cudaSuccess)
      return pc::fail(PC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[device] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[device];
  return PC_OK;
}

}  // namespace

extern "C" int pc_sqa_anneal_noalloc(int device, void *stream, uint64_t seed, const int32_t *dims,
                                     const int8_t *J, int P, double T, int n_sweeps,
                                     const double *gamma, int R, uint32_t run0, int32_t *E_dev,
                                     int32_t *best_dev) try {
  using namespace pc;
  if (!dims || !J || (n_sweeps > 0 && !gamma) || (R > 0 && !E_dev))
    return fail(PC_EINVAL, "NULL argument");
  Lattice lat;
  int rc = check_lattice(dims, J, &lat);
  if (rc) return rc;
  if (P < 16 || P % 16 || P > 128) return fail(PC_EINVAL, "P must be a multiple of 16 in [16, 128]");
  if ((int64_t)lat.N * P > 262144) return fail(PC_EINVAL, "N * P must be <= 262144");
  if (!(T > 0.0) || n_sweeps < 0) return fail(PC_EINVAL, "T must be > 0 and n_sweeps >= 0");
  if (n_sweeps > kNoallocMaxSweeps)
    return fail(PC_EINVAL, "pc_sqa_anneal_noalloc: n_sweeps exceeds the scratch limit of 10240");
  if (R < 0 || (uint64_t)run0 + (uint64_t)R > (1ull << 24))
    return fail(PC_EINVAL, "R must be >= 0 and run ids < 2^24");
  for (int s = 0; s < n_sweeps; ++s)
    if (!(gamma[s] > 0.0)) return fail(PC_EINVAL, "every Gamma must be > 0");
  PC_CUDA_TRY(cudaSetDevice(device));
  unsigned char *scratch = nullptr;
  if ((rc = noalloc_scratch(device, &scratch))) return rc;
  if (R == 0) return PC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *words = reinterpret_cast<uint32_t *>(scratch);
  StageChunk chunk_buf;
  StageChunk *chunk = &chunk_buf;

  // couplings: one 16-bit word per site (periodic: no absent bonds), two
  // per staged 32-bit word (N is even)
  {
    const int Lx = lat.L[0], Ly = lat.L[1], Lz = lat.L[2];
    uint16_t *jn = reinterpret_cast<uint16_t *>(chunk->w);
    for (int s = 0; s < lat.N; ++s) {
      const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
      const int xm = (x + Lx - 1) % Lx + Lx * (y + Ly * z);
      const int ym = x + Lx * ((y + Ly - 1) % Ly + Ly * z);
      const int zm = x + Lx * (y + Ly * ((z + Lz - 1) % Lz));
      const int8_t j6[6] = {J[3 * s], J[3 * xm], J[3 * s + 1], J[3 * ym + 1], J[3 * s + 2],
                            J[3 * zm + 2]};
      uint16_t m = 0;
      for (int d = 0; d < 6; ++d)
        if (j6[d] < 0) m |= (uint16_t)(1u << d);
      jn[s] = m;
    }
    chunk->off = 0;
    chunk->n = (uint32_t)lat.N / 2;
    if ((rc = stage_words(words, *chunk, st))) return rc;
  }
  // per-sweep threshold tables, kStageWords / kSqaTab sweeps per chunk
  {
    constexpr int W = pc::kSqaTab;
    constexpr int kSweepsPerChunk = kStageWords / W;
    const double beta_eff = 1.0 / ((double)P * T);
    for (int s0 = 0; s0 < n_sweeps; s0 += kSweepsPerChunk) {
      const int ns = (n_sweeps - s0 < kSweepsPerChunk) ? n_sweeps - s0 : kSweepsPerChunk;
      uint32_t *tab = chunk->w;
      for (int k = 0; k < ns; ++k) {
        const int32_t jq = pc_jperp_q(gamma[s0 + k], P, T);
        for (int e = 0; e < W; ++e) tab[W * k + e] = 0u;
        for (int m = 0; m < 3; ++m)
          for (int e = 0; e < 13; ++e) tab[W * k + e + 13 * m] = sqa_threshold(beta_eff, e - 6, jq, 2 * m - 2);
      }
      chunk->off = (uint32_t)(kNoallocJnegBytes / 4 + (size_t)s0 * W);
      chunk->n = (uint32_t)(ns * W);
      if ((rc = stage_words(words, *chunk, st))) return rc;
    }
  }
  SqaArgs a;
  a.Lx = lat.L[0];
  a.Ly = lat.L[1];
  a.Lz = lat.L[2];
  a.N = lat.N;
  a.P = P;
  a.NB = P / 16;
  a.S = n_sweeps;
  a.mLx = recip32((uint32_t)a.Lx);
  a.mLy = recip32((uint32_t)a.Ly);
  a.run0 = run0;
  a.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  a.k1 = (uint32_t)(seed >> 32);
  a.jneg = reinterpret_cast<const uint16_t *>(scratch);
  a.nbonds = 3 * lat.N;
  a.table = reinterpret_cast<const uint32_t *>(scratch + kNoallocJnegBytes);
  a.E = E_dev;
  a.best = best_dev;
  a.spins = nullptr;
  a.corr = nullptr;
  a.state = nullptr;   // one CTA per run: no state scratch
  a.done = a.queue = a.err = nullptr;
  a.R = R;
  a.K = n_sweeps;
  a.n_items = R;
  a.first_item = 0;
  a.wait_ns = 0;
  return sqa_launch(a, R, st);
} catch (...) {
  return pc::fail_exception();
}
