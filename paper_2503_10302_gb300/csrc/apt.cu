// Adaptive parallel tempering with isoenergetic cluster moves (Algorithm S2)
// as one persistent CTA per problem: checkerboard p-bit sweeps of every
// replica, replica energies, best-energy tracking, Houdayer cluster moves
// and replica exchange all run on chip between kernel launches.  The same
// kernel also drives the chains of the adaptive-ladder preprocessing
// (energy sums over a tail window) and of the pilot runs (energy
// histograms).
//
// Layout.  Replicas ("buffers") of one problem are packed eight to a 32-bit
// word, one spin per nibble (bit 0 = +1): group g holds buffers 8g..8g+7.
// Sites are split by checkerboard colour c = (x+y+z)&1 and indexed inside a
// colour by j = lin >> 1, so a word S[g][c][j] carries site (c, j) of eight
// replicas.  All replicas of a problem share the couplings, hence one word
// gives the nibble-packed satisfied-bond counts of eight replicas with six
// XOR/ADD pairs, and one Philox4x32-10 call gives their eight 16-bit
// uniforms.
//
// Replica slots are fixed: temperature r with ICM label a lives in buffer
// a*Tp + r (Tp = 8 ceil(T/8)), so the two labels of temperature r sit in the
// same nibble of groups h and h + G/2.  An accepted swap exchanges the two
// replicas' states (Algorithm S2) with SWAR nibble swaps, and the overlap of
// eight ICM pairs is one XOR of two words, which makes the cluster growth a
// nibble-parallel flood fill over all pairs at once.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "apt_dev.h"
#include "device.cuh"
#include "internal.h"

// Optional per-phase cycle counters of CTAs 0 and 1 (the two ranks of the
// first problem when problems split; build with -DPC_APT_PROFILE=1; read the
// 2 x 16 counters with pc_apt_profile_read).  Off by default.
#ifndef PC_APT_PROFILE
#define PC_APT_PROFILE 0
#endif
// The flood fill keeps a block's overlap words in registers across passes
// (build-time knob; 0 reloads them every pass).
#ifndef PC_APT_FILL_XREG
#define PC_APT_FILL_XREG 1
#endif
// Split problems keep the first entries of their swap tables in shared
// memory (build-time knob).
#ifndef PC_APT_STAGE_SWT
#define PC_APT_STAGE_SWT 1
#endif
#if PC_APT_PROFILE
__device__ unsigned long long g_apt_prof[32];
#define PROF_MARK(slot, t0)                                                     \
  do {                                                                          \
    if (blockIdx.x < 2 && threadIdx.x == 0) {                                   \
      const long long t1_ = clock64();                                          \
      atomicAdd(&g_apt_prof[16 * blockIdx.x + (slot)], (unsigned long long)(t1_ - (t0))); \
      (t0) = t1_;                                                               \
    }                                                                           \
  } while (0)
#else
#define PROF_MARK(slot, t0) do { } while (0)
#endif

namespace {
using namespace pcdev;
using pc::AptArgs;
using pc::AptProbDev;

constexpr int MAXGC = 4;   // groups handled per thread per site

struct Geo {
  int Lx, Ly, Lz, N, H, hx;
  uint32_t mhx, mLy, mLy2;
};

// Neighbours (other colour, colour-local index) of site (c, j), in the
// direction order +x, -x, +y, -y, +z, -z; periodic boundaries.
__device__ __forceinline__ void neighbours(const Geo &g, int c, int j, int (&n)[6]) {
  const int row = (int)fdiv((uint32_t)j, g.mhx);   // j / hx
  const int jx = j - row * g.hx;
  const int z = (int)fdiv((uint32_t)row, g.mLy);   // row / Ly
  const int y = row - z * g.Ly;
  const int p = (y + z + c) & 1;                   // x = 2 jx + p
  const int base = row * g.hx;
  int jxp, jxm;
  if (p == 0) {
    jxp = jx;
    jxm = (jx == 0) ? g.hx - 1 : jx - 1;
  } else {
    jxp = (jx + 1 == g.hx) ? 0 : jx + 1;
    jxm = jx;
  }
  n[0] = base + jxp;
  n[1] = base + jxm;
  const int yp = (y + 1 == g.Ly) ? 0 : y + 1, ym = (y == 0) ? g.Ly - 1 : y - 1;
  const int zp = (z + 1 == g.Lz) ? 0 : z + 1, zm = (z == 0) ? g.Lz - 1 : z - 1;
  n[2] = (yp + g.Ly * z) * g.hx + jx;
  n[3] = (ym + g.Ly * z) * g.hx + jx;
  n[4] = (y + g.Ly * zp) * g.hx + jx;
  n[5] = (y + g.Ly * zm) * g.hx + jx;
}

// lin = x + Lx (y + Ly z) of site (c, j).
__device__ __forceinline__ int lin_of(const Geo &g, int c, int j) {
  const int row = (int)fdiv((uint32_t)j, g.mhx);
  const int jx = j - row * g.hx;
  const int z = (int)fdiv((uint32_t)row, g.mLy);
  const int y = row - z * g.Ly;
  return 2 * jx + ((y + z + c) & 1) + g.Lx * row;
}


// Threshold of nibble i (thr points at the group's 128 entries: 8 buffers x
// 16, entry I + 6 for I = -6..6).  SCALE 1: C holds I + 6 per nibble;
// SCALE 2: C holds the satisfied count of a site with all six bonds, whose
// entry is 2C.
// thrh holds the thresholds' top halves t as 16-bit entries in the same
// [buffer][16] order, each group's 256 bytes starting on a 256-byte
// boundary of shared memory (tb, a shared-window address), so the entry of
// nibble i sits at tb | (32 i + 2 SCALE c_i), 32 i + 2 SCALE c_i <= 248:
// the offsets of 4 nibbles are formed in one word and each address is one
// byte permute of that word with tb.  The sign of d = v - t for the main
// half v is the decision, and the top 4 bits of each d are shifted into w
// so that bit 3 of nibble i carries half i's sign.  A zero product of the
// differences (mod 2^32) flags a possible tie, which refine8_grp settles
// exactly (a product that only wraps to 0 costs a needless refine).
template <int SCALE>
__device__ __forceinline__ uint32_t decide8_grp(const uint4 &x, uint32_t C, uint32_t tb, bool &tie) {
  // byte k of Dlo: offset of nibble 2k (64 k + 2 SCALE c); of Dhi: nibble 2k+1
  const uint32_t Dlo = (C & 0x0F0F0F0Fu) * (2u * SCALE) + 0xC0804000u;
  const uint32_t Dhi = ((C >> 4) & 0x0F0F0F0Fu) * (2u * SCALE) + 0xE0A06020u;
  uint32_t w = 0, tp = 1u;
#pragma unroll
  for (int i = 7; i >= 0; --i) {
    // byte 0 from the offsets, bytes 1-3 from tb
    const uint32_t addr = __byte_perm((i & 1) ? Dhi : Dlo, tb, 0x7650u + (uint32_t)(i >> 1));
    uint32_t th;
    asm("ld.shared.u16 %0, [%1];" : "=r"(th) : "r"(addr));
    const uint32_t d = half_lo(x, i) - th;
    w = __funnelshift_l(d, w, 4);
    tp *= d;
  }
  tie |= (tp == 0u);
  return (w >> 3) & 0x11111111u;
}

template <int SCALE>
__device__ __noinline__ uint32_t refine8_grp(uint32_t w, uint4 x, uint4 y, uint32_t C,
                                             const uint32_t *thr) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t t = thr[16 * i + SCALE * ((C >> (4 * i)) & 0xFu)];
    const uint32_t v = half_hi(x, i);
    if (v == (t & 0xFFFF0000u)) {
      const uint32_t u = v | half_lo(y, i);
      w = (u < t) ? (w | (1u << (4 * i))) : (w & ~(1u << (4 * i)));
    }
  }
  return w;
}

struct Shared {
  uint32_t *S;       // [Gc][2][H]
  uint32_t *thr;     // [Gc*8][16] p-bit thresholds, entry I + 6
  uint16_t *thrh;    // [Gc*8][16] their high halves (16-bit)
  int32_t *temp_of;  // [Gc*8]
  int32_t *buf_of;   // [Gc*8] (unused by the fixed-slot APT mode)
  int32_t *E;        // [Gc*8]
  int32_t *Eacc;     // [Gc*8]
  int32_t *satt, *sacc;   // [64] swap attempts / accepts of this launch
  int32_t *hist;     // pilot histogram [T][n_bins]
  int64_t *sum1, *sum2;   // ladder sums [Gc*8]
  int64_t *m64;      // best E, best sweep, hit sweep, target
  int32_t *m32;      // best buffer, flag, icm counters x3, any-swap flag
  uint16_t *jn;      // [2][H] coupling signs (bits 0-5) and missing bonds (8-13)
  uint32_t *V;       // ICM cluster bits [2][H], overlap bits [2][H], transposed overlaps [N/32][32]
  uint32_t *ikx;     // [64] per pair: Philox word 0, then k
  int32_t *ibit;     // [64] per pair: replica choice bit
  int32_t *inm;      // [64] per pair: mismatch count
  int32_t *isz;      // [64] per pair: cluster size
  uint32_t *imask;   // [3][8] per half-group: cluster-flip, whole-flip label 0, label 1
  uint32_t *swm;     // [8] per group: in-group swap nibble mask; [8] cross-group flags;
                     // [6] ICM matching nibble masks (4 labels)
  int32_t *gmap;     // [8] global group of each local group
  int32_t *xch;      // split problems: [2][4] boundary energies by attempt parity;
                     // [8] accepted boundary labels; [12..17] the peer's best at launch end
  uint32_t *stage;   // [2][4][64] peer boundary spins by attempt parity, one bit per site
  uint32_t *swt;     // split problems: [T-1][kSwtLen] first entries of each pair's swap table
};

// Entries of each pair's swap table (|dE| = 0, 2, .., 2 (kSwtLen - 1)) that a
// split problem's CTAs keep in shared memory; larger |dE| read the table in
// global memory.
constexpr int kSwtLen = 256;

struct Cta {
  Geo geo;
  int T, Tp, A, B, Bc, Gc, g0;
  // this CTA holds, for every label, the temperature groups [g0, g0 + Gu) of
  // the Glp groups per label (APT; ladder / pilot: A = 1, groups g0 ..);
  // split problems run as a cluster of two CTAs, rank 0 holding the hotter
  // (lower-beta, first) half
  int Gu, Glp, split, rank;
  int nbonds;        // bonds present (3N with periodic axes)
  int nreal;         // spins present (N without vacancies)
  uint32_t open;     // bit a: axis a open
  uint32_t ent;
  // thread chunking of the site loop: nch chunks of tpc threads, gc groups each
  int nch, tpc, gc;
};

// Satisfied-bond counts of NG groups in byte lanes: e8[u][0] byte k counts
// nibble 2k, e8[u][1] byte k nibble 2k + 1.  A site adds at most 6 to a
// lane, so a thread reduces them after at most kFlushSites sites.
constexpr int kFlushSites = 32;

// The NG groups [gbeg, gbeg + NG) of site (c, j): every neighbour word is
// loaded first, then the NG decisions run as one branch-free block whose
// Philox chains are independent, ties (a zero product of a word's eight
// differences, about 2^-13 per word) are settled after it, and the stores
// come last.  The field of 8 spins is C = n_neg 0x11111111 + sum_d eps_d W_d
// with eps_d = +1 (J > 0), -1 (J < 0) or 0 (absent bond): per nibble the
// count of satisfied present bonds (W ^ 1 for a negative bond is 1 - W),
// exact mod 2^32 because every final nibble lies in 0..6.
template <int NG, bool UPDATE, bool ENERGY, bool OPEN>
__device__ __forceinline__ void site_groups(const AptArgs &a, const Cta &k, const Shared &sh, int c, int j,
                                            uint32_t sweep, int gbeg, uint32_t (&e8)[NG][2]) {
  const int H = k.geo.H;
  const uint32_t tb0 = (uint32_t)__cvta_generic_to_shared(sh.thrh) + 256u * (uint32_t)gbeg;
  int n[6];
  neighbours(k.geo, c, j, n);
  const uint32_t jb = sh.jn[c * H + j];
  const uint32_t miss = OPEN ? (jb >> 8) & 0x3Fu : 0u;
  const uint32_t K = OPEN ? (uint32_t)__popc(miss) * 0x11111111u : 0u;
  uint32_t eps[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const uint32_t e = 1u - 2u * ((jb >> d) & 1u);
    eps[d] = (OPEN && ((miss >> d) & 1u)) ? 0u : e;
  }
  const uint32_t K0 = (uint32_t)__popc(jb & 0x3Fu & ~miss) * 0x11111111u;
  uint32_t C[NG], w[NG];
#pragma unroll
  for (int u = 0; u < NG; ++u) {
    const uint32_t *Wo = sh.S + (size_t)(2 * (gbeg + u) + (1 - c)) * H;
    uint32_t s = K0;
#pragma unroll
    for (int d = 0; d < 6; ++d) s += eps[d] * Wo[n[d]];
    C[u] = s;
  }
  if (UPDATE) {
    const uint32_t c2 = (uint32_t)c << 16, tag = (k.ent << 8) | a.tag_main;
    uint32_t tmask = 0u;
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      const uint4 x = philox((uint32_t)j, sweep, c2 | (uint32_t)sh.gmap[gbeg + u], tag, a.k0, a.k1);
      bool tie = false;
      // threshold index I + 6 = 2C + k per nibble (2C with every bond)
      const uint32_t D = OPEN ? 2u * C[u] + K : C[u];
      w[u] = decide8_grp<OPEN ? 1 : 2>(x, D, tb0 + 256u * (uint32_t)u, tie);
      tmask |= tie ? (1u << u) : 0u;
    }
    if (tmask) {
#pragma unroll
      for (int u = 0; u < NG; ++u) {
        if (!((tmask >> u) & 1u)) continue;
        const uint32_t g = (uint32_t)sh.gmap[gbeg + u];
        const uint4 x = philox((uint32_t)j, sweep, c2 | g, tag, a.k0, a.k1);
        const uint4 y = philox((uint32_t)j, sweep, c2 | g, (k.ent << 8) | a.tag_ref, a.k0, a.k1);
        const uint32_t D = OPEN ? 2u * C[u] + K : C[u];
        w[u] = refine8_grp<OPEN ? 1 : 2>(w[u], x, y, D, sh.thr + 128 * (gbeg + u));
      }
    }
#pragma unroll
    for (int u = 0; u < NG; ++u) sh.S[(size_t)(2 * (gbeg + u) + c) * H + j] = w[u];
  } else {
#pragma unroll
    for (int u = 0; u < NG; ++u) w[u] = sh.S[(size_t)(2 * (gbeg + u) + c) * H + j];
  }
  if (ENERGY) {
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      const uint32_t full = w[u] * 0xFu;    // nibble of all ones where the spin is +1
      const uint32_t sat = (C[u] & full) | ((0x66666666u - K - C[u]) & ~full);
      e8[u][0] += sat & 0x0F0F0F0Fu;
      e8[u][1] += (sat >> 4) & 0x0F0F0F0Fu;
    }
  }
}

// The sites j = j0, j0 + tpc, .. below j1 of colour c for the NG groups
// from gbeg; at most kFlushSites sites per thread, so that the byte lanes
// of the energy counts cannot overflow.  Every lane of a warp calls it
// (the warp reduction at the end).
template <int NG, bool UPDATE, bool ENERGY, bool OPEN>
__device__ __forceinline__ void site_loop(const AptArgs &a, const Cta &k, const Shared &sh, int c,
                                          uint32_t sweep, int j0, int j1, int gbeg) {
  uint32_t e8[NG][2];
#pragma unroll
  for (int u = 0; u < NG; ++u) e8[u][0] = e8[u][1] = 0u;
  for (int j = j0; j < j1; j += k.tpc) site_groups<NG, UPDATE, ENERGY, OPEN>(a, k, sh, c, j, sweep, gbeg, e8);
  if (ENERGY) {
    // lanes of a warp share the chunk (and NG); reduce 16-bit lanes across
    // the warp: word m of a group holds nibbles m (low) and m + 4 (high)
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < NG; ++u) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        uint32_t v = (e8[u][m & 1] >> (8 * (m >> 1))) & 0x00FF00FFu;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) {
          const int b = 8 * (gbeg + u) + m;
          atomicAdd(&sh.Eacc[b], (int)(v & 0xFFFFu));
          atomicAdd(&sh.Eacc[b + 4], (int)(v >> 16));
        }
      }
    }
  }
}

// Sites of colour c in blocks of kFlushSites per thread (one block unless
// H > kFlushSites * tpc).
template <int NG, bool UPDATE, bool ENERGY, bool OPEN>
__device__ __forceinline__ void site_blocks(const AptArgs &a, const Cta &k, const Shared &sh, int c,
                                            uint32_t sweep, int lt, int gbeg) {
  const int H = k.geo.H, span = kFlushSites * k.tpc;
  if (!ENERGY || H <= span) {
    site_loop<NG, UPDATE, ENERGY, OPEN>(a, k, sh, c, sweep, lt, H, gbeg);
    return;
  }
  for (int b0 = 0; b0 < H; b0 += span)
    site_loop<NG, UPDATE, ENERGY, OPEN>(a, k, sh, c, sweep, b0 + lt, min(H, b0 + span), gbeg);
}

// One colour phase of a sweep over the CTA's groups.  UPDATE: Eq. synapse +
// Eq. neuron for every site of colour c.  ENERGY: accumulate, per buffer,
// the satisfied bonds of the colour-c sites (every bond has exactly one
// colour-1 endpoint, so the colour-1 pass gives E = nbonds - 2 * satisfied).
// A site missing k of its six bonds (open boundaries) counts its satisfied
// present bonds C, so I = 2C - (6 - k); the threshold row is indexed by
// I + 6 = 2C + k, formed for eight spins at once as 2C + k * 0x11111111.
template <bool UPDATE, bool ENERGY, bool OPEN>
__device__ __forceinline__ void colour_phase_t(const AptArgs &a, const Cta &k, const Shared &sh,
                                               int c, uint32_t sweep, int gtot) {
  const int tid = threadIdx.x;
  const int q = tid / k.tpc, lt = tid - q * k.tpc;
  // groups [0, gtot) over the nch thread chunks (at most MAXGC per chunk)
  const int gper = gtot == k.Gc ? k.gc : (gtot + k.nch - 1) / k.nch;
  const int gbeg = q * gper;
  int gcnt = gtot - gbeg;
  if (gcnt > gper) gcnt = gper;
  if (gcnt >= 4)
    site_blocks<4, UPDATE, ENERGY, OPEN>(a, k, sh, c, sweep, lt, gbeg);
  else if (gcnt == 3)
    site_blocks<3, UPDATE, ENERGY, OPEN>(a, k, sh, c, sweep, lt, gbeg);
  else if (gcnt == 2)
    site_blocks<2, UPDATE, ENERGY, OPEN>(a, k, sh, c, sweep, lt, gbeg);
  else if (gcnt == 1)
    site_blocks<1, UPDATE, ENERGY, OPEN>(a, k, sh, c, sweep, lt, gbeg);
}

// Periodic problems take the path without absent-bond handling.
template <bool UPDATE, bool ENERGY>
__device__ __forceinline__ void colour_phase(const AptArgs &a, const Cta &k, const Shared &sh, int c,
                                             uint32_t sweep, int gtot) {
  if (k.open)
    colour_phase_t<UPDATE, ENERGY, true>(a, k, sh, c, sweep, gtot);
  else
    colour_phase_t<UPDATE, ENERGY, false>(a, k, sh, c, sweep, gtot);
}

// E_b = nbonds - 2 * (satisfied bonds); resets the accumulators.
__device__ __forceinline__ void finish_energies(const Cta &k, const Shared &sh) {
  for (int b = threadIdx.x; b < 8 * k.Gc; b += blockDim.x) {
    sh.E[b] = k.nbonds - 2 * sh.Eacc[b];
    sh.Eacc[b] = 0;
  }
}

// Minimum-energy selection (Algorithm S2 output): strict improvement, lowest
// slot index (r * A + a) on ties; copies the state of the new best replica.
// The two CTAs of a split problem track their own candidates (rank 1 into a
// scratch state) and combine them at the end of the launch: the global best
// is the lower energy, found at the earlier sweep, rank 0 (the lower slots)
// on ties, and the target is first hit at the earlier of the two hits.
__device__ void best_update(const AptArgs &a, const Cta &k, const Shared &sh, int p,
                            int64_t sweeps) {
  if (threadIdx.x < 32) {
    // the lowest energy, ties to the lowest slot r A + label: one warp
    // minimum of the key (E + 2^18) 2^8 + slot (|E| <= 3N < 2^18, slot < 2^8)
    const int lane = threadIdx.x;
    uint32_t key = 0xFFFFFFFFu;
    int bestb = 0;
    for (int b = lane; b < 8 * k.Gc; b += 32) {
      const int gb = 8 * sh.gmap[b >> 3] + (b & 7);
      const int r = gb % k.Tp, lab = gb / k.Tp;
      if (r >= k.T) continue;
      const uint32_t kb = ((uint32_t)(sh.E[b] + (1 << 18)) << 8) | (uint32_t)(r * k.A + lab);
      if (kb < key) {
        key = kb;
        bestb = b;
      }
    }
    const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, key);
    // the lane holding the minimum (keys are distinct), or lane 0 if no
    // buffer holds a temperature
    if (mn != 0xFFFFFFFFu ? key == mn : lane == 0) {
      const int bestE = mn != 0xFFFFFFFFu ? (int)(mn >> 8) - (1 << 18) : 0x7FFFFFFF;
      int flag = 0;
      if ((int64_t)bestE < sh.m64[0]) {
        sh.m64[0] = bestE;
        sh.m64[1] = sweeps;
        sh.m32[0] = 8 * sh.gmap[bestb >> 3] + (bestb & 7);
        sh.m32[7] = bestb;
        flag = 1;
      }
      if (sh.m64[2] < 0 && sh.m64[0] <= sh.m64[3]) sh.m64[2] = sweeps;
      sh.m32[1] = flag;
    }
  }
  __syncthreads();
  if (sh.m32[1]) {
    const int b = sh.m32[7];
    const int g = b >> 3, i = b & 7;
    const AptProbDev &P = a.prob[p];
    int8_t *dst = (k.rank ? a.best_spins2 : a.best_spins) + P.best_off;
    for (int kk = threadIdx.x; kk < k.geo.N; kk += blockDim.x) {
      const int c = kk >= k.geo.H ? 1 : 0, j = kk - c * k.geo.H;
      const uint32_t w = sh.S[(size_t)(2 * g + c) * k.geo.H + j];
      dst[lin_of(k.geo, c, j)] = ((w >> (4 * i)) & 1u) ? 1 : -1;
    }
  }
  __syncthreads();
}

// 32 x 32 bit-matrix transpose across a warp: lane l holds row l on entry
// (bit c = element (l, c)) and column l on exit (bit r = element (r, l)).
// Five butterfly stages exchange the off-diagonal blocks of size 16..1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                                                     : j == 2 ? 0x33333333u : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
    x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

// Nibble mask (bit 4i) <-> byte (bit i) of eight pairs.
__device__ __forceinline__ uint32_t nib_to_byte(uint32_t z) {
  uint32_t t = z & 0x11111111u;
  t = (t | (t >> 3)) & 0x03030303u;
  t = (t | (t >> 6)) & 0x000F000Fu;
  return (t | (t >> 12)) & 0xFFu;
}
__device__ __forceinline__ uint32_t byte_to_nib(uint32_t b) {
  uint32_t t = (b | (b << 12)) & 0x000F000Fu;
  t = (t | (t << 6)) & 0x03030303u;
  return (t | (t << 3)) & 0x11111111u;
}

// Union-find over 32-bit parent words in shared memory, every parent no
// larger than its child, so a root is the smallest index of its set.  A
// failed atomicMin means the word decreased meanwhile, which bounds the
// retries; the cap only guards the loop.
__device__ __forceinline__ uint32_t uf_find(volatile uint32_t *L, uint32_t x) {
  uint32_t p = L[x];
  for (int it = 0; p != x && it < 8192; ++it) {
    x = p;
    p = L[x];
  }
  return x;
}

__device__ __forceinline__ void uf_union(uint32_t *L, uint32_t a, uint32_t b) {
  volatile uint32_t *Lv = L;
  for (int it = 0; it < 1 << 16; ++it) {
    a = uf_find(Lv, a);
    b = uf_find(Lv, b);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicMin(&L[a], b);   // link the larger root under the smaller
    if (old == a) return;
    a = old;
  }
}

// Seeds of the cluster-seed rule ("randomly pick one cluster" read as a
// uniform choice among the mismatch clusters): for each pair in turn, a
// union-find over the lattice bonds between its mismatch sites labels the
// clusters by their first site in canonical order (c*H + j); with n
// clusters, the k-th root, k = floor(x0 n / 2^32), seeds the pair's flood
// fill.  The labels use the transposed-overlap words, which this rule does
// not need; R holds one root bit per site.
__device__ __forceinline__ void icm_cluster_seeds(const Cta &k, const Shared &sh, int nbits, int r0, int P) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int N = k.geo.N, H = k.geo.H, nchunk = (N + 31) >> 5;
  uint32_t *V = sh.V, *X = sh.V + N, *Lb = sh.V + 2 * N, *R = sh.V + 2 * N + 32 * nchunk;
  volatile uint32_t *Lv = Lb;
  for (int pb = 0; pb < nbits; ++pb) {
    if (r0 + 8 * ((pb >> 3) >> (P - 1)) + (pb & 7) >= k.T || sh.inm[pb] == 0) continue;
    for (int kk = tid; kk < N; kk += nt) Lb[kk] = ((X[kk] >> pb) & 1u) ? (uint32_t)kk : 0xFFFFFFFFu;
    __syncthreads();
    // every bond has one colour-0 end: unite each colour-0 mismatch site
    // with its mismatched neighbours over the bonds present
    for (int j = tid; j < H; j += nt) {
      if (!((X[j] >> pb) & 1u)) continue;
      int nb[6];
      neighbours(k.geo, 0, j, nb);
      const uint32_t miss = ((uint32_t)sh.jn[j] >> 8) & 0x3Fu;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int kk2 = H + nb[d];
        if (((miss >> d) & 1u) == 0u && ((X[kk2] >> pb) & 1u)) uf_union(Lb, (uint32_t)j, (uint32_t)kk2);
      }
    }
    __syncthreads();
    for (int ch = warp; ch < nchunk; ch += (nt >> 5)) {
      const int kk = ch * 32 + lane;
      const bool root = kk < N && ((X[kk] >> pb) & 1u) && uf_find(Lv, (uint32_t)kk) == (uint32_t)kk;
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, root);
      if (lane == 0) R[ch] = m;
    }
    __syncthreads();
    if (warp == 0) {
      int tot = 0;
      for (int ch = lane; ch < nchunk; ch += 32) tot += __popc(R[ch]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
      const int kth = (int)(((uint64_t)sh.ikx[pb] * (uint64_t)tot) >> 32);
      int base = 0;
      for (int ch0 = 0; ch0 < nchunk; ch0 += 32) {
        const int ch = ch0 + lane;
        uint32_t w = ch < nchunk ? R[ch] : 0u;
        const int cn = __popc(w);
        int inc = cn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (lane >= o) inc += y;
        }
        const int ex = base + inc - cn;
        const bool hit = kth >= ex && kth < ex + cn;
        if (hit) {
          int q = kth - ex, pos = 0;
#pragma unroll
          for (int h = 16; h >= 1; h >>= 1) {
            const int cl = __popc(w & ((1u << h) - 1u));
            if (q >= cl) {
              q -= cl;
              w >>= h;
              pos += h;
            }
          }
          V[ch * 32 + pos] |= 1u << pb;
        }
        if (__any_sync(0xFFFFFFFFu, hit)) break;
        base += __shfl_sync(0xFFFFFFFFu, inc, 31);
      }
    }
    __syncthreads();
  }
}

// ICMop of Algorithm S2 for every temperature at once.  With A labels per
// temperature (2 or 4) the labels of temperature r = 8h + i sit in nibble i
// of groups l*Gl + h, and pair p of the temperature's random matching owns
// bit 8 (h A/2 + p) + i of the per-site overlap word X, so the overlaps of
// eight pairs come from one XOR (two labels) or three masked XORs (four).
// The seed of a pair is the k-th site (canonical order c*H + j) with its
// bit set, k = floor(x0 n_minus / 2^32); its cluster grows by a flood fill
// V <- V | (X & OR_nbr V) until no cluster changes.  Clusters larger than
// N/2 flip one whole replica (x1 bit 0: the pair's first or second label),
// smaller ones flip in both replicas; then the energies are updated.
template <bool CSEED>
__device__ void icm_all(const AptArgs &a, const Cta &k, const Shared &sh, uint32_t t) {
  long long pt = clock64();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N = k.geo.N, H = k.geo.H;
  // A labels per temperature form A/2 pairs; label l's groups are
  // l*Gl .. l*Gl + Gl - 1.  Pair p of temperature r = 8h + i owns bit
  // 8 (h P + p) + i of the per-site overlap / cluster words.
  const int A = k.A, P = A >> 1, Gl = k.Gu, nbits = 8 * Gl * P;   // A is 2 or 4
  const int r0 = 8 * k.g0;   // first temperature held here
  const uint32_t *S = sh.S;
  uint32_t *V = sh.V;          // [2][H] cluster bits (one bit per pair)
  uint32_t *X = sh.V + N;      // [2][H] overlap bits
  int *match = sh.ibit + 32;   // [32] matching of the labels of each temperature
  if (tid < nbits) {
    const int pb = tid, beta = pb >> 3, h = beta >> (P - 1), p = beta - h * P, r = r0 + 8 * h + (pb & 7);
    if (r < k.T) {
      const uint4 x = philox((uint32_t)r, t, (uint32_t)p, (k.ent << 8) | TAG_ICM, a.k0, a.k1);
      sh.ikx[pb] = x.x;
      sh.ibit[pb] = (int)(x.y & 1u);
      // Algorithm S2 "randomly partition ICM replicas into pairs": with four
      // labels, one of the three perfect matchings, floor(3 x2 / 2^32) of
      // pair 0's draw; two labels always pair (0, 1)
      if (p == 0) match[r] = A == 4 ? (int)(((uint64_t)x.z * 3u) >> 32) : 0;
    }
  }
  if (tid < 24) sh.imask[tid] = 0;
  if (tid < 64) {
    sh.isz[tid] = 0;
    sh.inm[tid] = 0;
  }
  __syncthreads();
  if (A == 4 && tid < 3 * Gl) {
    // nibble masks of the temperatures of group h that use matching m
    const int h = tid / 3, m = tid - 3 * h;
    uint32_t mk = 0;
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + 8 * h + i;
      if (r < k.T && match[r] == m) mk |= 0xFu << (4 * i);
    }
    sh.swm[16 + tid] = mk;
  }
  __syncthreads();
  // (A) overlaps.  Warp w takes chunks of 32 sites in canonical order; the
  // transpose of the chunk's X words gives lane r the chunk's mismatch
  // bitmask of pair r, kept in Xt[chunk][r].
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5, nchunk = (N + 31) >> 5;
  uint32_t *Xt = sh.V + 2 * N;   // [nchunk][32]
  uint32_t nmis = 0;             // lane r: mismatches of pair r in this warp's chunks
  for (int ch = warp; ch < nchunk; ch += nw) {
    const int kk = ch * 32 + lane;
    uint32_t xb = 0;
    if (kk < N) {
      const int c = kk >= H ? 1 : 0, j = kk - c * H;
      if (A == 2) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if (h >= Gl) break;
          const uint32_t x = S[(2 * h + c) * H + j] ^ S[(2 * (h + Gl) + c) * H + j];
          xb |= nib_to_byte(x) << (8 * h);
        }
      } else {
        // the two labels of pair p depend on each temperature's matching:
        // select nibbles by the matching masks
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h >= Gl) break;
          uint32_t w[4];
#pragma unroll
          for (int l = 0; l < 4; ++l) w[l] = S[(2 * (l * Gl + h) + c) * H + j];
          const uint32_t m0 = sh.swm[16 + 3 * h], m1 = sh.swm[17 + 3 * h], m2 = sh.swm[18 + 3 * h];
          const uint32_t x0 = ((w[0] ^ w[1]) & m0) | ((w[0] ^ w[2]) & m1) | ((w[0] ^ w[3]) & m2);
          const uint32_t x1 = ((w[2] ^ w[3]) & m0) | ((w[1] ^ w[3]) & m1) | ((w[1] ^ w[2]) & m2);
          xb |= (nib_to_byte(x0) << (16 * h)) | (nib_to_byte(x1) << (16 * h + 8));
        }
      }
      if (sh.jn[kk] & 0x8000u) xb = 0;   // a vacancy has no overlap: never a seed or member
      X[kk] = xb;
      V[kk] = 0u;
    }
    const uint32_t col = warp_transpose32(xb);
    Xt[ch * 32 + lane] = col;
    nmis += __popc(col);
  }
  if (lane < nbits && nmis) atomicAdd(&sh.inm[lane], (int)nmis);
  __syncthreads();
  PROF_MARK(4, pt);
  // seeds: warp w finds the k-th mismatch of pairs w, w + nw, ...: chunk
  // counts by popcount, a warp scan over chunks, then the set bit inside
  // the chunk (the cluster-seed rule finds the k-th cluster instead)
  if (CSEED) icm_cluster_seeds(k, sh, nbits, r0, P);
  for (int r = warp; r < nbits && !CSEED; r += nw) {   // r: pair bit
    if (r0 + 8 * ((r >> 3) >> (P - 1)) + (r & 7) >= k.T) continue;
    const int nm = sh.inm[r];
    if (nm == 0) continue;
    const int kth = (int)(((uint64_t)sh.ikx[r] * (uint64_t)nm) >> 32);
    int base = 0;
    for (int ch0 = 0; ch0 < nchunk; ch0 += 32) {
      const int ch = ch0 + lane;
      uint32_t w = ch < nchunk ? Xt[ch * 32 + r] : 0u;
      const int cn = __popc(w);
      int inc = cn;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
      }
      const int ex = base + inc - cn;
      const bool hit = kth >= ex && kth < ex + cn;
      if (hit) {
        // position of set bit number q (from 0) of w: binary search on
        // popcounts of the low half of the remaining window
        int q = kth - ex, pos = 0;
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
          const int cl = __popc(w & ((1u << h) - 1u));
          if (q >= cl) {
            q -= cl;
            w >>= h;
            pos += h;
          }
        }
        atomicOr(&V[ch * 32 + pos], 1u << r);
      }
      if (__any_sync(0xFFFFFFFFu, hit)) break;
      base += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
  __syncthreads();
  PROF_MARK(5, pt);
  // (B) flood fill.  The cluster is the least fixed point of the monotone
  // update V <- V | (X & OR_nbr V).  A thread owns 2x2x2 blocks of sites
  // (bx, by, bz): per pass it reads the 24 outside neighbours of a block and
  // closes the block internally (the cube has diameter 3), so a pass moves
  // a cluster front by up to three sites.  Each site word has one writer,
  // so passes run without inner barriers (a stale neighbour read only delays
  // growth) and a pass with no change anywhere, started after a barrier,
  // proves the fixed point.
  {
    const Geo &g = k.geo;
    const int hx = g.hx, hy = g.Ly >> 1, nblk = N >> 3;
    // plain loads: a pass reads each neighbour word once, after the barrier
    // that ended the previous pass (a compiler fence as well), and a value
    // another thread writes during the pass is only seen one pass later
    const uint32_t *Vv = V;
    // block geometry: site i = dx + 2 dy + 4 dz of block (bx, by, bz) has
    // colour (dx+dy+dz)&1 and index bx + hx (y0 + dy + Ly (z0 + dz)) inside
    // its colour; an outside neighbour is the opposite corner's word of the
    // adjacent block, i.e. a site of this block shifted by one block step
    struct Blk {
      int kk[8];
      uint32_t dx2, dy2, dz2;   // (minus, plus) block steps as two int16 each
      uint32_t ok;              // bits -x,+x,-y,+y,-z,+z: outside neighbour present
    };
    auto make_blk = [&](int blk) {
      Blk B;
      const int rest = (int)fdiv((uint32_t)blk, g.mhx);           // blk / hx
      const int bx = blk - rest * hx;
      const int bz = (int)fdiv((uint32_t)rest, g.mLy2);           // rest / (Ly/2)
      const int by = rest - bz * hy;
      const int y0 = 2 * by, z0 = 2 * bz;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int dx = i & 1, dy = (i >> 1) & 1, dz = i >> 2;
        B.kk[i] = ((dx + dy + dz) & 1) * H + bx + hx * (y0 + dy + g.Ly * (z0 + dz));
      }
      const int LyHx = g.Ly * hx;
      auto pack = [](int m, int p) { return ((uint32_t)m & 0xFFFFu) | ((uint32_t)p << 16); };
      B.dx2 = pack(bx == 0 ? hx - 1 : -1, bx + 1 == hx ? 1 - hx : 1);
      B.dy2 = pack(hx * (y0 == 0 ? g.Ly - 2 : -2), hx * (y0 + 2 == g.Ly ? 2 - g.Ly : 2));
      B.dz2 = pack(LyHx * (z0 == 0 ? g.Lz - 2 : -2), LyHx * (z0 + 2 == g.Lz ? 2 - g.Lz : 2));
      // an open axis has no bond across its ends
      B.ok = 0x3Fu;
      if (k.open & 1u) B.ok &= ~((bx == 0 ? 1u : 0u) | (bx + 1 == hx ? 2u : 0u));
      if (k.open & 2u) B.ok &= ~((y0 == 0 ? 4u : 0u) | (y0 + 2 == g.Ly ? 8u : 0u));
      if (k.open & 4u) B.ok &= ~((z0 == 0 ? 16u : 0u) | (z0 + 2 == g.Lz ? 32u : 0u));
      return B;
    };
    // one relaxation of a block: outside neighbours, then the internal
    // closure (three rounds reach across the cube); writes changed words
    auto relax = [&](const Blk &B, const uint32_t (&x)[8], uint32_t (&v)[8]) {
      uint32_t nv[8];
      const int dxm = (int16_t)(B.dx2 & 0xFFFFu), dxp = (int16_t)(B.dx2 >> 16);
      const int dym = (int16_t)(B.dy2 & 0xFFFFu), dyp = (int16_t)(B.dy2 >> 16);
      const int dzm = (int16_t)(B.dz2 & 0xFFFFu), dzp = (int16_t)(B.dz2 >> 16);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int dx = i & 1, dy = (i >> 1) & 1, dz = i >> 2;
        const uint32_t mx = ((B.ok >> dx) & 1u) ? ~0u : 0u;
        const uint32_t my = ((B.ok >> (2 + dy)) & 1u) ? ~0u : 0u;
        const uint32_t mz = ((B.ok >> (4 + dz)) & 1u) ? ~0u : 0u;
        const uint32_t ox = Vv[B.kk[i ^ 1] + (dx ? dxp : dxm)] & mx;
        const uint32_t oy = Vv[B.kk[i ^ 2] + (dy ? dyp : dym)] & my;
        const uint32_t oz = Vv[B.kk[i ^ 4] + (dz ? dzp : dzm)] & mz;
        nv[i] = v[i] | (x[i] & (ox | oy | oz));
      }
#pragma unroll
      for (int round = 0; round < 3; ++round) {
#pragma unroll
        for (int i = 0; i < 8; ++i) nv[i] |= x[i] & (nv[i ^ 1] | nv[i ^ 2] | nv[i ^ 4]);
      }
      int ch = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (nv[i] != v[i]) {
          V[B.kk[i]] = nv[i];
          v[i] = nv[i];
          ch = 1;
        }
      }
      return ch;
    };
    if (nblk <= nt) {
      // one block per thread: its geometry and cluster words stay in
      // registers across passes (the thread is their only writer)
      Blk B;
      uint32_t v[8];
#if PC_APT_FILL_XREG
      uint32_t x[8];   // the block's overlap words do not change during the fill
#endif
      bool open = false;
      if (tid < nblk) {
        B = make_blk(tid);
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          v[i] = V[B.kk[i]];
#if PC_APT_FILL_XREG
          x[i] = X[B.kk[i]];
          o |= x[i] & ~v[i];
#else
          o |= X[B.kk[i]] & ~v[i];
#endif
        }
        open = o != 0;
      }
      for (int it = 0; it < N; ++it) {
        int changed = 0;
        if (open) {
          uint32_t o = 0;
#if !PC_APT_FILL_XREG
          uint32_t x[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) x[i] = X[B.kk[i]];
#endif
          changed = relax(B, x, v);
#pragma unroll
          for (int i = 0; i < 8; ++i) o |= x[i] & ~v[i];
          open = o != 0;
        }
        if (!__syncthreads_or(changed)) {
#if PC_APT_PROFILE
          if (blockIdx.x < 2 && tid == 0) atomicAdd(&g_apt_prof[16 * blockIdx.x + 11], (unsigned long long)(it + 1));
#endif
          break;
        }
      }
    } else {
      for (int it = 0; it < N; ++it) {
        int changed = 0;
        for (int blk = tid; blk < nblk; blk += nt) {
          const Blk B = make_blk(blk);
          uint32_t x[8], v[8];
          uint32_t open = 0;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            x[i] = X[B.kk[i]];
            v[i] = Vv[B.kk[i]];
            open |= x[i] & ~v[i];
          }
          if (open) changed |= relax(B, x, v);
        }
        if (!__syncthreads_or(changed)) break;
      }
    }
  }
  PROF_MARK(6, pt);
  // (C) cluster sizes: per chunk, lane r counts pair r's cluster sites
  {
    uint32_t sz = 0;
    for (int ch = warp; ch < nchunk; ch += nw) {
      const int kk = ch * 32 + lane;
      sz += __popc(warp_transpose32(kk < N ? V[kk] : 0u));
    }
    if (lane < nbits && sz) atomicAdd(&sh.isz[lane], (int)sz);
  }
  __syncthreads();
  // (D) decisions.  imask[(g P + p)] (g = l Gl + h): nibbles of label l's
  // group h flipped by pair p's cluster; imask[16 + g]: whole-replica flips.
  if (tid < nbits) {
    const int pb = tid, beta = pb >> 3, h = beta >> (P - 1), p = beta - h * P, i = pb & 7,
              r = r0 + 8 * h + i;
    if (r < k.T) {
      const int m = match[r];
      const int la = p == 0 ? 0 : (m == 0 ? 2 : 1);
      const int lb = p == 0 ? m + 1 : (m == 2 ? 2 : 3);
      const int size = sh.isz[pb];
      const uint32_t bit = 1u << (4 * i);
      if (sh.inm[pb] == 0) {
        atomicAdd(&sh.m32[2], 1);
      } else if (a.icm_big && 2 * size > k.nreal) {   // more than half of the spins present
        atomicOr(&sh.imask[16 + (sh.ibit[pb] ? lb : la) * Gl + h], bit);   // one whole replica
        atomicAdd(&sh.m32[4], 1);
      } else {
        atomicOr(&sh.imask[(la * Gl + h) * P + p], bit);                  // cluster, both replicas
        atomicOr(&sh.imask[(lb * Gl + h) * P + p], bit);
        atomicAdd(&sh.m32[3], 1);
      }
    }
  }
  __syncthreads();
  PROF_MARK(7, pt);
  // (E) flips.  With two labels the masks are read once into registers (a
  // store to S could alias them, so they would be reloaded after every one)
  uint32_t fm[4][4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const bool on = A == 2 && h < Gl;
    fm[h][0] = on ? sh.imask[h] : 0u;
    fm[h][1] = on ? sh.imask[16 + h] : 0u;
    fm[h][2] = on ? sh.imask[Gl + h] : 0u;
    fm[h][3] = on ? sh.imask[16 + Gl + h] : 0u;
  }
  for (int kk = tid; kk < N; kk += nt) {
    const int c = kk >= H ? 1 : 0, j = kk - c * H;
    const uint32_t v = V[kk];
    if (A == 2) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        if (h >= Gl) break;
        const uint32_t vv = byte_to_nib((v >> (8 * h)) & 0xFFu);
        uint32_t *p0 = sh.S + (size_t)(2 * h + c) * H + j, *p1 = sh.S + (size_t)(2 * (Gl + h) + c) * H + j;
        const uint32_t a0 = *p0, a1 = *p1;
        *p0 = a0 ^ ((vv & fm[h][0]) | fm[h][1]);
        *p1 = a1 ^ ((vv & fm[h][2]) | fm[h][3]);
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h >= Gl) break;
        const uint32_t n0 = byte_to_nib((v >> (16 * h)) & 0xFFu);
        const uint32_t n1 = byte_to_nib((v >> (16 * h + 8)) & 0xFFu);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const int g = l * Gl + h;
          sh.S[(2 * g + c) * H + j] ^= sh.imask[16 + g] | (n0 & sh.imask[2 * g]) | (n1 & sh.imask[2 * g + 1]);
        }
      }
    }
  }
  __syncthreads();
  PROF_MARK(8, pt);
  // (F) energies after the moves.  A Houdayer move keeps E_a + E_b of its
  // pair (the cluster's outside neighbours agree in both replicas; a whole
  // replica flip changes no energy at h = 0), so only label 0 is recounted
  // and label 1 follows as E_b' = E_a + E_b - E_a'.
  if (A == 2) {
    colour_phase<false, true>(a, k, sh, 1, 0u, Gl);
    __syncthreads();
    for (int b = tid; b < 8 * Gl; b += nt) {
      const int e0 = k.nbonds - 2 * sh.Eacc[b];
      sh.E[b + 8 * Gl] += sh.E[b] - e0;
      sh.E[b] = e0;
      sh.Eacc[b] = 0;
    }
  } else {
    // the pairs change with the temperature: recount every label
    colour_phase<false, true>(a, k, sh, 1, 0u, k.Gc);
    __syncthreads();
    finish_energies(k, sh);
  }
  __syncthreads();
  PROF_MARK(9, pt);
}

// Applies the swap masks of the last attempt (sh.swm) to the words
// [kb, ke) of every group plane ([0, H): colour 0, [H, 2H): colour 1).  A
// split problem's boundary swap (bmask: accepted labels) also writes the
// peer CTA's spins, pushed into `stage`, into this CTA's boundary nibble.
__device__ void swap_words(const Cta &k, const Shared &sh, int kb, int ke, uint32_t bmask,
                           const uint32_t *stage) {
  const int H = k.geo.H, G = k.Gc;
  // groups touched by the swaps, and the groups g whose nibble 7 pairs with
  // nibble 0 of g + 1
  uint32_t touch = 0, cross = 0;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    if (g < G && sh.swm[g]) touch |= 1u << g;
    if (g + 1 < G && sh.swm[8 + g]) cross |= 1u << g;
  }
  // rank 0 receives into nibble 7 of each label's last group, rank 1 into
  // nibble 0 of each label's first group
  const int bsh = k.rank == 0 ? 28 : 0, bgoff = k.rank == 0 ? k.Gu - 1 : 0;
  for (int kk = kb + threadIdx.x; kk < ke; kk += blockDim.x) {
    uint32_t *col = sh.S + kk;   // word (g, c, j) at col[g * 2H]
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      if ((touch >> g) & 1u) {
        const uint32_t w = col[(size_t)g * 2 * H], m = sh.swm[g];
        const uint32_t d = (w ^ (w >> 4)) & m;
        col[(size_t)g * 2 * H] = w ^ (d | (d << 4));
      }
    }
#pragma unroll
    for (int g = 0; g < 7; ++g) {
      if ((cross >> g) & 1u) {
        const uint32_t w0 = col[(size_t)g * 2 * H], w1 = col[(size_t)(g + 1) * 2 * H];
        const uint32_t d = ((w0 >> 28) ^ w1) & 1u;
        col[(size_t)g * 2 * H] = w0 ^ (d << 28);
        col[(size_t)(g + 1) * 2 * H] = w1 ^ d;
      }
    }
    if (bmask) {
      const int e = kk - kb;
      for (int l = 0; l < k.A; ++l) {
        if (!((bmask >> l) & 1u)) continue;
        const uint32_t bit = (stage[64 * l + (e >> 5)] >> (e & 31)) & 1u;
        uint32_t *wp = col + (size_t)(l * k.Gu + bgoff) * 2 * H;
        *wp = (*wp & ~(1u << bsh)) | (bit << bsh);
      }
    }
  }
}

// Split problems: writes this CTA's boundary spins of the words
// [kb, kb + H) (one colour), every label, one bit per site, into the peer
// CTA's stage[par] (distributed shared memory).  Rank 0 sends the last
// (coldest) temperature of its half (nibble 7 of each label's last group),
// rank 1 the first (hottest) of its half (nibble 0 of each label's first
// group).
__device__ void push_boundary(const Cta &k, const Shared &sh, int kb, int par, int w0 = 0) {
  namespace cg = cooperative_groups;
  const int H = k.geo.H;
  uint32_t *pstage = cg::this_cluster().map_shared_rank(sh.stage, k.rank ^ 1) + 256 * par;
  const int sh_own = k.rank == 0 ? 28 : 0, goff = k.rank == 0 ? k.Gu - 1 : 0;
  // warps w0 .. take part
  const int lane = threadIdx.x & 31, nw = (blockDim.x >> 5) - w0;
  for (int base = ((int)(threadIdx.x >> 5) - w0) * 32; base < H; base += nw * 32) {
    const int e = base + lane;
    for (int l = 0; l < k.A; ++l) {
      uint32_t bit = 0;
      if (e < H) bit = (sh.S[(size_t)(l * k.Gu + goff) * 2 * H + kb + e] >> sh_own) & 1u;
      const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
      if (lane == 0) pstage[64 * l + (base >> 5)] = word;
    }
  }
}

// Replica exchange of attempt t (Sec. "Comparison with Adaptive Parallel
// Tempering"; Methods): even t pairs (0,1),(2,3)..., odd t (1,2),(3,4)...;
// each label decides on its own; p_swap = min(1, exp(dbeta dE)).  Accepted
// pairs exchange their p-bit states (SWAR nibble swaps over all sites) and
// energies.  A split problem pushes its boundary spins and energies to the
// peer CTA before one cluster barrier; both CTAs then decide the boundary
// pair from the same energies and random word, and take the peer's spins
// for the accepted labels.  Buffers alternate with the attempt's parity, so
// one barrier per attempt orders every exchange.
template <bool SPLIT>
__device__ void swap_step(const AptArgs &a, const Cta &k, const Shared &sh, int p, uint32_t t) {
#if PC_APT_PROFILE
  long long pt = clock64();
#endif
  const AptProbDev &P = a.prob[p];
  const int A = k.A, q = (int)(t & 1u);
  const int r0 = 8 * k.g0, r1 = min(8 * (k.g0 + k.Gu), k.T);   // temperatures held here
  // local buffer of (label l, temperature r): l * 8 Gu + r - r0
  const int lb = 8 * k.Gu;
  auto swap_table = [&](int r, int dE) {
    const int kk = (-dE) >> 1;
    if (PC_APT_STAGE_SWT && SPLIT && a.stage_swt && kk < kSwtLen) return sh.swt[r * kSwtLen + kk];   // staged at launch
    const uint32_t off = a.swapidx[P.swapidx_off + 2 * r], len = a.swapidx[P.swapidx_off + 2 * r + 1];
    return ((uint32_t)kk < len) ? a.swaptab[off + kk] : 0u;
  };
  const int par = (int)(t & 1u);
  const int warp = threadIdx.x >> 5;
  if (k.split) {
    // energies of this side of the boundary pair, and its colour-1 spins
    // (warps 1 ..; warp 0 starts on the decisions meanwhile)
    const int rb_own = k.rank == 0 ? r1 - 1 : r0;
    int *pe = cooperative_groups::this_cluster().map_shared_rank(sh.xch, k.rank ^ 1) + 4 * par;
    if (threadIdx.x < A) pe[threadIdx.x] = sh.E[threadIdx.x * lb + rb_own - r0];
    if (warp >= 1) push_boundary(k, sh, k.geo.H, par, 1);
    // the boundary pair's draws do not depend on the energies: warp 1 takes
    // them now, before the cluster barrier
    const int rb = k.rank == 0 ? r1 : r0;
    const int lane1 = threadIdx.x - 32;
    if (warp == 1 && lane1 < A && rb < k.T && ((rb - 1) & 1) == q)
      sh.xch[18 + lane1] =
          (int)philox((uint32_t)(rb - 1), t, (uint32_t)lane1, (k.ent << 8) | TAG_SWAP, a.k0, a.k1).x;
  }
  PROF_MARK(12, pt);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane < 16) sh.swm[lane] = 0;
    __syncwarp();
    const int first = r0 + q;                          // r0 is even
    const int np = r1 - 1 > first ? (r1 - first) / 2 : 0;   // pairs (r, r + 1), r + 1 < r1
    int any = 0;
    // joint mode (Algorithm S2 read literally): lane idx decides pair idx
    // for all labels at once, with the summed energy difference
    const int nd = a.joint_swap ? np : np * A;
    for (int idx = lane; idx < nd; idx += 32) {
      const int r = first + 2 * (a.joint_swap ? idx : idx / A), al = a.joint_swap ? 0 : idx % A;
      // the draw first: it does not depend on the energies
      const uint32_t x0 = philox((uint32_t)r, t, (uint32_t)al, (k.ent << 8) | TAG_SWAP, a.k0, a.k1).x;
      const int bA = al * lb + r - r0, bB = bA + 1;
      int dE = sh.E[bB] - sh.E[bA];
      if (a.joint_swap)
        for (int l = 1; l < A; ++l) dE += sh.E[l * lb + r - r0 + 1] - sh.E[l * lb + r - r0];
      const bool acc = dE >= 0 || x0 < swap_table(r, dE);
      for (int l = al; l < (a.joint_swap ? A : al + 1); ++l) {
        const int lA = l * lb + r - r0, lB = lA + 1;
        sh.satt[r * A + l] += 1;
        if (acc) {
          sh.sacc[r * A + l] += 1;
          const int eA = sh.E[lA];
          sh.E[lA] = sh.E[lB];
          sh.E[lB] = eA;
          if ((lA & 7) != 7) atomicOr(&sh.swm[lA >> 3], 1u << (4 * (lA & 7)));
          else sh.swm[8 + (lA >> 3)] = 1u;
          any = 1;
        }
      }
    }
    any = __any_sync(0xFFFFFFFFu, any);
    if (lane == 0) sh.m32[5] = any;
  }
  PROF_MARK(13, pt);
  uint32_t bmask = 0;
  if (k.split) {
    cooperative_groups::this_cluster().sync();   // the peer's energies and spins have landed
    // the pair (rb - 1, rb) across the two CTAs, if this attempt's parity
    const int rb = k.rank == 0 ? r1 : r0;
    if (threadIdx.x == 0) {
      uint32_t accm = 0;
      if (rb < k.T && ((rb - 1) & 1) == q) {
        const int rb_own = k.rank == 0 ? r1 - 1 : r0;
        const int *pe = sh.xch + 4 * par;   // the peer's energies
        int e_lo[4], e_hi[4];               // energies at rb - 1 (rank 0's) and rb (rank 1's)
        for (int l = 0; l < A; ++l) {
          const int own = sh.E[l * lb + rb_own - r0];
          e_lo[l] = k.rank == 0 ? own : pe[l];
          e_hi[l] = k.rank == 0 ? pe[l] : own;
        }
        for (int l = 0; l < (a.joint_swap ? 1 : A); ++l) {
          int dE = e_hi[l] - e_lo[l];
          if (a.joint_swap)
            for (int m = 1; m < A; ++m) dE += e_hi[m] - e_lo[m];
          // the draw taken by warp 1 before the barrier
          const bool acc = dE >= 0 || (uint32_t)sh.xch[18 + l] < swap_table(rb - 1, dE);
          if (acc) accm |= a.joint_swap ? (1u << A) - 1u : 1u << l;
        }
        for (int l = 0; l < A; ++l) {
          if (k.rank == 0) sh.satt[(rb - 1) * A + l] += 1;   // counted once, by rank 0
          if ((accm >> l) & 1u) {
            if (k.rank == 0) sh.sacc[(rb - 1) * A + l] += 1;
            sh.E[l * lb + rb_own - r0] = k.rank == 0 ? e_hi[l] : e_lo[l];
          }
        }
      }
      sh.xch[8] = (int)accm;
    }
    __syncthreads();
    bmask = (uint32_t)sh.xch[8];
  } else {
    __syncthreads();
  }
  PROF_MARK(14, pt);
  if (!sh.m32[5] && !bmask) return;
  // colour 0 is rewritten by the next sweep without being read (a Gibbs
  // update depends on the neighbours only), so only colour 1 moves now; the
  // kernel applies the last attempt's swaps to colour 0 before it stores
  swap_words(k, sh, k.geo.H, 2 * k.geo.H, bmask, sh.stage + 256 * par);
  PROF_MARK(15, pt);
}

// MODE (pc::APT_MODE_*) and SPLIT (a cluster of two CTAs per problem) are
// template arguments, so that each kernel carries only its own code (the
// launcher picks the instantiation from a.mode and a.split).
template <int MODE, bool SPLIT, bool CSEED>
__global__ void __launch_bounds__(512) apt_kernel(const AptArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int cta = blockIdx.x;
  const int p = a.cta_prob[cta];
  const AptProbDev &P = a.prob[p];
  Cta k;
  k.geo.Lx = P.Lx;
  k.geo.Ly = P.Ly;
  k.geo.Lz = P.Lz;
  k.geo.N = P.N;
  k.geo.H = P.N >> 1;
  k.geo.hx = P.Lx >> 1;
  k.geo.mhx = P.mhx;
  k.geo.mLy = P.mLy;
  k.geo.mLy2 = P.mLy2;
  k.nbonds = P.nbonds;
  k.nreal = P.nreal;
  k.open = P.open;
  k.T = P.T;
  k.Tp = P.Tp;
  k.A = P.A;
  k.B = P.B;
  k.g0 = a.cta_g0[cta];
  k.Gc = a.cta_gc[cta];
  k.Bc = min(8 * k.Gc, P.B - 8 * k.g0);
  k.split = SPLIT;
  k.rank = SPLIT ? (int)cooperative_groups::this_cluster().block_rank() : 0;
  if (MODE == pc::APT_MODE_APT || MODE == pc::APT_MODE_ENERGY) {
    k.Gu = k.Gc / k.A;   // A is 1, 2 or 4
    k.Glp = k.Tp >> 3;
  } else {
    k.Gu = k.Gc;
    k.Glp = (k.B + 7) >> 3;
  }
  k.ent = P.ent;
  k.nch = a.cta_nch[cta];
  k.tpc = blockDim.x / k.nch;
  k.gc = (k.Gc + k.nch - 1) / k.nch;
  const int N = P.N;
  // both CTAs of a split problem carve shared memory alike (for the larger
  // of the two parts), so that distributed-shared-memory addresses correspond
  const int Gcarve = SPLIT ? k.A * max(k.Gu, k.Glp - k.Gu) : k.Gc, G8 = 8 * Gcarve;
  const int64_t s0 = a.ctr[0], t0 = a.ctr[1];
  const bool icm = MODE == pc::APT_MODE_APT && a.icm;
  // carve shared memory
  Shared sh;
  uint32_t *cur = smem;
  sh.S = cur;            cur += (size_t)Gcarve * N;
  sh.thr = cur;          cur += 16 * G8;
  // each group's 256-byte block of thrh on a 256-byte boundary of the
  // shared window (the same padding in both CTAs of a cluster)
  cur += ((256u - ((uint32_t)__cvta_generic_to_shared(cur) & 255u)) & 255u) >> 2;
  sh.thrh = reinterpret_cast<uint16_t *>(cur);   cur += 16 * G8;   // uses half of its carve
  sh.temp_of = reinterpret_cast<int32_t *>(cur);  cur += G8;
  sh.buf_of = reinterpret_cast<int32_t *>(cur);   cur += G8;
  sh.E = reinterpret_cast<int32_t *>(cur);        cur += G8;
  sh.Eacc = reinterpret_cast<int32_t *>(cur);     cur += G8;
  sh.satt = reinterpret_cast<int32_t *>(cur);     cur += 128;
  sh.sacc = reinterpret_cast<int32_t *>(cur);     cur += 128;
  sh.m32 = reinterpret_cast<int32_t *>(cur);      cur += 8;
  cur += ((uintptr_t)cur & 4) ? 1 : 0;            // 8-byte align
  sh.m64 = reinterpret_cast<int64_t *>(cur);      cur += 8;
  sh.sum1 = reinterpret_cast<int64_t *>(cur);     cur += 2 * G8;
  sh.sum2 = reinterpret_cast<int64_t *>(cur);     cur += 2 * G8;
  sh.hist = reinterpret_cast<int32_t *>(cur);     cur += MODE == pc::APT_MODE_PILOT ? k.T * a.n_bins : 0;
  sh.ikx = cur;                                   cur += 64;
  sh.ibit = reinterpret_cast<int32_t *>(cur);     cur += 64;
  sh.inm = reinterpret_cast<int32_t *>(cur);      cur += 64;
  sh.isz = reinterpret_cast<int32_t *>(cur);      cur += 64;
  sh.imask = cur;                                 cur += 24;
  sh.swm = cur;                                   cur += 24;
  sh.gmap = reinterpret_cast<int32_t *>(cur);     cur += 8;
  sh.xch = reinterpret_cast<int32_t *>(cur);      cur += 24;
  sh.stage = cur;                                 cur += SPLIT ? 512 : 0;
  sh.swt = cur;                                   cur += (SPLIT && MODE == pc::APT_MODE_APT && a.stage_swt) ? (size_t)max(k.T - 1, 0) * kSwtLen : 0;
  sh.V = cur;                                     cur += icm ? (size_t)3 * N + 31 + ((N + 31) >> 5) : 0;   // V, X, Xt, R
  sh.jn = reinterpret_cast<uint16_t *>(cur);

  // load state: local group u is global group gmap[u]
  if (threadIdx.x < 8)
    sh.gmap[threadIdx.x] = (threadIdx.x / max(k.Gu, 1)) * k.Glp + k.g0 + threadIdx.x % max(k.Gu, 1);
  __syncthreads();
  for (int i = threadIdx.x; i < k.Gc * N; i += blockDim.x)
    sh.S[i] = a.spins[P.spin_off + (size_t)sh.gmap[i / N] * N + i % N];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sh.jn[i] = a.jneg[P.jneg_off + i];
  for (int b = threadIdx.x; b < 8 * k.Gc; b += blockDim.x) {
    const int gb = 8 * sh.gmap[b >> 3] + (b & 7);
    const int tb = (b < k.Bc) ? a.temp_of[P.buf_off + gb] : 0;
    sh.temp_of[b] = tb;
    sh.buf_of[b] = (b < k.Bc) ? a.buf_of[P.buf_off + gb] : 0;
    sh.E[b] = (b < k.Bc) ? a.E[P.buf_off + gb] : 0;
    sh.Eacc[b] = 0;
    sh.sum1[b] = 0;
    sh.sum2[b] = 0;
    for (int e = 0; e < 16; ++e) {
      const uint32_t th = a.pbit[P.pbit_off + 16 * tb + e];
      sh.thr[16 * b + e] = th;
      sh.thrh[16 * b + e] = (uint16_t)(th >> 16);
    }
  }
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    sh.satt[i] = 0;
    sh.sacc[i] = 0;
  }
  if (threadIdx.x < 24) sh.xch[threadIdx.x] = 0;
  if (PC_APT_STAGE_SWT && SPLIT && MODE == pc::APT_MODE_APT && a.stage_swt)
    for (int i = threadIdx.x; i < (k.T - 1) * kSwtLen; i += blockDim.x) {
      const int r = i / kSwtLen, kk = i - r * kSwtLen;
      const uint32_t off = a.swapidx[P.swapidx_off + 2 * r], len = a.swapidx[P.swapidx_off + 2 * r + 1];
      sh.swt[i] = ((uint32_t)kk < len) ? a.swaptab[off + kk] : 0u;
    }
  if (MODE == pc::APT_MODE_PILOT)
    for (int i = threadIdx.x; i < k.T * a.n_bins; i += blockDim.x) sh.hist[i] = 0;
  if (threadIdx.x == 0) {
    sh.m64[0] = a.best_E[p];
    sh.m64[1] = a.best_sweep[p];
    sh.m64[2] = a.hit_sweep[p];
    sh.m64[3] = a.target[p];
    sh.m32[0] = a.best_buf[p];
    sh.m32[1] = 0;
    sh.m32[2] = sh.m32[3] = sh.m32[4] = 0;
    sh.m32[5] = sh.m32[6] = sh.m32[7] = 0;
  }
  __syncthreads();

  if (MODE == pc::APT_MODE_ENERGY) {
    colour_phase<false, true>(a, k, sh, 1, 0u, k.Gc);
    __syncthreads();
    finish_energies(k, sh);
    __syncthreads();
  } else {
    long long pt = clock64();
    for (int it = 0; it < a.n_iter; ++it) {
      const uint32_t t = (uint32_t)(t0 + it);
      for (int qq = 0; qq < a.spp; ++qq) {
        const uint32_t s = (uint32_t)(s0 + (int64_t)it * a.spp + qq);
        colour_phase<true, false>(a, k, sh, 0, s, k.Gc);
        __syncthreads();
        PROF_MARK(0, pt);
        if (MODE == pc::APT_MODE_APT && qq + 1 < a.spp) {
          // the APT mode reads energies only after the attempt's last sweep
          colour_phase<true, false>(a, k, sh, 1, s, k.Gc);
          __syncthreads();
          PROF_MARK(1, pt);
          continue;
        }
        colour_phase<true, true>(a, k, sh, 1, s, k.Gc);
        __syncthreads();
        finish_energies(k, sh);
        __syncthreads();
        PROF_MARK(1, pt);
        if (MODE == pc::APT_MODE_LADDER) {
          if ((int64_t)it * a.spp + qq >= a.window_from)
            for (int b = threadIdx.x; b < k.Bc; b += blockDim.x) {
              const int64_t e = sh.E[b];
              sh.sum1[b] += e;
              sh.sum2[b] += e * e;
            }
        } else if (MODE == pc::APT_MODE_PILOT) {
          if ((int64_t)s >= a.window_from)
            for (int b = threadIdx.x; b < k.Bc; b += blockDim.x) {
              const int64_t span = 3 * (int64_t)N;
              const int64_t num = ((int64_t)sh.E[b] + span) * a.n_bins;
              int64_t bin = num < 0 ? 0 : num / span;
              if (bin > a.n_bins - 1) bin = a.n_bins - 1;
              atomicAdd(&sh.hist[sh.temp_of[b] * a.n_bins + (int)bin], 1);
            }
        }
      }
      if (MODE != pc::APT_MODE_APT) continue;
      const int64_t sweeps = s0 + (int64_t)(it + 1) * a.spp;
      best_update(a, k, sh, p, sweeps);
      PROF_MARK(2, pt);
      if (icm) {
        icm_all<CSEED>(a, k, sh, t);
        pt = clock64();
        best_update(a, k, sh, p, sweeps);
        PROF_MARK(10, pt);
      }
      swap_step<SPLIT>(a, k, sh, p, t);
      __syncthreads();
      PROF_MARK(3, pt);
    }
  }

  // every thread's last histogram / sum update lands before the write-back,
  // and colour 0 takes the last attempt's swaps
  __syncthreads();
  if (MODE == pc::APT_MODE_APT && a.n_iter > 0) {
    const int lpar = (int)((t0 + a.n_iter - 1) & 1);   // parity of the last attempt
    uint32_t bmask = 0;
    if (k.split) {
      // colour-0 spins of the last boundary swap, and this rank's best
      // candidate, to the peer (the other parity's buffers are free)
      push_boundary(k, sh, 0, lpar ^ 1);
      if (threadIdx.x == 0) {
        int *px = cooperative_groups::this_cluster().map_shared_rank(sh.xch, k.rank ^ 1);
        px[12] = (int)sh.m64[0];
        px[13] = sh.m32[0];
        px[14] = (int)(uint32_t)((uint64_t)sh.m64[1] & 0xFFFFFFFFu);
        px[15] = (int)(uint32_t)((uint64_t)sh.m64[1] >> 32);
        px[16] = (int)(uint32_t)((uint64_t)sh.m64[2] & 0xFFFFFFFFu);
        px[17] = (int)(uint32_t)((uint64_t)sh.m64[2] >> 32);
      }
      cooperative_groups::this_cluster().sync();   // last access to the peer's memory
      if (threadIdx.x == 0) {
        const int64_t pE = sh.xch[12];
        const int64_t psw = (int64_t)(((uint64_t)(uint32_t)sh.xch[15] << 32) | (uint32_t)sh.xch[14]);
        const int64_t phit = (int64_t)(((uint64_t)(uint32_t)sh.xch[17] << 32) | (uint32_t)sh.xch[16]);
        // rank 0's candidate against rank 1's: lower energy, earlier sweep,
        // then rank 0 (its slots are the lower ones)
        const int64_t E0 = k.rank == 0 ? sh.m64[0] : pE, E1 = k.rank == 0 ? pE : sh.m64[0];
        const int64_t S0 = k.rank == 0 ? sh.m64[1] : psw, S1 = k.rank == 0 ? psw : sh.m64[1];
        const bool win1 = E1 < E0 || (E1 == E0 && S1 < S0);
        int copy = 0;
        if (k.rank == 0 && win1) {
          sh.m64[0] = pE;
          sh.m64[1] = psw;
          sh.m32[0] = sh.xch[13];
        }
        if (k.rank == 1) copy = win1 && sh.m64[0] == E1 && sh.m64[1] == S1 && sh.m64[1] >= s0;
        const int64_t h = sh.m64[2];
        sh.m64[2] = h < 0 ? phit : (phit < 0 ? h : min(h, phit));
        sh.m32[1] = copy;
      }
      __syncthreads();
      bmask = (uint32_t)sh.xch[8];
      if (sh.m32[1]) {   // rank 1 found the problem's best: it moves its state
        const AptProbDev &Pb = a.prob[p];
        for (int i = threadIdx.x; i < N; i += blockDim.x)
          a.best_spins[Pb.best_off + i] = a.best_spins2[Pb.best_off + i];
      }
    }
    if (sh.m32[5] || bmask) {
      swap_words(k, sh, 0, k.geo.H, bmask, sh.stage + 256 * (lpar ^ 1));
      __syncthreads();
    }
  }
  // store state
  for (int i = threadIdx.x; i < k.Gc * N; i += blockDim.x)
    a.spins[P.spin_off + (size_t)sh.gmap[i / N] * N + i % N] = sh.S[i];
  for (int b = threadIdx.x; b < k.Bc; b += blockDim.x) {
    const int gb = 8 * sh.gmap[b >> 3] + (b & 7);
    a.temp_of[P.buf_off + gb] = sh.temp_of[b];
    a.buf_of[P.buf_off + gb] = sh.buf_of[b];
    a.E[P.buf_off + gb] = sh.E[b];
    if (MODE == pc::APT_MODE_LADDER) {
      a.sum1[P.buf_off + gb] = sh.sum1[b];
      a.sum2[P.buf_off + gb] = sh.sum2[b];
    }
  }
  if (MODE == pc::APT_MODE_PILOT)
    for (int i = threadIdx.x; i < k.T * a.n_bins; i += blockDim.x)
      atomicAdd(reinterpret_cast<unsigned long long *>(&a.hist[P.hist_off + i]),
                (unsigned long long)sh.hist[i]);
  if (MODE == pc::APT_MODE_APT) {
    // statistics: both CTAs of a split problem add theirs
    unsigned long long *st = reinterpret_cast<unsigned long long *>(a.stats + P.stat_off);
    const int npair = (k.T - 1) * k.A;
    for (int i = threadIdx.x; i < npair; i += blockDim.x) {
      if (sh.satt[i]) atomicAdd(st + i, (unsigned long long)sh.satt[i]);
      if (sh.sacc[i]) atomicAdd(st + npair + i, (unsigned long long)sh.sacc[i]);
    }
    if (threadIdx.x < 3 && sh.m32[2 + threadIdx.x])
      atomicAdd(st + 2 * npair + threadIdx.x, (unsigned long long)sh.m32[2 + threadIdx.x]);
    if (threadIdx.x == 0 && k.rank == 0) {
      a.best_E[p] = sh.m64[0];
      a.best_sweep[p] = sh.m64[1];
      a.hit_sweep[p] = sh.m64[2];
      a.best_buf[p] = sh.m32[0];
    }
  }
}

__global__ void apt_advance_kernel(int64_t *ctr, int64_t sweeps, int64_t swaps) {
  ctr[0] += sweeps;
  ctr[1] += swaps;
}

// Random initial state of every replica: +1 iff the init half-word < 2^15.
__global__ void apt_init_kernel(const AptArgs a, int n_prob) {
  const int p = blockIdx.y;
  if (p >= n_prob) return;
  const AptProbDev &P = a.prob[p];
  const int N = P.N, H = N >> 1;
  const int G = (P.B + 7) >> 3;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G * N; idx += gridDim.x * blockDim.x) {
    const int g = idx / N, rem = idx - g * N, c = rem / H, j = rem - c * H;
    const uint4 x = philox((uint32_t)j, 0u, ((uint32_t)c << 16) | (uint32_t)g,
                           (P.ent << 8) | a.tag_init, a.k0, a.k1);
    uint32_t w = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) w |= (half_lo(x, i) < 0x8000u) ? (1u << (4 * i)) : 0u;
    a.spins[P.spin_off + idx] = w;
  }
}

}  // namespace

namespace pc {

size_t apt_smem_bytes(int N, int Gc, int nwarps, int mode, int icm, int T, int n_bins, int stage_swt) {
  const size_t G8 = 8 * (size_t)Gc;
  size_t words = (size_t)Gc * N + 32 * G8 + 4 * G8 + 128 + 8 + 1 + 16 + 8 * G8;
  words += 4 * 64 + 24 + 24 + 128 + 8 + 24 + 512;   // + larger swap stats, group map, exchange, stage
  if (mode == APT_MODE_PILOT) words += (size_t)T * n_bins;
  if (mode == APT_MODE_APT && stage_swt) words += (size_t)(T > 1 ? T - 1 : 0) * kSwtLen;   // staged swap tables
  // V, X, the transposed X (or the cluster labels) and the root masks
  if (mode == APT_MODE_APT && icm) words += (size_t)3 * N + 31 + (size_t)((N + 31) >> 5);
  return words * 4 + (size_t)N * 2 + 16 + 256;   // + the threshold table's alignment
}

template <int MODE, bool CSEED>
int apt_launch_mode(const AptArgs &a, int n_cta, int tpb, size_t smem, cudaStream_t st) {
  if (!a.split) {
    apt_kernel<MODE, false, CSEED><<<n_cta, tpb, smem, st>>>(a);
  } else {
    // split problems: consecutive CTA pairs form one cluster
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_cta);
    cfg.blockDim = dim3((unsigned)tpb);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.prio) {   // a mixed placement starts its clusters (the largest problems) first
      attr[1].id = cudaLaunchAttributePriority;
      attr[1].val.priority = a.prio;
      cfg.numAttrs = 2;
    }
    PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, apt_kernel<MODE, true, CSEED>, a));
  }
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

int apt_launch(const AptArgs &a, int n_cta, int tpb, size_t smem, cudaStream_t st) {
  if (n_cta <= 0) return PC_OK;
  // raise the dynamic shared-memory limit of every mode's kernel once per
  // device (never inside a stream capture: the first launch on a device
  // happens at load time)
  static size_t set_for[64] = {0};
  int dev = 0;
  PC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PC_EINVAL, "device index out of range");
  if (smem > set_for[dev]) {
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_APT, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_APT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_APT, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_APT, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_LADDER, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_LADDER, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_PILOT, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_PILOT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_ENERGY, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(apt_kernel<pc::APT_MODE_ENERGY, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set_for[dev] = smem;
  }
  switch (a.mode) {
    case pc::APT_MODE_APT:
      // the cluster-seed ICM rule has an instantiation of its own, so the
      // default rule's code is compiled without it
      return a.icm_seed ? apt_launch_mode<pc::APT_MODE_APT, true>(a, n_cta, tpb, smem, st)
                        : apt_launch_mode<pc::APT_MODE_APT, false>(a, n_cta, tpb, smem, st);
    case pc::APT_MODE_LADDER: return apt_launch_mode<pc::APT_MODE_LADDER, false>(a, n_cta, tpb, smem, st);
    case pc::APT_MODE_PILOT: return apt_launch_mode<pc::APT_MODE_PILOT, false>(a, n_cta, tpb, smem, st);
    case pc::APT_MODE_ENERGY: return apt_launch_mode<pc::APT_MODE_ENERGY, false>(a, n_cta, tpb, smem, st);
    default: return fail(PC_EINVAL, "unknown kernel mode");
  }
}

#if PC_APT_PROFILE
extern "C" int pc_apt_profile_read(unsigned long long *out, int reset) {
  PC_CUDA_TRY(cudaMemcpyFromSymbol(out, g_apt_prof, sizeof(unsigned long long) * 32));
  if (reset) {
    unsigned long long z[32] = {0};
    PC_CUDA_TRY(cudaMemcpyToSymbol(g_apt_prof, z, sizeof(z)));
  }
  return PC_OK;
}
#endif

int apt_advance_launch(int64_t *ctr, int64_t sweeps, int64_t swaps, cudaStream_t st) {
  apt_advance_kernel<<<1, 1, 0, st>>>(ctr, sweeps, swaps);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

int apt_init_launch(const AptArgs &a, int n_prob, int max_words, cudaStream_t st) {
  if (n_prob <= 0) return PC_OK;
  const int tpb = 256;
  int bx = (max_words + tpb - 1) / tpb;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  dim3 grid((unsigned)bx, (unsigned)n_prob);
  apt_init_kernel<<<grid, tpb, 0, st>>>(a, n_prob);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

}  // namespace pc
