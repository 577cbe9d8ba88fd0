// p-computer kernels on general sparse graphs: APT with replica exchange,
// ICM and minimum-energy tracking (Algorithm S2) and DT-SQA on the
// replicated network (Eq. S.3, Algorithm S1), both swept colour class by
// colour class as the colormap of the paper's graph-coloured architecture
// prescribes (Methods, "Graph Coloring of 3D Cubic Spin Glass Instances").
//
// Layout: one 32-bit word per (vertex, label) holds 32 replicas.  In APT
// they are the 32 temperatures of one label and a thread owns a (vertex,
// label) pair: the field of all 32 replicas is summed bit-sliced over the
// neighbour words, then each replica looks up Eq. neuron's threshold and
// compares it with its half of a Philox block that serves 8 replicas (16-bit
// halves; the refine block settles ties exactly, as in the lattice kernels).
// In DT-SQA the 32 bits are 32 independent runs and a thread owns one
// (slice, vertex) entry of the replicated network, in the same way.
#include <cuda_runtime.h>

#include <climits>
#include <cooperative_groups.h>
#include <cstdint>

#include "device.cuh"
#include "graph_dev.h"
#include "internal.h"

namespace pc {
namespace {

using pcdev::half_hi;
using pcdev::half_lo;
using pcdev::philox;

// Counter tags of the general-graph draws (the lattice kernels use 1..14).
enum : uint32_t {
  TAG_G_INIT = 15, TAG_G_SWEEP = 16, TAG_G_REFINE = 17, TAG_G_SWAP = 18, TAG_G_ICM = 19,
  TAG_GS_INIT = 20, TAG_GS_SWEEP = 21, TAG_GS_REFINE = 22
};

struct GShared {
  int off[kGMaxColours + 1];
  int32_t E[4][32];              // energy of label a, temperature r
  uint32_t wcnt[kGWarps][32];    // per-warp bit counts (ICM)
  uint32_t x0[2][32], x1[2][32]; // ICM draws per pair set and temperature
  uint32_t mcode[32];            // 4-label matching per temperature
  uint32_t nm[32];               // mismatch counts
  uint32_t sel[2][4];            // bit r: label k is the first / second of the pair
  uint32_t whole[4];             // bit r: label k flips entirely
  uint32_t small;                // bit r: the cluster flips in both replicas
  uint32_t swmask[4];            // accepted swaps per label (bit r: pair r, r+1)
  uint32_t att[128], acc[128];   // swap counters [r * A + a]
  unsigned long long icm[3];
  long long bestE, bestSweep, bestSlot, hit, target;
  int copy_slot;
};

struct GCta {
  int n, C, T, Imax, tid, lane, warp;
  int ths;                       // row length of the [temperature][field] table
  int ushift;                    // (entry >> 8) - ubase >> ushift = neighbour index
  uint32_t ubase;                // byte offset of the spin words from the dynamic base
  const char *dynb;              // dynamic shared-memory base
  uint32_t ent, k0, k1;
  uint32_t tag_init, tag_sweep, tag_refine;
  const int2 *vinfo;
  const uint32_t *adj;
  uint32_t *S;                   // [n][A]
  uint32_t *X;                   // [n] overlap mismatch (ICM)
  volatile uint32_t *Cl;         // [n] cluster bits (ICM)
  const uint32_t *Th;            // [2 Imax + 1][32]
  uint32_t *best_bits;
};

__device__ __forceinline__ int vi_deg(int2 v) { return v.y & 1023; }
__device__ __forceinline__ int vi_kl(int2 v) { return (v.y >> 10) & 1023; }
__device__ __forceinline__ int vi_h(int2 v) { return (int)(int8_t)(uint8_t)((uint32_t)v.y >> 20); }
__device__ __forceinline__ int ent_w(uint32_t e) { return (int)(int8_t)(uint8_t)(e & 0xFFu); }

template <bool SM>
__device__ __forceinline__ uint32_t ld_adj(const uint32_t *ad, int e) {
  if (SM) return ad[e];
  return __ldg(ad + e);
}
template <bool SM>
__device__ __forceinline__ int2 ld_vi(const int2 *vi, int p) {
  if (SM) return vi[p];
  return __ldg(vi + p);
}

// ---------------------------------------------------------------- bit-sliced sweeps
// A thread owns one (vertex, label) pair: its 32-bit spin word holds the
// label's 32 temperatures.  The field of all 32 replicas is summed
// bit-sliced: with t = the neighbour's word, inverted when w < 0 (bit set:
// w s_u = +|w|), C = sum_u |w_vu| t_u is kept as NP bit planes, and
// I = 2 C - W + h with W = sum_u |w_vu|.  Each replica then reads its count,
// looks up Eq. neuron's threshold in a [temperature][field] table (rows of
// odd length 2 Imax + 1, so lanes with different fields hit different
// banks) and compares it with its half of the group's Philox block.

// Adds wabs * t (wabs in 1..127) to the bit-sliced counter P (ripple carry).
template <int NP>
__device__ __forceinline__ void vadd(uint32_t (&P)[NP], uint32_t t, uint32_t wabs) {
  if (wabs == 1u) {
    uint32_t c = t;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const uint32_t n = P[q] & c;
      P[q] ^= c;
      c = n;
    }
    return;
  }
#pragma unroll
  for (int b = 0; b < 7; ++b) {
    if (!((wabs >> b) & 1u)) continue;
    uint32_t c = t;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if (q < b) continue;
      const uint32_t n = P[q] & c;
      P[q] ^= c;
      c = n;
    }
  }
}

// Count of replica r held in the planes (r a compile-time constant after unrolling).
template <int NP>
__device__ __forceinline__ int vget(const uint32_t (&P)[NP], int r) {
  int C = 0;
#pragma unroll
  for (int q = 0; q < NP; ++q) C |= (int)((P[q] >> r) & 1u) << q;
  return C;
}

// Bits 8g .. 8g+3 of w as the bytes of lo (bit 8g + i in byte i) and bits
// 8g+4 .. 8g+7 as the bytes of hi: the four bits of a nibble times
// 1 + 2^7 + 2^14 + 2^21 land, without carries, on bits 0, 8, 16 and 24.
__device__ __forceinline__ void spread_byte(uint32_t w, int g, uint32_t &lo, uint32_t &hi) {
  const uint32_t x = __byte_perm(w, 0u, 0x4440u + (uint32_t)g);
  lo = ((x & 0xFu) * 0x00204081u) & 0x01010101u;
  hi = ((x >> 4) * 0x00204081u) & 0x01010101u;
}

// Counts of replicas 8g .. 8g+7 from the NP planes, doubled, as bytes:
// C2lo holds 2 C of replicas 8g .. 8g+3, C2hi of 8g+4 .. 8g+7 (2 C is at
// most 2 (2^NP - 1) <= 254, so no byte carries into the next).
template <int NP>
__device__ __forceinline__ void counts2_bytes(const uint32_t (&P)[NP], int g, uint32_t &C2lo, uint32_t &C2hi) {
  C2lo = 0u;
  C2hi = 0u;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    uint32_t l, h;
    spread_byte(P[q], g, l, h);
    C2lo += l << (q + 1);
    C2hi += h << (q + 1);
  }
}

// Adds the neighbours [e0, e1) of one vertex, label a, into the planes;
// returns their sum of |w|.
template <int A, int NP, bool SM>
__device__ __forceinline__ int vfield(const char *dynb, const uint32_t *ad, int e0, int e1, int a,
                                      uint32_t (&P)[NP]) {
  int W = 0;
  for (int e = e0; e < e1; ++e) {
    const uint32_t en = ld_adj<SM>(ad, e);
    const int w = ent_w(en);
    uint32_t t = *reinterpret_cast<const uint32_t *>(dynb + (en >> 8) + 4 * a);
    if (w < 0) t = ~t;
    const uint32_t wabs = (uint32_t)(w < 0 ? -w : w);
    vadd<NP>(P, t, wabs);
    W += (int)wabs;
  }
  return W;
}

// Item i of a phase -> (vertex offset, label): the 32 threads of a warp share
// a label and take 32 consecutive vertices.
template <int A>
__device__ __forceinline__ void item_of(int i, int &v, int &a) {
  const int wi = i >> 5;
  a = wi % A;
  v = 32 * (wi / A) + (i & 31);
}

// Random initial states (Algorithm S2): replica b = 32 a + r takes half
// b & 7 of P(j, 0, (c << 16) | (b >> 3), (e << 8) | TAG_G_INIT); +1 iff it is
// below 2^15.
template <int A>
__device__ void g_init(const GCta &k, GShared &sh) {
  const uint32_t c3 = (k.ent << 8) | k.tag_init;
  for (int c = 0; c < k.C; ++c) {
    const int o0 = sh.off[c], nc = sh.off[c + 1] - o0;
    const int nitems = 32 * A * ((nc + 31) / 32);
    for (int it = k.tid; it < nitems; it += kGThreads) {
      int j, a;
      item_of<A>(it, j, a);
      if (j >= nc) continue;
      uint32_t word = 0;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint4 x = philox((uint32_t)j, 0u, ((uint32_t)c << 16) | (uint32_t)(4 * a + g), c3, k.k0, k.k1);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (8 * g + i < k.T && half_lo(x, i) < 0x8000u) word |= 1u << (8 * g + i);
      }
      k.S[(o0 + j) * A + a] = word;
    }
  }
  __syncthreads();
}

// One sweep, colour class by colour class (Algorithm S2's p-computer loop):
// every (vertex, label) of the class in parallel.  Replica b = 32 a + r
// takes half b & 7 of P(j, s, (c << 16) | (b >> 3), (e << 8) | TAG), so one
// Philox call serves 8 replicas of the vertex.
template <int A, int NP, bool SM>
__device__ void g_sweep(const GCta &k, GShared &sh, uint32_t s) {
  const uint32_t c3m = (k.ent << 8) | k.tag_sweep;
  const uint32_t c3r = (k.ent << 8) | k.tag_refine;
  for (int c = 0; c < k.C; ++c) {
    const int o0 = sh.off[c], nc = sh.off[c + 1] - o0;
    const int nitems = 32 * A * ((nc + 31) / 32);
    for (int it = k.tid; it < nitems; it += kGThreads) {
      int j, a;
      item_of<A>(it, j, a);
      if (j >= nc) continue;
      const int p = o0 + j;
      const int2 vi = ld_vi<SM>(k.vinfo, p);
      uint32_t P[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) P[q] = 0u;
      const int W = vfield<A, NP, SM>(k.dynb, k.adj + vi.x, 0, vi_deg(vi), a, P);
      const int base = vi_h(vi) - W + k.Imax;   // I + Imax = 2 C + base
      const uint32_t c2 = ((uint32_t)c << 16) | (uint32_t)(4 * a);
      // the sign of (main half - threshold top half) decides; per group of 8
      // replicas a zero product of the differences (mod 2^32) flags a
      // possible tie, settled exactly below (8 differences rarely wrap the
      // product to 0; a wrap only costs a needless check)
      uint32_t word = 0u, gmask = 0u;
#pragma unroll
      for (int g = 3; g >= 0; --g) {
        const uint4 x = philox((uint32_t)j, s, c2 + (uint32_t)g, c3m, k.k0, k.k1);
        uint32_t tp = 1u;
        // the group's table columns 2 C + base = I + Imax (at most
        // 2 Imax <= 254) as bytes, 4 replicas per word
        uint32_t Jlo, Jhi;
        counts2_bytes<NP>(P, g, Jlo, Jhi);
        Jlo += 0x01010101u * (uint32_t)base;
        Jhi += 0x01010101u * (uint32_t)base;
#pragma unroll
        for (int i = 7; i >= 0; --i) {
          const int r = 8 * g + i;
          const int col = (int)__byte_perm(i < 4 ? Jlo : Jhi, 0u, 0x4440u + (uint32_t)(i & 3));
          const uint32_t th = k.Th[r * k.ths + col];
          const uint32_t d = half_lo(x, i) - (th >> 16);
          word = __funnelshift_l(d, word, 1);   // shift in the sign of d as bit 0
          tp *= d;
        }
        gmask |= (tp == 0u ? 1u : 0u) << g;
      }
      if (gmask) {
#pragma unroll 1
        for (int g = 0; g < 4; ++g) {
          if (!((gmask >> g) & 1u)) continue;
          const uint4 x = philox((uint32_t)j, s, c2 + (uint32_t)g, c3m, k.k0, k.k1);
          uint4 y = make_uint4(0u, 0u, 0u, 0u);
          bool have_y = false;
#pragma unroll 1
          for (int i = 0; i < 8; ++i) {
            const int r = 8 * g + i;
            int C = 0;
            for (int q = 0; q < NP; ++q) C |= (int)((P[q] >> r) & 1u) << q;
            const uint32_t th = k.Th[r * k.ths + 2 * C + base];
            const uint32_t v = half_lo(x, i);
            if (v != (th >> 16)) continue;
            if (!have_y) {
              y = philox((uint32_t)j, s, c2 + (uint32_t)g, c3r, k.k0, k.k1);
              have_y = true;
            }
            const uint32_t u = (v << 16) | half_lo(y, i);
            word = (u < th) ? (word | (1u << r)) : (word & ~(1u << r));
          }
        }
      }
      k.S[p * A + a] = word;
    }
    __syncthreads();
  }
}

// Warp transpose of a 32 x 32 bit matrix: lane r returns the word whose bit
// l is bit r of lane l's x (block-recursive swap of off-diagonal blocks).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int d = 16 >> st;
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, d);
    x = (lane & d) ? ((x & ~M[st]) | ((y >> d) & M[st])) : ((x & M[st]) | ((y << d) & ~M[st]));
  }
  return x;
}

// Energies of all replicas from the current state (Eq. ising_energy), each
// bond counted at its endpoint of higher colour.  For vertex v with
// lower-colour count Cl (weights |w|), their sum of |w| W_l, and y = its spin
// word (inverted when h < 0):
//   e_v = W_l + |h| - 2 U,   U = (s_v = +1 ? Cl : W_l - Cl) + |h| y.
// U is formed bit-sliced (U <= Imax < 2^NP); each warp (one label, 32
// vertices) transposes the planes and counts bits per replica.
// AL: only the first AL labels are counted (their rows of E are rewritten).
template <int A, int NP, bool SM, int AL = A>
__device__ void g_energy(const GCta &k, GShared &sh) {
  if (k.tid < 32 * AL) sh.E[k.tid >> 5][k.tid & 31] = 0;
  __syncthreads();
  int eacc = 0, a_w = 0;
  const int nitems = 32 * AL * ((k.n + 31) / 32);
  for (int it0 = 32 * k.warp; it0 < nitems; it0 += kGThreads) {
    int v, a;
    item_of<AL>(it0 + k.lane, v, a);
    a_w = a;
    uint32_t U[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) U[q] = 0u;
    int K = 0;
    if (v < k.n) {
      const int2 vi = ld_vi<SM>(k.vinfo, v);
      uint32_t Pl[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) Pl[q] = 0u;
      const int Wl = vfield<A, NP, SM>(k.dynb, k.adj + vi.x, 0, vi_kl(vi), a, Pl);
      const uint32_t x = k.S[v * A + a];
      uint32_t cy = 0xFFFFFFFFu;   // Wl - Cl = Wl + ~Cl + 1
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const uint32_t wb = ((Wl >> q) & 1) ? 0xFFFFFFFFu : 0u, nb = ~Pl[q];
        const uint32_t d = wb ^ nb ^ cy;
        cy = (wb & nb) | (wb & cy) | (nb & cy);
        U[q] = (x & Pl[q]) | (~x & d);
      }
      const int h = vi_h(vi), ha = h < 0 ? -h : h;
      if (ha) vadd<NP>(U, h < 0 ? ~x : x, (uint32_t)ha);
      K = Wl + ha;
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) cnt += __popc(transpose32(U[q], k.lane)) << q;
    eacc += (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)K) - 2 * cnt;
  }
  atomicAdd(&sh.E[a_w][k.lane], eacc);
  __syncthreads();
}

// Minimum-energy tracking: lowest slot r*A + a on ties, strict improvement;
// an improvement copies that replica's state into the best-state bits.
template <int A>
__device__ void g_best(const GCta &k, GShared &sh, long long sweeps) {
  if (k.warp == 0) {
    int bE = INT_MAX, bB = INT_MAX;
    if (k.lane < k.T)
      for (int aa = 0; aa < A; ++aa) {
        const int e = sh.E[aa][k.lane];
        if (e < bE) { bE = e; bB = k.lane * A + aa; }
      }
    for (int o = 16; o; o >>= 1) {
      const int oE = __shfl_xor_sync(0xFFFFFFFFu, bE, o), oB = __shfl_xor_sync(0xFFFFFFFFu, bB, o);
      if (oE < bE || (oE == bE && oB < bB)) { bE = oE; bB = oB; }
    }
    if (k.lane == 0) {
      sh.copy_slot = -1;
      if ((long long)bE < sh.bestE) {
        sh.bestE = bE;
        sh.bestSweep = sweeps;
        sh.bestSlot = bB;
        sh.copy_slot = bB;
      }
      if (sh.hit < 0 && sh.bestE <= sh.target) sh.hit = sweeps;
    }
  }
  __syncthreads();
  const int cs = sh.copy_slot;
  if (cs >= 0) {
    const int r = cs / A, aa = cs % A;
    for (int w = k.warp; 32 * w < k.n; w += kGWarps) {
      const int p = 32 * w + k.lane;
      const bool bit = p < k.n && ((k.S[p * A + aa] >> r) & 1u);
      const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
      if (k.lane == 0) k.best_bits[w] = word;
    }
  }
  __syncthreads();
}

// Replica exchange at attempt t: pairs (r, r+1) with r = t mod 2, t mod 2 + 2,
// ...; per label (or jointly over labels) accept with min(1, exp(dbeta dE))
// through the pair's table by |dE|.  Accepted pairs exchange their states
// (bit r and r+1 of every word of the label) and energies.
template <int A>
__device__ void g_swap(const GCta &k, GShared &sh, uint32_t t, int joint, const uint32_t *swaptab,
                       const uint32_t *swapidx) {
  if (k.tid < 4) sh.swmask[k.tid] = 0u;
  __syncthreads();
  const int r0 = (int)(t & 1u), npairs = (k.T - r0) / 2;
  const uint32_t c3 = (k.ent << 8) | TAG_G_SWAP;
  if (joint) {
    if (k.tid < npairs) {
      const int r = r0 + 2 * k.tid;
      long long dE = 0;
      for (int aa = 0; aa < A; ++aa) dE += (long long)sh.E[aa][r + 1] - sh.E[aa][r];
      const uint32_t x = philox((uint32_t)r, t, 0u, c3, k.k0, k.k1).x;
      bool acc = dE >= 0;
      if (!acc) {
        const long long d = -dE;
        acc = d < (long long)swapidx[2 * r + 1] && x < swaptab[swapidx[2 * r] + d];
      }
      for (int aa = 0; aa < A; ++aa) {
        sh.att[r * A + aa]++;
        if (acc) {
          sh.acc[r * A + aa]++;
          atomicOr(&sh.swmask[aa], 1u << r);
        }
      }
    }
  } else if (k.tid < npairs * A) {
    const int r = r0 + 2 * (k.tid / A), aa = k.tid % A;
    const long long dE = (long long)sh.E[aa][r + 1] - sh.E[aa][r];
    const uint32_t x = philox((uint32_t)r, t, (uint32_t)aa, c3, k.k0, k.k1).x;
    bool acc = dE >= 0;
    if (!acc) {
      const long long d = -dE;
      acc = d < (long long)swapidx[2 * r + 1] && x < swaptab[swapidx[2 * r] + d];
    }
    sh.att[r * A + aa]++;
    if (acc) {
      sh.acc[r * A + aa]++;
      atomicOr(&sh.swmask[aa], 1u << r);
    }
  }
  __syncthreads();
  for (int i = k.tid; i < k.n * A; i += kGThreads) {
    const uint32_t M = sh.swmask[i % A];
    if (M) {
      const uint32_t w = k.S[i], d = (w ^ (w >> 1)) & M;
      k.S[i] = w ^ d ^ (d << 1);
    }
  }
  if (k.warp < A) {
    const uint32_t M = sh.swmask[k.warp];
    const int e = sh.E[k.warp][k.lane];
    int src = k.lane;
    if ((M >> k.lane) & 1u) src = k.lane + 1;
    else if (k.lane > 0 && ((M >> (k.lane - 1)) & 1u)) src = k.lane - 1;
    const int o = __shfl_sync(0xFFFFFFFFu, e, src);
    sh.E[k.warp][k.lane] = o;
  }
  __syncthreads();
}

// ICMop of Algorithm S2 for every temperature at once (bit r of the words =
// temperature r).  Per pair set: the overlap mismatch X, its count per
// temperature, the seed = the k-th mismatch vertex in canonical order
// (k = floor(x0 n_minus / 2^32)), the seed's connected component in X by a
// bit-parallel flood fill over the graph, then either the cluster flips in
// both replicas or, when it holds more than half of the n spins, one whole
// replica (x1 bit 0) flips.
template <int A, bool SM>
__device__ void g_icm(const GCta &k, GShared &sh, uint32_t t) {
  const uint32_t c3 = (k.ent << 8) | TAG_G_ICM;
  if (k.tid < 32 * (A / 2)) {
    const int pp = k.tid >> 5, r = k.tid & 31;
    if (r < k.T) {
      const uint4 x = philox((uint32_t)r, t, (uint32_t)pp, c3, k.k0, k.k1);
      sh.x0[pp][r] = x.x;
      sh.x1[pp][r] = x.y;
      if (pp == 0) sh.mcode[r] = (uint32_t)(((unsigned long long)x.z * 3ull) >> 32);
    }
  }
  __syncthreads();
  // warp ranges of whole 32-vertex blocks (counts by transpose and popcount)
  const int per = 32 * ((k.n + 32 * kGWarps - 1) / (32 * kGWarps));
  const int lo = min(k.n, k.warp * per), hi = min(k.n, lo + per);
  for (int pp = 0; pp < A / 2; ++pp) {
    if (k.warp == 0) {
      // the 4-label matchings (0,1)(2,3), (0,2)(1,3), (0,3)(1,2)
      const bool valid = k.lane < k.T;
      int la = 0, lb = 1;
      if (A == 4) {
        const int m = valid ? (int)sh.mcode[k.lane] : 0;
        const int M[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
        la = M[m][2 * pp];
        lb = M[m][2 * pp + 1];
      }
      for (int kk = 0; kk < A; ++kk) {
        const uint32_t sa = __ballot_sync(0xFFFFFFFFu, valid && la == kk);
        const uint32_t sb = __ballot_sync(0xFFFFFFFFu, valid && lb == kk);
        if (k.lane == 0) {
          sh.sel[0][kk] = sa;
          sh.sel[1][kk] = sb;
        }
      }
    }
    __syncthreads();
    uint32_t selA[A], selB[A];
#pragma unroll
    for (int kk = 0; kk < A; ++kk) {
      selA[kk] = sh.sel[0][kk];
      selB[kk] = sh.sel[1][kk];
    }
    for (int p = k.tid; p < k.n; p += kGThreads) {
      uint32_t xa = 0, xb = 0;
#pragma unroll
      for (int kk = 0; kk < A; ++kk) {
        const uint32_t w = k.S[p * A + kk];
        xa |= w & selA[kk];
        xb |= w & selB[kk];
      }
      k.X[p] = xa ^ xb;
      k.Cl[p] = 0u;
    }
    __syncthreads();
    uint32_t cnt = 0;
    for (int p0 = lo; p0 < hi; p0 += 32) {
      const int p = p0 + k.lane;
      cnt += __popc(transpose32(p < hi ? k.X[p] : 0u, k.lane));
    }
    sh.wcnt[k.warp][k.lane] = cnt;
    __syncthreads();
    {
      uint32_t pre = 0, tot = 0;
      for (int w = 0; w < kGWarps; ++w) {
        const uint32_t c = sh.wcnt[w][k.lane];
        pre += w < k.warp ? c : 0u;
        tot += c;
      }
      if (k.warp == 0) sh.nm[k.lane] = tot;
      if (k.lane < k.T && tot > 0) {
        const uint32_t kk = (uint32_t)(((unsigned long long)sh.x0[pp][k.lane] * tot) >> 32);
        if (kk >= pre && kk < pre + cnt) {
          uint32_t seen = pre;
          for (int p = lo; p < hi; ++p)
            if ((k.X[p] >> k.lane) & 1u) {
              if (seen == kk) {
                atomicOr((uint32_t *)&k.Cl[p], 1u << k.lane);
                break;
              }
              ++seen;
            }
        }
      }
    }
    __syncthreads();
    // flood fill: grow every seed inside X until nothing changes; each
    // change adds a bit, so at most 32 n passes
    for (;;) {
      int changed = 0;
      for (int p = k.tid; p < k.n; p += kGThreads) {
        const uint32_t cl = k.Cl[p], cand = k.X[p] & ~cl;
        if (cand) {
          const int2 vi = ld_vi<SM>(k.vinfo, p);
          const uint32_t *ad = k.adj + vi.x;
          uint32_t nb = 0;
          for (int e = 0, d = vi_deg(vi); e < d; ++e)
            nb |= k.Cl[((ld_adj<SM>(ad, e) >> 8) - k.ubase) >> k.ushift];
          const uint32_t nw = cl | (cand & nb);
          if (nw != cl) {
            k.Cl[p] = nw;
            changed = 1;
          }
        }
      }
      if (!__syncthreads_or(changed)) break;
    }
    cnt = 0;
    for (int p0 = lo; p0 < hi; p0 += 32) {
      const int p = p0 + k.lane;
      cnt += __popc(transpose32(p < hi ? k.Cl[p] : 0u, k.lane));
    }
    sh.wcnt[k.warp][k.lane] = cnt;
    __syncthreads();
    if (k.warp == 0) {
      uint32_t size = 0;
      for (int w = 0; w < kGWarps; ++w) size += sh.wcnt[w][k.lane];
      const bool valid = k.lane < k.T, has = valid && sh.nm[k.lane] > 0;
      const bool big = has && 2ull * size > (unsigned long long)k.n;
      const bool second = (sh.x1[pp][k.lane] & 1u) != 0u;
      const uint32_t smallM = __ballot_sync(0xFFFFFFFFu, has && !big);
      const uint32_t wA = __ballot_sync(0xFFFFFFFFu, big && !second);
      const uint32_t wB = __ballot_sync(0xFFFFFFFFu, big && second);
      const uint32_t none = __ballot_sync(0xFFFFFFFFu, valid && !has);
      if (k.lane == 0) {
        sh.small = smallM;
        for (int kk = 0; kk < A; ++kk) sh.whole[kk] = (wA & sh.sel[0][kk]) | (wB & sh.sel[1][kk]);
        sh.icm[0] += __popc(none);
        sh.icm[1] += __popc(smallM);
        sh.icm[2] += __popc(wA | wB);
      }
    }
    __syncthreads();
    const uint32_t smallM = sh.small;
    for (int i = k.tid; i < k.n * A; i += kGThreads) {
      const int p = i / A, kk = i % A;
      k.S[i] ^= (k.Cl[p] & smallM & (selA[kk] | selB[kk])) | sh.whole[kk];
    }
    __syncthreads();
  }
}

// NP: bit planes of the field counts (2^NP > Imax).  SM: the problem's
// vertex table and adjacency are staged in shared memory (when they fit)
// instead of being read through the L1 cache.
template <int A, int NP, bool SM>
__global__ void __launch_bounds__(kGThreads, 1) gapt_kernel(GAptArgs a, int init) {
  extern __shared__ __align__(16) uint32_t dyn[];
  __shared__ GShared sh;
  if (a.active && !a.active[blockIdx.x]) return;   // converged ladder problem
  const GProbDev &P = a.prob[blockIdx.x];
  GCta k;
  k.n = P.n;
  k.C = P.C;
  k.T = P.T;
  k.Imax = P.Imax;
  k.tid = threadIdx.x;
  k.lane = threadIdx.x & 31;
  k.warp = threadIdx.x >> 5;
  k.ent = P.ent;
  k.k0 = a.k0;
  k.k1 = a.k1;
  k.tag_init = a.tag_init;
  k.tag_sweep = a.tag_sweep;
  k.tag_refine = a.tag_refine;
  k.ushift = A == 1 ? 2 : (A == 2 ? 3 : 4);
  k.dynb = reinterpret_cast<const char *>(dyn);
  uint32_t *Th = dyn;
  const int nth = (2 * P.Imax + 1) * 32;
  k.Th = Th;
  k.S = Th + nth;
  k.ths = 2 * P.Imax + 1;
  k.ubase = 4u * (uint32_t)nth;
  k.X = k.S + (size_t)P.n * A;
  k.Cl = k.X + P.n;
  if (SM) {
    // vertex table at an 8-byte boundary after the cluster words, then the adjacency
    const size_t vo = ((size_t)(nth + P.n * (A + 2)) + 1) & ~(size_t)1;
    int2 *vs = reinterpret_cast<int2 *>(dyn + vo);
    uint32_t *as = dyn + vo + 2 * (size_t)P.n;
    for (int i = k.tid; i < P.n; i += kGThreads) vs[i] = a.vinfo[P.vbase + i];
    for (int i = k.tid; i < P.m; i += kGThreads) as[i] = a.adj[P.abase + i];
    k.vinfo = vs;
    k.adj = as;
  } else {
    k.vinfo = a.vinfo + P.vbase;
    k.adj = a.adj + P.abase;
  }
  k.best_bits = a.best_bits + P.bestbase;
  uint32_t *gS = a.spins + (size_t)P.vbase * A;
  if (k.tid <= k.C) sh.off[k.tid] = P.off[k.tid];
  for (int i = k.tid; i < nth; i += kGThreads) Th[i] = a.pbit[P.thbase + i];
  const long long *gb = a.best + 4 * (size_t)blockIdx.x;
  if (init) {
    __syncthreads();
    g_init<A>(k, sh);
    g_energy<A, NP, SM>(k, sh);
  } else {
    for (int i = k.tid; i < P.n * A; i += kGThreads) k.S[i] = gS[i];
    if (k.tid < 128) {
      sh.E[k.tid >> 5][k.tid & 31] = a.E[128 * (size_t)blockIdx.x + k.tid];
      sh.att[k.tid] = 0u;
      sh.acc[k.tid] = 0u;
    }
    if (k.tid == 0) {
      sh.bestE = gb[0];
      sh.bestSweep = gb[1];
      sh.bestSlot = gb[2];
      sh.hit = gb[3];
      sh.target = a.target[blockIdx.x];
      sh.icm[0] = sh.icm[1] = sh.icm[2] = 0ull;
    }
    __syncthreads();
    const uint32_t *swidx = a.swapidx + P.swbase;
    for (int t = 0; t < a.n_swaps; ++t) {
      const uint32_t tt = a.swap0 + (uint32_t)t;
      for (int q = 0; q < a.spp; ++q) g_sweep<A, NP, SM>(k, sh, a.sweep0 + (uint32_t)(t * a.spp + q));
      g_energy<A, NP, SM>(k, sh);
      if (a.ladder) {
        // thread tid reads (and next zeroes) only its own slot's energy
        if (t >= a.window_from && k.tid < 32 * A) {
          const long long e = sh.E[k.tid >> 5][k.tid & 31];
          a.sum1[128 * (size_t)blockIdx.x + k.tid] += e;
          a.sum2[128 * (size_t)blockIdx.x + k.tid] += e * e;
        }
        continue;
      }
      const long long done = (long long)a.sweep0 + (long long)(t + 1) * a.spp;
      g_best<A>(k, sh, done);
      if (A >= 2 && a.icm) {
        g_icm<A, SM>(k, sh, tt);
        if (A == 2) {
          // a cluster move keeps each pair's E_0 + E_1 and a whole-replica
          // flip keeps both (h = 0): recount label 0, label 1 follows
          int keep = 0;
          if (k.tid < 32) keep = sh.E[0][k.tid] + sh.E[1][k.tid];
          g_energy<A, NP, SM, 1>(k, sh);
          if (k.tid < 32) sh.E[1][k.tid] = keep - sh.E[0][k.tid];
          __syncthreads();
        } else {
          g_energy<A, NP, SM>(k, sh);
        }
        g_best<A>(k, sh, done);
      }
      g_swap<A>(k, sh, tt, a.joint, a.swaptab, swidx);
    }
    unsigned long long *st = a.stats + P.statbase;
    const int np = (P.T > 1 ? P.T - 1 : 0) * A;
    for (int i = k.tid; i < np; i += kGThreads) {
      st[i] += sh.att[i];
      st[np + i] += sh.acc[i];
    }
    if (k.tid == 0) {
      st[2 * np] += sh.icm[0];
      st[2 * np + 1] += sh.icm[1];
      st[2 * np + 2] += sh.icm[2];
      long long *b = a.best + 4 * (size_t)blockIdx.x;
      b[0] = sh.bestE;
      b[1] = sh.bestSweep;
      b[2] = sh.bestSlot;
      b[3] = sh.hit;
    }
  }
  for (int i = k.tid; i < P.n * A; i += kGThreads) gS[i] = k.S[i];
  if (k.tid < 128) a.E[128 * (size_t)blockIdx.x + k.tid] = sh.E[k.tid >> 5][k.tid & 31];
}

template <int A, int NP, bool SM>
int gapt_launch_t(const GAptArgs &a, int n_prob, size_t smem, bool init, cudaStream_t st) {
  PC_CUDA_TRY(cudaFuncSetAttribute(gapt_kernel<A, NP, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  gapt_kernel<A, NP, SM><<<n_prob, kGThreads, smem, st>>>(a, init ? 1 : 0);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

// DT-SQA on the replicated network of a graph (Eq. S.3, Algorithm S1),
// multi-spin coded: a CTA anneals 32 runs, whose spins of one (slice,
// vertex) share a word, and a thread owns one entry (slice k, vertex p) of
// the colour class being swept.  The in-slice field is summed bit-sliced
// over the neighbour words (NP planes); the two time neighbours' words give
// each run's count of +1 neighbours in imaginary time.  Run q takes half
// q & 7 of P(j, s, c, ((q >> 3) << 8) | TAG) (j: class-local index), so one
// Philox call serves 8 runs.  The sweep's [3][2 Imax + 1] table is staged in
// shared memory, one copy per lane when it is small (REP), so that threads
// with different fields do not collide on a bank.  All P n words stay in
// shared memory for the whole anneal.
//
// CL: the slices of a run group are split over a thread-block cluster of
// a.CS CTAs (rank r holds slices [r P / CS, (r+1) P / CS)), for anneals whose
// P n words do not fit one CTA.  Only the time neighbours of a range's end
// slices live in a neighbouring CTA; they are read through distributed
// shared memory, and every colour phase ends with a cluster barrier.
// SMG: the vertex table and adjacency are staged in shared memory (else
// they are read through the L1 cache).
template <int NP, bool REP, bool CL, bool SMG>
__global__ void __launch_bounds__(kGThreads, 1) gsqa_kernel(GSqaArgs a) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) uint32_t dyn[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = 2 * a.Imax + 1, ntab = 3 * nt, TB = REP ? 32 * ntab : ntab;
  const int n = a.n, P = a.P;
  const int CS = CL ? a.CS : 1, rank = CL ? (int)cg::this_cluster().block_rank() : 0;
  const int grp = (int)blockIdx.x / CS;                       // run group (32 runs)
  const int kb = rank * P / CS, ke = (rank + 1) * P / CS;     // own slices [kb, ke)
  const int nkmax = (P + CS - 1) / CS;                        // equal carve in every CTA
  uint32_t *tab = dyn;                       // [2][TB]
  uint32_t *W = dyn + 2 * TB;                // [nkmax][n]: slice k at (k - kb) n
  const size_t vo = (2 * (size_t)TB + (size_t)nkmax * n + 1) & ~(size_t)1;
  const int2 *vinfo = a.vinfo;
  const uint32_t *adj = a.adj;
  if (SMG) {   // staged vertex table and adjacency
    int2 *vs = reinterpret_cast<int2 *>(dyn + vo);
    uint32_t *as = dyn + vo + 2 * (size_t)n;
    for (int i = tid; i < n; i += kGThreads) vs[i] = a.vinfo[i];
    for (int i = tid; i < a.m; i += kGThreads) as[i] = a.adj[i];
    vinfo = vs;
    adj = as;
  }
  // the end slices' outer time neighbours: the last slice of rank - 1 and
  // the first slice of rank + 1 (this CTA itself without a cluster)
  const int rl = (rank + CS - 1) % CS, rr = (rank + 1) % CS;
  const uint32_t *Wl = W + (size_t)((rl + 1) * P / CS - rl * P / CS - 1) * n;
  const uint32_t *Wr = W;
  if (CL) {
    Wl = cg::this_cluster().map_shared_rank(W, rl) + (size_t)((rl + 1) * P / CS - rl * P / CS - 1) * n;
    Wr = cg::this_cluster().map_shared_rank(W, rr);
  }
  const uint32_t g0 = (a.run0 >> 3) + 4u * (uint32_t)grp;   // run group of bit 0 (run0 % 8 == 0)
  // this CTA's part of colour class c: entries [o0 + lo, o0 + hi) of the class list
  auto part = [&](int c, int &o0, int &lo, int &hi) {
    o0 = a.cls_off[c];
    lo = CL ? a.cls_rank[c * (CS + 1) + rank] : 0;
    hi = CL ? a.cls_rank[c * (CS + 1) + rank + 1] : a.cls_off[c + 1] - o0;
  };
  // Algorithm S1: random initial states of all slices
  for (int c = 0; c < a.Cp; ++c) {
    int o0, lo, hi;
    part(c, o0, lo, hi);
    for (int j = lo + tid; j < hi; j += kGThreads) {
      const uint32_t e = __ldg(a.cls + o0 + j);
      uint32_t word = 0u;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint4 x = philox((uint32_t)j, 0u, (uint32_t)c, ((g0 + g) << 8) | TAG_GS_INIT, a.k0, a.k1);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (half_lo(x, i) < 0x8000u) word |= 1u << (8 * g + i);
      }
      W[(size_t)((int)(e >> 20) - kb) * n + (e & 0xFFFFFu)] = word;
    }
  }
  if (CL) cg::this_cluster().sync();
  else __syncthreads();
  for (int s = 0; s < a.S; ++s) {
    uint32_t *T = tab + (s & 1) * TB;
    const uint32_t *gt = a.table + (size_t)s * ntab;
    for (int i = tid; i < TB; i += kGThreads) T[i] = __ldg(gt + (REP ? (i >> 5) : i));
    __syncthreads();
    for (int c = 0; c < a.Cp; ++c) {
      int o0, lo, hi;
      part(c, o0, lo, hi);
      for (int j = lo + tid; j < hi; j += kGThreads) {
        const uint32_t e = __ldg(a.cls + o0 + j);
        const int k = (int)(e >> 20), p = (int)(e & 0xFFFFFu);
        const uint32_t *Wk = W + (size_t)(k - kb) * n;
        const int2 vi = ld_vi<SMG>(vinfo, p);
        uint32_t Pl[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) Pl[q] = 0u;
        const int Ws = vfield<1, NP, SMG>(reinterpret_cast<const char *>(Wk), adj + vi.x, 0, vi_deg(vi), 0, Pl);
        const int base = vi_h(vi) - Ws + a.Imax;   // in-slice I + Imax = 2 C + base
        const uint32_t wd = k > kb ? Wk[p - n] : Wl[p];
        const uint32_t wu = k + 1 < ke ? Wk[p + n] : Wr[p];
        // decisions and the exact settlement of possible ties as in g_sweep
        uint32_t word = 0u, gmask = 0u;
#pragma unroll
        for (int g = 3; g >= 0; --g) {
          const uint4 x = philox((uint32_t)j, (uint32_t)s, (uint32_t)c, ((g0 + g) << 8) | TAG_GS_SWEEP, a.k0, a.k1);
          uint32_t tp = 1u;
          // three planes (Imax <= 7): the group's table indices
          // m nt + 2 C + base (below 2 nt + 2 Imax + 1 <= 59) as bytes,
          // 4 runs per word, m the time-neighbour count
          uint32_t Jlo = 0u, Jhi = 0u;
          if constexpr (NP == 3) {
            uint32_t dl, dh, ul, uh;
            counts2_bytes<NP>(Pl, g, Jlo, Jhi);
            spread_byte(wd, g, dl, dh);
            spread_byte(wu, g, ul, uh);
            Jlo += (dl + ul) * (uint32_t)nt + 0x01010101u * (uint32_t)base;
            Jhi += (dh + uh) * (uint32_t)nt + 0x01010101u * (uint32_t)base;
          }
#pragma unroll
          for (int i = 7; i >= 0; --i) {
            const int r = 8 * g + i;
            int idx;
            if constexpr (NP == 3) idx = (int)__byte_perm(i < 4 ? Jlo : Jhi, 0u, 0x4440u + (uint32_t)(i & 3));
            else idx = (int)(((wd >> r) & 1u) + ((wu >> r) & 1u)) * nt + 2 * vget<NP>(Pl, r) + base;
            const uint32_t th = REP ? T[32 * idx + lane] : T[idx];
            const uint32_t d = half_lo(x, i) - (th >> 16);
            word = __funnelshift_l(d, word, 1);   // shift in the sign of d as bit 0
            tp *= d;
          }
          gmask |= (tp == 0u ? 1u : 0u) << g;
        }
        if (gmask) {
#pragma unroll 1
          for (int g = 0; g < 4; ++g) {
            if (!((gmask >> g) & 1u)) continue;
            const uint32_t gq = (g0 + (uint32_t)g) << 8;
            const uint4 x = philox((uint32_t)j, (uint32_t)s, (uint32_t)c, gq | TAG_GS_SWEEP, a.k0, a.k1);
            uint4 y = make_uint4(0u, 0u, 0u, 0u);
            bool have_y = false;
#pragma unroll 1
            for (int i = 0; i < 8; ++i) {
              const int r = 8 * g + i;
              int C = 0;
              for (int q = 0; q < NP; ++q) C |= (int)((Pl[q] >> r) & 1u) << q;
              const int idx = (int)(((wd >> r) & 1u) + ((wu >> r) & 1u)) * nt + 2 * C + base;
              const uint32_t th = REP ? T[32 * idx + lane] : T[idx];
              const uint32_t v = half_lo(x, i);
              if (v != (th >> 16)) continue;
              if (!have_y) {
                y = philox((uint32_t)j, (uint32_t)s, (uint32_t)c, gq | TAG_GS_REFINE, a.k0, a.k1);
                have_y = true;
              }
              const uint32_t u = (v << 16) | half_lo(y, i);
              word = (u < th) ? (word | (1u << r)) : (word & ~(1u << r));
            }
          }
        }
        W[(size_t)(k - kb) * n + p] = word;
      }
      if (CL) cg::this_cluster().sync();
      else __syncthreads();
    }
  }
  // Algorithm S1: classical energy of every slice (bonds at their endpoint
  // of higher base colour, biases included), bit-sliced as in the APT
  // energy pass: e_v = W_l + |h| - 2 U per run, U counted per run by warp
  // transposes over blocks of 32 vertices
  const int runs_here = min(32, a.R - 32 * grp);
  const int nb32 = (n + 31) / 32;
  for (int it0 = 32 * warp; it0 < 32 * (ke - kb) * nb32; it0 += kGThreads) {
    const int blk = it0 >> 5, k = kb + blk / nb32, v = 32 * (blk % nb32) + lane;
    const uint32_t *Wk = W + (size_t)(k - kb) * n;
    uint32_t U[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) U[q] = 0u;
    int K = 0;
    if (v < n) {
      const int2 vi = ld_vi<SMG>(vinfo, v);
      uint32_t Pl[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) Pl[q] = 0u;
      const int Wl = vfield<1, NP, SMG>(reinterpret_cast<const char *>(Wk), adj + vi.x, 0, vi_kl(vi), 0, Pl);
      const uint32_t x = Wk[v];
      uint32_t cy = 0xFFFFFFFFu;   // Wl - Cl = Wl + ~Cl + 1
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const uint32_t wb = ((Wl >> q) & 1) ? 0xFFFFFFFFu : 0u, nb = ~Pl[q];
        const uint32_t d = wb ^ nb ^ cy;
        cy = (wb & nb) | (wb & cy) | (nb & cy);
        U[q] = (x & Pl[q]) | (~x & d);
      }
      const int h = vi_h(vi), ha = h < 0 ? -h : h;
      if (ha) vadd<NP>(U, h < 0 ? ~x : x, (uint32_t)ha);
      K = Wl + ha;
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) cnt += __popc(transpose32(U[q], lane)) << q;
    const long long ek = (long long)__reduce_add_sync(0xFFFFFFFFu, (unsigned)K) - 2LL * cnt;
    if (lane < runs_here)
      atomicAdd(reinterpret_cast<unsigned long long *>(&a.E[(size_t)(32 * grp + lane) * P + k]),
                (unsigned long long)ek);
  }
  if (a.spins)
    for (int i = tid; i < (ke - kb) * n; i += kGThreads) a.spins[((size_t)grp * P + kb) * n + i] = W[i];
}

}  // namespace

size_t gsqa_smem_bytes(int n, int P, int Imax, int m, int CS) {
  const size_t ntab = (size_t)3 * (2 * Imax + 1), TB = Imax <= 7 ? 32 * ntab : ntab;
  const size_t base = 2 * TB + (size_t)((P + CS - 1) / CS) * n;
  if (m < 0) return sizeof(uint32_t) * base;
  return sizeof(uint32_t) * (((base + 1) & ~(size_t)1) + 2 * (size_t)n + (size_t)m);
}

template <int NP, bool REP, bool CL, bool SMG>
int gsqa_launch_t(const GSqaArgs &a, size_t smem, cudaStream_t st) {
  auto kern = gsqa_kernel<NP, REP, CL, SMG>;
  PC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)(((a.R + 31) / 32) * (CL ? a.CS : 1));
  if (!CL) {
    kern<<<grid, kGThreads, smem, st>>>(a);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3((unsigned)kGThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  }
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

int gsqa_launch(const GSqaArgs &a, bool staged, size_t smem, cudaStream_t st) {
  const int sel = (a.Imax <= 7 ? 4 : 0) + (a.CS > 1 ? 2 : 0) + (staged ? 1 : 0);
  switch (sel) {
    case 0: return gsqa_launch_t<7, false, false, false>(a, smem, st);
    case 1: return gsqa_launch_t<7, false, false, true>(a, smem, st);
    case 2: return gsqa_launch_t<7, false, true, false>(a, smem, st);
    case 3: return gsqa_launch_t<7, false, true, true>(a, smem, st);
    case 4: return gsqa_launch_t<3, true, false, false>(a, smem, st);
    case 5: return gsqa_launch_t<3, true, false, true>(a, smem, st);
    case 6: return gsqa_launch_t<3, true, true, false>(a, smem, st);
    default: return gsqa_launch_t<3, true, true, true>(a, smem, st);
  }
}

size_t gapt_smem_bytes(int n, int A, int Imax, int m) {
  const size_t base = (size_t)(2 * Imax + 1) * 32 + (size_t)n * (A + 2);
  if (m < 0) return sizeof(uint32_t) * base;
  return sizeof(uint32_t) * (((base + 1) & ~(size_t)1) + 2 * (size_t)n + (size_t)m);
}

int gapt_launch(const GAptArgs &a, int n_prob, int A, int Imax, bool staged, size_t smem, bool init,
                cudaStream_t st) {
  const bool small = Imax <= 7;   // 3 planes hold every field count
  switch (A * 4 + (small ? 0 : 2) + (staged ? 1 : 0)) {
    case 4: return gapt_launch_t<1, 3, false>(a, n_prob, smem, init, st);
    case 5: return gapt_launch_t<1, 3, true>(a, n_prob, smem, init, st);
    case 6: return gapt_launch_t<1, 7, false>(a, n_prob, smem, init, st);
    case 7: return gapt_launch_t<1, 7, true>(a, n_prob, smem, init, st);
    case 8: return gapt_launch_t<2, 3, false>(a, n_prob, smem, init, st);
    case 9: return gapt_launch_t<2, 3, true>(a, n_prob, smem, init, st);
    case 10: return gapt_launch_t<2, 7, false>(a, n_prob, smem, init, st);
    case 11: return gapt_launch_t<2, 7, true>(a, n_prob, smem, init, st);
    case 16: return gapt_launch_t<4, 3, false>(a, n_prob, smem, init, st);
    case 17: return gapt_launch_t<4, 3, true>(a, n_prob, smem, init, st);
    case 18: return gapt_launch_t<4, 7, false>(a, n_prob, smem, init, st);
    case 19: return gapt_launch_t<4, 7, true>(a, n_prob, smem, init, st);
    default: return fail(PC_EINVAL, "n_labels must be 1, 2 or 4");
  }
}

}  // namespace pc
