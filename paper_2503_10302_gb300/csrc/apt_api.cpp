// C ABI of adaptive parallel tempering (Algorithm S2), the adaptive beta
// ladder (its preprocessing) and the pilot-run histograms.  Host side:
// validation, tables, batch packing, CTA scheduling and CUDA graphs; the
// work itself runs in apt.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "apt_dev.h"
#include "ctx.h"
#include "internal.h"

namespace pc {

namespace {

constexpr int kTpbDefault = 512; // threads per CTA of the sweep kernel (autotunable)
constexpr int kMaxGcCta = 8;     // groups (64 buffers) per CTA
constexpr int kChunkAttempts = 128;

// Batch of problems resident on the device (one per APT problem, or one per
// ladder/pilot instance).
struct Batch {
  std::vector<AptProbDev> prob;
  std::vector<int> G;            // groups per problem
  // device arrays
  DevBuf<AptProbDev> d_prob;
  DevBuf<uint32_t> d_spins, d_pbit, d_swaptab, d_swapidx;
  DevBuf<uint16_t> d_jneg;
  DevBuf<int32_t> d_temp, d_buf, d_E, d_bestbuf;
  DevBuf<int64_t> d_bestE, d_bestsweep, d_hit, d_target, d_stats, d_sum1, d_sum2, d_hist, d_ctr;
  DevBuf<int8_t> d_bestspins, d_bestspins2;   // best states; rank-1 candidates of split problems
  // CTA tables: the one-CTA part [4][n_u] (prob, g0, gc, nch), then the
  // two-CTA-cluster part [4][n_s]
  DevBuf<int> d_cta;
  int n_cta = 0;         // n_u + n_s
  int n_u = 0, n_s = 0;
  int tpb = kTpbDefault;
  int split = 0;         // every APT problem runs as a cluster of two CTAs (by temperature)
  int hybrid = 0;        // some problems run as clusters, the others as one CTA (two launches)
  int split_pref = 0;    // 0: when needed or when the batch fills at most half the SMs; 1: only when needed;
                         // 2: whenever possible; 3: the problems needing it or above the mean work per SM
  int nch_pref = 0;      // thread chunks per CTA: 0 = the cost model's choice, else this count where it fits
  int split_h = 0;       // split problems: temperature groups per label on rank 0 (0: half)
  size_t smem = 0;       // max of the two parts
  size_t smem_u = 0, smem_s = 0;
  int stage_swt = 1;     // the split part stages swap tables (when its CTAs still fit)
  std::vector<uint32_t> h_pbit, h_swaptab, h_swapidx;
};

// Split of a CTA's threads into nch chunks of tpb/nch threads, each chunk
// sweeping ceil(Gc/nch) groups of every site: `pref` where it fits (tpb a
// multiple of 32 nch, nch <= Gc, at most 4 groups per thread), else the
// choice that minimises the longest thread's work (site rounds x groups).
int choose_nch(int H, int Gc, int tpb, int pref) {
  if (pref > 0 && tpb % (32 * pref) == 0 && pref <= Gc && (Gc + pref - 1) / pref <= 4) return pref;
  int best = 1, best_cost = INT_MAX;
  for (int nch = 1; nch <= 8; nch *= 2) {
    if (tpb % (32 * nch)) continue;
    const int gc = (Gc + nch - 1) / nch;
    if (gc > 4) continue;
    const int tpc = tpb / nch;
    const int cost = ((H + tpc - 1) / tpc) * gc;
    if (cost < best_cost) {
      best_cost = cost;
      best = nch;
    }
  }
  return best;
}

// pack_jn16's words in (colour, j) order: coupling signs (bits 0-5), absent
// bonds (bits 8-13) and the vacancy flag (bit 15) of site (c, j).
std::vector<uint16_t> pack_jn_cj(const Lattice &lat, const uint8_t per[3], const uint8_t *present,
                                 const int8_t *J, int *nbonds, int *nreal) {
  std::vector<uint16_t> bylin = pack_jn16(lat, per, present, J, nbonds, nreal);
  const int Lx = lat.L[0], Ly = lat.L[1], H = lat.N / 2;
  std::vector<uint16_t> out((size_t)lat.N);
  for (int s = 0; s < lat.N; ++s) {
    const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
    out[(size_t)((x + y + z) & 1) * H + (s >> 1)] = bylin[(size_t)s];
  }
  return out;
}

// Host mirror of the spins of one problem, [B][N] in lin order.
void unpack_spins(const AptProbDev &P, const uint32_t *words, int B, int8_t *out) {
  const int N = P.N, H = N / 2, Lx = P.Lx, Ly = P.Ly;
  for (int s = 0; s < N; ++s) {
    const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
    const int c = (x + y + z) & 1, j = s >> 1;
    for (int b = 0; b < B; ++b) {
      const uint32_t w = words[((size_t)(b >> 3) * 2 + c) * H + j];
      out[(size_t)b * N + s] = ((w >> (4 * (b & 7))) & 1u) ? 1 : -1;
    }
  }
}

struct ProbSpec {
  Lattice lat;
  uint8_t per[3] = {1, 1, 1};     // periodic axes
  const uint8_t *present = nullptr;   // [N] 0 = vacancy, or none
  const int8_t *J;
  int T, Tp, A, B;
  uint32_t ent;
  std::vector<double> beta;       // [T] (ladder: 1 entry, pilot: n_beta)
  std::vector<int32_t> temp_of;   // [B]
  bool swaps;
};

// Allocates and fills the device arrays of a batch.
int build_batch(pc_ctx *c, Batch &bt, const std::vector<ProbSpec> &specs, int n_bins) {
  const int n = (int)specs.size();
  bt.prob.assign((size_t)n, AptProbDev{});
  bt.G.assign((size_t)n, 0);
  size_t spin_w = 0, jneg_b = 0, pbit_w = 0, swapidx_w = 0, buf_n = 0, best_b = 0, stat_n = 0,
         hist_n = 0;
  std::vector<uint16_t> h_jneg;
  bt.h_pbit.clear();
  bt.h_swaptab.clear();
  bt.h_swapidx.clear();
  std::vector<int32_t> h_temp, h_buf;
  for (int i = 0; i < n; ++i) {
    const ProbSpec &s = specs[(size_t)i];
    AptProbDev &P = bt.prob[(size_t)i];
    const int G = (s.B + 7) / 8;
    bt.G[(size_t)i] = G;
    P.Lx = s.lat.L[0];
    P.Ly = s.lat.L[1];
    P.Lz = s.lat.L[2];
    P.N = s.lat.N;
    P.mhx = recip32((uint32_t)(P.Lx / 2));
    P.mLy = recip32((uint32_t)P.Ly);
    P.mLy2 = recip32((uint32_t)(P.Ly / 2));
    P.T = s.T;
    P.Tp = s.Tp;
    P.A = s.A;
    P.B = s.B;
    P.ent = s.ent;
    P.spin_off = (uint32_t)spin_w;
    spin_w += (size_t)G * P.N;
    P.jneg_off = (uint32_t)jneg_b;
    std::vector<uint16_t> jn = pack_jn_cj(s.lat, s.per, s.present, s.J, &P.nbonds, &P.nreal);
    // bits 0-2: open axes; bit 3: some other absent bond (a vacancy).  Any
    // bit selects the sweep path that handles absent bonds.
    P.open = (s.per[0] ? 0u : 1u) | (s.per[1] ? 0u : 2u) | (s.per[2] ? 0u : 4u) |
             (P.nreal < P.N ? 8u : 0u);
    h_jneg.insert(h_jneg.end(), jn.begin(), jn.end());
    jneg_b += (size_t)P.N;
    P.pbit_off = (uint32_t)pbit_w;
    for (int t = 0; t < s.T; ++t) {
      // entry I + 6 for every local field I = -6..6 (odd I at open boundaries)
      for (int e = 0; e < 13; ++e) bt.h_pbit.push_back(pc_pbit_threshold(s.beta[(size_t)t], e - 6));
      for (int e = 13; e < 16; ++e) bt.h_pbit.push_back(0u);
    }
    pbit_w += (size_t)16 * s.T;
    P.swapidx_off = (uint32_t)swapidx_w;
    for (int r = 0; r + 1 < s.T; ++r) {
      const uint32_t off = (uint32_t)bt.h_swaptab.size();
      const double db = s.beta[(size_t)r + 1] - s.beta[(size_t)r];
      bt.h_swaptab.push_back(0xFFFFFFFFu);   // dE = 0: always accepted
      if (s.swaps) {
        // |dE| <= 6N per label; the joint rule sums the A labels
        for (int64_t k = 1; k <= 3 * (int64_t)P.N * s.A; ++k) {
          const uint32_t th = pc_swap_threshold(db, -2 * k);
          if (th == 0u) break;
          bt.h_swaptab.push_back(th);
        }
      }
      bt.h_swapidx.push_back(off);
      bt.h_swapidx.push_back((uint32_t)bt.h_swaptab.size() - off);
    }
    swapidx_w += (size_t)2 * (s.T > 1 ? s.T - 1 : 0);
    P.buf_off = (uint32_t)buf_n;
    for (int b = 0; b < 8 * G; ++b) {
      h_temp.push_back(b < s.B ? s.temp_of[(size_t)b] : 0);
      h_buf.push_back(b);
    }
    buf_n += (size_t)8 * G;
    P.best_off = (uint32_t)best_b;
    best_b += (size_t)P.N;
    P.stat_off = (uint32_t)stat_n;
    stat_n += (size_t)2 * (s.T > 1 ? s.T - 1 : 0) * s.A + 3;
    P.hist_off = (uint32_t)hist_n;
    hist_n += (size_t)s.T * (n_bins > 0 ? n_bins : 0);
  }
  if (bt.h_swaptab.empty()) bt.h_swaptab.push_back(0u);
  if (bt.h_swapidx.empty()) bt.h_swapidx.push_back(0u);
  if (spin_w > 0xFFFFFFFFull || bt.h_swaptab.size() > 0xFFFFFFFFull)
    return fail(PC_EINVAL, "batch too large");
  int rc;
  if ((rc = bt.d_prob.alloc((size_t)n)) || (rc = bt.d_spins.alloc(spin_w)) ||
      (rc = bt.d_jneg.alloc(jneg_b)) || (rc = bt.d_pbit.alloc(bt.h_pbit.size())) ||
      (rc = bt.d_swaptab.alloc(bt.h_swaptab.size())) || (rc = bt.d_swapidx.alloc(bt.h_swapidx.size())) ||
      (rc = bt.d_temp.alloc(buf_n)) || (rc = bt.d_buf.alloc(buf_n)) || (rc = bt.d_E.alloc(buf_n)) ||
      (rc = bt.d_sum1.alloc(buf_n)) || (rc = bt.d_sum2.alloc(buf_n)) ||
      (rc = bt.d_bestE.alloc((size_t)n)) || (rc = bt.d_bestsweep.alloc((size_t)n)) ||
      (rc = bt.d_hit.alloc((size_t)n)) || (rc = bt.d_target.alloc((size_t)n)) ||
      (rc = bt.d_bestbuf.alloc((size_t)n)) || (rc = bt.d_bestspins.alloc(best_b)) ||
      (rc = bt.d_bestspins2.alloc(best_b)) ||
      (rc = bt.d_stats.alloc(stat_n)) || (rc = bt.d_hist.alloc(hist_n)) || (rc = bt.d_ctr.alloc(2)))
    return rc;
  cudaStream_t st = c->stream;
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_prob.p, bt.prob.data(), sizeof(AptProbDev) * n, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_jneg.p, h_jneg.data(), h_jneg.size() * 2, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_pbit.p, bt.h_pbit.data(), bt.h_pbit.size() * 4, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_swaptab.p, bt.h_swaptab.data(), bt.h_swaptab.size() * 4,
                              cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_swapidx.p, bt.h_swapidx.data(), bt.h_swapidx.size() * 4,
                              cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_temp.p, h_temp.data(), h_temp.size() * 4, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_buf.p, h_buf.data(), h_buf.size() * 4, cudaMemcpyHostToDevice, st));
  std::vector<int64_t> big((size_t)n, INT64_MAX), neg((size_t)n, -1), low((size_t)n, INT64_MIN);
  std::vector<int32_t> negi((size_t)n, -1);
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_bestE.p, big.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_bestsweep.p, neg.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_hit.p, neg.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_target.p, low.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_bestbuf.p, negi.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st));
  if ((rc = bt.d_stats.zero(st)) || (rc = bt.d_hist.zero(st)) || (rc = bt.d_ctr.zero(st)) ||
      (rc = bt.d_E.zero(st)) || (rc = bt.d_sum1.zero(st)) || (rc = bt.d_sum2.zero(st)) ||
      (rc = bt.d_bestspins.zero(st)))
    return rc;
  // host vectors must outlive the async copies
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

AptArgs base_args(pc_ctx *c, Batch &bt) {
  AptArgs a;
  std::memset(&a, 0, sizeof(a));
  a.prob = bt.d_prob.p;
  a.cta_prob = bt.d_cta.p;
  a.cta_g0 = bt.d_cta.p + bt.n_cta;
  a.cta_gc = bt.d_cta.p + 2 * bt.n_cta;
  a.cta_nch = bt.d_cta.p + 3 * bt.n_cta;
  a.spins = bt.d_spins.p;
  a.jneg = bt.d_jneg.p;
  a.pbit = bt.d_pbit.p;
  a.swaptab = bt.d_swaptab.p;
  a.swapidx = bt.d_swapidx.p;
  a.split = bt.split;
  a.temp_of = bt.d_temp.p;
  a.buf_of = bt.d_buf.p;
  a.E = bt.d_E.p;
  a.best_E = bt.d_bestE.p;
  a.best_sweep = bt.d_bestsweep.p;
  a.hit_sweep = bt.d_hit.p;
  a.target = bt.d_target.p;
  a.best_buf = bt.d_bestbuf.p;
  a.best_spins = bt.d_bestspins.p;
  a.best_spins2 = bt.d_bestspins2.p;
  a.stats = bt.d_stats.p;
  a.sum1 = bt.d_sum1.p;
  a.sum2 = bt.d_sum2.p;
  a.hist = bt.d_hist.p;
  a.ctr = bt.d_ctr.p;
  a.k0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
  a.k1 = (uint32_t)(c->seed >> 32);
  a.spp = 1;
  a.icm_big = 1;
  a.icm_seed = 0;
  a.stage_swt = bt.stage_swt;
  return a;
}

// CTA list: problems in decreasing order of work (largest first, so the
// block scheduler packs the small ones behind), each split into CTAs of at
// most kMaxGcCta groups; only problems with active[i] set.
int schedule(pc_ctx *c, Batch &bt, const std::vector<char> &active, int mode, int icm, int n_bins) {
  const int n = (int)bt.prob.size();
  std::vector<int> order;
  for (int i = 0; i < n; ++i)
    if (active.empty() || active[(size_t)i]) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (int64_t)bt.prob[(size_t)x].N * bt.prob[(size_t)x].B > (int64_t)bt.prob[(size_t)y].N * bt.prob[(size_t)y].B;
  });
  // APT keeps a problem in one CTA (swaps and ICM couple all its groups), or
  // in a cluster of two CTAs that split its temperatures: needed above 64
  // replicas, and chosen for speed when the batch fills at most half the SMs
  // (pref 0), always (pref 2), or for the problems whose work alone exceeds
  // the batch's mean work per SM (pref 3: the rest run as one CTA each, in a
  // second, concurrent launch).  Ladder and pilot chains are independent, so
  // their groups spread over about one CTA per SM when the batch is small.
  bt.split = 0;
  bt.hybrid = 0;
  std::vector<char> ps((size_t)n, 0);
  if (mode == APT_MODE_APT && !order.empty()) {
    bool need = false, can = true;
    int64_t total = 0;
    for (int i : order) {
      const AptProbDev &P = bt.prob[(size_t)i];
      need = need || P.B > 64;
      can = can && (P.Tp >> 3) >= 2;
      total += (int64_t)P.N * P.B;
    }
    if (bt.split_pref == 3) {
      const int64_t per_sm = total / std::max(1, c->sms);
      for (int i : order) {
        const AptProbDev &P = bt.prob[(size_t)i];
        const bool need_i = P.B > 64, can_i = (P.Tp >> 3) >= 2;
        if (need_i && !can_i)
          return fail(PC_EINVAL, "a problem with more than 64 replicas needs >= 9 temperatures");
        ps[(size_t)i] = need_i || (can_i && (int64_t)P.N * P.B > per_sm);
      }
    } else {
      if (need && !can)
        return fail(PC_EINVAL, "a batch with more than 64 replicas in a problem needs >= 9 temperatures everywhere");
      const bool small = 2 * (int64_t)order.size() <= c->sms;
      const bool all = need || (can && (bt.split_pref == 2 || (bt.split_pref == 0 && small)));
      for (int i : order) ps[(size_t)i] = all;
    }
  }
  int gmax = kMaxGcCta;
  if (mode == APT_MODE_LADDER || mode == APT_MODE_PILOT) {
    int64_t total = 0;
    for (int i : order) total += bt.G[(size_t)i];
    const int sms = c->sms > 0 ? c->sms : 1;
    gmax = (int)std::min<int64_t>(kMaxGcCta, std::max<int64_t>(1, (total + sms - 1) / sms));
  }
  // [0]: one-CTA part, [1]: two-CTA-cluster part
  std::vector<int> cp[2], cg0[2], cgc[2], cnch[2];
  size_t smem[2] = {0, 0}, smem_ns = 0;   // smem_ns: the split part without staged swap tables
  for (int i : order) {
    const AptProbDev &P = bt.prob[(size_t)i];
    const int G = bt.G[(size_t)i];
    if (ps[(size_t)i]) {
      // rank 0: temperature groups [0, h1) of every label, rank 1: [h1, Glp)
      const int Glp = P.Tp >> 3;
      int h1 = bt.split_h > 0 ? std::min(bt.split_h, Glp - 1) : (Glp + 1) / 2;
      // each CTA holds at most kMaxGcCta groups (64 replicas, and 32 ICM
      // pair bits): an uneven split that breaks this falls back to the even one
      if (P.A * h1 > kMaxGcCta || P.A * (Glp - h1) > kMaxGcCta) h1 = (Glp + 1) / 2;
      for (int rank = 0; rank < 2; ++rank) {
        const int g0 = rank ? h1 : 0, gu = rank ? Glp - h1 : h1;
        cp[1].push_back(i);
        cg0[1].push_back(g0);
        cgc[1].push_back(P.A * gu);
        cnch[1].push_back(choose_nch(P.N / 2, P.A * gu, bt.tpb, bt.nch_pref));
      }
      const int gmx = P.A * std::max(h1, Glp - h1);
      smem[1] = std::max(smem[1], apt_smem_bytes(P.N, gmx, bt.tpb / 32, mode, icm, P.T, n_bins, 1));
      smem_ns = std::max(smem_ns, apt_smem_bytes(P.N, gmx, bt.tpb / 32, mode, icm, P.T, n_bins, 0));
      continue;
    }
    // equal chunks of at most gmax groups
    const int nchunk = (G + gmax - 1) / gmax, per = (G + nchunk - 1) / nchunk;
    for (int g0 = 0; g0 < G; g0 += per) {
      const int gc = std::min(per, G - g0);
      cp[0].push_back(i);
      cg0[0].push_back(g0);
      cgc[0].push_back(gc);
      cnch[0].push_back(choose_nch(P.N / 2, gc, bt.tpb, bt.nch_pref));
      smem[0] = std::max(smem[0], apt_smem_bytes(P.N, gc, bt.tpb / 32, mode, icm, P.T, n_bins, 0));
    }
  }
  // the split part stages its swap tables only where its CTAs still fit
  bt.stage_swt = smem[1] <= (size_t)c->smem_optin;
  if (!bt.stage_swt) smem[1] = smem_ns;
  bt.n_u = (int)cp[0].size();
  bt.n_s = (int)cp[1].size();
  bt.split = bt.n_s > 0 && bt.n_u == 0;
  bt.hybrid = bt.n_s > 0 && bt.n_u > 0;
  bt.smem_u = smem[0];
  bt.smem_s = smem[1];
  const size_t smem_max = std::max(smem[0], smem[1]);
  bt.n_cta = bt.n_u + bt.n_s;
  for (int part = 0; part < 2; ++part)
    for (int g : cgc[part])
      if (g < 1 || g > kMaxGcCta) return fail(PC_EINVAL, "internal: a CTA would hold more than 64 replicas");
  if (smem_max > (size_t)c->smem_optin) return fail(PC_EINVAL, "problem does not fit in shared memory");
  bt.smem = smem_max;
  std::vector<int> all;
  for (int part = 0; part < 2; ++part) {
    all.insert(all.end(), cp[part].begin(), cp[part].end());
    all.insert(all.end(), cg0[part].begin(), cg0[part].end());
    all.insert(all.end(), cgc[part].begin(), cgc[part].end());
    all.insert(all.end(), cnch[part].begin(), cnch[part].end());
  }
  int rc;
  if (bt.d_cta.n < all.size() && (rc = bt.d_cta.alloc(all.size()))) return rc;
  if (!all.empty())
    PC_CUDA_TRY(cudaMemcpyAsync(bt.d_cta.p, all.data(), all.size() * 4, cudaMemcpyHostToDevice, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
}

int set_counters(pc_ctx *c, Batch &bt, int64_t s0, int64_t t0) {
  const int64_t v[2] = {s0, t0};
  PC_CUDA_TRY(cudaMemcpyAsync(bt.d_ctr.p, v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
}

int max_words(const Batch &bt) {
  int m = 0;
  for (size_t i = 0; i < bt.prob.size(); ++i) m = std::max(m, bt.G[i] * bt.prob[i].N);
  return m;
}

// A second stream and two events for the two launches of a mixed batch.
struct Fork {
  cudaStream_t st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  Fork() = default;
  Fork(const Fork &) = delete;
  Fork &operator=(const Fork &) = delete;
  ~Fork() {
    if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  int ensure() {
    if (!st) PC_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (cudaEvent_t &e : ev)
      if (!e) PC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return PC_OK;
  }
};

// The APT kernel over a scheduled batch: one launch, or, when some problems
// run as two-CTA clusters and the others as one CTA (split preference 3),
// the cluster part on a second stream beside the one-CTA part, forked from
// and joined back into `st` with events (under stream capture the two become
// parallel nodes of the graph).  The parts hold disjoint problems, so their
// order does not matter.
int launch_parts(Batch &bt, AptArgs a, cudaStream_t st, Fork &f) {
  if (!bt.hybrid) {
    a.split = bt.split;
    return apt_launch(a, bt.n_cta, bt.tpb, bt.smem, st);
  }
  int rc;
  if ((rc = f.ensure())) return rc;
  AptArgs as = a, au = a;
  int *ts = bt.d_cta.p + 4 * bt.n_u;
  int least = 0, greatest = 0;
  PC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  as.split = 1;
  as.prio = greatest;
  as.cta_prob = ts;
  as.cta_g0 = ts + bt.n_s;
  as.cta_gc = ts + 2 * bt.n_s;
  as.cta_nch = ts + 3 * bt.n_s;
  au.split = 0;
  au.cta_prob = bt.d_cta.p;
  au.cta_g0 = bt.d_cta.p + bt.n_u;
  au.cta_gc = bt.d_cta.p + 2 * bt.n_u;
  au.cta_nch = bt.d_cta.p + 3 * bt.n_u;
  PC_CUDA_TRY(cudaEventRecord(f.ev[0], st));
  PC_CUDA_TRY(cudaStreamWaitEvent(f.st, f.ev[0], 0));
  if ((rc = apt_launch(as, bt.n_s, bt.tpb, bt.smem_s, f.st))) return rc;
  if ((rc = apt_launch(au, bt.n_u, bt.tpb, bt.smem_u, st))) return rc;
  PC_CUDA_TRY(cudaEventRecord(f.ev[1], f.st));
  PC_CUDA_TRY(cudaStreamWaitEvent(st, f.ev[1], 0));
  return PC_OK;
}

}  // namespace

// -------------------------------------------------------------------- APT
struct AptImpl {
  Batch bt;
  int A = 0;
  std::vector<ProbSpec> specs;        // the loaded problems (J copied below)
  std::vector<std::vector<int8_t>> Jcopy;
  std::vector<std::vector<uint8_t>> Pcopy;   // vacancy masks of the loaded problems
  bool icm_ok = false;
  // CUDA graph of one chunk of kChunkAttempts swap attempts
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int g_spp = -1, g_icm = -1;
  int joint = 0;                      // joint-label swap rule
  int icm_big = 1, icm_seed = 0;      // ICMop rules (pc_apt_set_icm_rules)
  Fork fork;                          // the second launch of a mixed placement
  ~AptImpl() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

}  // namespace pc

using namespace pc;

static AptImpl *apt_impl(pc_ctx *c) { return static_cast<AptImpl *>(c->apt_impl); }

void pc_apt_release_impl(pc_ctx *c) try {
  delete apt_impl(c);
  c->apt_impl = nullptr;
} catch (...) {
}

// ------------------------------------------------------------ checkpoints
namespace {

constexpr uint64_t kCkptMagic = 0x31544B43504D4350ull;   // "PCMPCKT1"

template <typename T>
int dev_io(FILE *f, DevBuf<T> &b, bool save) {
  std::vector<T> h(b.n);
  if (save) {
    PC_CUDA_TRY(cudaMemcpy(h.data(), b.p, b.n * sizeof(T), cudaMemcpyDeviceToHost));
    if (fwrite(h.data(), sizeof(T), b.n, f) != b.n) return fail(PC_EINVAL, "checkpoint write failed");
  } else {
    if (fread(h.data(), sizeof(T), b.n, f) != b.n) return fail(PC_EINVAL, "checkpoint is truncated");
    PC_CUDA_TRY(cudaMemcpy(b.p, h.data(), b.n * sizeof(T), cudaMemcpyHostToDevice));
  }
  return PC_OK;
}

// Identity of the loaded batch: problem shapes, ladders' sizes, entry ids
// and the seed; a checkpoint restores only into an identical batch.
std::vector<uint64_t> batch_identity(pc_ctx *c, const Batch &bt) {
  std::vector<uint64_t> id = {c->seed, (uint64_t)bt.prob.size()};
  for (const AptProbDev &P : bt.prob) {
    id.push_back(((uint64_t)P.Lx << 40) | ((uint64_t)P.Ly << 20) | (uint64_t)P.Lz);
    id.push_back(((uint64_t)P.T << 32) | ((uint64_t)P.A << 16) | (uint64_t)P.B);
    id.push_back(((uint64_t)P.open << 32) | P.ent);
  }
  return id;
}

int ckpt_io(pc_ctx *c, const char *path, bool save) {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (!path) return fail(PC_EINVAL, "path is NULL");
  Batch &bt = apt_impl(c)->bt;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  FILE *f = fopen(path, save ? "wb" : "rb");
  if (!f) return fail(PC_EINVAL, std::string("cannot open checkpoint ") + path);
  std::vector<uint64_t> id = batch_identity(c, bt);
  int rc = PC_OK;
  uint64_t hdr[3] = {kCkptMagic, (uint64_t)id.size(), 0};
  if (save) {
    hdr[2] = 0;
    int64_t ctrs[2] = {c->apt.sweeps, c->apt.swaps};
    if (fwrite(hdr, 8, 3, f) != 3 || fwrite(id.data(), 8, id.size(), f) != id.size() ||
        fwrite(ctrs, 8, 2, f) != 2)
      rc = fail(PC_EINVAL, "checkpoint write failed");
  } else {
    uint64_t h[3];
    std::vector<uint64_t> fid(id.size());
    int64_t ctrs[2];
    if (fread(h, 8, 3, f) != 3 || h[0] != kCkptMagic || h[1] != id.size() ||
        fread(fid.data(), 8, fid.size(), f) != fid.size() || fid != id || fread(ctrs, 8, 2, f) != 2)
      rc = fail(PC_EINVAL, "checkpoint does not match the loaded batch");
    else {
      c->apt.sweeps = ctrs[0];
      c->apt.swaps = ctrs[1];
    }
  }
  if (!rc) rc = dev_io(f, bt.d_spins, save);
  if (!rc) rc = dev_io(f, bt.d_E, save);
  if (!rc) rc = dev_io(f, bt.d_temp, save);
  if (!rc) rc = dev_io(f, bt.d_bestE, save);
  if (!rc) rc = dev_io(f, bt.d_bestsweep, save);
  if (!rc) rc = dev_io(f, bt.d_hit, save);
  if (!rc) rc = dev_io(f, bt.d_target, save);
  if (!rc) rc = dev_io(f, bt.d_bestbuf, save);
  if (!rc) rc = dev_io(f, bt.d_bestspins, save);
  if (!rc) rc = dev_io(f, bt.d_stats, save);
  if (!rc) rc = dev_io(f, bt.d_ctr, save);
  fclose(f);
  return rc;
}

}  // namespace

extern "C" {

int pc_apt_load(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, const int32_t *n_temps,
                const double *betas, int n_labels, uint32_t entry0) try {
  return pc_apt_load_bc(c, n_inst, dims, nullptr, nullptr, J, n_temps, betas, n_labels, entry0);
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_load_bc(pc_ctx *c, int n_inst, const int32_t *dims, const uint8_t *periodic,
                   const uint8_t *present, const int8_t *J, const int32_t *n_temps, const double *betas,
                   int n_labels, uint32_t entry0) try {
  if (!c || !dims || !J || !n_temps || !betas) return fail(PC_EINVAL, "NULL argument");
  if (n_inst < 1) return fail(PC_EINVAL, "n_inst must be >= 1");
  if (!(n_labels == 1 || n_labels == 2 || n_labels == 4))
    return fail(PC_EINVAL, "n_labels must be 1, 2 or 4");
  if ((uint64_t)entry0 + (uint64_t)n_inst > (1ull << 24)) return fail(PC_EINVAL, "entry ids must be < 2^24");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  std::vector<ProbSpec> specs((size_t)n_inst);
  size_t joff = 0, boff = 0;
  for (int i = 0; i < n_inst; ++i) {
    ProbSpec &s = specs[(size_t)i];
    int rc = check_lattice(dims + 3 * i, J + 3 * joff, &s.lat);
    if (rc) return rc;
    for (int ax = 0; ax < 3; ++ax) s.per[ax] = periodic ? (periodic[3 * i + ax] != 0) : 1;
    s.present = present ? present + joff : nullptr;
    s.J = J + 3 * joff;
    s.T = n_temps[i];
    s.A = n_labels;
    s.Tp = 8 * ((s.T + 7) / 8);
    s.B = s.Tp * n_labels;     // replica of (r, a) in buffer a * Tp + r
    // up to 64 replicas in one CTA; up to 128 (e.g. 32 temperatures x 4
    // labels) in a cluster of two CTAs that split the temperatures
    if (s.T < 1 || s.T > 32 || s.B > 128)
      return fail(PC_EINVAL, "need 1 <= n_temps <= 32 and 8*ceil(n_temps/8) * n_labels <= 128");
    s.ent = entry0 + (uint32_t)i;
    s.beta.assign(betas + boff, betas + boff + s.T);
    for (int t = 0; t < s.T; ++t) {
      if (!(s.beta[(size_t)t] >= 0.0) || !std::isfinite(s.beta[(size_t)t]))
        return fail(PC_EINVAL, "betas must be finite and >= 0");
      if (t > 0 && !(s.beta[(size_t)t] > s.beta[(size_t)t - 1]))
        return fail(PC_EINVAL, "betas must be strictly increasing");
    }
    s.temp_of.resize((size_t)s.B);
    for (int b = 0; b < s.B; ++b) s.temp_of[(size_t)b] = (b % s.Tp < s.T) ? b % s.Tp : 0;
    s.swaps = true;
    joff += (size_t)s.lat.N;
    boff += (size_t)s.T;
  }
  pc_apt_release_impl(c);
  AptImpl *im = new AptImpl();
  c->apt_impl = im;
  c->apt.ready = false;
  im->A = n_labels;
  im->Jcopy.resize(specs.size());
  im->Pcopy.resize(specs.size());
  for (size_t i = 0; i < specs.size(); ++i) {
    im->Jcopy[i].assign(specs[i].J, specs[i].J + 3 * (size_t)specs[i].lat.N);
    specs[i].J = im->Jcopy[i].data();
    if (specs[i].present) {
      im->Pcopy[i].assign(specs[i].present, specs[i].present + (size_t)specs[i].lat.N);
      specs[i].present = im->Pcopy[i].data();
    }
  }
  im->specs = specs;
  int rc = build_batch(c, im->bt, specs, 0);
  if (rc) return rc;
  if ((rc = schedule(c, im->bt, {}, APT_MODE_APT, n_labels >= 2, 0))) return rc;
  AptArgs a = base_args(c, im->bt);
  a.tag_init = 1;   // TAG_APT_INIT
  if ((rc = apt_init_launch(a, n_inst, max_words(im->bt), c->stream))) return rc;
  a.mode = APT_MODE_ENERGY;
  if ((rc = launch_parts(im->bt, a, c->stream, im->fork))) return rc;
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->apt.ready = true;
  c->apt.n = n_inst;
  c->apt.A = n_labels;
  c->apt.sweeps = 0;
  c->apt.swaps = 0;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

static int apt_enqueue(pc_ctx *c, AptImpl *im, int n_iter, int spp, int icm) {
  AptArgs a = base_args(c, im->bt);
  a.mode = APT_MODE_APT;
  a.n_iter = n_iter;
  a.spp = spp;
  a.icm = icm;
  a.joint_swap = im->joint;
  a.icm_big = im->icm_big;
  a.icm_seed = im->icm_seed;
  a.tag_main = 2;    // TAG_APT_SWEEP
  a.tag_ref = 3;     // TAG_APT_REFINE
  int rc = launch_parts(im->bt, a, c->stream, im->fork);
  if (rc) return rc;
  return apt_advance_launch(im->bt.d_ctr.p, (int64_t)n_iter * spp, n_iter, c->stream);
}

int pc_apt_set_joint_swap(pc_ctx *c, int joint) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  AptImpl *im = apt_impl(c);
  im->joint = joint ? 1 : 0;
  im->g_spp = -1;   // the captured chunk bakes the rule in: capture again
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_set_icm_rules(pc_ctx *c, int big_cluster_rule, int cluster_seed) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  AptImpl *im = apt_impl(c);
  im->icm_big = big_cluster_rule ? 1 : 0;
  im->icm_seed = cluster_seed ? 1 : 0;
  im->g_spp = -1;   // the captured chunk bakes the rules in: capture again
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_run(pc_ctx *c, int64_t n_swaps, int sweeps_per_swap, int icm) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (n_swaps < 0 || sweeps_per_swap < 1) return fail(PC_EINVAL, "n_swaps >= 0, sweeps_per_swap >= 1");
  AptImpl *im = apt_impl(c);
  if (icm && im->A < 2) return fail(PC_EINVAL, "ICM needs two or four labels per temperature");
  if (c->apt.sweeps + n_swaps * sweeps_per_swap > 0xFFFFFFFFll || c->apt.swaps + n_swaps > 0xFFFFFFFFll)
    return fail(PC_EINVAL, "sweep counter would exceed 2^32");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  icm = icm ? 1 : 0;
  int64_t left = n_swaps;
  // whole chunks replay one CUDA graph (sweep kernel + counter advance)
  if (left >= kChunkAttempts) {
    if (!im->exec || im->g_spp != sweeps_per_swap || im->g_icm != icm) {
      if (im->exec) cudaGraphExecDestroy(im->exec);
      if (im->graph) cudaGraphDestroy(im->graph);
      im->exec = nullptr;
      im->graph = nullptr;
      cudaStream_t cap;
      PC_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      int rc = PC_OK;
      if (e == cudaSuccess) {
        cudaStream_t saved = c->stream;
        c->stream = cap;
        rc = apt_enqueue(c, im, kChunkAttempts, sweeps_per_swap, icm);
        c->stream = saved;
        cudaError_t e2 = cudaStreamEndCapture(cap, &im->graph);
        if (!rc && e2 != cudaSuccess) rc = fail(PC_ECUDA, std::string("capture: ") + cudaGetErrorString(e2));
      } else {
        rc = fail(PC_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
      }
      cudaStreamDestroy(cap);
      if (rc) return rc;
      PC_CUDA_TRY(cudaGraphInstantiate(&im->exec, im->graph, 0));
      im->g_spp = sweeps_per_swap;
      im->g_icm = icm;
    }
    while (left >= kChunkAttempts) {
      PC_CUDA_TRY(cudaGraphLaunch(im->exec, c->stream));
      left -= kChunkAttempts;
    }
  }
  if (left > 0) {
    int rc = apt_enqueue(c, im, (int)left, sweeps_per_swap, icm);
    if (rc) return rc;
  }
  c->apt.sweeps += n_swaps * sweeps_per_swap;
  c->apt.swaps += n_swaps;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

}  // extern "C"

namespace {

// Re-schedules the loaded batch with a new launch shape; the chains do not
// move.  On failure the old shape is restored.
int apply_shape(pc_ctx *c, AptImpl *im, int tpb, int nch_pref, int split_pref, int split_h) {
  Batch &bt = im->bt;
  const int o_tpb = bt.tpb, o_nch = bt.nch_pref, o_split = bt.split_pref, o_h = bt.split_h;
  bt.tpb = tpb;
  bt.nch_pref = nch_pref;
  bt.split_pref = split_pref;
  bt.split_h = split_h;
  int rc = schedule(c, bt, {}, APT_MODE_APT, im->A >= 2, 0);
  if (rc) {
    bt.tpb = o_tpb;
    bt.nch_pref = o_nch;
    bt.split_pref = o_split;
    bt.split_h = o_h;
    schedule(c, bt, {}, APT_MODE_APT, im->A >= 2, 0);
    return rc;
  }
  if (im->exec) cudaGraphExecDestroy(im->exec);
  if (im->graph) cudaGraphDestroy(im->graph);
  im->exec = nullptr;
  im->graph = nullptr;
  // a mixed placement's second stream and events exist before any capture
  if (bt.hybrid) return im->fork.ensure();
  return PC_OK;
}

}  // namespace

extern "C" {

int pc_apt_autotune(pc_ctx *c, int trial_swaps, int icm, int *tpb_out, int *nch_out, int *split_out,
                    int *groups_out) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (trial_swaps < 1) return fail(PC_EINVAL, "trial_swaps must be >= 1");
  AptImpl *im = apt_impl(c);
  if (icm && im->A < 2) return fail(PC_EINVAL, "ICM needs two or four labels per temperature");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  // candidates: one CTA per problem or two-CTA clusters (where every
  // problem can split; problems above 64 replicas always split), threads
  // per CTA, and the threads' split over sites and replica groups
  bool can_split = true;
  for (const AptProbDev &P : im->bt.prob) can_split = can_split && (P.Tp >> 3) >= 2;
  int glp_max = 0;
  for (const AptProbDev &P : im->bt.prob) glp_max = std::max(glp_max, P.Tp >> 3);
  const int splits[3] = {1, 2, 3}, tpbs[5] = {256, 320, 384, 448, 512}, nchs[4] = {0, 1, 2, 4};
  struct Best { float ms; int tpb, nch, split, h; } best = {1e30f, im->bt.tpb, im->bt.nch_pref, im->bt.split_pref,
                                                            im->bt.split_h};
  cudaEvent_t e0, e1;
  PC_CUDA_TRY(cudaEventCreate(&e0));
  PC_CUDA_TRY(cudaEventCreate(&e1));
  int rc = PC_OK;
  for (int sp : splits)
   for (int h = 0; h <= (sp >= 2 ? std::min(3, glp_max - 1) : 0); ++h) {
    if (sp == 2 && !can_split) continue;
    if (sp >= 2 && h > 0 && 2 * h == glp_max) continue;   // the even split is h = 0
    for (int tpb : tpbs)
      for (int nch : nchs) {
        if (rc) break;
        // a scratch copy of the batch: the loaded chains are not advanced
        Batch tmp;
        tmp.tpb = tpb;
        tmp.split_pref = sp;
        tmp.nch_pref = nch;
        tmp.split_h = h;
        if ((rc = build_batch(c, tmp, im->specs, 0))) break;
        if (schedule(c, tmp, {}, APT_MODE_APT, im->A >= 2, 0)) continue;   // does not fit: skip
        if (sp == 3 && !tmp.hybrid) continue;   // the same placement as preference 1 or 2
        if (nch > 0) {   // skip a forced split that the schedule could not honour
          std::vector<int> h((size_t)tmp.n_cta);
          PC_CUDA_TRY(cudaMemcpy(h.data(), tmp.d_cta.p + 3 * tmp.n_cta, h.size() * 4, cudaMemcpyDeviceToHost));
          bool used = false;
          for (int v : h) used = used || v == nch;
          if (!used) continue;
        }
        AptArgs a = base_args(c, tmp);
        a.tag_init = 1;
        if ((rc = apt_init_launch(a, (int)im->specs.size(), max_words(tmp), c->stream))) break;
        a.mode = APT_MODE_APT;
        a.n_iter = trial_swaps;
        a.spp = 1;
        a.icm = icm ? 1 : 0;
        a.icm_big = im->icm_big;
        a.icm_seed = im->icm_seed;
        a.joint_swap = im->joint;
        a.tag_main = 2;
        a.tag_ref = 3;
        if ((rc = launch_parts(tmp, a, c->stream, im->fork))) break;   // warm-up
        PC_CUDA_TRY(cudaEventRecord(e0, c->stream));
        if ((rc = launch_parts(tmp, a, c->stream, im->fork))) break;
        PC_CUDA_TRY(cudaEventRecord(e1, c->stream));
        PC_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best.ms) best = {ms, tpb, nch, sp, h};
      }
   }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = apply_shape(c, im, best.tpb, best.nch, best.split, best.h))) return rc;
  if (tpb_out) *tpb_out = best.tpb;
  if (nch_out) *nch_out = best.nch;
  if (split_out) *split_out = im->bt.hybrid ? 2 : im->bt.split;
  if (groups_out) *groups_out = (im->bt.split || im->bt.hybrid) ? best.h : 0;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_set_launch(pc_ctx *c, int tpb, int nch, int split_pref, int split_groups) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (tpb < 64 || tpb > 512 || tpb % 64) return fail(PC_EINVAL, "tpb must be a multiple of 64 in [64, 512]");
  if (nch < 0 || nch > 8 || (nch & (nch - 1))) return fail(PC_EINVAL, "nch must be 0, 1, 2, 4 or 8");
  if (split_pref < 0 || split_pref > 3) return fail(PC_EINVAL, "split_pref must be 0, 1, 2 or 3");
  if (split_groups < 0 || split_groups > 3) return fail(PC_EINVAL, "split_groups must be 0 .. 3");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return apply_shape(c, apt_impl(c), tpb, nch, split_pref, split_groups);
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_set_split(pc_ctx *c, int pref) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (pref < 0 || pref > 3) return fail(PC_EINVAL, "pref must be 0, 1, 2 or 3");
  AptImpl *im = apt_impl(c);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return apply_shape(c, im, im->bt.tpb, im->bt.nch_pref, pref, im->bt.split_h);
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_is_split(pc_ctx *c, int *split) try {
  if (!c || !c->apt.ready || !apt_impl(c) || !split) return fail(PC_ESTATE, "pc_apt_load first");
  *split = apt_impl(c)->bt.hybrid ? 2 : apt_impl(c)->bt.split;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_set_block_threads(pc_ctx *c, int tpb) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (tpb < 64 || tpb > 512 || tpb % 64) return fail(PC_EINVAL, "tpb must be a multiple of 64 in [64, 512]");
  AptImpl *im = apt_impl(c);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return apply_shape(c, im, tpb, im->bt.nch_pref, im->bt.split_pref, im->bt.split_h);
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_progress(pc_ctx *c, int64_t *sweeps, int64_t *swaps) try {
  if (!c || !c->apt.ready) return fail(PC_ESTATE, "pc_apt_load first");
  if (sweeps) *sweeps = c->apt.sweeps;
  if (swaps) *swaps = c->apt.swaps;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

static int check_inst(pc_ctx *c, int inst) {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  if (inst < 0 || inst >= c->apt.n) return fail(PC_EINVAL, "instance index out of range");
  return PC_OK;
}

int pc_apt_save(pc_ctx *c, const char *path) try { return ckpt_io(c, path, true); } catch (...) { return pc::fail_exception(); }
int pc_apt_restore(pc_ctx *c, const char *path) try { return ckpt_io(c, path, false); } catch (...) { return pc::fail_exception(); }

int pc_apt_set_target(pc_ctx *c, int inst, int64_t e_target) try {
  int rc = check_inst(c, inst);
  if (rc) return rc;
  Batch &bt = apt_impl(c)->bt;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  int64_t best = 0, bsw = 0;
  PC_CUDA_TRY(cudaMemcpy(&best, bt.d_bestE.p + inst, 8, cudaMemcpyDeviceToHost));
  PC_CUDA_TRY(cudaMemcpy(&bsw, bt.d_bestsweep.p + inst, 8, cudaMemcpyDeviceToHost));
  const int64_t hit = (best <= e_target) ? bsw : -1;
  PC_CUDA_TRY(cudaMemcpy(bt.d_target.p + inst, &e_target, 8, cudaMemcpyHostToDevice));
  PC_CUDA_TRY(cudaMemcpy(bt.d_hit.p + inst, &hit, 8, cudaMemcpyHostToDevice));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_get_state(pc_ctx *c, int inst, int8_t *spins, int64_t *energies, int32_t *temp_of) try {
  int rc = check_inst(c, inst);
  if (rc) return rc;
  Batch &bt = apt_impl(c)->bt;
  const AptProbDev &P = bt.prob[(size_t)inst];
  const int G = bt.G[(size_t)inst];
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int nslot = P.T * P.A;
  if (spins) {
    std::vector<uint32_t> w((size_t)G * P.N);
    PC_CUDA_TRY(cudaMemcpy(w.data(), bt.d_spins.p + P.spin_off, w.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<int8_t> all((size_t)P.B * P.N);
    unpack_spins(P, w.data(), P.B, all.data());
    for (int sl = 0; sl < nslot; ++sl) {
      const int b = (sl % P.A) * P.Tp + sl / P.A;
      std::memcpy(spins + (size_t)sl * P.N, all.data() + (size_t)b * P.N, (size_t)P.N);
    }
  }
  if (energies) {
    std::vector<int32_t> e((size_t)P.B);
    PC_CUDA_TRY(cudaMemcpy(e.data(), bt.d_E.p + P.buf_off, e.size() * 4, cudaMemcpyDeviceToHost));
    for (int sl = 0; sl < nslot; ++sl) energies[sl] = e[(size_t)((sl % P.A) * P.Tp + sl / P.A)];
  }
  if (temp_of)
    for (int sl = 0; sl < nslot; ++sl) temp_of[sl] = sl / P.A;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_get_best(pc_ctx *c, int inst, int64_t *E, int64_t *sweep, int32_t *buf, int64_t *hit_sweep,
                    int8_t *spins) try {
  int rc = check_inst(c, inst);
  if (rc) return rc;
  Batch &bt = apt_impl(c)->bt;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (E) PC_CUDA_TRY(cudaMemcpy(E, bt.d_bestE.p + inst, 8, cudaMemcpyDeviceToHost));
  if (sweep) PC_CUDA_TRY(cudaMemcpy(sweep, bt.d_bestsweep.p + inst, 8, cudaMemcpyDeviceToHost));
  if (buf) {
    int32_t b = -1;
    PC_CUDA_TRY(cudaMemcpy(&b, bt.d_bestbuf.p + inst, 4, cudaMemcpyDeviceToHost));
    const AptProbDev &P = bt.prob[(size_t)inst];
    *buf = (b < 0) ? -1 : (b % P.Tp) * P.A + b / P.Tp;   // slot index
  }
  if (hit_sweep) PC_CUDA_TRY(cudaMemcpy(hit_sweep, bt.d_hit.p + inst, 8, cudaMemcpyDeviceToHost));
  if (spins)
    PC_CUDA_TRY(cudaMemcpy(spins, bt.d_bestspins.p + bt.prob[(size_t)inst].best_off,
                           (size_t)bt.prob[(size_t)inst].N, cudaMemcpyDeviceToHost));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_get_best_all(pc_ctx *c, int64_t *E, int64_t *hit_sweep) try {
  if (!c || !c->apt.ready || !apt_impl(c)) return fail(PC_ESTATE, "pc_apt_load first");
  Batch &bt = apt_impl(c)->bt;
  const size_t n = bt.prob.size();
  PC_CUDA_TRY(cudaSetDevice(c->device));
  if (E) PC_CUDA_TRY(cudaMemcpyAsync(E, bt.d_bestE.p, 8 * n, cudaMemcpyDeviceToHost, c->stream));
  if (hit_sweep) PC_CUDA_TRY(cudaMemcpyAsync(hit_sweep, bt.d_hit.p, 8 * n, cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_get_stats(pc_ctx *c, int inst, int64_t *att, int64_t *acc, int64_t *icm) try {
  int rc = check_inst(c, inst);
  if (rc) return rc;
  Batch &bt = apt_impl(c)->bt;
  const AptProbDev &P = bt.prob[(size_t)inst];
  const int np = (P.T - 1) * P.A;
  std::vector<int64_t> s((size_t)2 * np + 3);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  PC_CUDA_TRY(cudaMemcpy(s.data(), bt.d_stats.p + P.stat_off, s.size() * 8, cudaMemcpyDeviceToHost));
  if (att) std::memcpy(att, s.data(), 8 * (size_t)np);
  if (acc) std::memcpy(acc, s.data() + np, 8 * (size_t)np);
  if (icm) std::memcpy(icm, s.data() + 2 * np, 24);
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_get_pbit_table(pc_ctx *c, int inst, uint32_t *out) try {
  int rc = check_inst(c, inst);
  if (rc) return rc;
  Batch &bt = apt_impl(c)->bt;
  const AptProbDev &P = bt.prob[(size_t)inst];
  for (int t = 0; t < P.T; ++t)
    for (int cc = 0; cc < 7; ++cc) out[7 * t + cc] = bt.h_pbit[P.pbit_off + 16 * t + 2 * cc];
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_apt_get_swap_table(pc_ctx *c, int inst, int pair, uint32_t *out, int max_len, int *len) try {
  int rc = check_inst(c, inst);
  if (rc) return rc;
  Batch &bt = apt_impl(c)->bt;
  const AptProbDev &P = bt.prob[(size_t)inst];
  if (pair < 0 || pair + 1 >= P.T) return fail(PC_EINVAL, "pair out of range");
  const uint32_t off = bt.h_swapidx[P.swapidx_off + 2 * pair], n = bt.h_swapidx[P.swapidx_off + 2 * pair + 1];
  if (len) *len = (int)n;
  for (int k = 0; k < max_len && k < (int)n; ++k) out[k] = bt.h_swaptab[off + k];
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

// ------------------------------------------------------------------ ladder
}  // extern "C"

namespace {

// The adaptive beta ladder of Algorithm S2's preprocessing for n_inst
// lattices, instance i drawing with Philox entry ents[i]; outputs as
// pc_adaptive_ladder.  Arguments are checked by the callers.
int adaptive_impl(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, const uint32_t *ents,
                  double beta0, double alpha, int n_chains, int sweeps, int tail, double tol, int max_len,
                  double *beta_out, double *sigma_out, int32_t *len_out, int32_t *converged_out) {
  PC_CUDA_TRY(cudaSetDevice(c->device));
  std::vector<ProbSpec> specs((size_t)n_inst);
  size_t joff = 0;
  for (int i = 0; i < n_inst; ++i) {
    ProbSpec &s = specs[(size_t)i];
    int rc = check_lattice(dims + 3 * i, J + 3 * joff, &s.lat);
    if (rc) return rc;
    if ((int64_t)tail * 3 * s.lat.N * 3 * s.lat.N > (int64_t)1 << 62)
      return fail(PC_EINVAL, "tail too long for exact int64 sums");
    s.J = J + 3 * joff;
    s.T = 1;
    s.Tp = 1;
    s.A = 1;
    s.B = n_chains;
    s.ent = ents[i];
    s.beta.assign(1, beta0);
    s.temp_of.assign((size_t)n_chains, 0);
    s.swaps = false;
    joff += (size_t)s.lat.N;
  }
  Batch bt;
  int rc = build_batch(c, bt, specs, 0);
  if (rc) return rc;
  std::vector<double> beta((size_t)n_inst, beta0);
  std::vector<char> active((size_t)n_inst, 1);
  std::vector<int> len((size_t)n_inst, 0), conv((size_t)n_inst, 0);
  AptArgs a;
  if ((rc = schedule(c, bt, active, APT_MODE_LADDER, 0, 0))) return rc;
  a = base_args(c, bt);
  a.tag_init = 6;   // TAG_LAD_INIT
  if ((rc = apt_init_launch(a, n_inst, max_words(bt), c->stream))) return rc;
  std::vector<int64_t> s1, s2;
  for (int step = 0; step < max_len; ++step) {
    // thresholds of each active instance's current beta
    std::vector<uint32_t> pb((size_t)16 * n_inst, 0u);
    for (int i = 0; i < n_inst; ++i)
      for (int e = 0; e < 13; ++e) pb[(size_t)16 * i + e] = pc_pbit_threshold(beta[(size_t)i], e - 6);
    PC_CUDA_TRY(cudaMemcpyAsync(bt.d_pbit.p, pb.data(), pb.size() * 4, cudaMemcpyHostToDevice, c->stream));
    if ((rc = schedule(c, bt, active, APT_MODE_LADDER, 0, 0))) return rc;
    if ((rc = set_counters(c, bt, (int64_t)step * sweeps, 0))) return rc;
    a = base_args(c, bt);
    a.mode = APT_MODE_LADDER;
    a.n_iter = sweeps;
    a.spp = 1;
    a.window_from = sweeps - tail;
    a.tag_main = 7;   // TAG_LAD_SWEEP
    a.tag_ref = 8;    // TAG_LAD_REFINE
    if ((rc = apt_launch(a, bt.n_cta, bt.tpb, bt.smem, c->stream))) return rc;
    s1.resize(bt.d_sum1.n);
    s2.resize(bt.d_sum2.n);
    PC_CUDA_TRY(cudaMemcpyAsync(s1.data(), bt.d_sum1.p, s1.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    PC_CUDA_TRY(cudaMemcpyAsync(s2.data(), bt.d_sum2.p, s2.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
    bool any = false;
    for (int i = 0; i < n_inst; ++i) {
      if (!active[(size_t)i]) continue;
      const AptProbDev &P = bt.prob[(size_t)i];
      double mean_var = 0.0;
      for (int b = 0; b < n_chains; ++b) {
        const int64_t sE = s1[P.buf_off + b], sE2 = s2[P.buf_off + b];
        const int64_t num = (int64_t)tail * sE2 - sE * sE;
        mean_var += (double)num / ((double)tail * (double)(tail - 1));
      }
      mean_var /= (double)n_chains;
      const double sigma = std::sqrt(mean_var);
      beta_out[(size_t)i * max_len + len[(size_t)i]] = beta[(size_t)i];
      if (sigma_out) sigma_out[(size_t)i * max_len + len[(size_t)i]] = sigma;
      len[(size_t)i] += 1;
      if (sigma < tol) {
        conv[(size_t)i] = 1;
        active[(size_t)i] = 0;
      } else if (len[(size_t)i] == max_len) {
        active[(size_t)i] = 0;
      } else {
        beta[(size_t)i] = beta[(size_t)i] + alpha / sigma;
        any = true;
      }
    }
    if (!any) break;
  }
  for (int i = 0; i < n_inst; ++i) {
    len_out[i] = len[(size_t)i];
    if (converged_out) converged_out[i] = conv[(size_t)i];
  }
  return PC_OK;
}

int check_ladder_params(int n_chains, int sweeps, int tail, int max_len, double beta0, double alpha) {
  if (n_chains < 1 || n_chains > 4096 || sweeps < 1 || tail < 2 || tail > sweeps || max_len < 1 ||
      !(beta0 > 0.0) || !(alpha > 0.0))
    return fail(PC_EINVAL, "bad ladder parameters");
  if ((int64_t)sweeps * max_len > 0xFFFFFFFFll) return fail(PC_EINVAL, "sweep counter would exceed 2^32");
  return PC_OK;
}

}  // namespace

extern "C" {

int pc_adaptive_ladder(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
                       double beta0, double alpha, int n_chains, int sweeps, int tail, double tol,
                       int max_len, double *beta_out, double *sigma_out, int32_t *len_out,
                       int32_t *converged_out) try {
  if (!c || !dims || !J || !beta_out || !len_out) return fail(PC_EINVAL, "NULL argument");
  if (n_inst < 1) return fail(PC_EINVAL, "bad ladder parameters");
  int rc = check_ladder_params(n_chains, sweeps, tail, max_len, beta0, alpha);
  if (rc) return rc;
  if ((uint64_t)entry0 + (uint64_t)n_inst > (1ull << 24)) return fail(PC_EINVAL, "entry ids must be < 2^24");
  std::vector<uint32_t> ents((size_t)n_inst);
  for (int i = 0; i < n_inst; ++i) ents[(size_t)i] = entry0 + (uint32_t)i;
  return adaptive_impl(c, n_inst, dims, J, ents.data(), beta0, alpha, n_chains, sweeps, tail, tol, max_len,
                       beta_out, sigma_out, len_out, converged_out);
} catch (...) {
  return pc::fail_exception();
}

int pc_resample_ladder(const double *beta, int len, int n, double *out) try {
  if (!beta || !out || len < 1 || n < 2) return fail(PC_EINVAL, "bad arguments");
  if (len == 1) {
    for (int k = 0; k < n; ++k) out[k] = beta[0];
    return PC_OK;
  }
  for (int k = 0; k < n; ++k) {
    const double pos = (double)k * (double)(len - 1) / (double)(n - 1);
    int lo = (int)std::floor(pos);
    if (lo > len - 2) lo = len - 2;
    const double w = pos - (double)lo;
    out[k] = beta[lo] * (1.0 - w) + beta[lo + 1] * w;
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

// ------------------------------------------------------------------ pilot
}  // extern "C"

namespace {

int check_pilot_params(int n_inst, uint32_t entry0, int n_beta, const double *betas, int chains_per_beta,
                       int sweeps, int burn, int n_bins) {
  if (n_inst < 1 || n_beta < 1 || chains_per_beta < 1 || n_beta * chains_per_beta > 64 || sweeps < 1 ||
      burn < 0 || burn >= sweeps || n_bins < 1 || n_bins > 256 || n_beta * n_bins > 2048)
    return fail(PC_EINVAL, "bad pilot parameters (n_beta * chains_per_beta <= 64)");
  if ((uint64_t)entry0 + (uint64_t)n_inst > (1ull << 24)) return fail(PC_EINVAL, "entry ids must be < 2^24");
  for (int t = 0; t < n_beta; ++t)
    if (!(betas[t] >= 0.0) || !std::isfinite(betas[t])) return fail(PC_EINVAL, "betas must be finite and >= 0");
  return PC_OK;
}

// Runs the pilot chains of every instance on the device; the histograms stay
// in bt.d_hist ([n][n_beta][n_bins] at each problem's hist_off).
int pilot_run(pc_ctx *c, Batch &bt, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
              int n_beta, const double *betas, int chains_per_beta, int sweeps, int burn, int n_bins) {
  PC_CUDA_TRY(cudaSetDevice(c->device));
  std::vector<ProbSpec> specs((size_t)n_inst);
  size_t joff = 0;
  for (int i = 0; i < n_inst; ++i) {
    ProbSpec &s = specs[(size_t)i];
    int rc = check_lattice(dims + 3 * i, J + 3 * joff, &s.lat);
    if (rc) return rc;
    s.J = J + 3 * joff;
    s.T = n_beta;
    s.Tp = n_beta;
    s.A = 1;
    s.B = n_beta * chains_per_beta;
    s.ent = entry0 + (uint32_t)i;
    s.beta.assign(betas, betas + n_beta);
    s.temp_of.resize((size_t)s.B);
    for (int b = 0; b < s.B; ++b) s.temp_of[(size_t)b] = b / chains_per_beta;
    s.swaps = false;
    joff += (size_t)s.lat.N;
  }
  int rc = build_batch(c, bt, specs, n_bins);
  if (rc) return rc;
  if ((rc = schedule(c, bt, {}, APT_MODE_PILOT, 0, n_bins))) return rc;
  if ((rc = set_counters(c, bt, 0, 0))) return rc;
  AptArgs a = base_args(c, bt);
  a.tag_init = 9;   // TAG_PIL_INIT
  if ((rc = apt_init_launch(a, n_inst, max_words(bt), c->stream))) return rc;
  a.mode = APT_MODE_PILOT;
  a.n_iter = sweeps;
  a.spp = 1;
  a.window_from = burn;
  a.n_bins = n_bins;
  a.tag_main = 10;   // TAG_PIL_SWEEP
  a.tag_ref = 11;    // TAG_PIL_REFINE
  return apt_launch(a, bt.n_cta, bt.tpb, bt.smem, c->stream);
}

}  // namespace

extern "C" {

int pc_pilot_hist(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
                  int n_beta, const double *betas, int chains_per_beta, int sweeps, int burn, int n_bins,
                  int64_t *counts) try {
  if (!c || !dims || !J || !betas || !counts) return fail(PC_EINVAL, "NULL argument");
  int rc = check_pilot_params(n_inst, entry0, n_beta, betas, chains_per_beta, sweeps, burn, n_bins);
  if (rc) return rc;
  Batch bt;
  if ((rc = pilot_run(c, bt, n_inst, dims, J, entry0, n_beta, betas, chains_per_beta, sweeps, burn, n_bins)))
    return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(counts, bt.d_hist.p, (size_t)n_inst * n_beta * n_bins * 8,
                              cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_instance_features(const int32_t *dims, const int8_t *J, double *out3) try {
  if (!dims || !J || !out3) return fail(PC_EINVAL, "NULL argument");
  Lattice lat;
  int rc = check_lattice(dims, J, &lat);
  if (rc) return rc;
  const int Lx = lat.L[0], Ly = lat.L[1], Lz = lat.L[2], N = lat.N;
  auto at = [&](int x, int y, int z) { return ((x % Lx) + Lx * ((y % Ly) + Ly * (z % Lz))); };
  int64_t pos = 0, frust = 0;
  for (int s = 0; s < N; ++s) {
    const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
    for (int d = 0; d < 3; ++d) pos += J[3 * s + d] > 0;
    // plaquettes in the (x,y), (x,z), (y,z) planes with lower corner s
    const int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b) {
        const int sa = at(x + e[a][0], y + e[a][1], z + e[a][2]);
        const int sb = at(x + e[b][0], y + e[b][1], z + e[b][2]);
        const int prod = J[3 * s + a] * J[3 * sa + b] * J[3 * sb + a] * J[3 * s + b];
        frust += prod < 0;
      }
  }
  out3[0] = std::cbrt((double)N) / 16.0;
  out3[1] = (double)pos / (3.0 * N);
  out3[2] = (double)frust / (3.0 * N);
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

// ------------------------------------------------------- learned ladder
}  // extern "C"

namespace {

constexpr int kLearnedLen = 32;        // ladder length of the network's head
constexpr int kLearnedBins = 64;       // pilot histogram bins of its input
constexpr int kLearnedBetas = 4;       // pilot temperatures of its input
constexpr double kLadderGap = 1e-6;    // least gap of a predicted ladder

// Probe of given ladders: the first `attempts` APT attempts of one sweep,
// ICM (n_labels >= 2) and the swaps, on a scratch batch whose problem i
// draws with entry entry0 + i (the loaded APT batch is not touched).
// att / acc [n][T-1]: swap attempts and accepts of each pair summed over the
// labels.
int probe_impl(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0, int T,
               const double *betas, int n_labels, int attempts, std::vector<int64_t> &att,
               std::vector<int64_t> &acc) {
  PC_CUDA_TRY(cudaSetDevice(c->device));
  std::vector<ProbSpec> specs((size_t)n_inst);
  size_t joff = 0;
  for (int i = 0; i < n_inst; ++i) {
    ProbSpec &s = specs[(size_t)i];
    int rc = check_lattice(dims + 3 * i, J + 3 * joff, &s.lat);
    if (rc) return rc;
    s.J = J + 3 * joff;
    s.T = T;
    s.A = n_labels;
    s.Tp = 8 * ((T + 7) / 8);
    s.B = s.Tp * n_labels;
    s.ent = entry0 + (uint32_t)i;
    s.beta.assign(betas + (size_t)i * T, betas + (size_t)(i + 1) * T);
    for (int t = 0; t < T; ++t) {
      if (!(s.beta[(size_t)t] >= 0.0) || !std::isfinite(s.beta[(size_t)t]))
        return fail(PC_EINVAL, "betas must be finite and >= 0");
      if (t > 0 && !(s.beta[(size_t)t] > s.beta[(size_t)t - 1]))
        return fail(PC_EINVAL, "betas must be strictly increasing");
    }
    s.temp_of.resize((size_t)s.B);
    for (int b = 0; b < s.B; ++b) s.temp_of[(size_t)b] = (b % s.Tp < s.T) ? b % s.Tp : 0;
    s.swaps = true;
    joff += (size_t)s.lat.N;
  }
  Batch bt;
  const int icm = n_labels >= 2 ? 1 : 0;
  int rc = build_batch(c, bt, specs, 0);
  if (rc) return rc;
  if ((rc = schedule(c, bt, {}, APT_MODE_APT, icm, 0))) return rc;
  AptArgs a = base_args(c, bt);
  a.tag_init = 1;   // TAG_APT_INIT
  if ((rc = apt_init_launch(a, n_inst, max_words(bt), c->stream))) return rc;
  a.mode = APT_MODE_ENERGY;
  if ((rc = apt_launch(a, bt.n_cta, bt.tpb, bt.smem, c->stream))) return rc;
  for (int done = 0; done < attempts;) {
    const int n = std::min(kChunkAttempts, attempts - done);
    a = base_args(c, bt);
    a.mode = APT_MODE_APT;
    a.n_iter = n;
    a.spp = 1;
    a.icm = icm;
    a.tag_main = 2;   // TAG_APT_SWEEP
    a.tag_ref = 3;    // TAG_APT_REFINE
    if ((rc = apt_launch(a, bt.n_cta, bt.tpb, bt.smem, c->stream))) return rc;
    if ((rc = apt_advance_launch(bt.d_ctr.p, n, n, c->stream))) return rc;
    done += n;
  }
  std::vector<int64_t> st(bt.d_stats.n);
  PC_CUDA_TRY(cudaMemcpyAsync(st.data(), bt.d_stats.p, st.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  att.assign((size_t)n_inst * (T - 1), 0);
  acc.assign((size_t)n_inst * (T - 1), 0);
  for (int i = 0; i < n_inst; ++i) {
    const AptProbDev &P = bt.prob[(size_t)i];
    const int np = (T - 1) * n_labels;
    for (int r = 0; r + 1 < T; ++r)
      for (int l = 0; l < n_labels; ++l) {
        att[(size_t)i * (T - 1) + r] += st[P.stat_off + (size_t)r * n_labels + l];
        acc[(size_t)i * (T - 1) + r] += st[P.stat_off + (size_t)np + (size_t)r * n_labels + l];
      }
  }
  return PC_OK;
}

// Judge of a ladder by its swap-acceptance profile: the pooled acceptance
// acc/att of every pair that the probe attempted must reach acc_floor.
// acc_out [T-1] receives acc/att (-1 for a pair never attempted).
bool judge_pass(const int64_t *att, const int64_t *acc, int T, double acc_floor, double *acc_out) {
  bool pass = true;
  for (int r = 0; r + 1 < T; ++r) {
    if (att[r] <= 0) {
      if (acc_out) acc_out[r] = -1.0;
      continue;
    }
    if (acc_out) acc_out[r] = (double)acc[r] / (double)att[r];
    if ((double)acc[r] < acc_floor * (double)att[r]) pass = false;
  }
  return pass;
}

}  // namespace

extern "C" {

int pc_ladder_judge(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0, int n_temps,
                    const double *betas, int n_labels, int probe_attempts, double acc_floor, double *acc_out,
                    int32_t *pass_out) try {
  if (!c || !dims || !J || !betas || !pass_out) return fail(PC_EINVAL, "NULL argument");
  if (n_inst < 1 || n_temps < 2 || n_temps > 32 || probe_attempts < 1 ||
      !(n_labels == 1 || n_labels == 2 || n_labels == 4) || 8 * ((n_temps + 7) / 8) * n_labels > 128 ||
      !std::isfinite(acc_floor))
    return fail(PC_EINVAL, "bad judge parameters");
  if ((uint64_t)entry0 + (uint64_t)n_inst > (1ull << 24)) return fail(PC_EINVAL, "entry ids must be < 2^24");
  std::vector<int64_t> att, acc;
  int rc = probe_impl(c, n_inst, dims, J, entry0, n_temps, betas, n_labels, probe_attempts, att, acc);
  if (rc) return rc;
  for (int i = 0; i < n_inst; ++i)
    pass_out[i] = judge_pass(att.data() + (size_t)i * (n_temps - 1), acc.data() + (size_t)i * (n_temps - 1),
                             n_temps, acc_floor, acc_out ? acc_out + (size_t)i * (n_temps - 1) : nullptr)
                      ? 1
                      : 0;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_learned_features(pc_ctx *c, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
                        const pc_learned_opts *o, float *X_out) try {
  if (!c || !dims || !J || !o || !o->pilot_betas || !X_out) return fail(PC_EINVAL, "NULL argument");
  int rc = check_pilot_params(n_inst, entry0, kLearnedBetas, o->pilot_betas, o->pilot_chains, o->pilot_sweeps,
                              o->pilot_burn, kLearnedBins);
  if (rc) return rc;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  Batch bt;
  if ((rc = pilot_run(c, bt, n_inst, dims, J, entry0, kLearnedBetas, o->pilot_betas, o->pilot_chains,
                      o->pilot_sweeps, o->pilot_burn, kLearnedBins)))
    return rc;
  constexpr int kIn = 3 + kLearnedBetas * kLearnedBins;
  DevBuf<float> X;
  if ((rc = X.alloc((size_t)n_inst * kIn))) return rc;
  if ((rc = learned_features_launch(bt.d_prob.p, n_inst, bt.d_jneg.p, bt.d_hist.p, kLearnedBetas, kLearnedBins,
                                    X.p, kIn, c->stream)))
    return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(X_out, X.p, (size_t)n_inst * kIn * 4, cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_learned_ladder(pc_ctx *c, pc_mlp *m, int n_inst, const int32_t *dims, const int8_t *J, uint32_t entry0,
                      const pc_learned_opts *o, double *beta_out, double *acc_out, int32_t *fallback_out,
                      double *ready_s) try {
  const auto t_start = std::chrono::steady_clock::now();
  auto seconds = [&]() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  };
  if (!c || !m || !dims || !J || !o || !o->pilot_betas || !beta_out) return fail(PC_EINVAL, "NULL argument");
  if (mlp_context(m) != c) return fail(PC_EINVAL, "the network must belong to this context");
  if (n_inst < 1) return fail(PC_EINVAL, "n_inst must be >= 1");
  int rc = check_pilot_params(n_inst, entry0, kLearnedBetas, o->pilot_betas, o->pilot_chains, o->pilot_sweeps,
                              o->pilot_burn, kLearnedBins);
  if (rc) return rc;
  const bool judge = o->probe_attempts > 0;
  if (judge) {
    if (!(o->probe_labels == 1 || o->probe_labels == 2 || o->probe_labels == 4) || !std::isfinite(o->acc_floor))
      return fail(PC_EINVAL, "bad probe parameters");
    if ((rc = check_ladder_params(o->n_chains, o->sweeps, o->tail, o->max_len, o->beta0, o->alpha))) return rc;
  }
  PC_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  // (1) pilot histograms, (2) features, (3) the network, (4) monotone ladders
  {
    Batch bt;
    if ((rc = pilot_run(c, bt, n_inst, dims, J, entry0, kLearnedBetas, o->pilot_betas, o->pilot_chains,
                        o->pilot_sweeps, o->pilot_burn, kLearnedBins)))
      return rc;
    float *X = nullptr;
    if ((rc = mlp_input(m, n_inst, &X))) return rc;
    if ((rc = learned_features_launch(bt.d_prob.p, n_inst, bt.d_jneg.p, bt.d_hist.p, kLearnedBetas, kLearnedBins,
                                      X, 3 + kLearnedBetas * kLearnedBins, st)))
      return rc;
    const float *bf = nullptr;
    if ((rc = mlp_forward_input(m, n_inst, &bf))) return rc;
    DevBuf<double> d_beta;
    if ((rc = d_beta.alloc((size_t)n_inst * kLearnedLen))) return rc;
    if ((rc = ladder_monotone_launch(n_inst, kLearnedLen, bf, kLadderGap, d_beta.p, st))) return rc;
    PC_CUDA_TRY(cudaMemcpyAsync(beta_out, d_beta.p, (size_t)n_inst * kLearnedLen * 8, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (fallback_out)
    for (int i = 0; i < n_inst; ++i) fallback_out[i] = 0;
  if (!judge) {
    if (acc_out)
      for (size_t k = 0; k < (size_t)n_inst * (kLearnedLen - 1); ++k) acc_out[k] = -1.0;
    if (ready_s)
      for (int i = 0; i < n_inst; ++i) ready_s[i] = seconds();
    return PC_OK;
  }
  // (5) the judge: a short probe of every predicted ladder
  std::vector<int64_t> att, acc;
  if ((rc = probe_impl(c, n_inst, dims, J, entry0, kLearnedLen, beta_out, o->probe_labels, o->probe_attempts, att,
                       acc)))
    return rc;
  std::vector<int> fail_idx;
  for (int i = 0; i < n_inst; ++i) {
    const size_t off = (size_t)i * (kLearnedLen - 1);
    if (!judge_pass(att.data() + off, acc.data() + off, kLearnedLen, o->acc_floor, acc_out ? acc_out + off : nullptr))
      fail_idx.push_back(i);
  }
  const double t_judged = seconds();
  if (ready_s)
    for (int i = 0; i < n_inst; ++i) ready_s[i] = t_judged;
  if (fail_idx.empty()) return PC_OK;
  // (6) fallback: the adaptive procedure for the instances the judge
  // rejected (entry ids unchanged), resampled to the network's length
  std::vector<size_t> joff((size_t)n_inst + 1, 0);
  for (int i = 0; i < n_inst; ++i) joff[(size_t)i + 1] = joff[(size_t)i] + (size_t)dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2];
  const int nf = (int)fail_idx.size();
  std::vector<int32_t> fd;
  std::vector<int8_t> fJ;
  std::vector<uint32_t> fe;
  for (int i : fail_idx) {
    fd.insert(fd.end(), dims + 3 * i, dims + 3 * i + 3);
    fJ.insert(fJ.end(), J + 3 * joff[(size_t)i], J + 3 * joff[(size_t)i + 1]);
    fe.push_back(entry0 + (uint32_t)i);
  }
  std::vector<double> lad((size_t)nf * o->max_len);
  std::vector<int32_t> len((size_t)nf);
  if ((rc = adaptive_impl(c, nf, fd.data(), fJ.data(), fe.data(), o->beta0, o->alpha, o->n_chains, o->sweeps,
                          o->tail, o->tol, o->max_len, lad.data(), nullptr, len.data(), nullptr)))
    return rc;
  for (int k = 0; k < nf; ++k) {
    const int i = fail_idx[(size_t)k];
    if ((rc = pc_resample_ladder(lad.data() + (size_t)k * o->max_len, len[(size_t)k], kLearnedLen,
                                 beta_out + (size_t)i * kLearnedLen)))
      return rc;
    if (fallback_out) fallback_out[i] = 1;
  }
  if (ready_s)
    for (int i : fail_idx) ready_s[i] = seconds();
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

}  // extern "C"
