// Host side of the general-graph entry points: graph checks, DSATUR
// colouring, colour-major renumbering, threshold tables, and the APT batch
// and DT-SQA launches (kernels in graph.cu).
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstring>
#include <set>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "graph_dev.h"
#include "internal.h"

namespace pc {
namespace {

// A graph in colour-major numbering (see graph_dev.h).
struct HGraph {
  int n = 0, C = 0, Imax = 0;
  long long Ebound = 0;          // sum_edges |w| + sum_v |h|
  bool any_h = false;
  std::vector<int> newid;        // original -> new
  std::vector<int> orig;         // new -> original
  std::vector<int32_t> colour;   // original order
  std::vector<int2> vinfo;
  std::vector<uint32_t> adj;
  int off[kGMaxColours + 1] = {};
};

// Symmetric CSR with nonzero int8 weights, no self-loops, no repeats.
int check_graph(int n, const int32_t *rp, const int32_t *col, const int8_t *w) {
  if (n < 1 || n > (1 << 20)) return fail(PC_EINVAL, "graph: need 1 <= n <= 2^20 vertices");
  if (!rp || !col) return fail(PC_EINVAL, "graph: row_ptr / col is NULL");
  if (rp[0] != 0) return fail(PC_EINVAL, "graph: row_ptr[0] must be 0");
  for (int v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) return fail(PC_EINVAL, "graph: row_ptr must not decrease");
  std::vector<std::vector<std::pair<int, int>>> nb(n);
  for (int v = 0; v < n; ++v) {
    if (rp[v + 1] - rp[v] > kGMaxDeg) return fail(PC_EINVAL, "graph: degree above 1023");
    for (int q = rp[v]; q < rp[v + 1]; ++q) {
      const int u = col[q];
      if (u < 0 || u >= n || u == v) return fail(PC_EINVAL, "graph: neighbour out of range or self-loop");
      if (w && w[q] == 0) return fail(PC_EINVAL, "graph: zero weight");
      nb[v].push_back({u, w ? (int)w[q] : 0});
    }
    std::sort(nb[v].begin(), nb[v].end());
    for (size_t i = 1; i < nb[v].size(); ++i)
      if (nb[v][i].first == nb[v][i - 1].first) return fail(PC_EINVAL, "graph: repeated neighbour");
  }
  for (int v = 0; v < n; ++v)
    for (const auto &e : nb[v]) {
      const auto &L = nb[e.first];
      auto it = std::lower_bound(L.begin(), L.end(), std::make_pair(v, INT_MIN));
      if (it == L.end() || it->first != v) return fail(PC_EINVAL, "graph: edge listed in one direction only");
      if (it->second != e.second) return fail(PC_EINVAL, "graph: weights differ between directions");
    }
  return PC_OK;
}

// DSATUR with the tie rule of pc_graph_dsatur (ordered set of
// (-saturation, -uncoloured degree, v)).
int dsatur(int n, const int32_t *rp, const int32_t *col, std::vector<int32_t> &colour, int &C) {
  colour.assign(n, -1);
  std::vector<int> sat(n, 0), udeg(n);
  std::vector<uint32_t> seen(n, 0u);   // colours among coloured neighbours (< 32)
  std::set<std::tuple<int, int, int>> Q;
  for (int v = 0; v < n; ++v) {
    udeg[v] = rp[v + 1] - rp[v];
    Q.insert(std::make_tuple(0, -udeg[v], v));
  }
  C = 0;
  while (!Q.empty()) {
    const int v = std::get<2>(*Q.begin());
    Q.erase(Q.begin());
    const uint32_t freec = ~seen[v];
    if (!freec) return fail(PC_EINVAL, "graph: DSATUR needs more than 32 colours");
    const int c = __builtin_ctz(freec);
    colour[v] = c;
    C = std::max(C, c + 1);
    for (int q = rp[v]; q < rp[v + 1]; ++q) {
      const int u = col[q];
      if (colour[u] >= 0) continue;
      Q.erase(std::make_tuple(-sat[u], -udeg[u], u));
      --udeg[u];
      if (!((seen[u] >> c) & 1u)) {
        seen[u] |= 1u << c;
        ++sat[u];
      }
      Q.insert(std::make_tuple(-sat[u], -udeg[u], u));
    }
  }
  return PC_OK;
}

// Checks, colours (given or DSATUR) and renumbers one graph; adjacency
// entries carry the byte offset word_bytes * u of neighbour u's spin words.
int build_graph(int n, const int32_t *rp, const int32_t *col, const int8_t *w, const int8_t *h,
                const int32_t *colour, int word_bytes, HGraph &g) {
  int rc = check_graph(n, rp, col, w);
  if (rc) return rc;
  if (!w) return fail(PC_EINVAL, "graph: weights are NULL");
  g.n = n;
  if (colour) {
    g.colour.assign(colour, colour + n);
    g.C = 0;
    for (int v = 0; v < n; ++v) {
      if (colour[v] < 0 || colour[v] >= kGMaxColours)
        return fail(PC_EINVAL, "colour: values must lie in 0..31");
      g.C = std::max(g.C, colour[v] + 1);
      for (int q = rp[v]; q < rp[v + 1]; ++q)
        if (colour[col[q]] == colour[v]) return fail(PC_EINVAL, "colour: neighbours share a colour");
    }
  } else if ((rc = dsatur(n, rp, col, g.colour, g.C))) {
    return rc;
  }
  int cnt[kGMaxColours] = {};
  for (int v = 0; v < n; ++v) cnt[g.colour[v]]++;
  g.off[0] = 0;
  for (int c = 0; c < kGMaxColours; ++c) g.off[c + 1] = g.off[c] + cnt[c];
  g.newid.assign(n, 0);
  g.orig.assign(n, 0);
  int fill[kGMaxColours];
  for (int c = 0; c < kGMaxColours; ++c) fill[c] = g.off[c];
  for (int v = 0; v < n; ++v) {
    const int p = fill[g.colour[v]]++;
    g.newid[v] = p;
    g.orig[p] = v;
  }
  g.vinfo.assign(n, make_int2(0, 0));
  g.adj.clear();
  g.Imax = 0;
  g.Ebound = 0;
  g.any_h = false;
  std::vector<std::pair<int, int>> row;
  for (int p = 0; p < n; ++p) {
    const int v = g.orig[p];
    row.clear();
    long long bound = h ? std::abs((int)h[v]) : 0;
    for (int q = rp[v]; q < rp[v + 1]; ++q) {
      row.push_back({g.newid[col[q]], (int)w[q]});
      bound += std::abs((int)w[q]);
      if (col[q] > v) g.Ebound += std::abs((int)w[q]);
    }
    if (h) {
      g.Ebound += std::abs((int)h[v]);
      g.any_h |= h[v] != 0;
    }
    if (bound > kGMaxImax) return fail(PC_EINVAL, "graph: |h_v| + sum |w| exceeds 127");
    g.Imax = std::max(g.Imax, (int)bound);
    std::sort(row.begin(), row.end());
    const int lowest = g.off[g.colour[v]];
    int kl = 0;
    for (const auto &e : row) kl += e.first < lowest;
    const int hv = h ? (int)h[v] : 0;
    g.vinfo[p] = make_int2((int)g.adj.size(),
                           (int)((uint32_t)row.size() | ((uint32_t)kl << 10) | (((uint32_t)hv & 0xFFu) << 20)));
    for (const auto &e : row)
      g.adj.push_back(((uint32_t)(word_bytes * e.first) << 8) | ((uint32_t)e.second & 0xFFu));
  }
  return PC_OK;
}

template <typename T>
int upload(DevBuf<T> &d, const std::vector<T> &h, cudaStream_t st) {
  int rc = d.alloc(h.size());
  if (rc) return rc;
  if (!h.empty()) PC_CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return PC_OK;
}

struct GImpl {
  int n_prob = 0, A = 0, Imax = 0;   // Imax: largest field bound of the batch
  bool any_h = false;
  std::vector<HGraph> g;
  std::vector<int> T;
  std::vector<GProbDev> hp;
  DevBuf<GProbDev> d_prob;
  DevBuf<int2> d_vinfo;
  DevBuf<uint32_t> d_adj, d_pbit, d_swaptab, d_swapidx, d_spins, d_best_bits;
  DevBuf<int32_t> d_E;
  DevBuf<long long> d_best, d_target;
  DevBuf<unsigned long long> d_stats;
  size_t smem = 0, smem_staged = 0;
  bool staged = false;
  int64_t sweeps = 0, swaps = 0;
  int joint = 0;
  bool ready = false;
};

GImpl *gimpl(pc_ctx *c) { return static_cast<GImpl *>(c->graph_impl); }

int static_smem_guard(pc_ctx *c, size_t smem) {
  // the kernels' static shared memory is below 8 KB
  if (smem + 8192 > (size_t)c->smem_optin)
    return fail(PC_EINVAL, "graph problem too large for shared memory (" + std::to_string(smem) +
                               " bytes of state)");
  return PC_OK;
}

int gimpl_ready(pc_ctx *c, int prob) {
  if (!c) return fail(PC_EINVAL, "ctx is NULL");
  GImpl *im = gimpl(c);
  if (!im || !im->ready) return fail(PC_ESTATE, "no graph batch loaded (pc_gapt_load)");
  if (prob < 0 || prob >= im->n_prob) return fail(PC_EINVAL, "problem index out of range");
  return PC_OK;
}

GAptArgs make_args(pc_ctx *c, GImpl *im) {
  GAptArgs a{};
  a.prob = im->d_prob.p;
  a.vinfo = im->d_vinfo.p;
  a.adj = im->d_adj.p;
  a.pbit = im->d_pbit.p;
  a.swaptab = im->d_swaptab.p;
  a.swapidx = im->d_swapidx.p;
  a.spins = im->d_spins.p;
  a.E = im->d_E.p;
  a.best_bits = im->d_best_bits.p;
  a.best = im->d_best.p;
  a.target = im->d_target.p;
  a.stats = im->d_stats.p;
  a.k0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
  a.k1 = (uint32_t)(c->seed >> 32);
  a.joint = im->joint;
  a.tag_init = kTagGInit;
  a.tag_sweep = kTagGSweep;
  a.tag_refine = kTagGRefine;
  return a;
}

}  // namespace
}  // namespace pc

using namespace pc;

void pc_graph_release_impl(pc_ctx *c) try {
  delete gimpl(c);
  c->graph_impl = nullptr;
} catch (...) {
}

extern "C" {

int pc_graph_dsatur(int n, const int32_t *row_ptr, const int32_t *col, int32_t *colour,
                    int *n_colours) try {
  if (!colour) return fail(PC_EINVAL, "colour is NULL");
  int rc = check_graph(n, row_ptr, col, nullptr);
  if (rc) return rc;
  std::vector<int32_t> cl;
  int C = 0;
  if ((rc = dsatur(n, row_ptr, col, cl, C))) return rc;
  std::memcpy(colour, cl.data(), sizeof(int32_t) * n);
  if (n_colours) *n_colours = C;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

}  // extern "C"

namespace pc {
namespace {

// Builds a graph batch into im and draws its initial states with tag_init.
int gload(pc_ctx *c, GImpl *im, int n_prob, const int32_t *n_vert, const int32_t *row_ptr,
          const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
          const int32_t *n_temps, const double *betas, int n_labels, uint32_t entry0,
          uint32_t tag_init) {
  im->n_prob = n_prob;
  im->A = n_labels;
  im->g.resize(n_prob);
  im->T.resize(n_prob);
  std::vector<int2> vinfo;
  std::vector<uint32_t> adj, pbit, swaptab, swapidx;
  std::vector<unsigned long long> stats;
  size_t voff = 0, eoff = 0, roff = 0, boff = 0, bestw = 0;
  int rc;
  for (int i = 0; i < n_prob; ++i) {
    const int n = n_vert[i];
    HGraph &g = im->g[i];
    if (n < 1) return fail(PC_EINVAL, "n_vert must be >= 1");
    const int32_t *rpi = row_ptr + roff;
    if ((rc = build_graph(n, rpi, col + eoff, w + eoff, h ? h + voff : nullptr,
                          colour ? colour + voff : nullptr, 4 * n_labels, g)))
      return rc;
    // the kernel addresses spin words by their byte offset from the dynamic
    // shared-memory base, where they follow the [2 Imax + 1][32] p-bit table
    for (auto &e : g.adj) e += (uint32_t)(4 * (2 * g.Imax + 1) * 32) << 8;
    const int T = n_temps[i];
    if (T < 1 || T > 32) return fail(PC_EINVAL, "n_temps must lie in 1..32");
    const double *beta = betas + boff;
    for (int t = 1; t < T; ++t)
      if (!(beta[t] > beta[t - 1])) return fail(PC_EINVAL, "betas must increase strictly");
    im->T[i] = T;
    im->any_h |= g.any_h;
    im->Imax = std::max(im->Imax, g.Imax);
    GProbDev P{};
    P.n = n;
    P.C = g.C;
    P.T = T;
    P.A = n_labels;
    P.Imax = g.Imax;
    P.m = (int)g.adj.size();
    P.ent = entry0 + (uint32_t)i;
    P.vbase = (uint32_t)vinfo.size();
    P.abase = (uint32_t)adj.size();
    P.thbase = (uint32_t)pbit.size();
    P.swbase = (uint32_t)swapidx.size();
    P.bestbase = (uint32_t)bestw;
    P.statbase = (uint32_t)stats.size();
    for (int cc = 0; cc <= kGMaxColours; ++cc) P.off[cc] = g.off[cc];
    vinfo.insert(vinfo.end(), g.vinfo.begin(), g.vinfo.end());
    adj.insert(adj.end(), g.adj.begin(), g.adj.end());
    for (int r = 0; r < 32; ++r)
      for (int I = -g.Imax; I <= g.Imax; ++I) pbit.push_back(r < T ? pc_pbit_threshold(beta[r], I) : 0u);
    for (int r = 0; r + 1 < T; ++r) {
      const uint32_t o = (uint32_t)swaptab.size();
      const double db = beta[r + 1] - beta[r];
      swaptab.push_back(0xFFFFFFFFu);   // dE = 0
      // |dE| <= 2 Ebound per label; the joint rule sums the labels
      const long long cap = 2 * g.Ebound * n_labels;
      for (long long d = 1; d <= cap; ++d) {
        const uint32_t th = pc_swap_threshold(db, -d);
        if (th == 0u) break;
        swaptab.push_back(th);
      }
      swapidx.push_back(o);
      swapidx.push_back((uint32_t)swaptab.size() - o);
    }
    if (T == 1) swapidx.push_back(0u), swapidx.push_back(0u);
    stats.resize(stats.size() + 2 * (size_t)(T > 1 ? T - 1 : 0) * n_labels + 3, 0ull);
    bestw += (size_t)(n + 31) / 32;
    im->smem = std::max(im->smem, gapt_smem_bytes(n, n_labels, g.Imax, -1));
    im->smem_staged = std::max(im->smem_staged, gapt_smem_bytes(n, n_labels, g.Imax, (int)g.adj.size()));
    im->hp.push_back(P);
    voff += (size_t)n;
    eoff += (size_t)rpi[n];
    roff += (size_t)n + 1;
    boff += (size_t)T;
  }
  if ((rc = static_smem_guard(c, im->smem))) return rc;
  // stage vertex tables and adjacency in shared memory when the largest problem allows
  im->staged = im->smem_staged + 8192 <= (size_t)c->smem_optin;
  if (im->staged) im->smem = im->smem_staged;
  if (swaptab.empty()) swaptab.push_back(0u);
  if (adj.empty()) adj.push_back(0u);
  cudaStream_t st = c->stream;
  std::vector<long long> best(4 * (size_t)n_prob), target((size_t)n_prob, LLONG_MIN);
  for (int i = 0; i < n_prob; ++i) {
    best[4 * i] = LLONG_MAX;
    best[4 * i + 1] = -1;
    best[4 * i + 2] = -1;
    best[4 * i + 3] = -1;
  }
  if ((rc = upload(im->d_prob, im->hp, st)) || (rc = upload(im->d_vinfo, vinfo, st)) ||
      (rc = upload(im->d_adj, adj, st)) || (rc = upload(im->d_pbit, pbit, st)) ||
      (rc = upload(im->d_swaptab, swaptab, st)) || (rc = upload(im->d_swapidx, swapidx, st)) ||
      (rc = upload(im->d_stats, stats, st)) || (rc = upload(im->d_best, best, st)) ||
      (rc = upload(im->d_target, target, st)) ||
      (rc = im->d_spins.alloc(vinfo.size() * n_labels)) || (rc = im->d_best_bits.alloc(bestw)) ||
      (rc = im->d_E.alloc(128 * (size_t)n_prob)) || (rc = im->d_best_bits.zero(st)))
    return rc;
  GAptArgs a = make_args(c, im);
  a.tag_init = tag_init;
  if ((rc = gapt_launch(a, n_prob, n_labels, im->Imax, im->staged, im->smem, true, st))) return rc;
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  im->ready = true;
  return PC_OK;
}

}  // namespace
}  // namespace pc

extern "C" int pc_gapt_load(pc_ctx *c, int n_prob, const int32_t *n_vert, const int32_t *row_ptr,
                            const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
                            const int32_t *n_temps, const double *betas, int n_labels, uint32_t entry0) try {
  if (!c) return fail(PC_EINVAL, "ctx is NULL");
  if (n_prob < 1 || !n_vert || !row_ptr || !col || !w || !n_temps || !betas)
    return fail(PC_EINVAL, "pc_gapt_load: n_prob >= 1 and non-NULL arrays required");
  if (!(n_labels == 1 || n_labels == 2 || n_labels == 4))
    return fail(PC_EINVAL, "n_labels must be 1, 2 or 4");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  pc_graph_release_impl(c);
  GImpl *im = new GImpl();
  c->graph_impl = im;
  return gload(c, im, n_prob, n_vert, row_ptr, col, w, h, colour, n_temps, betas, n_labels, entry0,
               kTagGInit);
} catch (...) {
  return pc::fail_exception();
}

extern "C" {

int pc_gapt_run(pc_ctx *c, int64_t n_swaps, int sweeps_per_swap, int icm) try {
  int rc = gimpl_ready(c, 0);
  if (rc) return rc;
  GImpl *im = gimpl(c);
  if (n_swaps < 0 || sweeps_per_swap < 1) return fail(PC_EINVAL, "n_swaps >= 0, sweeps_per_swap >= 1");
  if (icm && im->A < 2) return fail(PC_EINVAL, "ICM needs n_labels 2 or 4");
  if (icm && im->any_h) return fail(PC_EINVAL, "ICM's whole-replica flip needs h = 0");
  if (im->sweeps + n_swaps * sweeps_per_swap > 0xFFFFFFFFll || im->swaps + n_swaps > 0xFFFFFFFFll)
    return fail(PC_EINVAL, "sweep counter would pass 2^32");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  GAptArgs a = make_args(c, im);
  a.spp = sweeps_per_swap;
  a.icm = icm ? 1 : 0;
  int64_t left = n_swaps;
  while (left > 0) {
    const int chunk = (int)std::min<int64_t>(left, 256);
    a.n_swaps = chunk;
    a.sweep0 = (uint32_t)im->sweeps;
    a.swap0 = (uint32_t)im->swaps;
    if ((rc = gapt_launch(a, im->n_prob, im->A, im->Imax, im->staged, im->smem, false, c->stream))) return rc;
    im->sweeps += (int64_t)chunk * sweeps_per_swap;
    im->swaps += chunk;
    left -= chunk;
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_set_joint_swap(pc_ctx *c, int joint) try {
  int rc = gimpl_ready(c, 0);
  if (rc) return rc;
  gimpl(c)->joint = joint != 0;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_set_target(pc_ctx *c, int prob, int64_t e_target) try {
  int rc = gimpl_ready(c, prob);
  if (rc) return rc;
  GImpl *im = gimpl(c);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  long long b[4];
  PC_CUDA_TRY(cudaMemcpyAsync(b, im->d_best.p + 4 * (size_t)prob, sizeof(b), cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  b[3] = (b[0] <= e_target) ? b[1] : -1;
  long long t = e_target;
  PC_CUDA_TRY(cudaMemcpyAsync(im->d_best.p + 4 * (size_t)prob, b, sizeof(b), cudaMemcpyHostToDevice, c->stream));
  PC_CUDA_TRY(cudaMemcpyAsync(im->d_target.p + prob, &t, sizeof(t), cudaMemcpyHostToDevice, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_get_energies(pc_ctx *c, int prob, int64_t *E) try {
  int rc = gimpl_ready(c, prob);
  if (rc) return rc;
  if (!E) return fail(PC_EINVAL, "E is NULL");
  GImpl *im = gimpl(c);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  int32_t e[128];
  PC_CUDA_TRY(cudaMemcpyAsync(e, im->d_E.p + 128 * (size_t)prob, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int T = im->T[prob], A = im->A;
  for (int r = 0; r < T; ++r)
    for (int a = 0; a < A; ++a) E[r * A + a] = e[32 * a + r];
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_get_spins(pc_ctx *c, int prob, int8_t *spins) try {
  int rc = gimpl_ready(c, prob);
  if (rc) return rc;
  if (!spins) return fail(PC_EINVAL, "spins is NULL");
  GImpl *im = gimpl(c);
  const HGraph &g = im->g[prob];
  const int A = im->A, T = im->T[prob], n = g.n;
  std::vector<uint32_t> wd((size_t)n * A);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaMemcpyAsync(wd.data(), im->d_spins.p + (size_t)im->hp[prob].vbase * A,
                              wd.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int r = 0; r < T; ++r)
    for (int a = 0; a < A; ++a)
      for (int v = 0; v < n; ++v)
        spins[((size_t)r * A + a) * n + v] = ((wd[(size_t)g.newid[v] * A + a] >> r) & 1u) ? 1 : -1;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_get_colours(pc_ctx *c, int prob, int32_t *colour) try {
  int rc = gimpl_ready(c, prob);
  if (rc) return rc;
  if (!colour) return fail(PC_EINVAL, "colour is NULL");
  const HGraph &g = gimpl(c)->g[prob];
  std::memcpy(colour, g.colour.data(), sizeof(int32_t) * g.n);
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_get_best(pc_ctx *c, int prob, int64_t *E, int64_t *sweep, int32_t *slot,
                     int64_t *hit_sweep, int8_t *spins) try {
  int rc = gimpl_ready(c, prob);
  if (rc) return rc;
  GImpl *im = gimpl(c);
  const HGraph &g = im->g[prob];
  long long b[4];
  std::vector<uint32_t> bits((size_t)(g.n + 31) / 32);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaMemcpyAsync(b, im->d_best.p + 4 * (size_t)prob, sizeof(b), cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaMemcpyAsync(bits.data(), im->d_best_bits.p + im->hp[prob].bestbase, bits.size() * 4,
                              cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (E) *E = b[0];
  if (sweep) *sweep = b[1];
  if (slot) *slot = (int32_t)b[2];
  if (hit_sweep) *hit_sweep = b[3];
  if (spins) {
    for (int v = 0; v < g.n; ++v) {
      const int p = g.newid[v];
      spins[v] = b[1] < 0 ? 0 : (((bits[p >> 5] >> (p & 31)) & 1u) ? 1 : -1);
    }
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gapt_get_stats(pc_ctx *c, int prob, int64_t *att, int64_t *acc, int64_t *icm) try {
  int rc = gimpl_ready(c, prob);
  if (rc) return rc;
  GImpl *im = gimpl(c);
  const int np = (im->T[prob] > 1 ? im->T[prob] - 1 : 0) * im->A;
  std::vector<unsigned long long> s((size_t)2 * np + 3);
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaMemcpyAsync(s.data(), im->d_stats.p + im->hp[prob].statbase, s.size() * 8,
                              cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < np; ++i) {
    if (att) att[i] = (int64_t)s[i];
    if (acc) acc[i] = (int64_t)s[np + i];
  }
  if (icm)
    for (int i = 0; i < 3; ++i) icm[i] = (int64_t)s[2 * np + i];
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_gsqa_anneal(pc_ctx *c, int n, const int32_t *row_ptr, const int32_t *col, const int8_t *w,
                   const int8_t *h, const int32_t *colour, int P, double T, int n_sweeps,
                   const double *gamma, int R, uint32_t run0, int64_t *E_out, int8_t *spins_out) try {
  if (!c) return fail(PC_EINVAL, "ctx is NULL");
  if (P < 2 || P > 2047 || !(T > 0) || n_sweeps < 0 || R < 1 || !E_out || (n_sweeps > 0 && !gamma))
    return fail(PC_EINVAL, "pc_gsqa_anneal: P in 2..2047, T > 0, R >= 1, gamma and E_out required");
  for (int s = 0; s < n_sweeps; ++s)
    if (!(gamma[s] > 0)) return fail(PC_EINVAL, "gamma must be > 0");
  // a word holds 32 runs and one Philox call serves 8 of them
  if (run0 % 8 != 0) return fail(PC_EINVAL, "run0 must be a multiple of 8");
  if ((uint64_t)run0 + (uint64_t)R + 32 > (1ull << 27)) return fail(PC_EINVAL, "run ids must stay below 2^27");
  HGraph g;
  int rc = build_graph(n, row_ptr, col, w, h, colour, 4, g);
  if (rc) return rc;
  // the slices of a run group go to a cluster of CS CTAs when one CTA cannot
  // hold them; the graph itself is staged in shared memory when it still fits
  const size_t budget = (size_t)c->smem_optin - 8192;
  int CS = 1;
  bool staged = true;
  auto fits = [&](int cs, bool st_) {
    return gsqa_smem_bytes(n, P, g.Imax, st_ ? (int)g.adj.size() : -1, cs) <= budget;
  };
  while (!fits(CS, true) && CS < 8 && 2 * CS <= P) CS *= 2;
  if (!fits(CS, true)) {
    staged = false;
    CS = 1;
    while (!fits(CS, false) && CS < 8 && 2 * CS <= P) CS *= 2;
  }
  const size_t smem = gsqa_smem_bytes(n, P, g.Imax, staged ? (int)g.adj.size() : -1, CS);
  if ((rc = static_smem_guard(c, smem))) return rc;
  // colour classes of the replicated network, each ordered by slice, then vertex
  const int Cp = std::max(g.C, (P & 1) ? 3 : 2);
  std::vector<uint32_t> cls;
  std::vector<int> cls_off(Cp + 1, 0);
  for (int cp = 0; cp < Cp; ++cp) {
    cls_off[cp] = (int)cls.size();
    for (int k = 0; k < P; ++k) {
      const int f = ((P & 1) && k == P - 1) ? 2 : (k & 1);
      const int base = ((cp - f) % Cp + Cp) % Cp;
      if (base >= g.C) continue;
      for (int p = g.off[base]; p < g.off[base + 1]; ++p) cls.push_back(((uint32_t)k << 20) | (uint32_t)p);
    }
  }
  cls_off[Cp] = (int)cls.size();
  // per class, the list offsets where each cluster rank's slices begin
  std::vector<int> cls_rank((size_t)Cp * (CS + 1), 0);
  for (int cp = 0; cp < Cp; ++cp)
    for (int r = 0; r <= CS; ++r) {
      const int kfirst = r * P / CS;
      int o = cls_off[cp];
      while (o < cls_off[cp + 1] && (int)(cls[o] >> 20) < kfirst) ++o;
      cls_rank[(size_t)cp * (CS + 1) + r] = o - cls_off[cp];
    }
  const int nt = 2 * g.Imax + 1;
  std::vector<uint32_t> table((size_t)std::max(n_sweeps, 1) * 3 * nt);
  const double beta_eff = 1.0 / ((double)P * T);
  for (int s = 0; s < n_sweeps; ++s) {
    const int32_t jq = pc_jperp_q(gamma[s], P, T);
    for (int nup = 0; nup < 3; ++nup)
      for (int I = -g.Imax; I <= g.Imax; ++I)
        table[((size_t)s * 3 + nup) * nt + (I + g.Imax)] = sqa_threshold(beta_eff, I, jq, 2 * nup - 2);
  }
  PC_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  DevBuf<int2> d_vinfo;
  DevBuf<uint32_t> d_adj, d_cls, d_table, d_spins;
  DevBuf<int> d_off, d_rank;
  DevBuf<long long> d_E;
  std::vector<uint32_t> adj = g.adj;
  if (adj.empty()) adj.push_back(0u);
  const int groups = (R + 31) / 32;
  if ((rc = upload(d_vinfo, g.vinfo, st)) || (rc = upload(d_adj, adj, st)) || (rc = upload(d_cls, cls, st)) ||
      (rc = upload(d_off, cls_off, st)) || (rc = upload(d_table, table, st)) ||
      (rc = upload(d_rank, cls_rank, st)) ||
      (rc = d_E.alloc((size_t)R * P)) || (rc = d_E.zero(st)))
    return rc;
  if (spins_out && (rc = d_spins.alloc((size_t)groups * P * n))) return rc;
  GSqaArgs a{};
  a.n = n;
  a.P = P;
  a.Cp = Cp;
  a.S = n_sweeps;
  a.Imax = g.Imax;
  a.R = R;
  a.m = (int)g.adj.size();
  a.run0 = run0;
  a.k0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
  a.k1 = (uint32_t)(c->seed >> 32);
  a.vinfo = d_vinfo.p;
  a.adj = d_adj.p;
  a.cls = d_cls.p;
  a.cls_off = d_off.p;
  a.table = d_table.p;
  a.E = d_E.p;
  a.spins = spins_out ? d_spins.p : nullptr;
  a.CS = CS;
  a.cls_rank = d_rank.p;
  if ((rc = gsqa_launch(a, staged, smem, st))) return rc;
  std::vector<long long> E((size_t)R * P);
  PC_CUDA_TRY(cudaMemcpyAsync(E.data(), d_E.p, E.size() * 8, cudaMemcpyDeviceToHost, st));
  std::vector<uint32_t> wd;
  if (spins_out) {
    wd.resize((size_t)groups * P * n);
    PC_CUDA_TRY(cudaMemcpyAsync(wd.data(), d_spins.p, wd.size() * 4, cudaMemcpyDeviceToHost, st));
  }
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  for (size_t i = 0; i < E.size(); ++i) E_out[i] = (int64_t)E[i];
  if (spins_out)
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < P; ++k)
        for (int v = 0; v < n; ++v)
          spins_out[((size_t)r * P + k) * n + v] =
              ((wd[((size_t)(r >> 5) * P + k) * n + g.newid[v]] >> (r & 31)) & 1u) ? 1 : -1;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_graph_adaptive_ladder(pc_ctx *c, int n_prob, const int32_t *n_vert, const int32_t *row_ptr,
                             const int32_t *col, const int8_t *w, const int8_t *h, const int32_t *colour,
                             uint32_t entry0, double beta0, double alpha, int n_chains, int sweeps,
                             int tail, double tol, int max_len, double *beta_out, double *sigma_out,
                             int32_t *len_out, int32_t *converged_out) try {
  if (!c || !beta_out || !len_out) return fail(PC_EINVAL, "NULL argument");
  if (n_prob < 1 || n_chains < 1 || n_chains > 128 || sweeps < 1 || tail < 2 || tail > sweeps ||
      max_len < 1 || !(beta0 > 0.0) || !(alpha > 0.0))
    return fail(PC_EINVAL, "bad ladder parameters (1 <= n_chains <= 128, 2 <= tail <= sweeps)");
  if ((int64_t)sweeps * max_len > 0xFFFFFFFFll) return fail(PC_EINVAL, "sweep counter would exceed 2^32");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  const int A = n_chains <= 32 ? 1 : (n_chains <= 64 ? 2 : 4);
  // the batch is built as 32 "temperatures" per label; every row of the
  // p-bit table is rewritten with the problem's current beta at each step
  std::vector<int32_t> nt((size_t)n_prob, 32);
  std::vector<double> dummy;
  for (int i = 0; i < n_prob; ++i)
    for (int r = 0; r < 32; ++r) dummy.push_back(1.0 + r);
  GImpl im;
  int rc = gload(c, &im, n_prob, n_vert, row_ptr, col, w, h, colour, nt.data(), dummy.data(), A, entry0,
                 kTagGLInit);
  if (rc) return rc;
  for (int i = 0; i < n_prob; ++i) {
    const long long eb = im.g[(size_t)i].Ebound;
    if ((double)tail * (double)eb * (double)eb > 4.0e18) return fail(PC_EINVAL, "tail too long for exact int64 sums");
  }
  DevBuf<long long> d_s1, d_s2;
  DevBuf<int> d_active;
  if ((rc = d_s1.alloc(128 * (size_t)n_prob)) || (rc = d_s2.alloc(128 * (size_t)n_prob)) ||
      (rc = d_active.alloc((size_t)n_prob)))
    return rc;
  cudaStream_t st = c->stream;
  std::vector<double> beta((size_t)n_prob, beta0);
  std::vector<int> active((size_t)n_prob, 1), len((size_t)n_prob, 0), conv((size_t)n_prob, 0);
  std::vector<uint32_t> pbit(im.d_pbit.n, 0u);
  std::vector<long long> s1(128 * (size_t)n_prob), s2(128 * (size_t)n_prob);
  for (int step = 0; step < max_len; ++step) {
    for (int i = 0; i < n_prob; ++i) {
      const int Imax = im.g[(size_t)i].Imax, nt2 = 2 * Imax + 1;
      uint32_t *row = pbit.data() + im.hp[(size_t)i].thbase;
      for (int I = -Imax; I <= Imax; ++I) row[I + Imax] = pc_pbit_threshold(beta[(size_t)i], I);
      for (int r = 1; r < 32; ++r) std::memcpy(row + (size_t)r * nt2, row, sizeof(uint32_t) * nt2);
    }
    PC_CUDA_TRY(cudaMemcpyAsync(im.d_pbit.p, pbit.data(), pbit.size() * 4, cudaMemcpyHostToDevice, st));
    PC_CUDA_TRY(cudaMemcpyAsync(d_active.p, active.data(), active.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if ((rc = d_s1.zero(st)) || (rc = d_s2.zero(st))) return rc;
    GAptArgs a = make_args(c, &im);
    a.tag_sweep = kTagGLSweep;
    a.tag_refine = kTagGLRefine;
    a.ladder = 1;
    a.window_from = sweeps - tail;
    a.sum1 = d_s1.p;
    a.sum2 = d_s2.p;
    a.active = d_active.p;
    a.spp = 1;
    a.n_swaps = sweeps;
    a.sweep0 = (uint32_t)((int64_t)step * sweeps);
    if ((rc = gapt_launch(a, n_prob, A, im.Imax, im.staged, im.smem, false, st))) return rc;
    PC_CUDA_TRY(cudaMemcpyAsync(s1.data(), d_s1.p, s1.size() * 8, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaMemcpyAsync(s2.data(), d_s2.p, s2.size() * 8, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    int left = 0;
    for (int i = 0; i < n_prob; ++i) {
      if (!active[(size_t)i]) continue;
      // sigma_E: square root of the chains' mean unbiased variance (chain b = slot 32 a + r)
      double mean_var = 0.0;
      for (int b = 0; b < n_chains; ++b) {
        const long long q1 = s1[128 * (size_t)i + b], q2 = s2[128 * (size_t)i + b];
        const long long num = (long long)tail * q2 - q1 * q1;
        mean_var += (double)num / ((double)tail * (double)(tail - 1));
      }
      mean_var /= (double)n_chains;
      const double sigma = std::sqrt(mean_var);
      beta_out[(size_t)i * max_len + len[(size_t)i]] = beta[(size_t)i];
      if (sigma_out) sigma_out[(size_t)i * max_len + len[(size_t)i]] = sigma;
      ++len[(size_t)i];
      if (sigma < tol) {
        conv[(size_t)i] = 1;
        active[(size_t)i] = 0;
      } else {
        beta[(size_t)i] = beta[(size_t)i] + alpha / sigma;
        left += len[(size_t)i] < max_len;
        if (len[(size_t)i] >= max_len) active[(size_t)i] = 0;
      }
    }
    if (!left) break;
  }
  for (int i = 0; i < n_prob; ++i) {
    len_out[i] = len[(size_t)i];
    if (converged_out) converged_out[i] = conv[(size_t)i];
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

}  // extern "C"
