// Device steps of the learned beta ladder that sit around the MLP: the
// network's input features of every instance, read from the pilot batch on
// the device (coupling words and pilot energy histograms), and the
// conversion of the network's fp32 ladders into strictly increasing double
// ladders.  The paper has no learned component; the network stands in for
// the adaptive-ladder preprocessing of Algorithm S2 on the grounds that
// ladders of one size are nearly the same across instances (Fig. S12).
#include <cuda_runtime.h>

#include "apt_dev.h"
#include "internal.h"

namespace {

using pc::AptProbDev;

constexpr int kFeatThreads = 256;

// One CTA per instance.  Instance features (all from the coupling words of
// the periodic lattice, whose bits 0, 2, 4 flag J < 0 on the +x, +y, +z bond
// of a site):
//   x0 = cbrt(N) / 16,
//   x1 = fraction of the 3N bonds with J > 0,
//   x2 = fraction of the 3N elementary plaquettes that are frustrated (an
//        odd number of negative couplings around the square),
// then the pilot histograms, each temperature's counts divided by their
// total (or by 1 when empty).  Integer counts are exact; the divisions are
// taken in double and rounded once to fp32.
__global__ void __launch_bounds__(kFeatThreads) features_kernel(const AptProbDev *prob,
                                                                const uint16_t *jneg,
                                                                const int64_t *hist, int n_beta,
                                                                int n_bins, float *X, int ldx) {
  const AptProbDev P = prob[blockIdx.x];
  const int Lx = P.Lx, Ly = P.Ly, Lz = P.Lz, N = P.N, H = N >> 1;
  const uint16_t *jn = jneg + P.jneg_off;
  // word of lattice site (x, y, z), coordinates taken modulo the lengths
  auto word = [&](int x, int y, int z) -> uint32_t {
    x = x == Lx ? 0 : x;
    y = y == Ly ? 0 : y;
    z = z == Lz ? 0 : z;
    const int lin = x + Lx * (y + Ly * z);
    return jn[((x + y + z) & 1) * H + (lin >> 1)];
  };
  int pos = 0, frust = 0;
  for (int s = threadIdx.x; s < N; s += blockDim.x) {
    const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
    const uint32_t w = word(x, y, z);
    const uint32_t wx = word(x + 1, y, z), wy = word(x, y + 1, z), wz = word(x, y, z + 1);
    // negative flags of the forward bonds: bit 0 (+x), bit 2 (+y), bit 4 (+z)
    pos += 3 - __popc(w & 0x15u);
    // plaquette (a, b) at s: J_a(s) J_b(s + a) J_a(s + b) J_b(s)
    const uint32_t pxy = (w >> 0) ^ (wx >> 2) ^ (wy >> 0) ^ (w >> 2);
    const uint32_t pxz = (w >> 0) ^ (wx >> 4) ^ (wz >> 0) ^ (w >> 4);
    const uint32_t pyz = (w >> 2) ^ (wy >> 4) ^ (wz >> 2) ^ (w >> 4);
    frust += (int)((pxy & 1u) + (pxz & 1u) + (pyz & 1u));
  }
  __shared__ int s_pos[kFeatThreads / 32], s_frust[kFeatThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    pos += __shfl_xor_sync(0xFFFFFFFFu, pos, o);
    frust += __shfl_xor_sync(0xFFFFFFFFu, frust, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_pos[warp] = pos;
    s_frust[warp] = frust;
  }
  __syncthreads();
  float *x = X + (size_t)blockIdx.x * ldx;
  if (threadIdx.x == 0) {
    int tp = 0, tf = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tp += s_pos[w];
      tf += s_frust[w];
    }
    x[0] = (float)(cbrt((double)N) / 16.0);
    x[1] = (float)((double)tp / (3.0 * (double)N));
    x[2] = (float)((double)tf / (3.0 * (double)N));
  }
  // histograms: one warp per temperature, total by warp reduction
  const int64_t *h = hist + P.hist_off;
  for (int t = warp; t < n_beta; t += (int)(blockDim.x >> 5)) {
    long long tot = 0;
    for (int b = lane; b < n_bins; b += 32) tot += h[(size_t)t * n_bins + b];
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    const double d = tot > 0 ? (double)tot : 1.0;
    for (int b = lane; b < n_bins; b += 32) x[3 + t * n_bins + b] = (float)((double)h[(size_t)t * n_bins + b] / d);
  }
}

// One thread per ladder: beta_0 = max(b_0, 0), beta_k = max(b_k,
// beta_{k-1} + gap), so that every ladder is strictly increasing (the
// network's cumulative softplus can stall in fp32 when a term underflows).
__global__ void monotone_kernel(int n, int len, const float *b, double gap, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double prev = 0.0;
  for (int k = 0; k < len; ++k) {
    double v = (double)b[(size_t)i * len + k];
    if (k == 0) {
      v = v > 0.0 ? v : 0.0;
    } else if (!(v >= prev + gap)) {
      v = prev + gap;
    }
    out[(size_t)i * len + k] = v;
    prev = v;
  }
}

}  // namespace

namespace pc {

int learned_features_launch(const AptProbDev *prob, int n_inst, const uint16_t *jneg, const int64_t *hist,
                            int n_beta, int n_bins, float *X, int ldx, cudaStream_t st) {
  if (n_inst <= 0) return PC_OK;
  features_kernel<<<n_inst, kFeatThreads, 0, st>>>(prob, jneg, hist, n_beta, n_bins, X, ldx);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

int ladder_monotone_launch(int n, int len, const float *b, double gap, double *out, cudaStream_t st) {
  if (n <= 0) return PC_OK;
  monotone_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, len, b, gap, out);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

}  // namespace pc
