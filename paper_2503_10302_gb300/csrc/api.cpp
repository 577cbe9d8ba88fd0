// C ABI: context, errors, host-side threshold tables, DT-SQA and the Philox
// check.  The adaptive-parallel-tempering, ladder and MLP entry points live
// in apt_api.cpp and mlp.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"
#include "internal.h"

namespace pc {

static thread_local std::string g_error;

void set_error(const std::string &msg) { g_error = msg; }

int fail(int code, const std::string &msg) {
  g_error = msg;
  return code;
}

int fail_exception() {
  try {
    throw;
  } catch (const std::bad_alloc &) {
    return fail(PC_ENOMEM, "host allocation failed");
  } catch (const std::length_error &) {
    return fail(PC_ENOMEM, "host allocation too large");
  } catch (const std::exception &e) {
    return fail(PC_EINVAL, std::string("unexpected error: ") + e.what());
  } catch (...) {
    return fail(PC_EINVAL, "unexpected error");
  }
}

uint32_t recip32(uint32_t d) {
  // ceil(2^32 / d): exact quotients for n, d < 2^16 through __umulhi; d = 1
  // (no 32-bit reciprocal) maps to 0, which the device divider treats as 1
  if (d <= 1) return 0u;
  return (uint32_t)((((uint64_t)1 << 32) + d - 1) / d);
}

int check_lattice(const int32_t *dims, const int8_t *J, Lattice *out) {
  if (!dims) return fail(PC_EINVAL, "dims is NULL");
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 2 || (dims[a] & 1))
      return fail(PC_EINVAL, "every lattice dimension must be even and >= 2 (periodic)");
    out->L[a] = dims[a];
  }
  out->N = dims[0] * dims[1] * dims[2];
  if (out->N > 4096) return fail(PC_EINVAL, "N = Lx*Ly*Lz must be <= 4096");
  if (J) {
    for (int i = 0; i < 3 * out->N; ++i)
      if (J[i] != 1 && J[i] != -1) return fail(PC_EINVAL, "couplings must be +1 or -1");
  }
  return PC_OK;
}

std::vector<uint8_t> pack_jneg(const Lattice &lat, const int8_t *J) {
  const int Lx = lat.L[0], Ly = lat.L[1], Lz = lat.L[2], N = lat.N;
  std::vector<uint8_t> out((size_t)N);
  for (int s = 0; s < N; ++s) {
    const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
    const int xm = (x + Lx - 1) % Lx + Lx * (y + Ly * z);
    const int ym = x + Lx * ((y + Ly - 1) % Ly + Ly * z);
    const int zm = x + Lx * (y + Ly * ((z + Lz - 1) % Lz));
    const int8_t j[6] = {J[3 * s + 0], J[3 * xm + 0], J[3 * s + 1],
                         J[3 * ym + 1], J[3 * s + 2], J[3 * zm + 2]};
    uint8_t m = 0;
    for (int d = 0; d < 6; ++d)
      if (j[d] < 0) m |= (uint8_t)(1u << d);
    out[(size_t)s] = m;
  }
  return out;
}

std::vector<uint16_t> pack_jn16(const Lattice &lat, const uint8_t per[3], const uint8_t *present,
                                const int8_t *J, int *nbonds, int *nreal) {
  std::vector<uint8_t> signs = pack_jneg(lat, J);
  const int Lx = lat.L[0], Ly = lat.L[1], Lz = lat.L[2];
  std::vector<uint16_t> out((size_t)lat.N);
  int nb = 0, nr = 0;
  for (int s = 0; s < lat.N; ++s) {
    const int x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
    uint16_t miss = 0;   // bit d: direction d (+x, -x, +y, -y, +z, -z) absent
    if (!per[0]) miss |= (uint16_t)((x == 0 ? 2 : 0) | (x == Lx - 1 ? 1 : 0));
    if (!per[1]) miss |= (uint16_t)((y == 0 ? 8 : 0) | (y == Ly - 1 ? 4 : 0));
    if (!per[2]) miss |= (uint16_t)((z == 0 ? 32 : 0) | (z == Lz - 1 ? 16 : 0));
    const bool vac = present && !present[s];
    if (vac) {
      miss = 0x3F;
    } else if (present) {
      const int xp = (x + 1) % Lx + Lx * (y + Ly * z), xm = (x + Lx - 1) % Lx + Lx * (y + Ly * z);
      const int yp = x + Lx * ((y + 1) % Ly + Ly * z), ym = x + Lx * ((y + Ly - 1) % Ly + Ly * z);
      const int zp = x + Lx * (y + Ly * ((z + 1) % Lz)), zm = x + Lx * (y + Ly * ((z + Lz - 1) % Lz));
      const int nbr[6] = {xp, xm, yp, ym, zp, zm};
      for (int d = 0; d < 6; ++d)
        if (!present[nbr[d]]) miss |= (uint16_t)(1u << d);
    }
    for (int d = 0; d < 6; d += 2) nb += ((miss >> d) & 1) ? 0 : 1;   // forward bonds
    nr += vac ? 0 : 1;
    out[(size_t)s] = (uint16_t)(((uint16_t)signs[(size_t)s] & ~miss & 0x3F) | (miss << 8) | (vac ? 0x8000 : 0));
  }
  *nbonds = nb;
  *nreal = nr;
  return out;
}

// floor(2^32 p) clamped to [0, 2^32 - 1].
static uint32_t threshold_of(double p) {
  const double t = std::floor(std::ldexp(p, 32));
  if (!(t > 0.0)) return 0u;
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)t;
}

uint32_t sqa_threshold(double beta_eff, int I, int32_t jq, int n) {
  const double h = (double)I + std::ldexp((double)jq, -16) * (double)n;
  const double p = 1.0 / (1.0 + std::exp(-2.0 * beta_eff * h));
  return threshold_of(p);
}

}  // namespace pc

using namespace pc;

extern "C" {

const char *pc_last_error(void) { return g_error.c_str(); }

uint32_t pc_pbit_threshold(double beta, int I) {
  const double p = 1.0 / (1.0 + std::exp(-2.0 * beta * (double)I));
  return threshold_of(p);
}

uint32_t pc_swap_threshold(double dbeta, int64_t dE) {
  const double p = std::exp(dbeta * (double)dE);
  if (p >= 1.0) return 0xFFFFFFFFu;
  return threshold_of(p);
}

int32_t pc_jperp_q(double gamma, int P, double T) {
  const double pt = (double)P * T;
  const double jp = -0.5 * pt * std::log(std::tanh(gamma / pt));
  return (int32_t)std::llround(jp * 65536.0);
}

int pc_create(pc_ctx **out, int device, uint64_t seed) try {
  if (!out) return fail(PC_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  PC_CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(PC_EINVAL, "no such CUDA device");
  PC_CUDA_TRY(cudaSetDevice(device));
  cudaDeviceProp prop;
  PC_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (prop.major * 10 + prop.minor < 100)
    return fail(PC_EINVAL, "the kernels are built for sm_103a (Blackwell Ultra)");
  pc_ctx *c = new pc_ctx();
  c->device = device;
  c->seed = seed;
  c->sms = prop.multiProcessorCount;
  c->smem_optin = (int)prop.sharedMemPerBlockOptin;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return fail(PC_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
  }
  c->own_stream = true;
  *out = c;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

void pc_destroy(pc_ctx *c) try {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  c->sqa.release();
  pc_apt_release_impl(c);
  pc_graph_release_impl(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
} catch (...) {
}

int pc_set_stream(pc_ctx *c, void *stream) try {
  if (!c) return fail(PC_EINVAL, "ctx is NULL");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->own_stream) cudaStreamDestroy(c->stream);
  c->stream = (cudaStream_t)stream;
  c->own_stream = false;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

static int sqa_check_device(pc_ctx *c);

int pc_synchronize(pc_ctx *c) try {
  if (!c) return fail(PC_EINVAL, "ctx is NULL");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return sqa_check_device(c);
} catch (...) {
  return pc::fail_exception();
}

int pc_device_sm_count(pc_ctx *c, int *sms) try {
  if (!c || !sms) return fail(PC_EINVAL, "NULL argument");
  *sms = c->sms;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_philox(pc_ctx *c, int64_t n, const uint32_t *ctr, uint32_t *out) try {
  if (!c || n < 0 || (n > 0 && (!ctr || !out))) return fail(PC_EINVAL, "bad arguments");
  if (n == 0) return PC_OK;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  DevBuf<uint32_t> dc, dout;
  int rc = dc.alloc((size_t)n * 4);
  if (rc) return rc;
  if ((rc = dout.alloc((size_t)n * 4))) return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(dc.p, ctr, (size_t)n * 16, cudaMemcpyHostToDevice, c->stream));
  if ((rc = philox_launch(dc.p, dout.p, n, (uint32_t)(c->seed & 0xFFFFFFFFu),
                          (uint32_t)(c->seed >> 32), c->stream)))
    return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(out, dout.p, (size_t)n * 16, cudaMemcpyDeviceToHost, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

// ------------------------------------------------------------------ DT-SQA
int pc_sqa_setup(pc_ctx *c, const int32_t *dims, const int8_t *J, int P, double T, int n_sweeps,
                 const double *gamma) try {
  return pc_sqa_setup_bc(c, dims, nullptr, nullptr, J, P, T, n_sweeps, gamma);
} catch (...) {
  return pc::fail_exception();
}

int pc_sqa_setup_bc(pc_ctx *c, const int32_t *dims, const uint8_t *periodic, const uint8_t *present,
                    const int8_t *J, int P, double T, int n_sweeps, const double *gamma) try {
  if (!c || !J || (n_sweeps > 0 && !gamma)) return fail(PC_EINVAL, "NULL argument");
  Lattice lat;
  int rc = check_lattice(dims, J, &lat);
  if (rc) return rc;
  uint8_t per[3];
  for (int ax = 0; ax < 3; ++ax) per[ax] = periodic ? (periodic[ax] != 0) : 1;
  if (P < 16 || P % 16 || P > 128) return fail(PC_EINVAL, "P must be a multiple of 16 in [16, 128]");
  if ((int64_t)lat.N * P > 262144) return fail(PC_EINVAL, "N * P must be <= 262144");
  if (!(T > 0.0) || n_sweeps < 0) return fail(PC_EINVAL, "T must be > 0 and n_sweeps >= 0");
  for (int s = 0; s < n_sweeps; ++s)
    if (!(gamma[s] > 0.0)) return fail(PC_EINVAL, "every Gamma must be > 0");
  if (sqa_smem_bytes(lat.N, P) > (size_t)c->smem_optin)
    return fail(PC_EINVAL, "run does not fit in shared memory");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  SqaState &q = c->sqa;
  // device buffers are kept from the previous setup when they are large
  // enough; the copies below are ordered after any anneal still queued on
  // the context's stream
  q.ready = false;
  q.last_err = nullptr;
  q.lat = lat;
  q.P = P;
  q.T = T;
  q.S = n_sweeps;
  q.jq.resize((size_t)n_sweeps);
  q.table.assign((size_t)(n_sweeps > 0 ? n_sweeps : 1) * kSqaTab, 0u);
  const double beta_eff = 1.0 / ((double)P * T);
  // every sweep's row is independent: long schedules are built by several
  // host threads (the rows do not depend on how they are split)
  auto rows = [&](int s0, int s1) {
    for (int s = s0; s < s1; ++s) {
      const int32_t jq = pc_jperp_q(gamma[s], P, T);
      q.jq[(size_t)s] = jq;
      // every in-slice field I = -6..6 (odd at open faces) and time count m
      for (int m = 0; m < 3; ++m)
        for (int e = 0; e < 13; ++e)
          q.table[(size_t)s * kSqaTab + e + 13 * m] = sqa_threshold(beta_eff, e - 6, jq, 2 * m - 2);
    }
  };
  int nth = (int)std::thread::hardware_concurrency();
  if (nth > 16) nth = 16;
  if (nth > n_sweeps / 512) nth = n_sweeps / 512;
  if (nth <= 1) {
    rows(0, n_sweeps);
  } else {
    auto lo = [&](int i) { return (int)((int64_t)n_sweeps * i / nth); };
    std::vector<std::thread> pool;
    int made = 1;   // parts 1 .. made-1 run on their own threads
    try {
      for (int i = 1; i < nth; ++i) {
        pool.emplace_back(rows, lo(i), lo(i + 1));
        ++made;
      }
    } catch (...) {
      // no thread could be started for part `made`: this thread builds it
      // and the rest below
    }
    rows(0, lo(1));
    for (int i = made; i < nth; ++i) rows(lo(i), lo(i + 1));
    for (auto &t : pool) t.join();
  }
  int nreal = 0;
  std::vector<uint16_t> jn = pack_jn16(lat, per, present, J, &q.nbonds, &nreal);
  if (q.d_jneg.n < jn.size() && (rc = q.d_jneg.alloc(jn.size()))) return rc;
  if (q.d_table.n < q.table.size() && (rc = q.d_table.alloc(q.table.size()))) return rc;
  // stage through pinned memory: one copy of each array
  const size_t tb = q.table.size() * 4, jb = (jn.size() * 2 + 15) / 16 * 16;
  if ((rc = q.stage.reserve(jb + tb))) return rc;
  std::memcpy(q.stage.p, jn.data(), jn.size() * 2);
  std::memcpy(q.stage.p + jb, q.table.data(), tb);
  if ((int64_t)(jn.size() * 2 + tb) != pc_sqa_upload_bytes(lat.N, n_sweeps))
    return fail(PC_EINVAL, "internal: upload size disagrees with pc_sqa_upload_bytes");
  PC_CUDA_TRY(cudaMemcpyAsync(q.d_jneg.p, q.stage.p, jn.size() * 2, cudaMemcpyHostToDevice, c->stream));
  PC_CUDA_TRY(cudaMemcpyAsync(q.d_table.p, q.stage.p + jb, tb, cudaMemcpyHostToDevice, c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  q.ready = true;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_sqa_get_table(pc_ctx *c, int sweep, uint32_t *out, int32_t *jq) try {
  if (!c || !c->sqa.ready) return fail(PC_ESTATE, "pc_sqa_setup first");
  if (sweep < 0 || sweep >= c->sqa.S) return fail(PC_EINVAL, "sweep out of range");
  for (int m = 0; m < 3; ++m)
    for (int cc = 0; cc < 7; ++cc) out[7 * m + cc] = c->sqa.table[(size_t)sweep * kSqaTab + 2 * cc + 13 * m];
  if (jq) *jq = c->sqa.jq[(size_t)sweep];
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

static int sqa_enqueue(pc_ctx *c, int R, uint32_t run0, int32_t *E_dev, int32_t *best_dev,
                       int8_t *spins_dev, int first_chunk = 0, uint64_t wait_ns = 10000000000ull,
                       int32_t *corr_dev = nullptr) {
  const SqaState &q = c->sqa;
  SqaArgs a;
  a.Lx = q.lat.L[0];
  a.Ly = q.lat.L[1];
  a.Lz = q.lat.L[2];
  a.N = q.lat.N;
  a.P = q.P;
  a.NB = q.P / 16;
  a.S = q.S;
  a.mLx = recip32((uint32_t)a.Lx);
  a.mLy = recip32((uint32_t)a.Ly);
  a.run0 = run0;
  a.k0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
  a.k1 = (uint32_t)(c->seed >> 32);
  a.jneg = q.d_jneg.p;
  a.nbonds = q.nbonds;
  a.table = q.d_table.p;
  a.E = E_dev;
  a.best = best_dev;
  a.spins = spins_dev;
  a.corr = corr_dev;
  a.state = nullptr;
  a.done = a.queue = a.err = nullptr;
  a.R = R;
  a.K = a.S;
  a.n_items = R;
  a.first_item = 0;
  a.wait_ns = wait_ns;
  if (a.S > 0) {
    // persistent time-sliced schedule: about 32 (run, chunk) items per SM
    SqaState &q = c->sqa;
    int nch = (32 * c->sms + R - 1) / R;
    if (nch > a.S) nch = a.S;
    if (nch < 1) nch = 1;
    a.K = (a.S + nch - 1) / nch;
    nch = (a.S + a.K - 1) / a.K;
    a.n_items = R * nch;
    a.first_item = first_chunk * R;
    const size_t words = (size_t)R * 2 * a.NB * a.N;
    int rc;
    if (q.d_state.n < words && (rc = q.d_state.alloc(words))) return rc;
    if (q.d_sync.n < (size_t)R + 2 && (rc = q.d_sync.alloc((size_t)R + 2))) return rc;
    PC_CUDA_TRY(cudaMemsetAsync(q.d_sync.p, 0, ((size_t)R + 2) * sizeof(int), c->stream));
    a.state = q.d_state.p;
    a.done = q.d_sync.p;
    a.queue = q.d_sync.p + R;
    a.err = q.d_sync.p + R + 1;
    q.last_err = a.err;
  }
  return sqa_launch(a, R, c->stream);
}

// Reads the device-side error flag of the last persistent anneal (after a
// stream synchronisation).
static int sqa_check_device(pc_ctx *c) {
  if (!c->sqa.last_err) return PC_OK;
  int e = 0;
  PC_CUDA_TRY(cudaMemcpy(&e, c->sqa.last_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) return fail(PC_EDEVICE, "anneal: a wait for the previous chunk of a run timed out");
  return PC_OK;
}

int pc_sqa_run_dev(pc_ctx *c, int R, uint32_t run0, int32_t *E_dev, int32_t *best_dev) try {
  if (!c || !c->sqa.ready) return fail(PC_ESTATE, "pc_sqa_setup first");
  if (R < 0 || (R > 0 && !E_dev)) return fail(PC_EINVAL, "bad arguments");
  if ((uint64_t)run0 + (uint64_t)R > (1ull << 24)) return fail(PC_EINVAL, "run ids must be < 2^24");
  if (R == 0) return PC_OK;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  return sqa_enqueue(c, R, run0, E_dev, best_dev, nullptr);
} catch (...) {
  return pc::fail_exception();
}

int pc_sqa_run_corr_dev(pc_ctx *c, int R, uint32_t run0, int32_t *E_dev, int32_t *best_dev,
                        int32_t *corr_dev) try {
  if (!c || !c->sqa.ready) return fail(PC_ESTATE, "pc_sqa_setup first");
  if (R < 0 || (R > 0 && (!E_dev || !corr_dev))) return fail(PC_EINVAL, "bad arguments");
  if ((uint64_t)run0 + (uint64_t)R > (1ull << 24)) return fail(PC_EINVAL, "run ids must be < 2^24");
  if (R == 0) return PC_OK;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  return sqa_enqueue(c, R, run0, E_dev, best_dev, nullptr, 0, 10000000000ull, corr_dev);
} catch (...) {
  return pc::fail_exception();
}

int pc_sqa_run(pc_ctx *c, int R, uint32_t run0, int64_t *E_out, int8_t *spins_out) try {
  if (!c || !c->sqa.ready) return fail(PC_ESTATE, "pc_sqa_setup first");
  if (R < 0) return fail(PC_EINVAL, "R must be >= 0");
  if ((uint64_t)run0 + (uint64_t)R > (1ull << 24)) return fail(PC_EINVAL, "run ids must be < 2^24");
  if (R == 0) return PC_OK;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  SqaState &q = c->sqa;
  const size_t nE = (size_t)R * q.P;
  int rc;
  if (q.d_E.n < nE && (rc = q.d_E.alloc(nE))) return rc;
  if (spins_out && q.d_spins.n < nE * (size_t)q.lat.N && (rc = q.d_spins.alloc(nE * (size_t)q.lat.N)))
    return rc;
  if ((rc = sqa_enqueue(c, R, run0, q.d_E.p, nullptr, spins_out ? q.d_spins.p : nullptr))) return rc;
  std::vector<int32_t> hE(nE);
  PC_CUDA_TRY(cudaMemcpyAsync(hE.data(), q.d_E.p, nE * 4, cudaMemcpyDeviceToHost, c->stream));
  if (spins_out)
    PC_CUDA_TRY(cudaMemcpyAsync(spins_out, q.d_spins.p, nE * (size_t)q.lat.N, cudaMemcpyDeviceToHost,
                                c->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if ((rc = sqa_check_device(c))) return rc;
  if (E_out)
    for (size_t i = 0; i < nE; ++i) E_out[i] = hE[i];
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_sqa_selftest_wait(pc_ctx *c, int *status) try {
  if (!c || !c->sqa.ready || !status) return fail(PC_ESTATE, "pc_sqa_setup first");
  if (c->sqa.S < 2) return fail(PC_EINVAL, "the self-test needs a schedule of at least 2 sweeps");
  PC_CUDA_TRY(cudaSetDevice(c->device));
  const int R = 2;
  SqaState &q = c->sqa;
  int rc;
  if (q.d_E.n < (size_t)R * q.P && (rc = q.d_E.alloc((size_t)R * q.P))) return rc;
  // queue starts at chunk 1: no chunk 0 ever completes, so every wait runs out
  if ((rc = sqa_enqueue(c, R, 0, q.d_E.p, nullptr, nullptr, 1, 50000000ull))) return rc;
  PC_CUDA_TRY(cudaStreamSynchronize(c->stream));
  *status = sqa_check_device(c);
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_sqa_anneal(pc_ctx *c, const int32_t *dims, const int8_t *J, int P, double T, int n_sweeps,
                  const double *gamma, int R, uint32_t run0, int64_t *E_out) try {
  int rc = pc_sqa_setup(c, dims, J, P, T, n_sweeps, gamma);
  if (rc) return rc;
  return pc_sqa_run(c, R, run0, E_out, nullptr);
} catch (...) {
  return pc::fail_exception();
}

int64_t pc_sqa_upload_bytes(int N, int n_sweeps) {
  if (N < 0) return 0;
  return (int64_t)N * 2 + (int64_t)kSqaTab * 4 * (n_sweeps > 0 ? n_sweeps : 1);
}

}  // extern "C"
