// C ABI of the TNMC library (declared in include/tnmc.h): context lifetime, device memory,
// argument checking and kernel launches.  No torch types cross this boundary.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tnmc.h"
#include "kernels.h"
#include "ctx_internal.h"

struct tnmc_ctx {
  int L = 0, n_real = 0, chi = 0, CHI = 0, precision = 0, n_chains = 1, n_therm = 0;
  int cap = 0;                    // realizations allocated; n_real <= cap are active
  double* pvec = nullptr;         // per-realization antiferromagnetic-bond probability
  int* nlimit = nullptr;          // per-realization number of proposals the chains use
  bool use_nlimit = false;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;
  int64_t launches = 0;
  int words = 0;
  // inputs
  int8_t* J = nullptr;
  double* beta = nullptr;
  uint64_t* seeds = nullptr;
  // environments
  void* env = nullptr;
  size_t env_bytes = 0, te_size = 0, t_size = 0;
  int* kdim = nullptr;
  int* dqr = nullptr;
  double* lam = nullptr;
  double* logz = nullptr;
  void* rowbuf = nullptr;
  void* Rstore = nullptr;
  void* mscratch = nullptr;       // environment-build M matrices for chi = 64 (nullptr otherwise)
  long long* stats = nullptr;
  unsigned* status = nullptr;
  unsigned* rstatus = nullptr;    // per-realization status bits (numeric failures of its proposals)
  int8_t* hfield = nullptr;       // external fields in units of beta, [real][L][L] (nullptr: none)
  int compression = TNMC_COMPRESS_CANONICAL;
  int8_t* hfield_buf = nullptr;   // the buffer behind hfield, allocated at the first tnmc_set_fields
  const int* chain_of = nullptr;  // chain index of each realization's draws (periodic driver), or nullptr
  // sampling
  void* work = nullptr;
  void* work_tc = nullptr;        // workspace of the tensor-core sampler (mixed TF32 path)
  uint32_t* packed = nullptr;
  double* logq = nullptr;
  int32_t* energy = nullptr;
  int32_t* magnet = nullptr;
  int64_t* clamps = nullptr;
  int cap_n = 0;
  int last_n = 0;
  uint64_t last_step0 = 0;
  bool have_props = false;
  bool env_built = false;
  // chains
  int* have_state = nullptr;
  double* cur_logq = nullptr;
  int32_t* cur_energy = nullptr;
  int32_t* cur_magnet = nullptr;
  uint32_t* cur_spins = nullptr;
  double* acc = nullptr;
  int* cur_idx = nullptr;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_sizes;
  // device buffers come from the stream-ordered allocator where the device has one, so that
  // freeing a context never waits for work on other streams (cudaFree synchronises the device)
  bool async_alloc = false;
  // the caller's allocator (tnmc_opts.alloc / free), when given
  tnmc_alloc_fn user_alloc = nullptr;
  tnmc_free_fn user_free = nullptr;
  void* alloc_user = nullptr;
  // pinned staging ring for the small per-batch host inputs (inverse temperatures, seeds),
  // so that host-to-device copies are truly asynchronous and the caller's buffers can be
  // reused at once; a slot is reused only after its copy has executed
  static constexpr int kStageSlots = 8;
  unsigned char* h_stage = nullptr;
  cudaEvent_t stage_ev[kStageSlots] = {};
  bool stage_used[kStageSlots] = {};
  int stage_next = 0;
};

static std::string g_create_err;

namespace {

tnmc_status fail(tnmc_ctx* c, tnmc_status s, const std::string& msg) {
  if (c) c->err = msg; else g_create_err = msg;
  return s;
}

tnmc_status cuda_fail(tnmc_ctx* c, cudaError_t e, const char* what) {
  return fail(c, TNMC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename P>
tnmc_status dalloc(tnmc_ctx* c, P** p, size_t bytes) {
  void* q = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->user_alloc) {
    q = c->user_alloc(bytes, reinterpret_cast<void*>(c->stream), c->alloc_user);
    if (!q) return fail(c, TNMC_ERR_OOM, "the caller's allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = c->async_alloc ? cudaMallocAsync(&q, bytes, c->stream) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, TNMC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                       cudaGetErrorString(e));
    }
  }
  c->allocs.push_back(q);
  c->alloc_sizes.push_back(bytes);
  *p = reinterpret_cast<P*>(q);
  return TNMC_OK;
}

// Return one block to whoever allocated it, in stream order on st.
void release_block(tnmc_ctx* c, void* p, size_t bytes, cudaStream_t st) {
  if (c->user_free) c->user_free(p, bytes, reinterpret_cast<void*>(st), c->alloc_user);
  else if (c->async_alloc) cudaFreeAsync(p, st);
  else cudaFree(p);
}

void dfree(tnmc_ctx* c, void* p) {
  if (!p) return;
  size_t bytes = 0;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      bytes = c->alloc_sizes[i];
      c->allocs.erase(c->allocs.begin() + i);
      c->alloc_sizes.erase(c->alloc_sizes.begin() + i);
      break;
    }
  release_block(c, p, bytes, c->stream);
}

int round_chi(int chi) {
  if (chi <= 4) return 4;
  if (chi <= 8) return 8;
  if (chi <= 16) return 16;
  if (chi <= 32) return 32;
  if (chi <= 64) return 64;
  return 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

tnmc_status check_status(tnmc_ctx* c) {
  unsigned st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
  if (st & tnmc::ST_NUMERIC)
    return fail(c, TNMC_ERR_NUMERIC, "a conditional weight w(+)+w(-) vanished or was not finite");
  if (st & tnmc::ST_TIMEOUT) return fail(c, TNMC_ERR_TIMEOUT, "a bounded device wait ran out");
  if (st & tnmc::ST_ARG) return fail(c, TNMC_ERR_ARG, "a kernel rejected its arguments");
  return TNMC_OK;
}

// Device bytes of every buffer a context holds, one function for the allocation and the
// capacity estimate so that the two cannot drift apart.
struct CtxSizes {
  size_t J, beta, seeds, pvec, nlimit, env, kdim, dqr, lam, logz, rowbuf, Rstore, mscratch, stats, status, rstatus,
      work, work_tc, clamps, have_state, cur_logq, cur_energy, cur_magnet, cur_spins, acc;
  size_t total() const {
    return J + beta + seeds + pvec + nlimit + env + kdim + dqr + lam + logz + rowbuf + Rstore + mscratch + stats +
           status + rstatus + work + work_tc + clamps + have_state + cur_logq + cur_energy + cur_magnet + cur_spins +
           acc;
  }
};

CtxSizes ctx_sizes(int L, int n_real, int CHI, int precision, int n_chains, int num_sms) {
  CtxSizes z{};
  const size_t tsz = precision == TNMC_FP64 ? 8 : 4;
  const size_t tesz = precision == TNMC_FP64 ? 8 : (precision == TNMC_MIXED_BF16 ? 2 : 4);
  const size_t D = 2 * (size_t)CHI, tile = (size_t)2 * CHI * CHI, R = (size_t)n_real;
  const size_t chains = R * n_chains, words = ((size_t)L * L + 31) / 32;
  z.J = (size_t)2 * L * (L - 1) * R;
  z.beta = 8 * R; z.seeds = 8 * R; z.pvec = 8 * R; z.nlimit = 4 * R;
  z.env = R * L * L * tile * tesz;
  z.kdim = 4 * R * L * (L + 1);
  z.dqr = 4 * R * (L + 1);
  z.lam = 8 * R * L;
  z.logz = 8 * R;
  z.rowbuf = R * 2 * L * tile * tsz;
  z.Rstore = R * L * D * D * tsz;
  z.mscratch = CHI > 32 ? R * D * D * tsz : 0;     // M of the environment build when it leaves shared memory
  z.stats = 4 * sizeof(long long) * R;
  z.status = sizeof(unsigned);
  z.rstatus = sizeof(unsigned) * R;
  z.work = tnmc::sample_work_bytes(L, CHI, precision, num_sms);
  z.work_tc = (precision == TNMC_MIXED_TF32 && tnmc::sample_tc_supported(CHI))
                  ? tnmc::sample_tc_work_bytes(L, CHI, num_sms) : 0;
  z.clamps = 8 * R;
  z.have_state = 4 * chains; z.cur_logq = 8 * chains; z.cur_energy = 4 * chains; z.cur_magnet = 4 * chains;
  z.cur_spins = 4 * chains * words;
  z.acc = 8 * R * tnmc::ACC_SLOTS;
  return z;
}

// Device bytes of the proposal buffers for n proposals per chain.
size_t props_bytes(int L, int n_real, int n_chains, int n) {
  const size_t items = (size_t)n_real * n_chains * n, words = ((size_t)L * L + 31) / 32;
  return items * (words * 4 + 8 + 4 + 4 + 4);
}

tnmc_status ensure_props(tnmc_ctx* c, int n) {
  if (n <= c->cap_n) return TNMC_OK;
  dfree(c, c->packed); dfree(c, c->logq); dfree(c, c->energy); dfree(c, c->magnet); dfree(c, c->cur_idx);
  c->packed = nullptr; c->logq = nullptr; c->energy = nullptr; c->magnet = nullptr; c->cur_idx = nullptr;
  const size_t items = (size_t)c->cap * c->n_chains * n;
  tnmc_status s;
  if ((s = dalloc(c, &c->packed, items * c->words * sizeof(uint32_t)))) return s;
  if ((s = dalloc(c, &c->logq, items * sizeof(double)))) return s;
  if ((s = dalloc(c, &c->energy, items * sizeof(int32_t)))) return s;
  if ((s = dalloc(c, &c->magnet, items * sizeof(int32_t)))) return s;
  if ((s = dalloc(c, &c->cur_idx, items * sizeof(int)))) return s;
  c->cap_n = n;
  return TNMC_OK;
}

}  // namespace


extern "C" {

int tnmc_version(void) { return 100; }

const char* tnmc_last_error(const tnmc_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

tnmc_status tnmc_couplings_pmj(int L, int n_real, const uint64_t* seeds_host, double p, int8_t* out_dev,
                               void* stream) {
  if (L < 2 || n_real < 1 || !seeds_host || !out_dev || !(p >= 0.0 && p <= 1.0))
    return fail(nullptr, TNMC_ERR_ARG, "tnmc_couplings_pmj: invalid argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* sd = nullptr;
  cudaError_t e = cudaMalloc(&sd, sizeof(uint64_t) * n_real);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, TNMC_ERR_OOM, "seed buffer"); }
  e = cudaMemcpyAsync(sd, seeds_host, sizeof(uint64_t) * n_real, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = tnmc::launch_couplings(L, n_real, sd, p, out_dev, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(sd);
  if (e != cudaSuccess) return fail(nullptr, TNMC_ERR_CUDA, std::string("couplings: ") + cudaGetErrorString(e));
  return TNMC_OK;
}

tnmc_status tnmc_create(int L, int n_real, const int8_t* couplings, const double* beta_host,
                        const uint64_t* seeds_host, int chi, const tnmc_opts* opts, tnmc_ctx** out) {
  if (!out) return fail(nullptr, TNMC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (L < 2 || L > 4096) return fail(nullptr, TNMC_ERR_ARG, "L must be in [2, 4096]");
  if (n_real < 1) return fail(nullptr, TNMC_ERR_ARG, "n_real must be >= 1");
  if (!couplings || !beta_host || !seeds_host || !opts) return fail(nullptr, TNMC_ERR_ARG, "NULL input");
  if (chi < 1) return fail(nullptr, TNMC_ERR_ARG, "chi must be >= 1");
  if (round_chi(chi) == 0) return fail(nullptr, TNMC_ERR_UNSUPPORTED, "chi > 64 is not built into this library");
  if (chi > 32 && opts && opts->precision == TNMC_FP64)
    return fail(nullptr, TNMC_ERR_UNSUPPORTED, "the FP64 path is built for chi <= 32 (chi = 64 needs 256 KB of shared memory)");
  if (opts->precision < 0 || opts->precision > 3) return fail(nullptr, TNMC_ERR_ARG, "unknown precision");
  if (opts->n_chains < 1 || opts->n_chains > 8) return fail(nullptr, TNMC_ERR_ARG, "n_chains must be in [1, 8]");
  if (opts->compression != TNMC_COMPRESS_CANONICAL && opts->compression != TNMC_COMPRESS_ZIPUP)
    return fail(nullptr, TNMC_ERR_ARG, "unknown compression");
  if ((opts->alloc == nullptr) != (opts->free == nullptr))
    return fail(nullptr, TNMC_ERR_ARG, "opts.alloc and opts.free must be given together");
  for (int k = 0; k < n_real; ++k)
    if (!(beta_host[k] > 0.0) || !std::isfinite(beta_host[k]))
      return fail(nullptr, TNMC_ERR_ARG, "beta must be positive and finite");
  const size_t nb = (size_t)2 * L * (L - 1);
  std::vector<int8_t> Jh(nb * n_real);
  if (cudaMemcpy(Jh.data(), couplings, Jh.size(), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, TNMC_ERR_ARG, "couplings pointer is neither host nor device memory");
  }
  for (size_t i = 0; i < Jh.size(); ++i)
    if (Jh[i] != 1 && Jh[i] != -1) return fail(nullptr, TNMC_ERR_ARG, "couplings must be +1 or -1");

  tnmc_ctx* c = new tnmc_ctx();
  c->L = L; c->n_real = n_real; c->cap = n_real; c->chi = chi; c->CHI = round_chi(chi);
  c->precision = opts->precision; c->n_chains = opts->n_chains; c->n_therm = opts->n_therm;
  c->compression = opts->compression;
  c->stream = reinterpret_cast<cudaStream_t>(opts->stream);
  c->words = (L * L + 31) / 32;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  int pools = 0;
  if (cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, c->device) != cudaSuccess) cudaGetLastError();
  c->async_alloc = pools != 0;
  c->user_alloc = opts->alloc; c->user_free = opts->free; c->alloc_user = opts->alloc_user;
  c->t_size = c->precision == TNMC_FP64 ? 8 : 4;
  c->te_size = c->precision == TNMC_FP64 ? 8 : (c->precision == TNMC_MIXED_BF16 ? 2 : 4);
  const int CHI = c->CHI;
  const CtxSizes z = ctx_sizes(L, n_real, CHI, c->precision, c->n_chains, c->num_sms);
  tnmc_status s;
#define TRY(x) do { if ((s = (x)) != TNMC_OK) { g_create_err = c->err; tnmc_destroy(c); return s; } } while (0)
  TRY(dalloc(c, &c->J, z.J));
  TRY(dalloc(c, &c->beta, z.beta));
  TRY(dalloc(c, &c->seeds, z.seeds));
  TRY(dalloc(c, &c->pvec, z.pvec));
  TRY(dalloc(c, &c->nlimit, z.nlimit));
  c->env_bytes = z.env;
  TRY(dalloc(c, &c->env, z.env));
  TRY(dalloc(c, &c->kdim, z.kdim));
  TRY(dalloc(c, &c->dqr, z.dqr));
  TRY(dalloc(c, &c->lam, z.lam));
  TRY(dalloc(c, &c->logz, z.logz));
  TRY(dalloc(c, &c->rowbuf, z.rowbuf));
  TRY(dalloc(c, &c->Rstore, z.Rstore));
  if (z.mscratch) TRY(dalloc(c, &c->mscratch, z.mscratch));
  TRY(dalloc(c, &c->stats, z.stats));
  TRY(dalloc(c, &c->status, z.status));
  TRY(dalloc(c, &c->rstatus, z.rstatus));
  TRY(dalloc(c, &c->work, z.work));
  if (z.work_tc) TRY(dalloc(c, &c->work_tc, z.work_tc));
  TRY(dalloc(c, &c->clamps, z.clamps));
  const size_t chains = (size_t)n_real * c->n_chains;
  TRY(dalloc(c, &c->have_state, z.have_state));
  TRY(dalloc(c, &c->cur_logq, z.cur_logq));
  TRY(dalloc(c, &c->cur_energy, z.cur_energy));
  TRY(dalloc(c, &c->cur_magnet, z.cur_magnet));
  TRY(dalloc(c, &c->cur_spins, z.cur_spins));
  TRY(dalloc(c, &c->acc, z.acc));
#undef TRY
  cudaError_t e = cudaMemcpyAsync(c->J, Jh.data(), Jh.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->beta, beta_host, sizeof(double) * n_real, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->seeds, seeds_host, sizeof(uint64_t) * n_real, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->rstatus, 0, sizeof(unsigned) * n_real, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->clamps, 0, sizeof(int64_t) * n_real, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->have_state, 0, sizeof(int) * chains, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(double) * (size_t)n_real * tnmc::ACC_SLOTS, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { cuda_fail(c, e, "create"); g_create_err = c->err; tnmc_destroy(c); return TNMC_ERR_CUDA; }
  *out = c;
  return TNMC_OK;
}

// Queue the copy of the small per-realization host inputs (inverse temperatures, seeds and,
// when given, bond probabilities and proposal limits) through the pinned staging ring.
static tnmc_status stage_small_inputs(tnmc_ctx* c, const double* beta_host, const uint64_t* seeds_host,
                                      const double* p_host = nullptr, const int* nlimit_host = nullptr) {
  const int n = c->n_real;
  for (int k = 0; k < n; ++k)
    if (!(beta_host[k] > 0.0) || !std::isfinite(beta_host[k])) return fail(c, TNMC_ERR_ARG, "beta must be positive and finite");
  const size_t slot_bytes = (size_t)32 * c->cap;
  cudaError_t e = cudaSuccess;
  if (!c->h_stage) {
    c->h_stage = static_cast<unsigned char*>(tnmc::pinned_get(slot_bytes * tnmc_ctx::kStageSlots));
    if (!c->h_stage) return fail(c, TNMC_ERR_OOM, "pinned staging");
    for (int s = 0; s < tnmc_ctx::kStageSlots; ++s) cudaEventCreateWithFlags(&c->stage_ev[s], cudaEventDisableTiming);
  }
  const int slot = c->stage_next;
  c->stage_next = (slot + 1) % tnmc_ctx::kStageSlots;
  if (c->stage_used[slot]) {
    e = cudaEventSynchronize(c->stage_ev[slot]);
    if (e != cudaSuccess) return cuda_fail(c, e, "staging wait");
  }
  unsigned char* h = c->h_stage + slot_bytes * slot;
  unsigned char* hb = h;
  unsigned char* hs = h + 8 * (size_t)c->cap;
  unsigned char* hp = h + 16 * (size_t)c->cap;
  unsigned char* hl = h + 24 * (size_t)c->cap;
  std::memcpy(hb, beta_host, sizeof(double) * n);
  std::memcpy(hs, seeds_host, sizeof(uint64_t) * n);
  e = cudaMemcpyAsync(c->beta, hb, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->seeds, hs, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && p_host) {
    std::memcpy(hp, p_host, sizeof(double) * n);
    e = cudaMemcpyAsync(c->pvec, hp, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess && nlimit_host) {
    std::memcpy(hl, nlimit_host, sizeof(int) * n);
    e = cudaMemcpyAsync(c->nlimit, hl, sizeof(int) * n, cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(c->stage_ev[slot], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "staging copy");
  c->stage_used[slot] = true;
  return TNMC_OK;
}

tnmc_status tnmc_set_couplings(tnmc_ctx* c, const int8_t* couplings, const double* beta_host,
                               const uint64_t* seeds_host) {
  if (!c || !couplings || !beta_host || !seeds_host) return fail(c, TNMC_ERR_ARG, "NULL argument");
  const size_t nb = (size_t)2 * c->L * (c->L - 1) * c->n_real;
  const bool dev = is_device_ptr(couplings);
  if (!dev)
    for (size_t i = 0; i < nb; ++i)
      if (couplings[i] != 1 && couplings[i] != -1) return fail(c, TNMC_ERR_ARG, "couplings must be +1 or -1");
  tnmc_status s = stage_small_inputs(c, beta_host, seeds_host);
  if (s) return s;
  cudaError_t e = cudaMemcpyAsync(c->J, couplings, nb, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set couplings");
  c->env_built = false;
  c->use_nlimit = false;
  return tnmc_reset_chains(c);
}

tnmc_status tnmc_set_realizations(tnmc_ctx* c, const uint64_t* seeds_host, const double* beta_host, double p) {
  if (!c || !seeds_host || !beta_host) return fail(c, TNMC_ERR_ARG, "NULL argument");
  if (!(p >= 0.0 && p <= 1.0)) return fail(c, TNMC_ERR_ARG, "p must be in [0, 1]");
  tnmc_status s = stage_small_inputs(c, beta_host, seeds_host);
  if (s) return s;
  c->use_nlimit = false;
  cudaError_t e = tnmc::launch_couplings(c->L, c->n_real, c->seeds, p, c->J, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "couplings launch");
  ++c->launches;
  c->env_built = false;
  return tnmc_reset_chains(c);
}

tnmc_status tnmc_build_env(tnmc_ctx* c, double* log_z_host) {
  if (!c) return fail(nullptr, TNMC_ERR_ARG, "NULL context");
  cudaError_t e;
  switch (c->precision) {
    case TNMC_FP64: {
      tnmc::EnvBuildArgs<double, double> a{c->L, c->n_real, c->chi, c->J, c->beta, (double*)c->env, c->kdim, c->dqr,
                                           c->lam, c->logz, (double*)c->rowbuf, (double*)c->Rstore, c->stats, c->status};
      a.hfield = c->hfield;
      a.zipup = c->compression == TNMC_COMPRESS_ZIPUP;
      e = tnmc::launch_env_build(a, c->CHI, c->stream);
      break;
    }
    case TNMC_MIXED_BF16: {
      tnmc::EnvBuildArgs<float, __nv_bfloat16> a{c->L, c->n_real, c->chi, c->J, c->beta, (__nv_bfloat16*)c->env, c->kdim,
                                                 c->dqr, c->lam, c->logz, (float*)c->rowbuf, (float*)c->Rstore, c->stats, c->status};
      a.Mscratch = (float*)c->mscratch;
      a.hfield = c->hfield;
      a.zipup = c->compression == TNMC_COMPRESS_ZIPUP;
      e = tnmc::launch_env_build(a, c->CHI, c->stream);
      break;
    }
    default: {
      tnmc::EnvBuildArgs<float, float> a{c->L, c->n_real, c->chi, c->J, c->beta, (float*)c->env, c->kdim, c->dqr,
                                         c->lam, c->logz, (float*)c->rowbuf, (float*)c->Rstore, c->stats, c->status};
      a.Mscratch = (float*)c->mscratch;
      a.hfield = c->hfield;
      a.zipup = c->compression == TNMC_COMPRESS_ZIPUP;
      e = tnmc::launch_env_build(a, c->CHI, c->stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "env build launch");
  ++c->launches;
  c->env_built = true;
  if (log_z_host) {
    tnmc_status s = check_status(c);
    if (s) return s;
    e = cudaMemcpy(log_z_host, c->logz, sizeof(double) * c->n_real, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "log Z copy");
  }
  return TNMC_OK;
}

static tnmc_status run_sample(tnmc_ctx* c, int n, uint64_t step0, const int8_t* forced, double* logq,
                              double* qplus, bool props) {
  tnmc::SampleArgs a{};
  a.L = c->L; a.n_real = c->n_real; a.n_chains = props ? c->n_chains : 1; a.n = n;
  a.n_items = props ? c->n_chains * n : n;
  a.step0 = step0; a.J = c->J; a.beta = c->beta; a.seeds = c->seeds; a.env = c->env;
  a.spins_packed = props ? c->packed : nullptr; a.words = c->words;
  a.logq = logq; a.energy = props ? c->energy : nullptr; a.magnet = props ? c->magnet : nullptr;
  a.clamps = props ? c->clamps : nullptr; a.forced = forced; a.qplus = qplus; a.work = c->work;
  a.status = c->status;
  a.real_status = props ? c->rstatus : nullptr;
  a.hfield = c->hfield;
  a.chain_of = props ? c->chain_of : nullptr;
  cudaError_t e;
  if (c->work_tc) {
    a.work = c->work_tc;
    e = tnmc::launch_sample_tc(a, c->CHI, c->num_sms, c->stream);
  } else {
    e = tnmc::launch_sample(a, c->precision, c->CHI, c->num_sms, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "sample launch");
  ++c->launches;
  return TNMC_OK;
}

tnmc_status tnmc_propose(tnmc_ctx* c, int n, uint64_t step0, double* logq_dev, int32_t* energy_dev,
                         int32_t* magnet_dev) {
  if (!c) return fail(nullptr, TNMC_ERR_ARG, "NULL context");
  if (!c->env_built) return fail(c, TNMC_ERR_STATE, "tnmc_propose before tnmc_build_env");
  if (n < 1) return fail(c, TNMC_ERR_ARG, "n must be >= 1");
  if (step0 + (uint64_t)n > 0xFFFFFFFFull) return fail(c, TNMC_ERR_ARG, "step indices must fit in 32 bits");
  tnmc_status s = ensure_props(c, n);
  if (s) return s;
  if ((s = run_sample(c, n, step0, nullptr, c->logq, nullptr, true))) return s;
  const size_t items = (size_t)c->n_real * c->n_chains * n;
  cudaError_t e = cudaSuccess;
  if (logq_dev) e = cudaMemcpyAsync(logq_dev, c->logq, items * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && energy_dev)
    e = cudaMemcpyAsync(energy_dev, c->energy, items * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && magnet_dev)
    e = cudaMemcpyAsync(magnet_dev, c->magnet, items * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "propose output copy");
  c->last_n = n; c->last_step0 = step0; c->have_props = true;
  return TNMC_OK;
}

tnmc_status tnmc_get_spins(tnmc_ctx* c, int8_t* spins_dev) {
  if (!c || !spins_dev) return fail(c, TNMC_ERR_ARG, "NULL argument");
  if (!c->have_props) return fail(c, TNMC_ERR_STATE, "no proposals");
  const int64_t n_cfg = (int64_t)c->n_real * c->n_chains * c->last_n;
  cudaError_t e = tnmc::launch_unpack(c->packed, c->words, c->L * c->L, n_cfg, spins_dev, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "unpack");
  ++c->launches;
  return TNMC_OK;
}

tnmc_status tnmc_eval_conditionals(tnmc_ctx* c, int n, const int8_t* spins_dev, double* logq_dev,
                                   double* qplus_dev) {
  if (!c || !spins_dev) return fail(c, TNMC_ERR_ARG, "NULL argument");
  if (!c->env_built) return fail(c, TNMC_ERR_STATE, "tnmc_eval_conditionals before tnmc_build_env");
  if (n < 1) return fail(c, TNMC_ERR_ARG, "n must be >= 1");
  if (!is_device_ptr(spins_dev)) return fail(c, TNMC_ERR_ARG, "spins_dev must be device memory");
  double* lq = logq_dev;
  double* tmp = nullptr;
  if (!lq) {
    tnmc_status sa = dalloc(c, &tmp, sizeof(double) * (size_t)c->n_real * n);
    if (sa) return sa;
    lq = tmp;
  }
  tnmc_status s = run_sample(c, n, 0, spins_dev, lq, qplus_dev, false);
  if (tmp) dfree(c, tmp);       // stream-ordered: the sweep that writes it runs first
  return s;
}

tnmc_status tnmc_accept(tnmc_ctx* c, uint8_t* accepted_dev, int64_t* n_accepted_host) {
  if (!c) return fail(nullptr, TNMC_ERR_ARG, "NULL context");
  if (!c->have_props) return fail(c, TNMC_ERR_STATE, "tnmc_accept before tnmc_propose");
  double before = 0.0;
  std::vector<double> acc_h;
  if (n_accepted_host) {
    acc_h.resize((size_t)c->n_real * tnmc::ACC_SLOTS);
    cudaError_t e = cudaMemcpyAsync(acc_h.data(), c->acc, acc_h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "accumulator read");
    for (int k = 0; k < c->n_real; ++k) before += acc_h[(size_t)k * tnmc::ACC_SLOTS + tnmc::ACC_NACC];
  }
  tnmc::AcceptArgs a{};
  a.L = c->L; a.n_real = c->n_real; a.n_chains = c->n_chains; a.n = c->last_n; a.words = c->words;
  a.n_therm = c->n_therm; a.step0 = c->last_step0; a.beta = c->beta; a.seeds = c->seeds;
  a.logq = c->logq; a.energy = c->energy; a.magnet = c->magnet; a.spins_packed = c->packed;
  a.accepted = accepted_dev; a.have_state = c->have_state; a.cur_logq = c->cur_logq;
  a.cur_energy = c->cur_energy; a.cur_magnet = c->cur_magnet; a.cur_spins = c->cur_spins;
  a.acc = c->acc; a.cur_idx = c->cur_idx; a.status = c->status;
  a.nlimit = c->use_nlimit ? c->nlimit : nullptr;
  cudaError_t e = tnmc::launch_accept(a, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "accept launch");
  ++c->launches;
  c->have_props = false;
  if (n_accepted_host) {
    tnmc_status s = check_status(c);
    if (s) return s;
    e = cudaMemcpy(acc_h.data(), c->acc, acc_h.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "accumulator read");
    double after = 0.0;
    for (int k = 0; k < c->n_real; ++k) after += acc_h[(size_t)k * tnmc::ACC_SLOTS + tnmc::ACC_NACC];
    *n_accepted_host = (int64_t)llround(after - before);
  }
  return TNMC_OK;
}

tnmc_status tnmc_observables(tnmc_ctx* c, tnmc_obs* out_host) {
  if (!c || !out_host) return fail(c, TNMC_ERR_ARG, "NULL argument");
  cudaError_t es = cudaStreamSynchronize(c->stream);
  if (es != cudaSuccess) return cuda_fail(c, es, "synchronise");
  std::vector<double> acc((size_t)c->n_real * tnmc::ACC_SLOTS);
  std::vector<int64_t> cl(c->n_real);
  cudaError_t e = cudaMemcpy(acc.data(), c->acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(cl.data(), c->clamps, cl.size() * sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "observables copy");
  std::vector<unsigned> rst(c->n_real);
  e = cudaMemcpy(rst.data(), c->rstatus, sizeof(unsigned) * rst.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "status copy");
  for (int k = 0; k < c->n_real; ++k) {
    tnmc::obs_from_acc(&acc[(size_t)k * tnmc::ACC_SLOTS], cl[k], &out_host[k]);
    out_host[k].status = (rst[k] & tnmc::ST_NUMERIC) ? TNMC_ERR_NUMERIC : TNMC_OK;
  }
  // every realization is filled in; a numeric failure of some is reported after the fact
  return check_status(c);
}

tnmc_status tnmc_reset_chains(tnmc_ctx* c) {
  if (!c) return fail(nullptr, TNMC_ERR_ARG, "NULL context");
  const size_t chains = (size_t)c->n_real * c->n_chains;
  cudaError_t e = cudaMemsetAsync(c->have_state, 0, sizeof(int) * chains, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->rstatus, 0, sizeof(unsigned) * c->n_real, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(double) * (size_t)c->n_real * tnmc::ACC_SLOTS, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->clamps, 0, sizeof(int64_t) * c->n_real, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset");
  c->have_props = false;
  return TNMC_OK;
}

tnmc_status tnmc_destroy(tnmc_ctx* c) {
  if (!c) return TNMC_OK;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  for (size_t i = 0; i < c->allocs.size(); ++i) release_block(c, c->allocs[i], c->alloc_sizes[i], c->stream);
  if (c->h_stage) {
    tnmc::pinned_put(c->h_stage, (size_t)32 * c->cap * tnmc_ctx::kStageSlots);
    for (int s = 0; s < tnmc_ctx::kStageSlots; ++s) if (c->stage_ev[s]) cudaEventDestroy(c->stage_ev[s]);
  }
  c->allocs.clear();
  c->alloc_sizes.clear();
  delete c;
  return TNMC_OK;
}

size_t tnmc_env_bytes(const tnmc_ctx* c) { return c ? c->env_bytes : 0; }

tnmc_status tnmc_build_stats(tnmc_ctx* c, int64_t* out_host) {
  if (!c || !out_host) return fail(c, TNMC_ERR_ARG, "NULL argument");
  if (!c->env_built) return fail(c, TNMC_ERR_STATE, "no environments");
  std::vector<long long> st((size_t)4 * c->n_real);
  cudaError_t e = cudaMemcpyAsync(st.data(), c->stats, st.size() * sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stats copy");
  int64_t mx = 0, unc = 0, tot = 0, nsvd = 0;
  for (int k = 0; k < c->n_real; ++k) {
    mx = st[4 * k] > mx ? st[4 * k] : mx; unc += st[4 * k + 1]; tot += st[4 * k + 2]; nsvd += st[4 * k + 3];
  }
  out_host[0] = mx; out_host[1] = unc; out_host[2] = tot; out_host[3] = nsvd;
  return TNMC_OK;
}

int64_t tnmc_launch_count(const tnmc_ctx* c) { return c ? c->launches : 0; }

tnmc_status tnmc_realization_status(tnmc_ctx* c, int32_t* out_host) {
  if (!c || !out_host) return fail(c, TNMC_ERR_ARG, "NULL argument");
  std::vector<unsigned> st(c->n_real);
  cudaError_t e = cudaMemcpyAsync(st.data(), c->rstatus, sizeof(unsigned) * st.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "status copy");
  for (int k = 0; k < c->n_real; ++k) out_host[k] = (st[k] & tnmc::ST_NUMERIC) ? TNMC_ERR_NUMERIC : TNMC_OK;
  return TNMC_OK;
}

tnmc_status tnmc_set_fields(tnmc_ctx* c, const int8_t* fields) {
  if (!c) return fail(nullptr, TNMC_ERR_ARG, "NULL context");
  if (!fields) {                       // back to no fields (the buffer stays for reuse)
    c->hfield = nullptr;
    c->env_built = false;
    return TNMC_OK;
  }
  const size_t nb = (size_t)c->n_real * c->L * c->L;
  if (!c->hfield_buf) {
    tnmc_status s = dalloc(c, &c->hfield_buf, nb);
    if (s) return s;
  }
  const bool dev = is_device_ptr(fields);
  cudaError_t e = cudaMemcpyAsync(c->hfield_buf, fields, nb, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(c->stream);   // the host buffer may go at once
  if (e != cudaSuccess) return cuda_fail(c, e, "fields copy");
  c->hfield = c->hfield_buf;
  c->env_built = false;
  return TNMC_OK;
}

tnmc_status tnmc_realization_status_async(tnmc_ctx* c, uint32_t* out_dev) {
  if (!c || !out_dev) return fail(c, TNMC_ERR_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(out_dev, c->rstatus, sizeof(unsigned) * c->n_real, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "status copy");
  return TNMC_OK;
}

tnmc_status tnmc_selftest_bounded_wait(int arrive, int64_t* elapsed_us) {
  unsigned* st = nullptr;
  cudaError_t e = cudaMalloc(&st, sizeof(unsigned));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, TNMC_ERR_OOM, "status word"); }
  unsigned h = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMemset(st, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventRecord(t0, nullptr);
  if (e == cudaSuccess) e = tnmc::launch_wait_probe(arrive, 1ll << 12, st, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(t1, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(unsigned), cudaMemcpyDeviceToHost);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "wait self-test");
  if (elapsed_us) *elapsed_us = (int64_t)(1000.0f * ms);
  if (h & tnmc::ST_TIMEOUT) return fail(nullptr, TNMC_ERR_TIMEOUT, "the bounded wait ran out (as the self-test intends when nothing arrives)");
  return TNMC_OK;
}

tnmc_status tnmc_env_build_occupancy(int L, int chi, int precision, int32_t* ctas_per_sm, int32_t* num_sms) {
  if (!ctas_per_sm || L < 2 || L > 4096 || precision < 0 || precision > 3)
    return fail(nullptr, TNMC_ERR_ARG, "bad arguments");
  const int CHI = round_chi(chi);
  if (chi < 1 || CHI == 0 || (CHI > 32 && precision == TNMC_FP64))
    return fail(nullptr, TNMC_ERR_UNSUPPORTED, "chi outside 1..64 (1..32 in FP64)");
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = tnmc::env_build_occupancy(L, CHI, precision, &per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "occupancy query");
  *ctas_per_sm = per_sm;
  if (num_sms) *num_sms = sms;
  return TNMC_OK;
}

size_t tnmc_device_bytes(const tnmc_ctx* c) {
  if (!c) return 0;
  size_t b = 0;
  for (size_t s : c->alloc_sizes) b += s;
  return b;
}

size_t tnmc_estimate_device_bytes(int L, int n_real, int chi, const tnmc_opts* opts, int n_max) {
  if (L < 2 || n_real < 1 || !opts || n_max < 0 || round_chi(chi) == 0) return 0;
  if (chi > 32 && opts->precision == TNMC_FP64) return 0;
  if (opts->n_chains < 1 || opts->n_chains > 8) return 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;  // without a device: the GB300 count, for planning on a host
  }
  return ctx_sizes(L, n_real, round_chi(chi), opts->precision, opts->n_chains, sms).total() +
         (n_max > 0 ? props_bytes(L, n_real, opts->n_chains, n_max) : 0);
}

tnmc_status tnmc_copy_env(tnmc_ctx* c, int real, int row, double* tiles_host, int32_t* dims_host, double* lam_host) {
  if (!c) return fail(nullptr, TNMC_ERR_ARG, "NULL context");
  if (real < 0 || real >= c->n_real || row < 0 || row >= c->L) return fail(c, TNMC_ERR_ARG, "index out of range");
  if (!c->env_built) return fail(c, TNMC_ERR_STATE, "no environments");
  tnmc_status s = check_status(c);
  if (s) return s;
  const int L = c->L, CHI = c->CHI, chi = c->chi;
  const size_t tile = (size_t)2 * CHI * CHI;
  const size_t off = ((size_t)real * L + row) * L * tile;
  std::vector<unsigned char> raw(L * tile * c->te_size);
  cudaError_t e = cudaMemcpy(raw.data(), (const unsigned char*)c->env + off * c->te_size, raw.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "env copy");
  if (tiles_host) {
    for (int cc = 0; cc < L; ++cc)
      for (int y = 0; y < 2; ++y)
        for (int a = 0; a < chi; ++a)
          for (int b = 0; b < chi; ++b) {
            const size_t src = (size_t)cc * tile + (size_t)y * CHI * CHI + (size_t)a * CHI + b;
            double v;
            if (c->te_size == 8) { std::memcpy(&v, &raw[src * 8], 8); }
            else if (c->te_size == 4) { float f; std::memcpy(&f, &raw[src * 4], 4); v = f; }
            else { uint16_t h; std::memcpy(&h, &raw[src * 2], 2); uint32_t bits = (uint32_t)h << 16; float f; std::memcpy(&f, &bits, 4); v = f; }
            tiles_host[(((size_t)cc * 2 + y) * chi + a) * chi + b] = v;
          }
  }
  if (dims_host) {
    e = cudaMemcpy(dims_host, c->kdim + ((size_t)real * L + row) * (L + 1), sizeof(int) * (L + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "dims copy");
  }
  if (lam_host) {
    e = cudaMemcpy(lam_host, c->lam + (size_t)real * L + row, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "lam copy");
  }
  return TNMC_OK;
}

}  // extern "C"

namespace tnmc {

// Pinned host blocks are kept for reuse instead of being returned with cudaFreeHost, which
// may synchronise the device; the cache is bounded by the largest set of contexts alive at once.
namespace {
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;
}  // namespace

void* pinned_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned_free.find(bytes);
    if (it != g_pinned_free.end()) {
      void* p = it->second;
      g_pinned_free.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return p;
}

void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.emplace(bytes, p);
}

void obs_from_acc(const double* a, int64_t clamps, tnmc_obs* out) {
  tnmc_obs& o = *out;
  std::memset(&o, 0, sizeof(o));
  o.n_prop = (int64_t)llround(a[ACC_NPROP]);
  o.n_acc = (int64_t)llround(a[ACC_NACC]);
  o.n_meas = (int64_t)llround(a[ACC_NMEAS]);
  o.n_meas_q = (int64_t)llround(a[ACC_NMEASQ]);
  o.clamps = clamps;
  const double nm = a[ACC_NMEAS] > 0 ? a[ACC_NMEAS] : 1.0;
  const double nq = a[ACC_NMEASQ] > 0 ? a[ACC_NMEASQ] : 1.0;
  o.E = a[ACC_E] / nm; o.E2 = a[ACC_E2] / nm; o.m_abs = a[ACC_MABS] / nm;
  o.m2 = a[ACC_M2] / nm; o.m4 = a[ACC_M4] / nm;
  o.q = a[ACC_Q] / nq; o.q_abs = a[ACC_QABS] / nq; o.q2 = a[ACC_Q2] / nq; o.q4 = a[ACC_Q4] / nq;
  o.m_edge = a[ACC_MEDGE] / nm; o.m_edge_abs = a[ACC_MEDGEABS] / nm; o.m_edge2 = a[ACC_MEDGE2] / nm;
  o.n_tests = (int64_t)llround(a[ACC_NTEST]);
  o.status = TNMC_OK;
}

// A new batch on a pooled context (used by the request server): n_active <= capacity
// realizations, each with its own seed, inverse temperature, bond probability and number of
// proposals per chain; couplings are generated on the device; all asynchronous.
tnmc_status ctx_begin_batch(tnmc_ctx* c, int n_active, const uint64_t* seeds, const double* betas,
                            const double* ps, const int* nlimits) {
  if (!c || n_active < 1 || n_active > c->cap) return fail(c, TNMC_ERR_ARG, "batch size outside the capacity");
  for (int k = 0; k < n_active; ++k)
    if (!(ps[k] >= 0.0 && ps[k] <= 1.0) || nlimits[k] < 1) return fail(c, TNMC_ERR_ARG, "bad p or n");
  c->n_real = n_active;
  tnmc_status s = stage_small_inputs(c, betas, seeds, ps, nlimits);
  if (s) return s;
  cudaError_t e = launch_couplings_pvec(c->L, c->n_real, c->seeds, c->pvec, c->J, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "couplings launch");
  ++c->launches;
  c->env_built = false;
  c->use_nlimit = true;
  const size_t chains = (size_t)c->n_real * c->n_chains;
  e = cudaMemsetAsync(c->have_state, 0, sizeof(int) * chains, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(double) * (size_t)c->n_real * ACC_SLOTS, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->clamps, 0, sizeof(int64_t) * c->n_real, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->rstatus, 0, sizeof(unsigned) * c->n_real, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset");
  c->have_props = false;
  return TNMC_OK;
}

// Queue the device-to-host copies of a batch's results into the caller's pinned buffers
// (acc: n_real x ACC_SLOTS, clamps, logz: n_real, stats: 4 n_real, status: 1, rstatus: n_real).
tnmc_status ctx_enqueue_readback(tnmc_ctx* c, double* acc_h, int64_t* clamps_h, double* logz_h,
                                 long long* stats_h, unsigned* status_h, unsigned* rstatus_h) {
  const size_t R = (size_t)c->n_real;
  cudaError_t e = cudaMemcpyAsync(acc_h, c->acc, sizeof(double) * R * ACC_SLOTS, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(clamps_h, c->clamps, sizeof(int64_t) * R, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(logz_h, c->logz, sizeof(double) * R, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stats_h, c->stats, sizeof(long long) * 4 * R, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_h, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rstatus_h, c->rstatus, sizeof(unsigned) * R, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "result copy");
  return TNMC_OK;
}

int ctx_capacity(const tnmc_ctx* c) { return c->cap; }

tnmc_status ctx_alloc(tnmc_ctx* c, void** p, size_t bytes) { return dalloc(c, p, bytes); }

int8_t* ctx_couplings_dev(tnmc_ctx* c) { return c->J; }

tnmc_status ctx_use_fields_dev(tnmc_ctx* c, int8_t* fields_dev) {
  c->hfield = fields_dev;
  c->env_built = false;
  return TNMC_OK;
}

void ctx_set_chain_of(tnmc_ctx* c, const int* chain_of_dev) { c->chain_of = chain_of_dev; }

const uint32_t* ctx_packed(const tnmc_ctx* c) { return c->packed; }
const double* ctx_logq(const tnmc_ctx* c) { return c->logq; }
const int32_t* ctx_energy(const tnmc_ctx* c) { return c->energy; }
const unsigned* ctx_realization_status_dev(const tnmc_ctx* c) { return c->rstatus; }
const int64_t* ctx_clamps_dev(const tnmc_ctx* c) { return c->clamps; }
int ctx_words(const tnmc_ctx* c) { return c->words; }
void ctx_add_launches(tnmc_ctx* c, int64_t n) { c->launches += n; }

cudaStream_t ctx_stream(const tnmc_ctx* c) { return c->stream; }

void ctx_set_stream(tnmc_ctx* c, cudaStream_t st) { c->stream = st; }

void ctx_release(tnmc_ctx* c, cudaStream_t st) {
  if (!c) return;
  for (size_t i = 0; i < c->allocs.size(); ++i) release_block(c, c->allocs[i], c->alloc_sizes[i], st);
  if (c->h_stage) {
    tnmc::pinned_put(c->h_stage, (size_t)32 * c->cap * tnmc_ctx::kStageSlots);
    for (int k = 0; k < tnmc_ctx::kStageSlots; ++k) if (c->stage_ev[k]) cudaEventDestroy(c->stage_ev[k]);
  }
  delete c;
}

}  // namespace tnmc
