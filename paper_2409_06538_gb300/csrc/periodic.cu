// Periodic boundaries by a pinned pair of lines (Sec. IV of arXiv 2409.06538).
//
// On an L x L torus each step of each chain fixes a row i0 and a column j0 (Philox draws), keeps
// their spins, and samples the rest -- an (L-1) x (L-1) region with open boundaries -- with the
// open-boundary method: the fixed spins act on their neighbours in the region as external fields
// (integers k in units of beta), the region's environments are built with those fields, one
// configuration x' is proposed, and it replaces the current region configuration x with the
// Metropolis probability of the region's conditional distribution given the fixed lines:
//   Delta = [-beta E_reg(x') + beta k.x' - log q(x')] - [-beta E_reg(x) + beta k.x - log q(x)],
//   accept iff Delta >= 0 or u < exp(Delta).
// One inner open-lattice context holds one region per (realization, chain): a kernel writes the
// regions' couplings, fields and current configurations into it, the inner context builds the
// environments, proposes one configuration per region and evaluates log q of the current one
// teacher-forced, and a second kernel takes the Metropolis decisions, writes accepted regions
// back into the torus states and measures the observables of the torus.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tnmc.h"
#include "common.cuh"
#include "ctx_internal.h"
#include "kernels.h"

struct tnmc_periodic {
  int L = 0, Lr = 0, n_real = 0, n_chains = 1, n_therm = 0, chi = 0, precision = 0;
  cudaStream_t stream = nullptr;
  tnmc_ctx* inner = nullptr;       // n_real * n_chains open regions of side L - 1
  int8_t* Jt = nullptr;            // torus couplings [real][2 L^2]: Jh [L][L] then Jv [L][L]
  double* beta = nullptr;          // [real]
  uint64_t* seeds = nullptr;       // [real]
  int8_t* state = nullptr;         // torus states [real][chain][L^2], +-1
  int8_t* fields = nullptr;        // [slot][Lr^2] fields of the fixed lines, units of beta
  int8_t* current = nullptr;       // [slot][Lr^2] current region configurations
  int* lines = nullptr;            // [slot][2] (i0, j0) of the step
  int* chain_of = nullptr;         // [slot] chain index of the region's draws
  double* logq_cur = nullptr;      // [slot] teacher-forced log q of the current region configuration
  double* acc = nullptr;           // [real][ACC_SLOTS] accumulators
  unsigned* rstat = nullptr;       // [real] status bits
  int64_t launches = 0;
  std::string err;
};

namespace {

std::string g_periodic_err;

tnmc_status pfail(tnmc_periodic* p, tnmc_status s, const std::string& m) {
  if (p) p->err = m; else g_periodic_err = m;
  return s;
}

__device__ __forceinline__ int block_sum_int(int v, int* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = tnmc::warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0;
  if (warp == 0) t = tnmc::warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const int out = red[0];
  __syncthreads();
  return out;
}

__global__ void torus_couplings_kernel(int L, int n_real, const uint64_t* seeds, double p, int8_t* out) {
  const int64_t nb = 2ll * L * L, total = nb * n_real;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int real = (int)(i / nb);
    const double u = tnmc::uniform(seeds[real], (uint32_t)(i % nb), 0u, 0u, tnmc::PURPOSE_BOND);
    out[i] = u < p ? (int8_t)-1 : (int8_t)1;
  }
}

struct PrepArgs {
  int L, Lr, n_chains;
  uint32_t step;
  const int8_t* Jt; const uint64_t* seeds; const int8_t* state;
  int8_t* Jreg; int8_t* fields; int8_t* current; int* lines;
};

// One CTA per (realization, chain): the lines of the step and the region's open-lattice problem.
__global__ void periodic_prepare_kernel(PrepArgs a) {
  const int slot = blockIdx.x, real = slot / a.n_chains, ch = slot % a.n_chains;
  const int L = a.L, Lr = a.Lr, N = L * L, Nr = Lr * Lr;
  const uint64_t seed = a.seeds[real];
  const double u0 = tnmc::uniform(seed, 0u, a.step, (uint32_t)ch, tnmc::PURPOSE_LINES);
  const double u1 = tnmc::uniform(seed, 1u, a.step, (uint32_t)ch, tnmc::PURPOSE_LINES);
  const int i0 = min((int)(u0 * L), L - 1), j0 = min((int)(u1 * L), L - 1);
  if (threadIdx.x == 0) { a.lines[2 * slot] = i0; a.lines[2 * slot + 1] = j0; }
  const int8_t* JhT = a.Jt + (size_t)real * 2 * N;
  const int8_t* JvT = JhT + N;
  const int8_t* s = a.state + (size_t)slot * N;
  int8_t* JhR = a.Jreg + (size_t)slot * 2 * Lr * (Lr - 1);
  int8_t* JvR = JhR + (size_t)Lr * (Lr - 1);
  auto R = [&](int r) { return (i0 + 1 + r) % L; };
  auto C = [&](int c) { return (j0 + 1 + c) % L; };
  for (int e = threadIdx.x; e < Lr * (Lr - 1); e += blockDim.x) {
    const int r = e / (Lr - 1), c = e % (Lr - 1);
    JhR[e] = JhT[R(r) * L + C(c)];
  }
  for (int e = threadIdx.x; e < (Lr - 1) * Lr; e += blockDim.x) {
    const int r = e / Lr, c = e % Lr;
    JvR[e] = JvT[R(r) * L + C(c)];
  }
  const int im = (i0 - 1 + L) % L, jm = (j0 - 1 + L) % L;
  for (int i = threadIdx.x; i < Nr; i += blockDim.x) {
    const int r = i / Lr, c = i % Lr, tr = R(r), tc = C(c);
    int k = 0;
    if (r == 0) k += JvT[i0 * L + tc] * s[i0 * L + tc];          // row i0 above
    if (r == Lr - 1) k += JvT[im * L + tc] * s[i0 * L + tc];     // row i0 below (across the seam)
    if (c == 0) k += JhT[tr * L + j0] * s[tr * L + j0];          // column j0 to the left
    if (c == Lr - 1) k += JhT[tr * L + jm] * s[tr * L + j0];     // column j0 to the right
    a.fields[(size_t)slot * Nr + i] = (int8_t)k;
    a.current[(size_t)slot * Nr + i] = s[tr * L + tc];
  }
}

struct AccArgs {
  int L, Lr, n_chains, words, n_therm;
  uint32_t step;
  const double* beta; const uint64_t* seeds;
  const int8_t* Jreg; const int8_t* fields; const int8_t* current; const int* lines;
  const uint32_t* packed; const double* logq_new; const int32_t* energy_new; const double* logq_cur;
  const unsigned* inner_status; const int8_t* Jt;
  int8_t* state; double* acc; unsigned* rstat;
};

// One CTA per realization: each chain's Metropolis decision, the accepted regions written back
// into the torus states, then the observables of the torus states.
__global__ void __launch_bounds__(256) periodic_accept_kernel(AccArgs a) {
  __shared__ int red[32];
  __shared__ int ok_s;
  __shared__ double e_s[8], m_s[8];
  const int real = blockIdx.x, tid = threadIdx.x, nc = a.n_chains;
  const int L = a.L, Lr = a.Lr, N = L * L, Nr = Lr * Lr;
  const double beta = a.beta[real];
  int nacc = 0;
  for (int ch = 0; ch < nc; ++ch) {
    const int slot = real * nc + ch;
    const int8_t* JhR = a.Jreg + (size_t)slot * 2 * Lr * (Lr - 1);
    const int8_t* JvR = JhR + (size_t)Lr * (Lr - 1);
    const int8_t* k = a.fields + (size_t)slot * Nr;
    const int8_t* x = a.current + (size_t)slot * Nr;
    const uint32_t* xp = a.packed + (size_t)slot * a.words;
    auto newspin = [&](int i) { return ((xp[i >> 5] >> (i & 31)) & 1u) ? -1 : 1; };
    int ecur = 0, kxc = 0, kxn = 0;
    for (int i = tid; i < Nr; i += blockDim.x) {
      const int r = i / Lr, c = i % Lr;
      if (c < Lr - 1) ecur -= JhR[r * (Lr - 1) + c] * x[i] * x[i + 1];
      if (r < Lr - 1) ecur -= JvR[r * Lr + c] * x[i] * x[i + Lr];
      kxc += k[i] * x[i];
      kxn += k[i] * newspin(i);
    }
    ecur = block_sum_int(ecur, red);
    kxc = block_sum_int(kxc, red);
    kxn = block_sum_int(kxn, red);
    if (tid == 0) {
      const double enew = (double)a.energy_new[slot];
      const double delta = (-beta * enew + beta * kxn - a.logq_new[slot]) -
                           (-beta * (double)ecur + beta * kxc - a.logq_cur[slot]);
      const double u = tnmc::uniform(a.seeds[real], 0u, a.step, (uint32_t)ch, tnmc::PURPOSE_ACCEPT);
      ok_s = (delta >= 0.0) || (u < exp(delta));
      if (a.inner_status[slot] & tnmc::ST_NUMERIC) atomicOr(a.rstat + real, tnmc::ST_NUMERIC);
    }
    __syncthreads();
    if (ok_s) {
      const int i0 = a.lines[2 * slot], j0 = a.lines[2 * slot + 1];
      int8_t* s = a.state + (size_t)slot * N;
      for (int i = tid; i < Nr; i += blockDim.x) {
        const int r = i / Lr, c = i % Lr;
        s[((i0 + 1 + r) % L) * L + (j0 + 1 + c) % L] = (int8_t)newspin(i);
      }
      if (tid == 0) ++nacc;
    }
    __syncthreads();
  }
  // observables of the torus states after the step
  if ((int64_t)a.step < (int64_t)a.n_therm) {
    if (tid == 0) {
      double* acc = a.acc + (size_t)real * tnmc::ACC_SLOTS;
      acc[tnmc::ACC_NPROP] += nc; acc[tnmc::ACC_NTEST] += nc; acc[tnmc::ACC_NACC] += nacc;
    }
    return;
  }
  const int8_t* JhT = a.Jt + (size_t)real * 2 * N;
  const int8_t* JvT = JhT + N;
  for (int ch = 0; ch < nc; ++ch) {
    const int8_t* s = a.state + (size_t)(real * nc + ch) * N;
    int e = 0, m = 0;
    for (int i = tid; i < N; i += blockDim.x) {
      const int r = i / L, c = i % L;
      e -= JhT[i] * s[i] * s[r * L + (c + 1) % L] + JvT[i] * s[i] * s[((r + 1) % L) * L + c];
      m += s[i];
    }
    e = block_sum_int(e, red);
    m = block_sum_int(m, red);
    if (tid == 0 && ch < 8) { e_s[ch] = (double)e; m_s[ch] = (double)m / N; }
  }
  int ov = 0;
  if (nc >= 2) {
    const int8_t* s0 = a.state + (size_t)(real * nc) * N;
    const int8_t* s1 = s0 + N;
    for (int i = tid; i < N; i += blockDim.x) ov += s0[i] * s1[i];
    ov = block_sum_int(ov, red);
  }
  if (tid == 0) {
    double* acc = a.acc + (size_t)real * tnmc::ACC_SLOTS;
    acc[tnmc::ACC_NPROP] += nc; acc[tnmc::ACC_NTEST] += nc; acc[tnmc::ACC_NACC] += nacc;
    for (int ch = 0; ch < nc && ch < 8; ++ch) {
      const double E = e_s[ch], mm = m_s[ch], m2 = mm * mm;
      acc[tnmc::ACC_NMEAS] += 1.0;
      acc[tnmc::ACC_E] += E; acc[tnmc::ACC_E2] += E * E;
      acc[tnmc::ACC_MABS] += fabs(mm); acc[tnmc::ACC_M2] += m2; acc[tnmc::ACC_M4] += m2 * m2;
    }
    if (nc >= 2) {
      const double q = (double)ov / N, q2 = q * q;
      acc[tnmc::ACC_NMEASQ] += 1.0;
      acc[tnmc::ACC_Q] += q; acc[tnmc::ACC_QABS] += fabs(q); acc[tnmc::ACC_Q2] += q2; acc[tnmc::ACC_Q4] += q2 * q2;
    }
  }
}

__global__ void fill_kernel(int8_t* p, int64_t n, int8_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void iota_mod_kernel(int* p, int n, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i % m;
}

}  // namespace

extern "C" {

tnmc_status tnmc_torus_couplings_pmj(int L, int n_real, const uint64_t* seeds_host, double p, int8_t* out_dev,
                                     void* stream) {
  if (L < 3 || n_real < 1 || !seeds_host || !out_dev || !(p >= 0.0 && p <= 1.0))
    return pfail(nullptr, TNMC_ERR_ARG, "tnmc_torus_couplings_pmj: invalid argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* sd = nullptr;
  cudaError_t e = cudaMalloc(&sd, sizeof(uint64_t) * n_real);
  if (e != cudaSuccess) { cudaGetLastError(); return pfail(nullptr, TNMC_ERR_OOM, "seed buffer"); }
  e = cudaMemcpyAsync(sd, seeds_host, sizeof(uint64_t) * n_real, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    int64_t blocks = (2ll * L * L * n_real + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    torus_couplings_kernel<<<(unsigned)blocks, 256, 0, st>>>(L, n_real, sd, p, out_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(sd);
  if (e != cudaSuccess) return pfail(nullptr, TNMC_ERR_CUDA, std::string("torus couplings: ") + cudaGetErrorString(e));
  return TNMC_OK;
}

tnmc_status tnmc_periodic_create(int L, int n_real, const int8_t* couplings, const double* beta_host,
                                 const uint64_t* seeds_host, int chi, const tnmc_opts* opts, tnmc_periodic** out) {
  if (!out) return pfail(nullptr, TNMC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (L < 3 || L > 4097 || n_real < 1 || !couplings || !beta_host || !seeds_host || !opts)
    return pfail(nullptr, TNMC_ERR_ARG, "tnmc_periodic_create: invalid argument");
  if (opts->n_chains < 1 || opts->n_chains > 8) return pfail(nullptr, TNMC_ERR_ARG, "n_chains must be in [1, 8]");
  const size_t nbt = (size_t)2 * L * L * n_real;
  std::vector<int8_t> Jh(nbt);
  if (cudaMemcpy(Jh.data(), couplings, nbt, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return pfail(nullptr, TNMC_ERR_ARG, "couplings pointer is neither host nor device memory");
  }
  for (size_t i = 0; i < nbt; ++i)
    if (Jh[i] != 1 && Jh[i] != -1) return pfail(nullptr, TNMC_ERR_ARG, "couplings must be +1 or -1");
  tnmc_periodic* p = new tnmc_periodic();
  p->L = L; p->Lr = L - 1; p->n_real = n_real; p->n_chains = opts->n_chains; p->n_therm = opts->n_therm;
  p->chi = chi; p->precision = opts->precision;
  p->stream = reinterpret_cast<cudaStream_t>(opts->stream);
  const int Lr = L - 1, nslot = n_real * p->n_chains;
  // the inner context: one open region per (realization, chain), its couplings written per step
  std::vector<int8_t> J0((size_t)nslot * 2 * Lr * (Lr - 1), 1);
  std::vector<double> b0(nslot);
  std::vector<uint64_t> s0(nslot);
  for (int k = 0; k < nslot; ++k) { b0[k] = beta_host[k / p->n_chains]; s0[k] = seeds_host[k / p->n_chains]; }
  tnmc_opts io = *opts;
  io.n_chains = 1;
  io.n_therm = 0;
  tnmc_status st = tnmc_create(Lr, nslot, J0.data(), b0.data(), s0.data(), chi, &io, &p->inner);
  if (st) { g_periodic_err = tnmc_last_error(nullptr); delete p; return st; }
  tnmc_ctx* in = p->inner;
  const int Nr = Lr * Lr, N = L * L;
#define PALLOC(ptr, bytes) do { void* q_ = nullptr; if ((st = tnmc::ctx_alloc(in, &q_, (bytes)))) { g_periodic_err = tnmc_last_error(in); tnmc_periodic_destroy(p); return st; } ptr = reinterpret_cast<decltype(ptr)>(q_); } while (0)
  PALLOC(p->Jt, nbt);
  PALLOC(p->beta, sizeof(double) * n_real);
  PALLOC(p->seeds, sizeof(uint64_t) * n_real);
  PALLOC(p->state, (size_t)nslot * N);
  PALLOC(p->fields, (size_t)nslot * Nr);
  PALLOC(p->current, (size_t)nslot * Nr);
  PALLOC(p->lines, sizeof(int) * 2 * nslot);
  PALLOC(p->chain_of, sizeof(int) * nslot);
  PALLOC(p->logq_cur, sizeof(double) * nslot);
  PALLOC(p->acc, sizeof(double) * n_real * tnmc::ACC_SLOTS);
  PALLOC(p->rstat, sizeof(unsigned) * n_real);
#undef PALLOC
  cudaError_t e = cudaMemcpyAsync(p->Jt, Jh.data(), nbt, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->beta, beta_host, sizeof(double) * n_real, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->seeds, seeds_host, sizeof(uint64_t) * n_real, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) {
    fill_kernel<<<256, 256, 0, p->stream>>>(p->state, (int64_t)nslot * N, (int8_t)1);   // start from all spins up
    iota_mod_kernel<<<(nslot + 255) / 256, 256, 0, p->stream>>>(p->chain_of, nslot, p->n_chains);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(p->acc, 0, sizeof(double) * n_real * tnmc::ACC_SLOTS, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->rstat, 0, sizeof(unsigned) * n_real, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    g_periodic_err = std::string("periodic create: ") + cudaGetErrorString(e);
    tnmc_periodic_destroy(p);
    return TNMC_ERR_CUDA;
  }
  tnmc::ctx_use_fields_dev(in, p->fields);
  tnmc::ctx_set_chain_of(in, p->chain_of);
  p->launches = 2;
  *out = p;
  return TNMC_OK;
}

tnmc_status tnmc_periodic_step(tnmc_periodic* p, int n_steps, uint64_t step0) {
  if (!p) return pfail(nullptr, TNMC_ERR_ARG, "NULL context");
  if (n_steps < 1 || step0 + (uint64_t)n_steps > 0xFFFFFFFFull) return pfail(p, TNMC_ERR_ARG, "bad step range");
  const int Lr = p->Lr, nslot = p->n_real * p->n_chains;
  tnmc_ctx* in = p->inner;
  for (int s = 0; s < n_steps; ++s) {
    const uint32_t t = (uint32_t)(step0 + s);
    PrepArgs pa{p->L, Lr, p->n_chains, t, p->Jt, p->seeds, p->state, tnmc::ctx_couplings_dev(in), p->fields,
                p->current, p->lines};
    periodic_prepare_kernel<<<nslot, 128, 0, p->stream>>>(pa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(p, TNMC_ERR_CUDA, std::string("periodic prepare: ") + cudaGetErrorString(e));
    tnmc::ctx_use_fields_dev(in, p->fields);        // marks the environments stale
    tnmc_status st = tnmc_build_env(in, nullptr);
    if (!st) st = tnmc_propose(in, 1, t, nullptr, nullptr, nullptr);
    if (!st) st = tnmc_eval_conditionals(in, 1, p->current, p->logq_cur, nullptr);
    if (st) return pfail(p, st, std::string("region step: ") + tnmc_last_error(in));
    AccArgs aa{p->L, Lr, p->n_chains, tnmc::ctx_words(in), p->n_therm, t, p->beta, p->seeds,
               tnmc::ctx_couplings_dev(in), p->fields, p->current, p->lines, tnmc::ctx_packed(in),
               tnmc::ctx_logq(in), tnmc::ctx_energy(in), p->logq_cur, tnmc::ctx_realization_status_dev(in), p->Jt,
               p->state, p->acc, p->rstat};
    periodic_accept_kernel<<<p->n_real, 256, 0, p->stream>>>(aa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(p, TNMC_ERR_CUDA, std::string("periodic accept: ") + cudaGetErrorString(e));
    p->launches += 2;
  }
  return TNMC_OK;
}

tnmc_status tnmc_periodic_observables(tnmc_periodic* p, tnmc_obs* out_host) {
  if (!p || !out_host) return pfail(p, TNMC_ERR_ARG, "NULL argument");
  std::vector<double> acc((size_t)p->n_real * tnmc::ACC_SLOTS);
  std::vector<unsigned> rs(p->n_real);
  std::vector<int64_t> cl((size_t)p->n_real * p->n_chains);
  cudaError_t e = cudaMemcpyAsync(acc.data(), p->acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rs.data(), p->rstat, rs.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cl.data(), tnmc::ctx_clamps_dev(p->inner), cl.size() * sizeof(int64_t),
                                            cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return pfail(p, TNMC_ERR_CUDA, std::string("observables copy: ") + cudaGetErrorString(e));
  for (int k = 0; k < p->n_real; ++k) {
    int64_t c = 0;
    for (int ch = 0; ch < p->n_chains; ++ch) c += cl[(size_t)k * p->n_chains + ch];
    tnmc::obs_from_acc(&acc[(size_t)k * tnmc::ACC_SLOTS], c, &out_host[k]);
    out_host[k].status = (rs[k] & tnmc::ST_NUMERIC) ? TNMC_ERR_NUMERIC : TNMC_OK;
  }
  return TNMC_OK;
}

tnmc_status tnmc_periodic_get_spins(tnmc_periodic* p, int8_t* spins_dev) {
  if (!p || !spins_dev) return pfail(p, TNMC_ERR_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(spins_dev, p->state, (size_t)p->n_real * p->n_chains * p->L * p->L,
                                  cudaMemcpyDeviceToDevice, p->stream);
  if (e != cudaSuccess) return pfail(p, TNMC_ERR_CUDA, std::string("spins copy: ") + cudaGetErrorString(e));
  return TNMC_OK;
}

int64_t tnmc_periodic_launch_count(const tnmc_periodic* p) {
  return p ? p->launches + tnmc_launch_count(p->inner) : 0;
}

const char* tnmc_periodic_last_error(const tnmc_periodic* p) { return p ? p->err.c_str() : g_periodic_err.c_str(); }

tnmc_status tnmc_periodic_destroy(tnmc_periodic* p) {
  if (!p) return TNMC_OK;
  tnmc_destroy(p->inner);          // every buffer above came from the inner context
  delete p;
  return TNMC_OK;
}

}  // extern "C"
