// Metropolis correction of the independent tensor-network proposals (Eq. accptanceratio with
// g(s'|s) = q(s'); App. A works the same filter for the 1D ring) and the observables of
// Sec. III.C, plus the seeded +-J disorder generator (Sec. III.A) and spin unpacking.
#include "common.cuh"
#include "kernels.h"

namespace tnmc {

constexpr int kAcceptThreads = 256;

template <typename T> __device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : T(0);
  if (warp == 0) s = warp_sum(s);
  if (threadIdx.x == 0) red[0] = s;
  __syncthreads();
  const T out = red[0];
  __syncthreads();
  return out;
}

// Spins -1 among packed bits b0..b1 (inclusive) of one configuration (bit = site r*L + c).
__device__ __forceinline__ int neg_in_range(const uint32_t* sp, int b0, int b1) {
  int neg = 0;
  for (int w = b0 >> 5; w <= (b1 >> 5); ++w) {
    uint32_t x = sp[w];
    const int lo = (w == (b0 >> 5)) ? (b0 & 31) : 0, hi = (w == (b1 >> 5)) ? (b1 & 31) : 31;
    x >>= lo;
    const int nb = hi - lo + 1;
    if (nb < 32) x &= (1u << nb) - 1u;
    neg += __popc(x);
  }
  return neg;
}

// Edge magnetisation of Sec. III.C: (1/2L) times the sum of the spins on the four edge
// segments at 1-based positions i = L/4 ... 3L/4 (every integer in that closed interval).
__device__ __forceinline__ double edge_magnetisation(const uint32_t* sp, int L) {
  const int i0 = (L + 3) / 4 - 1, i1 = (3 * L) / 4 - 1;
  int neg = neg_in_range(sp, i0, i1) + neg_in_range(sp, (L - 1) * L + i0, (L - 1) * L + i1);
  for (int r = i0; r <= i1; ++r) {
    const int a = r * L, b = r * L + L - 1;
    neg += (int)((sp[a >> 5] >> (a & 31)) & 1u) + (int)((sp[b >> 5] >> (b & 31)) & 1u);
  }
  const int nseg = i1 - i0 + 1;
  return (double)(4 * nseg - 2 * neg) / (2.0 * L);
}

// One CTA per realization.  Phase 1: each chain's decisions in step order (one thread per
// chain).  Phase 2: observables of the current states after every step.  Phase 3: carry the
// final current state to the next call.
__global__ void __launch_bounds__(kAcceptThreads) accept_kernel(AcceptArgs a) {
  const int real = blockIdx.x;
  const int tid = threadIdx.x;
  const int n = a.n, nc = a.n_chains;
  const double beta = a.beta[real];
  const uint64_t seed = a.seeds[real];
  const int N = a.L * a.L;
  __shared__ double red[32];
  __shared__ double nacc_s[8];
  __shared__ double ntest_s[8];
  int* cur = a.cur_idx + (size_t)real * nc * n;
  // proposals of this call that the realization uses: all n, or what is left of its own
  // per-realization total after step0 (the rest is skipped as if never drawn)
  int lim = n;
  if (a.nlimit) {
    const long long left = (long long)a.nlimit[real] - (long long)a.step0;
    lim = left <= 0 ? 0 : (left < n ? (int)left : n);
  }

  if (tid < nc) {
    const int ch = tid;
    const size_t base = ((size_t)real * nc + ch) * n;
    const size_t sidx = (size_t)real * nc + ch;
    bool have = a.have_state[sidx] != 0;
    double cE = have ? (double)a.cur_energy[sidx] : 0.0;
    double cq = have ? a.cur_logq[sidx] : 0.0;
    int c = -1;
    int64_t nacc = 0, ntest = 0;
    for (int k = 0; k < n; ++k) {
      if (k >= lim) {                       // beyond this realization's own proposal count
        if (a.accepted) a.accepted[base + k] = 0;
        cur[(size_t)ch * n + k] = c;
        continue;
      }
      const double E = (double)a.energy[base + k], lq = a.logq[base + k];
      bool ok;
      if (!have) {
        ok = true;
      } else {
        const double delta = (-beta * E - lq) - (-beta * cE - cq);
        const double u = uniform(seed, 0u, (uint32_t)(a.step0 + k), (uint32_t)ch, PURPOSE_ACCEPT);
        ok = (delta >= 0.0) || (u < exp(delta));
        ++ntest;
        if (ok) ++nacc;
      }
      if (ok) { have = true; cE = E; cq = lq; c = k; }
      if (a.accepted) a.accepted[base + k] = ok ? 1 : 0;
      cur[(size_t)ch * n + k] = c;
    }
    nacc_s[ch] = (double)nacc;
    ntest_s[ch] = (double)ntest;
  }
  __syncthreads();

  // ---- phase 2: observables
  const double invN = 1.0 / (double)N;
  double sE = 0, sE2 = 0, sMa = 0, sM2 = 0, sM4 = 0, nm = 0, sEd = 0, sEda = 0, sEd2 = 0;
  // items are dealt to threads by (chain, step < lim), so the sums depend only on the
  // realization's own proposals, whatever the call's n
  for (int idx = tid; idx < nc * lim; idx += blockDim.x) {
    const int ch = idx / lim, k = idx % lim;
    if ((int64_t)(a.step0 + k) < (int64_t)a.n_therm) continue;
    const int c = cur[(size_t)ch * n + k];
    const size_t sidx = (size_t)real * nc + ch;
    if (c < 0 && !a.have_state[sidx]) continue;
    const double E = c >= 0 ? (double)a.energy[sidx * n + c] : (double)a.cur_energy[sidx];
    const double m = (c >= 0 ? (double)a.magnet[sidx * n + c] : (double)a.cur_magnet[sidx]) * invN;
    const double m2 = m * m;
    sE += E; sE2 += E * E; sMa += fabs(m); sM2 += m2; sM4 += m2 * m2; nm += 1.0;
    const uint32_t* sp = c >= 0 ? a.spins_packed + (sidx * n + c) * a.words : a.cur_spins + sidx * a.words;
    const double me = edge_magnetisation(sp, a.L);
    sEd += me; sEda += fabs(me); sEd2 += me * me;
  }
  double sq = 0, sqa = 0, sq2 = 0, sq4 = 0, nq = 0;
  if (nc >= 2) {
    for (int k = tid; k < n; k += blockDim.x) {
      if (k >= lim) continue;
      if ((int64_t)(a.step0 + k) < (int64_t)a.n_therm) continue;
      const int c0 = cur[k], c1 = cur[(size_t)n + k];
      const size_t s0 = (size_t)real * nc + 0, s1 = (size_t)real * nc + 1;
      if ((c0 < 0 && !a.have_state[s0]) || (c1 < 0 && !a.have_state[s1])) continue;
      const uint32_t* p0 = c0 >= 0 ? a.spins_packed + (s0 * n + c0) * a.words : a.cur_spins + s0 * a.words;
      const uint32_t* p1 = c1 >= 0 ? a.spins_packed + (s1 * n + c1) * a.words : a.cur_spins + s1 * a.words;
      int diff = 0;
      for (int w = 0; w < a.words; ++w) diff += __popc(p0[w] ^ p1[w]);
      const double q = (double)(N - 2 * diff) * invN;
      const double q2 = q * q;
      sq += q; sqa += fabs(q); sq2 += q2; sq4 += q2 * q2; nq += 1.0;
    }
  }
  sE = block_sum(sE, red); sE2 = block_sum(sE2, red); sMa = block_sum(sMa, red);
  sM2 = block_sum(sM2, red); sM4 = block_sum(sM4, red); nm = block_sum(nm, red);
  sq = block_sum(sq, red); sqa = block_sum(sqa, red); sq2 = block_sum(sq2, red);
  sq4 = block_sum(sq4, red); nq = block_sum(nq, red);
  sEd = block_sum(sEd, red); sEda = block_sum(sEda, red); sEd2 = block_sum(sEd2, red);
  if (tid == 0) {
    double* acc = a.acc + (size_t)real * ACC_SLOTS;
    double na = 0, nt = 0;
    for (int ch = 0; ch < nc && ch < 8; ++ch) { na += nacc_s[ch]; nt += ntest_s[ch]; }
    acc[ACC_NPROP] += (double)nc * lim;
    acc[ACC_NACC] += na;
    acc[ACC_NTEST] += nt;
    acc[ACC_NMEAS] += nm;
    acc[ACC_NMEASQ] += nq;
    acc[ACC_E] += sE; acc[ACC_E2] += sE2; acc[ACC_MABS] += sMa; acc[ACC_M2] += sM2; acc[ACC_M4] += sM4;
    acc[ACC_Q] += sq; acc[ACC_QABS] += sqa; acc[ACC_Q2] += sq2; acc[ACC_Q4] += sq4;
    acc[ACC_MEDGE] += sEd; acc[ACC_MEDGEABS] += sEda; acc[ACC_MEDGE2] += sEd2;
  }
  __syncthreads();

  // ---- phase 3: carry the current states
  for (int ch = 0; ch < nc; ++ch) {
    const int c = cur[(size_t)ch * n + n - 1];
    if (c < 0) continue;
    const size_t sidx = (size_t)real * nc + ch;
    const uint32_t* src = a.spins_packed + (sidx * n + c) * a.words;
    for (int w = tid; w < a.words; w += blockDim.x) a.cur_spins[sidx * a.words + w] = src[w];
    if (tid == 0) {
      a.have_state[sidx] = 1;
      a.cur_energy[sidx] = a.energy[sidx * n + c];
      a.cur_logq[sidx] = a.logq[sidx * n + c];
      a.cur_magnet[sidx] = a.magnet[sidx * n + c];
    }
  }
}

cudaError_t launch_accept(const AcceptArgs& a, cudaStream_t st) {
  if (a.n_chains < 1 || a.n_chains > 8) return cudaErrorInvalidValue;
  accept_kernel<<<a.n_real, kAcceptThreads, 0, st>>>(a);
  return cudaGetLastError();
}

__global__ void couplings_kernel(int L, int n_real, const uint64_t* seeds, double p, const double* pvec, int8_t* out) {
  const int64_t nb = 2ll * L * (L - 1);
  const int64_t total = nb * n_real;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int real = (int)(i / nb);
    const uint32_t b = (uint32_t)(i % nb);
    const double u = uniform(seeds[real], b, 0u, 0u, PURPOSE_BOND);
    out[i] = (u < (pvec ? pvec[real] : p)) ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_couplings(int L, int n_real, const uint64_t* seeds_dev, double p, int8_t* out,
                             cudaStream_t st) {
  const int64_t total = 2ll * L * (L - 1) * n_real;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  couplings_kernel<<<(unsigned)blocks, 256, 0, st>>>(L, n_real, seeds_dev, p, nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_couplings_pvec(int L, int n_real, const uint64_t* seeds_dev, const double* p_dev, int8_t* out,
                                  cudaStream_t st) {
  const int64_t total = 2ll * L * (L - 1) * n_real;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  couplings_kernel<<<(unsigned)blocks, 256, 0, st>>>(L, n_real, seeds_dev, 0.0, p_dev, out);
  return cudaGetLastError();
}

__global__ void unpack_kernel(const uint32_t* packed, int words, int N, int64_t n_cfg, int8_t* out) {
  const int64_t total = n_cfg * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cfg = i / N;
    const int site = (int)(i % N);
    const uint32_t w = packed[cfg * words + (site >> 5)];
    out[i] = ((w >> (site & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_unpack(const uint32_t* packed, int words, int N, int64_t n_cfg, int8_t* out,
                          cudaStream_t st) {
  int64_t blocks = (n_cfg * N + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  unpack_kernel<<<(unsigned)blocks, 256, 0, st>>>(packed, words, N, n_cfg, out);
  return cudaGetLastError();
}

}  // namespace tnmc
