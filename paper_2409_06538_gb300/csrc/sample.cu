// Autoregressive proposals from the cached row environments (Sec. II.A Eq. approximate_bayes,
// Sec. II.B reverse-order sampling, Figs. fig:Z4 / fig:ZS4), and the same sweep with given
// spins (teacher forcing) for q(s) of arbitrary configurations.
//
// One warp per proposal, lanes over the bond index; the CTA's warps are NW proposals of the
// same realization and share every environment tile, staged once per site into shared
// memory with cp.async double buffering.  For row r (fields h_c = beta Jv[r-1][c] s_{r-1,c}):
//   right sweep  c = L-1..0 : v_y = B[c]^y R_{c+1}(y), stored to the warp's workspace;
//                 R_c(y') = sum_y exp(beta Jh[r][c-1] s_y' s_y + h_c s_y) v_y (jointly normalised)
//   left sweep   c = 0..L-1 : w(y) = exp(h_c s_y + beta Jh[r][c-1] s_{c-1} s_y) (l . v_y),
//                 clamp w >= 0, q(+) = w+/(w+ + w-), s = +1 iff u < q(+) with u the Philox
//                 uniform of counter (r*L+c, step, chain, 1); log q accumulates in FP64;
//                 l <- l B[c]^s (normalised).
#include "common.cuh"
#include "kernels.h"

namespace tnmc {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// The draw s = +1 iff u < q(+), u = m 2^-53 with m the 53-bit Philox integer.
// FP64 path: compared in double.  FP32 paths: the same comparison done exactly in integers,
// m < ceil(q 2^53), so that no FP64 instruction runs per lane.
__device__ __forceinline__ uint64_t philox_m53(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2) {
  const Philox4 o = philox4x32_10(c0, c1, c2, PURPOSE_SPIN, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((uint64_t)(o.x0 >> 5) << 26) | (uint64_t)(o.x1 >> 6);
}
__device__ __forceinline__ bool below(uint64_t m, double q) { return (double)m * (1.0 / 9007199254740992.0) < q; }
__device__ __forceinline__ bool below(uint64_t m, float q) {
  if (!(q > 0.0f)) return false;
  if (q >= 1.0f) return true;
  const uint32_t bits = __float_as_uint(q);
  const int e = (int)((bits >> 23) & 0xffu);
  const uint64_t mant = (e == 0) ? (uint64_t)(bits & 0x7fffffu) : (uint64_t)((bits & 0x7fffffu) | 0x800000u);
  const int sh = (e == 0 ? 1 : e) - 150 + 53;          // q 2^53 = mant 2^sh, sh <= 29 for q < 1
  uint64_t C;
  if (sh >= 0) C = mant << sh;
  else { const int k = -sh; C = (k >= 64) ? 1ull : ((mant + ((1ull << k) - 1ull)) >> k); }
  return m < C;
}
// log of the chosen conditional, accurate for q near 1 (log1p of the other branch)
__device__ __forceinline__ double log_q(double qs, double qo) { return qs > 0.5 ? log1p(-qo) : log(qs); }
__device__ __forceinline__ float log_q(float qs, float qo) { return qs > 0.5f ? log1pf(-qo) : logf(qs); }

template <typename T, typename TE, int CHI, int NW>
__global__ void __launch_bounds__(32 * NW)
sample_kernel(SampleArgs a) {
  constexpr int TILE = 2 * CHI * CHI;
  constexpr int NT = 32 * NW;
  constexpr int CHUNKS = TILE * (int)sizeof(TE) / 16;
  const int L = a.L, N = L * L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int al = lane & (CHI - 1);            // bond index handled by this lane
  const bool active_lane = lane < CHI;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  TE* stage0 = reinterpret_cast<TE*>(smem_raw);
  TE* stage1 = stage0 + TILE;
  int8_t* jh_s = reinterpret_cast<int8_t*>(stage1 + TILE);   // L
  int8_t* jv_s = jh_s + L;                                    // L
  int8_t* rows = jv_s + L;                                    // [NW][2][L]

  const int tiles_per_real = (a.n_items + NW - 1) / NW;
  const int64_t total = (int64_t)tiles_per_real * a.n_real;
  T* work = reinterpret_cast<T*>(a.work) + ((size_t)blockIdx.x * NW + warp) * (size_t)L * 2 * CHI;

  for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int real = (int)(tile / tiles_per_real);
    const int k = (int)(tile % tiles_per_real) * NW + warp;
    const bool valid = k < a.n_items;
    const int64_t item = (int64_t)real * a.n_items + k;
    const int chain = a.forced ? 0 : (a.chain_of ? a.chain_of[real] : k / a.n);
    const uint32_t step = (uint32_t)(a.step0 + (uint64_t)(a.forced ? 0 : k % a.n));
    const uint64_t seed = a.seeds[real];
    const double betad = a.beta[real];
    const T eb = (T)exp(betad), ebm = (T)exp(-betad);
    const int8_t* J = a.J + (size_t)real * 2 * L * (L - 1);
    const TE* envr = reinterpret_cast<const TE*>(a.env) + (size_t)real * L * L * TILE;
    int8_t* prow = rows + (size_t)warp * 2 * L;      // previous row spins
    int8_t* crow = prow + L;                          // current row spins
    const int8_t* forced = (a.forced && valid) ? a.forced + (size_t)item * N : nullptr;
    const int8_t* hf = a.hfield ? a.hfield + (size_t)real * N : nullptr;

    double logq = 0.0;          // FP64 total
    int energy = 0, magnet = 0;
    int64_t nclamp = 0;
    uint32_t word = 0;

    for (int r = 0; r < L; ++r) {
      __syncthreads();   // previous users of jh_s/jv_s/rows are done
      for (int c = tid; c < L - 1; c += NT) jh_s[c] = J[(size_t)r * (L - 1) + c];
      if (r > 0)
        for (int c = tid; c < L; c += NT) jv_s[c] = J[(size_t)L * (L - 1) + (size_t)(r - 1) * L + c];
      const TE* erow = envr + (size_t)r * L * TILE;

      // ---------------- right sweep ----------------
      T R0 = (al == 0 && active_lane) ? T(1) : T(0), R1 = R0;   // R_L(y) for y = 0, 1
      for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(stage0) + 16 * i,
                                                        reinterpret_cast<const char*>(erow + (size_t)(L - 1) * TILE) + 16 * i);
      cp_async_commit();
      for (int ci = 0; ci < L; ++ci) {
        const int c = L - 1 - ci;
        cp_async_wait_all();
        __syncthreads();
        const TE* tl = (ci & 1) ? stage1 : stage0;
        if (ci + 1 < L) {
          TE* nx = (ci & 1) ? stage0 : stage1;
          for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(nx) + 16 * i,
                                                            reinterpret_cast<const char*>(erow + (size_t)(c - 1) * TILE) + 16 * i);
          cp_async_commit();
        }
        // v_y[al] = sum_be B^y[al][be] R(y)[be]  (diagonal order: conflict-free smem reads)
        T v0 = 0, v1 = 0;
#pragma unroll 8
        for (int t = 0; t < CHI; ++t) {
          const int be = (al + t) & (CHI - 1);
          const T r0 = __shfl_sync(0xffffffffu, R0, be);
          const T r1 = __shfl_sync(0xffffffffu, R1, be);
          v0 += env_load<T, TE>(tl[al * CHI + be]) * r0;
          v1 += env_load<T, TE>(tl[CHI * CHI + al * CHI + be]) * r1;
        }
        if (!active_lane) { v0 = 0; v1 = 0; }
        if (active_lane) { work[(size_t)c * 2 * CHI + al] = v0; work[(size_t)c * 2 * CHI + CHI + al] = v1; }
        if (c > 0) {
          // R_c(y') = sum_y exp(beta Jh s_y' s_y) exp(h_c s_y) v_y
          const int jh = jh_s[c - 1];
          T f0 = 1, f1 = 1;                     // exp(h_c s_y) for y = 0 (+1), 1 (-1)
          if (r > 0) { const int sg = jv_s[c] * prow[c]; f0 = sg > 0 ? eb : ebm; f1 = sg > 0 ? ebm : eb; }
          if (hf) { const int kh = hf[(size_t)r * L + c]; if (kh) { f0 *= num<T>::exp_((T)(betad * kh)); f1 *= num<T>::exp_((T)(-betad * kh)); } }
          const T same = jh > 0 ? eb : ebm, diff = jh > 0 ? ebm : eb;
          const T n0 = same * f0 * v0 + diff * f1 * v1;   // y' = +1
          const T n1 = diff * f0 * v0 + same * f1 * v1;   // y' = -1
          T mx = tabs(n0) > tabs(n1) ? tabs(n0) : tabs(n1);
          mx = warp_max(mx);
          const T inv = mx > T(0) ? T(1) / mx : T(1);
          R0 = n0 * inv; R1 = n1 * inv;
        }
      }
      __syncwarp();

      // ---------------- left sweep ----------------
      T ell = (al == 0 && active_lane) ? T(1) : T(0);
      int sprev = 0;
      T rsum = 0, rcomp = 0;      // compensated row sum of log q terms
      for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(stage0) + 16 * i,
                                                        reinterpret_cast<const char*>(erow) + 16 * i);
      cp_async_commit();
      for (int c = 0; c < L; ++c) {
        cp_async_wait_all();
        __syncthreads();
        const TE* tl = (c & 1) ? stage1 : stage0;
        if (c + 1 < L) {
          TE* nx = (c & 1) ? stage0 : stage1;
          for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(nx) + 16 * i,
                                                            reinterpret_cast<const char*>(erow + (size_t)(c + 1) * TILE) + 16 * i);
          cp_async_commit();
        }
        const T v0 = active_lane ? work[(size_t)c * 2 * CHI + al] : T(0);
        const T v1 = active_lane ? work[(size_t)c * 2 * CHI + CHI + al] : T(0);
        T d0 = warp_sum(ell * v0), d1 = warp_sum(ell * v1);
        T f0 = 1, f1 = 1;
        if (r > 0) { const int sg = jv_s[c] * prow[c]; f0 = sg > 0 ? eb : ebm; f1 = sg > 0 ? ebm : eb; }
        if (c > 0) { const int sg = jh_s[c - 1] * sprev; f0 *= sg > 0 ? eb : ebm; f1 *= sg > 0 ? ebm : eb; }
        if (hf) { const int kh = hf[(size_t)r * L + c]; if (kh) { f0 *= num<T>::exp_((T)(betad * kh)); f1 *= num<T>::exp_((T)(-betad * kh)); } }
        T w0 = f0 * d0, w1 = f1 * d1;
        if (w0 < T(0)) { w0 = 0; ++nclamp; }
        if (w1 < T(0)) { w1 = 0; ++nclamp; }
        const T tot = w0 + w1;
        int s;
        T qp = T(0.5), lqs;
        if (!(tot > T(0)) || !isfinite(tot)) {
          if (lane == 0 && valid) {
            set_status(a.status, ST_NUMERIC);
            if (a.real_status) set_status(a.real_status + real, ST_NUMERIC);
          }
          // the realization is flagged; the spin is still drawn from the q = 1/2 it logs,
          // so that log q stays the probability the proposal was drawn with
          if (forced) s = forced[(size_t)r * L + c];
          else s = (philox_m53(seed, (uint32_t)(r * L + c), step, (uint32_t)chain) < (1ull << 52)) ? 1 : -1;
          lqs = T(-0.6931471805599453);
        } else {
          qp = w0 / tot;
          const T qm = w1 / tot;
          if (forced) {
            s = forced[(size_t)r * L + c];
          } else {
            s = below(philox_m53(seed, (uint32_t)(r * L + c), step, (uint32_t)chain), qp) ? 1 : -1;
          }
          lqs = (s == 1) ? log_q(qp, qm) : log_q(qm, qp);
        }
        {   // Kahan: the row's log q terms summed with FP64-grade accuracy in the compute type
          const T yk = lqs - rcomp;
          const T tk = rsum + yk;
          rcomp = (tk - rsum) - yk;
          rsum = tk;
        }
        if (a.qplus && valid && lane == 0) a.qplus[(size_t)item * N + (size_t)r * L + c] = (double)qp;
        // l <- l B^s
        const TE* bs = tl + (s == 1 ? 0 : CHI * CHI);
        T acc = 0;
#pragma unroll 8
        for (int t = 0; t < CHI; ++t) {
          const T lt = __shfl_sync(0xffffffffu, ell, t);
          acc += lt * env_load<T, TE>(bs[t * CHI + al]);
        }
        if (!active_lane) acc = 0;
        T mx = warp_max(tabs(acc));
        ell = mx > T(0) ? acc / mx : acc;
        // energy and magnetisation (Eq. E)
        if (c > 0) energy -= jh_s[c - 1] * sprev * s;
        if (r > 0) energy -= jv_s[c] * prow[c] * s;
        magnet += s;
        if (lane == 0) crow[c] = (int8_t)s;
        sprev = s;
        const int site = r * L + c;
        if (s < 0) word |= 1u << (site & 31);
        if ((site & 31) == 31 || site == N - 1) {
          if (lane == 0 && valid && a.spins_packed) a.spins_packed[(size_t)item * a.words + (site >> 5)] = word;
          word = 0;
        }
      }
      logq += (double)rsum;
      __syncwarp();
      for (int c = lane; c < L; c += 32) prow[c] = crow[c];
      __syncwarp();
    }
    if (lane == 0 && valid) {
      if (a.logq) a.logq[item] = logq;
      if (a.energy) a.energy[item] = energy;
      if (a.magnet) a.magnet[item] = magnet;
      if (a.clamps && nclamp) atomicAdd(reinterpret_cast<unsigned long long*>(a.clamps + real),
                                        (unsigned long long)nclamp);
    }
  }
}

// The same sweep for CHI = 64 (bond indices lane and lane + 32 on each lane).
template <typename T, typename TE, int CHI, int NW>
__global__ void __launch_bounds__(32 * NW)
sample_kernel_wide(SampleArgs a) {
  constexpr int E = CHI / 32;                 // bond indices per lane: lane + 32 e
  constexpr int TILE = 2 * CHI * CHI;
  constexpr int NT = 32 * NW;
  constexpr int CHUNKS = TILE * (int)sizeof(TE) / 16;
  const int L = a.L, N = L * L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  TE* stage0 = reinterpret_cast<TE*>(smem_raw);
  TE* stage1 = stage0 + TILE;
  int8_t* jh_s = reinterpret_cast<int8_t*>(stage1 + TILE);   // L
  int8_t* jv_s = jh_s + L;                                    // L
  int8_t* rows = jv_s + L;                                    // [NW][2][L]

  const int tiles_per_real = (a.n_items + NW - 1) / NW;
  const int64_t total = (int64_t)tiles_per_real * a.n_real;
  T* work = reinterpret_cast<T*>(a.work) + ((size_t)blockIdx.x * NW + warp) * (size_t)L * 2 * CHI;

  for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int real = (int)(tile / tiles_per_real);
    const int k = (int)(tile % tiles_per_real) * NW + warp;
    const bool valid = k < a.n_items;
    const int64_t item = (int64_t)real * a.n_items + k;
    const int chain = a.forced ? 0 : (a.chain_of ? a.chain_of[real] : k / a.n);
    const uint32_t step = (uint32_t)(a.step0 + (uint64_t)(a.forced ? 0 : k % a.n));
    const uint64_t seed = a.seeds[real];
    const double betad = a.beta[real];
    const T eb = (T)exp(betad), ebm = (T)exp(-betad);
    const int8_t* J = a.J + (size_t)real * 2 * L * (L - 1);
    const TE* envr = reinterpret_cast<const TE*>(a.env) + (size_t)real * L * L * TILE;
    int8_t* prow = rows + (size_t)warp * 2 * L;      // previous row spins
    int8_t* crow = prow + L;                          // current row spins
    const int8_t* forced = (a.forced && valid) ? a.forced + (size_t)item * N : nullptr;
    const int8_t* hf = a.hfield ? a.hfield + (size_t)real * N : nullptr;

    double logq = 0.0;          // FP64 total
    int energy = 0, magnet = 0;
    int64_t nclamp = 0;
    uint32_t word = 0;

    for (int r = 0; r < L; ++r) {
      __syncthreads();   // previous users of jh_s/jv_s/rows are done
      for (int c = tid; c < L - 1; c += NT) jh_s[c] = J[(size_t)r * (L - 1) + c];
      if (r > 0)
        for (int c = tid; c < L; c += NT) jv_s[c] = J[(size_t)L * (L - 1) + (size_t)(r - 1) * L + c];
      const TE* erow = envr + (size_t)r * L * TILE;

      // ---------------- right sweep ----------------
      T R0[E], R1[E];                                   // R_L(y) for y = 0, 1
#pragma unroll
      for (int e = 0; e < E; ++e) { R0[e] = (lane == 0 && e == 0) ? T(1) : T(0); R1[e] = R0[e]; }
      for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(stage0) + 16 * i,
                                                        reinterpret_cast<const char*>(erow + (size_t)(L - 1) * TILE) + 16 * i);
      cp_async_commit();
      for (int ci = 0; ci < L; ++ci) {
        const int c = L - 1 - ci;
        cp_async_wait_all();
        __syncthreads();
        const TE* tl = (ci & 1) ? stage1 : stage0;
        if (ci + 1 < L) {
          TE* nx = (ci & 1) ? stage0 : stage1;
          for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(nx) + 16 * i,
                                                            reinterpret_cast<const char*>(erow + (size_t)(c - 1) * TILE) + 16 * i);
          cp_async_commit();
        }
        // v_y[al] = sum_be B^y[al][be] R(y)[be] for al = lane + 32 e (diagonal order within
        // each half of be: conflict-free smem reads)
        T v0[E], v1[E];
#pragma unroll
        for (int e = 0; e < E; ++e) { v0[e] = 0; v1[e] = 0; }
#pragma unroll
        for (int h = 0; h < E; ++h) {
#pragma unroll 8
          for (int t = 0; t < 32; ++t) {
            const int j = (lane + t) & 31, be = 32 * h + j;
            const T r0 = __shfl_sync(0xffffffffu, R0[h], j);
            const T r1 = __shfl_sync(0xffffffffu, R1[h], j);
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int al = lane + 32 * e;
              v0[e] += env_load<T, TE>(tl[al * CHI + be]) * r0;
              v1[e] += env_load<T, TE>(tl[CHI * CHI + al * CHI + be]) * r1;
            }
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          work[(size_t)c * 2 * CHI + lane + 32 * e] = v0[e];
          work[(size_t)c * 2 * CHI + CHI + lane + 32 * e] = v1[e];
        }
        if (c > 0) {
          // R_c(y') = sum_y exp(beta Jh s_y' s_y) exp(h_c s_y) v_y
          const int jh = jh_s[c - 1];
          T f0 = 1, f1 = 1;                     // exp(h_c s_y) for y = 0 (+1), 1 (-1)
          if (r > 0) { const int sg = jv_s[c] * prow[c]; f0 = sg > 0 ? eb : ebm; f1 = sg > 0 ? ebm : eb; }
          if (hf) { const int kh = hf[(size_t)r * L + c]; if (kh) { f0 *= num<T>::exp_((T)(betad * kh)); f1 *= num<T>::exp_((T)(-betad * kh)); } }
          const T same = jh > 0 ? eb : ebm, diff = jh > 0 ? ebm : eb;
          T n0[E], n1[E], mx = 0;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            n0[e] = same * f0 * v0[e] + diff * f1 * v1[e];   // y' = +1
            n1[e] = diff * f0 * v0[e] + same * f1 * v1[e];   // y' = -1
            mx = tabs(n0[e]) > mx ? tabs(n0[e]) : mx;
            mx = tabs(n1[e]) > mx ? tabs(n1[e]) : mx;
          }
          mx = warp_max(mx);
          const T inv = mx > T(0) ? T(1) / mx : T(1);
#pragma unroll
          for (int e = 0; e < E; ++e) { R0[e] = n0[e] * inv; R1[e] = n1[e] * inv; }
        }
      }
      __syncwarp();

      // ---------------- left sweep ----------------
      T ell[E];
#pragma unroll
      for (int e = 0; e < E; ++e) ell[e] = (lane == 0 && e == 0) ? T(1) : T(0);
      int sprev = 0;
      T rsum = 0, rcomp = 0;      // compensated row sum of log q terms
      for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(stage0) + 16 * i,
                                                        reinterpret_cast<const char*>(erow) + 16 * i);
      cp_async_commit();
      for (int c = 0; c < L; ++c) {
        cp_async_wait_all();
        __syncthreads();
        const TE* tl = (c & 1) ? stage1 : stage0;
        if (c + 1 < L) {
          TE* nx = (c & 1) ? stage0 : stage1;
          for (int i = tid; i < CHUNKS; i += NT) cp_async16(reinterpret_cast<char*>(nx) + 16 * i,
                                                            reinterpret_cast<const char*>(erow + (size_t)(c + 1) * TILE) + 16 * i);
          cp_async_commit();
        }
        T p0 = 0, p1 = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          p0 += ell[e] * work[(size_t)c * 2 * CHI + lane + 32 * e];
          p1 += ell[e] * work[(size_t)c * 2 * CHI + CHI + lane + 32 * e];
        }
        T d0 = warp_sum(p0), d1 = warp_sum(p1);
        T f0 = 1, f1 = 1;
        if (r > 0) { const int sg = jv_s[c] * prow[c]; f0 = sg > 0 ? eb : ebm; f1 = sg > 0 ? ebm : eb; }
        if (c > 0) { const int sg = jh_s[c - 1] * sprev; f0 *= sg > 0 ? eb : ebm; f1 *= sg > 0 ? ebm : eb; }
        if (hf) { const int kh = hf[(size_t)r * L + c]; if (kh) { f0 *= num<T>::exp_((T)(betad * kh)); f1 *= num<T>::exp_((T)(-betad * kh)); } }
        T w0 = f0 * d0, w1 = f1 * d1;
        if (w0 < T(0)) { w0 = 0; ++nclamp; }
        if (w1 < T(0)) { w1 = 0; ++nclamp; }
        const T tot = w0 + w1;
        int s;
        T qp = T(0.5), lqs;
        if (!(tot > T(0)) || !isfinite(tot)) {
          if (lane == 0 && valid) {
            set_status(a.status, ST_NUMERIC);
            if (a.real_status) set_status(a.real_status + real, ST_NUMERIC);
          }
          // the realization is flagged; the spin is still drawn from the q = 1/2 it logs,
          // so that log q stays the probability the proposal was drawn with
          if (forced) s = forced[(size_t)r * L + c];
          else s = (philox_m53(seed, (uint32_t)(r * L + c), step, (uint32_t)chain) < (1ull << 52)) ? 1 : -1;
          lqs = T(-0.6931471805599453);
        } else {
          qp = w0 / tot;
          const T qm = w1 / tot;
          if (forced) {
            s = forced[(size_t)r * L + c];
          } else {
            s = below(philox_m53(seed, (uint32_t)(r * L + c), step, (uint32_t)chain), qp) ? 1 : -1;
          }
          lqs = (s == 1) ? log_q(qp, qm) : log_q(qm, qp);
        }
        {   // Kahan: the row's log q terms summed with FP64-grade accuracy in the compute type
          const T yk = lqs - rcomp;
          const T tk = rsum + yk;
          rcomp = (tk - rsum) - yk;
          rsum = tk;
        }
        if (a.qplus && valid && lane == 0) a.qplus[(size_t)item * N + (size_t)r * L + c] = (double)qp;
        // l <- l B^s
        const TE* bs = tl + (s == 1 ? 0 : CHI * CHI);
        T acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0;
#pragma unroll
        for (int h = 0; h < E; ++h) {
#pragma unroll 8
          for (int j = 0; j < 32; ++j) {
            const T lt = __shfl_sync(0xffffffffu, ell[h], j);
            const int t = 32 * h + j;
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] += lt * env_load<T, TE>(bs[t * CHI + lane + 32 * e]);
          }
        }
        T mx = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) mx = tabs(acc[e]) > mx ? tabs(acc[e]) : mx;
        mx = warp_max(mx);
#pragma unroll
        for (int e = 0; e < E; ++e) ell[e] = mx > T(0) ? acc[e] / mx : acc[e];
        // energy and magnetisation (Eq. E)
        if (c > 0) energy -= jh_s[c - 1] * sprev * s;
        if (r > 0) energy -= jv_s[c] * prow[c] * s;
        magnet += s;
        if (lane == 0) crow[c] = (int8_t)s;
        sprev = s;
        const int site = r * L + c;
        if (s < 0) word |= 1u << (site & 31);
        if ((site & 31) == 31 || site == N - 1) {
          if (lane == 0 && valid && a.spins_packed) a.spins_packed[(size_t)item * a.words + (site >> 5)] = word;
          word = 0;
        }
      }
      logq += (double)rsum;
      __syncwarp();
      for (int c = lane; c < L; c += 32) prow[c] = crow[c];
      __syncwarp();
    }
    if (lane == 0 && valid) {
      if (a.logq) a.logq[item] = logq;
      if (a.energy) a.energy[item] = energy;
      if (a.magnet) a.magnet[item] = magnet;
      if (a.clamps && nclamp) atomicAdd(reinterpret_cast<unsigned long long*>(a.clamps + real),
                                        (unsigned long long)nclamp);
    }
  }
}

template <int CHI, int NW>
static size_t sample_smem(int L, size_t te) {
  return 2 * (size_t)(2 * CHI * CHI) * te + 2 * (size_t)L + (size_t)NW * 2 * L + 16;
}

constexpr int kSampleWarps = 8;

template <typename T, typename TE, int CHI>
static cudaError_t launch_sample_t(const SampleArgs& a, int num_sms, cudaStream_t st) {
  constexpr int NW = kSampleWarps;
  const size_t smem = sample_smem<CHI, NW>(a.L, sizeof(TE));
  void (*kern)(SampleArgs);
  if constexpr (CHI > 32) kern = sample_kernel_wide<T, TE, CHI, NW>;
  else kern = sample_kernel<T, TE, CHI, NW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * NW, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  const int64_t tiles = (int64_t)((a.n_items + NW - 1) / NW) * a.n_real;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 32 * NW, smem, st>>>(a);
  return cudaGetLastError();
}

size_t sample_work_bytes(int L, int CHI, int precision, int num_sms) {
  const size_t el = precision == 0 ? 8 : 4;
  return (size_t)num_sms * 4 * kSampleWarps * (size_t)L * 2 * CHI * el;
}

cudaError_t launch_sample(const SampleArgs& a, int precision, int CHI, int num_sms, cudaStream_t st) {
#define TNMC_SAMPLE_CASE(T, TE)                                        \
  switch (CHI) {                                                       \
    case 4: return launch_sample_t<T, TE, 4>(a, num_sms, st);          \
    case 8: return launch_sample_t<T, TE, 8>(a, num_sms, st);          \
    case 16: return launch_sample_t<T, TE, 16>(a, num_sms, st);        \
    case 32: return launch_sample_t<T, TE, 32>(a, num_sms, st);        \
    case 64: return launch_sample_t<T, TE, 64>(a, num_sms, st);        \
    default: return cudaErrorInvalidValue;                             \
  }
  if (precision == 0) {
    if (CHI > 32) return cudaErrorInvalidValue;     // the FP64 build stops at CHI = 32
    TNMC_SAMPLE_CASE(double, double)
  }
  if (precision == 2) { TNMC_SAMPLE_CASE(float, __nv_bfloat16) }
  TNMC_SAMPLE_CASE(float, float)
#undef TNMC_SAMPLE_CASE
}

}  // namespace tnmc
