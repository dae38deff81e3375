// Tensor-core sampling sweep for the mixed-precision path (sm_103a tcgen05).
//
// The same autoregressive sweep as sample.cu (Sec. II.B: right-to-left contraction of the
// cached process tensors with the previous row's spins as fields, then left-to-right
// conditionals and draws), with the per-site contractions of a tile of 128 proposals done
// as (128 x CHI)(CHI x CHI) products on the tensor cores:
//   right sweep: v_y[m][al] = sum_be R_{c+1}(y)[m][be] B^y[al][be]     (A = R(y), B = B^y)
//   left sweep : u_y[m][be] = sum_al l[m][al]        B^y[al][be]       (A = l,    B = B^y^T)
// Thread m of the CTA owns proposal m, which is also TMEM lane m of the accumulator, so
// every per-proposal step (fields, normalisation, conditionals, the Philox draw, log q,
// the energy) runs in that thread's registers.
//
// Precision: operands are split x = hi + lo with hi = tf32(x) and lo = tf32(x - hi), and
// each product is hi.hi + hi.lo + lo.hi (three kind::tf32 MMAs with FP32 accumulation),
// which keeps the conditionals at FP32 accuracy; single TF32 operands would not meet the
// 1e-3 conditional tolerance because the contraction of a sign-indefinite MPS amplifies
// operand rounding.
//
// Shared-memory operands use the K-major, no-swizzle canonical layout: 8-row x 16-byte
// core matrices, 128 B apart along K (LBO) and 32*CHI B apart along M/N (SBO).
#include "common.cuh"
#include "kernels.h"

namespace tnmc {
namespace tc {

constexpr int M = 128;            // proposals per tile (MMA M)

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((128u & 0x3FFFFu) >> 4) << 16;       // LBO: next core matrix along K
  d |= (uint64_t)((sbo_bytes & 0x3FFFFu) >> 4) << 32;  // SBO: next 8-row group along M/N
  d |= (uint64_t)1 << 46;                               // descriptor version of this architecture
  return d;                                             // base offset 0, no swizzle
}

template <int N>
__host__ __device__ constexpr uint32_t idesc_tf32() {
  // FP32 accumulator, A and B TF32, both K-major, N/8 and M/16 fields
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar)));
}
// Bounded wait for the given phase parity; false when the limit ran out.
__device__ __forceinline__ bool wait_parity(uint64_t* mbar, uint32_t parity, long long limit = 1ll << 20) {
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(su32(mbar)), "r"(parity) : "memory");
  }
  return done != 0;
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int NC> struct TmemLd;
template <> struct TmemLd<32> {
  static __device__ __forceinline__ void ld(uint32_t ta, float* v) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
  }
};
template <> struct TmemLd<16> {
  static __device__ __forceinline__ void ld(uint32_t ta, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
  }
};
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Float offset of element (row r, k) in a (rows x KD) K-major canonical operand.
template <int KD> __device__ __forceinline__ int koff(int r, int k) {
  return (r >> 3) * (8 * KD) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// Write this thread's row (CHI values) of an A operand as hi/lo TF32 parts.
template <int CHI>
__device__ __forceinline__ void put_row_split(float* hi, float* lo, int m, const float* x) {
#pragma unroll
  for (int kg = 0; kg < CHI / 4; ++kg) {
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) { h[t] = tf32_rna(x[4 * kg + t]); l[t] = tf32_rna(x[4 * kg + t] - h[t]); }
    const int o = koff<CHI>(m, 4 * kg);
    *reinterpret_cast<float4*>(hi + o) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + o) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

}  // namespace tc

template <int CHI>
__global__ void __launch_bounds__(128) sample_tc_kernel(SampleArgs a) {
  using namespace tc;
  constexpr int AOP = M * CHI;            // floats of one A operand
  constexpr int BOP = CHI * CHI;          // floats of one B operand
  constexpr int TILE = 2 * CHI * CHI;     // floats of one cached site tile [y][al][be]
  constexpr int PRE = TILE / M;           // tile floats each thread prefetches
  constexpr int KSTEPS = CHI / 8;
  constexpr uint32_t SBO = 32 * CHI;      // bytes between 8-row groups (K = CHI)
  constexpr uint32_t IDESC = idesc_tf32<CHI>();
  constexpr int TCOLS = 2 * CHI < 32 ? 32 : 2 * CHI;
  const int L = a.L, N = L * L;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int words_row = (L + 31) / 32;

  extern __shared__ __align__(1024) float smf[];
  float* Abuf = smf;                                  // 4 operands: [0]=R0/l hi [1]=R0/l lo [2]=R1 hi [3]=R1 lo
  float* Bbuf = Abuf + 4 * AOP;                       // [stage][y][hi,lo]
  const int LP = (L + 15) & ~15;                      // keeps the uint32 arrays 16-byte aligned
  int8_t* jh_s = reinterpret_cast<int8_t*>(Bbuf + 8 * BOP);
  int8_t* jv_s = jh_s + LP;
  uint32_t* prow = reinterpret_cast<uint32_t*>(jv_s + LP);              // [words_row][M]
  uint32_t* crow = prow + (size_t)words_row * M;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tslot;
  const uint32_t tlane = (uint32_t)(warp * 32) << 16;
  uint32_t phase = 0;

  // issue the 3xTF32 products for y = 0, 1 into TMEM columns [y*CHI, y*CHI + CHI)
  auto issue = [&](const float* A0h, const float* A0l, const float* A1h, const float* A1l, const float* Bst) {
    if (tid == 0) {
      fence_after();
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const float* Ah = y ? A1h : A0h;
        const float* Al = y ? A1l : A0l;
        const float* Bh = Bst + (y * 2 + 0) * BOP;
        const float* Bl = Bst + (y * 2 + 1) * BOP;
        const uint32_t d = tbase + (uint32_t)(y * CHI);
        int first = 1;
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const float* A = term == 2 ? Al : Ah;
          const float* B = term == 1 ? Bl : Bh;
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk) {
            mma_tf32(d, kmajor_desc(su32(A) + 256u * kk, SBO), kmajor_desc(su32(B) + 256u * kk, SBO), IDESC,
                     first ? 0u : 1u);
            first = 0;
          }
        }
      }
      mma_commit(&mbar);
    }
  };
  // Wait for the products and load them.  On a timeout the thread records it, zeroes its
  // values and carries on to the barrier that ends the site, where every thread sees the
  // abort flag and leaves together.
  auto finish = [&](float* v0, float* v1) -> bool {
    const bool ok = wait_parity(&mbar, phase);
    phase ^= 1u;
    if (!ok) {
      set_status(a.status, ST_TIMEOUT);
      abort_flag = 1;
#pragma unroll
      for (int j = 0; j < CHI; ++j) { v0[j] = 0.0f; v1[j] = 0.0f; }
      return false;
    }
    fence_after();
    TmemLd<CHI>::ld(tbase + tlane + 0, v0);
    TmemLd<CHI>::ld(tbase + tlane + CHI, v1);
    tmem_wait_ld();
    return true;
  };
  // convert prefetched tile values into a B stage (right: row al / K be; left: row be / K al)
  auto convert = [&](const float* pre, float* Bst, bool left) {
#pragma unroll
    for (int i = 0; i < PRE; ++i) {
      const int e = tid + M * i;                      // destination index over [y][d]
      const int y = e / BOP, d = e % BOP;
      const float x = pre[i];
      const float h = tf32_rna(x), l = tf32_rna(x - h);
      Bst[(y * 2 + 0) * BOP + d] = h;
      Bst[(y * 2 + 1) * BOP + d] = l;
    }
    (void)left;
  };
  // source index (into the cached tile) of destination e for the right / left layouts
  auto src_index = [&](int e, bool left) -> int {
    const int y = e / BOP, d = e % BOP;
    const int g = d / (8 * CHI), rem = d % (8 * CHI);
    const int kg = rem / 32, rr = (rem % 32) / 4, kq = rem % 4;
    const int row = 8 * g + rr, k = 4 * kg + kq;
    return left ? (y * BOP + k * CHI + row) : (y * BOP + row * CHI + k);
  };
  auto prefetch = [&](const float* tile, float* pre, bool left) {
#pragma unroll
    for (int i = 0; i < PRE; ++i) pre[i] = __ldg(tile + src_index(tid + M * i, left));
  };

  const int tiles_per_real = (a.n_items + M - 1) / M;
  const int64_t total = (int64_t)tiles_per_real * a.n_real;
  float* work = reinterpret_cast<float*>(a.work) + (size_t)blockIdx.x * L * 2 * M * CHI;

  for (int64_t tileid = blockIdx.x; tileid < total; tileid += gridDim.x) {
    const int real = (int)(tileid / tiles_per_real);
    const int k = (int)(tileid % tiles_per_real) * M + tid;
    const bool valid = k < a.n_items;
    const int64_t item = (int64_t)real * a.n_items + k;
    const int chain = a.forced ? 0 : (a.chain_of ? a.chain_of[real] : k / a.n);
    const uint32_t step = (uint32_t)(a.step0 + (uint64_t)(a.forced ? 0 : k % a.n));
    const uint64_t seed = a.seeds[real];
    const double betad = a.beta[real];
    const float eb = (float)exp(betad), ebm = (float)exp(-betad);
    const int8_t* J = a.J + (size_t)real * 2 * L * (L - 1);
    const float* envr = reinterpret_cast<const float*>(a.env) + (size_t)real * L * L * TILE;
    const int8_t* forced = (a.forced && valid) ? a.forced + (size_t)item * N : nullptr;
    const int8_t* hf = a.hfield ? a.hfield + (size_t)real * N : nullptr;
    double logq = 0.0;
    int energy = 0, magnet = 0;
    long long nclamp = 0;
    uint32_t gword = 0;

    for (int r = 0; r < L; ++r) {
      __syncthreads();
      for (int c = tid; c < L - 1; c += M) jh_s[c] = J[(size_t)r * (L - 1) + c];
      if (r > 0)
        for (int c = tid; c < L; c += M) jv_s[c] = J[(size_t)L * (L - 1) + (size_t)(r - 1) * L + c];
      const float* erow = envr + (size_t)r * L * TILE;
      float pre[PRE];

      // ---------------- right sweep ----------------
      float R0[CHI], R1[CHI];
#pragma unroll
      for (int j = 0; j < CHI; ++j) { R0[j] = (j == 0) ? 1.0f : 0.0f; R1[j] = R0[j]; }
      put_row_split<CHI>(Abuf + 0 * AOP, Abuf + 1 * AOP, tid, R0);
      put_row_split<CHI>(Abuf + 2 * AOP, Abuf + 3 * AOP, tid, R1);
      prefetch(erow + (size_t)(L - 1) * TILE, pre, false);
      convert(pre, Bbuf, false);
      if (L > 1) prefetch(erow + (size_t)(L - 2) * TILE, pre, false);
      fence_async_smem();
      fence_before();
      __syncthreads();
      for (int ci = 0; ci < L; ++ci) {
        const int c = L - 1 - ci, st = ci & 1;
        issue(Abuf + 0 * AOP, Abuf + 1 * AOP, Abuf + 2 * AOP, Abuf + 3 * AOP, Bbuf + st * 4 * BOP);
        if (c > 0) {
          convert(pre, Bbuf + (st ^ 1) * 4 * BOP, false);
          if (c > 1) prefetch(erow + (size_t)(c - 2) * TILE, pre, false);
          fence_async_smem();
        }
        float v0[CHI], v1[CHI];
        finish(v0, v1);
        // R_{c+1}(y) -> workspace (read back by the left sweep at site c)
        float* wsl = work + ((size_t)(c * 2) * M + tid) * CHI;
#pragma unroll
        for (int j = 0; j < CHI; j += 4) {
          *reinterpret_cast<float4*>(wsl + j) = make_float4(R0[j], R0[j + 1], R0[j + 2], R0[j + 3]);
          *reinterpret_cast<float4*>(wsl + (size_t)M * CHI + j) = make_float4(R1[j], R1[j + 1], R1[j + 2], R1[j + 3]);
        }
        if (c > 0) {
          const int jh = jh_s[c - 1];
          float f0 = 1.0f, f1 = 1.0f;
          if (r > 0) {
            const int sp = ((prow[(c >> 5) * M + tid] >> (c & 31)) & 1u) ? -1 : 1;
            const int sg = jv_s[c] * sp;
            f0 = sg > 0 ? eb : ebm; f1 = sg > 0 ? ebm : eb;
          }
          if (hf) { const int kh = hf[(size_t)r * L + c]; if (kh) { f0 *= expf((float)(betad * kh)); f1 *= expf((float)(-betad * kh)); } }
          const float same = jh > 0 ? eb : ebm, diff = jh > 0 ? ebm : eb;
          float mx = 0.0f;
#pragma unroll
          for (int j = 0; j < CHI; ++j) {
            const float n0 = same * f0 * v0[j] + diff * f1 * v1[j];
            const float n1 = diff * f0 * v0[j] + same * f1 * v1[j];
            R0[j] = n0; R1[j] = n1;
            mx = fmaxf(mx, fmaxf(fabsf(n0), fabsf(n1)));
          }
          const float inv = mx > 0.0f ? 1.0f / mx : 1.0f;
#pragma unroll
          for (int j = 0; j < CHI; ++j) { R0[j] *= inv; R1[j] *= inv; }
          put_row_split<CHI>(Abuf + 0 * AOP, Abuf + 1 * AOP, tid, R0);
          put_row_split<CHI>(Abuf + 2 * AOP, Abuf + 3 * AOP, tid, R1);
          fence_async_smem();
        }
        fence_before();
        __syncthreads();
        if (abort_flag) break;
      }
      if (abort_flag) break;

      // ---------------- left sweep ----------------
      float ell[CHI];
#pragma unroll
      for (int j = 0; j < CHI; ++j) ell[j] = (j == 0) ? 1.0f : 0.0f;
      put_row_split<CHI>(Abuf + 0 * AOP, Abuf + 1 * AOP, tid, ell);
      prefetch(erow, pre, true);
      convert(pre, Bbuf, true);
      if (L > 1) prefetch(erow + (size_t)1 * TILE, pre, true);
      fence_async_smem();
      fence_before();
      __syncthreads();
      int sprev = 0;
      float rsum = 0.0f, rcomp = 0.0f;
      uint32_t rword = 0;
      for (int c = 0; c < L; ++c) {
        const int st = c & 1;
        issue(Abuf + 0 * AOP, Abuf + 1 * AOP, Abuf + 0 * AOP, Abuf + 1 * AOP, Bbuf + st * 4 * BOP);
        if (c + 1 < L) {
          convert(pre, Bbuf + (st ^ 1) * 4 * BOP, true);
          if (c + 2 < L) prefetch(erow + (size_t)(c + 2) * TILE, pre, true);
          fence_async_smem();
        }
        float Rw0[CHI], Rw1[CHI];
        const float* wsl = work + ((size_t)(c * 2) * M + tid) * CHI;
#pragma unroll
        for (int j = 0; j < CHI; j += 4) {
          const float4 p0 = *reinterpret_cast<const float4*>(wsl + j);
          const float4 p1 = *reinterpret_cast<const float4*>(wsl + (size_t)M * CHI + j);
          Rw0[j] = p0.x; Rw0[j + 1] = p0.y; Rw0[j + 2] = p0.z; Rw0[j + 3] = p0.w;
          Rw1[j] = p1.x; Rw1[j + 1] = p1.y; Rw1[j + 2] = p1.z; Rw1[j + 3] = p1.w;
        }
        float u0[CHI], u1[CHI];
        finish(u0, u1);
        float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
        for (int j = 0; j < CHI; ++j) { d0 += u0[j] * Rw0[j]; d1 += u1[j] * Rw1[j]; }
        float f0 = 1.0f, f1 = 1.0f;
        int sp = 0;
        if (r > 0) {
          sp = ((prow[(c >> 5) * M + tid] >> (c & 31)) & 1u) ? -1 : 1;
          const int sg = jv_s[c] * sp;
          f0 = sg > 0 ? eb : ebm; f1 = sg > 0 ? ebm : eb;
        }
        if (c > 0) { const int sg = jh_s[c - 1] * sprev; f0 *= sg > 0 ? eb : ebm; f1 *= sg > 0 ? ebm : eb; }
        if (hf) { const int kh = hf[(size_t)r * L + c]; if (kh) { f0 *= expf((float)(betad * kh)); f1 *= expf((float)(-betad * kh)); } }
        float w0 = f0 * d0, w1 = f1 * d1;
        if (w0 < 0.0f) { w0 = 0.0f; ++nclamp; }
        if (w1 < 0.0f) { w1 = 0.0f; ++nclamp; }
        const float tot = w0 + w1;
        int s;
        float qp = 0.5f, lqs;
        if (!(tot > 0.0f) || !isfinite(tot)) {
          if (valid) {
            set_status(a.status, ST_NUMERIC);
            if (a.real_status) set_status(a.real_status + real, ST_NUMERIC);
          }
          // the realization is flagged; the spin is still drawn from the q = 1/2 it logs,
          // so that log q stays the probability the proposal was drawn with
          if (forced) {
            s = forced[(size_t)r * L + c];
          } else {
            const Philox4 o = philox4x32_10((uint32_t)(r * L + c), step, (uint32_t)chain, PURPOSE_SPIN,
                                            (uint32_t)seed, (uint32_t)(seed >> 32));
            s = ((o.x0 >> 5) < (1u << 26)) ? 1 : -1;      // m53 < 2^52
          }
          lqs = -0.6931471805599453f;
        } else {
          qp = w0 / tot;
          const float qm = w1 / tot;
          if (forced) {
            s = forced[(size_t)r * L + c];
          } else {
            const Philox4 o = philox4x32_10((uint32_t)(r * L + c), step, (uint32_t)chain, PURPOSE_SPIN,
                                            (uint32_t)seed, (uint32_t)(seed >> 32));
            const uint64_t m53 = ((uint64_t)(o.x0 >> 5) << 26) | (uint64_t)(o.x1 >> 6);
            // u < q(+) exactly: m < ceil(q 2^53) (q a float in (0, 1))
            bool below = false;
            if (qp >= 1.0f) below = true;
            else if (qp > 0.0f) {
              const uint32_t bits = __float_as_uint(qp);
              const int ex = (int)((bits >> 23) & 0xffu);
              const uint64_t mant = (ex == 0) ? (uint64_t)(bits & 0x7fffffu) : (uint64_t)((bits & 0x7fffffu) | 0x800000u);
              const int sh = (ex == 0 ? 1 : ex) - 150 + 53;
              uint64_t C;
              if (sh >= 0) C = mant << sh;
              else { const int kq = -sh; C = (kq >= 64) ? 1ull : ((mant + ((1ull << kq) - 1ull)) >> kq); }
              below = m53 < C;
            }
            s = below ? 1 : -1;
          }
          const float qs = s == 1 ? qp : qm, qo = s == 1 ? qm : qp;
          lqs = qs > 0.5f ? log1pf(-qo) : logf(qs);
        }
        { const float yk = lqs - rcomp; const float tk = rsum + yk; rcomp = (tk - rsum) - yk; rsum = tk; }
        if (a.qplus && valid) a.qplus[(size_t)item * N + (size_t)r * L + c] = (double)qp;
        // l <- u_s, normalised
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < CHI; ++j) { ell[j] = s == 1 ? u0[j] : u1[j]; mx = fmaxf(mx, fabsf(ell[j])); }
        const float inv = mx > 0.0f ? 1.0f / mx : 1.0f;
#pragma unroll
        for (int j = 0; j < CHI; ++j) ell[j] *= inv;
        put_row_split<CHI>(Abuf + 0 * AOP, Abuf + 1 * AOP, tid, ell);
        fence_async_smem();
        if (c > 0) energy -= jh_s[c - 1] * sprev * s;
        if (r > 0) energy -= jv_s[c] * sp * s;
        magnet += s;
        sprev = s;
        if (s < 0) rword |= 1u << (c & 31);
        if ((c & 31) == 31 || c == L - 1) { crow[(c >> 5) * M + tid] = rword; rword = 0; }
        const int site = r * L + c;
        if (s < 0) gword |= 1u << (site & 31);
        if ((site & 31) == 31 || site == N - 1) {
          if (valid && a.spins_packed) a.spins_packed[(size_t)item * a.words + (site >> 5)] = gword;
          gword = 0;
        }
        fence_before();
        __syncthreads();
        if (abort_flag) break;
      }
      if (abort_flag) break;
      logq += (double)rsum;
      for (int w = 0; w < words_row; ++w) prow[w * M + tid] = crow[w * M + tid];
    }
    if (valid && !abort_flag) {
      if (a.logq) a.logq[item] = logq;
      if (a.energy) a.energy[item] = energy;
      if (a.magnet) a.magnet[item] = magnet;
      if (a.clamps && nclamp) atomicAdd(reinterpret_cast<unsigned long long*>(a.clamps + real), (unsigned long long)nclamp);
    }
    if (abort_flag) break;
  }
  fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
}

template <int CHI>
static size_t sample_tc_smem(int L) {
  const int words_row = (L + 31) / 32;
  return (size_t)(4 * tc::M * CHI + 8 * CHI * CHI) * sizeof(float) + (size_t)2 * ((L + 15) & ~15) +
         (size_t)2 * words_row * tc::M * sizeof(uint32_t) + 64;
}

int sample_tc_grid(int n_items, int n_real, int num_sms) {
  const int64_t tiles = (int64_t)((n_items + tc::M - 1) / tc::M) * n_real;
  int64_t grid = (int64_t)num_sms * 2;
  if (grid > tiles) grid = tiles;
  return grid < 1 ? 1 : (int)grid;
}

size_t sample_tc_work_bytes(int L, int CHI, int num_sms) {
  return (size_t)num_sms * 2 * (size_t)L * 2 * tc::M * CHI * sizeof(float);
}

template <int CHI>
static cudaError_t launch_tc_t(const SampleArgs& a, int num_sms, cudaStream_t st) {
  const size_t smem = sample_tc_smem<CHI>(a.L);
  cudaError_t e = cudaFuncSetAttribute(sample_tc_kernel<CHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = sample_tc_grid(a.n_items, a.n_real, num_sms);
  sample_tc_kernel<CHI><<<grid, tc::M, smem, st>>>(a);
  return cudaGetLastError();
}

bool sample_tc_supported(int CHI) { return CHI == 16 || CHI == 32; }

// Self-test of the bounded wait the sampler uses on its MMA completions: one CTA waits on an
// mbarrier of arrival count 1; with arrive != 0 one thread arrives first, otherwise nothing
// does and every wait must give up after `limit` polls and record ST_TIMEOUT.  The kernel
// returns normally either way.
__global__ void wait_probe_kernel(int arrive, long long limit, unsigned* status) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::su32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(tc::su32(&mbar)) : "memory");
  }
  __syncthreads();
  if (!tc::wait_parity(&mbar, 0u, limit)) set_status(status, ST_TIMEOUT);
}

cudaError_t launch_wait_probe(int arrive, long long limit, unsigned* status_dev, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(arrive, limit, status_dev);
  return cudaGetLastError();
}

cudaError_t launch_sample_tc(const SampleArgs& a, int CHI, int num_sms, cudaStream_t st) {
  if (CHI == 32) return launch_tc_t<32>(a, num_sms, st);
  if (CHI == 16) return launch_tc_t<16>(a, num_sms, st);
  return cudaErrorInvalidValue;
}

}  // namespace tnmc
