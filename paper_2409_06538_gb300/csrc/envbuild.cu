// Boundary-MPS row environments (Sec. II.B of arXiv 2409.06538) on sm_103a.
//
// For every realization (one CTA each) and every row r = L-2 .. 0:
//   A[c] = O_r[c] . Gt_{r+1}[c]  -- the row-transfer MPO (bond 2: the T tensors, copy tensor
//          with the right and bottom Boltzmann matrices absorbed) applied to the cached MPS;
//          A[c]^x_{(a,al),(b,be)} = W(x,a,b) B[c]^b_{al,be},
//          W(x,a,b) = exp(beta Jv[r][c] s_x s_b) * exp(beta Jh[r+1][c-1] s_a s_b)   (c > 0),
//          the right MPO bond b of the last site summed.
//   forward sweep  c = 0..L-2 : R_{c+1} = R-factor of [R_c A[c]^{x=0}; R_c A[c]^{x=1}]
//          (Householder; R_c^T R_c is the Gram matrix of the left part, so the left part is
//          represented without squaring its condition number);
//   backward sweep c = L-1..1 : M = A[c] contracted with the already-truncated right part,
//          Y = R_c M has the singular values and right singular vectors of the state cut
//          before site c (the left part is Q_{<c} R_c with Q an isometry).  Its SVD: two
//          Householder QRs (Y = Q1 R1, R1^T = Q2 R2) and a one-sided (Hestenes) Jacobi on R2^T,
//          V = Q2 Z (the QR-preconditioned one-sided Jacobi of Drmac and Veselic); the top
//          k = min(chi, d_c, 2 k_{c+1}) right singular vectors V give B_r[c] = V^T
//          (right-canonical), P = M V carries the rest of the state to site c-1.  Site 0 keeps
//          the normalised remainder; lam_r = log of the removed scale.
// This is the QR-sweep + truncating-SVD-sweep compression of the oracle, computed without
// forming Q: the truncated MPS is the same up to gauge (and rounding).
// Zip-up mode (args.zipup, a compression variant): no forward sweep and Y = M, the Jacobi on M
// itself (graded by columns); the rows alternate their sweep direction, a left-to-right row
// running as this backward sweep over the mirrored row (frame site f = lattice site L-1-f,
// bonds swapped, horizontal bond factors at the bond's right site).
#include "common.cuh"
#include "kernels.h"

namespace tnmc {

// Convergence: a pair counts as orthogonal when |y_p . y_q| <= tol |y_p| |y_q|, with tol =
// sqrt(D) eps, the rounding floor of a D-long dot product.  The residual non-orthogonality
// tilts the kept singular subspace where sigma_chi and sigma_{chi+1} are close; in FP32 at
// L = 256, chi = 32 a four times looser tolerance left environments whose conditionals drifted
// by up to 5e-3 from FP64 and produced doubly clamped sites (measured), for about 1 % more
// sweeps it does not.
template <typename T> struct JacobiTol;
template <> struct JacobiTol<float> { static constexpr int maxsw = 30; };
template <> struct JacobiTol<double> { static constexpr int maxsw = 40; };
template <typename T, int D> __device__ __forceinline__ T jacobi_tol() {
  return num<T>::sqrt_(T(D)) * num<T>::eps;
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };
__device__ __forceinline__ float dot16(const float4& a, const float4& b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ double dot16(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ void rot16(float4& u, float4& v, float c, float s) {
  const float4 a = u, b = v;
  u = make_float4(c * a.x - s * b.x, c * a.y - s * b.y, c * a.z - s * b.z, c * a.w - s * b.w);
  v = make_float4(s * a.x + c * b.x, s * a.y + c * b.y, s * a.z + c * b.z, s * a.w + c * b.w);
}
__device__ __forceinline__ void rot16(double2& u, double2& v, double c, double s) {
  const double2 a = u, b = v;
  u = make_double2(c * a.x - s * b.x, c * a.y - s * b.y);
  v = make_double2(s * a.x + c * b.x, s * a.y + c * b.y);
}
// Jacobi rotation (c, s) that makes columns p, q orthogonal, from a = |y_p|^2, b = |y_q|^2,
// g = y_p . y_q (y_p' = c y_p - s y_q, y_q' = s y_p + c y_q).  The angle solves
// tan 2theta = 2g / (b - a) with |theta| <= pi/4:
//   r = sqrt((b-a)^2 + 4 g^2), cos 2theta = |b-a| / r, c = sqrt((1 + cos 2theta) / 2),
//   s = sgn(b-a) g / (r c)   (sgn(0) = +1),
// two reciprocal square roots in sequence instead of the divide/sqrt chain of the tangent
// form.  FP32 uses the hardware rsqrt with one Newton step each, so c^2 + s^2 = 1 to
// working precision; FP64 uses IEEE operations.
__device__ __forceinline__ float rsqrt_nr(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ void rotation_from_gram(double a, double b, double g, double& c, double& s) {
  const double d = b - a;
  const double rinv = 1.0 / sqrt(d * d + 4.0 * g * g);
  const double h = 0.5 + 0.5 * fabs(d) * rinv;
  const double ic = 1.0 / sqrt(h);
  c = h * ic;
  s = (d < 0.0 ? -g : g) * rinv * ic;
}
__device__ __forceinline__ void rotation_from_gram(float a, float b, float g, float& c, float& s) {
  const float d = b - a;
  const float rinv = rsqrt_nr(fmaf(d, d, 4.0f * g * g));
  const float h = fmaf(0.5f * fabsf(d), rinv, 0.5f);
  const float ic = rsqrt_nr(h);
  c = h * ic;
  s = (d < 0.0f ? -g : g) * rinv * ic;
}

template <typename T> __device__ __forceinline__ T group8_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}
__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// 4-element shared-memory vectors (16 B for float, 2 x 16 B for double); callers keep the
// index a multiple of 4 so the accesses are aligned.
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void cp_async16_env(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit_env() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_env() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// Copy `bytes` (a multiple of 16) from global to shared memory with cp.async (no wait).
__device__ __forceinline__ void prefetch_async(void* smem, const void* gmem, int bytes, int tid, int nt) {
  for (int i = tid; i < bytes / 16; i += nt)
    cp_async16_env(static_cast<char*>(smem) + 16 * i, static_cast<const char*>(gmem) + 16 * i);
  cp_async_commit_env();
}

template <int CHI> struct EnvCfg {
  static constexpr int D = 2 * CHI;                 // MPO bond x MPS bond
  // 8 lanes per Jacobi pair (8*CHI threads); CHI = 32 runs 256 threads so that three
  // realizations fit on one SM in FP32 (80 registers, 72 KB of shared memory each)
  // CHI = 64 runs 512 threads (64 Jacobi pairs) with one CTA per SM
  static constexpr int NWARP = CHI > 32 ? 16 : (CHI < 4 ? 4 : (CHI > 8 ? 8 : CHI));
  static constexpr int NT = 32 * NWARP;
  static constexpr int TILE = 2 * CHI * CHI;        // [y][alpha][beta]
};

// Column stride of Y and V: at least 8 lanes x 16 bytes, so that the 8 lanes of a Jacobi
// pair read one contiguous 128-byte segment per vector load (no bank conflicts).
template <typename T, int CHI> struct JStride {
  static constexpr int D = 2 * CHI;
  static constexpr int VEC = 16 / (int)sizeof(T);
  static constexpr int DP = D > 8 * VEC ? D : 8 * VEC;
};

template <typename T, int CHI>
__host__ __device__ constexpr size_t env_smem_elems() {
  // CHI = 64: only Y and V (D*DP each) and the Householder vectors (three of 2D) stay in shared memory;
  // M lives in per-realization global scratch and R, the tile are read from global memory
  if (CHI > 32) return (size_t)2 * (2 * CHI) * JStride<T, CHI>::DP + (size_t)6 * (2 * CHI);
  // backward: M, R (D*D each), Y, V (D*DP each) + tile (2*CHI*CHI); P (D*CHI) lives in the Y
  //           region and Q (2*CHI*CHI) in the V region between their uses
  // forward : X (2D*D, aliases M and Y) + R (D*D) + tile; the Householder vectors use V
  // (FP32, CHI = 32: 72 KB, so three CTAs fit on one SM)
  return (size_t)2 * (2 * CHI) * (2 * CHI) + (size_t)2 * (2 * CHI) * JStride<T, CHI>::DP +
         (size_t)2 * CHI * CHI;
}

// Householder R factor of the first nc <= NC columns of an MR-row matrix A (column j at
// A + j*ld) in place, by all threads of the CTA: warp j % NWARP owns column j; reflector j is
// applied to every column a warp owns with the dot products reduced in one interleaved
// butterfly, and the owner of column j+1 forms reflector j+1 first, deferring its other columns
// by one step (reflectors rotate through three slots of vbuf).  On return the upper triangle of
// A holds R, zeros below.  With vsave (MR x NC, column j = reflector j, zero above row j) and
// csave (nc coefficients 2/|v|^2) the reflectors are kept, so that Q = H_0 H_1 ... H_{nc-1} can
// be applied afterwards.  Not inlined: one body serves both QRs of a site (measured 3 % faster
// than two inlined copies).  A Givens QR in the parallel Sameh-Kuck order (one barrier per
// stage, no reductions) measured slower per QR and less accurate once Q is accumulated.
template <typename T, int MR, int NC, int NWARP>
__device__ __noinline__ void householder_r(T* A, int ld, int nc, T (*vbuf)[MR], T* vcoef, T* vsave,
                                              T* csave, int lane, int warp) {
  constexpr int RPL = MR / 32 > 0 ? MR / 32 : 1;
  constexpr int CPW = (NC + NWARP - 1) / NWARP;
  const T tiny = (sizeof(T) == 4) ? T(1e-36) : T(1e-300);
  auto house = [&](int j) {
    T* col = A + (size_t)j * ld;
    T xr[RPL];
    T ss = 0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = lane + 32 * t;
      xr[t] = (i < MR && i >= j) ? col[i] : T(0);
      ss += xr[t] * xr[t];
    }
    ss = warp_sum(ss);
    const T x0 = col[j];
    __syncwarp();
    T* vj = vbuf[j % 3];
    T coef = T(0);
    if (ss <= tiny) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        if (i < MR) { vj[i] = T(0); if (i > j) col[i] = T(0); if (vsave) vsave[(size_t)j * MR + i] = T(0); }
      }
    } else {
      const T nrm = num<T>::sqrt_(ss);
      const T alpha = x0 >= T(0) ? -nrm : nrm;
      const T v0 = x0 - alpha;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        if (i < MR) {
          const T vi = (i == j) ? v0 : xr[t];
          vj[i] = vi;
          if (vsave) vsave[(size_t)j * MR + i] = vi;
          if (i >= j) col[i] = (i == j) ? alpha : T(0);
        }
      }
      coef = T(1) / (nrm * (nrm + (x0 >= T(0) ? x0 : -x0)));
    }
    if (lane == 0) { vcoef[j % 3] = coef; if (csave) csave[j] = coef; }
  };
  auto apply1 = [&](int jj, int k) {
    const T coef = vcoef[jj % 3];
    if (coef == T(0)) return;
    const T* v = vbuf[jj % 3];
    T* col = A + (size_t)k * ld;
    T xr[RPL], vr[RPL];
    T d = 0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = lane + 32 * t;
      xr[t] = i < MR ? col[i] : T(0);
      vr[t] = i < MR ? v[i] : T(0);
      d += vr[t] * xr[t];
    }
    d = warp_sum(d) * coef;
#pragma unroll
    for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; if (i < MR) col[i] = xr[t] - d * vr[t]; }
  };
  auto apply_batch = [&](int jj, int lo) {
    const T coef = vcoef[jj % 3];
    if (coef == T(0)) return;
    const T* v = vbuf[jj % 3];
    T vr[RPL], d[CPW];
#pragma unroll
    for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; vr[t] = i < MR ? v[i] : T(0); }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int k = warp + NWARP * q;
      d[q] = 0;
      if (k > lo && k < nc) {
        const T* col = A + (size_t)k * ld;
#pragma unroll
        for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; if (i < MR) d[q] += vr[t] * col[i]; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < CPW; ++q) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int k = warp + NWARP * q;
      if (k > lo && k < nc) {
        T* col = A + (size_t)k * ld;
        const T dc = d[q] * coef;
#pragma unroll
        for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; if (i < MR) col[i] -= dc * vr[t]; }
      }
    }
  };
  __syncthreads();
  if (nc <= 0) return;
  if (warp == 0) house(0);
  int pend = -1;
  for (int j = 0; j < nc; ++j) {
    __syncthreads();
    if (pend >= 0) { apply_batch(pend, pend + 1); pend = -1; }
    const int nxt = j + 1;
    if (nxt < nc && warp == nxt % NWARP) {
      apply1(j, nxt);
      __syncwarp();
      house(nxt);
      pend = j;
    } else {
      apply_batch(j, j);
    }
    __syncwarp();
  }
  __syncthreads();
}

template <int CHI> struct Pair {
  // round-robin ("circle") schedule over n columns (n even): n-1 rounds of n/2 disjoint pairs
  static __device__ __forceinline__ void get(int n, int round, int w, int& p, int& q) {
    const int m = n - 1;
    if (w == 0) { p = n - 1; q = round; }
    else { p = (round + w) % m; q = (round - w + m) % m; }
  }
};

template <typename T, typename TE, int CHI>
__global__ void __launch_bounds__(EnvCfg<CHI>::NT, (sizeof(T) == 8 || CHI > 32) ? 1 : 3)
env_build_kernel(EnvBuildArgs<T, TE> args) {
  using C = EnvCfg<CHI>;
  constexpr int D = C::D, NWARP = C::NWARP, NT = C::NT, TILE = C::TILE;
  const int L = args.L;
  const int real = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int chi = args.chi;
  const double beta = args.beta[real];

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  // CHI = 64 (kBig): M in global scratch, R_c and the previous-row tile read from global
  // memory where they are stored (the pointers move with the site), shared memory for Y, V
  constexpr bool kBig = CHI > 32;
  T* const Rstore_r = args.Rstore + (size_t)real * args.L * D * D;
  // backward-phase layout
  constexpr int DP = JStride<T, CHI>::DP;
  T* Mc = kBig ? args.Mscratch + (size_t)real * D * D : sm;   // D x D col-major, columns j = x*kn + g
  T* Yc = kBig ? sm : Mc + D * D;  // n columns of stride DP (rows >= D zero)
  T* Vc = Yc + D * DP;        // n columns of stride DP (rows >= n zero)
  T* Rc = kBig ? Rstore_r : Vc + D * DP;   // D x D col-major R_c
  T* Bt = kBig ? nullptr : Rc + D * D;     // previous-row tile [y][al][be]
  // P is written after the SVD (Y is dead by then) and read by the next site's Q = B P before
  // that site's Y is formed; Q is written after this site's V is dead and read before the next
  // V is initialised: so P takes the Y region and Q the V region
  T* Ps = Yc;                 // D x CHI col-major: P[(b,be)][g] at g*D + b*CHI + be
  T* Qs = Vc;                 // 2 x CHI x CHI: Q[b][al][g]
  // forward-phase layout (aliases M/Y/V; R stays at Rc)
  T* Xs = sm;                 // 2D x D col-major

  __shared__ T Wc[8];               // W[x][a][b] at x*4 + a*2 + b
  int8_t* jv_s = reinterpret_cast<int8_t*>(kBig ? Vc + D * DP + 6 * D : Bt + TILE);   // Jv[r][c], L entries
  int8_t* jh_s = jv_s + args.L;                                // Jh[r+1][c], L-1 entries
  const T eb = (T)exp(beta), ebm = (T)exp(-beta);             // exp(+-beta): every Boltzmann weight
  // Householder vectors (three slots; the V region is idle in the forward sweep unless
  // the forward matrix X fills Y and V, as for kBig)
  T (*vbuf)[2 * D] = reinterpret_cast<T (*)[2 * D]>(kBig ? Vc + D * DP : Vc);
  __shared__ T vcoef[3];
  __shared__ T csave[D];            // coefficients of the backward sweep's second QR
  __shared__ T red[32];
  __shared__ T sig[D];
  __shared__ int sel[CHI];
  __shared__ int rot[3];            // per-sweep 'any rotation' flags, a ring of three
  __shared__ int knext_s;

  const int8_t* J = args.J + (size_t)real * 2 * L * (L - 1);
  // external fields (units of beta) of this realization: the row MPO carries those of the row
  // below as a site weight exp(beta k s_b), the top-row closure of log Z those of row 0
  const int8_t* hf = args.hfield ? args.hfield + (size_t)real * L * L : nullptr;
  const int8_t* Jh = J;                          // [r][c], c < L-1
  const int8_t* Jv = J + (size_t)L * (L - 1);    // [r][c], r < L-1
  int* kd = args.kdim + (size_t)real * L * (L + 1);
  int* dqr = args.dqr + (size_t)real * (L + 1);
  T* rowbuf = args.rowbuf + (size_t)real * 2 * L * TILE;
  T* Rstore = args.Rstore + (size_t)real * L * D * D;
  TE* env = args.env + (size_t)real * L * L * TILE;
  double* lam = args.lam + (size_t)real * L;

  // ---- row L-1: the exact all-ones environment G_{L-1}(x) = 1
  {
    T* prev = rowbuf + (size_t)((L - 1) & 1) * L * TILE;
    TE* erow = env + (size_t)(L - 1) * L * TILE;
    for (int e = tid; e < L * TILE; e += NT) {
      const int t = e % TILE;
      const T v = (t == 0 || t == CHI * CHI) ? T(1) : T(0);
      prev[e] = v;
      erow[e] = env_store<TE, T>(v);
    }
    for (int c = tid; c <= L; c += NT) kd[(size_t)(L - 1) * (L + 1) + c] = 1;
    if (tid == 0) lam[L - 1] = 0.0;
  }
  __syncthreads();

  int max_sweeps_seen = 0, unconverged = 0;
  long long total_sweeps = 0, n_svd = 0;

  for (int r = L - 2; r >= 0; --r) {
    const T* prev = rowbuf + (size_t)((r + 1) & 1) * L * TILE;
    T* cur = rowbuf + (size_t)(r & 1) * L * TILE;
    TE* erow = env + (size_t)r * L * TILE;
    const int* kold = kd + (size_t)(r + 1) * (L + 1);
    int* knew = kd + (size_t)r * (L + 1);

    // Zip-up rows alternate their sweep direction; a left-to-right row runs as the right-to-left
    // sweep of the mirrored row.  The backward sweep below works in the sweep's frame: frame site
    // f is site osite(f) of the lattice, whose bonds are swapped when the row is mirrored.
    const bool zip = args.zipup != 0;
    const bool mir = zip && ((L - 2 - r) % 2 == 0);
    auto osite = [&](int f) { return mir ? L - 1 - f : f; };
    // canonical: QR bond dimensions d_c of the MPO x MPS (left-canonical form); zip-up: the
    // rows of frame site f's matrix M, (MPO bond) x (previous row's bond into f)
    if (tid == 0) {
      if (zip) {
        for (int f = 0; f < L; ++f) dqr[f] = (f == 0 ? 1 : 2) * (mir ? kold[L - f] : kold[f]);
      } else {
        dqr[0] = 1;
        for (int c = 0; c < L - 1; ++c) dqr[c + 1] = min(2 * dqr[c], 2 * kold[c + 1]);
      }
    }
    for (int c = tid; c < L; c += NT) jv_s[c] = Jv[(size_t)r * L + c];
    for (int c = tid; c < L - 1; c += NT) jh_s[c] = Jh[(size_t)(r + 1) * (L - 1) + c];
    // W(x,a,b) of (frame) site c from exp(+-beta): the vertical bond to the row below and the
    // horizontal bond of the row below to the previous frame site (absent at c = 0, where only
    // a = 0 exists) -- in a mirrored row that is the bond to the lattice site on the right
    auto set_w = [&](int c) {
      if (tid < 8) {
        const int x = tid >> 2, a = (tid >> 1) & 1, b = tid & 1;
        const int co = osite(c);
        T w = (jv_s[co] * spin_of(x) * spin_of(b) > 0) ? eb : ebm;
        if (c > 0) w *= (jh_s[mir ? co : c - 1] * spin_of(a) * spin_of(b) > 0) ? eb : ebm;
        else if (a == 1) w = T(0);
        if (hf) { const int k = hf[(size_t)(r + 1) * L + co]; if (k) w *= (T)exp(beta * (double)(k * spin_of(b))); }
        Wc[tid] = w;
      }
    };
    // R_0 = [1]
    if constexpr (kBig) Rc = Rstore;
    for (int e = tid; e < D * D; e += NT) Rc[e] = (e == 0) ? T(1) : T(0);
    if (!kBig && tid == 0) {
      for (int e = 0; e < D * D; ++e) Rstore[e] = (e == 0) ? T(1) : T(0);
    }
    // the tile the first sweep starts on: site 0 (forward sweep), frame site L-1 (zip-up)
    if constexpr (!kBig) prefetch_async(Bt, prev + (size_t)(zip ? osite(L - 1) : 0) * TILE, TILE * (int)sizeof(T), tid, NT);
    __syncthreads();

    // ---------------- forward sweep: R factors of the left parts (canonical only) ----------------
    for (int c = 0; !zip && c < L - 1; ++c) {
      set_w(c);
      if constexpr (kBig) {
        Rc = Rstore + (size_t)c * D * D;
        Bt = const_cast<T*>(prev + (size_t)c * TILE);
      }
      cp_async_wait_env();
      __syncthreads();
      // X[(x,i),(b,be)] = sum_al (W(x,0,b) R[i][al] + W(x,1,b) R[i][CHI+al]) B[b][al][be]:
      // four (D x CHI) = (D x CHI)(CHI x CHI) products, 4 x 4 register tiles
      constexpr int TI = D / 4, TB = CHI / 4;
      for (int u = tid; u < 4 * TI * TB; u += NT) {
        const int xb = u / (TI * TB), rem = u % (TI * TB);
        const int x = xb >> 1, b = xb & 1, i0 = (rem % TI) * 4, b0 = (rem / TI) * 4;
        const T w0 = Wc[x * 4 + 0 * 2 + b], w1 = Wc[x * 4 + 1 * 2 + b];
        T acc[4][4] = {};
#pragma unroll 4
        for (int al = 0; al < CHI; ++al) {
          T r0[4], r1[4], bv[4];
          ld4(Rc + al * D + i0, r0);
          ld4(Rc + (CHI + al) * D + i0, r1);
          ld4(Bt + b * CHI * CHI + al * CHI + b0, bv);
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            const T rw = w0 * r0[ii] + w1 * r1[ii];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += rw * bv[jj];
          }
        }
        // row (x, i) of X is stored at 2 i + x: the two blocks R_c A^0 and R_c A^1 share
        // R_c's row scale, which falls with i, so interleaving them lets the reflectors meet
        // the rows in order of scale (measured at L = 256 in FP32: two orders of magnitude
        // fewer clamped weights than the two blocks one after the other)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          T* xc = Xs + (size_t)(b * CHI + b0 + jj) * (2 * D);
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) xc[2 * (i0 + ii) + x] = acc[ii][jj];
        }
      }
      __syncthreads();
      // the next site's tile streams in while the QR runs
      if constexpr (!kBig) prefetch_async(Bt, prev + (size_t)(c + 1) * TILE, TILE * (int)sizeof(T), tid, NT);
      // Householder QR of X (m = 2D rows, D columns); warp (j % NWARP) owns column j.
      constexpr int m = 2 * D;
      const T tiny = (sizeof(T) == 4) ? T(1e-36) : T(1e-300);
      // Each lane owns rows lane + 32 t (t < m/32) of a column; the reflector vector is
      // stored zero above its pivot row, so the updates run over all rows unconditionally.
      constexpr int RPL = m / 32 > 0 ? m / 32 : 1;     // rows per lane
      constexpr int CPW = (D + NWARP - 1) / NWARP;      // columns a warp owns: k = warp + NWARP t
      auto house = [&](int j) {   // executed by the owning warp for column j
        T* col = Xs + (size_t)j * m;
        T xr[RPL];
        T ss = 0;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int i = lane + 32 * t;
          xr[t] = (i < m && i >= j) ? col[i] : T(0);
          ss += xr[t] * xr[t];
        }
        ss = warp_sum(ss);
        const T x0 = col[j];
        __syncwarp();                 // every lane has read the pivot before any lane writes
        T* vj = vbuf[j % 3];
        if (ss <= tiny) {
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if (i < m) { vj[i] = T(0); if (i > j) col[i] = T(0); }
          }
          if (lane == 0) vcoef[j % 3] = T(0);
        } else {
          const T nrm = num<T>::sqrt_(ss);
          const T alpha = x0 >= T(0) ? -nrm : nrm;
          const T v0 = x0 - alpha;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if (i < m) {
              vj[i] = (i == j) ? v0 : xr[t];
              if (i >= j) col[i] = (i == j) ? alpha : T(0);
            }
          }
          if (lane == 0) vcoef[j % 3] = T(1) / (nrm * (nrm + (x0 >= T(0) ? x0 : -x0)));  // 2/|v|^2
        }
      };
      // reflector jj applied to one column k (the pivot owner's next column)
      auto apply1 = [&](int jj, int k) {
        const T coef = vcoef[jj % 3];
        if (coef == T(0)) return;
        const T* v = vbuf[jj % 3];
        T* col = Xs + (size_t)k * m;
        T xr[RPL], vr[RPL];
        T d = 0;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int i = lane + 32 * t;
          xr[t] = i < m ? col[i] : T(0);
          vr[t] = i < m ? v[i] : T(0);
          d += vr[t] * xr[t];
        }
        d = warp_sum(d) * coef;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int i = lane + 32 * t;
          if (i < m) col[i] = xr[t] - d * vr[t];
        }
      };
      // reflector jj applied to every column k > lo this warp owns: the dot products of all of
      // them are reduced in one interleaved butterfly instead of one reduction after another
      auto apply_batch = [&](int jj, int lo) {
        const T coef = vcoef[jj % 3];
        if (coef == T(0)) return;
        const T* v = vbuf[jj % 3];
        T vr[RPL], d[CPW];
#pragma unroll
        for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; vr[t] = i < m ? v[i] : T(0); }
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
          const int k = warp + NWARP * q;
          d[q] = 0;
          if (k > lo && k < D) {
            const T* col = Xs + (size_t)k * m;
#pragma unroll
            for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; if (i < m) d[q] += vr[t] * col[i]; }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int q = 0; q < CPW; ++q) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
          const int k = warp + NWARP * q;
          if (k > lo && k < D) {
            T* col = Xs + (size_t)k * m;
            const T dc = d[q] * coef;
#pragma unroll
            for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; if (i < m) col[i] -= dc * vr[t]; }
          }
        }
      };
      // Step j: the owner of column j+1 applies reflector j to that column and forms reflector
      // j+1 at once (the critical path), deferring its other columns to the next step; every
      // other warp applies reflector j to its columns.  Reflectors rotate through three slots,
      // so a deferred one is still intact when its owner applies it.
      if (warp == 0) house(0);
      int pend = -1;                  // reflector this warp still owes its columns > pend + 1
      for (int j = 0; j < D; ++j) {
        __syncthreads();
        if (pend >= 0) { apply_batch(pend, pend + 1); pend = -1; }
        const int nxt = j + 1;
        if (nxt < D && warp == nxt % NWARP) {
          apply1(j, nxt);
          __syncwarp();
          house(nxt);
          pend = j;
        } else {
          apply_batch(j, j);
        }
        __syncwarp();
      }
      __syncthreads();
      // scale: max |R_jj|; R_{c+1} = X[0:D, :] / scale (col-major), also to Rstore[c+1]
      if (warp == 0) {
        T mx = 0;
        for (int j = lane; j < D; j += 32) { T v = Xs[(size_t)j * m + j]; v = v < 0 ? -v : v; mx = v > mx ? v : mx; }
        mx = warp_max(mx);
        if (lane == 0) red[0] = mx > T(0) ? T(1) / mx : T(1);
      }
      __syncthreads();
      const T inv = red[0];
      T* Rout = Rstore + (size_t)(c + 1) * D * D;
      for (int e = tid; e < D * D; e += NT) {
        const int i = e % D, j = e / D;
        const T v = (i <= j) ? Xs[(size_t)j * m + i] * inv : T(0);
        if constexpr (!kBig) Rc[e] = v;      // kBig reads R_{c+1} back from Rstore
        Rout[e] = v;
      }
      __syncthreads();
    }

    // ---------------- backward sweep: truncating SVDs ----------------
    // P_L[(b,be)][g] = delta(be,0) delta(g,0) for both b (closes the right MPO bond)
    for (int e = tid; e < D * CHI; e += NT) {
      const int row = e % D, g = e / D;
      Ps[e] = (g == 0 && (row % CHI) == 0) ? T(1) : T(0);
    }
    int kn = 1;             // k_{c+1}
    double logs = 0.0;
    if (tid == 0) knew[L] = 1;
    __syncthreads();
    for (int c = L - 1; c >= 0; --c) {
      // Bt (tile c) and Rc (R_c) were prefetched during the previous site
      set_w(c);
      if constexpr (kBig) {
        Rc = Rstore + (size_t)c * D * D;
        Bt = const_cast<T*>(prev + (size_t)osite(c) * TILE);
      }
      cp_async_wait_env();
      __syncthreads();
      // Q[b][al][g] = sum_be B[b][al][be] P[(b,be)][g]: 4 x 4 register tiles (a mirrored row
      // reads the previous row's tile with its bonds swapped)
      {
        constexpr int TA = CHI / 4;
        const int sA = mir ? 1 : CHI, sB = mir ? CHI : 1;
        for (int u = tid; u < 2 * TA * TA; u += NT) {
          const int b = u / (TA * TA), a0 = ((u % (TA * TA)) % TA) * 4, g0 = ((u % (TA * TA)) / TA) * 4;
          T acc[4][4] = {};
          if (g0 < kn) {
#pragma unroll 4
            for (int be = 0; be < CHI; ++be) {
              T bv[4], pv[4];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii) bv[ii] = Bt[b * CHI * CHI + (a0 + ii) * sA + be * sB];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) pv[jj] = Ps[(g0 + jj) * D + b * CHI + be];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += bv[ii] * pv[jj];
            }
          }
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            T row4[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) row4[jj] = (g0 + jj < kn) ? acc[ii][jj] : T(0);
            st4(Qs + b * CHI * CHI + (a0 + ii) * CHI + g0, row4);
          }
        }
      }
      __syncthreads();
      if (!kBig && c > 0) prefetch_async(Bt, prev + (size_t)osite(c - 1) * TILE, TILE * (int)sizeof(T), tid, NT);
      const int n = 2 * kn;    // compact columns j = x*kn + g
      // M[(a,al)][j] = sum_b W(x,a,b) Q[b][al][g]
      for (int e = tid; e < D * n; e += NT) {
        const int row = e % D, j = e / D;
        const int a = row / CHI, al = row % CHI, x = j / kn, g = j % kn;
        Mc[e] = Wc[x * 4 + a * 2 + 0] * Qs[0 * CHI * CHI + al * CHI + g] +
                Wc[x * 4 + a * 2 + 1] * Qs[1 * CHI * CHI + al * CHI + g];
      }
      __syncthreads();
      if (c == 0) {
        // site 0: the whole remaining state, row (a=0, al=0) of M
        if (warp == 0) {
          T ss = 0;
          for (int j = lane; j < n; j += 32) ss += Mc[(size_t)j * D] * Mc[(size_t)j * D];
          ss = warp_sum(ss);
          if (lane == 0) red[0] = num<T>::sqrt_(ss);
        }
        __syncthreads();
        const T nrm = red[0];
        const T inv = nrm > T(0) ? T(1) / nrm : T(0);
        T* ctile0 = cur + (size_t)osite(0) * TILE;
        TE* etile0 = erow + (size_t)osite(0) * TILE;
        for (int e = tid; e < TILE; e += NT) {
          const int y = e / (CHI * CHI), i = (e / CHI) % CHI, j = e % CHI;
          const int al = mir ? j : i, be = mir ? i : j;     // frame bonds of lattice entry (i, j)
          const T v = (al == 0 && be < kn) ? Mc[(size_t)(y * kn + be) * D] * inv : T(0);
          ctile0[e] = v;
          etile0[e] = env_store<TE, T>(v);
        }
        if (tid == 0) { logs += log((double)nrm); knew[0] = 1; knew[L] = 1; }
        __syncthreads();
        break;
      }
      // Y = R_c M  (D x n; R_c, the R factor of the left part up to site c-1, was
      // prefetched): 4 x 4 register tiles over (rows, compact columns).  Zip-up: Y = M (the
      // previous row is canonical on the side not yet swept, so no R factor)
      T fro = 0;
      if (zip) {
        for (int e = tid; e < DP * n; e += NT) {
          const int i = e % DP, j = e / DP;
          const T v = i < D ? Mc[(size_t)j * D + i] : T(0);
          Yc[e] = v;
          fro += v * v;
        }
      } else {
        constexpr int TI = D / 4;
        const int TJ = (n + 3) / 4;
        for (int u = tid; u < TI * TJ; u += NT) {
          const int i0 = (u % TI) * 4, j0 = (u / TI) * 4;
          T acc[4][4] = {};
#pragma unroll 4
          for (int l = 0; l < D; ++l) {
            T rv[4], mv[4];
            ld4(Rc + l * D + i0, rv);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) mv[jj] = (j0 + jj < n) ? Mc[(size_t)(j0 + jj) * D + l] : T(0);
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += rv[ii] * mv[jj];
          }
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            if (j0 + jj < n) {
              const T col4[4] = {acc[0][jj], acc[1][jj], acc[2][jj], acc[3][jj]};
              st4(Yc + (size_t)(j0 + jj) * DP + i0, col4);
#pragma unroll
              for (int ii = 0; ii < 4; ++ii) fro += acc[ii][jj] * acc[ii][jj];
            }
          }
        }
        if constexpr (DP > D) {
          constexpr int PAD = DP > D ? DP - D : 1;
          for (int e = tid; e < PAD * n; e += NT) Yc[(size_t)(e / PAD) * DP + D + e % PAD] = T(0);
        }
      }
      // the Jacobi runs on npad = n rounded up to 8 columns (blocks of 4, an even number of
      // blocks); columns n..npad-1 of Y are zero and never rotate
      const int npad = (n + 7) & ~7;
      fro = warp_sum(fro);
      if (lane == 0) red[warp] = fro;
      if (tid == 0) { rot[0] = 0; rot[1] = 0; rot[2] = 0; }
      __syncthreads();
      if (warp == 0) {
        T f = lane < NWARP ? red[lane] : T(0);
        f = warp_sum(f);
        if (lane == 0) red[NWARP] = f;
      }
      __syncthreads();
      const T tinyY = red[NWARP] * num<T>::eps * num<T>::eps;
      if (zip) {
        // the zip-up's Y = M is graded by columns (P = U S), where the one-sided Jacobi is
        // accurate without preconditioning
        for (int e = tid; e < DP * npad; e += NT) { const int i = e % DP, j = e / DP; Vc[e] = (i == j) ? T(1) : T(0); }
        for (int e = tid; e < DP * (npad - n); e += NT) Yc[(size_t)n * DP + e] = T(0);
        __syncthreads();
      } else {
        // Preconditioning: Y = Q1 R1 (Householder, R1 n x n), R1^T = Q2 R2, so that
        // R1 = R2^T Q2^T and the right singular vectors of Y are V = Q2 Z with Z those of R2^T.
        // The Jacobi then runs on R2^T, whose columns are already close to orthogonal and
        // graded, so it needs fewer sweeps and leaves a smaller tilt in the kept subspace than
        // on Y itself (at L = 256, chi = 32 in FP32: about half the sweeps and a five-fold
        // smaller 99.9th percentile of the conditional error).  Q1 is not kept; Q2's reflectors
        // overwrite R_c (shared memory, or its slot of the global R store for CHI = 64: R_c is
        // not read again in this row), their coefficients go to csave.
        householder_r<T, D, D, NWARP>(Yc, DP, n, reinterpret_cast<T (*)[D]>(Vc), vcoef, nullptr, nullptr, lane, warp);
        for (int e = tid; e < DP * n; e += NT) {           // R1^T, rows n..DP-1 zero
          const int i = e % DP, j = e / DP;
          Vc[e] = (i < n && j <= i) ? Yc[(size_t)i * DP + j] : T(0);
        }
        householder_r<T, D, D, NWARP>(Vc, DP, n, reinterpret_cast<T (*)[D]>(Yc), vcoef, Rc, csave, lane, warp);
        for (int e = tid; e < DP * npad; e += NT) {        // R2^T in Y, zero outside n x n
          const int i = e % DP, j = e / DP;
          Yc[e] = (i < n && j < n && j <= i) ? Vc[(size_t)i * DP + j] : T(0);
        }
        __syncthreads();
        for (int e = tid; e < DP * npad; e += NT) { const int i = e % DP, j = e / DP; Vc[e] = (i == j) ? T(1) : T(0); }
        __syncthreads();
      }
      const T tol = jacobi_tol<T, D>();
      // One-sided Jacobi in a block-cyclic order.  The npad columns form NB = npad/4 blocks of
      // four; in each block-round (a round-robin over blocks) warp wj owns one block pair and
      // its four 8-lane groups orthogonalise the 16 cross pairs in four sub-rounds (group i:
      // column i of block A against column (i+t) mod 4 of block B), and in the first
      // block-round also the six pairs inside each of its two blocks (three sub-rounds).  Every
      // pair of columns meets once per sweep; the columns a warp touches in a block-round are
      // its own, so sub-rounds are ordered by __syncwarp and only block-rounds need the
      // CTA-wide barrier (NB-1 per sweep instead of npad-1).  8 lanes per pair, each lane
      // holding DP/8 rows of both columns in 16-byte vectors; the three dot products of a pair
      // are reduced together over the 8 lanes.
      constexpr int NJ = 8 * CHI;
      constexpr int VEC = JStride<T, CHI>::VEC;
      constexpr int NV = DP / (8 * VEC);
      using V16 = typename Vec16<T>::type;
      int sweep = 0;
      if (tid < NJ) {
        const int wj = tid >> 5, grp = (tid >> 3) & 3, li = tid & 7;
        const int NB = npad / 4, mb = NB - 1;
        const bool wact = wj < NB / 2;
        // The sweep is bound by shared-memory traffic at the occupancy the build runs at, so a
        // pair's V columns are read only when the pair rotates, and in the cross sub-rounds
        // each 8-lane group keeps its block-A column (Y and V) in registers.
        auto rotation = [&](const V16* u, const V16* w, T& cs, T& sn) -> bool {
          T g = 0, a = 0, b = 0;
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            g += dot16(u[k], w[k]);
            a += dot16(u[k], u[k]);
            b += dot16(w[k], w[k]);
          }
          g = group8_sum(g); a = group8_sum(a); b = group8_sum(b);
          if (a > tinyY && b > tinyY && g * g > tol * tol * a * b) {
            rotation_from_gram(a, b, g, cs, sn);
            return true;
          }
          return false;
        };
        auto jpair = [&](int p, int q) {          // both columns from shared memory
          V16* yp = reinterpret_cast<V16*>(Yc + (size_t)p * DP);
          V16* yq = reinterpret_cast<V16*>(Yc + (size_t)q * DP);
          V16 up[NV], uq[NV];
#pragma unroll
          for (int k = 0; k < NV; ++k) { up[k] = yp[li + 8 * k]; uq[k] = yq[li + 8 * k]; }
          T cs, sn;
          if (rotation(up, uq, cs, sn)) {
            V16* vp = reinterpret_cast<V16*>(Vc + (size_t)p * DP);
            V16* vq = reinterpret_cast<V16*>(Vc + (size_t)q * DP);
            V16 wp[NV], wq[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) { wp[k] = vp[li + 8 * k]; wq[k] = vq[li + 8 * k]; }
#pragma unroll
            for (int k = 0; k < NV; ++k) {
              rot16(up[k], uq[k], cs, sn);
              rot16(wp[k], wq[k], cs, sn);
              yp[li + 8 * k] = up[k];
              yq[li + 8 * k] = uq[k];
              vp[li + 8 * k] = wp[k];
              vq[li + 8 * k] = wq[k];
            }
            if (li == 0) rot[sweep % 3] = 1;
          }
        };
        for (; sweep < JacobiTol<T>::maxsw; ++sweep) {
          // clear the flag of sweep+1; the slot was last read at the end of sweep-2, and every
          // thread has passed a barrier of sweep-1 since (a two-slot ring would let a slow
          // thread read a flag that was already cleared and leave the loop alone)
          if (tid == 0) rot[(sweep + 1) % 3] = 0;
          for (int br = 0; br < mb; ++br) {
            if (wact) {       // warp-uniform: the shuffles of the reductions need the whole warp
              // block pair of slot wj (circle method: slot 0 keeps block NB-1)
              const int bA = wj == 0 ? NB - 1 : (br + wj) % mb;
              const int bB = wj == 0 ? br : (br - wj + mb) % mb;
              if (br == 0) {
                // pairs inside blocks A (groups 0, 1) and B (groups 2, 3):
                // {(0,1),(2,3)}, {(0,2),(1,3)}, {(0,3),(1,2)}
                const int blk = 4 * ((grp < 2) ? bA : bB), gi = grp & 1;
#pragma unroll 1
                for (int t = 0; t < 3; ++t) {
                  const int i = (t == 0) ? 2 * gi : gi;
                  const int j = (t == 0) ? 2 * gi + 1 : (t == 1 ? gi + 2 : 3 - gi);
                  jpair(blk + i, blk + j);
                  __syncwarp();
                }
              }
              // cross pairs: group grp holds column A = 4 bA + grp and meets the four columns
              // of block B in turn (B column (grp + t) mod 4 in sub-round t)
              const int pa = 4 * bA + grp;
              V16* ya_s = reinterpret_cast<V16*>(Yc + (size_t)pa * DP);
              V16* va_s = reinterpret_cast<V16*>(Vc + (size_t)pa * DP);
              V16 ya[NV], va[NV];
#pragma unroll
              for (int k = 0; k < NV; ++k) ya[k] = ya_s[li + 8 * k];
              bool va_held = false;   // group-uniform: every lane of a group sees the same sums
#pragma unroll 1
              for (int t = 0; t < 4; ++t) {
                const int q = 4 * bB + ((grp + t) & 3);
                V16* yq = reinterpret_cast<V16*>(Yc + (size_t)q * DP);
                V16 uq[NV];
#pragma unroll
                for (int k = 0; k < NV; ++k) uq[k] = yq[li + 8 * k];
                T cs, sn;
                if (rotation(ya, uq, cs, sn)) {
                  V16* vq = reinterpret_cast<V16*>(Vc + (size_t)q * DP);
                  V16 wq[NV];
                  if (!va_held) {
#pragma unroll
                    for (int k = 0; k < NV; ++k) va[k] = va_s[li + 8 * k];
                    va_held = true;
                  }
#pragma unroll
                  for (int k = 0; k < NV; ++k) wq[k] = vq[li + 8 * k];
#pragma unroll
                  for (int k = 0; k < NV; ++k) {
                    rot16(ya[k], uq[k], cs, sn);
                    rot16(va[k], wq[k], cs, sn);
                    yq[li + 8 * k] = uq[k];
                    vq[li + 8 * k] = wq[k];
                  }
                  if (li == 0) rot[sweep % 3] = 1;
                }
                __syncwarp();
              }
              if (va_held) {          // column A changed: back to shared memory
#pragma unroll
                for (int k = 0; k < NV; ++k) { ya_s[li + 8 * k] = ya[k]; va_s[li + 8 * k] = va[k]; }
              }
            }
            named_barrier(1, NJ);
          }
          if (rot[sweep % 3] == 0) break;
        }
      }
      __syncthreads();
      if (sweep + 1 > max_sweeps_seen) max_sweeps_seen = sweep + 1;
      if (sweep >= JacobiTol<T>::maxsw) ++unconverged;
      total_sweeps += (long long)min(sweep + 1, JacobiTol<T>::maxsw);
      ++n_svd;
      // singular values = column norms of the rotated Y
      for (int j = warp; j < n; j += NWARP) {
        T ss = 0;
        for (int i = lane; i < D; i += 32) ss += Yc[(size_t)j * DP + i] * Yc[(size_t)j * DP + i];
        ss = warp_sum(ss);
        if (lane == 0) sig[j] = ss;
      }
      __syncthreads();
      const int k = min(chi, min(dqr[c], n));
      if (tid < n) {
        const T sj = sig[tid];
        int rank = 0;
        for (int i = 0; i < n; ++i) { const T si = sig[i]; rank += (si > sj) || (si == sj && i < tid); }
        if (rank < k) sel[rank] = tid;
      }
      if (tid == 0) { knew[mir ? L - c : c] = k; knext_s = k; }
      __syncthreads();
      if (!zip) {
        // V_k = Q2 Z_sel = H_0 H_1 ... H_{n-1} Z_sel: each warp takes its selected columns into
        // registers, applies the reflectors from the last to the first, and writes the result to
        // column g of V (the selection becomes the identity)
        constexpr int RPL = D / 32 > 0 ? D / 32 : 1;
        constexpr int CPQ = (CHI + NWARP - 1) / NWARP;
        T xz[CPQ][RPL];
#pragma unroll
        for (int q = 0; q < CPQ; ++q) {
          const int g = warp + NWARP * q;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            xz[q][t] = (g < k && i < n) ? Vc[(size_t)sel[g] * DP + i] : T(0);
          }
        }
        __syncthreads();
        for (int j = n - 1; j >= 0; --j) {
          const T coef = csave[j];
          if (coef == T(0)) continue;
          T vr[RPL], d[CPQ];
#pragma unroll
          for (int t = 0; t < RPL; ++t) { const int i = lane + 32 * t; vr[t] = (i < n) ? Rc[(size_t)j * D + i] : T(0); }
#pragma unroll
          for (int q = 0; q < CPQ; ++q) {
            d[q] = 0;
#pragma unroll
            for (int t = 0; t < RPL; ++t) d[q] += vr[t] * xz[q][t];
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < CPQ; ++q) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
#pragma unroll
          for (int q = 0; q < CPQ; ++q) {
            const T dc = d[q] * coef;
#pragma unroll
            for (int t = 0; t < RPL; ++t) xz[q][t] -= dc * vr[t];
          }
        }
#pragma unroll
        for (int q = 0; q < CPQ; ++q) {
          const int g = warp + NWARP * q;
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if (g < k && i < n) Vc[(size_t)g * DP + i] = xz[q][t];
          }
        }
        __syncthreads();
        if (tid < k) sel[tid] = tid;
        __syncthreads();
        // R_{c-1} streams in while the tile and P are formed (the reflectors are consumed)
        if (!kBig && c > 1) prefetch_async(Rc, Rstore + (size_t)(c - 1) * D * D, D * D * (int)sizeof(T), tid, NT);
      }
      // B_r[c][y][al][be] = V[(y,be)][sel[al]]
      T* ctile = cur + (size_t)osite(c) * TILE;
      TE* etile = erow + (size_t)osite(c) * TILE;
      for (int e = tid; e < TILE; e += NT) {
        const int y = e / (CHI * CHI), i = (e / CHI) % CHI, j = e % CHI;
        const int al = mir ? j : i, be = mir ? i : j;       // frame bonds of lattice entry (i, j)
        T v = T(0);
        if (al < k && be < kn) v = Vc[(size_t)sel[al] * DP + y * kn + be];
        ctile[e] = v;
        etile[e] = env_store<TE, T>(v);
      }
      // P[(a,al)][g] = sum_j M[(a,al)][j] V[j][sel[g]]: 4 x 4 register tiles
      T pmax = 0;
      {
        constexpr int TI = D / 4, TG = CHI / 4;
        for (int u = tid; u < TI * TG; u += NT) {
          const int i0 = (u % TI) * 4, g0 = (u / TI) * 4;
          T acc[4][4] = {};
          if (g0 < k) {
            const T* vc[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) vc[jj] = Vc + (size_t)sel[(g0 + jj < k) ? g0 + jj : g0] * DP;
#pragma unroll 4
            for (int j = 0; j < n; ++j) {
              T mv[4], vv[4];
              ld4(Mc + (size_t)j * D + i0, mv);
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) vv[jj] = (g0 + jj < k) ? vc[jj][j] : T(0);
#pragma unroll
              for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += mv[ii] * vv[jj];
            }
          }
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const T col4[4] = {acc[0][jj], acc[1][jj], acc[2][jj], acc[3][jj]};
            st4(Ps + (size_t)(g0 + jj) * D + i0, col4);
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) { const T aa = acc[ii][jj] < T(0) ? -acc[ii][jj] : acc[ii][jj]; pmax = aa > pmax ? aa : pmax; }
          }
        }
      }
      pmax = warp_max(pmax);
      if (lane == 0) red[warp] = pmax;
      __syncthreads();
      if (warp == 0) {
        T f = lane < NWARP ? red[lane] : T(0);
        f = warp_max(f);
        if (lane == 0) red[NWARP] = f;
      }
      __syncthreads();
      const T pm = red[NWARP];
      const T pinv = pm > T(0) ? T(1) / pm : T(1);
      for (int e = tid; e < D * CHI; e += NT) Ps[e] *= pinv;
      if (tid == 0 && pm > T(0)) logs += log((double)pm);
      kn = knext_s;
      __syncthreads();
    }
    if (tid == 0) lam[r] = logs;
    __syncthreads();
  }

  // log Z = sum_r lam_r + log sum_x prod_c exp(beta Jh[0][c] s_c s_{c+1}) Gt_0(x)
  if constexpr (kBig) {
    // as below, each lane holding the bond indices lane + 32 e of the running vector
    constexpr int E = CHI / 32;
    if (warp == 0) {
      const T* row0 = rowbuf;
      double ell[2][E];
      double lsum = 0.0;
      for (int x = 0; x < 2; ++x) {
        const double h0 = hf ? exp(beta * (double)(hf[0] * spin_of(x))) : 1.0;
        for (int e = 0; e < E; ++e) ell[x][e] = h0 * (double)row0[x * CHI * CHI + 0 * CHI + lane + 32 * e];
      }
      for (int c = 1; c < L; ++c) {
        const T* t = row0 + (size_t)c * TILE;
        const double jb = beta * (double)Jh[c - 1];
        double nx[2][E];
        for (int x = 0; x < 2; ++x)
          for (int e = 0; e < E; ++e) nx[x][e] = 0.0;
        double f0[2], f1[2];
        for (int x = 0; x < 2; ++x) { f0[x] = exp(jb * spin_of(0) * spin_of(x)); f1[x] = exp(jb * spin_of(1) * spin_of(x)); }
        for (int h = 0; h < E; ++h)
          for (int j = 0; j < 32; ++j) {
            const int al = 32 * h + j;
            const double l0 = __shfl_sync(0xffffffffu, ell[0][h], j);
            const double l1 = __shfl_sync(0xffffffffu, ell[1][h], j);
            for (int x = 0; x < 2; ++x) {
              const double cf = f0[x] * l0 + f1[x] * l1;
              for (int e = 0; e < E; ++e) nx[x][e] += cf * (double)t[x * CHI * CHI + al * CHI + lane + 32 * e];
            }
          }
        if (hf)
          for (int x = 0; x < 2; ++x) {
            const double hc = exp(beta * (double)(hf[c] * spin_of(x)));
            for (int e = 0; e < E; ++e) nx[x][e] *= hc;
          }
        double mx = 0.0;
        for (int x = 0; x < 2; ++x)
          for (int e = 0; e < E; ++e) mx = fmax(mx, fabs(nx[x][e]));
        mx = warp_max(mx);
        for (int x = 0; x < 2; ++x)
          for (int e = 0; e < E; ++e) ell[x][e] = mx > 0.0 ? nx[x][e] / mx : nx[x][e];
        if (mx > 0.0) lsum += log(mx);
      }
      const double tot = __shfl_sync(0xffffffffu, ell[0][0] + ell[1][0], 0);
      if (lane == 0) {
        double s = 0.0;
        for (int rr = 0; rr < L; ++rr) s += lam[rr];
        args.logz[real] = s + lsum + log(tot);
        if (args.stats) {
          args.stats[real * 4 + 0] = max_sweeps_seen;
          args.stats[real * 4 + 1] = unconverged;
          args.stats[real * 4 + 2] = total_sweeps;
          args.stats[real * 4 + 3] = n_svd;
        }
      }
    }
  } else {
  if (warp == 0) {
    const T* row0 = rowbuf;   // row 0 lives in buffer (0 & 1) = 0
    double ell[2];            // lane holds ell[x][lane] for lane < CHI
    double lsum = 0.0;
    for (int x = 0; x < 2; ++x)
      ell[x] = (lane < CHI) ? (hf ? exp(beta * (double)(hf[0] * spin_of(x))) : 1.0) * (double)row0[x * CHI * CHI + 0 * CHI + lane] : 0.0;
    for (int c = 1; c < L; ++c) {
      const T* t = row0 + (size_t)c * TILE;
      const double jb = beta * (double)Jh[c - 1];
      double nx[2] = {0.0, 0.0};
      for (int al = 0; al < CHI; ++al) {
        const double l0 = __shfl_sync(0xffffffffu, ell[0], al);
        const double l1 = __shfl_sync(0xffffffffu, ell[1], al);
        for (int x = 0; x < 2; ++x) {
          const double f0 = exp(jb * spin_of(0) * spin_of(x)), f1 = exp(jb * spin_of(1) * spin_of(x));
          const double b = (lane < CHI) ? (double)t[x * CHI * CHI + al * CHI + lane] : 0.0;
          nx[x] += (f0 * l0 + f1 * l1) * b;
        }
      }
      if (hf) { nx[0] *= exp(beta * (double)hf[c]); nx[1] *= exp(-beta * (double)hf[c]); }
      double mx = fmax(fabs(nx[0]), fabs(nx[1]));
      mx = warp_max(mx);
      if (mx > 0.0) { nx[0] /= mx; nx[1] /= mx; lsum += log(mx); }
      ell[0] = nx[0]; ell[1] = nx[1];
    }
    const double tot = __shfl_sync(0xffffffffu, ell[0] + ell[1], 0);
    if (lane == 0) {
      double s = 0.0;
      for (int rr = 0; rr < L; ++rr) s += lam[rr];
      args.logz[real] = s + lsum + log(tot);
      if (args.stats) {
        args.stats[real * 4 + 0] = max_sweeps_seen;
        args.stats[real * 4 + 1] = unconverged;
        args.stats[real * 4 + 2] = total_sweeps;
        args.stats[real * 4 + 3] = n_svd;
      }
    }
  }
  }
}

template <typename T, typename TE, int CHI>
cudaError_t launch_env_build_t(const EnvBuildArgs<T, TE>& a, cudaStream_t st) {
  using C = EnvCfg<CHI>;
  // + the two rows' couplings (int8) staged behind the tile
  const size_t smem = env_smem_elems<T, CHI>() * sizeof(T) + (size_t)2 * a.L + 16;
  cudaError_t e = cudaFuncSetAttribute(env_build_kernel<T, TE, CHI>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  env_build_kernel<T, TE, CHI><<<a.n_real, C::NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, typename TE>
cudaError_t launch_env_build(const EnvBuildArgs<T, TE>& a, int CHI, cudaStream_t st) {
  switch (CHI) {
    case 4: return launch_env_build_t<T, TE, 4>(a, st);
    case 8: return launch_env_build_t<T, TE, 8>(a, st);
    case 16: return launch_env_build_t<T, TE, 16>(a, st);
    case 32: return launch_env_build_t<T, TE, 32>(a, st);
    case 64:
      if constexpr (sizeof(T) == 4) return launch_env_build_t<T, TE, 64>(a, st);  // FP64 does not fit
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_env_build<double, double>(const EnvBuildArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_env_build<float, float>(const EnvBuildArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_env_build<float, __nv_bfloat16>(const EnvBuildArgs<float, __nv_bfloat16>&, int, cudaStream_t);

template <typename T, typename TE, int CHI>
static cudaError_t occupancy_t(int L, int* per_sm) {
  using C = EnvCfg<CHI>;
  const size_t smem = env_smem_elems<T, CHI>() * sizeof(T) + (size_t)2 * L + 16;
  cudaError_t e = cudaFuncSetAttribute(env_build_kernel<T, TE, CHI>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, env_build_kernel<T, TE, CHI>, C::NT, smem);
}

cudaError_t env_build_occupancy(int L, int CHI, int precision, int* per_sm) {
#define TNMC_OCC(T, TE)                                           \
  switch (CHI) {                                                  \
    case 4: return occupancy_t<T, TE, 4>(L, per_sm);              \
    case 8: return occupancy_t<T, TE, 8>(L, per_sm);              \
    case 16: return occupancy_t<T, TE, 16>(L, per_sm);            \
    case 32: return occupancy_t<T, TE, 32>(L, per_sm);            \
    case 64:                                                      \
      if constexpr (sizeof(T) == 4) return occupancy_t<T, TE, 64>(L, per_sm); \
      return cudaErrorInvalidValue;                               \
    default: return cudaErrorInvalidValue;                        \
  }
  if (precision == 0) { TNMC_OCC(double, double) }
  if (precision == 2) { TNMC_OCC(float, __nv_bfloat16) }
  TNMC_OCC(float, float)
#undef TNMC_OCC
}

size_t env_build_smem_bytes(int CHI, bool fp64) {
  const size_t el = fp64 ? 8 : 4;
  switch (CHI) {
    case 4: return env_smem_elems<float, 4>() * el;
    case 8: return env_smem_elems<float, 8>() * el;
    case 16: return env_smem_elems<float, 16>() * el;
    case 32: return env_smem_elems<float, 32>() * el;
    case 64: return fp64 ? 0 : env_smem_elems<float, 64>() * el;
    default: return 0;
  }
}

}  // namespace tnmc
