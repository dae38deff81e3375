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
//          before site c (the left part is Q_{<c} R_c with Q an isometry).  One-sided
//          (Hestenes) Jacobi SVD of Y keeps the top k = min(chi, d_c, 2 k_{c+1}) right
//          singular vectors V; B_r[c] = V^T (right-canonical), P = M V carries the rest of
//          the state to site c-1.  Site 0 keeps the normalised remainder; lam_r = log of the
//          removed scale.
// This is the QR-sweep + truncating-SVD-sweep compression of the oracle, computed without
// forming Q: the truncated MPS is the same up to gauge (and rounding).
#include "common.cuh"
#include "kernels.h"

namespace tnmc {

// Convergence: a pair counts as orthogonal when |y_p . y_q| <= tol |y_p| |y_q|.  The
// rounding floor of a D-long dot product is about sqrt(D) eps, so tol = 4 sqrt(D) eps
// (the criterion of one-sided Jacobi SVD codes, scaled for a safety margin).
template <typename T> struct JacobiTol;
template <> struct JacobiTol<float> { static constexpr int maxsw = 30; };
template <> struct JacobiTol<double> { static constexpr int maxsw = 40; };
template <typename T, int D> __device__ __forceinline__ T jacobi_tol() {
  return T(4) * num<T>::sqrt_(T(D)) * num<T>::eps;
}

template <int CHI> struct EnvCfg {
  static constexpr int D = 2 * CHI;                 // MPO bond x MPS bond
  static constexpr int NWARP = CHI < 4 ? 4 : CHI;   // one warp per Jacobi pair
  static constexpr int NT = 32 * NWARP;
  static constexpr int TILE = 2 * CHI * CHI;        // [y][alpha][beta]
};

template <typename T, int CHI>
__host__ __device__ constexpr size_t env_smem_elems() {
  // backward: M, Y, V, R (D*D each) + P (D*CHI) + Q (2*CHI*CHI) + tile (2*CHI*CHI)
  // forward : X (2D*D) + R (D*D) + tile -- the union is the backward footprint
  return (size_t)4 * (2 * CHI) * (2 * CHI) + (size_t)(2 * CHI) * CHI + 2 * (size_t)2 * CHI * CHI;
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
__global__ void __launch_bounds__(EnvCfg<CHI>::NT)
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
  // backward-phase layout
  T* Mc = sm;                 // D x D   col-major, compact columns j = x*kn + g
  T* Yc = Mc + D * D;         // D x D   col-major
  T* Vc = Yc + D * D;         // D x D   col-major (rows < n)
  T* Rc = Vc + D * D;         // D x D   col-major R_c
  T* Ps = Rc + D * D;         // D x CHI col-major: P[(b,be)][g] at g*D + b*CHI + be
  T* Qs = Ps + D * CHI;       // 2 x CHI x CHI: Q[b][al][g]
  T* Bt = Qs + TILE;          // previous-row tile [y][al][be]
  // forward-phase layout (aliases M/Y/V; R stays at Rc)
  T* Xs = sm;                 // 2D x D col-major

  __shared__ T Wc[8];               // W[x][a][b] at x*4 + a*2 + b
  __shared__ T vbuf[2][2 * D];      // Householder vectors (double-buffered)
  __shared__ T vcoef[2];
  __shared__ T red[32];
  __shared__ T sig[D];
  __shared__ int sel[CHI];
  __shared__ int rot[2];
  __shared__ int knext_s;

  const int8_t* J = args.J + (size_t)real * 2 * L * (L - 1);
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

    // QR bond dimensions d_c of the MPO x MPS (left-canonical form)
    if (tid == 0) {
      dqr[0] = 1;
      for (int c = 0; c < L - 1; ++c) dqr[c + 1] = min(2 * dqr[c], 2 * kold[c + 1]);
    }
    // R_0 = [1]
    for (int e = tid; e < D * D; e += NT) Rc[e] = (e == 0) ? T(1) : T(0);
    if (tid == 0) {
      for (int e = 0; e < D * D; ++e) Rstore[e] = (e == 0) ? T(1) : T(0);
    }
    __syncthreads();

    // ---------------- forward sweep: R factors of the left parts ----------------
    for (int c = 0; c < L - 1; ++c) {
      const T* btile = prev + (size_t)c * TILE;
      for (int e = tid; e < TILE; e += NT) Bt[e] = btile[e];
      if (tid < 8) {
        const int x = tid >> 2, a = (tid >> 1) & 1, b = tid & 1;
        double w = exp(beta * (double)Jv[(size_t)r * L + c] * spin_of(x) * spin_of(b));
        if (c > 0) w *= exp(beta * (double)Jh[(size_t)(r + 1) * (L - 1) + c - 1] * spin_of(a) * spin_of(b));
        else if (a == 1) w = 0.0;
        Wc[tid] = (T)w;
      }
      __syncthreads();
      // X[(x,i),(b,be)] = sum_al (W(x,0,b) R[i][al] + W(x,1,b) R[i][CHI+al]) B[b][al][be]
      for (int e = tid; e < 2 * D * D; e += NT) {
        const int row = e % (2 * D), col = e / (2 * D);
        const int x = row / D, i = row % D, b = col / CHI, be = col % CHI;
        const T w0 = Wc[x * 4 + 0 * 2 + b], w1 = Wc[x * 4 + 1 * 2 + b];
        const T* bb = Bt + b * CHI * CHI + be;
        T acc = 0;
#pragma unroll 8
        for (int al = 0; al < CHI; ++al)
          acc += (w0 * Rc[al * D + i] + w1 * Rc[(CHI + al) * D + i]) * bb[al * CHI];
        Xs[e] = acc;
      }
      __syncthreads();
      // Householder QR of X (m = 2D rows, D columns); warp (j % NWARP) owns column j.
      constexpr int m = 2 * D;
      const T tiny = (sizeof(T) == 4) ? T(1e-36) : T(1e-300);
      auto house = [&](int j) {   // executed by the owning warp for column j
        T* col = Xs + (size_t)j * m;
        T ss = 0;
        for (int i = j + lane; i < m; i += 32) ss += col[i] * col[i];
        ss = warp_sum(ss);
        const T x0 = col[j];
        __syncwarp();
        if (ss <= tiny) {
          for (int i = j + 1 + lane; i < m; i += 32) col[i] = T(0);
          if (lane == 0) vcoef[j & 1] = T(0);
        } else {
          const T nrm = num<T>::sqrt_(ss);
          const T alpha = x0 >= T(0) ? -nrm : nrm;
          const T v0 = x0 - alpha;
          for (int i = j + lane; i < m; i += 32) vbuf[j & 1][i] = (i == j) ? v0 : col[i];
          __syncwarp();
          for (int i = j + lane; i < m; i += 32) col[i] = (i == j) ? alpha : T(0);
          if (lane == 0) vcoef[j & 1] = T(1) / (nrm * (nrm + (x0 >= T(0) ? x0 : -x0)));  // 2/|v|^2
        }
      };
      if (warp == 0) house(0);
      for (int j = 0; j < D; ++j) {
        __syncthreads();
        const T coef = vcoef[j & 1];
        if (coef != T(0)) {
          const T* v = vbuf[j & 1];
          for (int k = j + 1 + ((warp - (j + 1)) % NWARP + NWARP) % NWARP; k < D; k += NWARP) {
            T* col = Xs + (size_t)k * m;
            T d = 0;
            for (int i = j + lane; i < m; i += 32) d += v[i] * col[i];
            d = warp_sum(d) * coef;
            for (int i = j + lane; i < m; i += 32) col[i] -= d * v[i];
          }
        }
        __syncwarp();
        if (j + 1 < D && warp == (j + 1) % NWARP) house(j + 1);
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
        Rc[e] = v;
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
      const T* btile = prev + (size_t)c * TILE;
      for (int e = tid; e < TILE; e += NT) Bt[e] = btile[e];
      if (tid < 8) {
        const int x = tid >> 2, a = (tid >> 1) & 1, b = tid & 1;
        double w = exp(beta * (double)Jv[(size_t)r * L + c] * spin_of(x) * spin_of(b));
        if (c > 0) w *= exp(beta * (double)Jh[(size_t)(r + 1) * (L - 1) + c - 1] * spin_of(a) * spin_of(b));
        else if (a == 1) w = 0.0;
        Wc[tid] = (T)w;
      }
      __syncthreads();
      // Q[b][al][g] = sum_be B[b][al][be] P[(b,be)][g]
      for (int e = tid; e < TILE; e += NT) {
        const int b = e / (CHI * CHI), al = (e / CHI) % CHI, g = e % CHI;
        T acc = 0;
        if (g < kn) {
#pragma unroll 8
          for (int be = 0; be < CHI; ++be) acc += Bt[b * CHI * CHI + al * CHI + be] * Ps[g * D + b * CHI + be];
        }
        Qs[e] = acc;
      }
      __syncthreads();
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
        for (int e = tid; e < TILE; e += NT) {
          const int y = e / (CHI * CHI), al = (e / CHI) % CHI, be = e % CHI;
          const T v = (al == 0 && be < kn) ? Mc[(size_t)(y * kn + be) * D] * inv : T(0);
          cur[e] = v;
          erow[e] = env_store<TE, T>(v);
        }
        if (tid == 0) { logs += log((double)nrm); knew[0] = 1; }
        __syncthreads();
        break;
      }
      // Y = R_c M  (D x n); the R factor of the left part up to site c-1
      const T* Rin = Rstore + (size_t)c * D * D;
      for (int e = tid; e < D * D; e += NT) Rc[e] = Rin[e];
      __syncthreads();
      T fro = 0;
      for (int e = tid; e < D * n; e += NT) {
        const int i = e % D, j = e / D;
        T acc = 0;
#pragma unroll 8
        for (int l = 0; l < D; ++l) acc += Rc[l * D + i] * Mc[(size_t)j * D + l];
        Yc[e] = acc;
        fro += acc * acc;
      }
      for (int e = tid; e < D * n; e += NT) { const int i = e % D, j = e / D; Vc[e] = (i == j) ? T(1) : T(0); }
      fro = warp_sum(fro);
      if (lane == 0) red[warp] = fro;
      if (tid == 0) { rot[0] = 0; rot[1] = 0; }
      __syncthreads();
      if (warp == 0) {
        T f = lane < NWARP ? red[lane] : T(0);
        f = warp_sum(f);
        if (lane == 0) red[NWARP] = f;
      }
      __syncthreads();
      const T tinyY = red[NWARP] * num<T>::eps * num<T>::eps;
      const T tol = jacobi_tol<T, D>();
      int sweep = 0;
      for (; sweep < JacobiTol<T>::maxsw; ++sweep) {
        if (tid == 0) rot[(sweep + 1) & 1] = 0;
        for (int rd = 0; rd < n - 1; ++rd) {
          if (warp < n / 2) {
            int p, q;
            Pair<CHI>::get(n, rd, warp, p, q);
            T* yp = Yc + (size_t)p * D;
            T* yq = Yc + (size_t)q * D;
            T a = 0, b = 0, g = 0;
#pragma unroll
            for (int t = 0; t < D / 32 + (D % 32 ? 1 : 0); ++t) {
              const int i = lane + 32 * t;
              if (i < D) { const T u = yp[i], v = yq[i]; a += u * u; b += v * v; g += u * v; }
            }
            a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
            const T ag = g < T(0) ? -g : g;
            if (a > tinyY && b > tinyY && ag > tol * num<T>::sqrt_(a) * num<T>::sqrt_(b)) {
              const T z = (b - a) / (T(2) * g);
              const T az = z < T(0) ? -z : z;
              T t = (az > T(1e15)) ? T(0.5) / az : T(1) / (az + num<T>::sqrt_(T(1) + z * z));
              if (z < T(0)) t = -t;
              const T cs = T(1) / num<T>::sqrt_(T(1) + t * t), sn = cs * t;
#pragma unroll
              for (int tt = 0; tt < D / 32 + (D % 32 ? 1 : 0); ++tt) {
                const int i = lane + 32 * tt;
                if (i < D) { const T u = yp[i], v = yq[i]; yp[i] = cs * u - sn * v; yq[i] = sn * u + cs * v; }
                if (i < n) {
                  T* vp = Vc + (size_t)p * D; T* vq = Vc + (size_t)q * D;
                  const T u = vp[i], v = vq[i]; vp[i] = cs * u - sn * v; vq[i] = sn * u + cs * v;
                }
              }
              if (lane == 0) rot[sweep & 1] = 1;
            }
          }
          __syncthreads();
        }
        if (rot[sweep & 1] == 0) break;
      }
      if (sweep + 1 > max_sweeps_seen) max_sweeps_seen = sweep + 1;
      if (sweep >= JacobiTol<T>::maxsw) ++unconverged;
      total_sweeps += (long long)min(sweep + 1, JacobiTol<T>::maxsw);
      ++n_svd;
      // singular values = column norms of the rotated Y
      for (int j = warp; j < n; j += NWARP) {
        T ss = 0;
        for (int i = lane; i < D; i += 32) ss += Yc[(size_t)j * D + i] * Yc[(size_t)j * D + i];
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
      if (tid == 0) { knew[c] = k; knext_s = k; }
      __syncthreads();
      // B_r[c][y][al][be] = V[(y,be)][sel[al]]
      T* ctile = cur + (size_t)c * TILE;
      TE* etile = erow + (size_t)c * TILE;
      for (int e = tid; e < TILE; e += NT) {
        const int y = e / (CHI * CHI), al = (e / CHI) % CHI, be = e % CHI;
        T v = T(0);
        if (al < k && be < kn) v = Vc[(size_t)sel[al] * D + y * kn + be];
        ctile[e] = v;
        etile[e] = env_store<TE, T>(v);
      }
      // P[(a,al)][g] = sum_j M[(a,al)][j] V[j][sel[g]]
      T pmax = 0;
      for (int e = tid; e < D * CHI; e += NT) {
        const int row = e % D, g = e / D;
        T acc = 0;
        if (g < k) {
          const T* vcol = Vc + (size_t)sel[g] * D;
          for (int j = 0; j < n; ++j) acc += Mc[(size_t)j * D + row] * vcol[j];
        }
        Ps[e] = acc;
        const T aa = acc < T(0) ? -acc : acc;
        pmax = aa > pmax ? aa : pmax;
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
  if (warp == 0) {
    const T* row0 = rowbuf;   // row 0 lives in buffer (0 & 1) = 0
    double ell[2];            // lane holds ell[x][lane] for lane < CHI
    double lsum = 0.0;
    for (int x = 0; x < 2; ++x) ell[x] = (lane < CHI) ? (double)row0[x * CHI * CHI + 0 * CHI + lane] : 0.0;
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

template <typename T, typename TE, int CHI>
cudaError_t launch_env_build_t(const EnvBuildArgs<T, TE>& a, cudaStream_t st) {
  using C = EnvCfg<CHI>;
  const size_t smem = env_smem_elems<T, CHI>() * sizeof(T);
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
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_env_build<double, double>(const EnvBuildArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_env_build<float, float>(const EnvBuildArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_env_build<float, __nv_bfloat16>(const EnvBuildArgs<float, __nv_bfloat16>&, int, cudaStream_t);

size_t env_build_smem_bytes(int CHI, bool fp64) {
  const size_t el = fp64 ? 8 : 4;
  switch (CHI) {
    case 4: return env_smem_elems<float, 4>() * el;
    case 8: return env_smem_elems<float, 8>() * el;
    case 16: return env_smem_elems<float, 16>() * el;
    case 32: return env_smem_elems<float, 32>() * el;
    default: return 0;
  }
}

}  // namespace tnmc
