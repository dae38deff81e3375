// Device helpers shared by the TNMC kernels: Philox4x32-10, spin/tensor conventions,
// status bits and element conversions.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"

namespace tnmc {

enum : uint32_t { PURPOSE_BOND = 0u, PURPOSE_SPIN = 1u, PURPOSE_ACCEPT = 2u, PURPOSE_LINES = 3u };

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the multiply-xor bijection with
// the key bumped by the Weyl constants between rounds.
struct Philox4 { uint32_t x0, x1, x2, x3; };

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

// 53-bit uniform in [0,1) from two 32-bit words.
__host__ __device__ __forceinline__ double u53(uint32_t x0, uint32_t x1) {
  const double a = (double)(x0 >> 5), b = (double)(x1 >> 6);
  return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0);
}

__host__ __device__ __forceinline__ double uniform(uint64_t seed, uint32_t c0, uint32_t c1,
                                                   uint32_t c2, uint32_t purpose) {
  const Philox4 o = philox4x32_10(c0, c1, c2, purpose, (uint32_t)seed, (uint32_t)(seed >> 32));
  return u53(o.x0, o.x1);
}

// Spin value of tensor index 0/1.
__host__ __device__ __forceinline__ int spin_of(int idx) { return 1 - 2 * idx; }

template <typename T> struct num;
template <> struct num<double> {
  static constexpr double eps = 2.220446049250313e-16;
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
};
template <> struct num<float> {
  static constexpr float eps = 1.1920928955078125e-07f;
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
};

// Environment storage element conversions.
template <typename TE> __device__ __forceinline__ float to_f(TE v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename TE> __device__ __forceinline__ T env_load(TE v) { return (T)to_f<TE>(v); }
template <> __device__ __forceinline__ double env_load<double, double>(double v) { return v; }

template <typename TE, typename T> __device__ __forceinline__ TE env_store(T v);
template <> __device__ __forceinline__ double env_store<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float env_store<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float env_store<float, double>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 env_store<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ void set_status(unsigned* st, unsigned bit) {
  if (st) atomicOr(st, bit);
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) { T w = __shfl_xor_sync(0xffffffffu, v, o); v = v > w ? v : w; }
  return v;
}

}  // namespace tnmc
