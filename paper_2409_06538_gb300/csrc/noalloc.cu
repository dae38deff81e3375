// Environment build that allocates nothing: the scratch of the build kernel (the R factors
// of the forward sweep, the two working rows, the bond-dimension array, statistics and the
// status word) lives in one file-scope device array instead of cudaMalloc'd memory.
//
// Some callers cannot call cudaMalloc: an application that reserves all device memory up
// front and forbids allocation afterwards, or a latency-critical path where cudaMalloc's
// device-wide synchronisation is not allowed.  They pass every input and output buffer;
// this entry point uses only the array below for everything else.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <mutex>
#include <string>

#include "../../include/tnmc.h"
#include "kernels.h"

namespace {

// 32 MiB of scratch, held by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// The status code is the whole error report of this entry point; the text is kept for a
// debugger only (written under g_err_mu, since calls may come from several threads).
std::mutex g_err_mu;
std::string g_err;

tnmc_status err(tnmc_status s, const std::string& m) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = m;
  return s;
}

// Device address of the scratch array for the current device (set-up once per device, with
// that device current; host code must not use the symbol itself as an address).
tnmc_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(TNMC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return err(TNMC_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return err(TNMC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return TNMC_OK;
}

int round_chi(int chi) {
  return chi <= 4 ? 4 : chi <= 8 ? 8 : chi <= 16 ? 16 : chi <= 32 ? 32 : 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T, typename TE>
tnmc_status run(int L, int n_real, int chi, int CHI, const int8_t* J, const double* beta, void* env,
                int32_t* kdim, double* lam, double* logz, cudaStream_t st, unsigned char* base) {
  const int D = 2 * CHI;
  const size_t tile = (size_t)2 * CHI * CHI;
  size_t off = 0;
  unsigned* status = reinterpret_cast<unsigned*>(base + off);  off += align256(sizeof(unsigned));
  long long* stats = reinterpret_cast<long long*>(base + off); off += align256(sizeof(long long) * 4 * n_real);
  int* dqr = reinterpret_cast<int*>(base + off);               off += align256(sizeof(int) * (size_t)n_real * (L + 1));
  T* rowbuf = reinterpret_cast<T*>(base + off);                off += align256(sizeof(T) * (size_t)n_real * 2 * L * tile);
  T* Rstore = reinterpret_cast<T*>(base + off);                off += align256(sizeof(T) * (size_t)n_real * L * D * D);
  if (off > kNoAllocScratchBytes)
    return err(TNMC_ERR_ARG, "tnmc_build_env_noalloc: needs " + std::to_string(off) + " bytes of scratch, the limit is " +
                                 std::to_string(kNoAllocScratchBytes) + " (reduce n_real, L or chi)");
  // the build kernel writes no status (it has no failure to report), but the word is cleared
  // so that the scratch a call leaves behind never carries another call's bits; every other
  // scratch word is written before it is read
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return err(TNMC_ERR_CUDA, std::string("status reset: ") + cudaGetErrorString(e));
  tnmc::EnvBuildArgs<T, TE> a{L, n_real, chi, J, beta, static_cast<TE*>(env), kdim, dqr, lam, logz, rowbuf, Rstore,
                              stats, status};
  e = tnmc::launch_env_build(a, CHI, st);
  if (e != cudaSuccess) return err(TNMC_ERR_CUDA, std::string("env build launch: ") + cudaGetErrorString(e));
  return TNMC_OK;
}

}  // namespace

extern "C" tnmc_status tnmc_build_env_noalloc(int L, int n_real, int chi, int precision, const int8_t* couplings_dev,
                                              const double* beta_dev, void* env_dev, int32_t* kdim_dev,
                                              double* lam_dev, double* logz_dev, void* stream) {
  if (L < 2 || n_real < 1 || chi < 1) return err(TNMC_ERR_ARG, "tnmc_build_env_noalloc: invalid size");
  if (!couplings_dev || !beta_dev || !env_dev || !kdim_dev || !lam_dev || !logz_dev)
    return err(TNMC_ERR_ARG, "tnmc_build_env_noalloc: NULL buffer");
  const int CHI = round_chi(chi);
  if (!CHI) return err(TNMC_ERR_UNSUPPORTED, "tnmc_build_env_noalloc: chi > 32");
  unsigned char* base = nullptr;
  tnmc_status s = scratch_for_current_device(&base);
  if (s) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  switch (precision) {
    case TNMC_FP64:
      return run<double, double>(L, n_real, chi, CHI, couplings_dev, beta_dev, env_dev, kdim_dev, lam_dev, logz_dev, st, base);
    case TNMC_FP32:
    case TNMC_MIXED_TF32:
      return run<float, float>(L, n_real, chi, CHI, couplings_dev, beta_dev, env_dev, kdim_dev, lam_dev, logz_dev, st, base);
    case TNMC_MIXED_BF16:
      return run<float, __nv_bfloat16>(L, n_real, chi, CHI, couplings_dev, beta_dev, env_dev, kdim_dev, lam_dev, logz_dev, st, base);
    default:
      return err(TNMC_ERR_ARG, "tnmc_build_env_noalloc: unknown precision");
  }
}
