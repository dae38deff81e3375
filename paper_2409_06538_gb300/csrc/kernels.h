// Internal launch interface between the C ABI (capi.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

namespace tnmc {

// Device status bits (OR-ed into the context's status word).
enum : unsigned {
  ST_NUMERIC = 1u,   // w(+)+w(-) <= 0 or not finite while sampling
  ST_TIMEOUT = 2u,   // a bounded wait ran out
  ST_ARG = 4u,       // a kernel found an argument outside what it was built for
};

template <typename T, typename TE>
struct EnvBuildArgs {
  int L, n_real, chi;
  const int8_t* J;        // [real][2L(L-1)]
  const double* beta;     // [real]
  TE* env;                // [real][L rows][L sites][2*CHI*CHI]
  int* kdim;              // [real][L rows][L+1]
  int* dqr;               // [real][L+1] scratch
  double* lam;            // [real][L]
  double* logz;           // [real]
  T* rowbuf;              // [real][2][L][2*CHI*CHI] scratch (build precision)
  T* Rstore;              // [real][L][D*D] scratch
  long long* stats;       // [real][4]: max Jacobi sweeps, unconverged SVDs, total sweeps, SVDs (nullable)
  unsigned* status;
  T* Mscratch = nullptr;  // [real][D*D] scratch, used only when CHI = 64 (M does not fit in shared memory)
  const int8_t* hfield = nullptr;   // [real][L][L] external fields in units of beta (weight exp(beta k s)), nullable
  int zipup = 0;                    // 1: zip-up compression (tnmc_compression), else canonical
};

template <typename T, typename TE>
cudaError_t launch_env_build(const EnvBuildArgs<T, TE>& a, int CHI, cudaStream_t st);
size_t env_build_smem_bytes(int CHI, bool fp64);
// Environment-build CTAs (one per realization) that fit on one SM at this L, CHI and precision.
cudaError_t env_build_occupancy(int L, int CHI, int precision, int* per_sm);

struct SampleArgs {
  int L, n_real, n_chains, n;      // proposals per chain in this call
  int n_items;                     // per realization: n_chains * n (or n for eval)
  uint64_t step0;
  const int8_t* J;                 // [real][2L(L-1)]
  const double* beta;              // [real]
  const uint64_t* seeds;           // [real]
  const void* env;                 // [real][L][L][2*CHI*CHI] of TE
  // outputs (per item = real * n_items + k)
  uint32_t* spins_packed;          // [item][L*L/32 rounded up] bit 1 <-> s = -1
  int words;                       // packed words per configuration
  double* logq;                    // [item]
  int32_t* energy;                 // [item] (nullable)
  int32_t* magnet;                 // [item] (nullable)
  int64_t* clamps;                 // [real] accumulated (nullable)
  // teacher forcing
  const int8_t* forced;            // [item][L*L] +-1 or nullptr (then Philox draws)
  double* qplus;                   // [item][L*L] (nullable)
  // scratch
  void* work;                      // [grid][warps][L][2*CHI] of compute type
  unsigned* status;
  unsigned* real_status;           // [real] per-realization status bits (nullable)
  const int8_t* hfield;            // [real][L][L] external fields in units of beta (nullable)
  const int* chain_of;             // [real] chain index of the draws' counters (nullable: item / n)
};

cudaError_t launch_sample(const SampleArgs& a, int precision, int CHI, int num_sms, cudaStream_t st);
// tensor-core (tcgen05, 3xTF32) sampler of the mixed path; CHI 16 or 32
bool sample_tc_supported(int CHI);
// Self-test of the sampler's bounded mbarrier wait (see sample_tc.cu).
cudaError_t launch_wait_probe(int arrive, long long limit, unsigned* status_dev, cudaStream_t st);
cudaError_t launch_sample_tc(const SampleArgs& a, int CHI, int num_sms, cudaStream_t st);
size_t sample_tc_work_bytes(int L, int CHI, int num_sms);
size_t sample_work_bytes(int L, int CHI, int precision, int num_sms);

struct AcceptArgs {
  int L, n_real, n_chains, n, words, n_therm;
  uint64_t step0;
  const double* beta;
  const uint64_t* seeds;
  const double* logq;              // [real][chain][k]
  const int32_t* energy;
  const int32_t* magnet;
  const uint32_t* spins_packed;    // [real][chain][k][words]
  uint8_t* accepted;               // nullable
  // chain state (persist across calls), per (real, chain)
  int* have_state;                 // 0/1
  double* cur_logq;
  int32_t* cur_energy;
  int32_t* cur_magnet;
  uint32_t* cur_spins;             // [real][chain][words]
  double* acc;                     // [real][16] accumulators
  int* cur_idx;                    // [real][chain][k] scratch: current state after step k
  const int* nlimit;               // [real] proposals per chain a realization uses in all, counted
                                   // from step 0; later steps are skipped (nullable: no limit)
  unsigned* status;
};
cudaError_t launch_accept(const AcceptArgs& a, cudaStream_t st);

cudaError_t launch_couplings(int L, int n_real, const uint64_t* seeds_dev, double p, int8_t* out,
                             cudaStream_t st);
cudaError_t launch_couplings_pvec(int L, int n_real, const uint64_t* seeds_dev, const double* p_dev, int8_t* out,
                                  cudaStream_t st);
cudaError_t launch_unpack(const uint32_t* packed, int words, int N, int64_t n_cfg, int8_t* out,
                          cudaStream_t st);

// accumulator slots in AcceptArgs::acc
enum AccSlot {
  ACC_NPROP = 0, ACC_NACC, ACC_NMEAS, ACC_NMEASQ, ACC_E, ACC_E2, ACC_MABS, ACC_M2, ACC_M4,
  ACC_Q, ACC_QABS, ACC_Q2, ACC_Q4, ACC_MEDGE, ACC_MEDGEABS, ACC_MEDGE2,
  ACC_NTEST,            // Metropolis tests: proposals after each chain's initial state
  ACC_SLOTS = 17
};

}  // namespace tnmc
