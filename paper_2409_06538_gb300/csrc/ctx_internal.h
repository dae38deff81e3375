// Library-internal entry points on a TNMC context, used by the request server (server.cu) to
// run batches asynchronously on pooled contexts.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "../../include/tnmc.h"

namespace tnmc {

// Fill a tnmc_obs from one realization's accumulator row (ACC_SLOTS doubles) and clamp count.
void obs_from_acc(const double* acc_row, int64_t clamps, tnmc_obs* out);

// Start a batch of n_active <= capacity realizations with their own seeds, inverse
// temperatures, antiferromagnetic-bond probabilities and total proposals per chain:
// generates the couplings on the device and resets the chains.  Asynchronous on the
// context's stream; the host arrays may be reused on return.
tnmc_status ctx_begin_batch(tnmc_ctx* c, int n_active, const uint64_t* seeds, const double* betas,
                            const double* ps, const int* nlimits);

// Queue copies of the batch results into pinned host memory: accumulators (n_active x
// ACC_SLOTS), clamp counts and log Z (n_active), build statistics (4 n_active), the context's
// status word and the per-realization status words (n_active).
tnmc_status ctx_enqueue_readback(tnmc_ctx* c, double* acc_h, int64_t* clamps_h, double* logz_h,
                                 long long* stats_h, unsigned* status_h, unsigned* rstatus_h);

int ctx_capacity(const tnmc_ctx* c);

// Device memory owned by the context (released with it), from the same allocator as its buffers.
tnmc_status ctx_alloc(tnmc_ctx* c, void** p, size_t bytes);
// Device couplings [real][2L(L-1)] of the context, for a caller that writes them in place
// (the periodic driver) before tnmc_build_env.
int8_t* ctx_couplings_dev(tnmc_ctx* c);
// Use a device array [real][L][L] of external fields (units of beta) owned by the caller.
tnmc_status ctx_use_fields_dev(tnmc_ctx* c, int8_t* fields_dev);
// Chain index of each realization's spin draws (device [real]), or nullptr.
void ctx_set_chain_of(tnmc_ctx* c, const int* chain_of_dev);
// Outputs of the last tnmc_propose / state of the context, on the device.
const uint32_t* ctx_packed(const tnmc_ctx* c);
const double* ctx_logq(const tnmc_ctx* c);
const int32_t* ctx_energy(const tnmc_ctx* c);
const unsigned* ctx_realization_status_dev(const tnmc_ctx* c);
const int64_t* ctx_clamps_dev(const tnmc_ctx* c);
int ctx_words(const tnmc_ctx* c);
void ctx_add_launches(tnmc_ctx* c, int64_t n);

// Pinned host memory from a process-wide cache (never handed back with cudaFreeHost while
// the process runs, so that releasing it cannot synchronise the device).
void* pinned_get(size_t bytes);
void pinned_put(void* p, size_t bytes);
cudaStream_t ctx_stream(const tnmc_ctx* c);

// Move a context to another stream.  The caller orders the switch: all work queued on the
// old stream must have completed (or be ordered before the new stream's work).
void ctx_set_stream(tnmc_ctx* c, cudaStream_t st);

// Free a context whose work has all completed, queueing the device frees on `st` and
// waiting for nothing (tnmc_destroy first synchronises the context's stream).
void ctx_release(tnmc_ctx* c, cudaStream_t st);

}  // namespace tnmc
