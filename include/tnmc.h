/*
 * tnmc.h -- C ABI of the GB300 (sm_103a) Tensor Network Monte Carlo library for the
 * two-dimensional +-J random-bond Ising model with open boundaries (arXiv 2409.06538).
 *
 * The library runs the three parts of the method on one GPU:
 *   (a) the boundary-MPS contraction of the L x L partition-function network, row by row
 *       from the bottom, with every row environment cached (Sec. II.B, Figs. 2-3);
 *   (b) whole-lattice proposals drawn row by row from the conditionals those environments
 *       give, with log q(s) (Sec. II.A Eqs. Bayes / approximate_bayes; Sec. II.B, Figs. 4-5);
 *   (c) the Metropolis accept/reject against the Boltzmann weight (Eq. accptanceratio,
 *       App. A) and the sampled observables (Sec. III.C).
 *
 * Conventions shared by every entry point
 *   - Spin s = +1 or -1; in tensors index 0 <-> +1 and 1 <-> -1 (Sec. II.B copy tensor).
 *   - Lattice L x L, site i = r*L + c (row r from the top, column c from the left).
 *   - Couplings of one realization: 2L(L-1) int8 values +-1; first Jh[r][c] (bond
 *     (r,c)-(r,c+1)) row-major over r<L, c<L-1, then Jv[r][c] (bond (r,c)-(r+1,c))
 *     row-major over r<L-1, c<L.  E(s) = -sum J_ij s_i s_j (Eq. E).
 *   - Random numbers: Philox4x32-10 keyed by the realization's 64-bit seed (low word
 *     first); the uniform is ((x0>>5)*2^26 + (x1>>6)) * 2^-53 from the first two output
 *     words.  Counters: bond b -> (b,0,0,0); spin at site i of proposal `step` of chain
 *     `chain` -> (i, step, chain, 1); accept test of that proposal -> (0, step, chain, 2).
 *   - Pointers named *_dev are device pointers on the context's CUDA device; *_host are
 *     host pointers; "host or device" pointers are classified by cudaPointerGetAttributes.
 *     The caller owns every buffer it passes; the library copies inputs at the call and
 *     never keeps a caller pointer.
 *   - Every call returns a tnmc_status and never aborts the process.  Work is queued on the
 *     context's stream (opts.stream, a cudaStream_t, NULL = legacy default stream); calls
 *     that return host data synchronise that stream.  Device-side failures (a vanishing or
 *     non-finite conditional weight, a wait that ran out) are recorded in a device status
 *     word and returned by the next synchronising call; tnmc_last_error() gives the text.
 *   - Order of use: create -> build_env -> (propose -> accept)* -> observables -> destroy.
 *     Out-of-order use returns TNMC_ERR_STATE.
 */
#ifndef TNMC_H
#define TNMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNMC_OK = 0,
  TNMC_ERR_ARG = 1,         /* invalid argument (sizes, NULL where not allowed, |J| != 1, ...) */
  TNMC_ERR_OOM = 2,         /* device allocation failed */
  TNMC_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  TNMC_ERR_NUMERIC = 4,     /* w(+)+w(-) <= 0 after clamping, or not finite, at some site */
  TNMC_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
  TNMC_ERR_STATE = 6,       /* call out of order (e.g. propose before build_env) */
  TNMC_ERR_UNSUPPORTED = 7  /* configuration not built into this library (e.g. chi > 64, or > 32 in FP64) */
} tnmc_status;

typedef enum {
  TNMC_FP64 = 0,        /* everything in FP64 (chi <= 32) */
  TNMC_FP32 = 1,        /* environments built and stored in FP32, sampling in FP32 (FMA) */
  TNMC_MIXED_BF16 = 2,  /* FP32 build, BF16 cached environments read into FP32 sampling (FMA);
                           outside the 1e-3 conditional tolerance (measured, see the tests) */
  TNMC_MIXED_TF32 = 3   /* FP32 build and cache; sampling products on the tensor cores as
                           3xTF32 (FP32 accuracy) for chi = 16 and 32, FP32 FMA otherwise.
                           Every path keeps log-norms, log q and the Metropolis test in FP64. */
} tnmc_precision;

/* Device allocator of the caller (optional).  alloc(bytes, stream, user) returns device memory
 * on the context's device, usable in stream order on `stream` (NULL on failure); free(ptr,
 * bytes, stream, user) gives it back once the work queued on `stream` no longer needs it.  With
 * both set, every device buffer of the context comes from them (PyTorch's caching allocator,
 * a pool the application reserved up front, ...); with both NULL the library allocates with
 * cudaMallocAsync (cudaMalloc where the device has no memory pools).  They are called only from
 * tnmc_create, tnmc_propose (when it grows the proposal buffers), tnmc_eval_conditionals
 * (without logq_dev) and tnmc_destroy, on the calling thread. */
typedef void* (*tnmc_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*tnmc_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Compression of the boundary MPS (the environment build). */
typedef enum {
  TNMC_COMPRESS_CANONICAL = 0,  /* Sec. II.B: per row, a left-to-right QR sweep (R factors of the left
                                   parts) and a right-to-left truncating SVD sweep (the SVD QR-
                                   preconditioned); the best truncation at a given chi */
  TNMC_COMPRESS_ZIPUP = 1       /* zip-up: per row one truncating SVD sweep and no QR sweep.  It
                                   relies on the previous row being canonical on the side the sweep
                                   reaches last, so the sweep direction alternates: the row built
                                   from the bond-1 last row sweeps left to right, the next right to
                                   left, and so on.  A left-to-right row is computed as the
                                   right-to-left sweep of the mirrored row (sites reversed, bonds
                                   swapped, each horizontal bond factor at the bond's right site).
                                   Cheaper per site and less accurate at the same chi (lower
                                   acceptance); not available through tnmc_build_env_noalloc */
} tnmc_compression;

typedef struct {
  int precision;      /* tnmc_precision */
  int n_chains;       /* Markov chains (replicas) per realization, >= 1; the overlap q of
                         Sec. III.C is measured between chains 0 and 1 when n_chains >= 2 */
  int n_therm;        /* steps with global step index < n_therm are not measured */
  void* stream;       /* cudaStream_t for all work of this context; NULL = default stream */
  tnmc_alloc_fn alloc;   /* caller's device allocator, or NULL (then free must be NULL too) */
  tnmc_free_fn free;
  void* alloc_user;      /* passed to alloc and free unchanged */
  int compression;       /* tnmc_compression; 0 (zero-initialised options) is the canonical one */
} tnmc_opts;

/* Per-realization thermal means over measured steps (Sec. III.C).  m = (1/N) sum_i s_i,
 * q = (1/N) sum_i s_i^(0) s_i^(1) between the current states of chains 0 and 1 at the same
 * step; m_edge = (1/2L) sum over the 1-based positions i = L/4 ... 3L/4 (inclusive) of
 * s_{i,1} + s_{1,i} + s_{L,i} + s_{i,L} (the edge magnetisation of Sec. III.C, normalisation
 * and segment as printed); E, m and m_edge statistics pool all chains. */
typedef struct {
  int64_t n_prop;       /* proposals processed by accept (all chains) */
  int64_t n_acc;        /* Metropolis tests that accepted */
  int64_t n_meas;       /* measured (chain, step) pairs */
  int64_t n_meas_q;     /* measured steps for the overlap */
  int64_t clamps;       /* negative truncated weights clamped to zero while sampling */
  double E, E2, m_abs, m2, m4;
  double q, q_abs, q2, q4;
  double m_edge, m_edge_abs, m_edge2;
  int64_t n_tests;      /* Metropolis tests: every proposal except each chain's first ever, which
                           is its initial state; the acceptance rate is n_acc / n_tests */
  int32_t status;       /* TNMC_OK, or TNMC_ERR_NUMERIC when a proposal of this realization met a
                           site with w+ + w- not positive and finite (its means are then not
                           valid samples of the clamp reading and tnmc_disorder_average skips it) */
  int32_t reserved;
} tnmc_obs;

/* Disorder averages [.] over realizations (Sec. III.C): mean and standard error (sample
 * standard deviation / sqrt(n_used)) of each thermal mean, in the order of tnmc_obs:
 * E, E2, m_abs, m2, m4, q, q_abs, q2, q4, m_edge, m_edge_abs, m_edge2. */
enum { TNMC_DIS_E = 0, TNMC_DIS_E2, TNMC_DIS_MABS, TNMC_DIS_M2, TNMC_DIS_M4, TNMC_DIS_Q, TNMC_DIS_QABS,
       TNMC_DIS_Q2, TNMC_DIS_Q4, TNMC_DIS_MEDGE, TNMC_DIS_MEDGEABS, TNMC_DIS_MEDGE2, TNMC_DIS_N };
typedef struct {
  int32_t n_used;       /* realizations averaged (status TNMC_OK) */
  int32_t n_dropped;    /* realizations left out because their status was not TNMC_OK */
  double mean[TNMC_DIS_N], se[TNMC_DIS_N];
  double U_m;           /* Binder ratio [<m^4>] / [<m^2>]^2 (Eq. eq:binderEA applied to m) */
  double Q_q;           /* overlap Binder ratio [<q^4>] / [<q^2>]^2 (Eq. eq:binderEA, denominator read
                           as the square of the disorder mean) */
  double q2_sq;         /* [<q^2>^2], the other reading of that denominator */
  double chi_q;         /* (L^2 / T) ([<q^2>] - [<q>]^2), Eq. eq:susEA as printed */
  double chi_edge;      /* L [<m_edge^2>] (Sec. III.C) */
  double acceptance;    /* sum n_acc / sum n_tests over the realizations used */
  int64_t n_prop, n_tests, n_acc, clamps;   /* sums over the realizations used */
} tnmc_disorder;

/* Inverse temperature on the Nishimori line (Sec. III.A): exp(-2 beta) = p / (1 - p), i.e.
 * beta = (1/2) ln((1-p)/p), written to *beta_out.  TNMC_ERR_ARG unless 0 < p < 1/2. */
tnmc_status tnmc_nishimori_beta(double p, double* beta_out);

/* Disorder averages of n_real per-realization thermal means (as tnmc_observables returns them)
 * for lattice side L at inverse temperature beta (T = 1/beta in chi_q).  Realizations whose
 * status is not TNMC_OK are skipped and counted in n_dropped.  Host code only: no device is
 * needed.  Errors: TNMC_ERR_ARG for NULL pointers, n_real < 1, L < 2 or beta not positive and
 * finite; TNMC_ERR_NUMERIC when no realization is usable (out then holds NaN means). */
tnmc_status tnmc_disorder_average(const tnmc_obs* obs_host, int n_real, int L, double beta,
                                  tnmc_disorder* out_host);

typedef struct tnmc_ctx tnmc_ctx;

/* Library version (major*10000 + minor*100 + patch). */
int tnmc_version(void);

/* Seeded synthetic disorder (Sec. III.A, P(J) = (1-p) delta(J-1) + p delta(J+1)):
 * J_b = -1 iff u_b < p with u_b the Philox uniform of counter (b,0,0,0) under seeds[k].
 * Writes n_real * 2L(L-1) int8 couplings to out_dev (device) in the layout above.
 * Errors: TNMC_ERR_ARG for L < 2, n_real < 1, p outside [0,1] or NULL pointers. */
tnmc_status tnmc_couplings_pmj(int L, int n_real, const uint64_t* seeds_host, double p,
                               int8_t* out_dev, void* stream);

/* Create a context for n_real independent disorder realizations of one lattice size L
 * and one cut-off bond dimension chi (the largest bond dimension the boundary MPS keeps,
 * D in Table tableparameter).
 *   couplings : host or device, n_real * 2L(L-1) int8 +-1 (copied);
 *   beta_host : n_real inverse temperatures (Eq. P); on the Nishimori line
 *               beta = 0.5 ln((1-p)/p) (Sec. III.A);
 *   seeds_host: n_real Philox keys for the spin and accept draws;
 *   chi       : 1 <= chi <= 64 (<= 32 on the FP64 path; TNMC_ERR_UNSUPPORTED above).
 * Allocates the environment cache (n_real * L * L * 2 chi^2 words) and all scratch on the
 * current CUDA device.  Errors: TNMC_ERR_ARG, TNMC_ERR_OOM, TNMC_ERR_UNSUPPORTED, TNMC_ERR_CUDA. */
tnmc_status tnmc_create(int L, int n_real, const int8_t* couplings, const double* beta_host,
                        const uint64_t* seeds_host, int chi, const tnmc_opts* opts,
                        tnmc_ctx** out);

/* Replace the disorder realizations of an existing context (same L, n_real, chi): queues
 * the copy of new couplings (host or device, validated when on the host), inverse
 * temperatures and seeds on the context's stream, resets the chains and marks the
 * environments stale, so that one context serves successive batches without re-allocating
 * its caches.  Asynchronous: beta_host and seeds_host may be reused on return (they go
 * through a pinned staging ring); a host couplings buffer in pinned memory must stay
 * unchanged until the stream has executed the copy.  Errors as tnmc_create. */
tnmc_status tnmc_set_couplings(tnmc_ctx* ctx, const int8_t* couplings, const double* beta_host,
                               const uint64_t* seeds_host);

/* New realizations from seeds alone (Sec. III.A disorder, as tnmc_couplings_pmj): queues the
 * seeds and inverse temperatures, generates the +-J couplings with probability p of an
 * antiferromagnetic bond on the device, resets the chains and marks the environments
 * stale -- all asynchronous on the context's stream (no host synchronisation), so batches
 * of several contexts on several streams overlap.  Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_set_realizations(tnmc_ctx* ctx, const uint64_t* seeds_host, const double* beta_host,
                                  double p);

/* (a) Boundary-MPS contraction (Sec. II.B): for r = L-2 .. 0 apply the row-transfer MPO
 * (the T tensors: copy tensor with the Boltzmann matrices W absorbed) to the cached MPS of
 * row r+1, cut the bond dimension back to chi by SVD (keeping min(chi, rows, cols) singular
 * values at every bond, swept right to left from left-canonical form), normalise, and cache
 * the row with its FP64 log-norm.  log_z_host (nullable, n_real doubles) receives log Z of the
 * truncated network (exact when nothing is truncated); passing it synchronises. */
tnmc_status tnmc_build_env(tnmc_ctx* ctx, double* log_z_host);

/* (b) Draw n proposals per chain (global step indices step0 .. step0+n-1) from the cached
 * environments, row by row top to bottom and left to right (Sec. II.B), with log q(s) in
 * FP64 and the exact integer energy.  Proposals stay on the device for tnmc_accept.
 * Optional device outputs (each nullable), index [real][chain][k]:
 *   logq_dev (double), energy_dev (int32), magnet_dev (int32 sum of spins). */
tnmc_status tnmc_propose(tnmc_ctx* ctx, int n, uint64_t step0, double* logq_dev,
                         int32_t* energy_dev, int32_t* magnet_dev);

/* External fields (the paper's fixed spins of Sec. IV act this way): fields (host or device,
 * n_real * L * L int8, [real][r][c]) are integers k in units of beta, so that a configuration's
 * weight gains exp(beta sum_i k_i s_i); they enter the row MPO of the environments (the row below
 * each row) and the fields of the sampling sweep.  The environments become stale (build again).
 * NULL removes the fields.  Errors: TNMC_ERR_ARG, TNMC_ERR_OOM, TNMC_ERR_CUDA. */
tnmc_status tnmc_set_fields(tnmc_ctx* ctx, const int8_t* fields);

/* Unpack the spins of the last tnmc_propose call to spins_dev (device int8 +-1,
 * [real][chain][k][L*L]). */
tnmc_status tnmc_get_spins(tnmc_ctx* ctx, int8_t* spins_dev);

/* Teacher-forced evaluation of q on given configurations (the conditionals of Eq. cond
 * from the cached environments, with the given spins in place of draws).
 *   spins_dev: device int8 +-1, [real][k][L*L], n configurations per realization;
 *   logq_dev : device double [real][k] (nullable);
 *   qplus_dev: device double [real][k][L*L], q(s_i=+1 | s_<i) at every site (nullable). */
tnmc_status tnmc_eval_conditionals(tnmc_ctx* ctx, int n, const int8_t* spins_dev,
                                   double* logq_dev, double* qplus_dev);

/* (c) Metropolis accept/reject over the proposals of the last tnmc_propose call, in step
 * order per chain (Eq. accptanceratio with g(s'|s) = q(s')):
 *   Delta = [-beta E(s') - log q(s')] - [-beta E(s) - log q(s)],
 *   accept iff Delta >= 0 or u < exp(Delta).
 * A chain's first proposal ever is its initial state.  The current state carries over to
 * the next call.  Observables of every step with global index >= opts.n_therm accumulate.
 *   accepted_dev  : device uint8 [real][chain][k] (nullable);
 *   n_accepted_host: total accepted in this call (nullable; passing it synchronises). */
tnmc_status tnmc_accept(tnmc_ctx* ctx, uint8_t* accepted_dev, int64_t* n_accepted_host);

/* Per-realization thermal means (host array of n_real tnmc_obs).  Synchronises.  Every
 * realization is filled in, with its own status, before the context's status is returned: on
 * TNMC_ERR_NUMERIC the realizations whose status field is TNMC_ERR_NUMERIC (the ones
 * tnmc_realization_status flags) are not valid and the others are; on other errors nothing is
 * meaningful. */
tnmc_status tnmc_observables(tnmc_ctx* ctx, tnmc_obs* out_host);

/* Reset chain states, observable accumulators and the context's and every realization's
 * device status word (the environments stay cached). */
tnmc_status tnmc_reset_chains(tnmc_ctx* ctx);

/* Release every device allocation of the context.  NULL is accepted. */
tnmc_status tnmc_destroy(tnmc_ctx* ctx);

/* Text of the last error on this context (or of the last failed create when ctx is NULL). */
const char* tnmc_last_error(const tnmc_ctx* ctx);

/* Introspection used by tests and the benchmark.
 *   tnmc_env_bytes: bytes of the environment cache;
 *   tnmc_copy_env : copy the cached environment of (real, row) to host: tiles_host gets
 *                   L * 2 * chi * chi doubles ([c][y][alpha][beta], zero padded),
 *                   dims_host gets the L+1 bond dimensions, lam_host the row log-norm. */
size_t tnmc_env_bytes(const tnmc_ctx* ctx);
tnmc_status tnmc_copy_env(tnmc_ctx* ctx, int real, int row, double* tiles_host,
                          int32_t* dims_host, double* lam_host);

/* Statistics of the last tnmc_build_env, summed over realizations: out_host[0] = most
 * Jacobi sweeps any truncation needed, [1] = truncations that hit the sweep limit,
 * [2] = total sweeps, [3] = truncating SVDs performed.  Synchronises; reports only CUDA
 * errors (a sampling failure recorded in the status word is not the build's). */
tnmc_status tnmc_build_stats(tnmc_ctx* ctx, int64_t* out_host);

/* Environment build that allocates nothing.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc -- an application that reserves all
 * device memory up front and forbids allocation afterwards, or a latency-critical path where
 * cudaMalloc's device-wide synchronisation is not allowed.
 * It runs the same boundary-MPS build as tnmc_build_env for n_real realizations, reading and
 * writing only the caller's buffers plus one file-scope device array of 32 MiB that every GPU
 * which loads the library holds until the process exits (the R factors, working rows,
 * bond-dimension array, statistics and status word live there).
 *   couplings_dev: device, n_real * 2L(L-1) int8 +-1 in the layout above (not validated);
 *   beta_dev     : device, n_real doubles;
 *   precision    : tnmc_precision (the build runs in FP64 for TNMC_FP64, FP32 otherwise);
 *   env_dev      : device output, n_real * L * L tiles of 2*C*C elements ([real][row][site]
 *                  [y][alpha][beta], zero padded), C the smallest of 4, 8, 16, 32 that is
 *                  >= chi; elements are double (FP64), bfloat16 (MIXED_BF16) or float;
 *   kdim_dev     : device output, n_real * L * (L+1) int32 bond dimensions;
 *   lam_dev      : device output, n_real * L row log-norms; logz_dev: n_real log Z;
 *   stream       : cudaStream_t (NULL = default stream); the call only queues work.
 * The first call on a device looks up the device address of the array (once per device,
 * with that device current); make that first call before any stream capture.  Every call
 * shares the one array and leaves the last call's contents in it (the status word is cleared
 * at the start of each call): calls whose work overlaps on the GPU race and corrupt each
 * other, so serialise them (one stream, or events).
 * Errors: TNMC_ERR_ARG for bad sizes or NULL buffers, and when the scratch this build needs,
 * n_real * ((2*L*2*C*C + L*4*C*C) * w + 4*(L+1) + 32) + 4 bytes, each of its five parts
 * rounded up to 256 bytes (w = 8 for FP64, 4 otherwise; 32 bytes of statistics per realization
 * and one status word), exceeds the 32 MiB array; TNMC_ERR_UNSUPPORTED for chi > 32;
 * TNMC_ERR_CUDA for a failed launch.  The build has no device-side failure to report, and the
 * call does not synchronise. */
tnmc_status tnmc_build_env_noalloc(int L, int n_real, int chi, int precision,
                                   const int8_t* couplings_dev, const double* beta_dev,
                                   void* env_dev, int32_t* kdim_dev, double* lam_dev,
                                   double* logz_dev, void* stream);

/* Per-realization status: out_host[k] (n_real int32) is TNMC_ERR_NUMERIC when a proposal of
 * realization k met a site whose conditional weights w+ + w- were not positive and finite
 * after clamping (the context-wide status then reports TNMC_ERR_NUMERIC too), else TNMC_OK.
 * Cleared by tnmc_reset_chains (and so by tnmc_set_couplings / tnmc_set_realizations).
 * Lets a caller drop the affected realizations instead of the whole batch.  Synchronises. */
tnmc_status tnmc_realization_status(tnmc_ctx* ctx, int32_t* out_host);

/* The same per-realization failure flags without synchronising: queues on the context's stream
 * a copy of the n_real status words into out_dev (device, n_real uint32): 0 = no failure, bit 0
 * set = a numeric failure as above (bit 1: a bounded wait ran out).  Lets a caller that reuses a
 * context for successive batches keep each batch's flags.  Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_realization_status_async(tnmc_ctx* ctx, uint32_t* out_dev);

/* Kernel launch accounting: number of kernels this context launched since creation. */
int64_t tnmc_launch_count(const tnmc_ctx* ctx);

/* Failure-detection self-test (the paper has no counterpart).  Runs, on the current device and
 * the default stream, the bounded mbarrier wait that guards the tensor-core sampler's MMA
 * completions, in a one-CTA probe kernel: with arrive = 0 nothing arrives on the barrier, so
 * the wait gives up after 4096 polls, the kernel records the timeout in a status word and
 * returns normally, and this call returns TNMC_ERR_TIMEOUT; with arrive != 0 one thread
 * arrives first and the call returns TNMC_OK.  *elapsed_us (nullable) gets the probe's device
 * time.  The CUDA context stays usable afterwards.  Synchronises. */
tnmc_status tnmc_selftest_bounded_wait(int arrive, int64_t* elapsed_us);

/* Concurrency of the environment build on the current device: *ctas_per_sm gets how many
 * realizations (one CTA each) one SM holds at once for this L, chi and precision (shared
 * memory and registers decide), *num_sms (nullable) the SM count.  A batch of R
 * realizations fills R of ctas_per_sm * num_sms slots; callers size the number of batches
 * they keep in flight from it.  TNMC_ERR_ARG / TNMC_ERR_UNSUPPORTED for bad arguments,
 * TNMC_ERR_CUDA without a device. */
tnmc_status tnmc_env_build_occupancy(int L, int chi, int precision, int32_t* ctas_per_sm,
                                     int32_t* num_sms);

/* Device memory accounting.  tnmc_device_bytes: bytes the context holds now (its buffers
 * grow once to the largest n passed to tnmc_propose).  tnmc_estimate_device_bytes: bytes a
 * context of these arguments would hold after proposals of up to n_max per chain, without
 * allocating anything (0 for invalid arguments); it uses the current device's SM count, or
 * 152 when no device is present. */
size_t tnmc_device_bytes(const tnmc_ctx* ctx);
size_t tnmc_estimate_device_bytes(int L, int n_real, int chi, const tnmc_opts* opts, int n_max);

/* ------------------------------------------------------------------------------------------
 * Periodic boundaries (Sec. IV): each step of each chain pins a row i0 and a column j0 of the
 * L x L torus, keeps their spins fixed, and samples the remaining (L-1) x (L-1) region as an
 * open lattice whose fixed neighbours act as external fields; the proposal replaces the region
 * with the Metropolis probability of the region's conditional distribution given the lines,
 *   Delta = [-beta E_reg(x') + beta k.x' - log q(x')] - [-beta E_reg(x) + beta k.x - log q(x)],
 * so every step leaves the torus Boltzmann distribution invariant.  The environments depend on
 * the fixed spins and are rebuilt for every step of every chain (one proposal per build).
 * Torus couplings of one realization: 2 L^2 int8 +-1, first Jh[r][c] coupling (r, c)-(r, c+1 mod L)
 * row-major, then Jv[r][c] coupling (r, c)-(r+1 mod L, c) row-major.  Lines of step t of chain k:
 * i0 = floor(u L), j0 = floor(u' L) with u, u' the uniforms of counters (0, t, k, 3) and
 * (1, t, k, 3); region site (r, c) is torus site (i0+1+r, j0+1+c) mod L, its spin draw uses the
 * region's site index r (L-1) + c with counter (site, t, k, 1); the accept uniform is the counter
 * (0, t, k, 2).  Chains start from all spins up.
 * ------------------------------------------------------------------------------------------ */
typedef struct tnmc_periodic tnmc_periodic;

/* Seeded torus disorder: J_b = -1 iff u_b < p, u_b the uniform of counter (b, 0, 0, 0), for the
 * 2 L^2 bonds of each of n_real realizations, written to out_dev (device).  L >= 3. */
tnmc_status tnmc_torus_couplings_pmj(int L, int n_real, const uint64_t* seeds_host, double p,
                                     int8_t* out_dev, void* stream);

/* Context of n_real torus realizations (couplings host or device, n_real * 2 L^2), inverse
 * temperatures, seeds and the bond dimension chi of the regions' environments; opts as for
 * tnmc_create (n_chains chains per realization, the overlap between chains 0 and 1).  3 <= L.
 * Errors as tnmc_create. */
tnmc_status tnmc_periodic_create(int L, int n_real, const int8_t* couplings, const double* beta_host,
                                 const uint64_t* seeds_host, int chi, const tnmc_opts* opts,
                                 tnmc_periodic** out);

/* n_steps steps of every chain (global step indices step0 ...); observables of the torus states
 * (E with the periodic bonds, m, the overlap q) accumulate after every step with index >= n_therm.
 * Asynchronous on the context's stream.  A region that meets a doubly clamped site flags its
 * realization (tnmc_obs.status). */
tnmc_status tnmc_periodic_step(tnmc_periodic* ctx, int n_steps, uint64_t step0);

/* Per-realization thermal means of the torus (n_real tnmc_obs; m_edge fields are zero, the torus
 * has no edge; n_tests = n_prop = steps x chains).  Synchronises. */
tnmc_status tnmc_periodic_observables(tnmc_periodic* ctx, tnmc_obs* out_host);

/* Current torus states to spins_dev (device int8 +-1, [real][chain][L*L]). */
tnmc_status tnmc_periodic_get_spins(tnmc_periodic* ctx, int8_t* spins_dev);

int64_t tnmc_periodic_launch_count(const tnmc_periodic* ctx);
const char* tnmc_periodic_last_error(const tnmc_periodic* ctx);
tnmc_status tnmc_periodic_destroy(tnmc_periodic* ctx);

/* ------------------------------------------------------------------------------------------
 * Request server: continuous batching of independent realizations on one GPU.
 *
 * The paper runs its disorder realizations as fixed sets (Sec. III); each realization is an
 * independent problem: couplings (Sec. III.A), environments (Sec. II.B), proposals with
 * log q (Sec. II.B), Metropolis and observables (Sec. III.C).  The server takes such
 * problems one request at a time from any thread, groups requests of equal (L, chi) into
 * batches of up to max_batch, runs up to max_inflight batches at once (one pooled context and
 * CUDA stream each) and returns per-request results as they finish.  A native scheduler
 * thread makes every CUDA call.  Pooled contexts are kept for reuse and evicted, least
 * recently used first, when a new (L, chi) needs room within mem_budget; a batch's capacity
 * is halved until one context fits the budget.
 *
 * A request's result does not depend on the batch it ran in: draws are keyed by its seed
 * and counted by (site, step, chain), sampling runs in fixed steps of `chunk` proposals per
 * chain, and the Metropolis kernel stops each realization at its own n_samples.  The same
 * request, server options and library give the same bits alone or in any mix.
 * ------------------------------------------------------------------------------------------ */
typedef struct tnmc_server tnmc_server;

typedef struct {
  int precision;     /* tnmc_precision of every request */
  int n_chains;      /* independent chains per realization, 1..8 */
  int n_therm;       /* leading proposals per chain left out of the observables */
  int chunk;         /* proposals per chain per sampling launch (>= 1) */
  int max_batch;     /* most realizations in one batch (>= 1) */
  int max_inflight;  /* most batches on the device at once (>= 1) */
  int linger_us;     /* a batch short of max_batch waits up to this long for more requests */
  int device;        /* CUDA device ordinal */
  size_t mem_budget; /* device bytes all pooled contexts may hold; 0 = 90% of free memory */
} tnmc_server_opts;

typedef struct {
  uint64_t seed;     /* realization seed: couplings and every draw (as in tnmc_couplings_pmj) */
  int L;             /* lattice side, 2..4096 */
  int chi;           /* MPS bond dimension, 1..64 (1..32 when the server runs FP64) */
  double p;          /* probability of an antiferromagnetic bond, [0, 1] */
  double beta;       /* inverse temperature, finite and > 0 */
  int n_samples;     /* proposals per chain, >= 1 */
} tnmc_request;

typedef struct {
  int64_t id;
  int32_t status;          /* tnmc_status of this request */
  int32_t batch_size;      /* realizations in the batch it ran in (0: never launched) */
  double log_z;            /* log Z~ of its environment build */
  tnmc_obs obs;            /* thermal means, as tnmc_observables */
  int64_t build_stats[4];  /* as tnmc_build_stats, for this realization */
  double t_submit, t_start, t_done;  /* seconds on the server clock (tnmc_server_now) */
} tnmc_result;

/* Start a server (and its scheduler thread) on opts->device.  TNMC_ERR_ARG for invalid
 * options, TNMC_ERR_CUDA if the device cannot be queried.  Contexts are made lazily. */
tnmc_status tnmc_server_create(const tnmc_server_opts* opts, tnmc_server** out);

/* Queue one request; *id_out gets its id (> 0).  Thread-safe, never blocks on the GPU.
 * TNMC_ERR_ARG for a request outside the ranges above, TNMC_ERR_STATE while stopping. */
tnmc_status tnmc_server_submit(tnmc_server* srv, const tnmc_request* req, int64_t* id_out);

/* Move up to max_results finished results (in completion order) into out_host; returns
 * how many.  Thread-safe, non-blocking. */
int tnmc_server_poll(tnmc_server* srv, tnmc_result* out_host, int max_results);

/* Block until request `id` finishes (timeout_s < 0: no limit), then move its result into
 * out_host.  TNMC_ERR_TIMEOUT if it did not finish in time or was already collected. */
tnmc_status tnmc_server_wait(tnmc_server* srv, int64_t id, double timeout_s, tnmc_result* out_host);

/* Block until every submitted request has finished (results stay to be collected). */
tnmc_status tnmc_server_drain(tnmc_server* srv, double timeout_s);

/* out_host[8]: submitted, completed, failed, batches launched, contexts created, contexts
 * evicted, peak device bytes held by pooled contexts, kernels launched. */
tnmc_status tnmc_server_stats(tnmc_server* srv, int64_t* out_host);

/* Text of the last error; a copy owned by the calling thread, valid until its next call. */
const char* tnmc_server_last_error(tnmc_server* srv);

/* Seconds since tnmc_server_create on the server's steady clock. */
double tnmc_server_now(tnmc_server* srv);

/* Finish every queued request, stop the scheduler and free all pooled contexts. */
tnmc_status tnmc_server_destroy(tnmc_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* TNMC_H */
