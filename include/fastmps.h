/*
 * fastmps.h -- C ABI of the GB300 (sm_103a) MPS perfect-sampling library.
 *
 * What it computes (Sec. 2.2 "Parallel MPS Sampling", Fig. 1 workflow;
 * Algorithm 2 "Measurement"; Sec. 3.3.1 per-sample scaling):
 * N independent configurations s[n] = (s_0 .. s_{M-1}) are drawn from the Born
 * distribution |A_0[s_0] A_1[s_1] ... A_{M-1}[s_{M-1}]|^2 of a right-canonical
 * complex MPS with M sites, physical dimension d and bond dimensions
 * b_0 = 1, b_1 .. b_{M-1}, b_M = 1.  Site k holds A_k[chi_l = b_k][d][chi_r =
 * b_{k+1}].  For each sample n the left vector v (v_0 = [1]) is contracted with
 * the site tensor, y_s = v A_k[:, s, :]; the unnormalised probabilities
 * w_s = ||y_s||^2 are summed in s order into C_s with Z = C_{d-1}; the outcome
 * is s* = #{s < d-1 : C_s < u Z} for the Philox4x32-10 uniform u = U(seed, n,
 * k, job) in (0,1); log p(s[n]) accumulates log w_{s*} - log Z; and
 * v <- y_{s*} / sqrt(w_{s*}).
 *
 * The uniform: key = (seed & 0xffffffff, seed >> 32), counter = (n & 0xffffffff,
 * n >> 32, k, job); with Philox outputs x0, x1,
 * u = (((uint64)x0 << 21 | x1 >> 11) + 0.5) * 2^-53.  Row n's result depends
 * only on (site tensors, seed, n, job, precision), not on N, n0 or tiling
 * choices other than through floating-point rounding.
 *
 * Conventions for every call
 *  - Return 0 (FASTMPS_OK) on success or a negative FASTMPS_ERR_* code; the
 *    message of the last failure is kept per handle (fastmps_last_error).
 *  - No C++ exception crosses the ABI.  Calls on one handle are not
 *    thread-safe; distinct handles are independent.
 *  - Input arrays are owned by the caller and only read during the call.
 *    Output arrays may be host or device memory (detected with
 *    cudaPointerGetAttributes) and are owned by the caller.
 *  - fastmps_sample* is synchronous: outputs are complete on return.
 */
#ifndef FASTMPS_H
#define FASTMPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes */
#define FASTMPS_OK 0
#define FASTMPS_ERR_INVALID_ARG (-1)   /* null pointer, negative size, out-of-range enum */
#define FASTMPS_ERR_SHAPE (-2)         /* bond_dims disagree with loaded sites, d > 255, ... */
#define FASTMPS_ERR_NOT_LOADED (-3)    /* a site (or pool entry) was never loaded */
#define FASTMPS_ERR_OOM (-4)           /* device or pinned-host allocation failed */
#define FASTMPS_ERR_CUDA (-5)          /* a CUDA runtime/driver call failed */
#define FASTMPS_ERR_TIMEOUT (-6)       /* a bounded device-side wait gave up */
#define FASTMPS_ERR_UNSUPPORTED (-7)   /* not available on this device/build */
#define FASTMPS_ERR_NUMERIC (-8)       /* Z = sum_s w_s was not a positive finite number */

/*
 * Arithmetic of the per-site contraction (Sec. 3.3, adaptive mixed precision).
 * BF16 modes keep the site tensor B and the left operand V as BF16 planes of
 * successive rounding residuals (B = B0 [+ B1], V = V0 + V1 [+ V2]) and
 * accumulate a list of plane products in FP32 on the tensor cores.
 */
#define FASTMPS_FP32 0    /* complex64 storage, FP32 SIMT FMA (no tensor cores) */
#define FASTMPS_BF16X2 1  /* V0 B0 + V1 B0: B in BF16, v to ~16 bits; 2 products */
#define FASTMPS_BF16X3 2  /* V0 B0 + V1 B0 + V0 B1: B to ~16 bits, v to ~16 bits; 3 products */
#define FASTMPS_BF16X3L 3 /* V0 B0 + V1 B0 + V2 B0: B in BF16, v to ~24 bits; 3 products */
#define FASTMPS_BF16X4 4  /* V0 B0 + V1 B0 + V2 B0 + V0 B1: B ~16 bits, v ~24 bits; 4 products */
/* Experiment: B = e4m3(A * 2^a) with a per-site power of two putting max |Re|,|Im| in [224, 448],
 * each left row e4m3(v * 2^r) with a per-row power of two likewise; one kind::f8f6f4 product.
 * Both scales cancel in w / Z.  Resident residency only. */
#define FASTMPS_FP8X1 5
/* Experiment: as FP8X1, with the left row split into two E4M3 residual planes at the same per-row
 * scale (V = V0 + V1, V1 = e4m3(v 2^r - V0)); two kind::f8f6f4 products V0 B + V1 B. */
#define FASTMPS_FP8X2 6
/* V0 B0 + V1 B0 with FP16 (binary16) operands: B = fp16(A * 2^a) with a per-site power of two putting
 * max |Re|,|Im| in [16384, 32768] (11 significant bits against BF16's 8; Sec. 3.3.2 keeps the tensors
 * in a 16-bit format), each left row as two FP16 residual planes of v * 2^r with a per-row power of
 * two putting its largest entry in [16384, 32768] (22 significant bits against BF16x2's 16).  Both
 * scales cancel in w / Z.  Same tensor-core rate as BF16x2.  Resident or host-streamed tensors;
 * fastmps_sample, fastmps_sample_ex and fastmps_sample_traced only (not batched, displaced or
 * allocation-free sampling). */
#define FASTMPS_FP16X2 7
/* V0 B0 + V1 B0 + V0 B1 with FP16 operands: as FP16X2, with the site tensor kept as two binary16
 * planes at the same per-site scale (B0 = fp16(A 2^a), B1 = fp16(A 2^a - B0), ~22 significant bits),
 * so that the 16-bit store no longer moves the conditionals of long chains (the storage error of one
 * binary16 plane reaches several 1e-3 at the end of a 1024-site chain); 3 products.  Same entry points
 * as FP16X2. */
#define FASTMPS_FP16X3 8

/* Where site tensors live between uses (Sec. 3.1: I/O overlapped by a double buffer). */
#define FASTMPS_RESIDENT_HBM 0    /* repacked once at load time, kept in device memory */
#define FASTMPS_HOST_STREAM 1     /* kept in pinned host memory (BF16), copied per site into
                                     one of two device slots on a copy stream, overlapped
                                     with the previous site's compute */

/* Element type of tensors passed to fastmps_load_site / fastmps_load_pool */
#define FASTMPS_C64 0   /* interleaved complex float  (re, im) */
#define FASTMPS_C128 1  /* interleaved complex double (re, im) */

typedef struct fastmps_options {
    int precision;          /* FASTMPS_FP32 | _BF16X2 | _BF16X3 | _BF16X3L | _BF16X4 | _FP8X1 | _FP8X2 | _FP16X2 |
                               _FP16X3 */
    int residency;          /* FASTMPS_RESIDENT_HBM | FASTMPS_HOST_STREAM (BF16 and FP16 modes only) */
    int64_t max_microbatch; /* rows per contraction launch; 0 = chosen from free memory */
    int autotune;           /* 1: time the candidate tile shapes once per new shape */
    void *stream;           /* cudaStream_t to run on; NULL = a stream owned by the handle */
    int fused_measure;      /* BF16 modes: 0 (default) = separate measurement kernel, overlapped
                               on a second stream when there are several micro-batches;
                               1 = measurement warps inside the contraction kernel;
                               2 = single pass (Algorithm 2 fused into the contraction's
                               epilogue): a thread-block cluster holds a sample's whole row in
                               tensor memory, combines the per-tile sums of squares through
                               distributed shared memory and writes only the selected,
                               renormalised block -- no FP32 scratch.  Sites whose row does not
                               fit one cluster (more than 32 column tiles, or column tiles not
                               a multiple of 64 wide) take mode 0. */
    int k_split;            /* BF16 modes, separate measurement: 0 or 1 = one thread block per output
                               tile; 2..8 = a thread-block cluster of that many blocks per tile, each
                               summing its share of the contraction index, partial tiles added
                               through distributed shared memory (the paper's single- vs
                               double-site split of Sec. 3.2, inside one GPU; an experiment). */
    int accum_chunk;        /* tensor-core modes, separate measurement: 0 = each output accumulated
                               over the whole contraction index in one tensor-memory accumulator;
                               c > 0 = n-tiles of 128 columns whose index is accumulated c k-blocks
                               (64 entries each) at a time into fresh accumulators, the chunk sums
                               added in FP32 registers with round-to-nearest (the tensor cores'
                               own accumulation then only spans short partial sums). */
} fastmps_options;

typedef struct fastmps_ctx *fastmps_handle;

/* Per-call statistics of the last fastmps_sample* call on a handle. */
typedef struct fastmps_stats {
    double ms_total;        /* wall time of the call (host clock) */
    double ms_contract;     /* device time in contraction kernels (CUDA events) */
    double ms_measure;      /* device time in the measurement kernels */
    int64_t launches;       /* kernels launched by the call */
    int64_t contract_launches;
    double flops_algorithmic; /* 8 * N * sum_k chi_l d chi_r */
    double flops_issued;    /* algorithmic x the number of split products (BF16 modes) */
    int64_t h2d_bytes;      /* host->device bytes copied during the call */
    int64_t d2h_bytes;      /* device->host bytes copied during the call */
    double ms_h2d;          /* device time of the site-tensor copies (host streaming; CUDA events) */
} fastmps_stats;

/* Fill *opt with the defaults: FP32, resident, automatic micro-batch, no autotune, own stream,
 * separate measurement kernel.  (Precision: Sec. 3.3; residency: Sec. 3.1; micro-batch: the
 * paper's N2 samples per contraction of Algorithm 2.) */
void fastmps_default_options(fastmps_options *opt);

/*
 * Create a handle on CUDA device `device`.  opt may be NULL (defaults).
 * (Library plumbing: one handle holds one MPS on one device, the paper's
 * per-process state of Sec. 3.1 reduced to a single GPU.)
 * Fails with FASTMPS_ERR_UNSUPPORTED if the device is not compute capability
 * 10.3 (the library is built for sm_103a only).  *out receives the handle
 * (NULL on failure).
 */
int fastmps_create(fastmps_handle *out, int device, const fastmps_options *opt);

/* Release every resource of the handle.  NULL is accepted; a handle must not be used afterwards.
 * (Plumbing, no counterpart in the paper.) */
void fastmps_destroy(fastmps_handle h);

/*
 * (Plumbing, no counterpart in the paper.)
 * Message of the last failure on h (empty string if none).  With h == NULL,
 * the message of the last failed fastmps_create in this process.
 * The pointer stays valid until the next call on the same handle.
 */
const char *fastmps_last_error(fastmps_handle h);

/*
 * Load site k (Sec. 2.2: the site tensors of the MPS, here right-canonical
 * A_k[chi_l][d][chi_r]; Sec. 3.3.2: kept in a compact low-precision format for
 * storage and transfer in the BF16 modes): A is host or device memory (detected with
 * cudaPointerGetAttributes), shape [chi_l][d][chi_r] row-major, interleaved
 * complex of type dtype.  The tensor is copied and repacked into
 * the handle's arithmetic format (complex64, or BF16 planes of the real
 * stacked operand); the caller keeps ownership of A.  Loading k again
 * replaces the site.  In FASTMPS_HOST_STREAM residency the BF16 copy stays in
 * pinned host memory.  Requirements: 0 <= k < 65536, chi_l, chi_r >= 1,
 * 2 <= d <= 255, d * chi_r >= chi_l (an isometry must fit).
 */
int fastmps_load_site(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *A, int dtype);

/*
 * Pool extension (Sec. 3.1: site tensors are loaded once and streamed to the
 * compute while the previous site runs) for chains that reuse tensors (e.g. a pool of 16 interior
 * isometries shared by thousands of sites): load pool entry j (same layout
 * and rules as fastmps_load_site), then map site k to it.  A mapped site uses
 * the pool entry until it is mapped again or loaded with fastmps_load_site.
 */
int fastmps_load_pool(fastmps_handle h, int j, int chi_l, int d, int chi_r, const void *A, int dtype);
int fastmps_map_site(fastmps_handle h, int k, int j);

/*
 * Draw N samples, rows n = 0 .. N-1 (Sec. 2.2 sampling workflow, Fig. 1: the
 * site-by-site contraction of every sample's left environment; Algorithm 2:
 * probabilities, cumulative sum, threshold draw and left-environment update;
 * Sec. 3.3.1: per-sample rescaling, here the exact renormalisation).
 *   bond_dims   host array of M+1 ints with bond_dims[0] = bond_dims[M] = 1;
 *               site k must be loaded with shape (bond_dims[k], d, bond_dims[k+1]).
 *   out_samples N*M bytes, row n = sample n (out_samples[n*M + k] = s_k), or NULL.
 *   out_logprob N doubles, log p(s[n]) = sum_k log(w_{s_k} / Z_k), or NULL.
 * N = 0 is valid and does nothing.
 */
int fastmps_sample(fastmps_handle h, int M, int d, const int *bond_dims, int64_t N, uint64_t seed,
                   uint8_t *out_samples, double *out_logprob);

/*
 * (Sec. 3.1 data parallelism: disjoint row ranges on different devices or calls
 * give the rows of one large run, since the uniform is keyed by the global n.)
 * As fastmps_sample for rows n = n0 .. n0+N-1 (output row i is sample n0+i)
 * and Philox counter word `job`.  trace_rows > 0 with trace_probs != NULL
 * records the normalised conditionals w_s / Z of the first trace_rows rows at
 * every site: trace_probs[(k * trace_rows + i) * d + s] (doubles, host or
 * device memory), for parity checks.
 */
int fastmps_sample_ex(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                      uint64_t seed, uint32_t job, uint8_t *out_samples, double *out_logprob,
                      int64_t trace_rows, double *trace_probs);

/*
 * As fastmps_sample_ex, with the conditionals traced for an arbitrary list of
 * call rows (for parity checks of rows anywhere in a large call, e.g. in
 * every micro-batch).  trace_list: n_trace distinct call rows in [0, N), host
 * memory; trace_probs[(k * n_trace + i) * d + s] = w_s / Z of call row
 * trace_list[i] at site k (host or device, M * n_trace * d doubles).  The
 * conditionals are those of Algorithm 2's probability line (Sec. 2.2); row
 * lists with a repeated or out-of-range row give FASTMPS_ERR_INVALID_ARG.
 */
int fastmps_sample_traced(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                          uint64_t seed, uint32_t job, uint8_t *out_samples, double *out_logprob,
                          const int64_t *trace_list, int64_t n_trace, double *trace_probs);

/*
 * fastmps_sample_noalloc -- sampling that allocates no memory.  (An addition
 * of this library for callers that cannot allocate; the paper has no
 * counterpart.)
 *
 * Same result as fastmps_sample_ex for rows n0 .. n0+N-1 (no trace), for
 * callers that may not call cudaMalloc while they sample: runtimes whose
 * device memory belongs to their own caching allocator or a fixed budget,
 * and services that allocate only at start-up so that their memory use
 * cannot grow or fragment later.  Every per-call buffer (left operands, contraction scratch,
 * outcomes, log-probabilities, error word) is carved from one static device
 * array of 64 MiB that each device loading this library holds until the
 * process exits; the call makes no cudaMalloc, cudaFree or other allocating
 * call.  The handle and its site tensors must already exist (creating and
 * loading do allocate), with FASTMPS_RESIDENT_HBM residency.
 *   out_samples, out_logprob: DEVICE memory owned by the caller (N*M bytes,
 *   N doubles), or NULL; host pointers are rejected (FASTMPS_ERR_INVALID_ARG).
 *   A chain/row count whose buffers exceed the 64 MiB array is rejected with
 *   FASTMPS_ERR_INVALID_ARG and a message giving the size it needed.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents (accumulators are cleared at the start of each call); calls
 * that overlap on the GPU race on it, so serialise them.  The call runs on
 * the handle's stream and returns when its outputs are complete.
 */
int fastmps_sample_noalloc(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                           uint64_t seed, uint32_t job, uint8_t *out_samples, double *out_logprob);

/*
 * Batched sampling of many independent MPS in one engine call (the paper's
 * many-sample data parallelism of Sec. 3.1 extended to many chains; chains may
 * differ in M, d, bond dimensions (Sec. 3.4.2: site-varying bond dimensions)
 * and sample count).
 *
 * Each job names a handle `chain` whose sites hold that MPS (loaded with
 * fastmps_load_site / fastmps_load_pool); every chain must live on the
 * runner's device and use the runner's precision (a BF16 mode) with resident
 * tensors.  Each job's rows are taken in chunks and every chunk through all
 * of the job's sites; one persistent tcgen05 kernel runs every (job, chunk,
 * site) step of the call, handing out 128-row tiles from a device work queue
 * and ordering the steps of each 128-row block of a job with bounded waits on
 * per-block step counters, so that different jobs (and different row blocks
 * of one job) advance independently.  The call's launches are captured into a
 * CUDA graph on the first call with a given job table and replayed by later
 * calls with the same table (same chains, shapes, rows, seeds and output
 * pointers).  A dependency wait that runs out gives FASTMPS_ERR_TIMEOUT and
 * leaves the runner usable.
 * Per job: rows n0 .. n0+N-1, Philox counter word `job`; outputs as in
 * fastmps_sample_ex (host or device, or NULL).  Statistics of the call are
 * available from the runner with fastmps_get_stats.
 */
typedef struct fastmps_job {
    fastmps_handle chain;
    int M;
    int d;
    const int *bond_dims; /* M+1 entries, host memory */
    int64_t n0;
    int64_t N;
    uint64_t seed;
    uint32_t job;
    uint8_t *out_samples; /* N*M bytes or NULL */
    double *out_logprob;  /* N doubles or NULL */
} fastmps_job;

int fastmps_sample_batch(fastmps_handle runner, int count, const fastmps_job *jobs);

/*
 * Vidal-form sites (Sec. 2.2: the workflow contracts the tensors Gamma_i into
 * the left environment; Algorithm 2 weights the squared amplitudes by the
 * coefficient vector Lambda).  Gamma: [chi_l][d][chi_r] interleaved complex of
 * type dtype; Lambda: chi_r real numbers of the same precision (double for
 * FASTMPS_C128, float for FASTMPS_C64) -- the Schmidt coefficients of the bond
 * right of site k ([1] for the last site).  Both host or device memory, owned
 * by the caller and only read during the call.  The site is stored as
 * A_k[a, s, b] = Gamma_k[a, s, b] * Lambda_k[b] (scaled on the device before the
 * repack), which is right-canonical for a Vidal canonical form, and is then
 * sampled exactly like a site loaded with fastmps_load_site: the outcome
 * probabilities are sum_b |(v Gamma_k[s])_b|^2 Lambda_k[b]^2 / Z and the carried
 * left vector is (v Gamma_k[s*]) Lambda_k / sqrt(w_{s*}).  Same requirements and
 * error codes as fastmps_load_site / fastmps_load_pool, plus
 * FASTMPS_ERR_INVALID_ARG for a NULL Lambda.
 */
int fastmps_load_site_vidal(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *Gamma,
                            const void *Lambda, int dtype);
int fastmps_load_pool_vidal(fastmps_handle h, int j, int chi_l, int d, int chi_r, const void *Gamma,
                            const void *Lambda, int dtype);

/*
 * Gaussian-boson-sampling random displacement (Sec. 3.4.1).
 *
 * fastmps_displacement: for N complex amplitudes mu[n] (interleaved complex64,
 * host or device) write the d x d matrices
 *     D(mu) = exp(-|mu|^2 / 2) exp(mu a^+) exp(-mu^* a)
 * (the paper's Zassenhaus approximation of the displacement operator
 * exp(mu a^+ - mu^* a) in the d-level truncation, a|j> = sqrt(j)|j-1>) as
 * interleaved complex64 with the batch index last: D[2*((s*d + t)*N + n)] (re)
 * and +1 (im) for row s, column t, sample n (host or device memory, d*d*N
 * complex entries).  Device arrays must be 8-byte aligned.  The product of the
 * two triangular factors is computed entry by entry from their closed forms in
 * FP32; it equals the matrix elements <s|D(mu)|t> of the untruncated operator.
 * Runs on the handle's stream and returns when D is complete.
 *
 * fastmps_sample_displaced: as fastmps_sample_ex, with the physical index of
 * every sample's contracted tensor mixed by its own displacement before the
 * measurement: y_s <- sum_t D(mu)[s, t] y_t with mu = mu[2*(k*ld_mu + i)] (re),
 * +1 (im) for call row i (sample n0+i) at site k (interleaved complex64, host or
 * device, ld_mu >= N).  The probabilities, draw, log-probability and next left
 * vector are then those of fastmps_sample_ex on the mixed blocks.  Needs
 * 2 <= d <= 16 and the FP32 or a BF16 precision (FASTMPS_ERR_SHAPE /
 * FASTMPS_ERR_UNSUPPORTED otherwise); the measurement runs as a separate kernel
 * (fused_measure is ignored).  Host amplitudes are copied to a device buffer of
 * M * N * 8 bytes owned by the handle at the start of the call; device
 * amplitudes (8-byte aligned) are read in place.  The outcome draw is decided
 * as in FP64 on the FP32 probability sums (an FP32 comparison, redone in FP64
 * when the threshold lies within 1e-5 Z of a cumulative sum).
 */
int fastmps_displacement(fastmps_handle h, int64_t N, int d, const float *mu, float *D);
int fastmps_sample_displaced(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                             uint64_t seed, uint32_t job, const float *mu, int64_t ld_mu, uint8_t *out_samples,
                             double *out_logprob, int64_t trace_rows, double *trace_probs);

/*
 * Dynamic bond dimensions (Sec. 3.4.2: entanglement grows from the edges to
 * the centre, so a fixed bond dimension is redundant at the edges; the filter
 * keeps fewer coefficients there while the truncation error stays under
 * control).  Host-only: no device work, no handle.
 *   bond_in   M+1 ints, the bond dimensions of the chain (bond_in[0] = bond_in[M] = 1).
 *   lambdas   M-1 host pointers; lambdas[k] holds the bond_in[k+1] Schmidt coefficients of the
 *             bond right of site k (descending order is not required).
 *   chi       the fixed bond dimension of the reference filter (keep at most chi per bond).
 *   eps       discarded-weight budget per bond; eps <= 0 selects the largest discarded weight
 *             that keeping min(chi, n) coefficients incurs on any bond of this chain.
 *   align     >= 1; kept counts are rounded up to a multiple of align (capped at min(chi, n)) --
 *             1 keeps the least counts; a multiple of the contraction tile (e.g. 64) avoids padding.
 *   bond_out  M+1 ints: bond_out[k+1] = the least c in [1, min(chi, n)] whose discarded weight
 *             T_c / T_0 (T_c = sum_{j >= c} lambda_j^2, summed in FP64 from the last index down)
 *             is <= the budget (min(chi, n) if none), rounded up to the alignment, then raised
 *             left to right to ceil(bond_out[k] / d) so that d * chi_r >= chi_l holds at every site.
 *   discarded_out (nullable) M+1 doubles: the discarded weight of each bond (0 at the ends).
 * Returns FASTMPS_OK, FASTMPS_ERR_INVALID_ARG (null pointer, bad size, all-zero spectrum) or
 * FASTMPS_ERR_SHAPE (ends not 1).  Keeping the leading coefficients assumes each spectrum is
 * sorted in descending order, as Schmidt coefficients are.
 */
int fastmps_bond_filter(int M, int d, const int *bond_in, const double *const *lambdas, int chi, double eps,
                        int align, int *bond_out, double *discarded_out);

/*
 * Load the leading block Gamma[:keep_l, :, :keep_r], Lambda[:keep_r] of a Vidal-form site whose
 * arrays have the full shape (chi_l, d, chi_r) and (chi_r) -- the truncation chosen by
 * fastmps_bond_filter -- without a copy by the caller.  Otherwise as fastmps_load_site_vidal;
 * needs 1 <= keep_l <= chi_l, 1 <= keep_r <= chi_r and d * keep_r >= keep_l.
 */
int fastmps_load_site_vidal_truncated(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *Gamma,
                                      const void *Lambda, int dtype, int keep_l, int keep_r);

/* Statistics of the last fastmps_sample* call (measurement plumbing; the paper has no counterpart). */
int fastmps_get_stats(fastmps_handle h, fastmps_stats *out);

/*
 * Self-test of the bounded device-side waits (no fault, no hang): launches one
 * thread block on `device` that waits on a shared-memory barrier nothing ever
 * completes, with the same bounded-wait routine the pipelined kernels use,
 * giving up after limit_ms.  *status receives FASTMPS_ERR_TIMEOUT when the
 * wait ran out (the expected outcome) and *waited_ms the device time waited.
 * Returns FASTMPS_OK if the self-test ran.  (Library test hook; the paper
 * has no counterpart.)
 */
int fastmps_selftest_bounded_wait(int device, double limit_ms, int *status, double *waited_ms);

/* Library version string (static storage; plumbing, no counterpart in the paper). */
const char *fastmps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FASTMPS_H */
