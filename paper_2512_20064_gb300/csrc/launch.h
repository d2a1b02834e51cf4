// Host-side launchers of the library's kernels (internal; not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fastmps {

// Column layout of the contraction output of one site.  Output column
// c = s * Cs + p * chi_r + b holds the real (p = 0) or imaginary (p = 1) part
// of y_s[b]; columns chi_r*2 .. Cs-1 of each block are zero padding, so a tile
// of width bn never straddles two outcomes s.  K = 2*chi_l rows of the stacked
// real operand, padded to K_pad (a multiple of 64).
struct SiteLayout {
    int chi_l = 0, d = 0, chi_r = 0;
    int bn = 0;        // n-tile width of the contraction kernel
    int Cs = 0;        // columns per outcome block (multiple of bn)
    int ncols = 0;     // d * Cs
    int K_pad = 0;     // roundup(2 chi_l, bk)
    int tiles_per_s = 0;
    int bk = 64;       // operand elements per k-block: one 128-byte swizzle row (64 BF16 or 128 FP8)
};

// ---- repack of a complex site tensor (device staging copy) -----------------
// src: interleaved complex [chi_l][d][chi_r], float (is_f64 = 0) or double.
// Tensor-core operand: B[c][kappa] (K-major, ld = K_pad), BF16 hi (and lo).
void launch_repack_bf16(const void *src, int is_f64, const SiteLayout &L, __nv_bfloat16 *B_hi,
                        __nv_bfloat16 *B_lo, cudaStream_t st);
// Same from a compact BF16 complex copy [chi_l][d][chi_r] of (re, im) pairs
// (planes = 1: hi only; planes = 2: hi block followed by lo block).
void launch_expand_bf16(const __nv_bfloat16 *compact, int planes, const SiteLayout &L, __nv_bfloat16 *B_hi,
                        __nv_bfloat16 *B_lo, cudaStream_t st);
// FP8 E4M3 operand B[c][kappa] (K-major, ld = K_pad bytes) of value * scale (scale a power of two).
void launch_repack_e4m3(const void *src, int is_f64, const SiteLayout &L, float scale, uint8_t *B8,
                        cudaStream_t st);
// Largest |Re| or |Im| of an interleaved complex tensor (as float), into *out_dev (zeroed first).
void launch_absmax(const void *src, int is_f64, int64_t n_complex, float *out_dev, cudaStream_t st);
// FP16 operand B[c][kappa] (K-major, ld = K_pad) of value * scale (scale a power of two), binary16 bits;
// B16_lo (optional) receives the rounding residual fp16(value * scale - B16).
void launch_repack_f16(const void *src, int is_f64, const SiteLayout &L, float scale, uint16_t *B16,
                       uint16_t *B16_lo, cudaStream_t st);
// FP32 SIMT operand: Bt[kappa][c] (N-major, ld = ncols), float.
void launch_repack_f32(const void *src, int is_f64, const SiteLayout &L, float *Bt, cudaStream_t st);

// ---- left operand ----------------------------------------------------------
// Set rows [0, rows) of V to the boundary vector v_0 = [1] (row = [1, 0, ... 0], ld elements).
void launch_init_left_bf16(__nv_bfloat16 *const *Vp, int nplanes, int64_t rows, int ld, cudaStream_t st);
void launch_init_left_f32(float *V, int64_t rows, int ld, cudaStream_t st);
void launch_init_left_e4m3(uint8_t *V8, int64_t rows, int ld, cudaStream_t st);
// FP16 planes of v_0 = [1]: plane 0 holds 1.0 in column 0, plane 1 zeros.
void launch_init_left_f16(uint16_t *V0, uint16_t *V1, int64_t rows, int ld, cudaStream_t st);

// ---- contraction kernels ---------------------------------------------------
struct ContractOut {
    float *Y;          // [rows_pad][ldY] FP32 scratch
    int64_t ldY;
    float *P;          // [rows_pad][ldP] per-tile sums of squares
    int ldP;
    int rows_valid;    // rows of this micro-batch
};

// FP32 SIMT: Y = V[row0 : row0+rows_pad] (ld = ldV, K = L.K_pad) x Bt.
void launch_contract_f32(const float *V, int64_t ldV, int64_t row0, int64_t rows_pad, const float *Bt,
                         const SiteLayout &L, const ContractOut &o, cudaStream_t st);

// tcgen05 BF16 split-precision contraction.  tmA[p] / tmB[p] are tensor maps
// over the operand planes (a_planes in {1,2,3}, b_planes in {1,2}); the
// products accumulated are (prod_a[q], prod_b[q]) for q < nprod.
constexpr int kMaxProducts = 4;
struct TcArgs {
    bool fp8 = false;  // E4M3 operands (one plane each), kind::f8f6f4
    bool f16 = false;  // FP16 (binary16) operands instead of BF16, kind::f16
    bool has_tmY = false;  // tmY maps the FP32 scratch (ncols x rows, 32 x 128 boxes): TMA-store epilogue
    CUtensorMap tmY;
    CUtensorMap tmA[3];
    CUtensorMap tmB[2];
    int a_planes, b_planes;
    int nprod;
    int prod_a[kMaxProducts], prod_b[kMaxProducts];
    int64_t row0;     // first row of the micro-batch in the V planes
    int rows_pad;     // multiple of 128
};
int tc_max_smem_ok(int device);
struct MeasureArgs;
// fused != nullptr: the measurement of each m-tile runs inside the contraction
// kernel (one thread block per m-tile at a time; grid = min(m-tiles, SMs)).
cudaError_t launch_contract_tc(const TcArgs &a, const SiteLayout &L, const ContractOut &o, int num_sms,
                               int *d_err, cudaStream_t st, const MeasureArgs *fused = nullptr);
// Single-pass cluster variant (no scratch): true if the site's row fits one cluster's tensor memory
// (C CTAs of T n-tiles each, C <= 16, the n-tile width a multiple of 64).
bool cluster_plan(const SiteLayout &L, int *C, int *T);
// On-chip split-K (a study of the paper's single- vs double-site splitting inside one GPU): a cluster of
// ksplit CTAs per output tile, each accumulating 1/ksplit of the k-blocks; partial tiles are added
// through distributed shared memory into rank 0, which writes Y and P as launch_contract_tc does
// (a.has_tmY required).  The sum is taken in rank order, so Y differs from the unsplit kernel by
// rounding only.
cudaError_t launch_contract_tc_splitk(const TcArgs &a, const SiteLayout &L, const ContractOut &o, int ksplit,
                                      int *d_err, cudaStream_t st, int *clusters_out = nullptr);
// Promoted accumulation: as launch_contract_tc (two-pass outputs Y and P, a.has_tmY required) with
// n-tiles of 256 columns (L.bn == 256) whose contraction index is accumulated by the tensor cores
// kchunk k-blocks at a time into fresh accumulators, the chunk sums being added in FP32 registers.
cudaError_t launch_contract_tc_promoted(const TcArgs &a, const SiteLayout &L, const ContractOut &o, int kchunk,
                                        int num_sms, int *d_err, cudaStream_t st);
// Clusters of the site's plan that can be resident at once on the current device (0: not runnable).
int cluster_capacity(int a_planes, int b_planes, const SiteLayout &L);
// Contraction + measurement of rows_valid rows in one launch; m describes the draw and the next left
// rows (BF16 planes; Y, P unused).  *clusters_out (nullable): clusters launched.
cudaError_t launch_contract_tc_cluster(const TcArgs &a, const SiteLayout &L, int rows_valid, int *d_err,
                                       cudaStream_t st, const MeasureArgs &m, int *clusters_out = nullptr);

// ---- measurement (Algorithm 2) --------------------------------------------
struct MeasureArgs {
    const float *Y;
    int64_t ldY;
    const float *P;
    int ldP;
    int d, chi_r, Cs, tiles_per_s;
    int rows;                 // rows of this micro-batch
    uint64_t seed;
    uint64_t n_base;          // sample index of row 0 of the micro-batch
    uint32_t k, job;
    // next left operand, rows offset row0 (all N rows live in the V buffer)
    int64_t row0;
    int ld_next;              // ld of the next V buffer (elements)
    int K_next;               // entries of the next row that must be written (2 chi_r .. K_next-1 zeroed)
    float *V32;               // FP32 path (or nullptr)
    __nv_bfloat16 *Vp[3];     // BF16 paths: planes of successive residuals (FP16 path: binary16 bits)
    int nplanes;              // 2 or 3
    int f16 = 0;              // FP16 path: two binary16 planes of each row scaled by a per-row power of two
    uint8_t *V8 = nullptr;    // FP8 path: E4M3 row scaled by a per-row power of two
    uint8_t *V8lo = nullptr;  // FP8X2: E4M3 residual plane at the same per-row scale (or nullptr)
    const float2 *mu = nullptr;  // displaced measurement: amplitude of each row of this micro-batch
    const float *disp_tab = nullptr;   // displaced measurement: constants of the displacement entries
    float2 *disp_D = nullptr;          // displaced measurement: per-row matrices [row][d*d] (prep kernel output)
    double *disp_u = nullptr;          // displaced measurement: per-row uniforms (prep kernel output)
    uint8_t *outcomes;        // [rows] outcome bytes of this site (site-major buffer slice)
    double *logp;             // [rows] accumulated log-probability
    double *trace;            // nullable: [trace_rows][d] normalised conditionals of this site
    int trace_rows;           // traced rows: call rows 0 .. trace_rows-1, or the rows trace_slot lists
    const int *trace_slot = nullptr;  // nullable: per call row, its trace slot (-1: not traced)
    int *err;
};
void launch_measure(const MeasureArgs &a, cudaStream_t st);

// ---- Vidal form and GBS displacement (gbs.cu) ------------------------------
constexpr int kMaxDisplacedD = 16;
// A[a][s][b] *= lam[b] on an interleaved complex tensor (float or double, lam of the same type).
void launch_scale_columns(void *A, int is_f64, int64_t n_complex, int chi_r, const void *lam, cudaStream_t st);
// Constants of the displacement entries for dimension d: (s, t) at [(s*d + t) * (2d + 1)]:
// c_st = sqrt(max! / min!) / |s-t|!, then q_m = m / ((s-m+1)(t-m+1)) for m = 1 .. d (0 above
// min(s, t)) as float-float pairs (hi, lo).
void build_displacement_table(int d, float *tab /* d * d * (2d + 1) */);
// D[(s*d + t) * N + n] = Zassenhaus displacement matrix of mu[n] (complex64, batch index last).
void launch_displacement(const float2 *mu, int64_t N, int d, const float *tab, float2 *D, int num_sms,
                         cudaStream_t st);
// Measurement with the physical index of each row mixed by D(a.mu[row]) first (a.mu != nullptr,
// d <= kMaxDisplacedD, FP32 or BF16-plane next rows).  Launches a prep kernel (one thread per row:
// the row's matrix and uniform into a.disp_D / a.disp_u) and the measurement kernel.
void launch_measure_displaced(const MeasureArgs &a, int num_sms, cudaStream_t st);

// Self-test: one bounded mbarrier wait that nothing completes (status, device time waited).
void launch_bounded_wait_selftest(uint64_t limit_ns, int *status, unsigned long long *waited_ns, cudaStream_t st);

// out[n * M + k] = O[k * ldO + n] for n < N, k < M.
void launch_transpose_outcomes(const uint8_t *O, int64_t ldO, int64_t N, int M, uint8_t *out, cudaStream_t st);

}  // namespace fastmps

namespace fastmps {

// ---- persistent batched kernel: every round of every job in one launch --------------------------
// Tasks are the tiles of all segments of all rounds, in round order (segments of round r, each
// m-tile-major); a segment's tasks occupy [task_begin, task_begin + num_m_tiles * num_n_tiles).
struct PSegment {  // 64-byte aligned through its CUtensorMap members
    CUtensorMap tmA[3];
    CUtensorMap tmB[2];
    int64_t task_begin;
    int num_m_tiles, num_n_tiles, num_k_blocks, bn;
    uint32_t idesc, tx_bytes;
    int row0;            // TMA y coordinate of the chunk's first row in the job's left-operand buffers
    int step;            // c * M + k: measurements every m-tile of this chunk has had before this segment
    int64_t slot_base;   // measured[slot_base + mt]: measurements completed by m-tile slot mt of the job
    int64_t done_base;   // tiles_done[done_base + mt]: finished tiles of m-tile mt of this segment
    float *Y;
    int64_t ldY;
    float *P;
    int ldP;
    int rows_valid;
};

struct PersistentArgs {
    const PSegment *segs;      // device
    const MeasureArgs *meas;   // device, one per segment
    int nseg;
    int64_t total_tasks;
    int *queue;                // device: next task (zero at launch)
    int *measured;             // device: per job m-tile slot (zero at launch)
    int *tiles_done;           // device: per segment m-tile (zero at launch)
    int a_planes, b_planes, nprod;
    int prod_a[kMaxProducts], prod_b[kMaxProducts];
    uint64_t wait_limit_ns;    // bound of every wait (a dependency that never resolves ends the launch)
    int stall_test;            // test hook: dependencies ask for one measurement more than ever happens
};

// Sets the kernel's shared-memory attribute (call once before launching, outside stream capture).
cudaError_t prepare_batch_persistent();
cudaError_t launch_batch_persistent(const PersistentArgs &g, int num_sms, int *d_err, cudaStream_t st);

}  // namespace fastmps
