// Vidal-form input and Gaussian-boson-sampling displacement (device code).
//
// * Vidal form (Sec. 2.2 workflow over the tensors Gamma_i; Algorithm 2 takes
//   the coefficient vector Lambda): the site is stored as the right-canonical
//   A_k[a, s, b] = Gamma_k[a, s, b] * Lambda_k[b], scaled in the staging copy
//   before the repack, so that sampling runs the canonical path unchanged.
// * Displacement (Sec. 3.4.1): the displacement operator exp(mu a^+ - mu^* a)
//   on the physical index is taken as the Zassenhaus product
//   exp(-|mu|^2/2) exp(mu a^+) exp(-mu^* a) of a lower- and an upper-triangular
//   matrix, each of which has closed-form entries:
//     exp(mu a^+)[s][m]  = mu^(s-m)      sqrt(s!/m!) / (s-m)!   (s >= m)
//     exp(-mu^* a)[m][t] = (-mu^*)^(t-m) sqrt(t!/m!) / (t-m)!   (t >= m)
//   so one entry of the product is a sum of min(s, t) + 1 terms (a real
//   alternating series, summed in float-float arithmetic).  Every sample
//   has its own mu; batched matrices are written with the batch index last, so
//   consecutive threads of a warp write consecutive samples (coalesced).
// * Displaced measurement: for sample n at site k, the contracted blocks y_t
//   (t < d) are mixed, z_s = sum_t D(mu[k, n])[s, t] y_t, before the
//   probabilities w_s = ||z_s||^2 are formed; the draw is Algorithm 2's, and the
//   next left vector is z_{s*} / sqrt(w_{s*}).  The mixing couples all d blocks
//   of a row, which no contraction tile holds together (a tile covers columns
//   of one outcome), so this kernel reads the whole FP32 scratch row (staged in
//   shared memory, so that it crosses HBM once) to form the probabilities and
//   the selected combination.
// GB300's FP64 pipes are narrow (a warp-wide FP64 instruction costs an SM
// about 16 issue cycles): FP64 is kept to the draw itself; the displacement
// series uses float-float (error-free FP32 transformations) and the lane sums
// are reduced in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "launch.h"
#include "measure.cuh"

namespace fastmps {

// ---------------------------------------------------------------------------
// Vidal form: A[a, s, b] = Gamma[a, s, b] * Lambda[b], in place on the staging copy
// ---------------------------------------------------------------------------
__global__ void scale_columns_kernel(void *A, int is_f64, int64_t n_complex, int chi_r, const void *lam) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_complex;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e % chi_r);
        if (is_f64) {
            const double l = static_cast<const double *>(lam)[b];
            double *p = static_cast<double *>(A) + 2 * e;
            p[0] *= l;
            p[1] *= l;
        } else {
            const float l = static_cast<const float *>(lam)[b];
            float *p = static_cast<float *>(A) + 2 * e;
            p[0] *= l;
            p[1] *= l;
        }
    }
}

void launch_scale_columns(void *A, int is_f64, int64_t n_complex, int chi_r, const void *lam, cudaStream_t st) {
    if (n_complex <= 0) return;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n_complex + threads - 1) / threads, 152 * 16);
    scale_columns_kernel<<<(unsigned)blocks, threads, 0, st>>>(A, is_f64, n_complex, chi_r, lam);
}

// ---------------------------------------------------------------------------
// One entry of the Zassenhaus displacement matrix
//
// D[s][t] = g sum_{m <= min(s,t)} L[s][m] U[m][t], g = exp(-|mu|^2/2).  Along the sum, consecutive
// terms differ by a real factor:
//   term_{m-1} / term_m = -|mu|^2 q_m,  q_m = m / ((s-m+1)(t-m+1)),
// so D[s][t] = g c_st lead(mu) S with the leading power lead = mu^(s-t) (s >= t) or (-mu^*)^(t-s),
// c_st = sqrt(max(s,t)! / min(s,t)!) / |s-t|!, and the real alternating series
// S = 1 + sum_{m=min(s,t)}^{1} prod_{m' >= m} (-|mu|^2 q_m').  For large d and |mu| the series
// cancels heavily (terms of order 10^3, sum of order 1 at d = 16, |mu| = 2.5: a plain FP32 sum loses
// 7e-5), so S is carried as an unevaluated float-float pair (hi + lo, ~44 significant bits) built
// from exact FP32 products (fmaf) and exact sums (two-sum); |mu|^2 and q_m enter as float-float
// values too.  g, c_st and the leading power multiply the whole entry and are taken in FP32.
//
// Table layout (host-built by build_displacement_table): entry (s, t) at tab[(s*d + t) * (2d + 1)]:
// [c_st, hi(q_1), lo(q_1), ..., hi(q_d), lo(q_d)] (q_m = 0 for m > min(s, t)).
// ---------------------------------------------------------------------------
struct ffloat {
    float hi, lo;
};

__device__ __forceinline__ ffloat ff_two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ffloat ff_mul(ffloat a, ffloat b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return {h, e - (h - p)};
}

__device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// mx = -|mu|^2 as a float-float value, g = exp(-|mu|^2 / 2)
__device__ __forceinline__ ffloat neg_abs2(float2 mu) {
    const ffloat xr = ff_two_prod(mu.x, mu.x), xi = ff_two_prod(mu.y, mu.y);
    const ffloat x = ff_add(xr, xi);
    return {-x.hi, -x.lo};
}

__device__ float2 displacement_entry(float2 mu, ffloat mx, float g, int s, int t, int d,
                                     const float *__restrict__ tab) {
    const float *e = tab + (s * d + t) * (2 * d + 1);
    const int j = min(s, t), p = max(s, t) - j;
    const float2 base = s >= t ? mu : make_float2(-mu.x, mu.y);  // mu, or -mu^*
    float2 lead = make_float2(1.f, 0.f);
    for (int q = 0; q < p; ++q) lead = cmulf(lead, base);
    ffloat r = {1.f, 0.f}, S = {1.f, 0.f};
    for (int m = j; m >= 1; --m) {
        r = ff_mul(r, ff_mul(mx, ffloat{e[2 * m - 1], e[2 * m]}));
        S = ff_add(S, r);
    }
    const float f = g * e[0] * (S.hi + S.lo);
    return make_float2(f * lead.x, f * lead.y);
}

// One thread per sample: all d*d entries, written D[(s*d + t) * N + n] (batch index last, so each
// store instruction of a warp covers 32 consecutive samples)
__global__ void __launch_bounds__(256) displacement_kernel(const float2 *__restrict__ mu, int64_t N, int d,
                                                           const float *__restrict__ tab, float2 *__restrict__ D) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float2 m = mu[n];
        const ffloat mx = neg_abs2(m);
        const float g = expf(0.5f * (mx.hi + mx.lo));
        for (int s = 0; s < d; ++s)
            for (int t = 0; t < d; ++t) D[(int64_t)(s * d + t) * N + n] = displacement_entry(m, mx, g, s, t, d, tab);
    }
}

void launch_displacement(const float2 *mu, int64_t N, int d, const float *tab, float2 *D, int num_sms,
                         cudaStream_t st) {
    if (N <= 0) return;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((N + threads - 1) / threads, (int64_t)num_sms * 8);
    displacement_kernel<<<(unsigned)blocks, threads, 0, st>>>(mu, N, d, tab, D);
}

// ---------------------------------------------------------------------------
// Displaced measurement: one warp per sample row at a time
// ---------------------------------------------------------------------------
constexpr int DISP_WARPS = 4;

__device__ __forceinline__ void store_next(const MeasureArgs &a, int64_t grow, int i, float x) {
    if (a.V32) {
        a.V32[grow * a.ld_next + i] = x;
        return;
    }
    __nv_bfloat16 h0, h1, h2;
    write_planes(x, a.nplanes, h0, h1, h2);
    a.Vp[0][grow * a.ld_next + i] = h0;
    a.Vp[1][grow * a.ld_next + i] = h1;
    if (a.nplanes > 2) a.Vp[2][grow * a.ld_next + i] = h2;
}

__device__ __forceinline__ void stage_row(float *dst, const float *src, int nf, int lane) {
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(dst);
    for (int i = lane * 4; i < nf; i += 128)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 4u * (uint32_t)i), "l"(src + i)
                     : "memory");
}

// The measurement of one row given the row's scratch values (global or shared memory) and D.
template <int DMAX, bool kShared>
__device__ __forceinline__ void displaced_row(const MeasureArgs &a, int row, const float *yrow, const float2 *D,
                                              int lane) {
    const int d = a.d, chi_r = a.chi_r;
    const int64_t Cs = a.Cs;
    auto ld = [&](int64_t i) -> float { return kShared ? yrow[i] : __ldcg(yrow + i); };
    // pass 1: w_s = sum_b |sum_t D[s][t] y_t[b]|^2 (FP32; the lane sums are reduced in FP32)
    float w[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) w[s] = 0.f;
    for (int b = lane; b < chi_r; b += 32) {
        float2 y[DMAX];
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
            y[t] = t < d ? make_float2(ld(t * Cs + b), ld(t * Cs + chi_r + b)) : make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < DMAX; ++s) {
            if (s >= d) break;
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int t = 0; t < DMAX; ++t) {
                if (t >= d) break;
                const float2 c = D[s * d + t];
                zr = fmaf(c.x, y[t].x, fmaf(-c.y, y[t].y, zr));
                zi = fmaf(c.x, y[t].y, fmaf(c.y, y[t].x, zi));
            }
            w[s] = fmaf(zr, zr, fmaf(zi, zi, w[s]));
        }
    }
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w[s] += __shfl_xor_sync(0xffffffffu, w[s], o);
    }
    // the draw in FP64 on the reduced sums (every lane holds them): C_s in s order,
    // s* = first s with C_s >= u Z, else d-1
    double Z = 0.0;
#pragma unroll
    for (int s = 0; s < DMAX; ++s)
        if (s < d) Z += (double)w[s];
    const uint64_t n = a.n_base + (uint64_t)row;
    const double thr = sample_uniform(a.seed, n, a.k, a.job) * Z;
    int sstar = d - 1;
    float ws = 0.f;
    double C = 0.0;
    bool found = false;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        if (s < d && !found) {
            C += (double)w[s];
            if (s == d - 1 || C >= thr) {
                sstar = s;
                ws = w[s];
                found = true;
            }
        }
    }
    const bool ok = (Z > 0.0) && isfinite(Z) && (ws > 0.f);
    const int64_t grow = a.row0 + row;
    if (lane == 0) {
        a.outcomes[row] = (uint8_t)sstar;
        if (ok) a.logp[grow] += (double)(logf(ws) - logf((float)Z));
        else atomicExch(a.err, (int)kDevNumeric);
        if (a.trace && grow < a.trace_rows) {
#pragma unroll
            for (int s = 0; s < DMAX; ++s)
                if (s < d) a.trace[grow * d + s] = ok ? (double)w[s] / Z : 0.0;
        }
    }
    // pass 2: next left row = (sum_t D[s*][t] y_t) / sqrt(w_{s*}), written as [Re | Im | zero padding]
    const float scale = ok ? rsqrtf(ws) : 0.f;
    float2 c[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        const float2 e = t < d ? D[sstar * d + t] : make_float2(0.f, 0.f);
        c[t] = make_float2(e.x * scale, e.y * scale);
    }
    for (int b = lane; b < chi_r; b += 32) {
        float zr = 0.f, zi = 0.f;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
            if (t >= d) break;
            const float yr = ld(t * Cs + b), yi = ld(t * Cs + chi_r + b);
            zr = fmaf(c[t].x, yr, fmaf(-c[t].y, yi, zr));
            zi = fmaf(c[t].x, yi, fmaf(c[t].y, yr, zi));
        }
        store_next(a, grow, b, zr);
        store_next(a, grow, chi_r + b, zi);
    }
    for (int i = 2 * chi_r + lane; i < a.K_next; i += 32) store_next(a, grow, i, 0.f);
}

__device__ __forceinline__ void build_D(const MeasureArgs &a, int row, float2 *D, int lane) {
    const int d = a.d;
    const float2 mu = a.mu[row];
    const ffloat mx = neg_abs2(mu);
    const float g = expf(0.5f * (mx.hi + mx.lo));
    for (int e = lane; e < d * d; e += 32) D[e] = displacement_entry(mu, mx, g, e / d, e % d, d, a.disp_tab);
}

// Persistent, staged: each warp walks rows r = gw, gw + W, ... (W warps in the grid), with two shared
// buffers of one scratch row each: the row after next is copied (cp.async) while this one is measured.
template <int DMAX>
__global__ void __launch_bounds__(DISP_WARPS * 32) measure_displaced_staged_kernel(const MeasureArgs a,
                                                                                  int total_warps) {
    __shared__ float2 Dsh[DISP_WARPS][DMAX * DMAX];
    extern __shared__ __align__(16) float staged[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    if (gw >= a.rows) return;  // whole warps only: no block-level barrier below
    const int nf = a.d * a.Cs;  // floats of one row; a multiple of 32, and each row starts 128-byte aligned
    float *const mine = staged + (size_t)warp * 2 * nf;  // this warp's two row buffers
    stage_row(mine, a.Y + (int64_t)gw * a.ldY, nf, lane);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int cur = 0;
    for (int row = gw; row < a.rows; row += total_warps, cur ^= 1) {
        const int next = row + total_warps;
        if (next < a.rows) stage_row(mine + (size_t)(cur ^ 1) * nf, a.Y + (int64_t)next * a.ldY, nf, lane);
        asm volatile("cp.async.commit_group;" ::: "memory");
        build_D(a, row, Dsh[warp], lane);
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this row's copy (all but the newest group)
        __syncwarp();
        displaced_row<DMAX, true>(a, row, mine + (size_t)cur * nf, Dsh[warp], lane);
        __syncwarp();  // this buffer and D are reused by the next iterations
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Unstaged (rows above the shared-memory limit): one row per warp, the second pass relies on L2.
template <int DMAX>
__global__ void __launch_bounds__(DISP_WARPS * 32) measure_displaced_kernel(const MeasureArgs a) {
    __shared__ float2 Dsh[DISP_WARPS][DMAX * DMAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * DISP_WARPS + warp;
    if (row >= a.rows) return;
    build_D(a, row, Dsh[warp], lane);
    __syncwarp();
    displaced_row<DMAX, false>(a, row, a.Y + (int64_t)row * a.ldY, Dsh[warp], lane);
}

// Two row buffers per warp must fit: rows up to 48 KB are staged (4 warps x 2 x 48 KB would not fit
// one SM, so the warps per block shrink with the row size).
constexpr size_t kStageSmem = 200 * 1024;   // shared memory per block for staged rows
constexpr size_t kStageMaxRow = 48 * 1024;

template <int DMAX>
void launch_displaced_variant(const MeasureArgs &a, int num_sms, cudaStream_t st) {
    const size_t row_bytes = (size_t)a.d * a.Cs * sizeof(float);
    if (row_bytes > kStageMaxRow || (int64_t)a.d * a.Cs > a.ldY) {
        const int grid = (a.rows + DISP_WARPS - 1) / DISP_WARPS;
        measure_displaced_kernel<DMAX><<<grid, DISP_WARPS * 32, 0, st>>>(a);
        return;
    }
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(DISP_WARPS, kStageSmem / (2 * row_bytes)));
    const size_t smem = (size_t)wpb * 2 * row_bytes;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(measure_displaced_staged_kernel<DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kStageSmem);
        attr_set = true;
    }
    // blocks resident per SM (227 KB of shared memory, DMAX^2 * 8 bytes static per warp)
    const size_t per_block = smem + (size_t)DISP_WARPS * DMAX * DMAX * 8 + 1024;
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(227 * 1024) / per_block));
    const int64_t want = ((int64_t)a.rows + wpb - 1) / wpb;
    const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms * per_sm);
    measure_displaced_staged_kernel<DMAX><<<grid, wpb * 32, smem, st>>>(a, grid * wpb);
}

void launch_measure_displaced(const MeasureArgs &a, int num_sms, cudaStream_t st) {
    if (a.rows <= 0) return;
    if (a.d <= 4) launch_displaced_variant<4>(a, num_sms, st);
    else if (a.d <= 8) launch_displaced_variant<8>(a, num_sms, st);
    else launch_displaced_variant<kMaxDisplacedD>(a, num_sms, st);
}

}  // namespace fastmps

namespace fastmps {

void build_displacement_table(int d, float *tab) {
    for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t) {
            float *e = tab + (s * d + t) * (2 * d + 1);
            const int j = s < t ? s : t, hi = s < t ? t : s;
            double c = 1.0;
            for (int q = j + 1; q <= hi; ++q) c *= std::sqrt((double)q) / (double)(q - j);
            e[0] = (float)c;
            for (int m = 1; m <= d; ++m) {
                const double q = m <= j ? (double)m / ((double)(s - m + 1) * (double)(t - m + 1)) : 0.0;
                const float qh = (float)q;
                e[2 * m - 1] = qh;
                e[2 * m] = (float)(q - (double)qh);
            }
        }
}

}  // namespace fastmps
