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
//   so one entry of the product is a sum of min(s, t) + 1 terms (the real
//   series in FP64 from a table of constants).  Every sample
//   has its own mu; batched matrices are written with the batch index last, so
//   consecutive threads of a warp write consecutive samples (coalesced).
// * Displaced measurement: for sample n at site k, the contracted blocks y_t
//   (t < d) are mixed, z_s = sum_t D(mu[k, n])[s, t] y_t, before the
//   probabilities w_s = ||z_s||^2 are formed; the draw is Algorithm 2's, and the
//   next left vector is z_{s*} / sqrt(w_{s*}).  The mixing couples all d blocks
//   of a row, which no contraction tile holds together (a tile covers columns
//   of one outcome), so this kernel reads the whole FP32 scratch row: once for
//   the probabilities, once more (from L2) for the selected combination.
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
// cancels heavily (terms of order 10^3, sum of order 1 at d = 16, |mu| = 2.5), so S is summed in
// FP64 with the FP64 constants c_st and q_m of a host-built table; g and the leading power, which
// multiply the whole entry, are taken in FP32.  GB300's FP64 pipes are narrow: the table leaves
// three FP64 operations per series term and no FP64 division, square root or exponential.
//
// Table layout (host-built by build_displacement_table): entry (s, t) at tab[(s*d + t) * (d + 1)]:
// [c_st, q_1, ..., q_min(s,t)].
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ float2 displacement_entry(float2 mu, int s, int t, int d, const double *__restrict__ tab, float g) {
    const double *e = tab + (s * d + t) * (d + 1);
    const int j = min(s, t), p = max(s, t) - j;
    const float2 base = s >= t ? mu : make_float2(-mu.x, mu.y);  // mu, or -mu^*
    float2 lead = make_float2(1.f, 0.f);
    for (int q = 0; q < p; ++q) lead = cmulf(lead, base);
    const double mx = -((double)mu.x * (double)mu.x + (double)mu.y * (double)mu.y);
    double r = 1.0, S = 1.0;
    for (int m = j; m >= 1; --m) {
        r *= mx * e[m];
        S += r;
    }
    const float f = g * (float)(e[0] * S);
    return make_float2(f * lead.x, f * lead.y);
}

// D[(s*d + t) * N + n] for every sample n (batch index last)
__global__ void displacement_kernel(const float2 *__restrict__ mu, int64_t N, int d, const double *__restrict__ tab,
                                    float2 *__restrict__ D) {
    const int st = blockIdx.y;  // s * d + t
    const int s = st / d, t = st % d;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float2 m = mu[n];
        const float g = expf(-0.5f * (m.x * m.x + m.y * m.y));
        D[(int64_t)st * N + n] = displacement_entry(m, s, t, d, tab, g);
    }
}

void launch_displacement(const float2 *mu, int64_t N, int d, const double *tab, float2 *D, cudaStream_t st) {
    if (N <= 0) return;
    const int threads = 256;
    const int64_t bx = std::min<int64_t>((N + threads - 1) / threads, 4096);
    dim3 grid((unsigned)bx, (unsigned)(d * d));
    displacement_kernel<<<grid, threads, 0, st>>>(mu, N, d, tab, D);
}

// ---------------------------------------------------------------------------
// Displaced measurement: one warp per sample row
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

// kStaged: the warp first copies its whole scratch row (d * Cs floats) into shared memory with
// cp.async (16-byte copies, all in flight at once), so both passes read shared memory and the row
// crosses HBM once.  Otherwise (rows too large for shared memory) both passes read global memory and
// the second relies on L2.
template <int DMAX, bool kStaged>
__global__ void __launch_bounds__(DISP_WARPS * 32) measure_displaced_kernel(const MeasureArgs a, int rows_per_block) {
    __shared__ float2 Dsh[DISP_WARPS][DMAX * DMAX];
    extern __shared__ __align__(16) float staged[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * rows_per_block + warp;
    if (row >= a.rows) return;  // whole warps only: no block-level barrier below
    const int d = a.d, chi_r = a.chi_r;
    const int64_t Cs = a.Cs;
    const float *yrow = a.Y + (int64_t)row * a.ldY;
    if (kStaged) {
        const int nf = d * (int)Cs;  // multiple of 32 floats; the row start is 128-byte aligned
        float *srow = staged + (size_t)warp * nf;
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(srow);
        for (int i = lane * 4; i < nf; i += 128)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 4u * (uint32_t)i), "l"(yrow + i)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    float2 *D = Dsh[warp];
    const float2 mu = a.mu[row];
    const float g = expf(-0.5f * (mu.x * mu.x + mu.y * mu.y));
    for (int e = lane; e < d * d; e += 32) D[e] = displacement_entry(mu, e / d, e % d, d, a.disp_tab, g);
    if (kStaged) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        yrow = staged + (size_t)warp * d * (int)Cs;
    }
    __syncwarp();
    auto ld = [&](int64_t i) -> float { return kStaged ? yrow[i] : __ldcg(yrow + i); };

    // pass 1: w_s = sum_b |sum_t D[s][t] y_t[b]|^2, FP32 per lane, FP64 across lanes
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
    double wd[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        double v = (double)w[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        wd[s] = v;
    }

    // the draw (every lane holds the sums): C_s in s order, s* = first s with C_s >= u Z, else d-1
    double Z = 0.0;
#pragma unroll
    for (int s = 0; s < DMAX; ++s)
        if (s < d) Z += wd[s];
    const uint64_t n = a.n_base + (uint64_t)row;
    const double thr = sample_uniform(a.seed, n, a.k, a.job) * Z;
    int sstar = d - 1;
    double ws = 0.0, C = 0.0;
    bool found = false;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        if (s < d && !found) {
            C += wd[s];
            if (s == d - 1 || C >= thr) {
                sstar = s;
                ws = wd[s];
                found = true;
            }
        }
    }
    const bool ok = (Z > 0.0) && isfinite(Z) && (ws > 0.0);
    const int64_t grow = a.row0 + row;
    if (lane == 0) {
        a.outcomes[row] = (uint8_t)sstar;
        if (ok) a.logp[grow] += (double)(logf((float)ws) - logf((float)Z));
        else atomicExch(a.err, (int)kDevNumeric);
        if (a.trace && grow < a.trace_rows) {
#pragma unroll
            for (int s = 0; s < DMAX; ++s)
                if (s < d) a.trace[grow * d + s] = ok ? wd[s] / Z : 0.0;
        }
    }

    // pass 2: next left row = (sum_t D[s*][t] y_t) / sqrt(w_{s*}), written as [Re | Im | zero padding]
    const float scale = ok ? rsqrtf((float)ws) : 0.f;
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

// Shared memory of the staged variant: at most 96 KB of rows per block (two blocks per SM),
// rows above 200 KB (e.g. d = 3, chi = 10^4) use the unstaged variant.
constexpr int kStageBudget = 96 * 1024;
constexpr int kStageMaxRow = 200 * 1024;

template <int DMAX>
void launch_displaced_variant(const MeasureArgs &a, cudaStream_t st) {
    const size_t row_bytes = (size_t)a.d * a.Cs * sizeof(float);
    if (row_bytes > (size_t)kStageMaxRow || (int64_t)a.d * a.Cs > a.ldY) {
        const int grid = (a.rows + DISP_WARPS - 1) / DISP_WARPS;
        measure_displaced_kernel<DMAX, false><<<grid, DISP_WARPS * 32, 0, st>>>(a, DISP_WARPS);
        return;
    }
    const int rpb = (int)std::max<size_t>(1, std::min<size_t>(DISP_WARPS, kStageBudget / row_bytes));
    const size_t smem = (size_t)rpb * row_bytes;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(measure_displaced_kernel<DMAX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStageMaxRow + 1024);
        attr_set = true;
    }
    const int grid = (a.rows + rpb - 1) / rpb;
    measure_displaced_kernel<DMAX, true><<<grid, rpb * 32, smem, st>>>(a, rpb);
}

void launch_measure_displaced(const MeasureArgs &a, cudaStream_t st) {
    if (a.rows <= 0) return;
    if (a.d <= 4) launch_displaced_variant<4>(a, st);
    else if (a.d <= 8) launch_displaced_variant<8>(a, st);
    else launch_displaced_variant<kMaxDisplacedD>(a, st);
}

}  // namespace fastmps

namespace fastmps {

void build_displacement_table(int d, double *tab) {
    for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t) {
            double *e = tab + (s * d + t) * (d + 1);
            const int j = s < t ? s : t, hi = s < t ? t : s;
            double c = 1.0;
            for (int q = j + 1; q <= hi; ++q) c *= std::sqrt((double)q) / (double)(q - j);
            e[0] = c;
            for (int m = 1; m <= d; ++m)
                e[m] = m <= j ? (double)m / ((double)(s - m + 1) * (double)(t - m + 1)) : 0.0;
        }
}

}  // namespace fastmps
