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
//   of one outcome), so this kernel reads the whole FP32 scratch row (held in
//   registers by one small thread block per row, so that it crosses HBM once)
//   to form the probabilities and the selected combination.
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

// The d*d entries of one sample for d <= DMAX, loops unrolled at compile time: the powers mu^k and
// (-mu^*)^k are formed once per sample and each entry's series has a fixed length.  out(e, value)
// receives entry e = s*d + t.
template <int DMAX, class Out>
__device__ __forceinline__ void displacement_matrix(float2 mu, int d, const float *__restrict__ tab, Out out) {
    const ffloat mx = neg_abs2(mu);
    const float g = expf(0.5f * (mx.hi + mx.lo));
    float2 pw[DMAX], pc[DMAX];  // mu^k and (-mu^*)^k
    pw[0] = pc[0] = make_float2(1.f, 0.f);
    const float2 nmc = make_float2(-mu.x, mu.y);
#pragma unroll
    for (int k = 1; k < DMAX; ++k) {
        pw[k] = cmulf(pw[k - 1], mu);
        pc[k] = cmulf(pc[k - 1], nmc);
    }
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        if (s >= d) break;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
            if (t >= d) break;
            const float *e = tab + (s * d + t) * (2 * d + 1);
            const int j = s < t ? s : t;
            ffloat r = {1.f, 0.f}, S = {1.f, 0.f};
#pragma unroll
            for (int m = DMAX - 1; m >= 1; --m) {
                if (m > j) continue;
                r = ff_mul(r, ff_mul(mx, ffloat{e[2 * m - 1], e[2 * m]}));
                S = ff_add(S, r);
            }
            const float f = g * e[0] * (S.hi + S.lo);
            const float2 lead = s >= t ? pw[s - t] : pc[t - s];
            out(s * d + t, make_float2(f * lead.x, f * lead.y));
        }
    }
}

template <int DMAX>
__global__ void __launch_bounds__(256) displacement_small_kernel(const float2 *__restrict__ mu, int64_t N, int d,
                                                                 const float *tab, float2 *D) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        // entries arrive in order e = 0, 1, ...: a running pointer (stride N) instead of e * N per entry
        float2 *q = D + n;
        displacement_matrix<DMAX>(mu[n], d, tab, [&](int, float2 v) {
            *q = v;
            q += N;
        });
    }
}

void launch_displacement(const float2 *mu, int64_t N, int d, const float *tab, float2 *D, int num_sms,
                         cudaStream_t st) {
    if (N <= 0) return;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((N + threads - 1) / threads, (int64_t)num_sms * 8);
    // (a fully unrolled 16 x 16 matrix no longer fits the register file: d > 8 takes the loop form)
    if (d <= 4) displacement_small_kernel<4><<<(unsigned)blocks, threads, 0, st>>>(mu, N, d, tab, D);
    else if (d <= 8) displacement_small_kernel<8><<<(unsigned)blocks, threads, 0, st>>>(mu, N, d, tab, D);
    else displacement_kernel<<<(unsigned)blocks, threads, 0, st>>>(mu, N, d, tab, D);
}

// Per-row inputs of the displaced measurement, one thread per row: the row's displacement matrix
// D[row][s*d + t] and its uniform u = U(seed, n, k, job), so that the measurement kernel's
// per-row serial section is only the draw.
template <int DMAX>
__global__ void __launch_bounds__(256) displaced_prep_kernel(const MeasureArgs a) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.rows) return;
    float2 *out = a.disp_D + (int64_t)row * a.d * a.d;
    displacement_matrix<DMAX>(a.mu[row], a.d, a.disp_tab, [&](int e, float2 v) { out[e] = v; });
    a.disp_u[row] = sample_uniform(a.seed, a.n_base + (uint64_t)row, a.k, a.job);
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

// ---------------------------------------------------------------------------
// Register-resident displaced measurement: one thread block per sample row.  Thread j holds columns
// of all d blocks of the row in registers (four consecutive columns per 16-byte load in the vector
// variant, single columns in the scalar one), so the row crosses HBM once and both passes read
// registers.  The d x d matrix of the row (prep kernel) is read by every thread through L1.
// The lane sums are reduced in FP32 (shuffles, then across warps through shared memory: the only
// block barrier), and every thread takes the same draw:
//   * fast path in FP32: prefix sums C_s and threshold u Z.  Their rounding error is below
//     16 * 2^-24 Z for d <= 16, so when every |C_s - u Z| exceeds 1e-5 Z the FP32 comparison
//     decides exactly as the FP64 one on the same sums;
//   * otherwise (about 2 d 1e-5 of the draws) the prefix sums and the threshold in FP64.
// This keeps GB300's narrow FP64 pipes off the common path while the decision stays the FP64 one.
// ---------------------------------------------------------------------------
template <int DMAX>
__device__ __forceinline__ int displaced_draw(const float (&w)[DMAX], int d, double u, float &wsel, float &Z32) {
    float C32[DMAX];
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        if (s < d) acc += w[s];
        C32[s] = acc;
    }
    Z32 = acc;
    const float thr32 = (float)u * acc;
    const float band = 1e-5f * acc;
    int sstar = d - 1;
    bool near = false;
#pragma unroll
    for (int s = DMAX - 1; s >= 0; --s) {
        if (s < d - 1) {
            if (C32[s] >= thr32) sstar = s;
            if (fabsf(C32[s] - thr32) <= band) near = true;
        }
    }
    if (near) {
        double C[DMAX];
        double a64 = 0.0;
#pragma unroll
        for (int s = 0; s < DMAX; ++s) {
            if (s < d) a64 += (double)w[s];
            C[s] = a64;
        }
        const double thr = u * a64;
        sstar = d - 1;
#pragma unroll
        for (int s = DMAX - 1; s >= 0; --s)
            if (s < d - 1 && C[s] >= thr) sstar = s;
    }
    wsel = 0.f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s)
        if (s == sstar) wsel = w[s];
    return sstar;
}

// Block-wide FP32 reduction of w[DMAX] (same summation order in every thread, so every thread ends
// with identical sums).
template <int DMAX>
__device__ __forceinline__ void block_reduce_w(float (&w)[DMAX], float (*red)[DMAX], int lane, int warp, int nw) {
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w[s] += __shfl_xor_sync(0xffffffffu, w[s], o);
    }
    if (nw == 1) return;
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < DMAX; ++s) red[warp][s] = w[s];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        float acc = 0.f;
        for (int q = 0; q < nw; ++q) acc += red[q][s];
        w[s] = acc;
    }
}

// Outcome, log-probability, trace (thread 0 of the block).
template <int DMAX>
__device__ __forceinline__ void displaced_outputs(const MeasureArgs &a, int row, int sstar, float wsel, float Z32,
                                                  const float (&w)[DMAX]) {
    const int d = a.d;
    const bool ok = (Z32 > 0.f) && isfinite(Z32) && (wsel > 0.f);
    const int64_t grow = a.row0 + row;
    a.outcomes[row] = (uint8_t)sstar;
    if (ok) a.logp[grow] += log((double)wsel / (double)Z32);  // FP64 log of the FP32 sums' ratio
    else atomicExch(a.err, (int)kDevNumeric);
    const int64_t slot = a.trace ? (a.trace_slot ? (int64_t)a.trace_slot[grow] : (grow < a.trace_rows ? grow : -1))
                                 : -1;
    if (slot >= 0) {
#pragma unroll
        for (int s = 0; s < DMAX; ++s)
            if (s < d) a.trace[slot * d + s] = ok ? (double)w[s] / (double)Z32 : 0.0;
    }
}

// Unstaged fallback (rows too wide for the register-resident and shared-memory variants, e.g.
// chi = 10^4): one warp per row, two passes over the row in global memory (the second from L2).
template <int DMAX>
__global__ void __launch_bounds__(DISP_WARPS * 32) measure_displaced_kernel(const MeasureArgs a) {
    __shared__ float2 Dsh[DISP_WARPS][DMAX * DMAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * DISP_WARPS + warp;
    if (row >= a.rows) return;
    const int d = a.d, chi_r = a.chi_r, dd = d * d;
    const int64_t Cs = a.Cs;
    float2 *D = Dsh[warp];
    for (int e = lane; e < dd; e += 32) D[e] = a.disp_D[(int64_t)row * dd + e];
    __syncwarp();
    const float *yrow = a.Y + (int64_t)row * a.ldY;
    float w[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) w[s] = 0.f;
    for (int b = lane; b < chi_r; b += 32) {
        float2 y[DMAX];
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
            y[t] = t < d ? make_float2(__ldcg(yrow + t * Cs + b), __ldcg(yrow + t * Cs + chi_r + b))
                         : make_float2(0.f, 0.f);
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
    block_reduce_w<DMAX>(w, nullptr, lane, 0, 1);
    float wsel, Z32;
    const int sstar = displaced_draw<DMAX>(w, d, a.disp_u[row], wsel, Z32);
    if (lane == 0) displaced_outputs<DMAX>(a, row, sstar, wsel, Z32, w);
    const float scale = wsel > 0.f && Z32 > 0.f && isfinite(Z32) ? rsqrtf(wsel) : 0.f;
    float2 c[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        const float2 e = t < d ? D[sstar * d + t] : make_float2(0.f, 0.f);
        c[t] = make_float2(e.x * scale, e.y * scale);
    }
    const int64_t grow = a.row0 + row;
    for (int b = lane; b < chi_r; b += 32) {
        float zr = 0.f, zi = 0.f;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
            if (t >= d) break;
            const float yr = __ldcg(yrow + t * Cs + b), yi = __ldcg(yrow + t * Cs + chi_r + b);
            zr = fmaf(c[t].x, yr, fmaf(-c[t].y, yi, zr));
            zi = fmaf(c[t].x, yi, fmaf(c[t].y, yr, zi));
        }
        store_next(a, grow, b, zr);
        store_next(a, grow, chi_r + b, zi);
    }
    for (int i = 2 * chi_r + lane; i < a.K_next; i += 32) store_next(a, grow, i, 0.f);
}

template <int DMAX, int VPT>
__global__ void __launch_bounds__(256) measure_displaced_rows_kernel(const MeasureArgs a) {
    __shared__ float red[8][DMAX];
    const int row = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x;
    const int d = a.d, chi_r = a.chi_r, dd = d * d;
    const int64_t Cs = a.Cs;
    const float *yrow = a.Y + (int64_t)row * a.ldY;
    const float2 *Drow = a.disp_D + (int64_t)row * dd;
    const double u = a.disp_u[row];
    float2 y[VPT][DMAX];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int b = tid + T * v;
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
            y[v][t] = (t < d && b < chi_r) ? make_float2(__ldcs(yrow + t * Cs + b), __ldcs(yrow + t * Cs + chi_r + b))
                                          : make_float2(0.f, 0.f);
    }
    float w[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        w[s] = 0.f;
        if (s >= d) continue;
        float2 c[DMAX];
#pragma unroll
        for (int t = 0; t < DMAX; ++t) c[t] = t < d ? Drow[s * d + t] : make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int t = 0; t < DMAX; ++t) {
                zr = fmaf(c[t].x, y[v][t].x, fmaf(-c[t].y, y[v][t].y, zr));
                zi = fmaf(c[t].x, y[v][t].y, fmaf(c[t].y, y[v][t].x, zi));
            }
            w[s] = fmaf(zr, zr, fmaf(zi, zi, w[s]));
        }
    }
    block_reduce_w<DMAX>(w, red, lane, warp, T >> 5);
    float wsel, Z32;
    const int sstar = displaced_draw<DMAX>(w, d, u, wsel, Z32);
    if (tid == 0) displaced_outputs<DMAX>(a, row, sstar, wsel, Z32, w);
    const float scale = wsel > 0.f && Z32 > 0.f && isfinite(Z32) ? rsqrtf(wsel) : 0.f;
    float2 c[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        const float2 e = t < d ? Drow[sstar * d + t] : make_float2(0.f, 0.f);
        c[t] = make_float2(e.x * scale, e.y * scale);
    }
    const int64_t grow = a.row0 + row;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int b = tid + T * v;
        if (b >= chi_r) break;
        float zr = 0.f, zi = 0.f;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
            zr = fmaf(c[t].x, y[v][t].x, fmaf(-c[t].y, y[v][t].y, zr));
            zi = fmaf(c[t].x, y[v][t].y, fmaf(c[t].y, y[v][t].x, zi));
        }
        store_next(a, grow, b, zr);
        store_next(a, grow, chi_r + b, zi);
    }
    for (int i = 2 * chi_r + tid; i < a.K_next; i += T) store_next(a, grow, i, 0.f);
}

// Vectorised variant (chi_r a multiple of 4): thread j holds the four consecutive columns
// b = 4g .. 4g+3 of groups g = j + T v (v < G), loaded as 16-byte vectors, and writes the next row
// with 16-byte (FP32) or 8-byte (BF16 plane) stores.
__device__ __forceinline__ void store_next4(const MeasureArgs &a, int64_t grow, int i, float4 x) {
    if (a.V32) {
        *reinterpret_cast<float4 *>(a.V32 + grow * a.ld_next + i) = x;
        return;
    }
    const float v[4] = {x.x, x.y, x.z, x.w};
    __align__(8) __nv_bfloat16 p0[4], p1[4], p2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) write_planes(v[e], a.nplanes, p0[e], p1[e], p2[e]);
    const int64_t off = grow * a.ld_next + i;
    *reinterpret_cast<uint2 *>(a.Vp[0] + off) = *reinterpret_cast<const uint2 *>(p0);
    *reinterpret_cast<uint2 *>(a.Vp[1] + off) = *reinterpret_cast<const uint2 *>(p1);
    if (a.nplanes > 2) *reinterpret_cast<uint2 *>(a.Vp[2] + off) = *reinterpret_cast<const uint2 *>(p2);
}

__device__ __forceinline__ void cmac4(float2 c, const float4 &yr, const float4 &yi, float4 &zr, float4 &zi) {
    zr.x = fmaf(c.x, yr.x, fmaf(-c.y, yi.x, zr.x));
    zr.y = fmaf(c.x, yr.y, fmaf(-c.y, yi.y, zr.y));
    zr.z = fmaf(c.x, yr.z, fmaf(-c.y, yi.z, zr.z));
    zr.w = fmaf(c.x, yr.w, fmaf(-c.y, yi.w, zr.w));
    zi.x = fmaf(c.x, yi.x, fmaf(c.y, yr.x, zi.x));
    zi.y = fmaf(c.x, yi.y, fmaf(c.y, yr.y, zi.y));
    zi.z = fmaf(c.x, yi.z, fmaf(c.y, yr.z, zi.z));
    zi.w = fmaf(c.x, yi.w, fmaf(c.y, yr.w, zi.w));
}

template <int DMAX, int G>
__global__ void __launch_bounds__(256) measure_displaced_vec4_kernel(const MeasureArgs a) {
    __shared__ float red[8][DMAX];
    const int row = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x;
    const int d = a.d, chi_r = a.chi_r, ngroups = chi_r >> 2, dd = d * d;
    const int64_t Cs = a.Cs;
    const float *yrow = a.Y + (int64_t)row * a.ldY;
    const float2 *Drow = a.disp_D + (int64_t)row * dd;
    const double u = a.disp_u[row];
    float4 yr[G][DMAX], yi[G][DMAX];
#pragma unroll
    for (int v = 0; v < G; ++v) {
        const int g = tid + T * v;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
            if (t < d && g < ngroups) {
                yr[v][t] = __ldcs(reinterpret_cast<const float4 *>(yrow + t * Cs) + g);
                yi[v][t] = __ldcs(reinterpret_cast<const float4 *>(yrow + t * Cs + chi_r) + g);
            } else {
                yr[v][t] = make_float4(0.f, 0.f, 0.f, 0.f);
                yi[v][t] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    float w[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        w[s] = 0.f;
        if (s >= d) continue;
#pragma unroll
        for (int v = 0; v < G; ++v) {
            float4 zr = make_float4(0.f, 0.f, 0.f, 0.f), zi = zr;
#pragma unroll
            for (int t = 0; t < DMAX; ++t)
                if (t < d) cmac4(Drow[s * d + t], yr[v][t], yi[v][t], zr, zi);
            w[s] += zr.x * zr.x + zr.y * zr.y + zr.z * zr.z + zr.w * zr.w + zi.x * zi.x + zi.y * zi.y +
                    zi.z * zi.z + zi.w * zi.w;
        }
    }
    block_reduce_w<DMAX>(w, red, lane, warp, T >> 5);
    float wsel, Z32;
    const int sstar = displaced_draw<DMAX>(w, d, u, wsel, Z32);
    if (tid == 0) displaced_outputs<DMAX>(a, row, sstar, wsel, Z32, w);
    const float scale = wsel > 0.f && Z32 > 0.f && isfinite(Z32) ? rsqrtf(wsel) : 0.f;
    float2 c[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        const float2 e = t < d ? Drow[sstar * d + t] : make_float2(0.f, 0.f);
        c[t] = make_float2(e.x * scale, e.y * scale);
    }
    const int64_t grow = a.row0 + row;
#pragma unroll
    for (int v = 0; v < G; ++v) {
        const int g = tid + T * v;
        if (g >= ngroups) break;
        float4 zr = make_float4(0.f, 0.f, 0.f, 0.f), zi = zr;
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
            if (t < d) cmac4(c[t], yr[v][t], yi[v][t], zr, zi);
        store_next4(a, grow, 4 * g, zr);
        store_next4(a, grow, chi_r + 4 * g, zi);
    }
    for (int i = 2 * chi_r + 4 * tid; i < a.K_next; i += 4 * T)
        store_next4(a, grow, i, make_float4(0.f, 0.f, 0.f, 0.f));
}

// Narrow rows (d * chi_r <= 2048, chi_r a multiple of 4): one warp per row, the row's d blocks
// copied to shared memory with cp.async (16-byte chunks, all in flight at once) instead of registers,
// so that about 28 rows per SM are in flight (shared memory bounds it, not registers).
template <int DMAX>
__global__ void __launch_bounds__(32) measure_displaced_smem_kernel(const MeasureArgs a) {
    extern __shared__ __align__(16) float srow[];  // d blocks of [Re (chi_r) | Im (chi_r)]
    const int row = blockIdx.x, lane = threadIdx.x;
    const int d = a.d, chi_r = a.chi_r, nf2 = 2 * chi_r, ngroups = chi_r >> 2, dd = d * d;
    const int64_t Cs = a.Cs;
    const float *yrow = a.Y + (int64_t)row * a.ldY;
    {
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(srow);
        for (int t = 0; t < d; ++t)
            for (int i = lane * 4; i < nf2; i += 128)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 4u * (uint32_t)(t * nf2 + i)),
                             "l"(yrow + t * Cs + i)
                             : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const float2 *Drow = a.disp_D + (int64_t)row * dd;
    const double u = a.disp_u[row];
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    const float4 *s4 = reinterpret_cast<const float4 *>(srow);
    const int q = nf2 >> 2;  // float4 per block
    float w[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        w[s] = 0.f;
        if (s >= d) continue;
        float2 c[DMAX];
#pragma unroll
        for (int t = 0; t < DMAX; ++t) c[t] = t < d ? Drow[s * d + t] : make_float2(0.f, 0.f);
        for (int g = lane; g < ngroups; g += 32) {
            float4 zr = make_float4(0.f, 0.f, 0.f, 0.f), zi = zr;
#pragma unroll
            for (int t = 0; t < DMAX; ++t)
                if (t < d) cmac4(c[t], s4[t * q + g], s4[t * q + ngroups + g], zr, zi);
            w[s] += zr.x * zr.x + zr.y * zr.y + zr.z * zr.z + zr.w * zr.w + zi.x * zi.x + zi.y * zi.y +
                    zi.z * zi.z + zi.w * zi.w;
        }
    }
    block_reduce_w<DMAX>(w, nullptr, lane, 0, 1);
    float wsel, Z32;
    const int sstar = displaced_draw<DMAX>(w, d, u, wsel, Z32);
    if (lane == 0) displaced_outputs<DMAX>(a, row, sstar, wsel, Z32, w);
    const float scale = wsel > 0.f && Z32 > 0.f && isfinite(Z32) ? rsqrtf(wsel) : 0.f;
    float2 c[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        const float2 e = t < d ? Drow[sstar * d + t] : make_float2(0.f, 0.f);
        c[t] = make_float2(e.x * scale, e.y * scale);
    }
    const int64_t grow = a.row0 + row;
    for (int g = lane; g < ngroups; g += 32) {
        float4 zr = make_float4(0.f, 0.f, 0.f, 0.f), zi = zr;
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
            if (t < d) cmac4(c[t], s4[t * q + g], s4[t * q + ngroups + g], zr, zi);
        store_next4(a, grow, 4 * g, zr);
        store_next4(a, grow, chi_r + 4 * g, zi);
    }
    for (int i = 2 * chi_r + 4 * lane; i < a.K_next; i += 128)
        store_next4(a, grow, i, make_float4(0.f, 0.f, 0.f, 0.f));
}

template <int DMAX>
bool launch_smem_variant(const MeasureArgs &a, cudaStream_t st) {
    if constexpr (DMAX > 8) {
        return false;
    } else {
        if ((a.chi_r & 3) || (a.K_next & 3) || (a.ld_next & 3) || a.d * a.chi_r > 2048) return false;
        const size_t smem = (size_t)a.d * 2 * a.chi_r * sizeof(float);
        measure_displaced_smem_kernel<DMAX><<<(unsigned)a.rows, 32, smem, st>>>(a);
        return true;
    }
}

template <int DMAX>
bool launch_vec4_variant(const MeasureArgs &a, cudaStream_t st) {
    if constexpr (DMAX > 8) {
        return false;
    } else {
        if ((a.chi_r & 3) || (a.K_next & 3) || (a.ld_next & 3)) return false;
        const int ngroups = a.chi_r >> 2;
        // one warp per row when G groups per thread cover the row, else up to 256 threads
        for (int cap : {32, 128, 256}) {
            for (int G : {1, 2}) {
                if (G * DMAX > 8) break;
                const int need = (ngroups + G - 1) / G;
                if (need > cap) continue;
                const int T = std::max(32, (need + 31) / 32 * 32);
                const dim3 grid((unsigned)a.rows);
                if (G == 1) measure_displaced_vec4_kernel<DMAX, 1><<<grid, T, 0, st>>>(a);
                else if constexpr (2 * DMAX <= 8) measure_displaced_vec4_kernel<DMAX, 2><<<grid, T, 0, st>>>(a);
                return true;
            }
        }
        return false;
    }
}

// Scalar variant: the fewest columns per thread (VPT in {1, 2, 4, 8}) that cover chi_r with at most
// 128 threads (else 256), under a register cap of VPT * DMAX <= 32 complex values; false if none fits.
template <int DMAX>
bool launch_rows_variant(const MeasureArgs &a, cudaStream_t st) {
    const int chi_r = a.chi_r;
    for (int cap : {128, 256}) {
        for (int vpt : {1, 2, 4, 8}) {
            if (vpt * DMAX > 32) break;
            const int need = (chi_r + vpt - 1) / vpt;
            if (need > cap) continue;
            const int T = std::max(32, (need + 31) / 32 * 32);
            const dim3 grid((unsigned)a.rows);
            switch (vpt) {
                case 1: measure_displaced_rows_kernel<DMAX, 1><<<grid, T, 0, st>>>(a); break;
                case 2: measure_displaced_rows_kernel<DMAX, 2><<<grid, T, 0, st>>>(a); break;
                case 4:
                    if constexpr (4 * DMAX <= 32) measure_displaced_rows_kernel<DMAX, 4><<<grid, T, 0, st>>>(a);
                    break;
                default:
                    if constexpr (8 * DMAX <= 32) measure_displaced_rows_kernel<DMAX, 8><<<grid, T, 0, st>>>(a);
                    break;
            }
            return true;
        }
    }
    return false;
}

template <int DMAX>
void launch_displaced_variant(const MeasureArgs &a, cudaStream_t st) {
    if (launch_smem_variant<DMAX>(a, st)) return;
    if (launch_vec4_variant<DMAX>(a, st)) return;
    if (launch_rows_variant<DMAX>(a, st)) return;
    const int grid = (a.rows + DISP_WARPS - 1) / DISP_WARPS;
    measure_displaced_kernel<DMAX><<<grid, DISP_WARPS * 32, 0, st>>>(a);
}

void launch_measure_displaced(const MeasureArgs &a, int num_sms, cudaStream_t st) {
    (void)num_sms;
    if (a.rows <= 0) return;
    const unsigned pg = (unsigned)((a.rows + 255) / 256);
    if (a.d <= 4) displaced_prep_kernel<4><<<pg, 256, 0, st>>>(a);
    else if (a.d <= 8) displaced_prep_kernel<8><<<pg, 256, 0, st>>>(a);
    else displaced_prep_kernel<kMaxDisplacedD><<<pg, 256, 0, st>>>(a);
    if (a.d <= 4) launch_displaced_variant<4>(a, st);
    else if (a.d <= 8) launch_displaced_variant<8>(a, st);
    else launch_displaced_variant<kMaxDisplacedD>(a, st);
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
