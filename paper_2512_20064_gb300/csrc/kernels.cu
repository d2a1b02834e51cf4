// Site-tensor repacking, FP32 SIMT contraction, measurement (Algorithm 2) and
// output transposition kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "launch.h"
#include "measure.cuh"

namespace fastmps {

// ---------------------------------------------------------------------------
// Stacked real operand of the complex contraction.
//
// With v = vr + i vi and A = Ar + i Ai, y = v A has
//   Re y =  vr Ar - vi Ai,   Im y = vr Ai + vi Ar,
// so with the left row [vr | vi] (length 2 chi_l) the output column
// (s, p = 0, b) takes the operand column [Ar[:, s, b] ; -Ai[:, s, b]] and the
// column (s, p = 1, b) takes [Ai[:, s, b] ; Ar[:, s, b]].  That is four real
// products per complex multiply-add, 8 chi_l d chi_r flops per sample.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float load_part(const void *src, int is_f64, int64_t cidx, int part) {
    if (is_f64) return (float)(static_cast<const double *>(src)[2 * cidx + part]);
    return static_cast<const float *>(src)[2 * cidx + part];
}

// Returns the operand value at output column c and reduction index kappa and
// sets *zero when the position is padding.  (re_part, sign) say which part of
// A[a, s, b] it is: value = sign * (re_part ? Re : Im) A[a, s, b].
struct StackedPos {
    int64_t cidx;  // complex index a*d*chi_r + s*chi_r + b
    int re_part;   // 1: real part, 0: imaginary part
    float sign;
    bool zero;
};

__device__ __forceinline__ StackedPos stacked_pos(int c, int kappa, int chi_l, int d, int chi_r, int Cs) {
    StackedPos q;
    const int s = c / Cs;
    const int r = c - s * Cs;
    q.zero = (r >= 2 * chi_r) || (kappa >= 2 * chi_l) || (s >= d);
    if (q.zero) {
        q.cidx = 0;
        q.re_part = 1;
        q.sign = 0.f;
        return q;
    }
    const int p = r >= chi_r;
    const int b = r - p * chi_r;
    const int second = kappa >= chi_l;
    const int a = second ? kappa - chi_l : kappa;
    q.cidx = ((int64_t)a * d + s) * chi_r + b;
    if (p == 0) {  // real output column: [Ar ; -Ai]
        q.re_part = second ? 0 : 1;
        q.sign = second ? -1.f : 1.f;
    } else {       // imaginary output column: [Ai ; Ar]
        q.re_part = second ? 1 : 0;
        q.sign = 1.f;
    }
    return q;
}

__global__ void repack_bf16_kernel(const void *__restrict__ src, int is_f64, int chi_l, int d, int chi_r, int Cs,
                                   int ncols, int K_pad, __nv_bfloat16 *__restrict__ B_hi,
                                   __nv_bfloat16 *__restrict__ B_lo) {
    const int64_t total = (int64_t)ncols * K_pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / K_pad);
        const int kappa = (int)(i - (int64_t)c * K_pad);
        const StackedPos q = stacked_pos(c, kappa, chi_l, d, chi_r, Cs);
        float x = 0.f;
        if (!q.zero) x = q.sign * load_part(src, is_f64, q.cidx, q.re_part ? 0 : 1);
        __nv_bfloat16 hi, lo;
        split_bf16(x, hi, lo);
        B_hi[i] = hi;
        if (B_lo) B_lo[i] = lo;
    }
}

__global__ void expand_bf16_kernel(const __nv_bfloat16 *__restrict__ compact, int planes, int chi_l, int d,
                                   int chi_r, int Cs, int ncols, int K_pad, __nv_bfloat16 *__restrict__ B_hi,
                                   __nv_bfloat16 *__restrict__ B_lo) {
    const int64_t total = (int64_t)ncols * K_pad;
    const int64_t plane = (int64_t)chi_l * d * chi_r * 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / K_pad);
        const int kappa = (int)(i - (int64_t)c * K_pad);
        const StackedPos q = stacked_pos(c, kappa, chi_l, d, chi_r, Cs);
        __nv_bfloat16 hi = __float2bfloat16_rn(0.f), lo = hi;
        if (!q.zero) {
            const int64_t e = 2 * q.cidx + (q.re_part ? 0 : 1);
            // 16-bit values moved as bits (BF16 or FP16 planes); negation flips the sign bit of either format
            hi = compact[e];
            if (q.sign < 0.f) hi = __ushort_as_bfloat16((unsigned short)(__bfloat16_as_ushort(hi) ^ 0x8000u));
            if (planes > 1) {
                lo = compact[plane + e];
                if (q.sign < 0.f) lo = __ushort_as_bfloat16((unsigned short)(__bfloat16_as_ushort(lo) ^ 0x8000u));
            }
        }
        B_hi[i] = hi;
        if (B_lo) B_lo[i] = lo;
    }
}

__global__ void repack_f32_kernel(const void *__restrict__ src, int is_f64, int chi_l, int d, int chi_r, int Cs,
                                  int ncols, int K_pad, float *__restrict__ Bt) {
    const int64_t total = (int64_t)ncols * K_pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kappa = (int)(i / ncols);
        const int c = (int)(i - (int64_t)kappa * ncols);
        const StackedPos q = stacked_pos(c, kappa, chi_l, d, chi_r, Cs);
        float x = 0.f;
        if (!q.zero) x = q.sign * load_part(src, is_f64, q.cidx, q.re_part ? 0 : 1);
        Bt[i] = x;
    }
}

__global__ void repack_e4m3_kernel(const void *__restrict__ src, int is_f64, int chi_l, int d, int chi_r, int Cs,
                                   int ncols, int K_pad, float scale, uint8_t *__restrict__ B8) {
    const int64_t total = (int64_t)ncols * K_pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / K_pad);
        const int kappa = (int)(i - (int64_t)c * K_pad);
        const StackedPos q = stacked_pos(c, kappa, chi_l, d, chi_r, Cs);
        float x = 0.f;
        if (!q.zero) x = q.sign * load_part(src, is_f64, q.cidx, q.re_part ? 0 : 1);
        B8[i] = (uint8_t)__nv_cvt_float_to_fp8(x * scale, __NV_SATFINITE, __NV_E4M3);
    }
}

__global__ void repack_f16_kernel(const void *__restrict__ src, int is_f64, int chi_l, int d, int chi_r, int Cs,
                                  int ncols, int K_pad, float scale, uint16_t *__restrict__ B16,
                                  uint16_t *__restrict__ B16_lo) {
    const int64_t total = (int64_t)ncols * K_pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / K_pad);
        const int kappa = (int)(i - (int64_t)c * K_pad);
        const StackedPos q = stacked_pos(c, kappa, chi_l, d, chi_r, Cs);
        float x = 0.f;
        if (!q.zero) x = q.sign * load_part(src, is_f64, q.cidx, q.re_part ? 0 : 1);
        const float xs = x * scale;  // exact: a power-of-two scale
        const __half hi = __float2half_rn(xs);
        B16[i] = __half_as_ushort(hi);
        if (B16_lo) B16_lo[i] = __half_as_ushort(__float2half_rn(xs - __half2float(hi)));  // the residual is exact
    }
}

// max over |Re|, |Im| (as float) of n complex entries; non-negative floats order like their bit patterns
__global__ void absmax_kernel(const void *__restrict__ src, int is_f64, int64_t n2, float *out) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = is_f64 ? (float)static_cast<const double *>(src)[i] : static_cast<const float *>(src)[i];
        m = fmaxf(m, fabsf(x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int *>(out), __float_as_uint(m));
}

static int grid_for(int64_t total, int block) {
    int64_t g = (total + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

void launch_repack_bf16(const void *src, int is_f64, const SiteLayout &L, __nv_bfloat16 *B_hi, __nv_bfloat16 *B_lo,
                        cudaStream_t st) {
    const int64_t total = (int64_t)L.ncols * L.K_pad;
    repack_bf16_kernel<<<grid_for(total, 256), 256, 0, st>>>(src, is_f64, L.chi_l, L.d, L.chi_r, L.Cs, L.ncols,
                                                              L.K_pad, B_hi, B_lo);
}

void launch_expand_bf16(const __nv_bfloat16 *compact, int planes, const SiteLayout &L, __nv_bfloat16 *B_hi,
                        __nv_bfloat16 *B_lo, cudaStream_t st) {
    const int64_t total = (int64_t)L.ncols * L.K_pad;
    expand_bf16_kernel<<<grid_for(total, 256), 256, 0, st>>>(compact, planes, L.chi_l, L.d, L.chi_r, L.Cs, L.ncols,
                                                              L.K_pad, B_hi, B_lo);
}

void launch_repack_e4m3(const void *src, int is_f64, const SiteLayout &L, float scale, uint8_t *B8,
                        cudaStream_t st) {
    const int64_t total = (int64_t)L.ncols * L.K_pad;
    repack_e4m3_kernel<<<grid_for(total, 256), 256, 0, st>>>(src, is_f64, L.chi_l, L.d, L.chi_r, L.Cs, L.ncols,
                                                              L.K_pad, scale, B8);
}

void launch_repack_f16(const void *src, int is_f64, const SiteLayout &L, float scale, uint16_t *B16,
                       uint16_t *B16_lo, cudaStream_t st) {
    const int64_t total = (int64_t)L.ncols * L.K_pad;
    repack_f16_kernel<<<grid_for(total, 256), 256, 0, st>>>(src, is_f64, L.chi_l, L.d, L.chi_r, L.Cs, L.ncols,
                                                             L.K_pad, scale, B16, B16_lo);
}

void launch_absmax(const void *src, int is_f64, int64_t n_complex, float *out_dev, cudaStream_t st) {
    cudaMemsetAsync(out_dev, 0, sizeof(float), st);
    absmax_kernel<<<grid_for(2 * n_complex, 256), 256, 0, st>>>(src, is_f64, 2 * n_complex, out_dev);
}

void launch_repack_f32(const void *src, int is_f64, const SiteLayout &L, float *Bt, cudaStream_t st) {
    const int64_t total = (int64_t)L.ncols * L.K_pad;
    repack_f32_kernel<<<grid_for(total, 256), 256, 0, st>>>(src, is_f64, L.chi_l, L.d, L.chi_r, L.Cs, L.ncols,
                                                             L.K_pad, Bt);
}

// ---------------------------------------------------------------------------
// Left boundary v_0 = [1]: row = [1, 0, ..., 0] (real part 1, imaginary 0).
// ---------------------------------------------------------------------------
__global__ void init_left_bf16_kernel(__nv_bfloat16 *V0, __nv_bfloat16 *V1, __nv_bfloat16 *V2, int64_t rows,
                                      int ld) {
    const int64_t total = rows * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const bool one = (i % ld) == 0;
        V0[i] = __float2bfloat16_rn(one ? 1.f : 0.f);
        V1[i] = __float2bfloat16_rn(0.f);
        if (V2) V2[i] = __float2bfloat16_rn(0.f);
    }
}

__global__ void init_left_f32_kernel(float *V, int64_t rows, int ld) {
    const int64_t total = rows * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        V[i] = (i % ld) == 0 ? 1.f : 0.f;
}

__global__ void init_left_e4m3_kernel(uint8_t *V8, int64_t rows, int ld) {
    const int64_t total = rows * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        V8[i] = (uint8_t)__nv_cvt_float_to_fp8((i % ld) == 0 ? 1.f : 0.f, __NV_SATFINITE, __NV_E4M3);
}

__global__ void init_left_f16_kernel(uint16_t *V0, uint16_t *V1, int64_t rows, int ld) {
    const int64_t total = rows * ld;
    const uint16_t one = __half_as_ushort(__float2half_rn(1.f)), zero = __half_as_ushort(__float2half_rn(0.f));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        V0[i] = (i % ld) == 0 ? one : zero;
        V1[i] = zero;
    }
}

void launch_init_left_f16(uint16_t *V0, uint16_t *V1, int64_t rows, int ld, cudaStream_t st) {
    init_left_f16_kernel<<<grid_for(rows * ld, 256), 256, 0, st>>>(V0, V1, rows, ld);
}

void launch_init_left_e4m3(uint8_t *V8, int64_t rows, int ld, cudaStream_t st) {
    init_left_e4m3_kernel<<<grid_for(rows * ld, 256), 256, 0, st>>>(V8, rows, ld);
}

void launch_init_left_bf16(__nv_bfloat16 *const *Vp, int nplanes, int64_t rows, int ld, cudaStream_t st) {
    init_left_bf16_kernel<<<grid_for(rows * ld, 256), 256, 0, st>>>(Vp[0], Vp[1], nplanes > 2 ? Vp[2] : nullptr,
                                                                      rows, ld);
}

void launch_init_left_f32(float *V, int64_t rows, int ld, cudaStream_t st) {
    init_left_f32_kernel<<<grid_for(rows * ld, 256), 256, 0, st>>>(V, rows, ld);
}

// ---------------------------------------------------------------------------
// FP32 SIMT contraction (the plain path): Y = V Bt over a 128 x 128 tile per
// block, 8 x 8 outputs per thread, K staged 8 at a time in double-buffered
// shared memory.  Epilogue: store the tile to the FP32 scratch and one sum of
// squares per row (the tile lies inside one outcome block s).
//
// Chunked accumulation: each output sums its K = 2 chi_l products in chunks
// of F32_CHUNK, every chunk in its own FP32 accumulator that is then added to
// a running FP32 total.  One sequential FP32 sum over K = 2048 has a rounding
// error ~ sqrt(K) units in the last place of the result, and because the
// left vector's direction error is carried, not forgotten, along a chain of
// random isometries, those errors add up over the sites and surface in the
// last sites' conditionals; chunks of 64 cut the per-site error about five
// times (2.3e-5 -> 4.7e-6 at M = 1024, chi = 1024 in a CPU emulation of both
// orders), at the cost of a second register tile.
// ---------------------------------------------------------------------------
constexpr int F32_BM = 128, F32_BN = 128, F32_BK = 8, F32_THREADS = 256;
constexpr int F32_CHUNK = 64;  // K entries per partial accumulator (a multiple of F32_BK)

__global__ void __launch_bounds__(F32_THREADS, 1)
contract_f32_kernel(const float *__restrict__ V, int64_t ldV, int64_t row0, const float *__restrict__ Bt, int ldB,
                    int K, float *__restrict__ Y, int64_t ldY, float *__restrict__ P, int ldP, int rows_valid) {
    __shared__ __align__(16) float As[2][F32_BK][F32_BM];
    __shared__ __align__(16) float Bs[2][F32_BK][F32_BN];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * F32_BM;
    const int n0 = blockIdx.x * F32_BN;
    const float *Ag = V + (row0 + m0) * ldV;
    const int a_row = tid >> 1, a_k = (tid & 1) * 4;
    const int b_k = tid >> 5, b_n = (tid & 31) * 4;

    float4 ra = *reinterpret_cast<const float4 *>(Ag + (int64_t)a_row * ldV + a_k);
    float4 rb = *reinterpret_cast<const float4 *>(Bt + (int64_t)b_k * ldB + n0 + b_n);
    As[0][a_k + 0][a_row] = ra.x;
    As[0][a_k + 1][a_row] = ra.y;
    As[0][a_k + 2][a_row] = ra.z;
    As[0][a_k + 3][a_row] = ra.w;
    *reinterpret_cast<float4 *>(&Bs[0][b_k][b_n]) = rb;
    __syncthreads();

    const int ty = tid >> 4, tx = tid & 15;
    float acc[8][8], tot[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            acc[i][j] = 0.f;
            tot[i][j] = 0.f;
        }

    const int nk = K / F32_BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) {
            const int k0 = (kt + 1) * F32_BK;
            ra = *reinterpret_cast<const float4 *>(Ag + (int64_t)a_row * ldV + k0 + a_k);
            rb = *reinterpret_cast<const float4 *>(Bt + (int64_t)(k0 + b_k) * ldB + n0 + b_n);
        }
#pragma unroll
        for (int kk = 0; kk < F32_BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if ((kt + 1) % (F32_CHUNK / F32_BK) == 0 || kt + 1 == nk) {
            // end of a K chunk: fold its partial sums into the running totals
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    tot[i][j] += acc[i][j];
                    acc[i][j] = 0.f;
                }
        }
        if (kt + 1 < nk) {
            const int nxt = cur ^ 1;
            As[nxt][a_k + 0][a_row] = ra.x;
            As[nxt][a_k + 1][a_row] = ra.y;
            As[nxt][a_k + 2][a_row] = ra.z;
            As[nxt][a_k + 3][a_row] = ra.w;
            *reinterpret_cast<float4 *>(&Bs[nxt][b_k][b_n]) = rb;
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        float ss = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) ss = fmaf(tot[i][j], tot[i][j], ss);
        ss += __shfl_xor_sync(0xffffffffu, ss, 1);
        ss += __shfl_xor_sync(0xffffffffu, ss, 2);
        ss += __shfl_xor_sync(0xffffffffu, ss, 4);
        ss += __shfl_xor_sync(0xffffffffu, ss, 8);
        if (r < rows_valid) {
            float *yr = Y + (int64_t)r * ldY + n0;
            *reinterpret_cast<float4 *>(yr + tx * 4) = make_float4(tot[i][0], tot[i][1], tot[i][2], tot[i][3]);
            *reinterpret_cast<float4 *>(yr + 64 + tx * 4) = make_float4(tot[i][4], tot[i][5], tot[i][6], tot[i][7]);
            if (tx == 0) P[(int64_t)r * ldP + blockIdx.x] = ss;
        }
    }
}

void launch_contract_f32(const float *V, int64_t ldV, int64_t row0, int64_t rows_pad, const float *Bt,
                         const SiteLayout &L, const ContractOut &o, cudaStream_t st) {
    dim3 grid(L.ncols / F32_BN, (unsigned)(rows_pad / F32_BM));
    contract_f32_kernel<<<grid, F32_THREADS, 0, st>>>(V, ldV, row0, Bt, L.ncols, L.K_pad, o.Y, o.ldY, o.P, o.ldP,
                                                       o.rows_valid);
}

constexpr int MEASURE_THREADS = 128;
constexpr int MEASURE_WARPS = MEASURE_THREADS / 32;

// Stand-alone measurement (FP32 path, and BF16 paths when not fused): a warp
// handles 32 samples, one per lane for the draw, then the warp writes each
// sample's next left row with coalesced loads.
__global__ void __launch_bounds__(MEASURE_THREADS) measure_kernel(const MeasureArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int base = (blockIdx.x * MEASURE_WARPS + warp) * 32;
    if (base >= a.rows) return;
    const int row = base + lane;
    int sstar = 0;
    float scale = 0.f;
    if (row < a.rows) sstar = measure_draw(a, row, &scale);
    const int count = min(32, a.rows - base);
    for (int j = 0; j < count; ++j) {
        const int sj = __shfl_sync(0xffffffffu, sstar, j);
        const float scj = __shfl_sync(0xffffffffu, scale, j);
        const int r = base + j;
        const float *ysrc = a.Y + (int64_t)r * a.ldY + (int64_t)sj * a.Cs;
        measure_write_row(a, lane, ysrc, scj, a.row0 + r);
    }
}

void launch_measure(const MeasureArgs &a, cudaStream_t st) {
    if (a.rows <= 0) return;
    const int rows_per_block = MEASURE_WARPS * 32;
    const int grid = (a.rows + rows_per_block - 1) / rows_per_block;
    measure_kernel<<<grid, MEASURE_THREADS, 0, st>>>(a);
}

// ---------------------------------------------------------------------------
// Outcomes are produced site-major (coalesced writes per site); the caller
// wants sample-major rows.  32 x 32 byte tiles through shared memory.
// ---------------------------------------------------------------------------
__global__ void transpose_u8_kernel(const uint8_t *__restrict__ O, int64_t ldO, int64_t N, int M,
                                    uint8_t *__restrict__ out) {
    __shared__ uint8_t t[32][33];
    const int64_t n0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int k = k0 + j;
        const int64_t n = n0 + threadIdx.x;
        if (k < M && n < N) t[j][threadIdx.x] = O[(int64_t)k * ldO + n];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t n = n0 + j;
        const int k = k0 + threadIdx.x;
        if (k < M && n < N) out[n * M + k] = t[threadIdx.x][j];
    }
}

void launch_transpose_outcomes(const uint8_t *O, int64_t ldO, int64_t N, int M, uint8_t *out, cudaStream_t st) {
    if (N <= 0 || M <= 0) return;
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32));
    transpose_u8_kernel<<<grid, dim3(32, 8), 0, st>>>(O, ldO, N, M, out);
}

}  // namespace fastmps

namespace fastmps {

// Self-test of the bounded wait used by the pipelined kernels: waits on an
// mbarrier that nothing ever arrives on; the wait gives up after limit_ns and
// the kernel records kDevTimeoutProducer and returns (no fault, no hang).
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int *status, unsigned long long *waited_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = global_ns();
        const bool ok = mbar_wait_bounded(&bar, 0u, &abort_flag, limit_ns);
        *waited_ns = global_ns() - t0;
        *status = ok ? kDevOk : kDevTimeoutProducer;
    }
}

void launch_bounded_wait_selftest(uint64_t limit_ns, int *status, unsigned long long *waited_ns, cudaStream_t st) {
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, status, waited_ns);
}

}  // namespace fastmps
