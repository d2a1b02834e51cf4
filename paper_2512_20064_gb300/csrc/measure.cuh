// Measurement step shared by the stand-alone measurement kernel and the
// measurement warps fused into the tcgen05 contraction (device code, internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "common.cuh"
#include "launch.h"

namespace fastmps {

// ---------------------------------------------------------------------------
// Measurement (Algorithm 2 with the exact per-sample rescaling of Sec. 3.3.1).
// Phase 1, one thread per sample (measure_draw):
//  * w_s = sum of the FP32 per-tile sums of squares of outcome block s,
//    accumulated in FP64;
//  * C_s = w_0 + ... + w_s in s order (FP64), Z = C_{d-1}, Philox uniform u,
//    s* = #{s < d-1 : C_s < u Z}: the decision is taken in FP64 as in the
//    oracle;
//  * log p accumulates log(w_{s*} / Z) in FP64: the ratio and its logarithm
//    are taken in FP64 (one log per sample per site, O(N M) work), since a
//    rare outcome has w_{s*} << 1 and the absolute error of an FP32 log
//    there would add up over thousands of sites.
// Phase 2, a warp per sample (measure_write_row): the selected block y_{s*} is scaled
// by 1/sqrt(w_{s*}) (FP32; the scale cancels in every later ratio w/Z) and
// written as the next left row -- FP32, or BF16 planes of successive
// residuals -- with coalesced 16-byte loads.
// GB300's FP64 pipes are narrow, so FP64 is kept to the O(d) per-sample
// operations of the draw and the accumulation, one sample per lane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_planes(float x, int nplanes, __nv_bfloat16 &h0, __nv_bfloat16 &h1,
                                             __nv_bfloat16 &h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    h2 = __float2bfloat16_rn(r1 - __bfloat162float(h1));
    if (nplanes < 3) h2 = __float2bfloat16_rn(0.f);
}

__device__ __forceinline__ void measure_write_row(const MeasureArgs &a, int lane, const float *ysrc, float scale,
                                                  int64_t grow) {
    const int nreal = 2 * a.chi_r;
    if (a.V32) {
        float *dst = a.V32 + grow * a.ld_next;
        if ((nreal & 3) == 0) {
            constexpr int U = 4;
            for (int base = 4 * lane; base < a.K_next; base += 128 * U) {
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = base + 128 * u;
                    v[u] = i < nreal ? __ldcg(reinterpret_cast<const float4 *>(ysrc + i))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = base + 128 * u;
                    if (i >= a.K_next) break;
                    *reinterpret_cast<float4 *>(dst + i) =
                        make_float4(v[u].x * scale, v[u].y * scale, v[u].z * scale, v[u].w * scale);
                }
            }
        } else {
            for (int i = lane; i < a.K_next; i += 32) dst[i] = i < nreal ? ysrc[i] * scale : 0.f;
        }
        return;
    }
    if (a.f16) {
        // FP16 row: scale the unit-norm row by the power of two that puts its largest entry in
        // [16384, 32768] (the scale cancels in w/Z at the next site; small entries stay normal), then
        // two binary16 planes of successive residuals, each rounded to nearest even
        float m = 0.f;
        for (int i = lane; i < nreal; i += 32) m = fmaxf(m, fabsf(__ldcg(ysrc + i) * scale));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float s16 = m > 0.f ? exp2f(floorf(log2f(32768.f / m))) : 1.f;
        uint16_t *d0 = reinterpret_cast<uint16_t *>(a.Vp[0]) + grow * a.ld_next;
        uint16_t *d1 = reinterpret_cast<uint16_t *>(a.Vp[1]) + grow * a.ld_next;
        for (int i = lane; i < a.K_next; i += 32) {
            const float x = i < nreal ? (__ldcg(ysrc + i) * scale) * s16 : 0.f;
            const __half h = __float2half_rn(x);
            d0[i] = __half_as_ushort(h);
            d1[i] = __half_as_ushort(__float2half_rn(x - __half2float(h)));
        }
        return;
    }
    if (a.V8) {
        // E4M3 row: scale the unit-norm row by the power of two that puts its largest entry in
        // [224, 448] (the scale cancels in w/Z at the next site), then round to nearest even
        float m = 0.f;
        for (int i = lane; i < nreal; i += 32) m = fmaxf(m, fabsf(__ldcg(ysrc + i) * scale));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float s8 = m > 0.f ? exp2f(floorf(log2f(448.f / m))) : 1.f;
        uint8_t *dst = a.V8 + grow * a.ld_next;
        uint8_t *dlo = a.V8lo ? a.V8lo + grow * a.ld_next : nullptr;
        for (int i = lane; i < a.K_next; i += 32) {
            const float x = i < nreal ? __ldcg(ysrc + i) * scale * s8 : 0.f;
            const __nv_fp8_storage_t h = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
            dst[i] = (uint8_t)h;
            if (dlo) {
                // residual at the same scale: the two planes' products add up to (V0 + V1) B
                const float hv = __half2float(__half(__nv_cvt_fp8_to_halfraw(h, __NV_E4M3)));
                dlo[i] = (uint8_t)__nv_cvt_float_to_fp8(x - hv, __NV_SATFINITE, __NV_E4M3);
            }
        }
        return;
    }
    __nv_bfloat16 *d0 = a.Vp[0] + grow * a.ld_next;
    __nv_bfloat16 *d1 = a.Vp[1] + grow * a.ld_next;
    __nv_bfloat16 *d2 = a.nplanes > 2 ? a.Vp[2] + grow * a.ld_next : nullptr;
    if ((nreal & 3) == 0) {
        // four 16-byte loads in flight per lane before any store
        constexpr int U = 4;
        for (int base = 4 * lane; base < a.K_next; base += 128 * U) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = base + 128 * u;
                v[u] = i < nreal ? __ldcg(reinterpret_cast<const float4 *>(ysrc + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = base + 128 * u;
                if (i >= a.K_next) break;
                const float x[4] = {v[u].x * scale, v[u].y * scale, v[u].z * scale, v[u].w * scale};
                __align__(8) __nv_bfloat16 p0[4], p1[4], p2[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) write_planes(x[e], a.nplanes, p0[e], p1[e], p2[e]);
                *reinterpret_cast<uint2 *>(d0 + i) = *reinterpret_cast<const uint2 *>(p0);
                *reinterpret_cast<uint2 *>(d1 + i) = *reinterpret_cast<const uint2 *>(p1);
                if (d2) *reinterpret_cast<uint2 *>(d2 + i) = *reinterpret_cast<const uint2 *>(p2);
            }
        }
    } else {
        for (int i = lane; i < a.K_next; i += 32) {
            const float x = i < nreal ? ysrc[i] * scale : 0.f;
            __nv_bfloat16 h0, h1, h2;
            write_planes(x, a.nplanes, h0, h1, h2);
            d0[i] = h0;
            d1[i] = h1;
            if (d2) d2[i] = h2;
        }
    }
}

// Phase 1 for sample `row` of the micro-batch (row < a.rows): draw, outcome,
// log-probability, optional trace.  Returns the outcome and sets *scale to
// 1/sqrt(w_{s*}).  P is read through L2 (it may have been written by other
// thread blocks of the same kernel).
__device__ __forceinline__ int measure_draw(const MeasureArgs &a, int row, float *scale_out) {
    int sstar = 0;
    float scale = 0.f;
    {
        const float *Prow = a.P + (int64_t)row * a.ldP;
        const int T = a.tiles_per_s;
        // pass 1: Z = w_0 + ... + w_{d-1} in s order
        double Z = 0.0;
        for (int s = 0; s < a.d; ++s) {
            double acc = 0.0;
            for (int j = 0; j < T; ++j) acc += (double)__ldcg(Prow + s * T + j);
            Z += acc;
        }
        const uint64_t n = a.n_base + (uint64_t)row;
        const double t = sample_uniform(a.seed, n, a.k, a.job) * Z;
        // pass 2: the same partial sums again; s* is the first s < d-1 with C_s >= t (else d-1),
        // which equals #{s < d-1 : C_s < t} because C is non-decreasing
        double C = 0.0, ws = 0.0;
        sstar = a.d - 1;
        for (int s = 0; s < a.d; ++s) {
            double acc = 0.0;
            for (int j = 0; j < T; ++j) acc += (double)__ldcg(Prow + s * T + j);
            C += acc;
            if (s == a.d - 1 || C >= t) {
                sstar = s;
                ws = acc;
                break;
            }
        }
        const bool ok = (Z > 0.0) && isfinite(Z) && (ws > 0.0);
        const int64_t grow = a.row0 + row;
        a.outcomes[row] = (uint8_t)sstar;
        if (ok) a.logp[grow] += log(ws / Z);
        else atomicExch(a.err, (int)kDevNumeric);
        const int64_t slot = a.trace ? (a.trace_slot ? (int64_t)a.trace_slot[grow] : (grow < a.trace_rows ? grow : -1))
                                     : -1;
        if (slot >= 0) {
            for (int s = 0; s < a.d; ++s) {
                double acc = 0.0;
                for (int j = 0; j < T; ++j) acc += (double)__ldcg(Prow + s * T + j);
                a.trace[slot * a.d + s] = ok ? acc / Z : 0.0;
            }
        }
        scale = ok ? rsqrtf((float)ws) : 0.f;
    }
    *scale_out = scale;
    return sstar;
}

}  // namespace fastmps
