// Handle state and host helpers shared by the library's host translation units (internal; not
// part of the ABI): the handle (struct fastmps_ctx) with its grow-only work buffers and loaded site
// tensors, error reporting, the precision plans and site layouts, tensor-map encoding and the host
// 16-bit conversions.  runtime.cu defines the helpers, loader.cu the site loader and the autotuner,
// engine.cu the per-call sampling engine, api.cu the C entry points.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/fastmps.h"
#include "common.cuh"
#include "launch.h"

namespace fastmps {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver (nullptr if the driver does not export it).
EncodeTiledFn get_encode_fn();

inline int64_t roundup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Host-side fault injection for tests: FASTMPS_FAIL_ALLOC_AFTER=n makes the
// (n+1)-th and later device allocations of work buffers report failure.
bool injected_alloc_failure();

// A device or pinned-host buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool host = false;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (host) cudaFreeHost(p);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    bool ensure(size_t want) {
        if (want <= bytes) return true;
        release();
        if (want == 0) return true;
        if (!host && injected_alloc_failure()) return false;
        cudaError_t e = host ? cudaHostAlloc(&p, want, cudaHostAllocDefault) : cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        bytes = want;
        return true;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

struct Tensor {
    SiteLayout L;
    int measure_mode = 0;  // autotuned: 2 = single-pass cluster kernel for this site, 0 = two-pass
    // resident operands (device)
    DevBuf B_hi, B_lo, Bt, B8;
    float fp8_scale = 1.f;  // FP8: stored value = e4m3(A * fp8_scale); FP16: fp16(A * fp8_scale)
    CUtensorMap tmB[2];
    // streamed operand (pinned host, compact BF16 [chi_l][d][chi_r] (re, im), hi block then lo block)
    DevBuf host_compact;
    int planes = 1;
};

}  // namespace fastmps

struct fastmps_ctx {
    int device = 0;
    fastmps_options opt{};
    cudaStream_t stream = nullptr, copy_stream = nullptr, measure_stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string last_error;
    std::map<int, std::unique_ptr<fastmps::Tensor>> site_tensor;  // private tensor of site k
    std::map<int, std::unique_ptr<fastmps::Tensor>> pool_tensor;  // pool entry j
    std::map<int, int> site_pool;                        // site k -> pool entry j
    // work buffers (grow only)
    fastmps::DevBuf V[2][3];  // [ping-pong][plane]  BF16 planes, or V[x][0] FP32
    fastmps::DevBuf Y[2], P[2], logp, O, Dout, Dlogp, trace, trace_slot, err;
    fastmps::DevBuf staging;  // device copy of a tensor being loaded
    fastmps::DevBuf lam;      // device copy of the Schmidt coefficients of a Vidal-form site being loaded
    fastmps::DevBuf mu;       // device copy of host displacement amplitudes (displaced sampling)
    fastmps::DevBuf disp_io;  // device staging of fastmps_displacement's host inputs / outputs
    fastmps::DevBuf trunc;    // device gather of the leading block of a truncated Vidal-form site
    fastmps::DevBuf disp_tab; // constants of the displacement entries for dimension disp_tab_d
    fastmps::DevBuf disp_D, disp_u;  // per-row matrices and uniforms of one displaced micro-batch
    int disp_tab_d = 0;
    std::vector<float> disp_tab_host;
    fastmps::DevBuf slot_compact[2], slot_hi, slot_lo;  // streaming slots
    cudaEvent_t copy_done[2] = {nullptr, nullptr}, slot_free[2] = {nullptr, nullptr};
    cudaEvent_t contract_done[2] = {nullptr, nullptr}, measure_done[2] = {nullptr, nullptr};
    fastmps_stats stats{};
    std::vector<cudaEvent_t> ev_pool;
};

namespace fastmps {

// Records msg as the handle's last error (if h) and returns code.
int fail(fastmps_handle h, int code, const std::string &msg);
// A failed CUDA call: FASTMPS_ERR_OOM for allocation failures, FASTMPS_ERR_CUDA otherwise.
int cuda_fail(fastmps_handle h, cudaError_t e, const char *what);

// Tensor-core precision modes (BF16 split planes or FP8); FP32 is the SIMT path.
inline bool is_bf16(const fastmps_handle h) { return h->opt.precision != FASTMPS_FP32; }
inline bool is_fp8(const fastmps_handle h) { return h->opt.precision == FASTMPS_FP8X1 || h->opt.precision == FASTMPS_FP8X2; }
inline bool is_f16(const fastmps_handle h) {
    return h->opt.precision == FASTMPS_FP16X2 || h->opt.precision == FASTMPS_FP16X3;
}

// Planes of the split-precision operands and the products accumulated per precision mode.
struct PrecisionPlan {
    int a_planes, b_planes, nprod;
    int pa[kMaxProducts], pb[kMaxProducts];
};

PrecisionPlan plan_of(int precision);

// bn_override > 0 (tensor-core modes): n-tile width chosen by the autotuner.
SiteLayout make_layout(int precision, int chi_l, int d, int chi_r, int bn_override = 0);

// 2-D tensor maps with the 128-byte swizzle: [outer][ld_elems] arrays, (box_inner x box_outer) boxes.
bool encode_2d(CUtensorMap *map, CUtensorMapDataType type, int elem_bytes, const void *base, uint64_t inner,
               uint64_t outer, uint64_t ld_elems, uint32_t box_inner, uint32_t box_outer);
bool encode_2d_bf16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                    uint32_t box_inner, uint32_t box_outer);
// FP32 contraction scratch [rows][ld] (TMA-store epilogue): 32 x 128 boxes, 128-byte swizzle
bool encode_2d_f32_scratch(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint64_t ld_elems);
bool encode_2d_f16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                   uint32_t box_inner, uint32_t box_outer);
// FP8 operands: rows of ld_elems bytes, 128-byte (128-element) boxes along K
bool encode_2d_u8(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                  uint32_t box_outer);

// Host round-to-nearest-even float -> bfloat16 bits (finite inputs).
inline uint16_t host_bf16_bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}
// Host float -> binary16 bits, round to nearest, ties to even (finite inputs below 65520 in
// magnitude): 11 significant bits for normals (exponent >= -14), multiples of 2^-24 below.
inline uint16_t host_f16_bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    const uint32_t sign = (u >> 16) & 0x8000u;
    const uint32_t a = u & 0x7FFFFFFFu;
    if (a >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u);  // 65520 and above round past 65504
    if (a <= 0x33000000u) return (uint16_t)sign;              // at most 2^-25: zero (a tie goes to even 0)
    const int e = (int)(a >> 23) - 127;
    const uint32_t mant = (a & 0x7FFFFFu) | 0x800000u;        // 24 significant bits
    const uint32_t shift = e >= -14 ? 13u : (uint32_t)(13 + (-14 - e));
    if (shift > 24) return (uint16_t)sign;
    const uint32_t rem = mant & ((1u << shift) - 1u), half = 1u << (shift - 1u);
    uint32_t m = mant >> shift;
    if (rem > half || (rem == half && (m & 1u))) m += 1u;
    if (e < -14) return (uint16_t)(sign | m);                  // subnormal (m = 0x400 is the least normal)
    uint32_t he = (uint32_t)(e + 15);
    if (m == 0x800u) {                                         // carry into the exponent
        m = 0x400u;
        he += 1u;
    }
    return (uint16_t)(sign | (he << 10) | (m & 0x3FFu));
}

// binary16 bits -> float (exact; finite inputs)
inline float host_f16_float(uint16_t b) {
    const int e = (b >> 10) & 0x1F;
    const float m = (float)(b & 0x3FF);
    const float v = e == 0 ? std::ldexp(m, -24) : std::ldexp(1024.f + m, e - 25);
    return (b & 0x8000u) ? -v : v;
}

inline float host_bf16_float(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Shape rules of a site tensor (fastmps_load_site and its variants).
int check_shape_args(fastmps_handle h, int chi_l, int d, int chi_r, const void *A, int dtype);
// Device (or managed) memory according to cudaPointerGetAttributes.
bool is_device_ptr(const void *p);

// ---- loader.cu ----
// Copy and repack one tensor into t.  lam (nullable, host or device, chi_r entries of the
// tensor's real type): Vidal form, the stored tensor is A[a][s][b] * lam[b].
int load_tensor(fastmps_handle h, Tensor &t, int chi_l, int d, int chi_r, const void *A, int dtype,
                const void *lam = nullptr);
// The tensor site k uses (its own or its pool entry), or nullptr.
Tensor *site_tensor_of(fastmps_handle h, int k);

// ---- engine.cu ----
// Device table of the displacement constants for dimension d (built and uploaded once per d).
const float *displacement_table(fastmps_handle h, int d);
// One sampling call (fastmps_sample_ex / _traced / _displaced).
// mu_dev (nullable, device): displaced sampling, amplitude of call row i at site k at mu_dev[k * ld_mu + i].
// trace_list (nullable, host): the trace_rows call rows to trace, in place of rows 0 .. trace_rows-1.
int run_sample(fastmps_handle h, int M, int d, const int *bonds, int64_t n0, int64_t N, uint64_t seed, uint32_t job,
               uint8_t *out_samples, double *out_logprob, int64_t trace_rows, double *trace_probs,
               const float2 *mu_dev = nullptr, int64_t ld_mu = 0, const int64_t *trace_list = nullptr);

}  // namespace fastmps
