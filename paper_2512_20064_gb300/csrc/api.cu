// C ABI and host engine of the sampling library (see include/fastmps.h).
//
// Engine per call (Sec. 3.1 data-parallel scheme on one device): all N rows
// of the left operand stay resident in device memory (the macro-batch);
// for each site k the rows are processed in micro-batches: one contraction
// launch writes the FP32 scratch Y and per-tile sums of squares, one
// measurement launch draws the outcome and writes the next left operand.  In
// host-streaming residency the BF16 site tensor of site k+1 is copied from
// pinned host memory into one of two device slots on a copy stream while site
// k computes (Sec. 3.1 double buffer; Sec. 3.3.2 16-bit storage).
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

using namespace fastmps;

namespace fastmps {
void batch_release(fastmps_handle h);
}

namespace {

std::string g_create_error;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

inline int64_t roundup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Error {
    int code;
    std::string msg;
};

// Host-side fault injection for tests: FASTMPS_FAIL_ALLOC_AFTER=n makes the
// (n+1)-th and later device allocations of work buffers report failure.
long long g_alloc_budget = -2;  // -2: not read yet, -1: no injection
bool injected_alloc_failure() {
    if (g_alloc_budget == -2) {
        const char *v = getenv("FASTMPS_FAIL_ALLOC_AFTER");
        g_alloc_budget = v ? atoll(v) : -1;
    }
    if (g_alloc_budget < 0) return false;
    if (g_alloc_budget == 0) return true;
    --g_alloc_budget;
    return false;
}

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

}  // namespace

struct fastmps_ctx {
    int device = 0;
    fastmps_options opt{};
    cudaStream_t stream = nullptr, copy_stream = nullptr, measure_stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string last_error;
    std::map<int, std::unique_ptr<Tensor>> site_tensor;  // private tensor of site k
    std::map<int, std::unique_ptr<Tensor>> pool_tensor;  // pool entry j
    std::map<int, int> site_pool;                        // site k -> pool entry j
    // work buffers (grow only)
    DevBuf V[2][3];  // [ping-pong][plane]  BF16 planes, or V[x][0] FP32
    DevBuf Y[2], P[2], logp, O, Dout, Dlogp, trace, trace_slot, err;
    DevBuf staging;  // device copy of a tensor being loaded
    DevBuf lam;      // device copy of the Schmidt coefficients of a Vidal-form site being loaded
    DevBuf mu;       // device copy of host displacement amplitudes (displaced sampling)
    DevBuf disp_io;  // device staging of fastmps_displacement's host inputs / outputs
    DevBuf trunc;    // device gather of the leading block of a truncated Vidal-form site
    DevBuf disp_tab; // constants of the displacement entries for dimension disp_tab_d
    DevBuf disp_D, disp_u;  // per-row matrices and uniforms of one displaced micro-batch
    int disp_tab_d = 0;
    std::vector<float> disp_tab_host;
    DevBuf slot_compact[2], slot_hi, slot_lo;  // streaming slots
    cudaEvent_t copy_done[2] = {nullptr, nullptr}, slot_free[2] = {nullptr, nullptr};
    cudaEvent_t contract_done[2] = {nullptr, nullptr}, measure_done[2] = {nullptr, nullptr};
    fastmps_stats stats{};
    std::vector<cudaEvent_t> ev_pool;
};

namespace {

int fail(fastmps_handle h, int code, const std::string &msg) {
    if (h) h->last_error = msg;
    return code;
}

int cuda_fail(fastmps_handle h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? FASTMPS_ERR_OOM : FASTMPS_ERR_CUDA, m);
}

// Tensor-core precision modes (BF16 split planes or FP8); FP32 is the SIMT path.
bool is_bf16(const fastmps_handle h) { return h->opt.precision != FASTMPS_FP32; }
bool is_fp8(const fastmps_handle h) { return h->opt.precision == FASTMPS_FP8X1 || h->opt.precision == FASTMPS_FP8X2; }
bool is_f16(const fastmps_handle h) {
    return h->opt.precision == FASTMPS_FP16X2 || h->opt.precision == FASTMPS_FP16X3;
}

// Planes of the split-precision operands and the products accumulated per precision mode.
struct PrecisionPlan {
    int a_planes, b_planes, nprod;
    int pa[kMaxProducts], pb[kMaxProducts];
};

PrecisionPlan plan_of(int precision) {
    switch (precision) {
        case FASTMPS_BF16X2: return {2, 1, 2, {0, 1, 0, 0}, {0, 0, 0, 0}};
        case FASTMPS_BF16X3: return {2, 2, 3, {0, 1, 0, 0}, {0, 0, 1, 0}};
        case FASTMPS_BF16X3L: return {3, 1, 3, {0, 1, 2, 0}, {0, 0, 0, 0}};
        case FASTMPS_BF16X4: return {3, 2, 4, {0, 1, 2, 0}, {0, 0, 0, 1}};
        case FASTMPS_FP8X1: return {1, 1, 1, {0, 0, 0, 0}, {0, 0, 0, 0}};
        case FASTMPS_FP8X2: return {2, 1, 2, {0, 1, 0, 0}, {0, 0, 0, 0}};
        case FASTMPS_FP16X2: return {2, 1, 2, {0, 1, 0, 0}, {0, 0, 0, 0}};
        case FASTMPS_FP16X3: return {2, 2, 3, {0, 1, 0, 0}, {0, 0, 1, 0}};
        default: return {1, 1, 1, {0, 0, 0, 0}, {0, 0, 0, 0}};
    }
}

// bn_override > 0 (tensor-core modes): n-tile width chosen by the autotuner.
SiteLayout make_layout(int precision, int chi_l, int d, int chi_r, int bn_override = 0) {
    SiteLayout L;
    L.chi_l = chi_l;
    L.d = d;
    L.chi_r = chi_r;
    L.bk = (precision == FASTMPS_FP8X1 || precision == FASTMPS_FP8X2) ? 128 : 64;
    L.K_pad = (int)roundup(2 * (int64_t)chi_l, L.bk);
    if (precision == FASTMPS_FP32) {
        L.bn = 128;
    } else {
        L.bn = (int)std::min<int64_t>(256, roundup(2 * (int64_t)chi_r, 32));
        if (bn_override > 0 && bn_override < L.bn) L.bn = bn_override;
    }
    L.Cs = (int)roundup(2 * (int64_t)chi_r, L.bn);
    L.ncols = d * L.Cs;
    L.tiles_per_s = L.Cs / L.bn;
    return L;
}

bool encode_2d(CUtensorMap *map, CUtensorMapDataType type, int elem_bytes, const void *base, uint64_t inner,
               uint64_t outer, uint64_t ld_elems, uint32_t box_inner, uint32_t box_outer) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    cuuint64_t gdim[2] = {inner, outer};
    cuuint64_t gstride[1] = {ld_elems * (uint64_t)elem_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, type, 2, const_cast<void *>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_2d_bf16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                    uint32_t box_inner, uint32_t box_outer) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, inner, outer, ld_elems, box_inner, box_outer);
}

// FP32 contraction scratch [rows][ld] (TMA-store epilogue): 32 x 128 boxes, 128-byte swizzle
bool encode_2d_f32_scratch(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint64_t ld_elems) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, cols, rows, ld_elems, 32, 128);
}

bool encode_2d_f16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                   uint32_t box_inner, uint32_t box_outer) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, inner, outer, ld_elems, box_inner, box_outer);
}

// FP8 operands: rows of ld_elems bytes, 128-byte (128-element) boxes along K
bool encode_2d_u8(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                  uint32_t box_outer) {
    return encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, base, inner, outer, ld_elems, 128, box_outer);
}

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

int check_shape_args(fastmps_handle h, int chi_l, int d, int chi_r, const void *A, int dtype) {
    if (!A) return fail(h, FASTMPS_ERR_INVALID_ARG, "tensor pointer is NULL");
    if (dtype != FASTMPS_C64 && dtype != FASTMPS_C128) return fail(h, FASTMPS_ERR_INVALID_ARG, "unknown dtype");
    if (chi_l < 1 || chi_r < 1 || d < 2 || d > 255)
        return fail(h, FASTMPS_ERR_SHAPE, "need chi_l >= 1, chi_r >= 1, 2 <= d <= 255");
    if ((int64_t)d * chi_r < chi_l) return fail(h, FASTMPS_ERR_SHAPE, "d * chi_r < chi_l: not an isometry shape");
    if ((int64_t)chi_l > (1 << 20) || (int64_t)chi_r > (1 << 20))
        return fail(h, FASTMPS_ERR_SHAPE, "bond dimension above 2^20");
    return FASTMPS_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// Autotuner: n-tile width and measurement mode per site shape.
// Candidates are the two-pass path (contraction + measurement kernel) with
// 256, 128 and 64 columns per n-tile (those not wider than the padded block
// 2 chi_r), and the single-pass cluster kernel where the site's row fits one
// cluster; each is timed on a probe of 8192 rows (contraction and
// measurement of one site), best of three.  The pipeline depth is not a
// candidate: with one thread block per SM the deepest ring that fits shared
// memory never loses.  Results are cached per process and, when
// FASTMPS_TUNE_CACHE names a file, in that file as a flat JSON object
// {"precision:chi_l:d:chi_r": bn + 10000 * mode, ...} (mode 2: cluster).
// ---------------------------------------------------------------------------
std::mutex g_tune_mutex;
std::map<std::string, int> g_tuned;
bool g_tune_loaded = false;

std::string tune_key(int precision, int chi_l, int d, int chi_r) {
    return std::to_string(precision) + ":" + std::to_string(chi_l) + ":" + std::to_string(d) + ":" +
           std::to_string(chi_r);
}

void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("FASTMPS_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    fclose(f);
    size_t i = 0;
    while ((i = text.find('"', i)) != std::string::npos) {
        const size_t j = text.find('"', i + 1);
        if (j == std::string::npos) break;
        const size_t c = text.find(':', j);
        if (c == std::string::npos) break;
        g_tuned[text.substr(i + 1, j - i - 1)] = atoi(text.c_str() + c + 1);
        i = j + 1;
    }
}

void tune_cache_store() {
    const char *path = getenv("FASTMPS_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fputc('{', f);
    bool first = true;
    for (auto &kv : g_tuned) {
        fprintf(f, "%s\"%s\": %d", first ? "" : ", ", kv.first.c_str(), kv.second);
        first = false;
    }
    fputs("}\n", f);
    fclose(f);
}

// Times the candidates on the staged tensor; returns bn + 10000 * mode of the fastest.
int autotune_bn(fastmps_handle h, int chi_l, int d, int chi_r, int is_f64) {
    const PrecisionPlan plan = plan_of(h->opt.precision);
    const int widest = (int)std::min<int64_t>(256, roundup(2 * (int64_t)chi_r, 32));
    const int64_t rows = 8192;
    int best = widest;
    float best_ms = 1e30f;
    const int K_next = (int)roundup(2 * (int64_t)chi_r, 64);
    DevBuf Vn[3], O, logp, err;
    bool ok = O.ensure((size_t)rows) && logp.ensure((size_t)rows * 8) && err.ensure(sizeof(int));
    for (int p = 0; p < plan.a_planes; ++p) ok = ok && Vn[p].ensure((size_t)rows * K_next * 2);
    if (!ok) return best;
    for (int cand = 0; cand < 4; ++cand) {
        const bool cluster = cand == 3;
        const int bn = cluster ? widest : (cand == 0 ? 256 : cand == 1 ? 128 : 64);
        if (bn > widest) continue;
        SiteLayout L = make_layout(h->opt.precision, chi_l, d, chi_r, bn);
        int cC = 0, cT = 0;
        if (cluster && !(cluster_plan(L, &cC, &cT) && cluster_capacity(plan.a_planes, plan.b_planes, L) > 0))
            continue;
        DevBuf B[2], V[3], Y, P;
        for (int p = 0; p < plan.b_planes; ++p) ok = ok && B[p].ensure((size_t)L.ncols * L.K_pad * 2);
        for (int p = 0; p < plan.a_planes; ++p) ok = ok && V[p].ensure((size_t)rows * L.K_pad * 2);
        if (!cluster)
            ok = ok && Y.ensure((size_t)rows * L.ncols * 4) && P.ensure((size_t)rows * (L.ncols / L.bn) * 4);
        if (!ok) break;
        launch_repack_bf16(h->staging.p, is_f64, L, B[0].as<__nv_bfloat16>(),
                           plan.b_planes > 1 ? B[1].as<__nv_bfloat16>() : nullptr, h->stream);
        __nv_bfloat16 *Vp[3] = {nullptr, nullptr, nullptr};
        for (int p = 0; p < plan.a_planes; ++p) Vp[p] = V[p].as<__nv_bfloat16>();
        launch_init_left_bf16(Vp, plan.a_planes, rows, L.K_pad, h->stream);  // every row the vector [1, 0, ...]
        cudaMemsetAsync(err.p, 0, sizeof(int), h->stream);
        TcArgs ta;
        ta.a_planes = plan.a_planes;
        ta.b_planes = plan.b_planes;
        ta.nprod = plan.nprod;
        for (int q = 0; q < kMaxProducts; ++q) {
            ta.prod_a[q] = plan.pa[q];
            ta.prod_b[q] = plan.pb[q];
        }
        for (int p = 0; p < 3; ++p)
            ok = ok && encode_2d_bf16(&ta.tmA[p], V[p < plan.a_planes ? p : 0].p, L.K_pad, rows, L.K_pad, 64, 128);
        for (int p = 0; p < 2; ++p)
            ok = ok && encode_2d_bf16(&ta.tmB[p], B[p < plan.b_planes ? p : 0].p, L.K_pad, L.ncols, L.K_pad, 64, L.bn);
        if (!ok) break;
        ta.row0 = 0;
        ta.rows_pad = (int)rows;
        ContractOut co{Y.as<float>(), L.ncols, P.as<float>(), L.ncols / L.bn, (int)rows};
        ta.has_tmY = !cluster && encode_2d_f32_scratch(&ta.tmY, Y.p, L.ncols, rows, L.ncols);
        MeasureArgs ma{};
        ma.Y = co.Y;
        ma.ldY = co.ldY;
        ma.P = co.P;
        ma.ldP = co.ldP;
        ma.d = d;
        ma.chi_r = chi_r;
        ma.Cs = L.Cs;
        ma.tiles_per_s = L.tiles_per_s;
        ma.rows = (int)rows;
        ma.seed = 1;
        ma.ld_next = K_next;
        ma.K_next = K_next;
        for (int p = 0; p < plan.a_planes; ++p) ma.Vp[p] = Vn[p].as<__nv_bfloat16>();
        ma.nplanes = plan.a_planes;
        ma.outcomes = O.as<uint8_t>();
        ma.logp = logp.as<double>();
        ma.err = err.as<int>();
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, h->stream);
            if (cluster) {
                launch_contract_tc_cluster(ta, L, (int)rows, err.as<int>(), h->stream, ma);
            } else {
                launch_contract_tc(ta, L, co, h->num_sms, err.as<int>(), h->stream);
                launch_measure(ma, h->stream);
            }
            cudaEventRecord(e1, h->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = bn + (cluster ? 20000 : 0);
        }
    }
    return best;
}

// Copy and repack one tensor into t.  lam (nullable, host or device, chi_r entries of the
// tensor's real type): Vidal form, the stored tensor is A[a][s][b] * lam[b].
int load_tensor(fastmps_handle h, Tensor &t, int chi_l, int d, int chi_r, const void *A, int dtype,
                const void *lam = nullptr) {
    int rc = check_shape_args(h, chi_l, d, chi_r, A, dtype);
    if (rc) return rc;
    const size_t lam_bytes = (size_t)chi_r * (dtype == FASTMPS_C128 ? 8 : 4);
    t.L = make_layout(h->opt.precision, chi_l, d, chi_r);
    const int64_t nelem = (int64_t)chi_l * d * chi_r;
    const bool tune = h->opt.autotune && is_bf16(h) && !is_fp8(h) && !is_f16(h) && h->opt.accum_chunk == 0 &&
                      h->opt.residency == FASTMPS_RESIDENT_HBM;
    const size_t src_bytes = (size_t)nelem * (dtype == FASTMPS_C128 ? 16 : 8);
    cudaError_t e;
    const bool a_on_device = is_device_ptr(A);
    std::vector<uint8_t> host_copy;
    if (a_on_device && h->opt.residency == FASTMPS_HOST_STREAM) {
        host_copy.resize(src_bytes);
        e = cudaMemcpy(host_copy.data(), A, src_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of site tensor");
        A = host_copy.data();
    }
    std::vector<uint8_t> lam_host;
    if (lam && h->opt.residency == FASTMPS_HOST_STREAM) {
        lam_host.resize(lam_bytes);
        e = cudaMemcpy(lam_host.data(), lam, lam_bytes, is_device_ptr(lam) ? cudaMemcpyDeviceToHost
                                                                             : cudaMemcpyHostToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of Schmidt coefficients");
    }
    if (h->opt.residency == FASTMPS_HOST_STREAM) {
        // compact BF16 copy in pinned host memory
        t.planes = plan_of(h->opt.precision).b_planes;
        t.host_compact.host = true;
        if (!t.host_compact.ensure((size_t)nelem * 2 * 2 * t.planes))
            return fail(h, FASTMPS_ERR_OOM, "pinned host allocation for a streamed tensor failed");
        uint16_t *dst = t.host_compact.as<uint16_t>();
        const int64_t n2 = nelem * 2;
        auto value = [&](int64_t i) -> float {
            if (dtype == FASTMPS_C128) {
                double v = static_cast<const double *>(A)[i];
                if (lam) v *= reinterpret_cast<const double *>(lam_host.data())[(i >> 1) % chi_r];
                return (float)v;
            }
            float x = static_cast<const float *>(A)[i];
            if (lam) x *= reinterpret_cast<const float *>(lam_host.data())[(i >> 1) % chi_r];
            return x;
        };
        if (is_f16(h)) {
            // binary16 at the per-site power-of-two scale that puts the largest |Re|, |Im| in [16384, 32768]
            float amax = 0.f;
            for (int64_t i = 0; i < n2; ++i) amax = std::max(amax, std::fabs(value(i)));
            t.fp8_scale = amax > 0.f ? (float)std::exp2(std::floor(std::log2(32768.0 / (double)amax))) : 1.f;
            for (int64_t i = 0; i < n2; ++i) {
                const float x = value(i) * t.fp8_scale;  // exact: a power-of-two scale
                const uint16_t hb = host_f16_bits(x);
                dst[i] = hb;
                if (t.planes > 1) dst[n2 + i] = host_f16_bits(x - host_f16_float(hb));
            }
            return FASTMPS_OK;
        }
        for (int64_t i = 0; i < n2; ++i) {
            const float x = value(i);
            uint16_t hb = host_bf16_bits(x);
            dst[i] = hb;
            if (t.planes > 1) dst[n2 + i] = host_bf16_bits(x - host_bf16_float(hb));
        }
        return FASTMPS_OK;
    }
    if (!h->staging.ensure(src_bytes)) return fail(h, FASTMPS_ERR_OOM, "staging allocation failed");
    e = cudaMemcpyAsync(h->staging.p, A, src_bytes, a_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy of site tensor");
    if (lam) {
        if (!h->lam.ensure(lam_bytes)) return fail(h, FASTMPS_ERR_OOM, "allocation failed");
        e = cudaMemcpyAsync(h->lam.p, lam, lam_bytes, is_device_ptr(lam) ? cudaMemcpyDeviceToDevice
                                                                          : cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of Schmidt coefficients");
        launch_scale_columns(h->staging.p, dtype == FASTMPS_C128, nelem, chi_r, h->lam.p, h->stream);
    }
    const size_t op_elems = (size_t)t.L.ncols * t.L.K_pad;
    if (is_fp8(h)) {
        // per-site power-of-two scale that puts the largest |Re|, |Im| in [224, 448]
        if (!t.B8.ensure(op_elems) || !h->err.ensure(256)) return fail(h, FASTMPS_ERR_OOM, "allocation failed");
        float amax = 0.f;
        launch_absmax(h->staging.p, dtype == FASTMPS_C128, nelem, h->err.as<float>(), h->stream);
        e = cudaMemcpyAsync(&amax, h->err.p, sizeof(float), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "site tensor maximum");
        t.fp8_scale = amax > 0.f ? (float)std::exp2(std::floor(std::log2(448.0 / (double)amax))) : 1.f;
        launch_repack_e4m3(h->staging.p, dtype == FASTMPS_C128, t.L, t.fp8_scale, t.B8.as<uint8_t>(), h->stream);
        if (!encode_2d_u8(&t.tmB[0], t.B8.p, t.L.K_pad, t.L.ncols, t.L.K_pad, t.L.bn))
            return fail(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
        t.tmB[1] = t.tmB[0];
    } else if (is_f16(h)) {
        // per-site power-of-two scale that puts the largest |Re|, |Im| in [16384, 32768]
        const bool two = plan_of(h->opt.precision).b_planes > 1;
        if (!t.B_hi.ensure(op_elems * 2) || (two && !t.B_lo.ensure(op_elems * 2)) || !h->err.ensure(256))
            return fail(h, FASTMPS_ERR_OOM, "allocation failed");
        float amax = 0.f;
        launch_absmax(h->staging.p, dtype == FASTMPS_C128, nelem, h->err.as<float>(), h->stream);
        e = cudaMemcpyAsync(&amax, h->err.p, sizeof(float), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "site tensor maximum");
        t.fp8_scale = amax > 0.f ? (float)std::exp2(std::floor(std::log2(32768.0 / (double)amax))) : 1.f;
        launch_repack_f16(h->staging.p, dtype == FASTMPS_C128, t.L, t.fp8_scale, t.B_hi.as<uint16_t>(),
                          two ? t.B_lo.as<uint16_t>() : nullptr, h->stream);
        if (!encode_2d_f16(&t.tmB[0], t.B_hi.p, t.L.K_pad, t.L.ncols, t.L.K_pad, 64, t.L.bn) ||
            (two && !encode_2d_f16(&t.tmB[1], t.B_lo.p, t.L.K_pad, t.L.ncols, t.L.K_pad, 64, t.L.bn)))
            return fail(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
        if (!two) t.tmB[1] = t.tmB[0];
    } else if (is_bf16(h)) {
        if (tune) {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            tune_cache_load();
            const std::string key = tune_key(h->opt.precision, chi_l, d, chi_r);
            auto it = g_tuned.find(key);
            int code;
            if (it != g_tuned.end()) {
                code = it->second;
            } else {
                code = autotune_bn(h, chi_l, d, chi_r, dtype == FASTMPS_C128);
                g_tuned[key] = code;
                tune_cache_store();
            }
            t.L = make_layout(h->opt.precision, chi_l, d, chi_r, code % 10000);
            t.measure_mode = code / 10000;
        }
        const size_t op_elems = (size_t)t.L.ncols * t.L.K_pad;
        if (!t.B_hi.ensure(op_elems * 2)) return fail(h, FASTMPS_ERR_OOM, "site operand allocation failed");
        __nv_bfloat16 *lo = nullptr;
        if (plan_of(h->opt.precision).b_planes > 1) {
            if (!t.B_lo.ensure(op_elems * 2)) return fail(h, FASTMPS_ERR_OOM, "site operand allocation failed");
            lo = t.B_lo.as<__nv_bfloat16>();
        }
        launch_repack_bf16(h->staging.p, dtype == FASTMPS_C128, t.L, t.B_hi.as<__nv_bfloat16>(), lo, h->stream);
        if (!encode_2d_bf16(&t.tmB[0], t.B_hi.p, t.L.K_pad, t.L.ncols, t.L.K_pad, 64, t.L.bn))
            return fail(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
        if (lo && !encode_2d_bf16(&t.tmB[1], t.B_lo.p, t.L.K_pad, t.L.ncols, t.L.K_pad, 64, t.L.bn))
            return fail(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
        if (!lo) t.tmB[1] = t.tmB[0];
    } else {
        if (!t.Bt.ensure(op_elems * 4)) return fail(h, FASTMPS_ERR_OOM, "site operand allocation failed");
        launch_repack_f32(h->staging.p, dtype == FASTMPS_C128, t.L, t.Bt.as<float>(), h->stream);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "repack launch");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "repack");
    return FASTMPS_OK;
}

Tensor *site_tensor_of(fastmps_handle h, int k) {
    auto it = h->site_pool.find(k);
    if (it != h->site_pool.end()) {
        auto p = h->pool_tensor.find(it->second);
        return p == h->pool_tensor.end() ? nullptr : p->second.get();
    }
    auto s = h->site_tensor.find(k);
    return s == h->site_tensor.end() ? nullptr : s->second.get();
}

struct EventTimer {
    fastmps_handle h;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> contract, measure, copy;
    size_t used = 0;
    explicit EventTimer(fastmps_handle hh) : h(hh) {}
    cudaEvent_t get() {
        if (used == h->ev_pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            h->ev_pool.push_back(e);
        }
        return h->ev_pool[used++];
    }
    double total(const std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v) {
        double s = 0;
        for (auto &p : v) {
            float ms = 0;
            cudaEventElapsedTime(&ms, p.first, p.second);
            s += ms;
        }
        return s;
    }
};

// Device table of the displacement constants for dimension d (built and uploaded once per d).
const float *displacement_table(fastmps_handle h, int d) {
    if (h->disp_tab_d == d) return h->disp_tab.as<float>();
    const size_t n = (size_t)d * d * (2 * d + 1);
    h->disp_tab_host.assign(n, 0.f);
    build_displacement_table(d, h->disp_tab_host.data());
    if (!h->disp_tab.ensure(n * sizeof(float))) return nullptr;
    if (cudaMemcpyAsync(h->disp_tab.p, h->disp_tab_host.data(), n * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
        return nullptr;
    h->disp_tab_d = d;
    return h->disp_tab.as<float>();
}

// mu_dev (nullable, device): displaced sampling, amplitude of call row i at site k at mu_dev[k * ld_mu + i].
// trace_list (nullable, host): the trace_rows call rows to trace, in place of rows 0 .. trace_rows-1.
int run_sample(fastmps_handle h, int M, int d, const int *bonds, int64_t n0, int64_t N, uint64_t seed, uint32_t job,
               uint8_t *out_samples, double *out_logprob, int64_t trace_rows, double *trace_probs,
               const float2 *mu_dev = nullptr, int64_t ld_mu = 0, const int64_t *trace_list = nullptr) {
    auto t_start = std::chrono::steady_clock::now();
    h->stats = fastmps_stats{};
    if (M < 1 || !bonds || N < 0 || n0 < 0) return fail(h, FASTMPS_ERR_INVALID_ARG, "need M >= 1, bonds, N >= 0, n0 >= 0");
    if (d < 2 || d > 255) return fail(h, FASTMPS_ERR_SHAPE, "need 2 <= d <= 255");
    if (bonds[0] != 1 || bonds[M] != 1) return fail(h, FASTMPS_ERR_SHAPE, "bond_dims[0] and bond_dims[M] must be 1");
    if (trace_rows < 0 || (trace_rows > 0 && !trace_probs))
        return fail(h, FASTMPS_ERR_INVALID_ARG, "trace_rows > 0 needs trace_probs");
    std::vector<Tensor *> ts(M);
    std::vector<char> on_cluster(M, 0);  // single-pass cluster contraction + measurement at site k
    const bool want_cluster = h->opt.fused_measure == 2 && is_bf16(h) && !is_fp8(h) && !is_f16(h) && !mu_dev;
    int ldV = 64;
    int ncols_max = 0, ldP_max = 0;
    double flops = 0;
    for (int k = 0; k < M; ++k) {
        Tensor *t = site_tensor_of(h, k);
        if (!t) return fail(h, FASTMPS_ERR_NOT_LOADED, "site " + std::to_string(k) + " is not loaded");
        if (t->L.chi_l != bonds[k] || t->L.d != d || t->L.chi_r != bonds[k + 1])
            return fail(h, FASTMPS_ERR_SHAPE, "site " + std::to_string(k) + " was loaded with shape (" +
                                                  std::to_string(t->L.chi_l) + ", " + std::to_string(t->L.d) + ", " +
                                                  std::to_string(t->L.chi_r) + ") but bond_dims/d say (" +
                                                  std::to_string(bonds[k]) + ", " + std::to_string(d) + ", " +
                                                  std::to_string(bonds[k + 1]) + ")");
        ts[k] = t;
        ldV = std::max(ldV, t->L.K_pad);
        int cC = 0, cT = 0;
        on_cluster[k] = (want_cluster || (t->measure_mode == 2 && h->opt.fused_measure == 0 && is_bf16(h) &&
                                          !is_fp8(h) && !mu_dev)) &&
                        cluster_plan(t->L, &cC, &cT) &&
                        cluster_capacity(plan_of(h->opt.precision).a_planes, plan_of(h->opt.precision).b_planes,
                                         t->L) > 0;
        if (!on_cluster[k]) {
            ncols_max = std::max(ncols_max, t->L.ncols);
            ldP_max = std::max(ldP_max, t->L.ncols / t->L.bn);
        }
        flops += 8.0 * bonds[k] * d * bonds[k + 1];
    }
    const PrecisionPlan plan = plan_of(h->opt.precision);
    const int prods = plan.nprod;
    h->stats.flops_algorithmic = flops * (double)N;
    h->stats.flops_issued = flops * (double)N * prods;
    if (N == 0) return FASTMPS_OK;
    const bool stream_mode = h->opt.residency == FASTMPS_HOST_STREAM;
    const bool bf16 = is_bf16(h);
    cudaStream_t st = h->stream;
    cudaError_t e;

    // ---- plan ---------------------------------------------------------------
    const int64_t N_pad = roundup(N, 128);
    int64_t N2;
    if (ncols_max == 0) {
        // every site runs the single-pass cluster kernel: no scratch, all rows in one launch per site
        N2 = h->opt.max_microbatch > 0 ? std::max<int64_t>(128, h->opt.max_microbatch / 128 * 128) : N_pad;
    } else if (h->opt.max_microbatch > 0) {
        N2 = std::max<int64_t>(128, h->opt.max_microbatch / 128 * 128);
    } else {
        // FP32 scratch budget per micro-batch buffer; with several micro-batches per site the
        // measurement of one overlaps the contraction of the next
        const int64_t budget = (int64_t)2 << 30;
        N2 = std::max<int64_t>(128, budget / ((int64_t)ncols_max * 4) / 128 * 128);
        // the fused BF16 kernel gives each thread block whole m-tiles: use whole waves of
        // (128 rows x SMs) so that every block gets the same number of m-tiles
        const int64_t wave = (int64_t)128 * h->num_sms;
        if (bf16 && h->opt.fused_measure && !mu_dev && N2 >= wave && N_pad > N2) N2 = N2 / wave * wave;
        // the displaced measurement reads whole scratch rows and takes a large share of a site: with at
        // least two micro-batches it overlaps the next micro-batch's contraction on the second stream
        if (mu_dev && N2 >= N_pad && N_pad >= 2 * wave) N2 = roundup((N_pad + 1) / 2, 128);
    }
    N2 = std::min(N2, N_pad);
    const int64_t J = (N + N2 - 1) / N2;  // micro-batches per site

    // ---- buffers -------------------------------------------------------------
    const bool fp8 = is_fp8(h);
    const int planes = bf16 ? plan.a_planes : 1;
    const size_t elem = fp8 ? 1 : (bf16 ? 2 : 4);
    if (fp8) ldV = (int)roundup(ldV, 128);
    for (int x = 0; x < 2; ++x)
        for (int p = 0; p < planes; ++p)
            if (!h->V[x][p].ensure((size_t)N_pad * ldV * elem))
                return fail(h, FASTMPS_ERR_OOM, "left-operand allocation failed");
    // BF16 modes measure inside the contraction kernel (no second launch, one scratch buffer)
    const bool fused = bf16 && !fp8 && h->opt.fused_measure == 1 && !mu_dev;
    const int nybuf = (J > 1 && !fused) ? 2 : 1;

    if (ncols_max > 0)
        for (int b = 0; b < nybuf; ++b)
            if (!h->Y[b].ensure((size_t)N2 * ncols_max * 4) || !h->P[b].ensure((size_t)N2 * ldP_max * 4))
                return fail(h, FASTMPS_ERR_OOM, "scratch allocation failed");
    if (!h->logp.ensure((size_t)N_pad * 8) || !h->O.ensure((size_t)M * N_pad) || !h->err.ensure(sizeof(int)))
        return fail(h, FASTMPS_ERR_OOM, "work-buffer allocation failed");
    const bool samples_dev = is_device_ptr(out_samples);
    const bool logp_dev = is_device_ptr(out_logprob);
    const bool trace_dev = is_device_ptr(trace_probs);
    if (out_samples && !samples_dev && !h->Dout.ensure((size_t)N * M))
        return fail(h, FASTMPS_ERR_OOM, "output staging allocation failed");
    double *trace_buf = nullptr;
    const int *trace_slot = nullptr;
    if (trace_list && trace_rows > 0) {
        // per-row slot map of the listed rows (distinct, inside the call)
        std::vector<int> slot((size_t)N, -1);
        for (int64_t i = 0; i < trace_rows; ++i) {
            const int64_t r = trace_list[i];
            if (r < 0 || r >= N || slot[(size_t)r] >= 0)
                return fail(h, FASTMPS_ERR_INVALID_ARG, "trace rows must be distinct call rows in [0, N)");
            slot[(size_t)r] = (int)i;
        }
        if (!h->trace_slot.ensure((size_t)N * sizeof(int))) return fail(h, FASTMPS_ERR_OOM, "trace allocation failed");
        e = cudaMemcpyAsync(h->trace_slot.p, slot.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vector is released on return
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of the trace rows");
        trace_slot = h->trace_slot.as<int>();
    }
    if (trace_rows > 0) {
        if (!trace_list) trace_rows = std::min(trace_rows, N);
        if (trace_dev) trace_buf = trace_probs;
        else {
            if (!h->trace.ensure((size_t)M * trace_rows * d * 8)) return fail(h, FASTMPS_ERR_OOM, "trace allocation failed");
            trace_buf = h->trace.as<double>();
        }
    }
    if (stream_mode) {
        size_t cmax = 0, opmax = 0;
        for (int k = 0; k < M; ++k) {
            cmax = std::max(cmax, ts[k]->host_compact.bytes);
            opmax = std::max(opmax, (size_t)ts[k]->L.ncols * ts[k]->L.K_pad * 2);
        }
        if (!h->slot_compact[0].ensure(cmax) || !h->slot_compact[1].ensure(cmax) || !h->slot_hi.ensure(opmax) ||
            (plan.b_planes > 1 && !h->slot_lo.ensure(opmax)))
            return fail(h, FASTMPS_ERR_OOM, "streaming slot allocation failed");
    }

    const float *disp_tab = nullptr;
    if (mu_dev && (!(disp_tab = displacement_table(h, d)) || !h->disp_D.ensure((size_t)N2 * d * d * 8) ||
                   !h->disp_u.ensure((size_t)N2 * 8)))
        return fail(h, FASTMPS_ERR_OOM, "displacement buffers allocation failed");
    int *d_err = h->err.as<int>();
    e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    cudaMemsetAsync(h->logp.p, 0, (size_t)N_pad * 8, st);
    __nv_bfloat16 *Vp[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    for (int x = 0; x < 2; ++x)
        for (int p = 0; p < planes && bf16 && !fp8; ++p) Vp[x][p] = h->V[x][p].as<__nv_bfloat16>();
    if (fp8) {
        launch_init_left_e4m3(h->V[0][0].as<uint8_t>(), N_pad, ldV, st);
        if (planes > 1) cudaMemsetAsync(h->V[0][1].p, 0, (size_t)N_pad * ldV, st);  // residual plane of [1]
    } else if (is_f16(h))
        launch_init_left_f16(h->V[0][0].as<uint16_t>(), h->V[0][1].as<uint16_t>(), N_pad, ldV, st);
    else if (bf16)
        launch_init_left_bf16(Vp[0], planes, N_pad, ldV, st);
    else
        launch_init_left_f32(h->V[0][0].as<float>(), N_pad, ldV, st);
    h->stats.launches += 1;

    EventTimer timer(h);
    cudaStream_t ms = h->measure_stream;
    int64_t g = 0;  // micro-batch counter over the whole call
    int64_t last_measured = -1;  // micro-batch whose measurement ran last on the measurement stream
    // the measurement stream starts after everything queued so far on the compute stream
    {
        cudaEvent_t ev = timer.get();
        cudaEventRecord(ev, st);
        cudaStreamWaitEvent(ms, ev, 0);
    }

    // streaming: prefetch site 0
    auto issue_copy = [&](int k) -> cudaError_t {
        const int slot = k & 1;
        cudaError_t ee = cudaStreamWaitEvent(h->copy_stream, h->slot_free[slot], 0);
        if (ee != cudaSuccess) return ee;
        cudaEvent_t q0 = timer.get(), q1 = timer.get();
        cudaEventRecord(q0, h->copy_stream);
        ee = cudaMemcpyAsync(h->slot_compact[slot].p, ts[k]->host_compact.p, ts[k]->host_compact.bytes,
                             cudaMemcpyHostToDevice, h->copy_stream);
        if (ee != cudaSuccess) return ee;
        cudaEventRecord(q1, h->copy_stream);
        timer.copy.push_back({q0, q1});
        h->stats.h2d_bytes += (int64_t)ts[k]->host_compact.bytes;
        return cudaEventRecord(h->copy_done[slot], h->copy_stream);
    };
    if (stream_mode) {
        // the copy stream must not run ahead of work already queued on the compute stream
        cudaEvent_t ev0 = timer.get();
        cudaEventRecord(ev0, st);
        cudaStreamWaitEvent(h->copy_stream, ev0, 0);
        e = issue_copy(0);
        if (e != cudaSuccess) return cuda_fail(h, e, "site copy");
    }

    for (int k = 0; k < M; ++k) {
        Tensor *t = ts[k];
        const SiteLayout &L = t->L;
        const int cur = k & 1, nxt = cur ^ 1;
        const int K_next = k + 1 < M ? ts[k + 1]->L.K_pad : 64;
        TcArgs ta;
        if (bf16) {
            const __nv_bfloat16 *Bh = t->B_hi.as<__nv_bfloat16>();
            const __nv_bfloat16 *Bl = t->B_lo.as<__nv_bfloat16>();
            if (stream_mode) {
                if (k + 1 < M) {
                    e = issue_copy(k + 1);
                    if (e != cudaSuccess) return cuda_fail(h, e, "site copy");
                }
                cudaStreamWaitEvent(st, h->copy_done[cur], 0);
                __nv_bfloat16 *lo = plan.b_planes > 1 ? h->slot_lo.as<__nv_bfloat16>() : nullptr;
                launch_expand_bf16(h->slot_compact[cur].as<__nv_bfloat16>(), t->planes, L,
                                   h->slot_hi.as<__nv_bfloat16>(), lo, st);
                h->stats.launches += 1;
                cudaEventRecord(h->slot_free[cur], st);
                Bh = h->slot_hi.as<__nv_bfloat16>();
                Bl = lo;
                auto map16 = [&](CUtensorMap *m, const void *base) {
                    return is_f16(h) ? encode_2d_f16(m, base, L.K_pad, L.ncols, L.K_pad, 64, L.bn)
                                     : encode_2d_bf16(m, base, L.K_pad, L.ncols, L.K_pad, 64, L.bn);
                };
                if (!map16(&ta.tmB[0], Bh) || (Bl && !map16(&ta.tmB[1], Bl)))
                    return fail(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
                if (!Bl) ta.tmB[1] = ta.tmB[0];
            } else {
                ta.tmB[0] = t->tmB[0];
                ta.tmB[1] = t->tmB[1];
            }
            ta.a_planes = plan.a_planes;
            ta.b_planes = plan.b_planes;
            ta.nprod = plan.nprod;
            for (int q = 0; q < kMaxProducts; ++q) {
                ta.prod_a[q] = plan.pa[q];
                ta.prod_b[q] = plan.pb[q];
            }
            ta.fp8 = fp8;
            ta.f16 = is_f16(h);
            for (int p = 0; p < 3; ++p) {
                const int src = p < plan.a_planes ? p : 0;
                const bool ok = fp8 ? encode_2d_u8(&ta.tmA[p], h->V[cur][src].p, L.K_pad, N_pad, ldV, 128)
                                : ta.f16 ? encode_2d_f16(&ta.tmA[p], h->V[cur][src].p, L.K_pad, N_pad, ldV, 64, 128)
                                         : encode_2d_bf16(&ta.tmA[p], h->V[cur][src].p, L.K_pad, N_pad, ldV, 64, 128);
                if (!ok) return fail(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
            }
        }
        for (int64_t r0 = 0; r0 < N; r0 += N2, ++g) {
            const int64_t rows = std::min<int64_t>(N2, N - r0);
            const int64_t rows_pad = roundup(rows, 128);
            const int yb = (int)(g % nybuf);
            if (on_cluster[k]) {
                // the rows come from the last measurement issued on the measurement stream, if any
                if (last_measured >= 0) cudaStreamWaitEvent(st, h->measure_done[last_measured % nybuf], 0);
                MeasureArgs ma{};
                ma.d = d;
                ma.chi_r = L.chi_r;
                ma.Cs = L.Cs;
                ma.tiles_per_s = L.tiles_per_s;
                ma.rows = (int)rows;
                ma.seed = seed;
                ma.n_base = (uint64_t)(n0 + r0);
                ma.k = (uint32_t)k;
                ma.job = job;
                ma.row0 = r0;
                ma.ld_next = ldV;
                ma.K_next = K_next;
                ma.V32 = nullptr;
                for (int p = 0; p < 3; ++p) ma.Vp[p] = Vp[nxt][p];
                ma.nplanes = planes;
                ma.outcomes = h->O.as<uint8_t>() + (int64_t)k * N_pad + r0;
                ma.logp = h->logp.as<double>();
                ma.trace = trace_buf ? trace_buf + (int64_t)k * trace_rows * d : nullptr;
                ma.trace_rows = (int)trace_rows;
                ma.trace_slot = trace_slot;
                ma.err = d_err;
                ta.row0 = r0;
                ta.rows_pad = (int)rows_pad;
                ta.has_tmY = false;
                cudaEvent_t c0 = timer.get(), c1 = timer.get();
                cudaEventRecord(c0, st);
                e = launch_contract_tc_cluster(ta, L, (int)rows, d_err, st, ma);
                if (e != cudaSuccess) return cuda_fail(h, e, "cluster contraction launch");
                cudaEventRecord(c1, st);
                timer.contract.push_back({c0, c1});
                h->stats.launches += 1;
                h->stats.contract_launches += 1;
                last_measured = -1;
                continue;
            }
            // the scratch buffer is free once the measurement two micro-batches back is done; with one
            // micro-batch per site the left rows of this contraction come from the previous measurement
            if (!fused && g >= nybuf) cudaStreamWaitEvent(st, h->measure_done[yb], 0);
            if (!fused && nybuf == 1 && g >= 1) cudaStreamWaitEvent(st, h->measure_done[0], 0);
            ContractOut co;
            co.Y = h->Y[yb].as<float>();
            co.ldY = L.ncols;
            co.P = h->P[yb].as<float>();
            co.ldP = L.ncols / L.bn;
            co.rows_valid = (int)rows;
            MeasureArgs ma;
            ma.Y = co.Y;
            ma.ldY = co.ldY;
            ma.P = co.P;
            ma.ldP = co.ldP;
            ma.d = d;
            ma.chi_r = L.chi_r;
            ma.Cs = L.Cs;
            ma.tiles_per_s = L.tiles_per_s;
            ma.rows = (int)rows;
            ma.seed = seed;
            ma.n_base = (uint64_t)(n0 + r0);
            ma.k = (uint32_t)k;
            ma.job = job;
            ma.row0 = r0;
            ma.ld_next = ldV;
            ma.K_next = K_next;
            ma.V32 = bf16 ? nullptr : h->V[nxt][0].as<float>();
            for (int p = 0; p < 3; ++p) ma.Vp[p] = fp8 ? nullptr : Vp[nxt][p];
            ma.nplanes = planes;
            ma.f16 = is_f16(h) ? 1 : 0;
            ma.V8 = fp8 ? h->V[nxt][0].as<uint8_t>() : nullptr;
            ma.V8lo = (fp8 && planes > 1) ? h->V[nxt][1].as<uint8_t>() : nullptr;
            ma.outcomes = h->O.as<uint8_t>() + (int64_t)k * N_pad + r0;
            ma.logp = h->logp.as<double>();
            ma.trace = trace_buf ? trace_buf + (int64_t)k * trace_rows * d : nullptr;
            ma.trace_rows = (int)trace_rows;
            ma.trace_slot = trace_slot;
            ma.err = d_err;
            ma.mu = mu_dev ? mu_dev + (int64_t)k * ld_mu + r0 : nullptr;
            ma.disp_tab = disp_tab;
            ma.disp_D = mu_dev ? h->disp_D.as<float2>() : nullptr;
            ma.disp_u = mu_dev ? h->disp_u.as<double>() : nullptr;
            cudaEvent_t c0 = timer.get(), c1 = timer.get();
            cudaEventRecord(c0, st);
            if (bf16) {
                ta.row0 = r0;
                ta.rows_pad = (int)rows_pad;
                ta.has_tmY = !fused && encode_2d_f32_scratch(&ta.tmY, co.Y, L.ncols, rows, L.ncols);
                if (h->opt.accum_chunk > 0 && ta.has_tmY && !fp8 && L.bn == 256)
                    e = launch_contract_tc_promoted(ta, L, co, h->opt.accum_chunk, h->num_sms, d_err, st);
                else if (h->opt.k_split >= 2 && ta.has_tmY && !fp8 && L.K_pad / L.bk >= h->opt.k_split)
                    e = launch_contract_tc_splitk(ta, L, co, h->opt.k_split, d_err, st);
                else
                    e = launch_contract_tc(ta, L, co, h->num_sms, d_err, st, fused ? &ma : nullptr);
                if (e != cudaSuccess) return cuda_fail(h, e, "contraction launch");
            } else {
                launch_contract_f32(h->V[cur][0].as<float>(), ldV, r0, rows_pad, t->Bt.as<float>(), L, co, st);
            }
            h->stats.launches += 1;
            h->stats.contract_launches += 1;
            cudaEventRecord(c1, st);
            timer.contract.push_back({c0, c1});
            if (!fused) {
                cudaEvent_t m0 = timer.get(), m1 = timer.get();
                cudaEventRecord(h->contract_done[yb], st);
                cudaStreamWaitEvent(ms, h->contract_done[yb], 0);
                cudaEventRecord(m0, ms);
                if (ma.mu) launch_measure_displaced(ma, h->num_sms, ms);
                else launch_measure(ma, ms);
                h->stats.launches += ma.mu ? 2 : 1;  // the displaced measurement has a prep kernel
                cudaEventRecord(m1, ms);
                cudaEventRecord(h->measure_done[yb], ms);
                timer.measure.push_back({m0, m1});
                last_measured = g;
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
        }
    }
    // the compute stream resumes after the last measurement
    if (last_measured >= 0) cudaStreamWaitEvent(st, h->measure_done[last_measured % nybuf], 0);

    // ---- outputs -------------------------------------------------------------
    if (out_samples) {
        uint8_t *dst = samples_dev ? out_samples : h->Dout.as<uint8_t>();
        launch_transpose_outcomes(h->O.as<uint8_t>(), N_pad, N, M, dst, st);
        h->stats.launches += 1;
        if (!samples_dev) {
            e = cudaMemcpyAsync(out_samples, dst, (size_t)N * M, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy of samples");
            h->stats.d2h_bytes += (int64_t)N * M;
        }
    }
    if (out_logprob) {
        e = cudaMemcpyAsync(out_logprob, h->logp.p, (size_t)N * 8,
                            logp_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of log-probabilities");
        if (!logp_dev) h->stats.d2h_bytes += N * 8;
    }
    if (trace_buf && !trace_dev) {
        e = cudaMemcpyAsync(trace_probs, trace_buf, (size_t)M * trace_rows * d * 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of trace");
    }
    int herr = 0;
    e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy of error word");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "sampling");
    h->stats.ms_contract = timer.total(timer.contract);
    h->stats.ms_measure = timer.total(timer.measure);
    h->stats.ms_h2d = timer.total(timer.copy);
    h->stats.ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (herr == kDevNumeric)
        return fail(h, FASTMPS_ERR_NUMERIC, "a sample's probabilities summed to zero or a non-finite value");
    if (herr != 0)
        return fail(h, FASTMPS_ERR_TIMEOUT,
                    "a bounded device wait in the contraction kernel gave up (code " + std::to_string(herr) + ")");
    return FASTMPS_OK;
}

}  // namespace

extern "C" {

void fastmps_default_options(fastmps_options *opt) {
    if (!opt) return;
    opt->precision = FASTMPS_FP32;
    opt->residency = FASTMPS_RESIDENT_HBM;
    opt->max_microbatch = 0;
    opt->autotune = 0;
    opt->stream = nullptr;
    opt->fused_measure = 0;
    opt->k_split = 0;
    opt->accum_chunk = 0;
}

int fastmps_create(fastmps_handle *out, int device, const fastmps_options *opt) {
    if (!out) {
        g_create_error = "out is NULL";
        return FASTMPS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fastmps_options o;
    fastmps_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < FASTMPS_FP32 || o.precision > FASTMPS_FP16X3) {
        g_create_error = "unknown precision";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.accum_chunk < 0 || o.accum_chunk > 4096) {
        g_create_error = "accum_chunk must be 0..4096";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.k_split < 0 || o.k_split > 8) {
        g_create_error = "k_split must be 0..8";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.residency != FASTMPS_RESIDENT_HBM && o.residency != FASTMPS_HOST_STREAM) {
        g_create_error = "unknown residency";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.residency == FASTMPS_HOST_STREAM &&
        (o.precision == FASTMPS_FP32 || o.precision == FASTMPS_FP8X1 || o.precision == FASTMPS_FP8X2)) {
        g_create_error = "host streaming keeps 16-bit tensors: use a BF16 or the FP16 precision";
        return FASTMPS_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_create_error = "no such CUDA device";
        return FASTMPS_ERR_CUDA;
    }
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    if (!(prop.major == 10 && prop.minor == 3)) {
        g_create_error = std::string("device ") + prop.name + " is sm_" + std::to_string(prop.major) +
                         std::to_string(prop.minor) + "; this library is built for sm_103a only";
        return FASTMPS_ERR_UNSUPPORTED;
    }
    if (o.precision != FASTMPS_FP32 && (!tc_max_smem_ok(device) || !get_encode_fn())) {
        g_create_error = "tensor-core path needs 227 KB shared memory and cuTensorMapEncodeTiled";
        return FASTMPS_ERR_UNSUPPORTED;
    }
    fastmps_ctx *h = new (std::nothrow) fastmps_ctx();
    if (!h) {
        g_create_error = "out of host memory";
        return FASTMPS_ERR_OOM;
    }
    h->device = device;
    h->opt = o;
    h->num_sms = prop.multiProcessorCount;
    cudaSetDevice(device);
    if (o.stream) {
        h->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            g_create_error = "stream creation failed";
            return FASTMPS_ERR_CUDA;
        }
        h->own_stream = true;
    }
    cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&h->measure_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2; ++i) {
        cudaEventCreateWithFlags(&h->copy_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&h->slot_free[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&h->contract_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&h->measure_done[i], cudaEventDisableTiming);
    }
    h->staging.host = false;
    *out = h;
    return FASTMPS_OK;
}

void fastmps_destroy(fastmps_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    fastmps::batch_release(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    if (h->measure_stream) cudaStreamSynchronize(h->measure_stream);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
        if (h->copy_done[i]) cudaEventDestroy(h->copy_done[i]);
        if (h->slot_free[i]) cudaEventDestroy(h->slot_free[i]);
        if (h->contract_done[i]) cudaEventDestroy(h->contract_done[i]);
        if (h->measure_done[i]) cudaEventDestroy(h->measure_done[i]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->measure_stream) cudaStreamDestroy(h->measure_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char *fastmps_last_error(fastmps_handle h) {
    if (!h) return g_create_error.c_str();
    return h->last_error.c_str();
}

int fastmps_load_site(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *A, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (k < 0 || k >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "site index out of range");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, A, dtype);
    if (rc) return rc;
    h->site_tensor[k] = std::move(t);
    h->site_pool.erase(k);
    return FASTMPS_OK;
}

int fastmps_load_pool(fastmps_handle h, int j, int chi_l, int d, int chi_r, const void *A, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (j < 0 || j >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "pool index out of range");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, A, dtype);
    if (rc) return rc;
    h->pool_tensor[j] = std::move(t);
    return FASTMPS_OK;
}

int fastmps_map_site(fastmps_handle h, int k, int j) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (k < 0 || k >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "site index out of range");
    if (h->pool_tensor.find(j) == h->pool_tensor.end())
        return fail(h, FASTMPS_ERR_NOT_LOADED, "pool entry " + std::to_string(j) + " is not loaded");
    h->site_pool[k] = j;
    h->site_tensor.erase(k);
    return FASTMPS_OK;
}

int fastmps_sample_ex(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N, uint64_t seed,
                      uint32_t job, uint8_t *out_samples, double *out_logprob, int64_t trace_rows,
                      double *trace_probs) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    try {
        return run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, trace_rows, trace_probs);
    } catch (const std::bad_alloc &) {
        return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(h, FASTMPS_ERR_CUDA, "unexpected host exception");
    }
}

int fastmps_sample_traced(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N, uint64_t seed,
                          uint32_t job, uint8_t *out_samples, double *out_logprob, const int64_t *trace_list,
                          int64_t n_trace, double *trace_probs) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (n_trace < 0 || (n_trace > 0 && (!trace_list || !trace_probs)))
        return fail(h, FASTMPS_ERR_INVALID_ARG, "n_trace > 0 needs trace_list and trace_probs");
    cudaSetDevice(h->device);
    try {
        return run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, n_trace, trace_probs,
                          nullptr, 0, n_trace > 0 ? trace_list : nullptr);
    } catch (const std::bad_alloc &) {
        return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(h, FASTMPS_ERR_CUDA, "unexpected host exception");
    }
}

int fastmps_sample(fastmps_handle h, int M, int d, const int *bond_dims, int64_t N, uint64_t seed,
                   uint8_t *out_samples, double *out_logprob) {
    return fastmps_sample_ex(h, M, d, bond_dims, 0, N, seed, 0, out_samples, out_logprob, 0, nullptr);
}

int fastmps_load_site_vidal(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *Gamma,
                            const void *Lambda, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (k < 0 || k >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "site index out of range");
    if (!Lambda) return fail(h, FASTMPS_ERR_INVALID_ARG, "Lambda is NULL");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, Gamma, dtype, Lambda);
    if (rc) return rc;
    h->site_tensor[k] = std::move(t);
    h->site_pool.erase(k);
    return FASTMPS_OK;
}

int fastmps_load_pool_vidal(fastmps_handle h, int j, int chi_l, int d, int chi_r, const void *Gamma,
                            const void *Lambda, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (j < 0 || j >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "pool index out of range");
    if (!Lambda) return fail(h, FASTMPS_ERR_INVALID_ARG, "Lambda is NULL");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, Gamma, dtype, Lambda);
    if (rc) return rc;
    h->pool_tensor[j] = std::move(t);
    return FASTMPS_OK;
}

int fastmps_load_site_vidal_truncated(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *Gamma,
                                      const void *Lambda, int dtype, int keep_l, int keep_r) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (!Gamma || !Lambda) return fail(h, FASTMPS_ERR_INVALID_ARG, "Gamma or Lambda is NULL");
    if (dtype != FASTMPS_C64 && dtype != FASTMPS_C128) return fail(h, FASTMPS_ERR_INVALID_ARG, "unknown dtype");
    if (chi_l < 1 || chi_r < 1 || d < 2 || d > 255 || keep_l < 1 || keep_l > chi_l || keep_r < 1 || keep_r > chi_r)
        return fail(h, FASTMPS_ERR_SHAPE, "need 1 <= keep_l <= chi_l, 1 <= keep_r <= chi_r, 2 <= d <= 255");
    if (keep_l == chi_l && keep_r == chi_r) return fastmps_load_site_vidal(h, k, chi_l, d, chi_r, Gamma, Lambda, dtype);
    cudaSetDevice(h->device);
    const size_t elem = dtype == FASTMPS_C128 ? 16 : 8;
    const size_t rows = (size_t)keep_l * d, width = (size_t)keep_r * elem, pitch = (size_t)chi_r * elem;
    // rows (a, s) of Gamma are contiguous runs of chi_r entries: the leading block is a 2D copy
    if (is_device_ptr(Gamma)) {
        if (!h->trunc.ensure(rows * width)) return fail(h, FASTMPS_ERR_OOM, "allocation failed");
        cudaError_t e = cudaMemcpy2DAsync(h->trunc.p, width, Gamma, pitch, width, rows, cudaMemcpyDeviceToDevice,
                                          h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "gather of the leading block");
        return fastmps_load_site_vidal(h, k, keep_l, d, keep_r, h->trunc.p, Lambda, dtype);
    }
    std::vector<uint8_t> block(rows * width);
    const uint8_t *src = static_cast<const uint8_t *>(Gamma);
    for (size_t r = 0; r < rows; ++r) memcpy(block.data() + r * width, src + r * pitch, width);
    return fastmps_load_site_vidal(h, k, keep_l, d, keep_r, block.data(), Lambda, dtype);
}

int fastmps_sample_displaced(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                             uint64_t seed, uint32_t job, const float *mu, int64_t ld_mu, uint8_t *out_samples,
                             double *out_logprob, int64_t trace_rows, double *trace_probs) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    try {
        if (!mu) return fail(h, FASTMPS_ERR_INVALID_ARG, "mu is NULL");
        if (M < 1 || N < 0 || ld_mu < N) return fail(h, FASTMPS_ERR_INVALID_ARG, "need M >= 1, N >= 0, ld_mu >= N");
        if (d < 2 || d > kMaxDisplacedD)
            return fail(h, FASTMPS_ERR_SHAPE, "displaced sampling supports 2 <= d <= " +
                                                  std::to_string(kMaxDisplacedD));
        if (is_fp8(h) || is_f16(h))
            return fail(h, FASTMPS_ERR_UNSUPPORTED, "displaced sampling needs FP32 or a BF16 precision");
        if (N == 0) return run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, trace_rows,
                                      trace_probs);
        const float2 *mu_dev;
        int64_t ld = ld_mu;
        if (is_device_ptr(mu)) {
            if (reinterpret_cast<uintptr_t>(mu) % 8 != 0)
                return fail(h, FASTMPS_ERR_INVALID_ARG, "device mu must be 8-byte aligned");
            mu_dev = reinterpret_cast<const float2 *>(mu);
        } else {
            if (!h->mu.ensure((size_t)M * N * 8)) return fail(h, FASTMPS_ERR_OOM, "amplitude allocation failed");
            cudaError_t e = cudaMemcpy2DAsync(h->mu.p, (size_t)N * 8, mu, (size_t)ld_mu * 8, (size_t)N * 8, M,
                                              cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy of displacement amplitudes");
            mu_dev = h->mu.as<float2>();
            ld = N;
        }
        int rc = run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, trace_rows,
                            trace_probs, mu_dev, ld);
        if (rc == FASTMPS_OK && !is_device_ptr(mu)) h->stats.h2d_bytes += (int64_t)M * N * 8;
        return rc;
    } catch (const std::bad_alloc &) {
        return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(h, FASTMPS_ERR_CUDA, "unexpected host exception");
    }
}

int fastmps_displacement(fastmps_handle h, int64_t N, int d, const float *mu, float *D) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (!mu || !D || N < 0) return fail(h, FASTMPS_ERR_INVALID_ARG, "need mu, D and N >= 0");
    if (d < 1 || d > 255) return fail(h, FASTMPS_ERR_SHAPE, "need 1 <= d <= 255");
    if (N == 0) return FASTMPS_OK;
    cudaSetDevice(h->device);
    const bool mu_dev = is_device_ptr(mu), D_dev = is_device_ptr(D);
    if ((mu_dev && reinterpret_cast<uintptr_t>(mu) % 8) || (D_dev && reinterpret_cast<uintptr_t>(D) % 8))
        return fail(h, FASTMPS_ERR_INVALID_ARG, "device arrays must be 8-byte aligned");
    const size_t mu_bytes = (size_t)N * 8, D_bytes = (size_t)N * d * d * 8;
    const size_t off = roundup((int64_t)mu_bytes, 256);
    if ((!mu_dev || !D_dev) && !h->disp_io.ensure(off + D_bytes))
        return fail(h, FASTMPS_ERR_OOM, "staging allocation failed");
    cudaStream_t st = h->stream;
    cudaError_t e;
    const float2 *mu_d = reinterpret_cast<const float2 *>(mu);
    if (!mu_dev) {
        e = cudaMemcpyAsync(h->disp_io.p, mu, mu_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of amplitudes");
        mu_d = h->disp_io.as<float2>();
    }
    float2 *D_d = D_dev ? reinterpret_cast<float2 *>(D)
                        : reinterpret_cast<float2 *>(static_cast<char *>(h->disp_io.p) + off);
    const float *tab = displacement_table(h, d);
    if (!tab) return fail(h, FASTMPS_ERR_OOM, "displacement table allocation failed");
    launch_displacement(mu_d, N, d, tab, D_d, h->num_sms, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "displacement launch");
    if (!D_dev) {
        e = cudaMemcpyAsync(D, D_d, D_bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of displacement matrices");
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "displacement");
    return FASTMPS_OK;
}

int fastmps_get_stats(fastmps_handle h, fastmps_stats *out) {
    if (!h || !out) return FASTMPS_ERR_INVALID_ARG;
    *out = h->stats;
    return FASTMPS_OK;
}

const char *fastmps_version(void) { return "fastmps-gb300 0.1 (sm_103a)"; }

int fastmps_selftest_bounded_wait(int device, double limit_ms, int *status, double *waited_ms) {
    if (!status || !waited_ms || limit_ms <= 0) return FASTMPS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return FASTMPS_ERR_CUDA;
    }
    int *d_status = nullptr;
    unsigned long long *d_ns = nullptr;
    if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (d_status) cudaFree(d_status);
        return FASTMPS_ERR_OOM;
    }
    launch_bounded_wait_selftest((uint64_t)(limit_ms * 1e6), d_status, d_ns, 0);
    int st = -1;
    unsigned long long ns = 0;
    cudaError_t e = cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost);
    cudaFree(d_status);
    cudaFree(d_ns);
    if (e != cudaSuccess) return FASTMPS_ERR_CUDA;
    *status = st == kDevOk ? FASTMPS_OK : FASTMPS_ERR_TIMEOUT;
    *waited_ms = (double)ns / 1e6;
    return FASTMPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Views for entry points implemented in other translation units.
// ---------------------------------------------------------------------------
#include "handle_view.h"

namespace fastmps {

int handle_view(fastmps_handle h, HandleView *out) {
    if (!h || !out) return FASTMPS_ERR_INVALID_ARG;
    out->device = h->device;
    out->precision = h->opt.precision;
    out->residency = h->opt.residency;
    out->stream = h->stream;
    out->num_sms = h->num_sms;
    out->max_microbatch = h->opt.max_microbatch;
    return FASTMPS_OK;
}

int site_view(fastmps_handle h, int k, SiteView *out) {
    Tensor *t = site_tensor_of(h, k);
    if (!t) return FASTMPS_ERR_NOT_LOADED;
    out->L = t->L;
    out->B0 = t->B_hi.as<__nv_bfloat16>();
    out->B1 = t->B_lo.as<__nv_bfloat16>();
    out->Bt = t->Bt.as<float>();
    out->tmB[0] = t->tmB[0];
    out->tmB[1] = t->tmB[1];
    return FASTMPS_OK;
}

int set_error(fastmps_handle h, int code, const char *msg) { return fail(h, code, msg); }

fastmps_stats *handle_stats(fastmps_handle h) { return &h->stats; }

void precision_products(int precision, int *a_planes, int *b_planes, int *nprod, int *pa, int *pb) {
    const PrecisionPlan p = plan_of(precision);
    *a_planes = p.a_planes;
    *b_planes = p.b_planes;
    *nprod = p.nprod;
    for (int q = 0; q < kMaxProducts; ++q) {
        pa[q] = p.pa[q];
        pb[q] = p.pb[q];
    }
}

bool encode_bf16_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                     uint32_t box_outer) {
    return encode_2d_bf16(map, base, inner, outer, ld_elems, 64, box_outer);
}

}  // namespace fastmps
