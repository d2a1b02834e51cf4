// Host helpers of the library (internal): error reporting, precision plans, site layouts, tensor-map
// encoding through the driver's cuTensorMapEncodeTiled, shape checks and pointer classification.
#include "context.h"

namespace fastmps {

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

namespace {
long long g_alloc_budget = -2;  // -2: not read yet, -1: no injection
}  // namespace

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

int fail(fastmps_handle h, int code, const std::string &msg) {
    if (h) h->last_error = msg;
    return code;
}

int cuda_fail(fastmps_handle h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? FASTMPS_ERR_OOM : FASTMPS_ERR_CUDA, m);
}

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

SiteLayout make_layout(int precision, int chi_l, int d, int chi_r, int bn_override) {
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

}  // namespace fastmps
