// Read-only views of a handle's state for entry points compiled outside the handle's own units (internal).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fastmps.h"
#include "launch.h"

namespace fastmps {

struct HandleView {
    int device;
    int precision;
    int residency;
    cudaStream_t stream;
    int num_sms;
    int64_t max_microbatch;  // rows per contraction launch requested in the options (0: automatic)
};

struct SiteView {
    SiteLayout L;
    const __nv_bfloat16 *B0, *B1;  // BF16 planes of the stacked operand (resident BF16 modes)
    const float *Bt;               // FP32 stacked operand (FP32 mode)
    CUtensorMap tmB[2];            // tensor maps over B0, B1 (resident BF16 modes)
};

// 0 on success; FASTMPS_ERR_NOT_LOADED if site k has no tensor.
int handle_view(fastmps_handle h, HandleView *out);
int site_view(fastmps_handle h, int k, SiteView *out);
// Records msg as the handle's last error and returns code.
int set_error(fastmps_handle h, int code, const char *msg);
// The product list of a BF16 precision mode (planes of V and B and the pairs multiplied).
void precision_products(int precision, int *a_planes, int *b_planes, int *nprod, int *pa, int *pb);
// cuTensorMapEncodeTiled over a BF16 matrix [outer][ld] with a (64 x box_outer) box, 128-byte swizzle.
bool encode_bf16_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                     uint32_t box_outer);

// Statistics of the handle's last call (written by the batch engine).
fastmps_stats *handle_stats(fastmps_handle h);
// Releases the batch engine's state of a handle (called by fastmps_destroy).
void batch_release(fastmps_handle h);

}  // namespace fastmps
