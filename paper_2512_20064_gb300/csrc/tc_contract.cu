// tcgen05 split-precision contraction of the left vectors with one site tensor.
//
// Y[row, c] = sum_kappa V[row, kappa] B[c, kappa] over the stacked real
// operands (K = 2 chi_l, padded to a multiple of 64), with V = V_0 + V_1 (+ V_2)
// and B = B_0 (+ B_1) held as BF16 planes of successive rounding residuals
// and a list of plane products accumulated in FP32 in tensor memory, e.g.
//   BF16x2 : V_0 B_0 + V_1 B_0
//   BF16x3 : V_0 B_0 + V_1 B_0 + V_0 B_1
//   BF16x3L: V_0 B_0 + V_1 B_0 + V_2 B_0
//   BF16x4 : V_0 B_0 + V_1 B_0 + V_2 B_0 + V_0 B_1
//
// Persistent kernel, one CTA per SM, 192 threads:
//   warp 0 : TMA producer (one thread) -- 128 x 64 tiles of each V plane and
//            bn x 64 tiles of each B plane per stage, 128-byte swizzle
//   warp 1 : TMEM allocator and MMA issuer (one thread), M = 128, N = bn, K = 16
//   warps 2-5 : epilogue -- tensor memory -> registers, one row per thread:
//            store the FP32 tile to the scratch Y and the row's sum of squares
//            over the tile (the tile lies in one outcome block s) to P.
// Two accumulator buffers of 256 columns let the epilogue of tile i overlap
// the main loop of tile i+1.  Every wait is bounded (common.cuh); on a
// timeout the kernel records an error word, drains its own in-flight copies
// and MMAs, frees tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "launch.h"

namespace fastmps {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;                      // BF16 elements per k-block = one 128-byte swizzle row
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;          // 2 accumulators x 256 columns
constexpr uint32_t kAccStride = 256;
constexpr uint32_t kATileBytes = kBM * kBK * 2;  // 16 KB
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 232448;           // 227 KB opt-in per block

struct TcParams {
    int num_m_tiles, num_n_tiles, num_k_blocks, bn;
    int a_planes, b_planes, stages, nprod;
    uint32_t prod_code;  // product q uses A plane (code >> 4q) & 3 and B plane (code >> (4q+2)) & 3
    uint32_t stage_bytes, b_plane_bytes;
    int row0;
    uint32_t idesc;
    float *Y;
    int64_t ldY;
    float *P;
    int ldP;
    int rows_valid;
    int *err;
};

__device__ __forceinline__ void record_error(int *err, volatile int *abort_flag, int code) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

// Time-bounded wait that ignores the abort flag (used while draining).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > 200000000ull) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 1)
tc_contract_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB0,
                   const __grid_constant__ CUtensorMap tmB1, const TcParams p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * p.stage_bytes);
    uint64_t *empty = full + p.stages;
    uint64_t *tfull = empty + p.stages;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull[0], 1);
        mbar_init(&tfull[1], 1);
        mbar_init(&tempty[0], 128);
        mbar_init(&tempty[1], 128);
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(&tmA0);
        if (p.a_planes > 1) prefetch_tmap(&tmA1);
        if (p.a_planes > 2) prefetch_tmap(&tmA2);
        prefetch_tmap(&tmB0);
        if (p.b_planes > 1) prefetch_tmap(&tmB1);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int total = p.num_m_tiles * p.num_n_tiles;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last_parity[s] = -1;
            bool failed = false;
            for (int tile = blockIdx.x; tile < total && !failed; tile += gridDim.x) {
                const int mt = tile / p.num_n_tiles;
                const int nt = tile - mt * p.num_n_tiles;
                const int y_a = p.row0 + mt * kBM;
                const int y_b = nt * p.bn;
                for (int kb = 0; kb < p.num_k_blocks; ++kb) {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag)) {
                        record_error(p.err, abort_flag, kDevTimeoutProducer);
                        failed = true;
                        break;
                    }
                    uint8_t *sbase = smem + (size_t)stage * p.stage_bytes;
                    mbar_arrive_expect_tx(&full[stage], p.stage_bytes);
                    const int x = kb * kBK;
                    tma_load_2d(sbase, &tmA0, &full[stage], x, y_a);
                    if (p.a_planes > 1) tma_load_2d(sbase + kATileBytes, &tmA1, &full[stage], x, y_a);
                    if (p.a_planes > 2) tma_load_2d(sbase + 2 * kATileBytes, &tmA2, &full[stage], x, y_a);
                    uint8_t *bbase = sbase + (size_t)p.a_planes * kATileBytes;
                    tma_load_2d(bbase, &tmB0, &full[stage], x, y_b);
                    if (p.b_planes > 1) tma_load_2d(bbase + p.b_plane_bytes, &tmB1, &full[stage], x, y_b);
                    last_parity[stage] = (int)phase;
                    if (++stage == p.stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (failed) {
                // let the copies this thread issued land before shared memory is released
                for (int s = 0; s < p.stages; ++s)
                    if (last_parity[s] >= 0) mbar_wait_drain(&full[s], (uint32_t)last_parity[s]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int lt = 0;
            bool failed = false;
            bool issued = false;
            for (int tile = blockIdx.x; tile < total && !failed; tile += gridDim.x, ++lt) {
                const int buf = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!mbar_wait_bounded(&tempty[buf], (use & 1u) ^ 1u, abort_flag)) {
                    record_error(p.err, abort_flag, kDevTimeoutMma);
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)buf * kAccStride;
                for (int kb = 0; kb < p.num_k_blocks; ++kb) {
                    if (!mbar_wait_bounded(&full[stage], phase, abort_flag)) {
                        record_error(p.err, abort_flag, kDevTimeoutMma);
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + (size_t)stage * p.stage_bytes);
                    const uint32_t sb = sa + (uint32_t)p.a_planes * kATileBytes;
                    for (int q = 0; q < p.nprod; ++q) {
                        const uint32_t pa = (p.prod_code >> (4 * q)) & 3u;
                        const uint32_t pb = (p.prod_code >> (4 * q + 2)) & 3u;
                        const uint32_t a_addr = sa + pa * kATileBytes;
                        const uint32_t b_addr = sb + pb * p.b_plane_bytes;
                        const uint64_t ad = sw128_kmajor_desc(a_addr);
                        const uint64_t bd = sw128_kmajor_desc(b_addr);
#pragma unroll
                        for (int k16 = 0; k16 < kBK / 16; ++k16) {
                            // +32 bytes along K inside the swizzle row = +2 in the address field
                            tc_mma_bf16(d_tmem, ad + (uint64_t)(2 * k16), bd + (uint64_t)(2 * k16), p.idesc,
                                        (kb | q | k16) != 0 ? 1u : 0u);
                        }
                    }
                    issued = true;
                    tc_commit(&empty[stage]);
                    if (++stage == p.stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (failed) break;
                tc_commit(&tfull[buf]);
            }
            if (failed && issued) {
                // wait for this thread's outstanding MMAs before tensor memory is freed
                tc_commit(drain);
                mbar_wait_drain(drain, 0u);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;  // tensor-memory lane quarter this warp may access
        int lt = 0;
        for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++lt) {
            const int buf = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            const int mt = tile / p.num_n_tiles;
            const int nt = tile - mt * p.num_n_tiles;
            if (!mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag)) {
                record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                break;
            }
            tc_fence_after();
            const int row = mt * kBM + quad * 32 + lane;
            const bool valid = row < p.rows_valid;
            float *yrow = p.Y + (int64_t)row * p.ldY + (int64_t)nt * p.bn;
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * kAccStride;
            float ss = 0.f;
            for (int ch = 0; ch < p.bn / 32; ++ch) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(taddr + (uint32_t)(ch * 32), r);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float v = __uint_as_float(r[j]);
                    ss = fmaf(v, v, ss);
                }
                if (valid) {
                    float4 *dst = reinterpret_cast<float4 *>(yrow + ch * 32);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                             __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[buf]);
            if (valid) p.P[(int64_t)row * p.ldP + nt] = ss;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

int stages_for(uint32_t stage_bytes) {
    const int fixed = 1024 /* alignment */ + 256 /* barriers */;
    int s = (kSmemLimit - fixed) / (int)stage_bytes;
    if (s > kMaxStages) s = kMaxStages;
    return s;
}

}  // namespace

int tc_max_smem_ok(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return v >= kSmemLimit;
}

cudaError_t launch_contract_tc(const TcArgs &a, const SiteLayout &L, const ContractOut &o, int num_sms, int *d_err,
                               cudaStream_t st) {
    TcParams p;
    p.num_m_tiles = a.rows_pad / kBM;
    p.num_n_tiles = L.ncols / L.bn;
    p.num_k_blocks = L.K_pad / kBK;
    p.bn = L.bn;
    p.a_planes = a.a_planes;
    p.b_planes = a.b_planes;
    if (a.nprod < 1 || a.nprod > kMaxProducts || a.a_planes < 1 || a.a_planes > 3 || a.b_planes < 1 ||
        a.b_planes > 2)
        return cudaErrorInvalidValue;
    p.nprod = a.nprod;
    p.prod_code = 0;
    for (int q = 0; q < a.nprod; ++q) {
        if (a.prod_a[q] < 0 || a.prod_a[q] >= a.a_planes || a.prod_b[q] < 0 || a.prod_b[q] >= a.b_planes)
            return cudaErrorInvalidValue;
        p.prod_code |= ((uint32_t)a.prod_a[q] | ((uint32_t)a.prod_b[q] << 2)) << (4 * q);
    }
    p.b_plane_bytes = (uint32_t)L.bn * kBK * 2;
    p.stage_bytes = (uint32_t)a.a_planes * kATileBytes + (uint32_t)a.b_planes * p.b_plane_bytes;
    p.stages = stages_for(p.stage_bytes);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    p.row0 = (int)a.row0;
    p.idesc = idesc_bf16_f32(kBM, L.bn);
    p.Y = o.Y;
    p.ldY = o.ldY;
    p.P = o.P;
    p.ldP = o.ldP;
    p.rows_valid = o.rows_valid;
    p.err = d_err;
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + 256;
    cudaError_t e = cudaFuncSetAttribute(tc_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    const int total = p.num_m_tiles * p.num_n_tiles;
    const int grid = total < num_sms ? total : num_sms;
    if (grid <= 0) return cudaSuccess;
    tc_contract_kernel<<<grid, kThreads, smem, st>>>(a.tmA[0], a.tmA[a.a_planes > 1 ? 1 : 0],
                                                     a.tmA[a.a_planes > 2 ? 2 : 0], a.tmB[0],
                                                     a.tmB[a.b_planes > 1 ? 1 : 0], p);
    return cudaGetLastError();
}

}  // namespace fastmps
