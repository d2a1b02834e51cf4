// Grouped contraction and measurement: many independent chains in one launch.
//
// A "round" advances every active job (one MPS, one chunk of its rows) by one
// site.  tc_contract_grouped_kernel is the persistent tcgen05 contraction of
// tc_contract.cu (TMA producer warp, MMA warp, four epilogue warps, two TMEM
// accumulators) run over the concatenated tile space of all segments of the
// round: each tile looks up its segment (tensor maps in device memory,
// n-tile width, K extent, scratch pointers), so jobs with different bond
// dimensions, physical dimensions and row counts share the GPU in one launch.
// measure_grouped_kernel then measures the rows of every segment
// (Algorithm 2), one warp per 32 rows.  All rounds of a batch are captured
// into one CUDA graph by the host engine.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "launch.h"
#include "measure.cuh"

namespace fastmps {

namespace {

constexpr int kBM = 128;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr uint32_t kATileBytes = 16384;      // 128 rows x 128 bytes
constexpr uint32_t kBPlaneBytesMax = 32768;  // 256 rows x 128 bytes
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 232448;
constexpr int kBarrierBytes = 512;

struct GParams {
    const TcSegment *segs;
    int nseg, total_tiles, stages, a_planes, b_planes, nprod;
    uint32_t prod_code, stage_bytes;
    int *err;
};

__device__ __forceinline__ void record_error(int *err, volatile int *abort_flag, int code) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

__device__ __forceinline__ bool mbar_wait_drain(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > 200000000ull) return false;
    }
    return true;
}

// Segment of global tile t, searching forward from *cursor (tiles visited in increasing order).
__device__ __forceinline__ const TcSegment *segment_of(const GParams &p, int t, int *cursor) {
    int s = *cursor;
    while (s + 1 < p.nseg && p.segs[s + 1].tile_begin <= t) ++s;
    *cursor = s;
    return &p.segs[s];
}

__global__ void __launch_bounds__(kThreads, 1) tc_contract_grouped_kernel(const GParams p) {
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
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0, cursor = 0;
            uint32_t phase = 0;
            int last_parity[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last_parity[s] = -1;
            bool failed = false;
            for (int t = blockIdx.x; t < p.total_tiles && !failed; t += gridDim.x) {
                const TcSegment *sg = segment_of(p, t, &cursor);
                const int lt = t - sg->tile_begin;
                const int mt = lt / sg->num_n_tiles;
                const int nt = lt - mt * sg->num_n_tiles;
                const int y_a = sg->row0 + mt * kBM;
                const int y_b = nt * sg->bn;
                for (int kb = 0; kb < sg->num_k_blocks; ++kb) {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag)) {
                        record_error(p.err, abort_flag, kDevTimeoutProducer);
                        failed = true;
                        break;
                    }
                    uint8_t *sbase = smem + (size_t)stage * p.stage_bytes;
                    mbar_arrive_expect_tx(&full[stage], sg->tx_bytes);
                    const int x = kb * 64;
                    for (int a = 0; a < p.a_planes; ++a)
                        tma_load_2d(sbase + a * kATileBytes, &sg->tmA[a], &full[stage], x, y_a);
                    uint8_t *bbase = sbase + (size_t)p.a_planes * kATileBytes;
                    for (int b = 0; b < p.b_planes; ++b)
                        tma_load_2d(bbase + b * kBPlaneBytesMax, &sg->tmB[b], &full[stage], x, y_b);
                    last_parity[stage] = (int)phase;
                    if (++stage == p.stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (failed)
                for (int s = 0; s < p.stages; ++s)
                    if (last_parity[s] >= 0) mbar_wait_drain(&full[s], (uint32_t)last_parity[s]);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0, lt = 0, cursor = 0;
            uint32_t phase = 0;
            bool failed = false, issued = false;
            for (int t = blockIdx.x; t < p.total_tiles && !failed; t += gridDim.x, ++lt) {
                const TcSegment *sg = segment_of(p, t, &cursor);
                const int buf = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!mbar_wait_bounded(&tempty[buf], (use & 1u) ^ 1u, abort_flag)) {
                    record_error(p.err, abort_flag, kDevTimeoutMma);
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)buf * kAccStride;
                for (int kb = 0; kb < sg->num_k_blocks; ++kb) {
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
                        const uint64_t ad = sw128_kmajor_desc(sa + pa * kATileBytes);
                        const uint64_t bd = sw128_kmajor_desc(sb + pb * kBPlaneBytesMax);
#pragma unroll
                        for (int k16 = 0; k16 < 4; ++k16)
                            tc_mma_bf16(d_tmem, ad + (uint64_t)(2 * k16), bd + (uint64_t)(2 * k16), sg->idesc,
                                        (kb | q | k16) != 0 ? 1u : 0u);
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
                tc_commit(drain);
                mbar_wait_drain(drain, 0u);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;
        int lt = 0, cursor = 0;
        for (int t = blockIdx.x; t < p.total_tiles; t += gridDim.x, ++lt) {
            const TcSegment *sg = segment_of(p, t, &cursor);
            const int buf = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            const int tl = t - sg->tile_begin;
            const int mt = tl / sg->num_n_tiles;
            const int nt = tl - mt * sg->num_n_tiles;
            if (!mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag)) {
                record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                break;
            }
            tc_fence_after();
            const int row = mt * kBM + quad * 32 + lane;
            const bool valid = row < sg->rows_valid;
            float *yrow = sg->Y + (int64_t)row * sg->ldY + (int64_t)nt * sg->bn;
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * kAccStride;
            float ss = 0.f;
            for (int ch = 0; ch < sg->bn / 32; ++ch) {
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
            if (valid) sg->P[(int64_t)row * sg->ldP + nt] = ss;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

constexpr int kMeasureThreads = 128;
constexpr int kMeasureWarps = kMeasureThreads / 32;

// One warp per 32 rows of one segment; warp w of the grid covers global 32-row block w.
__global__ void __launch_bounds__(kMeasureThreads)
measure_grouped_kernel(const TcSegment *__restrict__ segs, const MeasureArgs *__restrict__ meas, int nseg,
                       int total_blocks) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * kMeasureWarps + warp;
    if (gb >= total_blocks) return;
    int lo = 0, hi = nseg - 1;  // last segment with row_block_begin <= gb
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].row_block_begin <= gb) lo = mid;
        else hi = mid - 1;
    }
    const MeasureArgs &a = meas[lo];
    const int base = (gb - segs[lo].row_block_begin) * 32;
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
        measure_write_row(a, lane, a.Y + (int64_t)r * a.ldY + (int64_t)sj * a.Cs, scj, a.row0 + r);
    }
}

}  // namespace

cudaError_t prepare_contract_grouped() {
    return cudaFuncSetAttribute(tc_contract_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

cudaError_t launch_contract_grouped(const GroupedArgs &g, int num_sms, int *d_err, cudaStream_t st) {
    if (g.nseg <= 0 || g.total_tiles <= 0) return cudaSuccess;
    GParams p;
    p.segs = g.segs;
    p.nseg = g.nseg;
    p.total_tiles = g.total_tiles;
    p.a_planes = g.a_planes;
    p.b_planes = g.b_planes;
    p.nprod = g.nprod;
    if (g.nprod < 1 || g.nprod > kMaxProducts || g.a_planes < 1 || g.a_planes > 3 || g.b_planes < 1 ||
        g.b_planes > 2)
        return cudaErrorInvalidValue;
    p.prod_code = 0;
    for (int q = 0; q < g.nprod; ++q)
        p.prod_code |= ((uint32_t)g.prod_a[q] | ((uint32_t)g.prod_b[q] << 2)) << (4 * q);
    p.stage_bytes = (uint32_t)g.a_planes * kATileBytes + (uint32_t)g.b_planes * kBPlaneBytesMax;
    p.stages = (kSmemLimit - 1024 - kBarrierBytes) / (int)p.stage_bytes;
    if (p.stages > kMaxStages) p.stages = kMaxStages;
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    p.err = d_err;
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + kBarrierBytes;
    const int grid = g.total_tiles < num_sms ? g.total_tiles : num_sms;
    tc_contract_grouped_kernel<<<grid, kThreads, smem, st>>>(p);
    return cudaGetLastError();
}

void launch_measure_grouped(const GroupedArgs &g, cudaStream_t st) {
    if (g.nseg <= 0 || g.total_row_blocks <= 0) return;
    const int grid = (g.total_row_blocks + kMeasureWarps - 1) / kMeasureWarps;
    measure_grouped_kernel<<<grid, kMeasureThreads, 0, st>>>(g.segs, g.meas, g.nseg, g.total_row_blocks);
}

}  // namespace fastmps
