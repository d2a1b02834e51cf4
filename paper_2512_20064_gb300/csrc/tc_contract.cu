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
// the main loop of tile i+1.
//
// Fused variant (320 threads): warps 6-9 measure.  Each thread block owns
// whole m-tiles (128 rows) and walks all their n-tiles in order; after the
// last n-tile of an m-tile the epilogue hands it to the block's measurement
// warps through a shared-memory mbarrier ring (CTA-scope ordering only).
// They combine the per-tile sums of squares of the 128 rows in FP64, draw the
// outcomes and write the renormalised selected blocks as the next left rows
// (Algorithm 2) while the tensor cores work on the next m-tile.
//
// Every wait is bounded (common.cuh); on a timeout the kernel records an
// error word, drains its own in-flight copies and MMAs, frees tensor memory
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"
#include "launch.h"
#include "measure.cuh"

namespace fastmps {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;                      // BF16 elements per k-block = one 128-byte swizzle row (FP8: 128)
constexpr int kThreads = 192;                // TMA + MMA + 4 epilogue warps
constexpr int kThreadsFused = 320;           // + 4 measurement warps
constexpr int kRing = 4;                     // finished m-tiles queued for the measurement warps
constexpr int kBarrierBytes = 2048;          // mbarriers, ring, measurement staging
constexpr uint32_t kYStageBytes = 16384;     // one 128 x 32 FP32 chunk of the scratch tile (two buffers)
constexpr uint32_t kTmemCols = 512;          // 2 accumulators x 256 columns
constexpr uint32_t kAccStride = 256;
constexpr uint32_t kATileBytes = kBM * kBK * 2;  // 16 KB
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 232448;           // 227 KB opt-in per block

struct TcParams {
    int num_m_tiles, num_n_tiles, num_k_blocks, bn;
    int a_planes, b_planes, stages, nprod;
    uint32_t prod_code;  // product q uses A plane (code >> 4q) & 3 and B plane (code >> (4q+2)) & 3
    int tma_store;       // epilogue stages 128 x 32 chunks in shared memory and stores them with TMA
    uint32_t stage_bytes, b_plane_bytes;
    int row0;
    uint32_t idesc;
    float *Y;
    int64_t ldY;
    float *P;
    int ldP;
    int rows_valid;
    int *err;
    // fused measurement
    MeasureArgs m;
};

// Named barriers among a subset of warps.  The non-.aligned forms are used
// because lanes of one warp may reach them at different times.
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads: a
// group decides together whether to leave a loop, so no thread is left
// waiting at a later barrier for a thread that already left.
__device__ __forceinline__ bool named_bar_any(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

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

// The block's i-th tile.  Unfused: tiles are dealt round-robin in n-fastest
// order.  Fused: the block owns m-tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and visits all n-tiles of each (i % num_n_tiles == num_n_tiles - 1 ends an
// m-tile).  Returns false past the last tile.
template <bool kFused>
__device__ __forceinline__ bool tile_of(const TcParams &p, int i, int &mt, int &nt) {
    if (kFused) {
        const int q = i / p.num_n_tiles;
        nt = i - q * p.num_n_tiles;
        mt = blockIdx.x + q * gridDim.x;
        return mt < p.num_m_tiles;
    }
    const int tile = blockIdx.x + i * gridDim.x;
    mt = tile / p.num_n_tiles;
    nt = tile - mt * p.num_n_tiles;
    return tile < p.num_m_tiles * p.num_n_tiles;
}

template <bool kFused, bool kFp8>
__global__ void __launch_bounds__(kFused ? kThreadsFused : kThreads, 1)
tc_contract_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB0,
                   const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmY,
                   const TcParams p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

    uint8_t *ystage = smem + (size_t)p.stages * p.stage_bytes;  // 2 x 16 KB when p.tma_store
    uint64_t *full = reinterpret_cast<uint64_t *>(ystage + (p.tma_store ? 2 * kYStageBytes : 0u));
    uint64_t *empty = full + p.stages;
    uint64_t *tfull = empty + p.stages;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint64_t *mfull = drain + 1;     // [kRing] m-tile handed to the measurement warps
    uint64_t *mempty = mfull + kRing;
    int *mt_slot = reinterpret_cast<int *>(mempty + kRing);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mt_slot + kRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *m_sstar = reinterpret_cast<int *>(tmem_slot + 4);   // [128]
    float *m_scale = reinterpret_cast<float *>(m_sstar + kBM);  // [128]

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
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&mfull[r], 1);
            mbar_init(&mempty[r], kBM);
        }
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

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last_parity[s] = -1;
            bool failed = false;
            int mt, nt;
            for (int i = 0; !failed && tile_of<kFused>(p, i, mt, nt); ++i) {
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
                    const int x = kb * (kFp8 ? 2 * kBK : kBK);  // 128-byte rows: 64 BF16 or 128 FP8
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
            int mt, nt;
            for (int i = 0; !failed && tile_of<kFused>(p, i, mt, nt); ++i, ++lt) {
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
                            // (16 BF16 or 32 FP8 elements per MMA)
                            if (kFp8)
                                tc_mma_f8(d_tmem, ad + (uint64_t)(2 * k16), bd + (uint64_t)(2 * k16), p.idesc,
                                          (kb | q | k16) != 0 ? 1u : 0u);
                            else
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
    } else if (warp < 6) {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;  // tensor-memory lane quarter this warp may access
        int lt = 0;
        int ring = 0;               // (fused) next ring slot and its phase, tracked by thread 64
        uint32_t ring_phase = 0;
        int mt, nt;
        int chunk = 0;  // chunks staged so far (alternating staging buffers)
        const bool group_sync = kFused || p.tma_store;
        for (int i = 0; tile_of<kFused>(p, i, mt, nt); ++i, ++lt) {
            const int buf = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            const bool ready = mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag);
            if (group_sync ? named_bar_any(1, 128, !ready) : !ready) {
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
                if (!kFused && p.tma_store) {
                    // stage the 128 x 32 chunk (row = TMEM lane) with the 128-byte swizzle the tensor
                    // map expects, then one thread stores it with TMA
                    uint8_t *sb = ystage + (uint32_t)(chunk & 1) * kYStageBytes;
                    if (threadIdx.x == 64) bulk_wait_read_1();  // the store two chunks back has read sb
                    named_bar_sync(1, 128);
                    const int rl = quad * 32 + lane;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4 *>(sb + rl * 128 + ((j ^ (rl & 7)) * 16)) =
                            make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                        __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                    fence_proxy_async_smem();
                    named_bar_sync(1, 128);
                    if (threadIdx.x == 64) {
                        tma_store_2d(&tmY, sb, nt * p.bn + ch * 32, mt * kBM);
                        bulk_commit();
                    }
                    ++chunk;
                } else if (valid) {
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
            if (kFused && (i + 1) % p.num_n_tiles == 0) {
                // the m-tile is complete: the group barrier orders the 128 threads' stores before
                // the mbarrier arrive that hands the m-tile to the measurement warps
                named_bar_sync(1, 128);
                if (threadIdx.x == 64) {
                    if (!mbar_wait_bounded(&mempty[ring], ring_phase ^ 1u, abort_flag)) {
                        record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                    } else {
                        mt_slot[ring] = mt;
                        mbar_arrive(&mfull[ring]);
                        if (++ring == kRing) {
                            ring = 0;
                            ring_phase ^= 1u;
                        }
                    }
                }
                __syncwarp();
            }
        }
        if (!kFused && p.tma_store && threadIdx.x == 64) bulk_wait_all();  // scratch stores complete
        if (kFused && threadIdx.x == 64) {
            // no more m-tiles from this block: stop the measurement warps
            if (mbar_wait_bounded(&mempty[ring], ring_phase ^ 1u, abort_flag)) {
                mt_slot[ring] = -1;
                mbar_arrive(&mfull[ring]);
            }
        }
    } else if (kFused) {
        // ---------------- measurement: warps 6..9 ----------------
        const int m = threadIdx.x - 192;  // 0..127: the row of the m-tile this thread draws
        const int mw = m >> 5;
        int ring = 0;
        uint32_t ring_phase = 0;
        while (true) {
            const bool ready = mbar_wait_bounded(&mfull[ring], ring_phase, abort_flag);
            if (named_bar_any(2, 128, !ready)) {
                record_error(p.err, abort_flag, kDevTimeoutMeasure);
                break;
            }
            const int mt = mt_slot[ring];
            mbar_arrive(&mempty[ring]);
            if (++ring == kRing) {
                ring = 0;
                ring_phase ^= 1u;
            }
            if (mt < 0) break;
            const int row = mt * kBM + m;
            int sstar = 0;
            float scale = 0.f;
            if (row < p.rows_valid) sstar = measure_draw(p.m, row, &scale);
            m_sstar[m] = sstar;
            m_scale[m] = scale;
            named_bar_sync(2, 128);
            for (int j = 0; j < 32; ++j) {
                const int r = mt * kBM + mw * 32 + j;
                if (r >= p.rows_valid) break;
                const int sj = m_sstar[mw * 32 + j];
                const float *ysrc = p.Y + (int64_t)r * p.ldY + (int64_t)sj * p.m.Cs;
                measure_write_row(p.m, lane, ysrc, m_scale[mw * 32 + j], p.m.row0 + r);
            }
            named_bar_sync(2, 128);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

int stages_for(uint32_t stage_bytes, uint32_t extra = 0) {
    const int fixed = 1024 /* alignment */ + kBarrierBytes + (int)extra;
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
                               cudaStream_t st, const MeasureArgs *fused) {
    TcParams p;
    p.num_m_tiles = a.rows_pad / kBM;
    p.num_n_tiles = L.ncols / L.bn;
    p.num_k_blocks = L.K_pad / L.bk;
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
    p.b_plane_bytes = (uint32_t)L.bn * 128;  // bn rows of one 128-byte swizzle row
    p.stage_bytes = (uint32_t)a.a_planes * kATileBytes + (uint32_t)a.b_planes * p.b_plane_bytes;
    p.stages = stages_for(p.stage_bytes);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    // TMA-store epilogue when the staging buffers fit beside at least two pipeline stages
    p.tma_store = 0;
    if (a.has_tmY && !fused) {
        const int st2 = stages_for(p.stage_bytes, 2 * kYStageBytes);
        if (st2 >= 2) {
            p.stages = st2;
            p.tma_store = 1;
        }
    }
    p.row0 = (int)a.row0;
    p.idesc = a.fp8 ? idesc_e4m3_f32(kBM, L.bn) : idesc_bf16_f32(kBM, L.bn);
    if (a.fp8 && (fused || a.a_planes > 2 || a.b_planes != 1)) return cudaErrorInvalidValue;
    p.Y = o.Y;
    p.ldY = o.ldY;
    p.P = o.P;
    p.ldP = o.ldP;
    p.rows_valid = o.rows_valid;
    p.err = d_err;
    if (fused) {
        p.m = *fused;
    } else {
        p.m = MeasureArgs{};
    }
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + kBarrierBytes + (p.tma_store ? 2 * kYStageBytes : 0);
    const int units = fused ? p.num_m_tiles : p.num_m_tiles * p.num_n_tiles;  // fused blocks own m-tiles
    const int grid = units < num_sms ? units : num_sms;
    if (grid <= 0) return cudaSuccess;
    const CUtensorMap &a1 = a.tmA[a.a_planes > 1 ? 1 : 0], &a2 = a.tmA[a.a_planes > 2 ? 2 : 0];
    const CUtensorMap &b1 = a.tmB[a.b_planes > 1 ? 1 : 0];
    const CUtensorMap &ty = a.has_tmY ? a.tmY : a.tmA[0];  // unused when p.tma_store == 0
    cudaError_t e;
    if (a.fp8) {
        e = cudaFuncSetAttribute(tc_contract_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
        if (e != cudaSuccess) return e;
        tc_contract_kernel<false, true><<<grid, kThreads, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, ty, p);
    } else if (fused) {
        e = cudaFuncSetAttribute(tc_contract_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
        if (e != cudaSuccess) return e;
        tc_contract_kernel<true, false><<<grid, kThreadsFused, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, ty, p);
    } else {
        e = cudaFuncSetAttribute(tc_contract_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
        if (e != cudaSuccess) return e;
        tc_contract_kernel<false, false><<<grid, kThreads, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, ty, p);
    }
    return cudaGetLastError();
}

}  // namespace fastmps
