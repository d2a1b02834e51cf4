// Persistent batched contraction and measurement: many independent chains,
// every site, in one launch.
//
// The kernel is the tcgen05 contraction of tc_contract.cu (TMA producer warp,
// MMA warp, four epilogue warps, two TMEM accumulators) with four measurement
// warps, run over one task list: the tiles of every (job, chunk, site)
// segment in round order.  Each task looks up its segment (tensor maps in
// device memory, n-tile width, K extent, scratch pointers), so jobs with
// different bond dimensions, physical dimensions and row counts share the GPU
// in one launch; dependencies between consecutive sites of a job are kept per
// 128-row m-tile with counters in global memory.
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
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr uint32_t kATileBytes = 16384;      // 128 rows x 128 bytes
constexpr uint32_t kBPlaneBytesMax = 32768;  // 256 rows x 128 bytes
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 232448;

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

// ===========================================================================
// Persistent batched kernel: every round of every job in one launch.
//
// The tasks are the tiles of all segments of all rounds in round order.  The
// producer thread of each thread block takes the next task from a global
// counter (atomicAdd), so a block never waits on a task that no running block
// has taken: a task's predecessors come earlier in the order and have been
// taken already.  Before loading a task's left rows it waits -- bounded -- until
// the job's m-tile slot has been measured `step` times (the rows of chunk c at
// site k are written by the measurement of site k-1, and the chunk's scratch
// rows are free once the previous step's measurement has read them).  The
// epilogue stores the FP32 tile and its sums of squares and counts the finished
// tiles of the m-tile; the block that finishes the last one hands the m-tile to
// its four measurement warps, which draw, write the next left rows (Algorithm 2)
// and release the slot's counter.  Warps: 0 TMA producer, 1 MMA issuer, 2-5
// epilogue, 6-9 measurement (320 threads).
// ===========================================================================
constexpr int kPThreads = 320;
constexpr int kTaskRing = 16;
constexpr int kMRing = 4;
constexpr int kPBarrierBytes = 3072;

struct PParams {
    const PSegment *segs;
    const MeasureArgs *meas;
    int nseg;
    int64_t total_tasks;
    unsigned long long *queue;
    int *measured, *tiles_done;
    int stages, a_planes, b_planes, nprod;
    uint32_t prod_code, stage_bytes;
    uint64_t limit_ns;
    int stall;
    int *err;
};

// Last segment whose first task is <= t (segments ordered by task_begin).  A block takes tasks in
// increasing order, so the search gallops forward from the block's previous segment `from`.
__device__ __forceinline__ int psegment_of(const PParams &p, int64_t t, int from) {
    int lo = from, hi = from, step = 1;
    while (hi + 1 < p.nseg && p.segs[hi + 1].task_begin <= t) {
        lo = hi + 1;
        hi = hi + step < p.nseg - 1 ? hi + step : p.nseg - 1;
        step <<= 1;
        if (p.segs[hi].task_begin > t) break;
        lo = hi;
    }
    if (p.segs[hi].task_begin <= t) return hi;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.segs[mid].task_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Bounded wait for *cnt >= target (GPU-scope acquire).  Gives up early when any block has recorded
// an error; returns false then or when the limit runs out (*timed_out says which).
__device__ __forceinline__ bool wait_counter(const int *cnt, int target, const PParams &p, bool *timed_out) {
    *timed_out = false;
    if (ld_acquire_gpu(cnt) >= target) return true;
    const uint64_t t0 = global_ns();
    uint32_t iter = 0;
    while (ld_acquire_gpu(cnt) < target) {
        __nanosleep(100);
        if (((++iter) & 31u) == 0u) {
            if (*reinterpret_cast<volatile int *>(p.err) != 0) return false;
            if (global_ns() - t0 > p.limit_ns) {
                *timed_out = true;
                return false;
            }
        }
    }
    return true;
}

__global__ void __launch_bounds__(kPThreads, 1) tc_batch_persistent_kernel(const PParams p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * p.stage_bytes);
    uint64_t *empty = full + p.stages;
    uint64_t *tfull = empty + p.stages;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint64_t *task_full = drain + 1;            // [kTaskRing] task published by the producer
    uint64_t *task_empty = task_full + kTaskRing;  // [kTaskRing] read by the MMA thread and the epilogue
    uint64_t *mfull = task_empty + kTaskRing;    // [kMRing] m-tile handed to the measurement warps
    uint64_t *mempty = mfull + kMRing;
    int64_t *task_id = reinterpret_cast<int64_t *>(mempty + kMRing);  // [kTaskRing]
    int *task_seg = reinterpret_cast<int *>(task_id + kTaskRing);    // [kTaskRing]
    int *m_seg = task_seg + kTaskRing;                               // [kMRing]
    int *m_mt = m_seg + kMRing;                                      // [kMRing]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(m_mt + kMRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *m_sstar = reinterpret_cast<int *>(tmem_slot + 4);      // [128]
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
        for (int r = 0; r < kTaskRing; ++r) {
            mbar_init(&task_full[r], 1);
            mbar_init(&task_empty[r], 2);
        }
        for (int r = 0; r < kMRing; ++r) {
            mbar_init(&mfull[r], 1);
            mbar_init(&mempty[r], kBM);
        }
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
            // ---------------- TMA producer: takes tasks, waits for their left rows ----------------
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last_parity[s] = -1;
            bool failed = false;
            int seg_cursor = 0;
            for (int64_t seq = 0; !failed; ++seq) {
                const int slot = (int)(seq % kTaskRing);
                const uint32_t tpar = (uint32_t)((seq / kTaskRing) & 1);
                if (!mbar_wait_bounded(&task_empty[slot], tpar ^ 1u, abort_flag, p.limit_ns)) {
                    record_error(p.err, abort_flag, kDevTimeoutProducer);
                    break;
                }
                const int64_t t = (int64_t)atomicAdd(p.queue, 1ull);
                if (t >= p.total_tasks) {
                    task_id[slot] = -1;
                    mbar_arrive(&task_full[slot]);
                    break;
                }
                const int si = psegment_of(p, t, seg_cursor);
                seg_cursor = si;
                const PSegment *sg = &p.segs[si];
                const int64_t lt = t - sg->task_begin;
                const int mt = (int)(lt / sg->num_n_tiles);
                const int nt = (int)(lt - (int64_t)mt * sg->num_n_tiles);
                const int target = sg->step + p.stall;
                if (target > 0) {
                    bool timed_out;
                    if (!wait_counter(p.measured + sg->slot_base + mt, target, p, &timed_out)) {
                        if (timed_out) record_error(p.err, abort_flag, kDevTimeoutDependency);
                        else *abort_flag = 1;
                        break;
                    }
                    // the rows were written through the generic proxy by another block: order them
                    // before this thread's tensor-memory-access (async proxy) loads
                    fence_proxy_async_global();
                }
                task_id[slot] = t;
                task_seg[slot] = si;
                mbar_arrive(&task_full[slot]);
                const int y_a = sg->row0 + mt * kBM;
                const int y_b = nt * sg->bn;
                for (int kb = 0; kb < sg->num_k_blocks; ++kb) {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, p.limit_ns)) {
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
            if (*abort_flag)
                for (int s = 0; s < p.stages; ++s)
                    if (last_parity[s] >= 0) mbar_wait_drain(&full[s], (uint32_t)last_parity[s]);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            bool issued = false;
            for (int64_t seq = 0;; ++seq) {
                const int slot = (int)(seq % kTaskRing);
                if (!mbar_wait_bounded(&task_full[slot], (uint32_t)((seq / kTaskRing) & 1), abort_flag,
                                       p.limit_ns)) {
                    record_error(p.err, abort_flag, kDevTimeoutMma);
                    break;
                }
                const int64_t t = task_id[slot];
                const int si = task_seg[slot];
                mbar_arrive(&task_empty[slot]);
                if (t < 0) break;
                const PSegment *sg = &p.segs[si];
                const int buf = (int)(seq & 1);
                const uint32_t use = (uint32_t)(seq >> 1);
                if (!mbar_wait_bounded(&tempty[buf], (use & 1u) ^ 1u, abort_flag, p.limit_ns)) {
                    record_error(p.err, abort_flag, kDevTimeoutMma);
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)buf * kAccStride;
                const uint32_t idesc = sg->idesc;
                bool failed = false;
                for (int kb = 0; kb < sg->num_k_blocks; ++kb) {
                    if (!mbar_wait_bounded(&full[stage], phase, abort_flag, p.limit_ns)) {
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
                            tc_mma_bf16(d_tmem, ad + (uint64_t)(2 * k16), bd + (uint64_t)(2 * k16), idesc,
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
            if (*abort_flag && issued) {
                tc_commit(drain);
                mbar_wait_drain(drain, 0u);
            }
        }
        __syncwarp();
    } else if (warp < 6) {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;
        int ring = 0;
        uint32_t ring_phase = 0;
        for (int64_t seq = 0;; ++seq) {
            const int slot = (int)(seq % kTaskRing);
            const bool got = mbar_wait_bounded(&task_full[slot], (uint32_t)((seq / kTaskRing) & 1), abort_flag,
                                               p.limit_ns);
            if (named_bar_any(1, 128, !got)) {
                record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                break;
            }
            const int64_t t = task_id[slot];
            const int si = task_seg[slot];
            named_bar_sync(1, 128);  // every thread has read the slot
            if (threadIdx.x == 64) mbar_arrive(&task_empty[slot]);
            if (t < 0) break;
            const PSegment *sg = &p.segs[si];
            const int64_t lt = t - sg->task_begin;
            const int mt = (int)(lt / sg->num_n_tiles);
            const int nt = (int)(lt - (int64_t)mt * sg->num_n_tiles);
            const int buf = (int)(seq & 1);
            const uint32_t use = (uint32_t)(seq >> 1);
            const bool ready = mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag, p.limit_ns);
            if (named_bar_any(1, 128, !ready)) {
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
            // count the tile; the block that finishes the m-tile's last tile measures it
            named_bar_sync(1, 128);
            if (threadIdx.x == 64) {
                __threadfence();  // the group's stores (ordered by the barrier) before the count
                const int old = atomicAdd(p.tiles_done + sg->done_base + mt, 1);
                if (old == sg->num_n_tiles - 1) {
                    __threadfence();  // every block's tiles of this m-tile before the measurement reads them
                    if (!mbar_wait_bounded(&mempty[ring], ring_phase ^ 1u, abort_flag, p.limit_ns)) {
                        record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                    } else {
                        m_seg[ring] = si;
                        m_mt[ring] = mt;
                        mbar_arrive(&mfull[ring]);
                        if (++ring == kMRing) {
                            ring = 0;
                            ring_phase ^= 1u;
                        }
                    }
                }
            }
            __syncwarp();
        }
        if (threadIdx.x == 64) {
            // no more tiles from this block: stop the measurement warps
            if (mbar_wait_bounded(&mempty[ring], ring_phase ^ 1u, abort_flag, p.limit_ns)) {
                m_seg[ring] = -1;
                mbar_arrive(&mfull[ring]);
            }
        }
    } else {
        // ---------------- measurement: warps 6..9 ----------------
        const int m = threadIdx.x - 192;  // the row of the m-tile this thread draws
        const int mw = m >> 5;
        int ring = 0;
        uint32_t ring_phase = 0;
        while (true) {
            const bool ready = mbar_wait_bounded(&mfull[ring], ring_phase, abort_flag, p.limit_ns);
            if (named_bar_any(2, 128, !ready)) {
                record_error(p.err, abort_flag, kDevTimeoutMeasure);
                break;
            }
            const int si = m_seg[ring];
            const int mt = m_mt[ring];
            mbar_arrive(&mempty[ring]);
            if (++ring == kMRing) {
                ring = 0;
                ring_phase ^= 1u;
            }
            if (si < 0) break;
            const MeasureArgs &a = p.meas[si];
            const int rows = p.segs[si].rows_valid;
            const int row = mt * kBM + m;
            int sstar = 0;
            float scale = 0.f;
            if (row < rows) sstar = measure_draw(a, row, &scale);
            m_sstar[m] = sstar;
            m_scale[m] = scale;
            named_bar_sync(2, 128);
            for (int j = 0; j < 32; ++j) {
                const int r = mt * kBM + mw * 32 + j;
                if (r >= rows) break;
                const int sj = m_sstar[mw * 32 + j];
                const float *ysrc = a.Y + (int64_t)r * a.ldY + (int64_t)sj * a.Cs;
                measure_write_row(a, lane, ysrc, m_scale[mw * 32 + j], a.row0 + r);
            }
            named_bar_sync(2, 128);  // the m-tile's next left rows are written
            if (threadIdx.x == 192) {
                fence_proxy_async_global();
                red_release_add_gpu(p.measured + p.segs[si].slot_base + mt, 1);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

cudaError_t prepare_batch_persistent() {
    return cudaFuncSetAttribute(tc_batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

cudaError_t launch_batch_persistent(const PersistentArgs &g, int num_sms, int *d_err, cudaStream_t st) {
    if (g.nseg <= 0 || g.total_tasks <= 0) return cudaSuccess;
    if (g.nprod < 1 || g.nprod > kMaxProducts || g.a_planes < 1 || g.a_planes > 3 || g.b_planes < 1 ||
        g.b_planes > 2)
        return cudaErrorInvalidValue;
    PParams p;
    p.segs = g.segs;
    p.meas = g.meas;
    p.nseg = g.nseg;
    p.total_tasks = g.total_tasks;
    p.queue = reinterpret_cast<unsigned long long *>(g.queue);
    p.measured = g.measured;
    p.tiles_done = g.tiles_done;
    p.a_planes = g.a_planes;
    p.b_planes = g.b_planes;
    p.nprod = g.nprod;
    p.prod_code = 0;
    for (int q = 0; q < g.nprod; ++q)
        p.prod_code |= ((uint32_t)g.prod_a[q] | ((uint32_t)g.prod_b[q] << 2)) << (4 * q);
    p.stage_bytes = (uint32_t)g.a_planes * kATileBytes + (uint32_t)g.b_planes * kBPlaneBytesMax;
    p.stages = (kSmemLimit - 1024 - kPBarrierBytes) / (int)p.stage_bytes;
    if (p.stages > kMaxStages) p.stages = kMaxStages;
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    p.limit_ns = g.wait_limit_ns;
    p.stall = g.stall_test ? 1 : 0;
    p.err = d_err;
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + kPBarrierBytes;
    const int grid = g.total_tasks < num_sms ? (int)g.total_tasks : num_sms;
    tc_batch_persistent_kernel<<<grid, kPThreads, smem, st>>>(p);
    return cudaGetLastError();
}


}  // namespace fastmps
