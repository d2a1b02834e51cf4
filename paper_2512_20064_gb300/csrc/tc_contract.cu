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
// Cluster variant (single pass, no scratch): a thread-block cluster of C CTAs
// covers one m-tile's whole row, CTA rank r computing n-tiles r*T .. r*T+T-1
// and keeping their accumulators in tensor memory.  The epilogue warps square
// and sum their tiles per row, publish the 128 per-tile sums in shared memory
// and signal every CTA of the cluster through a remote mbarrier arrive; each
// CTA then reads all C*T partial sums of its rows through distributed shared
// memory, combines them in FP64 in tile order (the same sums, in the same
// order, as the two-pass measurement), draws the outcome -- identically in
// every CTA -- and writes the columns of the selected block it holds,
// scaled by 1/sqrt(w_{s*}), as BF16 planes of the next left row (Algorithm 2
// fused after the contraction; Sec. 3.3.1 per-sample scaling).  Rank 0 writes
// the outcome, log-probability and trace.  Nothing but the next left rows
// leaves the chip.
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
constexpr int kMaxClusterTiles = 32;         // cluster variant: n-tiles per m-tile (C * T)
constexpr int kMaxClusterCTAs = 16;          // largest (non-portable) cluster
constexpr uint32_t kClusterBytes = 64 + 4 * 128 * 4 * 2;  // 4 mbarriers + partial sums [2][T <= 4][128]

enum TcMode : int { kTwoPass = 0, kFusedCta = 1, kClusterFused = 2, kSplitK = 3, kPromoted = 4 };
// Promoted accumulation: warpgroup 0 = TMA, MMA and two idle warps; warpgroups 1 and 2 = 8 epilogue
// warps (two per tensor-memory lane quarter), each thread keeping a 128-column FP32 running sum.  Three
// warps per SM sub-partition cap the launch at 168 registers per thread; warpgroup 0 returns registers
// so that the epilogue warps can hold their sums without spilling.
constexpr int kThreadsPromoted = 384;
constexpr int kPromoRegsLaunch = 168;        // 65536 / (3 warps x 32 threads x 4 sub-partitions), rounded to 8
constexpr int kPromoRegsCtl = 72;            // warpgroup 0 after setmaxnreg.dec
constexpr int kPromoRegsEpi = 216;           // warpgroups 1 and 2 after setmaxnreg.inc
static_assert(kPromoRegsCtl * 128 + kPromoRegsEpi * 256 <= kPromoRegsLaunch * kThreadsPromoted,
              "register shares exceed the launch total");
static_assert((kPromoRegsCtl + 2 * kPromoRegsEpi) * 32 <= 16384, "one sub-partition's register file");

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
    int cl_T;  // cluster variant: n-tiles per CTA per m-tile (the cluster has num_n_tiles / cl_T CTAs)
    int ksplit;  // split-K variant: CTAs per cluster, each accumulating 1/ksplit of the k-blocks
    int kchunk;  // promoted accumulation: k-blocks per tensor-memory accumulator (n-tile of 128 columns)
    // fused measurement
    MeasureArgs m;
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

// The block's i-th tile.  Unfused: tiles are dealt round-robin in n-fastest
// order.  Fused: the block owns m-tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and visits all n-tiles of each (i % num_n_tiles == num_n_tiles - 1 ends an
// m-tile).  Cluster: the cluster owns m-tiles clusterid, clusterid + nclusters,
// ... and CTA rank r visits n-tiles r*T .. r*T+T-1 of each.  Returns false past
// the last tile.
template <int kMode>
__device__ __forceinline__ bool tile_of(const TcParams &p, int i, int &mt, int &nt) {
    if (kMode == kClusterFused) {
        const int q = i / p.cl_T;
        nt = (int)cluster_ctarank() * p.cl_T + (i - q * p.cl_T);
        mt = (int)cluster_id_x() + q * (int)cluster_count_x();
        return mt < p.num_m_tiles;
    }
    if (kMode == kSplitK) {
        const int tile = (int)cluster_id_x() + i * (int)cluster_count_x();
        mt = tile / p.num_n_tiles;
        nt = tile - mt * p.num_n_tiles;
        return tile < p.num_m_tiles * p.num_n_tiles;
    }
    if (kMode == kFusedCta) {
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

// ---------------------------------------------------------------------------
// Cluster variant: draw of one row from the partial sums of squares of all
// n-tiles of the row (pv[j] = sum over tile j, tiles in column order), exactly
// as measure_draw does from the scratch P: w_s in FP64 in tile order, Z, the
// Philox threshold, s* and log(w_{s*} / Z) in FP64.  The writer CTA (rank 0)
// stores the outcome, the log-probability and the trace.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cluster_draw(const MeasureArgs &a, int row, const float *pv, bool writer,
                                            float *scale_out) {
    const int T = a.tiles_per_s;
    double Z = 0.0;
    for (int s = 0; s < a.d; ++s) {
        double acc = 0.0;
        for (int j = 0; j < T; ++j) acc += (double)pv[s * T + j];
        Z += acc;
    }
    const uint64_t n = a.n_base + (uint64_t)row;
    const double t = sample_uniform(a.seed, n, a.k, a.job) * Z;
    double C = 0.0, ws = 0.0;
    int sstar = a.d - 1;
    for (int s = 0; s < a.d; ++s) {
        double acc = 0.0;
        for (int j = 0; j < T; ++j) acc += (double)pv[s * T + j];
        C += acc;
        if (s == a.d - 1 || C >= t) {
            sstar = s;
            ws = acc;
            break;
        }
    }
    const bool ok = (Z > 0.0) && isfinite(Z) && (ws > 0.0);
    if (writer) {
        const int64_t grow = a.row0 + row;
        a.outcomes[row] = (uint8_t)sstar;
        if (ok) a.logp[grow] += log(ws / Z);
        else atomicExch(a.err, (int)kDevNumeric);
        const int64_t slot = a.trace ? (a.trace_slot ? (int64_t)a.trace_slot[grow] : (grow < a.trace_rows ? grow : -1))
                                     : -1;
        if (slot >= 0) {
            for (int s = 0; s < a.d; ++s) {
                double acc = 0.0;
                for (int j = 0; j < T; ++j) acc += (double)pv[s * T + j];
                a.trace[slot * a.d + s] = ok ? acc / Z : 0.0;
            }
        }
    }
    *scale_out = ok ? rsqrtf((float)ws) : 0.f;
    return sstar;
}

// 32 consecutive entries (columns c0 .. c0+31 of the selected block, c0 a multiple of 32) of one next
// left row: value * scale, zero at and beyond 2 chi_r, as BF16 planes of successive residuals.
__device__ __forceinline__ void write_row_chunk(const MeasureArgs &a, int64_t grow, int c0, const uint32_t (&r)[32],
                                                float scale) {
    const int nreal = 2 * a.chi_r;
    __nv_bfloat16 *d0 = a.Vp[0] + grow * a.ld_next + c0;
    __nv_bfloat16 *d1 = a.Vp[1] + grow * a.ld_next + c0;
    __nv_bfloat16 *d2 = a.nplanes > 2 ? a.Vp[2] + grow * a.ld_next + c0 : nullptr;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = 8 * g + e;
            const float x = (c0 + j < nreal) ? __uint_as_float(r[j]) * scale : 0.f;
            write_planes(x, a.nplanes, p0[e], p1[e], p2[e]);
        }
        *reinterpret_cast<uint4 *>(d0 + 8 * g) = *reinterpret_cast<const uint4 *>(p0);
        *reinterpret_cast<uint4 *>(d1 + 8 * g) = *reinterpret_cast<const uint4 *>(p1);
        if (d2) *reinterpret_cast<uint4 *>(d2 + 8 * g) = *reinterpret_cast<const uint4 *>(p2);
    }
}

// Epilogue warps (2..5) of the cluster variant.  part: [2][cl_T][128] partial sums of this CTA;
// pready[b] / pfree[b]: count = cluster size, one remote arrive per CTA (b = m-tile parity).
__device__ __forceinline__ void cluster_epilogue(const TcParams &p, uint32_t tmem_base, uint64_t *tfull,
                                                 uint64_t *tempty, uint64_t *pready, uint64_t *pfree, float *part,
                                                 volatile int *abort_flag, int warp, int lane) {
    const int quad = warp & 3;  // tensor-memory lane quarter this warp may access
    const int r = quad * 32 + lane;
    const int T = p.cl_T;
    const int NT = p.num_n_tiles;
    const uint32_t C = (uint32_t)(NT / T);
    const uint32_t rank = cluster_ctarank();
    const int cid = (int)cluster_id_x(), ncl = (int)cluster_count_x();
    const MeasureArgs &a = p.m;
    const int tps = a.tiles_per_s;
    const uint32_t part_addr = smem_u32(part);
    int lt = 0;
    for (int u = 0;; ++u) {
        const int mt = cid + u * ncl;
        if (mt >= p.num_m_tiles) break;
        const int slot = u & 1;
        const uint32_t use = (uint32_t)(u >> 1);
        // this slot's partial sums may be overwritten once every CTA has read them (two m-tiles back)
        if (use >= 1) {
            const bool ok = mbar_wait_cluster_bounded(&pfree[slot], (use - 1) & 1u, abort_flag);
            if (named_bar_any(1, 128, !ok)) {
                record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                return;
            }
        }
        // 1. sums of squares of this CTA's tiles, same order as the two-pass epilogue
        for (int t = 0; t < T; ++t) {
            const int buf = (lt + t) & 1;
            const uint32_t tuse = (uint32_t)((lt + t) >> 1);
            const bool ready = mbar_wait_bounded(&tfull[buf], tuse & 1u, abort_flag);
            if (named_bar_any(1, 128, !ready)) {
                record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                return;
            }
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * kAccStride;
            float ss = 0.f;
            for (int ch = 0; ch < p.bn / 32; ++ch) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(taddr + (uint32_t)(ch * 32), v);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float x = __uint_as_float(v[j]);
                    ss = fmaf(x, x, ss);
                }
            }
            part[(slot * T + t) * 128 + r] = ss;
        }
        // 2. publish to every CTA of the cluster, then gather all partial sums of the row
        named_bar_sync(1, 128);
        if (threadIdx.x == 64) {
            const uint32_t bar = smem_u32(&pready[slot]);
            for (uint32_t c = 0; c < C; ++c) mbar_arrive_cluster(mapa_shared(bar, c));
        }
        const bool all = mbar_wait_cluster_bounded(&pready[slot], use & 1u, abort_flag);
        if (named_bar_any(1, 128, !all)) {
            record_error(p.err, abort_flag, kDevTimeoutEpilogue);
            return;
        }
        float pv[kMaxClusterTiles];
#pragma unroll
        for (int j = 0; j < kMaxClusterTiles; ++j) {
            if (j < NT) {
                const uint32_t owner = (uint32_t)(j / T);
                const int t = j - (int)owner * T;
                pv[j] = ld_shared_cluster_f32(mapa_shared(part_addr + (uint32_t)(((slot * T + t) * 128 + r) * 4), owner));
            }
        }
        named_bar_sync(1, 128);
        if (threadIdx.x == 64) {
            const uint32_t bar = smem_u32(&pfree[slot]);
            for (uint32_t c = 0; c < C; ++c) mbar_arrive_cluster(mapa_shared(bar, c));
        }
        // 3. the draw, identical in every CTA of the cluster
        const int row = mt * kBM + r;
        const bool valid = row < p.rows_valid;
        int sstar = -1;
        float scale = 0.f;
        if (valid) sstar = cluster_draw(a, row, pv, rank == 0, &scale);
        // 4. this CTA's columns of the selected block
        for (int t = 0; t < T; ++t) {
            const int j = (int)rank * T + t;
            const int s_here = j / tps;
            const int col0 = (j - s_here * tps) * p.bn;
            const bool mine = valid && sstar == s_here;
            if (!__any_sync(0xffffffffu, mine)) continue;  // tensor-memory loads are warp-collective
            const int buf = (lt + t) & 1;
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * kAccStride;
            for (int ch = 0; ch < p.bn / 32; ++ch) {
                const int c0 = col0 + ch * 32;
                if (c0 >= a.K_next) break;
                uint32_t v[32];
                tmem_ld_32x32b_x32(taddr + (uint32_t)(ch * 32), v);
                tc_wait_ld();
                if (mine) write_row_chunk(a, a.row0 + row, c0, v, scale);
            }
        }
        tc_fence_before();
        for (int t = 0; t < T; ++t) mbar_arrive(&tempty[(lt + t) & 1]);
        lt += T;
    }
}

// ---------------------------------------------------------------------------
// Split-K variant: a cluster of S CTAs computes one output tile, CTA rank j
// accumulating k-blocks [j*nkb/S, (j+1)*nkb/S) in its own tensor memory.  Ranks
// j >= 1 stage each 128 x 32 chunk of their partial tile in shared memory (the
// swizzled layout of the scratch store) and signal rank 0 with a remote
// mbarrier arrive; rank 0 adds the partial chunks to its own through
// distributed shared memory (rank order), releases the staging buffer, and
// stores the sum and the row's sum of squares like the two-pass epilogue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ld_shared_cluster_v4(uint32_t cluster_addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(cluster_addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ void splitk_epilogue(const TcParams &p, const CUtensorMap *tmY, uint32_t tmem_base,
                                                uint64_t *tfull, uint64_t *tempty, uint64_t *chunk_ready,
                                                uint64_t *chunk_free, uint8_t *ystage, volatile int *abort_flag,
                                                int warp, int lane) {
    const int quad = warp & 3;
    const int rl = quad * 32 + lane;  // row of the tile (tensor-memory lane)
    const uint32_t rank = cluster_ctarank();
    const uint32_t S = (uint32_t)p.ksplit;
    const uint32_t ystage_addr = smem_u32(ystage);
    int lt = 0;
    uint32_t q = 0;  // chunks handled so far (staging buffer q & 1)
    int mt, nt;
    for (int i = 0; tile_of<kSplitK>(p, i, mt, nt); ++i, ++lt) {
        const int buf = lt & 1;
        const uint32_t use = (uint32_t)(lt >> 1);
        const bool ready = mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag);
        if (named_bar_any(1, 128, !ready)) {
            record_error(p.err, abort_flag, kDevTimeoutEpilogue);
            return;
        }
        tc_fence_after();
        const int row = mt * kBM + rl;
        const bool valid = row < p.rows_valid;
        const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * kAccStride;
        float ss = 0.f;
        for (int ch = 0; ch < p.bn / 32; ++ch, ++q) {
            const uint32_t sbuf = q & 1u, sphase = (q >> 1) & 1u;
            uint8_t *sb = ystage + sbuf * kYStageBytes;
            uint32_t r[32];
            tmem_ld_32x32b_x32(taddr + (uint32_t)(ch * 32), r);
            tc_wait_ld();
            if (rank != 0) {
                // stage this rank's partial chunk once rank 0 has consumed the buffer's previous chunk
                if (q >= 2) {
                    const bool fr = mbar_wait_cluster_bounded(&chunk_free[sbuf], sphase ^ 1u, abort_flag);
                    if (named_bar_any(1, 128, !fr)) {
                        record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                        return;
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    *reinterpret_cast<float4 *>(sb + rl * 128 + ((j ^ (rl & 7)) * 16)) =
                        make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                    __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                named_bar_sync(1, 128);
                if (threadIdx.x == 64) mbar_arrive_cluster(mapa_shared(smem_u32(&chunk_ready[sbuf]), 0));
                continue;
            }
            // rank 0: add the other ranks' partial chunks in rank order
            if (S > 1) {
                const bool rd = mbar_wait_cluster_bounded(&chunk_ready[sbuf], sphase, abort_flag);
                if (named_bar_any(1, 128, !rd)) {
                    record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                    return;
                }
                for (uint32_t j = 1; j < S; ++j) {
                    const uint32_t base = mapa_shared(ystage_addr + sbuf * kYStageBytes, j);
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const float4 v = ld_shared_cluster_v4(base + (uint32_t)(rl * 128 + ((g ^ (rl & 7)) * 16)));
                        r[4 * g] = __float_as_uint(__uint_as_float(r[4 * g]) + v.x);
                        r[4 * g + 1] = __float_as_uint(__uint_as_float(r[4 * g + 1]) + v.y);
                        r[4 * g + 2] = __float_as_uint(__uint_as_float(r[4 * g + 2]) + v.z);
                        r[4 * g + 3] = __float_as_uint(__uint_as_float(r[4 * g + 3]) + v.w);
                    }
                }
                named_bar_sync(1, 128);  // every row's remote reads of this buffer are done
                if (threadIdx.x == 64)
                    for (uint32_t j = 1; j < S; ++j) mbar_arrive_cluster(mapa_shared(smem_u32(&chunk_free[sbuf]), j));
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float v = __uint_as_float(r[j]);
                ss = fmaf(v, v, ss);
            }
            // stage the summed chunk in this CTA's buffer and store it with TMA (as the two-pass epilogue)
            if (threadIdx.x == 64) bulk_wait_read_1();
            named_bar_sync(1, 128);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4 *>(sb + rl * 128 + ((j ^ (rl & 7)) * 16)) =
                    make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            fence_proxy_async_smem();
            named_bar_sync(1, 128);
            if (threadIdx.x == 64) {
                tma_store_2d(tmY, sb, nt * p.bn + ch * 32, mt * kBM);
                bulk_commit();
            }
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
        if (rank == 0 && valid) p.P[(int64_t)row * p.ldP + nt] = ss;
    }
    if (rank == 0 && threadIdx.x == 64) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Promoted accumulation: the MMA issuer accumulates every p.kchunk k-blocks of
// the contraction index into a fresh accumulator (two of 256 columns in
// rotation), and eight epilogue warps add the chunk sums in FP32 registers,
// rounding to nearest: warps w and w+4 share tensor-memory lane quarter w % 4
// (the tile's rows) and take the low and high 128 columns of the tile.  The
// tensor cores' accumulation then spans a few k-blocks only, where its partial
// sums are small, and the long sum over the whole index is taken with correctly
// rounded FP32 additions.  The tile is stored like the two-pass epilogue (TMA
// stores of 128 x 32 chunks, each half through its own staging buffer) and
// the row's sum of squares is the sum of the two halves' sums.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void promoted_epilogue(const TcParams &p, const CUtensorMap *tmY, uint32_t tmem_base,
                                                  uint64_t *tfull, uint64_t *tempty, uint8_t *ystage, float *ss_hi,
                                                  volatile int *abort_flag, int warp, int lane) {
    const int quad = warp & 3;
    const int half = (warp - 4) >> 2;        // 0: columns 0..127 of the tile, 1: columns 128..255
    const int rl = quad * 32 + lane;
    const int elected = half == 0 ? 128 : 256;  // first thread of each half
    const int nch = (p.num_k_blocks + p.kchunk - 1) / p.kchunk;
    uint8_t *sb = ystage + (uint32_t)half * kYStageBytes;  // this half's staging buffer
    uint32_t cq = 0;  // chunks consumed (buffer cq % 2)
    int mt, nt;
    for (int i = 0; tile_of<kPromoted>(p, i, mt, nt); ++i) {
        float acc[128];
        for (int c = 0; c < nch; ++c, ++cq) {
            const int buf = (int)(cq & 1u);
            const uint32_t use = cq >> 1;
            const bool ready = mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag);
            if (named_bar_any(1, 256, !ready)) {
                record_error(p.err, abort_flag, kDevTimeoutEpilogue);
                return;
            }
            tc_fence_after();
            const uint32_t taddr =
                tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * kAccStride + (uint32_t)(half * 128);
#pragma unroll
            for (int g = 0; g < 4; g += 2) {
                // two 32-column loads in flight per wait
                uint32_t r0[32], r1[32];
                tmem_ld_32x32b_x32(taddr + (uint32_t)(g * 32), r0);
                tmem_ld_32x32b_x32(taddr + (uint32_t)(g * 32 + 32), r1);
                tc_wait_ld();
                if (c == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        acc[g * 32 + j] = __uint_as_float(r0[j]);
                        acc[g * 32 + 32 + j] = __uint_as_float(r1[j]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        acc[g * 32 + j] += __uint_as_float(r0[j]);
                        acc[g * 32 + 32 + j] += __uint_as_float(r1[j]);
                    }
                }
            }
            // the warp's tensor-memory reads are complete: one arrive per warp frees the buffer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        const int row = mt * kBM + rl;
        float ss = 0.f;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
#pragma unroll
            for (int j = 0; j < 32; ++j) ss = fmaf(acc[g * 32 + j], acc[g * 32 + j], ss);
            if (threadIdx.x == elected) bulk_wait_read_0();  // this half's previous store has read sb
            named_bar_sync(2 + half, 128);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4 *>(sb + rl * 128 + ((j ^ (rl & 7)) * 16)) =
                    make_float4(acc[g * 32 + 4 * j], acc[g * 32 + 4 * j + 1], acc[g * 32 + 4 * j + 2],
                                acc[g * 32 + 4 * j + 3]);
            fence_proxy_async_smem();
            named_bar_sync(2 + half, 128);
            if (threadIdx.x == elected) {
                tma_store_2d(tmY, sb, nt * p.bn + half * 128 + g * 32, mt * kBM);
                bulk_commit();
            }
        }
        // the row's sum of squares: low half + high half
        if (half == 1) ss_hi[rl] = ss;
        named_bar_sync(1, 256);
        if (half == 0 && row < p.rows_valid) p.P[(int64_t)row * p.ldP + nt] = ss + ss_hi[rl];
        named_bar_sync(1, 256);  // ss_hi is free for the next tile
    }
    if (threadIdx.x == elected) bulk_wait_all();
}

template <int kMode, bool kFp8>
__global__ void __launch_bounds__(kMode == kFusedCta ? kThreadsFused : (kMode == kPromoted ? kThreadsPromoted : kThreads), 1)
tc_contract_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB0,
                   const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmY,
                   const TcParams p) {
    constexpr bool kFused = kMode == kFusedCta;
    constexpr bool kCluster = kMode == kClusterFused;
    constexpr bool kSplit = kMode == kSplitK;
    constexpr bool kPromo = kMode == kPromoted;
    // split-K: this CTA's share of the k-blocks
    const int kb_lo = kSplit ? (int)(cluster_ctarank() * (uint32_t)p.num_k_blocks / (uint32_t)p.ksplit) : 0;
    const int kb_hi = kSplit ? (int)((cluster_ctarank() + 1) * (uint32_t)p.num_k_blocks / (uint32_t)p.ksplit)
                             : p.num_k_blocks;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

    uint8_t *ystage = smem + (size_t)p.stages * p.stage_bytes;  // 2 x 16 KB when p.tma_store
    uint64_t *full = reinterpret_cast<uint64_t *>(ystage + (p.tma_store ? 2 * kYStageBytes : 0u));
    uint64_t *empty = full + p.stages;
    uint64_t *tfull = empty + p.stages;  // [4]: accumulator buffers (two 256-column, or four 128-column)
    uint64_t *tempty = tfull + 4;
    uint64_t *drain = tempty + 4;
    uint64_t *mfull = drain + 1;     // [kRing] m-tile handed to the measurement warps
    uint64_t *mempty = mfull + kRing;
    int *mt_slot = reinterpret_cast<int *>(mempty + kRing);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mt_slot + kRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *m_sstar = reinterpret_cast<int *>(tmem_slot + 4);   // [128]
    float *m_scale = reinterpret_cast<float *>(m_sstar + kBM);  // [128]
    // cluster variant: behind the barrier region
    uint64_t *pready = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(full) + kBarrierBytes);  // [2]
    uint64_t *pfree = pready + 2;                                                                      // [2]
    float *part = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(pready) + 64);  // [2][cl_T][128]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kPromo ? 8 : 128);  // promoted: one arrive per epilogue warp
        }
        mbar_init(drain, 1);
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&mfull[r], 1);
            mbar_init(&mempty[r], kBM);
        }
        if (kCluster) {
            const uint32_t csize = (uint32_t)(p.num_n_tiles / p.cl_T);  // one arrive from every CTA
            for (int b = 0; b < 2; ++b) {
                mbar_init(&pready[b], csize);
                mbar_init(&pfree[b], csize);
            }
        }
        if (kSplit) {  // pready: a chunk staged by every other rank (rank 0); pfree: buffer consumed (ranks > 0)
            for (int b = 0; b < 2; ++b) {
                mbar_init(&pready[b], p.ksplit > 1 ? (uint32_t)(p.ksplit - 1) : 1u);
                mbar_init(&pfree[b], 1);
            }
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
    // cluster variants: every CTA's barriers are initialised before any remote arrive
    if (kCluster || kSplit) cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // ---------------- TMA producer (warp 0) ----------------
    auto run_producer = [&]() {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) last_parity[s] = -1;
            bool failed = false;
            int mt, nt;
            for (int i = 0; !failed && tile_of<kMode>(p, i, mt, nt); ++i) {
                const int y_a = p.row0 + mt * kBM;
                const int y_b = nt * p.bn;
                for (int kb = kb_lo; kb < kb_hi; ++kb) {
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
    };
    // ---------------- MMA issuer (warp 1) ----------------
    auto run_mma = [&]() {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int lt = 0;
            bool failed = false;
            bool issued = false;
            int mt, nt;
            uint32_t cq = 0;  // promoted accumulation: chunks issued so far (buffer cq % 2)
            for (int i = 0; !failed && tile_of<kMode>(p, i, mt, nt); ++i, ++lt) {
                int buf = lt & 1;
                uint32_t d_tmem = 0;
                if (!kPromo) {
                    const uint32_t use = (uint32_t)(lt >> 1);
                    if (!mbar_wait_bounded(&tempty[buf], (use & 1u) ^ 1u, abort_flag)) {
                        record_error(p.err, abort_flag, kDevTimeoutMma);
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    d_tmem = tmem_base + (uint32_t)buf * kAccStride;
                }
                for (int kb = kb_lo; kb < kb_hi; ++kb) {
                    const int kin = kPromo ? (kb - kb_lo) % p.kchunk : kb - kb_lo;  // k-block within the accumulator
                    if (kPromo && kin == 0) {
                        // a fresh 128-column accumulator for the next chunk of the contraction index
                        buf = (int)(cq & 1u);
                        const uint32_t use = cq >> 1;
                        if (!mbar_wait_bounded(&tempty[buf], (use & 1u) ^ 1u, abort_flag)) {
                            record_error(p.err, abort_flag, kDevTimeoutMma);
                            failed = true;
                            break;
                        }
                        tc_fence_after();
                        d_tmem = tmem_base + (uint32_t)buf * kAccStride;
                    }
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
                            const uint32_t acc = (kin | q | k16) != 0 ? 1u : 0u;
                            if (kFp8)
                                tc_mma_f8(d_tmem, ad + (uint64_t)(2 * k16), bd + (uint64_t)(2 * k16), p.idesc, acc);
                            else
                                tc_mma_bf16(d_tmem, ad + (uint64_t)(2 * k16), bd + (uint64_t)(2 * k16), p.idesc, acc);
                        }
                    }
                    issued = true;
                    tc_commit(&empty[stage]);
                    if (++stage == p.stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    if (kPromo && (kin == p.kchunk - 1 || kb == kb_hi - 1)) {
                        tc_commit(&tfull[buf]);
                        ++cq;
                    }
                }
                if (failed) break;
                if (!kPromo) tc_commit(&tfull[buf]);
            }
            if (failed && issued) {
                // wait for this thread's outstanding MMAs before tensor memory is freed
                tc_commit(drain);
                mbar_wait_drain(drain, 0u);
            }
        }
        __syncwarp();
    };

    if (kPromo) {
        // each warpgroup sets its register budget before its warps take their roles
        if (warp < 4) {
            setmaxnreg_dec<kPromoRegsCtl>();
            if (warp == 0)
                run_producer();
            else if (warp == 1)
                run_mma();
        } else {
            setmaxnreg_inc<kPromoRegsEpi>();
            // ---------------- promoted-accumulation epilogue: warps 4..11 ----------------
            promoted_epilogue(p, &tmY, tmem_base, tfull, tempty, ystage, m_scale, abort_flag, warp, lane);
        }
    } else if (warp == 0) {
        run_producer();
    } else if (warp == 1) {
        run_mma();
    } else if (kCluster && warp < 6) {
        // ---------------- cluster epilogue: warps 2..5 ----------------
        cluster_epilogue(p, tmem_base, tfull, tempty, pready, pfree, part, abort_flag, warp, lane);
    } else if (kSplit && warp < 6) {
        // ---------------- split-K epilogue: warps 2..5 ----------------
        splitk_epilogue(p, &tmY, tmem_base, tfull, tempty, pready, pfree, ystage, abort_flag, warp, lane);
    } else if (warp < 6) {
        // ---------------- epilogue: warps 2..5 ----------------
        const int quad = warp & 3;  // tensor-memory lane quarter this warp may access
        int lt = 0;
        int ring = 0;               // (fused) next ring slot and its phase, tracked by thread 64
        uint32_t ring_phase = 0;
        int mt, nt;
        int chunk = 0;  // chunks staged so far (alternating staging buffers)
        const bool group_sync = kFused || p.tma_store;
        for (int i = 0; tile_of<kMode>(p, i, mt, nt); ++i, ++lt) {
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
    // cluster variants: no CTA leaves while another may still read its shared memory or arrive on its barriers
    if (kCluster || kSplit) cluster_sync_all();
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
    p.idesc = a.fp8 ? idesc_e4m3_f32(kBM, L.bn) : (a.f16 ? idesc_f16_f32(kBM, L.bn) : idesc_bf16_f32(kBM, L.bn));
    if (a.fp8 && (fused || a.a_planes > 2 || a.b_planes != 1)) return cudaErrorInvalidValue;
    p.Y = o.Y;
    p.ldY = o.ldY;
    p.P = o.P;
    p.ldP = o.ldP;
    p.rows_valid = o.rows_valid;
    p.err = d_err;
    p.cl_T = 1;
    p.ksplit = 1;
    p.kchunk = 0;
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
        e = cudaFuncSetAttribute(tc_contract_kernel<kTwoPass, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
        if (e != cudaSuccess) return e;
        tc_contract_kernel<kTwoPass, true><<<grid, kThreads, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, ty, p);
    } else if (fused) {
        e = cudaFuncSetAttribute(tc_contract_kernel<kFusedCta, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
        if (e != cudaSuccess) return e;
        tc_contract_kernel<kFusedCta, false><<<grid, kThreadsFused, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, ty, p);
    } else {
        e = cudaFuncSetAttribute(tc_contract_kernel<kTwoPass, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
        if (e != cudaSuccess) return e;
        tc_contract_kernel<kTwoPass, false><<<grid, kThreads, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, ty, p);
    }
    return cudaGetLastError();
}

bool cluster_plan(const SiteLayout &L, int *C_out, int *T_out) {
    if (L.bn % 64 != 0 || L.ncols % L.bn != 0) return false;
    const int NT = L.ncols / L.bn;
    if (NT > kMaxClusterTiles || L.K_pad < 64) return false;
    // K_next <= Cs: the block's own columns cover the next row's padding up to its K extent
    if ((int)(((2 * (int64_t)L.chi_r) + 63) / 64 * 64) > L.Cs) return false;
    // the two 256-column accumulators hold all T tiles of an m-tile until its draw: T <= 2
    for (int T = 1; T <= 2; ++T) {
        if (NT % T != 0 || L.bn > (int)kAccStride || (T * 128 * 4 * 2) > (int)(kClusterBytes - 64)) continue;
        const int C = NT / T;
        if (C > kMaxClusterCTAs) continue;
        *C_out = C;
        *T_out = T;
        return true;
    }
    return false;
}

namespace {

// Launch configuration of the cluster kernel for a site layout and plane counts; returns the largest
// number of clusters that can be resident at once (0: the configuration cannot run).
int cluster_config(int a_planes, int b_planes, const SiteLayout &L, int C, cudaLaunchConfig_t &cfg,
                   cudaLaunchAttribute *attr, size_t *smem_out, int *stages_out) {
    const uint32_t stage_bytes = (uint32_t)a_planes * kATileBytes + (uint32_t)b_planes * (uint32_t)L.bn * 128;
    const int stages = stages_for(stage_bytes, kClusterBytes);
    if (stages < 2) return 0;
    const size_t smem = (size_t)stages * stage_bytes + 1024 + kBarrierBytes + kClusterBytes;
    auto kern = tc_contract_kernel<kClusterFused, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) != cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cfg = cudaLaunchConfig_t{};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)C);
    // resident clusters per (cluster size, shared-memory size), cached
    static int cache[kMaxClusterCTAs + 1][8] = {};
    const int sidx = (int)((smem >> 15) & 7);
    if (cache[C][sidx] == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        cache[C][sidx] = n > 0 ? n : -1;
    }
    *smem_out = smem;
    *stages_out = stages;
    return cache[C][sidx] > 0 ? cache[C][sidx] : 0;
}

}  // namespace

int cluster_capacity(int a_planes, int b_planes, const SiteLayout &L) {
    int C = 0, T = 0;
    if (!cluster_plan(L, &C, &T)) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    size_t smem = 0;
    int stages = 0;
    return cluster_config(a_planes, b_planes, L, C, cfg, attr, &smem, &stages);
}

cudaError_t launch_contract_tc_cluster(const TcArgs &a, const SiteLayout &L, int rows_valid, int *d_err,
                                       cudaStream_t st, const MeasureArgs &m, int *clusters_out) {
    int C = 0, T = 0;
    // FP16 rows are scaled by their largest entry, which no single CTA of the cluster sees
    if (a.fp8 || a.f16 || !cluster_plan(L, &C, &T)) return cudaErrorInvalidConfiguration;
    if (a.nprod < 1 || a.nprod > kMaxProducts || a.a_planes < 1 || a.a_planes > 3 || a.b_planes < 1 ||
        a.b_planes > 2 || m.nplanes != a.a_planes)
        return cudaErrorInvalidValue;
    TcParams p;
    p.num_m_tiles = a.rows_pad / kBM;
    p.num_n_tiles = L.ncols / L.bn;
    p.num_k_blocks = L.K_pad / L.bk;
    p.bn = L.bn;
    p.a_planes = a.a_planes;
    p.b_planes = a.b_planes;
    p.nprod = a.nprod;
    p.prod_code = 0;
    for (int q = 0; q < a.nprod; ++q) {
        if (a.prod_a[q] < 0 || a.prod_a[q] >= a.a_planes || a.prod_b[q] < 0 || a.prod_b[q] >= a.b_planes)
            return cudaErrorInvalidValue;
        p.prod_code |= ((uint32_t)a.prod_a[q] | ((uint32_t)a.prod_b[q] << 2)) << (4 * q);
    }
    p.b_plane_bytes = (uint32_t)L.bn * 128;
    p.stage_bytes = (uint32_t)a.a_planes * kATileBytes + (uint32_t)a.b_planes * p.b_plane_bytes;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    size_t smem = 0;
    const int max_clusters = cluster_config(a.a_planes, a.b_planes, L, C, cfg, attr, &smem, &p.stages);
    if (max_clusters <= 0) return cudaErrorInvalidConfiguration;
    p.tma_store = 0;
    p.row0 = (int)a.row0;
    p.idesc = a.f16 ? idesc_f16_f32(kBM, L.bn) : idesc_bf16_f32(kBM, L.bn);
    p.Y = nullptr;
    p.ldY = 0;
    p.P = nullptr;
    p.ldP = 0;
    p.rows_valid = rows_valid;
    p.err = d_err;
    p.cl_T = T;
    p.ksplit = 1;
    p.kchunk = 0;
    p.m = m;
    if (p.num_m_tiles <= 0) return cudaSuccess;
    (void)smem;
    // persistent: as many clusters as can be resident at once (at most one per m-tile)
    const int ncl = p.num_m_tiles < max_clusters ? p.num_m_tiles : max_clusters;
    if (clusters_out) *clusters_out = ncl;
    cfg.gridDim = dim3((unsigned)(ncl * C));
    cfg.stream = st;
    auto kern = tc_contract_kernel<kClusterFused, false>;
    cudaError_t e;
    const CUtensorMap &a1 = a.tmA[a.a_planes > 1 ? 1 : 0], &a2 = a.tmA[a.a_planes > 2 ? 2 : 0];
    const CUtensorMap &b1 = a.tmB[a.b_planes > 1 ? 1 : 0];
    e = cudaLaunchKernelEx(&cfg, kern, a.tmA[0], a1, a2, a.tmB[0], b1, a.tmA[0], p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_contract_tc_splitk(const TcArgs &a, const SiteLayout &L, const ContractOut &o, int ksplit,
                                      int *d_err, cudaStream_t st, int *clusters_out) {
    if (a.fp8 || !a.has_tmY || ksplit < 2 || ksplit > 8) return cudaErrorInvalidValue;
    if (a.nprod < 1 || a.nprod > kMaxProducts || a.a_planes < 1 || a.a_planes > 3 || a.b_planes < 1 ||
        a.b_planes > 2)
        return cudaErrorInvalidValue;
    TcParams p;
    p.num_m_tiles = a.rows_pad / kBM;
    p.num_n_tiles = L.ncols / L.bn;
    p.num_k_blocks = L.K_pad / L.bk;
    if (p.num_k_blocks < ksplit) return cudaErrorInvalidValue;
    p.bn = L.bn;
    p.a_planes = a.a_planes;
    p.b_planes = a.b_planes;
    p.nprod = a.nprod;
    p.prod_code = 0;
    for (int q = 0; q < a.nprod; ++q) {
        if (a.prod_a[q] < 0 || a.prod_a[q] >= a.a_planes || a.prod_b[q] < 0 || a.prod_b[q] >= a.b_planes)
            return cudaErrorInvalidValue;
        p.prod_code |= ((uint32_t)a.prod_a[q] | ((uint32_t)a.prod_b[q] << 2)) << (4 * q);
    }
    p.b_plane_bytes = (uint32_t)L.bn * 128;
    p.stage_bytes = (uint32_t)a.a_planes * kATileBytes + (uint32_t)a.b_planes * p.b_plane_bytes;
    p.stages = stages_for(p.stage_bytes, 2 * kYStageBytes + kClusterBytes);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    p.tma_store = 1;
    p.row0 = (int)a.row0;
    p.idesc = a.f16 ? idesc_f16_f32(kBM, L.bn) : idesc_bf16_f32(kBM, L.bn);
    p.Y = o.Y;
    p.ldY = o.ldY;
    p.P = o.P;
    p.ldP = o.ldP;
    p.rows_valid = o.rows_valid;
    p.err = d_err;
    p.cl_T = 1;
    p.ksplit = ksplit;
    p.kchunk = 0;
    p.m = MeasureArgs{};
    const int tiles = p.num_m_tiles * p.num_n_tiles;
    if (tiles <= 0) return cudaSuccess;
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + kBarrierBytes + 2 * kYStageBytes + kClusterBytes;
    auto kern = tc_contract_kernel<kSplitK, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ksplit;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)ksplit);
    int ncl_max = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl_max, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (ncl_max <= 0) return cudaErrorInvalidConfiguration;
    const int ncl = tiles < ncl_max ? tiles : ncl_max;
    if (clusters_out) *clusters_out = ncl;
    cfg.gridDim = dim3((unsigned)(ncl * ksplit));
    cfg.stream = st;
    const CUtensorMap &a1 = a.tmA[a.a_planes > 1 ? 1 : 0], &a2 = a.tmA[a.a_planes > 2 ? 2 : 0];
    const CUtensorMap &b1 = a.tmB[a.b_planes > 1 ? 1 : 0];
    e = cudaLaunchKernelEx(&cfg, kern, a.tmA[0], a1, a2, a.tmB[0], b1, a.tmY, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_contract_tc_promoted(const TcArgs &a, const SiteLayout &L, const ContractOut &o, int kchunk,
                                        int num_sms, int *d_err, cudaStream_t st) {
    if (a.fp8 || !a.has_tmY || L.bn != 256 || kchunk < 1) return cudaErrorInvalidValue;
    if (a.nprod < 1 || a.nprod > kMaxProducts || a.a_planes < 1 || a.a_planes > 3 || a.b_planes < 1 ||
        a.b_planes > 2)
        return cudaErrorInvalidValue;
    TcParams p;
    p.num_m_tiles = a.rows_pad / kBM;
    p.num_n_tiles = L.ncols / L.bn;
    p.num_k_blocks = L.K_pad / L.bk;
    p.bn = L.bn;
    p.a_planes = a.a_planes;
    p.b_planes = a.b_planes;
    p.nprod = a.nprod;
    p.prod_code = 0;
    for (int q = 0; q < a.nprod; ++q) {
        if (a.prod_a[q] < 0 || a.prod_a[q] >= a.a_planes || a.prod_b[q] < 0 || a.prod_b[q] >= a.b_planes)
            return cudaErrorInvalidValue;
        p.prod_code |= ((uint32_t)a.prod_a[q] | ((uint32_t)a.prod_b[q] << 2)) << (4 * q);
    }
    p.b_plane_bytes = (uint32_t)L.bn * 128;
    p.stage_bytes = (uint32_t)a.a_planes * kATileBytes + (uint32_t)a.b_planes * p.b_plane_bytes;
    p.stages = stages_for(p.stage_bytes, 2 * kYStageBytes);
    if (p.stages < 2) return cudaErrorInvalidConfiguration;
    p.tma_store = 1;
    p.row0 = (int)a.row0;
    p.idesc = a.f16 ? idesc_f16_f32(kBM, L.bn) : idesc_bf16_f32(kBM, L.bn);
    p.Y = o.Y;
    p.ldY = o.ldY;
    p.P = o.P;
    p.ldP = o.ldP;
    p.rows_valid = o.rows_valid;
    p.err = d_err;
    p.cl_T = 1;
    p.ksplit = 1;
    p.kchunk = kchunk < p.num_k_blocks ? kchunk : p.num_k_blocks;
    p.m = MeasureArgs{};
    const int tiles = p.num_m_tiles * p.num_n_tiles;
    if (tiles <= 0) return cudaSuccess;
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + kBarrierBytes + 2 * kYStageBytes;
    auto kern = tc_contract_kernel<kPromoted, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    // the epilogue warpgroups' register increase is served from the launch's own registers: refuse a
    // build whose launch count would leave the increase waiting
    static int regs = -1;
    if (regs < 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        regs = fa.numRegs;
    }
    if (regs * kThreadsPromoted < kPromoRegsCtl * 128 + kPromoRegsEpi * 256) return cudaErrorInvalidConfiguration;
    const int grid = tiles < num_sms ? tiles : num_sms;
    const CUtensorMap &a1 = a.tmA[a.a_planes > 1 ? 1 : 0], &a2 = a.tmA[a.a_planes > 2 ? 2 : 0];
    const CUtensorMap &b1 = a.tmB[a.b_planes > 1 ? 1 : 0];
    kern<<<grid, kThreadsPromoted, smem, st>>>(a.tmA[0], a1, a2, a.tmB[0], b1, a.tmY, p);
    return cudaGetLastError();
}

}  // namespace fastmps
