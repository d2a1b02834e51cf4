// fastmps_sample_batch: many independent MPS sampled together.
//
// Schedule.  Job j has M_j sites and N_j rows, processed in C_j chunks of at
// most N2_j rows (N2_j bounded by a shared FP32-scratch budget).  Round r
// advances every job with r < C_j * M_j by one step: chunk c = r / M_j at
// site k = r % M_j.  One persistent kernel runs every round of every job:
// its task list is the tiles of all segments (job, chunk, site) in round
// order, taken from a device counter, and a task waits (bounded) only for the
// measurement of its own job's rows at the previous step -- not for a whole
// round -- so rounds of different jobs overlap freely.  The segment table is
// built on the host and copied to device memory once; the call's launches
// (counter resets, left-boundary initialisation, the persistent kernel, the
// output transposes) are captured into a CUDA graph that later calls with the
// same job table replay.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/fastmps.h"
#include "common.cuh"
#include "handle_view.h"
#include "launch.h"

namespace fastmps {

namespace {

inline int64_t roundup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    bool host = false;
    ~Buf() { release(); }
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

struct JobBufs {
    Buf V[2][3], Y, P, logp, O, stage_out;
};

struct BatchState {
    std::vector<std::unique_ptr<JobBufs>> jobs;
    Buf segs_dev, meas_dev, segs_host, meas_host, err, counters;
    std::vector<uint64_t> signature;
    int64_t launches = 0;  // kernels of one replay of the graph
    cudaGraphExec_t graph = nullptr;
    ~BatchState() {
        if (graph) cudaGraphExecDestroy(graph);
    }
};

std::mutex g_batch_mutex;
std::map<fastmps_handle, std::unique_ptr<BatchState>> g_batch;

BatchState *state_of(fastmps_handle h) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    auto &p = g_batch[h];
    if (!p) p.reset(new BatchState());
    return p.get();
}

bool device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct JobPlan {
    int M, d, ldV, ncols_max, ldP_max;
    int64_t N, N_pad, N2, chunks, rounds;
};

// Test hook: FASTMPS_TEST_STALL_DEPENDENCY=1 makes every task wait for one measurement more than ever
// happens, with a 100 ms wait limit, so the persistent kernel's bounded waits run out.
bool stall_test_requested() {
    const char *v = getenv("FASTMPS_TEST_STALL_DEPENDENCY");
    return v && v[0] == '1';
}

}  // namespace

void batch_release(fastmps_handle h) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    g_batch.erase(h);
}

}  // namespace fastmps

using namespace fastmps;

extern "C" int fastmps_sample_batch(fastmps_handle runner, int count, const fastmps_job *jobs) {
    if (!runner) return FASTMPS_ERR_INVALID_ARG;
    auto t_start = std::chrono::steady_clock::now();
    HandleView rv;
    handle_view(runner, &rv);
    if (cudaSetDevice(rv.device) != cudaSuccess) return set_error(runner, FASTMPS_ERR_CUDA, "cudaSetDevice failed");
    fastmps_stats *stats = handle_stats(runner);
    *stats = fastmps_stats{};
    if (count < 0 || (count > 0 && !jobs)) return set_error(runner, FASTMPS_ERR_INVALID_ARG, "bad job table");
    if (rv.precision == FASTMPS_FP32 || rv.precision == FASTMPS_FP8X1 || rv.precision == FASTMPS_FP8X2 ||
        rv.precision == FASTMPS_FP16X2 || rv.precision == FASTMPS_FP16X3)
        return set_error(runner, FASTMPS_ERR_UNSUPPORTED, "batched sampling runs the BF16 tensor-core modes");
    char msg[256];
    int a_planes, b_planes, nprod, pa[kMaxProducts], pb[kMaxProducts];
    precision_products(rv.precision, &a_planes, &b_planes, &nprod, pa, pb);

    // ---- validate and plan -------------------------------------------------
    std::vector<JobPlan> plan(count);
    const int64_t budget = (int64_t)4 << 30;  // FP32 scratch shared by all jobs
    int64_t total_rows = 0;
    for (int j = 0; j < count; ++j) total_rows += std::max<int64_t>(0, jobs[j].N);
    int64_t R = 0;
    double flops = 0;
    for (int j = 0; j < count; ++j) {
        const fastmps_job &J = jobs[j];
        HandleView cv;
        if (!J.chain || handle_view(J.chain, &cv) != FASTMPS_OK)
            return set_error(runner, FASTMPS_ERR_INVALID_ARG, "job without a chain handle");
        if (cv.device != rv.device || cv.precision != rv.precision || cv.residency != FASTMPS_RESIDENT_HBM) {
            snprintf(msg, sizeof msg, "job %d: chain must be resident, on the runner's device, with its precision", j);
            return set_error(runner, FASTMPS_ERR_INVALID_ARG, msg);
        }
        if (J.M < 1 || !J.bond_dims || J.N < 0 || J.n0 < 0 || J.d < 2 || J.d > 255 || J.bond_dims[0] != 1 ||
            J.bond_dims[J.M] != 1) {
            snprintf(msg, sizeof msg, "job %d: bad M, d, N, n0 or bond_dims", j);
            return set_error(runner, FASTMPS_ERR_SHAPE, msg);
        }
        JobPlan &P = plan[j];
        P.M = J.M;
        P.d = J.d;
        P.N = J.N;
        P.ldV = 64;
        P.ncols_max = 0;
        P.ldP_max = 0;
        for (int k = 0; k < J.M; ++k) {
            SiteView sv;
            if (site_view(J.chain, k, &sv) != FASTMPS_OK) {
                snprintf(msg, sizeof msg, "job %d: site %d is not loaded", j, k);
                return set_error(runner, FASTMPS_ERR_NOT_LOADED, msg);
            }
            if (sv.L.chi_l != J.bond_dims[k] || sv.L.d != J.d || sv.L.chi_r != J.bond_dims[k + 1]) {
                snprintf(msg, sizeof msg, "job %d: site %d does not match bond_dims / d", j, k);
                return set_error(runner, FASTMPS_ERR_SHAPE, msg);
            }
            P.ldV = std::max(P.ldV, sv.L.K_pad);
            P.ncols_max = std::max(P.ncols_max, sv.L.ncols);
            P.ldP_max = std::max(P.ldP_max, sv.L.ncols / sv.L.bn);
            flops += 8.0 * sv.L.chi_l * sv.L.d * sv.L.chi_r * (double)J.N;
        }
        P.N_pad = roundup(std::max<int64_t>(J.N, 1), 128);
        // scratch share proportional to the job's rows
        const int64_t share = std::max<int64_t>((int64_t)256 << 20,
                                                total_rows > 0 ? budget * std::max<int64_t>(J.N, 1) / total_rows : 0);
        P.N2 = std::min(P.N_pad, std::max<int64_t>(128, share / ((int64_t)P.ncols_max * 4) / 128 * 128));
        if (rv.max_microbatch > 0)  // the runner's option caps the rows of a chunk
            P.N2 = std::min(P.N2, std::max<int64_t>(128, rv.max_microbatch / 128 * 128));
        P.chunks = J.N > 0 ? (J.N + P.N2 - 1) / P.N2 : 0;
        P.rounds = P.chunks * J.M;
        R = std::max(R, P.rounds);
    }
    stats->flops_algorithmic = flops;
    stats->flops_issued = flops * nprod;
    if (R == 0) return FASTMPS_OK;

    // ---- buffers ---------------------------------------------------------------
    BatchState *bs = state_of(runner);
    while ((int)bs->jobs.size() < count) bs->jobs.emplace_back(new JobBufs());
    for (int j = 0; j < count; ++j) {
        const JobPlan &P = plan[j];
        JobBufs &B = *bs->jobs[j];
        for (int x = 0; x < 2; ++x)
            for (int p = 0; p < a_planes; ++p)
                if (!B.V[x][p].ensure((size_t)P.N_pad * P.ldV * 2))
                    return set_error(runner, FASTMPS_ERR_OOM, "left-operand allocation failed");
        if (!B.Y.ensure((size_t)P.N2 * P.ncols_max * 4) || !B.P.ensure((size_t)P.N2 * P.ldP_max * 4) ||
            !B.logp.ensure((size_t)P.N_pad * 8) || !B.O.ensure((size_t)P.M * P.N_pad))
            return set_error(runner, FASTMPS_ERR_OOM, "work-buffer allocation failed");
        if (jobs[j].out_samples && !device_pointer(jobs[j].out_samples) &&
            !B.stage_out.ensure((size_t)P.N * P.M))
            return set_error(runner, FASTMPS_ERR_OOM, "output staging allocation failed");
    }
    if (!bs->err.ensure(256)) return set_error(runner, FASTMPS_ERR_OOM, "allocation failed");
    int *d_err = bs->err.as<int>();

    // ---- signature: reuse the captured graph when nothing changed -----------------
    const bool stall = stall_test_requested();
    std::vector<uint64_t> sig;
    sig.push_back((uint64_t)count);
    sig.push_back((uint64_t)stall);
    for (int j = 0; j < count; ++j) {
        const fastmps_job &J = jobs[j];
        const uint64_t f[] = {(uint64_t)(uintptr_t)J.chain, (uint64_t)J.M, (uint64_t)J.d, (uint64_t)J.n0,
                              (uint64_t)J.N, J.seed, (uint64_t)J.job, (uint64_t)(uintptr_t)bs->jobs[j]->V[0][0].p,
                              (uint64_t)(uintptr_t)bs->jobs[j]->Y.p, (uint64_t)(uintptr_t)J.out_samples,
                              (uint64_t)(uintptr_t)bs->jobs[j]->stage_out.p};
        sig.insert(sig.end(), f, f + sizeof f / sizeof f[0]);
        for (int k = 0; k <= J.M; ++k) sig.push_back((uint64_t)J.bond_dims[k]);
        for (int k = 0; k < J.M; ++k) {
            SiteView sv;
            site_view(J.chain, k, &sv);
            sig.push_back((uint64_t)(uintptr_t)(sv.B0));
        }
    }
    cudaStream_t st = rv.stream;
    cudaError_t e;
    if (!(bs->graph && sig == bs->signature)) {
        if (bs->graph) {
            cudaGraphExecDestroy(bs->graph);
            bs->graph = nullptr;
        }
        // ---- segment table of every round, in task order ----------------------------
        size_t total_segs = 0;
        for (int64_t r = 0; r < R; ++r)
            for (int j = 0; j < count; ++j) total_segs += r < plan[j].rounds ? 1 : 0;
        // m-tile slots of each job (counters of completed measurements)
        std::vector<int64_t> slot_base(count + 1, 0);
        for (int j = 0; j < count; ++j) slot_base[j + 1] = slot_base[j] + plan[j].N2 / 128;
        if (!bs->segs_host.host) bs->segs_host.host = true;
        if (!bs->meas_host.host) bs->meas_host.host = true;
        if (!bs->segs_host.ensure(total_segs * sizeof(PSegment)) ||
            !bs->meas_host.ensure(total_segs * sizeof(MeasureArgs)) ||
            !bs->segs_dev.ensure(total_segs * sizeof(PSegment)) ||
            !bs->meas_dev.ensure(total_segs * sizeof(MeasureArgs)))
            return set_error(runner, FASTMPS_ERR_OOM, "segment-table allocation failed");
        PSegment *hs = bs->segs_host.as<PSegment>();
        MeasureArgs *hm = bs->meas_host.as<MeasureArgs>();
        int64_t task = 0, done = 0;
        size_t si = 0;
        for (int64_t r = 0; r < R; ++r) {
            for (int j = 0; j < count; ++j) {
                const JobPlan &P = plan[j];
                if (r >= P.rounds) continue;
                const fastmps_job &J = jobs[j];
                JobBufs &B = *bs->jobs[j];
                const int64_t c = r / P.M;
                const int k = (int)(r % P.M);
                SiteView sv;
                site_view(J.chain, k, &sv);
                const SiteLayout &L = sv.L;
                const int cur = k & 1, nxt = cur ^ 1;
                int K_next = 64;
                if (k + 1 < P.M) {
                    SiteView sn;
                    site_view(J.chain, k + 1, &sn);
                    K_next = sn.L.K_pad;
                }
                const int64_t row0 = c * P.N2;
                const int64_t rows = std::min<int64_t>(P.N2, P.N - row0);
                PSegment &S = hs[si];
                memset(&S, 0, sizeof S);
                for (int p = 0; p < 3; ++p)
                    if (!encode_bf16_map(&S.tmA[p], B.V[cur][p < a_planes ? p : 0].p, L.K_pad, P.N_pad, P.ldV, 128))
                        return set_error(runner, FASTMPS_ERR_CUDA, "tensor map encoding failed");
                S.tmB[0] = sv.tmB[0];
                S.tmB[1] = sv.tmB[1];
                S.task_begin = task;
                S.num_m_tiles = (int)(roundup(rows, 128) / 128);
                S.num_n_tiles = L.ncols / L.bn;
                S.num_k_blocks = L.K_pad / 64;
                S.bn = L.bn;
                S.idesc = idesc_bf16_f32(128, L.bn);
                S.tx_bytes = (uint32_t)a_planes * 16384u + (uint32_t)b_planes * (uint32_t)L.bn * 128u;
                S.row0 = (int)row0;
                S.step = (int)r;  // chunk c at site k is the job's step c * M + k = r
                S.slot_base = slot_base[j];
                S.done_base = done;
                // fixed row strides (the job's widest site): m-tiles of consecutive steps run
                // concurrently, so a row's scratch must not move when the site's width changes
                S.Y = B.Y.as<float>();
                S.ldY = P.ncols_max;
                S.P = B.P.as<float>();
                S.ldP = P.ldP_max;
                S.rows_valid = (int)rows;
                MeasureArgs &m = hm[si];
                m = MeasureArgs{};
                m.Y = S.Y;
                m.ldY = S.ldY;
                m.P = S.P;
                m.ldP = S.ldP;
                m.d = J.d;
                m.chi_r = L.chi_r;
                m.Cs = L.Cs;
                m.tiles_per_s = L.tiles_per_s;
                m.rows = (int)rows;
                m.seed = J.seed;
                m.n_base = (uint64_t)(J.n0 + row0);
                m.k = (uint32_t)k;
                m.job = J.job;
                m.row0 = row0;
                m.ld_next = P.ldV;
                m.K_next = K_next;
                m.V32 = nullptr;
                for (int p = 0; p < 3; ++p) m.Vp[p] = p < a_planes ? B.V[nxt][p].as<__nv_bfloat16>() : nullptr;
                m.nplanes = a_planes;
                m.outcomes = B.O.as<uint8_t>() + (int64_t)k * P.N_pad + row0;
                m.logp = B.logp.as<double>();
                m.trace = nullptr;
                m.trace_rows = 0;
                m.err = d_err;
                task += (int64_t)S.num_m_tiles * S.num_n_tiles;
                done += S.num_m_tiles;
                ++si;
            }
        }
        // counters: [0, 2) task queue (64-bit), then measured[slot], then tiles_done[segment m-tile]
        const size_t counter_ints = 4 + (size_t)slot_base[count] + (size_t)done;
        if (!bs->counters.ensure(counter_ints * sizeof(int)))
            return set_error(runner, FASTMPS_ERR_OOM, "counter allocation failed");
        e = cudaMemcpyAsync(bs->segs_dev.p, hs, total_segs * sizeof(PSegment), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bs->meas_dev.p, hm, total_segs * sizeof(MeasureArgs), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(runner, FASTMPS_ERR_CUDA, "segment-table upload failed");

        // ---- capture the call: resets, initialisation, one persistent launch, transposes ------
        std::vector<uint8_t *> out_dst(count, nullptr);
        for (int j = 0; j < count; ++j)
            if (jobs[j].out_samples)
                out_dst[j] = device_pointer(jobs[j].out_samples) ? jobs[j].out_samples
                                                                 : bs->jobs[j]->stage_out.as<uint8_t>();
        e = prepare_batch_persistent();
        if (e != cudaSuccess) return set_error(runner, FASTMPS_ERR_CUDA, "kernel attribute setup failed");
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(runner, FASTMPS_ERR_CUDA, "stream creation failed");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return set_error(runner, FASTMPS_ERR_CUDA, "stream capture failed to start");
        }
        int64_t launches = 0;
        cudaMemsetAsync(d_err, 0, sizeof(int), cap);
        cudaMemsetAsync(bs->counters.p, 0, counter_ints * sizeof(int), cap);
        for (int j = 0; j < count; ++j) {
            const JobPlan &P = plan[j];
            if (P.rounds == 0) continue;
            JobBufs &B = *bs->jobs[j];
            __nv_bfloat16 *V0[3] = {nullptr, nullptr, nullptr};
            for (int p = 0; p < a_planes; ++p) V0[p] = B.V[0][p].as<__nv_bfloat16>();
            cudaMemsetAsync(B.logp.p, 0, (size_t)P.N_pad * 8, cap);
            launch_init_left_bf16(V0, a_planes, P.N_pad, P.ldV, cap);
            ++launches;
        }
        PersistentArgs g;
        g.segs = bs->segs_dev.as<PSegment>();
        g.meas = bs->meas_dev.as<MeasureArgs>();
        g.nseg = (int)total_segs;
        g.total_tasks = task;
        int *ctr = bs->counters.as<int>();
        g.queue = ctr;
        g.measured = ctr + 4;
        g.tiles_done = ctr + 4 + slot_base[count];
        g.a_planes = a_planes;
        g.b_planes = b_planes;
        g.nprod = nprod;
        for (int q = 0; q < kMaxProducts; ++q) {
            g.prod_a[q] = pa[q];
            g.prod_b[q] = pb[q];
        }
        g.wait_limit_ns = stall ? 100000000ull : kWaitLimitNs;
        g.stall_test = stall ? 1 : 0;
        const cudaError_t le = launch_batch_persistent(g, rv.num_sms, d_err, cap);
        ++launches;
        for (int j = 0; j < count; ++j) {
            const JobPlan &P = plan[j];
            if (P.rounds == 0 || !jobs[j].out_samples) continue;
            JobBufs &B = *bs->jobs[j];
            launch_transpose_outcomes(B.O.as<uint8_t>(), P.N_pad, P.N, P.M, out_dst[j], cap);
            ++launches;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (le != cudaSuccess || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return set_error(runner, FASTMPS_ERR_CUDA, "capture of the batched launches failed");
        }
        e = cudaGraphInstantiate(&bs->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            bs->graph = nullptr;
            return set_error(runner, FASTMPS_ERR_CUDA, "graph instantiation failed");
        }
        bs->signature = sig;
        bs->launches = launches;
    }
    stats->launches = bs->launches;
    stats->contract_launches = 1;  // one persistent launch runs every round of every job

    // ---- run ----------------------------------------------------------------------
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    e = cudaGraphLaunch(bs->graph, st);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return set_error(runner, FASTMPS_ERR_CUDA, "graph launch failed");
    }
    for (int j = 0; j < count; ++j) {
        const JobPlan &P = plan[j];
        if (P.rounds == 0) continue;
        JobBufs &B = *bs->jobs[j];
        if (jobs[j].out_samples && !device_pointer(jobs[j].out_samples)) {
            cudaMemcpyAsync(jobs[j].out_samples, B.stage_out.p, (size_t)P.N * P.M, cudaMemcpyDeviceToHost, st);
            stats->d2h_bytes += P.N * P.M;
        }
        if (jobs[j].out_logprob) {
            const bool dev = device_pointer(jobs[j].out_logprob);
            cudaMemcpyAsync(jobs[j].out_logprob, B.logp.p, (size_t)P.N * 8,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
            if (!dev) stats->d2h_bytes += P.N * 8;
        }
    }
    int herr = 0;
    e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    stats->ms_contract = ms;  // device time of the whole graph (contraction + measurement)
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (e != cudaSuccess) return set_error(runner, FASTMPS_ERR_CUDA, cudaGetErrorString(e));
    if (herr == kDevNumeric)
        return set_error(runner, FASTMPS_ERR_NUMERIC, "a sample's probabilities summed to zero or a non-finite value");
    if (herr != 0) return set_error(runner, FASTMPS_ERR_TIMEOUT, "a bounded device wait gave up");
    return FASTMPS_OK;
}
