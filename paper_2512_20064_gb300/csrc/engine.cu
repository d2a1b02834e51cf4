// Host engine of one sampling call.
//
// Engine per call (Sec. 3.1 data-parallel scheme on one device): all N rows
// of the left operand stay resident in device memory (the macro-batch);
// for each site k the rows are processed in micro-batches: one contraction
// launch writes the FP32 scratch Y and per-tile sums of squares, one
// measurement launch draws the outcome and writes the next left operand.  In
// host-streaming residency the BF16 site tensor of site k+1 is copied from
// pinned host memory into one of two device slots on a copy stream while site
// k computes (Sec. 3.1 double buffer; Sec. 3.3.2 16-bit storage).
#include "context.h"

namespace fastmps {

namespace {

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

}  // namespace

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

int run_sample(fastmps_handle h, int M, int d, const int *bonds, int64_t n0, int64_t N, uint64_t seed, uint32_t job,
               uint8_t *out_samples, double *out_logprob, int64_t trace_rows, double *trace_probs,
               const float2 *mu_dev, int64_t ld_mu, const int64_t *trace_list) {
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

}  // namespace fastmps
