// Site loading (a-1 of the hot path, once per load): copy of a complex site tensor (host or device,
// optionally scaled by a Vidal-form coefficient vector), repack into the handle's arithmetic format
// (BF16 or binary16 planes of the stacked real operand, E4M3, or the FP32 transpose) and the tensor
// maps over it; compact 16-bit copies in pinned host memory for host streaming; and the autotuner
// that picks the n-tile width and the measurement mode per site shape.
#include "context.h"

namespace fastmps {

namespace {

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

}  // namespace

int load_tensor(fastmps_handle h, Tensor &t, int chi_l, int d, int chi_r, const void *A, int dtype,
                const void *lam) {
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

}  // namespace fastmps
