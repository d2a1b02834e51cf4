// C ABI of the sampling library (see include/fastmps.h): argument checks, handle creation and
// destruction, site loading, the sampling entry points (which run the engine of engine.cu), the
// displacement call, statistics, and read-only views of a handle for the entry points compiled in
// other translation units (batch.cu, noalloc.cu).
#include "context.h"
#include "handle_view.h"

using namespace fastmps;

namespace {
std::string g_create_error;
}  // namespace

extern "C" {

void fastmps_default_options(fastmps_options *opt) {
    if (!opt) return;
    opt->precision = FASTMPS_FP32;
    opt->residency = FASTMPS_RESIDENT_HBM;
    opt->max_microbatch = 0;
    opt->autotune = 0;
    opt->stream = nullptr;
    opt->fused_measure = 0;
    opt->k_split = 0;
    opt->accum_chunk = 0;
}

int fastmps_create(fastmps_handle *out, int device, const fastmps_options *opt) {
    if (!out) {
        g_create_error = "out is NULL";
        return FASTMPS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fastmps_options o;
    fastmps_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < FASTMPS_FP32 || o.precision > FASTMPS_FP16X3) {
        g_create_error = "unknown precision";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.accum_chunk < 0 || o.accum_chunk > 4096) {
        g_create_error = "accum_chunk must be 0..4096";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.k_split < 0 || o.k_split > 8) {
        g_create_error = "k_split must be 0..8";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.residency != FASTMPS_RESIDENT_HBM && o.residency != FASTMPS_HOST_STREAM) {
        g_create_error = "unknown residency";
        return FASTMPS_ERR_INVALID_ARG;
    }
    if (o.residency == FASTMPS_HOST_STREAM &&
        (o.precision == FASTMPS_FP32 || o.precision == FASTMPS_FP8X1 || o.precision == FASTMPS_FP8X2)) {
        g_create_error = "host streaming keeps 16-bit tensors: use a BF16 or the FP16 precision";
        return FASTMPS_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_create_error = "no such CUDA device";
        return FASTMPS_ERR_CUDA;
    }
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    if (!(prop.major == 10 && prop.minor == 3)) {
        g_create_error = std::string("device ") + prop.name + " is sm_" + std::to_string(prop.major) +
                         std::to_string(prop.minor) + "; this library is built for sm_103a only";
        return FASTMPS_ERR_UNSUPPORTED;
    }
    if (o.precision != FASTMPS_FP32 && (!tc_max_smem_ok(device) || !get_encode_fn())) {
        g_create_error = "tensor-core path needs 227 KB shared memory and cuTensorMapEncodeTiled";
        return FASTMPS_ERR_UNSUPPORTED;
    }
    fastmps_ctx *h = new (std::nothrow) fastmps_ctx();
    if (!h) {
        g_create_error = "out of host memory";
        return FASTMPS_ERR_OOM;
    }
    h->device = device;
    h->opt = o;
    h->num_sms = prop.multiProcessorCount;
    cudaSetDevice(device);
    if (o.stream) {
        h->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            g_create_error = "stream creation failed";
            return FASTMPS_ERR_CUDA;
        }
        h->own_stream = true;
    }
    cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&h->measure_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2; ++i) {
        cudaEventCreateWithFlags(&h->copy_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&h->slot_free[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&h->contract_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&h->measure_done[i], cudaEventDisableTiming);
    }
    h->staging.host = false;
    *out = h;
    return FASTMPS_OK;
}

void fastmps_destroy(fastmps_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    fastmps::batch_release(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    if (h->measure_stream) cudaStreamSynchronize(h->measure_stream);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
        if (h->copy_done[i]) cudaEventDestroy(h->copy_done[i]);
        if (h->slot_free[i]) cudaEventDestroy(h->slot_free[i]);
        if (h->contract_done[i]) cudaEventDestroy(h->contract_done[i]);
        if (h->measure_done[i]) cudaEventDestroy(h->measure_done[i]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->measure_stream) cudaStreamDestroy(h->measure_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char *fastmps_last_error(fastmps_handle h) {
    if (!h) return g_create_error.c_str();
    return h->last_error.c_str();
}

int fastmps_load_site(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *A, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (k < 0 || k >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "site index out of range");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, A, dtype);
    if (rc) return rc;
    h->site_tensor[k] = std::move(t);
    h->site_pool.erase(k);
    return FASTMPS_OK;
}

int fastmps_load_pool(fastmps_handle h, int j, int chi_l, int d, int chi_r, const void *A, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (j < 0 || j >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "pool index out of range");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, A, dtype);
    if (rc) return rc;
    h->pool_tensor[j] = std::move(t);
    return FASTMPS_OK;
}

int fastmps_map_site(fastmps_handle h, int k, int j) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (k < 0 || k >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "site index out of range");
    if (h->pool_tensor.find(j) == h->pool_tensor.end())
        return fail(h, FASTMPS_ERR_NOT_LOADED, "pool entry " + std::to_string(j) + " is not loaded");
    h->site_pool[k] = j;
    h->site_tensor.erase(k);
    return FASTMPS_OK;
}

int fastmps_sample_ex(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N, uint64_t seed,
                      uint32_t job, uint8_t *out_samples, double *out_logprob, int64_t trace_rows,
                      double *trace_probs) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    try {
        return run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, trace_rows, trace_probs);
    } catch (const std::bad_alloc &) {
        return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(h, FASTMPS_ERR_CUDA, "unexpected host exception");
    }
}

int fastmps_sample_traced(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N, uint64_t seed,
                          uint32_t job, uint8_t *out_samples, double *out_logprob, const int64_t *trace_list,
                          int64_t n_trace, double *trace_probs) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (n_trace < 0 || (n_trace > 0 && (!trace_list || !trace_probs)))
        return fail(h, FASTMPS_ERR_INVALID_ARG, "n_trace > 0 needs trace_list and trace_probs");
    cudaSetDevice(h->device);
    try {
        return run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, n_trace, trace_probs,
                          nullptr, 0, n_trace > 0 ? trace_list : nullptr);
    } catch (const std::bad_alloc &) {
        return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(h, FASTMPS_ERR_CUDA, "unexpected host exception");
    }
}

int fastmps_sample(fastmps_handle h, int M, int d, const int *bond_dims, int64_t N, uint64_t seed,
                   uint8_t *out_samples, double *out_logprob) {
    return fastmps_sample_ex(h, M, d, bond_dims, 0, N, seed, 0, out_samples, out_logprob, 0, nullptr);
}

int fastmps_load_site_vidal(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *Gamma,
                            const void *Lambda, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (k < 0 || k >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "site index out of range");
    if (!Lambda) return fail(h, FASTMPS_ERR_INVALID_ARG, "Lambda is NULL");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, Gamma, dtype, Lambda);
    if (rc) return rc;
    h->site_tensor[k] = std::move(t);
    h->site_pool.erase(k);
    return FASTMPS_OK;
}

int fastmps_load_pool_vidal(fastmps_handle h, int j, int chi_l, int d, int chi_r, const void *Gamma,
                            const void *Lambda, int dtype) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (j < 0 || j >= 65536) return fail(h, FASTMPS_ERR_INVALID_ARG, "pool index out of range");
    if (!Lambda) return fail(h, FASTMPS_ERR_INVALID_ARG, "Lambda is NULL");
    cudaSetDevice(h->device);
    std::unique_ptr<Tensor> t(new (std::nothrow) Tensor());
    if (!t) return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    int rc = load_tensor(h, *t, chi_l, d, chi_r, Gamma, dtype, Lambda);
    if (rc) return rc;
    h->pool_tensor[j] = std::move(t);
    return FASTMPS_OK;
}

int fastmps_load_site_vidal_truncated(fastmps_handle h, int k, int chi_l, int d, int chi_r, const void *Gamma,
                                      const void *Lambda, int dtype, int keep_l, int keep_r) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (!Gamma || !Lambda) return fail(h, FASTMPS_ERR_INVALID_ARG, "Gamma or Lambda is NULL");
    if (dtype != FASTMPS_C64 && dtype != FASTMPS_C128) return fail(h, FASTMPS_ERR_INVALID_ARG, "unknown dtype");
    if (chi_l < 1 || chi_r < 1 || d < 2 || d > 255 || keep_l < 1 || keep_l > chi_l || keep_r < 1 || keep_r > chi_r)
        return fail(h, FASTMPS_ERR_SHAPE, "need 1 <= keep_l <= chi_l, 1 <= keep_r <= chi_r, 2 <= d <= 255");
    if (keep_l == chi_l && keep_r == chi_r) return fastmps_load_site_vidal(h, k, chi_l, d, chi_r, Gamma, Lambda, dtype);
    cudaSetDevice(h->device);
    const size_t elem = dtype == FASTMPS_C128 ? 16 : 8;
    const size_t rows = (size_t)keep_l * d, width = (size_t)keep_r * elem, pitch = (size_t)chi_r * elem;
    // rows (a, s) of Gamma are contiguous runs of chi_r entries: the leading block is a 2D copy
    if (is_device_ptr(Gamma)) {
        if (!h->trunc.ensure(rows * width)) return fail(h, FASTMPS_ERR_OOM, "allocation failed");
        cudaError_t e = cudaMemcpy2DAsync(h->trunc.p, width, Gamma, pitch, width, rows, cudaMemcpyDeviceToDevice,
                                          h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "gather of the leading block");
        return fastmps_load_site_vidal(h, k, keep_l, d, keep_r, h->trunc.p, Lambda, dtype);
    }
    std::vector<uint8_t> block(rows * width);
    const uint8_t *src = static_cast<const uint8_t *>(Gamma);
    for (size_t r = 0; r < rows; ++r) memcpy(block.data() + r * width, src + r * pitch, width);
    return fastmps_load_site_vidal(h, k, keep_l, d, keep_r, block.data(), Lambda, dtype);
}

int fastmps_sample_displaced(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                             uint64_t seed, uint32_t job, const float *mu, int64_t ld_mu, uint8_t *out_samples,
                             double *out_logprob, int64_t trace_rows, double *trace_probs) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    try {
        if (!mu) return fail(h, FASTMPS_ERR_INVALID_ARG, "mu is NULL");
        if (M < 1 || N < 0 || ld_mu < N) return fail(h, FASTMPS_ERR_INVALID_ARG, "need M >= 1, N >= 0, ld_mu >= N");
        if (d < 2 || d > kMaxDisplacedD)
            return fail(h, FASTMPS_ERR_SHAPE, "displaced sampling supports 2 <= d <= " +
                                                  std::to_string(kMaxDisplacedD));
        if (is_fp8(h) || is_f16(h))
            return fail(h, FASTMPS_ERR_UNSUPPORTED, "displaced sampling needs FP32 or a BF16 precision");
        if (N == 0) return run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, trace_rows,
                                      trace_probs);
        const float2 *mu_dev;
        int64_t ld = ld_mu;
        if (is_device_ptr(mu)) {
            if (reinterpret_cast<uintptr_t>(mu) % 8 != 0)
                return fail(h, FASTMPS_ERR_INVALID_ARG, "device mu must be 8-byte aligned");
            mu_dev = reinterpret_cast<const float2 *>(mu);
        } else {
            if (!h->mu.ensure((size_t)M * N * 8)) return fail(h, FASTMPS_ERR_OOM, "amplitude allocation failed");
            cudaError_t e = cudaMemcpy2DAsync(h->mu.p, (size_t)N * 8, mu, (size_t)ld_mu * 8, (size_t)N * 8, M,
                                              cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy of displacement amplitudes");
            mu_dev = h->mu.as<float2>();
            ld = N;
        }
        int rc = run_sample(h, M, d, bond_dims, n0, N, seed, job, out_samples, out_logprob, trace_rows,
                            trace_probs, mu_dev, ld);
        if (rc == FASTMPS_OK && !is_device_ptr(mu)) h->stats.h2d_bytes += (int64_t)M * N * 8;
        return rc;
    } catch (const std::bad_alloc &) {
        return fail(h, FASTMPS_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(h, FASTMPS_ERR_CUDA, "unexpected host exception");
    }
}

int fastmps_displacement(fastmps_handle h, int64_t N, int d, const float *mu, float *D) {
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    if (!mu || !D || N < 0) return fail(h, FASTMPS_ERR_INVALID_ARG, "need mu, D and N >= 0");
    if (d < 1 || d > 255) return fail(h, FASTMPS_ERR_SHAPE, "need 1 <= d <= 255");
    if (N == 0) return FASTMPS_OK;
    cudaSetDevice(h->device);
    const bool mu_dev = is_device_ptr(mu), D_dev = is_device_ptr(D);
    if ((mu_dev && reinterpret_cast<uintptr_t>(mu) % 8) || (D_dev && reinterpret_cast<uintptr_t>(D) % 8))
        return fail(h, FASTMPS_ERR_INVALID_ARG, "device arrays must be 8-byte aligned");
    const size_t mu_bytes = (size_t)N * 8, D_bytes = (size_t)N * d * d * 8;
    const size_t off = roundup((int64_t)mu_bytes, 256);
    if ((!mu_dev || !D_dev) && !h->disp_io.ensure(off + D_bytes))
        return fail(h, FASTMPS_ERR_OOM, "staging allocation failed");
    cudaStream_t st = h->stream;
    cudaError_t e;
    const float2 *mu_d = reinterpret_cast<const float2 *>(mu);
    if (!mu_dev) {
        e = cudaMemcpyAsync(h->disp_io.p, mu, mu_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of amplitudes");
        mu_d = h->disp_io.as<float2>();
    }
    float2 *D_d = D_dev ? reinterpret_cast<float2 *>(D)
                        : reinterpret_cast<float2 *>(static_cast<char *>(h->disp_io.p) + off);
    const float *tab = displacement_table(h, d);
    if (!tab) return fail(h, FASTMPS_ERR_OOM, "displacement table allocation failed");
    launch_displacement(mu_d, N, d, tab, D_d, h->num_sms, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "displacement launch");
    if (!D_dev) {
        e = cudaMemcpyAsync(D, D_d, D_bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy of displacement matrices");
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "displacement");
    return FASTMPS_OK;
}

int fastmps_get_stats(fastmps_handle h, fastmps_stats *out) {
    if (!h || !out) return FASTMPS_ERR_INVALID_ARG;
    *out = h->stats;
    return FASTMPS_OK;
}

const char *fastmps_version(void) { return "fastmps-gb300 0.1 (sm_103a)"; }

int fastmps_selftest_bounded_wait(int device, double limit_ms, int *status, double *waited_ms) {
    if (!status || !waited_ms || limit_ms <= 0) return FASTMPS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return FASTMPS_ERR_CUDA;
    }
    int *d_status = nullptr;
    unsigned long long *d_ns = nullptr;
    if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (d_status) cudaFree(d_status);
        return FASTMPS_ERR_OOM;
    }
    launch_bounded_wait_selftest((uint64_t)(limit_ms * 1e6), d_status, d_ns, 0);
    int st = -1;
    unsigned long long ns = 0;
    cudaError_t e = cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost);
    cudaFree(d_status);
    cudaFree(d_ns);
    if (e != cudaSuccess) return FASTMPS_ERR_CUDA;
    *status = st == kDevOk ? FASTMPS_OK : FASTMPS_ERR_TIMEOUT;
    *waited_ms = (double)ns / 1e6;
    return FASTMPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Views for entry points implemented in other translation units.
// ---------------------------------------------------------------------------

namespace fastmps {

int handle_view(fastmps_handle h, HandleView *out) {
    if (!h || !out) return FASTMPS_ERR_INVALID_ARG;
    out->device = h->device;
    out->precision = h->opt.precision;
    out->residency = h->opt.residency;
    out->stream = h->stream;
    out->num_sms = h->num_sms;
    out->max_microbatch = h->opt.max_microbatch;
    return FASTMPS_OK;
}

int site_view(fastmps_handle h, int k, SiteView *out) {
    Tensor *t = site_tensor_of(h, k);
    if (!t) return FASTMPS_ERR_NOT_LOADED;
    out->L = t->L;
    out->B0 = t->B_hi.as<__nv_bfloat16>();
    out->B1 = t->B_lo.as<__nv_bfloat16>();
    out->Bt = t->Bt.as<float>();
    out->tmB[0] = t->tmB[0];
    out->tmB[1] = t->tmB[1];
    return FASTMPS_OK;
}

int set_error(fastmps_handle h, int code, const char *msg) { return fail(h, code, msg); }

fastmps_stats *handle_stats(fastmps_handle h) { return &h->stats; }

void precision_products(int precision, int *a_planes, int *b_planes, int *nprod, int *pa, int *pb) {
    const PrecisionPlan p = plan_of(precision);
    *a_planes = p.a_planes;
    *b_planes = p.b_planes;
    *nprod = p.nprod;
    for (int q = 0; q < kMaxProducts; ++q) {
        pa[q] = p.pa[q];
        pb[q] = p.pb[q];
    }
}

bool encode_bf16_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                     uint32_t box_outer) {
    return encode_2d_bf16(map, base, inner, outer, ld_elems, 64, box_outer);
}

}  // namespace fastmps
