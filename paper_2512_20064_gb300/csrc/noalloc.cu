// fastmps_sample_noalloc: the sampling path with every per-call buffer taken
// from one fixed device array instead of allocated memory.
//
// Who needs it: callers that may not call cudaMalloc while they sample --
// runtimes whose device memory is owned by their own caching allocator or a
// fixed budget, and long-running services that forbid allocation after
// start-up so that memory use cannot grow or fragment.
// fastmps_sample grows per-handle work buffers with cudaMalloc on demand;
// this entry point instead uses kNoAllocScratchBytes of static device memory
// that every device which loads this library holds until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// device address of the array with cudaGetSymbolAddress, once per device;
// that first call should come before any stream capture begins.  Every call
// shares the one array, which keeps the previous call's contents: the
// log-probability accumulators and the error word are cleared at the start
// of each call, everything else is fully written before it is read.  Calls
// that overlap on the GPU (on different streams, or from different handles on
// the same device) race on the array and must be serialised by the caller.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "../../include/fastmps.h"
#include "common.cuh"
#include "handle_view.h"
#include "launch.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

inline int64_t roundup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Device address of the array on `device` (which must be current).
int scratch_address(fastmps_handle h, int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices)
        return fastmps::set_error(h, FASTMPS_ERR_UNSUPPORTED, "device index beyond the no-alloc set-up table");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char m[160];
            snprintf(m, sizeof m, "cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorName(e));
            return fastmps::set_error(h, FASTMPS_ERR_CUDA, m);
        }
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return FASTMPS_OK;
}

bool device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Carves 256-byte-aligned pieces out of the array.
struct Carver {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t bytes) {
        T *p = reinterpret_cast<T *>(base + used);
        used += (size_t)roundup((int64_t)bytes, 256);
        return p;
    }
};

}  // namespace

extern "C" int fastmps_sample_noalloc(fastmps_handle h, int M, int d, const int *bond_dims, int64_t n0, int64_t N,
                                      uint64_t seed, uint32_t job, uint8_t *out_samples, double *out_logprob) {
    using namespace fastmps;
    if (!h) return FASTMPS_ERR_INVALID_ARG;
    HandleView hv;
    handle_view(h, &hv);
    if (cudaSetDevice(hv.device) != cudaSuccess) return set_error(h, FASTMPS_ERR_CUDA, "cudaSetDevice failed");
    if (M < 1 || !bond_dims || N < 0 || n0 < 0)
        return set_error(h, FASTMPS_ERR_INVALID_ARG, "need M >= 1, bond_dims, N >= 0, n0 >= 0");
    if (d < 2 || d > 255) return set_error(h, FASTMPS_ERR_SHAPE, "need 2 <= d <= 255");
    if (bond_dims[0] != 1 || bond_dims[M] != 1)
        return set_error(h, FASTMPS_ERR_SHAPE, "bond_dims[0] and bond_dims[M] must be 1");
    if (hv.residency != FASTMPS_RESIDENT_HBM)
        return set_error(h, FASTMPS_ERR_UNSUPPORTED, "fastmps_sample_noalloc needs resident site tensors");
    if (hv.precision == FASTMPS_FP8X1 || hv.precision == FASTMPS_FP8X2 || hv.precision == FASTMPS_FP16X2 ||
        hv.precision == FASTMPS_FP16X3)
        return set_error(h, FASTMPS_ERR_UNSUPPORTED, "fastmps_sample_noalloc runs FP32 and the BF16 modes");
    if (N > 0 && ((out_samples && !device_pointer(out_samples)) || (out_logprob && !device_pointer(out_logprob))))
        return set_error(h, FASTMPS_ERR_INVALID_ARG, "fastmps_sample_noalloc writes device memory only");
    // site views are read again in the site loop: no host container is allocated
    int ldV = 64, ncols_max = 0, ldP_max = 0;
    char msg[256];
    for (int k = 0; k < M; ++k) {
        SiteView sv;
        if (site_view(h, k, &sv) != FASTMPS_OK) {
            snprintf(msg, sizeof msg, "site %d is not loaded", k);
            return set_error(h, FASTMPS_ERR_NOT_LOADED, msg);
        }
        const SiteLayout &L = sv.L;
        if (L.chi_l != bond_dims[k] || L.d != d || L.chi_r != bond_dims[k + 1]) {
            snprintf(msg, sizeof msg, "site %d was loaded with shape (%d, %d, %d), bond_dims/d say (%d, %d, %d)", k,
                     L.chi_l, L.d, L.chi_r, bond_dims[k], d, bond_dims[k + 1]);
            return set_error(h, FASTMPS_ERR_SHAPE, msg);
        }
        ldV = std::max(ldV, L.K_pad);
        ncols_max = std::max(ncols_max, L.ncols);
        ldP_max = std::max(ldP_max, L.ncols / L.bn);
    }
    if (N == 0) return FASTMPS_OK;

    const bool bf16 = hv.precision != FASTMPS_FP32;
    int a_planes = 1, b_planes = 1, nprod = 1, pa[kMaxProducts], pb[kMaxProducts];
    if (bf16) precision_products(hv.precision, &a_planes, &b_planes, &nprod, pa, pb);
    const int planes = bf16 ? a_planes : 1;
    const size_t elem = bf16 ? 2 : 4;
    const int64_t N_pad = roundup(N, 128);

    // size check: fixed part for all rows, then as many micro-batch rows as fit
    const size_t fixed = 256 + (size_t)roundup(N_pad * 8, 256) + (size_t)roundup((int64_t)M * N_pad, 256) +
                         2 * (size_t)planes * (size_t)roundup(N_pad * ldV * (int64_t)elem, 256);
    const size_t per_row = (size_t)ncols_max * 4 + (size_t)ldP_max * 4;
    int64_t N2 = 0;
    if (fixed + 128 * per_row + 512 <= kNoAllocScratchBytes)
        N2 = std::min<int64_t>(N_pad, (int64_t)((kNoAllocScratchBytes - fixed - 512) / per_row) / 128 * 128);
    if (N2 < 128) {
        snprintf(msg, sizeof msg,
                 "fastmps_sample_noalloc: %lld rows of this chain need %zu MiB of scratch but the static scratch "
                 "holds %zu MiB; sample fewer rows per call",
                 (long long)N, (fixed + 128 * per_row + ((size_t)1 << 20) - 1) >> 20, kNoAllocScratchBytes >> 20);
        return set_error(h, FASTMPS_ERR_INVALID_ARG, msg);
    }

    unsigned char *base = nullptr;
    int rc = scratch_address(h, hv.device, &base);
    if (rc) return rc;
    Carver c{base};
    int *d_err = c.take<int>(256);
    double *logp = c.take<double>((size_t)N_pad * 8);
    uint8_t *O = c.take<uint8_t>((size_t)M * N_pad);
    __nv_bfloat16 *Vp[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    float *V32[2] = {nullptr, nullptr};
    for (int x = 0; x < 2; ++x) {
        if (bf16)
            for (int p = 0; p < planes; ++p) Vp[x][p] = c.take<__nv_bfloat16>((size_t)N_pad * ldV * 2);
        else
            V32[x] = c.take<float>((size_t)N_pad * ldV * 4);
    }
    float *Y = c.take<float>((size_t)N2 * ncols_max * 4);
    float *P = c.take<float>((size_t)N2 * ldP_max * 4);
    if (c.used > kNoAllocScratchBytes) return set_error(h, FASTMPS_ERR_INVALID_ARG, "no-alloc scratch overflow");

    cudaStream_t st = hv.stream;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(logp, 0, (size_t)N_pad * 8, st);
    if (e != cudaSuccess) return set_error(h, FASTMPS_ERR_CUDA, "cudaMemsetAsync failed");
    if (bf16) launch_init_left_bf16(Vp[0], planes, N_pad, ldV, st);
    else launch_init_left_f32(V32[0], N_pad, ldV, st);

    for (int k = 0; k < M; ++k) {
        SiteView sv, sv_next;
        site_view(h, k, &sv);
        const SiteLayout &L = sv.L;
        const int cur = k & 1, nxt = cur ^ 1;
        int K_next = 64;
        if (k + 1 < M) {
            site_view(h, k + 1, &sv_next);
            K_next = sv_next.L.K_pad;
        }
        TcArgs ta;
        if (bf16) {
            ta.tmB[0] = sv.tmB[0];
            ta.tmB[1] = sv.tmB[1];
            ta.a_planes = a_planes;
            ta.b_planes = b_planes;
            ta.nprod = nprod;
            for (int q = 0; q < kMaxProducts; ++q) {
                ta.prod_a[q] = pa[q];
                ta.prod_b[q] = pb[q];
            }
            for (int p = 0; p < 3; ++p)
                if (!encode_bf16_map(&ta.tmA[p], Vp[cur][p < planes ? p : 0], L.K_pad, N_pad, ldV, 128))
                    return set_error(h, FASTMPS_ERR_CUDA, "tensor map encoding failed");
        }
        for (int64_t r0 = 0; r0 < N; r0 += N2) {
            const int64_t rows = std::min<int64_t>(N2, N - r0);
            ContractOut co;
            co.Y = Y;
            co.ldY = L.ncols;
            co.P = P;
            co.ldP = L.ncols / L.bn;
            co.rows_valid = (int)rows;
            if (bf16) {
                ta.row0 = r0;
                ta.rows_pad = (int)roundup(rows, 128);
                e = launch_contract_tc(ta, L, co, hv.num_sms, d_err, st);
                if (e != cudaSuccess) return set_error(h, FASTMPS_ERR_CUDA, "contraction launch failed");
            } else {
                launch_contract_f32(V32[cur], ldV, r0, roundup(rows, 128), sv.Bt, L, co, st);
            }
            MeasureArgs ma;
            ma.Y = Y;
            ma.ldY = L.ncols;
            ma.P = P;
            ma.ldP = L.ncols / L.bn;
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
            ma.V32 = bf16 ? nullptr : V32[nxt];
            for (int p = 0; p < 3; ++p) ma.Vp[p] = Vp[nxt][p];
            ma.nplanes = planes;
            ma.outcomes = O + (int64_t)k * N_pad + r0;
            ma.logp = logp;
            ma.trace = nullptr;
            ma.trace_rows = 0;
            ma.err = d_err;
            launch_measure(ma, st);
            e = cudaGetLastError();
            if (e != cudaSuccess) return set_error(h, FASTMPS_ERR_CUDA, "kernel launch failed");
        }
    }
    if (out_samples) launch_transpose_outcomes(O, N_pad, N, M, out_samples, st);
    if (out_logprob) {
        e = cudaMemcpyAsync(out_logprob, logp, (size_t)N * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return set_error(h, FASTMPS_ERR_CUDA, "copy of log-probabilities failed");
    }
    int herr = 0;
    e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(h, FASTMPS_ERR_CUDA, cudaGetErrorString(e));
    if (herr == kDevNumeric)
        return set_error(h, FASTMPS_ERR_NUMERIC, "a sample's probabilities summed to zero or a non-finite value");
    if (herr != 0) return set_error(h, FASTMPS_ERR_TIMEOUT, "a bounded device wait in the contraction kernel gave up");
    return FASTMPS_OK;
}
