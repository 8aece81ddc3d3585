// extern "C" entry points of libcdmd: argument checks, workspace, dispatch.
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "cdmd_internal.cuh"

namespace cdmd {

namespace {
thread_local char g_last_error[512] = "";

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
}  // namespace

cdmd_status fail(cdmd_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

cdmd_status cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? CDMD_ERR_NOMEM : CDMD_ERR_CUDA;
}

void clear_error() { g_last_error[0] = '\0'; }

cdmd_status ensure_buffer(cdmd_ctx* ctx, BufferId id, size_t bytes, void** out) {
    Buffer& b = ctx->buf[id];
    if (bytes == 0) bytes = 256;
    if (b.bytes < bytes) {
        if (b.ptr != nullptr) {
            CDMD_CHECK_CUDA(cudaDeviceSynchronize());
            CDMD_CHECK_CUDA(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        const size_t want = ((bytes + bytes / 8) + 255) & ~static_cast<size_t>(255);
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(CDMD_ERR_NOMEM, "workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        }
        b.ptr = p;
        b.bytes = want;
    }
    *out = b.ptr;
    return CDMD_OK;
}

static cdmd_status check_video(const uint8_t* D, int64_t m, int n, int64_t ldd) {
    CDMD_REQUIRE(D != nullptr, "D is NULL");
    CDMD_REQUIRE(m >= 1, "m must be >= 1 (got %lld)", static_cast<long long>(m));
    CDMD_REQUIRE(m <= 0x7fffffffLL, "m must fit a 32-bit Philox counter word (got %lld)", static_cast<long long>(m));
    CDMD_REQUIRE(n >= 2, "n must be >= 2 (got %d)", n);
    CDMD_REQUIRE(ldd >= m, "ldd (%lld) must be >= m (%lld)", static_cast<long long>(ldd), static_cast<long long>(m));
    return CDMD_OK;
}

// Prefix the current error message with the clip it concerns.
static cdmd_status fail_clip(cdmd_status st, int clip) {
    char msg[sizeof(g_last_error)];
    snprintf(msg, sizeof(msg), "%s", g_last_error);
    return fail(st, "clip %d: %s", clip, msg);
}

constexpr int kMaxSharedRun = 8;   // clips per cdmd_run_shared / cdmd_run_host_shared call

}  // namespace cdmd

using namespace cdmd;

extern "C" {

const char* cdmd_last_error(void) { return g_last_error; }

const char* cdmd_status_string(cdmd_status s) {
    switch (s) {
        case CDMD_OK: return "CDMD_OK";
        case CDMD_ERR_INVALID_ARG: return "CDMD_ERR_INVALID_ARG";
        case CDMD_ERR_CUDA: return "CDMD_ERR_CUDA";
        case CDMD_ERR_NOMEM: return "CDMD_ERR_NOMEM";
        case CDMD_ERR_NOT_CONVERGED: return "CDMD_ERR_NOT_CONVERGED";
        case CDMD_ERR_RANK_DEFICIENT: return "CDMD_ERR_RANK_DEFICIENT";
        case CDMD_ERR_NONFINITE: return "CDMD_ERR_NONFINITE";
        case CDMD_ERR_UNSUPPORTED: return "CDMD_ERR_UNSUPPORTED";
        case CDMD_ERR_TIMEOUT: return "CDMD_ERR_TIMEOUT";
    }
    return "CDMD_ERR_UNKNOWN";
}

cdmd_status cdmd_create(cdmd_ctx** ctx, int device) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    *ctx = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return cuda_fail(e, "cudaGetDeviceCount"); }
    CDMD_REQUIRE(device >= 0 && device < count, "device %d out of range (%d devices)", device, count);
    DeviceGuard g(device);
    cdmd_ctx* c = new cdmd_ctx();
    c->device = device;
    e = cudaDeviceGetAttribute(&c->device_sms, cudaDevAttrMultiProcessorCount, device);
    c->num_sms = c->device_sms;
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return cuda_fail(e, "cdmd_create");
    }
    *ctx = c;
    return CDMD_OK;
}

cdmd_status cdmd_set_sm_limit(cdmd_ctx* ctx, int max_sms) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(max_sms >= 0, "max_sms = %d must be >= 0", max_sms);
    ctx->num_sms = (max_sms == 0) ? ctx->device_sms : std::min(max_sms, ctx->device_sms);
    return CDMD_OK;
}

void cdmd_destroy(cdmd_ctx* ctx) {
    if (ctx == nullptr) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto& b : ctx->buf)
        if (b.ptr) cudaFree(b.ptr);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
}

cdmd_status cdmd_status_sync(cdmd_ctx* ctx, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CDMD_CHECK_CUDA(cudaStreamSynchronize(s));
    int h = 0;
    CDMD_CHECK_CUDA(cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CDMD_CHECK_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (h != 0) return fail(static_cast<cdmd_status>(h), "device reported %s", cdmd_status_string(static_cast<cdmd_status>(h)));
    return CDMD_OK;
}

cdmd_status cdmd_selftest_wait(cdmd_ctx* ctx, uint32_t limit_us, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(limit_us >= 1 && limit_us <= 2000000, "limit_us must be in [1, 2000000] (got %u)", limit_us);
    DeviceGuard g(ctx->device);
    return launch_selftest_wait(ctx, static_cast<uint64_t>(limit_us) * 1000ull, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_selftest_recip(cdmd_ctx* ctx, const double* a, int64_t n, double* rcp, double* rsqrt,
                                void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(n >= 0, "n must be >= 0 (got %lld)", static_cast<long long>(n));
    CDMD_REQUIRE(n == 0 || a != nullptr, "a is NULL");
    DeviceGuard g(ctx->device);
    return launch_selftest_recip(a, n, rcp, rsqrt, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_measure_sparse_nnz(cdmd_ctx* ctx, int64_t m, int k, uint64_t seed, double density, int64_t* nnz,
                                    void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && nnz != nullptr, "ctx or nnz is NULL");
    CDMD_REQUIRE(m >= 1 && m <= 0x7fffffffLL, "m out of range");
    CDMD_REQUIRE(k >= 1, "k must be >= 1");
    CDMD_REQUIRE(density > 0.0 && density <= 1.0, "density must be in (0, 1]");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t* counts = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SMALL, static_cast<size_t>(m + 1) * sizeof(int64_t),
                                   reinterpret_cast<void**>(&counts));
    if (st != CDMD_OK) return st;
    st = launch_measure_sparse_count(ctx, m, k, seed, density, counts, s);
    if (st != CDMD_OK) return st;
    std::vector<int64_t> h(static_cast<size_t>(m));
    CDMD_CHECK_CUDA(cudaMemcpyAsync(h.data(), counts, m * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CDMD_CHECK_CUDA(cudaStreamSynchronize(s));
    int64_t total = 0;
    for (int64_t v : h) total += v;
    *nnz = total;
    return CDMD_OK;
}

cdmd_status cdmd_measure_build(cdmd_ctx* ctx, cdmd_measure* meas, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && meas != nullptr, "ctx or meas is NULL");
    CDMD_REQUIRE(meas->m >= 1 && meas->m <= 0x7fffffffLL, "meas->m out of range");
    CDMD_REQUIRE(meas->k >= 1, "meas->k must be >= 1");
    DeviceGuard g(ctx->device);
    if (meas->ctype == CDMD_C_ROWSAMPLE) {
        CDMD_REQUIRE(meas->k <= meas->m, "ROWSAMPLE needs k <= m");
        CDMD_REQUIRE(meas->rows != nullptr, "meas->rows is NULL");
    } else if (meas->ctype == CDMD_C_SRFT) {
        CDMD_REQUIRE((static_cast<int64_t>(meas->k) + 1) / 2 <= meas->m, "SRFT needs ceil(k/2) <= m");
        CDMD_REQUIRE(meas->k <= 8192, "SRFT supports k <= 8192");
        CDMD_REQUIRE(meas->rows != nullptr, "meas->rows is NULL");
    } else if (meas->ctype == CDMD_C_SPARSE) {
        CDMD_REQUIRE(meas->density > 0.0 && meas->density <= 1.0, "density must be in (0, 1]");
        CDMD_REQUIRE(meas->col_ptr != nullptr && meas->row_idx != nullptr, "CSC arrays are NULL");
        CDMD_REQUIRE(meas->k <= 0x7fffffff, "k too large");
        int64_t nnz = 0;
        cdmd_status st = cdmd_measure_sparse_nnz(ctx, meas->m, meas->k, meas->seed, meas->density, &nnz, stream);
        if (st != CDMD_OK) return st;
        CDMD_REQUIRE(meas->nnz_capacity >= nnz, "nnz_capacity %lld < nnz %lld", static_cast<long long>(meas->nnz_capacity),
                     static_cast<long long>(nnz));
    } else {
        return fail(CDMD_ERR_INVALID_ARG, "cdmd_measure_build takes SPARSE, ROWSAMPLE or SRFT");
    }
    return launch_measure_build(ctx, meas, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_sketch(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, cdmd_ctype ctype, int k,
                        uint64_t seed, cdmd_prec prec, double* DY, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    CDMD_REQUIRE(DY != nullptr, "DY is NULL");
    CDMD_REQUIRE(k >= 1 && k <= (1 << 20), "k must be in [1, 2^20] (got %d)", k);
    CDMD_REQUIRE(ctype == CDMD_C_GAUSSIAN || ctype == CDMD_C_RADEMACHER,
                 "cdmd_sketch generates GAUSSIAN or RADEMACHER C; use cdmd_sketch_gather for the others");
    CDMD_REQUIRE(aligned(DY, 8), "DY must be 8-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == CDMD_PREC_FP32) return launch_sketch_fp32(ctx, D, m, n, ldd, ctype, k, seed, DY, s);
    if (prec == CDMD_PREC_BF16X2) {
        return launch_sketch_tc(ctx, D, m, n, ldd, ctype, k, seed, DY, s);
    }
    return fail(CDMD_ERR_INVALID_ARG, "unknown precision %d", static_cast<int>(prec));
}

cdmd_status cdmd_sketch_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m, const int* n,
                               const int64_t* ldd, cdmd_ctype ctype, int k, uint64_t seed, cdmd_prec prec,
                               double* const* DY, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(nclips >= 1, "nclips must be >= 1 (got %d)", nclips);
    CDMD_REQUIRE(D != nullptr && n != nullptr && ldd != nullptr && DY != nullptr, "NULL array argument");
    for (int i = 0; i < nclips; ++i) {
        cdmd_status st = check_video(D[i], m, n[i], ldd[i]);
        if (st != CDMD_OK) return fail_clip(st, i);
        CDMD_REQUIRE(DY[i] != nullptr && aligned(DY[i], 8), "clip %d: DY is NULL or not 8-byte aligned", i);
    }
    CDMD_REQUIRE(k >= 1 && k <= (1 << 20), "k must be in [1, 2^20] (got %d)", k);
    CDMD_REQUIRE(ctype == CDMD_C_GAUSSIAN || ctype == CDMD_C_RADEMACHER,
                 "cdmd_sketch_shared generates GAUSSIAN or RADEMACHER C");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == CDMD_PREC_BF16X2) return launch_sketch_tc_shared(ctx, nclips, D, m, n, ldd, ctype, k, seed, DY, s);
    if (prec != CDMD_PREC_FP32 && prec != CDMD_PREC_BF16X2)
        return fail(CDMD_ERR_INVALID_ARG, "unknown precision %d", static_cast<int>(prec));
    for (int i = 0; i < nclips; ++i) {
        cdmd_status st = cdmd_sketch(ctx, D[i], m, n[i], ldd[i], ctype, k, seed, prec, DY[i], stream);
        if (st != CDMD_OK) return st;
    }
    return CDMD_OK;
}

cdmd_status cdmd_sketch_gather(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               const cdmd_measure* meas, double* DY, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && meas != nullptr, "ctx or meas is NULL");
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    CDMD_REQUIRE(DY != nullptr, "DY is NULL");
    CDMD_REQUIRE(meas->m == m, "meas was built for m = %lld, video has m = %lld", static_cast<long long>(meas->m),
                 static_cast<long long>(m));
    CDMD_REQUIRE(meas->ctype == CDMD_C_SPARSE || meas->ctype == CDMD_C_ROWSAMPLE || meas->ctype == CDMD_C_SRFT,
                 "meas must be SPARSE, ROWSAMPLE or SRFT");
    if (meas->ctype == CDMD_C_SPARSE) {
        CDMD_REQUIRE(meas->col_ptr && meas->row_idx, "CSC arrays are NULL");
        CDMD_REQUIRE(static_cast<size_t>(meas->k) * 17 * sizeof(int32_t) <= 232448,
                     "SPARSE gather supports k <= %d", static_cast<int>(232448 / 68));
    } else {
        CDMD_REQUIRE(meas->rows != nullptr, "meas->rows is NULL");
    }
    DeviceGuard g(ctx->device);
    return launch_sketch_gather(ctx, D, m, n, ldd, meas, DY, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_decompose(cdmd_ctx* ctx, const double* DY, int k, int n, int r, int K, cdmd_selector selector,
                           double* sigma, double* lambda, double* G, double* PhiY, double* beta, int32_t* sel,
                           int32_t* nsel, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(DY && sigma && lambda && G && beta && sel && nsel, "a required pointer is NULL");
    CDMD_REQUIRE(n >= 2 && n <= 512, "n must be in [2, 512] (got %d)", n);
    CDMD_REQUIRE(k >= 1, "k must be >= 1");
    CDMD_REQUIRE(r >= 1 && r <= 32 && r <= k && r <= n - 1, "r must be in [1, min(32, k, n-1)] (got %d)", r);
    CDMD_REQUIRE(K >= 1 && K <= r, "K must be in [1, r] (got %d)", K);
    CDMD_REQUIRE(selector == CDMD_SEL_OMP || selector == CDMD_SEL_LSTSQ || selector == CDMD_SEL_MLP,
                 "unknown selector %d", static_cast<int>(selector));
    CDMD_REQUIRE(selector != CDMD_SEL_MLP || ctx->selector_loaded,
                 "CDMD_SEL_MLP needs a model (cdmd_selector_load)");
    DeviceGuard g(ctx->device);
    return launch_decompose(ctx, DY, k, n, r, K, selector, sigma, lambda, G, PhiY, beta, sel, nsel,
                            static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_decompose_auto(cdmd_ctx* ctx, const double* DY, int k, int n, int r_max, int K,
                                cdmd_selector selector, double* sigma, double* lambda, double* G, double* PhiY,
                                double* beta, int32_t* sel, int32_t* nsel, int* r_out, double* tau_out, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(DY && sigma && lambda && G && beta && sel && nsel && r_out, "a required pointer is NULL");
    CDMD_REQUIRE(n >= 2 && n <= 512, "n must be in [2, 512] (got %d)", n);
    CDMD_REQUIRE(k >= 1, "k must be >= 1");
    CDMD_REQUIRE(r_max >= 1 && r_max <= 32 && r_max <= k && r_max <= n - 1,
                 "r_max must be in [1, min(32, k, n-1)] (got %d)", r_max);
    CDMD_REQUIRE(K >= 1 && K <= r_max, "K must be in [1, r_max] (got %d)", K);
    CDMD_REQUIRE(selector == CDMD_SEL_OMP || selector == CDMD_SEL_LSTSQ || selector == CDMD_SEL_MLP,
                 "unknown selector %d", static_cast<int>(selector));
    CDMD_REQUIRE(selector != CDMD_SEL_MLP || ctx->selector_loaded,
                 "CDMD_SEL_MLP needs a model (cdmd_selector_load)");
    DeviceGuard g(ctx->device);
    return launch_decompose_auto(ctx, DY, k, n, r_max, K, selector, sigma, lambda, G, PhiY, beta, sel, nsel, r_out,
                                 tau_out, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_snapshot_gram(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, double* R,
                               void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    CDMD_REQUIRE(R != nullptr && aligned(R, 8), "R is NULL or not 8-byte aligned");
    DeviceGuard g(ctx->device);
    return launch_gram_tc(ctx, D, m, n, ldd, R, static_cast<cudaStream_t>(stream));
}

static cdmd_status check_exact_selector(cdmd_selector selector) {
    CDMD_REQUIRE(selector == CDMD_SEL_OMP || selector == CDMD_SEL_LSTSQ,
                 "exact DMD selects by OMP or least squares (got selector %d)", static_cast<int>(selector));
    return CDMD_OK;
}

cdmd_status cdmd_decompose_gram(cdmd_ctx* ctx, const double* R, int n, int r, int K, cdmd_selector selector,
                                double* sigma, double* lambda, double* G, double* beta, int32_t* sel, int32_t* nsel,
                                void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(R && sigma && lambda && G && beta && sel && nsel, "a required pointer is NULL");
    CDMD_REQUIRE(n >= 2 && n <= 512, "n must be in [2, 512] (got %d)", n);
    CDMD_REQUIRE(r >= 1 && r <= 32 && r <= n - 1, "r must be in [1, min(32, n-1)] (got %d)", r);
    CDMD_REQUIRE(K >= 1 && K <= r, "K must be in [1, r] (got %d)", K);
    cdmd_status st = check_exact_selector(selector);
    if (st != CDMD_OK) return st;
    DeviceGuard g(ctx->device);
    return launch_decompose_gram(ctx, R, n, r, K, selector, sigma, lambda, G, beta, sel, nsel,
                                 static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_lift(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const double* G, int r,
                      const int32_t* cols, int ncols, cdmd_prec prec, float* Phi, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    CDMD_REQUIRE(G != nullptr && Phi != nullptr, "G or Phi is NULL");
    CDMD_REQUIRE(n <= 512, "n must be <= 512");
    CDMD_REQUIRE(r >= 1 && ncols >= 1 && ncols <= 64, "need r >= 1 and 1 <= ncols <= 64");
    CDMD_REQUIRE(cols != nullptr || ncols <= r, "ncols > r needs an explicit cols list");
    CDMD_REQUIRE(aligned(Phi, 8), "Phi must be 8-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == CDMD_PREC_FP32) return launch_lift_fp32(ctx, D, m, n, ldd, G, r, cols, ncols, Phi, s);
    if (prec == CDMD_PREC_BF16X2) return launch_lift_tc(ctx, D, m, n, ldd, G, r, cols, ncols, Phi, s);
    return fail(CDMD_ERR_INVALID_ARG, "unknown precision %d", static_cast<int>(prec));
}

cdmd_status cdmd_subtract(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const float* Phi, int ncols,
                          const int32_t* cols, const double* beta, const double* lambda, int r, float tau,
                          cdmd_bgmode mode, uint32_t* mask, float* bg, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    CDMD_REQUIRE(Phi && beta && lambda && mask, "a required pointer is NULL");
    CDMD_REQUIRE(n <= 512, "n must be <= 512");
    CDMD_REQUIRE(ncols >= 1 && ncols <= 32, "ncols must be in [1, 32]");
    CDMD_REQUIRE(r >= 1, "r must be >= 1");
    CDMD_REQUIRE(cols != nullptr || ncols <= r, "ncols > r needs an explicit cols list");
    CDMD_REQUIRE(tau >= 0.0f, "tau must be >= 0");
    CDMD_REQUIRE(mode == CDMD_BG_MODULUS || mode == CDMD_BG_REAL || mode == CDMD_BG_STATIC, "unknown background mode");
    CDMD_REQUIRE(aligned(Phi, 8), "Phi must be 8-byte aligned");
    DeviceGuard g(ctx->device);
    return launch_subtract(ctx, D, m, n, ldd, Phi, ncols, cols, beta, lambda, r, tau, mode, mask, bg,
                           static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_median3x3(cdmd_ctx* ctx, const uint32_t* mask, int64_t W, int64_t H, int n, uint32_t* out,
                           void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && mask != nullptr && out != nullptr, "ctx, mask or out is NULL");
    CDMD_REQUIRE(W >= 1 && H >= 1, "W and H must be >= 1");
    CDMD_REQUIRE(W <= 0x7fffffffLL / H, "W*H must be <= 2^31 - 1");
    CDMD_REQUIRE(n >= 1 && n <= 262140, "n must be in [1, 262140]");
    CDMD_REQUIRE(aligned(mask, 4) && aligned(out, 4), "mask and out must be 4-byte aligned");
    const int64_t bytes = (W * H + 31) / 32 * 4 * static_cast<int64_t>(n);
    const uintptr_t a = reinterpret_cast<uintptr_t>(mask), b = reinterpret_cast<uintptr_t>(out);
    CDMD_REQUIRE(a + bytes <= b || b + bytes <= a, "mask and out overlap");
    DeviceGuard g(ctx->device);
    return launch_median3x3(mask, W, H, n, out, static_cast<cudaStream_t>(stream));
}

namespace {

cdmd_status check_run(const uint8_t* D, int64_t m, int n, int64_t ldd, const cdmd_params* p) {
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    const int k = p->k, r = p->r, K = p->K;
    CDMD_REQUIRE(k >= 1, "k must be >= 1");
    CDMD_REQUIRE(r == 0 || (r >= 1 && r <= 32 && r <= k && r <= n - 1),
                 "r must be 0 (automatic) or in [1, min(32, k, n-1)]");
    const int r_bound = r == 0 ? std::min(32, std::min(k, n - 1)) : r;
    CDMD_REQUIRE(K >= 1 && K <= r_bound, "K must be in [1, r] (r = 0: [1, min(32, k, n-1)])");
    return CDMD_OK;
}

// Steps 4-9 of cdmd_run on a sketch DY already in device memory, or, with
// DY NULL, of exact DMD on the snapshot Gram R (the context's small-solve and
// Phi buffers are reused, stream-ordered).
cdmd_status run_from(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const cdmd_params* p,
                     double* DY, const double* R, uint32_t* mask, void* stream) {
    const int k = p->k, K = p->K;
    // r == 0: the rank comes from the optimal hard threshold (Remark 2), at
    // most min(32, k, n-1); buffers are sized for that bound
    const bool auto_rank = p->r == 0;
    int r = auto_rank ? std::min(32, std::min(k, n - 1)) : p->r;
    const int p1 = n - 1;
    const int ncols_max = (p->selector == CDMD_SEL_LSTSQ) ? r : K;
    void* v = nullptr;
    const size_t n_small = static_cast<size_t>(r) + 2 * r + 2 * static_cast<size_t>(p1) * r + 2 * r + 8;
    cdmd_status st = ensure_buffer(ctx, BUF_RUN_SMALL, n_small * sizeof(double) + (r + 8) * sizeof(int32_t), &v);
    if (st != CDMD_OK) return st;
    double* sigma = static_cast<double*>(v);
    double* lambda = sigma + r;
    double* Gm = lambda + 2 * r;
    double* beta = Gm + 2 * static_cast<size_t>(p1) * r;
    int32_t* sel = reinterpret_cast<int32_t*>(beta + 2 * r + 8);
    int32_t* nsel = sel + r + 4;
    st = ensure_buffer(ctx, BUF_RUN_PHI, static_cast<size_t>(m) * ncols_max * 2 * sizeof(float), &v);
    if (st != CDMD_OK) return st;
    float* Phi = static_cast<float*>(v);
    ctx->run_DY = DY; ctx->run_sigma = sigma; ctx->run_lambda = lambda; ctx->run_G = Gm;
    ctx->run_beta = beta; ctx->run_sel = sel; ctx->run_nsel = nsel; ctx->run_Phi = Phi;

    if (DY != nullptr && auto_rank)
        st = cdmd_decompose_auto(ctx, DY, k, n, r, K, p->selector, sigma, lambda, Gm, nullptr, beta, sel, nsel, &r,
                                 nullptr, stream);
    else if (DY != nullptr)
        st = cdmd_decompose(ctx, DY, k, n, r, K, p->selector, sigma, lambda, Gm, nullptr, beta, sel, nsel, stream);
    else
        st = cdmd_decompose_gram(ctx, R, n, r, K, p->selector, sigma, lambda, Gm, beta, sel, nsel, stream);
    if (st != CDMD_OK) return st;
    const int ncols = (p->selector == CDMD_SEL_LSTSQ) ? r : std::min(K, r);
    // OMP: lift and subtract only the selected modes (sel, -1 padded);
    // LSTSQ: every mode carries an amplitude, so all r are used.
    const int32_t* cols = (p->selector == CDMD_SEL_LSTSQ) ? nullptr : sel;
    st = cdmd_lift(ctx, D, m, n, ldd, Gm, r, cols, ncols, p->prec, Phi, stream);
    if (st != CDMD_OK) return st;
    return cdmd_subtract(ctx, D, m, n, ldd, Phi, ncols, cols, beta, lambda, r, p->tau, p->bgmode, mask, nullptr,
                         stream);
}

}  // namespace

cdmd_status cdmd_run(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const cdmd_params* p,
                     uint32_t* mask, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && p != nullptr && mask != nullptr, "ctx, params or mask is NULL");
    cdmd_status st = check_run(D, m, n, ldd, p);
    if (st != CDMD_OK) return st;
    DeviceGuard g(ctx->device);
    void* v = nullptr;
    st = ensure_buffer(ctx, BUF_RUN_DY, static_cast<size_t>(p->k) * n * sizeof(double), &v);
    if (st != CDMD_OK) return st;
    double* DY = static_cast<double*>(v);
    st = cdmd_sketch(ctx, D, m, n, ldd, p->ctype, p->k, p->seed, p->prec, DY, stream);
    if (st != CDMD_OK) return st;
    return run_from(ctx, D, m, n, ldd, p, DY, nullptr, mask, stream);
}

cdmd_status cdmd_run_exact(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const cdmd_params* p,
                           uint32_t* mask, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && p != nullptr && mask != nullptr, "ctx, params or mask is NULL");
    cdmd_status st = check_video(D, m, n, ldd);
    if (st != CDMD_OK) return st;
    CDMD_REQUIRE(p->r >= 1 && p->r <= 32 && p->r <= n - 1 && p->r <= m, "r must be in [1, min(32, m, n-1)]");
    CDMD_REQUIRE(p->K >= 1 && p->K <= p->r, "K must be in [1, r]");
    st = check_exact_selector(p->selector);
    if (st != CDMD_OK) return st;
    DeviceGuard g(ctx->device);
    void* v = nullptr;
    st = ensure_buffer(ctx, BUF_RUN_GRAM, static_cast<size_t>(n) * n * sizeof(double), &v);
    if (st != CDMD_OK) return st;
    double* R = static_cast<double*>(v);
    st = cdmd_snapshot_gram(ctx, D, m, n, ldd, R, stream);
    if (st != CDMD_OK) return st;
    return run_from(ctx, D, m, n, ldd, p, nullptr, R, mask, stream);
}

cdmd_status cdmd_run_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m, const int* n,
                            const int64_t* ldd, const cdmd_params* p, uint32_t* const* mask, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && p != nullptr, "ctx or params is NULL");
    CDMD_REQUIRE(nclips >= 1, "nclips must be >= 1 (got %d)", nclips);
    CDMD_REQUIRE(D != nullptr && n != nullptr && ldd != nullptr && mask != nullptr, "NULL array argument");
    size_t off[kMaxSharedRun + 1] = {0};
    CDMD_REQUIRE(nclips <= kMaxSharedRun, "nclips must be <= %d (got %d)", kMaxSharedRun, nclips);
    for (int i = 0; i < nclips; ++i) {
        cdmd_status st = check_run(D[i], m, n[i], ldd[i], p);
        if (st != CDMD_OK) return fail_clip(st, i);
        CDMD_REQUIRE(mask[i] != nullptr, "clip %d: mask is NULL", i);
        off[i + 1] = off[i] + static_cast<size_t>(p->k) * n[i];
    }
    DeviceGuard g(ctx->device);
    void* v = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_RUN_DY, off[nclips] * sizeof(double), &v);
    if (st != CDMD_OK) return st;
    double* DYs[kMaxSharedRun];
    for (int i = 0; i < nclips; ++i) DYs[i] = static_cast<double*>(v) + off[i];
    st = cdmd_sketch_shared(ctx, nclips, D, m, n, ldd, p->ctype, p->k, p->seed, p->prec, DYs, stream);
    if (st != CDMD_OK) return st;
    for (int i = 0; i < nclips; ++i) {
        st = run_from(ctx, D[i], m, n[i], ldd[i], p, DYs[i], nullptr, mask[i], stream);
        if (st != CDMD_OK) return st;
    }
    return CDMD_OK;
}

cdmd_status cdmd_run_host(cdmd_ctx* ctx, const uint8_t* D_host, int64_t m, int n, const cdmd_params* p,
                          uint32_t* mask_host, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && D_host != nullptr && mask_host != nullptr && p != nullptr, "NULL argument");
    cdmd_status st = check_video(D_host, m, n, m);
    if (st != CDMD_OK) return st;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vbytes = static_cast<size_t>(m) * n;
    const size_t wpf = static_cast<size_t>((m + 31) / 32);
    const size_t mbytes = wpf * n * sizeof(uint32_t);
    void* dv = nullptr;
    void* dm = nullptr;
    st = ensure_buffer(ctx, BUF_RUN_VIDEO, vbytes, &dv);
    if (st != CDMD_OK) return st;
    st = ensure_buffer(ctx, BUF_RUN_MASK, mbytes, &dm);
    if (st != CDMD_OK) return st;
    CDMD_CHECK_CUDA(cudaMemcpyAsync(dv, D_host, vbytes, cudaMemcpyHostToDevice, s));
    st = cdmd_run(ctx, static_cast<const uint8_t*>(dv), m, n, m, p, static_cast<uint32_t*>(dm), stream);
    if (st != CDMD_OK) return st;
    CDMD_CHECK_CUDA(cudaMemcpyAsync(mask_host, dm, mbytes, cudaMemcpyDeviceToHost, s));
    return cdmd_status_sync(ctx, stream);
}

cdmd_status cdmd_run_host_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D_host, int64_t m, const int* n,
                                 const cdmd_params* p, uint32_t* const* mask_host, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && p != nullptr && D_host != nullptr && n != nullptr && mask_host != nullptr,
                 "NULL argument");
    CDMD_REQUIRE(nclips >= 1 && nclips <= kMaxSharedRun, "nclips must be in [1, %d] (got %d)", kMaxSharedRun, nclips);
    size_t voff[kMaxSharedRun + 1] = {0}, moff[kMaxSharedRun + 1] = {0};
    const size_t wpf = static_cast<size_t>((m + 31) / 32);
    for (int i = 0; i < nclips; ++i) {
        CDMD_REQUIRE(D_host[i] != nullptr && mask_host[i] != nullptr, "clip %d: NULL buffer", i);
        cdmd_status st = check_video(D_host[i], m, n[i], m);
        if (st != CDMD_OK) return fail_clip(st, i);
        voff[i + 1] = voff[i] + (static_cast<size_t>(m) * n[i] + 255) / 256 * 256;
        moff[i + 1] = moff[i] + wpf * n[i] * sizeof(uint32_t);
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* dv = nullptr;
    void* dm = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_RUN_VIDEO, voff[nclips], &dv);
    if (st != CDMD_OK) return st;
    st = ensure_buffer(ctx, BUF_RUN_MASK, moff[nclips], &dm);
    if (st != CDMD_OK) return st;
    const uint8_t* Dd[kMaxSharedRun];
    uint32_t* Md[kMaxSharedRun];
    int64_t ldd[kMaxSharedRun];
    for (int i = 0; i < nclips; ++i) {
        Dd[i] = static_cast<const uint8_t*>(dv) + voff[i];
        Md[i] = reinterpret_cast<uint32_t*>(static_cast<char*>(dm) + moff[i]);
        ldd[i] = m;
        CDMD_CHECK_CUDA(cudaMemcpyAsync(const_cast<uint8_t*>(Dd[i]), D_host[i], static_cast<size_t>(m) * n[i],
                                        cudaMemcpyHostToDevice, s));
    }
    st = cdmd_run_shared(ctx, nclips, Dd, m, n, ldd, p, Md, stream);
    if (st != CDMD_OK) return st;
    for (int i = 0; i < nclips; ++i)
        CDMD_CHECK_CUDA(cudaMemcpyAsync(mask_host[i], Md[i], moff[i + 1] - moff[i], cudaMemcpyDeviceToHost, s));
    return cdmd_status_sync(ctx, stream);
}

cdmd_status cdmd_workspace_views(cdmd_ctx* ctx, double** DY, double** sigma, double** lambda, double** G,
                                 double** beta, int32_t** sel, int32_t** nsel, float** Phi) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(ctx->run_DY != nullptr, "no cdmd_run on this context yet");
    if (DY) *DY = ctx->run_DY;
    if (sigma) *sigma = ctx->run_sigma;
    if (lambda) *lambda = ctx->run_lambda;
    if (G) *G = ctx->run_G;
    if (beta) *beta = ctx->run_beta;
    if (sel) *sel = ctx->run_sel;
    if (nsel) *nsel = ctx->run_nsel;
    if (Phi) *Phi = ctx->run_Phi;
    return CDMD_OK;
}


// ---------------------------------------------------------------------------
// learned mode selector
// ---------------------------------------------------------------------------

cdmd_status cdmd_selector_load(cdmd_ctx* ctx, const float* blob, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(blob != nullptr, "blob is NULL");
    DeviceGuard g(ctx->device);
    void* buf = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SELECTOR, kSelBytes, &buf);
    if (st != CDMD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CDMD_CHECK_CUDA(cudaMemcpyAsync(buf, blob, CDMD_MLP_BLOB * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CDMD_CHECK_CUDA(cudaMemsetAsync(static_cast<char*>(buf) + kSelOrderOff, 0, kSelBytes - kSelOrderOff, s));
    ctx->selector_loaded = true;
    return CDMD_OK;
}

cdmd_status cdmd_selector_features(cdmd_ctx* ctx, const double* lambda, const int32_t* sel, int r, int K,
                                   float* feats, float* labels, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(lambda != nullptr && feats != nullptr, "lambda and feats are required");
    CDMD_REQUIRE(ctx->last_M != nullptr && ctx->last_r == r, "no decomposition with r = %d on this context", r);
    CDMD_REQUIRE(K >= 0 && K <= r, "K must be in [0, r] (got %d)", K);
    CDMD_REQUIRE(labels == nullptr || sel != nullptr || K == 0, "labels need sel");
    DeviceGuard g(ctx->device);
    return launch_selector_features(ctx, lambda, sel, r, K, feats, labels, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_selector_relabel(cdmd_ctx* ctx, const double* DY, int k, int n, const double* G,
                                  const double* lambda, int r, const double* y_target, int K, int32_t* sel,
                                  void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(DY && G && lambda && y_target && sel, "DY, G, lambda, y_target and sel are required");
    CDMD_REQUIRE(ctx->last_M != nullptr && ctx->last_r == r, "no decomposition with r = %d on this context", r);
    CDMD_REQUIRE(n >= 2 && n <= 512 && k >= 1, "bad sizes");
    CDMD_REQUIRE(K >= 1 && K <= r, "K must be in [1, r] (got %d)", K);
    DeviceGuard g(ctx->device);
    return launch_selector_relabel(ctx, DY, k, n, G, lambda, r, y_target, K, sel, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_selector_fallbacks(cdmd_ctx* ctx, int64_t* count, int reset, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && count != nullptr, "ctx and count are required");
    CDMD_REQUIRE(ctx->selector_loaded, "no selector model loaded");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long v = 0;
    CDMD_CHECK_CUDA(cudaMemcpyAsync(&v, selector_fallbacks(ctx), sizeof(v), cudaMemcpyDeviceToHost, s));
    if (reset) CDMD_CHECK_CUDA(cudaMemsetAsync(selector_fallbacks(ctx), 0, sizeof(v), s));
    CDMD_CHECK_CUDA(cudaStreamSynchronize(s));
    *count = static_cast<int64_t>(v);
    return CDMD_OK;
}

cdmd_status cdmd_mlp_forward(cdmd_ctx* ctx, const float* blob, const float* X, int64_t N, int bf16, float* s,
                             float* p, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(blob != nullptr && (X != nullptr || N == 0), "blob and X are required");
    CDMD_REQUIRE(N >= 0, "N must be >= 0");
    DeviceGuard g(ctx->device);
    return launch_mlp_forward(ctx, blob, X, N, bf16, s, p, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_mlp_grad(cdmd_ctx* ctx, const float* blob, const float* X, const float* Y, int64_t N, float* grad,
                          float* loss, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(blob && X && Y && grad, "blob, X, Y and grad are required");
    CDMD_REQUIRE(N >= 1, "N must be >= 1");
    DeviceGuard g(ctx->device);
    return launch_mlp_train(ctx, 0, const_cast<float*>(blob), nullptr, nullptr, 1, 0.0f, 0.0f, 0.0f, 0.0f, X, Y, N,
                            grad, loss, static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_mlp_train_step(cdmd_ctx* ctx, float* blob, float* m, float* v, int step, float lr, float beta1,
                                float beta2, float eps, const float* X, const float* Y, int64_t N, float* loss,
                                void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr, "ctx is NULL");
    CDMD_REQUIRE(blob && m && v && X && Y, "blob, m, v, X and Y are required");
    CDMD_REQUIRE(N >= 1 && step >= 1, "N and step must be >= 1");
    CDMD_REQUIRE(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f,
                 "Adam needs 0 <= beta1, beta2 < 1 and eps > 0");
    DeviceGuard g(ctx->device);
    return launch_mlp_train(ctx, 1, blob, m, v, step, lr, beta1, beta2, eps, X, Y, N, nullptr, loss,
                            static_cast<cudaStream_t>(stream));
}

cdmd_status cdmd_synth_clip(cdmd_ctx* ctx, int width, int height, int n, const float* waves, int nw,
                            const float* objects, int nobj, int ellipse, float drift, float noise_sigma,
                            uint64_t seed, uint8_t* D, int64_t ldd, void* stream) {
    clear_error();
    CDMD_REQUIRE(ctx != nullptr && D != nullptr, "ctx and D are required");
    CDMD_REQUIRE(width >= 1 && height >= 1 && n >= 1, "width, height and n must be >= 1");
    CDMD_REQUIRE(n <= 65535, "n must be <= 65535");
    CDMD_REQUIRE(ldd >= static_cast<int64_t>(width) * height, "ldd must be >= width * height");
    CDMD_REQUIRE(nw >= 0 && (nw == 0 || waves != nullptr), "waves missing");
    CDMD_REQUIRE(nobj >= 0 && (nobj == 0 || objects != nullptr), "objects missing");
    DeviceGuard g(ctx->device);
    return launch_synth_clip(width, height, n, waves, nw, objects, nobj, ellipse, drift, noise_sigma, seed, D, ldd,
                             static_cast<cudaStream_t>(stream));
}

}  // extern "C"
