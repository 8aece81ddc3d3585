// Internal declarations shared by the libcdmd translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>

#include "cdmd.h"

namespace cdmd {

// ---------------------------------------------------------------------------
// Host-side error plumbing: every extern "C" entry returns a cdmd_status and
// leaves a message in a thread-local buffer (cdmd_last_error).
// ---------------------------------------------------------------------------
cdmd_status fail(cdmd_status s, const char* fmt, ...);
cdmd_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define CDMD_CHECK_CUDA(call)                                          \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return ::cdmd::cuda_fail(_e, #call);    \
    } while (0)

#define CDMD_CHECK_LAUNCH(name)                                        \
    do {                                                               \
        cudaError_t _e = cudaGetLastError();                           \
        if (_e != cudaSuccess) return ::cdmd::cuda_fail(_e, name);     \
    } while (0)

#define CDMD_REQUIRE(cond, ...)                                        \
    do {                                                               \
        if (!(cond)) return ::cdmd::fail(CDMD_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

// Device status word: the first numerical error recorded wins.
__device__ __forceinline__ void record_status(int* status, int code) {
    if (status != nullptr) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 bit products with Weyl-bumped round keys.
// ---------------------------------------------------------------------------
// 1/a and 1/sqrt(a) in FP64 by the Newton-Raphson method: start from the
// hardware's approximate reciprocal (rcp.approx.ftz.f64) or reciprocal square
// root (rsqrt.approx.ftz.f64) and take two Newton steps for the root of
// f(x) = 1/x - a, x <- x (2 - a x) = x + x (1 - a x), or of f(y) = 1/y^2 - a,
// y <- y (3 - a y^2) / 2 = y + y (1/2 - (a/2) y^2).  Each step roughly doubles
// the number of correct bits, so two steps from the approximation reach FP64
// rounding level (a few ulp; bounded by a GPU test against IEEE division and
// square root).  Zero and subnormal inputs are flushed (ftz); callers pass
// normal positive values.  They replace a division or square root (hundreds of
// cycles in FP64 on this GPU) on the latency-critical paths of the small solves.
__device__ __forceinline__ double rcp64(double a) {
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(a));
    double e = fma(-a, x, 1.0);
    x = fma(x, e, x);
    e = fma(-a, x, 1.0);
    x = fma(x, e, x);
    return x;
}

__device__ __forceinline__ double rsqrt64(double a) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    const double h = 0.5 * a;
    double t = fma(-h * y, y, 0.5);
    y = fma(y, t, y);
    t = fma(-h * y, y, 0.5);
    y = fma(y, t, y);
    return y;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 key) {
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd > 0) {
            key.x += 0x9E3779B9u;
            key.y += 0xBB67AE85u;
        }
        // one 32x32 -> 64-bit product per word pair (a single wide multiply)
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ key.x, static_cast<uint32_t>(p1),
                       static_cast<uint32_t>(p0 >> 32) ^ c.w ^ key.y, static_cast<uint32_t>(p0));
    }
    return c;
}

// The same generator with its ten round keys computed once by the caller
// (key + i * (0x9E3779B9, 0xBB67AE85)); for loops that draw many counters
// under one key.
struct PhiloxKeys {
    uint32_t x[10], y[10];
};
__host__ __device__ __forceinline__ PhiloxKeys philox_round_keys(uint2 key) {
    PhiloxKeys k;
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        k.x[rnd] = key.x + static_cast<uint32_t>(rnd) * 0x9E3779B9u;
        k.y[rnd] = key.y + static_cast<uint32_t>(rnd) * 0xBB67AE85u;
    }
    return k;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& k) {
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k.x[rnd], static_cast<uint32_t>(p1),
                       static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k.y[rnd], static_cast<uint32_t>(p0));
    }
    return c;
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
    return make_uint2(static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32));
}

// Box-Muller pair from two Philox words, FP32, accurate library functions.
// U(w) = (w + 1/2) 2^-32.  ln U is taken as logf(U) when U < 1/2 and as
// log1pf(-(1 - U)) otherwise, where 1 - U = (~w + 1/2) 2^-32 is formed from
// the integer, so neither branch cancels.  The angle 2 pi U(wb) is split into
// a quarter turn q (top two bits of wb) and a remainder f = (low 30 bits +
// 1/2) 2^-30 in (0, 1) so that sincospif sees an argument below 1/2.
__device__ __forceinline__ void box_muller_accurate(uint32_t wa, uint32_t wb, float& z_cos, float& z_sin) {
    const float two_m32 = 2.3283064365386963e-10f;   // 2^-32
    float ln_u;
    if (wa < 0x80000000u) {
        ln_u = logf((__uint2float_rn(wa) + 0.5f) * two_m32);
    } else {
        ln_u = log1pf(-((__uint2float_rn(~wa) + 0.5f) * two_m32));
    }
    const float radius = sqrtf(-2.0f * ln_u);
    const uint32_t quarter = wb >> 30;
    const float f = (__uint2float_rn(wb & 0x3fffffffu) + 0.5f) * 9.313225746154785e-10f;   // 2^-30
    float s, c;
    sincospif(0.5f * f, &s, &c);
    float cs, sn;   // rotate by quarter * pi/2
    switch (quarter) {
        case 0: cs = c; sn = s; break;
        case 1: cs = -s; sn = c; break;
        case 2: cs = -c; sn = -s; break;
        default: cs = s; sn = -c; break;
    }
    z_cos = radius * cs;
    z_sin = radius * sn;
}

// Four Gaussian entries C[4q + 0..3, j] from counter (j, q, 0, 0).
__device__ __forceinline__ float4 gaussian_quad(uint2 key, uint32_t j, uint32_t q) {
    const uint4 w = philox4x32_10(make_uint4(j, q, 0u, 0u), key);
    float4 z;
    box_muller_accurate(w.x, w.y, z.x, z.y);
    box_muller_accurate(w.z, w.w, z.z, z.w);
    return z;
}

// Four Rademacher entries C[4q + 0..3, j]: bits of counter (j, i/128, 1, 0).
__device__ __forceinline__ float4 rademacher_quad(uint2 key, uint32_t j, uint32_t q) {
    const uint32_t i0 = 4u * q;
    const uint4 w = philox4x32_10(make_uint4(j, i0 >> 7, 1u, 0u), key);
    const uint32_t b = i0 & 127u;
    const uint32_t word = (b >> 5) == 0 ? w.x : (b >> 5) == 1 ? w.y : (b >> 5) == 2 ? w.z : w.w;
    const uint32_t bits = word >> (b & 31u);
    float4 z;
    z.x = (bits & 1u) ? -1.0f : 1.0f;
    z.y = (bits & 2u) ? -1.0f : 1.0f;
    z.z = (bits & 4u) ? -1.0f : 1.0f;
    z.w = (bits & 8u) ? -1.0f : 1.0f;
    return z;
}

// ---------------------------------------------------------------------------
// Context: device, status word and a grow-only workspace of named buffers.
// ---------------------------------------------------------------------------
struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

enum BufferId {
    BUF_SKETCH_PARTIAL = 0,   // sketch split partials (float)
    BUF_SKETCH_WIDE,          // BF16 copies of the frames of clips sketched together
    BUF_GRAM,                 // snapshot Gram split partials (float)
    BUF_EIG,                  // eigen-solver scratch (double)
    BUF_SMALL,                // small-solve scratch (double)
    BUF_RUN_DY,               // cdmd_run intermediates
    BUF_RUN_SMALL,
    BUF_RUN_PHI,
    BUF_RUN_VIDEO,            // cdmd_run_host device copy of the video
    BUF_RUN_MASK,
    BUF_SUBTRACT_TABLE,       // lambda^t table and amplitudes for pass (c)
    BUF_SELECTOR,             // selector model blob, pick order, accept flag, fallback count
    BUF_MLP_PARTS,            // selector training: per-warp partial gradients
    BUF_RELABEL,              // selector training: OMP against a second target
    BUF_RUN_GRAM,             // cdmd_run_exact: the n x n snapshot Gram (double)
    BUF_COUNT
};

}  // namespace cdmd

struct cdmd_ctx {
    int device = 0;
    int device_sms = 0;    // SMs of the device
    int num_sms = 0;       // SMs the full-data passes size their grids for (cdmd_set_sm_limit)
    int* d_status = nullptr;
    cdmd::Buffer buf[cdmd::BUF_COUNT];
    bool selector_loaded = false;
    // Gram quantities of the last cdmd_decompose (decompose workspace)
    const double* last_M = nullptr;
    const double* last_cvec = nullptr;
    const double* last_R = nullptr;
    int last_r = 0;
    // views of the last cdmd_run
    double* run_DY = nullptr;
    double* run_sigma = nullptr;
    double* run_lambda = nullptr;
    double* run_G = nullptr;
    double* run_beta = nullptr;
    int32_t* run_sel = nullptr;
    int32_t* run_nsel = nullptr;
    float* run_Phi = nullptr;
};

namespace cdmd {

// Selector buffer: model blob (FP32, 2 KB slot), pick order (32 int32),
// accept flag (int), fallback count (uint64).
constexpr size_t kSelOrderOff = 2048;
constexpr size_t kSelAcceptOff = 2176;
constexpr size_t kSelFallbackOff = 2184;
constexpr size_t kSelBytes = 2304;
inline float* selector_blob(cdmd_ctx* ctx) { return static_cast<float*>(ctx->buf[BUF_SELECTOR].ptr); }
inline int32_t* selector_order(cdmd_ctx* ctx) {
    return reinterpret_cast<int32_t*>(static_cast<char*>(ctx->buf[BUF_SELECTOR].ptr) + kSelOrderOff);
}
inline int* selector_accept(cdmd_ctx* ctx) {
    return reinterpret_cast<int*>(static_cast<char*>(ctx->buf[BUF_SELECTOR].ptr) + kSelAcceptOff);
}
inline unsigned long long* selector_fallbacks(cdmd_ctx* ctx) {
    return reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->buf[BUF_SELECTOR].ptr) + kSelFallbackOff);
}

// Grow-only workspace buffer (never shrinks; synchronises the device before
// freeing an older, smaller allocation).
cdmd_status ensure_buffer(cdmd_ctx* ctx, BufferId id, size_t bytes, void** out);

// Pass launchers (implemented in the kernel translation units).
cdmd_status launch_sketch_fp32(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               cdmd_ctype ctype, int k, uint64_t seed, double* DY,
                               cudaStream_t stream);
cdmd_status launch_sketch_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                             cdmd_ctype ctype, int k, uint64_t seed, double* DY,
                             cudaStream_t stream);
// Several clips of the same pixel count sketched with one C (same k, seed):
// up to 512 frames of them share each draw of C.
cdmd_status launch_sketch_tc_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m, const int* n,
                                    const int64_t* ldd, cdmd_ctype ctype, int k, uint64_t seed, double* const* DY,
                                    cudaStream_t stream);
// The subtract pass's per-clip table as the tensor-core pass reads it: the
// amplitudes and lambda^t powers per selected column and, when the selected
// modes are real or complete conjugate pairs (hdr[1] = 1), per real term
// (hdr[0] terms, Phi column term_col[e], amplitude term_amp[e]).
struct SubTcTable {
    const int* hdr;
    const int* term_col;
    const float2* amp;           // beta per column
    const float2* term_amp;      // 2 beta per pair, beta per real mode
    const float2* lam_t;         // lambda^t per column, [n][nc_pad]
    const float2* term_lam_t;    // lambda^t per real term, [n][nc_pad]
};
// Pass (c) on the tensor cores for mask-only MODULUS / REAL calls with
// 32 <= n <= 1024 frames, ncols <= 16, a 16-byte aligned video and Phi.
bool subtract_tc_supported(int n, int ncols, cdmd_bgmode mode, const uint8_t* D, int64_t ldd, int64_t m,
                           const float* Phi, const float* bg);
cdmd_status launch_subtract_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const float* Phi,
                               int ncols, const SubTcTable& tb, int nc_pad, float tau, cdmd_bgmode mode,
                               uint32_t* mask, cudaStream_t stream);
cdmd_status launch_selftest_wait(cdmd_ctx* ctx, uint64_t limit_ns, cudaStream_t stream);
cdmd_status launch_selftest_recip(const double* a, int64_t n, double* r, double* q, cudaStream_t stream);
cdmd_status launch_gram_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, double* R,
                           cudaStream_t stream);
cdmd_status launch_decompose_auto(cdmd_ctx* ctx, const double* DY, int k, int n, int r_max, int K,
                                  cdmd_selector selector, double* sigma, double* lambda, double* G, double* PhiY,
                                  double* beta, int32_t* sel, int32_t* nsel, int* r_out, double* tau_out,
                                  cudaStream_t stream);
cdmd_status launch_decompose_gram(cdmd_ctx* ctx, const double* R, int n, int r, int K, cdmd_selector selector,
                                  double* sigma, double* lambda, double* G, double* beta, int32_t* sel,
                                  int32_t* nsel, cudaStream_t stream);
cdmd_status launch_median3x3(const uint32_t* mask, int64_t W, int64_t H, int n, uint32_t* out,
                             cudaStream_t stream);
cdmd_status launch_sketch_gather(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                                 const cdmd_measure* meas, double* DY, cudaStream_t stream);
cdmd_status launch_measure_sparse_count(cdmd_ctx* ctx, int64_t m, int k, uint64_t seed,
                                        double density, int64_t* d_counts, cudaStream_t stream);
cdmd_status launch_measure_build(cdmd_ctx* ctx, cdmd_measure* meas, cudaStream_t stream);
cdmd_status launch_sketch_srft(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               const cdmd_measure* meas, double* DY, cudaStream_t stream);
cdmd_status launch_decompose(cdmd_ctx* ctx, const double* DY, int k, int n, int r, int K,
                             cdmd_selector selector, double* sigma, double* lambda, double* G,
                             double* PhiY, double* beta, int32_t* sel, int32_t* nsel,
                             cudaStream_t stream);
cdmd_status launch_lift_fp32(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                             const double* G, int r, const int32_t* cols, int ncols, float* Phi,
                             cudaStream_t stream);
cdmd_status launch_lift_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                           const double* G, int r, const int32_t* cols, int ncols, float* Phi,
                           cudaStream_t stream);
cdmd_status launch_subtract(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                            const float* Phi, int ncols, const int32_t* cols, const double* beta,
                            const double* lambda, int r, float tau, cdmd_bgmode mode,
                            uint32_t* mask, float* bg, cudaStream_t stream);
cdmd_status launch_synth_clip(int width, int height, int n, const float* waves, int nw, const float* objects,
                              int nobj, int ellipse, float drift, float noise_sigma, uint64_t seed, uint8_t* D,
                              int64_t ldd, cudaStream_t stream);
cdmd_status launch_selector_features(cdmd_ctx* ctx, const double* lambda, const int32_t* sel, int r, int K,
                                     float* feats, float* labels, cudaStream_t stream);
cdmd_status launch_selector_relabel(cdmd_ctx* ctx, const double* DY, int k, int n, const double* G,
                                    const double* lambda, int r, const double* y_target, int K, int32_t* sel,
                                    cudaStream_t stream);
cdmd_status launch_mlp_select(cdmd_ctx* ctx, const double* lambda, const double* M, const double* cvec,
                              const double* R, int r, int K, cudaStream_t stream);
cdmd_status launch_mlp_forward(cdmd_ctx* ctx, const float* blob, const float* X, int64_t N, int bf16,
                               float* s, float* p, cudaStream_t stream);
cdmd_status launch_mlp_train(cdmd_ctx* ctx, int apply, float* blob, float* m, float* v, int step, float lr,
                             float beta1, float beta2, float eps, const float* X, const float* Y, int64_t N,
                             float* grad, float* loss, cudaStream_t stream);

}  // namespace cdmd
