// Pass (a), plain form: DY = C D with C generated in-kernel (Algorithm 1
// steps 2-3, Eq. YCX), FP32 CUDA-core FMA.
//
// Grid: (row tiles of 64 rows of C) x (pixel splits).  Each CTA walks its
// pixel range in chunks of 32 pixels: it draws the 64 x 32 block of C from
// Philox into shared memory, stages the 32 pixels of every frame (uint8 ->
// float) and accumulates a 64 x (frames) tile in registers: warp w owns rows
// 8w..8w+7, lane l owns frames l, l+32, ...  Every C entry is drawn once.
// Partial sums (one per split) are written as float [split][k][n] and summed
// in FP64 by sketch_reduce_kernel in a fixed order (deterministic).
#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr int kRowsPerCta = 64;
constexpr int kPixPerChunk = 32;
constexpr int kThreads = 256;

template <int TQ, int CTYPE>
__global__ void __launch_bounds__(kThreads, 2)
sketch_fp32_kernel(const uint8_t* __restrict__ D, int64_t m, int n_slab, int t0, int64_t ldd,
                   int k, uint2 key, int64_t pix_per_split, int n_total,
                   float* __restrict__ part) {
    constexpr int NP = 32 * TQ;      // padded frames of the slab
    constexpr int DS = NP + 1;       // shared row stride (odd: fewer conflicts)
    __shared__ __align__(16) float Cs[kPixPerChunk][kRowsPerCta];
    extern __shared__ float Ds[];    // [kPixPerChunk][DS]

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int row0 = blockIdx.x * kRowsPerCta;
    const int64_t pbeg = static_cast<int64_t>(blockIdx.y) * pix_per_split;
    const int64_t pend = min(m, pbeg + pix_per_split);

    for (int idx = tid; idx < kPixPerChunk * DS; idx += kThreads) Ds[idx] = 0.0f;

    float acc[8][TQ];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < TQ; ++q) acc[a][q] = 0.0f;

    const bool vec_ok = ((ldd & 3) == 0) && ((reinterpret_cast<uintptr_t>(D) & 3) == 0);

    for (int64_t j0 = pbeg; j0 < pend; j0 += kPixPerChunk) {
        __syncthreads();   // previous chunk fully consumed
        // C block: 16 quads of rows x 32 pixels = 512 Philox calls.
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = tid + kThreads * h;
            const int quad = c & 15;
            const int jj = c >> 4;
            const int64_t j = j0 + jj;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < pend && row0 + 4 * quad < k) {
                const uint32_t q = static_cast<uint32_t>((row0 >> 2) + quad);
                z = (CTYPE == CDMD_C_GAUSSIAN) ? gaussian_quad(key, static_cast<uint32_t>(j), q)
                                               : rademacher_quad(key, static_cast<uint32_t>(j), q);
            }
            *reinterpret_cast<float4*>(&Cs[jj][4 * quad]) = z;
        }
        // D block: frames t0 .. t0+n_slab-1, pixels j0 .. j0+31 (4 per thread).
        const bool full = vec_ok && (j0 + kPixPerChunk <= pend);
        for (int idx = tid; idx < n_slab * 8; idx += kThreads) {
            const int t = idx >> 3;
            const int g = idx & 7;
            const uint8_t* src = D + static_cast<int64_t>(t0 + t) * ldd + j0 + 4 * g;
            uint32_t w = 0;
            if (full) {
                w = __ldg(reinterpret_cast<const uint32_t*>(src));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + 4 * g + e < pend) w |= static_cast<uint32_t>(src[e]) << (8 * e);
            }
            float* dst = Ds + (4 * g) * DS + t;
            dst[0] = static_cast<float>(w & 255u);
            dst[DS] = static_cast<float>((w >> 8) & 255u);
            dst[2 * DS] = static_cast<float>((w >> 16) & 255u);
            dst[3 * DS] = static_cast<float>(w >> 24);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < kPixPerChunk; ++jj) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Cs[jj][warp * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Cs[jj][warp * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int q = 0; q < TQ; ++q) {
                const float b = Ds[jj * DS + lane + 32 * q];
#pragma unroll
                for (int a = 0; a < 8; ++a) acc[a][q] = fmaf(av[a], b, acc[a][q]);
            }
        }
    }
    // part[(split * k + i) * n_total + t0 + t]
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = row0 + warp * 8 + a;
        if (i >= k) continue;
        float* dst = part + (static_cast<int64_t>(blockIdx.y) * k + i) * n_total + t0;
#pragma unroll
        for (int q = 0; q < TQ; ++q) {
            const int t = lane + 32 * q;
            if (t < n_slab) dst[t] = acc[a][q];
        }
    }
}

// DY[t*k + i] = sum_s part[(s*k + i)*n + t], FP64, fixed order.
__global__ void sketch_reduce_kernel(const float* __restrict__ part, int splits, int k, int n,
                                     double* __restrict__ DY, int* status) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<int64_t>(k) * n) return;
    const int i = static_cast<int>(idx / n);
    const int t = static_cast<int>(idx % n);
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += static_cast<double>(part[(static_cast<int64_t>(sp) * k + i) * n + t]);
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    DY[static_cast<int64_t>(t) * k + i] = s;
}

template <int CTYPE>
cdmd_status launch_slab(int tq, dim3 grid, size_t smem, cudaStream_t stream, const uint8_t* D,
                        int64_t m, int n_slab, int t0, int64_t ldd, int k, uint2 key,
                        int64_t pps, int n_total, float* part) {
#define CDMD_SKETCH_CASE(TQV)                                                                    \
    case TQV: {                                                                                  \
        auto kern = sketch_fp32_kernel<TQV, CTYPE>;                                              \
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                             static_cast<int>(smem)));                           \
        kern<<<grid, kThreads, smem, stream>>>(D, m, n_slab, t0, ldd, k, key, pps, n_total, part); \
        break;                                                                                   \
    }
    switch (tq) {
        CDMD_SKETCH_CASE(1)
        CDMD_SKETCH_CASE(2)
        CDMD_SKETCH_CASE(3)
        CDMD_SKETCH_CASE(4)
        CDMD_SKETCH_CASE(5)
        CDMD_SKETCH_CASE(6)
        CDMD_SKETCH_CASE(7)
        CDMD_SKETCH_CASE(8)
        default:
            return fail(CDMD_ERR_INVALID_ARG, "internal: frame slab too wide");
    }
#undef CDMD_SKETCH_CASE
    CDMD_CHECK_LAUNCH("sketch_fp32_kernel");
    return CDMD_OK;
}

}  // namespace

cdmd_status launch_sketch_fp32(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               cdmd_ctype ctype, int k, uint64_t seed, double* DY,
                               cudaStream_t stream) {
    constexpr int kMaxSlab = 256;   // frames per launch (TQ <= 8)
    const int row_tiles = (k + kRowsPerCta - 1) / kRowsPerCta;
    const int64_t chunks = (m + kPixPerChunk - 1) / kPixPerChunk;
    // about two waves of two CTAs per SM; at least 16 chunks per split
    int64_t splits = (4LL * ctx->num_sms + row_tiles - 1) / row_tiles;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, (chunks + 15) / 16));
    splits = std::min<int64_t>(splits, 65535);
    const int64_t chunks_per_split = (chunks + splits - 1) / splits;
    const int64_t pps = chunks_per_split * kPixPerChunk;
    splits = (m + pps - 1) / pps;

    float* part = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL,
                                   static_cast<size_t>(splits) * k * n * sizeof(float),
                                   reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    const uint2 key = seed_key(seed);
    for (int t0 = 0; t0 < n; t0 += kMaxSlab) {
        const int n_slab = std::min(kMaxSlab, n - t0);
        const int tq = (n_slab + 31) / 32;
        const size_t smem = static_cast<size_t>(kPixPerChunk) * (32 * tq + 1) * sizeof(float);
        const dim3 grid(row_tiles, static_cast<unsigned>(splits));
        st = (ctype == CDMD_C_GAUSSIAN)
                 ? launch_slab<CDMD_C_GAUSSIAN>(tq, grid, smem, stream, D, m, n_slab, t0, ldd, k, key, pps, n, part)
                 : launch_slab<CDMD_C_RADEMACHER>(tq, grid, smem, stream, D, m, n_slab, t0, ldd, k, key, pps, n, part);
        if (st != CDMD_OK) return st;
    }
    const int64_t total = static_cast<int64_t>(k) * n;
    sketch_reduce_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, stream>>>(
        part, static_cast<int>(splits), k, n, DY, ctx->d_status);
    CDMD_CHECK_LAUNCH("sketch_reduce_kernel");
    return CDMD_OK;
}

}  // namespace cdmd

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP32 sketch (cdmd_sketch_noalloc).
//
// Some callers cannot allocate device memory at run time: code that runs
// under a memory budget fixed at start-up, real-time or safety-certified
// pipelines that forbid allocation after initialisation, and hosts where
// another runtime owns the device allocator.  For them the split partials of
// the sketch live in a fixed array of this file instead of a context's
// workspace.  The array is a static device variable: every GPU that loads
// this library holds its 16 MiB until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

// 4 Mi FP32 partial sums (16 MiB) for the allocation-free sketch.
static __device__ __align__(256) float g_sketch_noalloc_scratch[static_cast<size_t>(4) << 20];

namespace cdmd {
namespace {

constexpr size_t kNoAllocScratchFloats = static_cast<size_t>(4) << 20;   // elements of the array above

// Host-side set-up per device: the array's device address (host code cannot
// use the symbol itself: its host-side name is only a stand-in) and the SM
// count, taken once with that device current.
struct NoAllocDevice {
    bool ready = false;
    float* scratch = nullptr;
    int num_sms = 0;
};
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoAllocDevice g_noalloc_devices[kNoAllocMaxDevices];

}  // namespace
}  // namespace cdmd

extern "C" cdmd_status cdmd_sketch_noalloc(const uint8_t* D, int64_t m, int n, int64_t ldd, cdmd_ctype ctype,
                                           int k, uint64_t seed, double* DY, void* stream) {
    using namespace cdmd;
    clear_error();
    CDMD_REQUIRE(D != nullptr && DY != nullptr, "D or DY is NULL");
    CDMD_REQUIRE(m >= 1 && m <= 0x7fffffffLL, "m must be in [1, 2^31) (got %lld)", static_cast<long long>(m));
    CDMD_REQUIRE(n >= 2, "n must be >= 2 (got %d)", n);
    CDMD_REQUIRE(ldd >= m, "ldd (%lld) must be >= m (%lld)", static_cast<long long>(ldd), static_cast<long long>(m));
    CDMD_REQUIRE(k >= 1, "k must be >= 1 (got %d)", k);
    CDMD_REQUIRE(ctype == CDMD_C_GAUSSIAN || ctype == CDMD_C_RADEMACHER, "ctype must be GAUSSIAN or RADEMACHER");
    CDMD_REQUIRE(static_cast<size_t>(k) * static_cast<size_t>(n) <= kNoAllocScratchFloats,
                 "k * n = %lld exceeds the fixed scratch of cdmd_sketch_noalloc (%zu partial sums); "
                 "use cdmd_sketch", static_cast<long long>(k) * n, kNoAllocScratchFloats);
    int dev = -1;
    CDMD_CHECK_CUDA(cudaGetDevice(&dev));
    CDMD_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, "device index %d out of range", dev);
    NoAllocDevice setup;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoAllocDevice& s = g_noalloc_devices[dev];
        if (!s.ready) {
            void* p = nullptr;
            CDMD_CHECK_CUDA(cudaGetSymbolAddress(&p, g_sketch_noalloc_scratch));
            int sms = 0;
            CDMD_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            s.scratch = static_cast<float*>(p);
            s.num_sms = sms;
            s.ready = true;
        }
        setup = s;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    constexpr int kMaxSlab = 256;
    const int row_tiles = (k + kRowsPerCta - 1) / kRowsPerCta;
    const int64_t chunks = (m + kPixPerChunk - 1) / kPixPerChunk;
    const int64_t cap_splits = static_cast<int64_t>(kNoAllocScratchFloats / (static_cast<size_t>(k) * n));
    int64_t splits = (4LL * setup.num_sms + row_tiles - 1) / row_tiles;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, (chunks + 15) / 16));
    splits = std::min<int64_t>(std::min<int64_t>(splits, cap_splits), 65535);
    const int64_t chunks_per_split = (chunks + splits - 1) / splits;
    const int64_t pps = chunks_per_split * kPixPerChunk;
    splits = (m + pps - 1) / pps;   // never more than before: every split gets pixels
    const uint2 key = seed_key(seed);
    for (int t0 = 0; t0 < n; t0 += kMaxSlab) {
        const int n_slab = std::min(kMaxSlab, n - t0);
        const int tq = (n_slab + 31) / 32;
        const size_t smem = static_cast<size_t>(kPixPerChunk) * (32 * tq + 1) * sizeof(float);
        const dim3 grid(row_tiles, static_cast<unsigned>(splits));
        const cdmd_status s2 =
            (ctype == CDMD_C_GAUSSIAN)
                ? launch_slab<CDMD_C_GAUSSIAN>(tq, grid, smem, st, D, m, n_slab, t0, ldd, k, key, pps, n, setup.scratch)
                : launch_slab<CDMD_C_RADEMACHER>(tq, grid, smem, st, D, m, n_slab, t0, ldd, k, key, pps, n,
                                                 setup.scratch);
        if (s2 != CDMD_OK) return s2;
    }
    const int64_t total = static_cast<int64_t>(k) * n;
    sketch_reduce_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(
        setup.scratch, static_cast<int>(splits), k, n, DY, nullptr);
    CDMD_CHECK_LAUNCH("sketch_reduce_kernel (noalloc)");
    return CDMD_OK;
}
