// Pass (b), plain form: full-state modes Phi = X' G with G = V S^-1 W
// (Algorithm 1 step 8, Eq. cDMDModes), FP32 CUDA-core FMA.
//
// Each thread owns 4 consecutive pixels (one 32-bit load per frame) and a
// tile of 8 complex modes; G for the tile is converted FP64 -> FP32 into
// shared memory by the CTA.  Grid: (pixel blocks of 1024) x (mode tiles).
#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 256;
constexpr int kPx = 4;
constexpr int kCt = 8;

__global__ void __launch_bounds__(kThreads)
lift_fp32_kernel(const uint8_t* __restrict__ D, int64_t m, int n, int64_t ldd,
                 const double* __restrict__ G, int r, const int32_t* __restrict__ cols, int ncols,
                 float* __restrict__ Phi) {
    extern __shared__ float2 Gs[];   // [(n-1)][kCt]
    const int p = n - 1;
    const int c0 = blockIdx.y * kCt;
    for (int idx = threadIdx.x; idx < p * kCt; idx += kThreads) {
        const int t = idx / kCt;
        const int c = idx % kCt;
        float2 g = make_float2(0.f, 0.f);
        if (c0 + c < ncols) {
            const int s = cols ? cols[c0 + c] : c0 + c;
            if (s >= 0 && s < r) {
                const double* src = G + 2 * (static_cast<int64_t>(s) * p + t);
                g = make_float2(static_cast<float>(src[0]), static_cast<float>(src[1]));
            }
        }
        Gs[idx] = g;
    }
    __syncthreads();

    const int64_t j0 = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) * kPx;
    if (j0 >= m) return;
    const bool vec = (j0 + kPx <= m) && ((ldd & 3) == 0) && ((reinterpret_cast<uintptr_t>(D) & 3) == 0);
    float2 acc[kPx][kCt];
#pragma unroll
    for (int e = 0; e < kPx; ++e)
#pragma unroll
        for (int c = 0; c < kCt; ++c) acc[e][c] = make_float2(0.f, 0.f);

    for (int t = 0; t < p; ++t) {
        const uint8_t* src = D + static_cast<int64_t>(t + 1) * ldd + j0;
        uint32_t w = 0;
        if (vec) {
            w = __ldg(reinterpret_cast<const uint32_t*>(src));
        } else {
#pragma unroll
            for (int e = 0; e < kPx; ++e)
                if (j0 + e < m) w |= static_cast<uint32_t>(src[e]) << (8 * e);
        }
        float x[kPx];
#pragma unroll
        for (int e = 0; e < kPx; ++e) x[e] = static_cast<float>((w >> (8 * e)) & 255u);
        const float2* gt = Gs + t * kCt;
#pragma unroll
        for (int c = 0; c < kCt; ++c) {
            const float2 g = gt[c];
#pragma unroll
            for (int e = 0; e < kPx; ++e) {
                acc[e][c].x = fmaf(x[e], g.x, acc[e][c].x);
                acc[e][c].y = fmaf(x[e], g.y, acc[e][c].y);
            }
        }
    }
    const int cn = min(kCt, ncols - c0);
#pragma unroll
    for (int e = 0; e < kPx; ++e) {
        if (j0 + e >= m) break;
        float2* dst = reinterpret_cast<float2*>(Phi) + (j0 + e) * ncols + c0;
#pragma unroll
        for (int c = 0; c < kCt; ++c)
            if (c < cn) dst[c] = acc[e][c];
    }
}

}  // namespace

cdmd_status launch_lift_fp32(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                             const double* G, int r, const int32_t* cols, int ncols, float* Phi,
                             cudaStream_t stream) {
    (void)ctx;
    const int64_t pix_per_cta = static_cast<int64_t>(kThreads) * kPx;
    const dim3 grid(static_cast<unsigned>((m + pix_per_cta - 1) / pix_per_cta),
                    static_cast<unsigned>((ncols + kCt - 1) / kCt));
    const size_t smem = static_cast<size_t>(n - 1) * kCt * sizeof(float2);
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(lift_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    lift_fp32_kernel<<<grid, kThreads, smem, stream>>>(D, m, n, ldd, G, r, cols, ncols, Phi);
    CDMD_CHECK_LAUNCH("lift_fp32_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
