// Pass (c): background reconstruction from the selected modes, foreground
// threshold and bit-packed mask, fused in one pass over the video.
//
//   bg_jt = | sum_c Phi_jc beta_{s_c} lambda_{s_c}^t |   (Eq. DMDTerms, MODULUS)
//   mask_jt = |x_jt - bg_jt| > tau                       (Eq. thres, strict)
//
// subtract_table_kernel (one CTA) forms lambda^t for t < n by repeated FP64
// multiplication and the amplitudes; the main kernel keeps, per pixel, the
// ncols products a_jc = Phi_jc beta_c in registers and walks the frames:
// lane l of a warp owns pixels base + l + 32e (e < PX), so the ballot of
// sub-position e is exactly mask word base/32 + e of frame t.
#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 256;

// table[t * nc_pad + c] = lambda_{s_c}^t ; amp[c] = beta_{s_c} (0 for unused c)
__global__ void subtract_table_kernel(const int32_t* __restrict__ cols, int ncols, int nc_pad,
                                      const double* __restrict__ beta,
                                      const double* __restrict__ lambda, int r, int n,
                                      float2* __restrict__ table, float2* __restrict__ amp) {
    const int c = threadIdx.x;
    if (c >= nc_pad) return;
    int s = -1;
    if (c < ncols) s = cols ? cols[c] : c;
    const bool ok = (s >= 0 && s < r);
    const double lr = ok ? lambda[2 * s] : 0.0;
    const double li = ok ? lambda[2 * s + 1] : 0.0;
    amp[c] = ok ? make_float2(static_cast<float>(beta[2 * s]), static_cast<float>(beta[2 * s + 1]))
                : make_float2(0.f, 0.f);
    double pr = 1.0, pi = 0.0;
    for (int t = 0; t < n; ++t) {
        table[static_cast<int64_t>(t) * nc_pad + c] =
            ok ? make_float2(static_cast<float>(pr), static_cast<float>(pi)) : make_float2(0.f, 0.f);
        const double nr = pr * lr - pi * li;
        const double ni = pr * li + pi * lr;
        pr = nr;
        pi = ni;
    }
}

template <int NC, int PX, int MODE>
__global__ void __launch_bounds__(kThreads)
subtract_kernel(const uint8_t* __restrict__ D, int64_t m, int n, int64_t ldd,
                const float2* __restrict__ Phi, int ncols, const float2* __restrict__ table,
                const float2* __restrict__ amp, float tau, uint32_t* __restrict__ mask,
                int64_t words_per_frame, float* __restrict__ bg_out) {
    extern __shared__ float2 Ls[];   // [n][NC]
    for (int idx = threadIdx.x; idx < n * NC; idx += kThreads) Ls[idx] = table[idx];
    __syncthreads();

    constexpr int FB = 8;   // frames whose bytes are loaded ahead of the arithmetic
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = static_cast<int64_t>(gridDim.x) * (kThreads / 32);
    const int64_t tiles = (m + 32 * PX - 1) / (32 * PX);
    for (int64_t tile = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5; tile < tiles;
         tile += warps_total) {
        const int64_t base = tile * 32 * PX;
        float2 a[PX][NC];
#pragma unroll
        for (int e = 0; e < PX; ++e) {
            const int64_t j = base + lane + 32 * e;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float2 v = make_float2(0.f, 0.f);
                if (j < m && c < ncols) {
                    const float2 ph = Phi[j * ncols + c];
                    const float2 b = amp[c];
                    v = make_float2(ph.x * b.x - ph.y * b.y, ph.x * b.y + ph.y * b.x);
                }
                a[e][c] = v;
            }
        }
        float bg_static[PX];
        if (MODE == CDMD_BG_STATIC) {
#pragma unroll
            for (int e = 0; e < PX; ++e) {
                float zr = 0.f, zi = 0.f;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    zr += a[e][c].x;
                    zi += a[e][c].y;
                }
                bg_static[e] = sqrtf(zr * zr + zi * zi);
            }
        }
        const int64_t word0 = tile * PX;
        for (int t0 = 0; t0 < n; t0 += FB) {
            float xv[FB][PX];
#pragma unroll
            for (int f = 0; f < FB; ++f)
#pragma unroll
                for (int e = 0; e < PX; ++e) {
                    const int64_t j = base + lane + 32 * e;
                    xv[f][e] = (t0 + f < n && j < m)
                                   ? static_cast<float>(__ldg(D + static_cast<int64_t>(t0 + f) * ldd + j)) : 0.0f;
                }
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                const int t = t0 + f;
                if (t >= n) break;
                const float2* lt = Ls + t * NC;
                uint32_t words[PX];
#pragma unroll
                for (int e = 0; e < PX; ++e) {
                    const int64_t j = base + lane + 32 * e;
                    const float x = xv[f][e];
                    bool bit;
                    float bg = 0.0f;
                    if (MODE == CDMD_BG_STATIC) {
                        bg = bg_static[e];
                        bit = fabsf(x - bg) > tau;
                    } else {
                        float zr = 0.f, zi = 0.f;
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const float2 l = lt[c];
                            zr = fmaf(a[e][c].x, l.x, zr);
                            zr = fmaf(-a[e][c].y, l.y, zr);
                            zi = fmaf(a[e][c].x, l.y, zi);
                            zi = fmaf(a[e][c].y, l.x, zi);
                        }
                        if (MODE == CDMD_BG_REAL) {
                            bg = zr;
                            bit = fabsf(x - bg) > tau;
                        } else if (bg_out != nullptr) {
                            bg = sqrtf(zr * zr + zi * zi);
                            bit = fabsf(x - bg) > tau;
                        } else {
                            // |x - |z|| > tau  <=>  |z|^2 > (x + tau)^2  or  (x - tau > 0 and |z|^2 < (x - tau)^2)
                            const float q = fmaf(zr, zr, zi * zi);
                            const float up = x + tau, dn = x - tau;
                            bit = (q > up * up) || (dn > 0.0f && q < dn * dn);
                        }
                    }
                    bit = bit && (j < m);
                    if (bg_out != nullptr && j < m) bg_out[static_cast<int64_t>(t) * m + j] = bg;
                    words[e] = __ballot_sync(0xffffffffu, bit);
                }
                if (lane < PX) {
                    uint32_t w = words[0];
#pragma unroll
                    for (int e = 1; e < PX; ++e)
                        if (lane == e) w = words[e];
                    const int64_t wi = word0 + lane;
                    if (wi < words_per_frame) mask[static_cast<int64_t>(t) * words_per_frame + wi] = w;
                }
            }
        }
    }
}

template <int NC, int PX>
cdmd_status launch_nc(cdmd_bgmode mode, const uint8_t* D, int64_t m, int n, int64_t ldd,
                      const float2* Phi, int ncols, const float2* table, const float2* amp,
                      float tau, uint32_t* mask, float* bg, int sms, cudaStream_t stream) {
    const int64_t warps = (m + 32 * PX - 1) / (32 * PX);
    // persistent: a few CTAs per SM walk the pixel tiles (the lambda^t table
    // is staged once per CTA)
    const int64_t blocks = std::min<int64_t>((warps * 32 + kThreads - 1) / kThreads, static_cast<int64_t>(sms) * 3);
    const size_t smem = static_cast<size_t>(n) * NC * sizeof(float2);
    const int64_t wpf = (m + 31) / 32;
#define CDMD_SUB_MODE(MV)                                                                         \
    {                                                                                             \
        auto kern = subtract_kernel<NC, PX, MV>;                                                  \
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                             static_cast<int>(smem)));                            \
        kern<<<static_cast<unsigned>(blocks), kThreads, smem, stream>>>(D, m, n, ldd, Phi, ncols, \
                                                                        table, amp, tau, mask,    \
                                                                        wpf, bg);                 \
    }
    if (mode == CDMD_BG_MODULUS) CDMD_SUB_MODE(CDMD_BG_MODULUS)
    else if (mode == CDMD_BG_REAL) CDMD_SUB_MODE(CDMD_BG_REAL)
    else CDMD_SUB_MODE(CDMD_BG_STATIC)
#undef CDMD_SUB_MODE
    CDMD_CHECK_LAUNCH("subtract_kernel");
    return CDMD_OK;
}

}  // namespace

cdmd_status launch_subtract(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                            const float* Phi, int ncols, const int32_t* cols, const double* beta,
                            const double* lambda, int r, float tau, cdmd_bgmode mode,
                            uint32_t* mask, float* bg, cudaStream_t stream) {
    int nc_pad;
    if (ncols <= 4) nc_pad = 4;
    else if (ncols <= 8) nc_pad = 8;
    else if (ncols <= 10) nc_pad = 10;
    else if (ncols <= 12) nc_pad = 12;
    else if (ncols <= 16) nc_pad = 16;
    else if (ncols <= 20) nc_pad = 20;
    else if (ncols <= 24) nc_pad = 24;
    else nc_pad = 32;
    void* tbl = nullptr;
    const size_t table_bytes = static_cast<size_t>(n) * nc_pad * sizeof(float2);
    cdmd_status st = ensure_buffer(ctx, BUF_SUBTRACT_TABLE, table_bytes + 32 * sizeof(float2), &tbl);
    if (st != CDMD_OK) return st;
    float2* table = static_cast<float2*>(tbl);
    float2* amp = table + static_cast<size_t>(n) * nc_pad;
    subtract_table_kernel<<<1, 32, 0, stream>>>(cols, ncols, nc_pad, beta, lambda, r, n, table, amp);
    CDMD_CHECK_LAUNCH("subtract_table_kernel");
    const float2* ph = reinterpret_cast<const float2*>(Phi);
    switch (nc_pad) {
        case 4: return launch_nc<4, 4>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        case 8: return launch_nc<8, 4>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        case 10: return launch_nc<10, 2>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        case 12: return launch_nc<12, 2>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        case 16: return launch_nc<16, 2>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        case 20: return launch_nc<20, 1>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        case 24: return launch_nc<24, 1>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
        default: return launch_nc<32, 1>(mode, D, m, n, ldd, ph, ncols, table, amp, tau, mask, bg, ctx->num_sms, stream);
    }
}

}  // namespace cdmd
