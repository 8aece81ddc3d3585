// Pass (b), mixed form: Phi = X' G on the 5th-generation tensor cores
// (Algorithm 1 step 8, Eq. cDMDModes).
//
// As a real GEMM: M = 128 pixels per tile, K = frames 1..n-1, N = 4 columns
// per mode: (hi re, lo re, hi im, lo im) of G = V S^-1 W split into BF16 hi +
// lo parts.  uint8 pixels are exact in BF16.  The epilogue adds the hi and lo
// products, so Phi carries G to ~2^-16 relative with FP32 accumulation.
//
// Persistent CTAs walk the pixel tiles.  Per tile:
//   warp 0      TMA: D[frames 1..n-1][128 pixels] uint8 box -> staging
//   warps 2-7   transpose 8 x 8 byte blocks of the staging tile into the
//               K-major 128-byte swizzled BF16 A tile (rows = pixels)
//   warp 1      one thread issues tcgen05.mma over the K blocks into one of
//               two TMEM accumulators
//   warps 8-11  tcgen05.ld the accumulator (one pixel per thread), add hi + lo
//               and store Phi (complex64, pixel-major)
// G (the B operand) is converted once per CTA.  At most 16 modes and 255
// frames per launch; the launcher loops over groups of 16 modes and over
// frame chunks (later chunks add into Phi).  Waits are bounded as in the
// sketch.
#include "tc_common.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 384;
constexpr int kStages = 2;
constexpr int kPix = 128;
constexpr int kConv = 192;               // converter threads (warps 2-7)
constexpr int kMaxModes = 16;
constexpr uint32_t kAccCols = 64;        // TMEM columns per accumulator
constexpr uint32_t kTmemCols = 128;

struct LiftLayout {
    int p, kpad, nkb, npad;
    uint32_t a_stage, b_off, b_bytes, st_off, st_stage, bar_off, misc_off, total;
};

__host__ __device__ inline LiftLayout lift_layout(int n, int nmodes) {
    LiftLayout L;
    L.p = n - 1;
    L.kpad = (L.p + 15) / 16 * 16;
    L.nkb = (L.kpad + 63) / 64;
    L.npad = (4 * nmodes + 15) / 16 * 16;
    L.a_stage = static_cast<uint32_t>(L.nkb) * kPix * 128u;
    L.b_off = kStages * L.a_stage;
    L.b_bytes = static_cast<uint32_t>(L.nkb) * L.npad * 128u;
    L.st_off = L.b_off + (L.b_bytes + 1023u) / 1024u * 1024u;
    L.st_stage = static_cast<uint32_t>(L.p) * kPix;
    L.bar_off = (L.st_off + kStages * L.st_stage + 127u) / 128u * 128u;
    L.misc_off = L.bar_off + (4 * kStages + 4) * 8;
    L.total = L.misc_off + 64;
    return L;
}

__device__ __forceinline__ uint16_t bf16_rn_bits(float x) {
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

__global__ void __launch_bounds__(kThreads, 1)
lift_tc_kernel(const __grid_constant__ CUtensorMap tmap, int64_t m, int n, const double* __restrict__ G, int ldg,
               int r, const int32_t* __restrict__ cols, int col0, int nmodes, int ncols_total, int64_t ntiles,
               int accumulate, float* __restrict__ Phi, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const LiftLayout L = lift_layout(n, nmodes);
    uint8_t* A = smem;
    uint8_t* Bop = smem + L.b_off;
    uint8_t* St = smem + L.st_off;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* tma_full = bars;
    uint64_t* st_free = bars + kStages;
    uint64_t* a_full = bars + 2 * kStages;
    uint64_t* a_free = bars + 3 * kStages;
    uint64_t* acc_full = bars + 4 * kStages;        // [2]
    uint64_t* acc_empty = bars + 4 * kStages + 2;   // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p = L.p;
    int64_t my_tiles = 0;
    if (blockIdx.x < ntiles) my_tiles = (ntiles - 1 - blockIdx.x) / gridDim.x + 1;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&st_free[s], kConv);
            tc::mbar_init(&a_full[s], kConv);
            tc::mbar_init(&a_free[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&acc_full[a], 1);
            tc::mbar_init(&acc_empty[a], 128);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // B operand: row 4c + {0,1,2,3} = (hi re, lo re, hi im, lo im) of mode c,
    // K = frame t (0-based within X'), zero outside the modes and frames.
    for (int idx = tid; idx < L.npad * L.kpad; idx += kThreads) {
        const int row = idx / L.kpad, t = idx % L.kpad;
        const int c = row >> 2, part = row & 3;
        float val = 0.0f;
        if (c < nmodes && t < p) {
            const int s = cols ? cols[col0 + c] : col0 + c;
            if (s >= 0 && s < r) {
                const float g = static_cast<float>(G[2 * (static_cast<int64_t>(s) * ldg + t) + (part >> 1)]);
                const uint16_t hb = bf16_rn_bits(g);
                const float hf = __uint_as_float(static_cast<uint32_t>(hb) << 16);
                val = (part & 1) ? (g - hf) : hf;
            }
        }
        const int kb = t >> 6;
        const uint32_t off = static_cast<uint32_t>(kb) * L.npad * 128u +
                             tc::sw128_offset(static_cast<uint32_t>(row), static_cast<uint32_t>((t & 63) >> 3)) +
                             static_cast<uint32_t>(t & 7) * 2u;
        *reinterpret_cast<uint16_t*>(Bop + off) = bf16_rn_bits(val);
    }
    tc::fence_proxy_async_smem();
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            for (int64_t i = 0; i < my_tiles; ++i) {
                const int s = static_cast<int>(i % kStages);
                const uint32_t u = static_cast<uint32_t>(i / kStages);
                if (u >= 1 && !tc::mbar_wait(&st_free[s], (u - 1) & 1u, abort_flag, status)) break;
                const int64_t tile = blockIdx.x + i * gridDim.x;
                tc::mbar_arrive_expect_tx(&tma_full[s], static_cast<uint32_t>(p) * kPix);
                tc::tma_load_2d(St + s * L.st_stage, &tmap, static_cast<int>(tile * kPix), 1, &tma_full[s]);
            }
            for (int s = 0; s < kStages; ++s) {
                const int64_t uses = (my_tiles - s + kStages - 1) / kStages;
                if (uses >= 1) tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(128, L.npad);
            for (int64_t i = 0; i < my_tiles; ++i) {
                const int s = static_cast<int>(i % kStages);
                const uint32_t u = static_cast<uint32_t>(i / kStages);
                const int a = static_cast<int>(i & 1);
                const uint32_t v = static_cast<uint32_t>(i >> 1);
                if (!tc::mbar_wait(&a_full[s], u & 1u, abort_flag, status)) break;
                if (v >= 1 && !tc::mbar_wait(&acc_empty[a], (v - 1) & 1u, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + s * L.a_stage);
                const uint32_t b_base = tc::smem_u32(Bop);
                for (int kb = 0; kb < L.nkb; ++kb) {
                    for (int kk = 0; kk < 4; ++kk) {
                        const int k0 = kb * 64 + kk * 16;
                        if (k0 >= L.kpad) break;
                        const uint64_t adesc = tc::desc_sw128(a_base + kb * kPix * 128 + kk * 32);
                        const uint64_t bdesc = tc::desc_sw128(b_base + kb * L.npad * 128 + kk * 32);
                        tc::mma_bf16(tmem_base + a * kAccCols, adesc, bdesc, idesc, k0 > 0 ? 1u : 0u);
                    }
                }
                tc::mma_commit(&a_free[s]);
                tc::mma_commit(&acc_full[a]);
            }
        }
    } else if (warp < 8) {
        const int ct = tid - 64;
        const int groups = L.kpad / 8;
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int s = static_cast<int>(i % kStages);
            const uint32_t u = static_cast<uint32_t>(i / kStages);
            if (!tc::mbar_wait(&tma_full[s], u & 1u, abort_flag, status)) break;
            if (u >= 1 && !tc::mbar_wait(&a_free[s], (u - 1) & 1u, abort_flag, status)) break;
            const uint8_t* src = St + s * L.st_stage;
            uint8_t* dst = A + s * L.a_stage;
            for (int it = ct; it < 16 * groups; it += kConv) {
                const int pg = it & 15, fg = it >> 4;
                uint2 raw[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int f = fg * 8 + e;
                    raw[e] = (f < p) ? *reinterpret_cast<const uint2*>(src + f * kPix + pg * 8) : make_uint2(0u, 0u);
                }
                uint8_t* blk = dst + (fg >> 3) * kPix * 128;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    // pixel qq of the 8 this item holds: rotated by lane, so the
                    // warp's 16-byte stores hit every swizzle phase (row & 7)
                    // and no bank twice per wavefront
                    const uint32_t qq = static_cast<uint32_t>(q + lane) & 7u;
                    const uint32_t sel0 = 0x7540u | (qq & 3u);   // byte qq&3 under exponent 2^23
                    uint32_t w[4];
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const uint32_t w0 = (qq < 4u) ? raw[2 * e2].x : raw[2 * e2].y;
                        const uint32_t w1 = (qq < 4u) ? raw[2 * e2 + 1].x : raw[2 * e2 + 1].y;
                        const float f0 = __uint_as_float(__byte_perm(w0, 0x4B000000u, sel0)) - 8388608.0f;
                        const float f1 = __uint_as_float(__byte_perm(w1, 0x4B000000u, sel0)) - 8388608.0f;
                        w[e2] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
                    }
                    *reinterpret_cast<uint4*>(blk + tc::sw128_offset(static_cast<uint32_t>(pg * 8) + qq,
                                                                     static_cast<uint32_t>(fg & 7))) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&st_free[s]);
            tc::mbar_arrive(&a_full[s]);
        }
    } else {
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int a = static_cast<int>(i & 1);
            const uint32_t v = static_cast<uint32_t>(i >> 1);
            if (!tc::mbar_wait(&acc_full[a], v & 1u, abort_flag, status)) break;
            tc::tc_fence_after();
            const int64_t tile = blockIdx.x + i * gridDim.x;
            const int64_t j = tile * kPix + row;
            for (int c0 = 0; c0 < L.npad; c0 += 16) {
                uint32_t rv[16];
                tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + a * kAccCols + c0, rv);
                tc::tmem_wait_ld();
                if (j < m) {
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int c = c0 / 4 + q4;
                        if (c < nmodes) {
                            float re = __uint_as_float(rv[4 * q4]) + __uint_as_float(rv[4 * q4 + 1]);
                            float im = __uint_as_float(rv[4 * q4 + 2]) + __uint_as_float(rv[4 * q4 + 3]);
                            float2* dst = reinterpret_cast<float2*>(Phi + 2 * (j * ncols_total + col0 + c));
                            if (accumulate) {
                                const float2 prev = *dst;
                                re += prev.x;
                                im += prev.y;
                            }
                            *dst = make_float2(re, im);
                        }
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acc_empty[a]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        // every MMA committed to the last accumulator barrier must be done
        if (my_tiles > 0 && *abort_flag) {
            const int64_t last = my_tiles - 1;
            tc::mbar_wait(&acc_full[last & 1], static_cast<uint32_t>(last >> 1) & 1u, abort_flag, status, 2000000000ull);
        }
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

cdmd_status launch_lift_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const double* G, int r,
                           const int32_t* cols, int ncols, float* Phi, cudaStream_t stream) {
    if ((reinterpret_cast<uintptr_t>(D) & 15) != 0 || (ldd & 15) != 0)
        return fail(CDMD_ERR_INVALID_ARG, "BF16X2 lift needs a 16-byte aligned video and ldd %% 16 == 0");
    // frames of X' in chunks of at most 255 (the operand tile and the tensor
    // copy box hold one chunk); the product is linear in the frames, so
    // chunks after the first add into Phi.  Chunk q covers X' frames
    // [t0, t0 + cnt) = video frames t0+1 .. t0+cnt, seen as a clip of cnt+1
    // frames starting at frame t0, with G rows t0.. (leading dimension n-1).
    const int pt = n - 1;
    const int nch = (pt + 254) / 255;
    const int per = (pt + nch - 1) / nch;
    const int64_t ntiles = (m + kPix - 1) / kPix;
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>(ntiles, ctx->num_sms));
    for (int q = 0; q < nch; ++q) {
        const int t0 = q * per;
        const int cnt = std::min(per, pt - t0);
        const int nq = cnt + 1;
        const uint8_t* Dq = D + static_cast<int64_t>(t0) * ldd;
        CUtensorMap tmap;
        cdmd_status st = make_video_tmap(&tmap, Dq, m, nq, ldd, kPix, nq - 1);
        if (st != CDMD_OK) return st;
        for (int col0 = 0; col0 < ncols; col0 += kMaxModes) {
            const int nmodes = std::min(kMaxModes, ncols - col0);
            const LiftLayout L = lift_layout(nq, nmodes);
            const size_t smem = L.total + 1024;
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(lift_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 232448));
            (void)smem;
            lift_tc_kernel<<<grid, kThreads, L.total + 1024, stream>>>(tmap, m, nq, G + 2 * static_cast<int64_t>(t0),
                                                                         pt, r, cols, col0, nmodes, ncols, ntiles,
                                                                         q > 0 ? 1 : 0, Phi, ctx->d_status);
            CDMD_CHECK_LAUNCH("lift_tc_kernel");
        }
    }
    return CDMD_OK;
}

}  // namespace cdmd
