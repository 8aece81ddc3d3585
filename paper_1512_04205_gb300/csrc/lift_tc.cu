// Pass (b), mixed form: Phi = X' G on the 5th-generation tensor cores
// (Algorithm 1 step 8, Eq. cDMDModes).
//
// As a real GEMM: M = 128 pixels per tile, K = frames 1..n-1, N = 4 columns
// per mode: (hi re, lo re, hi im, lo im) of G = V S^-1 W, scaled by a power
// of two per mode and split into FP16 hi + lo parts.  uint8 pixels are exact
// in FP16.  The epilogue adds the hi and lo products and undoes the scale, so
// Phi carries G to ~2^-21 relative with FP32 accumulation.
//
// A is fed MN-major: the video is frame-major, so a frame's 128 pixels of a
// tile are already contiguous, and the converters only widen bytes (byte
// permute 0x64vv = 1024 + v, minus 1024 in f16x2) into 128-byte swizzled rows
// (64 pixels x 8 frames per 1024-byte atom).  No byte transpose.
//
// Persistent CTAs walk the pixel tiles.  Per tile:
//   warp 0      TMA: D[frames 1..n-1][128 pixels] uint8 box -> staging ring
//               (three stages where they fit, else two)
//   warps 2-7   widen the staging tile into one of two FP16 A tiles
//   warp 1      one thread issues tcgen05.mma over the K steps into one of
//               two TMEM accumulators
//   warps 8-15  two epilogue groups, one per accumulator (alternate tiles):
//               tcgen05.ld (one pixel per thread), add hi + lo, scale, store
//               Phi (complex64, pixel-major)
// G (the B operand) is converted once per CTA.  At most 16 modes and 255
// frames per launch; the launcher loops over groups of 16 modes and over
// frame chunks (later chunks add into Phi).  Waits are bounded as in the
// sketch.
#include "tc_common.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 512;
constexpr int kPix = 128;
constexpr int kConv = 192;               // converter threads (warps 2-7)
constexpr int kMaxModes = 16;
constexpr int kMaxSt = 3;                // staging stages at most
constexpr uint32_t kAccCols = 64;        // TMEM columns per accumulator
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kSmemLimit = 232448;

struct LiftLayout {
    int p, kpad, nkb, npad, nst;
    uint32_t a_stage, b_off, b_bytes, st_off, st_stage, bar_off, misc_off, total;
};

__host__ __device__ inline LiftLayout lift_layout(int n, int nmodes) {
    LiftLayout L;
    L.p = n - 1;
    L.kpad = (L.p + 15) / 16 * 16;
    L.nkb = (L.kpad + 63) / 64;
    L.npad = (4 * nmodes + 15) / 16 * 16;
    // A (MN-major): per 8 frames, two 1024-byte atoms (pixels 0-63, 64-127)
    L.a_stage = static_cast<uint32_t>(L.kpad) * 256u;
    L.b_off = 2 * L.a_stage;
    L.b_bytes = static_cast<uint32_t>(L.nkb) * L.npad * 128u;
    L.st_off = L.b_off + (L.b_bytes + 1023u) / 1024u * 1024u;
    L.st_stage = static_cast<uint32_t>(L.p) * kPix;
    for (L.nst = kMaxSt; L.nst > 2; --L.nst) {
        const uint32_t bar = (L.st_off + L.nst * L.st_stage + 127u) / 128u * 128u;
        if (bar + (2 * kMaxSt + 8) * 8 + 256 + 1024 <= kSmemLimit) break;
    }
    L.bar_off = (L.st_off + L.nst * L.st_stage + 127u) / 128u * 128u;
    L.misc_off = L.bar_off + (2 * kMaxSt + 8) * 8;
    // misc: TMEM slot, abort flag, 16 float inverse scales, 16 double scales
    L.total = L.misc_off + 256;
    return L;
}

__device__ __forceinline__ uint16_t f16_rn_bits(float x) {
    uint16_t h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

__device__ __forceinline__ float f16_to_f32(uint16_t h) {
    float x;
    asm("cvt.f32.f16 %0, %1;" : "=f"(x) : "h"(h));
    return x;
}

// Shared-memory descriptor of an MN-major operand with 128-byte swizzling:
// 8 rows of K, 128 bytes (64 FP16 elements of M) each, per 1024-byte atom;
// lbo = byte distance between atoms along M, sbo = between atoms along K.
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(lbo >> 4) << 16;
    d |= static_cast<uint64_t>(sbo >> 4) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(2u) << 61;
    return d;
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
    uint64_t* tma_full = bars;                      // [nst]
    uint64_t* st_free = bars + kMaxSt;              // [nst]
    uint64_t* a_full = bars + 2 * kMaxSt;           // [2]
    uint64_t* a_free = bars + 2 * kMaxSt + 2;       // [2]
    uint64_t* acc_full = bars + 2 * kMaxSt + 4;     // [2]
    uint64_t* acc_empty = bars + 2 * kMaxSt + 6;    // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 8);
    float* inv_scale = reinterpret_cast<float*>(smem + L.misc_off + 64);       // [16]
    double* scale = reinterpret_cast<double*>(smem + L.misc_off + 128);        // [16]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p = L.p;
    const int nst = L.nst;
    int64_t my_tiles = 0;
    if (blockIdx.x < ntiles) my_tiles = (ntiles - 1 - blockIdx.x) / gridDim.x + 1;

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&st_free[s], kConv);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&a_full[s], kConv);
            tc::mbar_init(&a_free[s], 1);
            tc::mbar_init(&acc_full[s], 1);
            tc::mbar_init(&acc_empty[s], 128);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // Scale of mode c: 2^s with max_t max(|Re G|, |Im G|) * 2^s in [2^14, 2^15),
    // so the FP16 hi and lo parts stay normal and far from overflow.
    for (int c = warp; c < kMaxModes; c += kThreads / 32) {
        double mx = 0.0;
        const int s = (c < nmodes) ? (cols ? cols[col0 + c] : col0 + c) : -1;
        if (s >= 0 && s < r) {
            for (int t = lane; t < p; t += 32) {
                const double* g = G + 2 * (static_cast<int64_t>(s) * ldg + t);
                mx = fmax(mx, fmax(fabs(g[0]), fabs(g[1])));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            int e = 0;
            if (mx > 0.0 && mx <= 1.0e300) frexp(mx, &e);
            const int sh = max(-100, min(100, 15 - e));
            scale[c] = ldexp(1.0, sh);
            inv_scale[c] = static_cast<float>(ldexp(1.0, -sh));
        }
    }
    // frames p .. kpad-1 of both A tiles are zeroed once (the converters never
    // write them): B is zero there, but uninitialised shared memory could hold
    // FP16 infinities or NaNs, which a zero factor does not cancel
    for (int idx = tid; idx < 2 * (L.kpad - p) * 16; idx += kThreads) {
        const int a = idx / ((L.kpad - p) * 16);
        const int rem = idx % ((L.kpad - p) * 16);
        const int f = p + (rem >> 4), q = rem & 15;
        *reinterpret_cast<uint4*>(A + a * L.a_stage + (f >> 3) * 2048 + (q >> 3) * 1024 + (f & 7) * 128 +
                                  (q & 7) * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    // B operand: row 4c + {0,1,2,3} = (hi re, lo re, hi im, lo im) of mode c
    // times its scale, K = frame t (0-based within X'), zero outside the modes
    // and frames.
    for (int idx = tid; idx < L.npad * L.kpad; idx += kThreads) {
        const int row = idx / L.kpad, t = idx % L.kpad;
        const int c = row >> 2, part = row & 3;
        uint16_t bits = 0;
        if (c < nmodes && t < p) {
            const int s = cols ? cols[col0 + c] : col0 + c;
            if (s >= 0 && s < r) {
                const double g = G[2 * (static_cast<int64_t>(s) * ldg + t) + (part >> 1)] * scale[c];
                const uint16_t hb = f16_rn_bits(static_cast<float>(g));
                bits = (part & 1) ? f16_rn_bits(static_cast<float>(g - static_cast<double>(f16_to_f32(hb)))) : hb;
            }
        }
        const int kb = t >> 6;
        const uint32_t off = static_cast<uint32_t>(kb) * L.npad * 128u +
                             tc::sw128_offset(static_cast<uint32_t>(row), static_cast<uint32_t>((t & 63) >> 3)) +
                             static_cast<uint32_t>(t & 7) * 2u;
        *reinterpret_cast<uint16_t*>(Bop + off) = bits;
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
            int s = 0;
            uint32_t u = 0;
            for (int64_t i = 0; i < my_tiles; ++i) {
                if (u >= 1 && !tc::mbar_wait(&st_free[s], (u - 1) & 1u, abort_flag, status)) break;
                const int64_t tile = blockIdx.x + i * gridDim.x;
                tc::mbar_arrive_expect_tx(&tma_full[s], static_cast<uint32_t>(p) * kPix);
                tc::tma_load_2d(St + s * L.st_stage, &tmap, static_cast<int>(tile * kPix), 1, &tma_full[s]);
                if (++s == nst) {
                    s = 0;
                    ++u;
                }
            }
            for (int q = 0; q < nst; ++q) {
                const int64_t uses = (my_tiles - q + nst - 1) / nst;
                if (uses >= 1) tc::mbar_wait(&tma_full[q], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // A MN-major (transpose bit 15), B K-major, both FP16, FP32 accumulate
            const uint32_t idesc = tc::idesc_f16_f32(128, L.npad) | (1u << 15);
            const int nk = L.kpad / 16;
            for (int64_t i = 0; i < my_tiles; ++i) {
                const int a = static_cast<int>(i & 1);
                const uint32_t v = static_cast<uint32_t>(i >> 1);
                if (!tc::mbar_wait(&a_full[a], v & 1u, abort_flag, status)) break;
                if (v >= 1 && !tc::mbar_wait(&acc_empty[a], (v - 1) & 1u, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + a * L.a_stage);
                const uint32_t b_base = tc::smem_u32(Bop);
                for (int kk = 0; kk < nk; ++kk) {
                    // 16 frames = two 2048-byte groups of A; B in K atoms of 64
                    const uint64_t adesc = desc_mn_sw128(a_base + static_cast<uint32_t>(kk) * 4096u, 1024u, 2048u);
                    const uint64_t bdesc = tc::desc_sw128(b_base + static_cast<uint32_t>(kk >> 2) * L.npad * 128u +
                                                          static_cast<uint32_t>(kk & 3) * 32u);
                    tc::mma_f16(tmem_base + a * kAccCols, adesc, bdesc, idesc, kk > 0 ? 1u : 0u);
                }
                tc::mma_commit(&a_free[a]);
                tc::mma_commit(&acc_full[a]);
            }
        }
    } else if (warp < 8) {
        // Item (frame f, 16-pixel chunk pc): one 16-byte load of the staging
        // row, two 16-byte stores of FP16 pixels.  Within each 8-lane phase
        // four lanes take frame f (chunks 0-3 or 4-7) and four take frame
        // f + 1 (the other half), so the loads cover 128 distinct bytes and
        // the stores, one atom row each, every swizzle position once.
        const int ct = tid - 64;
        const int nitems = ((p + 1) >> 1) * 16;
        int s = 0;
        uint32_t u = 0;
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int a = static_cast<int>(i & 1);
            const uint32_t v = static_cast<uint32_t>(i >> 1);
            if (!tc::mbar_wait(&tma_full[s], u & 1u, abort_flag, status)) break;
            if (v >= 1 && !tc::mbar_wait(&a_free[a], (v - 1) & 1u, abort_flag, status)) break;
            const uint8_t* src = St + s * L.st_stage;
            uint8_t* dst = A + a * L.a_stage;
            for (int it = ct; it < nitems; it += kConv) {
                const int w = it & 15;
                const int fo = (w >> 2) & 1;
                const int pc = (w & 3) | ((((w >> 2) ^ (w >> 3)) & 1) << 2);
                const int f = 2 * (it >> 4) + fo;
                if (f < p) {
                    const uint4 raw = *reinterpret_cast<const uint4*>(src + f * kPix + pc * 16);
                    uint32_t o[8];
                    o[0] = tc::sub_1024_f16x2(__byte_perm(raw.x, 0x64646464u, 0x4140u));
                    o[1] = tc::sub_1024_f16x2(__byte_perm(raw.x, 0x64646464u, 0x4342u));
                    o[2] = tc::sub_1024_f16x2(__byte_perm(raw.y, 0x64646464u, 0x4140u));
                    o[3] = tc::sub_1024_f16x2(__byte_perm(raw.y, 0x64646464u, 0x4342u));
                    o[4] = tc::sub_1024_f16x2(__byte_perm(raw.z, 0x64646464u, 0x4140u));
                    o[5] = tc::sub_1024_f16x2(__byte_perm(raw.z, 0x64646464u, 0x4342u));
                    o[6] = tc::sub_1024_f16x2(__byte_perm(raw.w, 0x64646464u, 0x4140u));
                    o[7] = tc::sub_1024_f16x2(__byte_perm(raw.w, 0x64646464u, 0x4342u));
                    const uint32_t rr = static_cast<uint32_t>(f & 7);
                    uint8_t* row = dst + (f >> 3) * 2048 + (pc >> 2) * 1024 + rr * 128u;
                    const uint32_t c0 = static_cast<uint32_t>(pc & 3) * 2u;
                    *reinterpret_cast<uint4*>(row + ((c0 ^ rr) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
                    *reinterpret_cast<uint4*>(row + (((c0 + 1u) ^ rr) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&st_free[s]);
            tc::mbar_arrive(&a_full[a]);
            if (++s == nst) {
                s = 0;
                ++u;
            }
        }
    } else {
        // group g (warps 8-11 or 12-15) takes the tiles i = g, g + 2, ...,
        // always accumulator g
        const int g = (warp - 8) >> 2;
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        for (int64_t i = g; i < my_tiles; i += 2) {
            const uint32_t v = static_cast<uint32_t>(i >> 1);
            if (!tc::mbar_wait(&acc_full[g], v & 1u, abort_flag, status)) break;
            tc::tc_fence_after();
            const int64_t tile = blockIdx.x + i * gridDim.x;
            const int64_t j = tile * kPix + row;
            for (int c0 = 0; c0 < L.npad; c0 += 16) {
                uint32_t rv[16];
                tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + g * kAccCols + c0, rv);
                tc::tmem_wait_ld();
                if (j < m) {
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int c = c0 / 4 + q4;
                        if (c < nmodes) {
                            const float sc = inv_scale[c];
                            float re = (__uint_as_float(rv[4 * q4]) + __uint_as_float(rv[4 * q4 + 1])) * sc;
                            float im = (__uint_as_float(rv[4 * q4 + 2]) + __uint_as_float(rv[4 * q4 + 3])) * sc;
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
            tc::mbar_arrive(&acc_empty[g]);
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
            if (smem > kSmemLimit) return fail(CDMD_ERR_INVALID_ARG, "lift tile does not fit in shared memory");
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(lift_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(kSmemLimit)));
            lift_tc_kernel<<<grid, kThreads, smem, stream>>>(tmap, m, nq, G + 2 * static_cast<int64_t>(t0),
                                                                         pt, r, cols, col0, nmodes, ncols, ntiles,
                                                                         q > 0 ? 1 : 0, Phi, ctx->d_status);
            CDMD_CHECK_LAUNCH("lift_tc_kernel");
        }
    }
    return CDMD_OK;
}

}  // namespace cdmd
