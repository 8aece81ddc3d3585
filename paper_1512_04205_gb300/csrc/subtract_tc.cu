// Pass (c) on the 5th-generation tensor cores: the background of a tile of
// 128 pixels over all frames as a small GEMM, then threshold and bit-pack.
//
//   bg_jt = | sum_s a_js lambda_s^t |,  a_js = Phi_js beta_s     (Eq. DMDTerms)
//   mask_jt = |x_jt - bg_jt| > tau                              (Eq. thres)
//
// With a_js = u + i v and lambda_s^t = p + i q:
//   Re = sum_s (u p - v q) = [u, v] . [p, -q]
//   Im = sum_s (v p + u q) = [v, -u] . [p, -q]
// so one B operand, rows = frames t holding (p, -q) per mode, serves both
// parts: A rows (u, v) give Re and A' rows (v, -u) give Im.  K = 2 ncols
// (<= 32, zero padded: one 128-byte row of FP32 words).  The MMA is
// kind::tf32, which reads 11 significant bits of each FP32 word, so both
// operands are split: hi = the word with its low 13 mantissa bits cleared
// (exact in TF32), lo = the rest (exact in FP32, read to 11 bits).  Three
// products accumulate in FP32 in tensor memory (hi.hi + hi.lo + lo.hi), about
// 2^-19 relative per term, with FP32 range for modes that grow or decay.
//
// Tensor memory holds the frames in two halves, each with its Re (column
// 256h) and Im (256h + 128) accumulators, so the MMAs of one half overlap the
// epilogue of the other.  Per 128-pixel tile (persistent CTAs):
//   warp 0      TMA: D[frames][128 pixels] uint8 box -> staging (2 stages)
//   warp 1      one thread: 3 x ceil(2 ncols / 8) K8 MMAs per part (Re, and
//               Im unless REAL) and half, commits per half
//   warps 2-3   a = Phi beta for the tile's pixels -> A, A' hi / lo tiles
//   warps 4-7   epilogue of frame half 0, warps 8-11 of half 1: tcgen05.ld,
//               |x - bg| > tau, one ballot per frame = one mask word
// Waits are bounded as in the sketch.
#include <algorithm>

#include "tc_common.cuh"
#include "batch_internal.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 384;
constexpr int kPix = 128;                 // pixels per tile (MMA M)
constexpr int kMaxModes = 16;             // K = 2 ncols <= 32
constexpr int kTileBytes = kPix * 128;    // one 128-row SW128 tile (32 FP32 per row)
constexpr uint32_t kTmemCols = 512;

__host__ __device__ inline int pad16(int n) { return (n + 15) / 16 * 16; }

// Frames of half 0 (a multiple of 16, at most 128) and half 1.
__host__ __device__ inline int half0(int n) { return (pad16(n) / 16 + 1) / 2 * 16; }

struct SubLayout {
    uint32_t a_off, b_off, b_bytes, d_off, d_stage, amp_off, bar_off, misc_off, total;
};

__host__ __device__ inline SubLayout sub_layout(int n) {
    SubLayout L;
    L.a_off = 0;                                          // A hi, A lo, A' hi, A' lo
    L.b_off = 4 * kTileBytes;
    L.b_bytes = static_cast<uint32_t>(pad16(n)) * 128u;   // one of B hi, B lo
    L.d_off = L.b_off + 2 * L.b_bytes;
    L.d_stage = static_cast<uint32_t>(n) * kPix;
    L.amp_off = L.d_off + 2 * L.d_stage;
    L.bar_off = L.amp_off + kMaxModes * 8;
    L.misc_off = L.bar_off + 12 * 8;
    L.total = L.misc_off + 64;
    return L;
}

struct SubTcArgs {
    const float2* Phi;          // m x ncols complex, pixel-major
    const float2* lam_t;        // lambda^t, [n][nc_pad]
    const float2* amp;          // beta per column
    uint32_t* mask;
    int64_t m, words_per_frame, ntiles;
    int n, ncols, nc_pad;
    float tau;
};

// TF32 hi (low 13 mantissa bits cleared) and the FP32 rest of a float.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

// Store 4 FP32 values as hi and lo 16-byte chunks.
__device__ __forceinline__ void store_split4(uint8_t* hi_tile, uint8_t* lo_tile, uint32_t off, float a, float b,
                                             float c, float d) {
    float h[4], l[4];
    split_tf32(a, h[0], l[0]);
    split_tf32(b, h[1], l[1]);
    split_tf32(c, h[2], l[2]);
    split_tf32(d, h[3], l[3]);
    *reinterpret_cast<float4*>(hi_tile + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo_tile + off) = make_float4(l[0], l[1], l[2], l[3]);
}

// The tiles tile_first + li * tile_stride (li < my_tiles) of one clip.
template <bool kReal>
__device__ __forceinline__ void subtract_tc_body(const CUtensorMap* tmap, const SubTcArgs& a, int64_t tile_first,
                                                 int64_t tile_stride, int64_t my_tiles, int* status, uint8_t* smem) {
    const int n = a.n;
    const SubLayout L = sub_layout(n);
    uint8_t* Ahi = smem + L.a_off;
    uint8_t* Alo = Ahi + kTileBytes;
    uint8_t* Aphi = Ahi + 2 * kTileBytes;
    uint8_t* Aplo = Ahi + 3 * kTileBytes;
    uint8_t* Bhi = smem + L.b_off;
    uint8_t* Blo = Bhi + L.b_bytes;
    uint8_t* Dst = smem + L.d_off;
    float2* amp = reinterpret_cast<float2*>(smem + L.amp_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* tma_full = bars;          // [2]
    uint64_t* d_free = bars + 2;        // [2]
    uint64_t* a_full = bars + 4;
    uint64_t* a_free = bars + 5;
    uint64_t* acc_full = bars + 6;      // [2]
    uint64_t* acc_free = bars + 8;      // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 8);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int npad = pad16(n);
    const int nh0 = half0(n);
    const int ncols = a.ncols;
    const float tau = a.tau;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&d_free[s], 256);
            tc::mbar_init(&acc_full[s], 1);
            tc::mbar_init(&acc_free[s], 128);
        }
        tc::mbar_init(a_full, 64);
        tc::mbar_init(a_free, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // per-CTA constants: amplitudes, the B operand
    if (tid < kMaxModes) amp[tid] = tid < ncols ? a.amp[tid] : make_float2(0.f, 0.f);
    // B rows t: (Re lambda_s^t, -Im lambda_s^t) for s < ncols in K = 2s, 2s+1;
    // 4 K values (2 modes) per 16-byte chunk, chunks 0..7 of the 128-byte row
    for (int it = tid; it < npad * 8; it += kThreads) {
        const int t = it >> 3, c = it & 7;
        float2 l0 = make_float2(0.f, 0.f), l1 = make_float2(0.f, 0.f);
        if (t < n && 2 * c < ncols) l0 = a.lam_t[static_cast<int64_t>(t) * a.nc_pad + 2 * c];
        if (t < n && 2 * c + 1 < ncols) l1 = a.lam_t[static_cast<int64_t>(t) * a.nc_pad + 2 * c + 1];
        const uint32_t off = tc::sw128_offset(static_cast<uint32_t>(t), static_cast<uint32_t>(c));
        store_split4(Bhi, Blo, off, l0.x, -l0.y, l1.x, -l1.y);
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
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            for (int64_t li = 0; li < my_tiles; ++li) {
                const int s = static_cast<int>(li & 1);
                const uint32_t u = static_cast<uint32_t>(li >> 1);
                if (u >= 1 && !tc::mbar_wait(&d_free[s], (u - 1) & 1u, abort_flag, status)) break;
                tc::mbar_arrive_expect_tx(&tma_full[s], static_cast<uint32_t>(n) * kPix);
                const int64_t tile = tile_first + li * tile_stride;
                tc::tma_load_2d(Dst + s * L.d_stage, tmap, static_cast<int>(tile * kPix), 0, &tma_full[s]);
            }
            for (int s = 0; s < 2; ++s) {
                const int64_t uses = (my_tiles - s + 1) / 2;
                if (uses >= 1) tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const int nh[2] = {nh0, npad - nh0};
            const uint32_t idesc0 = tc::idesc_tf32_f32(128, nh[0]);
            const uint32_t idesc1 = tc::idesc_tf32_f32(128, nh[1] > 0 ? nh[1] : 16);
            const int nk = (2 * ncols + 7) / 8;      // K8 steps covering K = 2 ncols
            const uint32_t ahi = tc::smem_u32(Ahi), alo = tc::smem_u32(Alo);
            const uint32_t aphi = tc::smem_u32(Aphi), aplo = tc::smem_u32(Aplo);
            const uint32_t bhi = tc::smem_u32(Bhi), blo = tc::smem_u32(Blo);
            for (int64_t li = 0; li < my_tiles; ++li) {
                const uint32_t par = static_cast<uint32_t>(li & 1);
                if (!tc::mbar_wait(a_full, par, abort_flag, status)) break;
                bool ok = true;
                for (int h = 0; h < 2; ++h) {
                    if (li >= 1 && !tc::mbar_wait(&acc_free[h], par ^ 1u, abort_flag, status)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t boff = static_cast<uint32_t>(h * nh0) * 128u;
                    const uint32_t idesc = h ? idesc1 : idesc0;
#pragma unroll
                    for (int part = 0; part < (kReal ? 1 : 2); ++part) {
                        const uint32_t acc = tmem_base + 256u * h + 128u * part;
                        const uint32_t ah = part ? aphi : ahi;
                        const uint32_t al = part ? aplo : alo;
#pragma unroll 1
                        for (int kk = 0; kk < nk; ++kk) {
                            const uint64_t dbh = tc::desc_sw128(bhi + boff + kk * 32);
                            const uint64_t dbl = tc::desc_sw128(blo + boff + kk * 32);
                            const uint64_t dah = tc::desc_sw128(ah + kk * 32);
                            const uint64_t dal = tc::desc_sw128(al + kk * 32);
                            tc::mma_tf32(acc, dah, dbh, idesc, kk ? 1u : 0u);
                            tc::mma_tf32(acc, dah, dbl, idesc, 1u);
                            tc::mma_tf32(acc, dal, dbh, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&acc_full[h]);
                }
                if (!ok) break;
                tc::mma_commit(a_free);
            }
        }
    } else if (warp < 4) {
        // ---------------- A builders: a = Phi beta ----------------
        // Phi of the next tile is loaded into registers while the MMAs of the
        // current one run, so the global latency stays off the critical path
        const int ct = tid - 64;
        float2 f[2][kMaxModes];
        auto load_phi = [&](int64_t li) {
            const int64_t tile = tile_first + li * tile_stride;
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int64_t p = tile * kPix + ct + 64 * jj;
#pragma unroll
                for (int s = 0; s < kMaxModes; ++s)
                    f[jj][s] = (p < a.m && s < ncols) ? a.Phi[p * ncols + s] : make_float2(0.f, 0.f);
            }
        };
        if (my_tiles > 0) load_phi(0);
        for (int64_t li = 0; li < my_tiles; ++li) {
            if (li >= 1 && !tc::mbar_wait(a_free, static_cast<uint32_t>((li - 1) & 1), abort_flag, status)) break;
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int j = ct + 64 * jj;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float2 b0 = amp[2 * c], b1 = amp[2 * c + 1];
                    const float2 f0 = f[jj][2 * c], f1 = f[jj][2 * c + 1];
                    const float u0 = f0.x * b0.x - f0.y * b0.y, v0 = f0.x * b0.y + f0.y * b0.x;
                    const float u1 = f1.x * b1.x - f1.y * b1.y, v1 = f1.x * b1.y + f1.y * b1.x;
                    const uint32_t off = tc::sw128_offset(static_cast<uint32_t>(j), static_cast<uint32_t>(c));
                    store_split4(Ahi, Alo, off, u0, v0, u1, v1);                          // A row: (u, v)
                    if (!kReal) store_split4(Aphi, Aplo, off, v0, -u0, v1, -u1);        // A' row: (v, -u)
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(a_full);
            if (li + 1 < my_tiles) load_phi(li + 1);
        }
    } else {
        // ---------------- epilogue: warps 4-7 frame half 0, 8-11 half 1 ----------------
        const int h = (warp - 4) >> 2;
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int t0 = h * nh0;
        const int t1 = h ? n : (nh0 < n ? nh0 : n);
        for (int64_t li = 0; li < my_tiles; ++li) {
            const int s = static_cast<int>(li & 1);
            const uint32_t u = static_cast<uint32_t>(li >> 1);
            if (!tc::mbar_wait(&acc_full[h], static_cast<uint32_t>(li & 1), abort_flag, status)) break;
            if (!tc::mbar_wait(&tma_full[s], u & 1u, abort_flag, status)) break;
            tc::tc_fence_after();
            const int64_t tile = tile_first + li * tile_stride;
            const int64_t p = tile * kPix + row;
            const bool valid = p < a.m;
            const bool warp_full = __all_sync(0xffffffffu, valid);
            const int64_t widx = tile * (kPix / 32) + quarter;
            const uint8_t* xs = Dst + s * L.d_stage + row;
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + 256u * h;
            for (int c0 = t0; c0 < t1; c0 += 16) {
                const int nq = t1 - c0 < 16 ? t1 - c0 : 16;       // frames in this chunk (warp-uniform)
                uint32_t re[16], im[16];
                tc::tmem_ld_x16(taddr + static_cast<uint32_t>(c0 - t0), re);
                if (!kReal) tc::tmem_ld_x16(taddr + 128u + static_cast<uint32_t>(c0 - t0), im);
                // all 16 grey levels first (independent loads that overlap the
                // tensor-memory load), then the decisions and ballots
                uint32_t xv[16];
                uint32_t keep = 0u;
                if (nq == 16 && warp_full) {
                    // a full chunk of a warp whose pixels are all below m:
                    // no per-frame or per-pixel guards
#pragma unroll
                    for (int q = 0; q < 16; ++q) xv[q] = xs[(c0 + q) * kPix];
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        // grey level as a float: 2^23 + x, exact, minus 2^23
                        const float x = __uint_as_float(0x4B000000u | xv[q]) - 8388608.0f;
                        const float r = __uint_as_float(re[q]);
                        float bgv;
                        if (kReal) {
                            bgv = r;
                        } else {
                            const float i2 = __uint_as_float(im[q]);
                            asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(bgv) : "f"(fmaf(r, r, i2 * i2)));
                        }
                        const uint32_t w = __ballot_sync(0xffffffffu, fabsf(x - bgv) > tau);
                        keep = lane == q ? w : keep;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) xv[q] = q < nq ? xs[(c0 + q) * kPix] : 0u;
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float x = __uint_as_float(0x4B000000u | xv[q]) - 8388608.0f;
                        const float r = __uint_as_float(re[q]);
                        float bgv;
                        if (kReal) {
                            bgv = r;
                        } else {
                            const float i2 = __uint_as_float(im[q]);
                            asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(bgv) : "f"(fmaf(r, r, i2 * i2)));
                        }
                        const bool fg = fabsf(x - bgv) > tau;
                        const uint32_t w = __ballot_sync(0xffffffffu, fg && valid && q < nq);
                        keep = lane == q ? w : keep;
                    }
                }
                if (lane < nq && widx < a.words_per_frame)
                    a.mask[static_cast<int64_t>(c0 + lane) * a.words_per_frame + widx] = keep;
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acc_free[h]);
            tc::mbar_arrive(&d_free[s]);
        }
    }
    // teardown: every MMA has finished before TMEM is released
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0 && my_tiles > 0 && !*abort_flag) {
        // the last tile's commits are complete once its epilogues ran; wait for
        // a_free too so no MMA is in flight at the dealloc
        tc::mbar_wait(a_free, static_cast<uint32_t>((my_tiles - 1) & 1), abort_flag, status);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

template <bool kReal>
__global__ void __launch_bounds__(kThreads, 1)
subtract_tc_kernel(const __grid_constant__ CUtensorMap tmap, const SubTcArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    int64_t my_tiles = 0;
    if (static_cast<int64_t>(blockIdx.x) < a.ntiles)
        my_tiles = (a.ntiles - 1 - static_cast<int64_t>(blockIdx.x)) / gridDim.x + 1;
    subtract_tc_body<kReal>(&tmap, a, blockIdx.x, gridDim.x, my_tiles, status, smem);
}

// Grouped: CTA b runs item items[b], consecutive tiles of one clip; the
// clip's tensor map lives in global memory.
template <bool kReal>
__global__ void __launch_bounds__(kThreads, 1)
subtract_tc_grouped_kernel(const SubTcClip* __restrict__ clips, const SubtractItem* __restrict__ items, float tau,
                           int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const SubtractItem it = items[blockIdx.x];
    const SubTcClip c = clips[it.clip];
    SubTcArgs a;
    a.Phi = c.Phi;
    a.lam_t = c.lam_t;
    a.amp = c.amp;
    a.mask = c.mask;
    a.m = c.m;
    a.words_per_frame = (c.m + 31) / 32;
    a.ntiles = (c.m + kPix - 1) / kPix;
    a.n = c.n;
    a.ncols = c.ncols;
    a.nc_pad = c.nc_pad;
    a.tau = tau;
    subtract_tc_body<kReal>(c.tmap, a, it.tile0, 1, it.ntiles, status, smem);
}

}  // namespace

bool subtract_tc_supported(int n, int ncols, cdmd_bgmode mode, const uint8_t* D, int64_t ldd, int64_t m,
                           const float* bg) {
    return bg == nullptr && (mode == CDMD_BG_MODULUS || mode == CDMD_BG_REAL) && n >= 32 && n <= 1024 &&
           ncols >= 1 && ncols <= kMaxModes && (reinterpret_cast<uintptr_t>(D) % 16 == 0) && (ldd % 16 == 0) &&
           m <= 0x7fffffffLL - kPix;
}

size_t subtract_tc_smem(int n) { return sub_layout(n).total + 1024; }

int subtract_tc_tile_pixels() { return kPix; }

cdmd_status make_subtract_tc_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd) {
    return make_video_tmap(map, D, m, n, ldd, kPix, n);
}

cdmd_status launch_subtract_tc_grouped(const SubTcClip* clips, const SubtractItem* items, int nitems, int max_n,
                                       cdmd_bgmode mode, float tau, int* status, cudaStream_t stream) {
    const size_t smem = subtract_tc_smem(max_n);
    if (mode == CDMD_BG_REAL) {
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(subtract_tc_grouped_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        subtract_tc_grouped_kernel<true><<<static_cast<unsigned>(nitems), kThreads, smem, stream>>>(clips, items, tau,
                                                                                                   status);
    } else {
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(subtract_tc_grouped_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        subtract_tc_grouped_kernel<false><<<static_cast<unsigned>(nitems), kThreads, smem, stream>>>(clips, items, tau,
                                                                                                    status);
    }
    CDMD_CHECK_LAUNCH("subtract_tc_grouped_kernel");
    return CDMD_OK;
}

cdmd_status launch_subtract_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const float* Phi,
                               int ncols, const void* lam_t, const void* amp, int nc_pad, float tau, cdmd_bgmode mode,
                               uint32_t* mask, cudaStream_t stream) {
    // frames in chunks of at most 256 (the MMA N and the tensor copy box);
    // frames are independent here, so chunk q is the clip of frames
    // t0 .. t0+cnt-1 with its rows of the lambda^t table and of the mask
    const int nch = (n + 255) / 256;
    const int per = (n + nch - 1) / nch;
    const int64_t wpf = (m + 31) / 32;
    for (int q = 0; q < nch; ++q) {
        const int t0 = q * per;
        const int cnt = std::min(per, n - t0);
        CUtensorMap tmap;
        cdmd_status st = make_video_tmap(&tmap, D + static_cast<int64_t>(t0) * ldd, m, cnt, ldd, kPix, cnt);
        if (st != CDMD_OK) return st;
        SubTcArgs a{};
        a.Phi = reinterpret_cast<const float2*>(Phi);
        a.lam_t = static_cast<const float2*>(lam_t) + static_cast<int64_t>(t0) * nc_pad;
        a.amp = static_cast<const float2*>(amp);
        a.mask = mask + static_cast<int64_t>(t0) * wpf;
        a.m = m;
        a.words_per_frame = wpf;
        a.ntiles = (m + kPix - 1) / kPix;
        a.n = cnt;
        a.ncols = ncols;
        a.nc_pad = nc_pad;
        a.tau = tau;
        const size_t smem = sub_layout(cnt).total + 1024;
        const unsigned grid = static_cast<unsigned>(std::min<int64_t>(a.ntiles, ctx->num_sms));
        if (mode == CDMD_BG_REAL) {
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(subtract_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 232448));
            subtract_tc_kernel<true><<<grid, kThreads, smem, stream>>>(tmap, a, ctx->d_status);
        } else {
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(subtract_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 232448));
            subtract_tc_kernel<false><<<grid, kThreads, smem, stream>>>(tmap, a, ctx->d_status);
        }
        CDMD_CHECK_LAUNCH("subtract_tc_kernel");
    }
    return CDMD_OK;
}

}  // namespace cdmd
