// Exact DMD's one full-data contraction: the snapshot Gram R = D^T D of the
// uint8 video (R[s][t] = sum_j D[s][j] D[t][j], n x n), on the tensor cores.
//
// Exact DMD (Section 2.1) takes the SVD of X itself.  In the method of
// snapshots every quantity the small solves need (X^T X, X^T X', X'^T X',
// X'^T x1) is a block of this one Gram matrix, so the decomposition that
// follows is the compressed one's with R in place of DY^T DY, and the lift
// and subtract passes are shared.  This is the comparator of the paper's
// Computational Performance section.
//
// uint8 values are exact in FP16 and so are their products; the sums
// accumulate in FP32 in tensor memory, per CTA over a contiguous pixel range,
// and a second kernel adds the CTAs' partials in FP64.  FP16 rather than
// BF16 because both operands are frames and FP16 converts in two
// instructions per pixel pair: 1024 + b (b < 1024) is exact in FP16, so a
// byte permute builds the halves 0x6400 | b and one packed subtract of 1024
// leaves b.  Frames are both the
// A and the B operand, taken from the same shared-memory tile:
//   tile 0   A = frames 0..127   x  B = frames 0..n-1    (R rows 0..127)
//   tile 1   A = frames 128..255 x  B = frames 128..n-1  (n > 128 only)
// The block of rows 128.. against columns 0..127 is the transpose of part of
// tile 0 and is not computed; the reduce reads every entry from the upper
// triangle, so R comes out exactly symmetric.
//
// One CTA per SM, 384 threads:
//   warp 0       TMA: the uint8 bytes of 64 pixels x n frames per K step,
//                into an 8-slot staging ring (8 loads in flight)
//   warp 1       tcgen05.mma issue (M 128, K 16) and commits
//   warps 2-11   convert the staged bytes to an FP16 tile in the 128-byte
//                swizzled K-major layout (rows = frames), 16 pixels per item,
//                into a 3-slot ring of operand tiles
//   warps 4-7    epilogue: tcgen05.ld of the accumulators, FP32 partials of
//                the upper triangle
// Every mbarrier wait is bounded; on a timeout the CTA records
// CDMD_ERR_TIMEOUT, drains its copies and MMAs, frees TMEM and returns.
#include "tc_common.cuh"

namespace cdmd {
namespace {

constexpr int kGThreads = 384;
constexpr int kGConv = 320;                  // warps 2-11
constexpr int kGStg = 8;                     // uint8 staging slots (loads in flight)
constexpr int kGBuf = 3;                     // FP16 operand tiles
constexpr int kGKStep = 64;                  // pixels per K step
constexpr uint32_t kGBTile = 256u * 128u;    // 256 frame rows x 128 bytes of FP16
constexpr uint32_t kGStaging = 256u * 64u;   // 256 frames x 64 uint8 pixels
constexpr uint32_t kGTmemCols = 512;

__host__ __device__ inline int gpad16(int n) { return (n + 15) / 16 * 16; }

__host__ __device__ inline uint32_t gram_smem_bytes() {
    return kGBuf * kGBTile + kGStg * kGStaging + (2 * kGStg + 2 * kGBuf + 1) * 8 + 64;
}

struct GramArgs {
    float* part;        // [ctas][t][s] FP32 partial sums, s <= t
    int64_t m;          // pixels
    int64_t total_steps, steps_per_cta;
    int n;
};

__global__ void __launch_bounds__(kGThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ GramArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* B = smem;                                    // kGBuf FP16 tiles (1024-byte aligned)
    uint8_t* Dst = smem + kGBuf * kGBTile;                // kGStg uint8 stagings
    uint64_t* bars = reinterpret_cast<uint64_t*>(Dst + kGStg * kGStaging);
    uint64_t* tma_full = bars;                            // [kGStg] bytes landed
    uint64_t* d_free = bars + kGStg;                      // [kGStg] bytes converted
    uint64_t* b_full = bars + 2 * kGStg;                  // [kGBuf] tile written
    uint64_t* mma_done = bars + 2 * kGStg + kGBuf;        // [kGBuf] tile read by the MMAs
    uint64_t* accum_done = bars + 2 * kGStg + 2 * kGBuf;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int n = a.n;
    const int n16 = gpad16(n);
    const bool two_tiles = n > 128;
    const int64_t step0 = static_cast<int64_t>(blockIdx.x) * a.steps_per_cta;
    int64_t nsteps = a.total_steps - step0;
    if (nsteps > a.steps_per_cta) nsteps = a.steps_per_cta;
    if (nsteps < 0) nsteps = 0;

    if (tid == 0) {
        for (int s = 0; s < kGStg; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&d_free[s], kGConv);
        }
        for (int s = 0; s < kGBuf; ++s) {
            tc::mbar_init(&b_full[s], kGConv);
            tc::mbar_init(&mma_done[s], 1);
        }
        tc::mbar_init(accum_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // frame rows n..255 of every B tile are read by the MMAs (A rows of a
    // 128-row tile, B rows up to n16) but never written: zero them once
    for (int s = 0; s < kGBuf; ++s)
        for (uint32_t off = static_cast<uint32_t>(n) * 128u + tid * 16u; off < kGBTile; off += kGThreads * 16u)
            *reinterpret_cast<uint4*>(B + s * kGBTile + off) = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_proxy_async_smem();
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, kGTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint32_t bytes = static_cast<uint32_t>(n) * kGKStep;
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kGStg);
                const uint32_t u = static_cast<uint32_t>(ks / kGStg);
                // the staging slot is free once its bytes were converted
                if (u >= 1 && !tc::mbar_wait(&d_free[s], (u - 1) & 1u, abort_flag, status)) break;
                tc::mbar_arrive_expect_tx(&tma_full[s], bytes);
                tc::tma_load_2d(Dst + s * kGStaging, &tmap, static_cast<int>((step0 + ks) * kGKStep), 0, &tma_full[s]);
            }
            // drain: the last load of each stage must have landed before exit
            for (int s = 0; s < kGStg; ++s) {
                const int64_t uses = (nsteps - s + kGStg - 1) / kGStg;
                if (uses >= 1) tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc0 = tc::idesc_f16_f32(128, n16);
            const uint32_t idesc1 = tc::idesc_f16_f32(128, two_tiles ? n16 - 128 : 16);
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kGBuf);
                const uint32_t par = static_cast<uint32_t>(ks / kGBuf) & 1u;
                if (!tc::mbar_wait(&b_full[s], par, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t base = tc::smem_u32(B + s * kGBTile);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t d0 = tc::desc_sw128(base + kk * 32);                 // frames 0..
                    tc::mma_f16(tmem_base, d0, d0, idesc0, (ks | kk) ? 1u : 0u);
                }
                if (two_tiles) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t d1 = tc::desc_sw128(base + 128u * 128u + kk * 32);   // frames 128..
                        tc::mma_f16(tmem_base + 256u, d1, d1, idesc1, (ks | kk) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&mma_done[s]);
            }
            tc::mma_commit(accum_done);   // fires once every MMA issued above has finished
        }
    } else {
        // ---------------- converters (warps 2-11): uint8 -> FP16, 16 pixels of one frame per item ----------------
        const int ct = tid - 64;
        const int items = n * 4;
        for (int64_t ks = 0; ks < nsteps; ++ks) {
            const int sg = static_cast<int>(ks % kGStg);
            const uint32_t ug = static_cast<uint32_t>(ks / kGStg);
            const int sb = static_cast<int>(ks % kGBuf);
            const uint32_t ub = static_cast<uint32_t>(ks / kGBuf);
            // the B tile is free once the MMAs of its previous use finished
            if (ub >= 1 && !tc::mbar_wait(&mma_done[sb], (ub - 1) & 1u, abort_flag, status)) break;
            if (!tc::mbar_wait(&tma_full[sg], ug & 1u, abort_flag, status)) break;
            const uint8_t* src = Dst + sg * kGStaging;
            uint8_t* dst = B + sb * kGBTile;
            for (int it = ct; it < items; it += kGConv) {
                const int t = it >> 2, c16 = it & 3;
                const uint4 raw = *reinterpret_cast<const uint4*>(src + t * kGKStep + c16 * 16);
                uint32_t w[8];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const uint32_t word = h == 0 ? raw.x : h == 1 ? raw.y : h == 2 ? raw.z : raw.w;
                    // halves 0x6400 | b = 1024 + b for bytes (0, 1) and (2, 3), then minus 1024, exact
                    w[h * 2 + 0] = tc::sub_1024_f16x2(__byte_perm(word, 0x64646464u, 0x4140u));
                    w[h * 2 + 1] = tc::sub_1024_f16x2(__byte_perm(word, 0x64646464u, 0x4342u));
                }
                // two 16-byte chunks of the swizzled row; a quarter warp covers
                // an even and an odd row, so its eight stores hit distinct banks
                const uint32_t row = static_cast<uint32_t>(t);
                *reinterpret_cast<uint4*>(dst + tc::sw128_offset(row, 2u * c16)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(dst + tc::sw128_offset(row, 2u * c16 + 1u)) = make_uint4(w[4], w[5], w[6], w[7]);
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&d_free[sg]);
            tc::mbar_arrive(&b_full[sb]);
        }
        // ---------------- epilogue (warps 4-7): FP32 partials of the upper block ----------------
        if (warp >= 4) {
            const bool ok = tc::mbar_wait(accum_done, 0u, abort_flag, status) && !*abort_flag;
            tc::tc_fence_after();
            if (ok) {
                const int quarter = warp & 3;
                float* part = a.part + static_cast<int64_t>(blockIdx.x) * n * n;
                for (int tile = 0; tile < (two_tiles ? 2 : 1); ++tile) {
                    const int srow = tile * 128 + quarter * 32 + lane;   // frame of this thread's accumulator row
                    const int ncol = tile ? n16 - 128 : n16;
                    for (int c0 = 0; c0 < ncol; c0 += 16) {
                        uint32_t v[16];
                        tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + tile * 256u + c0, v);
                        tc::tmem_wait_ld();
                        // column-major partials: for each t the warp's 32 rows
                        // are 32 consecutive floats
                        if (srow < n) {
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const int t = tile * 128 + c0 + q;
                                if (t >= srow && t < n) part[static_cast<int64_t>(t) * n + srow] = __uint_as_float(v[q]);
                            }
                        }
                    }
                }
            }
        }
    }
    // teardown: every MMA has finished (accum_done) before TMEM is released
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (*abort_flag) tc::mbar_wait(accum_done, 0u, abort_flag, status, 2000000000ull);
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, kGTmemCols);
    }
}

// R[s][t] = R[t][s] = sum over CTAs of part[c][t][s] (s <= t), FP64, in a
// fixed order.  blockIdx.y = t; a block covers 32 consecutive s and its 8
// warps split the CTAs (warp g adds CTAs g, g+8, ...), then warp 0 adds the
// 8 sums in warp order.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(32 * kRedWarps)
gram_tc_reduce_kernel(const float* __restrict__ part, int ctas, int n, double* __restrict__ R, int* status) {
    __shared__ double red[kRedWarps][32];
    const int t = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int g = threadIdx.x >> 5;
    const int s = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 > t) return;   // the whole block is below the diagonal
    const bool live = s <= t;
    const int64_t nn = static_cast<int64_t>(n) * n;
    const int64_t src = static_cast<int64_t>(t) * n + s;
    double v = 0.0;
    if (live) {
#pragma unroll 4
        for (int c = g; c < ctas; c += kRedWarps) v += static_cast<double>(part[c * nn + src]);
    }
    red[g][lane] = v;
    __syncthreads();
    if (g == 0 && live) {
        double tot = 0.0;
#pragma unroll
        for (int i = 0; i < kRedWarps; ++i) tot += red[i][lane];
        if (!isfinite(tot)) record_status(status, CDMD_ERR_NONFINITE);
        R[src] = tot;                                   // R[t][s]
        R[static_cast<int64_t>(s) * n + t] = tot;       // R[s][t]
    }
}

}  // namespace

cdmd_status launch_gram_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, double* R,
                           cudaStream_t stream) {
    if (n < 2 || n > 256)
        return fail(CDMD_ERR_UNSUPPORTED, "the snapshot Gram covers 2 <= n <= 256 frames (got %d)", n);
    if ((reinterpret_cast<uintptr_t>(D) & 15u) != 0 || (ldd & 15) != 0)
        return fail(CDMD_ERR_UNSUPPORTED, "the snapshot Gram needs a 16-byte aligned video with ldd %% 16 == 0");
    CUtensorMap tmap;
    cdmd_status st = make_video_tmap(&tmap, D, m, n, ldd, kGKStep, n);
    if (st != CDMD_OK) return st;
    const int64_t steps = (m + kGKStep - 1) / kGKStep;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 1;
    int64_t ctas = steps < sms ? steps : sms;
    const int64_t per = (steps + ctas - 1) / ctas;
    ctas = (steps + per - 1) / per;
    float* part = nullptr;
    st = ensure_buffer(ctx, BUF_GRAM, static_cast<size_t>(ctas) * n * n * sizeof(float), reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    GramArgs a;
    a.part = part;
    a.m = m;
    a.total_steps = steps;
    a.steps_per_cta = per;
    a.n = n;
    const size_t smem = gram_smem_bytes() + 1024;
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    gram_tc_kernel<<<static_cast<unsigned>(ctas), kGThreads, smem, stream>>>(tmap, a, ctx->d_status);
    CDMD_CHECK_LAUNCH("gram_tc_kernel");
    gram_tc_reduce_kernel<<<dim3((n + 31) / 32, n), 32 * kRedWarps, 0, stream>>>(part, static_cast<int>(ctas), n, R,
                                                                                 ctx->d_status);
    CDMD_CHECK_LAUNCH("gram_tc_reduce_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
