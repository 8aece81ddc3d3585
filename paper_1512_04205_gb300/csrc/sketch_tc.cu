// Pass (a), mixed form: DY = C D on the 5th-generation tensor cores
// (Algorithm 1 steps 2-3, Eq. YCX).
//
// uint8 pixels are exact in BF16; the Gaussian C is split into BF16 hi + lo
// parts (C = hi + lo to ~2^-17 relative) and both products accumulate in FP32
// in tensor memory: D_acc += C_hi D + C_lo D.  C is drawn in-kernel from
// Philox4x32-10 (Box-Muller with the fast MUFU log2 / sin / cos) and never
// touches HBM.
//
// One persistent CTA per SM owns a pair of 128-row M tiles of C (256 rows)
// and a contiguous pixel range; the whole frame dimension (n <= 256) is the
// MMA N.  Per 64-pixel K step and pipeline stage:
//   warp 0      TMA: D[frames][64 pixels] uint8 box -> staging buffer
//   warps 2-3   convert the staged bytes to BF16 in the 128-byte swizzled
//               K-major layout (B operand, rows = frames)
//   warps 4-11  draw the 256 x 64 block of C and write hi / lo BF16 tiles in
//               the same layout (A operands, rows = rows of C)
//   warp 1      one thread issues 2 tiles x 4 K16 steps x (hi, lo) = 16
//               tcgen05.mma (M 128, N = frames padded to 16, K 16) into two
//               TMEM accumulators and commits to the stage's barrier
// After the last K step warps 4-7 read the accumulators (tcgen05.ld) and write
// FP32 partials [split][frame][row]; a second kernel sums the splits in FP64.
// Every mbarrier wait is bounded in time; on a timeout the CTA records
// CDMD_ERR_TIMEOUT, drains its copies and MMAs, frees TMEM and returns.
#include <cudaTypedefs.h>

#include "tc_common.cuh"
#include "batch_internal.cuh"

namespace cdmd {

cdmd_status make_video_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd, int box_x,
                            int box_y) {
    // resolved once (thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (encode == nullptr) return fail(CDMD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(n)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldd)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_x), static_cast<cuuint32_t>(box_y)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(D), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CDMD_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", static_cast<int>(r));
    return CDMD_OK;
}

namespace {

constexpr int kThreads = 384;
constexpr int kStages = 2;
constexpr int kKStep = 64;                  // pixels per K step (one 128-byte BF16 row)
constexpr int kTileBytes = 128 * 128;       // 128 rows x 128 bytes
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxFrames = 256;             // frames per launch: MMA N and TMA box height limits

// Fast Box-Muller pair (MUFU lg2 / sqrt / sin / cos), same definition as the
// accurate form: U(w) = (w + 1/2) 2^-32, angle split into quarter turns: the
// top two bits of wb pick the quadrant and the hardware sine / cosine see only
// the remainder (pi/2) f, f in (0, 1) from the next 23 bits (a float in
// [1, 2) built from the bits, minus 1, plus half a step; no I2F).  The
// quadrant map sends the approximation error of cos and sin to +c, -s, -c,
// +s in turn, so its mean cancels; handed the whole angle, the hardware
// functions leave a bias of ~5e-7 per draw that a sketch over 2 M pixels of
// mean ~128 grey levels turns into ~1e-4 relative.
__device__ __forceinline__ void box_muller_fast(uint32_t wa, uint32_t wb, float& zc, float& zs) {
    const float u = fmaf(__uint2float_rn(wa), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float x = -1.3862943611198906f * __log2f(u);   // -2 ln u
    float rad;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rad) : "f"(x));
    const float f = __uint_as_float(0x3F800000u | ((wb >> 7) & 0x7FFFFFu)) - (1.0f - 5.9604645e-08f);
    float s, c;
    __sincosf(1.5707963267948966f * f, &s, &c);
    const uint32_t qt = wb >> 30;
    float cs = (qt & 1u) ? -s : c;
    float sn = (qt & 1u) ? c : s;
    if (qt & 2u) { cs = -cs; sn = -sn; }
    zc = rad * cs;
    zs = rad * sn;
}

struct SmemLayout {
    uint32_t a_off, b_off, dst_off, bar_off, misc_off, total;
    uint32_t b_stage_bytes, dst_stage_bytes;
};

__host__ __device__ inline SmemLayout smem_layout(int n) {
    SmemLayout L;
    const int npad = (n + 15) / 16 * 16;
    L.a_off = 0;
    L.b_stage_bytes = static_cast<uint32_t>(npad) * 128u;
    L.b_off = L.a_off + kStages * 4 * kTileBytes;
    // tensor copies need a 128-byte aligned shared-memory destination: pad
    // the staging stride (n * 64 bytes is only 64-byte aligned for odd n)
    L.dst_stage_bytes = (static_cast<uint32_t>(n) * kKStep + 127u) / 128u * 128u;
    L.dst_off = L.b_off + kStages * ((L.b_stage_bytes + 1023u) / 1024u * 1024u);
    L.bar_off = (L.dst_off + kStages * L.dst_stage_bytes + 127u) / 128u * 128u;
    L.misc_off = L.bar_off + (5 * kStages + 1) * 8;
    L.total = L.misc_off + 64;
    return L;
}

// One CTA's share of C D: rows pair*256 .. pair*256+255 of C over the
// 64-pixel K steps step0 .. step0+nsteps-1, written to part[t * k + row]
// (this split's partial sums).  Used by the per-clip and the grouped launch.
__device__ __forceinline__ void sketch_tc_body(const CUtensorMap* tmap, int64_t m, int n, int k, uint2 key, int pair,
                                               int64_t step0, int64_t nsteps, float* __restrict__ part, int* status,
                                               uint8_t* smem) {
    const SmemLayout L = smem_layout(n);
    const int npad = (n + 15) / 16 * 16;
    uint8_t* A = smem + L.a_off;
    uint8_t* B = smem + L.b_off;
    uint8_t* Dst = smem + L.dst_off;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* tma_full = bars;
    uint64_t* d_free = bars + kStages;
    uint64_t* b_full = bars + 2 * kStages;
    uint64_t* a_full = bars + 3 * kStages;
    uint64_t* mma_done = bars + 4 * kStages;
    uint64_t* accum_done = bars + 5 * kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 8);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    if (nsteps < 0) nsteps = 0;
    const uint32_t b_stride = (L.b_stage_bytes + 1023u) / 1024u * 1024u;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&d_free[s], 64);
            tc::mbar_init(&b_full[s], 64);
            tc::mbar_init(&a_full[s], 256);
            tc::mbar_init(&mma_done[s], 1);
        }
        tc::mbar_init(accum_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // zero the padding rows (frames n..npad-1) of both B stages once
    for (int s = 0; s < kStages; ++s)
        for (uint32_t off = static_cast<uint32_t>(n) * 128u + tid * 16u; off < L.b_stage_bytes; off += kThreads * 16u)
            *reinterpret_cast<uint4*>(B + s * b_stride + off) = make_uint4(0u, 0u, 0u, 0u);
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
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kStages);
                const uint32_t u = static_cast<uint32_t>(ks / kStages);
                if (u >= 1 && !tc::mbar_wait(&d_free[s], (u - 1) & 1u, abort_flag, status)) break;
                tc::mbar_arrive_expect_tx(&tma_full[s], static_cast<uint32_t>(n) * kKStep);
                tc::tma_load_2d(Dst + s * L.dst_stage_bytes, tmap, static_cast<int>((step0 + ks) * kKStep), 0,
                                &tma_full[s]);
            }
            // drain: the last load of each stage must have landed before exit
            for (int s = 0; s < kStages; ++s) {
                const int64_t uses = (nsteps - s + kStages - 1) / kStages;
                if (uses >= 1) tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(128, npad);
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kStages);
                const uint32_t par = static_cast<uint32_t>(ks / kStages) & 1u;
                if (!tc::mbar_wait(&a_full[s], par, abort_flag, status)) break;
                if (!tc::mbar_wait(&b_full[s], par, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + s * 4 * kTileBytes);
                const uint32_t b_base = tc::smem_u32(B + s * b_stride);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bdesc = tc::desc_sw128(b_base + kk * 32);
#pragma unroll
                        for (int hl = 0; hl < 2; ++hl) {
                            const uint64_t adesc = tc::desc_sw128(a_base + (mt * 2 + hl) * kTileBytes + kk * 32);
                            tc::mma_bf16(tmem_base + mt * 256, adesc, bdesc, idesc, (ks | kk | hl) ? 1u : 0u);
                        }
                    }
                }
                tc::mma_commit(&mma_done[s]);
            }
            tc::mma_commit(accum_done);   // fires once every MMA issued above has finished
        }
    } else if (warp < 4) {
        // ---------------- uint8 -> BF16 converters ----------------
        const int ct = tid - 64;
        for (int64_t ks = 0; ks < nsteps; ++ks) {
            const int s = static_cast<int>(ks % kStages);
            const uint32_t u = static_cast<uint32_t>(ks / kStages);
            if (!tc::mbar_wait(&tma_full[s], u & 1u, abort_flag, status)) break;
            if (u >= 1 && !tc::mbar_wait(&mma_done[s], (u - 1) & 1u, abort_flag, status)) break;
            const uint8_t* src = Dst + s * L.dst_stage_bytes;
            uint8_t* dst = B + s * b_stride;
            for (int it = ct; it < n * 8; it += 64) {
                const int t = it >> 3, g = it & 7;
                const uint2 raw = *reinterpret_cast<const uint2*>(src + t * kKStep + g * 8);
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t word = h ? raw.y : raw.x;
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float f0 = __uint_as_float(0x4B000000u | ((word >> (16 * e)) & 0xFFu)) - 8388608.0f;
                        const float f1 = __uint_as_float(0x4B000000u | ((word >> (16 * e + 8)) & 0xFFu)) - 8388608.0f;
                        w[h * 2 + e] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
                    }
                }
                *reinterpret_cast<uint4*>(dst + tc::sw128_offset(static_cast<uint32_t>(t), static_cast<uint32_t>(g))) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&d_free[s]);
            tc::mbar_arrive(&b_full[s]);
        }
    } else {
        // ---------------- C generators (256 threads) ----------------
        const int gt = tid - 128;
        const int row_pair0 = pair * 256;
        const PhiloxKeys rk = philox_round_keys(key);   // the same for every draw of this CTA
        for (int64_t ks = 0; ks < nsteps; ++ks) {
            const int s = static_cast<int>(ks % kStages);
            const uint32_t u = static_cast<uint32_t>(ks / kStages);
            if (u >= 1 && !tc::mbar_wait(&mma_done[s], (u - 1) & 1u, abort_flag, status)) break;
            const int64_t j0 = (step0 + ks) * kKStep;
            uint8_t* a_stage = A + s * 4 * kTileBytes;
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int it = gt + 256 * h;
                const int g = it & 7;        // 8-pixel group within the K step
                const int q = it >> 3;       // quad of rows within the pair (0..63)
                const int mt = q >> 5;
                const uint32_t row_t = static_cast<uint32_t>(4 * (q & 31));
                const uint32_t gq = static_cast<uint32_t>((row_pair0 >> 2) + q);
                float z[4][8];
                const int64_t jg = j0 + 8 * g;
                if (row_pair0 + 4 * q < k && jg + 8 <= m) {
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        const uint4 wv = philox4x32_10(make_uint4(static_cast<uint32_t>(jg + p), gq, 0u, 0u), rk);
                        box_muller_fast(wv.x, wv.y, z[0][p], z[1][p]);
                        box_muller_fast(wv.z, wv.w, z[2][p], z[3][p]);
                    }
                } else if (row_pair0 + 4 * q < k) {
                    // pixels past m (last K step only) are drawn and then zeroed
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        const uint4 wv = philox4x32_10(make_uint4(static_cast<uint32_t>(jg + p), gq, 0u, 0u), rk);
                        box_muller_fast(wv.x, wv.y, z[0][p], z[1][p]);
                        box_muller_fast(wv.z, wv.w, z[2][p], z[3][p]);
                        const bool in = (jg + p) < m;
#pragma unroll
                        for (int e = 0; e < 4; ++e) z[e][p] = in ? z[e][p] : 0.0f;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int p = 0; p < 8; ++p) z[e][p] = 0.0f;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int p2 = 0; p2 < 4; ++p2) {
                        const float a = z[e][2 * p2], b = z[e][2 * p2 + 1];
                        const uint32_t ua = __float_as_uint(a) & 0xFFFF0000u;   // hi by truncation
                        const uint32_t ub = __float_as_uint(b) & 0xFFFF0000u;
                        hi[p2] = __byte_perm(ua, ub, 0x7632);
                        lo[p2] = tc::pack_bf16_rn(a - __uint_as_float(ua), b - __uint_as_float(ub));
                    }
                    const uint32_t off = tc::sw128_offset(row_t + e, static_cast<uint32_t>(g));
                    *reinterpret_cast<uint4*>(a_stage + (mt * 2 + 0) * kTileBytes + off) =
                        make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4*>(a_stage + (mt * 2 + 1) * kTileBytes + off) =
                        make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&a_full[s]);
        }
        // ---------------- epilogue (warps 4-7) ----------------
        if (warp < 8) {
            const bool ok = tc::mbar_wait(accum_done, 0u, abort_flag, status) && !*abort_flag;
            tc::tc_fence_after();
            if (ok) {
                const int quarter = warp & 3;
                const int row_in_tile = quarter * 32 + lane;
                for (int mt = 0; mt < 2; ++mt) {
                    const int row = pair * 256 + mt * 128 + row_in_tile;
                    for (int c0 = 0; c0 < npad; c0 += 16) {
                        uint32_t v[16];
                        tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + mt * 256 + c0, v);
                        tc::tmem_wait_ld();
                        if (row < k) {
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const int t = c0 + q;
                                if (t < n) part[static_cast<int64_t>(t) * k + row] = __uint_as_float(v[q]);
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
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_kernel(const __grid_constant__ CUtensorMap tmap, int64_t m, int n, int k, uint2 key,
                 int64_t steps_per_split, int64_t total_steps, float* __restrict__ part, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // the runtime aligns dynamic shared memory to at least 16 bytes; round up
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int split = blockIdx.y;
    const int64_t step0 = static_cast<int64_t>(split) * steps_per_split;
    int64_t nsteps = total_steps - step0;
    if (nsteps > steps_per_split) nsteps = steps_per_split;
    sketch_tc_body(&tmap, m, n, k, key, blockIdx.x, step0, nsteps, part + static_cast<int64_t>(split) * n * k, status,
                   smem);
}

// Grouped launch: CTA b runs work item items[b] (any clip, frame chunk,
// row pair and pixel range); the tensor maps live in global memory.
__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_grouped_kernel(const SketchItem* __restrict__ items, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const SketchItem it = items[blockIdx.x];
    sketch_tc_body(it.tmap, it.m, it.n, it.k, it.key, it.pair, it.step0, it.nsteps, it.part, status, smem);
}

// Grouped fixed-order reduce: element idx of the concatenated outputs belongs
// to chunk c with prefix[c] <= idx < prefix[c+1].
__global__ void sketch_reduce_grouped_kernel(const ReduceChunk* __restrict__ chunks, const int64_t* __restrict__ prefix,
                                             int nchunks, int64_t total, int* status) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int lo = 0, hi = nchunks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    const ReduceChunk c = chunks[lo];
    const int64_t e = idx - prefix[lo];
    double s = 0.0;
    for (int sp = 0; sp < c.splits; ++sp) s += static_cast<double>(c.part[static_cast<int64_t>(sp) * c.elems + e]);
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    c.DY[e] = s;
}

// DY[t*k + i] = sum_s part[(s*n + t)*k + i], FP64, fixed order.
__global__ void sketch_tc_reduce_kernel(const float* __restrict__ part, int splits, int k, int n,
                                        double* __restrict__ DY, int* status) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t total = static_cast<int64_t>(k) * n;
    if (idx >= total) return;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += static_cast<double>(part[static_cast<int64_t>(sp) * total + idx]);
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    DY[idx] = s;
}

}  // namespace

cdmd_status launch_sketch_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, cdmd_ctype ctype,
                             int k, uint64_t seed, double* DY, cudaStream_t stream) {
    if (ctype != CDMD_C_GAUSSIAN)
        return fail(CDMD_ERR_UNSUPPORTED, "BF16X2 sketch is built for the Gaussian measurement matrix");
    if ((reinterpret_cast<uintptr_t>(D) & 15) != 0 || (ldd & 15) != 0)
        return fail(CDMD_ERR_INVALID_ARG, "BF16X2 sketch needs a 16-byte aligned video and ldd %% 16 == 0");
    if (n > kMaxFrames) {
        // the sketch is linear in the frames: DY[t0:t1] = C D[:, t0:t1]
        for (int t0 = 0; t0 < n; t0 += kMaxFrames) {
            const int nc = std::min(kMaxFrames, n - t0);
            cdmd_status st = launch_sketch_tc(ctx, D + static_cast<int64_t>(t0) * ldd, m, nc, ldd, ctype, k, seed,
                                              DY + static_cast<int64_t>(t0) * k, stream);
            if (st != CDMD_OK) return st;
        }
        return CDMD_OK;
    }
    CUtensorMap tmap;
    cdmd_status st = make_video_tmap(&tmap, D, m, n, ldd, kKStep, n);
    if (st != CDMD_OK) return st;
    const int pairs = (k + 255) / 256;
    const int64_t total_steps = (m + kKStep - 1) / kKStep;
    int64_t splits = std::max<int64_t>(1, ctx->num_sms / pairs);
    splits = std::min<int64_t>(splits, total_steps);
    const int64_t steps_per_split = (total_steps + splits - 1) / splits;
    splits = (total_steps + steps_per_split - 1) / steps_per_split;
    float* part = nullptr;
    st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL, static_cast<size_t>(splits) * n * k * sizeof(float),
                       reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    const SmemLayout L = smem_layout(n);
    const size_t smem = L.total + 1024;   // room to align the base to 1024 bytes
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    sketch_tc_kernel<<<dim3(pairs, static_cast<unsigned>(splits)), kThreads, smem, stream>>>(
        tmap, m, n, k, seed_key(seed), steps_per_split, total_steps, part, ctx->d_status);
    CDMD_CHECK_LAUNCH("sketch_tc_kernel");
    const int64_t tot = static_cast<int64_t>(k) * n;
    sketch_tc_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, stream>>>(
        part, static_cast<int>(splits), k, n, DY, ctx->d_status);
    CDMD_CHECK_LAUNCH("sketch_tc_reduce_kernel");
    return CDMD_OK;
}

}  // namespace cdmd

namespace cdmd {

size_t sketch_tc_smem_bytes(int n) { return smem_layout(n).total + 1024; }

cdmd_status launch_sketch_grouped(const SketchItem* items, int nitems, size_t smem, const ReduceChunk* chunks,
                                  const int64_t* prefix, int nchunks, int64_t total, int* status, cudaStream_t stream) {
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(sketch_tc_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    sketch_tc_grouped_kernel<<<static_cast<unsigned>(nitems), kThreads, smem, stream>>>(items, status);
    CDMD_CHECK_LAUNCH("sketch_tc_grouped_kernel");
    sketch_reduce_grouped_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, stream>>>(chunks, prefix, nchunks,
                                                                                                total, status);
    CDMD_CHECK_LAUNCH("sketch_reduce_grouped_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
