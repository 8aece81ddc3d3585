// Pass (a), mixed form: DY = C D on the 5th-generation tensor cores
// (Algorithm 1 steps 2-3, Eq. YCX).
//
// uint8 pixels are exact in BF16; the Gaussian C is split into BF16 hi + lo
// parts (C = hi + lo to ~2^-17 relative) and both products accumulate in FP32
// in tensor memory: D_acc += C_hi D + C_lo D.  C is drawn in-kernel from
// Philox4x32-10 (Box-Muller with the fast MUFU log2 / sin / cos) and never
// touches HBM.
//
// One persistent CTA per SM owns a block of C rows and a contiguous pixel
// range.  Tensor memory holds 512 FP32 columns of 128 rows: every Gaussian a
// CTA draws is applied to as many frames as fit there.
//   per clip   two 128-row tiles of C against one clip's frames (n <= 256 per
//              launch).  Warp 0 TMA-loads the uint8 bytes (64 pixels x n
//              frames per K step) into a staging buffer and warps 2-11
//              convert them to BF16 B tiles in the 128-byte swizzled layout.
//   packed     one 128-row tile of C against up to 512 frames of several
//              clips under the same C (same pixel count, k and seed: windows
//              of one camera).  The frames, widened to BF16 copies in HBM
//              beforehand (`widen_kernel`), are cut into segments packed into
//              two 256-row slots; each segment's tensor copy lands in the B
//              operand directly, so the conversion is done once per clip and
//              not again in every row block.
//   packed, Rademacher C   the same packing, but the +1 / -1 entries are
//              exact in FP16: one product, and sixteen warps convert the
//              uint8 bytes (loaded into registers two K steps ahead) to FP16
//              B tiles in the kernel, so no BF16 copy is made.  With the
//              Gaussian draw the in-kernel conversion costs more issue slots
//              than the widen pass, which overlaps other clips' launches.
// In the per-clip and the Gaussian packed form, warp 1 issues tcgen05.mma
// (M 128, N = frames per slot padded to 16, K 16, hi and lo) into the
// accumulators and commits to the stage's barrier, and warps 4-11 draw the C
// block (rows x 64 pixels) from Philox, split into BF16 hi / lo A tiles.
// After the last K step warps 4-7 read the accumulators (tcgen05.ld) and write
// FP32 partials [split][frame][row]; a second kernel sums the splits in FP64.
// Every mbarrier wait is bounded in time; on a timeout the CTA records
// CDMD_ERR_TIMEOUT, drains its copies and MMAs, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "tc_common.cuh"
#include "batch_internal.cuh"

namespace cdmd {

namespace {

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

// cuTensorMapEncodeTiled from the driver, resolved once (thread-safe static
// initialisation); NULL if the driver does not provide it.
EncodeFn tmap_encoder() {
    static const EncodeFn encode = []() -> EncodeFn {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeFn>(fn);
    }();
    return encode;
}

}  // namespace

cdmd_status make_video_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd, int box_x,
                            int box_y, int swizzle_bytes) {
    const EncodeFn encode = tmap_encoder();
    if (encode == nullptr) return fail(CDMD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(n)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldd)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_x), static_cast<cuuint32_t>(box_y)};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                        : CU_TENSOR_MAP_SWIZZLE_NONE;
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(D), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CDMD_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", static_cast<int>(r));
    return CDMD_OK;
}

// BF16 frames (dim0 = pixels, dim1 = frames, row stride ldw elements), box
// 64 pixels x box_y frames landing in the 128-byte swizzled K-major layout
// the MMA reads (8-row atoms of 1024 bytes); pixels past m read as zero.
static cdmd_status make_wide_tmap(CUtensorMap* map, const uint16_t* W, int64_t m, int n, int64_t ldw, int box_y) {
    const EncodeFn encode = tmap_encoder();
    if (encode == nullptr) return fail(CDMD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(n)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldw) * 2u};
    const cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(box_y)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(W), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CDMD_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", static_cast<int>(r));
    return CDMD_OK;
}

namespace {

constexpr int kThreads = 384;
constexpr int kWorkers = 320;               // warps 2-11
constexpr int kStages = 2;
constexpr int kKStep = 64;                  // pixels per K step (one 128-byte BF16 row)
constexpr int kTileBytes = 128 * 128;       // 128 rows x 128 bytes
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCols = 256;          // one accumulator slot (128 lanes x 256 FP32 columns)
constexpr int kMaxFrames = 256;             // frames per clip and launch: MMA N and TMA box height limits
constexpr size_t kMaxSmem = 232448;         // opt-in shared memory per CTA

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

__host__ __device__ inline int pad16(int n) { return (n + 15) / 16 * 16; }

// Shared memory of one CTA: per stage the A tiles (hi, lo per 128-row tile),
// the B tiles of each clip (frames padded to 16 rows; each clip's region
// starts 2048-byte aligned) and the uint8 staging of each clip (128-byte
// aligned tensor-copy destinations), then the barriers.
struct SmemLayout {
    uint32_t a_stage, b_stage, dst_stage;    // bytes per stage
    uint32_t b_clip[2], dst_clip[2];         // clip offsets inside a stage
    uint32_t a_off, b_off, dst_off, bar_off, misc_off, total;
};

__host__ __device__ inline SmemLayout smem_layout(int mtiles, int nclips, int n0, int n1) {
    SmemLayout L;
    L.a_stage = 2u * static_cast<uint32_t>(mtiles) * kTileBytes;
    uint32_t b = 0, d = 0;
    for (int g = 0; g < 2; ++g) {
        L.b_clip[g] = b;
        L.dst_clip[g] = d;
        if (g < nclips) {
            const int n = g ? n1 : n0;
            b += static_cast<uint32_t>(pad16(n)) * 128u;
            d += (static_cast<uint32_t>(n) * kKStep + 127u) / 128u * 128u;
        }
    }
    L.b_stage = (b + 1023u) / 1024u * 1024u;
    L.dst_stage = d;
    L.a_off = 0;
    L.b_off = kStages * L.a_stage;
    L.dst_off = L.b_off + kStages * L.b_stage;
    L.bar_off = L.dst_off + kStages * L.dst_stage;
    L.misc_off = L.bar_off + (4 * kStages + 1) * 8;
    L.total = L.misc_off + 64;
    return L;
}

// Draw this thread's share of one K step of C: mtiles items of 4 rows x 8
// pixels (gt + 256 h, h < mtiles) of the rows row0 .. row0 + 128 mtiles - 1
// and pixels j0 .. j0 + 63, split into BF16 hi / lo and stored in the A
// stage's 128-byte swizzled K-major tiles (hi, lo per 128-row tile).  Rows
// past k and pixels past m are zero.
__device__ __forceinline__ void draw_c_tiles(uint8_t* a_stage, int gt, int mtiles, int row0, int k, int64_t j0,
                                             int64_t m, const PhiloxKeys& rk) {
#pragma unroll 1
    for (int h = 0; h < mtiles; ++h) {
        const int it = gt + 256 * h;
        const int g = it & 7;        // 8-pixel group within the K step
        const int q = it >> 3;       // quad of rows within the block (0 .. 32 mtiles - 1)
        const int mt = q >> 5;
        const uint32_t row_t = static_cast<uint32_t>(4 * (q & 31));
        const uint32_t gq = static_cast<uint32_t>((row0 >> 2) + q);
        float z[4][8];
        const int64_t jg = j0 + 8 * g;
        if (row0 + 4 * q < k && jg + 8 <= m) {
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const uint4 wv = philox4x32_10(make_uint4(static_cast<uint32_t>(jg + p), gq, 0u, 0u), rk);
                box_muller_fast(wv.x, wv.y, z[0][p], z[1][p]);
                box_muller_fast(wv.z, wv.w, z[2][p], z[3][p]);
            }
        } else if (row0 + 4 * q < k) {
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
            *reinterpret_cast<uint4*>(a_stage + (mt * 2 + 0) * kTileBytes + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(a_stage + (mt * 2 + 1) * kTileBytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

// One 128-row Rademacher tile of C (rows row0 .. row0 + 127, row0 a multiple
// of 128; pixels j0 .. j0 + 63) as BF16 +1 / -1 in the 128-byte swizzled
// K-major layout.  Entry (i, j) is bit (i % 128) % 32 of word (i % 128) / 32
// of the Philox counter (j, i / 128, 1, 0): clear = +1, set = -1.  One counter
// gives all 128 rows of a pixel, so generator warp gw (0 .. 7) covers the rows
// of one word, 32 (gw & 3) .. +31, and 32 pixels, 32 (gw >> 2) .. +31: each
// lane draws one pixel's counter and the warp passes the word round by
// shuffles, lane l keeping bit l (its row).  Rows past k and pixels past m
// are zero.  +1 and -1 are exact in BF16, so C needs no lo part.
__device__ __forceinline__ void draw_rademacher_tile(uint8_t* a_tile, int gw, int lane, int row0, int k, int64_t j0,
                                                     int64_t m, const PhiloxKeys& rk) {
    const int wi = gw & 3;
    const int64_t jb = j0 + 32 * (gw >> 2);
    const uint4 w = philox4x32_10(
        make_uint4(static_cast<uint32_t>(jb + lane), static_cast<uint32_t>(row0 >> 7), 1u, 0u), rk);
    const uint32_t word = wi == 0 ? w.x : wi == 1 ? w.y : wi == 2 ? w.z : w.w;
    const uint32_t row = static_cast<uint32_t>(32 * wi + lane);
    const bool row_ok = row0 + static_cast<int>(row) < k;
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
        uint32_t out[4];
#pragma unroll
        for (int p2 = 0; p2 < 4; ++p2) {
            const int src = gg * 8 + 2 * p2;
            const uint32_t b0 = (__shfl_sync(0xffffffffu, word, src) >> lane) & 1u;
            const uint32_t b1 = (__shfl_sync(0xffffffffu, word, src + 1) >> lane) & 1u;
            const uint32_t e0 = (row_ok && jb + src < m) ? (0x3F80u | (b0 << 15)) : 0u;
            const uint32_t e1 = (row_ok && jb + src + 1 < m) ? (0x3F80u | (b1 << 15)) : 0u;
            out[p2] = e0 | (e1 << 16);
        }
        const uint32_t chunk = static_cast<uint32_t>(4 * (gw >> 2) + gg);   // 8 pixels per 16-byte chunk
        *reinterpret_cast<uint4*>(a_tile + tc::sw128_offset(row, chunk)) = make_uint4(out[0], out[1], out[2], out[3]);
    }
}

// One CTA's share of C D: the rows of C in row block U.rowblk (128 mtiles
// rows) over the 64-pixel K steps step0 .. step0+nsteps-1, against each of
// U.nclips clips, written to U.part[g][t * k + row] (this split's partial
// sums).  Used by the per-clip and the grouped launch.
// U.tmap[g] maps the uint8 frames; the bytes are staged and converted to BF16
// by warps 2-11.
template <bool kRad>
__device__ __forceinline__ void sketch_tc_body(const SketchItem& U, int* status, uint8_t* smem) {
    const int nclips = U.nclips, mtiles = U.mtiles, k = U.k;
    const int n0 = U.n[0], n1 = nclips > 1 ? U.n[1] : 0;
    const SmemLayout L = smem_layout(mtiles, nclips, n0, n1);
    uint8_t* A = smem + L.a_off;
    uint8_t* B = smem + L.b_off;
    uint8_t* Dst = smem + L.dst_off;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* tma_full = bars;
    uint64_t* d_free = bars + kStages;
    uint64_t* ab_full = bars + 2 * kStages;
    uint64_t* mma_done = bars + 3 * kStages;
    uint64_t* accum_done = bars + 4 * kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 8);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int64_t nsteps = U.nsteps < 0 ? 0 : U.nsteps;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&d_free[s], kWorkers);
            tc::mbar_init(&ab_full[s], kWorkers);
            tc::mbar_init(&mma_done[s], 1);
        }
        tc::mbar_init(accum_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // zero the padding rows (frames n..npad-1) of every B region once
    for (int s = 0; s < kStages; ++s)
        for (int g = 0; g < nclips; ++g) {
            const int n = g ? n1 : n0;
            uint8_t* base = B + s * L.b_stage + (g ? L.b_clip[1] : 0u);
            for (uint32_t off = static_cast<uint32_t>(n) * 128u + tid * 16u; off < static_cast<uint32_t>(pad16(n)) * 128u;
                 off += kThreads * 16u)
                *reinterpret_cast<uint4*>(base + off) = make_uint4(0u, 0u, 0u, 0u);
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
            const uint32_t bytes = static_cast<uint32_t>(n0 + n1) * kKStep;
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kStages);
                const uint32_t u = static_cast<uint32_t>(ks / kStages);
                // the slot is free once its bytes were converted
                if (u >= 1 && !tc::mbar_wait(&d_free[s], (u - 1) & 1u, abort_flag, status)) break;
                tc::mbar_arrive_expect_tx(&tma_full[s], bytes);
                const int x = static_cast<int>((U.step0 + ks) * kKStep);
                for (int g = 0; g < nclips; ++g)
                    tc::tma_load_2d(Dst + s * L.dst_stage + (g ? L.dst_clip[1] : 0u), g ? U.tmap[1] : U.tmap[0], x, 0,
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
            const uint32_t idesc0 = tc::idesc_bf16_f32(128, pad16(n0));
            const uint32_t idesc1 = tc::idesc_bf16_f32(128, pad16(n1 > 0 ? n1 : 16));
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kStages);
                const uint32_t par = static_cast<uint32_t>(ks / kStages) & 1u;
                if (!tc::mbar_wait(&ab_full[s], par, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + s * L.a_stage);
                const uint32_t b_base = tc::smem_u32(B + s * L.b_stage);
#pragma unroll 1
                for (int mt = 0; mt < mtiles; ++mt) {
#pragma unroll 1
                    for (int g = 0; g < nclips; ++g) {
                        const uint32_t acc = tmem_base + static_cast<uint32_t>(mt * nclips + g) * kAccCols;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bdesc = tc::desc_sw128(b_base + (g ? L.b_clip[1] : 0u) + kk * 32);
#pragma unroll
                            for (int hl = 0; hl < (kRad ? 1 : 2); ++hl) {
                                const uint64_t adesc = tc::desc_sw128(a_base + (mt * 2 + hl) * kTileBytes + kk * 32);
                                tc::mma_bf16(acc, adesc, bdesc, g ? idesc1 : idesc0, (ks | kk | hl) ? 1u : 0u);
                            }
                        }
                    }
                }
                tc::mma_commit(&mma_done[s]);
            }
            tc::mma_commit(accum_done);   // fires once every MMA issued above has finished
        }
    } else {
        // ---------------- workers: C generators (warps 4-11) and converters (warps 2-11) ----------------
        const int wt = tid - 64;
        const bool gen = warp >= 4;
        const int gt = tid - 128;
        const int row0 = U.rowblk * 128 * mtiles;
        const int conv0 = n0 * 8, conv_total = (n0 + n1) * 8;
        const PhiloxKeys rk = philox_round_keys(U.key);   // the same for every draw of this CTA
        for (int64_t ks = 0; ks < nsteps; ++ks) {
            const int s = static_cast<int>(ks % kStages);
            const uint32_t u = static_cast<uint32_t>(ks / kStages);
            if (u >= 1 && !tc::mbar_wait(&mma_done[s], (u - 1) & 1u, abort_flag, status)) break;
            if (gen) {
                if constexpr (kRad) {
                    for (int mt = 0; mt < mtiles; ++mt)
                        draw_rademacher_tile(A + s * L.a_stage + (mt * 2) * kTileBytes, warp - 4, lane,
                                             row0 + 128 * mt, k, (U.step0 + ks) * kKStep, U.m, rk);
                } else {
                    draw_c_tiles(A + s * L.a_stage, gt, mtiles, row0, k, (U.step0 + ks) * kKStep, U.m, rk);
                }
            }
            // uint8 -> BF16: 8 pixels of one frame per item, over both clips
            if (!tc::mbar_wait(&tma_full[s], u & 1u, abort_flag, status)) break;
            const uint8_t* src_stage = Dst + s * L.dst_stage;
            uint8_t* b_stage = B + s * L.b_stage;
            for (int it = wt; it < conv_total; it += kWorkers) {
                const int g = it >= conv0 ? 1 : 0;
                const int li = it - (g ? conv0 : 0);
                const int t = li >> 3, c8 = li & 7;
                const uint2 raw = *reinterpret_cast<const uint2*>(src_stage + (g ? L.dst_clip[1] : 0u) + t * kKStep + c8 * 8);
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t word = h ? raw.y : raw.x;
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        // byte b of the word into a float with exponent 2^23: 2^23 + b, exact
                        const float f0 = __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7540u + 2u * e)) - 8388608.0f;
                        const float f1 = __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7541u + 2u * e)) - 8388608.0f;
                        w[h * 2 + e] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
                    }
                }
                *reinterpret_cast<uint4*>(b_stage + (g ? L.b_clip[1] : 0u) +
                                          tc::sw128_offset(static_cast<uint32_t>(t), static_cast<uint32_t>(c8))) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&d_free[s]);
            tc::mbar_arrive(&ab_full[s]);
        }
        // ---------------- epilogue (warps 4-7) ----------------
        if (warp >= 4 && warp < 8) {
            const bool ok = tc::mbar_wait(accum_done, 0u, abort_flag, status) && !*abort_flag;
            tc::tc_fence_after();
            if (ok) {
                const int quarter = warp & 3;
                const int row_in_tile = quarter * 32 + lane;
                for (int mt = 0; mt < mtiles; ++mt) {
                    const int row = row0 + mt * 128 + row_in_tile;
                    for (int g = 0; g < nclips; ++g) {
                        const int n = g ? n1 : n0;
                        float* part = g ? U.part[1] : U.part[0];
                        const uint32_t col = static_cast<uint32_t>(mt * nclips + g) * kAccCols;
                        for (int c0 = 0; c0 < pad16(n); c0 += 16) {
                            uint32_t v[16];
                            tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + col + c0, v);
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

struct SketchArgs {
    float* part[2];             // [splits][n_g][k] partial sums of each clip
    int n[2];
    int nclips, mtiles, k;
    int64_t m, steps_per_split, total_steps;
    uint2 key;
};

template <bool kRad>
__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_kernel(const __grid_constant__ CUtensorMap tmap0, const __grid_constant__ CUtensorMap tmap1,
                 const SketchArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // the runtime aligns dynamic shared memory to at least 16 bytes; round up
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int split = blockIdx.y;
    SketchItem U;
    U.tmap[0] = &tmap0;
    U.tmap[1] = &tmap1;
    U.step0 = static_cast<int64_t>(split) * a.steps_per_split;
    U.nsteps = a.total_steps - U.step0;
    if (U.nsteps > a.steps_per_split) U.nsteps = a.steps_per_split;
    U.n[0] = a.n[0];
    U.n[1] = a.n[1];
    U.part[0] = a.part[0] + static_cast<int64_t>(split) * a.n[0] * a.k;
    U.part[1] = a.nclips > 1 ? a.part[1] + static_cast<int64_t>(split) * a.n[1] * a.k : nullptr;
    U.m = a.m;
    U.key = a.key;
    U.nclips = a.nclips;
    U.mtiles = a.mtiles;
    U.k = a.k;
    U.rowblk = blockIdx.x;
    sketch_tc_body<kRad>(U, status, smem);
}

// Grouped launch: CTA b runs work item items[b] (any clip or clip pair, frame
// chunk, row block and pixel range); the tensor maps live in global memory.
__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_grouped_kernel(const SketchItem* __restrict__ items, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const SketchItem it = items[blockIdx.x];
    sketch_tc_body<false>(it, status, smem);
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

// ---------------------------------------------------------------------------
// Packed form: the frames of several clips under one C, cut into segments of
// consecutive frames and packed into two 256-row B slots (512 rows = the 512
// FP32 columns of tensor memory).  One 128-row tile of C per CTA: each
// Gaussian drawn feeds up to 512 frames of whichever clips the launch holds.
// Segments start on 8-row boundaries (1024-byte swizzle atoms) and never
// cross a slot; a segment's frames come from the BF16 copy of its clip by
// one tensor copy of box 64 pixels x L frames.  Rows no segment covers stay
// zero.  Partials are [split][B row][k]; a reduce per segment writes the
// clip's DY columns f0 .. f0 + L - 1.
// ---------------------------------------------------------------------------
constexpr int kPackRows = 512;
constexpr int kMaxSeg = 8;
constexpr uint32_t kPackBStage = kPackRows * 128u;     // bytes of one B stage
constexpr uint32_t kPackAStage = 2u * kTileBytes;      // hi, lo of one 128-row tile

struct PackSeg {
    double* DY;        // the clip's DY (frame-major, k per frame)
    int row0, L, f0;   // B rows row0 .. row0 + L - 1 hold frames f0 .. f0 + L - 1
    int pad;
};

struct PackArgs {
    CUtensorMap tmap[kMaxSeg];   // per segment: the clip's BF16 frames, box 64 x L
    PackSeg seg[kMaxSeg];
    float* part;                 // [splits][kPackRows][k]
    int nseg, k;
    int nslot[2];                // rows of each slot the MMAs cover (multiples of 16, 0 = unused)
    int64_t m, steps_per_split, total_steps;
    uint2 key;
};

__host__ __device__ inline uint32_t pack_smem_bytes() {
    return kStages * (kPackAStage + kPackBStage) + (3 * kStages + 1) * 8 + 64;
}

__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_packed_kernel(const __grid_constant__ PackArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* A = smem;
    uint8_t* B = smem + kStages * kPackAStage;
    uint64_t* bars = reinterpret_cast<uint64_t*>(B + kStages * kPackBStage);
    uint64_t* tma_full = bars;
    uint64_t* ab_full = bars + kStages;
    uint64_t* mma_done = bars + 2 * kStages;
    uint64_t* accum_done = bars + 3 * kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kStages + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int k = a.k;
    const int split = blockIdx.y;
    const int row0 = blockIdx.x * 128;
    const int64_t step0 = static_cast<int64_t>(split) * a.steps_per_split;
    int64_t nsteps = a.total_steps - step0;
    if (nsteps > a.steps_per_split) nsteps = a.steps_per_split;
    if (nsteps < 0) nsteps = 0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&ab_full[s], 256);
            tc::mbar_init(&mma_done[s], 1);
        }
        tc::mbar_init(accum_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // rows no segment covers must read as zero: clear both B stages once
    for (uint32_t off = tid * 16u; off < kStages * kPackBStage; off += kThreads * 16u)
        *reinterpret_cast<uint4*>(B + off) = make_uint4(0u, 0u, 0u, 0u);
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
            uint32_t bytes = 0;
            for (int i = 0; i < a.nseg; ++i) bytes += static_cast<uint32_t>(a.seg[i].L) * 128u;
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kStages);
                const uint32_t u = static_cast<uint32_t>(ks / kStages);
                // the slot's B rows are free once the MMAs that read them finished
                if (u >= 1 && !tc::mbar_wait(&mma_done[s], (u - 1) & 1u, abort_flag, status)) break;
                tc::mbar_arrive_expect_tx(&tma_full[s], bytes);
                const int x = static_cast<int>((step0 + ks) * kKStep);
                for (int i = 0; i < a.nseg; ++i)
                    tc::tma_load_2d(B + s * kPackBStage + static_cast<uint32_t>(a.seg[i].row0) * 128u, &a.tmap[i], x,
                                    a.seg[i].f0, &tma_full[s]);
            }
            for (int s = 0; s < kStages; ++s) {
                const int64_t uses = (nsteps - s + kStages - 1) / kStages;
                if (uses >= 1) tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc0 = tc::idesc_bf16_f32(128, a.nslot[0] > 0 ? a.nslot[0] : 16);
            const uint32_t idesc1 = tc::idesc_bf16_f32(128, a.nslot[1] > 0 ? a.nslot[1] : 16);
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kStages);
                const uint32_t par = static_cast<uint32_t>(ks / kStages) & 1u;
                if (!tc::mbar_wait(&ab_full[s], par, abort_flag, status)) break;
                if (!tc::mbar_wait(&tma_full[s], par, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + s * kPackAStage);
                const uint32_t b_base = tc::smem_u32(B + s * kPackBStage);
#pragma unroll
                for (int slot = 0; slot < 2; ++slot) {
                    if (a.nslot[slot] == 0) continue;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bdesc = tc::desc_sw128(b_base + slot * (kPackBStage / 2) + kk * 32);
#pragma unroll
                        for (int hl = 0; hl < 2; ++hl) {
                            const uint64_t adesc = tc::desc_sw128(a_base + hl * kTileBytes + kk * 32);
                            tc::mma_bf16(tmem_base + slot * kAccCols, adesc, bdesc, slot ? idesc1 : idesc0,
                                         (ks | kk | hl) ? 1u : 0u);
                        }
                    }
                }
                tc::mma_commit(&mma_done[s]);
            }
            tc::mma_commit(accum_done);
        }
    } else if (warp >= 4) {
        // ---------------- C generators (warps 4-11) ----------------
        const int gt = tid - 128;
        const PhiloxKeys rk = philox_round_keys(a.key);
        for (int64_t ks = 0; ks < nsteps; ++ks) {
            const int s = static_cast<int>(ks % kStages);
            const uint32_t u = static_cast<uint32_t>(ks / kStages);
            if (u >= 1 && !tc::mbar_wait(&mma_done[s], (u - 1) & 1u, abort_flag, status)) break;
            draw_c_tiles(A + s * kPackAStage, gt, 1, row0, k, (step0 + ks) * kKStep, a.m, rk);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&ab_full[s]);
        }
        // ---------------- epilogue (warps 4-7): partials of every used B row ----------------
        if (warp < 8) {
            const bool ok = tc::mbar_wait(accum_done, 0u, abort_flag, status) && !*abort_flag;
            tc::tc_fence_after();
            if (ok) {
                const int quarter = warp & 3;
                const int row = row0 + quarter * 32 + lane;
                float* part = a.part + static_cast<int64_t>(split) * kPackRows * k;
                for (int slot = 0; slot < 2; ++slot) {
                    for (int c0 = 0; c0 < a.nslot[slot]; c0 += 16) {
                        uint32_t v[16];
                        tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + slot * kAccCols + c0,
                                        v);
                        tc::tmem_wait_ld();
                        if (row < k) {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                part[static_cast<int64_t>(slot * 256 + c0 + q) * k + row] = __uint_as_float(v[q]);
                        }
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (*abort_flag) tc::mbar_wait(accum_done, 0u, abort_flag, status, 2000000000ull);
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Packed form on CTA pairs (cta_group::2): the CTAs of row blocks 2c and 2c + 1
// form a cluster and one 2-SM MMA (M = 256) covers both 128-row tiles of C.
// Each CTA draws its own tile of C (A) and holds half of every 256-row B slot
// (rows 0-127 in the leader, rank 0; 128-255 in the other), so each copies
// and reads half of the frames a single-CTA launch needs: the frame stages
// shrink to 32 KB and three of them fit beside four stages of C (the draw of
// step k + 4 never waits for the MMAs of step k; three frame stages cover a
// copy's latency at this step rate).
//   warp 0      TMA (both CTAs): this CTA's segments of each stage, on its
//               own stage barrier (so each CTA can drain its own copies
//               before it leaves)
//   warp 2      the other CTA: when its half of a stage has landed, arrives
//               on the leader's barrier for that stage (cluster scope)
//   warp 1      leader: the pair MMAs (N = 256 per used slot), commits to
//               the stage barriers of both CTAs (multicast)
//   warp 3      the other CTA: when its tile of C is drawn, arrives on the
//               leader's barrier for that stage (cluster scope)
//   warps 4-11  both CTAs: draw C; one arrival per warp on this CTA's
//               barrier (a cluster-scope release costs about a thousand
//               cycles, so only the relay threads pay it)
//   warps 4-7   after the last K step: this CTA's accumulators (its 128
//               rows of C x every frame column) to the FP32 partials
// Segments never cross a 128-row half (the host cuts them there).
// ---------------------------------------------------------------------------
constexpr int kQAStages = 4;
constexpr int kQBStages = 3;
constexpr uint32_t kQBStage = kPackRows * 128u / 2u;     // this CTA's half of 512 B rows
constexpr uint32_t kQHalf = 128u * 128u;                 // one slot's half: 128 rows x 128 bytes

__host__ __device__ inline uint32_t pair_smem_bytes() {
    return kQAStages * kPackAStage + kQBStages * kQBStage + (3 * kQAStages + 3 * kQBStages + 1) * 8 + 64;
}

__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_pair_kernel(const __grid_constant__ PackArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* A = smem;
    uint8_t* B = smem + kQAStages * kPackAStage;
    uint64_t* bars = reinterpret_cast<uint64_t*>(B + kQBStages * kQBStage);
    uint64_t* tma_full = bars;                          // [kQBStages] this CTA's half landed
    uint64_t* b_free = bars + kQBStages;                // [kQBStages] pair MMAs done with the frames
    uint64_t* peer_ready = bars + 2 * kQBStages;        // [kQBStages] leader: the other half landed
    uint64_t* a_full = bars + 3 * kQBStages;            // [kQAStages] leader: both tiles of C drawn
    uint64_t* a_free = a_full + kQAStages;              // [kQAStages] pair MMAs done with C
    uint64_t* a_local = a_free + kQAStages;             // [kQAStages] this CTA's tile of C drawn
    uint64_t* accum_done = a_local + kQAStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int k = a.k;
    const uint32_t crank = tc::cluster_ctarank();
    const bool leader = crank == 0;
    const int split = blockIdx.y;
    const int row0 = blockIdx.x * 128;
    const int64_t step0 = static_cast<int64_t>(split) * a.steps_per_split;
    int64_t nsteps = a.total_steps - step0;
    if (nsteps > a.steps_per_split) nsteps = a.steps_per_split;
    if (nsteps < 0) nsteps = 0;

    if (tid == 0) {
        for (int s = 0; s < kQBStages; ++s) {
            tc::mbar_init(&tma_full[s], 1);
            tc::mbar_init(&b_free[s], 1);
            tc::mbar_init(&peer_ready[s], 1);
        }
        for (int s = 0; s < kQAStages; ++s) {
            tc::mbar_init(&a_full[s], 8 + 1);          // the leader's drawing warps + the other CTA's relay
            tc::mbar_init(&a_free[s], 1);
            tc::mbar_init(&a_local[s], 8);
        }
        tc::mbar_init(accum_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // rows no segment covers must read as zero: clear this CTA's B stages once
    for (uint32_t off = tid * 16u; off < kQBStages * kQBStage; off += kThreads * 16u)
        *reinterpret_cast<uint4*>(B + off) = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_proxy_async_smem();
    if (warp == 0) {
        tc::tmem_alloc_cg2(tmem_slot, kTmemCols);
        tc::tmem_relinquish_cg2();
    }
    tc::tc_fence_before();
    __syncthreads();
    // both CTAs' barriers exist before either signals the other's
    tc::cluster_sync_all();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            uint32_t bytes_own = 0;
            for (int i = 0; i < a.nseg; ++i)
                if (static_cast<uint32_t>((a.seg[i].row0 & 255) >> 7) == crank)
                    bytes_own += static_cast<uint32_t>(a.seg[i].L) * 128u;
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kQBStages);
                const uint32_t u = static_cast<uint32_t>(ks / kQBStages);
                // this CTA's half of the stage is free once the pair MMAs that read it finished
                if (u >= 1 && !tc::mbar_wait_cl(&b_free[s], (u - 1) & 1u, abort_flag, status)) break;
                tc::mbar_arrive_expect_tx(&tma_full[s], bytes_own);
                const int x = static_cast<int>((step0 + ks) * kKStep);
                for (int i = 0; i < a.nseg; ++i) {
                    const int r0 = a.seg[i].row0;
                    if (static_cast<uint32_t>((r0 & 255) >> 7) != crank) continue;
                    uint8_t* dst = B + s * kQBStage + static_cast<uint32_t>(r0 >> 8) * kQHalf +
                                   static_cast<uint32_t>(r0 & 127) * 128u;
                    tc::tma_load_2d(dst, &a.tmap[i], x, a.seg[i].f0, &tma_full[s]);
                }
            }
            // drain: this CTA's last copies of each stage have landed before it
            // leaves (bounded in time only: an abort elsewhere must not cut it short)
            volatile int no_abort = 0;
            for (int s = 0; s < kQBStages; ++s) {
                const int64_t uses = (nsteps - s + kQBStages - 1) / kQBStages;
                if (uses >= 1) tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(uses - 1) & 1u, &no_abort, status);
            }
        }
    } else if (warp == 3) {
        // ---------------- relay of the drawn C tiles (the other CTA) ----------------
        if (lane == 0 && !leader) {
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int sa = static_cast<int>(ks % kQAStages);
                if (!tc::mbar_wait(&a_local[sa], static_cast<uint32_t>(ks / kQAStages) & 1u, abort_flag, status))
                    break;
                tc::mbar_arrive_cluster(tc::mapa_u32(tc::smem_u32(&a_full[sa]), 0u));
            }
        }
    } else if (warp == 2) {
        // ---------------- forwarder (the other CTA) ----------------
        if (lane == 0 && !leader) {
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kQBStages);
                if (!tc::mbar_wait(&tma_full[s], static_cast<uint32_t>(ks / kQBStages) & 1u, abort_flag, status))
                    break;
                tc::mbar_arrive_cluster(tc::mapa_u32(tc::smem_u32(&peer_ready[s]), 0u));
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (leader) ----------------
        if (lane == 0 && leader) {
            const uint32_t idesc = tc::idesc_bf16_f32(256, 256);
            for (int64_t ks = 0; ks < nsteps; ++ks) {
                const int s = static_cast<int>(ks % kQBStages);
                const uint32_t pb = static_cast<uint32_t>(ks / kQBStages) & 1u;
                const int sa = static_cast<int>(ks % kQAStages);
                const uint32_t pa = static_cast<uint32_t>(ks / kQAStages) & 1u;
                if (!tc::mbar_wait_cl(&a_full[sa], pa, abort_flag, status)) break;
                if (!tc::mbar_wait(&tma_full[s], pb, abort_flag, status)) break;
                if (!tc::mbar_wait_cl(&peer_ready[s], pb, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + sa * kPackAStage);
                const uint32_t b_base = tc::smem_u32(B + s * kQBStage);
#pragma unroll
                for (int slot = 0; slot < 2; ++slot) {
                    if (a.nslot[slot] == 0) continue;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bdesc = tc::desc_sw128(b_base + slot * kQHalf + kk * 32);
#pragma unroll
                        for (int hl = 0; hl < 2; ++hl) {
                            const uint64_t adesc = tc::desc_sw128(a_base + hl * kTileBytes + kk * 32);
                            tc::mma_bf16_cg2(tmem_base + slot * kAccCols, adesc, bdesc, idesc,
                                             (ks | kk | hl) ? 1u : 0u);
                        }
                    }
                }
                tc::mma_commit_cg2(&b_free[s], 3);
                tc::mma_commit_cg2(&a_free[sa], 3);
            }
            tc::mma_commit_cg2(accum_done, 3);
        }
    } else if (warp >= 4) {
        // ---------------- C generators (warps 4-11, both CTAs) ----------------
        const int gt = tid - 128;
        const PhiloxKeys rk = philox_round_keys(a.key);
        for (int64_t ks = 0; ks < nsteps; ++ks) {
            const int sa = static_cast<int>(ks % kQAStages);
            const uint32_t u = static_cast<uint32_t>(ks / kQAStages);
            if (u >= 1 && !tc::mbar_wait_cl(&a_free[sa], (u - 1) & 1u, abort_flag, status)) break;
            draw_c_tiles(A + sa * kPackAStage, gt, 1, row0, k, (step0 + ks) * kKStep, a.m, rk);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(leader ? &a_full[sa] : &a_local[sa]);
        }
        // ---------------- epilogue (warps 4-7): this CTA's 128 rows ----------------
        if (warp < 8) {
            const bool ok = tc::mbar_wait_cl(accum_done, 0u, abort_flag, status) && !*abort_flag;
            tc::tc_fence_after();
            if (ok) {
                const int quarter = warp & 3;
                const int row = row0 + quarter * 32 + lane;
                float* part = a.part + static_cast<int64_t>(split) * kPackRows * k;
                for (int slot = 0; slot < 2; ++slot) {
                    for (int c0 = 0; c0 < a.nslot[slot]; c0 += 16) {
                        uint32_t v[16];
                        tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + slot * kAccCols + c0,
                                        v);
                        tc::tmem_wait_ld();
                        if (row < k) {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                part[static_cast<int64_t>(slot * 256 + c0 + q) * k + row] = __uint_as_float(v[q]);
                        }
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0) {
        // no pair MMA may still read either CTA's shared memory or write
        // tensor memory when the CTAs leave: wait for the last commit
        volatile int no_abort = 0;
        tc::mbar_wait_cl(accum_done, 0u, &no_abort, status);
    }
    __syncthreads();
    tc::cluster_sync_all();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc_cg2(tmem_base, kTmemCols);
    }
}

// DY of segment blockIdx.y: DY[(f0 + t) k + i] = sum_s part[s][row0 + t][i], FP64, fixed order.
__global__ void sketch_packed_reduce_kernel(const __grid_constant__ PackArgs a, int splits, int* status) {
    const PackSeg sg = a.seg[blockIdx.y];
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t total = static_cast<int64_t>(sg.L) * a.k;
    if (idx >= total) return;
    const int64_t src = static_cast<int64_t>(sg.row0) * a.k + idx;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += static_cast<double>(a.part[static_cast<int64_t>(sp) * kPackRows * a.k + src]);
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    sg.DY[static_cast<int64_t>(sg.f0) * a.k + idx] = s;
}

// W[t * ldw + j] = D[t * ldd + j] as BF16 (exact for uint8) for j < m, zero for
// m <= j < ldw; 16 pixels per thread, blockIdx.y = frame.
__global__ void widen_kernel(const uint8_t* __restrict__ D, int64_t m, int64_t ldd, uint16_t* __restrict__ W,
                             int64_t ldw) {
    const int64_t t = blockIdx.y;
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 16;
    if (j >= ldw) return;
    const uint8_t* src = D + t * ldd + j;
    uint32_t b[4];
    if (j + 16 <= m) {
        const uint4 raw = *reinterpret_cast<const uint4*>(src);
        b[0] = raw.x; b[1] = raw.y; b[2] = raw.z; b[3] = raw.w;
    } else {
        // the last chunk of a row: read only the bytes below m
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            b[w] = 0u;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (j + 4 * w + e < m) b[w] |= static_cast<uint32_t>(src[4 * w + e]) << (8 * e);
        }
    }
    uint32_t o[8];
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float f0 = __uint_as_float(__byte_perm(b[w], 0x4B000000u, 0x7540u + 2u * e)) - 8388608.0f;
            const float f1 = __uint_as_float(__byte_perm(b[w], 0x4B000000u, 0x7541u + 2u * e)) - 8388608.0f;
            o[2 * w + e] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
        }
    uint4* dst = reinterpret_cast<uint4*>(W + t * ldw + j);
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

// ---------------------------------------------------------------------------
// Packed form for the Rademacher C, straight from the uint8 frames.  The
// entries +1 / -1 are exact in FP16, so one product suffices and the B tiles
// are built in the kernel: each of warps 1-16 loads the bytes of four B rows
// (16 pixels each) into registers two 64-pixel K steps ahead and converts
// them to FP16 (the byte permute 0x6400 | b = 1024 + b, then one packed
// subtract of 1024) in the 128-byte swizzled K-major layout.  With only a
// Philox counter per 32 pixels to draw, the Gaussian form's widened BF16
// copies would leave this kernel bound by their tensor copies (eight
// row-block CTAs each read every BF16 tile); reading the bytes halves that
// traffic and needs no copy of the frames.
//   warp 0       tensor-memory allocation; lane 0 issues tcgen05.mma per K
//                step (per slot four K16 quarters) into 2 x 256 FP32 columns
//   warps 1-16   per K step: the C tile (row g / 4, 16 pixels) into the A
//                stage, four B rows into the B stage; 2 operand stages.
//                Lane 0 waits for a stage and arrives for its warp.
//   warps 1-16   after the last K step: the accumulators to FP32 partials
//                [split][B row][k]; a reduce per segment sums the splits in
//                FP64 into the clip's DY columns f0 .. f0 + L - 1.
// Rows no segment covers read as zero: the B stages are cleared once and
// those rows are never written.
// ---------------------------------------------------------------------------
constexpr int kRadRows = 512;
constexpr int kRadMaxSeg = 8;
constexpr int kRThreads = 544;                           // warp 0 + 16 generator warps
constexpr int kRGenWarps = 16;                           // warps 1-16
constexpr int kRKStep = 64;                              // pixels per K step
constexpr int kRBuf = 2;                                 // operand stages = K steps of bytes in flight
constexpr uint32_t kRAStage = 128u * 128u;               // 128 rows x 128 bytes of FP16
constexpr uint32_t kRSlotBytes = 256u * 128u;            // one 256-row slot of B
constexpr uint32_t kRBStage = 2u * kRSlotBytes;          // 512 rows x 128 bytes of FP16

struct RadSeg {
    double* DY;             // the clip's DY (frame-major, k per frame)
    const uint8_t* D;       // the segment's first frame
    int64_t ldd;            // bytes between frames
    int row0, L, f0;        // B rows row0 .. row0 + L - 1 hold frames f0 .. f0 + L - 1
    int pad;
};

struct RadArgs {
    RadSeg seg[kRadMaxSeg];
    PhiloxKeys rk;               // round keys of the seed (constant for the launch)
    float* part;                 // [splits][kRadRows][k]
    int nseg, k;
    int nslot[2];                // rows of each slot the MMAs cover (multiples of 16, 0 = unused)
    int64_t m;
    int steps_per_split, total_steps;
};

__host__ __device__ inline uint32_t rad_smem_bytes() {
    return kRBuf * (kRAStage + kRBStage) + (2 * kRBuf + 1) * 8 + 64;
}

// 16 bytes of a B row at pixel j (16-byte aligned), streaming; pixels at or
// past m and rows no segment covers (src == nullptr) read as zero.
__device__ __forceinline__ uint4 load_row16(const uint8_t* src, int64_t j, int64_t m) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (src == nullptr || j >= m) return v;
    const uint8_t* p = src + j;
    if (j + 16 <= m) {
        asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p));
        return v;
    }
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 16; ++e)
        if (j + e < m) w[e >> 2] |= static_cast<uint32_t>(p[e]) << (8 * (e & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// The same where the whole 16 bytes are below m (every split but the one
// holding the ragged end of the frame).
__device__ __forceinline__ uint4 load_row16_full(const uint8_t* src, int64_t j) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (src != nullptr)
        asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(src + j));
    return v;
}

// 16 uint8 pixels as FP16 into two 16-byte chunks (off_a, off_a ^ 16 apart
// by the swizzle) of a B row.
__device__ __forceinline__ void convert_row16(uint8_t* b_stage, uint32_t off_a, uint32_t off_b, uint4 raw) {
    uint32_t w[8];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint32_t word = h == 0 ? raw.x : h == 1 ? raw.y : h == 2 ? raw.z : raw.w;
        w[h * 2 + 0] = tc::sub_1024_f16x2(__byte_perm(word, 0x64646464u, 0x4140u));
        w[h * 2 + 1] = tc::sub_1024_f16x2(__byte_perm(word, 0x64646464u, 0x4342u));
    }
    *reinterpret_cast<uint4*>(b_stage + off_a) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(b_stage + off_b) = make_uint4(w[4], w[5], w[6], w[7]);
}

// One Rademacher item as FP16 +1 / -1: row r = g / 4 of the tile, pixels
// j0 + 16 (g mod 4) .. + 15, two 16-byte chunks.  Entry (i, j) is bit
// (i % 128) % 32 of word (i % 128) / 32 of the Philox counter (j, i / 128,
// 1, 0): clear = +1, set = -1.  Lane l draws the counters of pixels j0 + l
// and j0 + 32 + l (every row of a warp lies in one word) and the warp passes
// the words round by shuffles.  Rows past k and pixels past m are zero.
__device__ __forceinline__ void draw_rademacher_f16(uint8_t* a_stage, uint32_t off_a, uint32_t off_b, int lane, int r,
                                                    int pg, int row0, int k, int64_t j0, int64_t m,
                                                    const PhiloxKeys& rk) {
    const uint32_t blk = static_cast<uint32_t>(row0 >> 7);
    const uint4 wa = philox4x32_10(make_uint4(static_cast<uint32_t>(j0) + lane, blk, 1u, 0u), rk);
    const uint4 wb = philox4x32_10(make_uint4(static_cast<uint32_t>(j0) + 32u + lane, blk, 1u, 0u), rk);
    const int wi = r >> 5;
    const uint32_t word_a = wi == 0 ? wa.x : wi == 1 ? wa.y : wi == 2 ? wa.z : wa.w;
    const uint32_t word_b = wi == 0 ? wb.x : wi == 1 ? wb.y : wi == 2 ? wb.z : wb.w;
    const bool row_ok = row0 + r < k;
    const bool hi_half = pg >= 2;                   // pixels 32 .. 63 of the step
    uint32_t out[8];
#pragma unroll
    for (int p2 = 0; p2 < 8; ++p2) {
        const int src = 16 * (pg & 1) + 2 * p2;     // lane of the counter
        const uint32_t a0 = __shfl_sync(0xffffffffu, word_a, src), a1 = __shfl_sync(0xffffffffu, word_a, src + 1);
        const uint32_t b0 = __shfl_sync(0xffffffffu, word_b, src), b1 = __shfl_sync(0xffffffffu, word_b, src + 1);
        const uint32_t s0 = ((hi_half ? b0 : a0) >> (r & 31)) & 1u;
        const uint32_t s1 = ((hi_half ? b1 : a1) >> (r & 31)) & 1u;
        const int64_t jp = j0 + 16 * pg + 2 * p2;
        const uint32_t e0 = (row_ok && jp < m) ? (0x3C00u | (s0 << 15)) : 0u;
        const uint32_t e1 = (row_ok && jp + 1 < m) ? (0x3C00u | (s1 << 15)) : 0u;
        out[p2] = e0 | (e1 << 16);
    }
    *reinterpret_cast<uint4*>(a_stage + off_a) = make_uint4(out[0], out[1], out[2], out[3]);
    *reinterpret_cast<uint4*>(a_stage + off_b) = make_uint4(out[4], out[5], out[6], out[7]);
}

__global__ void __launch_bounds__(kRThreads, 1)
sketch_rad_u8_kernel(const __grid_constant__ RadArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* A = smem;                                   // kRBuf x C tiles
    uint8_t* B = smem + kRBuf * kRAStage;                // kRBuf x 512-row FP16 tiles
    uint64_t* bars = reinterpret_cast<uint64_t*>(B + kRBuf * kRBStage);
    uint64_t* ab_full = bars;                            // [kRBuf] A and B written
    uint64_t* mma_done = bars + kRBuf;                   // [kRBuf] read by the MMAs
    uint64_t* accum_done = bars + 2 * kRBuf;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int k = a.k;
    const int split = blockIdx.y;
    const int row0 = blockIdx.x * 128;
    const int nslot0 = a.nslot[0], nslot1 = a.nslot[1];
    const int step0 = split * a.steps_per_split;
    int nsteps = a.total_steps - step0;
    if (nsteps > a.steps_per_split) nsteps = a.steps_per_split;
    if (nsteps < 0) nsteps = 0;

    if (tid == 0) {
        for (int s = 0; s < kRBuf; ++s) {
            tc::mbar_init(&ab_full[s], kRGenWarps);
            tc::mbar_init(&mma_done[s], 1);
        }
        tc::mbar_init(accum_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // rows no segment covers must read as zero: clear the B stages once
    for (uint32_t off = tid * 16u; off < kRBuf * kRBStage; off += kRThreads * 16u)
        *reinterpret_cast<uint4*>(B + off) = make_uint4(0u, 0u, 0u, 0u);
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
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc0 = tc::idesc_f16_f32(128, nslot0 > 0 ? nslot0 : 16);
            const uint32_t idesc1 = tc::idesc_f16_f32(128, nslot1 > 0 ? nslot1 : 16);
            int s = 0;
            uint32_t ph = 0;
            for (int ks = 0; ks < nsteps; ++ks) {
                if (!tc::mbar_wait(&ab_full[s], ph, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(A + s * kRAStage);
                const uint32_t b_base = tc::smem_u32(B + s * kRBStage);
#pragma unroll
                for (int slot = 0; slot < 2; ++slot) {
                    if ((slot ? nslot1 : nslot0) == 0) continue;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bdesc = tc::desc_sw128(b_base + slot * kRSlotBytes + kk * 32);
                        const uint64_t adesc = tc::desc_sw128(a_base + kk * 32);
                        tc::mma_f16(tmem_base + slot * kAccCols, adesc, bdesc, slot ? idesc1 : idesc0,
                                    (ks | kk) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&mma_done[s]);
                if (++s == kRBuf) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            tc::mma_commit(accum_done);   // fires once every MMA issued above has finished
        }
    } else {
        // ---------------- generators / converters (warps 1-16) ----------------
        const int g = tid - 32;
        // C item and the converted B rows: row r (+ 128 t), 16 pixels pg
        const int r = g >> 2, pg = g & 3;
        const uint32_t off_a = tc::sw128_offset(static_cast<uint32_t>(r), static_cast<uint32_t>(2 * pg));
        const uint32_t off_b = tc::sw128_offset(static_cast<uint32_t>(r), static_cast<uint32_t>(2 * pg + 1));
        // B rows r + 128 t (t < 4) differ from row r by 16 KB in the layout
        const uint8_t* src[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int row = r + 128 * t;
            const int slot = row >> 8;
            src[t] = nullptr;
            if (row - 256 * slot < (slot ? nslot1 : nslot0)) {
                for (int i = 0; i < a.nseg; ++i) {
                    const RadSeg& sg = a.seg[i];
                    if (row >= sg.row0 && row < sg.row0 + sg.L)
                        src[t] = sg.D + static_cast<int64_t>(row - sg.row0) * sg.ldd + 16 * pg;
                }
            }
        }
        const int64_t m = a.m;
        // no pixel of this split's K steps lies past m: loads need no tail checks
        const bool full = static_cast<int64_t>(step0 + nsteps) * kRKStep <= m;
        // bytes of K steps 0 and 1
        uint4 buf[kRBuf][4];
#pragma unroll
        for (int d = 0; d < kRBuf; ++d)
#pragma unroll
            for (int t = 0; t < 4; ++t)
                buf[d][t] = d < nsteps ? load_row16(src[t], static_cast<int64_t>(step0 + d) * kRKStep, m)
                                       : make_uint4(0u, 0u, 0u, 0u);
        uint32_t ph = 0;      // parity of the current use of the stages
        bool ok = true;
        // after an abort the remaining steps only skip their work
        for (int kb = 0; kb < nsteps; kb += kRBuf) {
#pragma unroll
            for (int s = 0; s < kRBuf; ++s) {
                const int ks = kb + s;
                if (ks >= nsteps) break;
                // the stage is free once the MMAs of its previous use finished
                // (lane 0 waits for the warp, then the warp syncs)
                if (kb > 0 && ok) {
                    bool free_ok = true;
                    if (lane == 0) {
                        free_ok = tc::mbar_wait(&mma_done[s], ph ^ 1u, abort_flag, status);
                    }
                    __syncwarp();
                    ok = __shfl_sync(0xffffffffu, free_ok ? 1 : 0, 0) != 0;
                }
                const int64_t j0 = static_cast<int64_t>(step0 + ks) * kRKStep;
                uint8_t* a_stage = A + s * kRAStage;
                uint8_t* b_stage = B + s * kRBStage;
                if (ok) {
                    draw_rademacher_f16(a_stage, off_a, off_b, lane, r, pg, row0, k, j0, m, a.rk);
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (src[t] != nullptr)
                            convert_row16(b_stage, off_a + t * 16384u, off_b + t * 16384u, buf[s][t]);
                }
                // every lane's writes are ordered before the async proxy's
                // reads, then one arrival per warp
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0 && ok) tc::mbar_arrive(&ab_full[s]);
                // the bytes of K step ks + kRBuf into the registers just used
                if (ks + kRBuf < nsteps && ok) {
                    if (full) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) buf[s][t] = load_row16_full(src[t], j0 + kRBuf * kRKStep);
                    } else {
#pragma unroll
                        for (int t = 0; t < 4; ++t) buf[s][t] = load_row16(src[t], j0 + kRBuf * kRKStep, m);
                    }
                }
            }
            ph ^= 1u;
        }
        // ---------------- epilogue: partials of every used B row ----------------
        const bool done = tc::mbar_wait(accum_done, 0u, abort_flag, status) && !*abort_flag;
        tc::tc_fence_after();
        if (done) {
            const int quarter = warp & 3;
            const int cg = (warp - 1) >> 2;                 // column group 0 .. 3
            const int row = row0 + quarter * 32 + lane;
            float* part = a.part + static_cast<int64_t>(split) * kRadRows * k;
            for (int slot = 0; slot < 2; ++slot) {
                for (int c0 = 16 * cg; c0 < (slot ? nslot1 : nslot0); c0 += 64) {
                    uint32_t v[16];
                    tc::tmem_ld_x16(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + slot * kAccCols + c0, v);
                    tc::tmem_wait_ld();
                    if (row < k) {
#pragma unroll
                        for (int qq = 0; qq < 16; ++qq)
                            part[static_cast<int64_t>(slot * 256 + c0 + qq) * k + row] = __uint_as_float(v[qq]);
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

// DY of segment blockIdx.y: DY[(f0 + t) k + i] = sum_s part[s][row0 + t][i], FP64, fixed order.
__global__ void sketch_rad_reduce_kernel(const __grid_constant__ RadArgs a, int splits, int* status) {
    const RadSeg sg = a.seg[blockIdx.y];
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t total = static_cast<int64_t>(sg.L) * a.k;
    if (idx >= total) return;
    const int64_t src = static_cast<int64_t>(sg.row0) * a.k + idx;
    const int64_t stride = static_cast<int64_t>(kRadRows) * a.k;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += static_cast<double>(a.part[sp * stride + src]);
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    sg.DY[static_cast<int64_t>(sg.f0) * a.k + idx] = s;
}

// DY_g[t*k + i] = sum_s part_g[(s*n_g + t)*k + i], FP64, fixed order; blockIdx.y = clip.
__global__ void sketch_tc_reduce_kernel(const SketchArgs a, int splits, double* DY0, double* DY1, int* status) {
    const int g = blockIdx.y;
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t total = static_cast<int64_t>(a.k) * (g ? a.n[1] : a.n[0]);
    if (idx >= total) return;
    const float* part = g ? a.part[1] : a.part[0];
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += static_cast<double>(part[static_cast<int64_t>(sp) * total + idx]);
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    (g ? DY1 : DY0)[idx] = s;
}

}  // namespace

// Shared memory of a CTA in the given shape (bytes, with room to align the
// base to 1024); larger than kMaxSmem when the shape does not fit.
size_t sketch_tc_smem_bytes(int mtiles, int nclips, int n0, int n1) {
    return smem_layout(mtiles, nclips, n0, n1).total + 1024;
}

bool sketch_tc_pair_fits(int n0, int n1) {
    return n0 >= 1 && n1 >= 1 && n0 <= kMaxFrames && n1 <= kMaxFrames &&
           sketch_tc_smem_bytes(1, 2, n0, n1) <= kMaxSmem;
}

namespace {

// One launch: nclips (1 or 2) clips of <= 256 frames, each its own DY.
cdmd_status launch_sketch_tc_unit(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m, const int* n,
                                  const int64_t* ldd, bool rad, int k, uint64_t seed, double* const* DY,
                                  cudaStream_t stream) {
    const int mtiles = nclips == 1 ? 2 : 1;
    CUtensorMap tmap[2];
    for (int g = 0; g < nclips; ++g) {
        cdmd_status st = make_video_tmap(&tmap[g], D[g], m, n[g], ldd[g], kKStep, n[g]);
        if (st != CDMD_OK) return st;
    }
    if (nclips == 1) tmap[1] = tmap[0];
    const int rowblks = (k + 128 * mtiles - 1) / (128 * mtiles);
    const int64_t total_steps = (m + kKStep - 1) / kKStep;
    int64_t splits = std::max<int64_t>(1, ctx->num_sms / rowblks);
    splits = std::min<int64_t>(splits, total_steps);
    const int64_t steps_per_split = (total_steps + splits - 1) / splits;
    splits = (total_steps + steps_per_split - 1) / steps_per_split;
    size_t floats = 0;
    for (int g = 0; g < nclips; ++g) floats += static_cast<size_t>(splits) * n[g] * k;
    float* part = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL, floats * sizeof(float), reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    SketchArgs a{};
    a.part[0] = part;
    a.part[1] = nclips > 1 ? part + static_cast<size_t>(splits) * n[0] * k : nullptr;
    a.n[0] = n[0];
    a.n[1] = nclips > 1 ? n[1] : 0;
    a.nclips = nclips;
    a.mtiles = mtiles;
    a.k = k;
    a.m = m;
    a.steps_per_split = steps_per_split;
    a.total_steps = total_steps;
    a.key = seed_key(seed);
    const size_t smem = smem_layout(mtiles, nclips, a.n[0], a.n[1]).total + 1024;
    if (smem > kMaxSmem) return fail(CDMD_ERR_UNSUPPORTED, "sketch: %zu bytes of shared memory per CTA", smem);
    auto kern = rad ? sketch_tc_kernel<true> : sketch_tc_kernel<false>;
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    kern<<<dim3(rowblks, static_cast<unsigned>(splits)), kThreads, smem, stream>>>(tmap[0], tmap[1], a, ctx->d_status);
    CDMD_CHECK_LAUNCH("sketch_tc_kernel");
    const int64_t tot = static_cast<int64_t>(k) * std::max(a.n[0], a.n[1]);
    sketch_tc_reduce_kernel<<<dim3(static_cast<unsigned>((tot + 255) / 256), nclips), 256, 0, stream>>>(
        a, static_cast<int>(splits), DY[0], nclips > 1 ? DY[1] : nullptr, ctx->d_status);
    CDMD_CHECK_LAUNCH("sketch_tc_reduce_kernel");
    return CDMD_OK;
}

// Shared sketch of several clips under one Rademacher C from the uint8 frames
// (no BF16 copies); launches of up to 512 packed frames.
cdmd_status launch_sketch_rad_u8(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m, const int* n,
                                 const int64_t* ldd, int k, uint64_t seed, double* const* DY, cudaStream_t stream) {
    if (m > (static_cast<int64_t>(1) << 31) - kRKStep)
        return fail(CDMD_ERR_UNSUPPORTED, "packed sketch: m = %lld pixels (at most 2^31 - 64)", static_cast<long long>(m));
    const int rowblks = (k + 127) / 128;
    const int64_t total_steps = (m + kRKStep - 1) / kRKStep;
    int64_t splits = std::max<int64_t>(1, ctx->num_sms / rowblks);
    splits = std::min<int64_t>(splits, total_steps);
    const int64_t steps_per_split = (total_steps + splits - 1) / splits;
    splits = (total_steps + steps_per_split - 1) / steps_per_split;
    float* part = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL, static_cast<size_t>(splits) * kRadRows * k * sizeof(float),
                                   reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    const size_t smem = rad_smem_bytes() + 1024;
    if (smem > kMaxSmem) return fail(CDMD_ERR_UNSUPPORTED, "packed sketch: %zu bytes of shared memory per CTA", smem);
    // the attribute is the largest any launch of this kernel uses (the same
    // for every call, so concurrent host threads never lower it)
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(sketch_rad_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kMaxSmem)));
    RadArgs a{};
    a.part = part;
    a.k = k;
    a.m = m;
    a.steps_per_split = static_cast<int>(steps_per_split);
    a.total_steps = static_cast<int>(total_steps);
    a.rk = philox_round_keys(seed_key(seed));
    int rows = 0;     // B rows used so far in this launch (a multiple of 8)
    auto flush = [&]() -> cdmd_status {
        if (a.nseg == 0) return CDMD_OK;
        a.nslot[0] = rows >= 256 ? 256 : (rows + 15) / 16 * 16;
        a.nslot[1] = rows > 256 ? (rows - 256 + 15) / 16 * 16 : 0;
        int maxL = 0;
        for (int i = 0; i < a.nseg; ++i) maxL = std::max(maxL, a.seg[i].L);
        sketch_rad_u8_kernel<<<dim3(rowblks, static_cast<unsigned>(splits)), kRThreads, smem, stream>>>(a, ctx->d_status);
        CDMD_CHECK_LAUNCH("sketch_rad_u8_kernel");
        const int64_t tot = static_cast<int64_t>(maxL) * k;
        sketch_rad_reduce_kernel<<<dim3(static_cast<unsigned>((tot + 255) / 256), a.nseg), 256, 0, stream>>>(
            a, static_cast<int>(splits), ctx->d_status);
        CDMD_CHECK_LAUNCH("sketch_rad_reduce_kernel");
        a.nseg = 0;
        rows = 0;
        return CDMD_OK;
    };
    for (int i = 0; i < nclips; ++i) {
        for (int f = 0; f < n[i];) {
            if (a.nseg == kRadMaxSeg || rows == kRadRows) {
                st = flush();
                if (st != CDMD_OK) return st;
            }
            const int space = 256 - (rows & 255);            // rows left in the current slot
            const int L = std::min(n[i] - f, space);
            RadSeg& sg = a.seg[a.nseg];
            sg.DY = DY[i];
            sg.D = D[i] + static_cast<int64_t>(f) * ldd[i];
            sg.ldd = ldd[i];
            sg.row0 = rows;
            sg.L = L;
            sg.f0 = f;
            ++a.nseg;
            rows += (L + 7) / 8 * 8;
            f += L;
        }
    }
    return flush();
}

cdmd_status check_tc_video(const uint8_t* D, int64_t ldd) {
    if ((reinterpret_cast<uintptr_t>(D) & 15) != 0 || (ldd & 15) != 0)
        return fail(CDMD_ERR_INVALID_ARG, "BF16X2 sketch needs a 16-byte aligned video and ldd %% 16 == 0");
    return CDMD_OK;
}

}  // namespace

cdmd_status launch_sketch_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, cdmd_ctype ctype,
                             int k, uint64_t seed, double* DY, cudaStream_t stream) {
    if (ctype != CDMD_C_GAUSSIAN && ctype != CDMD_C_RADEMACHER)
        return fail(CDMD_ERR_UNSUPPORTED, "BF16X2 sketch generates GAUSSIAN or RADEMACHER C");
    cdmd_status st = check_tc_video(D, ldd);
    if (st != CDMD_OK) return st;
    // the sketch is linear in the frames: DY[t0:t1] = C D[:, t0:t1]
    for (int t0 = 0; t0 < n; t0 += kMaxFrames) {
        const int nc = std::min(kMaxFrames, n - t0);
        const uint8_t* Dc = D + static_cast<int64_t>(t0) * ldd;
        double* DYc = DY + static_cast<int64_t>(t0) * k;
        st = launch_sketch_tc_unit(ctx, 1, &Dc, m, &nc, &ldd, ctype == CDMD_C_RADEMACHER, k, seed, &DYc, stream);
        if (st != CDMD_OK) return st;
    }
    return CDMD_OK;
}

cdmd_status launch_sketch_tc_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m, const int* n,
                                    const int64_t* ldd, cdmd_ctype ctype, int k, uint64_t seed, double* const* DY,
                                    cudaStream_t stream) {
    for (int i = 0; i < nclips; ++i) {
        cdmd_status st = check_tc_video(D[i], ldd[i]);
        if (st != CDMD_OK) return st;
    }
    if (nclips == 1) return launch_sketch_tc(ctx, D[0], m, n[0], ldd[0], ctype, k, seed, DY[0], stream);
    if (ctype == CDMD_C_RADEMACHER) return launch_sketch_rad_u8(ctx, nclips, D, m, n, ldd, k, seed, DY, stream);
    // BF16 copies of every clip's frames (one HBM-bound pass each)
    const int64_t ldw = (m + 15) / 16 * 16;
    size_t elems = 0;
    for (int i = 0; i < nclips; ++i) elems += static_cast<size_t>(n[i]) * ldw;
    uint16_t* W = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SKETCH_WIDE, elems * sizeof(uint16_t), reinterpret_cast<void**>(&W));
    if (st != CDMD_OK) return st;
    std::vector<const uint16_t*> Wc(nclips);
    for (int i = 0; i < nclips; ++i) {
        const unsigned bx = static_cast<unsigned>((ldw / 16 + 255) / 256);
        widen_kernel<<<dim3(bx, static_cast<unsigned>(n[i])), 256, 0, stream>>>(D[i], m, ldd[i], W, ldw);
        CDMD_CHECK_LAUNCH("widen_kernel");
        Wc[i] = W;
        W += static_cast<size_t>(n[i]) * ldw;
    }
    // launches of up to 512 packed frames
    const int rowblks = (k + 127) / 128;
    const int64_t total_steps = (m + kKStep - 1) / kKStep;
    int64_t splits = std::max<int64_t>(1, ctx->num_sms / rowblks);
    splits = std::min<int64_t>(splits, total_steps);
    const int64_t steps_per_split = (total_steps + splits - 1) / splits;
    splits = (total_steps + steps_per_split - 1) / steps_per_split;
    float* part = nullptr;
    st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL, static_cast<size_t>(splits) * kPackRows * k * sizeof(float),
                       reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    // CTA pairs (one 2-SM MMA over two 128-row tiles of C) when the row
    // blocks pair up; single CTAs otherwise
    const bool pairs = rowblks % 2 == 0;
    const size_t smem = (pairs ? pair_smem_bytes() : pack_smem_bytes()) + 1024;
    auto packed = pairs ? sketch_tc_pair_kernel : sketch_tc_packed_kernel;
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(packed, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    PackArgs a{};
    a.part = part;
    a.k = k;
    a.m = m;
    a.steps_per_split = steps_per_split;
    a.total_steps = total_steps;
    a.key = seed_key(seed);
    int rows = 0;     // B rows used so far in this launch (a multiple of 8)
    auto flush = [&]() -> cdmd_status {
        if (a.nseg == 0) return CDMD_OK;
        a.nslot[0] = rows >= 256 ? 256 : (rows + 15) / 16 * 16;
        a.nslot[1] = rows > 256 ? (rows - 256 + 15) / 16 * 16 : 0;
        int maxL = 0;
        for (int i = 0; i < a.nseg; ++i) maxL = std::max(maxL, a.seg[i].L);
        if (pairs) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(static_cast<unsigned>(rowblks), static_cast<unsigned>(splits), 1);
            cfg.blockDim = dim3(kThreads, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CDMD_CHECK_CUDA(cudaLaunchKernelEx(&cfg, sketch_tc_pair_kernel, a, ctx->d_status));
        } else {
            packed<<<dim3(rowblks, static_cast<unsigned>(splits)), kThreads, smem, stream>>>(a, ctx->d_status);
        }
        CDMD_CHECK_LAUNCH("sketch_tc_packed_kernel");
        const int64_t tot = static_cast<int64_t>(maxL) * k;
        sketch_packed_reduce_kernel<<<dim3(static_cast<unsigned>((tot + 255) / 256), a.nseg), 256, 0, stream>>>(
            a, static_cast<int>(splits), ctx->d_status);
        CDMD_CHECK_LAUNCH("sketch_packed_reduce_kernel");
        a.nseg = 0;
        rows = 0;
        return CDMD_OK;
    };
    for (int i = 0; i < nclips; ++i) {
        for (int f = 0; f < n[i];) {
            if (a.nseg == kMaxSeg || rows == kPackRows) {
                st = flush();
                if (st != CDMD_OK) return st;
            }
            // rows left in the current slot (in the current half of it for CTA
            // pairs, where each half lives in one CTA)
            const int space = pairs ? 128 - (rows & 127) : 256 - (rows & 255);
            const int L = std::min(n[i] - f, space);
            PackSeg& sg = a.seg[a.nseg];
            sg.DY = DY[i];
            sg.row0 = rows;
            sg.L = L;
            sg.f0 = f;
            st = make_wide_tmap(&a.tmap[a.nseg], Wc[i], m, n[i], ldw, L);
            if (st != CDMD_OK) return st;
            ++a.nseg;
            rows += (L + 7) / 8 * 8;
            f += L;
        }
    }
    return flush();
}

cdmd_status launch_sketch_grouped(const SketchItem* items, int nitems, size_t smem, const ReduceChunk* chunks,
                                  const int64_t* prefix, int nchunks, int64_t total, int* status, cudaStream_t stream) {
    if (smem > kMaxSmem) return fail(CDMD_ERR_UNSUPPORTED, "grouped sketch: %zu bytes of shared memory per CTA", smem);
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
