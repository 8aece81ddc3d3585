// Pass (c) on the 5th-generation tensor cores: the background of a tile of
// 128 pixels over all frames as a small GEMM, then threshold and bit-pack.
//
//   bg_jt = | sum_s a_js lambda_s^t |,  a_js = Phi_js beta_s     (Eq. DMDTerms)
//   mask_jt = |x_jt - bg_jt| > tau                              (Eq. thres)
//
// Frames are the MMA's M dimension and pixels its N dimension: an epilogue
// thread owns one frame and reads 32 consecutive pixels of it from tensor
// memory, so its grey levels are two 16-byte shared-memory loads and its 32
// decisions are one mask word, with no ballot.
//
// With a_js = u + i v and lambda_s^t = p + i q:
//   Re = sum_s (u p - v q) = [p, -q] . [u,  v]
//   Im = sum_s (u q + v p) = [p, -q] . [v, -u]
// A (frames x K, built once per CTA) holds (p, -q) per term; B (pixels x K,
// built per unit) holds (u, v) of 128 pixels or, when Im is needed, (u, v)
// of 64 pixels in rows 0-63 and (v, -u) in rows 64-127, so one MMA chain of
// N = 128 per frame block yields Re of the whole tile, or Re in columns 0-63
// and Im in 64-127 of half of it (a unit: one tile, or half a tile).  The
// cost of an MMA here is mostly per instruction (a few hundred cycles at
// N = 64 or 128), so the widest N that tensor memory allows is used.  A pair
// is one 32-bit word of two BF16.  Both
// operands are split into BF16 hi + lo and term s takes the three words 3s,
// 3s+1, 3s+2 of K,
//   A: hi, hi, lo      B: hi, lo, hi      ->   hi.hi + hi.lo + lo.hi,
// about 2^-16 relative per term, with FP32 range (modes that grow or decay)
// and FP32 accumulation.
//
// When the selected modes are real modes and complete conjugate pairs with
// conjugate amplitudes (the table kernel decides and writes one real term per
// real mode or pair), the sum is real: only Re is formed, and MODULUS is |Re|.
//
// Tensor memory: a ring of unit stages (4 for one frame block, else 2) x
// frame blocks (frames 0-127, 128-255) x 128 columns.  B has a ring of 4
// stages (2 when its rows span two K atoms).  Per tile (persistent CTAs):
//   warp 0      TMA: a 128-pixel tile's bytes (box 128 pixels x n frames,
//               128-byte swizzle: half as many copy rows per byte as a
//               64-pixel box) and its rows of Phi (one bulk copy) into a ring
//               of stages
//   warp 1      one thread: the MMAs of every frame block of a unit, commits
//   builders    thread = pixel: a = Phi beta split into hi / lo words of B;
//               warps 2 and 3, and 11 and 19 when lane quadrant 3 of frame
//               block 1 holds no frame (n <= 224)
//   warps 4-19  epilogue in two groups (warps 4-11 even units, 12-19 odd
//               ones, so the groups' latencies overlap): warp (frame block h,
//               lane quadrant q = warp % 4) covers frames 128 h + 32 q + lane
//               and the pixels of its units
// Waits are bounded as in the sketch.
#include <algorithm>
#include <type_traits>

#include "tc_common.cuh"
#include "batch_internal.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 640;
constexpr int kPix = 64;                       // pixels of a unit with Re and Im
constexpr int kTile = 128;                     // pixels per tensor copy (one tile)
constexpr int kMaxModes = 16;                  // terms per part: 3 x 16 words <= 2 K atoms
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kATile = 128u * 128u;       // one K atom of A: 128 rows x 128 bytes
constexpr uint32_t kBAtom = 2u * kPix * 128u;  // one K atom of B: 128 rows x 128 bytes (128 pixels, or 64 and their (v, -u) rows)
constexpr uint32_t kPhiStage = kTile * kMaxModes * 8u;
constexpr int kMaxStages = 6;
constexpr int kMaxAcc = 4;
constexpr uint32_t kSmemLimit = 232448;        // opt-in shared memory per CTA
constexpr int kNumBars = 2 * kMaxStages + 4 * kMaxAcc + 1;

__host__ __device__ inline uint32_t round1k(uint32_t x) { return (x + 1023u) & ~1023u; }

// K atoms (64 BF16 = 32 words per row) holding 3 words per term
__host__ __device__ constexpr int k_atoms(int nc) { return (3 * nc + 31) / 32; }

// B stages: as many as the tensor-memory ring (up to 4) when B is one atom
__host__ __device__ constexpr int b_stages_max(int natoms) { return natoms == 1 ? 4 : 2; }

struct SubLayout {
    uint32_t b_off, x_off, x_stage, phi_off, bar_off, misc_off, total;
    int nstages;
};

// A tiles [block][atom], the B ring [stage][atom], then a ring of stages of
// frame bytes and Phi rows as deep as the shared memory allows.
__host__ __device__ inline SubLayout sub_layout(int n, int natoms, int nblk) {
    SubLayout L;
    const uint32_t a_bytes = static_cast<uint32_t>(nblk * natoms) * kATile;
    const uint32_t b_bytes = static_cast<uint32_t>(b_stages_max(natoms) * natoms) * kBAtom;
    L.b_off = a_bytes;
    L.x_off = a_bytes + b_bytes;
    L.x_stage = round1k(static_cast<uint32_t>(n) * kTile);
    const uint32_t fixed = a_bytes + b_bytes + 2048u;   // barriers, constants, alignment slack
    const int ns = static_cast<int>((kSmemLimit - fixed) / (L.x_stage + kPhiStage));
    L.nstages = ns > kMaxStages ? kMaxStages : ns;
    L.phi_off = L.x_off + static_cast<uint32_t>(L.nstages) * L.x_stage;
    L.bar_off = L.phi_off + static_cast<uint32_t>(L.nstages) * kPhiStage;
    L.misc_off = L.bar_off + kNumBars * 8;
    L.total = L.misc_off + 256;
    return L;
}

struct SubTcArgs {
    const float2* Phi;          // m x ncols complex, pixel-major, 16-byte aligned
    SubTcTable tb;              // amplitudes, lambda^t tables, real-term split
    uint32_t* mask;
    int64_t m, words_per_frame, ntiles;
    int n, ncols, nc_pad;
    float tau;
};

// BF16 hi (round to nearest) and lo (the rounded rest) of a pair, x in the
// low half of each word.
__device__ __forceinline__ void split_pair(float x, float y, uint32_t& hi, uint32_t& lo) {
    hi = tc::pack_bf16_rn(x, y);
    const float hx = __uint_as_float(hi << 16);
    const float hy = __uint_as_float(hi & 0xFFFF0000u);
    lo = tc::pack_bf16_rn(x - hx, y - hy);
}

// Byte offset of the 16-byte chunk holding words 4 ch .. 4 ch + 3 of row
// `row` in K-major 128-byte swizzled atoms of `atom_bytes` each.
__device__ __forceinline__ uint32_t chunk_offset(uint32_t row, int ch, uint32_t atom_bytes) {
    return static_cast<uint32_t>(ch >> 3) * atom_bytes + tc::sw128_offset(row, static_cast<uint32_t>(ch & 7));
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// tcgen05.wait::ld that the compiler sees as producing r, so no use of the
// loaded registers can be scheduled above it.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// The same, making the registers of a second load (im) depend on it too.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&r)[32], uint32_t (&s)[32]) {
    tmem_wait_ld32(r);
    asm volatile(""
                 : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]), "+r"(s[7]),
                   "+r"(s[8]), "+r"(s[9]), "+r"(s[10]), "+r"(s[11]), "+r"(s[12]), "+r"(s[13]), "+r"(s[14]),
                   "+r"(s[15]), "+r"(s[16]), "+r"(s[17]), "+r"(s[18]), "+r"(s[19]), "+r"(s[20]), "+r"(s[21]),
                   "+r"(s[22]), "+r"(s[23]), "+r"(s[24]), "+r"(s[25]), "+r"(s[26]), "+r"(s[27]), "+r"(s[28]),
                   "+r"(s[29]), "+r"(s[30]), "+r"(s[31])
                 :
                 : "memory");
}

// 32 decisions (bit i = pixel i) from 32 grey levels (two 16-byte rows in
// pixel order) and the accumulators.  V: 0 bg = Re (REAL), 1 bg = |Re|
// (MODULUS of a real sum), 2 bg = |Re + i Im|.
template <int V>
__device__ __forceinline__ uint32_t decide32(const uint4& x0, const uint4& x1, const uint32_t (&re)[32],
                                             const uint32_t (&im)[32], float tau) {
    uint32_t bits = 0u;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const uint4& xw = i < 16 ? x0 : x1;
        const int wq = (i >> 2) & 3;
        const uint32_t word = wq == 0 ? xw.x : wq == 1 ? xw.y : wq == 2 ? xw.z : xw.w;
        // grey level as a float: 2^23 + x, exact, minus 2^23
        const float x = __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7650u + static_cast<uint32_t>(i & 3))) -
                        8388608.0f;
        const float r = __uint_as_float(re[i]);
        float bg;
        if (V == 0) {
            bg = r;
        } else if (V == 1) {
            bg = fabsf(r);
        } else {
            const float q = __uint_as_float(im[i]);
            asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(bg) : "f"(fmaf(r, r, q * q)));
        }
        if (fabsf(x - bg) > tau) bits |= 1u << i;
    }
    return bits;
}

// The 128-pixel tiles tile_first + i * tile_stride (i < my_tiles) of one
// clip, each one tensor copy and one or two units; NC
// (4, 8, 10 or 16) >= ncols fixes the positions of each term's words in B.
template <bool kReal, int NC>
__device__ __forceinline__ void subtract_tc_body(const CUtensorMap* tmap, const SubTcArgs& a, int64_t tile_first,
                                                 int64_t tile_stride, int64_t my_tiles, int* status, uint8_t* smem) {
    constexpr int natoms = k_atoms(NC);
    constexpr int kChunks = (3 * NC + 3) / 4;       // 16-byte chunks of a B row holding terms
    const int n = a.n;
    const int ncols = a.ncols;
    const int nblk = (n + 127) >> 7;
    const SubLayout L = sub_layout(n, natoms, nblk);
    const int S = L.nstages;
    // the terms: one per real mode or conjugate pair when the sum is real,
    // else one per selected column
    const bool real_only = a.tb.hdr[1] != 0;
    int cnt = real_only ? a.tb.hdr[0] : ncols;
    cnt = cnt < 0 ? 0 : (cnt > ncols ? ncols : cnt);
    const int parts = (!kReal && !real_only) ? 2 : 1;
    // a unit of work is one MMA of N = 128 per frame block: the whole
    // 128-pixel tile when only Re is formed, else half of it (Re and Im)
    const int upt = parts;                                      // units per tile
    const int upx = kTile / upt;                                // pixels per unit
    const int64_t my_units = my_tiles * upt;
    const int nk = cnt > 0 ? (3 * cnt + 7) / 8 : 1;             // K16 steps: 8 words each
    const int acc_cols = nblk * 128;                            // tensor-memory columns of a unit
    const int nacc = acc_cols <= 128 ? kMaxAcc : 2;
    constexpr int nb = b_stages_max(natoms);

    uint8_t* A = smem;
    uint8_t* B = smem + L.b_off;
    uint8_t* X = smem + L.x_off;
    uint8_t* PhiS = smem + L.phi_off;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* x_full = bars;                      // [S] bytes and Phi rows landed
    uint64_t* x_free = bars + kMaxStages;         // [S] read by the builders and the epilogue
    uint64_t* b_full = bars + 2 * kMaxStages;     // [nb] B built
    uint64_t* b_free = b_full + kMaxAcc;          // [nb] MMAs done with B
    uint64_t* acc_full = b_free + kMaxAcc;        // [nacc] accumulators ready
    uint64_t* acc_free = acc_full + kMaxAcc;      // [nacc] accumulators read
    uint64_t* drain = acc_free + kMaxAcc;         // every MMA finished
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.misc_off + 8);
    float2* amps = reinterpret_cast<float2*>(smem + L.misc_off + 16);        // [16]
    int* cols = reinterpret_cast<int*>(smem + L.misc_off + 16 + 8 * kMaxModes);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const float tau = a.tau;

    // epilogue warps whose frames exist (the same count in both groups);
    // builders on the spare scheduler
    auto epi_active = [&](int w) {
        const int h = ((w - 4) >> 2) & 1;
        return w >= 4 && h < nblk && 128 * h + 32 * (w & 3) < n;
    };
    int n_epi = 0;
    for (int w = 4; w < kThreads / 32; ++w) n_epi += epi_active(w) ? 1 : 0;
    const int n_epi_g = n_epi / 2;
    // builders: warps 2 and 3, and 11 and 19 when lane quadrant 3 of frame
    // block 1 holds no frame (their scheduler has the least epilogue work)
    const bool spare = !epi_active(11) && !epi_active(19);
    const int nbw = spare ? 4 : 2;
    const int bidx = warp == 2 ? 0 : warp == 3 ? 1 : (spare && warp == 11) ? 2 : (spare && warp == 19) ? 3 : -1;
    const bool is_builder = bidx >= 0;
    // a stage is read by the builders and by the epilogue groups that take
    // its units (both when a tile is two units)
    const int x_consumers = nbw + (upt == 2 ? n_epi : n_epi_g);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&x_full[s], 1);
            tc::mbar_init(&x_free[s], x_consumers);
        }
        for (int i = 0; i < kMaxAcc; ++i) {
            tc::mbar_init(&b_full[i], nbw);
            tc::mbar_init(&b_free[i], 1);
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_free[i], n_epi_g);
        }
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (tid < kMaxModes) {
        const bool on = tid < cnt;
        amps[tid] = on ? (real_only ? a.tb.term_amp[tid] : a.tb.amp[tid]) : make_float2(0.f, 0.f);
        cols[tid] = on ? (real_only ? a.tb.term_col[tid] : tid) : 0;
    }
    // A: row t of frame block h; words 3s, 3s+1, 3s+2 hold term s's (p, -q)
    // as hi, hi, lo.  Frames past n and words past 3 cnt are zero.
    {
        const float2* lt = real_only ? a.tb.term_lam_t : a.tb.lam_t;
        constexpr int wrow = natoms * 32;
        const int total = nblk * 128 * wrow;
        for (int idx = tid; idx < total; idx += kThreads) {
            const int w = idx % wrow;
            const int rest = idx / wrow;
            const int row = rest & 127;
            const int h = rest >> 7;
            const int t = 128 * h + row;
            const int s = w / 3, b = w - 3 * s;
            uint32_t val = 0u;
            if (t < n && s < cnt) {
                const float2 l = lt[static_cast<int64_t>(t) * a.nc_pad + s];
                uint32_t hi, lo;
                split_pair(l.x, -l.y, hi, lo);
                val = b < 2 ? hi : lo;
            }
            *reinterpret_cast<uint32_t*>(A + static_cast<uint32_t>(h * natoms) * kATile +
                                         chunk_offset(static_cast<uint32_t>(row), w >> 2, kATile) + (w & 3) * 4u) = val;
        }
    }
    // B: chunks past the terms' words are never written and must read as zero
    for (uint32_t off = tid * 16u; off < static_cast<uint32_t>(nb * natoms) * kBAtom;
         off += kThreads * 16u)
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
    const uint32_t x_bytes = static_cast<uint32_t>(n) * kTile;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            // ring position and phase kept as counters (no division per tile)
            int s = 0;
            uint32_t ph = 0u;
            for (int64_t li = 0; li < my_tiles; ++li) {
                if (li >= S && !tc::mbar_wait(&x_free[s], ph ^ 1u, abort_flag, status)) break;
                const int64_t tile = tile_first + li * tile_stride;
                const int64_t p0 = tile * kTile;
                const int64_t npx = a.m - p0 < kTile ? a.m - p0 : kTile;
                const uint32_t bulk = static_cast<uint32_t>(npx * ncols * 8) & ~15u;
                tc::mbar_arrive_expect_tx(&x_full[s], x_bytes + bulk);
                tc::tma_load_2d(X + s * L.x_stage, tmap, static_cast<int>(p0), 0, &x_full[s]);
                if (bulk > 0u) tc::bulk_load(PhiS + s * kPhiStage, a.Phi + p0 * ncols, bulk, &x_full[s]);
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            // drain: the last copies of each stage must have landed before exit
            for (s = 0; s < S; ++s) {
                const int64_t uses = (my_tiles - s + S - 1) / S;
                if (uses >= 1) tc::mbar_wait(&x_full[s], static_cast<uint32_t>(uses - 1) & 1u, abort_flag, status);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // N = 128: 128 pixels (Re) or 64 pixels' Re and Im (rows of B, B')
            const uint32_t idesc = tc::idesc_bf16_f32(128, 128);
            const uint32_t a_base = tc::smem_u32(A), b_base = tc::smem_u32(B);
            int sa = 0, sb = 0;
            uint32_t pa = 0u, pb = 0u;
            for (int64_t u = 0; u < my_units; ++u) {
                if (!tc::mbar_wait(&b_full[sb], pb, abort_flag, status)) break;
                if (u >= nacc && !tc::mbar_wait(&acc_free[sa], pa ^ 1u, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint64_t bd0 = tc::desc_sw128(b_base + static_cast<uint32_t>(sb * natoms) * kBAtom);
                for (int h = 0; h < nblk; ++h) {
                    const uint32_t acc = tmem_base + static_cast<uint32_t>(sa * acc_cols + h * 128);
                    const uint64_t ad0 = tc::desc_sw128(a_base + static_cast<uint32_t>(h * natoms) * kATile);
#pragma unroll 1
                    for (int kk = 0; kk < nk; ++kk) {
                        // start-address field: 16-byte units; K16 step = 32 bytes
                        // within an atom, whole atoms beyond
                        const uint64_t ka = static_cast<uint64_t>((kk >> 2) * (kATile >> 4) + (kk & 3) * 2);
                        const uint64_t kb = static_cast<uint64_t>((kk >> 2) * (kBAtom >> 4) + (kk & 3) * 2);
                        tc::mma_bf16(acc, ad0 + ka, bd0 + kb, idesc, kk ? 1u : 0u);
                    }
                }
                tc::mma_commit(&b_free[sb]);
                tc::mma_commit(&acc_full[sa]);
                if (++sa == nacc) {
                    sa = 0;
                    pa ^= 1u;
                }
                if (++sb == nb) {
                    sb = 0;
                    pb ^= 1u;
                }
            }
            tc::mma_commit(drain);
        }
    } else if (is_builder) {
        // ---------------- B builders: a = Phi beta, thread = pixel ----------------
        int s = 0, sb = 0;
        uint32_t px = 0u, pb = 0u;
        for (int64_t u = 0; u < my_units; ++u) {
            const int64_t i2 = upt == 2 ? (u >> 1) : u;                   // the 128-pixel tile
            const int sub = upt == 2 ? static_cast<int>(u & 1) : 0;
            if (!tc::mbar_wait(&x_full[s], px, abort_flag, status)) break;
            if (u >= nb && !tc::mbar_wait(&b_free[sb], pb ^ 1u, abort_flag, status)) break;
            const int64_t p0 = (tile_first + i2 * tile_stride) * kTile;   // first pixel of the tile
            const int64_t ntp = a.m - p0 < kTile ? a.m - p0 : kTile;      // its pixels below m
            const int bulk = static_cast<int>(ntp * ncols * 8) & ~15;     // bytes the bulk copy brought
            uint8_t* brow = B + static_cast<uint32_t>(sb * natoms) * kBAtom;
            // uniform: every entry of the tile came with the bulk copy
            const bool full = ntp == kTile && bulk == kTile * ncols * 8;
            for (int jj = bidx * 32 + lane; jj < upx; jj += nbw * 32) {
                const int ii = upx * sub + jj;                            // this thread's pixel in the tile
                const float2* ps = reinterpret_cast<const float2*>(PhiS + s * kPhiStage) + ii * ncols;
                // every load of the row (columns, Phi entries, amplitudes)
                // ahead of its stores, so none waits behind a store it might alias
                int cl[NC];
#pragma unroll
                for (int e = 0; e < NC; ++e) cl[e] = cols[e];
                float2 ph[NC], am[NC];
                if (full) {
#pragma unroll
                    for (int e = 0; e < NC; ++e) ph[e] = ps[cl[e]];
                } else {
#pragma unroll
                    for (int e = 0; e < NC; ++e) {
                        ph[e] = make_float2(0.f, 0.f);
                        if (ii < ntp) {
                            // the bulk copy covers whole 16-byte units; a last odd
                            // 8 bytes come from global memory
                            const int idx = ii * ncols + cl[e];
                            ph[e] = idx * 8 < bulk ? ps[cl[e]] : a.Phi[p0 * ncols + idx];
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < NC; ++e) am[e] = amps[e];
                // words 3e .. 3e+2 of term e in row jj (u, v) and, for Im, row
                // 64 + jj (v, -u: the halves swapped, the new high half
                // negated); a 16-byte chunk is stored as soon as its four words
                // are known (words past 3 NC are zero)
                uint32_t wv[4 * kChunks];
#pragma unroll
                for (int w = 3 * NC; w < 4 * kChunks; ++w) wv[w] = 0u;
#pragma unroll
                for (int e = 0; e < NC; ++e) {
                    uint32_t hi, lo;
                    split_pair(ph[e].x * am[e].x - ph[e].y * am[e].y, ph[e].x * am[e].y + ph[e].y * am[e].x, hi,
                               lo);
                    wv[3 * e] = hi;
                    wv[3 * e + 1] = lo;
                    wv[3 * e + 2] = hi;
#pragma unroll
                    for (int ch = 0; ch < kChunks; ++ch) {
                        const int last = 4 * ch + 3 < 3 * NC ? 4 * ch + 3 : 3 * NC - 1;   // last term word
                        if (last / 3 == e) {
                            const uint32_t off = chunk_offset(static_cast<uint32_t>(jj), ch, kBAtom);
                            *reinterpret_cast<uint4*>(brow + off) =
                                make_uint4(wv[4 * ch], wv[4 * ch + 1], wv[4 * ch + 2], wv[4 * ch + 3]);
                            if (parts == 2) {
                                uint32_t r4[4];
#pragma unroll
                                for (int k = 0; k < 4; ++k)
                                    r4[k] = 4 * ch + k < 3 * NC
                                                ? (__byte_perm(wv[4 * ch + k], 0u, 0x1032u) ^ 0x80000000u)
                                                : 0u;
                                // row 64 + jj: eight 8-row groups further, same swizzle phase
                                *reinterpret_cast<uint4*>(brow + off + 8u * 1024u) =
                                    make_uint4(r4[0], r4[1], r4[2], r4[3]);
                            }
                        }
                    }
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&b_full[sb]);
                if (sub == upt - 1) tc::mbar_arrive(&x_free[s]);   // the tile's Phi rows read
            }
            if (++sb == nb) {
                sb = 0;
                pb ^= 1u;
            }
            if (sub == upt - 1 && ++s == S) {
                s = 0;
                px ^= 1u;
            }
        }
    } else if (epi_active(warp)) {
        // ---------------- epilogue ----------------
        // group g (warps 4-11, 12-19) takes the units u = g, g + 2, ..., so
        // one group's hand-off and tensor-memory latencies overlap the other
        // group's arithmetic; warp (h, q) of a group covers frames
        // 128 h + 32 q + lane and all pixels of its units
        const int q = warp & 3;
        const int h = ((warp - 4) >> 2) & 1;
        const int g = (warp - 4) >> 3;
        const int t = 128 * h + 32 * q + lane;
        const bool tv = t < n;
        const int variant = parts == 2 ? 2 : (kReal ? 0 : 1);
        const int xstep = upt == 2 ? 1 : 2;           // tiles between this group's units
        // one loop per background form, so no form's branch sits in another's
        // unrolled body
        auto run = [&](auto vtag) {
            constexpr int V = decltype(vtag)::value;
            int s = upt == 2 ? 0 : g, sa = g;
            uint32_t px = 0u, pa = 0u;
            for (int64_t u = g; u < my_units; u += 2) {
                const int64_t i2 = upt == 2 ? (u >> 1) : u;       // the 128-pixel tile
                const int sub = upt == 2 ? g : 0;
                if (!tc::mbar_wait(&x_full[s], px, abort_flag, status)) break;
                if (!tc::mbar_wait(&acc_full[sa], pa, abort_flag, status)) break;
                tc::tc_fence_after();
                const uint8_t* row = X + s * L.x_stage + t * kTile;
                const uint32_t sw = static_cast<uint32_t>(t) & 7u;
                const uint32_t taddr = tmem_base + (static_cast<uint32_t>(32 * q) << 16) +
                                       static_cast<uint32_t>(sa * acc_cols + h * 128);
                constexpr int kWords = V == 2 ? 2 : 4;            // 32-pixel words of a unit
                uint32_t word[kWords];
#pragma unroll
                for (int c = 0; c < kWords; ++c) {
                    uint32_t re[32], im[32];
                    tmem_ld_x32(taddr + 32u * c, re);
                    if (V == 2) tmem_ld_x32(taddr + 64u + 32u * c, im);
                    // frame t's bytes of pixels upx sub + 32 c .. + 31: 16-byte
                    // chunks 4 sub + 2 c and the next of its 128-byte row,
                    // 128-byte swizzle (chunk ^ (t & 7))
                    uint4 x0 = make_uint4(0u, 0u, 0u, 0u), x1 = x0;
                    if (tv) {
                        const uint32_t ch = 4u * sub + 2u * c;
                        x0 = *reinterpret_cast<const uint4*>(row + ((ch ^ sw) << 4));
                        x1 = *reinterpret_cast<const uint4*>(row + (((ch + 1u) ^ sw) << 4));
                    }
                    if (V == 2) tmem_wait_ld32(re, im);
                    else tmem_wait_ld32(re);
                    word[c] = decide32<V>(x0, x1, re, V == 2 ? im : re, tau);
                }
                // this warp is done with the accumulators and the bytes
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(&acc_free[sa]);
                    tc::mbar_arrive(&x_free[s]);
                }
                if ((sa += 2) >= nacc) {
                    sa -= nacc;
                    pa ^= 1u;
                }
                if ((s += xstep) >= S) {
                    s -= S;
                    px ^= 1u;
                }
                // first pixel of the unit
                const int64_t pc = (tile_first + i2 * tile_stride) * kTile + upx * sub;
#pragma unroll
                for (int c = 0; c < kWords; ++c) {
                    const int64_t wi = (pc >> 5) + c;
                    if (tv && wi < a.words_per_frame) {
                        const int64_t left = a.m - (pc + 32 * c);        // pixels of this word below m
                        uint32_t w = word[c];
                        if (left < 32) w &= left > 0 ? (1u << left) - 1u : 0u;
                        a.mask[static_cast<int64_t>(t) * a.words_per_frame + wi] = w;
                    }
                }
            }
        };
        if (variant == 2) run(std::integral_constant<int, 2>{});
        else if (variant == 1) run(std::integral_constant<int, 1>{});
        else run(std::integral_constant<int, 0>{});
    }
    // teardown: every MMA has finished before tensor memory is released
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0) {
        volatile int no_abort = 0;
        tc::mbar_wait(drain, 0u, &no_abort, status);
    }
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

template <bool kReal, int NC>
__global__ void __launch_bounds__(kThreads, 1)
subtract_tc_kernel(const __grid_constant__ CUtensorMap tmap, const SubTcArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    int64_t my_tiles = 0;
    if (static_cast<int64_t>(blockIdx.x) < a.ntiles)
        my_tiles = (a.ntiles - 1 - static_cast<int64_t>(blockIdx.x)) / gridDim.x + 1;
    subtract_tc_body<kReal, NC>(&tmap, a, blockIdx.x, gridDim.x, my_tiles, status, smem);
}

// Grouped: CTA b runs item items[b], consecutive tiles of one clip; the
// clip's tensor map lives in global memory.
template <bool kReal, int NC>
__global__ void __launch_bounds__(kThreads, 1)
subtract_tc_grouped_kernel(const SubTcClip* __restrict__ clips, const SubtractItem* __restrict__ items, float tau,
                           int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const SubtractItem it = items[blockIdx.x];
    const SubTcClip c = clips[it.clip];
    SubTcArgs a;
    a.Phi = c.Phi;
    a.tb = c.tb;
    a.mask = c.mask;
    a.m = c.m;
    a.words_per_frame = (c.m + 31) / 32;
    a.ntiles = (c.m + kTile - 1) / kTile;
    a.n = c.n;
    a.ncols = c.ncols;
    a.nc_pad = c.nc_pad;
    a.tau = tau;
    subtract_tc_body<kReal, NC>(c.tmap, a, it.tile0, 1, it.ntiles, status, smem);
}

template <typename K>
cdmd_status set_smem(K kern) {
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemLimit)));
    return CDMD_OK;
}

// The term-count instantiation covering ncols columns.
__host__ inline int nc_class(int ncols) { return ncols <= 4 ? 4 : ncols <= 8 ? 8 : ncols <= 10 ? 10 : 16; }

template <int NC>
cdmd_status launch_plain(const CUtensorMap& tmap, const SubTcArgs& a, cdmd_bgmode mode, unsigned grid, int* status,
                         cudaStream_t stream) {
    if (mode == CDMD_BG_REAL) {
        cdmd_status st = set_smem(subtract_tc_kernel<true, NC>);
        if (st != CDMD_OK) return st;
        subtract_tc_kernel<true, NC><<<grid, kThreads, kSmemLimit, stream>>>(tmap, a, status);
    } else {
        cdmd_status st = set_smem(subtract_tc_kernel<false, NC>);
        if (st != CDMD_OK) return st;
        subtract_tc_kernel<false, NC><<<grid, kThreads, kSmemLimit, stream>>>(tmap, a, status);
    }
    CDMD_CHECK_LAUNCH("subtract_tc_kernel");
    return CDMD_OK;
}

template <int NC>
cdmd_status launch_grouped(const SubTcClip* clips, const SubtractItem* items, int nitems, cdmd_bgmode mode,
                           float tau, int* status, cudaStream_t stream) {
    if (mode == CDMD_BG_REAL) {
        cdmd_status st = set_smem(subtract_tc_grouped_kernel<true, NC>);
        if (st != CDMD_OK) return st;
        subtract_tc_grouped_kernel<true, NC><<<static_cast<unsigned>(nitems), kThreads, kSmemLimit, stream>>>(
            clips, items, tau, status);
    } else {
        cdmd_status st = set_smem(subtract_tc_grouped_kernel<false, NC>);
        if (st != CDMD_OK) return st;
        subtract_tc_grouped_kernel<false, NC><<<static_cast<unsigned>(nitems), kThreads, kSmemLimit, stream>>>(
            clips, items, tau, status);
    }
    CDMD_CHECK_LAUNCH("subtract_tc_grouped_kernel");
    return CDMD_OK;
}

}  // namespace

bool subtract_tc_supported(int n, int ncols, cdmd_bgmode mode, const uint8_t* D, int64_t ldd, int64_t m,
                           const float* Phi, const float* bg) {
    return bg == nullptr && (mode == CDMD_BG_MODULUS || mode == CDMD_BG_REAL) && n >= 32 && n <= 1024 &&
           ncols >= 1 && ncols <= kMaxModes && (reinterpret_cast<uintptr_t>(D) % 16 == 0) && (ldd % 16 == 0) &&
           (reinterpret_cast<uintptr_t>(Phi) % 16 == 0) && m <= 0x7fffffffLL - kTile;
}

size_t subtract_tc_smem(int) { return kSmemLimit; }

int subtract_tc_tile_pixels() { return kTile; }

cdmd_status make_subtract_tc_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd) {
    return make_video_tmap(map, D, m, n, ldd, kTile, n, 128);
}

cdmd_status launch_subtract_tc_grouped(const SubTcClip* clips, const SubtractItem* items, int nitems, int max_ncols,
                                       cdmd_bgmode mode, float tau, int* status, cudaStream_t stream) {
    switch (nc_class(max_ncols)) {
        case 4: return launch_grouped<4>(clips, items, nitems, mode, tau, status, stream);
        case 8: return launch_grouped<8>(clips, items, nitems, mode, tau, status, stream);
        case 10: return launch_grouped<10>(clips, items, nitems, mode, tau, status, stream);
        default: return launch_grouped<16>(clips, items, nitems, mode, tau, status, stream);
    }
}

cdmd_status launch_subtract_tc(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd, const float* Phi,
                               int ncols, const SubTcTable& tb, int nc_pad, float tau, cdmd_bgmode mode,
                               uint32_t* mask, cudaStream_t stream) {
    // frames in chunks of at most 256 (two 128-row frame blocks, the tensor
    // copy's box height); frames are independent here, so chunk q is the clip
    // of frames t0 .. t0+cnt-1 with its rows of the lambda^t tables and mask
    const int nch = (n + 255) / 256;
    const int per = (n + nch - 1) / nch;
    const int64_t wpf = (m + 31) / 32;
    for (int q = 0; q < nch; ++q) {
        const int t0 = q * per;
        const int cnt = std::min(per, n - t0);
        CUtensorMap tmap;
        cdmd_status st = make_video_tmap(&tmap, D + static_cast<int64_t>(t0) * ldd, m, cnt, ldd, kTile, cnt, 128);
        if (st != CDMD_OK) return st;
        SubTcArgs a{};
        a.Phi = reinterpret_cast<const float2*>(Phi);
        a.tb = tb;
        a.tb.lam_t = tb.lam_t + static_cast<int64_t>(t0) * nc_pad;
        a.tb.term_lam_t = tb.term_lam_t + static_cast<int64_t>(t0) * nc_pad;
        a.mask = mask + static_cast<int64_t>(t0) * wpf;
        a.m = m;
        a.words_per_frame = wpf;
        a.ntiles = (m + kTile - 1) / kTile;
        a.n = cnt;
        a.ncols = ncols;
        a.nc_pad = nc_pad;
        a.tau = tau;
        const unsigned grid = static_cast<unsigned>(std::min<int64_t>(a.ntiles, ctx->num_sms));
        switch (nc_class(ncols)) {
            case 4: st = launch_plain<4>(tmap, a, mode, grid, ctx->d_status, stream); break;
            case 8: st = launch_plain<8>(tmap, a, mode, grid, ctx->d_status, stream); break;
            case 10: st = launch_plain<10>(tmap, a, mode, grid, ctx->d_status, stream); break;
            default: st = launch_plain<16>(tmap, a, mode, grid, ctx->d_status, stream); break;
        }
        if (st != CDMD_OK) return st;
    }
    return CDMD_OK;
}

}  // namespace cdmd
