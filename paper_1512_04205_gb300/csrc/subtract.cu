// Pass (c): background reconstruction from the selected modes, foreground
// threshold and bit-packed mask, fused in one pass over the video.
//
//   bg_jt = | sum_c Phi_jc beta_{s_c} lambda_{s_c}^t |   (Eq. DMDTerms, MODULUS)
//   mask_jt = |x_jt - bg_jt| > tau                       (Eq. thres, strict)
//
// subtract_table_kernel (one block: lane = selected column, eight warps =
// eight blocks of frames) forms lambda^t for t < n in FP64, each warp from
// lambda^t0 by binary powering and then by repeated multiplication, and the
// amplitudes.  It also classifies the selected modes:
// the video is real, so the modes of a real A~ come as real eigenvalues and
// conjugate pairs with conjugate modes and (least-squares) amplitudes, and a
// pair contributes phi b lambda^t + conj(phi b lambda^t) = 2 Re(phi b lambda^t).
// When every selected complex mode has its partner selected, the sum is real
// and the main kernel accumulates one real term per real mode or pair (two
// FMAs per term instead of four per mode); otherwise it sums every mode in
// complex arithmetic.  Per pixel, the main kernel keeps the products
// a_c = Phi_jc beta_c in registers and walks the frames: lane l of a warp
// owns pixels base + l + 32e (e < PX), so the ballot of sub-position e is
// exactly mask word base/32 + e of frame t.
#include "cdmd_internal.cuh"
#include "tc_common.cuh"
#include "batch_internal.cuh"

namespace cdmd {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxCols = 32;
constexpr int kTableThreads = 256;     // table kernel: 8 warps, one block of frames each

// Table layout (one allocation):
//   hdr[4] int32            nterms, real_only
//   term_col[32] int32      column of Phi for each real term
//   amp[32] float2          beta per column (complex path)
//   term_amp[32] float2     scale * beta per real term (2 for a pair, 1 for a real mode)
//   table[n][nc_pad] float2 lambda^t per column (complex path)
//   ttable[n][nc_pad] float2 lambda^t per real term
struct Table {
    int* hdr;
    int* term_col;
    float2* amp;
    float2* term_amp;
    float2* table;
    float2* ttable;
};

__host__ __device__ inline size_t table_bytes(int n, int nc_pad) {
    return 16 + 4 * kMaxCols + 2 * 8 * kMaxCols + 2 * static_cast<size_t>(n) * nc_pad * sizeof(float2);
}

__host__ __device__ inline Table table_views(void* base, int n, int nc_pad) {
    char* p = static_cast<char*>(base);
    Table t;
    t.hdr = reinterpret_cast<int*>(p);
    t.term_col = reinterpret_cast<int*>(p + 16);
    t.amp = reinterpret_cast<float2*>(p + 16 + 4 * kMaxCols);
    t.term_amp = t.amp + kMaxCols;
    t.table = t.term_amp + kMaxCols;
    t.ttable = t.table + static_cast<size_t>(n) * nc_pad;
    return t;
}

__device__ __forceinline__ void build_table(const int32_t* __restrict__ cols, int ncols, int nc_pad,
                                            const double* __restrict__ beta, const double* __restrict__ lambda, int r,
                                            int n, const Table& tb) {
    // lane c = selected column; warp w = block w of the frames (every warp
    // classifies the columns the same way, warp 0 writes the per-column data)
    const int c = threadIdx.x & 31;
    const int wb = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    int s = -1;
    if (c < ncols) s = cols ? cols[c] : c;
    const bool ok = (s >= 0 && s < r);
    const double lr = ok ? lambda[2 * s] : 0.0;
    const double li = ok ? lambda[2 * s + 1] : 0.0;
    const double br = ok ? beta[2 * s] : 0.0;
    const double bi = ok ? beta[2 * s + 1] : 0.0;
    // classify: real, lead of a pair (Im > 0), follower (Im < 0), or lone
    const double mag = hypot(lr, li);
    const bool is_real = ok && fabs(li) <= 1e-12 * fmax(mag, 1e-300);
    const double tol = 1e-9 * fmax(1.0, mag);
    int partner = -1;
    for (int d = 0; d < 32; ++d) {
        const double dr = __shfl_sync(0xffffffffu, lr, d);
        const double di = __shfl_sync(0xffffffffu, li, d);
        const bool dok = __shfl_sync(0xffffffffu, ok, d);
        const bool dreal = __shfl_sync(0xffffffffu, is_real, d);
        if (partner < 0 && ok && !is_real && dok && !dreal && d != c && (di > 0.0) != (li > 0.0) &&
            hypot(dr - lr, di + li) <= tol)
            partner = d;
    }
    // a pair counts only when each side names the other and the amplitudes
    // are conjugate to working precision
    const int back = __shfl_sync(0xffffffffu, partner, partner < 0 ? c : partner);
    const double pbr = __shfl_sync(0xffffffffu, br, partner < 0 ? c : partner);
    const double pbi = __shfl_sync(0xffffffffu, bi, partner < 0 ? c : partner);
    const bool paired = partner >= 0 && back == c && hypot(pbr - br, pbi + bi) <= 1e-6 * fmax(hypot(br, bi), 1e-300);
    const bool lead = paired && li > 0.0;
    const bool real_ok = is_real && fabs(bi) <= 1e-6 * fmax(fabs(br), 1e-300);
    const bool term = real_ok || lead;
    const bool lone = ok && !(real_ok || paired);
    const unsigned tmask = __ballot_sync(0xffffffffu, term);
    const bool real_only = __ballot_sync(0xffffffffu, lone) == 0u;
    const int u = __popc(tmask & ((1u << c) - 1u));
    if (c == 0 && wb == 0) {
        tb.hdr[0] = __popc(tmask);
        tb.hdr[1] = real_only ? 1 : 0;
    }
    if (c >= nc_pad) return;
    const double scale = lead ? 2.0 : 1.0;
    const int nt = __popc(tmask);
    if (wb == 0) {
        tb.amp[c] = ok ? make_float2(static_cast<float>(br), static_cast<float>(bi)) : make_float2(0.f, 0.f);
        if (term) {
            tb.term_col[u] = c;
            tb.term_amp[u] = make_float2(static_cast<float>(scale * br), static_cast<float>(scale * bi));
        }
        // unused real-term slots: zero amplitude, zero powers
        if (c >= nt) {
            tb.term_col[c] = 0;
            tb.term_amp[c] = make_float2(0.f, 0.f);
        }
    }
    // frames t0 .. t1-1 of this warp: lambda^t0 by binary powering, then
    // repeated multiplication
    const int per = (n + nwb - 1) / nwb;
    const int t0 = wb * per;
    const int t1 = t0 + per < n ? t0 + per : n;
    double pr = 1.0, pi = 0.0;
    {
        double xr = lr, xi = li;
        for (int e = t0; e > 0; e >>= 1) {
            if (e & 1) {
                const double nr = pr * xr - pi * xi;
                pi = pr * xi + pi * xr;
                pr = nr;
            }
            const double sr = xr * xr - xi * xi;
            xi = 2.0 * xr * xi;
            xr = sr;
        }
    }
    for (int t = t0; t < t1; ++t) {
        const float2 v = ok ? make_float2(static_cast<float>(pr), static_cast<float>(pi)) : make_float2(0.f, 0.f);
        tb.table[static_cast<int64_t>(t) * nc_pad + c] = v;
        if (term) tb.ttable[static_cast<int64_t>(t) * nc_pad + u] = v;
        if (c >= nt) tb.ttable[static_cast<int64_t>(t) * nc_pad + c] = make_float2(0.f, 0.f);
        const double nr = pr * lr - pi * li;
        const double ni = pr * li + pi * lr;
        pr = nr;
        pi = ni;
    }
}

__global__ void __launch_bounds__(kTableThreads)
subtract_table_kernel(const int32_t* __restrict__ cols, int ncols, int nc_pad, const double* __restrict__ beta,
                      const double* __restrict__ lambda, int r, int n, Table tb) {
    build_table(cols, ncols, nc_pad, beta, lambda, r, n, tb);
}

// Grouped: one block per clip, tables with the common column stride nc.
__global__ void __launch_bounds__(kTableThreads)
subtract_table_grouped_kernel(const SubtractClip* __restrict__ clips, int nc) {
    const SubtractClip c = clips[blockIdx.x];
    build_table(c.cols, c.ncols, nc, c.beta, c.lambda, c.r, c.n, table_views(c.table, c.n, nc));
}

// One pixel tile for every frame.  REAL: accumulate real terms only (the
// sum is real); otherwise complex arithmetic over every selected column.
template <int NC, int PX, int MODE, bool REAL, int LSTRIDE>
__device__ __forceinline__ void subtract_tile(const uint8_t* __restrict__ D, int64_t m, int n, int64_t ldd,
                                              const float2* __restrict__ Phi, int ncols, const Table& tb,
                                              int nterms, const float2* Ls, float tau, uint32_t* __restrict__ mask,
                                              int64_t words_per_frame, float* __restrict__ bg_out, int64_t tile,
                                              int lane) {
    constexpr int FB = 8;   // frames whose bytes are loaded ahead of the arithmetic
    const int64_t base = tile * 32 * PX;
    // a[e][c] = Phi_jc beta_c (complex path) or Phi_j,col(u) * scale_u beta_u (real terms)
    float2 a[PX][NC];
#pragma unroll
    for (int e = 0; e < PX; ++e) {
        const int64_t j = base + lane + 32 * e;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float2 v = make_float2(0.f, 0.f);
            const int col = REAL ? tb.term_col[c] : c;
            const float2 b = REAL ? tb.term_amp[c] : tb.amp[c];
            if (j < m && c < nterms && col < ncols) {
                const float2 ph = Phi[j * ncols + col];
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
            const float2* lt = Ls + t * LSTRIDE;
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
                } else if (REAL) {
                    // sum of real terms Re(a_u lambda_u^t); padded terms are zero
                    float zr = 0.f;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float2 l = lt[c];
                        zr = fmaf(a[e][c].x, l.x, zr);
                        zr = fmaf(-a[e][c].y, l.y, zr);
                    }
                    bg = (MODE == CDMD_BG_REAL) ? zr : fabsf(zr);
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

template <int NC, int PX, int MODE>
__global__ void __launch_bounds__(kThreads)
subtract_kernel(const uint8_t* __restrict__ D, int64_t m, int n, int64_t ldd,
                const float2* __restrict__ Phi, int ncols, Table tb, float tau, uint32_t* __restrict__ mask,
                int64_t words_per_frame, float* __restrict__ bg_out) {
    extern __shared__ float2 Ls[];   // [n][NC] lambda^t per real term, or per column
    const bool real_only = (MODE != CDMD_BG_STATIC) && tb.hdr[1] != 0;
    const float2* src = real_only ? tb.ttable : tb.table;
    for (int idx = threadIdx.x; idx < n * NC; idx += kThreads) Ls[idx] = src[idx];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = static_cast<int64_t>(gridDim.x) * (kThreads / 32);
    const int64_t tiles = (m + 32 * PX - 1) / (32 * PX);
    const int64_t first = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
    if (real_only) {
        // real terms, unrolled for the smallest of three sizes that holds them
        // (the lambda^t rows keep their stride NC)
        constexpr int N1 = (NC + 1) / 2, N2 = (3 * NC + 3) / 4;
        const int nterms = tb.hdr[0];
        if (nterms <= N1) {
            for (int64_t tile = first; tile < tiles; tile += warps_total)
                subtract_tile<N1, PX, MODE, true, NC>(D, m, n, ldd, Phi, ncols, tb, nterms, Ls, tau, mask,
                                                      words_per_frame, bg_out, tile, lane);
        } else if (nterms <= N2) {
            for (int64_t tile = first; tile < tiles; tile += warps_total)
                subtract_tile<N2, PX, MODE, true, NC>(D, m, n, ldd, Phi, ncols, tb, nterms, Ls, tau, mask,
                                                      words_per_frame, bg_out, tile, lane);
        } else {
            for (int64_t tile = first; tile < tiles; tile += warps_total)
                subtract_tile<NC, PX, MODE, true, NC>(D, m, n, ldd, Phi, ncols, tb, nterms, Ls, tau, mask,
                                                      words_per_frame, bg_out, tile, lane);
        }
    } else {
        for (int64_t tile = first; tile < tiles; tile += warps_total)
            subtract_tile<NC, PX, MODE, false, NC>(D, m, n, ldd, Phi, ncols, tb, NC, Ls, tau, mask, words_per_frame,
                                                   bg_out, tile, lane);
    }
}

// TMA-staged variant for 16-byte aligned frames and up to 12 columns: a
// producer warp streams [16 frames x 960 pixels] chunks of the video into a
// ring of shared-memory stages with 2-D tensor loads (out-of-range pixels and
// frames read as zero), so 90 KB per SM are in flight independently of the
// consumers' registers.  Consumer warp w owns pixels 64w .. 64w + 63 of
// the CTA tile, lane l the pixels 64w + l and 64w + l + 32, so each of the
// two ballots of a frame is one mask word.  Waits are bounded: after
// 2 s the kernel records CDMD_ERR_TIMEOUT, stops, and waits (again bounded)
// for its own loads in flight before it exits.
constexpr int kTmaPxl = 2;                          // adjacent pixels per lane
constexpr int kTmaConsumers = 15;                   // + 1 producer warp = 16 warps (128 registers each)
constexpr int kTmaThreads = 32 * (kTmaConsumers + 1);
constexpr int kTmaFB = 16;                          // frames per chunk
constexpr int kTmaWarpPx = 32 * kTmaPxl;            // pixels per consumer warp
constexpr int kTmaTile = kTmaWarpPx * kTmaConsumers;   // pixels per CTA tile (960)
constexpr int kTmaBox = 192;                        // pixels per tensor load (3 warps; box width <= 256)
static_assert(kTmaTile % kTmaBox == 0 && kTmaBox % kTmaWarpPx == 0 && kTmaTile % 32 == 0, "tile layout");
static_assert(kTmaBox % 16 == 0, "tensor-load x offsets must be multiples of 16 bytes");
static_assert(kTmaPxl == 2, "a lane owns pixels l and l + 32 of its warp's 64");
constexpr int kTmaStages = 6;
constexpr int kChunkBytes = kTmaFB * kTmaTile;


__host__ __device__ inline size_t tma_ls_offset() { return static_cast<size_t>(kTmaStages) * kChunkBytes; }
__host__ __device__ inline size_t tma_bar_offset(int n, int nc) {
    return (tma_ls_offset() + static_cast<size_t>(n) * nc * sizeof(float2) + 15) & ~static_cast<size_t>(15);
}
__host__ __device__ inline size_t tma_smem_bytes(int n, int nc) {
    return tma_bar_offset(n, nc) + 2 * kTmaStages * sizeof(uint64_t) + 16;
}

// Consumer side: every chunk of every tile of this CTA.
template <int NT, int MODE, bool REAL, int LSTRIDE>
__device__ __forceinline__ void tma_consume(const uint8_t* stages, uint64_t* full, uint64_t* empty, volatile int* abort,
                                            int* status, int64_t tile0, int64_t tstride, int64_t my_tiles, int nch,
                                            int64_t m, int n,
                                            const float2* __restrict__ Phi, int ncols, const Table& tb, int nterms,
                                            const float2* Ls, float tau, uint32_t* __restrict__ mask,
                                            int64_t words_per_frame, float* __restrict__ bg_out, int warp, int lane) {
    for (int64_t ti = 0; ti < my_tiles; ++ti) {
        const int64_t tile = tile0 + ti * tstride;
        // lane l owns pixels j0 + l and j0 + l + 32 of the warp's 64, so each
        // ballot is one mask word as it stands
        const int64_t j0 = tile * kTmaTile + warp * kTmaWarpPx + lane;
        float2 a[kTmaPxl][NT];
#pragma unroll
        for (int e = 0; e < kTmaPxl; ++e) {
            const int64_t j = j0 + 32 * e;
#pragma unroll
            for (int c = 0; c < NT; ++c) {
                float2 v = make_float2(0.f, 0.f);
                const int col = REAL ? tb.term_col[c] : c;
                const float2 b = REAL ? tb.term_amp[c] : tb.amp[c];
                if (j < m && c < nterms && col < ncols) {
                    const float2 ph = Phi[j * ncols + col];
                    v = make_float2(ph.x * b.x - ph.y * b.y, ph.x * b.y + ph.y * b.x);
                }
                a[e][c] = v;
            }
        }
        float bg_static[kTmaPxl];
        if (MODE == CDMD_BG_STATIC) {
#pragma unroll
            for (int e = 0; e < kTmaPxl; ++e) {
                float zr = 0.f, zi = 0.f;
#pragma unroll
                for (int c = 0; c < NT; ++c) {
                    zr += a[e][c].x;
                    zi += a[e][c].y;
                }
                bg_static[e] = sqrtf(zr * zr + zi * zi);
            }
        }
        for (int ch = 0; ch < nch; ++ch) {
            const int64_t g = ti * nch + ch;
            const int s = static_cast<int>(g % kTmaStages);
            if (!tc::mbar_wait(&full[s], static_cast<uint32_t>(g / kTmaStages) & 1u, abort, status)) return;
            constexpr int kWarpsPerBox = kTmaBox / kTmaWarpPx;
            const uint8_t* buf = stages + static_cast<size_t>(s) * kChunkBytes +
                                 (warp / kWarpsPerBox) * (kTmaFB * kTmaBox) + (warp % kWarpsPerBox) * kTmaWarpPx + lane;
            const int t0 = ch * kTmaFB;
            // the chunk's 16 frames x 2 mask words: lane 2f + e keeps word e
            // of frame f and every lane stores one word after the chunk
            static_assert(2 * kTmaFB == 32 && kTmaPxl == 2, "one mask word per lane per chunk");
            uint32_t keep = 0;
#pragma unroll 4
            for (int f = 0; f < kTmaFB; ++f) {
                const int t = t0 + f;
                if (t >= n) break;
                // this frame's lambda^t row, two terms per 16-byte load (rows
                // start 16-byte aligned: LSTRIDE is even)
                static_assert(LSTRIDE % 2 == 0, "lambda^t rows must hold an even number of columns");
                const float2* lt = Ls + t * LSTRIDE;
                float2 lv[NT];
#pragma unroll
                for (int c = 0; c + 1 < NT; c += 2) {
                    const float4 q = *reinterpret_cast<const float4*>(lt + c);
                    lv[c] = make_float2(q.x, q.y);
                    lv[c + 1] = make_float2(q.z, q.w);
                }
                if (NT & 1) lv[NT - 1] = lt[NT - 1];
                uint32_t bal[kTmaPxl];
#pragma unroll
                for (int e = 0; e < kTmaPxl; ++e) {
                    const int64_t j = j0 + 32 * e;
                    // the byte as a float: 2^23 + b built from the bits, minus 2^23 (exact)
                    const uint32_t b = buf[f * kTmaBox + 32 * e];
                    const float x = __uint_as_float(0x4B000000u | b) - 8388608.0f;
                    bool bit;
                    float bg = 0.0f;
                    if (MODE == CDMD_BG_STATIC) {
                        bg = bg_static[e];
                        bit = fabsf(x - bg) > tau;
                    } else if (REAL) {
                        // two partial sums (even / odd terms) halve the FMA dependency chain
                        float z0 = 0.f, z1 = 0.f;
#pragma unroll
                        for (int c = 0; c < NT; ++c) {
                            const float2 l = lv[c];
                            float& z = (c & 1) ? z1 : z0;
                            z = fmaf(a[e][c].x, l.x, z);
                            z = fmaf(-a[e][c].y, l.y, z);
                        }
                        const float zr = z0 + z1;
                        bg = (MODE == CDMD_BG_REAL) ? zr : fabsf(zr);
                        bit = fabsf(x - bg) > tau;
                    } else {
                        float zr = 0.f, zi = 0.f;
#pragma unroll
                        for (int c = 0; c < NT; ++c) {
                            const float2 l = lv[c];
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
                            const float q = fmaf(zr, zr, zi * zi);
                            const float up = x + tau, dn = x - tau;
                            bit = (q > up * up) || (dn > 0.0f && q < dn * dn);
                        }
                    }
                    bit = bit && (j < m);
                    if (bg_out != nullptr && j < m) bg_out[static_cast<int64_t>(t) * m + j] = bg;
                    bal[e] = __ballot_sync(0xffffffffu, bit);
                }
                if (lane == 2 * f) keep = bal[0];
                if (lane == 2 * f + 1) keep = bal[1];
            }
            {
                const int t = t0 + (lane >> 1);
                const int64_t wi = tile * (kTmaTile / 32) + warp * kTmaPxl + (lane & 1);
                if (t < n && wi < words_per_frame) mask[static_cast<int64_t>(t) * words_per_frame + wi] = keep;
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
        }
    }
}

template <int NC, int MODE>
__device__ __forceinline__ void subtract_tma_body(const CUtensorMap* tmap, int64_t m, int n,
                                                  const float2* __restrict__ Phi, int ncols, const Table& tb, float tau,
                                                  uint32_t* __restrict__ mask, int64_t words_per_frame,
                                                  float* __restrict__ bg_out, int* status, int64_t tile0,
                                                  int64_t tstride, int64_t my_tiles, uint8_t* smem) {
    uint8_t* stages = smem;
    float2* Ls = reinterpret_cast<float2*>(smem + tma_ls_offset());
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + tma_bar_offset(n, NC));
    uint64_t* empty = full + kTmaStages;
    volatile int* abort = reinterpret_cast<volatile int*>(empty + kTmaStages);
    int* issued_sm = reinterpret_cast<int*>(empty + kTmaStages) + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool real_only = (MODE != CDMD_BG_STATIC) && tb.hdr[1] != 0;
    const float2* src = real_only ? tb.ttable : tb.table;
    for (int idx = threadIdx.x; idx < n * NC; idx += kTmaThreads) Ls[idx] = src[idx];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kTmaConsumers);
        }
        *abort = 0;
        *issued_sm = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    const int nch = (n + kTmaFB - 1) / kTmaFB;
    const int64_t total = my_tiles * nch;
    if (warp == kTmaConsumers) {
        if (lane == 0) {
            int64_t g = 0;
            for (; g < total; ++g) {
                const int s = static_cast<int>(g % kTmaStages);
                const int64_t u = g / kTmaStages;
                if (u >= 1 && !tc::mbar_wait(&empty[s], static_cast<uint32_t>(u - 1) & 1u, abort, status)) break;
                if (*abort) break;
                const int64_t tile = tile0 + (g / nch) * tstride;
                const int t0 = static_cast<int>(g % nch) * kTmaFB;
                tc::mbar_arrive_expect_tx(&full[s], kChunkBytes);
#pragma unroll
                for (int q = 0; q < kTmaTile / kTmaBox; ++q)
                    tc::tma_load_2d(stages + static_cast<size_t>(s) * kChunkBytes + q * (kTmaFB * kTmaBox), tmap,
                                    static_cast<int>(tile * kTmaTile + q * kTmaBox), t0, &full[s]);
            }
            *issued_sm = static_cast<int>(g);
        }
    } else if (real_only) {
        // one real term per real mode or conjugate pair: K/2 to (K+1)/2 + 1
        // terms when most modes pair up
        constexpr int N1 = (NC + 1) / 2, N2 = N1 + 1, N3 = N1 + 2;
        const int nterms = tb.hdr[0];
        if (nterms <= N1)
            tma_consume<N1, MODE, true, NC>(stages, full, empty, abort, status, tile0, tstride, my_tiles, nch, m, n, Phi, ncols, tb,
                                            nterms, Ls, tau, mask, words_per_frame, bg_out, warp, lane);
        else if (nterms <= N2)
            tma_consume<N2, MODE, true, NC>(stages, full, empty, abort, status, tile0, tstride, my_tiles, nch, m, n, Phi, ncols, tb,
                                            nterms, Ls, tau, mask, words_per_frame, bg_out, warp, lane);
        else if (nterms <= N3)
            tma_consume<N3, MODE, true, NC>(stages, full, empty, abort, status, tile0, tstride, my_tiles, nch, m, n, Phi, ncols, tb,
                                            nterms, Ls, tau, mask, words_per_frame, bg_out, warp, lane);
        else
            tma_consume<NC, MODE, true, NC>(stages, full, empty, abort, status, tile0, tstride, my_tiles, nch, m, n, Phi, ncols, tb,
                                            nterms, Ls, tau, mask, words_per_frame, bg_out, warp, lane);
    } else {
        tma_consume<NC, MODE, false, NC>(stages, full, empty, abort, status, tile0, tstride, my_tiles, nch, m, n, Phi, ncols, tb, NC,
                                         Ls, tau, mask, words_per_frame, bg_out, warp, lane);
    }
    __syncthreads();
    // after an abort, wait (bounded) for this CTA's own tensor loads in flight
    if (threadIdx.x == 0 && *abort) {
        const int64_t issued = *issued_sm;
        volatile int never = 0;
        for (int64_t g = (issued > kTmaStages ? issued - kTmaStages : 0); g < issued; ++g)
            tc::mbar_wait(&full[g % kTmaStages], static_cast<uint32_t>(g / kTmaStages) & 1u, &never, status);
    }
}

template <int NC, int MODE>
__global__ void __launch_bounds__(kTmaThreads, 1)   // 16 warps x 128 registers fill the 64K register file
subtract_tma_kernel(const __grid_constant__ CUtensorMap tmap, int64_t m, int n, const float2* __restrict__ Phi,
                    int ncols, Table tb, float tau, uint32_t* __restrict__ mask, int64_t words_per_frame,
                    float* __restrict__ bg_out, int* status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int64_t tiles = (m + kTmaTile - 1) / kTmaTile;
    const int64_t my_tiles = (static_cast<int64_t>(blockIdx.x) < tiles) ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    subtract_tma_body<NC, MODE>(&tmap, m, n, Phi, ncols, tb, tau, mask, words_per_frame, bg_out, status, blockIdx.x,
                                gridDim.x, my_tiles, smem);
}

// Grouped: CTA b runs item items[b], consecutive tiles of one clip.
template <int NC, int MODE>
__global__ void __launch_bounds__(kTmaThreads, 1)
subtract_tma_grouped_kernel(const SubtractClip* __restrict__ clips, const SubtractItem* __restrict__ items,
                            float tau, int* status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const SubtractItem it = items[blockIdx.x];
    const SubtractClip c = clips[it.clip];
    subtract_tma_body<NC, MODE>(c.tmap, c.m, c.n, reinterpret_cast<const float2*>(c.Phi), c.ncols,
                                table_views(c.table, c.n, NC), tau, c.mask, c.words_per_frame, nullptr, status,
                                it.tile0, 1, it.ntiles, smem);
}

template <int NC>
cdmd_status launch_nc_tma(cdmd_ctx* ctx, cdmd_bgmode mode, const uint8_t* D, int64_t m, int n, int64_t ldd,
                          const float2* Phi, int ncols, const Table& tb, float tau, uint32_t* mask, float* bg,
                          cudaStream_t stream) {
    CUtensorMap tmap;
    cdmd_status st = make_video_tmap(&tmap, D, m, n, ldd, kTmaBox, kTmaFB);
    if (st != CDMD_OK) return st;
    const int64_t tiles = (m + kTmaTile - 1) / kTmaTile;
    const int64_t blocks = std::min<int64_t>(tiles, static_cast<int64_t>(ctx->num_sms));
    const size_t smem = tma_smem_bytes(n, NC);
    const int64_t wpf = (m + 31) / 32;
#define CDMD_SUBT_MODE(MV)                                                                              \
    {                                                                                                   \
        auto kern = subtract_tma_kernel<NC, MV>;                                                        \
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                             static_cast<int>(smem)));                                  \
        kern<<<static_cast<unsigned>(blocks), kTmaThreads, smem, stream>>>(tmap, m, n, Phi, ncols, tb, tau, \
                                                                           mask, wpf, bg, ctx->d_status); \
    }
    if (mode == CDMD_BG_MODULUS) CDMD_SUBT_MODE(CDMD_BG_MODULUS)
    else if (mode == CDMD_BG_REAL) CDMD_SUBT_MODE(CDMD_BG_REAL)
    else CDMD_SUBT_MODE(CDMD_BG_STATIC)
#undef CDMD_SUBT_MODE
    CDMD_CHECK_LAUNCH("subtract_tma_kernel");
    return CDMD_OK;
}

template <int NC, int PX>
cdmd_status launch_nc(cdmd_bgmode mode, const uint8_t* D, int64_t m, int n, int64_t ldd,
                      const float2* Phi, int ncols, const Table& tb, float tau, uint32_t* mask, float* bg, int sms,
                      cudaStream_t stream) {
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
                                                                        tb, tau, mask, wpf, bg);  \
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
    cdmd_status st = ensure_buffer(ctx, BUF_SUBTRACT_TABLE, table_bytes(n, nc_pad), &tbl);
    if (st != CDMD_OK) return st;
    const Table tb = table_views(tbl, n, nc_pad);
    subtract_table_kernel<<<1, kTableThreads, 0, stream>>>(cols, ncols, nc_pad, beta, lambda, r, n, tb);
    CDMD_CHECK_LAUNCH("subtract_table_kernel");
    if (subtract_tc_supported(n, ncols, mode, D, ldd, m, Phi, bg))
        return launch_subtract_tc(ctx, D, m, n, ldd, Phi, ncols, subtract_tc_table(tbl, n, nc_pad), nc_pad, tau, mode,
                                  mask, stream);
    const float2* ph = reinterpret_cast<const float2*>(Phi);
    // TMA needs a 16-byte aligned base and row stride; n <= 512 keeps the
    // lambda^t table within shared memory next to the stages
    const bool tma_ok = (reinterpret_cast<uintptr_t>(D) % 16 == 0) && (ldd % 16 == 0) && nc_pad <= 12 && n <= 512 &&
                        m <= 0x7fffffffLL - 2 * kTmaTile;
    if (tma_ok) {
        switch (nc_pad) {
            case 4: return launch_nc_tma<4>(ctx, mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, stream);
            case 8: return launch_nc_tma<8>(ctx, mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, stream);
            case 10: return launch_nc_tma<10>(ctx, mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, stream);
            default: return launch_nc_tma<12>(ctx, mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, stream);
        }
    }
    switch (nc_pad) {
        case 4: return launch_nc<4, 4>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        case 8: return launch_nc<8, 4>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        case 10: return launch_nc<10, 2>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        case 12: return launch_nc<12, 2>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        case 16: return launch_nc<16, 2>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        case 20: return launch_nc<20, 1>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        case 24: return launch_nc<24, 1>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
        default: return launch_nc<32, 1>(mode, D, m, n, ldd, ph, ncols, tb, tau, mask, bg, ctx->num_sms, stream);
    }
}

}  // namespace cdmd

namespace cdmd {

size_t subtract_table_bytes_nc(int n, int nc) { return table_bytes(n, nc); }

SubTcTable subtract_tc_table(void* table, int n, int nc) {
    const Table t = table_views(table, n, nc);
    SubTcTable r;
    r.hdr = t.hdr;
    r.term_col = t.term_col;
    r.amp = t.amp;
    r.term_amp = t.term_amp;
    r.lam_t = t.table;
    r.term_lam_t = t.ttable;
    return r;
}
size_t subtract_tma_smem(int n, int nc) { return tma_smem_bytes(n, nc); }
int subtract_tile_pixels() { return kTmaTile; }

cdmd_status make_subtract_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd) {
    return make_video_tmap(map, D, m, n, ldd, kTmaBox, kTmaFB);
}

cdmd_status launch_subtract_grouped(const SubtractClip* clips, int nclips, const SubtractItem* items, int nitems,
                                    int nc, int max_n, cdmd_bgmode mode, float tau, int* status, cudaStream_t stream) {
    subtract_table_grouped_kernel<<<static_cast<unsigned>(nclips), kTableThreads, 0, stream>>>(clips, nc);
    CDMD_CHECK_LAUNCH("subtract_table_grouped_kernel");
    if (nitems == 0) return CDMD_OK;
    const size_t smem = tma_smem_bytes(max_n, nc);
#define CDMD_SUBG(NCV, MV)                                                                                   \
    {                                                                                                        \
        auto kern = subtract_tma_grouped_kernel<NCV, MV>;                                                    \
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                             static_cast<int>(smem)));                                       \
        kern<<<static_cast<unsigned>(nitems), kTmaThreads, smem, stream>>>(clips, items, tau, status);       \
    }
#define CDMD_SUBG_NC(MV)                                \
    switch (nc) {                                       \
        case 4: CDMD_SUBG(4, MV) break;                 \
        case 8: CDMD_SUBG(8, MV) break;                 \
        case 10: CDMD_SUBG(10, MV) break;               \
        case 12: CDMD_SUBG(12, MV) break;               \
        default: return fail(CDMD_ERR_INVALID_ARG, "grouped subtract: column stride %d", nc); \
    }
    if (mode == CDMD_BG_MODULUS) { CDMD_SUBG_NC(CDMD_BG_MODULUS) }
    else if (mode == CDMD_BG_REAL) { CDMD_SUBG_NC(CDMD_BG_REAL) }
    else { CDMD_SUBG_NC(CDMD_BG_STATIC) }
#undef CDMD_SUBG_NC
#undef CDMD_SUBG
    CDMD_CHECK_LAUNCH("subtract_tma_grouped_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
