// SRFT sketch (Section 3.3, "Measurement Matrices": C = R F D, the
// subsampled randomized Fourier transform), applied with a fast transform.
//
// Row 2a of the real sketch is Re(F D)[s_a, :] and row 2a+1 is Im(F D)[s_a, :],
// F the unnormalised m-point DFT, D = diag(exp(i theta_j)), s_0 < s_1 < ...
// the kept frequencies (see cdmd.h, CDMD_C_SRFT).  So the sketch of frame x is
// X[s_a] = sum_j exp(-2 pi i s_a j / m) d_j x_j at the kept frequencies.
//
// Four-step factorisation of the m-point DFT: with m = N1 N2 and pixel
// j = c + N1 y (c < N1, y < N2),
//     X[f] = sum_c exp(-2 pi i f c / m) Z_c[f mod N2],
//     Z_c[g] = sum_y exp(-2 pi i g y / N2) d_{c + N1 y} x_{c + N1 y},
// i.e. an N2-point FFT down each of the N1 strided "columns", then for each
// kept frequency a sum over the columns with one twiddle each.  N2 is the
// largest divisor of m up to 1024 made of the factors 2, 3 and 5, so the
// column FFTs run as mixed-radix (4, 2, 3, 5) Stockham passes in shared
// memory; the cost is O(m log N2 + |R| N1) per frame instead of the dense
// O(k m).
//
// Kernel layout: a CTA owns a group of column tiles (S columns each) and a
// range of frames.  Per tile it tabulates d_j for the tile's S x N2 pixels
// (one Philox draw per pixel, reused for every frame), then per frame loads
// the tile (uint8 -> complex d_j x_j), runs the FFT passes, and adds the
// tile's share of every kept frequency into an FP32 accumulator in shared
// memory.  After its last tile it writes the accumulator as partials
// [tile group][frame][frequency]; a second kernel adds the groups in FP64 in
// a fixed order and writes D_Y.
#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr int kSrftThreads = 1024;
constexpr int kSrftMaxN2 = 1024;
constexpr int kSrftAccElems = 4096;        // accumulator: frames per CTA x kept frequencies (32 KB)
constexpr size_t kSrftSmemBudget = 220 * 1024;
constexpr int kSrftMaxStages = 16;
constexpr uint32_t kStreamSrftPhase = 5u;

struct SrftStages {
    int n;
    int radix[kSrftMaxStages];
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// exp(i theta_j) of the diagonal D, theta_j = 2 pi U(w0), w0 word 0 of
// Philox counter (j, 0, 5, 0)
__device__ __forceinline__ float2 srft_phase(uint2 key, int64_t j) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), 0u, kStreamSrftPhase, 0u), key);
    const float u = fmaf(__uint2float_rn(w.x), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    float s, c;
    sincospif(2.0f * u, &s, &c);
    return make_float2(c, s);
}

// Radix-R butterflies of the forward DFT (exp(-2 pi i q r / R)): inputs
// src[r L] times the stage twiddle tw[r tb], outputs dst[q Ns].
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_neg_i(float2 a) { return make_float2(a.y, -a.x); }   // a * (-i)

__device__ __forceinline__ float2 load_tw(const float2* src, int r, int L, const float2* tw, int tb) {
    const float2 a = src[r * L];
    return tb == 0 ? a : cmulf(a, tw[r * tb]);
}

__device__ __forceinline__ void butterfly2(const float2* src, float2* dst, int L, int Ns, const float2* tw, int tb) {
    const float2 a = src[0], b = load_tw(src, 1, L, tw, tb);
    dst[0] = cadd2(a, b);
    dst[Ns] = csub2(a, b);
}

__device__ __forceinline__ void butterfly4(const float2* src, float2* dst, int L, int Ns, const float2* tw, int tb) {
    const float2 a = src[0], b = load_tw(src, 1, L, tw, tb), c = load_tw(src, 2, L, tw, tb),
                 d = load_tw(src, 3, L, tw, tb);
    const float2 s0 = cadd2(a, c), d0 = csub2(a, c), s1 = cadd2(b, d), d1 = mul_neg_i(csub2(b, d));
    dst[0] = cadd2(s0, s1);            // a + b + c + d
    dst[Ns] = cadd2(d0, d1);           // a - i b - c + i d
    dst[2 * Ns] = csub2(s0, s1);       // a - b + c - d
    dst[3 * Ns] = csub2(d0, d1);       // a + i b - c - i d
}

__device__ __forceinline__ void butterfly3(const float2* src, float2* dst, int L, int Ns, const float2* tw, int tb) {
    const float2 a = src[0], b = load_tw(src, 1, L, tw, tb), c = load_tw(src, 2, L, tw, tb);
    const float h = 0.8660254037844386f;                         // sin(2 pi / 3)
    const float2 t = cadd2(b, c);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    const float2 u = csub2(b, c);
    const float2 w = make_float2(h * u.y, -h * u.x);             // -i sin(2 pi/3) (b - c)
    dst[0] = cadd2(a, t);
    dst[Ns] = cadd2(m, w);
    dst[2 * Ns] = csub2(m, w);
}

__device__ __forceinline__ void butterfly5(const float2* src, float2* dst, int L, int Ns, const float2* tw, int tb) {
    float2 v[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) v[r] = load_tw(src, r, L, tw, tb);
    // cos and sin of 2 pi q / 5, q = 0..4
    const float cq[5] = {1.0f, 0.30901699437494745f, -0.8090169943749473f, -0.8090169943749473f, 0.30901699437494745f};
    const float sq[5] = {0.0f, 0.9510565162951535f, 0.5877852522924732f, -0.5877852522924732f, -0.9510565162951535f};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        float2 sum = v[0];
#pragma unroll
        for (int r = 1; r < 5; ++r) {
            const int e = (q * r) % 5;                           // exp(-2 pi i e / 5) = (c, -s)
            sum.x = fmaf(v[r].x, cq[e], fmaf(v[r].y, sq[e], sum.x));
            sum.y = fmaf(v[r].y, cq[e], fmaf(-v[r].x, sq[e], sum.y));
        }
        dst[q * Ns] = sum;
    }
}

__global__ void __launch_bounds__(kSrftThreads)
srft_partial_kernel(const uint8_t* __restrict__ D, int64_t m, int n, int64_t ldd, int64_t N1, int N2, int S,
                    SrftStages st, uint2 key, const int64_t* __restrict__ freqs, int nf, int tiles,
                    int tiles_per_group, int fpc, float2* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char srft_smem[];
    // column c of a tile starts at c * P: the odd pad spreads the tile-load
    // stores (one per column, same row) over the banks
    const int P = N2 + 1;
    const int elems = S * P;
    float2* bufA = reinterpret_cast<float2*>(srft_smem);
    float2* bufB = bufA + elems;
    float2* dtab = bufB + elems;
    float2* tw = dtab + elems;                     // exp(-2 pi i e / N2), e < N2
    float2* acc = tw + N2;                         // [fpc][nf]
    int64_t* ph0 = reinterpret_cast<int64_t*>(acc + static_cast<size_t>(fpc) * nf);   // (s_a x0) mod m
    const int tid = threadIdx.x;
    const int group = blockIdx.x;
    const int t0 = blockIdx.y * fpc;
    const int t1 = min(n, t0 + fpc);
    const float inv_m = 1.0f / static_cast<float>(m);

    for (int e = tid; e < N2; e += kSrftThreads) {
        float s, c;
        sincospif(-2.0f * static_cast<float>(e) / static_cast<float>(N2), &s, &c);
        tw[e] = make_float2(c, s);
    }
    for (int e = tid; e < fpc * nf; e += kSrftThreads) acc[e] = make_float2(0.0f, 0.0f);

    const int tile_lo = group * tiles_per_group;
    const int tile_hi = min(tiles, tile_lo + tiles_per_group);
    for (int tile = tile_lo; tile < tile_hi; ++tile) {
        const int64_t x0 = static_cast<int64_t>(tile) * S;
        __syncthreads();                            // previous tile's readers of dtab / ph0 are done
        for (int e = tid; e < S * N2; e += kSrftThreads) {
            const int c = e / N2, y = e - c * N2;
            const int64_t x = x0 + c;
            dtab[c * P + y] = (x < N1) ? srft_phase(key, x + N1 * y) : make_float2(0.0f, 0.0f);
        }
        for (int a = tid; a < nf; a += kSrftThreads) ph0[a] = (freqs[a] % m) * x0 % m;
        for (int t = t0; t < t1; ++t) {
            __syncthreads();                        // dtab ready; previous frame's readers of the buffers done
            const uint8_t* Dt = D + static_cast<int64_t>(t) * ldd;
            for (int e = tid; e < S * N2; e += kSrftThreads) {
                // consecutive threads read consecutive columns of one row
                const int y = e / S, c = e - y * S;
                const int64_t x = x0 + c;
                const float v = (x < N1) ? static_cast<float>(Dt[x + N1 * y]) : 0.0f;
                const float2 d = dtab[c * P + y];
                bufA[c * P + y] = make_float2(v * d.x, v * d.y);
            }
            // Stockham passes: sub-transforms of size Ns grow by each radix R;
            // butterfly j (of L = N2 / R) reads j + r L, twiddles by
            // exp(-2 pi i r (j mod Ns) / (Ns R)), and writes its R outputs Ns apart
            float2* in = bufA;
            float2* out = bufB;
            int Ns = 1;
            for (int s = 0; s < st.n; ++s) {
                const int R = st.radix[s];
                const int L = N2 / R;
                const int twstep = N2 / (Ns * R);
                // exact quotients of small non-negative ints by a float reciprocal
                const float inv_L = 1.0f / static_cast<float>(L);
                const float inv_Ns = 1.0f / static_cast<float>(Ns);
                __syncthreads();
                for (int b = tid; b < S * L; b += kSrftThreads) {
                    const int c = static_cast<int>((static_cast<float>(b) + 0.5f) * inv_L);
                    const int j = b - c * L;
                    const int g = static_cast<int>((static_cast<float>(j) + 0.5f) * inv_Ns);
                    const int kk = j - g * Ns;
                    const float2* src = in + c * P + j;
                    float2* dst = out + c * P + g * Ns * R + kk;
                    const int tb = kk * twstep;
                    if (R == 4) butterfly4(src, dst, L, Ns, tw, tb);
                    else if (R == 2) butterfly2(src, dst, L, Ns, tw, tb);
                    else if (R == 3) butterfly3(src, dst, L, Ns, tw, tb);
                    else butterfly5(src, dst, L, Ns, tw, tb);
                }
                float2* tmp = in;
                in = out;
                out = tmp;
                Ns *= R;
            }
            __syncthreads();
            // the tile's share of every kept frequency s_a:
            //   sum_c exp(-2 pi i s_a (x0 + c) / m) Z_c[s_a mod N2]
            float2* accf = acc + static_cast<size_t>(t - t0) * nf;
            for (int a = tid; a < nf; a += kSrftThreads) {
                const int64_t f = freqs[a] % m;
                const int g = static_cast<int>(f % N2);
                int64_t ph = ph0[a];
                float2 sum = make_float2(0.0f, 0.0f);
                for (int c = 0; c < S; ++c) {
                    if (x0 + c >= N1) break;
                    float s, co;
                    sincospif(-2.0f * (static_cast<float>(ph) * inv_m), &s, &co);
                    const float2 p = cmulf(in[c * P + g], make_float2(co, s));
                    sum.x += p.x;
                    sum.y += p.y;
                    ph += f;
                    if (ph >= m) ph -= m;
                }
                accf[a].x += sum.x;
                accf[a].y += sum.y;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < (t1 - t0) * nf; e += kSrftThreads) {
        const int tl = e / nf, a = e - tl * nf;
        partial[(static_cast<int64_t>(group) * n + t0 + tl) * nf + a] = acc[e];
    }
}

// DY[t k + i] = sum over tile groups (FP64, fixed order) of the real (even i)
// or imaginary (odd i) part of frequency i / 2
__global__ void srft_reduce_kernel(const float2* __restrict__ partial, int groups, int n, int nf, int k,
                                   double* __restrict__ DY) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<int64_t>(n) * k) return;
    const int t = static_cast<int>(idx / k), i = static_cast<int>(idx % k);
    const int a = i >> 1;
    double s = 0.0;
    for (int g = 0; g < groups; ++g) {
        const float2 v = partial[(static_cast<int64_t>(g) * n + t) * nf + a];
        s += static_cast<double>((i & 1) ? v.y : v.x);
    }
    DY[idx] = s;
}

// largest divisor of m up to kSrftMaxN2 whose prime factors are 2, 3 and 5
int64_t srft_fft_length(int64_t m) {
    int64_t best = 1;
    for (int64_t d = 2; d <= kSrftMaxN2 && d <= m; ++d) {
        if (m % d != 0) continue;
        int64_t r = d;
        for (int p : {2, 3, 5})
            while (r % p == 0) r /= p;
        if (r == 1) best = d;
    }
    return best;
}

SrftStages srft_stages(int64_t N2) {
    SrftStages s{};
    int64_t r = N2;
    while (r % 4 == 0) { s.radix[s.n++] = 4; r /= 4; }
    while (r % 2 == 0) { s.radix[s.n++] = 2; r /= 2; }
    while (r % 3 == 0) { s.radix[s.n++] = 3; r /= 3; }
    while (r % 5 == 0) { s.radix[s.n++] = 5; r /= 5; }
    return s;
}

}  // namespace

cdmd_status launch_sketch_srft(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               const cdmd_measure* meas, double* DY, cudaStream_t stream) {
    const int k = meas->k;
    const int nf = (k + 1) / 2;
    CDMD_REQUIRE(nf <= kSrftAccElems, "SRFT keeps at most %d frequencies (k <= %d)", kSrftAccElems,
                 2 * kSrftAccElems);
    const int64_t N2 = srft_fft_length(m);
    const int64_t N1 = m / N2;
    int fpc = std::max(1, std::min(n, kSrftAccElems / nf));
    // columns per tile: as many as the three column buffers leave room for (<= 16)
    const size_t fixed = static_cast<size_t>(N2 + fpc * nf) * sizeof(float2) + static_cast<size_t>(nf) * sizeof(int64_t);
    const size_t per_col = 3 * static_cast<size_t>(N2 + 1) * sizeof(float2);
    const int S = static_cast<int>(std::min<size_t>(16, (kSrftSmemBudget - fixed) / per_col));
    CDMD_REQUIRE(S >= 1, "SRFT tile does not fit in shared memory");
    const int tiles = static_cast<int>((N1 + S - 1) / S);
    // about one CTA per SM (one fits: the tile buffers fill the shared
    // memory): tile groups first, then more frame groups if tiles run out
    int fgroups = (n + fpc - 1) / fpc;
    int groups = std::max(1, std::min(tiles, (ctx->num_sms + fgroups / 2) / fgroups));
    if (groups == tiles && groups * fgroups < ctx->num_sms) {
        fgroups = std::min(n, (ctx->num_sms + groups - 1) / groups);
        fpc = (n + fgroups - 1) / fgroups;
        fgroups = (n + fpc - 1) / fpc;
    }
    const int tiles_per_group = (tiles + groups - 1) / groups;
    groups = (tiles + tiles_per_group - 1) / tiles_per_group;
    float* part = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL,
                                   static_cast<size_t>(groups) * n * nf * sizeof(float2),
                                   reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    const size_t smem = fixed + static_cast<size_t>(S) * per_col;
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(srft_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    srft_partial_kernel<<<dim3(groups, fgroups), kSrftThreads, smem, stream>>>(
        D, m, n, ldd, N1, static_cast<int>(N2), S, srft_stages(N2), seed_key(meas->seed), meas->rows, nf, tiles,
        tiles_per_group, fpc, reinterpret_cast<float2*>(part));
    CDMD_CHECK_LAUNCH("srft_partial_kernel");
    const int64_t tot = static_cast<int64_t>(n) * k;
    srft_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, stream>>>(
        reinterpret_cast<const float2*>(part), groups, n, nf, k, DY);
    CDMD_CHECK_LAUNCH("srft_reduce_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
