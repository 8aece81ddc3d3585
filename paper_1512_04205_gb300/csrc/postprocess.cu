// Post-processing of the bit-packed foreground mask: a 3 x 3 median filter of
// each frame (Section 4, the BMC figure's median-filtered masks; the
// Discussion names the median filter as the post-pass that cuts false
// positives).  Pixel j of a frame sits at row j / W, column j % W; pixels
// outside the frame count as background.
//
// On 0/1 values the median of nine is 1 iff at least five are 1, so each
// thread filters 32 pixels at once: it forms the nine shifted 32-bit windows
// (row above, same row, row below; left, centre, right), clears the
// neighbours that would wrap across a row end, and counts the ones per bit
// with a bit-sliced adder.  A thread keeps one word position for four frames,
// so its row-edge masks are computed once, and loads all their words before
// it uses any (36 loads in flight).  HBM traffic is one read and one write of
// the mask; the row above and below come from L1/L2.
#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr int kMedianThreads = 256;
constexpr int kMedianFrames = 4;   // frames per thread

__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t& sum, uint32_t& carry) {
    const uint32_t t = a ^ b;
    sum = t ^ c;
    carry = (a & b) | (t & c);
}

__global__ void __launch_bounds__(kMedianThreads) median3x3_kernel(const uint32_t* __restrict__ in,
                                                                   uint32_t* __restrict__ out, uint32_t W,
                                                                   uint32_t m, int64_t nw, int n) {
    const int64_t w = static_cast<int64_t>(blockIdx.x) * kMedianThreads + threadIdx.x;
    if (w >= nw) return;
    const uint32_t p0 = static_cast<uint32_t>(w) * 32u;
    const uint32_t tail = (m & 31u) ? ((1u << (m & 31u)) - 1u) : 0xffffffffu;

    // bits whose pixel is in column 0 (their left neighbour would wrap) and in
    // column W-1 (their right neighbour would wrap)
    const uint32_t x0 = p0 % W;
    uint32_t left = 0u, right = 0u;
    for (uint32_t b = (x0 == 0u) ? 0u : W - x0; b < 32u; b += W) left |= 1u << b;
    for (uint32_t b = W - 1u - x0; b < 32u; b += W) right |= 1u << b;

    // Frame-independent part: row dy's window starts one pixel left of
    // p0 + (dy - 1) W, i.e. at bit sh[dy] of word wq[dy]; the three words
    // wq .. wq+2 cover it.
    int64_t wq[3];
    uint32_t sh[3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const int64_t q = static_cast<int64_t>(p0) + static_cast<int64_t>(dy - 1) * W - 1;
        wq[dy] = q >> 5;   // floor for negative q too
        sh[dy] = static_cast<uint32_t>(q) & 31u;
    }
    const uint32_t rmask = (w == nw - 1) ? tail : 0xffffffffu;
    const int f0 = static_cast<int>(blockIdx.y) * kMedianFrames;
    const int nf = min(kMedianFrames, n - f0);

    // all frames' words are loaded before any is used, so each thread keeps
    // 9 x kMedianFrames loads in flight.  Almost every thread reads nine
    // words inside the frame, none of them the last: plain loads.  The rest
    // zero the words outside the frame and mask the last word's spare bits.
    uint32_t win[kMedianFrames][3][3];
    if (wq[0] >= 0 && wq[2] + 2 < nw - 1) {
#pragma unroll
        for (int i = 0; i < kMedianFrames; ++i) {
            const uint32_t* fr = in + static_cast<int64_t>(f0 + min(i, nf - 1)) * nw;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int c = 0; c < 3; ++c) win[i][dy][c] = __ldg(fr + wq[dy] + c);
        }
    } else {
        uint32_t keep[3][3];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t x = wq[dy] + c;
                keep[dy][c] = (x < 0 || x >= nw) ? 0u : (x == nw - 1 ? tail : 0xffffffffu);
            }
#pragma unroll
        for (int i = 0; i < kMedianFrames; ++i) {
            const uint32_t* fr = in + static_cast<int64_t>(f0 + min(i, nf - 1)) * nw;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    win[i][dy][c] = keep[dy][c] ? (__ldg(fr + wq[dy] + c) & keep[dy][c]) : 0u;
        }
    }
#pragma unroll
    for (int i = 0; i < kMedianFrames; ++i) {
        uint32_t v[9];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            // bits s .. s+31 and s+32 .. s+63 of the 96-bit string c:b:a; the
            // centre and right windows start one and two bits later
            const uint32_t lo = __funnelshift_r(win[i][dy][0], win[i][dy][1], sh[dy]);
            const uint32_t hi = __funnelshift_r(win[i][dy][1], win[i][dy][2], sh[dy]);
            v[3 * dy + 0] = lo & ~left;
            v[3 * dy + 1] = __funnelshift_r(lo, hi, 1u);
            v[3 * dy + 2] = __funnelshift_r(lo, hi, 2u) & ~right;
        }
        uint32_t s1, c1, s2, c2, s3, c3, S, C, t1, t2;
        full_add(v[0], v[1], v[2], s1, c1);
        full_add(v[3], v[4], v[5], s2, c2);
        full_add(v[6], v[7], v[8], s3, c3);
        full_add(s1, s2, s3, S, C);   // count = S + 2 (C + c1 + c2 + c3)
        full_add(c1, c2, c3, t1, t2); // c1 + c2 + c3 = t1 + 2 t2
        // twos = C + t1 + 2 t2; count >= 5 iff twos >= 3, or twos >= 2 and S
        const uint32_t ge3 = t2 & (C | t1);
        const uint32_t ge2 = t2 | (C & t1);
        if (i < nf) out[static_cast<int64_t>(f0 + i) * nw + w] = (ge3 | (ge2 & S)) & rmask;
    }
}

}  // namespace

cdmd_status launch_median3x3(const uint32_t* mask, int64_t W, int64_t H, int n, uint32_t* out, cudaStream_t stream) {
    const int64_t m = W * H;
    const int64_t nw = (m + 31) / 32;
    const dim3 grid(static_cast<unsigned>((nw + kMedianThreads - 1) / kMedianThreads),
                    static_cast<unsigned>((n + kMedianFrames - 1) / kMedianFrames));
    median3x3_kernel<<<grid, kMedianThreads, 0, stream>>>(mask, out, static_cast<uint32_t>(W),
                                                          static_cast<uint32_t>(m), nw, n);
    CDMD_CHECK_LAUNCH("median3x3_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
