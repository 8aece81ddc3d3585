// Synthetic clip renderer: the training data of the learned selector is made
// on the device, one clip per call, never stored.  The scene is the recipe of
// the seeded input generator (textured low-rank background of plane waves,
// constant-intensity moving objects, global illumination drift, per-pixel
// sensor noise); the scene parameters come from the caller, the noise from
// Philox4x32-10 keyed by the clip's seed.
#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr float kTwoPi = 6.283185307179586f;

__global__ void synth_kernel(int W, int H, int n, const float* __restrict__ waves, int nw,
                             const float* __restrict__ objs, int nobj, int ellipse, float drift, float sigma,
                             uint2 key, uint8_t* __restrict__ D, int64_t ldd) {
    const int64_t m = static_cast<int64_t>(W) * H;
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (j >= m || t >= n) return;
    const float x = static_cast<float>(j % W), y = static_cast<float>(j / W);
    float v = 128.0f;
    for (int w = 0; w < nw; ++w) {
        const float amp = waves[4 * w], period = waves[4 * w + 1], th = waves[4 * w + 2], ph = waves[4 * w + 3];
        float s, c;
        sincosf(th, &s, &c);
        v += amp * sinf((x * c + y * s) * (kTwoPi / period) + ph);
    }
    const float xs = x + 0.5f, ys = y + 0.5f;
    for (int q = 0; q < nobj; ++q) {
        const float* o = objs + (static_cast<int64_t>(t) * nobj + q) * 5;
        const float dx = xs - o[0], dy = ys - o[1], hw = 0.5f * o[2], hh = 0.5f * o[3];
        bool inside;
        if (ellipse) {
            const float ex = dx / hw, ey = dy / hh;
            inside = ex * ex + ey * ey <= 1.0f;
        } else {
            inside = fabsf(dx) <= hw && fabsf(dy) <= hh;
        }
        if (inside) v = o[4];
    }
    if (drift != 0.0f && n > 1) v *= 1.0f + drift * (2.0f * static_cast<float>(t) / static_cast<float>(n - 1) - 1.0f);
    if (sigma > 0.0f) {
        const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(t), 4u, 0u), key);
        float zc, zs;
        box_muller_accurate(w.x, w.y, zc, zs);
        v += sigma * zc;
    }
    v = fminf(fmaxf(floorf(v + 0.5f), 0.0f), 255.0f);
    D[static_cast<int64_t>(t) * ldd + j] = static_cast<uint8_t>(v);
}

}  // namespace

cdmd_status launch_synth_clip(int width, int height, int n, const float* waves, int nw, const float* objects,
                              int nobj, int ellipse, float drift, float noise_sigma, uint64_t seed, uint8_t* D,
                              int64_t ldd, cudaStream_t stream) {
    const int64_t m = static_cast<int64_t>(width) * height;
    const int threads = 256;
    const dim3 grid(static_cast<unsigned>((m + threads - 1) / threads), static_cast<unsigned>(n));
    synth_kernel<<<grid, threads, 0, stream>>>(width, height, n, waves, nw, objects, nobj, ellipse, drift, noise_sigma,
                                               seed_key(seed), D, ldd);
    CDMD_CHECK_LAUNCH("synth_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
