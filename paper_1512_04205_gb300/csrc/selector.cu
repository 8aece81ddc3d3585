// Learned background-mode selector: training (loss gradient + Adam), batch
// inference, feature export and the in-decompose selection.
//
// The paper chooses the background modes by sparse coding (Section 2.3,
// Eq. sparsecoding, applied to the compressed modes in Remark 3).  The
// selector scores every mode with a 2-layer MLP over four per-mode features
// (selector_common.cuh), keeps the K best, and hands them to the Gram-form
// least-squares solver of the decomposition; when the fitted residual exceeds
// the model's tolerance the sparse-coding solver runs instead.
//
// Training kernels:
//   mlp_grad_kernel   one warp per row at a time, lane u owns hidden units u
//                     and u + 32, so the backward pass accumulates every
//                     gradient entry in registers; each warp writes one
//                     partial gradient (385 values + loss)
//   mlp_update_kernel one CTA per parameter reduces the partials in a fixed
//                     order in FP64 (deterministic), divides by N, then
//                     either stores the gradient or applies one Adam step
//                     (Kingma & Ba, Algorithm 1)
#include "cdmd_internal.cuh"
#include "selector_common.cuh"

namespace cdmd {
namespace {

using namespace sel;

constexpr int kPart = kParams + 1;   // gradient entries + loss
constexpr int kGradThreads = 256;
constexpr int kUpdateThreads = 256;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(kGradThreads)
mlp_grad_kernel(const float* __restrict__ blob, const float* __restrict__ X, const float* __restrict__ Y,
                int64_t N, float* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    float mu[kFeat], sd[kFeat];
#pragma unroll
    for (int i = 0; i < kFeat; ++i) {
        mu[i] = blob[i];
        sd[i] = blob[4 + i];
    }
    float w1[2][kFeat], b1[2], w2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int u = lane + 32 * q;
#pragma unroll
        for (int i = 0; i < kFeat; ++i) w1[q][i] = blob[kOffW1 + u * kFeat + i];
        b1[q] = blob[kOffB1 + u];
        w2[q] = blob[kOffW2 + u];
    }
    const float b2 = blob[kOffB2];
    float gW1[2][kFeat] = {}, gb1[2] = {}, gw2[2] = {};
    float gb2 = 0.0f, loss = 0.0f;
    for (int64_t row = gw; row < N; row += nw) {
        float xh[kFeat];
#pragma unroll
        for (int i = 0; i < kFeat; ++i) xh[i] = (X[row * kFeat + i] - mu[i]) / sd[i];
        float hp[2], h[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            hp[q] = b1[q];
#pragma unroll
            for (int i = 0; i < kFeat; ++i) hp[q] = fmaf(w1[q][i], xh[i], hp[q]);
            h[q] = fmaxf(hp[q], 0.0f);
        }
        const float s = warp_sum_f(fmaf(w2[0], h[0], w2[1] * h[1])) + b2;
        const float y = Y[row];
        const float ds = 1.0f / (1.0f + expf(-s)) - y;   // dL/ds times N
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            gw2[q] = fmaf(ds, h[q], gw2[q]);
            const float dh = hp[q] > 0.0f ? ds * w2[q] : 0.0f;
            gb1[q] += dh;
#pragma unroll
            for (int i = 0; i < kFeat; ++i) gW1[q][i] = fmaf(dh, xh[i], gW1[q][i]);
        }
        gb2 += ds;
        loss += fmaxf(s, 0.0f) + log1pf(expf(-fabsf(s))) - y * s;
    }
    float* out = part + gw * kPart;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int u = lane + 32 * q;
#pragma unroll
        for (int i = 0; i < kFeat; ++i) out[u * kFeat + i] = gW1[q][i];
        out[kHidden * kFeat + u] = gb1[q];
        out[kHidden * kFeat + kHidden + u] = gw2[q];
    }
    if (lane == 0) {
        out[kParams - 1] = gb2;
        out[kParams] = loss;
    }
}

// One CTA per entry t of the partial rows: fixed-order FP64 reduction, then
// grad[t] (apply == 0) or an Adam step on parameter t (apply == 1).
__global__ void __launch_bounds__(kUpdateThreads)
mlp_update_kernel(const float* __restrict__ part, int64_t nparts, int64_t N, int apply, float* blob,
                  float* m, float* v, int step, float lr, float beta1, float beta2, float eps,
                  float* grad, float* loss) {
    __shared__ double red[kUpdateThreads];
    const int t = blockIdx.x;
    double acc = 0.0;
    for (int64_t p = threadIdx.x; p < nparts; p += kUpdateThreads) acc += static_cast<double>(part[p * kPart + t]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kUpdateThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double g = red[0] / static_cast<double>(N);
    if (t == kParams) {
        if (loss != nullptr) *loss = static_cast<float>(g);
        return;
    }
    if (!apply) {
        grad[t] = static_cast<float>(g);
        return;
    }
    const float gf = static_cast<float>(g);
    const float mt = beta1 * m[t] + (1.0f - beta1) * gf;
    const float vt = beta2 * v[t] + (1.0f - beta2) * gf * gf;
    m[t] = mt;
    v[t] = vt;
    const float bc1 = static_cast<float>(1.0 - pow(static_cast<double>(beta1), step));
    const float bc2 = static_cast<float>(1.0 - pow(static_cast<double>(beta2), step));
    const float mhat = mt / bc1;
    const float vhat = vt / bc2;
    blob[kHeader + t] -= lr * mhat / (sqrtf(vhat) + eps);
}

// Batch inference: one thread per row, the model in shared memory.
__global__ void mlp_forward_kernel(const float* __restrict__ blob, const float* __restrict__ X, int64_t N,
                                   int bf16, float* __restrict__ s_out, float* __restrict__ p_out) {
    __shared__ float wsm[kBlob];
    for (int i = threadIdx.x; i < kBlob; i += blockDim.x) wsm[i] = blob[i];
    __syncthreads();
    const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= N) return;
    float f[kFeat], xh[kFeat];
#pragma unroll
    for (int i = 0; i < kFeat; ++i) f[i] = X[row * kFeat + i];
    normalise(wsm, f, bf16 != 0, xh);
    const float s = mlp_logit(wsm, xh, bf16 != 0);
    if (s_out != nullptr) s_out[row] = s;
    if (p_out != nullptr) p_out[row] = 1.0f / (1.0f + expf(-s));
}

// Features of lane j's mode from the decomposition's Gram quantities:
// M (column-major r x r complex, M[a][c] at 2 (c r + a)), cvec, R_00.
__device__ __forceinline__ void lane_features(int lane, int r, const double* lam, const double* M,
                                              const double* cvec, const double* R, float f[kFeat]) {
    const bool live = lane < r;
    const double mjj = live ? M[2 * (static_cast<int64_t>(lane) * r + lane)] : 0.0;
    const double nmax = warp_max_d(live ? sqrt(fmax(mjj, 0.0)) : 0.0);
    if (live) {
        mode_features(lam[2 * lane], lam[2 * lane + 1], mjj, cvec[2 * lane], cvec[2 * lane + 1], nmax, R[0], f);
    } else {
#pragma unroll
        for (int i = 0; i < kFeat; ++i) f[i] = 0.0f;
    }
}

__global__ void __launch_bounds__(32)
selector_features_kernel(const double* __restrict__ lam, const double* __restrict__ M,
                         const double* __restrict__ cvec, const double* __restrict__ R, int r,
                         const int32_t* __restrict__ sel, int K, float* __restrict__ feats,
                         float* __restrict__ labels) {
    const int lane = threadIdx.x;
    float f[kFeat];
    lane_features(lane, r, lam, M, cvec, R, f);
    if (lane >= r) return;
#pragma unroll
    for (int i = 0; i < kFeat; ++i) feats[lane * kFeat + i] = f[i];
    if (labels != nullptr) {
        float y = 0.0f;
        for (int q = 0; q < K; ++q)
            if (sel[q] == lane) y = 1.0f;
        labels[lane] = y;
    }
}

// Scores every mode (BF16 inference) and writes the pick order: order[q] is
// the mode of rank q (descending logit, equal logits by index) for q < K,
// -1 after.
__global__ void __launch_bounds__(32)
mlp_select_kernel(const float* __restrict__ blob, const double* __restrict__ lam, const double* __restrict__ M,
                  const double* __restrict__ cvec, const double* __restrict__ R, int r, int K,
                  int32_t* __restrict__ order) {
    const int lane = threadIdx.x;
    float f[kFeat], xh[kFeat];
    lane_features(lane, r, lam, M, cvec, R, f);
    float s = -INFINITY;
    if (lane < r) {
        normalise(blob, f, true, xh);
        s = mlp_logit(blob, xh, true);
        if (isnan(s)) s = -INFINITY;
    }
    int rank = 0;
    for (int i = 0; i < r; ++i) {
        const float si = __shfl_sync(0xffffffffu, s, i);
        if (i != lane && (si > s || (si == s && i < lane))) ++rank;
    }
    const int kc = min(K, r);
    if (lane >= kc) order[lane] = -1;
    if (lane < r && rank < kc) order[rank] = lane;
}

}  // namespace

cdmd_status launch_selector_features(cdmd_ctx* ctx, const double* lambda, const int32_t* sel, int r, int K,
                                     float* feats, float* labels, cudaStream_t stream) {
    selector_features_kernel<<<1, 32, 0, stream>>>(lambda, ctx->last_M, ctx->last_cvec, ctx->last_R, r, sel, K,
                                                   feats, labels);
    CDMD_CHECK_LAUNCH("selector_features_kernel");
    return CDMD_OK;
}

cdmd_status launch_mlp_select(cdmd_ctx* ctx, const double* lambda, const double* M, const double* cvec,
                              const double* R, int r, int K, cudaStream_t stream) {
    mlp_select_kernel<<<1, 32, 0, stream>>>(selector_blob(ctx), lambda, M, cvec, R, r, K, selector_order(ctx));
    CDMD_CHECK_LAUNCH("mlp_select_kernel");
    return CDMD_OK;
}

cdmd_status launch_mlp_forward(cdmd_ctx* ctx, const float* blob, const float* X, int64_t N, int bf16,
                               float* s, float* p, cudaStream_t stream) {
    (void)ctx;
    if (N == 0) return CDMD_OK;
    const int threads = 256;
    mlp_forward_kernel<<<static_cast<unsigned>((N + threads - 1) / threads), threads, 0, stream>>>(blob, X, N, bf16,
                                                                                                 s, p);
    CDMD_CHECK_LAUNCH("mlp_forward_kernel");
    return CDMD_OK;
}

cdmd_status launch_mlp_train(cdmd_ctx* ctx, int apply, float* blob, float* m, float* v, int step, float lr,
                             float beta1, float beta2, float eps, const float* X, const float* Y, int64_t N,
                             float* grad, float* loss, cudaStream_t stream) {
    const int64_t warps_per_block = kGradThreads / 32;
    // a few rows per warp, at most four CTAs per SM
    int64_t blocks = (N + warps_per_block * 4 - 1) / (warps_per_block * 4);
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, static_cast<int64_t>(ctx->num_sms) * 4));
    const int64_t nparts = blocks * warps_per_block;
    void* buf = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_MLP_PARTS, static_cast<size_t>(nparts) * kPart * sizeof(float), &buf);
    if (st != CDMD_OK) return st;
    float* part = static_cast<float*>(buf);
    mlp_grad_kernel<<<static_cast<unsigned>(blocks), kGradThreads, 0, stream>>>(blob, X, Y, N, part);
    CDMD_CHECK_LAUNCH("mlp_grad_kernel");
    mlp_update_kernel<<<kPart, kUpdateThreads, 0, stream>>>(part, nparts, N, apply, blob, m, v, step, lr, beta1,
                                                            beta2, eps, grad, loss);
    CDMD_CHECK_LAUNCH("mlp_update_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
