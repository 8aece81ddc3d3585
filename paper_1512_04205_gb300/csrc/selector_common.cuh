// Learned background-mode selector: model layout, per-mode features and the
// network's logit, shared by the training, batch-inference and in-decompose
// selection kernels so that every path computes the same numbers.
//
// Features of mode j (Section 2.2 relates background modes to |lambda| near 1
// and arg lambda near 0; the compressed modes are those of Section 3.2):
//   f0 = max(log|lambda_j|, -30)
//   f1 = |arg lambda_j|                      (conjugate pairs share features)
//   f2 = max(log(||phi_j|| / max_i ||phi_i||), -30)
//   f3 = |phi_j^H y1| / (||phi_j|| ||y1||)
// taken in Gram form: ||phi_j||^2 = M_jj with M = Phi_Y^H Phi_Y, and
// phi_j^H y1 = cvec_j, ||y1||^2 = R_00.
//
// Network: xh = (f - mu) / sd; h = relu(W1 xh + b1) (64 units); s = w2.h + b2.
// Model blob (FP32): mu[4] sd[4] tol pad[3] | W1[64][4] b1[64] w2[64] b2.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace cdmd {
namespace sel {

constexpr int kFeat = 4;
constexpr int kHidden = 64;
constexpr int kParams = kHidden * kFeat + kHidden + kHidden + 1;   // 385
constexpr int kHeader = 12;
constexpr int kBlob = kHeader + kParams;                           // 397
constexpr int kOffW1 = kHeader;
constexpr int kOffB1 = kOffW1 + kHidden * kFeat;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kHidden;
constexpr int kOffTol = 8;
constexpr double kFloor = -30.0;

__device__ __forceinline__ float bf16r(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// Features of one mode from its eigenvalue (lr, li), ||phi||^2 = mjj,
// phi^H y1 = (cr, ci), the largest ||phi|| over the modes and ||y1||^2.
__device__ __forceinline__ void mode_features(double lr, double li, double mjj, double cr, double ci,
                                              double nmax, double y2, float f[kFeat]) {
    const double absl = hypot(lr, li);
    const double nrm = sqrt(fmax(mjj, 0.0));
    f[0] = static_cast<float>(absl > 0.0 ? fmax(log(absl), kFloor) : kFloor);
    f[1] = static_cast<float>(fabs(atan2(li, lr)));
    f[2] = static_cast<float>((nrm > 0.0 && nmax > 0.0) ? fmax(log(nrm / nmax), kFloor) : kFloor);
    const double den = nrm * sqrt(fmax(y2, 0.0));
    f[3] = static_cast<float>(den > 0.0 ? hypot(cr, ci) / den : 0.0);
}

// Normalised input of the network; rounded to BF16 for BF16 inference.
__device__ __forceinline__ void normalise(const float* blob, const float f[kFeat], bool bf16,
                                          float xh[kFeat]) {
#pragma unroll
    for (int i = 0; i < kFeat; ++i) {
        const float v = (f[i] - blob[i]) / blob[4 + i];
        xh[i] = bf16 ? bf16r(v) : v;
    }
}

// Logit of one row: FP32 accumulation over the hidden units in index order;
// with bf16 every matrix operand (xh, W1, h, w2) is a BF16 value.
__device__ __forceinline__ float mlp_logit(const float* blob, const float xh[kFeat], bool bf16) {
    float acc = 0.0f;
    for (int u = 0; u < kHidden; ++u) {
        float hp = blob[kOffB1 + u];
#pragma unroll
        for (int i = 0; i < kFeat; ++i) {
            const float w = blob[kOffW1 + u * kFeat + i];
            hp = fmaf(bf16 ? bf16r(w) : w, xh[i], hp);
        }
        float h = fmaxf(hp, 0.0f);
        float w2 = blob[kOffW2 + u];
        if (bf16) {
            h = bf16r(h);
            w2 = bf16r(w2);
        }
        acc = fmaf(w2, h, acc);
    }
    return acc + blob[kOffB2];
}

}  // namespace sel
}  // namespace cdmd
