// Small solves on the device, FP64 (Algorithm 1 steps 4-7 and 9, Remark 3).
//
// Everything after the sketch is derived from the n x n Gram matrix
// R = DY^T DY of the sketch (for exact DMD, R = D^T D of the video itself,
// computed by the snapshot Gram pass, and DY is never formed):
//   Y^T Y  = R[0:p, 0:p]     (p = n-1)      -> V, S   (SVD of Y, step 4)
//   Y^T Y' = R[0:p, 1:n]                     -> A~ = S^-1 V^T (Y^T Y') V S^-1 (step 6)
//   Y'^T Y'= R[1:n, 1:n], Y'^T y1 = R[1:n, 0] -> Gram form of the OMP on the
//            compressed modes Phi_Y = Y' G (Remark 3)
// so no kernel after the Gram touches the k-long sketch rows again.
//
// FP64 on this GPU is slow in both senses: about 1/64 of the FP32 FMA rate,
// 64 cycles for a dependent FMA and ~640 for a division or square root.  So
// the O(p^3) / O(p^2 r) stages are spread over SMs, serial chains are kept
// short (several independent accumulators, more lanes), divisions and square
// roots on critical paths become approximate reciprocals refined by Newton
// steps, and the one iteration-heavy r x r stage runs in FP32 with an FP64
// Newton correction per eigenpair:
//   gram_partial / gram_reduce   multi-CTA, split over the sketch rows
//   tridiag                      Householder tridiagonalisation of Y^T Y on a
//                                thread-block cluster, rows distributed over
//                                the CTAs' shared memory, vectors exchanged
//                                through distributed shared memory
//   tridiag_eigpair              one CTA per wanted eigenvalue: Sturm-count
//                                multisection (64 shifts per pass), then
//                                inverse iteration with reciprocal pivots
//   orthonormalise               classical Gram-Schmidt, twice (one CTA)
//   backtransform                one CTA per eigenvector: V = Q z
//   bmat, atilde                 B = (Y^T Y') V, A~ = S^-1 V^T B S^-1
//   eig_f32                      one warp: Hessenberg + complex-shift QR on A~
//                                in FP32, eigenvectors by back-substitution
//   eig_refine                   one CTA per eigenpair: FP64 Newton on
//                                (A~ - mu) w = 0 with one entry of w fixed
//   eig_order                    normalise, order (conjugate pairs adjacent)
//   gmat                         G = V S^-1 W
//   hmat                         H = (Y'^T Y') G, M = G^H H, c = G^H (Y'^T y1)
//   omp                          one warp: OMP / least squares in Gram form
//   phiy (optional)              Phi_Y = Y' G
#include <cooperative_groups.h>

#include "cdmd_internal.cuh"

namespace cg = cooperative_groups;

namespace cdmd {
namespace {

constexpr double kEps = 2.220446049250313e-16;
// An eigenvalue of Y^T Y at most kRankTol p eps times the largest is taken as
// zero (sigma_r of the sketch vanishes): the Gram and the reduction leave
// rounding of order (k + p) eps in them, so a bound of p eps alone would sit
// at the noise level of an exactly rank-deficient sketch.
constexpr double kRankTol = 64.0;
constexpr int kMaxR = 32;
constexpr size_t kMaxOptInSmem = 232448;      // opt-in shared memory per CTA

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; `red` holds >= 32 doubles of shared scratch.  All threads
// of the block must call it; every thread gets the total.
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const double out = red[0];
    __syncthreads();
    return out;
}

// complex helpers
struct cd {
    double x, y;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.x, -a.y}; }
__device__ __forceinline__ double cabs2(cd a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }
// 1/a for complex a != 0
__device__ __forceinline__ cd cinv(cd a) {
    const double s = rcp64(cabs2(a));
    return {a.x * s, -a.y * s};
}
__device__ __forceinline__ cd shfl_cd(cd v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// ---------------------------------------------------------------------------
// 1. Gram matrix R = DY^T DY (n x n), split over the k rows
// ---------------------------------------------------------------------------
constexpr int kGT = 32;

__global__ void __launch_bounds__(256)
gram_partial_kernel(const double* __restrict__ DY, int k, int n, int kchunk,
                    double* __restrict__ part) {
    const int ta = blockIdx.y, tb = blockIdx.x;
    if (ta > tb) return;
    __shared__ double As[kGT][kGT + 1];
    __shared__ double Bs[kGT][kGT + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int a0 = ta * kGT, b0 = tb * kGT;
    const int ibeg = blockIdx.z * kchunk;
    const int iend = min(k, ibeg + kchunk);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = ibeg; i0 < iend; i0 += kGT) {
        for (int idx = tid; idx < kGT * kGT; idx += 256) {
            const int ii = idx & 31, cc = idx >> 5;
            const int i = i0 + ii;
            As[ii][cc] = (i < iend && a0 + cc < n) ? DY[static_cast<int64_t>(a0 + cc) * k + i] : 0.0;
            Bs[ii][cc] = (i < iend && b0 + cc < n) ? DY[static_cast<int64_t>(b0 + cc) * k + i] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int ii = 0; ii < kGT; ++ii) {
            const double bv = Bs[ii][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(As[ii][ty + 8 * q], bv, acc[q]);
        }
        __syncthreads();
    }
    double* dst = part + static_cast<int64_t>(blockIdx.z) * n * n;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int a = a0 + ty + 8 * q, b = b0 + tx;
        if (a < n && b < n) dst[a * n + b] = acc[q];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int splits, int n,
                                   double* __restrict__ R, int* status) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int a = idx / n, b = idx % n;
    if (a / kGT > b / kGT) { const int t = a; a = b; b = t; }
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[static_cast<int64_t>(sp) * n * n + a * n + b];
    if (!isfinite(s)) record_status(status, CDMD_ERR_NONFINITE);
    R[idx] = s;
}

// ---------------------------------------------------------------------------
// 2. Householder tridiagonalisation of A = R[0:p, 0:p] on a cluster of P CTAs.
// Row i lives in CTA i % P (local slot i / P), full length p.  Step j:
//   the owner of row j (= column j by symmetry) has formed the reflector
//   H_j = I - tau v v^T with H_j A[j+1:, j] = alpha e_1 (v scaled to a
//   leading 1, tau in [1, 2]) and written v and tau
//   into every CTA (distributed shared memory, buffer j % 2);
//   barrier; every CTA forms u_i = (A v)_i on its rows i > j and its share
//   of v^T u, and writes them into every CTA;
//   barrier; every CTA forms w = tau u - (tau^2/2)(v^T u) v and applies the
//   rank-2 update A -= v w^T + w v^T to its rows.  The owner of row j+1
//   updates that row first and forms the next reflector into the other
//   buffer while the rest of the cluster is still updating, so the next
//   step starts right after one barrier.
// Two cluster barriers per step, the same sequence in every CTA.
// Outputs: diagonal dd[p], off-diagonal ee[p-1], reflectors Hv[j*p + l]
// (l > j) and htau[j], with A = Q T Q^T, Q = H_0 H_1 ... H_{p-3}.
// ---------------------------------------------------------------------------
constexpr int kTriThreads = 512;

// Reflector of step j from the owner's copy of row j, formed by one warp
// (the other warps of the owning CTA keep updating their rows meanwhile):
// tail2 = sum_{l > j+1} row[l]^2 (the caller's partial sums per lane), then v
// (entries j+1..p-1) and tau go into buffer `b` of every CTA, and the step's
// outputs to global memory.
__device__ void tri_reflector_warp(cg::cluster_group& cluster, int P, const double* row, int j, int p,
                                   double tail_part, double* vbuf, double* tau_slot, int b, double* Hv,
                                   double* htau, double* dd, double* ee) {
    const int lane = threadIdx.x & 31;
    const double tail2 = warp_sum(tail_part);
    const double x0 = row[j + 1];
    // scaled form: v = (1, x_{j+2} / v0, ...), tau = 2 v0^2 / (v0^2 + tail2)
    // in [1, 2], so neither grows however small the column is
    double alpha, tau, inv_v0;
    if (!(tail2 > 1e-280)) {              // nothing below the sub-diagonal (or a subnormal remainder)
        alpha = x0;
        tau = 0.0;
        inv_v0 = 0.0;
    } else {
        const double s2 = fma(x0, x0, tail2);
        const double nrm = s2 * rsqrt64(s2);
        alpha = (x0 >= 0.0) ? -nrm : nrm;
        const double v0 = x0 - alpha;     // |v0| >= nrm > 0
        inv_v0 = rcp64(v0);
        tau = 2.0 * rcp64(fma(tail2 * inv_v0, inv_v0, 1.0));
    }
    const int L = p - j - 1;
    for (int l = j + 1 + lane; l < p; l += 32) {
        const double val = (tau == 0.0) ? 0.0 : ((l == j + 1) ? 1.0 : row[l] * inv_v0);
        Hv[static_cast<int64_t>(j) * p + l] = val;
        for (int rr = 0; rr < P; ++rr) *cluster.map_shared_rank(vbuf + b * p + l, rr) = val;
    }
    (void)L;
    if (lane < P) *cluster.map_shared_rank(tau_slot + b, lane) = tau;
    if (lane == 0) {
        dd[j] = row[j];
        ee[j] = alpha;
        htau[j] = tau;
    }
}

__global__ void __launch_bounds__(kTriThreads)
tridiag_kernel(const double* __restrict__ R, int n, int p, double* __restrict__ Hv,
               double* __restrict__ htau, double* __restrict__ dd, double* __restrict__ ee) {
    cg::cluster_group cluster = cg::this_cluster();
    const int P = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int rows_per = (p + P - 1) / P;
    extern __shared__ double sm[];
    double* Aloc = sm;                                          // rows_per * p
    double* vbuf = Aloc + static_cast<size_t>(rows_per) * p;   // 2 * p
    double* ubuf = vbuf + 2 * p;                                // p: u gathered from every CTA
    double* wv = ubuf + p;                                      // p
    double* red = wv + p;                                       // 32 scratch
    double* slot = red + 32;                                    // 32: each CTA's share of v^T u
    double* tau_slot = slot + 32;                               // 2
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = kTriThreads / 32;

    for (int idx = tid; idx < rows_per * p; idx += kTriThreads) {
        const int li = idx / p, l = idx % p;
        const int i = rank + P * li;
        Aloc[idx] = (i < p) ? R[static_cast<int64_t>(i) * n + l] : 0.0;
    }
    // every CTA of the cluster has started (and loaded its rows) before any
    // CTA writes into another's shared memory
    cluster.sync();
    if (rank == 0 && wid == 0) {
        double tp = 0.0;
        for (int l = 2 + lane; l < p; l += 32) tp = fma(Aloc[l], Aloc[l], tp);
        tri_reflector_warp(cluster, P, Aloc, 0, p, tp, vbuf, tau_slot, 0, Hv, htau, dd, ee);
    }
    cluster.sync();

    for (int j = 0; j + 2 < p; ++j) {
        const int b = j & 1;
        const double* v = vbuf + b * p;
        const double tau = tau_slot[b];
        // local rows i > j start at li_first
        const int li_first = (j + 1 > rank) ? (j + 1 - rank + P - 1) / P : 0;
        if (tau != 0.0) {
            // u_i = sum_l A_il v_l on own rows (one warp per row), broadcast to every CTA
            double part = 0.0;
            for (int li = li_first + wid; li < rows_per; li += nwarps) {
                const int i = rank + P * li;
                if (i >= p) break;
                const double* row = Aloc + static_cast<size_t>(li) * p;
                double s0 = 0.0, s1 = 0.0;
                int l = j + 1 + lane;
                for (; l + 32 < p; l += 64) {
                    s0 = fma(row[l], v[l], s0);
                    s1 = fma(row[l + 32], v[l + 32], s1);
                }
                if (l < p) s0 = fma(row[l], v[l], s0);
                const double u = warp_sum(s0 + s1);
                if (lane < P) *cluster.map_shared_rank(ubuf + i, lane) = u;
                part = fma(v[i], u, part);
            }
            if (lane == 0) red[wid] = part;
            __syncthreads();
            if (tid < P) {
                double t = 0.0;
                for (int q = 0; q < nwarps; ++q) t += red[q];
                *cluster.map_shared_rank(slot + rank, tid) = t;
            }
        }
        cluster.sync();
        const int nxt = j + 1;
        const bool own_next = (nxt + 2 < p) && (nxt % P == rank);
        const int li_next = nxt / P;
        if (tau != 0.0) {
            double vtu = 0.0;
            for (int q = 0; q < P; ++q) vtu += slot[q];
            const double kc = 0.5 * tau * tau * vtu;
            for (int l = j + 1 + tid; l < p; l += kTriThreads) wv[l] = fma(tau, ubuf[l], -kc * v[l]);
            __syncthreads();
            if (own_next && wid == 0) {
                // warp 0: the next reflector's row first, then the reflector
                double* row = Aloc + static_cast<size_t>(li_next) * p;
                const double vi = v[nxt], wi = wv[nxt];
                double tp = 0.0;
                for (int l = j + 1 + lane; l < p; l += 32) {
                    const double a = fma(-vi, wv[l], fma(-wi, v[l], row[l]));
                    row[l] = a;
                    if (l > nxt + 1) tp = fma(a, a, tp);
                }
                __syncwarp();
                tri_reflector_warp(cluster, P, row, nxt, p, tp, vbuf, tau_slot, b ^ 1, Hv, htau, dd, ee);
            } else {
                // the other rows (all warps, or warps 1.. on the owner of the next row)
                const int L = p - j - 1;
                const int nrows = rows_per - li_first;
                const bool own_split = own_next;
                const int t0 = own_split ? tid - 32 : tid;
                const int nt = own_split ? kTriThreads - 32 : kTriThreads;
                for (int idx = t0; idx < nrows * L; idx += nt) {
                    const int li = li_first + idx / L;
                    const int l = j + 1 + idx % L;
                    const int i = rank + P * li;
                    if (i >= p || (own_split && li == li_next)) continue;
                    double* a = Aloc + static_cast<size_t>(li) * p + l;
                    *a = fma(-v[i], wv[l], fma(-wv[i], v[l], *a));
                }
            }
        } else if (own_next && wid == 0) {
            const double* row = Aloc + static_cast<size_t>(li_next) * p;
            double tp = 0.0;
            for (int l = nxt + 2 + lane; l < p; l += 32) tp = fma(row[l], row[l], tp);
            tri_reflector_warp(cluster, P, row, nxt, p, tp, vbuf, tau_slot, b ^ 1, Hv, htau, dd, ee);
        }
        cluster.sync();
    }
    // trailing 2x2 block
    if (tid == 0) {
        for (int i = max(p - 2, 0); i < p; ++i) {
            if (i % P != rank) continue;
            const double* row = Aloc + static_cast<size_t>(i / P) * p;
            dd[i] = row[i];
            if (i + 1 < p) ee[i] = row[i + 1];
        }
    }
}

// p <= 2: the leading block of R is already tridiagonal (no reflectors).
__global__ void tiny_tridiag_kernel(const double* R, int n, int p, double* dd, double* ee, double* htau) {
    for (int i = 0; i < p; ++i) {
        dd[i] = R[i * n + i];
        if (i + 1 < p) ee[i] = R[i * n + i + 1];
        htau[i] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// 3. Eigenpairs of the symmetric tridiagonal T (d, e), the r largest.
// Sturm count N(x) = #eigenvalues < x = sign changes in the leading minors
// p_i(x) = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{-1} = 1).  Signs are read
// from the high words (no compare on the critical path); the pair (p_i,
// p_{i-1}) is rescaled by a power of two every eight steps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rescale_pair(double& a, double& b) {
    const int e = (__double2hiint(a) >> 20) & 0x7ff;
    if (e > 1023 + 400 || (e > 0 && e < 1023 - 400)) {
        const double s = __hiloint2double((2046 - e) << 20, 0);   // 2^(1023 - e)
        a *= s;
        b *= s;
    }
}

__device__ __forceinline__ void sturm_count2(const double* d, const double* e2, int p, double x0, double x1,
                                             int& n0, int& n1) {
    double a0 = d[0] - x0, a1 = d[0] - x1, b0 = 1.0, b1 = 1.0;
    int c0 = static_cast<int>(static_cast<unsigned>(__double2hiint(a0)) >> 31);
    int c1 = static_cast<int>(static_cast<unsigned>(__double2hiint(a1)) >> 31);
    for (int i = 1; i < p; ++i) {
        const double ei = e2[i - 1], di = d[i];
        const double t0 = fma(di - x0, a0, -ei * b0);
        const double t1 = fma(di - x1, a1, -ei * b1);
        c0 += static_cast<int>(static_cast<unsigned>(__double2hiint(t0) ^ __double2hiint(a0)) >> 31);
        c1 += static_cast<int>(static_cast<unsigned>(__double2hiint(t1) ^ __double2hiint(a1)) >> 31);
        b0 = a0;
        a0 = t0;
        b1 = a1;
        a1 = t1;
        if ((i & 7) == 0) {
            rescale_pair(a0, b0);
            rescale_pair(a1, b1);
        }
    }
    n0 = c0;
    n1 = c1;
}

constexpr int kShifts = 64;   // shifts tested per multisection pass (two per lane)

__global__ void __launch_bounds__(32)
tridiag_eigpair_kernel(const double* __restrict__ dd, const double* __restrict__ ee, int p, int r, double* lam,
                       double* Z, int* status) {
    extern __shared__ double tsm[];
    double* d = tsm;            // p
    double* e = d + p;          // p (e[p-1] = 0)
    double* e2 = e + p;         // p
    double* lmul = e2 + p;      // p: elimination multipliers
    double* udg = lmul + p;     // p: U diagonal
    double* u1 = udg + p;       // p: U first super-diagonal
    double* u2 = u1 + p;        // p: U second super-diagonal
    double* invd = u2 + p;      // p: 1 / U diagonal
    double* z = invd + p;       // p: iterate
    int* piv = reinterpret_cast<int*>(z + p);   // p
    const int w = blockIdx.x;
    const int lane = threadIdx.x;
    for (int i = lane; i < p; i += 32) {
        d[i] = dd[i];
        e[i] = (i + 1 < p) ? ee[i] : 0.0;
        e2[i] = e[i] * e[i];
    }
    __syncwarp();
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int i = lane; i < p; i += 32) {
        const double rad = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);
        lo = fmin(lo, d[i] - rad);
        hi = fmax(hi, d[i] + rad);
        tn = fmax(tn, fabs(d[i]) + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    }
    const double pad = 2.0 * kEps * tn + 1e-300;
    lo -= pad;
    hi += pad;
    const int idx = p - 1 - w;   // ascending index of the target eigenvalue
    bool converged = false;
    for (int it = 0; it < 40; ++it) {
        const double width = hi - lo;
        if (width <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)) + kEps * tn + 1e-300) { converged = true; break; }
        const double step = width * (1.0 / (kShifts + 1));
        int n0, n1;
        sturm_count2(d, e2, p, fma(step, static_cast<double>(lane + 1), lo),
                     fma(step, static_cast<double>(lane + 33), lo), n0, n1);
        const unsigned b0 = __ballot_sync(0xffffffffu, n0 > idx);
        const unsigned b1 = __ballot_sync(0xffffffffu, n1 > idx);
        const int f = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : kShifts);
        const double nlo = (f == 0) ? lo : fma(step, static_cast<double>(f), lo);
        const double nhi = (f == kShifts) ? hi : fma(step, static_cast<double>(f + 1), lo);
        if (nlo >= nhi || (nlo == lo && nhi == hi)) { converged = true; break; }
        lo = nlo;
        hi = nhi;
    }
    const double lambda = 0.5 * (lo + hi);
    if (!converged && lane == 0) record_status(status, CDMD_ERR_NOT_CONVERGED);
    if (lane == 0) lam[w] = lambda;
    if (!(lambda > kRankTol * static_cast<double>(p) * kEps * tn)) {
        // a numerically zero eigenvalue: sigma_r of the sketch vanishes
        if (lane == 0) record_status(status, CDMD_ERR_RANK_DEFICIENT);
        for (int i = lane; i < p; i += 32) Z[static_cast<int64_t>(w) * p + i] = (i == w) ? 1.0 : 0.0;
        return;
    }
    // inverse iteration: LU with partial pivoting of T - mu I, reciprocal pivots
    const double mu = lambda + kEps * tn;   // keeps T - mu I away from exact singularity
    const double tiny = kEps * tn + 1e-300;
    for (int i = lane; i < p; i += 32) {
        udg[i] = d[i] - mu;
        lmul[i] = e[i];
        u1[i] = e[i];
        u2[i] = 0.0;
        piv[i] = 0;
        // start vector: 1 + a hash of (i, w) in [0, 1)
        uint32_t h = (static_cast<uint32_t>(i) + 1u) * 0x9E3779B9u ^ (static_cast<uint32_t>(w) + 1u) * 0x85EBCA6Bu;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        z[i] = 1.0 + static_cast<double>(h & 0xffff) * (1.0 / 65536.0);
    }
    __syncwarp();
    if (lane == 0) {
        for (int i = 0; i + 1 < p; ++i) {
            if (fabs(udg[i]) >= fabs(lmul[i])) {
                if (udg[i] == 0.0) udg[i] = tiny;
                const double inv = rcp64(udg[i]);
                invd[i] = inv;
                const double fct = lmul[i] * inv;
                lmul[i] = fct;
                udg[i + 1] = fma(-fct, u1[i], udg[i + 1]);
            } else {
                const double inv = rcp64(lmul[i]);
                invd[i] = inv;
                const double fct = udg[i] * inv;
                udg[i] = lmul[i];
                lmul[i] = fct;
                const double tmp = u1[i];
                u1[i] = udg[i + 1];
                udg[i + 1] = fma(-fct, udg[i + 1], tmp);
                if (i + 2 < p) {
                    u2[i] = u1[i + 1];
                    u1[i + 1] = -fct * u1[i + 1];
                }
                piv[i] = 1;
            }
        }
        if (udg[p - 1] == 0.0) udg[p - 1] = tiny;
        invd[p - 1] = rcp64(udg[p - 1]);
    }
    for (int itr = 0; itr < 2; ++itr) {
        if (lane == 0) {
            for (int i = 0; i + 1 < p; ++i) {
                if (piv[i] == 0) {
                    z[i + 1] = fma(-lmul[i], z[i], z[i + 1]);
                } else {
                    const double tmp = z[i];
                    z[i] = z[i + 1];
                    z[i + 1] = fma(-lmul[i], z[i], tmp);
                }
            }
            z[p - 1] *= invd[p - 1];
            if (p > 1) z[p - 2] = fma(-u1[p - 2], z[p - 1], z[p - 2]) * invd[p - 2];
            for (int i = p - 3; i >= 0; --i) z[i] = fma(-u2[i], z[i + 2], fma(-u1[i], z[i + 1], z[i])) * invd[i];
        }
        __syncwarp();
        double s0 = 0.0;
        for (int i = lane; i < p; i += 32) s0 = fma(z[i], z[i], s0);
        const double nrm2 = warp_sum(s0);
        if (!(nrm2 > 0.0) || !isfinite(nrm2)) {
            if (lane == 0) record_status(status, CDMD_ERR_NOT_CONVERGED);
            break;
        }
        const double inv = rsqrt64(nrm2);
        for (int i = lane; i < p; i += 32) z[i] *= inv;
        __syncwarp();
    }
    for (int i = lane; i < p; i += 32) Z[static_cast<int64_t>(w) * p + i] = z[i];
}

// ---------------------------------------------------------------------------
// Target rank by the optimal hard threshold for singular values (Remark 2;
// Gavish and Donoho, unknown noise level): the singular values of Y are the
// square roots of the eigenvalues of T.  One warp finds the median of the q
// largest by multisection on Sturm counts, sets tau = omega * median and
// counts the eigenvalues above tau^2 with one more Sturm count.
// ---------------------------------------------------------------------------
__device__ double kth_eigenvalue(const double* d, const double* e2, int p, int idx, double lo, double hi, double tn,
                                 int* status) {
    const int lane = threadIdx.x & 31;
    bool converged = false;
    for (int it = 0; it < 40; ++it) {
        const double width = hi - lo;
        if (width <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)) + kEps * tn + 1e-300) { converged = true; break; }
        const double step = width * (1.0 / (kShifts + 1));
        int n0, n1;
        sturm_count2(d, e2, p, fma(step, static_cast<double>(lane + 1), lo),
                     fma(step, static_cast<double>(lane + 33), lo), n0, n1);
        const unsigned b0 = __ballot_sync(0xffffffffu, n0 > idx);
        const unsigned b1 = __ballot_sync(0xffffffffu, n1 > idx);
        const int f = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : kShifts);
        const double nlo = (f == 0) ? lo : fma(step, static_cast<double>(f), lo);
        const double nhi = (f == kShifts) ? hi : fma(step, static_cast<double>(f + 1), lo);
        if (nlo >= nhi || (nlo == lo && nhi == hi)) { converged = true; break; }
        lo = nlo;
        hi = nhi;
    }
    if (!converged && lane == 0) record_status(status, CDMD_ERR_NOT_CONVERGED);
    return 0.5 * (lo + hi);
}

__global__ void __launch_bounds__(32)
gd_rank_kernel(const double* __restrict__ dd, const double* __restrict__ ee, int p, int q, double omega, int r_max,
               int* r_out, double* tau_out, int* status) {
    extern __shared__ double gsm[];
    double* d = gsm;        // p
    double* e2 = d + p;     // p (e2[p-1] = 0)
    const int lane = threadIdx.x;
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int i = lane; i < p; i += 32) {
        const double e = (i + 1 < p) ? ee[i] : 0.0;
        const double em = (i > 0) ? ee[i - 1] : 0.0;
        d[i] = dd[i];
        e2[i] = e * e;
        const double rad = fabs(e) + fabs(em);
        lo = fmin(lo, dd[i] - rad);
        hi = fmax(hi, dd[i] + rad);
        tn = fmax(tn, fabs(dd[i]) + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    }
    __syncwarp();
    const double pad = 2.0 * kEps * tn + 1e-300;
    lo -= pad;
    hi += pad;
    // descending positions j0 <= j1 of the median of the q largest
    const int j0 = (q - 1) / 2, j1 = q / 2;
    const double l0 = kth_eigenvalue(d, e2, p, p - 1 - j0, lo, hi, tn, status);
    const double l1 = (j1 == j0) ? l0 : kth_eigenvalue(d, e2, p, p - 1 - j1, lo, hi, tn, status);
    const double ymed = 0.5 * (sqrt(fmax(l0, 0.0)) + sqrt(fmax(l1, 0.0)));
    const double tau = omega * ymed;
    int below, unused;
    sturm_count2(d, e2, p, tau * tau, tau * tau, below, unused);   // eigenvalues < tau^2
    if (lane == 0) {
        const int above = p - below;
        *r_out = above < 1 ? 1 : (above > r_max ? r_max : above);
        *tau_out = tau;
    }
}

// 4a. Classical Gram-Schmidt over the r columns of Z (descending eigenvalue
// order), applied twice: the dots of a column with all earlier columns are
// taken in parallel (one warp each).  Z is not __restrict__: threads read
// entries other threads wrote, ordered by __syncthreads.
__global__ void __launch_bounds__(1024)
orthonormalise_kernel(double* Z, int p, int r) {
    // classical Gram-Schmidt, twice, on the r columns held in shared memory
    extern __shared__ double osm[];
    double* Zs = osm;                         // r columns of p
    double* dots = Zs + static_cast<size_t>(r) * p;   // 32
    double* red = dots + 32;                  // 32
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < r * p; i += blockDim.x) Zs[i] = Z[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < r; ++c) {
            double* zc = Zs + static_cast<size_t>(c) * p;
            if (wid < c) {
                const double* zq = Zs + static_cast<size_t>(wid) * p;
                double s0 = 0.0, s1 = 0.0;
                int i = lane;
                for (; i + 32 < p; i += 64) {
                    s0 = fma(zq[i], zc[i], s0);
                    s1 = fma(zq[i + 32], zc[i + 32], s1);
                }
                if (i < p) s0 = fma(zq[i], zc[i], s0);
                const double s = warp_sum(s0 + s1);
                if (lane == 0) dots[wid] = s;
            }
            __syncthreads();
            double nacc = 0.0;
            for (int i = threadIdx.x; i < p; i += blockDim.x) {
                double a0 = zc[i], a1 = 0.0;
                int q = 0;
                for (; q + 1 < c; q += 2) {
                    a0 = fma(-dots[q], Zs[static_cast<size_t>(q) * p + i], a0);
                    a1 = fma(-dots[q + 1], Zs[static_cast<size_t>(q + 1) * p + i], a1);
                }
                if (q < c) a0 = fma(-dots[q], Zs[static_cast<size_t>(q) * p + i], a0);
                const double a = a0 + a1;
                zc[i] = a;
                nacc = fma(a, a, nacc);
            }
            const double nrm2 = block_sum(nacc, red);
            const double inv = nrm2 > 0.0 ? rsqrt64(nrm2) : 0.0;
            for (int i = threadIdx.x; i < p; i += blockDim.x) zc[i] *= inv;
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < r * p; i += blockDim.x) Z[i] = Zs[i];
}

// 4b. V[:, c] = Q z_c (apply H_{p-3}, ..., H_0) and sigma_c = sqrt(lambda_c);
// one CTA (one warp) per column, four partial sums per lane.  Each lane
// holds its entries of the next reflector in registers, loaded one step
// ahead, so the L2 latency of the reflector rows is off the critical path.
// kBtPer: reflector entries per lane, 8 for p <= 256 and 16 up to p = 511
template <int kBtPer>
__global__ void __launch_bounds__(32)
backtransform_kernel(const double* __restrict__ Z, const double* __restrict__ Hv,
                     const double* __restrict__ htau, const double* __restrict__ lam, int p, int r,
                     double* __restrict__ V, double* __restrict__ sigma, int* status) {
    extern __shared__ double ysm[];   // p
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    for (int i = lane; i < p; i += 32) ysm[i] = Z[static_cast<int64_t>(c) * p + i];
    __syncwarp();
    // entry q of lane: index lane + 32 q of the reflector row
    double cur[kBtPer], nxt[kBtPer];
    double tau_cur = 0.0, tau_nxt = 0.0;
    int j = p - 3;
    if (j >= 0) {
        tau_cur = htau[j];
#pragma unroll
        for (int q = 0; q < kBtPer; ++q) {
            const int l = lane + 32 * q;
            cur[q] = (l > j && l < p) ? Hv[static_cast<int64_t>(j) * p + l] : 0.0;
        }
    }
    for (; j >= 0; --j) {
        if (j > 0) {
            tau_nxt = htau[j - 1];
#pragma unroll
            for (int q = 0; q < kBtPer; ++q) {
                const int l = lane + 32 * q;
                nxt[q] = (l > j - 1 && l < p) ? Hv[static_cast<int64_t>(j - 1) * p + l] : 0.0;
            }
        }
        if (tau_cur != 0.0) {
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int q = 0; q < kBtPer; q += 2) {
                const int l0 = lane + 32 * q, l1 = l0 + 32;
                if (l0 < p) s0 = fma(cur[q], ysm[l0], s0);
                if (l1 < p) s1 = fma(cur[q + 1], ysm[l1], s1);
            }
            const double s = warp_sum(s0 + s1) * tau_cur;
#pragma unroll
            for (int q = 0; q < kBtPer; ++q) {
                const int l = lane + 32 * q;
                if (l > j && l < p) ysm[l] = fma(-s, cur[q], ysm[l]);
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < kBtPer; ++q) cur[q] = nxt[q];
        tau_cur = tau_nxt;
    }
    for (int i = lane; i < p; i += 32) V[static_cast<int64_t>(c) * p + i] = ysm[i];
    if (lane == 0) {
        const double l0 = lam[0];
        const double lc = lam[c];
        if (!(lc > kRankTol * static_cast<double>(p) * kEps * fabs(l0))) record_status(status, CDMD_ERR_RANK_DEFICIENT);
        sigma[c] = lc > 0.0 ? lc * rsqrt64(lc) : 0.0;
    }
}

// 4c. B[a][c] = sum_b R[a][b+1] V[b][c] = ((Y^T Y') V)[a][c]; one warp per entry.
__global__ void __launch_bounds__(256)
bmat_kernel(const double* __restrict__ R, const double* __restrict__ V, int n, int p, double* __restrict__ B) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * 8 + wid;
    const int c = blockIdx.y;
    if (a >= p) return;
    const double* row = R + static_cast<int64_t>(a) * n + 1;
    const double* vc = V + static_cast<int64_t>(c) * p;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < p; b += 64) {
        s0 = fma(row[b], vc[b], s0);
        s1 = fma(row[b + 32], vc[b + 32], s1);
    }
    if (b < p) s0 = fma(row[b], vc[b], s0);
    const double s = warp_sum(s0 + s1);
    if (lane == 0) B[static_cast<int64_t>(c) * p + a] = s;
}

// 5. A~[a][c] = V[:,a]^T B[:,c] / (sigma_a sigma_c), one CTA per column c.
__global__ void __launch_bounds__(32)
atilde_kernel(const double* __restrict__ V, const double* __restrict__ B,
              const double* __restrict__ sigma, int p, int r, double* __restrict__ At) {
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    const double* bc = B + static_cast<int64_t>(c) * p;
    for (int a = 0; a < r; ++a) {
        const double* va = V + static_cast<int64_t>(a) * p;
        double s = 0.0;
        for (int i = lane; i < p; i += 32) s = fma(va[i], bc[i], s);
        s = warp_sum(s);
        if (lane == 0) {
            const double den = sigma[a] * sigma[c];
            At[static_cast<int64_t>(c) * r + a] = den > 0.0 ? s * rcp64(den) : 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// 6. Eigen-decomposition of the real r x r A~ (r <= 32).
// 6a (FP32, one warp): Householder Hessenberg reduction, complex single-shift
//     QR (Wilkinson shift, bulge chase with Givens rotations) to a complex
//     Schur form, eigenvectors by back-substitution, W = Q Z X.
// 6b (FP64, one CTA per eigenpair): Newton's method on (A~ - mu I) w = 0 with
//     the largest entry of w held at 1: each step solves the bordered linear
//     system for (delta w, delta mu) by Gaussian elimination with partial
//     pivoting; quadratic convergence from the FP32 start.
// 6c (one warp): unit-norm eigenvectors with the largest-modulus entry real
//     positive; eigenvalues ordered by descending modulus, conjugate pairs
//     adjacent with the positive imaginary part first.
// ---------------------------------------------------------------------------
struct cf {
    float x, y;
};
__device__ __forceinline__ cf fmulc(cf a, cf b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cf faddc(cf a, cf b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cf fsubc(cf a, cf b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cf fconjc(cf a) { return {a.x, -a.y}; }
__device__ __forceinline__ float fabs2c(cf a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float fabsc(cf a) { return hypotf(a.x, a.y); }
__device__ __forceinline__ cf fdivc(cf a, cf b) {
    const float s = fabsf(b.x) + fabsf(b.y);
    const cf as = {a.x / s, a.y / s}, bs = {b.x / s, b.y / s};
    const float den = bs.x * bs.x + bs.y * bs.y;
    return {(as.x * bs.x + as.y * bs.y) / den, (as.y * bs.x - as.x * bs.y) / den};
}
__device__ __forceinline__ cf fsqrtc(cf a) {
    const float m = fabsc(a);
    if (m == 0.0f) return {0.0f, 0.0f};
    float re = sqrtf(0.5f * (m + fabsf(a.x)));
    float im = 0.5f * a.y / re;
    if (a.x < 0.0f) {
        const float t = re;
        re = fabsf(im);
        im = (a.y >= 0.0f) ? t : -t;
    }
    return {re, im};
}

__global__ void __launch_bounds__(32)
eig_f32_kernel(const double* __restrict__ At, int r, float2* __restrict__ lam32, float2* __restrict__ W32,
               int* fallback) {
    __shared__ float Hr[kMaxR][kMaxR + 1];
    __shared__ float Q[kMaxR][kMaxR + 1];
    __shared__ cf T[kMaxR][kMaxR + 1];
    __shared__ cf Zs[kMaxR][kMaxR + 1];
    __shared__ cf X[kMaxR][kMaxR + 1];
    __shared__ float hv[kMaxR];
    const int lane = threadIdx.x;
    for (int idx = lane; idx < r * r; idx += 32) {
        const int i = idx % r, c = idx / r;
        Hr[i][c] = static_cast<float>(At[static_cast<int64_t>(c) * r + i]);
        Q[i][c] = (i == c) ? 1.0f : 0.0f;
    }
    __syncwarp();
    for (int j = 0; j + 2 < r; ++j) {
        const float hj = (lane > j && lane < r) ? Hr[lane][j] : 0.0f;
        float nrm2 = hj * hj;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
        const float nrm = sqrtf(nrm2);
        const float x0 = Hr[j + 1][j];
        const float v0 = x0 + (x0 >= 0.0f ? nrm : -nrm);
        // ||v||^2 = v0^2 + (nrm^2 - x0^2)
        const float vn = fmaf(v0, v0, fmaxf(nrm2 - x0 * x0, 0.0f));
        const float beta = (nrm > 0.0f && vn > 0.0f) ? 2.0f / vn : 0.0f;
        __syncwarp();
        if (lane > j && lane < r) hv[lane] = (lane == j + 1) ? v0 : hj;
        __syncwarp();
        if (beta != 0.0f) {
            if (lane < r) {
                float s = 0.0f;
                for (int i = j + 1; i < r; ++i) s += hv[i] * Hr[i][lane];
                s *= beta;
                for (int i = j + 1; i < r; ++i) Hr[i][lane] -= s * hv[i];
            }
            __syncwarp();
            if (lane < r) {
                float s = 0.0f, sq = 0.0f;
                for (int c = j + 1; c < r; ++c) {
                    s += Hr[lane][c] * hv[c];
                    sq += Q[lane][c] * hv[c];
                }
                s *= beta;
                sq *= beta;
                for (int c = j + 1; c < r; ++c) {
                    Hr[lane][c] -= s * hv[c];
                    Q[lane][c] -= sq * hv[c];
                }
            }
            __syncwarp();
            if (lane >= j + 2 && lane < r) Hr[lane][j] = 0.0f;
        }
        __syncwarp();
    }
    for (int idx = lane; idx < r * r; idx += 32) {
        const int i = idx % r, c = idx / r;
        T[i][c] = {Hr[i][c], 0.0f};
        Zs[i][c] = {(i == c) ? 1.0f : 0.0f, 0.0f};
    }
    __syncwarp();
    const float eps32 = 1.1920929e-07f;
    int hi = r - 1, its = 0, total = 0;
    bool failed = false;
    while (hi > 0) {
        // deflation: the largest lo <= hi with a negligible T[lo][lo-1] (or 0)
        bool small = false;
        if (lane >= 1 && lane <= hi) {
            const float sc = fabsc(T[lane - 1][lane - 1]) + fabsc(T[lane][lane]);
            small = fabsc(T[lane][lane - 1]) <= eps32 * sc;
        }
        const unsigned sm_mask = __ballot_sync(0xffffffffu, small);
        const int lo = sm_mask ? 31 - __clz(sm_mask) : 0;
        if (lo > 0 && lane == 0) T[lo][lo - 1] = {0.0f, 0.0f};
        __syncwarp();
        if (lo == hi) { --hi; its = 0; continue; }
        ++its;
        ++total;
        if (its > 60 || total > 60 * r) { failed = true; break; }
        cf mu;
        {
            const cf a = T[hi - 1][hi - 1], b = T[hi - 1][hi], c = T[hi][hi - 1], dv = T[hi][hi];
            if (its % 11 == 0) {
                mu = {dv.x + fabsc(c), dv.y};
            } else {
                const cf half = {0.5f * (a.x - dv.x), 0.5f * (a.y - dv.y)};
                const cf bc = fmulc(b, c);
                const cf disc = fsqrtc(faddc(fmulc(half, half), bc));
                const cf s1 = faddc(half, disc), s2 = fsubc(half, disc);
                cf mu1 = dv, mu2 = dv;
                if (fabs2c(s1) > 0.0f) mu1 = fsubc(dv, fdivc(bc, s1));
                if (fabs2c(s2) > 0.0f) mu2 = fsubc(dv, fdivc(bc, s2));
                mu = (fabs2c(fsubc(mu1, dv)) <= fabs2c(fsubc(mu2, dv))) ? mu1 : mu2;
            }
        }
        // bulge chase: rotation q acts on rows q, q+1 (lanes = columns), then
        // on columns q, q+1 (lanes = rows) and on Z; the entry T[q+1][q-1]
        // the row rotation zeroes is written 0 by its lane
        for (int q = lo; q < hi; ++q) {
            cf x, y;
            if (q == lo) { x = fsubc(T[lo][lo], mu); y = T[lo + 1][lo]; }
            else { x = T[q][q - 1]; y = T[q + 1][q - 1]; }
            const float rr = sqrtf(fabs2c(x) + fabs2c(y));
            cf cg_ = {1.0f, 0.0f}, sg = {0.0f, 0.0f};
            if (rr > 0.0f) {
                const float inv = 1.0f / rr;
                cg_ = {x.x * inv, x.y * inv};
                sg = {y.x * inv, y.y * inv};
            }
            __syncwarp();
            const int col0 = max(q - 1, 0);
            if (lane >= col0 && lane < r) {
                const cf t0 = T[q][lane], t1 = T[q + 1][lane];
                T[q][lane] = faddc(fmulc(fconjc(cg_), t0), fmulc(fconjc(sg), t1));
                T[q + 1][lane] = (q > lo && lane == q - 1) ? cf{0.0f, 0.0f} : fsubc(fmulc(cg_, t1), fmulc(sg, t0));
            }
            __syncwarp();
            const int row1 = min(q + 3, hi + 1);
            if (lane < r) {
                if (lane < row1) {
                    const cf t0 = T[lane][q], t1 = T[lane][q + 1];
                    T[lane][q] = faddc(fmulc(t0, cg_), fmulc(t1, sg));
                    T[lane][q + 1] = fsubc(fmulc(t1, fconjc(cg_)), fmulc(t0, fconjc(sg)));
                }
                const cf z0 = Zs[lane][q], z1 = Zs[lane][q + 1];
                Zs[lane][q] = faddc(fmulc(z0, cg_), fmulc(z1, sg));
                Zs[lane][q + 1] = fsubc(fmulc(z1, fconjc(cg_)), fmulc(z0, fconjc(sg)));
            }
            __syncwarp();
        }
    }
    // a failed FP32 iteration hands the whole problem to the FP64 QR fallback
    if (lane == 0) *fallback = failed ? 1 : 0;
    __syncwarp();
    float tmax = 0.0f;
    for (int i = 0; i < r; ++i)
        for (int c = i; c < r; ++c) tmax = fmaxf(tmax, fabsc(T[i][c]));
    const float small = eps32 * fmaxf(tmax, 1e-30f);
    if (lane < r) {
        const int j = lane;
        for (int i = 0; i < r; ++i) X[i][j] = {i == j ? 1.0f : 0.0f, 0.0f};
        for (int i = j - 1; i >= 0; --i) {
            cf s = {0.0f, 0.0f};
            for (int q = i + 1; q <= j; ++q) s = faddc(s, fmulc(T[i][q], X[q][j]));
            cf den = fsubc(T[i][i], T[j][j]);
            if (fabsc(den) < small) den = {small, 0.0f};
            const cf v = fdivc(s, den);
            X[i][j] = {-v.x, -v.y};
        }
    }
    __syncwarp();
    if (lane < r) {
        const int j = lane;
        cf tmp[kMaxR];
        for (int i = 0; i < r; ++i) {
            cf s = {0.0f, 0.0f};
            for (int q = 0; q <= j; ++q) s = faddc(s, fmulc(Zs[i][q], X[q][j]));
            tmp[i] = s;
        }
        for (int i = 0; i < r; ++i) {
            float re = 0.0f, im = 0.0f;
            for (int q = 0; q < r; ++q) {
                re += Q[i][q] * tmp[q].x;
                im += Q[i][q] * tmp[q].y;
            }
            W32[static_cast<int64_t>(j) * r + i] = make_float2(re, im);
        }
        lam32[j] = make_float2(T[j][j].x, T[j][j].y);
    }
}

__global__ void __launch_bounds__(32)
eig_refine_kernel(const double* __restrict__ At, int r, const float2* __restrict__ lam32,
                  const float2* __restrict__ W32, double* __restrict__ lamR, double* __restrict__ WR, int* fallback) {
    __shared__ double A[kMaxR][kMaxR + 1];
    __shared__ cd Mx[kMaxR][kMaxR + 1];
    __shared__ cd wv[kMaxR];
    __shared__ cd rhs[kMaxR];
    __shared__ cd zz[kMaxR];
    __shared__ int perm[kMaxR];
    const int j = blockIdx.x;
    const int lane = threadIdx.x;
    for (int idx = lane; idx < r * r; idx += 32) {
        const int i = idx % r, c = idx / r;
        A[i][c] = At[static_cast<int64_t>(c) * r + i];
    }
    cd mu = {static_cast<double>(lam32[j].x), static_cast<double>(lam32[j].y)};
    cd w = {0.0, 0.0};
    if (lane < r) {
        const float2 v = W32[static_cast<int64_t>(j) * r + lane];
        w = {static_cast<double>(v.x), static_cast<double>(v.y)};
    }
    // hold the largest entry of w at 1
    double key = (lane < r) ? cabs2(w) : -1.0;
    const double kmax = warp_max(key);
    const unsigned at = __ballot_sync(0xffffffffu, key == kmax && lane < r);
    const int pidx = at ? __ffs(at) - 1 : 0;   // no candidate only with non-finite entries
    const cd wp = shfl_cd(w, pidx);
    if (kmax > 0.0) w = cmul(w, cinv(wp));
    if (lane == pidx) w = {1.0, 0.0};
    if (lane < r) wv[lane] = w;
    __syncwarp();
    bool done = false;
    for (int it = 0; it < 4 && !done; ++it) {
        // residual and the bordered matrix: column pidx replaced by -w
        if (lane < r) {
            cd res = {-mu.x * wv[lane].x + mu.y * wv[lane].y, -mu.x * wv[lane].y - mu.y * wv[lane].x};
            for (int c = 0; c < r; ++c) {
                res.x = fma(A[lane][c], wv[c].x, res.x);
                res.y = fma(A[lane][c], wv[c].y, res.y);
                Mx[lane][c] = (c == pidx) ? cd{-wv[lane].x, -wv[lane].y}
                                          : cd{A[lane][c] - (c == lane ? mu.x : 0.0), c == lane ? -mu.y : 0.0};
            }
            rhs[lane] = {-res.x, -res.y};
            perm[lane] = lane;
        }
        __syncwarp();
        // Gaussian elimination with partial pivoting; lane q owns logical row q
        for (int k = 0; k < r; ++k) {
            const double mag = (lane >= k && lane < r) ? cabs2(Mx[perm[lane]][k]) : -1.0;
            const double mbest = warp_max(mag);
            const unsigned bb = __ballot_sync(0xffffffffu, mag == mbest && lane >= k && lane < r);
            const int pk = bb ? __ffs(bb) - 1 : k;   // non-finite column: keep the order
            __syncwarp();
            if (lane == 0 && pk != k) {
                const int t = perm[k];
                perm[k] = perm[pk];
                perm[pk] = t;
            }
            __syncwarp();
            const int prow = perm[k];
            const cd pv = Mx[prow][k];
            if (cabs2(pv) == 0.0) continue;
            const cd inv = cinv(pv);
            if (lane > k && lane < r) {
                const int row = perm[lane];
                const cd l = cmul(Mx[row][k], inv);
                for (int c = k + 1; c < r; ++c) Mx[row][c] = csub(Mx[row][c], cmul(l, Mx[prow][c]));
                rhs[row] = csub(rhs[row], cmul(l, rhs[prow]));
            }
            __syncwarp();
        }
        // back substitution in logical order, column by column: lane i keeps
        // b_i = rhs[perm[i]]; z_q = b_q / U_qq goes to every lane, which
        // subtracts U_iq z_q from its b_i (the reciprocal pivots in parallel)
        {
            const int row_l = (lane < r) ? perm[lane] : 0;
            cd bl = (lane < r) ? rhs[row_l] : cd{0.0, 0.0};
            cd invu = {0.0, 0.0};
            if (lane < r) {
                const cd pv = Mx[row_l][lane];
                if (cabs2(pv) > 0.0) invu = cinv(pv);
            }
            for (int q = r - 1; q >= 0; --q) {
                const cd zq = shfl_cd(cmul(bl, invu), q);
                if (lane == q) zz[q] = zq;
                if (lane < q) bl = csub(bl, cmul(Mx[row_l][q], zq));
            }
            __syncwarp();
        }
        // update: z_pidx is the eigenvalue correction, the rest correct w
        const cd dmu = zz[pidx];
        double dw = 0.0;
        if (lane < r && lane != pidx) {
            wv[lane] = cadd(wv[lane], zz[lane]);
            dw = cabs2(zz[lane]);
        }
        mu = cadd(mu, dmu);
        dw = warp_max(dw);
        done = (cabs2(dmu) <= 1e-28 * cabs2(mu)) && (dw <= 1e-26) && it > 0;
        __syncwarp();
    }
    // no quadratic convergence (a cluster or a nearly defective pair): the
    // FP64 QR fallback recomputes every eigenpair
    if (!done && lane == 0) atomicExch(fallback, 1);
    if (lane == 0) {
        lamR[2 * j] = mu.x;
        lamR[2 * j + 1] = mu.y;
    }
    if (lane < r) {
        WR[2 * (static_cast<int64_t>(j) * r + lane)] = wv[lane].x;
        WR[2 * (static_cast<int64_t>(j) * r + lane) + 1] = wv[lane].y;
    }
}

// FP64 fallback of steps 6b/6c for the rare A~ on which the FP32 solve or
// the Newton refinement did not converge (clustered or nearly defective
// eigenvalues, e.g. a conjugate pair about to meet on the real axis), or whose
// refined eigenvalues coincide.  One CTA: Householder Hessenberg reduction,
// complex single-shift QR with Wilkinson shifts (exceptional shift every 11
// iterations) to a complex Schur form T = Z^H H Z, eigenvectors of T by
// back-substitution, W = Q Z X.  Returns at once when nothing was flagged.
__device__ __forceinline__ double cabsd(cd a) { return hypot(a.x, a.y); }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    const double sc = fabs(b.x) + fabs(b.y);
    const cd as = {a.x / sc, a.y / sc}, bs = {b.x / sc, b.y / sc};
    const double den = bs.x * bs.x + bs.y * bs.y;
    return {(as.x * bs.x + as.y * bs.y) / den, (as.y * bs.x - as.x * bs.y) / den};
}
__device__ __forceinline__ cd csqrt_(cd a) {
    const double m = cabsd(a);
    if (m == 0.0) return {0.0, 0.0};
    double re = sqrt(0.5 * (m + fabs(a.x)));
    double im = 0.5 * a.y / re;
    if (a.x < 0.0) {
        const double t = re;
        re = fabs(im);
        im = (a.y >= 0.0) ? t : -t;
    }
    return {re, im};
}

constexpr int kQrThreads = 64;
constexpr size_t kQrSmem = 2 * kMaxR * (kMaxR + 1) * sizeof(double) + 3 * kMaxR * (kMaxR + 1) * sizeof(cd);

__global__ void __launch_bounds__(kQrThreads)
eig_qr64_kernel(const double* __restrict__ At, int r, double* lamR, double* WR, int* fallback, int* status) {
    extern __shared__ double qsm[];
    typedef double RowD[kMaxR + 1];
    typedef cd RowC[kMaxR + 1];
    RowD* Hr = reinterpret_cast<RowD*>(qsm);
    RowD* Q = Hr + kMaxR;
    RowC* T = reinterpret_cast<RowC*>(Q + kMaxR);
    RowC* Zs = T + kMaxR;
    RowC* X = Zs + kMaxR;
    __shared__ double hv[kMaxR];
    __shared__ double scal[4];
    __shared__ cd rot[2];
    __shared__ int flag[2];
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    if (tid == 0) {
        int go = *fallback;
        for (int i = 0; i < r && !go; ++i)
            for (int q = i + 1; q < r && !go; ++q) {
                const cd li = {lamR[2 * i], lamR[2 * i + 1]}, lq = {lamR[2 * q], lamR[2 * q + 1]};
                const double tol = 1e-8 * fmax(1.0, cabsd(li));
                if (!(cabs2(csub(li, lq)) > tol * tol)) go = 1;   // coincident (or NaN) eigenvalues
            }
        flag[1] = go;
    }
    __syncthreads();
    if (!flag[1]) return;
    for (int idx = tid; idx < r * r; idx += nt) {
        const int i = idx % r, c = idx / r;
        Hr[i][c] = At[static_cast<int64_t>(c) * r + i];
        Q[i][c] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = 0; j + 2 < r; ++j) {
        if (tid == 0) {
            double nrm2 = 0.0;
            for (int i = j + 1; i < r; ++i) nrm2 += Hr[i][j] * Hr[i][j];
            const double nrm = sqrt(nrm2);
            if (nrm == 0.0) {
                scal[0] = 0.0;
            } else {
                for (int i = j + 1; i < r; ++i) hv[i] = Hr[i][j];
                hv[j + 1] += (Hr[j + 1][j] >= 0.0 ? nrm : -nrm);
                double vn = 0.0;
                for (int i = j + 1; i < r; ++i) vn += hv[i] * hv[i];
                scal[0] = vn > 0.0 ? 2.0 / vn : 0.0;
            }
        }
        __syncthreads();
        const double beta = scal[0];
        if (beta != 0.0) {
            for (int c = tid; c < r; c += nt) {
                double sacc = 0.0;
                for (int i = j + 1; i < r; ++i) sacc += hv[i] * Hr[i][c];
                sacc *= beta;
                for (int i = j + 1; i < r; ++i) Hr[i][c] -= sacc * hv[i];
            }
            __syncthreads();
            for (int i = tid; i < r; i += nt) {
                double sh = 0.0, sq = 0.0;
                for (int c = j + 1; c < r; ++c) {
                    sh += Hr[i][c] * hv[c];
                    sq += Q[i][c] * hv[c];
                }
                sh *= beta;
                sq *= beta;
                for (int c = j + 1; c < r; ++c) {
                    Hr[i][c] -= sh * hv[c];
                    Q[i][c] -= sq * hv[c];
                }
            }
            __syncthreads();
            for (int i = j + 2 + tid; i < r; i += nt) Hr[i][j] = 0.0;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < r * r; idx += nt) {
        const int i = idx % r, c = idx / r;
        T[i][c] = {Hr[i][c], 0.0};
        Zs[i][c] = {(i == c) ? 1.0 : 0.0, 0.0};
    }
    __syncthreads();
    int hi = r - 1, its = 0, total = 0;
    bool failed = false;
    while (hi > 0) {
        if (tid == 0) {
            int lo = hi;
            while (lo > 0) {
                const double sc = cabsd(T[lo - 1][lo - 1]) + cabsd(T[lo][lo]);
                if (cabsd(T[lo][lo - 1]) <= kEps * sc) { T[lo][lo - 1] = {0.0, 0.0}; break; }
                --lo;
            }
            flag[0] = lo;
        }
        __syncthreads();
        const int lo = flag[0];
        if (lo == hi) { --hi; its = 0; __syncthreads(); continue; }
        ++its;
        ++total;
        if (its > 60 || total > 60 * r) { failed = true; break; }
        if (tid == 0) {
            const cd a = T[hi - 1][hi - 1], b = T[hi - 1][hi], c = T[hi][hi - 1], d = T[hi][hi];
            cd mu;
            if (its % 11 == 0) {
                mu = {d.x + cabsd(c), d.y};
            } else {
                const cd half = {0.5 * (a.x - d.x), 0.5 * (a.y - d.y)};
                const cd bc = cmul(b, c);
                const cd disc = csqrt_(cadd(cmul(half, half), bc));
                const cd s1 = cadd(half, disc), s2 = csub(half, disc);
                cd mu1 = d, mu2 = d;
                if (cabs2(s1) > 0.0) mu1 = csub(d, cdiv(bc, s1));
                if (cabs2(s2) > 0.0) mu2 = csub(d, cdiv(bc, s2));
                mu = (cabs2(csub(mu1, d)) <= cabs2(csub(mu2, d))) ? mu1 : mu2;
            }
            rot[1] = mu;
        }
        __syncthreads();
        const cd mu = rot[1];
        for (int q = lo; q < hi; ++q) {
            if (tid == 0) {
                cd x, y;
                if (q == lo) { x = csub(T[lo][lo], mu); y = T[lo + 1][lo]; }
                else { x = T[q][q - 1]; y = T[q + 1][q - 1]; }
                const double rr = sqrt(cabs2(x) + cabs2(y));
                if (rr == 0.0) { rot[0] = {1.0, 0.0}; scal[1] = 0.0; scal[2] = 0.0; }
                else { rot[0] = {x.x / rr, x.y / rr}; scal[1] = y.x / rr; scal[2] = y.y / rr; }
            }
            __syncthreads();
            const cd cg_ = rot[0];
            const cd sg = {scal[1], scal[2]};
            const int col0 = max(q - 1, 0);
            for (int c = col0 + tid; c < r; c += nt) {
                const cd t0 = T[q][c], t1 = T[q + 1][c];
                T[q][c] = cadd(cmul(cconj(cg_), t0), cmul(cconj(sg), t1));
                T[q + 1][c] = csub(cmul(cg_, t1), cmul(sg, t0));
            }
            __syncthreads();
            const int row1 = min(q + 3, hi + 1);
            for (int i = tid; i < r; i += nt) {
                if (i < row1) {
                    const cd t0 = T[i][q], t1 = T[i][q + 1];
                    T[i][q] = cadd(cmul(t0, cg_), cmul(t1, sg));
                    T[i][q + 1] = csub(cmul(t1, cconj(cg_)), cmul(t0, cconj(sg)));
                }
                const cd z0 = Zs[i][q], z1 = Zs[i][q + 1];
                Zs[i][q] = cadd(cmul(z0, cg_), cmul(z1, sg));
                Zs[i][q + 1] = csub(cmul(z1, cconj(cg_)), cmul(z0, cconj(sg)));
            }
            __syncthreads();
            if (tid == 0 && q > lo) T[q + 1][q - 1] = {0.0, 0.0};
            __syncthreads();
        }
    }
    if (failed && tid == 0) record_status(status, CDMD_ERR_NOT_CONVERGED);
    if (tid == 0) {
        double tmax = 0.0;
        for (int i = 0; i < r; ++i)
            for (int c = i; c < r; ++c) tmax = fmax(tmax, cabsd(T[i][c]));
        scal[3] = kEps * fmax(tmax, 1e-300);
    }
    __syncthreads();
    const double small = scal[3];
    for (int j = tid; j < r; j += nt) {
        for (int i = 0; i < r; ++i) X[i][j] = {i == j ? 1.0 : 0.0, 0.0};
        for (int i = j - 1; i >= 0; --i) {
            cd acc = {0.0, 0.0};
            for (int q = i + 1; q <= j; ++q) acc = cadd(acc, cmul(T[i][q], X[q][j]));
            cd den = csub(T[i][i], T[j][j]);
            if (cabsd(den) < small) den = {small, 0.0};
            const cd v = cdiv(acc, den);
            X[i][j] = {-v.x, -v.y};
        }
        lamR[2 * j] = T[j][j].x;
        lamR[2 * j + 1] = T[j][j].y;
    }
    __syncthreads();
    // W = Q (Z X); column j by one thread (X upper triangular)
    for (int j = tid; j < r; j += nt) {
        cd zx[kMaxR];
        for (int q = 0; q < r; ++q) {
            cd acc = {0.0, 0.0};
            for (int u = 0; u <= j; ++u) acc = cadd(acc, cmul(Zs[q][u], X[u][j]));
            zx[q] = acc;
        }
        for (int i = 0; i < r; ++i) {
            double re = 0.0, im = 0.0;
            for (int q = 0; q < r; ++q) {
                re += Q[i][q] * zx[q].x;
                im += Q[i][q] * zx[q].y;
            }
            WR[2 * (static_cast<int64_t>(j) * r + i)] = re;
            WR[2 * (static_cast<int64_t>(j) * r + i) + 1] = im;
        }
    }
    if (tid == 0) *fallback = 0;
}

__global__ void __launch_bounds__(32)
eig_order_kernel(const double* __restrict__ lamR, const double* __restrict__ WR, int r, double* __restrict__ lam_out,
                 double* __restrict__ W_out) {
    __shared__ int order[kMaxR];
    const int lane = threadIdx.x;
    if (lane == 0) {
        bool used[kMaxR];
        double key_abs[kMaxR], key_im[kMaxR];
        int first[kMaxR], second[kMaxR];
        int nu = 0;
        for (int i = 0; i < r; ++i) used[i] = false;
        for (int pass = 0; pass < r; ++pass) {
            int i = -1;
            for (int q = 0; q < r; ++q)
                if (!used[q] && (i < 0 || lamR[2 * q + 1] > lamR[2 * i + 1])) i = q;
            if (i < 0) break;
            used[i] = true;
            const cd li = {lamR[2 * i], lamR[2 * i + 1]};
            int partner = -1;
            if (li.y > 0.0) {
                double bd = 1e300;
                for (int q = 0; q < r; ++q) {
                    if (used[q]) continue;
                    const cd lq = {lamR[2 * q], lamR[2 * q + 1]};
                    const double d2 = cabs2(csub(lq, cconj(li)));
                    if (d2 < bd) { bd = d2; partner = q; }
                }
                const double tol = 1e-9 * fmax(1.0, sqrt(cabs2(li)));
                if (partner >= 0 && !(bd <= tol * tol)) partner = -1;
                if (partner >= 0) used[partner] = true;
            }
            key_abs[nu] = cabs2(li);
            key_im[nu] = li.y;
            first[nu] = i;
            second[nu] = partner;
            ++nu;
        }
        int perm[kMaxR];
        for (int u = 0; u < nu; ++u) perm[u] = u;
        for (int u = 1; u < nu; ++u) {
            const int cur = perm[u];
            int v = u - 1;
            while (v >= 0) {
                const int o = perm[v];
                const bool before = (key_abs[cur] > key_abs[o]) || (key_abs[cur] == key_abs[o] && key_im[cur] > key_im[o]);
                if (!before) break;
                perm[v + 1] = perm[v];
                --v;
            }
            perm[v + 1] = cur;
        }
        int pos = 0;
        for (int u = 0; u < nu; ++u) {
            order[pos++] = first[perm[u]];
            if (second[perm[u]] >= 0) order[pos++] = second[perm[u]];
        }
    }
    __syncwarp();
    if (lane < r) {
        const int s = order[lane];
        lam_out[2 * lane] = lamR[2 * s];
        lam_out[2 * lane + 1] = lamR[2 * s + 1];
        // unit 2-norm, largest-modulus entry real positive
        double n2 = 0.0, best = -1.0;
        int bi = 0;
        for (int i = 0; i < r; ++i) {
            const cd v = {WR[2 * (static_cast<int64_t>(s) * r + i)], WR[2 * (static_cast<int64_t>(s) * r + i) + 1]};
            const double a2 = cabs2(v);
            n2 += a2;
            if (a2 > best) { best = a2; bi = i; }
        }
        const cd vb = {WR[2 * (static_cast<int64_t>(s) * r + bi)], WR[2 * (static_cast<int64_t>(s) * r + bi) + 1]};
        const double inv_b = best > 0.0 ? rsqrt64(best) : 0.0;
        const double inv_n = n2 > 0.0 ? rsqrt64(n2) : 0.0;
        const cd ph = {vb.x * inv_b * inv_n, -vb.y * inv_b * inv_n};   // conj(v_b)/|v_b| / ||v||
        for (int i = 0; i < r; ++i) {
            const cd v = {WR[2 * (static_cast<int64_t>(s) * r + i)], WR[2 * (static_cast<int64_t>(s) * r + i) + 1]};
            cd o = cmul(v, ph);
            if (i == bi) o.y = 0.0;
            W_out[2 * (static_cast<int64_t>(lane) * r + i)] = o.x;
            W_out[2 * (static_cast<int64_t>(lane) * r + i) + 1] = o.y;
        }
    }
}

// 7. G[t][c] = sum_a V[t][a] / sigma_a * W[a][c]   (column-major complex)
__global__ void gmat_kernel(const double* __restrict__ V, const double* __restrict__ sigma,
                            const double* __restrict__ W, int p, int r, double* __restrict__ G) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p * r) return;
    const int t = idx % p, c = idx / p;
    double re = 0.0, im = 0.0;
    for (int a = 0; a < r; ++a) {
        const double va = V[static_cast<int64_t>(a) * p + t] / sigma[a];
        re = fma(va, W[2 * (static_cast<int64_t>(c) * r + a)], re);
        im = fma(va, W[2 * (static_cast<int64_t>(c) * r + a) + 1], im);
    }
    G[2 * static_cast<int64_t>(idx)] = re;
    G[2 * static_cast<int64_t>(idx) + 1] = im;
}

// 8. h = (Y'^T Y') G[:, c];  M[a][c] = G[:,a]^H h;  cvec[c] = G[:,c]^H (Y'^T y1).
// One CTA of 16 warps per column c, one warp per row of h, then per entry.
__global__ void __launch_bounds__(512)
hmat_kernel(const double* __restrict__ R, const double* __restrict__ G, int n, int p, int r,
            double* __restrict__ M, double* __restrict__ cvec) {
    extern __shared__ double hsm[];   // h: 2p
    const int c = blockIdx.x;
    const double* gc = G + 2 * static_cast<int64_t>(c) * p;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = wid; t < p; t += nw) {
        const double* row = R + static_cast<int64_t>(t + 1) * n + 1;
        double re = 0.0, im = 0.0;
        for (int b = lane; b < p; b += 32) {
            re = fma(row[b], gc[2 * b], re);
            im = fma(row[b], gc[2 * b + 1], im);
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) { hsm[2 * t] = re; hsm[2 * t + 1] = im; }
    }
    __syncthreads();
    for (int a = wid; a <= r; a += nw) {
        // a < r: M[a][c]; a == r: cvec[c]
        double re = 0.0, im = 0.0;
        if (a < r) {
            const double* ga = G + 2 * static_cast<int64_t>(a) * p;
            for (int t = lane; t < p; t += 32) {
                const double gr = ga[2 * t], gi = ga[2 * t + 1];
                const double hr = hsm[2 * t], hi = hsm[2 * t + 1];
                re += gr * hr + gi * hi;   // conj(g) h
                im += gr * hi - gi * hr;
            }
        } else {
            for (int t = lane; t < p; t += 32) {
                const double y = R[static_cast<int64_t>(t + 1) * n];   // (Y'^T y1)_t
                re += gc[2 * t] * y;
                im -= gc[2 * t + 1] * y;
            }
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            if (a < r) {
                M[2 * (static_cast<int64_t>(c) * r + a)] = re;
                M[2 * (static_cast<int64_t>(c) * r + a) + 1] = im;
            } else {
                cvec[2 * c] = re;
                cvec[2 * c + 1] = im;
            }
        }
    }
}

// 9. OMP in Gram form, one warp (r <= 32; lane j owns mode j).  M = Phi_Y^H
// Phi_Y (Hermitian, column-major), cvec = Phi_Y^H y1, ||y1||^2 = R[0][0].
// Scores |phi_j^H rho|^2 / ||phi_j||^2 with phi_j^H rho = c_j - sum_q M[j][S_q]
// beta_q; ties (relative 2e-9 on the squared score, i.e. 1e-9 on the score)
// go to the largest Im(lambda), then the lowest index.  The least-squares fit
// on the selected set solves M_SS beta = c_S through a Cholesky factor
// M_SS = L L^H grown by one row per pick; every triangular solve is
// right-looking (one row per lane, one broadcast per step).
__global__ void __launch_bounds__(32)
omp_kernel(const double* __restrict__ M, const double* __restrict__ cvec, const double* __restrict__ R,
           const double* __restrict__ lam, int r, int K, int lstsq, double* __restrict__ beta,
           int32_t* __restrict__ sel, int32_t* __restrict__ nsel_out, int* status,
           const int32_t* __restrict__ order, const float* __restrict__ blob, int* accept,
           unsigned long long* fallbacks) {
    // Modes of operation:
    //   order == nullptr, accept == nullptr   greedy OMP (or lstsq over all r)
    //   order != nullptr                      least squares on the learned pick
    //                                         order; accepted (outputs written,
    //                                         *accept = 1) when the relative
    //                                         residual is within the model's tol,
    //                                         else *accept = 0 and one fallback
    //                                         is counted
    //   order == nullptr, accept != nullptr   greedy OMP unless *accept == 1
    if (order == nullptr && accept != nullptr && *accept == 1) return;
    __shared__ cd L[kMaxR][kMaxR + 1];   // L[u][q], u >= q
    __shared__ double invdiag[kMaxR];
    __shared__ cd bsel[kMaxR];
    __shared__ int S[kMaxR];
    const int lane = threadIdx.x;
    auto Mel = [&](int i, int jj) -> cd {
        return {M[2 * (static_cast<int64_t>(jj) * r + i)], M[2 * (static_cast<int64_t>(jj) * r + i) + 1]};
    };
    const bool live = lane < r;
    const double mjj = live ? Mel(lane, lane).x : 0.0;
    const double inv_m = (live && mjj > 0.0) ? rcp64(mjj) : 0.0;
    const cd cj = live ? cd{cvec[2 * lane], cvec[2 * lane + 1]} : cd{0.0, 0.0};
    const double imlam = live ? lam[2 * lane + 1] : 0.0;
    bool used = false;
    const double y2 = R[0];
    const int kmax_steps = lstsq ? r : min(K, r);
    int ns = 0;
    double res2 = y2;
    for (int step = 0; step < kmax_steps; ++step) {
        if (!lstsq && order == nullptr && res2 <= 1e-24 * y2) break;
        int best;
        if (order != nullptr) {
            best = order[step];
            if (best < 0 || best >= r) break;
        } else if (lstsq) {
            best = step;
        } else {
            double score = -1.0;
            if (live && !used && mjj > 0.0) {
                cd g = cj;
                for (int q = 0; q < ns; ++q) g = csub(g, cmul(Mel(lane, S[q]), bsel[q]));
                score = cabs2(g) * inv_m;
            }
            const double bmax = warp_max(score);
            if (!(bmax > 0.0)) break;
            const bool cand = score >= bmax * (1.0 - 2e-9);
            const double key = cand ? imlam : -1e300;
            const double kbest = warp_max(key);
            const unsigned bb = __ballot_sync(0xffffffffu, cand && key == kbest);
            if (bb == 0u) break;                    // non-finite scores: no pick
            best = __ffs(bb) - 1;
        }
        // new Cholesky row: solve L x = m (m_q = M[S_q][best]); row = conj(x)
        cd t = (lane < ns) ? Mel(S[lane], best) : cd{0.0, 0.0};
        double xs2 = 0.0;
        for (int q = 0; q < ns; ++q) {
            cd xq = {0.0, 0.0};
            if (lane == q) xq = cscale(t, invdiag[q]);
            xq = shfl_cd(xq, q);
            if (lane == q) { L[ns][q] = cconj(xq); xs2 = cabs2(xq); }
            if (lane > q && lane < ns) t = csub(t, cmul(L[lane][q], xq));
        }
        const double diag2 = Mel(best, best).x - warp_sum(xs2);
        if (!(diag2 > kEps * Mel(best, best).x)) {
            if (lstsq && lane == 0) record_status(status, CDMD_ERR_RANK_DEFICIENT);
            break;
        }
        const double invd = rsqrt64(diag2);
        if (lane == 0) {
            L[ns][ns] = {diag2 * invd, 0.0};
            invdiag[ns] = invd;
            S[ns] = best;
        }
        if (lane == best) used = true;
        ++ns;
        __syncwarp();
        // beta: L y = c_S (forward), then L^H beta = y (backward); lane u owns row u
        cd v = (lane < ns) ? cd{cvec[2 * S[lane]], cvec[2 * S[lane] + 1]} : cd{0.0, 0.0};
        for (int q = 0; q < ns; ++q) {
            cd yq = {0.0, 0.0};
            if (lane == q) { yq = cscale(v, invdiag[q]); v = yq; }
            yq = shfl_cd(yq, q);
            if (lane > q && lane < ns) v = csub(v, cmul(L[lane][q], yq));
        }
        for (int q = ns - 1; q >= 0; --q) {
            cd bq = {0.0, 0.0};
            if (lane == q) { bq = cscale(v, invdiag[q]); v = bq; }
            bq = shfl_cd(bq, q);
            if (lane < q) v = csub(v, cmul(cconj(L[q][lane]), bq));
        }
        if (lane < ns) bsel[lane] = v;
        __syncwarp();
        double cb = 0.0;
        if (lane < ns) {
            const cd c = {cvec[2 * S[lane]], cvec[2 * S[lane] + 1]};
            cb = fma(c.x, v.x, c.y * v.y);
        }
        res2 = y2 - warp_sum(cb);
    }
    if (order != nullptr) {
        const double tol = static_cast<double>(blob[8]);
        const bool ok = tol >= 0.0 && res2 <= tol * tol * y2;   // a negative tol rejects every pick
        if (lane == 0) {
            *accept = ok ? 1 : 0;
            if (!ok) atomicAdd(fallbacks, 1ull);
        }
        if (!ok) return;
    }
    if (live) {
        beta[2 * lane] = 0.0;
        beta[2 * lane + 1] = 0.0;
    }
    __syncwarp();
    if (lane < ns) {
        beta[2 * S[lane]] = bsel[lane].x;
        beta[2 * S[lane] + 1] = bsel[lane].y;
    }
    if (lane < K) sel[lane] = (lane < ns) ? S[lane] : -1;
    if (lane == 0) *nsel_out = ns;
}

// 10. Phi_Y[i][c] = sum_t DY[(t+1)*k + i] G[t][c]
__global__ void phiy_kernel(const double* __restrict__ DY, const double* __restrict__ G, int k, int p,
                            int r, double* __restrict__ PhiY) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<int64_t>(k) * r) return;
    const int i = static_cast<int>(idx % k), c = static_cast<int>(idx / k);
    double re = 0.0, im = 0.0;
    for (int t = 0; t < p; ++t) {
        const double y = DY[static_cast<int64_t>(t + 1) * k + i];
        re = fma(y, G[2 * (static_cast<int64_t>(c) * p + t)], re);
        im = fma(y, G[2 * (static_cast<int64_t>(c) * p + t) + 1], im);
    }
    PhiY[2 * idx] = re;
    PhiY[2 * idx + 1] = im;
}

// OMP against another target y_t (k values) on the same decomposition:
// cvec_t[c] = G[:,c]^H (Y'^T y_t), y2_t = ||y_t||^2.
__global__ void __launch_bounds__(256)
relabel_target_kernel(const double* __restrict__ DY, int k, int p, const double* __restrict__ G, int r,
                      const double* __restrict__ yt, double* __restrict__ u, double* __restrict__ cvec_t,
                      double* __restrict__ y2_t) {
    // one CTA: first u = Y'^T y_t (warp per frame), then cvec_t, then ||y_t||^2
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = wid; t < p; t += nw) {
        const double* col = DY + static_cast<int64_t>(t + 1) * k;
        double acc = 0.0;
        for (int i = lane; i < k; i += 32) acc = fma(col[i], yt[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) u[t] = acc;
    }
    __syncthreads();
    for (int c = wid; c <= r; c += nw) {
        double re = 0.0, im = 0.0;
        if (c < r) {
            const double* gc = G + 2 * static_cast<int64_t>(c) * p;
            for (int t = lane; t < p; t += 32) {
                re = fma(gc[2 * t], u[t], re);
                im = fma(-gc[2 * t + 1], u[t], im);
            }
        } else {
            for (int i = lane; i < k; i += 32) re = fma(yt[i], yt[i], re);
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            if (c < r) {
                cvec_t[2 * c] = re;
                cvec_t[2 * c + 1] = im;
            } else {
                *y2_t = re;
            }
        }
    }
}

}  // namespace

cdmd_status launch_selector_relabel(cdmd_ctx* ctx, const double* DY, int k, int n, const double* G,
                                    const double* lambda, int r, const double* y_target, int K, int32_t* sel,
                                    cudaStream_t stream) {
    const int p = n - 1;
    void* buf = nullptr;
    const size_t doubles = static_cast<size_t>(p) + 4 * r + 8;
    cdmd_status st = ensure_buffer(ctx, BUF_RELABEL, doubles * sizeof(double) + 64, &buf);
    if (st != CDMD_OK) return st;
    double* u = static_cast<double*>(buf);
    double* cvec_t = u + p;
    double* beta_t = cvec_t + 2 * r;
    double* y2_t = beta_t + 2 * r;
    int32_t* nsel_t = reinterpret_cast<int32_t*>(y2_t + 1);
    relabel_target_kernel<<<1, 256, 0, stream>>>(DY, k, p, G, r, y_target, u, cvec_t, y2_t);
    CDMD_CHECK_LAUNCH("relabel_target_kernel");
    omp_kernel<<<1, 32, 0, stream>>>(ctx->last_M, cvec_t, y2_t, lambda, r, K, 0, beta_t, sel, nsel_t,
                                     ctx->d_status, nullptr, nullptr, nullptr, nullptr);
    CDMD_CHECK_LAUNCH("omp_kernel");
    return CDMD_OK;
}

namespace {

// Steps 4-7 and 9 from the Gram of the sketch DY (k x n), or, when Rin is
// given, from that n x n Gram directly (DY and PhiY unused).
struct AutoRank {
    int* r_host;        // receives the chosen rank
    double* tau_host;   // receives the threshold (may be NULL)
};

cdmd_status decompose_impl(cdmd_ctx* ctx, const double* DY, int k, const double* Rin, int n, int r, int K,
                           cdmd_selector selector, double* sigma, double* lambda, double* G, double* PhiY,
                           double* beta, int32_t* sel, int32_t* nsel, cudaStream_t stream,
                           const AutoRank* autor = nullptr) {
    const int p = n - 1;
    // ---- workspace layout (doubles) ----
    const int ntiles = (n + kGT - 1) / kGT;
    const int kchunk = 128;
    const int splits = Rin != nullptr ? 0 : (k + kchunk - 1) / kchunk;
    const size_t n_gram_part = static_cast<size_t>(splits) * n * n;
    const size_t n_R = static_cast<size_t>(n) * n;
    const size_t n_Hv = static_cast<size_t>(p) * p;
    const size_t n_vec = static_cast<size_t>(p);
    const size_t n_Z = static_cast<size_t>(p) * r;
    const size_t n_small = static_cast<size_t>(r) * r * 2;
    const size_t total = n_gram_part + n_R + n_Hv + 3 * n_vec + r + 3 * n_Z + 5 * n_small + 6 * r + 64;
    // + one slot for the eigen-solver's fallback flag and two for the rank
    // threshold's result; with an automatic rank, r is its upper bound here
    double* ws = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_EIG, (total + 3) * sizeof(double), reinterpret_cast<void**>(&ws));
    if (st != CDMD_OK) return st;
    int* eig_flag = reinterpret_cast<int*>(ws + total);   // written by eig_f32_kernel before any read
    int* gd_r = reinterpret_cast<int*>(ws + total + 1);
    double* gd_tau = ws + total + 2;
    double* gpart = ws;
    double* Rws = gpart + n_gram_part;
    const double* R = Rin != nullptr ? Rin : Rws;
    double* Hv = Rws + n_R;
    double* htau = Hv + n_Hv;
    double* dd = htau + n_vec;
    double* ee = dd + n_vec;
    double* lamT = ee + n_vec;
    // the regions below depend on r; with an automatic rank they are laid out
    // again once the rank is known (a smaller r fits the same allocation)
    double *Z, *V, *B, *At, *W, *M, *WR, *lamR, *cvec;
    float *lam32, *W32;
    auto lay_out = [&](int rr) {
        const size_t nz = static_cast<size_t>(p) * rr, ns = static_cast<size_t>(rr) * rr * 2;
        Z = lamT + rr;
        V = Z + nz;
        B = V + nz;
        At = B + nz;
        W = At + ns;
        M = W + ns;
        WR = M + ns;
        lamR = WR + ns;
        cvec = lamR + 2 * rr;
        lam32 = reinterpret_cast<float*>(cvec + 2 * rr);    // 2r floats
        W32 = reinterpret_cast<float*>(cvec + 4 * rr);      // 2r^2 floats (ns/2 doubles)
    };
    lay_out(r);

    // 1. Gram
    if (Rin == nullptr) {
        gram_partial_kernel<<<dim3(ntiles, ntiles, splits), 256, 0, stream>>>(DY, k, n, kchunk, gpart);
        CDMD_CHECK_LAUNCH("gram_partial_kernel");
        gram_reduce_kernel<<<(n * n + 255) / 256, 256, 0, stream>>>(gpart, splits, n, Rws, ctx->d_status);
        CDMD_CHECK_LAUNCH("gram_reduce_kernel");
    }

    // 2. tridiagonalisation on a cluster of 8 CTAs (else 4).  A cluster must
    // fit in one GPC beside other clips' full-data passes: 8 CTAs gave 3.8 %
    // more clips/s than 16 with clips in flight, at 2 % more latency
    if (p >= 3) {
        // cluster size: 8 CTAs first (fits one GPC beside other clips' passes),
        // else 16 (non-portable; large n), else 4
        const int csize_pref = 8;
        const int cands[3] = {csize_pref, csize_pref == 16 ? 8 : 16, 4};
        bool launched = false;
        for (int ci = 0; ci < 3 && !launched; ++ci) {
            const int csize = cands[ci];
            const int rows_per = (p + csize - 1) / csize;
            const size_t smem = (static_cast<size_t>(rows_per) * p + 4 * static_cast<size_t>(p) + 66) * sizeof(double);
            if (smem > kMaxOptInSmem) continue;
            // the opt-in maximum, the same value on every call: concurrent
            // contexts (and captured graphs) never see it lowered
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(kMaxOptInSmem)));
            if (csize > 8)
                CDMD_CHECK_CUDA(cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(csize, 1, 1);
            cfg.blockDim = dim3(kTriThreads, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = csize;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            const cudaError_t oe = cudaOccupancyMaxActiveClusters(&nclusters, tridiag_kernel, &cfg);
            if (oe != cudaSuccess || nclusters < 1) {
                (void)cudaGetLastError();
                continue;
            }
            CDMD_CHECK_CUDA(cudaLaunchKernelEx(&cfg, tridiag_kernel, static_cast<const double*>(R), n, p, Hv,
                                               htau, dd, ee));
            launched = true;
        }
        if (!launched) return fail(CDMD_ERR_UNSUPPORTED, "no cluster size fits the tridiagonalisation of p = %d", p);
    } else {
        tiny_tridiag_kernel<<<1, 1, 0, stream>>>(R, n, p, dd, ee, htau);
        CDMD_CHECK_LAUNCH("tiny_tridiag_kernel");
    }
    // 2b. optional automatic rank (Remark 2): the one host synchronisation of
    // the decomposition, since the launches below are sized by r
    if (autor != nullptr) {
        const int q = k < p ? k : p;
        const double bq = static_cast<double>(q) / static_cast<double>(k > p ? k : p);
        const double omega = ((0.56 * bq - 0.95) * bq + 1.82) * bq + 1.43;
        gd_rank_kernel<<<1, 32, 2 * static_cast<size_t>(p) * sizeof(double), stream>>>(dd, ee, p, q, omega, r, gd_r,
                                                                                         gd_tau, ctx->d_status);
        CDMD_CHECK_LAUNCH("gd_rank_kernel");
        int hr = 0;
        double ht = 0.0;
        CDMD_CHECK_CUDA(cudaMemcpyAsync(&hr, gd_r, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CDMD_CHECK_CUDA(cudaMemcpyAsync(&ht, gd_tau, sizeof(double), cudaMemcpyDeviceToHost, stream));
        CDMD_CHECK_CUDA(cudaStreamSynchronize(stream));
        if (hr < 1 || hr > r) return fail(CDMD_ERR_CUDA, "rank threshold returned %d (bound %d)", hr, r);
        // picks past the capped K read as "no mode"
        CDMD_CHECK_CUDA(cudaMemsetAsync(sel, 0xff, static_cast<size_t>(K) * sizeof(int32_t), stream));
        r = hr;
        if (K > r) K = r;
        *autor->r_host = r;
        if (autor->tau_host != nullptr) *autor->tau_host = ht;
        lay_out(r);
    }
    // 3. eigenpairs of T, orthonormalisation, back-transform
    {
        const size_t esm = 10 * static_cast<size_t>(p) * sizeof(double);
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(tridiag_eigpair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kMaxOptInSmem)));
        tridiag_eigpair_kernel<<<r, 32, esm, stream>>>(dd, ee, p, r, lamT, Z, ctx->d_status);
        CDMD_CHECK_LAUNCH("tridiag_eigpair_kernel");
    }
    {
        const size_t osm = (static_cast<size_t>(r) * p + 64) * sizeof(double);
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(orthonormalise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kMaxOptInSmem)));
        orthonormalise_kernel<<<1, 1024, osm, stream>>>(Z, p, r);
    }
    CDMD_CHECK_LAUNCH("orthonormalise_kernel");
    static_assert(32 * 16 >= 511, "the back-transform covers p = n - 1 <= 511 (n <= 512)");
    if (p <= 256)
        backtransform_kernel<8><<<r, 32, p * sizeof(double), stream>>>(Z, Hv, htau, lamT, p, r, V, sigma,
                                                                       ctx->d_status);
    else
        backtransform_kernel<16><<<r, 32, p * sizeof(double), stream>>>(Z, Hv, htau, lamT, p, r, V, sigma,
                                                                        ctx->d_status);
    CDMD_CHECK_LAUNCH("backtransform_kernel");
    // 4. A~ and its eigen-decomposition
    bmat_kernel<<<dim3((p + 7) / 8, r), 256, 0, stream>>>(R, V, n, p, B);
    CDMD_CHECK_LAUNCH("bmat_kernel");
    atilde_kernel<<<r, 32, 0, stream>>>(V, B, sigma, p, r, At);
    CDMD_CHECK_LAUNCH("atilde_kernel");
    eig_f32_kernel<<<1, 32, 0, stream>>>(At, r, reinterpret_cast<float2*>(lam32), reinterpret_cast<float2*>(W32),
                                         eig_flag);
    CDMD_CHECK_LAUNCH("eig_f32_kernel");
    eig_refine_kernel<<<r, 32, 0, stream>>>(At, r, reinterpret_cast<const float2*>(lam32),
                                            reinterpret_cast<const float2*>(W32), lamR, WR, eig_flag);
    CDMD_CHECK_LAUNCH("eig_refine_kernel");
    CDMD_CHECK_CUDA(cudaFuncSetAttribute(eig_qr64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kQrSmem)));
    eig_qr64_kernel<<<1, kQrThreads, kQrSmem, stream>>>(At, r, lamR, WR, eig_flag, ctx->d_status);
    CDMD_CHECK_LAUNCH("eig_qr64_kernel");
    eig_order_kernel<<<1, 32, 0, stream>>>(lamR, WR, r, lambda, W);
    CDMD_CHECK_LAUNCH("eig_order_kernel");
    // 5. G, Gram-form quantities, selection
    gmat_kernel<<<(p * r + 127) / 128, 128, 0, stream>>>(V, sigma, W, p, r, G);
    CDMD_CHECK_LAUNCH("gmat_kernel");
    hmat_kernel<<<r, 512, 2 * p * sizeof(double), stream>>>(R, G, n, p, r, M, cvec);
    CDMD_CHECK_LAUNCH("hmat_kernel");
    ctx->last_M = M;
    ctx->last_cvec = cvec;
    ctx->last_R = R;
    ctx->last_r = r;
    if (selector == CDMD_SEL_MLP) {
        // learned pick order -> least squares on it -> OMP only if rejected
        st = launch_mlp_select(ctx, lambda, M, cvec, R, r, K, stream);
        if (st != CDMD_OK) return st;
        omp_kernel<<<1, 32, 0, stream>>>(M, cvec, R, lambda, r, K, 0, beta, sel, nsel, ctx->d_status,
                                         selector_order(ctx), selector_blob(ctx), selector_accept(ctx),
                                         selector_fallbacks(ctx));
        CDMD_CHECK_LAUNCH("omp_kernel");
        omp_kernel<<<1, 32, 0, stream>>>(M, cvec, R, lambda, r, K, 0, beta, sel, nsel, ctx->d_status, nullptr,
                                         nullptr, selector_accept(ctx), nullptr);
    } else {
        omp_kernel<<<1, 32, 0, stream>>>(M, cvec, R, lambda, r, K, selector == CDMD_SEL_LSTSQ ? 1 : 0, beta, sel,
                                         nsel, ctx->d_status, nullptr, nullptr, nullptr, nullptr);
    }
    CDMD_CHECK_LAUNCH("omp_kernel");
    if (PhiY != nullptr && DY != nullptr) {
        const int64_t tot = static_cast<int64_t>(k) * r;
        phiy_kernel<<<static_cast<unsigned>((tot + 127) / 128), 128, 0, stream>>>(DY, G, k, p, r, PhiY);
        CDMD_CHECK_LAUNCH("phiy_kernel");
    }
    return CDMD_OK;
}

}  // namespace

cdmd_status launch_decompose(cdmd_ctx* ctx, const double* DY, int k, int n, int r, int K,
                             cdmd_selector selector, double* sigma, double* lambda, double* G,
                             double* PhiY, double* beta, int32_t* sel, int32_t* nsel,
                             cudaStream_t stream) {
    return decompose_impl(ctx, DY, k, nullptr, n, r, K, selector, sigma, lambda, G, PhiY, beta, sel, nsel, stream);
}

cdmd_status launch_decompose_auto(cdmd_ctx* ctx, const double* DY, int k, int n, int r_max, int K,
                                  cdmd_selector selector, double* sigma, double* lambda, double* G, double* PhiY,
                                  double* beta, int32_t* sel, int32_t* nsel, int* r_out, double* tau_out,
                                  cudaStream_t stream) {
    const AutoRank a{r_out, tau_out};
    return decompose_impl(ctx, DY, k, nullptr, n, r_max, K, selector, sigma, lambda, G, PhiY, beta, sel, nsel, stream,
                          &a);
}

cdmd_status launch_decompose_gram(cdmd_ctx* ctx, const double* R, int n, int r, int K, cdmd_selector selector,
                                  double* sigma, double* lambda, double* G, double* beta, int32_t* sel,
                                  int32_t* nsel, cudaStream_t stream) {
    return decompose_impl(ctx, nullptr, 0, R, n, r, K, selector, sigma, lambda, G, nullptr, beta, sel, nsel, stream);
}

}  // namespace cdmd
