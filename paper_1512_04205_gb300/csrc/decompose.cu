// Small solves on the device, FP64 (Algorithm 1 steps 4-7 and 9, Remark 3).
//
// Everything after the sketch is derived from the n x n Gram matrix
// R = DY^T DY of the sketch:
//   Y^T Y  = R[0:p, 0:p]     (p = n-1)      -> V, S   (SVD of Y, step 4)
//   Y^T Y' = R[0:p, 1:n]                     -> A~ = S^-1 V^T (Y^T Y') V S^-1 (step 6)
//   Y'^T Y'= R[1:n, 1:n], Y'^T y1 = R[1:n, 0] -> Gram form of the OMP on the
//            compressed modes Phi_Y = Y' G (Remark 3)
// so no kernel after the Gram touches the k-long sketch rows again.
//
// FP64 on this GPU runs at about 1/64 of the FP32 rate, so each O(p^3) or
// O(p^2 r) stage is spread over many SMs:
//   gram_partial / gram_reduce   multi-CTA, split over the sketch rows
//   tridiag                      Householder tridiagonalisation of Y^T Y on a
//                                thread-block cluster, rows distributed over
//                                the CTAs' shared memory, vectors exchanged
//                                through distributed shared memory
//   tridiag_eigpair              one CTA per wanted eigenvalue: Sturm-count
//                                multisection, then inverse iteration
//   orthonormalise               modified Gram-Schmidt, twice (one CTA)
//   backtransform                one CTA per eigenvector: V = Q z, B = (Y^T Y') V
//   atilde                       one CTA per column of A~
//   eig_small                    one CTA: Hessenberg + complex-shift QR on A~
//   gmat                         G = V S^-1 W
//   hmat                         H = (Y'^T Y') G, M = G^H H, c = G^H (Y'^T y1)
//   omp                          one CTA: OMP / least squares in Gram form
//   phiy (optional)              Phi_Y = Y' G
#include <cooperative_groups.h>

#include "cdmd_internal.cuh"

namespace cg = cooperative_groups;

namespace cdmd {
namespace {

constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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
// Row i lives in CTA i % P (local slot i / P).  Step j: the owner of row j
// (= column j by symmetry) forms the reflector H_j = I - tau v v^T with
// H_j A[j+1:, j] = alpha e_1 and broadcasts v; every CTA forms u = A v on its
// rows and broadcasts it; every CTA then applies the rank-2 update
// A -= v w^T + w v^T, w = tau u - (tau^2/2)(v^T u) v, to its rows.
// Outputs: diagonal dd[p], off-diagonal ee[p-1], reflectors Hv[j*p + l]
// (l > j) and htau[j], with A = Q T Q^T, Q = H_0 H_1 ... H_{p-3}.
// ---------------------------------------------------------------------------
constexpr int kTriThreads = 256;

__global__ void __launch_bounds__(kTriThreads)
tridiag_kernel(const double* __restrict__ R, int n, int p, double* __restrict__ Hv,
               double* __restrict__ htau, double* __restrict__ dd, double* __restrict__ ee) {
    cg::cluster_group cluster = cg::this_cluster();
    const int P = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int rows_per = (p + P - 1) / P;
    extern __shared__ double sm[];
    double* Aloc = sm;                              // rows_per * p
    double* vbuf = Aloc + static_cast<size_t>(rows_per) * p;   // 2 * p
    double* ubuf = vbuf + 2 * p;                    // p
    double* wv = ubuf + p;                          // p
    double* red = wv + p;                           // 32 scratch + 2 tau slots
    double* tau_slot = red + 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = kTriThreads / 32;

    for (int idx = tid; idx < rows_per * p; idx += kTriThreads) {
        const int li = idx / p, l = idx % p;
        const int i = rank + P * li;
        Aloc[idx] = (i < p) ? R[static_cast<int64_t>(i) * n + l] : 0.0;
    }
    cluster.sync();

    for (int j = 0; j + 2 < p; ++j) {
        const int buf = j & 1;
        const int owner = j % P;
        if (rank == owner) {
            const double* row = Aloc + static_cast<size_t>(j / P) * p;
            double s = 0.0;
            for (int l = j + 2 + tid; l < p; l += kTriThreads) s += row[l] * row[l];
            const double tail2 = block_sum(s, red);
            const double x0 = row[j + 1];
            double alpha, tau, v0;
            if (tail2 == 0.0) {
                alpha = x0; tau = 0.0; v0 = 0.0;
            } else {
                const double nrm = sqrt(x0 * x0 + tail2);
                alpha = (x0 >= 0.0) ? -nrm : nrm;
                v0 = x0 - alpha;
                tau = 2.0 / (v0 * v0 + tail2);
            }
            for (int rr = 0; rr < P; ++rr) {
                double* rv = cluster.map_shared_rank(vbuf + buf * p, rr);
                for (int l = j + 1 + tid; l < p; l += kTriThreads)
                    rv[l] = (l == j + 1) ? v0 : (tau == 0.0 ? 0.0 : row[l]);
                if (tid == 0) *cluster.map_shared_rank(tau_slot + buf, rr) = tau;
            }
            for (int l = j + 1 + tid; l < p; l += kTriThreads)
                Hv[static_cast<int64_t>(j) * p + l] = (l == j + 1) ? v0 : (tau == 0.0 ? 0.0 : row[l]);
            if (tid == 0) {
                dd[j] = row[j];
                ee[j] = alpha;
                htau[j] = tau;
            }
        }
        cluster.sync();
        const double* v = vbuf + buf * p;
        const double tau = tau_slot[buf];
        if (tau != 0.0) {
            // (b) u_i = sum_l A_il v_l for owned rows i > j; one warp per row
            const int li_first = (j + 1 - rank + P - 1) / P;   // smallest li with rank + P li >= j+1
            for (int li = li_first + wid; li < rows_per; li += nwarps) {
                const int i = rank + P * li;
                if (i >= p) break;
                const double* row = Aloc + static_cast<size_t>(li) * p;
                double s = 0.0;
                for (int l = j + 1 + lane; l < p; l += 32) s = fma(row[l], v[l], s);
                s = warp_sum(s);
                if (lane < P) *cluster.map_shared_rank(ubuf + i, lane) = s;
            }
        }
        cluster.sync();
        if (tau != 0.0) {
            double s = 0.0;
            for (int l = j + 1 + tid; l < p; l += kTriThreads) s = fma(v[l], ubuf[l], s);
            const double vtu = block_sum(s, red);
            const double kc = 0.5 * tau * tau * vtu;
            for (int l = j + 1 + tid; l < p; l += kTriThreads) wv[l] = tau * ubuf[l] - kc * v[l];
            __syncthreads();
            const int li_first = (j + 1 - rank + P - 1) / P;
            const int L = p - j - 1;
            const int nrows = rows_per - li_first;
            for (int idx = tid; idx < nrows * L; idx += kTriThreads) {
                const int li = li_first + idx / L;
                const int l = j + 1 + idx % L;
                const int i = rank + P * li;
                if (i >= p) continue;
                double* a = Aloc + static_cast<size_t>(li) * p + l;
                *a = *a - v[i] * wv[l] - wv[i] * v[l];
            }
        }
        __syncthreads();
    }
    // trailing 2x2 (or smaller) block
    if (tid == 0) {
        for (int i = max(p - 2, 0); i < p; ++i) {
            if (i % P != rank) continue;
            const double* row = Aloc + static_cast<size_t>(i / P) * p;
            dd[i] = row[i];
            if (i + 1 < p) ee[i] = row[i + 1];
        }
    }
    cluster.sync();
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
// Sturm count N(x) = #eigenvalues < x = sign changes of the leading minors
// p_i(x) = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}, rescaled to stay in range.
// ---------------------------------------------------------------------------
__device__ int sturm_count(const double* d, const double* e2, int p, double x) {
    double a = d[0] - x;   // p_0
    double b = 1.0;        // p_{-1}
    int cnt = (a < 0.0) ? 1 : 0;
    if (a == 0.0) { a = -kEps; cnt = 1; }
    for (int i = 1; i < p; ++i) {
        double c = fma(d[i] - x, a, -e2[i - 1] * b);
        if (c == 0.0) c = (a < 0.0) ? kEps : -kEps;   // zero counts as a change
        cnt += ((c < 0.0) != (a < 0.0)) ? 1 : 0;
        b = a;
        a = c;
        const double m = fabs(a);
        if (m > 1e150) { a *= 1e-150; b *= 1e-150; }
        else if (m < 1e-150 && fabs(b) < 1e-150) { a *= 1e150; b *= 1e150; }
    }
    return cnt;
}

constexpr int kSections = 8;   // lanes used by the multisection

// Every array this kernel writes and reads back lives in shared memory, so
// no load can be served from a read-only cache path that misses the write.
__global__ void __launch_bounds__(32)
tridiag_eigpair_kernel(const double* __restrict__ dd, const double* __restrict__ ee, int p, int r,
                       double* lam, double* Z, int* status) {
    extern __shared__ double tsm[];
    double* d = tsm;          // p
    double* e = d + p;        // p (e[p-1] = 0)
    double* e2 = e + p;       // p
    double* work = e2 + p;    // 6 p: LU factors, pivots, iterate
    const int w = blockIdx.x;             // w-th largest
    const int lane = threadIdx.x;
    for (int i = lane; i < p; i += 32) {
        d[i] = dd[i];
        e[i] = (i + 1 < p) ? ee[i] : 0.0;
        e2[i] = e[i] * e[i];
    }
    __syncwarp();
    // Gershgorin interval
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
    const int idx = p - 1 - w;   // ascending index of the target
    bool converged = false;
    for (int it = 0; it < 80; ++it) {
        const double width = hi - lo;
        if (width <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)) + kEps * tn + 1e-300) { converged = true; break; }
        const double x = lo + width * static_cast<double>(lane + 1) / (kSections + 1);
        int cnt = 0;
        if (lane < kSections) cnt = sturm_count(d, e2, p, x);
        const unsigned above = __ballot_sync(0xffffffffu, lane < kSections && cnt > idx);
        const int f = above ? __ffs(above) - 1 : kSections;
        const double xf = lo + width * static_cast<double>(f + 1) / (kSections + 1);
        const double xl = lo + width * static_cast<double>(f) / (kSections + 1);
        const double nlo = (f == 0) ? lo : xl;
        const double nhi = (f == kSections) ? hi : xf;
        if (nlo >= nhi || (nlo == lo && nhi == hi)) { converged = true; break; }
        lo = nlo;
        hi = nhi;
    }
    const double lambda = 0.5 * (lo + hi);
    if (!converged && lane == 0) record_status(status, CDMD_ERR_NOT_CONVERGED);
    if (lane == 0) lam[w] = lambda;

    // inverse iteration by lane 0: LU with partial pivoting of T - mu I
    if (lane == 0) {
        double* ldl = work;                                    // sub multipliers
        double* ldd = ldl + p;                                 // U diagonal
        double* ldu = ldd + p;                                 // U first super
        double* ldu2 = ldu + p;                                // U second super
        double* piv = ldu2 + p;                                // 1.0 = rows swapped
        double* z = piv + p;
        const double mu = lambda + kEps * tn;   // keep the shifted matrix non-singular
        const double tiny = kEps * tn + 1e-300;
        for (int i = 0; i < p; ++i) {
            ldd[i] = d[i] - mu;
            ldl[i] = (i + 1 < p) ? e[i] : 0.0;
            ldu[i] = (i + 1 < p) ? e[i] : 0.0;
            ldu2[i] = 0.0;
            piv[i] = 0.0;
        }
        for (int i = 0; i + 1 < p; ++i) {
            if (fabs(ldd[i]) >= fabs(ldl[i])) {
                if (ldd[i] == 0.0) ldd[i] = tiny;
                const double fct = ldl[i] / ldd[i];
                ldl[i] = fct;
                ldd[i + 1] -= fct * ldu[i];
            } else {
                const double fct = ldd[i] / ldl[i];
                ldd[i] = ldl[i];
                ldl[i] = fct;
                const double tmp = ldu[i];
                ldu[i] = ldd[i + 1];
                ldd[i + 1] = tmp - fct * ldd[i + 1];
                if (i + 2 < p) {
                    ldu2[i] = ldu[i + 1];
                    ldu[i + 1] = -fct * ldu[i + 1];
                }
                piv[i] = 1.0;
            }
        }
        if (ldd[p - 1] == 0.0) ldd[p - 1] = tiny;
        // deterministic start vector
        uint32_t hs = 0x9E3779B9u * static_cast<uint32_t>(w + 1);
        for (int i = 0; i < p; ++i) {
            hs ^= hs << 13; hs ^= hs >> 17; hs ^= hs << 5;
            z[i] = 1.0 + static_cast<double>(hs & 0xffff) * (1.0 / 65536.0);
        }
        for (int itr = 0; itr < 3; ++itr) {
            for (int i = 0; i + 1 < p; ++i) {
                if (piv[i] == 0.0) {
                    z[i + 1] -= ldl[i] * z[i];
                } else {
                    const double tmp = z[i];
                    z[i] = z[i + 1];
                    z[i + 1] = tmp - ldl[i] * z[i];
                }
            }
            z[p - 1] /= ldd[p - 1];
            if (p > 1) z[p - 2] = (z[p - 2] - ldu[p - 2] * z[p - 1]) / ldd[p - 2];
            for (int i = p - 3; i >= 0; --i)
                z[i] = (z[i] - ldu[i] * z[i + 1] - ldu2[i] * z[i + 2]) / ldd[i];
            double nrm = 0.0;
            for (int i = 0; i < p; ++i) nrm = fma(z[i], z[i], nrm);
            nrm = sqrt(nrm);
            if (!(nrm > 0.0) || !isfinite(nrm)) { record_status(status, CDMD_ERR_NOT_CONVERGED); nrm = 1.0; }
            const double inv = 1.0 / nrm;
            for (int i = 0; i < p; ++i) z[i] *= inv;
        }
        for (int i = 0; i < p; ++i) Z[static_cast<int64_t>(w) * p + i] = z[i];
    }
}

// 4a. Modified Gram-Schmidt over the r columns of Z (descending eigenvalue
// order), applied twice.
// Threads read entries other threads wrote (ordered by __syncthreads), so Z
// is deliberately not __restrict__: its loads must stay coherent.
__global__ void __launch_bounds__(256)
orthonormalise_kernel(double* Z, int p, int r) {
    __shared__ double red[32];
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < r; ++c) {
            double* zc = Z + static_cast<int64_t>(c) * p;
            for (int q = 0; q < c; ++q) {
                const double* zq = Z + static_cast<int64_t>(q) * p;
                double s = 0.0;
                for (int i = threadIdx.x; i < p; i += blockDim.x) s = fma(zq[i], zc[i], s);
                const double dot = block_sum(s, red);
                for (int i = threadIdx.x; i < p; i += blockDim.x) zc[i] -= dot * zq[i];
                __syncthreads();
            }
            double s = 0.0;
            for (int i = threadIdx.x; i < p; i += blockDim.x) s = fma(zc[i], zc[i], s);
            const double nrm = sqrt(block_sum(s, red));
            const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
            for (int i = threadIdx.x; i < p; i += blockDim.x) zc[i] *= inv;
            __syncthreads();
        }
    }
}

// 4b. V[:, c] = Q z_c (apply H_{p-3}, ..., H_0), sigma_c = sqrt(lambda_c),
// B[:, c] = (Y^T Y') V[:, c].  One CTA (one warp) per column.
__global__ void __launch_bounds__(32)
backtransform_kernel(const double* __restrict__ Z, const double* __restrict__ Hv,
                     const double* __restrict__ htau, const double* __restrict__ lam,
                     const double* __restrict__ R, int n, int p, int r,
                     double* __restrict__ V, double* __restrict__ B, double* __restrict__ sigma,
                     int* status) {
    extern __shared__ double ysm[];   // p
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    for (int i = lane; i < p; i += 32) ysm[i] = Z[static_cast<int64_t>(c) * p + i];
    __syncwarp();
    for (int j = p - 3; j >= 0; --j) {
        const double tau = htau[j];
        if (tau == 0.0) continue;
        const double* v = Hv + static_cast<int64_t>(j) * p;
        double s = 0.0;
        for (int l = j + 1 + lane; l < p; l += 32) s = fma(v[l], ysm[l], s);
        s = warp_sum(s) * tau;
        for (int l = j + 1 + lane; l < p; l += 32) ysm[l] -= s * v[l];
        __syncwarp();
    }
    for (int i = lane; i < p; i += 32) V[static_cast<int64_t>(c) * p + i] = ysm[i];
    if (lane == 0) {
        const double l0 = lam[0];
        const double lc = lam[c];
        if (!(lc > static_cast<double>(p) * kEps * fabs(l0))) record_status(status, CDMD_ERR_RANK_DEFICIENT);
        sigma[c] = sqrt(fmax(lc, 0.0));
    }
    // B[a][c] = sum_b R[a][b+1] V[b][c]
    for (int a = 0; a < p; ++a) {
        const double* row = R + static_cast<int64_t>(a) * n + 1;
        double s = 0.0;
        for (int b = lane; b < p; b += 32) s = fma(row[b], ysm[b], s);
        s = warp_sum(s);
        if (lane == 0) B[static_cast<int64_t>(c) * p + a] = s;
    }
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
            At[static_cast<int64_t>(c) * r + a] = den > 0.0 ? s / den : 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// 6. Eigen-decomposition of the real r x r A~ in one CTA: Householder
// Hessenberg reduction, complex single-shift QR (Wilkinson shift, bulge chase
// with Givens rotations) to a complex Schur form, eigenvectors by
// back-substitution, W = Q Z X; columns scaled to unit norm with the
// largest-modulus entry real positive; eigenvalues ordered by descending
// modulus with conjugate pairs adjacent (+Im first).
// ---------------------------------------------------------------------------
struct cplx {
    double x, y;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.x, -a.y}; }
__device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double cabsd(cplx a) { return hypot(a.x, a.y); }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    const double s = fabs(b.x) + fabs(b.y);
    const cplx as = {a.x / s, a.y / s}, bs = {b.x / s, b.y / s};
    const double den = bs.x * bs.x + bs.y * bs.y;
    return {(as.x * bs.x + as.y * bs.y) / den, (as.y * bs.x - as.x * bs.y) / den};
}
__device__ __forceinline__ cplx csqrt_(cplx a) {
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

constexpr int kMaxR = 32;

__global__ void __launch_bounds__(64)
eig_small_kernel(const double* __restrict__ At, int r, double* __restrict__ lam_out,
                 double* __restrict__ W_out, int* status) {
    extern __shared__ double esm[];
    typedef double RowD[kMaxR + 1];
    typedef cplx RowC[kMaxR + 1];
    RowD* Hr = reinterpret_cast<RowD*>(esm);
    RowD* Q = Hr + kMaxR;
    RowC* T = reinterpret_cast<RowC*>(Q + kMaxR);
    RowC* Zs = T + kMaxR;
    RowC* X = Zs + kMaxR;
    __shared__ double hv[kMaxR];
    __shared__ cplx lamv[kMaxR];
    __shared__ int order[kMaxR];
    __shared__ double scal[4];
    __shared__ cplx rot[2];
    __shared__ int flag[2];
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    for (int idx = tid; idx < r * r; idx += nt) {
        const int i = idx % r, c = idx / r;
        Hr[i][c] = At[static_cast<int64_t>(c) * r + i];
        Q[i][c] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    // --- Hessenberg reduction ---
    for (int j = 0; j + 2 < r; ++j) {
        if (tid == 0) {
            double nrm2 = 0.0;
            for (int i = j + 1; i < r; ++i) nrm2 += Hr[i][j] * Hr[i][j];
            const double nrm = sqrt(nrm2);
            const double x0 = Hr[j + 1][j];
            if (nrm == 0.0) {
                scal[0] = 0.0;
            } else {
                for (int i = j + 1; i < r; ++i) hv[i] = Hr[i][j];
                hv[j + 1] += (x0 >= 0.0 ? nrm : -nrm);
                double vn = 0.0;
                for (int i = j + 1; i < r; ++i) vn += hv[i] * hv[i];
                scal[0] = vn > 0.0 ? 2.0 / vn : 0.0;
            }
        }
        __syncthreads();
        const double beta = scal[0];
        if (beta != 0.0) {
            // rows: H[j+1:, c] -= beta v (v^T H[j+1:, c]) for every column c
            for (int c = tid; c < r; c += nt) {
                double s = 0.0;
                for (int i = j + 1; i < r; ++i) s += hv[i] * Hr[i][c];
                s *= beta;
                for (int i = j + 1; i < r; ++i) Hr[i][c] -= s * hv[i];
            }
            __syncthreads();
            // columns: H[i, j+1:] -= beta (H[i, j+1:] v) v^T, same for Q
            for (int i = tid; i < r; i += nt) {
                double s = 0.0, sq = 0.0;
                for (int c = j + 1; c < r; ++c) {
                    s += Hr[i][c] * hv[c];
                    sq += Q[i][c] * hv[c];
                }
                s *= beta;
                sq *= beta;
                for (int c = j + 1; c < r; ++c) {
                    Hr[i][c] -= s * hv[c];
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
    // --- complex Schur form by single-shift QR ---
    int hi = r - 1, its = 0, total = 0;
    bool failed = false;
    while (hi > 0) {
        if (tid == 0) {
            int lo = hi;
            while (lo > 0) {
                const double s = cabsd(T[lo - 1][lo - 1]) + cabsd(T[lo][lo]);
                if (cabsd(T[lo][lo - 1]) <= kEps * s) { T[lo][lo - 1] = {0.0, 0.0}; break; }
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
            const cplx a = T[hi - 1][hi - 1], b = T[hi - 1][hi], c = T[hi][hi - 1], d = T[hi][hi];
            cplx mu;
            if (its % 11 == 0) {
                mu = {d.x + cabsd(c), d.y};
            } else {
                const cplx half = {0.5 * (a.x - d.x), 0.5 * (a.y - d.y)};
                const cplx bc = cmul(b, c);
                const cplx disc = csqrt_(cadd(cmul(half, half), bc));
                const cplx s1 = cadd(half, disc), s2 = csub(half, disc);
                cplx mu1 = d, mu2 = d;
                if (cabs2(s1) > 0.0) mu1 = csub(d, cdiv(bc, s1));
                if (cabs2(s2) > 0.0) mu2 = csub(d, cdiv(bc, s2));
                mu = (cabs2(csub(mu1, d)) <= cabs2(csub(mu2, d))) ? mu1 : mu2;
            }
            rot[1] = mu;
        }
        __syncthreads();
        const cplx mu = rot[1];
        for (int q = lo; q < hi; ++q) {
            if (tid == 0) {
                cplx x, y;
                if (q == lo) { x = csub(T[lo][lo], mu); y = T[lo + 1][lo]; }
                else { x = T[q][q - 1]; y = T[q + 1][q - 1]; }
                const double rr = sqrt(cabs2(x) + cabs2(y));
                if (rr == 0.0) { rot[0] = {1.0, 0.0}; scal[1] = 0.0; scal[2] = 0.0; }
                else { rot[0] = {x.x / rr, x.y / rr}; scal[1] = y.x / rr; scal[2] = y.y / rr; }
            }
            __syncthreads();
            const cplx cg_ = rot[0];
            const cplx sg = {scal[1], scal[2]};
            // rows q, q+1: [conj(c) conj(s); -s c] applied from the left
            const int col0 = max(q - 1, 0);
            for (int c = col0 + tid; c < r; c += nt) {
                const cplx t0 = T[q][c], t1 = T[q + 1][c];
                T[q][c] = cadd(cmul(cconj(cg_), t0), cmul(cconj(sg), t1));
                T[q + 1][c] = csub(cmul(cg_, t1), cmul(sg, t0));
            }
            __syncthreads();
            // columns q, q+1: multiply by G^H from the right
            const int row1 = min(q + 3, hi + 1);
            for (int i = tid; i < r; i += nt) {
                if (i < row1) {
                    const cplx t0 = T[i][q], t1 = T[i][q + 1];
                    T[i][q] = cadd(cmul(t0, cg_), cmul(t1, sg));
                    T[i][q + 1] = csub(cmul(t1, cconj(cg_)), cmul(t0, cconj(sg)));
                }
                const cplx z0 = Zs[i][q], z1 = Zs[i][q + 1];
                Zs[i][q] = cadd(cmul(z0, cg_), cmul(z1, sg));
                Zs[i][q + 1] = csub(cmul(z1, cconj(cg_)), cmul(z0, cconj(sg)));
            }
            __syncthreads();
            if (tid == 0 && q > lo) T[q + 1][q - 1] = {0.0, 0.0};
            __syncthreads();
        }
    }
    if (failed) {
        if (tid == 0) record_status(status, CDMD_ERR_NOT_CONVERGED);
    }
    __syncthreads();
    // --- eigenvectors of the triangular T ---
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
            cplx s = {0.0, 0.0};
            for (int q = i + 1; q <= j; ++q) s = cadd(s, cmul(T[i][q], X[q][j]));
            cplx den = csub(T[i][i], T[j][j]);
            if (cabsd(den) < small) den = {small, 0.0};
            const cplx v = cdiv(s, den);
            X[i][j] = {-v.x, -v.y};
        }
        lamv[j] = T[j][j];
    }
    __syncthreads();
    // W = Q (Z X): first Zs <- Zs X (column j by thread j), then Q
    for (int j = tid; j < r; j += nt) {
        cplx tmp[kMaxR];
        for (int i = 0; i < r; ++i) {
            // X is upper triangular: X[q][j] = 0 for q > j
            cplx s = {0.0, 0.0};
            for (int q = 0; q <= j; ++q) s = cadd(s, cmul(Zs[i][q], X[q][j]));
            tmp[i] = s;
        }
        for (int i = 0; i < r; ++i) {
            double re = 0.0, im = 0.0;
            for (int q = 0; q < r; ++q) {
                re += Q[i][q] * tmp[q].x;
                im += Q[i][q] * tmp[q].y;
            }
            X[i][j] = {re, im};   // column j is only touched by this thread
        }
    }
    __syncthreads();
    // normalise: unit norm, largest-modulus entry real positive
    for (int j = tid; j < r; j += nt) {
        double nrm2 = 0.0, best = -1.0;
        int bi = 0;
        for (int i = 0; i < r; ++i) {
            const double a2 = cabs2(X[i][j]);
            nrm2 += a2;
            if (a2 > best) { best = a2; bi = i; }
        }
        const double nrm = sqrt(nrm2);
        cplx ph = {1.0, 0.0};
        if (best > 0.0) {
            const double ab = sqrt(best);
            ph = {X[bi][j].x / ab, -X[bi][j].y / ab};   // conj(x_b) / |x_b|
        }
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int i = 0; i < r; ++i) {
            const cplx v = cmul(X[i][j], ph);
            X[i][j] = {v.x * inv, v.y * inv};
        }
        X[bi][j].y = 0.0;
    }
    __syncthreads();
    // ordering (pair-aware, as the paper's modes come in conjugate pairs)
    if (tid == 0) {
        bool used[kMaxR];
        double key_abs[kMaxR], key_im[kMaxR];
        int first[kMaxR], second[kMaxR];
        int nu = 0;
        for (int i = 0; i < r; ++i) used[i] = false;
        for (int pass = 0; pass < r; ++pass) {
            // next unused index with the largest imaginary part
            int i = -1;
            for (int q = 0; q < r; ++q)
                if (!used[q] && (i < 0 || lamv[q].y > lamv[i].y)) i = q;
            used[i] = true;
            int partner = -1;
            if (lamv[i].y > 0.0) {
                double bd = 1e300;
                for (int q = 0; q < r; ++q) {
                    if (used[q]) continue;
                    const cplx cj = cconj(lamv[i]);
                    const double dd2 = cabsd(csub(lamv[q], cj));
                    if (dd2 < bd) { bd = dd2; partner = q; }
                }
                if (partner >= 0 && !(bd <= 1e-9 * fmax(1.0, cabsd(lamv[i])))) partner = -1;
                if (partner >= 0) used[partner] = true;
            }
            if (i >= 0) {
                key_abs[nu] = cabsd(lamv[i]);
                key_im[nu] = lamv[i].y;
                first[nu] = i;
                second[nu] = partner;
                ++nu;
            }
            bool all = true;
            for (int q = 0; q < r; ++q) all = all && used[q];
            if (all) break;
        }
        // insertion sort of units by (-|lambda|, -Im)
        int perm[kMaxR];
        for (int u = 0; u < nu; ++u) perm[u] = u;
        for (int u = 1; u < nu; ++u) {
            const int cur = perm[u];
            int v = u - 1;
            while (v >= 0) {
                const int o = perm[v];
                const bool before = (key_abs[cur] > key_abs[o]) ||
                                    (key_abs[cur] == key_abs[o] && key_im[cur] > key_im[o]);
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
    __syncthreads();
    for (int j = tid; j < r; j += nt) {
        const int s = order[j];
        lam_out[2 * j] = lamv[s].x;
        lam_out[2 * j + 1] = lamv[s].y;
        for (int i = 0; i < r; ++i) {
            W_out[2 * (static_cast<int64_t>(j) * r + i)] = X[i][s].x;
            W_out[2 * (static_cast<int64_t>(j) * r + i) + 1] = X[i][s].y;
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
__global__ void __launch_bounds__(128)
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

// 9. OMP in Gram form (one thread; r <= 64).  M = Phi_Y^H Phi_Y (Hermitian,
// column-major), cvec = Phi_Y^H y1, y2 = ||y1||^2.  The least-squares fit on
// the selected set solves M_SS beta = c_S through an incrementally grown
// Cholesky factor.
__global__ void omp_kernel(const double* __restrict__ M, const double* __restrict__ cvec,
                           const double* __restrict__ R, const double* __restrict__ lam, int r,
                           int K, int lstsq, double* __restrict__ beta, int32_t* __restrict__ sel,
                           int32_t* __restrict__ nsel_out, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    cplx L[kMaxR][kMaxR];
    cplx bsel[kMaxR];
    cplx ytmp[kMaxR];
    int S[kMaxR];
    bool used[kMaxR];
    const double y2 = R[0];
    auto Mel = [&](int i, int j) -> cplx {   // M[i][j], column-major storage
        return {M[2 * (static_cast<int64_t>(j) * r + i)], M[2 * (static_cast<int64_t>(j) * r + i) + 1]};
    };
    auto cv = [&](int i) -> cplx { return {cvec[2 * i], cvec[2 * i + 1]}; };
    for (int i = 0; i < r; ++i) { used[i] = false; beta[2 * i] = 0.0; beta[2 * i + 1] = 0.0; }
    const int kmax = lstsq ? r : min(K, r);
    int ns = 0;
    double res2 = y2;
    for (int step = 0; step < kmax; ++step) {
        if (!lstsq && res2 <= 1e-24 * y2) break;
        int best = -1;
        if (lstsq) {
            best = step;
        } else {
            double bscore = -1.0;
            double score[kMaxR];
            for (int j = 0; j < r; ++j) {
                score[j] = -1.0;
                if (used[j]) continue;
                const double mjj = Mel(j, j).x;
                if (!(mjj > 0.0)) continue;
                cplx g = cv(j);
                for (int q = 0; q < ns; ++q) g = csub(g, cmul(Mel(j, S[q]), bsel[q]));
                score[j] = sqrt(cabs2(g) / mjj);
                bscore = fmax(bscore, score[j]);
            }
            if (!(bscore > 0.0)) break;
            for (int j = 0; j < r; ++j) {
                if (score[j] < bscore * (1.0 - 1e-9)) continue;
                if (best < 0 || lam[2 * j + 1] > lam[2 * best + 1]) best = j;
            }
        }
        // grow the Cholesky factor with column `best`
        cplx lrow[kMaxR];
        double diag = Mel(best, best).x;
        for (int q = 0; q < ns; ++q) {
            cplx s = Mel(S[q], best);   // M[S_q][best]
            for (int u = 0; u < q; ++u) s = csub(s, cmul(L[q][u], cconj(lrow[u])));
            // L[ns][q] = conj(s / L[q][q]) in the convention M = L L^H
            const cplx v = {s.x / L[q][q].x, s.y / L[q][q].x};
            lrow[q] = cconj(v);
            diag -= cabs2(lrow[q]);
        }
        if (!(diag > kEps * Mel(best, best).x)) {
            if (lstsq) record_status(status, CDMD_ERR_RANK_DEFICIENT);
            break;
        }
        for (int q = 0; q < ns; ++q) L[ns][q] = lrow[q];
        L[ns][ns] = {sqrt(diag), 0.0};
        S[ns] = best;
        used[best] = true;
        ++ns;
        // solve L y = c_S, L^H beta = y
        for (int q = 0; q < ns; ++q) {
            cplx s = cv(S[q]);
            for (int u = 0; u < q; ++u) s = csub(s, cmul(L[q][u], ytmp[u]));
            ytmp[q] = {s.x / L[q][q].x, s.y / L[q][q].x};
        }
        for (int q = ns - 1; q >= 0; --q) {
            cplx s = ytmp[q];
            for (int u = q + 1; u < ns; ++u) s = csub(s, cmul(cconj(L[u][q]), bsel[u]));
            bsel[q] = {s.x / L[q][q].x, s.y / L[q][q].x};
        }
        double cb = 0.0;   // Re(c_S^H beta)
        for (int q = 0; q < ns; ++q) {
            const cplx c = cv(S[q]);
            cb += c.x * bsel[q].x + c.y * bsel[q].y;
        }
        res2 = y2 - cb;
    }
    for (int q = 0; q < ns; ++q) {
        beta[2 * S[q]] = bsel[q].x;
        beta[2 * S[q] + 1] = bsel[q].y;
    }
    for (int q = 0; q < K; ++q) sel[q] = (q < ns) ? S[q] : -1;
    *nsel_out = ns;
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

}  // namespace

cdmd_status launch_decompose(cdmd_ctx* ctx, const double* DY, int k, int n, int r, int K,
                             cdmd_selector selector, double* sigma, double* lambda, double* G,
                             double* PhiY, double* beta, int32_t* sel, int32_t* nsel,
                             cudaStream_t stream) {
    const int p = n - 1;
    // ---- workspace layout (doubles) ----
    const int ntiles = (n + kGT - 1) / kGT;
    const int kchunk = 128;
    const int splits = (k + kchunk - 1) / kchunk;
    const size_t n_gram_part = static_cast<size_t>(splits) * n * n;
    const size_t n_R = static_cast<size_t>(n) * n;
    const size_t n_Hv = static_cast<size_t>(p) * p;
    const size_t n_vec = static_cast<size_t>(p);
    const size_t n_Z = static_cast<size_t>(p) * r;
    const size_t n_work = static_cast<size_t>(r) * 6 * p;
    const size_t n_small = static_cast<size_t>(r) * r * 2;
    size_t total = n_gram_part + n_R + n_Hv + 3 * n_vec + r + n_Z + n_work + 2 * n_Z + n_small * 3 + 2 * r + 64;
    double* ws = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_EIG, total * sizeof(double), reinterpret_cast<void**>(&ws));
    if (st != CDMD_OK) return st;
    double* gpart = ws;
    double* R = gpart + n_gram_part;
    double* Hv = R + n_R;
    double* htau = Hv + n_Hv;
    double* dd = htau + n_vec;
    double* ee = dd + n_vec;
    double* lamT = ee + n_vec;
    double* Z = lamT + r;
    double* work = Z + n_Z;
    double* V = work + n_work;
    double* B = V + n_Z;
    double* At = B + n_Z;
    double* W = At + n_small;
    double* M = W + n_small;
    double* cvec = M + n_small;

    // 1. Gram
    gram_partial_kernel<<<dim3(ntiles, ntiles, splits), 256, 0, stream>>>(DY, k, n, kchunk, gpart);
    CDMD_CHECK_LAUNCH("gram_partial_kernel");
    gram_reduce_kernel<<<(n * n + 255) / 256, 256, 0, stream>>>(gpart, splits, n, R, ctx->d_status);
    CDMD_CHECK_LAUNCH("gram_reduce_kernel");

    // 2. tridiagonalisation on a cluster (16 CTAs if the device allows, else 8)
    if (p >= 3) {
        int csize = 16;
        for (;;) {
            const int rows_per = (p + csize - 1) / csize;
            const size_t smem = (static_cast<size_t>(rows_per) * p + 5 * static_cast<size_t>(p) + 34) * sizeof(double);
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem)));
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
                if (csize > 8) { csize = 8; continue; }
                return fail(CDMD_ERR_UNSUPPORTED, "no room for a %d-CTA cluster of %zu bytes each", csize, smem);
            }
            CDMD_CHECK_CUDA(cudaLaunchKernelEx(&cfg, tridiag_kernel, static_cast<const double*>(R), n, p, Hv,
                                               htau, dd, ee));
            break;
        }
    } else {
        // p <= 2: A is already tridiagonal
        tiny_tridiag_kernel<<<1, 1, 0, stream>>>(R, n, p, dd, ee, htau);
        CDMD_CHECK_LAUNCH("tiny_tridiag_kernel");
    }
    // 3. eigenpairs of T
    {
        const size_t esm = 9 * static_cast<size_t>(p) * sizeof(double);
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(tridiag_eigpair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(esm)));
        tridiag_eigpair_kernel<<<r, 32, esm, stream>>>(dd, ee, p, r, lamT, Z, ctx->d_status);
    }
    CDMD_CHECK_LAUNCH("tridiag_eigpair_kernel");
    orthonormalise_kernel<<<1, 256, 0, stream>>>(Z, p, r);
    CDMD_CHECK_LAUNCH("orthonormalise_kernel");
    backtransform_kernel<<<r, 32, p * sizeof(double), stream>>>(Z, Hv, htau, lamT, R, n, p, r, V, B, sigma,
                                                                 ctx->d_status);
    CDMD_CHECK_LAUNCH("backtransform_kernel");
    // 4. A~ and its eigen-decomposition
    atilde_kernel<<<r, 32, 0, stream>>>(V, B, sigma, p, r, At);
    CDMD_CHECK_LAUNCH("atilde_kernel");
    {
        const size_t esmem = static_cast<size_t>(kMaxR) * (kMaxR + 1) * (2 * sizeof(double) + 3 * sizeof(cplx));
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(eig_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(esmem)));
        eig_small_kernel<<<1, 64, esmem, stream>>>(At, r, lambda, W, ctx->d_status);
    }
    CDMD_CHECK_LAUNCH("eig_small_kernel");
    // 5. G, Gram-form quantities, selection
    gmat_kernel<<<(p * r + 127) / 128, 128, 0, stream>>>(V, sigma, W, p, r, G);
    CDMD_CHECK_LAUNCH("gmat_kernel");
    hmat_kernel<<<r, 128, 2 * p * sizeof(double), stream>>>(R, G, n, p, r, M, cvec);
    CDMD_CHECK_LAUNCH("hmat_kernel");
    omp_kernel<<<1, 32, 0, stream>>>(M, cvec, R, lambda, r, K, selector == CDMD_SEL_LSTSQ ? 1 : 0, beta, sel,
                                     nsel, ctx->d_status);
    CDMD_CHECK_LAUNCH("omp_kernel");
    if (PhiY != nullptr) {
        const int64_t tot = static_cast<int64_t>(k) * r;
        phiy_kernel<<<static_cast<unsigned>((tot + 127) / 128), 128, 0, stream>>>(DY, G, k, p, r, PhiY);
        CDMD_CHECK_LAUNCH("phiy_kernel");
    }
    return CDMD_OK;
}

}  // namespace cdmd
