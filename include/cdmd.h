/*
 * cdmd.h -- C ABI of libcdmd: compressed dynamic mode decomposition (cDMD)
 * for video background modelling on one NVIDIA GB300 (sm_103a).
 *
 * Method: Erichson, Brunton & Kutz, "Compressed Dynamic Mode Decomposition for
 * Background Modeling" (arXiv 1512.04205), Algorithm 1 with the sparse-coding
 * mode selection of Remark 3 and the threshold mask of Eq. (thres).
 *
 * Letters (the paper swaps some of them; see its Appendix A):
 *   m  pixels per frame        (paper: n)
 *   n  frames in the clip      (paper: m)
 *   k  sketch rows / measurements (paper: p)
 *   r  target rank             (paper: k)
 *   K  non-zero amplitudes kept by the sparse coding (paper: K)
 *
 * Data layout (all device memory unless stated otherwise):
 *   D      uint8 video, frame-major: pixel j of frame t at D[t*ldd + j],
 *          ldd >= m.  This is the paper's m x n video matrix stored by columns.
 *   DY     double, k x n column-major (DY[t*k + i]): the sketch C*D.  Its
 *          columns 0..n-2 are Y and columns 1..n-1 are Y' (Eq. YCX).
 *   complex values are interleaved (re, im) pairs of the stated real type.
 *   G      double complex, (n-1) x r column-major: G = V S^-1 W.
 *   Phi    float complex, pixel-major: mode c of pixel j at Phi[j*ncols + c].
 *   mask   uint32, frame-major: frame t holds ceil(m/32) words at
 *          mask[t*ceil(m/32) + j/32]; pixel j is bit j%32 (LSB first).
 *
 * Ownership: the caller owns every pointer it passes; the library never frees
 * them.  A context owns only its workspace and its device status word.
 *
 * Execution: every call that takes a stream enqueues its kernels on that
 * stream (a cudaStream_t passed as void*; NULL = legacy default stream) and
 * returns without synchronising.  Argument and launch errors are returned
 * synchronously.  Numerical errors found on the device (iteration limits,
 * rank deficiency, non-finite data) are recorded in the context's status word
 * and returned by cdmd_status_sync().  No call traps, aborts or spins without
 * a bound.  Calls on one context must not run concurrently from several host
 * threads.  A context's workspace grows on first use of a larger problem; the
 * first call at the largest size must happen before any stream capture.
 */
#ifndef CDMD_H
#define CDMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CDMD_OK = 0,
    CDMD_ERR_INVALID_ARG = 1,    /* bad size, pointer, alignment or enum     */
    CDMD_ERR_CUDA = 2,           /* a CUDA runtime call or launch failed     */
    CDMD_ERR_NOMEM = 3,          /* workspace allocation failed              */
    CDMD_ERR_NOT_CONVERGED = 4,  /* an eigen-iteration hit its bound         */
    CDMD_ERR_RANK_DEFICIENT = 5, /* sigma_r of the sketch is zero            */
    CDMD_ERR_NONFINITE = 6,      /* NaN or Inf met in the sketch             */
    CDMD_ERR_UNSUPPORTED = 7,    /* valid request the library does not serve */
    CDMD_ERR_TIMEOUT = 8         /* a kernel's bounded wait gave up          */
} cdmd_status;

/* Measurement matrix C (Section 3.3).  Gaussian and Rademacher entries are
 * pure functions of (seed, row i, pixel j) through Philox4x32-10 and are
 * generated inside the sketch kernel, never stored:
 *   GAUSSIAN    counter (j, i/4, 0, 0), word i%4; words (0,1) and (2,3) are
 *               Box-Muller pairs with U(w) = (w + 1/2) 2^-32:
 *               z_even = sqrt(-2 ln U(w_a)) cos(2 pi U(w_b)),
 *               z_odd  = sqrt(-2 ln U(w_a)) sin(2 pi U(w_b)).
 *   RADEMACHER  counter (j, i/128, 1, 0); bit (i%128)%32 of word (i%128)/32;
 *               clear = +1, set = -1.
 * The gather forms are built once into a caller-owned cdmd_measure:
 *   SPARSE      counter (j, i/4, 2, 0), word w = word i%4; entry non-zero iff
 *               w < floor(2^32 * density), then +1 for even w, else -1.
 *   ROWSAMPLE   Floyd's sampling of k distinct pixels (row i of C = the i-th
 *               smallest selected pixel): for t = m-k .. m-1 the draw is
 *               v = floor(((w1 << 32) | w0) * (t+1) / 2^64) from words 0,1 of
 *               counter (t, 0, 3, 0); v is taken unless already taken, else t.
 *   SRFT        subsampled randomized Fourier transform C = R F D (Section
 *               3.3, after Woolfe et al.): D = diag(exp(i theta_j)) with
 *               theta_j = 2 pi U(w0), w0 word 0 of counter (j, 0, 5, 0); F the
 *               unnormalised m-point DFT, F(f, j) = exp(-2 pi i f j / m); R
 *               keeps q = ceil(k/2) distinct frequencies s_0 < s_1 < ... drawn
 *               from [0, m) by Floyd's sampling as for ROWSAMPLE but on
 *               counters (t, 0, 6, 0).  The real sketch rows are the real and
 *               imaginary parts of the kept complex measurements: row 2a =
 *               Re(F D)[s_a, :], row 2a+1 = Im(F D)[s_a, :] (odd k: the last
 *               frequency keeps its real row only).  Applied by an FFT, never
 *               formed.
 * The key of every counter is (seed & 0xffffffff, seed >> 32). */
typedef enum {
    CDMD_C_GAUSSIAN = 0,
    CDMD_C_RADEMACHER = 1,
    CDMD_C_SPARSE = 2,
    CDMD_C_ROWSAMPLE = 3,
    CDMD_C_SRFT = 4
} cdmd_ctype;

/* Arithmetic of the two contractions (sketch and lift).
 *   FP32    CUDA-core FP32 FMA, FP32 partial sums over pixel chunks reduced
 *           in FP64.
 *   BF16X2  tcgen05 tensor cores: the sketch's uint8 pixels are exact in
 *           BF16 and its Gaussian C is split into hi + lo BF16 parts
 *           (Rademacher C, +1 / -1, is exact and takes one product); the
 *           lift's pixels are exact in FP16 and G, scaled by a power of two
 *           per mode, is split into hi + lo FP16 parts.  FP32 accumulation
 *           in tensor memory. */
typedef enum { CDMD_PREC_FP32 = 0, CDMD_PREC_BF16X2 = 1 } cdmd_prec;

/* Background of pixel j in frame t from the selected modes S:
 *   MODULUS  | sum_{s in S} Phi_js beta_s lambda_s^t |        (time-varying)
 *   REAL     Re( sum_{s in S} Phi_js beta_s lambda_s^t )     (footnote of
 *            Eq. DMDTerms: only the real part is kept)
 *   STATIC   | sum_{s in S} Phi_js beta_s |, the x_BG = Phi beta of
 *            Section 2.3, the same for every frame. */
typedef enum { CDMD_BG_MODULUS = 0, CDMD_BG_REAL = 1, CDMD_BG_STATIC = 2 } cdmd_bgmode;

/* Amplitudes / mode selection (Algorithm 1 step 9, Remark 3).
 *   OMP    orthogonal matching pursuit on the compressed modes Phi_Y with
 *          target y1 = DY[:,0], K picks.
 *   LSTSQ  least squares on all r compressed modes (OMP with K = r).
 *   MLP    learned selection (no counterpart in the paper, which uses sparse
 *          coding, Section 2.3): the K modes of highest score under the model
 *          loaded by cdmd_selector_load, amplitudes by least squares on them;
 *          if the relative residual ||y1 - Phi_Y,S beta|| / ||y1|| exceeds the
 *          model's tol, OMP runs instead (counted, see
 *          cdmd_selector_fallbacks). */
typedef enum { CDMD_SEL_OMP = 0, CDMD_SEL_LSTSQ = 1, CDMD_SEL_MLP = 2 } cdmd_selector;

typedef struct cdmd_ctx cdmd_ctx;

/* Gather / transform measurement matrix, device arrays owned by the caller.
 *   SPARSE     CSC by pixel: col_ptr[m+1] (int64), row_idx[nnz] (int32):
 *              bits 0..30 = row i, bit 31 set = entry -1 (clear = +1).
 *   ROWSAMPLE  rows[k] (int64): the selected pixel of row i, increasing.
 *   SRFT       rows[ceil(k/2)] (int64): the kept frequencies, increasing.
 * cdmd_measure_build fills it; its capacity fields say how large the caller's
 * arrays are. */
typedef struct {
    cdmd_ctype ctype;
    int32_t k;
    int64_t m;
    uint64_t seed;
    double density;
    int64_t* col_ptr;       /* SPARSE: m+1 entries                         */
    int32_t* row_idx;       /* SPARSE: nnz_capacity entries                */
    int64_t nnz_capacity;   /* SPARSE: entries available at row_idx        */
    int64_t* rows;          /* ROWSAMPLE: k entries                        */
} cdmd_measure;

/* ---- context ------------------------------------------------------------ */

/* Create a context bound to CUDA device `device`.  Allocates the device
 * status word.  Returns CDMD_ERR_INVALID_ARG for a NULL ctx or bad device. */
cdmd_status cdmd_create(cdmd_ctx** ctx, int device);

/* Free the context's workspace and status word (NULL is ignored).  Waits for
 * the device to finish work that uses the workspace. */
void cdmd_destroy(cdmd_ctx* ctx);

/* Cap the grids of the full-data passes (sketch, lift, subtract) issued
 * through this context at `max_sms` streaming multiprocessors' worth of CTAs
 * (0 = the whole device; larger values are clamped to it).  The paper has no
 * counterpart: Algorithm 1 treats one clip at a time.  The cap leaves SMs free
 * so that the latency-bound small solves of another clip, issued through
 * another context on another stream, run beside this context's passes.
 * The cap changes results only through the split of the sketch's pixel sums
 * (rounding order).  CDMD_ERR_INVALID_ARG for a NULL ctx or a negative cap. */
cdmd_status cdmd_set_sm_limit(cdmd_ctx* ctx, int max_sms);

/* Message of the last error returned on this host thread ("" if none). */
const char* cdmd_last_error(void);

/* Name of a status code. */
const char* cdmd_status_string(cdmd_status s);

/* Synchronise `stream`, then return and clear the numerical status recorded
 * on the device by the calls enqueued so far (CDMD_OK if none). */
cdmd_status cdmd_status_sync(cdmd_ctx* ctx, void* stream);

/* Failure detection without a GPU fault: enqueue on `stream` one kernel that
 * waits on an mbarrier nothing ever arrives at, with the bounded wait every
 * tensor-core kernel of the library uses (a global-timer limit of limit_us
 * microseconds, 1..2,000,000).  The wait gives up, records
 * CDMD_ERR_TIMEOUT in the context's status word (returned and cleared by the
 * next cdmd_status_sync) and the kernel returns; the context stays usable.
 * CDMD_ERR_INVALID_ARG for a NULL ctx or limit_us outside the range. */
cdmd_status cdmd_selftest_wait(cdmd_ctx* ctx, uint32_t limit_us, void* stream);

/* The FP64 reciprocal and reciprocal square root the small solves use on
 * their latency-critical paths (Newton-Raphson from the hardware
 * approximations, two steps), applied to n doubles: rcp[i] = 1/a[i],
 * rsqrt[i] = 1/sqrt(a[i]) (either output may be NULL).  The paper has no
 * counterpart; this lets a test bound their error against IEEE division and
 * square root.  Inputs must be normal positive numbers whose reciprocal is
 * normal (subnormals are flushed to zero).  Device arrays, enqueued on
 * `stream`.  CDMD_ERR_INVALID_ARG for a NULL ctx, n < 0 or a NULL a. */
cdmd_status cdmd_selftest_recip(cdmd_ctx* ctx, const double* a, int64_t n, double* rcp, double* rsqrt,
                                void* stream);

/* ---- measurement matrices (Section 3.3) ---------------------------------- */

/* Exact number of non-zeros of the SPARSE matrix for (m, k, seed, density),
 * counted on the device and returned on the host (synchronises `stream`).
 * Use it to size row_idx before cdmd_measure_build. */
cdmd_status cdmd_measure_sparse_nnz(cdmd_ctx* ctx, int64_t m, int k, uint64_t seed,
                                    double density, int64_t* nnz, void* stream);

/* Fill a SPARSE, ROWSAMPLE or SRFT cdmd_measure (fields ctype, k, m, seed,
 * density and the arrays must be set).  Enqueued on `stream`; ROWSAMPLE and
 * SRFT are drawn on the device with no host round trip (graph-capturable
 * once the context's workspace has been sized by a first call).  ROWSAMPLE
 * needs 1 <= k <= m; SRFT needs ceil(k/2) <= m and k <= 8192; SPARSE needs
 * 0 < density <= 1 and nnz_capacity >= the count from
 * cdmd_measure_sparse_nnz (else CDMD_ERR_INVALID_ARG). */
cdmd_status cdmd_measure_build(cdmd_ctx* ctx, cdmd_measure* meas, void* stream);

/* ---- pass (a): sketch  DY = C D  (Algorithm 1 steps 2-3, Eq. YCX) -------- */

/* Dense Gaussian / Rademacher C generated in-kernel from `seed` (never
 * stored).  D: m x n frames (n >= 2), ldd >= m.  DY: k x n doubles
 * (column-major, ld = k), overwritten.  prec selects FP32 CUDA-core or
 * tensor-core arithmetic (BF16X2: hi+lo BF16 for Gaussian C, one exact BF16
 * product for Rademacher C, whose sketch is then exact while every partial
 * sum stays below 2^24; needs a 16-byte aligned D with ldd % 16 == 0, and
 * sketches clips longer than 256 frames in 256-frame pieces, the product
 * being linear in the frames). */
cdmd_status cdmd_sketch(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                        cdmd_ctype ctype, int k, uint64_t seed, cdmd_prec prec,
                        double* DY, void* stream);

/* Several clips sketched with one measurement matrix (Algorithm 1 steps 2-3
 * for each clip, one C): DY[i] = C D[i] for i < nclips, where every clip has
 * the same pixel count m and C is drawn from the same (ctype, k, seed) as
 * cdmd_sketch draws it.  This is the case of one camera (one sensing matrix)
 * whose video is processed window by window.  With prec = CDMD_PREC_BF16X2,
 * a Gaussian or Rademacher C and nclips >= 2, each clip's frames are first
 * widened to a BF16 copy in the context's workspace (2 m n bytes per clip),
 * then the frames of all clips are packed 512 to a launch: each entry of C
 * drawn feeds every frame of the launch, whichever clip it belongs to.  A
 * single clip, and the FP32 precision, go as cdmd_sketch would.  D[i],
 * n[i], ldd[i], DY[i] as for cdmd_sketch; the four arrays are host arrays of
 * nclips entries (D[i], DY[i] device pointers).  Results agree with
 * cdmd_sketch's up to the rounding order of the split partial sums.
 * CDMD_ERR_INVALID_ARG (naming the clip) for nclips < 1 or any argument
 * cdmd_sketch would reject. */
cdmd_status cdmd_sketch_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m,
                               const int* n, const int64_t* ldd, cdmd_ctype ctype, int k,
                               uint64_t seed, cdmd_prec prec, double* const* DY, void* stream);

/* Sparse or single-pixel C applied as a gather (one pass over D; exact
 * integer sums), or SRFT C applied by a fast transform (one pass over D: an
 * FFT of length N2 down the N1 strided columns of each frame, m = N1 N2 with
 * N2 the largest divisor of m up to 1024 whose prime factors are 2, 3 and 5,
 * then one twiddled sum over the columns per kept frequency; FP32 arithmetic,
 * FP64 sums of the column-group partials).  meas must have been filled by
 * cdmd_measure_build for the same m.  DY as for cdmd_sketch with
 * k = meas->k. */
cdmd_status cdmd_sketch_gather(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               const cdmd_measure* meas, double* DY, void* stream);

/* ---- small solves on the device (Algorithm 1 steps 4-7, 9; Remark 3) ----- */

/* From DY (k x n, ld = k) compute, in FP64 on the device:
 *   sigma  [r]            leading singular values of Y = DY[:, 0:n-1]
 *   lambda [2r]           eigenvalues of A~ = U^T Y' V S^-1 (complex)
 *   G      [2 (n-1) r]    V S^-1 W, column-major complex (eigenvectors W of
 *                         unit 2-norm, largest-modulus entry real positive)
 *   PhiY   [2 k r]        Y' G, column-major complex (may be NULL)
 *   beta   [2r]           amplitude of each mode, 0 for modes not selected
 *   sel    [K]            selected modes in pick order, -1 after the last
 *   nsel   [1]            number of modes selected
 * Eigenvalues are ordered by descending modulus (conjugate pairs adjacent,
 * positive imaginary part first).  The SVD is taken from the eigen-
 * decomposition of the Gram matrix Y^T Y (method of snapshots).
 * Requires 1 <= r <= min(k, n-1), 1 <= K <= r, n <= 512, k >= 1. */
cdmd_status cdmd_decompose(cdmd_ctx* ctx, const double* DY, int k, int n, int r, int K,
                           cdmd_selector selector, double* sigma, double* lambda,
                           double* G, double* PhiY, double* beta, int32_t* sel,
                           int32_t* nsel, void* stream);

/* ---- exact DMD, the comparator (Section 2.1; Section 4, Computational
 * Performance) --------------------------------------------------------------
 *
 * Exact DMD takes the SVD of X itself instead of a sketch.  In the method of
 * snapshots every quantity the small solves use is a block of the n x n Gram
 * R = D^T D of the video (X^T X, X^T X', X'^T X', X'^T x1), so exact DMD is
 * cdmd_snapshot_gram, cdmd_decompose_gram, then the same lift and subtract.
 *
 * cdmd_snapshot_gram: R[s*n + t] = sum_j D[s*ldd + j] D[t*ldd + j] (FP64,
 * device, n x n, exactly symmetric).  The products are exact (uint8 in
 * FP16 on the tensor cores); sums accumulate in FP32 over each SM's pixel
 * range (the accumulation truncates: relative error <= 2^-23 per 16-pixel
 * step of that range, coherent) and the ranges are added in FP64.  Needs 2 <= n <= 256, D 16-byte aligned and
 * ldd % 16 == 0 (else CDMD_ERR_UNSUPPORTED).
 *
 * cdmd_decompose_gram: the outputs of cdmd_decompose (no PhiY) from a Gram R
 * (device, n x n, symmetric) instead of DY: the SVD of X = D[:, 0:n-1] from
 * the eigen-decomposition of R[0:n-1, 0:n-1], A~ = S^-1 V^T R[0:n-1, 1:n] V
 * S^-1, and the selection on the full modes Phi = X' G with x1 = D[:, 0]
 * (Section 2.3, Eq. sparsecoding) in Gram form.  Selector OMP or LSTSQ
 * (CDMD_ERR_INVALID_ARG for MLP, whose network is trained on compressed
 * modes).  Requires 1 <= r <= min(32, n-1), 1 <= K <= r, n <= 512. */
cdmd_status cdmd_snapshot_gram(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                               double* R, void* stream);
cdmd_status cdmd_decompose_gram(cdmd_ctx* ctx, const double* R, int n, int r, int K,
                                cdmd_selector selector, double* sigma, double* lambda,
                                double* G, double* beta, int32_t* sel, int32_t* nsel,
                                void* stream);

/* cdmd_decompose with the target rank chosen on the device by the optimal
 * hard threshold for singular values (Remark 2; Gavish and Donoho, unknown
 * noise level; Section 4 uses it for every batch): with q = min(k, n-1),
 * beta = q / max(k, n-1) and y_med the median of the q largest singular
 * values of Y, tau = omega(beta) y_med with
 *   omega(beta) = 0.56 beta^3 - 0.95 beta^2 + 1.82 beta + 1.43,
 * and r = #{sigma_i > tau} clamped to [1, r_max].  K is capped at r.
 * Outputs are sized as for cdmd_decompose with r = r_max; the first r
 * entries (columns) are written and sel holds -1 past the capped K.
 * *r_out (host) receives r, *tau_out (host, may be NULL) tau.  Unlike the
 * other calls this one synchronises `stream` once (after the tridiagonal
 * reduction), because the launches that follow are sized by r; it is not
 * graph-capturable.  Requires 1 <= r_max <= min(32, k, n-1), 1 <= K <= r_max. */
cdmd_status cdmd_decompose_auto(cdmd_ctx* ctx, const double* DY, int k, int n, int r_max, int K,
                                cdmd_selector selector, double* sigma, double* lambda,
                                double* G, double* PhiY, double* beta, int32_t* sel,
                                int32_t* nsel, int* r_out, double* tau_out, void* stream);

/* ---- pass (b): mode lift  Phi = X' G  (Algorithm 1 step 8, Eq. cDMDModes) */

/* Phi[j*ncols + c] = sum_{t=0}^{n-2} D[(t+1)*ldd + j] * G[:, cols[c]] for the
 * ncols modes listed in `cols` (device int32, NULL = modes 0..ncols-1; a
 * negative entry yields a zero column).  G: (n-1) x r complex double.
 * Phi: m x ncols complex float, pixel-major.  ncols <= 64.  BF16X2 (FP16
 * hi + lo parts of G on the tensor cores, about 2^-21 relative) needs a
 * 16-byte aligned D and ldd % 16 == 0 (else CDMD_ERR_INVALID_ARG); clips
 * longer than 256 frames are lifted in chunks of at most 255 frames of X',
 * the later chunks adding into Phi (the product is linear in the frames). */
cdmd_status cdmd_lift(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                      const double* G, int r, const int32_t* cols, int ncols,
                      cdmd_prec prec, float* Phi, void* stream);

/* ---- pass (c): background, threshold, bit-packed mask (Eq. DMDTerms, thres)
 *
 * For column c of Phi (c < ncols) the mode is s = cols[c] (device int32;
 * c skipped when negative); its amplitude is beta[s] and eigenvalue
 * lambda[s] (both complex double, length r).  mask bit (j, t) is set iff
 * |D[t*ldd + j] - bg_jt| > tau with bg_jt as selected by `mode`.  bg, if not
 * NULL, receives bg_jt as float, frame-major (bg[t*m + j]).
 * Mask-only MODULUS and REAL calls (bg NULL) with 32 <= n <= 1024, at most 16
 * columns and 16-byte aligned D, ldd and Phi run on the tensor cores, with
 * the background formed from BF16 hi + lo parts (about 2^-16 relative per
 * term): a decision within about a hundredth of a grey level of tau may
 * differ from that of a call with a background output, which sums in FP32. */
cdmd_status cdmd_subtract(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                          const float* Phi, int ncols, const int32_t* cols,
                          const double* beta, const double* lambda, int r,
                          float tau, cdmd_bgmode mode, uint32_t* mask, float* bg,
                          void* stream);

/* ---- mask post-pass: 3 x 3 median filter (Section 4: the BMC figure's
 * median-filtered masks; the Discussion's median-filter post-processing)
 *
 * mask and out are device arrays of n frames of ceil(W*H/32) uint32 words,
 * laid out as for cdmd_subtract with pixel j of a frame at row j / W,
 * column j % W.  Output bit (j, t) is the median of the 3 x 3 neighbourhood
 * of pixel j in frame t, neighbours outside the frame counting as 0, i.e. 1
 * iff at least five of the nine are 1.  Bits of mask past W*H are ignored;
 * those of out are written 0.  The caller owns both; they must not overlap
 * (no in-place filtering) and must be 4-byte aligned.
 * CDMD_ERR_INVALID_ARG for NULL or overlapping arrays, W or H < 1,
 * W*H > 2^31 - 1, or n outside [1, 262140]. */
cdmd_status cdmd_median3x3(cdmd_ctx* ctx, const uint32_t* mask, int64_t W, int64_t H, int n,
                           uint32_t* out, void* stream);

/* ---- whole pipeline ------------------------------------------------------ */

typedef struct {
    int32_t k;              /* sketch rows                                  */
    int32_t r;              /* target rank; 0 = automatic (cdmd_decompose_auto,
                               at most min(32, k, n-1); cdmd_run and
                               cdmd_run_shared then synchronise once per clip) */
    int32_t K;              /* modes kept by the selection                  */
    cdmd_ctype ctype;       /* GAUSSIAN or RADEMACHER (dense, in-kernel)    */
    uint64_t seed;
    cdmd_prec prec;
    cdmd_selector selector;
    cdmd_bgmode bgmode;
    float tau;              /* threshold in grey levels                     */
} cdmd_params;

/* Sketch -> decompose -> lift of the selected modes -> subtract, on device
 * buffers, enqueued on `stream`; intermediates live in the context's
 * workspace and stay valid until the next call on the context (see
 * cdmd_workspace_views).  mask as described above. */
cdmd_status cdmd_run(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                     const cdmd_params* p, uint32_t* mask, void* stream);

/* Exact DMD end to end (Section 2.1 with the selection of Section 2.3):
 * snapshot Gram -> decompose from the Gram -> lift -> subtract, as cdmd_run
 * with no sketch (p->k, p->ctype and p->seed are ignored; p->prec picks the
 * lift).  Requires 1 <= r <= min(32, m, n-1), 1 <= K <= r, selector OMP or
 * LSTSQ, and the snapshot Gram's limits (n <= 256, aligned D). */
cdmd_status cdmd_run_exact(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                           const cdmd_params* p, uint32_t* mask, void* stream);

/* cdmd_run on host memory: copies D_host (m x n frame-major, ldd = m; pinned
 * memory gives full copy bandwidth) to the device, runs the pipeline and
 * copies the mask back to mask_host, all on `stream`, then synchronises the
 * stream and returns the numerical status as cdmd_status_sync does. */
cdmd_status cdmd_run_host(cdmd_ctx* ctx, const uint8_t* D_host, int64_t m, int n,
                          const cdmd_params* p, uint32_t* mask_host, void* stream);

/* cdmd_run for 1..8 clips of the same pixel count and parameters (one
 * measurement matrix): the sketches go through cdmd_sketch_shared, then each
 * clip's small solves, lift and subtract run in order on `stream`, reusing
 * the context's workspace (cdmd_workspace_views then shows the last clip).
 * D, n, ldd and mask are host arrays of nclips entries; each clip as for
 * cdmd_run.  CDMD_ERR_INVALID_ARG (naming the clip) as cdmd_run would, or for
 * nclips outside [1, 8]. */
cdmd_status cdmd_run_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D, int64_t m,
                            const int* n, const int64_t* ldd, const cdmd_params* p,
                            uint32_t* const* mask, void* stream);

/* cdmd_run_shared on host memory: copies each D_host[i] (m x n[i], ldd = m)
 * to the device, runs cdmd_run_shared and copies each mask back to
 * mask_host[i], all on `stream`; then synchronises the stream and returns the
 * numerical status as cdmd_status_sync does. */
cdmd_status cdmd_run_host_shared(cdmd_ctx* ctx, int nclips, const uint8_t* const* D_host,
                                 int64_t m, const int* n, const cdmd_params* p,
                                 uint32_t* const* mask_host, void* stream);

/* Device pointers to the intermediates of the last cdmd_run on ctx (any
 * output pointer may be NULL).  Valid until the next call on the context. */
cdmd_status cdmd_workspace_views(cdmd_ctx* ctx, double** DY, double** sigma, double** lambda,
                                 double** G, double** beta, int32_t** sel, int32_t** nsel,
                                 float** Phi);

/* ---- batches of clips -------------------------------------------------------
 *
 * The paper processes long videos as independent 200-frame batches
 * (Section 4.1); a batch here is many clips of uneven resolution and length
 * run through one plan.  cdmd_batch_create validates the clips, allocates
 * every per-clip buffer and workspace once, picks the execution knobs (see
 * cdmd_batch_tuning) by timing candidates on the batch itself when asked,
 * and captures the whole batch into one CUDA graph; cdmd_batch_run replays
 * it.  Every clip gets the same results as a cdmd_run with the same
 * parameters up to the rounding order of the sketch's split sums.
 *
 * A clip: device video D (frame-major, n frames of m pixels, row stride
 * ldd), its sketch size k, rank r, K selected modes, measurement seed, and
 * the device mask it receives (n x ceil(m/32) words, as for cdmd_subtract).
 * The caller owns D and mask and keeps them alive, at fixed addresses, for
 * the life of the batch; the graph reads and writes them on every run. */
typedef struct {
    const uint8_t* D;
    int64_t m;
    int32_t n;
    int64_t ldd;
    int32_t k, r, K;
    uint64_t seed;
    uint32_t* mask;
} cdmd_clip;

/* flags */
#define CDMD_BATCH_GRAPH 1      /* capture the batch into a CUDA graph (else eager launches) */
#define CDMD_BATCH_AUTOTUNE 2   /* time candidate knobs on the batch and keep the fastest    */
#define CDMD_BATCH_GROUPED 4    /* the subtract pass of all clips, and with BF16X2 their sketch,
                                   as one grouped launch each (else per-clip launches); dropped
                                   silently for clips it does not cover (unaligned D or ldd,
                                   more than 12 modes)                                        */

typedef struct {
    cdmd_prec prec;
    cdmd_selector selector;
    cdmd_bgmode bgmode;
    float tau;
    int32_t lanes;                /* streams (each with its own workspace); 0 = default 8      */
    int32_t flags;
    const float* selector_blob;   /* device model blob for CDMD_SEL_MLP, else NULL             */
} cdmd_batch_params;

typedef struct cdmd_batch cdmd_batch;

/* Plan a batch of nclips clips on `device`; work done while planning (a warm-up
 * run, autotuning runs, the capture) is enqueued on `stream` and waited for.
 * Requirements per clip as for cdmd_run (Gaussian C); with BF16X2, D must be
 * 16-byte aligned with ldd % 16 == 0.  CDMD_ERR_INVALID_ARG names the first
 * offending clip. */
cdmd_status cdmd_batch_create(cdmd_batch** batch, int device, const cdmd_clip* clips, int nclips,
                              const cdmd_batch_params* params, void* stream);

/* Run the whole batch on `stream` (asynchronous; graph replay if captured). */
cdmd_status cdmd_batch_run(cdmd_batch* batch, void* stream);

/* Synchronise `stream`, then return and clear the first numerical status
 * recorded by any clip of the batch (CDMD_OK if none). */
cdmd_status cdmd_batch_status_sync(cdmd_batch* batch, void* stream);

/* Device pointers to clip `clip`'s results of the last run: DY (k x n),
 * lambda (2r), beta (2r), sel (K), Phi (m x ncols complex float); any output
 * pointer may be NULL. */
cdmd_status cdmd_batch_views(cdmd_batch* batch, int clip, double** DY, double** lambda, double** beta,
                             int32_t** sel, float** Phi);

/* The knobs the plan runs with: lanes (streams), the SM cap of each lane's
 * full-data passes (0 = none), the number of waves the grouped passes are
 * split into (0 without CDMD_BATCH_GROUPED; the small solves of one wave
 * overlap the grouped sketch of the next), the sketch work-item size
 * (64-pixel steps per CTA) and the subtract work-item size (pixel tiles per
 * CTA) of the grouped launches, and the measured time of one run in
 * milliseconds (0 if not autotuned).  Any output pointer may be NULL. */
cdmd_status cdmd_batch_tuning(cdmd_batch* batch, int32_t* lanes, int32_t* sm_limit, int32_t* waves,
                              int32_t* sketch_steps, int32_t* subtract_tiles, float* run_ms);

void cdmd_batch_destroy(cdmd_batch* batch);

/* Copy `bytes` between any two host or device addresses, ordered on
 * `stream` (a convenience for bindings reading the views above). */
cdmd_status cdmd_copy(void* dst, const void* src, size_t bytes, void* stream);

/* ---- learned mode selector ------------------------------------------------
 *
 * The paper selects background modes by sparse coding (Section 2.3,
 * Eq. sparsecoding; Remark 3 for the compressed modes).  These calls train
 * and apply a small network that predicts that selection from four per-mode
 * features (FP32, row-major r x 4):
 *   f0 = max(log|lambda_j|, -30), f1 = |arg lambda_j|,
 *   f2 = max(log(||phi_j|| / max_i ||phi_i||), -30),
 *   f3 = |phi_j^H y1| / (||phi_j|| ||y1||),
 * phi_j = column j of Phi_Y, y1 = DY[:,0] (Section 2.2 ties background modes
 * to |lambda| near 1 and arg lambda near 0).  The network is
 *   xh = (f - mu) / sd,  h = relu(W1 xh + b1) (64 units),  s = w2 . h + b2,
 *   p = 1 / (1 + exp(-s)),
 * trained with the mean binary cross-entropy against OMP labels and Adam.
 *
 * Model blob: CDMD_MLP_BLOB floats (device memory, caller-owned):
 *   [0..3] mu, [4..7] sd, [8] tol, [9..11] zero,
 *   then CDMD_MLP_PARAMS parameters: W1 (64 x 4 row-major), b1 (64), w2 (64),
 *   b2 (1).  Gradients and Adam moments use the parameter layout. */
#define CDMD_MLP_FEATURES 4
#define CDMD_MLP_HIDDEN 64
#define CDMD_MLP_PARAMS 385
#define CDMD_MLP_HEADER 12
#define CDMD_MLP_BLOB 397

/* Copy a model blob (device) into the context for CDMD_SEL_MLP and reset the
 * fallback count; the caller's blob may be freed after the copy completes on
 * `stream`.  Inference rounds the network's matrix operands (xh, W1, h, w2)
 * to bfloat16 and accumulates in FP32. */
cdmd_status cdmd_selector_load(cdmd_ctx* ctx, const float* blob, void* stream);

/* Features (r x 4) of the modes of the last cdmd_decompose on ctx, computed
 * from its Gram quantities (valid until the next cdmd_decompose or cdmd_run
 * on ctx); lambda is that call's lambda output.  If labels is not NULL,
 * labels[j] = 1 when mode j appears among sel[0..K-1] (the call's sel
 * output), else 0.  Device pointers; enqueued on `stream`.
 * CDMD_ERR_INVALID_ARG if no decomposition with this r was run on ctx. */
cdmd_status cdmd_selector_features(cdmd_ctx* ctx, const double* lambda, const int32_t* sel, int r, int K,
                                   float* feats, float* labels, void* stream);

/* OMP (Remark 3) on the compressed modes of the last cdmd_decompose on ctx
 * against another target y_target (k doubles, device) instead of y1, e.g. the
 * sketch of a clip's clean background frame when labelling training data:
 * sel[0..K-1] receives the picks (-1 after the last).  DY, G and lambda are
 * that call's input and outputs (k, n, r as there); 1 <= K <= r. */
cdmd_status cdmd_selector_relabel(cdmd_ctx* ctx, const double* DY, int k, int n, const double* G,
                                  const double* lambda, int r, const double* y_target, int K, int32_t* sel,
                                  void* stream);

/* Number of CDMD_SEL_MLP decompositions on ctx that fell back to OMP since
 * the last load or reset.  Synchronises `stream`; reset != 0 zeroes it. */
cdmd_status cdmd_selector_fallbacks(cdmd_ctx* ctx, int64_t* count, int reset, void* stream);

/* Batch inference: logits s[N] and probabilities p[N] (either may be NULL)
 * for N feature rows X (N x 4), with bf16 != 0 the BF16 operand rounding of
 * the in-decompose selection, else FP32 throughout. */
cdmd_status cdmd_mlp_forward(cdmd_ctx* ctx, const float* blob, const float* X, int64_t N, int bf16,
                             float* s, float* p, void* stream);

/* Mean loss and its gradient over N >= 1 rows (X: N x 4, Y: N labels in
 * {0, 1}) at the blob's parameters, FP32 arithmetic with FP64 reduction of
 * per-warp partial sums in a fixed order (deterministic).  grad:
 * CDMD_MLP_PARAMS floats; loss: 1 float; device pointers. */
cdmd_status cdmd_mlp_grad(cdmd_ctx* ctx, const float* blob, const float* X, const float* Y, int64_t N,
                          float* grad, float* loss, void* stream);

/* One Adam step (Kingma & Ba, Algorithm 1) on the blob's parameters from the
 * gradient over N rows: m and v (CDMD_MLP_PARAMS floats each, zero before
 * step 1) are updated in place; step >= 1 counts updates; loss (may be NULL)
 * receives the loss before the update. */
cdmd_status cdmd_mlp_train_step(cdmd_ctx* ctx, float* blob, float* m, float* v, int step, float lr, float beta1,
                                float beta2, float eps, const float* X, const float* Y, int64_t N, float* loss,
                                void* stream);

/* ---- synthetic clips (selector training data) ----------------------------
 *
 * Renders a seeded synthetic clip on the device, shaped like the paper's
 * surveillance workloads (Section 4: static textured scene, moving
 * foreground, illumination change, sensor noise).  For frame t and pixel
 * j = y * width + x (frame-major, D[t * ldd + j]):
 *   v  = 128 + sum_w amp_w sin((x cos th_w + y sin th_w) 2 pi / period_w + phase_w)
 *   v  = intensity_q for every object q (in order) whose frame-t rectangle
 *        (|x + 1/2 - cx| <= w/2 and |y + 1/2 - cy| <= h/2) or ellipse
 *        (ellipse != 0) contains the pixel centre
 *   v *= 1 + drift (2 t / (n - 1) - 1)                        (n > 1)
 *   v += noise_sigma z, z standard normal (Box-Muller on Philox4x32-10 words
 *        0, 1 of counter (j, t, 4, 0) under key = seed)
 *   D  = clamp(floor(v + 1/2), 0, 255)
 * waves: nw x 4 floats [amp, period, theta, phase]; objects: n x nobj x 5
 * floats [cx, cy, w, h, intensity] (state at frame t); device pointers.
 * Requires width, height, n >= 1 and ldd >= width * height. */
cdmd_status cdmd_synth_clip(cdmd_ctx* ctx, int width, int height, int n, const float* waves, int nw,
                            const float* objects, int nobj, int ellipse, float drift, float noise_sigma,
                            uint64_t seed, uint8_t* D, int64_t ldd, void* stream);

/* ---- allocation-free sketch ---------------------------------------------
 *
 * The paper has no counterpart to this call.  It serves callers that cannot
 * allocate device memory once they are running: pipelines whose memory
 * budget is fixed at start-up, real-time or certified code that forbids
 * allocation after initialisation, and hosts whose device allocator belongs
 * to another runtime.  cdmd_sketch keeps its split partial sums in a
 * context's workspace, which may grow; this variant keeps them in a fixed
 * 16 MiB array compiled into the library instead (every GPU that loads
 * libcdmd holds that array until the process exits) and allocates nothing.
 *
 * Same arguments and result as cdmd_sketch with prec = CDMD_PREC_FP32, minus
 * the context.  Runs on the calling thread's current device, enqueued on
 * `stream`.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Rejects k * n > 4,194,304 with CDMD_ERR_INVALID_ARG.  Every call shares the
 * one array and overwrites every partial sum it later reads, so nothing has
 * to be cleared between calls; calls whose kernels overlap on the GPU
 * (different streams without ordering between them) race on the array.
 * There is no context status word, so the non-finite check that cdmd_sketch
 * reports through cdmd_status_sync is not available here. */
cdmd_status cdmd_sketch_noalloc(const uint8_t* D, int64_t m, int n, int64_t ldd, cdmd_ctype ctype, int k,
                                uint64_t seed, double* DY, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDMD_H */
