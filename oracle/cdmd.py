"""Compressed DMD for background modelling, plain FP64 CPU oracle.

TEST INFRASTRUCTURE.  This is the slow, obviously-correct reference that the
CUDA path is checked against.  Only tests, the smoke check and the CPU
baseline leg of the benchmark may import it; the product never does.

It follows Algorithm 1 of Erichson, Brunton & Kutz (arXiv 1512.04205) in the
paper's order, with the letters used throughout this repository:
m pixels per frame, n frames, k sketch rows, r target rank, K non-zero
amplitudes.  The video D is m x n (column t = frame t).

  step (1)  X = D[:, 0:n-1], X' = D[:, 1:n]                     Eq. (FullData)
  step (2)  C (k x m)                                 Section 3.3, measurement.py
  step (3)  Y = C X, Y' = C X'  (one product C D, then column slices)  Eq. (YCX)
  step (4)  truncated SVD  Y = U S V^T  at rank r                     Eq. (svd)
  step (6)  A~ = U^T Y' V S^-1                          Section 3.2, projected map
  step (7)  A~ W = W Lambda                                     eigen-decomposition
  Phi_Y = Y' V S^-1 W                              compressed modes, Section 3.2
  step (8)  Phi = X' V S^-1 W                                   Eq. (cDMDModes)
  step (9)  amplitudes: lstsq (Eq. b) or OMP on the compressed modes (Remark 3,
            Eq. sparsecoding) with y1 = Y[:, 0]
  background  bg_jt = | sum_{s in sel} Phi_js beta_s lambda_s^t |        Eq. (DMDTerms)
  mask        M_jt = 1  iff  |x_jt - bg_jt| > tau                       Eq. (thres)
  F-measure   harmonic mean of precision and recall            Section 4 (Results)
  post-pass   3 x 3 median filter of each mask frame, zero padding    Section 4 (BMC figure, Discussion)
  rank        optional: r from the optimal hard threshold on the singular values
              of Y (Remark 2)
  exact DMD   the same steps on X itself (no C; Section 2.1), the comparator of
              Section 4 (Computational Performance)

Readings where the paper is silent (all FP64):
* SVD: one-sided (Hestenes) Jacobi on Y, cyclic pair order, until every pair
  is orthogonal to 1e-15 relative; singular values sorted descending.
* eig: Householder reduction to Hessenberg form, complex single-shift QR with
  Wilkinson shifts to a complex Schur form, eigenvectors by back-substitution.
  Each eigenvector column has unit 2-norm and its largest-modulus entry real
  and positive.  Eigenvalues are ordered by descending modulus, then by
  descending imaginary part.
* OMP: correlation |phi_j^H rho| / ||phi_j||; candidates within 1e-9 relative of
  the best score are ties and go to the largest Im(lambda), then lowest index;
  beta is re-solved by complex least squares on the selected columns after each
  pick; stop at K picks or when ||rho|| <= 1e-12 ||y1||.
* Background modes: MODULUS (the default: modulus of the complex sum), REAL (footnote to Eq. DMDTerms),
  STATIC (x_BG = Phi beta of Section 2.3, i.e. t = 0 for every frame).
* Median filter: the paper gives neither the window nor the border rule;
  the window is 3 x 3 and pixels outside the frame count as background.
"""
import numpy as np

# ----------------------------------------------------------------------------
# Steps (1) and (3)
# ----------------------------------------------------------------------------


def split_snapshots(D):
    """Left and right snapshot sequences X, X' (Eq. FullData)."""
    D = np.asarray(D, dtype=np.float64)
    return D[:, :-1], D[:, 1:]


def sketch(C, D):
    """Compressed data D_Y = C D (Eq. YCX, Algorithm 1 step 3)."""
    return np.asarray(C, dtype=np.float64) @ np.asarray(D, dtype=np.float64)


# ----------------------------------------------------------------------------
# Step (4): truncated SVD by one-sided Jacobi
# ----------------------------------------------------------------------------


def jacobi_svd(Y, tol=1e-15, max_sweeps=80):
    """Thin SVD Y = U diag(s) V^T by one-sided Jacobi rotations.

    Columns of a working copy of Y are rotated pairwise until they are mutually
    orthogonal; the rotations accumulate into V.  Returns (U, s, V, sweeps)
    with s descending; columns of U for zero singular values are zero.
    """
    A = np.array(Y, dtype=np.float64, copy=True)
    p = A.shape[1]
    V = np.eye(p)
    sweeps = 0
    # columns whose squared norm is below (eps ||Y||_F)^2 are numerically zero
    # (rank < p); rotating them against each other would never terminate
    negligible = (np.finfo(np.float64).eps * np.linalg.norm(A)) ** 2
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for a in range(p - 1):
            for b in range(a + 1, p):
                alpha = A[:, a] @ A[:, a]
                beta = A[:, b] @ A[:, b]
                gamma = A[:, a] @ A[:, b]
                if alpha <= negligible or beta <= negligible:
                    continue
                if gamma == 0.0 or abs(gamma) <= tol * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                if abs(zeta) > 1e150:
                    t = 0.5 / zeta
                else:
                    t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                col_a = A[:, a].copy()
                A[:, a] = c * col_a - s * A[:, b]
                A[:, b] = s * col_a + c * A[:, b]
                v_a = V[:, a].copy()
                V[:, a] = c * v_a - s * V[:, b]
                V[:, b] = s * v_a + c * V[:, b]
        if not rotated:
            break
    else:
        raise RuntimeError("Jacobi SVD did not converge")
    sig = np.sqrt(np.einsum("ij,ij->j", A, A))
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    A = A[:, order]
    V = V[:, order]
    U = np.zeros_like(A)
    nz = sig > 0
    U[:, nz] = A[:, nz] / sig[nz]
    return U, sig, V, sweeps


def truncated_svd(Y, r):
    """Rank-r truncation of the Jacobi SVD (Algorithm 1 step 4)."""
    U, s, V, _ = jacobi_svd(Y)
    if s[r - 1] <= 0.0:
        raise ValueError("rank-deficient sketch: sigma_r == 0")
    return U[:, :r], s[:r], V[:, :r]


# ----------------------------------------------------------------------------
# Step (7): eigen-decomposition of the real nonsymmetric A~
# ----------------------------------------------------------------------------


def hessenberg(A):
    """Householder reduction A = Q H Q^T with H upper Hessenberg."""
    H = np.array(A, dtype=np.float64, copy=True)
    n = H.shape[0]
    Q = np.eye(n)
    for j in range(n - 2):
        x = H[j + 1:, j].copy()
        normx = np.linalg.norm(x)
        if normx == 0.0:
            continue
        v = x.copy()
        v[0] += (1.0 if x[0] >= 0 else -1.0) * normx
        v /= np.linalg.norm(v)
        # P = I - 2 v v^T acting on rows/cols j+1..n-1
        H[j + 1:, :] -= 2.0 * np.outer(v, v @ H[j + 1:, :])
        H[:, j + 1:] -= 2.0 * np.outer(H[:, j + 1:] @ v, v)
        Q[:, j + 1:] -= 2.0 * np.outer(Q[:, j + 1:] @ v, v)
        H[j + 2:, j] = 0.0
    return H, Q


def _givens(x, y):
    """Unitary G = [[conj(c), conj(s)], [-s, c]] with G [x, y]^T = [r, 0]^T."""
    r = np.sqrt(abs(x) ** 2 + abs(y) ** 2)
    if r == 0.0:
        return 1.0 + 0j, 0j
    return x / r, y / r


def complex_schur(H, max_iter_per_eig=60):
    """Complex Schur form H = Z T Z^H of an upper Hessenberg matrix.

    Single-shift QR steps (bulge chasing with Givens rotations) on the active
    window, Wilkinson shift from its trailing 2x2 block, deflation when a
    sub-diagonal entry is below machine precision relative to its neighbours.
    """
    T = np.array(H, dtype=np.complex128, copy=True)
    n = T.shape[0]
    Z = np.eye(n, dtype=np.complex128)
    eps = np.finfo(np.float64).eps
    hi = n - 1
    its = 0
    while hi > 0:
        lo = hi
        while lo > 0:
            if abs(T[lo, lo - 1]) <= eps * (abs(T[lo - 1, lo - 1]) + abs(T[lo, lo])):
                T[lo, lo - 1] = 0.0
                break
            lo -= 1
        if lo == hi:
            hi -= 1
            its = 0
            continue
        its += 1
        if its > max_iter_per_eig:
            raise RuntimeError("complex Schur iteration did not converge")
        a, b = T[hi - 1, hi - 1], T[hi - 1, hi]
        c, d = T[hi, hi - 1], T[hi, hi]
        if its % 11 == 0:
            mu = d + abs(c)          # exceptional shift breaks cycles
        else:
            half = 0.5 * (a - d)
            disc = np.sqrt(half * half + b * c)
            mu1 = d - b * c / (half + disc) if (half + disc) != 0 else d
            mu2 = d - b * c / (half - disc) if (half - disc) != 0 else d
            mu = mu1 if abs(mu1 - d) <= abs(mu2 - d) else mu2
        x = T[lo, lo] - mu
        y = T[lo + 1, lo]
        for q in range(lo, hi):
            if q > lo:
                x = T[q, q - 1]
                y = T[q + 1, q - 1]
            cg, sg = _givens(x, y)
            G = np.array([[np.conj(cg), np.conj(sg)], [-sg, cg]])
            col0 = max(q - 1, 0)
            T[q:q + 2, col0:] = G @ T[q:q + 2, col0:]
            row1 = min(q + 3, hi + 1)
            T[:row1, q:q + 2] = T[:row1, q:q + 2] @ G.conj().T
            Z[:, q:q + 2] = Z[:, q:q + 2] @ G.conj().T
            if q > lo:
                T[q + 1, q - 1] = 0.0
    return T, Z


def triangular_eigenvectors(T):
    """Eigenvectors of an upper-triangular T by back-substitution."""
    n = T.shape[0]
    X = np.zeros((n, n), dtype=np.complex128)
    small = np.finfo(np.float64).eps * max(np.abs(T).max(), np.finfo(np.float64).tiny)
    for j in range(n):
        X[j, j] = 1.0
        for i in range(j - 1, -1, -1):
            denom = T[i, i] - T[j, j]
            if abs(denom) < small:
                denom = small
            X[i, j] = -(T[i, i + 1:j + 1] @ X[i + 1:j + 1, j]) / denom
    return X


def normalize_modes(W):
    """Unit 2-norm columns whose largest-modulus entry is real positive."""
    W = np.array(W, dtype=np.complex128, copy=True)
    for j in range(W.shape[1]):
        nrm = np.linalg.norm(W[:, j])
        if nrm == 0.0:
            continue
        W[:, j] /= nrm
        p = int(np.argmax(np.abs(W[:, j])))
        W[:, j] *= np.conj(W[p, j]) / abs(W[p, j])
    return W


def order_eigen(lam, pair_rel=1e-9):
    """Index order of the eigenvalues.

    An eigenvalue with positive imaginary part is paired with the closest
    unpaired eigenvalue within pair_rel * max(1, |lambda|) of its conjugate.
    Pairs and single eigenvalues are sorted by descending modulus, then by
    descending imaginary part, of their positive-imaginary member; a pair
    lists its positive-imaginary member first.  (The two members of a pair
    differ in modulus only by rounding, so a plain sort could split them.)
    """
    lam = np.asarray(lam, dtype=np.complex128)
    used = np.zeros(len(lam), dtype=bool)
    units = []
    for i in np.argsort(-lam.imag, kind="stable"):
        if used[i]:
            continue
        used[i] = True
        members = [int(i)]
        if lam[i].imag > 0:
            dist = np.abs(lam - np.conj(lam[i]))
            dist[used] = np.inf
            j = int(np.argmin(dist))
            if dist[j] <= pair_rel * max(1.0, abs(lam[i])):
                used[j] = True
                members.append(j)
        units.append((-abs(lam[i]), -lam[i].imag, members))
    units.sort(key=lambda u: (u[0], u[1]))
    return np.array([q for u in units for q in u[2]], dtype=np.int64)


def eig_nonsymmetric(A):
    """Eigenvalues and eigenvectors of a real square matrix (step 7)."""
    H, Q = hessenberg(A)
    T, Z = complex_schur(H)
    lam = np.diag(T).copy()
    W = Q @ Z @ triangular_eigenvectors(T)
    W = normalize_modes(W)
    order = order_eigen(lam)
    return lam[order], W[:, order]


# ----------------------------------------------------------------------------
# Step (9): amplitudes and sparse mode selection
# ----------------------------------------------------------------------------


def omp(PhiY, y1, K, lam, tie_rel=1e-9, stop_rel=1e-12):
    """Orthogonal matching pursuit on the compressed modes (Remark 3).

    Returns (sel, beta_sel): the selected mode indices in pick order and their
    complex amplitudes from the least-squares fit on the selected columns.
    """
    PhiY = np.asarray(PhiY, dtype=np.complex128)
    y1 = np.asarray(y1, dtype=np.complex128)
    r = PhiY.shape[1]
    norms = np.linalg.norm(PhiY, axis=0)
    sel = []
    beta = np.zeros(0, dtype=np.complex128)
    rho = y1.copy()
    y_norm = np.linalg.norm(y1)
    for _ in range(min(K, r)):
        if np.linalg.norm(rho) <= stop_rel * y_norm:
            break
        corr = np.abs(PhiY.conj().T @ rho)
        score = np.where(norms > 0, corr / np.where(norms > 0, norms, 1.0), -1.0)
        score[sel] = -np.inf
        best = score.max()
        if best <= 0:
            break
        ties = [j for j in range(r) if score[j] >= best * (1.0 - tie_rel)]
        j = sorted(ties, key=lambda q: (-lam[q].imag, q))[0]
        sel.append(j)
        beta = np.linalg.lstsq(PhiY[:, sel], y1, rcond=None)[0]
        rho = y1 - PhiY[:, sel] @ beta
    return np.array(sel, dtype=np.int64), beta


def lstsq_amplitudes(Phi, x1):
    """All-mode amplitudes b = argmin ||x1 - Phi b|| (Eq. b, step 9)."""
    return np.linalg.lstsq(np.asarray(Phi, dtype=np.complex128),
                           np.asarray(x1, dtype=np.complex128), rcond=None)[0]


# ----------------------------------------------------------------------------
# Whole decomposition (Algorithm 1 with Remark 3)
# ----------------------------------------------------------------------------


def decompose(DY, r, K):
    """Steps (4)-(7), compressed modes and OMP from the sketch D_Y (k x n)."""
    DY = np.asarray(DY, dtype=np.float64)
    Y, Yp = DY[:, :-1], DY[:, 1:]
    U, s, V = truncated_svd(Y, r)
    Atil = (U.T @ Yp @ V) / s[None, :]
    lam, W = eig_nonsymmetric(Atil)
    G = (V / s[None, :]) @ W                  # V S^-1 W, (n-1) x r
    PhiY = Yp @ G
    sel, beta = omp(PhiY, DY[:, 0], K, lam)
    return dict(U=U, sigma=s, V=V, Atilde=Atil, lam=lam, W=W, G=G, PhiY=PhiY,
                sel=sel, beta=beta)


def gd_omega(beta):
    """Coefficient of the optimal hard threshold for singular values when the
    noise level is unknown (Gavish and Donoho, the work cited in Remark 2): the
    cubic approximation they publish, within about 0.02 of the exact value."""
    return 0.56 * beta ** 3 - 0.95 * beta ** 2 + 1.82 * beta + 1.43


def gd_rank(s, shape, r_max):
    """Target rank by the optimal hard threshold (Remark 2, Section 4's
    evaluation settings): with beta = min(shape) / max(shape) and y_med the
    median of the min(shape) singular values s of the matrix, keep the
    singular values above tau = gd_omega(beta) * y_med.  Returns (r, tau) with
    r clamped to [1, r_max]."""
    q = min(shape)
    s = np.sort(np.asarray(s, dtype=np.float64))[::-1][:q]
    beta = q / max(shape)
    tau = gd_omega(beta) * float(np.median(s))
    r = int(np.sum(s > tau))
    return max(1, min(r, r_max)), tau


def decompose_auto(DY, r_max, K):
    """Steps (4)-(9) with the target rank chosen by gd_rank on the singular
    values of Y = DY[:, 0:n-1] (Remark 2: the threshold combined with step 4);
    K is capped at that rank."""
    DY = np.asarray(DY, dtype=np.float64)
    Y = DY[:, :-1]
    _, sv, _, _ = jacobi_svd(Y)
    r, tau = gd_rank(sv, Y.shape, r_max)
    out = decompose(DY, r, min(K, r))
    out["rank"] = r
    out["rank_tau"] = tau
    return out


def lift(D, G):
    """Full-state modes Phi = X' V S^-1 W = X' G (Eq. cDMDModes, step 8)."""
    _, Xp = split_snapshots(D)
    return Xp @ G


def cdmd(D, C, r, K):
    """Algorithm 1 (+ Remark 3) on a video D (m x n) with measurement C."""
    DY = sketch(C, D)
    out = decompose(DY, r, K)
    out["DY"] = DY
    out["Phi"] = lift(D, out["G"])
    return out


def exact_dmd(D, r, K):
    """Exact DMD (Section 2.1) with the sparse-coding selection of Section 2.3.

    Steps (4)-(9) run on the snapshots themselves, with no measurement: the
    SVD is that of X, A~ = U^T X' V S^-1, the modes Phi = X' V S^-1 W are the
    full-resolution ones, and OMP works on them with x1 = D[:, 0].  Same
    keys as cdmd(); "Phi" is the (m x r) mode matrix.
    """
    out = decompose(D, r, K)
    out["Phi"] = out["PhiY"]
    return out


def snapshot_gram(D):
    """R = D^T D (n x n), the inner products of every pair of frames, in exact
    integer arithmetic for a uint8 video (sums of m products < 2^63)."""
    D = np.asarray(D)
    if np.issubdtype(D.dtype, np.integer):
        Di = D.astype(np.int64)
        return Di.T @ Di
    D = D.astype(np.float64)
    return D.T @ D


# ----------------------------------------------------------------------------
# Background, foreground mask, F-measure
# ----------------------------------------------------------------------------

BG_MODULUS, BG_REAL, BG_STATIC = "modulus", "real", "static"


def background(Phi_sel, beta_sel, lam_sel, n, mode=BG_MODULUS):
    """Background video from the selected modes (Eq. DMDTerms, Section 2.3)."""
    Phi_sel = np.asarray(Phi_sel, dtype=np.complex128)
    amp = Phi_sel * np.asarray(beta_sel, dtype=np.complex128)[None, :]
    if mode == BG_STATIC:
        z = amp.sum(axis=1)
        return np.repeat(np.abs(z)[:, None], n, axis=1)
    vander = np.asarray(lam_sel, dtype=np.complex128)[:, None] ** np.arange(n)[None, :]
    z = amp @ vander
    if mode == BG_MODULUS:
        return np.abs(z)
    if mode == BG_REAL:
        return z.real
    raise ValueError(mode)


def foreground_mask(D, bg, tau):
    """M_jt = 1 iff |x_jt - bg_jt| > tau (Eq. thres, strict)."""
    return np.abs(np.asarray(D, dtype=np.float64) - bg) > tau


def pack_mask(mask):
    """Bit-pack an m x n boolean mask frame by frame.

    Frame t occupies ceil(m/32) uint32 words; pixel j is bit j%32 (LSB first)
    of word j//32.  Returns an (n, ceil(m/32)) uint32 array.
    """
    mask = np.asarray(mask, dtype=bool)
    m, n = mask.shape
    words = (m + 31) // 32
    out = np.zeros((n, words), dtype=np.uint32)
    for j in range(m):
        out[:, j // 32] |= mask[j, :].astype(np.uint32) << np.uint32(j % 32)
    return out


def fmeasure(pred, truth):
    """(precision, recall, F) of a predicted foreground mask (Section 4)."""
    pred = np.asarray(pred, dtype=bool)
    truth = np.asarray(truth, dtype=bool)
    tp = int(np.sum(pred & truth))
    fp = int(np.sum(pred & ~truth))
    fn = int(np.sum(~pred & truth))
    precision = tp / (tp + fp) if tp + fp > 0 else 0.0
    recall = tp / (tp + fn) if tp + fn > 0 else 0.0
    f = 2 * precision * recall / (precision + recall) if precision + recall > 0 else 0.0
    return precision, recall, f


# ----------------------------------------------------------------------------
# Mask post-processing (Section 4: the BMC figure's median-filtered masks and
# the Discussion's remark that a median filter cuts false positives)
# ----------------------------------------------------------------------------

def median3x3_mask(mask, W, H):
    """3 x 3 median filter of each frame of an m x n boolean mask.

    Pixel j of a frame sits at row j // W, column j % W (m = W * H).  The
    window is the pixel and its eight neighbours; neighbours outside the frame
    count as background (zero padding).  Written as the definition: stack the
    nine shifted frames and take their median, which for 0/1 values is the
    fifth-smallest of the nine.
    """
    mask = np.asarray(mask, dtype=bool)
    m, n = mask.shape
    if m != W * H:
        raise ValueError("m != W * H")
    frames = mask.T.reshape(n, H, W).astype(np.uint8)
    padded = np.zeros((n, H + 2, W + 2), dtype=np.uint8)
    padded[:, 1:H + 1, 1:W + 1] = frames
    window = np.stack([padded[:, 1 + dy:H + 1 + dy, 1 + dx:W + 1 + dx]
                       for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)
    med = np.median(window, axis=0)
    return (med > 0.5).reshape(n, m).T
