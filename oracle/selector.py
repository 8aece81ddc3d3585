"""Learned background-mode selector, plain FP64 CPU oracle.

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU legs of the
benchmark may import it; the product never does.

The paper picks the background modes and their amplitudes by sparse coding
(Section 2.3, Eq. sparsecoding; Remark 3 applies it to the compressed modes).
This module defines a small learned replacement for the selection step and
keeps the sparse-coding solver as its fallback and as the reference its
selections are checked against:

  features   per mode j of the decomposition (the continuous-time reading of
             Section 2.2 ties background modes to |lambda| near 1 and arg
             lambda near 0):
               f0 = log |lambda_j|                                 (floored at -30)
               f1 = |arg lambda_j|          (conjugate pairs share their features)
               f2 = log(||phi_j|| / max_i ||phi_i||)               (floored at -30)
               f3 = |phi_j^H y1| / (||phi_j|| ||y1||)     (first OMP correlation)
             with phi_j the compressed mode (column j of Phi_Y) and y1 the
             first sketched frame.
  network    xh = (x - mu) / sd;  h = relu(W1 xh + b1) (64 units);
             s = w2 . h + b2;  p = sigmoid(s).
  loss       mean binary cross-entropy of p against the OMP label of the mode,
             written as softplus(s) - y s.
  optimiser  Adam (Kingma & Ba, ICLR 2015, Algorithm 1).
  selection  the K modes of largest logit s (equivalently p; equal s: lower
             index first; ranking by s avoids the ties a saturated sigmoid
             would create); amplitudes
             by least squares on the selected compressed modes (Eq. b in the
             compressed form of Remark 3); if the relative residual
             ||y1 - Phi_Y,S beta|| / ||y1|| exceeds tol the OMP result is used.

Parameter vector layout (shared with the device kernels' C ABI):
  W1 (64 x 4, row-major: W1[u][i]), b1 (64), w2 (64), b2 (1)  -> 385 values.
Model blob: mu (4), sd (4), tol, 3 zeros, then the 385 parameters.
"""
import numpy as np

from oracle import cdmd as O

N_FEAT = 4
HIDDEN = 64
N_PARAM = HIDDEN * N_FEAT + HIDDEN + HIDDEN + 1
HEADER = 12
FLOOR = -30.0


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------


def features(lam, PhiY, y1):
    """Per-mode features (r x 4, FP64) from the eigenvalues, compressed modes
    and first sketched frame."""
    lam = np.asarray(lam, dtype=np.complex128)
    PhiY = np.asarray(PhiY, dtype=np.complex128)
    y1 = np.asarray(y1, dtype=np.complex128)
    r = lam.shape[0]
    norms = np.linalg.norm(PhiY, axis=0)
    ynorm = np.linalg.norm(y1)
    nmax = norms.max() if r else 0.0
    X = np.zeros((r, N_FEAT))
    with np.errstate(divide="ignore"):
        X[:, 0] = np.maximum(np.log(np.abs(lam)), FLOOR)
        X[:, 1] = np.abs(np.angle(lam))
        X[:, 2] = np.where(norms > 0, np.maximum(np.log(norms / nmax), FLOOR), FLOOR) if nmax > 0 else FLOOR
    corr = np.abs(PhiY.conj().T @ y1)
    den = norms * ynorm
    X[:, 3] = np.where(den > 0, corr / np.where(den > 0, den, 1.0), 0.0)
    return X


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + HIDDEN * N_FEAT].reshape(HIDDEN, N_FEAT)
    o += HIDDEN * N_FEAT
    b1 = theta[o:o + HIDDEN]
    o += HIDDEN
    w2 = theta[o:o + HIDDEN]
    o += HIDDEN
    b2 = theta[o]
    return W1, b1, w2, b2


def pack(W1, b1, w2, b2):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(w2), [b2]]).astype(np.float64)


def init_params(seed):
    """He-uniform first layer, small second layer (any start works for the tests)."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1.0, 1.0, (HIDDEN, N_FEAT)) * np.sqrt(6.0 / N_FEAT)
    b1 = np.zeros(HIDDEN)
    w2 = rng.uniform(-1.0, 1.0, HIDDEN) * np.sqrt(6.0 / HIDDEN) * 0.1
    return pack(W1, b1, w2, 0.0)


def bf16_round(x):
    """Round FP64 values to the nearest bfloat16 (ties to even), as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, mu, sd, bf16=False):
    """Logits s and probabilities p of the selector for feature rows X (N x 4).

    bf16=True rounds every matrix operand (normalised features, W1, hidden
    activations, w2) to bfloat16 and keeps biases and sums exact, the
    inference precision of the device kernels (FP32 accumulation).
    """
    W1, b1, w2, b2 = unpack(theta)
    Xh = (np.asarray(X, dtype=np.float64) - mu) / sd
    if bf16:
        Xh = bf16_round(Xh)
        W1 = bf16_round(W1)
        w2 = bf16_round(w2)
    hpre = Xh @ W1.T + b1
    h = np.maximum(hpre, 0.0)
    if bf16:
        h = bf16_round(h)
    s = h @ w2 + b2
    return s, 1.0 / (1.0 + np.exp(-s))


def loss_and_grad(theta, X, Y, mu, sd):
    """Mean BCE loss over the rows and its exact gradient (FP64).

    L = (1/N) sum_i softplus(s_i) - y_i s_i;  dL/ds_i = (sigmoid(s_i) - y_i)/N,
    back-propagated through the output layer and the ReLU layer.
    """
    W1, b1, w2, b2 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    N = X.shape[0]
    Xh = (X - mu) / sd
    hpre = Xh @ W1.T + b1
    h = np.maximum(hpre, 0.0)
    s = h @ w2 + b2
    loss = np.mean(np.maximum(s, 0.0) + np.log1p(np.exp(-np.abs(s))) - Y * s)
    ds = (1.0 / (1.0 + np.exp(-s)) - Y) / N
    g_w2 = h.T @ ds
    g_b2 = ds.sum()
    dh = np.outer(ds, w2) * (hpre > 0.0)
    g_W1 = dh.T @ Xh
    g_b1 = dh.sum(axis=0)
    return loss, pack(g_W1, g_b1, g_w2, g_b2)


def adam_step(theta, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1); step counts from 1.

    Returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ----------------------------------------------------------------------------
# selection with OMP fallback
# ----------------------------------------------------------------------------


def rank_modes(s):
    """Mode indices by descending logit; equal values keep index order."""
    s = np.asarray(s)
    return np.array(sorted(range(len(s)), key=lambda j: (-s[j], j)), dtype=np.int64)


def select(theta, mu, sd, tol, lam, PhiY, y1, K, bf16=True):
    """Learned selection of K background modes and their amplitudes.

    Returns dict(sel, beta, fallback, residual, s, p): sel in pick order, beta the
    least-squares amplitudes on sel; fallback=True when the learned set's
    relative residual exceeded tol and OMP's (sel, beta) were returned.
    """
    PhiY = np.asarray(PhiY, dtype=np.complex128)
    y1 = np.asarray(y1, dtype=np.complex128)
    X = features(lam, PhiY, y1)
    s, p = forward(theta, X, mu, sd, bf16=bf16)
    r = PhiY.shape[1]
    sel = rank_modes(s)[:min(K, r)]
    beta = np.linalg.lstsq(PhiY[:, sel], y1, rcond=None)[0]
    res = np.linalg.norm(y1 - PhiY[:, sel] @ beta) / np.linalg.norm(y1)
    if res > tol:
        osel, obeta = O.omp(PhiY, y1, K, lam)
        return dict(sel=osel, beta=obeta, fallback=True, residual=res, s=s, p=p)
    return dict(sel=sel, beta=beta, fallback=False, residual=res, s=s, p=p)


def labels(r, sel):
    """OMP labels: 1 for each selected mode, 0 otherwise."""
    y = np.zeros(r)
    y[np.asarray(sel, dtype=np.int64)] = 1.0
    return y


def blob(theta, mu, sd, tol):
    """Model blob in the device layout (FP32)."""
    head = np.zeros(HEADER)
    head[0:4] = mu
    head[4:8] = sd
    head[8] = tol
    return np.concatenate([head, np.asarray(theta, dtype=np.float64)]).astype(np.float32)


def from_blob(b):
    b = np.asarray(b, dtype=np.float64)
    return b[HEADER:], b[0:4], b[4:8], float(b[8])
