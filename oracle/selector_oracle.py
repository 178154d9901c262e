"""CPU oracle of the learned sketch-precision selector -- TEST INFRASTRUCTURE.

The paper leaves choosing the sketch precision to the caller: a coarse
regime of kappa_2(A) decides half (< 1e4), single (< 1e8) or double
(Sec. II-C).  It suggests a CholQR probe or a 1-norm estimator, and names
machine-learned condition estimators as a further option.  The selector is
that option: 16 cheap features of the R_s that an FP16 sketch produces, an
MLP 16-64-64-3 (ReLU) trained with class-weighted cross-entropy, and a
choice that minimises the expected cost of the precision ladder (a too-low
precision costs its run plus every rerun up to the right one).

Plain FP64 numpy, written from these definitions; shares nothing with the
CUDA kernels.
"""
from __future__ import annotations

import math

import numpy as np

NUM_FEATURES = 16
HIDDEN = 64
CLASSES = 3            # 0: fp16, 1: fp32, 2: fp64
SHAPES = [(HIDDEN, NUM_FEATURES), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (CLASSES, HIDDEN), (CLASSES,)]
NUM_PARAMS = sum(int(np.prod(s)) for s in SHAPES)
POWER_STEPS = 3


def _power_norm(apply, applyT, n):
    """3-step power iteration for ||M||_2 with x0 = ones / sqrt(n): each step
    x <- M^T M x, normalised; returns sqrt of the last norm."""
    x = np.full(n, 1.0 / math.sqrt(n))
    nrm = 0.0
    for _ in range(POWER_STEPS):
        x = applyT(apply(x))
        nrm = float(np.linalg.norm(x))
        if nrm == 0.0 or not np.isfinite(nrm):
            return nrm
        x = x / nrm
    return math.sqrt(nrm)


def _solve_upper(R, b):
    n = len(b)
    x = b.copy()
    for j in range(n - 1, -1, -1):
        x[j] /= R[j, j]
        x[:j] -= R[:j, j] * x[j]
    return x


def _solve_upper_T(R, b):
    # R^T x = b, R^T lower triangular: forward substitution
    n = len(b)
    x = b.copy()
    for j in range(n):
        x[j] /= R[j, j]
        x[j + 1:] -= R[j, j + 1:] * x[j]
    return x


def _cond_est(R):
    n = R.shape[0]
    nr = _power_norm(lambda x: R @ x, lambda y: R.T @ y, n)
    ni = _power_norm(lambda x: _solve_upper(R, x), lambda y: _solve_upper_T(R, y), n)
    return nr * ni


def features(R: np.ndarray, m: int) -> np.ndarray:
    """The 16 selector features of an upper-triangular R with positive
    diagonal (n x n), for a problem with m rows."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    d = np.abs(np.diag(R))
    tiny = np.finfo(np.float64).tiny
    L = np.log10(np.maximum(d, tiny))
    Lmax, Lmin = L.max(), L.min()
    Ls = np.sort(L)
    q = lambda p: Ls[int(math.floor(p * (n - 1)))]
    f = np.zeros(NUM_FEATURES)
    f[0] = Lmax - Lmin
    f[1] = Lmax - q(0.10)
    f[2] = Lmax - q(0.50)
    f[3] = float(np.mean(Lmax - L))
    f[4] = float(np.sqrt(np.mean((L - L.mean()) ** 2)))
    f[5] = math.log10(max(_cond_est(R), 1.0))
    f[6] = math.log10(max(_cond_est(R / np.maximum(d, tiny)[None, :]), 1.0))
    cn = np.linalg.norm(R, axis=0)
    f[7] = math.log10(max(cn.max(), tiny) / max(cn.min(), tiny))
    f[8] = float(np.linalg.norm(np.triu(R, 1)) / max(np.linalg.norm(d), tiny))
    f[9] = n / 512.0
    f[10] = math.log2(m) / 22.0
    dmax = d.max()
    f[11] = float(np.mean(d < 2.0 ** -11 * dmax))
    f[12] = float(np.mean(d < 2.0 ** -20 * dmax))
    h = max(n // 2, 2)
    i = np.arange(h, dtype=np.float64)
    slope = float(np.sum((i - i.mean()) * (L[:h] - L[:h].mean())) / np.sum((i - i.mean()) ** 2))
    f[13] = -slope * (n - 1)
    f[14] = Lmax - L[-1]
    f[15] = 1.0
    return f


# --- MLP 16-64-64-3 --------------------------------------------------------------

def unpack(theta: np.ndarray):
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (8 significand bits), round-to-nearest-even, from FP32."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def normalize(X, mu, sd):
    return (np.asarray(X, np.float64) - mu) / sd


def forward(theta, Xn):
    """Logits and the activations backprop needs (FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    a1 = Xn @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3.T + b3
    return z, (a1, h1, a2, h2)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grad(theta, Xn, y, class_w):
    """Class-weighted mean cross-entropy and its gradient (FP64)."""
    B = Xn.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z, (a1, h1, a2, h2) = forward(theta, Xn)
    p = softmax(z)
    w = class_w[y]
    loss = float(np.sum(w * -np.log(p[np.arange(B), y])) / B)
    dz = p.copy()
    dz[np.arange(B), y] -= 1.0
    dz *= (w / B)[:, None]
    gW3 = dz.T @ h2
    gb3 = dz.sum(0)
    dh2 = (dz @ W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ Xn
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adamw_step(theta, g, m, v, step, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW update (decoupled weight decay), bias-corrected."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v


def cost_matrix(costs):
    """C[k][y]: cost of starting the ladder at k when y is the cheapest
    precision that passes: cost(k) if k >= y, else every run from k to y."""
    c = np.asarray(costs, dtype=np.float64)
    C = np.zeros((CLASSES, CLASSES))
    for k in range(CLASSES):
        for t in range(CLASSES):
            C[k, t] = c[k] if k >= t else c[k:t + 1].sum()
    return C


def choose(theta, Xn, costs):
    """argmin_k sum_y p(y | x) C[k][y]."""
    z, _ = forward(theta, Xn)
    p = softmax(z)
    return np.argmin(p @ cost_matrix(costs).T, axis=1)
