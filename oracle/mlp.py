"""FP64 reference of the learned Metropolis proposal for the hidden variables.

ORACLE / TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper allows any proposal for the paths' Metropolis update as long as the
acceptance keeps the sampled trial exact (Sec. III A, the discussion after Eq.
(23)).  This proposal is conditioned on walker features f (length K) and is a
diagonal Gaussian q(x | f) = N(mu(f), diag exp(logv(f))) with

    mu(f)   = f + out[:K],      logv(f) = clip(out[K:], LOGV_MIN, LOGV_MAX),
    out     = W3 tanh(W2 tanh(W1 f + b1) + b2) + b3,

two hidden layers of width H.  The features are the gradient at x = 0 of
log|<Phi(x)|phi>| (Phi(x) = exp(sum_k x_k U_k) Phi0):

    f_k = Re sum_s Tr[(Phi0_s^T phi_s)^-1 Phi0_s^T U_k phi_s],

so that the untrained network already proposes around the linearised target.
Training minimises the Gaussian negative log-likelihood of the paths' states,

    loss = 1/(W P) sum_wp 1/2 sum_k [(x_wpk - mu_wk)^2 / v_wk + logv_wk].

Parameters are one flat FP32-ordered vector: W1 (H x K), b1 (H), W2 (H x H),
b2 (H), W3 (2K x H), b3 (2K), all row-major.
"""

from __future__ import annotations

import numpy as np

LOGV_MIN = -6.0
LOGV_MAX = 3.0


def n_params(K: int, H: int = 256) -> int:
    return H * K + H + H * H + H + 2 * K * H + 2 * K


def unpack(theta: np.ndarray, K: int, H: int = 256):
    o = 0
    def take(*shape):
        nonlocal o
        n = int(np.prod(shape))
        a = theta[o:o + n].reshape(shape)
        o += n
        return a
    W1, b1 = take(H, K), take(H)
    W2, b2 = take(H, H), take(H)
    W3, b3 = take(2 * K, H), take(2 * K)
    return W1, b1, W2, b2, W3, b3


def features(Phi0: np.ndarray, U: np.ndarray, phi_up: np.ndarray, phi_dn: np.ndarray) -> np.ndarray:
    """f_k for walkers phi (W, N, n_s); Phi0 (N, n_up); U (K, N, N)."""
    f = np.zeros((phi_up.shape[0], U.shape[0]))
    for phi in (phi_up, phi_dn):
        n = phi.shape[2]
        if n == 0:
            continue
        P0 = Phi0[:, :n]
        A = np.einsum("ia,wib->wab", P0, phi)
        Theta0 = phi @ np.linalg.inv(A)                        # (W, N, n)
        UP = np.einsum("kij,ja->kia", U, P0)                   # U_k Phi0
        f += np.einsum("wia,kia->wk", Theta0, UP).real
    return f


def forward(theta, f, K, H=256):
    W1, b1, W2, b2, W3, b3 = unpack(theta, K, H)
    z1 = f @ W1.T + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2.T + b2
    h2 = np.tanh(z2)
    out = h2 @ W3.T + b3
    mu = f + out[:, :K]
    logv_raw = out[:, K:]
    logv = np.clip(logv_raw, LOGV_MIN, LOGV_MAX)
    return dict(h1=h1, h2=h2, out=out, mu=mu, logv=logv, logv_raw=logv_raw)


def loss_and_grad(theta, f, x, K, H=256):
    """f (W, K); x (W, P, K).  Returns (loss, grad) with grad the flat gradient."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, K, H)
    c = forward(theta, f, K, H)
    Wn, P = x.shape[:2]
    r = x - c["mu"][:, None, :]
    iv = np.exp(-c["logv"])[:, None, :]
    loss = 0.5 * np.sum(r * r * iv + c["logv"][:, None, :]) / (Wn * P)
    dmu = -np.sum(r * iv, axis=1) / (Wn * P)
    dlogv = 0.5 * np.sum(1.0 - r * r * iv, axis=1) / (Wn * P)
    dlogv = dlogv * ((c["logv_raw"] > LOGV_MIN) & (c["logv_raw"] < LOGV_MAX))
    dout = np.concatenate([dmu, dlogv], axis=1)
    gW3 = dout.T @ c["h2"]
    gb3 = dout.sum(axis=0)
    dz2 = (dout @ W3) * (1.0 - c["h2"] ** 2)
    gW2 = dz2.T @ c["h1"]
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - c["h1"] ** 2)
    gW1 = dz1.T @ f
    gb1 = dz1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad


def log_q(x, mu, logv):
    """log N(x; mu, diag exp(logv)) up to the constant shared by x and x'."""
    r = x - mu
    return -0.5 * np.sum(r * r * np.exp(-logv) + logv, axis=-1)
