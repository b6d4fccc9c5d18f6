"""FP64 oracle of the learned boundary upsampler (test infrastructure only).

The paper interpolates the DNS boundary velocity linearly between samples
(Sec. 3, after Eq. 1).  The learned form predicts, per face site and coarse
interval [jK, (j+1)K], the difference between the true boundary velocity at
the K substeps and the cubic Hermite (Catmull-Rom) interpolant of the coarse
samples; the boundary then uses Hermite plus that residual.

Network (one row per face site and interval):
  features x (24, zero-padded to 32), divided by u_max:
    u at samples j-1, j, j+1, j+2 (3 components each; j-1 clamped to 0),
    in-face differences du/dp and du/dq at samples j and j+1 (central, one
    sided at face edges)
  h1 = relu(x W1 + b1)   (128)
  h2 = relu(h1 W2 + b2)  (128)
  y  = h2 W3 + b3        (3 K), y[3 (s - 1) + c] = residual of component c at
                          substep s, in units of u_max / OUT_DIV.

The output unit is a fraction of u_max because the Hermite residual is a few
thousandths of u_max: with targets that small, Adam's step (a fixed fraction
of a weight's scale per update) is large against the output weights the fit
needs, and training stalls at a noisy fit.

Rows are ordered face-major: row = (f E + q) E + p, faces x-, x+, y-, y+, z-, z+
with the in-face coordinates of the sample layout ([6][3][E][E], (q, p)).
"""
from __future__ import annotations

import numpy as np

NFEAT = 24
NIN = 32
HIDDEN = 128
OUT_DIV = 64.0  # network output unit: u_max / OUT_DIV


def _face_grad(U):
    """In-face differences of U [6][3][E][E] along p (last axis) and q."""
    gp = np.empty_like(U)
    gq = np.empty_like(U)
    gp[..., 1:-1] = 0.5 * (U[..., 2:] - U[..., :-2])
    gp[..., 0] = U[..., 1] - U[..., 0]
    gp[..., -1] = U[..., -1] - U[..., -2]
    gq[..., 1:-1, :] = 0.5 * (U[..., 2:, :] - U[..., :-2, :])
    gq[..., 0, :] = U[..., 1, :] - U[..., 0, :]
    gq[..., -1, :] = U[..., -1, :] - U[..., -2, :]
    return gp, gq


def features(samples, j, u_max):
    """Feature matrix [6 E^2][32] of interval j from coarse samples [J][6][3][E][E]."""
    S = np.asarray(samples, np.float64)
    E = S.shape[-1]
    cols = []
    for jj in (max(j - 1, 0), j, j + 1, j + 2):
        cols.append(S[jj])
    for jj in (j, j + 1):
        gp, gq = _face_grad(S[jj])
        cols.append(gp)
        cols.append(gq)
    X = np.zeros((6 * E * E, NIN))
    k = 0
    for blk in cols:  # blk [6][3][E][E]
        for c in range(3):
            X[:, k] = blk[:, c].reshape(-1) / u_max
            k += 1
    assert k == NFEAT
    return X


def hermite(samples, j, s, K):
    """Catmull-Rom cubic Hermite value [6][3][E][E] at t = jK + s (one-sided
    tangent on the first interval)."""
    S = np.asarray(samples, np.float64)
    th = s / K
    h00 = 2 * th ** 3 - 3 * th ** 2 + 1
    h10 = th ** 3 - 2 * th ** 2 + th
    h01 = -2 * th ** 3 + 3 * th ** 2
    h11 = th ** 3 - th ** 2
    m0 = 0.5 * (S[j + 1] - S[j - 1]) if j >= 1 else S[1] - S[0]
    m1 = 0.5 * (S[j + 2] - S[j])
    return h00 * S[j] + h10 * m0 + h01 * S[j + 1] + h11 * m1


def targets(fine, samples, j, K, u_max):
    """Target matrix [6 E^2][3 K]: (fine boundary velocity - Hermite) in units
    of u_max / OUT_DIV at t = jK + s, s = 1..K.  fine: [T][6][3][E][E] sampled
    every step."""
    E = np.asarray(samples).shape[-1]
    T = np.zeros((6 * E * E, 3 * K))
    for s in range(1, K + 1):
        r = (np.asarray(fine[j * K + s], np.float64) - hermite(samples, j, s, K)) * (OUT_DIV / u_max)
        for c in range(3):
            T[:, 3 * (s - 1) + c] = r[:, c].reshape(-1)
    return T


def init_params(seed, K, scale=1.0):
    """He-style initial weights (float64), W stored [in][out]."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.normal(0, np.sqrt(2.0 / NFEAT), (NIN, HIDDEN)) * scale,
        "b1": np.zeros(HIDDEN),
        "W2": rng.normal(0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN)) * scale,
        "b2": np.zeros(HIDDEN),
        "W3": rng.normal(0, np.sqrt(1.0 / HIDDEN), (HIDDEN, 3 * K)) * scale * 0.1,
        "b3": np.zeros(3 * K),
    }
    p["W1"][NFEAT:] = 0.0
    return p


def forward(p, X):
    """(y, cache) of the three-layer network."""
    a1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"] + p["b3"]
    return y, (X, a1, h1, a2, h2)


def loss(y, T):
    """Mean squared error over all elements."""
    return float(np.mean((y - T) ** 2))


def backward(p, cache, y, T):
    """Gradients of loss(y, T) with respect to every parameter."""
    X, a1, h1, a2, h2 = cache
    dy = 2.0 * (y - T) / y.size
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dh2 = dy @ p["W3"].T
    da2 = dh2 * (a2 > 0)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (a1 > 0)
    g["W1"] = X.T @ da1
    g["b1"] = da1.sum(0)
    return g


def residual_block(p, samples, j, K, u_max):
    """Residual [6][3][K][E][E] (velocity units) of interval j for the LB
    boundary (the oracle's time interpolation MLP mode)."""
    E = np.asarray(samples).shape[-1]
    y, _ = forward(p, features(samples, j, u_max))
    R = np.zeros((6, 3, K, E, E))
    for s in range(K):
        for c in range(3):
            R[:, c, s] = (y[:, 3 * s + c] * (u_max / OUT_DIV)).reshape(6, E, E)
    return R
