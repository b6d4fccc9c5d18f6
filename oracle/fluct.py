"""FP64 oracle of the fluctuating lattice Boltzmann collision (test
infrastructure only: the GPU's lb_set_fluctuation is checked against it).

The hybrid method the paper builds on (Sec. 1, the Ahlrichs-Duenweg coupling)
pairs thermal noise on the beads with a fluctuating fluid, so that kT > 0 is
consistent on both sides.  The collision runs in the D3Q19 orthogonal mode
basis: with weights w_i the 19 polynomials e_k(c) below satisfy
sum_i w_i e_k(c_i) e_l(c_i) = b_k delta_kl.  Modes 0-3 (mass and momentum) are
conserved; each other mode relaxes towards its equilibrium value and receives
noise of the amplitude the fluctuation-dissipation theorem fixes:

    m_k* = m_k^eq + gamma_k (m_k - m_k^eq) + sqrt(mu rho b_k (1 - gamma_k^2)) xi_k,

mu = kT / c_s^2 (unit particle mass), xi_k of unit variance.  With kT = 0 and
gamma_k = 1 - 1/tau for every non-conserved mode this is the BGK collision.
Random numbers: Philox4x32-10 with counter (step, site, mode block, 0xF1) and
the seed as key, words mapped to unit-variance uniforms on [-sqrt3, sqrt3), as
for the bead noise, so a GPU implementation can match it bit for bit.
Numpy, periodic boxes only (streaming by rolls).
"""
from __future__ import annotations

import numpy as np

from . import lattice

CS2 = 1.0 / 3.0
_M0, _M1, _W0, _W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85


def mode_basis():
    """e [19][19] (mode k at velocity i) and the norms b [19]."""
    c, w = lattice()
    cx, cy, cz = (c[:, a].astype(np.float64) for a in range(3))
    c2 = cx * cx + cy * cy + cz * cz
    e = np.array([
        np.ones(19), cx, cy, cz,
        c2 - 1.0, 3.0 * cx * cx - c2, cy * cy - cz * cz,
        cx * cy, cy * cz, cz * cx,
        (3.0 * c2 - 5.0) * cx, (3.0 * c2 - 5.0) * cy, (3.0 * c2 - 5.0) * cz,
        (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz,
        3.0 * c2 * c2 - 6.0 * c2 + 1.0,
        (2.0 * c2 - 3.0) * (3.0 * cx * cx - c2), (2.0 * c2 - 3.0) * (cy * cy - cz * cz),
    ])
    b = (e * e * w[None, :]).sum(axis=1)
    return e, b


def philox4x32_10_vec(ctr, key):
    """Philox4x32-10 of counters ctr [..., 4] (uint32) with key (k0, k1)."""
    x = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(_W0)) & mask
            k1 = (k1 + np.uint64(_W1)) & mask
        p0 = np.uint64(_M0) * x[0]
        p1 = np.uint64(_M1) * x[2]
        y0 = ((p1 >> np.uint64(32)) ^ x[1] ^ k0) & mask
        y1 = p1 & mask
        y2 = ((p0 >> np.uint64(32)) ^ x[3] ^ k1) & mask
        y3 = p0 & mask
        x = [y0, y1, y2, y3]
    return np.stack(x, axis=-1).astype(np.uint32)


def mode_noise(step, nsites, seed):
    """Unit-variance uniforms xi [15][nsites] for modes 4..18 of every site at
    a step: counter (step, site, block, 0xF1), blocks 0..3 give 4 words each."""
    site = np.arange(nsites, dtype=np.uint64)
    words = []
    for blk in range(4):
        ctr = np.zeros((nsites, 4), dtype=np.uint64)
        ctr[:, 0] = np.uint64(step & 0xFFFFFFFF)
        ctr[:, 1] = site
        ctr[:, 2] = np.uint64(blk)
        ctr[:, 3] = np.uint64(0xF1)
        words.append(philox4x32_10_vec(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)))
    v = np.concatenate(words, axis=1)[:, :15].T.astype(np.float64)  # [15][nsites]
    return np.sqrt(3.0) * (2.0 * (v * (1.0 / 4294967296.0)) - 1.0)


def equilibrium_modes(e, rho, u):
    """Equilibrium moments m_k^eq [19][sites] of f^eq(rho, u)."""
    c, w = lattice()
    cu = c.astype(np.float64) @ u                       # [19][sites]
    usq = (u * u).sum(axis=0)
    feq = w[:, None] * rho[None, :] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq[None, :])
    return e @ feq


def collide(f, gamma, kT, step, seed):
    """Fluctuating collision of populations f [19][sites]: gamma [19] (modes
    0-3 ignored, they are conserved)."""
    e, b = mode_basis()
    c, w = lattice()
    m = e @ f
    rho = m[0]
    u = m[1:4] / rho[None, :]
    meq = equilibrium_modes(e, rho, u)
    ms = m.copy()
    g = np.asarray(gamma, dtype=np.float64)
    ms[4:] = meq[4:] + g[4:, None] * (m[4:] - meq[4:])
    if kT > 0.0:
        mu = kT / CS2
        xi = mode_noise(step, f.shape[1], seed)
        ms[4:] += np.sqrt(mu * rho[None, :] * b[4:, None] * (1.0 - g[4:, None] ** 2)) * xi
    # back to populations: f_i = w_i sum_k e_k(c_i) m_k / b_k
    return w[:, None] * (e.T @ (ms / b[:, None]))


def stream_periodic(f, E):
    """Pull streaming in a periodic box: f_i(x) <- f_i(x - c_i)."""
    c, _ = lattice()
    g = f.reshape(19, E, E, E)
    out = np.empty_like(g)
    for i in range(19):
        out[i] = np.roll(g[i], shift=(int(c[i, 2]), int(c[i, 1]), int(c[i, 0])), axis=(0, 1, 2))
    return out.reshape(19, -1)


def run_periodic(f, E, gamma, kT, seed, n0, nsteps, observe=None):
    """Collide-then-stream steps n0 .. n0 + nsteps - 1 of a periodic box
    (populations [19][E^3]); observe(step, f) after every step."""
    for n in range(n0, n0 + nsteps):
        f = stream_periodic(collide(f, gamma, kT, n, seed), E)
        if observe is not None:
            observe(n, f)
    return f
