"""Seeded synthetic inputs for the tracer-box method.

This module draws the random inputs that both the CUDA path and the CPU
oracle consume, so that both see bit-identical numbers.  It holds none of the
lattice Boltzmann, boundary or bead arithmetic.

The paper feeds its fine lattice Boltzmann box with velocity samples of a
1024^3 DNS recorded around Lagrangian tracers (Sec. 2 and 3).  That record is
not available; a synthetic divergence-free random-phase field with a
Kolmogorov spectrum stands in for it:

    u(x, t) = sum_m amp_m cos(kvec_m . (x - xc) + omega_m t + phi_m)

  k_m      = k_min (k_max / k_min)^(m / (M - 1))         (log spaced)
  khat_m   uniform on the unit sphere, kvec_m = (2 pi k_m / E) khat_m
  e_m      unit vector perpendicular to khat_m, uniform angle (divergence free)
  A_m      = sqrt(Ek(k_m) dk_m), Ek(k) = k^(-5/3) exp(-(k / 16)^2),
             dk_m = k_m ln(k_max / k_min) / (M - 1)
  phi_m    uniform on [0, 2 pi)
  omega_m  = u_max (2 pi / E) k_m^(2/3)
  amp_m    = S A_m e_m, S such that max |u(x, 0)| = u_max over the sample
             lattice (every max(1, E // 32)-th site per axis plus the last
             site, so the maximum is exact for E < 64 and a close lower bound
             of the true maximum above that).

Bead chains start as seeded self-avoiding random walks (bond length 0.97,
directions uniform on the sphere, every bead at least 1.0 from all earlier
non-adjacent beads) translated so the centre of mass sits at the box centre,
redrawn until every bead lies in [1, E - 2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Modes:
    """Mode table of the synthetic coarse flow (float64, C-contiguous)."""
    kvec: np.ndarray   # [M][3] wave vectors in lattice units (radians per site)
    amp: np.ndarray    # [M][3] amplitude vectors S A_m e_m
    omega: np.ndarray  # [M] angular frequencies (radians per LB step)
    phi: np.ndarray    # [M] phases
    E: int
    u_max: float

    @property
    def M(self) -> int:
        return int(self.kvec.shape[0])


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)]))


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, n)
    a = rng.uniform(0.0, 2.0 * np.pi, n)
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(a), r * np.sin(a), z], axis=1)


def sample_lattice(E: int) -> np.ndarray:
    """Points at which the normalisation maximum is taken: [n][3]."""
    stride = max(1, E // 32)
    ax = np.unique(np.concatenate([np.arange(0, E, stride), [E - 1]])).astype(np.float64)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def mode_table(seed: int, M: int, k_min: float, k_max: float, E: int, u_max: float = 0.05) -> Modes:
    """Draw the Kolmogorov-spectrum mode table for one box (see module doc)."""
    rng = _rng(seed, 1)
    m = np.arange(M, dtype=np.float64)
    if M > 1:
        k = k_min * (k_max / k_min) ** (m / (M - 1))
        dk = k * np.log(k_max / k_min) / (M - 1)
    else:
        k = np.array([k_min], dtype=np.float64)
        dk = np.array([1.0])
    khat = _unit_vectors(rng, M)
    # orthonormal pair perpendicular to khat, then a uniform angle in that plane
    helper = np.where(np.abs(khat[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    a1 = np.cross(khat, helper)
    a1 /= np.linalg.norm(a1, axis=1, keepdims=True)
    a2 = np.cross(khat, a1)
    ang = rng.uniform(0.0, 2.0 * np.pi, M)
    e = np.cos(ang)[:, None] * a1 + np.sin(ang)[:, None] * a2
    spectrum = k ** (-5.0 / 3.0) * np.exp(-(k / 16.0) ** 2)
    A = np.sqrt(spectrum * dk)
    phi = rng.uniform(0.0, 2.0 * np.pi, M)
    omega = u_max * (2.0 * np.pi / E) * k ** (2.0 / 3.0)
    kvec = (2.0 * np.pi * k / E)[:, None] * khat
    amp = A[:, None] * e
    # normalise: max |u(x, 0)| over the sample lattice equals u_max
    pts = sample_lattice(E) - 0.5 * (E - 1)
    umax_seen = 0.0
    for s in range(0, pts.shape[0], 4096):
        ph = pts[s:s + 4096] @ kvec.T + phi[None, :]
        u = np.cos(ph) @ amp
        umax_seen = max(umax_seen, float(np.sqrt((u * u).sum(axis=1)).max()))
    amp = amp * (u_max / umax_seen)
    return Modes(kvec=np.ascontiguousarray(kvec), amp=np.ascontiguousarray(amp),
                 omega=np.ascontiguousarray(omega), phi=np.ascontiguousarray(phi), E=E, u_max=u_max)


def single_mode(E: int, kvec, amp, omega: float = 0.0, phi: float = 0.0) -> Modes:
    """A one-mode table (for closed-form checks)."""
    return Modes(kvec=np.ascontiguousarray(np.reshape(np.asarray(kvec, np.float64), (1, 3))),
                 amp=np.ascontiguousarray(np.reshape(np.asarray(amp, np.float64), (1, 3))),
                 omega=np.array([float(omega)]), phi=np.array([float(phi)]), E=E, u_max=0.0)


def chain_start(seed: int, nbeads: int, E: int, bond: float = 0.97, min_dist: float = 1.0,
                max_tries: int = 1000) -> np.ndarray:
    """Self-avoiding random-walk chain start [nbeads][3] centred at
    ((E-1)/2)^3, all beads in [1, E-2)."""
    rng = _rng(seed, 2)
    centre = 0.5 * (E - 1)
    for _ in range(max_tries):
        pos = np.zeros((nbeads, 3))
        ok = True
        for b in range(1, nbeads):
            for _attempt in range(200):
                cand = pos[b - 1] + bond * _unit_vectors(rng, 1)[0]
                if b < 2 or np.min(np.sum((pos[:b - 1] - cand) ** 2, axis=1)) >= min_dist ** 2:
                    pos[b] = cand
                    break
            else:
                ok = False
                break
        if not ok:
            continue
        pos += centre - pos.mean(axis=0)
        if np.all(pos >= 1.0) and np.all(pos < E - 2):
            return np.ascontiguousarray(pos)
    raise ValueError("chain of %d beads does not fit a box of edge %d" % (nbeads, E))


def batch_edges(seed: int, nboxes: int, choices=(24, 32, 48, 64)) -> np.ndarray:
    """Box edges drawn uniformly from ``choices``."""
    rng = _rng(seed, 3)
    return np.asarray(choices, dtype=np.int64)[rng.integers(0, len(choices), nboxes)]


def batch_chain_lengths(seed: int, edges) -> np.ndarray:
    """Chain length per box, uniform on [32, min(128, 2 E)]."""
    rng = _rng(seed, 4)
    edges = np.asarray(edges)
    hi = np.minimum(128, 2 * edges)
    return (32 + np.floor(rng.uniform(0.0, 1.0, edges.shape[0]) * (hi - 32 + 1))).astype(np.int64)


def mlp_init(seed: int, K: int, scale: float = 1.0) -> np.ndarray:
    """Seeded initial weights of the learned boundary upsampler as one float32
    vector in master layout: W1 [32][128] (rows 24..31 zero: padding inputs),
    b1 [128], W2 [128][128], b2 [128], W3 [128][3K], b3 [3K]; He-style normal
    draws, biases zero, the output layer scaled down by 10."""
    rng = _rng(seed, 5)
    W1 = rng.normal(0.0, np.sqrt(2.0 / 24), (32, 128)) * scale
    W1[24:] = 0.0
    W2 = rng.normal(0.0, np.sqrt(2.0 / 128), (128, 128)) * scale
    W3 = rng.normal(0.0, np.sqrt(1.0 / 128), (128, 3 * K)) * scale * 0.1
    return np.concatenate([W1.ravel(), np.zeros(128), W2.ravel(), np.zeros(128), W3.ravel(),
                           np.zeros(3 * K)]).astype(np.float32)


def tracer_velocity(modes: Modes, t) -> np.ndarray:
    """Velocity of the synthetic field at the box centre (the tracer's own
    velocity v(t), which the co-moving frame subtracts) at times t: [len(t)][3]."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.cos(modes.omega[None, :] * t[:, None] + modes.phi[None, :]) @ modes.amp


def tracer_frame_accel(modes: Modes, t) -> np.ndarray:
    """Frame acceleration -dv/dt of the tracer at the box centre at times t:
    [len(t)][3] (the time derivative of tracer_velocity, negated)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return (modes.omega[None, :] * np.sin(modes.omega[None, :] * t[:, None] + modes.phi[None, :])) @ modes.amp

