"""Pins of the fluctuating-LB oracle (the thermal fluid of the hybrid method the
paper builds on): orthogonal mode basis, BGK limit, conservation with noise,
equipartition, and the vectorised Philox against the pinned scalar one."""
from fractions import Fraction

import numpy as np
import pytest


@pytest.fixture(scope="module")
def fl(orc):
    from oracle import fluct
    return fluct


def test_mode_basis_is_orthogonal_exactly(orc, fl):
    c, _ = orc.lattice()
    w = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12
    e, b = fl.mode_basis()
    ei = np.rint(e).astype(int)
    assert np.array_equal(ei, e)  # integer polynomials of integer velocities
    for k in range(19):
        for l in range(19):
            s = sum(w[i] * int(ei[k, i]) * int(ei[l, i]) for i in range(19))
            if k == l:
                assert s > 0 and float(s) == pytest.approx(b[k], rel=1e-15)
            else:
                assert s == 0, (k, l)


def test_vectorised_philox_matches_the_pinned_scalar_one(orc, fl):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(5, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    v = fl.philox4x32_10_vec(ctr.astype(np.uint64), key)
    for r in range(5):
        assert np.array_equal(v[r], orc.philox4x32_10(ctr[r], np.array(key, np.uint32)))


def _smooth_state(orc, E, amp=0.02):
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    k = 2 * np.pi / E
    u = np.stack([amp * np.sin(k * Y), amp * np.cos(k * Z + 0.3), amp * 0.5 * np.sin(k * X + 1.0)])
    box = orc.BoxParams(E=E, tau=0.8, periodic=(True, True, True))
    return box, orc.init(box, u)


def test_zero_temperature_single_rate_is_bgk(orc, fl):
    E, tau = 8, 0.8
    box, A = _smooth_state(orc, E)
    A = A + 1e-4 * np.sin(np.arange(A.size).reshape(A.shape))  # off equilibrium
    gamma = np.full(19, 1.0 - 1.0 / tau)
    Bf = fl.collide(fl.stream_periodic(A.reshape(19, -1), E), gamma, 0.0, 0, 1)
    st, Bref, _, _, _ = orc.step_from(box, A, np.zeros((1, 6, 3, E, E)), 0)
    assert st == 0
    assert np.abs(Bf - Bref.reshape(19, -1)).max() < 1e-15


def test_noise_conserves_mass_and_momentum(orc, fl):
    E = 6
    box, A = _smooth_state(orc, E)
    f = A.reshape(19, -1)
    c, _ = orc.lattice()
    g = fl.collide(f, np.zeros(19), 1e-3, 7, 3)
    assert np.abs(g.sum(0) - f.sum(0)).max() < 1e-15
    assert np.abs(c.T.astype(float) @ g - c.T.astype(float) @ f).max() < 1e-15
    assert not np.allclose(g, fl.collide(f, np.zeros(19), 0.0, 7, 3))  # the noise is there


def test_equipartition_of_the_velocity(orc, fl):
    # periodic box at rest, all non-conserved modes fully thermalised (gamma 0):
    # <u_a^2> = kT / rho per component (minus the conserved total momentum)
    E, kT = 8, 1e-5
    box = orc.BoxParams(E=E, tau=1.0, periodic=(True, True, True))
    f = orc.init(box, np.zeros((3, E, E, E))).reshape(19, -1)
    c, _ = orc.lattice()
    acc = []

    def obs(n, g):
        if n >= 100:
            rho = g.sum(0)
            u = (c.T.astype(float) @ g) / rho
            acc.append((u * u).mean())

    fl.run_periodic(f, E, np.zeros(19), kT, 11, 0, 900, obs)
    ref = kT * (1.0 - 1.0 / E ** 3)
    assert np.mean(acc) == pytest.approx(ref, rel=0.03)


def test_noise_is_reproducible(orc, fl):
    a = fl.mode_noise(5, 64, 99)
    assert np.array_equal(a, fl.mode_noise(5, 64, 99))
    assert not np.array_equal(a, fl.mode_noise(6, 64, 99))
    big = fl.mode_noise(5, 4096, 99)  # 61,440 draws: mean 0, variance 1, bounded by sqrt(3)
    assert abs(big.mean()) < 0.02 and big.var() == pytest.approx(1.0, rel=0.02)
    assert np.abs(big).max() < np.sqrt(3.0)
