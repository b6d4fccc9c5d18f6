"""Pins of the oracle's vorticity diagnostic (mean |curl u| over a cube by
central differences, Sec. 3, Figs. 1 and 2) against closed forms."""
import numpy as np
import pytest

from flowcases import abc_flow, vol_from


def test_abc_flow_curl_is_sin_k_times_u(orc):
    # Beltrami field: curl u = k u.  On the lattice a central difference of
    # sin(k x) is sin(k) cos(k x), so the discrete curl is exactly sin(k) u.
    E = 24
    fn, nu, k = abc_flow(E, 0.8)
    u = vol_from(fn, E)
    for lo, hi in ((1, E - 2), (9, 14), (5, 5)):
        ref = np.sin(k) * np.sqrt((u ** 2).sum(0))[lo:hi + 1, lo:hi + 1, lo:hi + 1].mean()
        assert orc.vorticity_mean(u, lo, hi) == pytest.approx(ref, rel=1e-13)


def test_rigid_rotation_has_curl_twice_the_rate(orc):
    # u = Omega x (r - r0): central differences are exact on a linear field,
    # curl u = 2 Omega everywhere
    E = 16
    Om = np.array([0.003, -0.002, 0.005])
    ar = np.arange(E, dtype=float) - 7.3
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    u = np.stack([Om[1] * Z - Om[2] * Y, Om[2] * X - Om[0] * Z, Om[0] * Y - Om[1] * X])
    assert orc.vorticity_mean(u, 1, E - 2) == pytest.approx(2 * np.linalg.norm(Om), rel=1e-12)


def test_gradient_field_has_no_curl(orc):
    # u = grad(x^2 + y z) = (2x, z, y): linear, irrotational
    E = 12
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    u = np.stack([2 * X, Z, Y]) * 1e-3
    assert orc.vorticity_mean(u, 1, E - 2) < 1e-15


def test_component_order_matters(orc):
    # a shear u_x = s y has curl (0, 0, -s): a swapped derivative or sign would
    # give a different magnitude on the mixed field below
    E = 12
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    s, t = 2e-3, 7e-4
    u = np.stack([s * Y, t * X, np.zeros_like(X)])  # curl = (0, 0, t - s)
    assert orc.vorticity_mean(u, 2, 9) == pytest.approx(abs(t - s), rel=1e-12)
    u2 = np.stack([s * Y, np.zeros_like(X), t * Y])  # curl = (t, 0, -s)
    assert orc.vorticity_mean(u2, 2, 9) == pytest.approx(np.hypot(t, s), rel=1e-12)
