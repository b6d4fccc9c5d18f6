"""Pins of the co-moving-frame body force (Sec. 2: the flow in the tracer's
frame, w = u - v(t), feels the force density rho (-dv/dt)) on the oracle."""
import numpy as np
import pytest


def test_frame_accel_interpolates_linearly(orc):
    # samples of a linear-in-time acceleration are reproduced exactly between samples
    K = 4
    samp = np.array([[0.1 * j, -0.2 * j + 1.0, 0.05] for j in range(6)]) * 1e-5
    for n in range(0, 4 * K):
        t = n / K
        ref = np.array([0.1 * t, -0.2 * t + 1.0, 0.05]) * 1e-5 + np.array([1e-6, 0, 0])
        assert np.allclose(orc.frame_accel_at((1e-6, 0, 0), samp, K, n), ref, rtol=0, atol=1e-20)


def test_periodic_uniform_flow_integrates_the_frame_force(orc):
    # A uniform state in a fully periodic box stays uniform; BGK with Guo
    # forcing adds exactly rho a(n) to the momentum each step, and the reported
    # velocity carries half of the current step's force:
    #   u(N) = u0 + sum_{m < N} a(m) + a(N) / 2.
    E, K, N = 8, 2, 9
    rng = np.random.default_rng(3)
    samp = rng.normal(size=(N // K + 3, 3)) * 2e-5
    box = orc.BoxParams(E=E, tau=0.7, periodic=(True, True, True), K=K)
    u0 = np.array([0.01, -0.02, 0.005])
    A = orc.init(box, np.broadcast_to(u0[:, None, None, None], (3, E, E, E)).copy())
    st, A, _, _ = orc.run_frame(box, A, np.zeros((1, 6, 3, E, E)), samp, 0, N)
    assert st == 0
    from dataclasses import replace
    aN = orc.frame_accel_at(box.accel, samp, K, N)
    _, u = orc.fields(replace(box, accel=tuple(aN)), A)
    ref = u0 + sum(orc.frame_accel_at(box.accel, samp, K, m) for m in range(N)) + 0.5 * aN
    for c in range(3):
        assert np.abs(u[c] - ref[c]).max() < 1e-15
