"""Eq. (1) unit matching (Sec. 3) against the numbers the paper prints for its
case study (Sec. 3), and the synthetic tracer's frame acceleration."""
import math

import numpy as np
import pytest

from paper_0809_4958_gb300 import inputs, scaling


def _paper_map(tau=1.0):
    eta, tau_eta = scaling.kolmogorov(1.0 / 400.0, 0.1)  # run 4: nu = 1/400, eps = 0.1
    return scaling.UnitMap(eta=eta, tau_eta=tau_eta, delta=2 * math.pi / 1024, z=6, tau=tau), eta, tau_eta


def test_kolmogorov_scales_of_the_case_study():
    m, eta, tau_eta = _paper_map()
    assert eta == pytest.approx(0.0199, abs=5e-5)       # printed 0.0199
    assert tau_eta == pytest.approx(0.158, abs=5e-4)    # printed 0.158
    assert eta / m.delta == pytest.approx(3.24, abs=5e-3)  # printed 3.26 (reading: computed value used)


def test_mach_number_and_sampling_of_the_case_study():
    # tau = 1 (nu~ = 1/6) reproduces the printed Ma = 1.49e-2 at z = 6
    m, eta, tau_eta = _paper_map(1.0)
    assert m.mach == pytest.approx(1.49e-2, rel=5e-3)
    assert m.eta_lb == pytest.approx(6 * eta / m.delta)
    # one DNS sample every 0.05 tau_eta, 81 tau_eta in all
    assert m.steps(0.05 * tau_eta) == pytest.approx(113.4, abs=0.5)
    assert m.steps(81 * tau_eta) == pytest.approx(1.84e5, rel=5e-3)
    # Eq. (1): a Kolmogorov-unit velocity maps to a Kolmogorov-unit velocity
    assert (eta / tau_eta) * m.velocity == pytest.approx(m.eta_lb / m.tau_eta_lb, rel=1e-14)
    assert m.acceleration == pytest.approx(m.velocity / m.time, rel=1e-14)


def test_tracer_frame_accel_is_minus_dv_dt():
    modes = inputs.mode_table(2, 64, 1.0, 16.0, 32)
    t = np.array([0.0, 13.0, 57.5])
    h = 1e-3
    fd = -(inputs.tracer_velocity(modes, t + h) - inputs.tracer_velocity(modes, t - h)) / (2 * h)
    assert np.abs(inputs.tracer_frame_accel(modes, t) - fd).max() < 1e-9 * np.abs(fd).max() + 1e-15
