"""Pins of the oracle's lattice Boltzmann update (stream-collide, velocity
boundary, forcing) against closed-form flows and conservation laws."""
import numpy as np
import pytest

from paper_0809_4958_gb300 import inputs
from flowcases import abc_flow, faces_from, vol_from


def _const_samples(E, u, J=2):
    S = np.zeros((J, 6, 3, E, E))
    for c in range(3):
        S[:, :, c] = u[c]
    return S


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.3])
def test_uniform_flow_is_a_fixed_point(orc, tau):
    # constant velocity on every face and in the interior stays exactly constant
    E = 8
    u = (0.03, -0.02, 0.01)
    box = orc.BoxParams(E=E, tau=tau, K=1)
    sim = orc.Sim(box, vol_from(lambda X, Y, Z, t: u, E), _const_samples(E, u, J=60))
    assert sim.run(50) == 0
    rho, uf = sim.fields()
    assert np.abs(rho - 1).max() < 1e-14
    for c in range(3):
        assert np.abs(uf[c] - u[c]).max() < 1e-15


def test_periodic_conservation_with_chain(orc):
    # all axes periodic, chain with noise, no pinning: mass and total momentum
    # (fluid + beads) are conserved to rounding over 1000 steps
    E = 16
    mt = inputs.mode_table(1, 64, 1, 4, E)
    u0 = orc.volume_field(mt, E, 0.0)
    box = orc.BoxParams(E=E, tau=0.8, periodic=(True, True, True))
    ch = orc.ChainParams(nbeads=8, kT=1e-4, seed=11, pin_com=0, n_md=50)
    pos0 = inputs.chain_start(4, 8, E)
    sim = orc.Sim(box, u0, np.zeros((2, 6, 3, E, E)), ch, pos0, vel0=np.full((8, 3), 0.01))
    c0 = sim.conservation()
    assert sim.run(1000) == 0
    c1 = sim.conservation()
    mass = E ** 3
    assert abs(c1[0] - c0[0]) <= 1e-12 * mass
    p0 = c0[1:4] + c0[4:7]
    p1 = c1[1:4] + c1[4:7]
    pscale = mass * 0.05
    assert np.abs(p1 - p0).max() <= 1e-12 * pscale
    # and momentum really was exchanged between beads and fluid
    assert np.abs(c1[4:7] - c0[4:7]).max() > 1e-4
    # a mistake in the force sign or the half-force shift would break this
    assert np.abs(c1[1:4] - c0[1:4]).max() > 1e-4


def _taylor_green_nu(orc, E, tau):
    k = 2 * np.pi / E
    U = 1e-4
    fn = lambda X, Y, Z, t: (U * np.cos(k * X) * np.sin(k * Y), -U * np.sin(k * X) * np.cos(k * Y), 0 * X)
    nu = (tau - 0.5) / 3
    box = orc.BoxParams(E=E, tau=tau, periodic=(True, True, True))
    sim = orc.Sim(box, vol_from(fn, E), np.zeros((2, 6, 3, E, E)))
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    basis = np.cos(k * X) * np.sin(k * Y)
    chunk = max(1, int(0.6 / (2 * nu * k * k)) // 20)
    ts, amps = [], []
    for _ in range(20):
        assert sim.run(chunk) == 0
        u = sim.fields()[1]
        ts.append(sim.n)
        amps.append((u[0] * basis).sum() / (basis * basis).sum())
    rate = -np.polyfit(np.array(ts[5:]), np.log(np.array(amps[5:])), 1)[0]
    return rate / (2 * k * k), nu


def test_taylor_green_viscosity(orc):
    # the 2-D Taylor-Green mode decays as exp(-2 nu k^2 t) with
    # nu = cs^2 (tau - 1/2); the fitted nu converges at second order in E
    nu16, nu = _taylor_green_nu(orc, 16, 0.8)
    nu32, _ = _taylor_green_nu(orc, 32, 0.8)
    e16, e32 = abs(nu16 / nu - 1), abs(nu32 / nu - 1)
    assert e32 < 0.01
    assert e16 / e32 > 3.0
    nu32b, nub = _taylor_green_nu(orc, 32, 0.55)
    assert abs(nu32b / nub - 1) < 0.01


def _couette(orc, E, tau, u0_linear):
    U = 0.01
    lin = lambda X, Y, Z, t: (U * Y / (E - 1), 0 * X, 0 * X)
    box = orc.BoxParams(E=E, tau=tau, periodic=(True, False, True), K=10 ** 6)
    S = faces_from(lin, E, 2, 10 ** 6)
    u0 = vol_from(lin, E) if u0_linear else np.zeros((3, E, E, E))
    return orc.Sim(box, u0, S), U


def test_couette_exact_at_tau_one(orc):
    # at tau = 1 the post-collision populations are equilibria, and for D3Q19
    # the quadratic terms cancel (sum w c_x^2 c_y^2 = 1/9): the linear profile
    # between equilibrium walls is an exact fixed point ...
    E = 8
    sim, U = _couette(orc, E, 1.0, True)
    assert sim.run(100) == 0
    u = sim.fields()[1]
    y = np.arange(E)
    assert np.abs(u[0] - (U * y / (E - 1))[None, :, None]).max() < 1e-15
    assert np.abs(u[1:]).max() < 1e-15
    # ... and it is reached from rest
    sim, U = _couette(orc, E, 1.0, False)
    assert sim.run(1200) == 0
    prof = sim.fields()[1][0, E // 2, :, E // 2]
    assert np.abs(prof - U * y / (E - 1)).max() < 1e-12 * U


def test_couette_converges_for_other_tau(orc):
    errs = []
    for E in (8, 16):
        sim, U = _couette(orc, E, 0.8, True)
        assert sim.run(int(20 * E * E / 0.1 / np.pi ** 2)) == 0
        prof = sim.fields()[1][0, E // 2, :, E // 2]
        y = np.arange(E)
        errs.append(np.abs(prof - U * y / (E - 1)).max() / U)
    assert errs[0] < 0.03 and errs[1] < 0.015 and errs[0] / errs[1] > 1.6


def test_poiseuille_profile(orc):
    # body acceleration a along x between equilibrium walls at y = 0, E-1:
    # u_x = a / (2 nu) y (E - 1 - y); equilibrium walls carry no
    # non-equilibrium part, so the profile is not exact, but it converges
    # at second order (measured: 1/72 at E = 8, 1/336 at E = 16)
    errs = []
    for E in (8, 16):
        tau, a = 1.0, 1e-6
        nu = (tau - 0.5) / 3
        ex = lambda X, Y, Z, t: (a / (2 * nu) * Y * (E - 1 - Y), 0 * X, 0 * X)
        box = orc.BoxParams(E=E, tau=tau, periodic=(True, False, True), accel=(a, 0, 0), K=10 ** 6)
        sim = orc.Sim(box, vol_from(ex, E), np.zeros((2, 6, 3, E, E)))
        assert sim.run(int(20 * E * E / nu / np.pi ** 2)) == 0
        y = np.arange(E, dtype=float)
        exact = a / (2 * nu) * y * (E - 1 - y)
        prof = sim.fields()[1][0, E // 2, :, E // 2]
        errs.append(np.abs(prof - exact).max() / exact.max())
    assert errs[1] < 3.5e-3
    assert errs[0] / errs[1] > 4.0


def test_abc_flow_recovered_from_boundary(orc):
    # Sec. 2: with the initial field everywhere and the velocity only on the
    # boundary afterwards, the interior must follow the unique Navier-Stokes
    # solution.  The decaying ABC flow is such a solution; the lattice result
    # approaches it as the resolution grows.
    errs = []
    for E in (16, 32):
        tau = 0.8
        fn, nu, k = abc_flow(E, tau)
        T = int(1.0 / (nu * k * k))
        box = orc.BoxParams(E=E, tau=tau, K=1)
        sim = orc.Sim(box, vol_from(fn, E), faces_from(fn, E, T + 2, 1))
        assert sim.run(T) == 0
        u = sim.fields()[1]
        ex = vol_from(fn, E, float(T))
        sl = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
        errs.append(np.sqrt(((u[sl] - ex[sl]) ** 2).sum() / (ex[sl] ** 2).sum()))
    assert errs[0] < 0.06 and errs[1] < 0.03
    assert errs[0] / errs[1] > 1.8


def test_storage_emulation_rounds_deviations(orc):
    # with 16-bit storage every stored population is w_i + (a binary16 value)
    E = 8
    _, w = orc.lattice()
    mt = inputs.mode_table(2, 16, 1, 3, E)
    for st, rnd in [(orc.STORE_F16, lambda v: float(np.float64(v).astype(np.float16))), (orc.STORE_BF16, orc.round_bf16)]:
        box = orc.BoxParams(E=E, tau=0.8, storage=st)
        sim = orc.Sim(box, orc.volume_field(mt, E), orc.face_samples(mt, E, 1, 0, 6))
        assert sim.run(3) == 0
        d = sim.f - w[:, None, None, None]
        sample = d.ravel()[:: 97]
        # w_i + r is held in FP64, so r comes back to within an FP64 ulp of w_i
        assert all(abs(rnd(v) - v) <= 2e-17 for v in sample)
