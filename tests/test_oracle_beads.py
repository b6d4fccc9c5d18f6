"""Pins of the oracle's bead-fluid coupling (Stokes friction point particles,
trilinear interpolation and spreading, FENE chain, centre-of-mass pinning)."""
import numpy as np
import pytest

from paper_0809_4958_gb300 import inputs
from flowcases import lattice_shift_state


def test_trilinear_interpolation_exact_on_linear_field(orc):
    E = 12
    u0 = np.array([0.01, -0.02, 0.005])
    G = np.array([[1e-3, 2e-4, -3e-4], [-5e-4, 1e-4, 7e-4], [2e-4, -6e-4, 3e-4]])
    lin = lambda X, Y, Z: tuple(u0[a] + G[a, 0] * X + G[a, 1] * Y + G[a, 2] * Z for a in range(3))
    # rho = 1 only to first order in u for the shifted state; keep u small and
    # check against the moments the oracle itself reports at the sites
    A = lattice_shift_state(orc, E, lin)
    box = orc.BoxParams(E=E, tau=0.8)
    rho, uf = orc.fields(box, A)
    rng = np.random.default_rng(0)
    for _ in range(20):
        R = rng.uniform(1.0, E - 2.0 - 1e-9, 3)
        st, u = orc.interp_velocity(box, A, R)
        assert st == 0
        i0 = np.floor(R).astype(int)
        d = R - i0
        # trilinear combination of the site values ...
        ref = np.zeros(3)
        for c in range(8):
            o = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
            wgt = np.prod(np.where(o == 1, d, 1 - d))
            s = i0 + o
            ref += wgt * uf[:, s[2], s[1], s[0]]
        assert np.allclose(u, ref, atol=1e-17, rtol=1e-13)
    # ... and the site values are the linear field up to the O(u^2) density
    # variation of the shifted state, so the interpolant is the linear field
    R = np.array([4.3, 6.7, 5.1])
    st, u = orc.interp_velocity(box, A, R)
    assert np.allclose(u, u0 + G @ R, atol=2e-6)
    # stencil leaving the interior on a velocity axis is an error
    assert orc.interp_velocity(box, A, np.array([0.5, 5.0, 5.0]))[0] == orc.ERR_BEAD_OOB
    assert orc.interp_velocity(box, A, np.array([5.0, 10.0, 5.0]))[0] == orc.ERR_BEAD_OOB


def _uniform_state(orc, E, u):
    feq = orc.equilibrium(1.0, u)
    return np.ascontiguousarray(np.broadcast_to(feq[:, None, None, None], (19, E, E, E)))


def test_single_substep_friction_update(orc):
    # one substep of length 1 in uniform flow u0: V1 = V0 - zeta (V0 - u0) / m,
    # R1 = R0 + V1, momentum -zeta (V0 - u0) ... given to the fluid with
    # opposite sign, spread with the trilinear weights of R0
    E = 8
    u0 = np.array([0.02, -0.01, 0.005])
    A = _uniform_state(orc, E, u0)
    box = orc.BoxParams(E=E, tau=0.8)
    R0 = np.array([[3.25, 4.5, 2.75]])
    V0 = np.array([[0.1, 0.03, -0.02]])
    zeta, m = 0.7, 2.0
    ch = orc.ChainParams(nbeads=1, zeta=zeta, mass=m, n_md=1, pin_com=0)
    st, pos, vel, g = orc.chain_couple(box, ch, A, 0, R0, V0)
    assert st == 0
    V1 = V0[0] - zeta * (V0[0] - u0) / m
    assert np.allclose(vel[0], V1, atol=1e-17, rtol=1e-15)
    assert np.allclose(pos[0], R0[0] + V1, atol=1e-15)
    P = zeta * (V0[0] - u0)  # momentum given to the fluid: -(F_fric) dt
    i0 = np.floor(R0[0]).astype(int)
    d = R0[0] - i0
    nz = np.argwhere(np.abs(g).sum(0) > 0)
    assert len(nz) == 8
    for c in range(8):
        o = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        wgt = np.prod(np.where(o == 1, d, 1 - d))
        s = i0 + o
        assert np.allclose(g[:, s[2], s[1], s[0]], wgt * P, atol=1e-18, rtol=1e-14)


def test_momentum_given_to_fluid_equals_bead_momentum_loss(orc):
    E = 16
    mt = inputs.mode_table(3, 32, 1, 4, E)
    box = orc.BoxParams(E=E, tau=0.8, periodic=(True, True, True))
    A = orc.init(box, orc.volume_field(mt, E))
    pos = inputs.chain_start(1, 16, E)
    vel = np.random.default_rng(0).normal(0, 0.01, (16, 3))
    ch = orc.ChainParams(nbeads=16, kT=1e-3, seed=5, pin_com=0)
    st, p1, v1, g = orc.chain_couple(box, ch, A, 7, pos, vel)
    assert st == 0
    dP_beads = ch.mass * (v1 - vel).sum(0)
    assert np.allclose(g.reshape(3, -1).sum(1), -dP_beads, atol=1e-15)
    assert np.abs(dP_beads).max() > 1e-3


def test_centre_of_mass_pinning(orc):
    E = 16
    box = orc.BoxParams(E=E, tau=0.8)
    A = _uniform_state(orc, E, np.array([0.03, 0.0, -0.02]))
    pos = inputs.chain_start(2, 12, E)
    vel = np.random.default_rng(1).normal(0, 0.02, (12, 3))
    for pin in (1, 2):
        ch = orc.ChainParams(nbeads=12, pin_com=pin)
        st, p1, v1, _ = orc.chain_couple(box, ch, A, 0, pos, vel)
        assert st == 0
        assert np.allclose(p1.mean(0), 7.5, atol=1e-13)
        if pin == 2:
            assert np.allclose(v1.mean(0), 0.0, atol=1e-16)
        else:
            assert np.abs(v1.mean(0)).max() > 1e-3


def test_free_bead_shares_momentum_with_periodic_fluid(orc):
    # a bead with V0 in a periodic fluid at rest ends at the common velocity
    # m V0 / (m + rho E^3).  The explicit coupling also excites a slowly
    # damped period-2 oscillation of the bead velocity (alternating sign from
    # step to step), so the check averages two consecutive steps.
    E = 8
    box = orc.BoxParams(E=E, tau=1.0, periodic=(True, True, True))
    V0 = np.array([[0.05, -0.02, 0.01]])
    ch = orc.ChainParams(nbeads=1, pin_com=0, n_md=10)
    sim = orc.Sim(box, np.zeros((3, E, E, E)), np.zeros((2, 6, 3, E, E)), ch, np.array([[3.3, 3.6, 4.1]]), V0)
    assert sim.run(1500) == 0
    v_a = sim.vel[0].copy()
    u_a = sim.fields()[1].reshape(3, -1).mean(1)
    assert sim.run(1) == 0
    v_b = sim.vel[0].copy()
    u_b = sim.fields()[1].reshape(3, -1).mean(1)
    final = ch.mass * V0[0] / (ch.mass + E ** 3)
    assert np.allclose(0.5 * (v_a + v_b), final, rtol=1e-3, atol=1e-9)
    assert np.allclose(0.5 * (u_a + u_b), final, rtol=1e-3)


def test_stokes_drag_on_single_bead(orc):
    # constant force f on one bead, the opposite force spread uniformly over the
    # fluid so the box as a whole does not accelerate.  The bead drifts at
    # V = mobility * f with mobility 1/zeta + 1/(g rho nu a) (Ahlrichs-Duenweg,
    # g ~ 25 for trilinear coupling) minus the periodic-image correction
    # 2.837 / (6 pi rho nu E) (Hasimoto).  Loose pin: 10 %.
    E, tau = 16, 1.0
    nu = (tau - 0.5) / 3
    f = 1e-4
    box = orc.BoxParams(E=E, tau=tau, periodic=(True, True, True), accel=(-f / E ** 3, 0, 0))
    ch = orc.ChainParams(nbeads=1, zeta=1.0, pin_com=0, n_md=10, f_ext=(f, 0, 0))
    sim = orc.Sim(box, np.zeros((3, E, E, E)), np.zeros((2, 6, 3, E, E)), ch, np.array([[7.5, 7.5, 7.5]]))
    assert sim.run(600) == 0
    mob = sim.vel[0, 0] / f
    expect = 1.0 / ch.zeta + 1.0 / (25.0 * nu) - 2.837 / (6 * np.pi * nu * E)
    assert abs(mob / expect - 1) < 0.10, (mob, expect)


def test_noise_statistics(orc):
    # unit-variance uniform numbers from Philox words: mean 0, variance 1
    n = 20000
    xs = []
    for i in range(n // 4):
        r = orc.philox4x32_10([i, 3, 1, 0], [99, 0])
        xs.extend(np.sqrt(3.0) * (2.0 * (r.astype(np.float64) / 2.0 ** 32) - 1.0))
    xs = np.array(xs)
    assert abs(xs.mean()) < 3 / np.sqrt(n)
    assert abs(xs.var() - 1) < 3 * np.sqrt(0.8 / n)


def test_fene_overstretch_is_reported(orc):
    E = 16
    box = orc.BoxParams(E=E, tau=0.8)
    A = _uniform_state(orc, E, np.zeros(3))
    pos = np.array([[7.0, 7.0, 7.0], [8.45, 7.0, 7.0]])
    vel = np.array([[-5.0, 0, 0], [5.0, 0, 0]])  # jumps past R0 within one substep
    ch = orc.ChainParams(nbeads=2, pin_com=0, k_fene=0.1)
    st, *_ = orc.chain_couple(box, ch, A, 0, pos, vel)
    assert st == orc.ERR_FENE
