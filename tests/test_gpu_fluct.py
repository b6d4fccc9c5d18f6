"""Fluctuating collision on the GPU (lb_set_fluctuation) against the
fluctuating-LB oracle (oracle/fluct.py), through the C ABI.

The GPU's pull step is collide(stream(f)); the oracle runs the same order
from its own initial state (oracle.init of the same seeded velocity field),
with the same Philox counters (step, site, block, 0xF1), so with FP64 storage
every site agrees to rounding -- a single noise word that differed would show
as an error of the size of the noise itself.  Then the physics: mass and
momentum conserved with noise, and equipartition <u_a^2> = kT / rho.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_4958_gb300 import lbtracer
    lbtracer.load()
    return lbtracer


@pytest.fixture(scope="module")
def fl():
    oracle.build()
    from oracle import fluct
    return fluct


def smooth_u0(E, amp=0.02):
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    k = 2 * np.pi / E
    return np.stack([amp * np.sin(k * Y), amp * np.cos(k * Z + 0.3), amp * 0.5 * np.sin(k * X + 1.0)])


def periodic_box(lbt, E, tau, storage, u0):
    tr = lbt.Tracers([lbt.box_desc(E, tau, periodic=(True, True, True))], storage)
    real = np.float64 if storage == lbt.LB_STORE_F64 else np.float32
    tr.lb_init(0, np.ascontiguousarray(u0, real))
    tr.lb_sync()
    return tr


def gammas(tau, bulk=None, odd=None, even=None):
    g = np.full(19, 1.0 - 1.0 / tau)
    if bulk is not None:
        g[4] = bulk
    if odd is not None:
        g[10:16] = odd
    if even is not None:
        g[16:19] = even
    return g


def run_oracle(fl, A, E, gamma, kT, seed, nsteps):
    f = A.reshape(19, -1)
    for n in range(nsteps):
        f = fl.collide(fl.stream_periodic(f, E), gamma, kT, n, seed)
    return f


@pytest.mark.parametrize("case", ["bgk_limit", "thermal"])
def test_fp64_steps_match_the_oracle_sitewise(lbt, fl, case):
    E, tau, seed = 16, 0.8, 0x1234ABCD5678
    u0 = smooth_u0(E)
    if case == "bgk_limit":
        g, kT = gammas(tau), 0.0
    else:  # every mode class relaxed differently, strong noise so a wrong word shows
        g, kT = gammas(tau, bulk=0.2, odd=-0.3, even=0.1), 1e-2
    tr = periodic_box(lbt, E, tau, lbt.LB_STORE_F64, u0)
    tr.lb_set_fluctuation(0, kT, seed, g)
    _, w = oracle.lattice()
    A0 = oracle.init(oracle.BoxParams(E=E, tau=tau, periodic=(True, True, True)), u0)
    for nsteps in (1, 3):
        if nsteps == 3:
            tr.lb_step(2)
        else:
            tr.lb_step(1)
        d = tr.deviations(0).reshape(19, -1)
        ref = run_oracle(fl, A0, E, g, kT, seed, nsteps) - w[:, None]
        err = np.abs(d - ref).max()
        print("%s, %d steps: max |GPU - oracle| %.2e (deviations up to %.2e)" % (case, nsteps, err, np.abs(ref).max()))
        assert err < 1e-13
    if case == "bgk_limit":  # and the same as the plain BGK kernel
        plain = periodic_box(lbt, E, tau, lbt.LB_STORE_F64, u0)
        plain.lb_step(3)
        assert np.abs(plain.deviations(0).reshape(19, -1) - d).max() < 1e-15


def test_fp32_thermal_steps_match_the_oracle(lbt, fl):
    # FP32 noise takes the top 24 bits of each Philox word: relative 2^-24 of the noise
    E, tau, seed, kT = 16, 0.8, 77, 1e-4
    u0 = smooth_u0(E)
    g = gammas(tau, bulk=0.2, odd=0.0, even=0.0)
    tr = periodic_box(lbt, E, tau, lbt.LB_STORE_F32, u0)
    tr.lb_set_fluctuation(0, kT, seed, g)
    tr.lb_step(4)
    _, w = oracle.lattice()
    A0 = oracle.init(oracle.BoxParams(E=E, tau=tau, periodic=(True, True, True)), u0)
    ref = run_oracle(fl, A0, E, g, kT, seed, 4) - w[:, None]
    err = np.abs(tr.deviations(0).reshape(19, -1) - ref).max()
    print("FP32, 4 steps: max |GPU - oracle| %.2e" % err)
    assert err < 2e-6


def test_noise_conserves_mass_and_momentum(lbt):
    E, tau = 16, 0.8
    tr = periodic_box(lbt, E, tau, lbt.LB_STORE_F64, smooth_u0(E))
    tr.lb_set_fluctuation(0, 1e-3, 5, gammas(tau, bulk=0.0, odd=0.0, even=0.0))
    c0 = tr.lb_conservation(0)
    tr.lb_step(50)
    c1 = tr.lb_conservation(0)
    assert abs(c1[0] - c0[0]) <= 1e-12 * c0[0]
    assert np.abs(c1[1:4] - c0[1:4]).max() <= 1e-12 * c0[0]
    assert np.abs(tr.deviations(0) - periodic_box(lbt, E, tau, lbt.LB_STORE_F64, smooth_u0(E)).deviations(0)).max() > 0


def test_equipartition_of_the_velocity(lbt):
    # periodic box at rest, every non-conserved mode fully thermalised each
    # step (gamma 0): <u_a^2> = kT / rho per component, less the conserved
    # total momentum's share 1/E^3
    E, kT = 16, 1e-5
    tr = periodic_box(lbt, E, 1.0, lbt.LB_STORE_F32, np.zeros((3, E, E, E)))
    tr.lb_set_fluctuation(0, kT, 11, np.zeros(19))
    u = torch.empty((3, E, E, E), dtype=torch.float32, device="cuda")
    acc = []
    for n in range(1000):
        tr.lb_step(1)
        if n >= 100:
            tr.lb_read_fields(0, lbt.LB_FIELD_U, u)
            acc.append(float((u.double() ** 2).mean()))
    ref = kT * (1.0 - 1.0 / E ** 3)
    print("<u_a^2> = %.4e, kT / rho = %.4e" % (np.mean(acc), ref))
    assert np.mean(acc) == pytest.approx(ref, rel=0.03)


def test_refused_where_the_collision_cannot_run(lbt):
    tr = lbt.Tracers([lbt.box_desc(16, 0.8, nbeads=4)], lbt.LB_STORE_F32)
    with pytest.raises(lbt.LBError) as ei:
        tr.lb_set_fluctuation(0, 1e-4, 1, gammas(0.8))  # a box with chain capacity
    assert ei.value.code == lbt.LB_ERR_ARG
    tr2 = lbt.Tracers([lbt.box_desc(16, 0.8, periodic=(True, True, True))], lbt.LB_STORE_F32)
    with pytest.raises(lbt.LBError) as ei:
        tr2.lb_set_fluctuation(0, 1e-4, 1, np.full(19, 1.0))  # gamma must lie in (-1, 1)
    assert ei.value.code == lbt.LB_ERR_ARG
    tr2.lb_set_fluctuation(0, 1e-4, 1, gammas(0.8))
    with pytest.raises(lbt.LBError) as ei:
        tr2.lb_set_launch(lbt.LB_KERNEL_REGISTER, 128, 0, 0)
    assert ei.value.code == lbt.LB_ERR_STATE
    tr2.lb_set_fluctuation(0, 0.0, 0, None)  # back to BGK: the register kernel is allowed again
    tr2.lb_set_launch(lbt.LB_KERNEL_REGISTER, 128, 0, 0)
