"""Co-moving-frame body force through the C ABI (Sec. 2: the tracer frame adds
the force density rho (-dv/dt), given as time samples and interpolated
linearly in time): GPU against the oracle, step by step."""
import numpy as np
import pytest

import oracle
from gpucases import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ST64, ST32 = 0, 1


@pytest.fixture(scope="module")
def lbt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_4958_gb300 import lbtracer
    lbtracer.load()
    return lbtracer


def _drive(lbt, tr, c, fsamp, nsteps, dev_samples):
    """Steps with the face and frame-acceleration samples pushed as needed."""
    pushed_f = pushed_a = -1
    for n in range(nsteps):
        j = n // c.K
        if not all(c.periodic):
            while pushed_f < j + 1:
                pushed_f += 1
                tr.lb_set_boundary(0, pushed_f, dev_samples[pushed_f])
        while pushed_a < j + 1:
            pushed_a += 1
            tr.lb_set_frame_accel(0, pushed_a, fsamp[pushed_a])
        tr.lb_step(1)


def test_periodic_box_integrates_the_frame_force(lbt):
    E, K, N = 16, 3, 14
    rng = np.random.default_rng(5)
    fsamp = rng.normal(size=(N // K + 3, 3)) * 2e-5
    u0 = np.array([0.01, -0.015, 0.004])
    tr = lbt.Tracers([lbt.box_desc(E, 0.7, periodic=(True, True, True), K=K, frame_accel=True)], ST64)
    tr.lb_init(0, np.broadcast_to(u0[:, None, None, None], (3, E, E, E)).copy())
    c = Case.__new__(Case)
    c.K, c.periodic = K, (True, True, True)
    _drive(lbt, tr, c, fsamp, N, None)
    u = np.zeros((3, E, E, E))
    tr.lb_read_fields(0, lbt.LB_FIELD_U, u)
    aN = oracle.frame_accel_at((0, 0, 0), fsamp, K, N)
    ref = u0 + sum(oracle.frame_accel_at((0, 0, 0), fsamp, K, m) for m in range(N)) + 0.5 * aN
    for a in range(3):
        assert np.abs(u[a] - ref[a]).max() < 1e-14
    tr.close()


@pytest.mark.parametrize("storage,kernel", [(ST64, "staged"), (ST64, "register"), (ST32, "staged")])
def test_frame_force_with_boundaries_and_chain_matches_oracle(lbt, storage, kernel):
    # velocity faces, a noisy chain and a time-dependent frame acceleration
    # (K = 2, samples interpolated at every step): populations and beads
    # against the oracle stepped with the same per-step acceleration
    c = Case(16, 0.8, 6, seed=4, M=16, nbeads=6, K=2)
    c.kT = 1e-4
    N = 6
    rng = np.random.default_rng(9)
    fsamp = rng.normal(size=(N // c.K + 3, 3)) * 3e-5
    d = c.gpu_desc(lbt)
    d.frame_accel = 1
    tr = lbt.Tracers([d], storage)
    if kernel == "register":
        tr.lb_set_launch(lbt.LB_KERNEL_REGISTER, 256, 0, 0)
    real = torch.float64 if storage == ST64 else torch.float32
    dev_samples = torch.from_numpy(c.samples).to("cuda", real)
    torch.cuda.synchronize()
    tr.lb_init(0, torch.from_numpy(c.u0).to("cuda", real).contiguous())
    tr.chain_couple(0, c.gpu_chain(lbt), np.ascontiguousarray(c.pos0), None)
    tr.lb_sync()
    _, w = oracle.lattice()
    A0 = oracle.init(c.oracle_box(), c.u0)
    _drive(lbt, tr, c, fsamp, N, dev_samples)
    B = tr.deviations(0).astype(np.float64)
    pos, vel = tr.chain(0, c.nbeads)
    st, Aref, pref, vref = oracle.run_frame(c.oracle_box(), A0, c.samples, fsamp, 0, N, c.oracle_chain(),
                                            c.pos0, np.zeros_like(c.pos0))
    assert st == 0
    dref = Aref - w[:, None, None, None]
    if storage == ST64:
        assert np.abs(B - dref).max() < 1e-13
        assert np.abs(pos - pref).max() < 1e-11 and np.abs(vel - vref).max() < 1e-10
    else:
        assert np.abs(B - dref).max() < 5e-5  # FP32 chain dynamics (see the 128^3 sampled-step test)
        assert np.abs(pos - pref).max() < 1e-5 and np.abs(vel - vref).max() < 3e-4
    tr.close()
