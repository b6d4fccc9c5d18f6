"""The paper-shaped replay (Secs. 2-4): a box of 128 sites per axis (the
paper's 121, rounded to the kernels' 8-site alignment) zoomed z = 6 from a
coarse face grid, tau = 1, one coarse sample every 113 LB steps (0.05 tau_eta
mapped by Eq. 1), the flow in the tracer's co-moving frame (w = u - v(t) on
the boundary and in the initial field) with the frame force rho (-dv/dt) from
the tracer's acceleration, and a chain at the centre.  After stepping across
a coarse-interval boundary, one GPU step is compared site by site with one
oracle step from the same state."""
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


def test_paper_shaped_replay_step(lbt):
    from paper_0809_4958_gb300 import inputs, scaling
    eta, tau_eta = scaling.kolmogorov(1.0 / 400.0, 0.1)
    um = scaling.UnitMap(eta=eta, tau_eta=tau_eta, delta=2 * np.pi / 1024, z=6, tau=1.0)
    K = int(round(um.steps(0.05 * tau_eta)))  # 113
    E, z, nb = 128, 6, 16
    Ec = oracle.coarse_points(E, z)
    u_eta = um.eta_lb / um.tau_eta_lb  # Kolmogorov velocity in lattice units
    modes = inputs.mode_table(21, 256, 1.0, 10.0, E, u_max=3 * u_eta)
    n0 = 150
    J = n0 // K + 3
    faces = lbt.synth_faces(modes, E, K, 0, J, torch.float64, zoom=z).cpu().numpy()
    v = inputs.tracer_velocity(modes, np.arange(J) * K)
    faces = faces - v[:, None, :, None, None]  # co-moving frame
    u0 = lbt.synth_volume(modes, E, 0.0, torch.float64, zoom=z).cpu().numpy() - v[0][:, None, None, None]
    fsamp = inputs.tracer_frame_accel(modes, np.arange(J) * K)
    d = lbt.box_desc(E, 1.0, K=K, nbeads=nb, zoom=z, frame_accel=True)
    tr = lbt.Tracers([d], lbt.LB_STORE_F32)
    dev_faces = torch.from_numpy(faces).to("cuda", torch.float32)
    torch.cuda.synchronize()
    tr.lb_init(0, torch.from_numpy(u0).to("cuda", torch.float32).contiguous())
    pos0 = inputs.chain_start(3, nb, E)
    ch = lbt.chain_desc(nb, kT=1e-4, seed=5)
    tr.chain_couple(0, ch, pos0, None)
    pushed = -1

    def step_to(n1):
        nonlocal pushed
        while tr.lb_current_step() < n1:
            j = tr.lb_current_step() // K
            while pushed < j + 1:
                pushed += 1
                tr.lb_set_boundary(0, pushed, dev_faces[pushed])
                tr.lb_set_frame_accel(0, pushed, fsamp[pushed])
            tr.lb_step(1)

    step_to(n0)
    _, w = oracle.lattice()
    A = tr.deviations(0).astype(np.float64) + w[:, None, None, None]
    pos, vel = tr.chain(0, nb)
    step_to(n0 + 1)
    B = tr.deviations(0).astype(np.float64)
    pos1, vel1 = tr.chain(0, nb)
    a_n = oracle.frame_accel_at((0.0, 0.0, 0.0), fsamp, K, n0)
    box = oracle.BoxParams(E=E, tau=1.0, K=K, zoom=z, accel=tuple(a_n))
    chain = oracle.ChainParams(nbeads=nb, kT=1e-4, seed=5)
    st, Bref, pref, vref, _ = oracle.step_from(box, A, faces, n0, chain, pos, vel)
    assert st == 0
    dref = Bref - w[:, None, None, None]
    print("paper-shaped: K %d, eta~ %.2f sites, tau~_eta %.0f steps, Ma %.4f, max |a| %.2e, max |B - ref| %.2e"
          % (K, um.eta_lb, um.tau_eta_lb, um.mach, np.abs(fsamp).max(), np.abs(B - dref).max()))
    assert np.abs(B - dref).max() < 2e-7
    assert np.abs(pos1 - pref).max() < 1e-5 and np.abs(vel1 - vref).max() < 3e-4
    tr.close()
