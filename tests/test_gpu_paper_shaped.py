"""The paper-shaped replay (Secs. 2-4): a box of 128 sites per axis (the
paper's 121, rounded to the kernels' 8-site alignment) zoomed z = 6 from a
coarse face grid, tau = 1, one coarse sample every 113 LB steps (0.05 tau_eta
mapped by Eq. 1), the flow in the tracer's co-moving frame (w = u - v(t) on
the boundary and in the initial field) with the frame force rho (-dv/dt) from
the tracer's acceleration, and a chain at the centre.  GPU (FP32) and oracle
(FP64) both run 151 steps, across a coarse-interval boundary, from the same
inputs drawn by the oracle's generator, and are compared site by site."""
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
    faces = oracle.face_samples(modes, E, K, 0, J, zoom=z)
    v = inputs.tracer_velocity(modes, np.arange(J) * K)
    faces = faces - v[:, None, :, None, None]  # co-moving frame
    u0 = oracle.volume_field(modes, E, 0.0, zoom=z) - v[0][:, None, None, None]
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
    while tr.lb_current_step() < n0 + 1:
        j = tr.lb_current_step() // K
        while pushed < j + 1:
            pushed += 1
            tr.lb_set_boundary(0, pushed, dev_faces[pushed])
            tr.lb_set_frame_accel(0, pushed, fsamp[pushed])
        tr.lb_step(1)
    B = tr.deviations(0).astype(np.float64)
    u = tr.fields(0)[1]
    pos1, vel1 = tr.chain(0, nb)
    box = oracle.BoxParams(E=E, tau=1.0, K=K, zoom=z)
    chain = oracle.ChainParams(nbeads=nb, kT=1e-4, seed=5)
    st, Aref, pref, vref = oracle.run_frame(box, oracle.init(box, u0), faces, fsamp, 0, n0 + 1, chain, pos0,
                                            np.zeros_like(pos0))
    assert st == 0
    _, w = oracle.lattice()
    dref = Aref - w[:, None, None, None]
    # reported velocity of the oracle state at step n0 + 1 (its body acceleration is the frame's at t_{n0+1})
    box_n = oracle.BoxParams(E=E, tau=1.0, K=K, zoom=z, accel=tuple(oracle.frame_accel_at((0.0, 0.0, 0.0), fsamp, K,
                                                                                            n0 + 1)))
    u_ref = oracle.fields(box_n, Aref)[1]
    e_u = float(np.sqrt(((u - u_ref)[:, 1:-1, 1:-1, 1:-1] ** 2).sum() / (u_ref[:, 1:-1, 1:-1, 1:-1] ** 2).sum()))
    print("paper-shaped: K %d, eta~ %.2f sites, tau~_eta %.0f steps, Ma %.4f, max |a| %.2e, after %d steps: "
          "max |B - ref| %.2e, velocity rel L2 %.2e, beads %.2e / %.2e"
          % (K, um.eta_lb, um.tau_eta_lb, um.mach, np.abs(fsamp).max(), n0 + 1, np.abs(B - dref).max(), e_u,
             np.abs(pos1 - pref).max(), np.abs(vel1 - vref).max()))
    assert np.abs(B - dref).max() < 5e-6
    assert e_u <= 1e-5
    assert np.abs(pos1 - pref).max() < 1e-3 and np.abs(vel1 - vref).max() < 1e-2
    tr.close()
