"""GPU path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from gpucases import Case, GpuRunner, interior, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_4958_gb300 import lbtracer
    lbtracer.load()
    return lbtracer


ST64, ST32 = 0, 1


def gpu_run(lbt, case, storage, nsteps=None):
    r = GpuRunner(lbt, torch, [case], storage)
    r.step(case.nsteps if nsteps is None else nsteps)
    return r


def test_generator_matches_oracle(lbt):
    from paper_0809_4958_gb300 import inputs
    for E, M, kmax in [(16, 64, 8), (24, 256, 12)]:
        modes = inputs.mode_table(3, M, 1, kmax, E)
        ref = oracle.face_samples(modes, E, 5, 2, 3)
        got = lbt.synth_faces(modes, E, 5, 2, 3, torch.float64).cpu().numpy()
        assert np.abs(got - ref).max() < 1e-14
        got32 = lbt.synth_faces(modes, E, 5, 2, 3, torch.float32).cpu().numpy()
        assert np.abs(got32 - ref).max() < 1e-8
        vref = oracle.volume_field(modes, E, 7.0)
        vgot = lbt.synth_volume(modes, E, 7.0, torch.float64).cpu().numpy()
        assert np.abs(vgot - vref).max() < 1e-14


def test_single_step_f64_matches_oracle_sitewise(lbt):
    c = Case(16, 0.8, 1, nbeads=6, M=32)
    r = gpu_run(lbt, c, ST64)
    _, w = oracle.lattice()
    sim = c.run_oracle()
    d = r.tr.deviations(0)
    assert np.abs(d - (sim.f - w[:, None, None, None])).max() < 1e-15
    pos, vel = r.tr.chain(0, c.nbeads)
    # the MD sums each bead's substep displacements before adding them to the
    # FP64 position, so positions and velocities agree to FP64 rounding of the
    # 50 substeps, not bitwise
    assert np.abs(pos - sim.pos).max() < 1e-12 and np.abs(vel - sim.vel).max() < 1e-11


@pytest.fixture(scope="module")
def cfg0():
    # plain method, one 32^3 box, tau 0.8, 256 modes with |k| in [1, 16],
    # one 16-bead FENE chain (k 30, R0 1.5, zeta 1, kT 0), 1000 steps
    c = Case(32, 0.8, 1000, seed=0, M=256, k_max=16, nbeads=16)
    sim = c.run_oracle()
    return c, sim


@pytest.mark.parametrize("storage,tol", [(ST64, 1e-12), (ST32, 1e-5)])
def test_cfg0_1000_steps(lbt, cfg0, storage, tol):
    c, sim = cfg0
    r = gpu_run(lbt, c, storage)
    rho, u = r.tr.fields(0)
    _, u_ref = sim.fields()
    err = rel_l2(interior(u), interior(u_ref))
    assert err <= tol, err
    pos, _ = r.tr.chain(0, c.nbeads)
    assert np.abs(pos - sim.pos).max() < (1e-10 if storage == ST64 else 1e-4)


@pytest.mark.parametrize("storage,tol", [(ST64, 1e-12), (ST32, 1e-5)])
@pytest.mark.parametrize("shape", ["E8", "E24", "xper", "allper_accel", "yz_per", "hermite"])
def test_edge_shapes(lbt, storage, tol, shape):
    kw = dict(E8=dict(E=8, tau=0.6, nsteps=60, M=16),
              E24=dict(E=24, tau=0.8, nsteps=80, M=64, nbeads=20),
              xper=dict(E=16, tau=0.7, nsteps=80, M=32, periodic=(True, False, False), nbeads=8),
              allper_accel=dict(E=16, tau=0.9, nsteps=80, M=32, periodic=(True, True, True), accel=(1e-5, -2e-5, 5e-6),
                                nbeads=8, pin_com=0, kT=1e-4),
              yz_per=dict(E=24, tau=1.2, nsteps=60, M=32, periodic=(False, True, True), accel=(0, 1e-5, 0)),
              hermite=dict(E=16, tau=0.8, nsteps=64, M=32, K=4, time_interp=1, nbeads=4))[shape]
    c = Case(**kw)
    sim = c.run_oracle()
    r = gpu_run(lbt, c, storage)
    rho, u = r.tr.fields(0)
    rho_ref, u_ref = sim.fields()
    # periodic boxes lose most of their velocity to viscosity within the run,
    # while FP32 rounding acts on O(1) populations: the error is measured
    # against the norm of the initial field on the same sites
    d = interior(u, c.periodic).astype(np.float64) - interior(u_ref, c.periodic)
    norm = max(np.sqrt((interior(u_ref, c.periodic) ** 2).sum()), np.sqrt((interior(c.u0, c.periodic) ** 2).sum()))
    assert np.sqrt((d ** 2).sum()) / norm <= tol
    assert np.abs(rho - rho_ref).max() <= (1e-13 if storage == ST64 else 1e-6)
    # boundary layer: equilibrium of the interpolated boundary velocity
    assert np.abs(u - u_ref).max() <= (1e-13 if storage == ST64 else 1e-6)


def test_periodic_conservation_f64(lbt):
    c = Case(16, 0.8, 400, M=32, periodic=(True, True, True), nbeads=10, kT=1e-4, pin_com=0,
             vel0=np.full((10, 3), 0.01))
    r = GpuRunner(lbt, torch, [c], ST64)
    c0 = r.tr.lb_conservation(0)
    r.step(400)
    c1 = r.tr.lb_conservation(0)
    mass = 16 ** 3
    assert abs(c1[0] - c0[0]) <= 1e-12 * mass
    assert np.abs((c1[1:4] + c1[4:7]) - (c0[1:4] + c0[4:7])).max() <= 1e-12 * mass * 0.05
    assert np.abs(c1[4:7] - c0[4:7]).max() > 1e-5  # momentum really moved between beads and fluid
    sim = c.run_oracle()
    ref = sim.conservation()
    # the oracle adds the 19 * 16^3 populations one by one in FP64: its mass sum
    # carries a rounding error of order sqrt(n) eps mass ~ 1e-10 (absolute);
    # the GPU sums deviations in a tree
    assert abs(c1[0] - ref[0]) <= 1e-13 * mass
    assert np.abs(c1[1:] - ref[1:]).max() <= 1e-10


@pytest.mark.parametrize("storage", [ST64, ST32])
def test_bead_lanes_agree(lbt, storage):
    # the lanes of a bead only split its pair forces: every choice gives the
    # same chain up to the order of the force sums
    c = Case(24, 0.8, 20, M=32, nbeads=40, kT=1e-4)
    runs = []
    for lanes, bpt in ((1, 1), (1, 2), (2, 1), (4, 1), (8, 1), (2, 0)):
        r = GpuRunner(lbt, torch, [c], storage)
        r.tr.lb_set_bead_launch(lanes, bpt)
        r.step(20)
        runs.append((r.tr.chain(0, c.nbeads), r.tr.deviations(0)))
    (p0, v0), d0 = runs[0]
    # FP32: the substep displacements round at 2^-24 of positions ~E/2 and the
    # differences of summation order grow over 20 steps of 50 substeps
    tol_p, tol_d = (1e-12, 1e-14) if storage == ST64 else (1e-4, 1e-6)
    for (p, v), d in runs[1:]:
        assert np.abs(p - p0).max() <= tol_p and np.abs(d - d0).max() <= tol_d


@pytest.mark.parametrize("ctas", [0, 7])
def test_batch_with_many_tiles_per_block_equals_single_boxes(lbt, ctas):
    # four 64^3 Hermite boxes (K = 16): every persistent block takes tiles of
    # several boxes in turn, so a tile header must stay valid while the next
    # tile of another box is already being staged
    cases = [Case(64, 0.8, 40, seed=s, M=64, K=16, time_interp=1) for s in range(4)]
    rb = GpuRunner(lbt, torch, cases, ST32)
    rb.tr.lb_set_launch(lbt.LB_KERNEL_STAGED, 0, ctas, 0)
    rb.step(40)
    for b in (0, 3):
        r1 = GpuRunner(lbt, torch, [cases[b]], ST32)
        r1.step(40)
        assert np.array_equal(rb.tr.deviations(b), r1.tr.deviations(0)), b
    u = rb.tr.fields(0)[1]
    u_ref = cases[0].run_oracle().fields()[1]
    assert rel_l2(interior(u), interior(u_ref)) <= 1e-5


def test_batch_of_uneven_boxes_equals_single_boxes(lbt):
    cases = [Case(24, 0.8, 30, seed=1, M=32, nbeads=12), Case(16, 0.7, 30, seed=2, M=16),
             Case(32, 0.9, 30, seed=3, M=32, nbeads=20)]
    rb = GpuRunner(lbt, torch, cases, ST32)
    rb.step(30)
    for b, c in enumerate(cases):
        rs = GpuRunner(lbt, torch, [c], ST32)
        rs.step(30)
        assert np.array_equal(rb.tr.deviations(b), rs.tr.deviations(0))
        if c.nbeads:  # noise-free chains: the noise counter would carry the box index
            assert np.array_equal(rb.tr.chain(b, c.nbeads)[0], rs.tr.chain(0, c.nbeads)[0])


def test_graph_replay_equals_steps(lbt):
    c = Case(24, 0.8, 40, M=32, nbeads=8, periodic=(True, True, True))
    ra = GpuRunner(lbt, torch, [c], ST32)
    ra.step(40)
    rg = GpuRunner(lbt, torch, [c], ST32)
    rg.tr.lb_graph_capture(10)
    for _ in range(4):
        rg.tr.lb_graph_launch()
    assert rg.tr.lb_current_step() == 40
    assert np.array_equal(ra.tr.deviations(0), rg.tr.deviations(0))
    assert np.array_equal(ra.tr.chain(0, 8)[0], rg.tr.chain(0, 8)[0])


@pytest.fixture(scope="module")
def fullsize_128_inputs():
    # 128^3 box, 1024 modes with |k| in [1, 64]: boundary samples and initial
    # field from the oracle's own generator (nothing the oracle sees comes
    # from the GPU)
    from paper_0809_4958_gb300 import inputs
    E = 128
    modes = inputs.mode_table(11, 1024, 1.0, 64.0, E)
    return modes, oracle.face_samples(modes, E, 1, 0, 14), oracle.volume_field(modes, E, 0.0)


@pytest.mark.parametrize("tau", [0.55, 0.8])
def test_fullsize_128_against_oracle(lbt, fullsize_128_inputs, tau):
    # the default workload's shape: 128^3 FP32 box, 64-bead chain with noise
    # at kT 1e-4; GPU and oracle both run 11 steps from the same inputs, and
    # the GPU's sampled step 10 -> 11 is also compared with the oracle's
    from paper_0809_4958_gb300 import inputs
    modes, samples, u0 = fullsize_128_inputs
    E, nsteps = 128, 11
    c = Case.__new__(Case)
    c.E, c.tau, c.K, c.time_interp, c.periodic, c.accel = E, tau, 1, 0, (False, False, False), (0.0, 0.0, 0.0)
    c.zoom = 1
    c.nsteps, c.nbeads, c.kT, c.n_md, c.pin_com, c.chain_seed, c.vel0 = nsteps, 64, 1e-4, 50, 2, 9, None
    c.modes, c.samples, c.u0 = modes, samples, u0
    c.J = samples.shape[0]
    c.pos0 = inputs.chain_start(5, 64, E)
    r = GpuRunner(lbt, torch, [c], ST32)
    r.step(nsteps)
    d = r.tr.deviations(0).astype(np.float64)
    u = r.tr.fields(0)[1]
    pos, vel = r.tr.chain(0, 64)
    sim = c.run_oracle()
    _, w = oracle.lattice()
    dref = sim.f - w[:, None, None, None]
    e_u = rel_l2(interior(u), interior(sim.fields()[1]))
    e_d = np.abs(d - dref).max()
    e_p, e_v = np.abs(pos - sim.pos).max(), np.abs(vel - sim.vel).max()
    print("128^3 tau %.2f after %d steps: velocity rel L2 %.2e, max |d - ref| %.2e, beads %.2e / %.2e"
          % (tau, nsteps, e_u, e_d, e_p, e_v))
    # FP32 rounding of O(1) quantities (rho, w_i rho) over 11 steps is a few
    # 1e-7 absolute on the deviations; at the forced sites the FP32 chain MD
    # hands the fluid a force that differs from the FP64 one (bead velocities
    # differ by ~1e-4, see below), which at tau 0.55 (over-relaxed, slowly
    # damped) leaves up to ~1e-5 there.  Velocity: the spec FP32 bound.
    assert e_d < 2e-5
    assert e_u <= 1e-5
    # the FP32 chain MD (50 stiff substeps per step, forces up to ~50 rounded
    # to 2^-24 with a 2-ulp fast reciprocal) differs from the FP64 oracle by
    # ~1e-6 in position and ~1e-4 in velocity per step; friction and the
    # centre-of-mass pin keep it from growing fast over 11 steps
    assert e_p < 1e-4 and e_v < 3e-3


def test_chain_recoupled_at_an_odd_step(lbt):
    # A chain re-coupled at step 3 (odd) at new positions: the bead kernel of
    # that step must gather, move and spread from the new positions, and the
    # forced re-collision must rewrite exactly the new stencil sites.  GPU and
    # oracle both run 3 steps, re-place the chain and run one more.
    c = Case(16, 0.8, 6, seed=3, M=16, nbeads=6)
    r = GpuRunner(lbt, torch, [c], ST64)
    r.step(3)
    pos_new = np.ascontiguousarray(c.pos0 + np.array([1.3, 0.4, -0.7]))
    r.tr.chain_couple(0, c.gpu_chain(lbt), pos_new, None)
    r.step(1)
    B = r.tr.deviations(0).astype(np.float64)
    pos1, vel1 = r.tr.chain(0, 6)
    sim = oracle.Sim(c.oracle_box(), c.u0, c.samples, c.oracle_chain(), c.pos0)
    assert sim.run(3) == 0
    sim.pos = pos_new.copy()
    sim.vel = np.zeros_like(pos_new)
    assert sim.run(1) == 0
    _, w = oracle.lattice()
    assert np.abs(B - (sim.f - w[:, None, None, None])).max() < 1e-13
    assert np.abs(pos1 - sim.pos).max() < 1e-11 and np.abs(vel1 - sim.vel).max() < 1e-10


def test_error_flags_freeze_only_the_failing_box(lbt):
    good = Case(16, 0.8, 5, seed=1, M=16, nbeads=6)
    bad = Case(16, 0.8, 5, seed=2, M=16, nbeads=6)
    bad.vel0 = np.zeros((6, 3))
    bad.vel0[0] = [-40.0, 0, 0]
    bad.vel0[1] = [40.0, 0, 0]
    r = GpuRunner(lbt, torch, [good, bad], ST64)
    r.step(3)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_sync()
    assert ei.value.code == lbt.LB_ERR_FENE
    assert r.tr.lb_status(0) == 0 and r.tr.lb_status(1) == lbt.LB_ERR_FENE
    d1 = np.zeros((19, 16, 16, 16))
    r.tr.lb_read_fields(0, lbt.LB_FIELD_DEV, d1)
    r.step(2)
    d2 = np.zeros_like(d1)
    r.tr.lb_read_fields(0, lbt.LB_FIELD_DEV, d2)
    assert not np.array_equal(d1, d2)  # the healthy box keeps stepping
    b1 = np.zeros_like(d1)
    with pytest.raises(lbt.LBError):
        r.tr.lb_read_fields(1, lbt.LB_FIELD_DEV, b1)


def test_bead_stencil_leaving_interior_is_flagged(lbt):
    c = Case(16, 0.8, 2, M=16, nbeads=2, pin_com=0)
    # the beads drift about 0.76 sites towards x = 0 in the first step, so the
    # stencil of the first (from x = 0.44) leaves the interior at the second;
    # the drift is gentle enough that the fluid they push stays finite (a
    # harder push can make the stream-collide flag LB_ERR_NONFINITE first:
    # the first error of a step wins)
    c.pos0 = np.array([[1.2, 7.0, 7.0], [2.17, 7.0, 7.0]])
    c.vel0 = np.array([[-1.2, 0, 0], [-1.2, 0, 0]])
    r = GpuRunner(lbt, torch, [c], ST32)
    r.step(2)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_sync()
    assert ei.value.code == lbt.LB_ERR_BEAD_OOB


def test_missing_boundary_sample_is_refused(lbt):
    c = Case(16, 0.8, 2, M=16)
    r = GpuRunner(lbt, torch, [c], ST32)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_step(1)  # nothing pushed yet
    assert ei.value.code == lbt.LB_ERR_STATE
    r.tr.lb_set_boundary(0, 0, r.dev_samples[0][0])
    with pytest.raises(lbt.LBError):
        r.tr.lb_set_boundary(0, 2, r.dev_samples[0][2])  # out of order


@pytest.mark.parametrize("storage", [ST64, ST32, 2, 3])
@pytest.mark.parametrize("periodic", [(True, False, False), (False, False, False), (True, True, True)])
def test_launch_shapes_agree(lbt, storage, periodic):
    # grid size and block size change only the work decomposition: bitwise the
    # same result for one kernel and one sites-per-thread instantiation; other
    # instantiations are separately compiled code whose FMA contraction may
    # differ in the last bit of a site's update
    accel = (1e-5, 0.0, -2e-5) if all(periodic) else (0.0, 0.0, 0.0)
    c = Case(24, 0.8, 12, M=32, nbeads=10, periodic=periodic, accel=accel, pin_com=0 if all(periodic) else 2)
    ref = GpuRunner(lbt, torch, [c], storage)  # default: staged kernel, one block per SM
    ref.step(12)
    d_ref = ref.tr.deviations(0)
    dv = {ST64: 2, ST32: 4, 2: 8, 3: 8}[storage]
    scale = np.abs(d_ref).max()
    # rounding acts on O(1) quantities (rho, w_i rho ...): FP64/FP32 differences
    # are a few eps absolute; a 16-bit store can flip by one storage ulp
    tol = {ST64: 8 * 2.2e-16, ST32: 8 * 1.2e-7, 2: 2.0 ** -10 * scale, 3: 2.0 ** -7 * scale}[storage]
    S, Rg = lbt.LB_KERNEL_STAGED, lbt.LB_KERNEL_REGISTER
    for kernel, threads, ctas, vw, exact in [(S, 0, 3, 0, True), (S, 0, 1, 0, True), (S, 0, 5, 1, storage == ST64),
                                             (Rg, 256, 0, 0, False),
                                             (Rg, 128, 0, dv // 2, False), (Rg, 96, 7, dv, False),
                                             (Rg, 64, 152, max(dv // 4, 1), False)]:
        r = GpuRunner(lbt, torch, [c], storage)
        r.tr.lb_set_launch(kernel, threads, ctas, vw)
        r.step(12)
        d = r.tr.deviations(0)
        if exact:
            assert np.array_equal(d, d_ref), (kernel, threads, ctas, vw)
        else:
            assert np.abs(d - d_ref).max() <= tol, (kernel, threads, ctas, vw)
