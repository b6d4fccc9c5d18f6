"""The chain-order MD layout of the bead kernel (lb_set_bead_launch(2, 0)):
two lanes per bead in chain order, one taking the bonds, the other the beads
two apart, the two splitting the Verlet list of the pairs further apart.
Checked against the FP64 oracle (all-pairs WCA, no lists) on a folded chain
whose rows touch, so that the listed pairs carry force, with velocities that
move beads past half the skin inside a step, so that the lists are rebuilt
between substeps."""
import numpy as np
import pytest

import oracle
from gpucases import Case, GpuRunner

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


def serpentine(nb, E, row, bond=0.97, h=1.08, turn_dx=0.8):
    """Chain folded into rows of `row` beads 0.97 apart, the rows 1.08 apart,
    one bead between rows at each turn (its two bonds 0.97 long): beads of
    adjacent rows at the same x sit inside the WCA cut-off (2^(1/6) = 1.122)
    with a mild repulsion, and most of those pairs are four or more places
    apart along the chain.  Every bond starts near its rest length."""
    pos = []
    r = 0
    while len(pos) < nb:
        xs = [c * bond for c in range(row)]
        if r % 2:
            xs = xs[::-1]
        for x in xs:
            if len(pos) < nb:
                pos.append([x, r * h, 0.0])
        if len(pos) < nb:
            pos.append([(row - 1) * bond + turn_dx if r % 2 == 0 else -turn_dx, (r + 0.5) * h, 0.0])
        r += 1
    pos = np.asarray(pos)
    return np.ascontiguousarray(pos + 0.5 * (E - 1) - pos.mean(axis=0))


def listed_contacts(pos, rc=2.0 ** (1.0 / 6.0)):
    n = len(pos)
    return sum(1 for i in range(n) for j in range(i + 3, n) if np.linalg.norm(pos[i] - pos[j]) < rc)


@pytest.mark.parametrize("nb,row", [(64, 8), (24, 6)])
def test_chain_order_layout_matches_oracle(lbt, nb, row):
    E = 24
    c = Case(E, 0.8, 3, seed=3, M=16, nbeads=nb, kT=1e-3, pin_com=2)
    c.pos0 = serpentine(nb, E, row)
    assert listed_contacts(c.pos0) >= nb // 3  # the lists carry force from the start
    rng = np.random.default_rng(11)
    # a common drift moves every bead past half the skin (0.15) inside the
    # first step; a small random part on top
    c.vel0 = np.ascontiguousarray(np.array([0.35, 0.0, 0.0]) + 0.03 * rng.standard_normal((nb, 3)))
    r = GpuRunner(lbt, torch, [c], ST64)
    r.tr.lb_set_bead_launch(2, 0)
    r.step(3)
    sim = c.run_oracle()
    pos, vel = r.tr.chain(0, nb)
    ep, ev = np.abs(pos - sim.pos).max(), np.abs(vel - sim.vel).max()
    print("%d beads, 3 steps: max |pos - oracle| %.2e, |vel - oracle| %.2e, moved %.2f"
          % (nb, ep, ev, np.abs(sim.pos - c.pos0).max()))
    assert np.abs(sim.pos - c.pos0).max() > 0.2
    # the two sides sum the same forces in different orders; the contacts
    # amplify those FP64 roundings over 150 substeps, a missed or misplaced
    # pair would show at the size of the force itself
    assert ep < 1e-9 and ev < 1e-8
    _, w = oracle.lattice()
    assert np.abs(r.tr.deviations(0) - (sim.f - w[:, None, None, None])).max() < 1e-11


@pytest.mark.parametrize("lanes,bpt", [(8, 1), (4, 1), (2, 1), (1, 1), (1, 2)])
def test_other_layouts_match_oracle_on_the_folded_chain(lbt, lanes, bpt):
    E, nb = 24, 64
    c = Case(E, 0.8, 2, seed=3, M=16, nbeads=nb, kT=1e-3, pin_com=2)
    c.pos0 = serpentine(nb, E, 8)
    c.vel0 = np.ascontiguousarray(np.tile([0.35, 0.0, 0.0], (nb, 1)))
    r = GpuRunner(lbt, torch, [c], ST64)
    r.tr.lb_set_bead_launch(lanes, bpt)
    r.step(2)
    sim = c.run_oracle()
    pos, vel = r.tr.chain(0, nb)
    assert np.abs(pos - sim.pos).max() < 1e-9 and np.abs(vel - sim.vel).max() < 1e-8


def test_chain_order_layout_agrees_with_eight_lanes_fp32(lbt):
    E, nb = 32, 64
    runs = []
    for lanes, bpt in ((8, 1), (2, 0)):
        c = Case(E, 0.8, 10, seed=4, M=16, nbeads=nb, kT=1e-4)
        c.pos0 = serpentine(nb, E, 8)
        r = GpuRunner(lbt, torch, [c], ST32)
        r.tr.lb_set_bead_launch(lanes, bpt)
        r.step(10)
        runs.append(r.tr.chain(0, nb)[0])
    assert np.abs(runs[0] - runs[1]).max() < 1e-4


def test_chain_order_layout_reports_a_broken_bond(lbt):
    c = Case(16, 0.8, 2, seed=2, M=16, nbeads=6)
    c.vel0 = np.zeros((6, 3))
    c.vel0[0] = [-40.0, 0, 0]
    c.vel0[1] = [40.0, 0, 0]
    r = GpuRunner(lbt, torch, [c], ST32)
    r.tr.lb_set_bead_launch(2, 0)
    r.step(2)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_sync()
    assert ei.value.code == lbt.LB_ERR_FENE


def test_chain_order_layout_refusals(lbt):
    tr = lbt.Tracers([lbt.box_desc(32, 0.8, nbeads=64)], lbt.LB_STORE_F32)
    for lanes in (1, 4, 8):
        with pytest.raises(lbt.LBError) as ei:
            tr.lb_set_bead_launch(lanes, 0)  # the chain-order layout takes two lanes per bead
        assert ei.value.code == lbt.LB_ERR_ARG
    tr.lb_set_bead_launch(2, 0)
    big = lbt.Tracers([lbt.box_desc(64, 0.8, nbeads=256)], lbt.LB_STORE_F32)
    big.lb_set_bead_launch(2, 0)  # the largest chain: 512 MD threads
