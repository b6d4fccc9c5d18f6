"""The chain trajectory ring (lb_set_chain_history): after every step the
bead kernel leaves the end-of-step positions in slot (n + 1) mod slots, for
plain steps and for graph replays alike, equal bit for bit to the positions
the context reports after that step."""
import numpy as np
import pytest

from gpucases import Case, GpuRunner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ST32 = 1


@pytest.fixture(scope="module")
def lbt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_4958_gb300 import lbtracer
    lbtracer.load()
    return lbtracer


def two_chains():
    # boxes of different capacity: the second chain starts at bead offset 12
    return [Case(24, 0.8, 12, seed=1, M=16, nbeads=12, kT=1e-4), Case(24, 0.8, 12, seed=2, M=16, nbeads=20, kT=1e-4)]


def positions_per_step(lbt, nsteps):
    r = GpuRunner(lbt, torch, two_chains(), ST32)
    out = []
    for _ in range(nsteps):
        r.step(1)
        out.append(np.concatenate([r.tr.chain(0, 12)[0], r.tr.chain(1, 20)[0]]))
    return out


def test_plain_steps_fill_the_ring(lbt):
    ref = positions_per_step(lbt, 7)
    r = GpuRunner(lbt, torch, two_chains(), ST32)
    slots = 5
    hist = torch.full((slots, 32, 3), np.nan, dtype=torch.float64, device="cuda")
    r.tr.lb_set_chain_history(hist, slots)
    r.step(7)
    r.tr.lb_sync()
    h = hist.cpu().numpy()
    for n in range(2, 7):  # steps 2..6 are in the ring (slot (n + 1) mod 5)
        assert np.array_equal(h[(n + 1) % slots], ref[n]), n


def test_graph_replays_fill_the_ring(lbt):
    ref = positions_per_step(lbt, 12)
    G = 4
    r = GpuRunner(lbt, torch, two_chains(), ST32, ring_slots=G + 4)
    hist = torch.zeros((G, 32, 3), dtype=torch.float64, device="cuda")
    r.tr.lb_set_chain_history(hist, G)
    r.tr.lb_graph_capture(G)  # captures steps, runs none
    for rep in range(3):  # steps 0..3, 4..7, 8..11
        r.push_for(r.n + G - 1)
        r.tr.lb_graph_launch()
        r.n += G
        r.tr.lb_sync()
        h = hist.cpu().numpy()
        for k in range(G):
            n = r.n - G + k
            assert np.array_equal(h[(n + 1) % G], ref[n]), (rep, n)


def test_refusals(lbt):
    r = GpuRunner(lbt, torch, two_chains(), ST32)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_set_chain_history(np.zeros((3, 32, 3)), 3)  # host memory
    assert ei.value.code == lbt.LB_ERR_ARG
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_set_chain_history(None, 3)
    assert ei.value.code == lbt.LB_ERR_ARG
    nochain = lbt.Tracers([lbt.box_desc(16, 0.8)], lbt.LB_STORE_F32)
    with pytest.raises(lbt.LBError) as ei:
        nochain.lb_set_chain_history(torch.zeros((2, 1, 3), dtype=torch.float64, device="cuda"), 2)
    assert ei.value.code == lbt.LB_ERR_STATE
    r.tr.lb_set_chain_history(None, 0)  # off
