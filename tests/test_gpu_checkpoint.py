"""Checkpoint and restore of a context (lb_save / lb_load) through the C ABI.

A run saved at step n and restored into a fresh context with the same boxes
must continue bit for bit like the run that was never interrupted: the
populations, the boundary ring, the chain (its noise is keyed on the step
number), the status words and the step counter all come back.
"""
import numpy as np
import pytest

from gpucases import Case, GpuRunner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_4958_gb300 import lbtracer
    lbtracer.load()
    return lbtracer


def cases():
    # a noisy chain in a linear-interpolation box and a Hermite box with K = 3
    return [Case(24, 0.8, 20, seed=4, M=32, nbeads=10, kT=1e-4), Case(16, 0.7, 20, seed=5, M=16, K=3, time_interp=1)]


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("where", ["host", "device"])
def test_restored_run_continues_bitwise(lbt, storage, where):
    n, k = 7, 9
    a = GpuRunner(lbt, torch, cases(), storage)
    a.step(n)
    size = a.tr.lb_checkpoint_bytes()
    buf = np.zeros(size, np.uint8) if where == "host" else torch.zeros(size, dtype=torch.uint8, device="cuda")
    a.tr.lb_save(buf)
    pushed = list(a.pushed)
    a.step(k)
    b = GpuRunner(lbt, torch, cases(), storage)
    b.tr.lb_load(buf)
    b.pushed, b.n = pushed, n
    assert b.tr.lb_current_step() == n
    b.step(k)
    for box in (0, 1):
        assert np.array_equal(a.tr.deviations(box), b.tr.deviations(box)), box
    pa, va = a.tr.chain(0, 10)
    pb, vb = b.tr.chain(0, 10)
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert b.tr.lb_current_step() == n + k


def test_checkpoint_of_another_context_is_refused(lbt):
    a = GpuRunner(lbt, torch, cases(), 1)
    a.step(2)
    buf = np.zeros(a.tr.lb_checkpoint_bytes(), np.uint8)
    a.tr.lb_save(buf)
    other = GpuRunner(lbt, torch, [Case(24, 0.8, 4, seed=4, M=32, nbeads=10, kT=1e-4)], 1)
    before = other.tr.deviations(0)
    with pytest.raises(lbt.LBError) as ei:
        other.tr.lb_load(np.zeros(other.tr.lb_checkpoint_bytes(), np.uint8))  # no header
    assert ei.value.code == lbt.LB_ERR_ARG
    with pytest.raises(lbt.LBError) as ei:
        other.tr.lb_load(buf)  # two boxes saved, one box here
    assert ei.value.code == lbt.LB_ERR_ARG
    assert np.array_equal(other.tr.deviations(0), before)  # nothing changed
