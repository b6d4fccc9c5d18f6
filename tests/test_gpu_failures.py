"""Failure detection through the C ABI, without faulting or hanging the GPU.

Each error code the library raises while stepping has a test here that would
fail if its detection were removed:
  - LB_ERR_TIMEOUT from the host's bounded wait on the stream (lb_sync), made
    certain by a bounded sleep kernel placed on the context stream;
  - LB_ERR_TIMEOUT from the stream-collide kernel's bounded barrier wait, made
    to run out by the test-only injection (lb_test_inject): the producer never
    arms one pipeline stage, the consumers give up after a short limit, flag
    that box and leave;
  - LB_ERR_NONFINITE from the in-step density check, raised by a NaN placed in
    the initial field of one box.
In every case the other box of a two-box context steps on bitwise as in a
clean run, and the context keeps stepping afterwards.
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


def raw_deviations(lbt, r, box):
    """Stored deviations of a box without the status check that synchronous
    reads make (a failed box's own reads return its error)."""
    E = r.tr.E(box)
    t = torch.empty((19, E, E, E), dtype=r.tr.real, device="cuda")
    r.tr.lb_read_fields(box, lbt.LB_FIELD_DEV | lbt.LB_FIELD_ASYNC, t)
    r.tr.stream.synchronize()
    return t.cpu().numpy()


def two_boxes():
    # box 0 carries a chain (the bead kernel and the forced re-collision run
    # beside the stream-collide); box 1 is the one that fails
    return [Case(24, 0.8, 8, seed=1, M=32, nbeads=10), Case(16, 0.8, 8, seed=2, M=16)]


def test_host_stream_wait_times_out_then_recovers(lbt):
    c = Case(24, 0.8, 4, M=16)
    r = GpuRunner(lbt, torch, [c], 1)
    r.step(2)
    with torch.cuda.stream(r.tr.stream):
        torch.cuda._sleep(800_000_000)  # a bounded spin of 8e8 cycles, about 0.4 s at 2 GHz
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_sync(timeout_ms=20)
    assert ei.value.code == lbt.LB_ERR_TIMEOUT
    r.tr.lb_sync()  # the stream drains: the context stays usable
    r.step(2)
    r.tr.lb_sync()
    assert r.tr.lb_current_step() == 4
    assert r.tr.lb_status(0) == lbt.LB_OK


def test_device_wait_runs_out_and_flags_only_its_box(lbt):
    ref = GpuRunner(lbt, torch, two_boxes(), 1)
    ref.step(3)
    r = GpuRunner(lbt, torch, two_boxes(), 1)
    r.step(2)
    r.tr.lb_test_inject(lbt.LB_INJECT_WITHHOLD_LAST_TILE, 2000)  # waits give up after 2 ms
    r.step(1)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_sync()
    assert ei.value.code == lbt.LB_ERR_TIMEOUT
    assert r.tr.lb_status(1) == lbt.LB_ERR_TIMEOUT
    assert r.tr.lb_status(0) == lbt.LB_OK
    assert np.array_equal(r.tr.deviations(0), ref.tr.deviations(0))
    # injection off: box 0 keeps stepping exactly as the clean run, box 1 stays frozen
    r.tr.lb_test_inject(lbt.LB_INJECT_NONE, 0)
    d1_err = raw_deviations(lbt, r, 1)
    r.step(2)
    ref.step(2)
    assert np.array_equal(r.tr.deviations(0), ref.tr.deviations(0))
    assert np.array_equal(raw_deviations(lbt, r, 1), d1_err)
    assert r.tr.lb_status(1) == lbt.LB_ERR_TIMEOUT


def test_injection_is_refused_for_the_register_kernel(lbt):
    r = GpuRunner(lbt, torch, [Case(16, 0.8, 2, M=16)], 1)
    r.tr.lb_set_launch(lbt.LB_KERNEL_REGISTER, 128, 0, 0)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_test_inject(lbt.LB_INJECT_WITHHOLD_LAST_TILE, 2000)
    assert ei.value.code == lbt.LB_ERR_STATE


@pytest.mark.parametrize("kernel", ["staged", "register"])
@pytest.mark.parametrize("storage", [0, 1, 2])
def test_nonfinite_density_flags_only_its_box_while_stepping(lbt, kernel, storage):
    clean = two_boxes()
    bad = two_boxes()
    bad[1].u0 = bad[1].u0.copy()
    bad[1].u0[0, 8, 8, 8] = np.nan  # one interior site of box 1
    ref = GpuRunner(lbt, torch, clean, storage)
    r = GpuRunner(lbt, torch, bad, storage)
    if kernel == "register":
        for x in (ref, r):
            x.tr.lb_set_launch(lbt.LB_KERNEL_REGISTER, 128, 0, 0)
    ref.step(3)
    r.step(3)
    with pytest.raises(lbt.LBError) as ei:
        r.tr.lb_sync()
    assert ei.value.code == lbt.LB_ERR_NONFINITE
    assert r.tr.lb_status(1) == lbt.LB_ERR_NONFINITE
    assert r.tr.lb_status(0) == lbt.LB_OK
    assert np.array_equal(r.tr.deviations(0), ref.tr.deviations(0))
    # the flagged box froze after the step that found the NaN
    d1 = raw_deviations(lbt, r, 1)
    r.step(1)
    ref.step(1)
    assert np.array_equal(raw_deviations(lbt, r, 1), d1, equal_nan=True)
    assert np.array_equal(r.tr.deviations(0), ref.tr.deviations(0))
