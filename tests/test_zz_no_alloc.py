"""The allocation-free sums entry point (lb_population_sums_noalloc) against
the context-based lb_conservation, through the C ABI.

Callers whose device memory is fully committed before the run (a framework
allocator that has reserved the GPU, or a loop that forbids allocations after
start-up) use the allocation-free call; it must give the same FP64 sums as the
regular entry point, on consecutive calls that share its fixed scratch array.
This file is collected last on purpose.
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


def _as_storage(dev, storage):
    """The read-out widens 16-bit storage to float32 exactly; hand the call
    the 16-bit deviations themselves."""
    if storage == 2:
        return dev.to(torch.float16).contiguous()
    if storage == 3:
        return dev.to(torch.bfloat16).contiguous()
    return dev.contiguous()


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_noalloc_sums_equal_conservation_on_two_calls(lbt, storage):
    E = 24
    c = Case(E, 0.8, 30, M=32, nbeads=12, periodic=(True, True, True), pin_com=0, kT=1e-4)
    r = GpuRunner(lbt, torch, [c], storage)
    real = torch.float64 if storage == 0 else torch.float32
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for call in range(2):
        r.step(15)
        ref = r.tr.lb_conservation(0)[:4]
        dev = torch.empty((19, E, E, E), dtype=real, device="cuda")
        r.tr.lb_read_fields(0, lbt.LB_FIELD_DEV, dev)
        pops, code = _as_storage(dev, storage), storage
        stream = torch.cuda.current_stream()
        lbt.lb_population_sums_noalloc(pops, code, E, out, stream)
        stream.synchronize()
        got = out.cpu().numpy()
        # same FP64 sums as lb_conservation up to summation order
        assert abs(got[0] - ref[0]) <= 1e-12 * E ** 3, (call, got, ref)
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-12 * E ** 3 * 0.05, (call, got, ref)
        assert got[0] > 0.9 * E ** 3


def test_noalloc_rejects_boxes_beyond_its_scratch(lbt):
    # a buffer of the right size for E = 401 passes the binding's checks; the
    # library refuses the edge because its fixed scratch covers E <= 400
    E = 401
    buf = torch.zeros(19 * E ** 3, dtype=torch.float16, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbt.LBError) as ei:
        lbt.lb_population_sums_noalloc(buf, lbt.LB_STORE_F16DEV, E, out)
    assert ei.value.code == lbt.LB_ERR_SIZE
    assert "E <= 400" in str(ei.value)
    del buf


def test_noalloc_accepts_the_largest_documented_box(lbt):
    # E = 400 is the documented maximum; zero deviations sum to exactly E^3
    E = 400
    pops = torch.zeros(19 * E ** 3, dtype=torch.float16, device="cuda")
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    lbt.lb_population_sums_noalloc(pops, lbt.LB_STORE_F16DEV, E, out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [float(E ** 3), 0.0, 0.0, 0.0]
    del pops

