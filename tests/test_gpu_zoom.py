"""Spatial zoom on the GPU (Sec. 3: boundary samples on a coarse grid of
spacing z sites, bilinear within each face; initial field trilinear) against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from gpucases import Case, GpuRunner, interior, rel_l2

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


@pytest.mark.parametrize("E,z", [(16, 3), (24, 5), (40, 6)])
def test_generator_on_the_coarse_grid(lbt, E, z):
    # (24, 5) and (40, 6): the last coarse cell reaches past the box
    from paper_0809_4958_gb300 import inputs
    modes = inputs.mode_table(4, 128, 1, E / 2, E)
    ref = oracle.face_samples(modes, E, 3, 1, 2, zoom=z)
    got = lbt.synth_faces(modes, E, 3, 1, 2, torch.float64, zoom=z).cpu().numpy()
    assert got.shape == ref.shape and np.abs(got - ref).max() < 1e-14
    vref = oracle.volume_field(modes, E, 2.0, zoom=z)
    vgot = lbt.synth_volume(modes, E, 2.0, torch.float64, zoom=z).cpu().numpy()
    assert vgot.shape == vref.shape and np.abs(vgot - vref).max() < 1e-14


@pytest.mark.parametrize("E,z,interp", [(16, 3, 0), (24, 5, 1), (40, 6, 0)])
def test_zoomed_steps_f64_sitewise(lbt, E, z, interp):
    # initial field trilinear from the coarse grid, a few steps with the
    # bilinear boundary: FP64 populations site by site
    c = Case(E, 0.8, 6, M=64, K=2, time_interp=interp, zoom=z, nbeads=6)
    r = GpuRunner(lbt, torch, [c], ST64)
    r.step(6)
    sim = c.run_oracle()
    _, w = oracle.lattice()
    assert np.abs(r.tr.deviations(0) - (sim.f - w[:, None, None, None])).max() < 1e-14


def test_zoomed_box_fp32_300_steps(lbt):
    # 64^3 box with z = 7 (ten coarse cells per side), Hermite in time, chain
    c = Case(64, 0.8, 300, M=256, k_max=16, K=4, time_interp=1, zoom=7, nbeads=16)
    r = GpuRunner(lbt, torch, [c], ST32)
    r.step(300)
    u = r.tr.fields(0)[1]
    u_ref = c.run_oracle().fields()[1]
    assert rel_l2(interior(u), interior(u_ref)) <= 1e-5


def test_zoom_is_refused_for_the_upsampler(lbt):
    with pytest.raises(Exception):
        lbt.Tracers([lbt.box_desc(16, 0.8, time_interp=lbt.LB_TIME_MLP, K=16, zoom=3)], ST32)
