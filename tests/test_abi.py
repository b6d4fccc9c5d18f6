"""The C ABI library builds, loads without a GPU and exports every function
that include/lbtracer.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbtracer.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_create", "lb_set_boundary", "lb_step", "chain_couple", "lb_read_fields"):
        assert required in names


def test_library_exports_every_declared_function():
    from paper_0809_4958_gb300 import build, lbtracer
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lbtracer.EXPORTS) == set(declared_functions())


def test_plan_validates_without_a_gpu():
    from paper_0809_4958_gb300 import lbtracer as lbt
    lib = lbt.load()
    n = ctypes.c_size_t()
    good = (lbt.lb_box_desc * 1)(lbt.box_desc(32, 0.8, nbeads=16))
    assert lib.lb_plan(good, 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_OK
    # two population buffers of 19 * 32^3 floats dominate the arena
    assert n.value >= 2 * 19 * 32 ** 3 * 4
    for bad in (lbt.box_desc(30, 0.8), lbt.box_desc(32, 0.5), lbt.box_desc(32, 0.8, K=0),
                lbt.box_desc(32, 0.8, nbeads=300)):
        arr = (lbt.lb_box_desc * 1)(bad)
        assert lib.lb_plan(arr, 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_ERR_ARG
    mixed = lbt.box_desc(32, 0.8)
    mixed.face_mode[0] = lbt.LB_FACE_PERIODIC  # x- periodic but x+ velocity
    assert lib.lb_plan((lbt.lb_box_desc * 1)(mixed), 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_ERR_ARG
    assert b"periodic" in lib.lb_last_error(None).lower() or b"axis" in lib.lb_last_error(None)
    assert lib.lb_plan(good, 1, lbt.LB_STORE_F32, 3, ctypes.byref(n)) == lbt.LB_ERR_ARG  # ring shorter than 4
    n20 = ctypes.c_size_t()
    assert lib.lb_plan(good, 1, lbt.LB_STORE_F32, 20, ctypes.byref(n20)) == lbt.LB_OK
    assert n20.value >= n.value + 16 * 6 * 3 * 32 * 32 * 4  # 16 more slots of six 32^2 faces


def test_plan_checks_frame_accel_and_zoom_without_a_gpu():
    from paper_0809_4958_gb300 import lbtracer as lbt
    lib = lbt.load()
    n = ctypes.c_size_t()
    ok = lbt.box_desc(32, 0.8, frame_accel=True, zoom=6)
    assert lib.lb_plan((lbt.lb_box_desc * 1)(ok), 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_OK
    bad = lbt.box_desc(32, 0.8)
    bad.frame_accel = 2
    assert lib.lb_plan((lbt.lb_box_desc * 1)(bad), 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_ERR_ARG
    assert b"frame_accel" in lib.lb_last_error(None)
    for zoom in (-1, 32):  # zoom must lie in [0, E - 1]
        bz = lbt.box_desc(32, 0.8, zoom=zoom)
        assert lib.lb_plan((lbt.lb_box_desc * 1)(bz), 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_ERR_ARG
    mlpz = lbt.box_desc(32, 0.8, time_interp=lbt.LB_TIME_MLP, K=16, zoom=2)  # the upsampler needs zoom <= 1
    assert lib.lb_plan((lbt.lb_box_desc * 1)(mlpz), 1, lbt.LB_STORE_F32, 0, ctypes.byref(n)) == lbt.LB_ERR_ARG
