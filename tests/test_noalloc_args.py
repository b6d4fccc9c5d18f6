"""Argument checks of the allocation-free sums call, without a GPU.

The C call takes no buffer sizes, so the binding rejects mismatched buffers
before any launch, and the library rejects box edges beyond its fixed scratch
before any CUDA call.  Stand-in objects play the tensors here: each case
differs from a valid call in one property only.
"""
import ctypes

import pytest
import torch

from paper_0809_4958_gb300 import lbtracer as lbt


class FakeTensor:
    def __init__(self, numel, elem, dtype, is_cuda=True):
        self._n, self._e, self.dtype, self.is_cuda = numel, elem, dtype, is_cuda

    def numel(self):
        return self._n

    def element_size(self):
        return self._e


E = 16
GOOD_POPS = {0: (8, torch.float64), 1: (4, torch.float32), 2: (2, torch.float16), 3: (2, torch.bfloat16)}


def good(storage=1):
    e, dt = GOOD_POPS[storage]
    return FakeTensor(19 * E ** 3, e, dt), FakeTensor(4, 8, torch.float64)


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_valid_arguments_pass_the_checks(storage):
    pops, out = good(storage)
    lbt.check_noalloc_args(pops, storage, E, out)


@pytest.mark.parametrize("case", ["host_pops", "short_pops", "f32_with_f64_storage", "f16_with_f32_storage",
                                  "host_out", "f32_out", "short_out", "bad_storage", "zero_edge"])
def test_mismatched_arguments_are_rejected(case):
    pops, out = good(1)
    storage, edge = 1, E
    if case == "host_pops":
        pops.is_cuda = False
    elif case == "short_pops":
        pops._n = 19 * E ** 3 - 1
    elif case == "f32_with_f64_storage":
        storage = 0
    elif case == "f16_with_f32_storage":
        pops._e, pops.dtype = 2, torch.float16
    elif case == "host_out":
        out.is_cuda = False
    elif case == "f32_out":
        out.dtype = torch.float32
    elif case == "short_out":
        out._n = 3
    elif case == "bad_storage":
        storage = 4
    elif case == "zero_edge":
        edge = 0
    with pytest.raises(lbt.LBError) as ei:
        lbt.check_noalloc_args(pops, storage, edge, out)
    assert ei.value.code == lbt.LB_ERR_ARG


@pytest.mark.parametrize("edge", [401, 406, 1024])
def test_library_rejects_edges_beyond_400_before_any_cuda_call(edge):
    lib = lbt.load()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.lb_population_sums_noalloc(dummy, lbt.LB_STORE_F32, edge, dummy, None) == lbt.LB_ERR_SIZE
    assert b"E <= 400" in lib.lb_last_error(None)


def test_library_rejects_null_and_unknown_storage_before_any_cuda_call():
    lib = lbt.load()
    dummy = ctypes.c_void_p(256)
    assert lib.lb_population_sums_noalloc(None, lbt.LB_STORE_F32, 8, dummy, None) == lbt.LB_ERR_ARG
    assert lib.lb_population_sums_noalloc(dummy, 7, 8, dummy, None) == lbt.LB_ERR_ARG
    assert lib.lb_population_sums_noalloc(dummy, lbt.LB_STORE_F32, 0, dummy, None) == lbt.LB_ERR_ARG
