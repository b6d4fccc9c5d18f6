"""Launch candidates of the autotuner (host logic, no GPU): every candidate is
a valid shape for the storage format, the staged kernel comes first with its
default sites per thread."""
import pytest

from paper_0809_4958_gb300 import autotune, lbtracer as lbt


@pytest.mark.parametrize("storage,vec", [(lbt.LB_STORE_F64, 2), (lbt.LB_STORE_F32, 4), (lbt.LB_STORE_F16DEV, 8),
                                         (lbt.LB_STORE_BF16DEV, 8)])
def test_candidates_are_valid_shapes(storage, vec):
    cands = autotune.candidates(storage, 152)
    assert cands[0][0] == lbt.LB_KERNEL_STAGED
    assert cands[0][3] == (1 if storage == lbt.LB_STORE_F64 else 2)  # default sites per thread
    assert len(set(cands)) == len(cands)
    for kernel, threads, ctas, x in cands:
        assert ctas == 0  # persistent grid sized by the library
        if kernel == lbt.LB_KERNEL_STAGED:
            assert threads == 0 and x in ((1,) if storage == lbt.LB_STORE_F64 else (1, 2))
        else:
            assert kernel == lbt.LB_KERNEL_REGISTER and threads in (128, 256)
            assert x >= 1 and vec % x == 0 and x >= vec // 4  # one, a half or a quarter of the vector width
