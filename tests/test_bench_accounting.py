"""The benchmark's roofline numerator and whole-job arithmetic, on the CPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_of_the_default_box():
    # 128^3 FP32 with linear time interpolation: interior sites read and write
    # 19 populations (152 B); the 96,776 boundary sites write 19 (76 B)
    # and reads 3 components of 2 FP32 samples (24 B)
    E = 128
    interior, boundary = 126 ** 3, 128 ** 3 - 126 ** 3
    assert boundary == 96776
    assert bench.alg_bytes_per_launch(E, 4, 4) == interior * 152 + boundary * (76 + 24) == 313734752


def test_algorithmic_bytes_scale_with_storage_and_interpolation():
    E = 32
    i, b = 30 ** 3, 32 ** 3 - 30 ** 3
    assert bench.alg_bytes_per_launch(E, 2, 4) == i * 76 + b * (38 + 24)          # 16-bit storage
    assert bench.alg_bytes_per_launch(E, 8, 8) == i * 304 + b * (152 + 48)        # FP64
    assert bench.alg_bytes_per_launch(E, 4, 4, time_interp=1) == i * 152 + b * (76 + 48)  # Hermite: 4 samples
