"""Host arithmetic of bench.py's roofline: the algorithmic bytes of the CGS2
passes and the TF32 peak derived from the measured bf16 peaks.  No GPU."""
import json
import os

import pytest

import bench


def test_krylov_bytes_hand_count():
    """One cycle of 3 steps: step j streams 2 (2j + 3) vectors (two passes, each
    j basis vectors + w read for the dots, j + w read + w written for the
    update): (10 + 14 + 18) vectors of N entries."""
    N, vb = 1000, 8
    assert bench.krylov_bytes(3, 1, 50, N, vb) == (10 + 14 + 18) * N * vb
    # a restart at 2: steps j = 1, 2, 1
    assert bench.krylov_bytes(3, 1, 2, N, vb) == (10 + 14 + 10) * N * vb
    # two cycles split the iterations 2 + 1, each from j = 1
    assert bench.krylov_bytes(3, 2, 50, N, vb) == (10 + 14 + 10) * N * vb
    assert bench.krylov_bytes(0, 1, 50, N, vb) == 0


def test_tf32_peak_from_measured_bf16():
    burst, sustained, kind = bench.measured_peak_tf32()
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if kind == "measured":
        d = json.load(open(path))
        assert burst == pytest.approx(d["bf16_tflops"] * 1.1 / 2.25)
        assert sustained == pytest.approx(d["bf16_tflops_sustained"] * 1.1 / 2.25)
    else:
        assert burst == pytest.approx(1900.0 * 1.1 / 2.25)
