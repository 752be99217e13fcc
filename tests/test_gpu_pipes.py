"""The benchmark's pipe probe (libbldtt_pipes.so, built apart from the
library) behind the roofline's issue ceilings returns plausible rates:
operations per clock per SM are positive, the packed FP32x2 FMA is at least as
fast per lane as the scalar one, and the MUFU unit is well below the FMA pipe
(the rates themselves are reported by bench.py)."""
import pytest
import torch

import bench

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    r = bench.pipe_rates(torch.cuda.current_stream())
    assert all(v > 0 for v in r.values())
    assert 32 <= r["ffma"] <= 256
    assert r["ffma2_lanes"] >= 0.9 * r["ffma"]
    assert r["mufu_rsqrt"] < r["ffma"] and r["mufu_ex2"] < r["ffma"]
    assert r["dfma"] < r["ffma"]
