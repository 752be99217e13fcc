"""The allocation-free entry point, checked against the allocating path.

bldtt_bounding_box_noalloc serves callers that cannot allocate device memory;
its result must equal the root-cluster box that bldtt_setup builds with
allocator-backed scratch (read back with bldtt_export_tree).  Min/max are
exact, so the comparison is bit-exact, the tolerance the tree tests use.
Two calls in a row, the second smaller than the first, check that nothing
left in the shared scratch array leaks into a later result.
"""
import numpy as np
import pytest
import torch

from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup_root_box(pts, q):
    dt = torch.from_numpy(pts).cuda()
    dq = torch.from_numpy(q).cuda()
    with B.Plan(dt, dt, dq, n=2, theta=0.7, N0=64, M0=64, precision=B.FP64) as plan:
        t = plan.export_tree(0)
    return np.concatenate([t["lo"][:, 0], t["hi"][:, 0]])


def test_noalloc_box_matches_allocating_path_twice():
    cases = [W.make_problem("plummer", 300_000, seed=31)[::2],
             W.make_problem("sphere", 5_000, seed=32)[::2]]
    for pts, q in cases:                      # two calls in a row, large then small
        want = _setup_root_box(pts, q)
        box, flag = B.bounding_box_noalloc(torch.from_numpy(pts).cuda())
        got = box.cpu().numpy()
        assert int(flag.item()) == 0
        assert np.array_equal(got, want)
        assert np.array_equal(got, np.concatenate([pts.min(axis=1), pts.max(axis=1)]))


def test_noalloc_box_flags_non_finite_and_rejects_bad_sizes():
    pts = W.make_problem("uniform", 4_000, seed=33)[0].copy()
    pts[2, 123] = np.nan
    box, flag = B.bounding_box_noalloc(torch.from_numpy(pts).cuda())
    assert int(flag.item()) == 1
    keep = np.ones(pts.shape[1], dtype=bool)
    keep[123] = False
    want = np.concatenate([pts[:, keep].min(axis=1), pts[:, keep].max(axis=1)])
    assert np.array_equal(box.cpu().numpy(), want)
    lib = B.load_library()
    dev = torch.zeros(6, dtype=torch.float64, device="cuda")
    import ctypes
    p = ctypes.c_void_p(dev.data_ptr())
    assert lib.bldtt_bounding_box_noalloc(p, 0, p, None, None) == 1
    assert lib.bldtt_bounding_box_noalloc(p, 2 ** 31, p, None, None) == 1
