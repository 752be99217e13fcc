"""The allocation-free entry point, checked against the allocating path.

bldtt_bounding_box_noalloc serves callers that cannot allocate device memory;
its result must equal the root-cluster box that bldtt_setup builds with
allocator-backed scratch (read back with bldtt_export_tree).  Min/max are
exact, so the comparison is bit for bit (on the float64 bit patterns, so that
-0.0 and +0.0 differ), the tolerance the tree tests use.  Calls in a row,
sizes going down and up, check that nothing left in the shared scratch array
leaks into a later result; the largest case exceeds one grid-stride pass of
the capped grid.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _setup_root_box(pts, q):
    dt = torch.from_numpy(pts).cuda()
    dq = torch.from_numpy(q).cuda()
    with B.Plan(dt, dt, dq, n=2, theta=0.7, N0=64, M0=64, precision=B.FP64) as plan:
        t = plan.export_tree(0)
    return np.concatenate([t["lo"][:, 0], t["hi"][:, 0]])


def _signed_zero_extremes():
    """Points whose x minimum and y maximum are zero, held by both -0.0 and
    +0.0 particles."""
    pts, _, q = W.make_problem("uniform", 3_000, seed=34)
    pts = pts.copy()
    pts[0] = np.abs(pts[0])
    pts[1] = -np.abs(pts[1])
    pts[0, [5, 900]] = [-0.0, 0.0]
    pts[1, [17, 2500]] = [0.0, -0.0]
    return pts, q


def test_noalloc_box_matches_allocating_path_twice():
    cases = [W.make_problem("plummer", 300_000, seed=31)[::2],   # 150k points
             W.make_problem("sphere", 5_000, seed=32)[::2],
             _signed_zero_extremes(),
             W.make_problem("uniform", 400_000, seed=35)[::2]]   # 400k: two grid-stride passes
    for pts, q in cases:                      # calls in a row, large, small, large
        want = _setup_root_box(pts, q)
        box, flag = B.bounding_box_noalloc(torch.from_numpy(pts).cuda())
        got = box.cpu().numpy()
        assert int(flag.item()) == 0
        assert np.array_equal(_bits(got), _bits(want))
        assert np.array_equal(got, np.concatenate([pts.min(axis=1), pts.max(axis=1)]))
    # the zero extremes come back as +0.0, as in the setup's root box
    pts, _ = _signed_zero_extremes()
    box, _ = B.bounding_box_noalloc(torch.from_numpy(pts).cuda())
    got = box.cpu().numpy()
    assert _bits(got[0]) == _bits(0.0) and _bits(got[4]) == _bits(0.0)


def test_noalloc_box_without_flag_pointer():
    pts, _, q = W.make_problem("uniform", 400_000, seed=36)
    dp = torch.from_numpy(pts).cuda()
    box = torch.empty(6, dtype=torch.float64, device="cuda")
    lib = B.load_library()
    rc = lib.bldtt_bounding_box_noalloc(ctypes.c_void_p(dp.data_ptr()), pts.shape[1],
                                        ctypes.c_void_p(box.data_ptr()), None, None)
    assert rc == 0
    torch.cuda.synchronize()
    assert np.array_equal(_bits(box.cpu().numpy()), _bits(_setup_root_box(pts, q)))


def test_noalloc_box_flags_non_finite_and_rejects_bad_sizes():
    pts = W.make_problem("uniform", 4_000, seed=33)[0].copy()
    pts[2, 123] = np.nan
    pts[0, 7] = np.inf
    pts[1, 3000] = -np.inf
    box, flag = B.bounding_box_noalloc(torch.from_numpy(pts).cuda())
    assert int(flag.item()) == 1
    finite = np.isfinite(pts)
    want = np.array([pts[d, finite[d]].min() for d in range(3)]
                    + [pts[d, finite[d]].max() for d in range(3)])
    assert np.array_equal(box.cpu().numpy(), want)       # infinities left out of the box
    lib = B.load_library()
    dev = torch.zeros(6, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dev.data_ptr())
    assert lib.bldtt_bounding_box_noalloc(p, 0, p, None, None) == 1
    assert lib.bldtt_bounding_box_noalloc(p, 2 ** 31, p, None, None) == 1
