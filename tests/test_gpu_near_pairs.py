"""FP32_BULK accuracy on close pairs.

The FP32 path carries coordinates relative to a frame centre per 256-source
chunk, so a pair at distance r inside a chunk of half-size rho sees a rounding
error of about u rho / r on r (u = 2^-24).  Targets near a particle chunk add
the frame residuals of both points, which keeps the error at a few u for any
r > 0.  These tests put points much closer than the chunk size and hold the
FP32 result to the FP64 plan target by target, and check that a target's
result does not depend on which warp evaluated it (the consumer layout)."""
import os

import numpy as np
import pytest

from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import max_rel, rel_l2, run_gpu

pytestmark = pytest.mark.gpu


def close_pairs(n_base, n_close, sep, seed, kind="uniform"):
    """n_base points of `kind` plus n_close partners, each at distance `sep`
    from a base point in a random direction."""
    rng = np.random.default_rng(seed)
    base, _, _ = W.make_problem(kind, n_base, seed=seed)
    pick = rng.choice(n_base, size=n_close, replace=False)
    u = rng.standard_normal((3, n_close))
    u /= np.linalg.norm(u, axis=0)
    pts = np.concatenate([base, base[:, pick] + sep * u], axis=1)
    q = rng.uniform(-1, 1, pts.shape[1])
    return np.ascontiguousarray(pts), q, n_base + np.arange(n_close), pick


@pytest.mark.parametrize("sep", [1e-5, 1e-7])
@pytest.mark.parametrize("kernel,kappa", [(B.COULOMB, 0.0), (B.YUKAWA, 1.3),
                                          (B.OSCILLATORY, 2.0)])
def test_close_pairs_fp32_matches_fp64(sep, kernel, kappa):
    pts, q, partners, pick = close_pairs(20_000, 200, sep, seed=11)
    kw = dict(kernel=kernel, kappa=kappa, n=5, theta=0.7, N0=400, M0=400)
    phi64, p64 = run_gpu(pts, pts, q, precision=B.FP64, **kw)
    p64.close()
    phi32, p32 = run_gpu(pts, pts, q, precision=B.FP32_BULK, **kw)
    p32.close()
    # the close pair's own term q/r dominates these targets' potentials
    idx = np.concatenate([partners, pick])
    assert max_rel(phi64[idx], phi32[idx]) <= 1e-5
    assert rel_l2(phi64[idx], phi32[idx]) <= 1e-6
    assert rel_l2(phi64, phi32) <= 1e-6


def test_sphere_surface_fp32_matches_fp64():
    """Points on the unit sphere (a 2-D set): nearest-neighbour distances far
    below the chunk size dominate the potentials of many targets."""
    pts, _, _ = W.make_problem("sphere", 60_000, seed=23)
    q = np.random.default_rng(23).standard_normal(60_000)
    for kernel, kappa in ((B.COULOMB, 0.0), (B.YUKAWA, 0.7)):
        kw = dict(kernel=kernel, kappa=kappa, n=6, theta=0.7, N0=500, M0=500)
        phi64, p64 = run_gpu(pts, pts, q, precision=B.FP64, **kw)
        p64.close()
        phi32, p32 = run_gpu(pts, pts, q, precision=B.FP32_BULK, **kw)
        p32.close()
        assert rel_l2(phi64, phi32) <= 1e-6, kernel


def test_result_independent_of_consumer_layout(monkeypatch):
    """Layouts group targets into warps differently; per-target results must
    be bit for bit the same (the careful and guarded paths keep the packed
    path's arithmetic for every target that does not need them)."""
    pts, q, _, _ = close_pairs(30_000, 300, 1e-6, seed=5)
    kw = dict(kernel=B.COULOMB, kappa=0.0, n=5, theta=0.7, N0=600, M0=600)
    out = []
    for layout in ("0", "1", "2", "3", "4", "5"):     # 3-5: the same with idle warps skipping
        monkeypatch.setenv("BLDTT_INTERACT_LAYOUT", layout)
        phi, plan = run_gpu(pts, pts, q, precision=B.FP32_BULK, **kw)
        plan.close()
        out.append(phi)
    for other in out[1:]:
        assert np.array_equal(out[0], other)
