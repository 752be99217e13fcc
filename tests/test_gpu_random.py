"""Seeded random problems against the oracle: the set-up's trees and lists
exactly, the potentials to the FP64 tolerance, on shapes the named cases do not
cover.

Each case draws its targets and sources from one of seven point sets (cube,
sphere surface, Plummer, Gaussian, a thin segment, tight clusters, a coarse
lattice with repeated points), a fifth of the sets tiny (1-20 points) and the
rest log-uniform in [200, 5000], leaf sizes log-uniform in [1, 200] (at least 8
when a set holds more than 500 points, to bound the oracle's time), degree 1-6,
theta 0 (the direct sum) or uniform in [0.4, 0.95], and one of the four
kernels.  Every case runs the cooperative tree build and traversal and must
give the oracle's clusters, leaf members, list entries per type and evaluation
counts exactly, FP64 potentials to rel-l2 1e-12 and max-norm 1e-10, and FP32
bulk potentials to rel-l2 1e-6."""
import numpy as np
import pytest

import oracle as O
from paper_2012_06925_gb300 import binding as B
from _gpu_util import (gpu_list_keys, gpu_tree_table, max_rel, oracle_list_keys, oracle_tree_table,
                       rel_l2, run_gpu, same_leaf_members)

pytestmark = pytest.mark.gpu

KINDS = ["cube", "sphere", "plummer", "gaussian", "segment", "clusters", "lattice"]
KERNELS = [B.COULOMB, B.YUKAWA, B.OSCILLATORY, B.REG_COULOMB]


def points(kind: str, n: int, rng: np.random.Generator) -> np.ndarray:
    if kind == "cube":
        return rng.uniform(-1, 1, (3, n))
    if kind == "sphere":
        v = rng.normal(size=(3, n))
        return v / np.linalg.norm(v, axis=0)
    if kind == "plummer":
        u = rng.uniform(0, 0.98518, n)
        r = 0.1 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        v = rng.normal(size=(3, n))
        return r * v / np.linalg.norm(v, axis=0)
    if kind == "gaussian":
        return rng.normal(size=(3, n))
    if kind == "segment":                      # nearly one-dimensional
        t = rng.uniform(-1, 1, n)
        return np.stack([t, 1e-3 * rng.normal(size=n), 0.5 + 1e-6 * rng.normal(size=n)])
    if kind == "clusters":                     # a few tight blobs far apart
        centres = rng.uniform(-5, 5, (3, 4))
        which = rng.integers(0, 4, n)
        return centres[:, which] + 1e-3 * rng.normal(size=(3, n))
    # coarse lattice: many points share coordinates and some coincide exactly
    return rng.integers(-4, 5, (3, n)).astype(np.float64) / 4.0


def draw(seed: int):
    rng = np.random.default_rng(1000 + seed)

    def size():   # a fifth tiny (1-20 points), the rest 200-5000
        if rng.uniform() < 0.2:
            return int(rng.integers(1, 21))
        return int(round(10 ** rng.uniform(np.log10(200), np.log10(5000))))

    m = size()
    shared = rng.uniform() < 0.3
    n = m if shared else size()
    tk = KINDS[rng.integers(len(KINDS))]
    sk = tk if shared else KINDS[rng.integers(len(KINDS))]
    tgt = points(tk, m, rng)
    src = tgt if shared else points(sk, n, rng)
    q = rng.uniform(-1, 1, n)

    def leaf(count):
        lo = 8 if count > 500 else 1
        return int(max(lo, round(10 ** rng.uniform(0, np.log10(200)))))

    m0 = leaf(m)
    n0 = m0 if shared else leaf(n)
    kernel = KERNELS[rng.integers(len(KERNELS))]
    kappa = 0.0 if kernel == B.COULOMB else float(rng.uniform(0.01, 2.0))
    theta = 0.0 if rng.uniform() < 0.15 else float(rng.uniform(0.4, 0.95))
    kw = dict(kernel=kernel, kappa=kappa, n=int(rng.integers(1, 7)), theta=theta, N0=n0, M0=m0)
    return f"{tk}/{sk} M={m} N={n}", tgt, src, q, kw


@pytest.mark.parametrize("seed", range(24))
def test_random_problem_matches_oracle(seed):
    desc, tgt, src, q, kw = draw(seed)
    ref = O.bldtt(tgt, src, q, **kw)
    phi, plan = run_gpu(tgt, src, q, precision=B.FP64, **kw)
    with plan:
        gt, gs = plan.export_tree(0), plan.export_tree(1)
        assert same_leaf_members(gt, ref.ttree), desc
        assert same_leaf_members(gs, ref.stree), desc
        assert gpu_tree_table(gt) == oracle_tree_table(ref.ttree), desc
        assert gpu_tree_table(gs) == oracle_tree_table(ref.stree), desc
        assert gpu_list_keys(gt, gs, plan.export_lists()) == oracle_list_keys(ref.ttree, ref.stree,
                                                                              ref.lists), desc
        st = plan.stats()
        assert st["interactions"] == [float(v) for v in ref.counts], desc
    if np.all(ref.phi == 0):
        assert np.all(phi == 0), desc
        return
    assert rel_l2(ref.phi, phi) <= 1e-12, desc
    assert max_rel(ref.phi, phi) <= 1e-10, desc
    phi32, plan32 = run_gpu(tgt, src, q, precision=B.FP32_BULK, **kw)
    plan32.close()
    assert rel_l2(ref.phi, phi32) <= 1e-6, desc
