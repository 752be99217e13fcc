"""Parity at the full size of the unequal-set workload: 1E7 uniform targets in
[-1,1]^3, 5E6 Plummer sources (scale radius 0.1, truncated at r = 1), Yukawa
kappa = 0.5, n = 7, theta = 0.8, leaves of 2000, in the launch configuration
the benchmark times for it.

Exact: both trees (boxes, levels, parents, leaf memberships) and all four
interaction lists against the oracle's.  Sampled: FP64 potentials at targets
the oracle evaluates one by one (Eq. (19) along each target's chain of
clusters).  FP32_BULK against FP64 on the whole output is checked by
test_gpu_full_size.py.  The oracle's set-up of 1.5E7 points is the longest
CPU step of the GPU suite (about 20 s on one core), so this file is collected
last."""
import numpy as np
import pytest

import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import (gpu_list_keys, gpu_tree_table, oracle_list_keys, oracle_tree_table,
                       same_leaf_members, to_dev)

pytestmark = pytest.mark.gpu


def test_unequal_yukawa_full_size_against_the_oracle():
    cfg = W.CONFIGS["unequal_yukawa"]
    tgt, src, q = W.make_problem(cfg["kind"], cfg["M"], cfg["N"], seed=cfg["seed"],
                                 sources_kind=cfg["sources_kind"])
    kw = dict(kernel=cfg["kernel"], kappa=cfg["kappa"], n=cfg["n"], theta=cfg["theta"],
              N0=cfg["N0"], M0=cfg["M0"])
    idx = np.random.default_rng(2025).choice(tgt.shape[1], size=24, replace=False)
    with B.Plan(to_dev(tgt), to_dev(src), to_dev(q), precision=B.FP64, **kw) as plan:
        got = plan.compute().cpu().numpy()[idx]
        plan.check_error()
        gt, gs = plan.export_tree(0), plan.export_tree(1)
        glists = gpu_list_keys(gt, gs, plan.export_lists())

    samp = O.SampledBLDTT(tgt, src, q, **kw)
    assert same_leaf_members(gt, samp.tt)
    assert same_leaf_members(gs, samp.st)
    assert gpu_tree_table(gt) == oracle_tree_table(samp.tt)
    assert gpu_tree_table(gs) == oracle_tree_table(samp.st)
    assert glists == oracle_list_keys(samp.tt, samp.st, samp.lists)

    ref = samp.potentials(idx)
    assert O.relative_l2_error(ref, got) <= 1e-12
    assert O.max_norm_error(ref, got) <= 1e-10
