"""Parity against the oracle at the full sizes of two benchmarked workloads,
in the launch configurations the benchmark times for them.

Unequal sets: 1E7 uniform targets in [-1,1]^3, 5E6 Plummer sources (scale
radius 0.1, truncated at r = 1), Yukawa kappa = 0.5, n = 7, theta = 0.8,
leaves of 2000.  Exact: both trees (boxes, levels, parents, leaf memberships)
and all four interaction lists.  Sampled: FP64 potentials at targets the
oracle evaluates one by one (Eq. (19) along each target's chain of clusters).
FP32_BULK against FP64 on the whole output is checked by test_gpu_full_size.py.

Batched: the 512 independent problems of the batched workload (1E3 to 1E5
points, half in the cube and half on the unit sphere, normal charges, Coulomb
or Yukawa with kappa in [0.1, 2]; n = 6, theta = 0.7, leaves of 500) in one
plan.  Every problem: FP32_BULK against FP64 within the 1e-6 budget.  Six
problems (the smallest, the largest and four others drawn at random): their trees'
clusters and all their list entries exactly as the oracle builds them for the
problem alone, and FP64 potentials at sampled targets.

The oracle's set-ups here are the longest CPU steps of the GPU suite (about
20 s for the 1.5E7 points of the unequal sets on one core), so this file is
collected last."""
import numpy as np
import pytest

import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import (gpu_list_keys, gpu_tree_table, max_rel, oracle_list_keys,
                       oracle_tree_table, rel_l2, same_leaf_members, to_dev)

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


BATCHED = dict(count=512, seed=4, n=6, theta=0.7, N0=500, M0=500)


def check_batched_problem(i, off, gt, gs, lists, phi64, samp, idx):
    """Problem i of a batch against the oracle's BLDTT of that problem alone
    (samp): cluster particle ranges and boxes, list entries, sampled FP64
    potentials.  Forest particle ranges are made problem-local by off[i]."""
    b, e = int(off[i]), int(off[i + 1])
    for tree_g, tree_o in ((gt, samp.tt), (gs, samp.st)):
        sel = np.flatnonzero((tree_g["begin"] >= b) & (tree_g["begin"] < e))
        got = sorted((int(tree_g["begin"][c]) - b, int(tree_g["end"][c]) - b,
                      tuple(tree_g["lo"][:, c].tolist()), tuple(tree_g["hi"][:, c].tolist()))
                     for c in sel)
        want = sorted((tree_o.begin[c], tree_o.end[c], tuple(float(v) for v in tree_o.lo[c]),
                       tuple(float(v) for v in tree_o.hi[c])) for c in range(tree_o.num_clusters))
        assert got == want, i
    for typ in range(4):
        t, s = lists[typ]
        sel = (gt["begin"][t] >= b) & (gt["begin"][t] < e)
        got = sorted(((int(gt["begin"][x]) - b, int(gt["end"][x]) - b),
                      (int(gs["begin"][y]) - b, int(gs["end"][y]) - b))
                     for x, y in zip(t[sel], s[sel]))
        want = sorted(((samp.tt.begin[x], samp.tt.end[x]), (samp.st.begin[y], samp.st.end[y]))
                      for x, y in samp.lists[typ])
        assert got == want, (i, typ)
    ref = samp.potentials(idx)
    got = phi64[b + idx]
    assert rel_l2(ref, got) <= 1e-12, i
    assert max_rel(ref, got) <= 1e-10, i


def test_batched_workload_full_size_against_the_oracle():
    probs = W.batched_problems(count=BATCHED["count"], seed=BATCHED["seed"])
    pts = np.concatenate([p["points"] for p in probs], axis=1)
    q = np.concatenate([p["charges"] for p in probs])
    off = np.cumsum([0] + [p["points"].shape[1] for p in probs])
    kernels = [p["kernel"] for p in probs]
    kappas = [p["kappa"] for p in probs]
    kw = dict(n=BATCHED["n"], theta=BATCHED["theta"], N0=BATCHED["N0"], M0=BATCHED["M0"])
    dt, dq = to_dev(pts), to_dev(q)
    with B.Plan.batch(dt, off, dt, off, dq, kernels, kappas, precision=B.FP64, **kw) as plan:
        phi64 = plan.compute().cpu().numpy()
        plan.check_error()
        gt, gs = plan.export_tree(0), plan.export_tree(1)
        lists = plan.export_lists()
    with B.Plan.batch(dt, off, dt, off, dq, kernels, kappas, precision=B.FP32_BULK, **kw) as plan:
        phi32 = plan.compute().cpu().numpy()
        plan.check_error()
    del dt, dq

    worst = max(rel_l2(phi64[off[i]:off[i + 1]], phi32[off[i]:off[i + 1]])
                for i in range(len(probs)))
    assert worst <= 1e-6

    sizes = np.diff(off)
    rng = np.random.default_rng(99)
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    rest = np.setdiff1d(np.arange(len(probs)), pick)
    pick += [int(i) for i in rng.choice(rest, size=4, replace=False)]
    for i in sorted(pick):
        p = probs[i]
        samp = O.SampledBLDTT(p["points"], p["points"], p["charges"], kernel=p["kernel"],
                              kappa=p["kappa"], **kw)
        idx = np.sort(rng.choice(int(sizes[i]), size=16, replace=False))
        check_batched_problem(i, off, gt, gs, lists, phi64, samp, idx)
