"""Batched problems (bldtt_setup_batch): one plan, one persistent interaction
launch for the Coulomb and Yukawa problems together (one more per other
kernel) and one CUDA graph for many independent problems.

Each problem of the batch must equal the oracle's BLDTT of that problem alone
(trees, lists and potentials), and the batched potentials must equal, bit for
bit, those of a separate single-problem plan: batching only concatenates the
work, it does not change any summation order."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu

KW = dict(n=3, theta=0.7, N0=40, M0=40)


def small_batch(seed=40):
    """Nine problems of 300..3000 particles: cube / sphere / Plummer, some with
    separate source sets, Coulomb, Yukawa, oscillatory and regularized kernels."""
    rng = np.random.default_rng(seed)
    specs = [("uniform", None, B.COULOMB, 0.0), ("sphere", None, B.YUKAWA, 0.4),
             ("uniform", "plummer", B.YUKAWA, 1.7), ("plummer", None, B.COULOMB, 0.0),
             ("gaussian", "uniform", B.OSCILLATORY, float(np.pi)),
             ("uniform", None, B.REG_COULOMB, 0.005), ("sphere", "sphere", B.COULOMB, 0.0),
             ("uniform", None, B.YUKAWA, 0.1), ("uniform", "uniform", B.COULOMB, 0.0)]
    probs = []
    for i, (kind, skind, kern, kappa) in enumerate(specs):
        m = int(rng.integers(300, 3000))
        nsrc = None if skind is None else int(rng.integers(300, 3000))
        t, s, q = W.make_problem(kind, m, nsrc, seed=seed + i, sources_kind=skind)
        probs.append(dict(t=t, s=s, q=q, kernel=kern, kappa=kappa))
    return probs


def concat(probs):
    tg = np.concatenate([p["t"] for p in probs], axis=1)
    sg = np.concatenate([p["s"] for p in probs], axis=1)
    qg = np.concatenate([p["q"] for p in probs])
    to = np.cumsum([0] + [p["t"].shape[1] for p in probs])
    so = np.cumsum([0] + [p["s"].shape[1] for p in probs])
    return tg, sg, qg, to, so


def batch_plan(probs, precision):
    tg, sg, qg, to, so = concat(probs)
    plan = B.Plan.batch(to_dev(tg), to, to_dev(sg), so, to_dev(qg), [p["kernel"] for p in probs],
                        [p["kappa"] for p in probs], precision=precision, **KW)
    return plan, to, so


@pytest.fixture(scope="module")
def probs():
    return small_batch()


def test_batch_matches_oracle_per_problem(probs):
    plan, to, so = batch_plan(probs, B.FP64)
    with plan:
        phi = plan.compute().cpu().numpy()
        plan.check_error()
        gt, gs = plan.export_tree(0), plan.export_tree(1)
        lists = plan.export_lists()
        st = plan.stats()
    assert st["num_target_clusters"] == gt["begin"].size
    for i, p in enumerate(probs):
        ref = O.bldtt(p["t"], p["s"], p["q"], kernel=p["kernel"], kappa=p["kappa"], **KW)
        got = phi[to[i]:to[i + 1]]
        assert rel_l2(ref.phi, got) <= 1e-12, i
        # the problem's clusters, with particle ranges made problem-local
        for tree_g, tree_o, off in ((gt, ref.ttree, to), (gs, ref.stree, so)):
            sel = (tree_g["begin"] >= off[i]) & (tree_g["begin"] < off[i + 1])
            keys = sorted(zip((tree_g["begin"][sel] - off[i]).tolist(),
                              (tree_g["end"][sel] - off[i]).tolist()))
            assert keys == sorted(zip(tree_o.begin, tree_o.end)), i
        for typ in range(4):
            t, s = lists[typ]
            sel = (gt["begin"][t] >= to[i]) & (gt["begin"][t] < to[i + 1])
            got_keys = sorted(((int(gt["begin"][a]) - to[i], int(gt["end"][a]) - to[i]),
                               (int(gs["begin"][b]) - so[i], int(gs["end"][b]) - so[i]))
                              for a, b in zip(t[sel], s[sel]))
            want = sorted(((ref.ttree.begin[a], ref.ttree.end[a]),
                           (ref.stree.begin[b], ref.stree.end[b])) for a, b in ref.lists[typ])
            assert got_keys == want, (i, typ)


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_BULK])
def test_batch_equals_separate_plans_bitwise(probs, precision):
    plan, to, so = batch_plan(probs, precision)
    with plan:
        phi = plan.compute().cpu().numpy()
        plan.check_error()
    for i, p in enumerate(probs):
        with B.Plan(to_dev(p["t"]), to_dev(p["s"]), to_dev(p["q"]), kernel=p["kernel"],
                    kappa=p["kappa"], precision=precision, **KW) as single:
            ref = single.compute().cpu().numpy()
        assert np.array_equal(ref, phi[to[i]:to[i + 1]]), i


def test_graph_replay_and_autotune(probs):
    plan, to, so = batch_plan(probs, B.FP32_BULK)
    stream = torch.cuda.Stream()
    with plan:
        ref = plan.compute().cpu().numpy()
        phi = torch.empty(plan.M, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(2):
                phi.fill_(0.0)
                plan.compute_graph(phi, stream)
                stream.synchronize()
                assert np.array_equal(phi.cpu().numpy(), ref)
        layout = plan.autotune(phi)
        assert layout in range(6)                    # layouts instantiated for Coulomb
        table = plan.autotune_table()                # (launch, kernel, layout, ms) per tried layout
        first = [r for r in table if r[0] == 0]
        assert sorted(r[2] for r in first) == list(range(6))
        assert min(first, key=lambda r: r[3])[2] == layout
        assert np.array_equal(plan.compute().cpu().numpy(), ref)
        plan.check_error()
