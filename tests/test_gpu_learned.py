"""The learned selector on the GPU against the oracle (oracle/learned.py):
network outputs bit for bit, gradients and Adam within float rounding, pair
features bit for bit, pair-error labels, the selector's decisions (identical
list entries), and the multi-degree BLDTT's potentials."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import learned as L
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import gpu_to_oracle_index, rel_l2, run_gpu, to_dev

pytestmark = pytest.mark.gpu


def random_params(nout, seed, scale=1.0):
    """Seeded float32 master weights in the packed order of the C ABI."""
    rng = np.random.default_rng(seed)
    p = {}
    dims = [(64, 6), (64, 64), (64, 64), (nout, 64)]
    for l, (o, i) in enumerate(dims, start=1):
        p[f"W{l}"] = (rng.standard_normal((o, i)) * np.sqrt(2.0 / i) * (scale if l == 4 else 1.0)
                      ).astype(np.float32)
        p[f"b{l}"] = (rng.standard_normal(o) * 0.1).astype(np.float32)
    return p


def pack(p):
    return np.concatenate([np.concatenate([p[f"W{l}"].ravel(), p[f"b{l}"]]) for l in (1, 2, 3, 4)])


def unpack(flat, nout):
    dims = [(64, 6), (64, 64), (64, 64), (nout, 64)]
    out, o = {}, 0
    for l, (a, b) in enumerate(dims, start=1):
        out[f"W{l}"] = flat[o:o + a * b].reshape(a, b)
        o += a * b
        out[f"b{l}"] = flat[o:o + a]
        o += a
    return out


def test_param_count_matches_layout():
    for m in (1, 3, 6, 8):
        assert B.param_count(m) == pack(random_params(3 * m, 0)).size
    assert B.param_count(0) == -1 and B.param_count(9) == -1


def test_forward_is_bit_exact():
    nout = 12
    p = random_params(nout, 1)
    X = np.random.default_rng(2).uniform(0, 1.2, (3000, 6))
    want, _ = L.forward_bf16(p, X)
    got = B.mlp_forward(torch.from_numpy(pack(p)).cuda(), nout,
                        torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()
    assert np.array_equal(got, want)


def test_gradients_and_adam_match_the_oracle():
    nout = 9
    p = random_params(nout, 3)
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 1, (700, 6))
    T = rng.standard_normal((700, nout)).astype(np.float32)
    mask = (rng.uniform(size=(700, nout)) < 0.7).astype(np.float32)
    y, cache = L.forward_bf16(p, X)
    loss, gy = L.loss_and_grad_out(y, T, mask)
    g = L.backward(cache, gy)
    flat = torch.from_numpy(pack(p)).cuda()
    grads, gl = B.mlp_gradients(flat, nout, torch.from_numpy(X.astype(np.float32)).cuda(),
                                torch.from_numpy(T).cuda(), torch.from_numpy(mask).cuda())
    gg = unpack(grads.cpu().numpy().astype(np.float64), nout)
    assert abs(gl.item() - loss) <= 1e-5 * loss
    for k in g:
        scale = np.abs(g[k]).max()
        assert np.abs(gg[k] - g[k]).max() <= 2e-4 * scale, k
    # one Adam step from zero moments
    m = torch.zeros_like(flat)
    v = torch.zeros_like(flat)
    B.mlp_adam(flat, m, v, grads, step=1, lr=1e-3)
    z = {k: np.zeros_like(vv, dtype=np.float64) for k, vv in gg.items()}
    want, _, _ = L.adam_step({k: vv.astype(np.float64) for k, vv in p.items()}, gg, z, z, 1, 1e-3)
    got = unpack(flat.cpu().numpy().astype(np.float64), nout)
    for k in want:
        assert np.abs(got[k] - want[k]).max() <= 1e-6, k


@pytest.fixture(scope="module")
def small_problem():
    t, s, q = W.make_problem("uniform", 3000, 2600, seed=21, sources_kind="plummer")
    return t, s, q


def _oracle_trees(t, s, leaf):
    return O.build_tree(t, leaf), O.build_tree(s, leaf)


def test_pair_features_bit_exact_and_errors_match(small_problem):
    t, s, q = small_problem
    kw = dict(kernel=B.COULOMB, kappa=0.0, n=4, theta=0.7, N0=60, M0=60)
    phi, plan = run_gpu(t, s, q, precision=B.FP64, **kw)
    with plan:
        gt, gs = plan.export_tree(0), plan.export_tree(1)
        tt, st = _oracle_trees(t, s, 60)
        mt, ms = gpu_to_oracle_index(gt, tt), gpu_to_oracle_index(gs, st)
        rng = np.random.default_rng(5)
        # pairs of similar levels, some well separated, some not
        cand = [(a, b) for a in range(gt["begin"].size) for b in range(gs["begin"].size)
                if abs(int(gt["level"][a]) - int(gs["level"][b])) <= 1]
        pick = [cand[i] for i in rng.choice(len(cand), size=300, replace=False)]
        pairs = torch.tensor(pick, dtype=torch.int32, device="cuda")
        f = B.pair_features(plan, pairs).cpu().numpy()
        for (a, b), fg in zip(pick, f):
            fo = L.pair_features(tt, mt[a], st, ms[b], 0.0)
            if fo is None:
                assert np.all(np.isnan(fg))
            else:
                assert np.array_equal(fg, fo)
        # labels on separated pairs with small target clusters (every target sampled)
        sep = [(a, b) for (a, b), fg in zip(pick, f)
               if not np.isnan(fg[0]) and fg[4] < 0.8 and gt["end"][a] - gt["begin"][a] <= 64][:12]
        assert len(sep) >= 4
        degrees = [2, 4, 6]
        err = B.pair_errors(plan, torch.tensor(sep, dtype=torch.int32, device="cuda"), degrees,
                            samples=64).cpu().numpy()
        for (a, b), eg in zip(sep, err):
            ta, sb = mt[a], ms[b]
            pos = np.arange(tt.begin[ta], tt.end[ta])
            eo = L.pair_errors(t, s, q, tt, st, ta, sb, degrees, pos)
            big = eo > 1e-11
            assert np.all(np.abs(np.log10(eg[big]) - np.log10(eo[big])) <= 1e-2)
            assert np.all(eg[~big] <= 1e-10)


def _selector_plan(t, s, q, sel_np, precision, kernel=B.COULOMB, kappa=0.0, theta=0.7, leaf=60):
    return B.Plan.learned(to_dev(t), to_dev(s), to_dev(q), sel_np, kernel=kernel, kappa=kappa,
                          theta=theta, N0=leaf, M0=leaf, precision=precision)


def _class_keys(plan, gt, gs, nclass):
    lists = plan.export_lists(nclass)
    out = []
    for tg, sg in lists:
        out.append(sorted(((int(gt["begin"][a]), int(gt["end"][a])),
                           (int(gs["begin"][b]), int(gs["end"][b]))) for a, b in zip(tg, sg)))
    return out


def _oracle_class_keys(tt, st, entries, nclass):
    out = [[] for _ in range(nclass)]
    for c, a, b in entries:
        out[c].append(((tt.begin[a], tt.end[a]), (st.begin[b], st.end[b])))
    return [sorted(x) for x in out]


def test_mac_fallback_plan_equals_the_standard_plan(small_problem):
    """No network: the MAC at the highest degree decides every pair; extra
    lower degrees carry proxies but no entries, so the potentials are those of
    the standard plan bit for bit."""
    t, s, q = small_problem
    for precision in (B.FP64, B.FP32_BULK):
        ref, p0 = run_gpu(t, s, q, precision=precision, kernel=B.COULOMB, n=5, theta=0.7, N0=60,
                          M0=60)
        p0.close()
        with _selector_plan(t, s, q, B.Selector([3, 5]), precision) as pl:
            got = pl.compute().cpu().numpy()
            pl.check_error()
            nclass, degrees = pl.list_classes()
            assert (nclass, degrees) == (7, [3, 5])
            counts = [len(a) for a, _ in pl.export_lists()]
            assert counts[1] == counts[2] == counts[3] == 0
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("kernel,kappa", [(B.COULOMB, 0.0), (B.YUKAWA, 0.8)])
def test_random_selector_lists_and_potentials_match_the_oracle(small_problem, kernel, kappa):
    t, s, q = small_problem
    degrees = [2, 3, 5]
    p = random_params(9, 10, scale=4.0)
    lo, hi = np.full(6, -10.0, np.float32), np.full(6, 10.0, np.float32)
    lo[4] = 0.05                      # pairs closer than this fall back to the MAC
    sel_np = B.Selector(degrees, pack(p), lo, hi, log10_budget=0.0)
    tt, st = _oracle_trees(t, s, 60)
    osel = L.Selector(p, degrees, 0.0, lo, hi, theta_fallback=0.7)
    entries = L.learned_traversal(tt, st, osel, kappa)
    classes = {c for c, _, _ in entries}
    assert len(classes) >= 5
    ref = L.bldtt_entries(t, s, q, tt, st, entries, degrees, kernel=kernel, kappa=kappa)
    for precision, tol in ((B.FP64, 1e-12), (B.FP32_BULK, 1e-6)):
        with _selector_plan(t, s, q, sel_np, precision, kernel=kernel, kappa=kappa) as pl:
            got = pl.compute().cpu().numpy()
            pl.check_error()
            gt, gs = pl.export_tree(0), pl.export_tree(1)
            assert _class_keys(pl, gt, gs, 10) == _oracle_class_keys(tt, st, entries, 10)
        assert rel_l2(ref, got) <= tol, precision
