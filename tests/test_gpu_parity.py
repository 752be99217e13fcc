"""GPU path against the oracle, stage by stage, through the C ABI.

Tolerances: trees, memberships and interaction lists must match exactly;
FP64 proxy charges / proxy potentials to 1e-12 of their largest magnitude;
potentials FP64 to rel-l2 1e-12 and max-norm 1e-10, FP32_BULK to rel-l2 1e-6
and max-norm 1e-5.  The FP32 budget: each evaluation carries ~u = 6e-8 from
the rsqrt plus the rounding of coordinates in a chunk's frame (at most ~13u
relative in r for targets beyond the close-pair distance of the chunk, a few
u with the frame residuals inside it), and chunk sums of 128 terms per lane
add ~u sqrt(128); summed over a target's ~1e4-1e5 terms with random signs this
stays well below 1e-6 (measured 1-3e-7), and the worst single term stays below
1e-5 of the largest potential on these small cases."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import (gpu_list_keys, gpu_to_oracle_index, gpu_tree_table, max_rel, oracle_list_keys,
                       oracle_tree_table, rel_l2, run_gpu, same_leaf_members, to_dev)

pytestmark = pytest.mark.gpu

FP64_L2, FP64_MAX = 1e-12, 1e-10
FP32_L2, FP32_MAX = 1e-6, 1e-5

CASES = [
    # name, problem kwargs, method kwargs
    ("uniform_eq", dict(kind="uniform", n_targets=6000, seed=1),
     dict(kernel=B.COULOMB, n=4, theta=0.7, N0=150, M0=150)),
    ("plummer_unequal_yukawa", dict(kind="uniform", n_targets=5000, n_sources=7000, seed=2,
                                    sources_kind="plummer"),
     dict(kernel=B.YUKAWA, kappa=0.5, n=3, theta=0.8, N0=60, M0=90)),
    ("sphere_small_leaves", dict(kind="sphere", n_targets=4000, seed=3),
     dict(kernel=B.COULOMB, n=2, theta=0.6, N0=10, M0=7)),
    ("gaussian_n6", dict(kind="gaussian", n_targets=3000, n_sources=2500, seed=4),
     dict(kernel=B.YUKAWA, kappa=1.7, n=6, theta=0.9, N0=400, M0=300)),
    ("oscillatory_pi", dict(kind="uniform", n_targets=4000, seed=15),
     dict(kernel=B.OSCILLATORY, kappa=float(np.pi), n=4, theta=0.7, N0=60, M0=60)),
    ("regularized_coulomb", dict(kind="sphere", n_targets=3500, n_sources=4000, seed=16,
                                 sources_kind="uniform"),
     dict(kernel=B.REG_COULOMB, kappa=0.005, n=3, theta=0.8, N0=40, M0=40)),
    ("cc_pp_only_variant", dict(kind="uniform", n_targets=5000, n_sources=4500, seed=17,
                                sources_kind="plummer"),
     dict(kernel=B.COULOMB, n=2, theta=0.7, N0=20, M0=20, variant=B.VARIANT_CC_PP_ONLY)),
]


def problem(pkw):
    pkw = dict(pkw)
    kind = pkw.pop("kind")
    return W.make_problem(kind, **pkw)


@pytest.mark.parametrize("name,pkw,mkw", CASES, ids=[c[0] for c in CASES])
def test_trees_lists_and_potentials_match_oracle(name, pkw, mkw):
    tgt, src, q = problem(pkw)
    ref = O.bldtt(tgt, src, q, **mkw)
    if mkw.get("variant") == B.VARIANT_CC_PP_ONLY:
        assert len(ref.lists[O.PC]) == 0 and len(ref.lists[O.CP]) == 0 and len(ref.lists[O.CC]) > 0
    phi, plan = run_gpu(tgt, src, q, precision=B.FP64, **mkw)
    with plan:
        gt, gs = plan.export_tree(0), plan.export_tree(1)
        # trees: identical clusters; same leaf members
        assert same_leaf_members(gt, ref.ttree)
        assert same_leaf_members(gs, ref.stree)
        assert gpu_tree_table(gt) == oracle_tree_table(ref.ttree)
        assert gpu_tree_table(gs) == oracle_tree_table(ref.stree)
        # interaction lists: identical sets per type
        assert gpu_list_keys(gt, gs, plan.export_lists()) == oracle_list_keys(ref.ttree, ref.stree,
                                                                              ref.lists)
        # proxy charges and proxy potentials
        ms = gpu_to_oracle_index(gs, ref.stree)
        mt = gpu_to_oracle_index(gt, ref.ttree)
        qh = plan.proxy_charges()
        assert np.max(np.abs(qh - ref.qhat[ms])) <= 1e-12 * np.max(np.abs(ref.qhat))
        pt = plan.proxy_potentials()
        scale = max(np.max(np.abs(ref.phit)), 1e-300)
        assert np.max(np.abs(pt - ref.phit[mt])) <= 1e-12 * scale
        st = plan.stats()
        assert st["list_entries"] == [len(l) for l in ref.lists]
        assert st["interactions"] == [float(v) for v in ref.counts]
    assert rel_l2(ref.phi, phi) <= FP64_L2
    assert max_rel(ref.phi, phi) <= FP64_MAX
    phi32, plan32 = run_gpu(tgt, src, q, precision=B.FP32_BULK, **mkw)
    plan32.close()
    assert rel_l2(ref.phi, phi32) <= FP32_L2
    assert max_rel(ref.phi, phi32) <= FP32_MAX


@pytest.mark.parametrize("precision,tol", [(B.FP64, 1e-12), (B.FP32_BULK, 1e-6)])
def test_degree_two_kernel_equals_direct_sum(precision, tol):
    """Every approximation is exact for the test kernel (n >= 2)."""
    tgt, src, q = W.make_problem("uniform", 4000, 3500, seed=6, sources_kind="plummer")
    ref = O.direct_sum(tgt, src, q, O.TEST_POLY)
    phi, plan = run_gpu(tgt, src, q, precision=precision, kernel=B.TEST_POLY, n=2, theta=0.7,
                        N0=20, M0=20)
    with plan:
        assert all(c > 0 for c in plan.stats()["list_entries"])
    assert rel_l2(ref, phi) <= tol


@pytest.mark.parametrize("kernel,kappa", [(B.COULOMB, 0.0), (B.YUKAWA, 0.9)])
def test_theta_zero_is_direct_sum(kernel, kappa):
    tgt, src, q = W.make_problem("sphere", 2500, 2000, seed=8, sources_kind="uniform")
    ref = O.direct_sum(tgt, src, q, kernel, kappa)
    phi, plan = run_gpu(tgt, src, q, precision=B.FP64, kernel=kernel, kappa=kappa, n=3, theta=0.0,
                        N0=64, M0=64)
    plan.close()
    assert rel_l2(ref, phi) <= 1e-13


def test_device_direct_sum_matches_oracle():
    tgt, src, q = W.make_problem("uniform", 1500, 2100, seed=9, sources_kind="plummer")
    src[:, :40] = tgt[:, :40]          # coincident pairs contribute nothing
    for kernel, kappa in ((B.COULOMB, 0.0), (B.YUKAWA, 0.5), (B.TEST_POLY, 0.0)):
        ref = O.direct_sum(tgt, src, q, kernel, kappa)
        got = B.direct_sum(to_dev(tgt), to_dev(src), to_dev(q), kernel, kappa).cpu().numpy()
        assert rel_l2(ref, got) <= 1e-14


@pytest.mark.parametrize("name,pts", [
    ("single_target_single_source", None),
    ("all_identical", np.full((3, 700), 0.25)),
    ("flat_plane", None),
    ("duplicated_pairs", None),
    ("signed_zeros", None),
])
def test_degenerate_inputs(name, pts):
    rng = np.random.default_rng(11)
    if name == "single_target_single_source":
        tgt = np.array([[0.1], [0.2], [0.3]])
        src = np.array([[0.5], [0.2], [0.3]])
        q = np.array([2.0])
        kw = dict(n=3, theta=0.7, N0=1, M0=1)
    elif name == "all_identical":
        tgt = src = pts
        q = rng.uniform(-1, 1, 700)
        kw = dict(n=4, theta=0.7, N0=5, M0=5)
    elif name == "flat_plane":
        tgt = rng.uniform(-1, 1, (3, 3000))
        tgt[2] = 0.0
        src = tgt
        q = rng.uniform(-1, 1, 3000)
        kw = dict(n=4, theta=0.7, N0=40, M0=40)
    elif name == "signed_zeros":
        # root box [-1, 1]^3, so the first midpoints are exactly 0; a fifth of
        # the coordinates are -0.0 or +0.0, which FP64 compares as equal (the
        # tree's integer keys must too)
        tgt = rng.uniform(-1, 1, (3, 2000))
        tgt[:, :6] = [[-1, 1, 0, 0, 0, 0], [0, 0, -1, 1, 0, 0], [0, 0, 0, 0, -1, 1]]
        zero = rng.random((3, 2000)) < 0.2
        neg = rng.random((3, 2000)) < 0.5
        zero[:, :6] = False
        tgt[zero & neg] = -0.0
        tgt[zero & ~neg] = 0.0
        assert np.signbit(tgt[zero & neg]).all()
        src = tgt
        q = rng.uniform(-1, 1, 2000)
        kw = dict(n=4, theta=0.7, N0=40, M0=40)
    else:
        base = rng.uniform(-1, 1, (3, 1500))
        tgt = np.concatenate([base, base], axis=1)
        src = tgt
        q = rng.uniform(-1, 1, 3000)
        kw = dict(n=3, theta=0.75, N0=30, M0=30)
    ref = O.bldtt(tgt, src, q, **kw)
    for prec, tol in ((B.FP64, FP64_L2), (B.FP32_BULK, FP32_L2)):
        phi, plan = run_gpu(tgt, src, q, precision=prec, **kw)
        with plan:
            gt = plan.export_tree(0)
            assert same_leaf_members(gt, ref.ttree)
            assert gpu_tree_table(gt) == oracle_tree_table(ref.ttree)
        if np.all(ref.phi == 0):
            assert np.all(phi == 0)
        else:
            assert rel_l2(ref.phi, phi) <= tol


def test_set_charges_and_solve_host():
    tgt, src, q = W.make_problem("uniform", 3000, seed=12)
    kw = dict(kernel=B.COULOMB, n=5, theta=0.7, N0=100, M0=100)
    q2 = np.random.default_rng(5).uniform(-1, 1, 3000)
    ref1 = O.bldtt(tgt, src, q, **kw).phi
    ref2 = O.bldtt(tgt, src, q2, **kw).phi
    phi, plan = run_gpu(tgt, src, q, precision=B.FP64, **kw)
    with plan:
        plan.set_charges(to_dev(q2))
        phi2 = plan.compute().cpu().numpy()
        phi1b = None
        plan.set_charges(to_dev(q))
        phi1b = plan.compute().cpu().numpy()
    assert rel_l2(ref1, phi) <= FP64_L2
    assert rel_l2(ref2, phi2) <= FP64_L2
    assert np.array_equal(phi, phi1b)            # deterministic
    host_phi, stats = B.solve_host(tgt, tgt, q, precision=B.FP64, **kw)
    assert np.array_equal(host_phi, phi)
    assert stats["launches_compute"] > 0


@pytest.mark.parametrize("level_by_level", [False, True])
def test_invalid_inputs_on_device(level_by_level, monkeypatch):
    if level_by_level:
        monkeypatch.setenv("BLDTT_LEVEL_BY_LEVEL", "1")
    tgt, src, q = W.make_problem("uniform", 500, seed=13)
    bad = tgt.copy()
    bad[1, 17] = np.nan
    with pytest.raises(B.BLDTTError) as e:
        B.Plan(to_dev(bad), to_dev(src), to_dev(q), n=3, N0=20, M0=20)
    assert e.value.status == 1
    qb = q.copy()
    qb[3] = np.inf
    with pytest.raises(B.BLDTTError) as e:
        B.Plan(to_dev(tgt), to_dev(src), to_dev(qb), n=3, N0=20, M0=20)
    assert e.value.status == 1
    # a bad source coordinate, found by the source-tree build
    bad_src = src.copy()
    bad_src[2, 400] = -np.inf
    with pytest.raises(B.BLDTTError) as e:
        B.Plan(to_dev(tgt), to_dev(bad_src), to_dev(q), n=3, N0=20, M0=20)
    assert e.value.status == 1
    # the library stays usable after the errors
    phi, plan = run_gpu(tgt, src.copy(), q, n=3, theta=0.7, N0=20, M0=20, precision=B.FP64)
    plan.close()
    assert np.all(np.isfinite(phi))


SET_UP_CASES = [CASES[0], CASES[1], CASES[2], CASES[6]]


@pytest.mark.parametrize("name,pkw,mkw", SET_UP_CASES, ids=[c[0] for c in SET_UP_CASES])
def test_cooperative_set_up_equals_level_by_level(name, pkw, mkw, monkeypatch):
    """The tree build and the traversal in one cooperative launch each give the
    trees, lists and potentials of the level-by-level host loops bit for bit
    (BLDTT_LEVEL_BY_LEVEL=1 selects the loops)."""
    tgt, src, q = problem(pkw)

    def run():
        phi, plan = run_gpu(tgt, src, q, precision=B.FP64, **mkw)
        with plan:
            trees = [plan.export_tree(k) for k in (0, 1)]
            lists = plan.export_lists()
            st = plan.stats()
        return phi, trees, lists, st

    phi_c, trees_c, lists_c, st_c = run()
    monkeypatch.setenv("BLDTT_LEVEL_BY_LEVEL", "1")
    phi_l, trees_l, lists_l, st_l = run()
    assert st_l["launches_setup"] > st_c["launches_setup"]     # the loops did run
    for a, b in zip(trees_c, trees_l):
        assert a.keys() == b.keys()
        for k in a:
            assert np.asarray(a[k]).tobytes() == np.asarray(b[k]).tobytes(), k
    for (tc, sc), (tl, sl) in zip(lists_c, lists_l):
        assert np.array_equal(tc, tl) and np.array_equal(sc, sl)
    assert np.array_equal(phi_c, phi_l)


def test_set_up_regrowth_gives_the_same_plan(monkeypatch):
    """The cooperative launches' capacity paths: a tree build that starts with
    room for 64 clusters (grown and resumed level by level), a traversal whose
    buffers overflow at least once (relaunched with doubled buffers), and one
    that never fits (three launches, then the level loop) all give the default
    plan's trees, lists and potentials bit for bit."""
    name, pkw, mkw = CASES[2]                     # sphere, leaves of 7: ~1000 clusters
    tgt, src, q = problem(pkw)

    def run():
        phi, plan = run_gpu(tgt, src, q, precision=B.FP64, **mkw)
        with plan:
            trees = [plan.export_tree(k) for k in (0, 1)]
            lists = plan.export_lists()
            st = plan.stats()
        return phi, trees, lists, st

    def same(a, b):
        assert np.array_equal(a[0], b[0])
        for ta, tb in zip(a[1], b[1]):
            for k in ta:
                assert np.asarray(ta[k]).tobytes() == np.asarray(tb[k]).tobytes(), k
        for (tc, sc), (tl, sl) in zip(a[2], b[2]):
            assert np.array_equal(tc, tl) and np.array_equal(sc, sl)

    base = run()
    assert base[3]["num_target_clusters"] > 256
    entries = int(sum(base[3]["list_entries"]))
    with monkeypatch.context() as m:
        m.setenv("BLDTT_TREE_CAPACITY", "8")
        grown = run()
    same(base, grown)
    assert grown[3]["launches_setup"] > base[3]["launches_setup"]      # resumed launches
    with monkeypatch.context() as m:                # 3 E/8 entries overflow at least once
        m.setenv("BLDTT_TRAVERSAL_CAPACITY", str(3 * entries // 8))
        relaunched = run()
    same(base, relaunched)
    assert relaunched[3]["launches_setup"] >= base[3]["launches_setup"] + 1
    with monkeypatch.context() as m:
        m.setenv("BLDTT_TRAVERSAL_CAPACITY", "1")
        looped = run()
    same(base, looped)
    assert looped[3]["launches_setup"] > base[3]["launches_setup"] + 2


def test_plans_on_two_host_threads():
    """Plans set up and computed at the same time from two host threads, each
    on its own stream, share the library's device memory pool and pinned read
    slots; each gives the result it gives alone, bit for bit."""
    import threading
    cases = [CASES[0], CASES[1]]
    inputs = [problem(pkw) for _, pkw, _ in cases]
    alone = []
    for (_, _, mkw), (tgt, src, q) in zip(cases, inputs):
        phi, plan = run_gpu(tgt, src, q, precision=B.FP32_BULK, **mkw)
        plan.close()
        alone.append(phi)
    dev = [(to_dev(t), to_dev(s_), to_dev(q)) for t, s_, q in inputs]
    torch.cuda.synchronize()
    out = [[None] * 3 for _ in cases]
    errors = []

    def work(i):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                for r in range(3):
                    with B.Plan(*dev[i], precision=B.FP32_BULK, stream=stream, **cases[i][2]) as plan:
                        phi = torch.empty(plan.M, dtype=torch.float64, device="cuda")
                        plan.compute(phi, stream=stream)
                        stream.synchronize()
                        out[i][r] = phi.cpu().numpy()
        except Exception as e:   # reported on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in range(len(cases)):
        for r in range(3):
            assert np.array_equal(out[i][r], alone[i]), (i, r)


def test_plain_fp64_workload_full_size():
    """The 2E4-particle plain FP64 workload (n=4, theta=0.7, leaves of 500):
    GPU FP64 equals the oracle BLDTT, and both are within the expected
    approximation error of the direct sum."""
    cfg = W.CONFIGS["plain_fp64_n2e4"]
    tgt, src, q = W.make_problem(cfg["kind"], cfg["M"], seed=cfg["seed"])
    kw = dict(kernel=cfg["kernel"], kappa=cfg["kappa"], n=cfg["n"], theta=cfg["theta"],
              N0=cfg["N0"], M0=cfg["M0"])
    ref = O.bldtt(tgt, src, q, **kw)
    direct = O.direct_sum(tgt, src, q)
    phi, plan = run_gpu(tgt, src, q, precision=B.FP64, **kw)
    plan.close()
    assert rel_l2(ref.phi, phi) <= FP64_L2
    assert max_rel(ref.phi, phi) <= FP64_MAX
    err = rel_l2(direct, phi)
    assert err == pytest.approx(rel_l2(direct, ref.phi), rel=1e-6)
    assert err < 1e-4


def test_plans_release_their_memory():
    """Set-ups and destroys in a loop (shared and separate trees, a batch, a
    set-up that fails on a non-finite source) leave the device's free memory
    where it was: every plan's arrays go back to the library's pool, whose
    reserve stays the same from one cycle to the next."""
    tgt, src, q = W.make_problem("uniform", 60_000, 40_000, seed=17, sources_kind="plummer")
    dt, ds, dq = to_dev(tgt), to_dev(src), to_dev(q)
    dq_t = to_dev(W.make_problem("uniform", 60_000, seed=17)[2])
    src_bad = src.copy()
    src_bad[1, 39_000] = np.nan
    ds_bad = to_dev(src_bad)
    torch.cuda.synchronize()

    def cycle():
        for prec in (B.FP64, B.FP32_BULK):
            with B.Plan(dt, dt, dq_t, n=5, theta=0.7, N0=200, M0=200, precision=prec) as p:
                p.compute()
            with B.Plan(dt, ds, dq, n=5, theta=0.7, N0=200, M0=200, precision=prec) as p:
                p.compute()
        off = [0, 30_000, 60_000]
        with B.Plan.batch(dt, off, dt, off, dq_t, [B.COULOMB, B.YUKAWA], [0.0, 0.5], n=4, N0=200,
                          M0=200) as p:
            p.compute()
        with pytest.raises(B.BLDTTError):    # a set-up that fails in the tree build frees all it took
            B.Plan(dt, ds_bad, dq, n=5, theta=0.7, N0=200, M0=200)
        torch.cuda.synchronize()

    cycle()                                   # first use: library state, module loading
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < 64 << 20, (free0, free1)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection without a fault: a wait on an mbarrier that nothing
    arrives on gives up after its limit with BLDTT_ETIMEOUT, and the device
    keeps computing correctly afterwards."""
    assert B.wait_probe(2_000_000) == 4          # BLDTT_ETIMEOUT, after 2 ms
    assert "gave up" in B.load_library().bldtt_last_error().decode()
    tgt, src, q = W.make_problem("uniform", 3000, seed=23)
    phi, plan = run_gpu(tgt, src, q, n=4, theta=0.0, N0=100, M0=100, precision=B.FP64)
    plan.close()
    assert rel_l2(O.direct_sum(tgt, src, q), phi) <= 1e-13
