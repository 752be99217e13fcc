"""Parity at the full size of the benchmarked workload: 1E6 uniform particles
in [-1,1]^3, Coulomb, n=8, theta=0.7, leaves of 2000, in the launch
configuration the benchmark times.

Exact: both trees and all four interaction lists.  Sampled: FP64 potentials
at targets the oracle evaluates one by one (Eq. (19) along each target's chain
of clusters).  Whole output: FP32_BULK against FP64 (the benchmark metric),
and both against the FP64 direct sum on sampled targets."""
import numpy as np
import pytest

import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import (gpu_list_keys, gpu_tree_table, oracle_list_keys, oracle_tree_table,
                       same_leaf_members, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    cfg = W.CONFIGS["uniform_n1e6"]
    tgt, src, q = W.make_problem(cfg["kind"], cfg["M"], seed=cfg["seed"])
    kw = dict(kernel=cfg["kernel"], kappa=cfg["kappa"], n=cfg["n"], theta=cfg["theta"],
              N0=cfg["N0"], M0=cfg["M0"])
    dt, dq = to_dev(tgt), to_dev(q)
    p64 = B.Plan(dt, dt, dq, precision=B.FP64, **kw)
    phi64 = p64.compute().cpu().numpy()
    p64.check_error()
    p32 = B.Plan(dt, dt, dq, precision=B.FP32_BULK, **kw)
    phi32 = p32.compute().cpu().numpy()
    p32.check_error()
    samp = O.SampledBLDTT(tgt, tgt, q, **kw)
    yield dict(tgt=tgt, q=q, kw=kw, p64=p64, p32=p32, phi64=phi64, phi32=phi32, samp=samp, dt=dt,
               dq=dq)
    p64.close()
    p32.close()


def test_trees_and_lists_exact(full):
    samp, p = full["samp"], full["p32"]
    gt, gs = p.export_tree(0), p.export_tree(1)
    assert same_leaf_members(gt, samp.tt)
    assert gpu_tree_table(gt) == oracle_tree_table(samp.tt)
    assert gpu_tree_table(gs) == oracle_tree_table(samp.st)
    assert same_leaf_members(gs, samp.st)
    assert gpu_list_keys(gt, gs, p.export_lists()) == oracle_list_keys(samp.tt, samp.st, samp.lists)


def test_sampled_fp64_potentials(full):
    rng = np.random.default_rng(2024)
    idx = rng.choice(full["tgt"].shape[1], size=40, replace=False)
    ref = full["samp"].potentials(idx)
    got = full["phi64"][idx]
    assert O.relative_l2_error(ref, got) <= 1e-12
    assert O.max_norm_error(ref, got) <= 1e-10


# Max-norm of FP32_BULK against FP64, relative to max|phi|: the same 1e-5 as
# on the small parity cases (the tolerance proposed for the metric beside its
# rel-l2 budget of 1e-6).  Why it holds at this size: every term whose pair
# distance r is below tau = 0.3|e| of a particle chunk (|e| its
# half-diagonal, ~0.1 here) takes the frame residuals and is back at a few u
# (u = 2^-24); the rest carry a relative error <= 2 u rho/tau ~ 2.4e-7 each
# (rho ~ 6e-2 the chunk's half size), and these errors have random signs, so
# a target's error grows like the square root of its ~1e5 near-field terms,
# not like their sum.  The measured value is printed.
FP32_MAX_FULL = 1e-5


def test_fp32_bulk_against_fp64_and_direct(full):
    err = O.relative_l2_error(full["phi64"], full["phi32"])
    mx = O.max_norm_error(full["phi64"], full["phi32"])
    print(f"uniform_n1e6: FP32 vs FP64 rel-l2 {err:.3e}, max-norm {mx:.3e}")
    assert err <= 1e-6
    assert mx <= FP32_MAX_FULL
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(full["tgt"].shape[1], size=2000, replace=False))
    ts = to_dev(full["tgt"][:, idx])
    direct = B.direct_sum(ts, full["dt"], full["dq"]).cpu().numpy()
    e64 = O.relative_l2_error(direct, full["phi64"][idx])
    e32 = O.relative_l2_error(direct, full["phi32"][idx])
    print(f"uniform_n1e6 vs direct sum (2000 targets): FP64 {e64:.3e}, FP32 {e32:.3e}")
    # Sec. 4.1 reports 3.67E-8 at this size; FP32 evaluation adds at most ~1E-6.
    assert 3e-9 <= e64 <= 3e-7
    assert e32 <= e64 + 1e-6


def test_unequal_yukawa_full_size():
    """The unequal-set workload at its full size (1E7 uniform targets, 5E6
    Plummer sources, Yukawa kappa=0.5, n=7, theta=0.8, leaves 2000) in the
    benchmarked configuration: FP32_BULK against the FP64 BLDTT on the whole
    output, and both against the FP64 direct sum on 2000 sampled targets."""
    cfg = W.CONFIGS["unequal_yukawa"]
    tgt, src, q = W.make_problem(cfg["kind"], cfg["M"], cfg["N"], seed=cfg["seed"],
                                 sources_kind=cfg["sources_kind"])
    kw = dict(kernel=cfg["kernel"], kappa=cfg["kappa"], n=cfg["n"], theta=cfg["theta"],
              N0=cfg["N0"], M0=cfg["M0"])
    dt, ds, dq = to_dev(tgt), to_dev(src), to_dev(q)
    phi = {}
    for prec in (B.FP64, B.FP32_BULK):
        with B.Plan(dt, ds, dq, precision=prec, **kw) as plan:
            phi[prec] = plan.compute().cpu().numpy()
            plan.check_error()
    err = O.relative_l2_error(phi[B.FP64], phi[B.FP32_BULK])
    assert err <= 1e-6
    idx = np.sort(np.random.default_rng(8).choice(tgt.shape[1], size=2000, replace=False))
    direct = B.direct_sum(to_dev(tgt[:, idx]), ds, dq, cfg["kernel"], cfg["kappa"]).cpu().numpy()
    e64 = O.relative_l2_error(direct, phi[B.FP64][idx])
    e32 = O.relative_l2_error(direct, phi[B.FP32_BULK][idx])
    print(f"unequal_yukawa: FP32 vs FP64 {err:.2e}, FP64 vs direct {e64:.2e}, FP32 vs direct {e32:.2e}")
    assert e64 <= 1e-5                # the method's error at n=7, theta=0.8
    assert e32 <= e64 + 1e-6
