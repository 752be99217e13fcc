"""The tensor-core (tcgen05) leaf contractions of FP32_BULK mode, Eq. (9)
(leaf proxy charges, Sec. 2.5) and Eq. (21) (leaf proxy potentials to the
particles, Sec. 2.7), against the oracle and against the SIMT kernels.

Tolerances: the proxy charges of the FP32 plan against the FP64 plan's,
relative l2 over all clusters <= 2e-6: each operand is held by its TF32 pair
to about 2^-22 (the TF32 rounding of the low part; all four products of the
pairs are taken), each 32-particle chunk is summed in FP32 (about
u sqrt(32) = 3.4e-7 of the chunk's root-sum-square), and the charges' mixed
signs make |qhat| smaller than the sum of |terms| by a further factor of a
few.  Potentials: the metric's 1e-6 relative l2 and 1e-5 max-norm against
the FP64 plan, and no more than twice (plus 1e-7) the SIMT engine's error on
the same problem."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import max_rel, rel_l2, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    dict(kind="uniform", M=20_000, N=None, sk=None, kernel=B.COULOMB, kappa=0.0, n=8, leaf=500),
    dict(kind="uniform", M=15_000, N=12_000, sk="plummer", kernel=B.YUKAWA, kappa=0.5, n=7, leaf=300),
    dict(kind="sphere", M=12_000, N=None, sk=None, kernel=B.COULOMB, kappa=0.0, n=3, leaf=150),
    dict(kind="gaussian", M=9_000, N=None, sk=None, kernel=B.COULOMB, kappa=0.0, n=10, leaf=1400),
    dict(kind="uniform", M=3_000, N=None, sk=None, kernel=B.COULOMB, kappa=0.0, n=1, leaf=37),
]


def _run(case, precision, engine=None):
    tgt, src, q = W.make_problem(case["kind"], case["M"], case["N"], seed=61, sources_kind=case["sk"])
    dt = to_dev(tgt)
    ds = dt if src is tgt else to_dev(src)
    with B.Plan(dt, ds, to_dev(q), kernel=case["kernel"], kappa=case["kappa"], n=case["n"],
                theta=0.7, N0=case["leaf"], M0=case["leaf"], precision=precision) as plan:
        if engine is not None:
            plan.set_pass_engine(engine, engine)
        phi = plan.compute().cpu().numpy()
        plan.check_error()
        used = (plan.pass_engine_used(0), plan.pass_engine_used(1))
        return phi, plan.proxy_charges(), used, (tgt, src, q)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['kind']}-n{c['n']}-leaf{c['leaf']}")
def test_tensor_leaf_passes_match_fp64_and_simt(case):
    phi64, qh64, used64, (tgt, src, q) = _run(case, B.FP64, B.PASS_TENSOR)
    assert used64 == (B.PASS_SIMT, B.PASS_SIMT)      # FP64 plans keep the SIMT kernels
    phis, qhs, useds, _ = _run(case, B.FP32_BULK, B.PASS_SIMT)
    phit, qht, usedt, _ = _run(case, B.FP32_BULK, B.PASS_TENSOR)
    assert useds == (B.PASS_SIMT,) * 2 and usedt == (B.PASS_TENSOR,) * 2
    e_q, e_qs = rel_l2(qh64.ravel(), qht.ravel()), rel_l2(qh64.ravel(), qhs.ravel())
    e_t, e_s = rel_l2(phi64, phit), rel_l2(phi64, phis)
    m_t = max_rel(phi64, phit)
    print(f"{case['kind']} n={case['n']}: qhat tensor {e_q:.2e}, simt {e_qs:.2e}; "
          f"phi tensor {e_t:.2e} (max {m_t:.2e}), simt {e_s:.2e}")
    assert e_q <= 2e-6
    assert e_t <= 1e-6 and m_t <= 1e-5
    assert e_t <= 2.0 * e_s + 1e-7


def test_tensor_leaf_passes_reproduce_the_degree_two_kernel():
    """With the test kernel of degree 2 per coordinate and n = 2 every
    approximation is exact, so the whole FP32 tensor-engine path must match
    the oracle's direct sum to FP32 rounding."""
    tgt, src, q = W.make_problem("uniform", 4_000, 3_500, seed=62, sources_kind="plummer")
    with B.Plan(to_dev(tgt), to_dev(src), to_dev(q), kernel=B.TEST_POLY, n=2, theta=0.7, N0=40,
                M0=40, precision=B.FP32_BULK) as plan:
        plan.set_pass_engine(B.PASS_TENSOR, B.PASS_TENSOR)
        phi = plan.compute().cpu().numpy()
        plan.check_error()
        assert plan.pass_engine_used(0) == plan.pass_engine_used(1) == B.PASS_TENSOR
        st = plan.stats()
    assert all(v > 0 for v in st["list_entries"])            # PP, PC, CP and CC all present
    ref = O.direct_sum(tgt, src, q, O.TEST_POLY)
    assert rel_l2(ref, phi) <= 1e-6


def test_tensor_engine_falls_back_beyond_eleven_points_and_shards_agree():
    tgt, _, q = W.make_problem("uniform", 30_000, seed=63)
    dt, dq = to_dev(tgt), to_dev(q)
    with B.Plan(dt, dt, dq, n=11, theta=0.7, N0=2000, M0=2000, precision=B.FP32_BULK) as plan:
        plan.set_pass_engine(B.PASS_TENSOR, B.PASS_TENSOR)
        assert plan.pass_engine_used(0) == plan.pass_engine_used(1) == B.PASS_SIMT   # 12 points
    # the default: upward on SIMT; downward on the tensor cores for target
    # leaves of 512 particles or more on average, else SIMT
    with B.Plan(dt, dt, dq, n=6, theta=0.7, N0=2000, M0=2000, precision=B.FP32_BULK) as plan:
        assert (plan.pass_engine_used(0), plan.pass_engine_used(1)) == (B.PASS_SIMT, B.PASS_TENSOR)
    with B.Plan(dt, dt, dq, n=6, theta=0.7, N0=300, M0=300, precision=B.FP32_BULK) as plan:
        assert (plan.pass_engine_used(0), plan.pass_engine_used(1)) == (B.PASS_SIMT, B.PASS_SIMT)
        plan.set_pass_engine(B.PASS_TENSOR, B.PASS_TENSOR)
        full = plan.compute()
        again = plan.compute()
        assert torch.equal(full.view(torch.int64), again.view(torch.int64))   # deterministic
        phi = torch.zeros_like(full)
        for k in range(3):
            plan.compute_shard(k, 3, phi)
        plan.check_error()
        assert torch.equal(phi.view(torch.int64), full.view(torch.int64))
    with pytest.raises(B.BLDTTError):
        with B.Plan(dt, dt, dq, n=3, theta=0.7, N0=300, M0=300) as plan:
            plan.set_pass_engine(B.PASS_SIMT, 7)
