"""Target-leaf sharding on one GPU: computing the shards of a plan one after
the other (bldtt_compute_shard) reproduces bldtt_compute's potentials bit for
bit, each shard writes exactly its own targets and leaves every other entry
untouched, and the shards' evaluation counts cover the plan's (shared
ancestors' proxy work is counted by every shard that computes it)."""
import numpy as np
import pytest
import torch

from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W
from _gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _bits(t):
    return t.cpu().numpy().view(np.uint64)


CASES = [
    dict(kind="uniform", M=200_000, N=None, sources_kind=None, kernel=B.COULOMB, kappa=0.0, n=6,
         theta=0.7, leaf=500, precision=B.FP32_BULK),
    dict(kind="uniform", M=120_000, N=90_000, sources_kind="plummer", kernel=B.YUKAWA, kappa=0.5,
         n=5, theta=0.8, leaf=300, precision=B.FP32_BULK),
    dict(kind="sphere", M=60_000, N=None, sources_kind=None, kernel=B.COULOMB, kappa=0.0, n=4,
         theta=0.7, leaf=200, precision=B.FP64),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['kind']}-{c['M']}-{c['precision']}")
def test_shards_reproduce_the_one_gpu_potentials(case):
    tgt, src, q = W.make_problem(case["kind"], case["M"], case["N"], seed=41,
                                 sources_kind=case["sources_kind"])
    dt = to_dev(tgt)
    ds = dt if src is tgt else to_dev(src)
    dq = to_dev(q)
    kw = dict(kernel=case["kernel"], kappa=case["kappa"], n=case["n"], theta=case["theta"],
              N0=case["leaf"], M0=case["leaf"], precision=case["precision"])
    with B.Plan(dt, ds, dq, **kw) as plan:
        full = plan.compute()
        plan.check_error()
        total = plan.stats()["computed_evaluations"]
        assert total == pytest.approx(sum(plan.stats()["interactions"]), rel=1e-12)
        for nshards in (2, 3, 7):
            phi = torch.full_like(full, float("nan"))
            written, evals = 0, 0.0
            for k in range(nshards):
                before = torch.isnan(phi)
                plan.compute_shard(k, nshards, phi)
                plan.check_error()
                evals += plan.stats()["computed_evaluations"]
                now = ~torch.isnan(phi) & before           # entries this shard wrote
                written += int(now.sum())
                # every entry written by an earlier shard is unchanged
                assert torch.equal(phi[~before].view(torch.int64), full[~before].view(torch.int64))
                assert torch.equal(phi[now].view(torch.int64), full[now].view(torch.int64))
            assert written == full.numel()
            assert np.array_equal(_bits(phi), _bits(full))
            assert total <= evals <= 1.25 * total
        # the one-GPU compute still gives the same bits after shards were run
        again = plan.compute()
        assert np.array_equal(_bits(again), _bits(full))


def test_shard_arguments_are_checked():
    tgt, _, q = W.make_problem("uniform", 5000, seed=42)
    dt, dq = to_dev(tgt), to_dev(q)
    with B.Plan(dt, dt, dq, n=3, theta=0.7, N0=100, M0=100) as plan:
        phi = torch.zeros(5000, dtype=torch.float64, device="cuda")
        for shard, nshards in ((2, 2), (-1, 2), (0, 0)):
            with pytest.raises(B.BLDTTError):
                plan.compute_shard(shard, nshards, phi)
        plan.compute_shard(0, 1, phi)          # one shard is the whole compute
        assert np.array_equal(_bits(phi), _bits(plan.compute()))
