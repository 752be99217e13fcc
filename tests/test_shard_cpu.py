"""Target-leaf sharding, host side (no GPU): the cost partition of the
library (bldtt_partition_leaves, a host-only entry point), the work each rank
of a two-rank gloo job takes from it, and the gather of the ranks' potentials
that bench.py uses.  The work lists come from the oracle's trees and Alg. 2
lists; a leaf's cost is its PP/PC evaluations plus its share of the CP/CC
evaluations of every cluster above it (the library's definition), and each
rank's real cost counts the proxy work of shared ancestors in full."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle as O
from paper_2012_06925_gb300 import binding as B
from paper_2012_06925_gb300 import workloads as W


def test_partition_of_equal_costs_is_even():
    assert list(B.partition_leaves(np.ones(12), 4)) == [0, 3, 6, 9, 12]
    assert list(B.partition_leaves(np.ones(10), 1)) == [0, 10]


def test_partition_takes_the_nearest_boundary_and_allows_empty_ranges():
    # cumulative 1, 2, 3, 13: half of 13 is 6.5, nearer to 3 (after leaf 2) than to 13
    assert list(B.partition_leaves([1.0, 1.0, 1.0, 10.0], 2)) == [0, 3, 4]
    assert list(B.partition_leaves([5.0, 5.0], 4)) == [0, 0, 1, 1, 2]    # more shards than leaves
    assert list(B.partition_leaves(np.zeros(6), 3)) == [0, 2, 4, 6]      # no cost: equal counts
    assert list(B.partition_leaves([], 2)) == [0, 0, 0]
    for bad in ([1.0, -1.0], [1.0, np.nan], [np.inf]):
        with pytest.raises(B.BLDTTError):
            B.partition_leaves(bad, 2)
    with pytest.raises(B.BLDTTError):
        B.partition_leaves([1.0], 0)


def _work(seed=5):
    """Oracle trees and lists of an unequal-set problem; per leaf (tree order)
    its particle-item evaluations, per cluster its proxy-item evaluations and
    its leaf range."""
    tgt, src, q = W.make_problem("uniform", 12_000, 9_000, seed=seed, sources_kind="plummer")
    n = 2
    n_p = (n + 1) ** 3
    tt, st, lists = O.build_lists(tgt, src, n, 0.7, 60, 60)
    leaves = sorted(tt.leaves(), key=lambda c: tt.begin[c])
    index = {c: i for i, c in enumerate(leaves)}
    first = {c: min(index[l] for l in leaves if tt.begin[c] <= tt.begin[l] < tt.end[c])
             for c in range(tt.num_clusters)}
    last = {c: 1 + max(index[l] for l in leaves if tt.begin[c] <= tt.begin[l] < tt.end[c])
            for c in range(tt.num_clusters)}
    part = np.zeros(tt.num_clusters)       # PP + PC of a cluster's own entries
    prox = np.zeros(tt.num_clusters)       # CP + CC
    for t, s in lists[O.PP]:
        part[t] += tt.count(t) * st.count(s)
    for t, s in lists[O.PC]:
        part[t] += tt.count(t) * n_p
    for t, s in lists[O.CP]:
        prox[t] += n_p * st.count(s)
    for t, s in lists[O.CC]:
        prox[t] += n_p * n_p
    # a leaf's particle items carry the PP/PC entries of its whole chain,
    # evaluated at its own particles
    leaf_part = np.zeros(len(leaves))
    for i, c in enumerate(leaves):
        a = c
        while a >= 0:
            leaf_part[i] += part[a] * tt.count(c) / tt.count(a)
            a = tt.parent[a]
    cost = leaf_part.copy()
    for i, c in enumerate(leaves):
        a = c
        while a >= 0:
            cost[i] += prox[a] / (last[a] - first[a])
            a = tt.parent[a]
    return dict(leaves=leaves, first=first, last=last, leaf_part=leaf_part, prox=prox, cost=cost,
                nclusters=tt.num_clusters)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _work()
        bounds = B.partition_leaves(w["cost"], world)
        lo, hi = int(bounds[rank]), int(bounds[rank + 1])
        mine_leaves = [i for i in range(lo, hi) if w["leaf_part"][i] > 0]
        mine_prox = [c for c in range(w["nclusters"])
                     if w["prox"][c] > 0 and w["first"][c] < hi and w["last"][c] > lo]
        cost = float(w["leaf_part"][lo:hi].sum() + sum(w["prox"][c] for c in mine_prox))
        got = [None] * world
        dist.all_gather_object(got, (mine_leaves, mine_prox, cost, list(bounds)))
        # the gather of potentials: each rank owns a disjoint set of entries
        phi = torch.zeros(1000, dtype=torch.float64)
        gen = torch.Generator().manual_seed(rank)
        own = torch.arange(rank, 1000, world)
        phi[own] = torch.randn(own.numel(), dtype=torch.float64, generator=gen)
        mine = phi.clone()
        bench.gather_potentials(phi, dist)
        out[rank] = dict(shards=got, phi=phi.numpy(), own=mine.numpy(),
                         total_part=int((w["leaf_part"] > 0).sum()),
                         total_prox=int((w["prox"] > 0).sum()),
                         total_cost=float(w["leaf_part"].sum() + w["prox"].sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_the_work_list_and_gather_the_potentials():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0["shards"] == r1["shards"]                     # every rank sees the same partition
    (l0, p0, c0, b0), (l1, p1, c1, b1) = r0["shards"]
    assert b0 == b1 and b0[0] == 0 and b0[1] == b1[1]
    # particle items: disjoint, their union is every leaf with PP/PC work
    assert not set(l0) & set(l1) and len(set(l0) | set(l1)) == r0["total_part"]
    # proxy items: every cluster with CP/CC work is computed by some rank
    assert len(set(p0) | set(p1)) == r0["total_prox"]
    # costs balance within 10 % (shared ancestors' proxy work counted in full)
    assert max(c0, c1) <= 1.10 * min(c0, c1)
    assert c0 + c1 >= r0["total_cost"]
    # the gathered potentials are the union of the ranks' entries, bit for bit
    want = r0["own"] + r1["own"]
    for r in (r0, r1):
        assert np.array_equal(r["phi"].view(np.uint64), want.view(np.uint64))
