"""Helpers shared by the GPU parity tests: run the library through the C ABI
and map its clusters onto the oracle's by their particle ranges."""
import numpy as np
import torch

import oracle as O
from paper_2012_06925_gb300 import binding as B


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def run_gpu(tgt, src, q, precision=B.FP64, **kw):
    """Set up and compute; returns (phi numpy, plan).  The plan stays open."""
    plan = B.Plan(to_dev(tgt), to_dev(src), to_dev(q), precision=precision, **kw)
    phi = plan.compute().cpu().numpy()
    plan.check_error()
    return phi, plan


def oracle_tree_table(tree: O.Tree):
    out = {}
    for c in range(tree.num_clusters):
        par = tree.parent[c]
        out[(tree.begin[c], tree.end[c])] = (tuple(tree.lo[c]), tuple(tree.hi[c]), tree.level[c],
                                             None if par < 0 else (tree.begin[par], tree.end[par]))
    return out


def gpu_tree_table(t: dict):
    out = {}
    C = t["begin"].size
    for c in range(C):
        par = int(t["parent"][c])
        out[(int(t["begin"][c]), int(t["end"][c]))] = (
            tuple(float(v) for v in t["lo"][:, c]), tuple(float(v) for v in t["hi"][:, c]),
            int(t["level"][c]),
            None if par < 0 else (int(t["begin"][par]), int(t["end"][par])))
    return out


def oracle_list_keys(tt, st, lists):
    return [sorted(((tt.begin[a], tt.end[a]), (st.begin[b], st.end[b])) for a, b in l)
            for l in lists]


def gpu_list_keys(gt, gs, lists):
    out = []
    for t, s in lists:
        out.append(sorted(((int(gt["begin"][a]), int(gt["end"][a])),
                           (int(gs["begin"][b]), int(gs["end"][b]))) for a, b in zip(t, s)))
    return out


def gpu_to_oracle_index(gtree: dict, otree: O.Tree):
    """Array m with m[gpu cluster] = oracle cluster (same particle range)."""
    okey = {(otree.begin[c], otree.end[c]): c for c in range(otree.num_clusters)}
    return np.array([okey[(int(b), int(e))] for b, e in zip(gtree["begin"], gtree["end"])])


def rel_l2(ref, got):
    return O.relative_l2_error(ref, got)


def max_rel(ref, got):
    return O.max_norm_error(ref, got)


def same_leaf_members(gtree: dict, otree: O.Tree) -> bool:
    """The GPU orders the particles inside each leaf along a Morton curve; the
    leaf memberships (sets) must still equal the oracle's."""
    gperm, operm = gtree["perm"], otree.perm
    for c in otree.leaves():
        b, e = otree.begin[c], otree.end[c]
        if sorted(gperm[b:e].tolist()) != sorted(operm[b:e].tolist()):
            return False
    return True
