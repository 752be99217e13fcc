"""Plain FP64 CPU oracle for the BLDTT compute phase.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
restatement of the method that the CUDA library is checked against.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code, table or helper with the CUDA
path and never calls it.

Everything is written from Wilson, Vaughn & Krasny, "A GPU-accelerated fast
summation method based on barycentric Lagrange interpolation and dual tree
traversal" (BLDTT).  Equation numbers follow the paper's numbering:

  Eq. (1)   direct sum                              Sec. 1
  Eq. (3)   1D barycentric Lagrange polynomial      Sec. 2.1
  Eqs. (4)-(5) Chebyshev points of the 2nd kind and their weights, Sec. 2.1
  Alg. 1    BLDTT driver                            Sec. 2.2
  tree building                                     Sec. 2.3
  Eq. (6)   PP potential                            Sec. 2.4
  Eqs. (8)-(9)  PC potential, proxy charges         Sec. 2.4
  Eqs. (11)-(12) CP potential, CP proxy potential   Sec. 2.4
  Eqs. (14)-(15) CC potential, CC proxy potential   Sec. 2.4
  Eq. (16)  upward pass child -> parent             Sec. 2.5, App. B
  Alg. 2    dual tree traversal                     Sec. 2.6
  Eq. (19)  per-level direct downward form          Sec. 2.7, App. C
  Eq. (20)  parent -> child proxy potentials        Sec. 2.7
  Eq. (21)  leaf proxies -> target particles        Sec. 2.7
  Eq. (22)  relative l2 error                       Sec. 4

Readings taken where the paper is silent or garbled (each is also applied,
independently, by the CUDA path):

  R1  Eq. (3) prints sum_k' w_k/(x - s_k'); the weight inside the sum is w_k'.
      In 3D the basis is the tensor product of three 1D bases (Sec. 2.1).
  R2  Proxy points adapted to a box [lo, hi] in one dimension are
      t_k = c + h*s_k with c = (lo+hi)*0.5, h = (hi-lo)*0.5 and
      s_k = cos(pi*k/n), symmetrised: s_0 = 1, s_n = -1, s_{n-k} = -s_k and
      s_{n/2} = 0 for even n.  The weights (-1)^k delta_k are unchanged by the
      affine map.
  R3  Coincident-point guard: if x - t_k == 0 exactly, L_k(x) = 1 and the
      other L_k'(x) = 0 in that dimension (the first such k when several are
      equal, which happens only for a zero-width box).
  R4  A cluster is a leaf iff |C| <= M0 (Alg. 1 speaks of the maximum number
      of particles per leaf), or if all of its box extents are zero.
  R5  Child count (Sec. 2.3): at most 1 split dimension when
      M0 < |C| <= 2 M0, at most 2 when 2 M0 < |C| <= 4 M0, else at most 3.
      A dimension is eligible iff L_d*L_d*2 >= L_max*L_max (aspect ratio
      sqrt 2); the split dimensions are the longest eligible ones, ties to the
      lower axis.  A particle goes to the upper half iff coord >= midpoint of
      the (shrunk) box.  Children are ordered by the (x, y, z) bit triple,
      empty ones dropped, and each child is shrunk to its bounding box.
      Particles keep their input order inside every cluster.
  R6  Cluster centre = box centre; cluster radius = half the box diagonal;
      R = distance between centres.  The MAC (r_t + r_s)/R < theta is
      evaluated as r_t + r_s < theta*R (Alg. 2).
  R7  |C| in Alg. 2 is the particle count; the comparisons with n_p=(n+1)^3
      are the strict '>' of Alg. 2.  When neither cluster is a leaf, the
      target is split iff |C_s| < |C_t|.
  R8  A pair with r == 0 contributes nothing, in the direct sum and in PP
      (Eq. (1) would otherwise divide by zero for i == j).
  R9  Eq. (16) sums over the actual (2, 4 or 8) children; the upper limit
      'b' in Eq. (14) is n.
  R10 G = 1/r (no 4 pi) and Yukawa G = exp(-kappa r)/r (Sec. 4.6).  The other
      kernels of Sec. 4.6 take their parameter from kappa: oscillatory
      G = sin(kappa r)/r (the paper's case is kappa = pi) and regularized
      Coulomb G = 1/sqrt(r^2 + kappa^2) (the paper's eps = 0.005).  R8 applies
      to every kernel, including the two that are finite at r = 0.
  R12 The CC+PP-only variant (Sec. 4.3): a well-separated pair is CC when both
      clusters hold more than n_p particles and PP otherwise.
  R11 Every cluster of both trees carries proxies; proxy potentials of
      clusters without CP/CC interactions stay zero but are still passed
      down.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

COULOMB = 0
YUKAWA = 1
OSCILLATORY = 2
REG_COULOMB = 3
TEST_POLY = 99

# Traversal variants: the full method, and the ablation of Sec. 4.3 that uses
# only CC and PP (PC/CP candidates are computed directly).
FULL = 0
CC_PP_ONLY = 1

PP, PC, CP, CC = 0, 1, 2, 3
TYPE_NAMES = ("PP", "PC", "CP", "CC")


# --------------------------------------------------------------------------
# Kernel functions G(x, y), d = x - y  (Eq. (1); Sec. 4.6; reading R8, R10)
# --------------------------------------------------------------------------

def kernel_values(kernel: int, kappa: float, dx, dy, dz):
    """G evaluated on arrays of separations d = x - y (target minus source).

    Pairs with r == 0 are given the value 0 (reading R8).
    TEST_POLY is a test-only kernel of degree <= 2 in every coordinate of x
    and of y separately, so interpolation of degree n >= 2 reproduces it
    exactly:  G(d) = 1 + d1 - 2 d2 + 3 d3 + d1 d2 - d2 d3 + d1^2 d3^2 - d2^2/2.
    """
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    dz = np.asarray(dz, dtype=np.float64)
    r2 = dx * dx + dy * dy + dz * dz
    zero = r2 == 0.0
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        if kernel == COULOMB:
            g = 1.0 / np.sqrt(r2)
        elif kernel == YUKAWA:
            r = np.sqrt(r2)
            g = np.exp(-kappa * r) / r
        elif kernel == OSCILLATORY:
            r = np.sqrt(r2)
            g = np.sin(kappa * r) / r
        elif kernel == REG_COULOMB:
            g = 1.0 / np.sqrt(r2 + kappa * kappa)
        elif kernel == TEST_POLY:
            g = (1.0 + dx - 2.0 * dy + 3.0 * dz + dx * dy - dy * dz
                 + dx * dx * dz * dz - 0.5 * dy * dy)
        else:
            raise ValueError(f"unknown kernel {kernel}")
    g = np.where(zero, 0.0, g)
    return g


def _block_sum(kernel, kappa, tx, ty, tz, sx, sy, sz, q, block_elems=2_000_000):
    """phi(t) = sum_j G(t - s_j) q_j for target arrays t, source arrays s."""
    m = tx.shape[0]
    out = np.zeros(m)
    ns = sx.shape[0]
    if ns == 0 or m == 0:
        return out
    step = max(1, block_elems // ns)
    for a in range(0, m, step):
        b = min(m, a + step)
        g = kernel_values(kernel, kappa,
                          tx[a:b, None] - sx[None, :],
                          ty[a:b, None] - sy[None, :],
                          tz[a:b, None] - sz[None, :])
        out[a:b] = g @ q
    return out


def direct_sum(targets, sources, charges, kernel=COULOMB, kappa=0.0):
    """Eq. (1): phi(x_i) = sum_j G(x_i, y_j) q_j, O(MN), FP64 (reading R8)."""
    t = np.asarray(targets, dtype=np.float64)
    s = np.asarray(sources, dtype=np.float64)
    q = np.asarray(charges, dtype=np.float64)
    return _block_sum(kernel, kappa, t[0], t[1], t[2], s[0], s[1], s[2], q)


def relative_l2_error(reference, approx):
    """Eq. (22): (sum (phi_ds - phi_fs)^2 / sum phi_ds^2)^(1/2)."""
    reference = np.asarray(reference, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    num = np.sum((reference - approx) ** 2)
    den = np.sum(reference ** 2)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def max_norm_error(reference, approx):
    reference = np.asarray(reference, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    den = np.max(np.abs(reference)) if reference.size else 0.0
    num = np.max(np.abs(reference - approx)) if reference.size else 0.0
    return num / den if den > 0 else num


# --------------------------------------------------------------------------
# Barycentric Lagrange interpolation (Sec. 2.1; readings R1-R3)
# --------------------------------------------------------------------------

def chebyshev_points(n: int) -> np.ndarray:
    """Eq. (4): s_k = cos(pi k / n), k = 0..n, symmetrised (reading R2)."""
    s = np.empty(n + 1)
    for k in range(n + 1):
        s[k] = math.cos(math.pi * k / n)
    for k in range(n // 2 + 1):
        s[n - k] = -s[k]
    s[0] = 1.0
    s[n] = -1.0
    if n % 2 == 0:
        s[n // 2] = 0.0
    return s


def chebyshev_weights(n: int) -> np.ndarray:
    """Eq. (5): w_k = (-1)^k delta_k, delta_k = 1/2 at k = 0, n, else 1."""
    w = np.empty(n + 1)
    for k in range(n + 1):
        delta = 0.5 if (k == 0 or k == n) else 1.0
        w[k] = delta if k % 2 == 0 else -delta
    return w


def box_nodes(lo: float, hi: float, n: int) -> np.ndarray:
    """Chebyshev points adapted to [lo, hi] (reading R2): c + h s_k."""
    c = (lo + hi) * 0.5
    h = (hi - lo) * 0.5
    return c + h * chebyshev_points(n)


def lagrange_1d(x, nodes, weights) -> np.ndarray:
    """Eq. (3), second barycentric form.  Returns L[k, j] = L_k(x_j).

    Coincident-point guard (reading R3): where x_j - t_k == 0 exactly the
    column is one-hot at the first such k.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nodes = np.asarray(nodes, dtype=np.float64)
    weights = np.asarray(weights, dtype=np.float64)
    d = x[None, :] - nodes[:, None]                 # (P, m): x_j - t_k
    hit = d == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = weights[:, None] / d                # w_k / (x - t_k)
        denom = terms.sum(axis=0)                   # sum_k' w_k' / (x - t_k')
        L = terms / denom[None, :]
    cols = np.nonzero(hit.any(axis=0))[0]
    for j in cols:
        k = int(np.argmax(hit[:, j]))
        L[:, j] = 0.0
        L[k, j] = 1.0
    return L


def lagrange_1d_product_form(x, nodes) -> np.ndarray:
    """Textbook Lagrange polynomials prod_{j!=k} (x - t_j)/(t_k - t_j).

    Not used by the method; it is the independent definition the barycentric
    form of Eq. (3) is checked against.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    P = len(nodes)
    L = np.ones((P, x.size))
    for k in range(P):
        for j in range(P):
            if j != k:
                L[k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
    return L


def general_weights(nodes) -> np.ndarray:
    """w_k = 1 / prod_{j!=k} (s_k - s_j), the general definition in Eq. (3)."""
    P = len(nodes)
    w = np.empty(P)
    for k in range(P):
        p = 1.0
        for j in range(P):
            if j != k:
                p *= nodes[k] - nodes[j]
        w[k] = 1.0 / p
    return w


# --------------------------------------------------------------------------
# Trees (Sec. 2.3; readings R4-R6)
# --------------------------------------------------------------------------

@dataclass
class Tree:
    """Clusters of one particle set, particles permuted into tree order.

    perm[p] is the input index of the particle at tree position p; cluster c
    holds tree positions [begin[c], end[c]).  Clusters are numbered in the
    order the recursion creates them (pre-order).
    """
    perm: np.ndarray
    begin: list = field(default_factory=list)
    end: list = field(default_factory=list)
    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)
    parent: list = field(default_factory=list)
    children: list = field(default_factory=list)
    level: list = field(default_factory=list)

    @property
    def num_clusters(self):
        return len(self.begin)

    def count(self, c):
        return self.end[c] - self.begin[c]

    def is_leaf(self, c):
        return len(self.children[c]) == 0

    def center(self, c):
        lo, hi = self.lo[c], self.hi[c]
        return ((lo[0] + hi[0]) * 0.5, (lo[1] + hi[1]) * 0.5, (lo[2] + hi[2]) * 0.5)

    def radius(self, c):
        """Half the box diagonal (reading R6)."""
        lo, hi = self.lo[c], self.hi[c]
        ex = hi[0] - lo[0]
        ey = hi[1] - lo[1]
        ez = hi[2] - lo[2]
        return math.sqrt(ex * ex + ey * ey + ez * ez) * 0.5

    def nodes(self, c, n):
        """Three 1D arrays of proxy coordinates of cluster c (reading R2)."""
        return [box_nodes(self.lo[c][d], self.hi[c][d], n) for d in range(3)]

    def leaves(self):
        return [c for c in range(self.num_clusters) if self.is_leaf(c)]

    def key(self, c):
        return (self.begin[c], self.end[c])


def split_plan(lo, hi, count, max_leaf):
    """Which dimensions a cluster is bisected in (Sec. 2.3, reading R5).

    Returns the list of split dimensions (empty for a leaf).
    """
    if count <= max_leaf:
        return []
    ext = [hi[d] - lo[d] for d in range(3)]
    lmax = max(ext)
    if lmax == 0.0:
        return []
    if count <= 2 * max_leaf:
        cap = 1
    elif count <= 4 * max_leaf:
        cap = 2
    else:
        cap = 3
    eligible = [d for d in range(3) if ext[d] * ext[d] * 2.0 >= lmax * lmax]
    eligible.sort(key=lambda d: (-ext[d], d))
    return sorted(eligible[:cap])


def build_tree(points, max_leaf: int) -> Tree:
    """Sec. 2.3: recursive midpoint bisection of shrunk boxes."""
    pts = np.asarray(points, dtype=np.float64)
    m = pts.shape[1]
    tree = Tree(perm=np.empty(m, dtype=np.int64))

    def make(idx, begin, level, parent):
        sub = pts[:, idx]
        lo = tuple(float(v) for v in sub.min(axis=1))
        hi = tuple(float(v) for v in sub.max(axis=1))
        cid = tree.num_clusters
        tree.begin.append(begin)
        tree.end.append(begin + idx.size)
        tree.lo.append(lo)
        tree.hi.append(hi)
        tree.parent.append(parent)
        tree.children.append([])
        tree.level.append(level)
        dims = split_plan(lo, hi, idx.size, max_leaf)
        if not dims:
            tree.perm[begin:begin + idx.size] = idx
            return cid
        code = np.zeros(idx.size, dtype=np.int64)
        for d in dims:
            mid = (lo[d] + hi[d]) * 0.5
            code |= (sub[d] >= mid).astype(np.int64) << (2 - d)
        pos = begin
        for child_code in range(8):
            sel = idx[code == child_code]          # keeps input order
            if sel.size == 0:
                continue
            ch = make(sel, pos, level + 1, cid)
            tree.children[cid].append(ch)
            pos += sel.size
        return cid

    if m > 0:
        make(np.arange(m, dtype=np.int64), 0, 0, -1)
    return tree


# --------------------------------------------------------------------------
# Dual tree traversal (Sec. 2.6, Algorithm 2; readings R6, R7)
# --------------------------------------------------------------------------

def well_separated(tt: Tree, t: int, st: Tree, s: int, theta: float) -> bool:
    ct = tt.center(t)
    cs = st.center(s)
    dx = ct[0] - cs[0]
    dy = ct[1] - cs[1]
    dz = ct[2] - cs[2]
    R = math.sqrt(dx * dx + dy * dy + dz * dz)
    return tt.radius(t) + st.radius(s) < theta * R


def dual_tree_traversal(tt: Tree, st: Tree, n: int, theta: float, variant: int = FULL):
    """Algorithm 2 from the root pair.  Returns four lists of (t, s) pairs.

    variant CC_PP_ONLY is the ablation of Sec. 4.3 (reading R12).
    """
    n_p = (n + 1) ** 3
    lists = ([], [], [], [])
    if tt.num_clusters == 0 or st.num_clusters == 0:
        return lists

    def dtt(t, s):
        if well_separated(tt, t, st, s, theta):
            big_t = tt.count(t) > n_p
            big_s = st.count(s) > n_p
            if big_t and big_s:
                lists[CC].append((t, s))
            elif variant == CC_PP_ONLY:
                lists[PP].append((t, s))
            elif big_t and not big_s:
                lists[CP].append((t, s))
            elif not big_t and big_s:
                lists[PC].append((t, s))
            else:
                lists[PP].append((t, s))
            return
        leaf_t = tt.is_leaf(t)
        leaf_s = st.is_leaf(s)
        if leaf_t and leaf_s:
            lists[PP].append((t, s))
        elif leaf_s:
            for c in tt.children[t]:
                dtt(c, s)
        elif leaf_t:
            for c in st.children[s]:
                dtt(t, c)
        elif st.count(s) < tt.count(t):
            for c in tt.children[t]:
                dtt(c, s)
        else:
            for c in st.children[s]:
                dtt(t, c)

    dtt(0, 0)
    return lists


# --------------------------------------------------------------------------
# Upward pass (Sec. 2.5, App. B)
# --------------------------------------------------------------------------

def tensor_basis(tree: Tree, c: int, n: int, px, py, pz):
    """The three 1D factor matrices L^(d)[k_d, j] of cluster c at points p."""
    w = chebyshev_weights(n)
    nx, ny, nz = tree.nodes(c, n)
    return lagrange_1d(px, nx, w), lagrange_1d(py, ny, w), lagrange_1d(pz, nz, w)


def proxy_charges_direct(tree: Tree, c: int, n: int, ys, qs):
    """Eq. (9): qhat_k = sum_{y_j in C} L_k(y_j) q_j, k a 3D index.

    ys is the (3, N) source array in tree order and qs the charges in tree
    order.  Returns an array of shape (n+1, n+1, n+1).
    """
    b, e = tree.begin[c], tree.end[c]
    B1, B2, B3 = tensor_basis(tree, c, n, ys[0, b:e], ys[1, b:e], ys[2, b:e])
    W = B2[:, None, :] * B3[None, :, :] * qs[b:e][None, None, :]
    return np.tensordot(B1, W, axes=([1], [2]))


def child_to_parent_matrices(tree: Tree, par: int, ch: int, n: int):
    """U_d[k, k'] = L^par_k(s^child_k') in each dimension (Eq. (16))."""
    w = chebyshev_weights(n)
    pn = tree.nodes(par, n)
    cn = tree.nodes(ch, n)
    return [lagrange_1d(cn[d], pn[d], w) for d in range(3)]


def upward_pass(tree: Tree, n: int, ys, qs):
    """Sec. 2.5: leaf proxy charges by Eq. (9), then parents by Eq. (16)."""
    P = n + 1
    qhat = np.zeros((tree.num_clusters, P, P, P))
    for c in tree.leaves():
        qhat[c] = proxy_charges_direct(tree, c, n, ys, qs)
    by_level = sorted(range(tree.num_clusters), key=lambda c: -tree.level[c])
    for c in by_level:
        if tree.is_leaf(c):
            continue
        acc = np.zeros((P, P, P))
        for ch in tree.children[c]:
            U1, U2, U3 = child_to_parent_matrices(tree, c, ch, n)
            acc += np.einsum("ai,bj,ck,ijk->abc", U1, U2, U3, qhat[ch])
        qhat[c] = acc
    return qhat


def proxy_grid(tree: Tree, c: int, n: int):
    """Flattened 3D Chebyshev grid of cluster c, k = (k1, k2, k3) row-major."""
    nx, ny, nz = tree.nodes(c, n)
    gx, gy, gz = np.meshgrid(nx, ny, nz, indexing="ij")
    return gx.ravel(), gy.ravel(), gz.ravel()


# --------------------------------------------------------------------------
# The four interactions (Sec. 2.4)
# --------------------------------------------------------------------------

def interact_pp(kernel, kappa, xs, tb, te, ys, qs, sb, se):
    """Eq. (6): phi(x_i) = sum_{y_j in C_s} G(x_i, y_j) q_j."""
    return _block_sum(kernel, kappa, xs[0, tb:te], xs[1, tb:te], xs[2, tb:te],
                      ys[0, sb:se], ys[1, sb:se], ys[2, sb:se], qs[sb:se])


def interact_pc(kernel, kappa, xs, tb, te, st, s, n, qhat):
    """Eq. (8): phi(x_i) = sum_k G(x_i, s_k) qhat_k."""
    gx, gy, gz = proxy_grid(st, s, n)
    return _block_sum(kernel, kappa, xs[0, tb:te], xs[1, tb:te], xs[2, tb:te],
                      gx, gy, gz, qhat[s].ravel())


def interact_cp(kernel, kappa, tt, t, n, ys, qs, sb, se):
    """Eq. (12): phi(t_l) = sum_{y_j in C_s} G(t_l, y_j) q_j."""
    gx, gy, gz = proxy_grid(tt, t, n)
    return _block_sum(kernel, kappa, gx, gy, gz,
                      ys[0, sb:se], ys[1, sb:se], ys[2, sb:se], qs[sb:se])


def interact_cc(kernel, kappa, tt, t, st, s, n, qhat):
    """Eq. (15): phi(t_l) = sum_k G(t_l, s_k) qhat_k."""
    tx, ty, tz = proxy_grid(tt, t, n)
    sx, sy, sz = proxy_grid(st, s, n)
    return _block_sum(kernel, kappa, tx, ty, tz, sx, sy, sz, qhat[s].ravel())


# --------------------------------------------------------------------------
# Downward pass (Sec. 2.7, App. C)
# --------------------------------------------------------------------------

def parent_to_child(tree: Tree, par: int, ch: int, n: int, phit_par):
    """Eq. (20): phi(t^child_k') = sum_k L^par_k(t^child_k') phi(t^par_k)."""
    D1, D2, D3 = child_to_parent_matrices(tree, par, ch, n)
    return np.einsum("ai,bj,ck,abc->ijk", D1, D2, D3, phit_par)


def leaf_to_particles(tree: Tree, c: int, n: int, xs, phit_leaf):
    """Eq. (21): phi(x_i) += sum_k L_k(x_i) phi(t_k) for x_i in leaf c."""
    b, e = tree.begin[c], tree.end[c]
    B1, B2, B3 = tensor_basis(tree, c, n, xs[0, b:e], xs[1, b:e], xs[2, b:e])
    return np.einsum("im,jm,km,ijk->m", B1, B2, B3, phit_leaf)


# --------------------------------------------------------------------------
# Driver (Algorithm 1)
# --------------------------------------------------------------------------

@dataclass
class Result:
    phi: np.ndarray            # potentials, input order of the targets
    phi_tree: np.ndarray       # potentials, target tree order
    ttree: Tree
    stree: Tree
    lists: tuple
    qhat: np.ndarray           # (num source clusters, P, P, P)
    phit_dtt: np.ndarray       # CP + CC proxy potentials after the traversal
    phit: np.ndarray           # proxy potentials after the downward pass
    counts: tuple              # kernel evaluations per type (PP, PC, CP, CC)


def build_lists(targets, sources, n, theta, N0, M0, variant=FULL):
    """Alg. 1 line 6 plus Alg. 2: trees and the four interaction lists."""
    tt = build_tree(targets, M0)
    st = build_tree(sources, N0)
    lists = dual_tree_traversal(tt, st, n, theta, variant)
    return tt, st, lists


def interaction_counts(tt, st, lists, n):
    n_p = (n + 1) ** 3
    pp = sum(tt.count(t) * st.count(s) for t, s in lists[PP])
    pc = sum(tt.count(t) * n_p for t, s in lists[PC])
    cp = sum(n_p * st.count(s) for t, s in lists[CP])
    cc = n_p * n_p * len(lists[CC])
    return pp, pc, cp, cc


def bldtt(targets, sources, charges, kernel=COULOMB, kappa=0.0, n=8, theta=0.7,
          N0=2000, M0=2000, variant=FULL) -> Result:
    """Algorithm 1: trees, upward pass, dual tree traversal, downward pass."""
    xs_in = np.asarray(targets, dtype=np.float64)
    ys_in = np.asarray(sources, dtype=np.float64)
    q_in = np.asarray(charges, dtype=np.float64)
    P = n + 1
    tt, st, lists = build_lists(xs_in, ys_in, n, theta, N0, M0, variant)
    xs = xs_in[:, tt.perm]
    ys = ys_in[:, st.perm]
    qs = q_in[st.perm]

    qhat = upward_pass(st, n, ys, qs)

    # Potentials at particles and at target proxies start at zero (Sec. 2.6).
    phi = np.zeros(xs.shape[1])
    phit = np.zeros((tt.num_clusters, P, P, P))
    for t, s in lists[PP]:
        phi[tt.begin[t]:tt.end[t]] += interact_pp(kernel, kappa, xs, tt.begin[t], tt.end[t],
                                                   ys, qs, st.begin[s], st.end[s])
    for t, s in lists[PC]:
        phi[tt.begin[t]:tt.end[t]] += interact_pc(kernel, kappa, xs, tt.begin[t], tt.end[t],
                                                   st, s, n, qhat)
    for t, s in lists[CP]:
        phit[t] += interact_cp(kernel, kappa, tt, t, n, ys, qs,
                               st.begin[s], st.end[s]).reshape(P, P, P)
    for t, s in lists[CC]:
        phit[t] += interact_cc(kernel, kappa, tt, t, st, s, n, qhat).reshape(P, P, P)
    phit_dtt = phit.copy()

    # Downward pass: root to leaves by Eq. (20), then leaves to targets, Eq. (21).
    for c in sorted(range(tt.num_clusters), key=lambda c: tt.level[c]):
        for ch in tt.children[c]:
            phit[ch] += parent_to_child(tt, c, ch, n, phit[c])
    for c in tt.leaves():
        phi[tt.begin[c]:tt.end[c]] += leaf_to_particles(tt, c, n, xs, phit[c])

    out = np.empty_like(phi)
    out[tt.perm] = phi
    return Result(phi=out, phi_tree=phi, ttree=tt, stree=st, lists=lists, qhat=qhat,
                  phit_dtt=phit_dtt, phit=phit,
                  counts=interaction_counts(tt, st, lists, n))


def downward_direct(tt: Tree, n: int, xs, phit_dtt, positions):
    """Eq. (19): sum over the chain of clusters containing each target of
    the interpolated CP/CC proxy potentials, without the recursion.

    positions are tree positions of targets; returns the downward share of
    phi at those targets.
    """
    w = chebyshev_weights(n)
    out = np.zeros(len(positions))
    leaf_of = _leaf_of_position(tt)
    for a, p in enumerate(positions):
        c = leaf_of[p]
        while c >= 0:
            nx, ny, nz = tt.nodes(c, n)
            l1 = lagrange_1d(xs[0, p], nx, w)[:, 0]
            l2 = lagrange_1d(xs[1, p], ny, w)[:, 0]
            l3 = lagrange_1d(xs[2, p], nz, w)[:, 0]
            out[a] += np.einsum("i,j,k,ijk->", l1, l2, l3, phit_dtt[c])
            c = tt.parent[c]
    return out


def _leaf_of_position(tt: Tree):
    leaf_of = np.full(tt.perm.size, -1, dtype=np.int64)
    for c in tt.leaves():
        leaf_of[tt.begin[c]:tt.end[c]] = c
    return leaf_of


class SampledBLDTT:
    """BLDTT potentials at selected targets only, for problems too large to
    run the whole oracle.

    The trees, the interaction lists and the upward pass are computed in full;
    the potential at a target x_i is then assembled along its chain of target
    clusters C^1 c C^2 c ... (Sec. 2.7): PP and PC terms of every cluster on
    the chain, plus the CP/CC proxy potentials of every cluster on the chain
    interpolated straight to x_i (Eq. (19)).  Equal to the full driver up to
    rounding order.
    """

    def __init__(self, targets, sources, charges, kernel=COULOMB, kappa=0.0, n=8,
                 theta=0.7, N0=2000, M0=2000, variant=FULL):
        self.kernel, self.kappa, self.n = kernel, kappa, n
        self.xs_in = np.asarray(targets, dtype=np.float64)
        ys_in = np.asarray(sources, dtype=np.float64)
        q_in = np.asarray(charges, dtype=np.float64)
        self.tt, self.st, self.lists = build_lists(self.xs_in, ys_in, n, theta, N0, M0, variant)
        self.xs = self.xs_in[:, self.tt.perm]
        self.ys = ys_in[:, self.st.perm]
        self.qs = q_in[self.st.perm]
        self.qhat = upward_pass(self.st, n, self.ys, self.qs)
        self.by_target = [dict((k, []) for k in range(4)) for _ in range(self.tt.num_clusters)]
        for typ in range(4):
            for t, s in self.lists[typ]:
                self.by_target[t][typ].append(s)
        self._phit = {}
        self.leaf_of = _leaf_of_position(self.tt)
        self.pos_of_input = np.empty_like(self.tt.perm)
        self.pos_of_input[self.tt.perm] = np.arange(self.tt.perm.size)

    def phit_dtt(self, c):
        """CP + CC proxy potentials of target cluster c (Eqs. (12), (15))."""
        if c not in self._phit:
            P = self.n + 1
            acc = np.zeros(P ** 3)
            for s in self.by_target[c][CP]:
                acc += interact_cp(self.kernel, self.kappa, self.tt, c, self.n, self.ys,
                                   self.qs, self.st.begin[s], self.st.end[s])
            for s in self.by_target[c][CC]:
                acc += interact_cc(self.kernel, self.kappa, self.tt, c, self.st, s,
                                   self.n, self.qhat)
            self._phit[c] = acc.reshape(P, P, P)
        return self._phit[c]

    def potentials(self, input_indices):
        """phi at the given targets (input order indices)."""
        w = chebyshev_weights(self.n)
        out = np.zeros(len(input_indices))
        for a, i in enumerate(input_indices):
            p = int(self.pos_of_input[i])
            xs = self.xs[:, p:p + 1]
            c = int(self.leaf_of[p])
            total = 0.0
            while c >= 0:
                for s in self.by_target[c][PP]:
                    total += interact_pp(self.kernel, self.kappa, xs, 0, 1, self.ys, self.qs,
                                         self.st.begin[s], self.st.end[s])[0]
                for s in self.by_target[c][PC]:
                    total += interact_pc(self.kernel, self.kappa, xs, 0, 1, self.st, s,
                                         self.n, self.qhat)[0]
                nx, ny, nz = self.tt.nodes(c, self.n)
                l1 = lagrange_1d(xs[0], nx, w)[:, 0]
                l2 = lagrange_1d(xs[1], ny, w)[:, 0]
                l3 = lagrange_1d(xs[2], nz, w)[:, 0]
                total += float(np.einsum("i,j,k,ijk->", l1, l2, l3, self.phit_dtt(c)))
                c = self.tt.parent[c]
            out[a] = total
        return out
