"""FP64 oracle of the far-field (treecode) mat-vec, Sec. 2.2.3.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests, the
smoke check and the CPU legs of ``bench.py`` use it; the library never does.

Sec. 2.2.3 writes the mat-vec of Eqs. 5-6 as N-body sums over sources with
"charges" ds_j phi_j and ds_j dphi/dnu_j, arranges the elements in a tree of
clusters (root box split into children until a cluster holds at most N0
elements), and evaluates each target's sum as particle-particle terms over
the near clusters plus, for every cluster c that is well separated from the
target (multipole acceptance criterion r_c / R <= theta, r_c the cluster
radius, R the distance from the target to the cluster centre), a p-th
order polynomial approximation of the kernel in the source position.

Reading T1 (what this oracle fixes where the section is silent or where
the CUDA path departs from it):
* Tree: a cluster is a range of elements in tree order; its box is the
  tight bounding box of its centroids (FP64, as given); a cluster with more
  than N0 elements is split in two at the median of the longest box side
  (elements ordered by that coordinate, ties by element index; the first
  half gets floor(count / 2)).  The root is every element in input order.
* Cluster centre x_c = box centre; radius r_c = half the box diagonal.
* Targets are taken leaf by leaf (a leaf B with centre x_B, radius r_B),
  and the MAC is applied to the whole leaf: c is far for B when
  r_c + theta r_B <= theta |x_B - x_c|, which guarantees r_c / |x - x_c| <=
  theta for every target x of B (the paper's particle-cluster criterion).
* The degree-p polynomial in the source position is the tensor-product
  Lagrange interpolant at (p+1)^3 Chebyshev points of the second kind on the
  cluster box (barycentric form), not the Taylor series about the centre:
  it turns every far-field term into the same pair sum over (p+1)^3 proxy
  sources with weights
      a_k = sum_{j in c} L_k(x_j) a_j,   m_k = sum_{j in c} L_k(x_j) m_j,
  with a_j = ds_j psi_j and m_j = ds_j phi_j n_j (the kernels K2 and K4 are
  linear in the source normal, so the weighted normal m_j interpolates like a
  charge).  A cluster that passes the MAC but holds no more elements than
  proxies is summed directly.
* Traversal per leaf: from the root, a far cluster contributes its proxies
  (or its elements when it is small), a near leaf its elements (the self
  pair j = i is omitted as in Eqs. 5-6), a near cluster its two children.

Every (target, source) pair is thus covered exactly once, by a direct term
or through exactly one far cluster.  Pins (tests/test_oracle_pins.py):
theta = 0 reproduces the direct mat-vec; the error against it falls
geometrically with p; the proxy weights reproduce every monomial moment of
degree <= p per coordinate; the lists cover each pair once and every far
entry meets the particle-cluster MAC for each of its targets.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _c, _p, lib


@dataclass
class Tree:
    perm: np.ndarray                 # tree position -> element index
    start: list = field(default_factory=list)   # per node: first tree position
    end: list = field(default_factory=list)     # per node: one past the last
    lo: list = field(default_factory=list)      # per node: box corner (3,)
    hi: list = field(default_factory=list)
    child: list = field(default_factory=list)   # per node: (left, right) or None
    leaves: list = field(default_factory=list)  # node ids of the leaves, in tree order


def build_tree(x, leaf_size):
    """Binary tree of clusters over centroids x (N, 3), leaves of at most leaf_size."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    perm = np.arange(n, dtype=np.int64)
    t = Tree(perm=perm)

    def node(s, e):
        pts = x[perm[s:e]]
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        k = len(t.start)
        t.start.append(s)
        t.end.append(e)
        t.lo.append(lo)
        t.hi.append(hi)
        t.child.append(None)
        return k

    stack = [node(0, n)]
    while stack:
        k = stack.pop()
        s, e = t.start[k], t.end[k]
        if e - s <= leaf_size:
            continue
        ext = t.hi[k] - t.lo[k]
        d = int(np.argmax(ext))  # first of equal maxima
        idx = perm[s:e]
        order = np.lexsort((idx, x[idx, d]))  # by coordinate, ties by element index
        perm[s:e] = idx[order]
        h = (e - s) // 2
        left, right = node(s, s + h), node(s + h, e)
        t.child[k] = (left, right)
        stack.append(right)
        stack.append(left)
    # leaves in tree order
    t.leaves = sorted((k for k in range(len(t.start)) if t.child[k] is None), key=lambda k: t.start[k])
    return t


def geometry(t, k):
    lo, hi = t.lo[k], t.hi[k]
    c = 0.5 * (lo + hi)
    r = float(np.sqrt(np.sum((0.5 * (hi - lo)) ** 2)))
    return c, r


def interaction_lists(t, theta, degree):
    """Per leaf: a list of ('direct', start, end) tree-position ranges and
    ('far', node) clusters, in traversal order (adjacent direct ranges merged)."""
    n_proxy = (degree + 1) ** 3
    lists = []
    for b in t.leaves:
        xb, rb = geometry(t, b)
        out = []

        def visit(k):
            xc, rc = geometry(t, k)
            dist = float(np.sqrt(np.sum((xb - xc) ** 2)))
            count = t.end[k] - t.start[k]
            if rc + theta * rb <= theta * dist:
                if count > n_proxy:
                    out.append(("far", k))
                else:
                    out.append(("direct", t.start[k], t.end[k]))
            elif t.child[k] is None:
                out.append(("direct", t.start[k], t.end[k]))
            else:
                visit(t.child[k][0])
                visit(t.child[k][1])

        visit(0)
        merged = []
        for e in out:
            if merged and e[0] == "direct" and merged[-1][0] == "direct" and merged[-1][2] == e[1]:
                merged[-1] = ("direct", merged[-1][1], e[2])
            else:
                merged.append(e)
        lists.append(merged)
    return lists


def cheb_box(lo, hi, degree):
    """Chebyshev points of the second kind on the cluster box, per coordinate
    ((3, degree + 1)), and their barycentric weights.  A box side shorter than
    1e-3 of the longest is widened to that length about its centre."""
    ext = hi - lo
    ext = np.maximum(ext, 1e-3 * ext.max())
    c = 0.5 * (lo + hi)
    tk = np.cos(np.pi * np.arange(degree + 1) / degree)
    nodes = c[:, None] + 0.5 * ext[:, None] * tk[None, :]
    w = (-1.0) ** np.arange(degree + 1)
    w[0] *= 0.5
    w[-1] *= 0.5
    return nodes, w


def lagrange_1d(t, nodes, w):
    """Barycentric Lagrange basis values l_i(t) for points t (m,) -> (m, degree+1)."""
    diff = t[:, None] - nodes[None, :]
    exact = diff == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        q = w[None, :] / diff
        out = q / q.sum(axis=1, keepdims=True)
    rows = exact.any(axis=1)
    out[rows] = exact[rows].astype(np.float64)
    return out


def proxies(t, k, x, a, m, degree):
    """Proxy positions (P, 3) and weights a_k (P,), m_k (P, 3) of cluster k."""
    nodes, w = cheb_box(t.lo[k], t.hi[k], degree)
    idx = t.perm[t.start[k]:t.end[k]]
    L = [lagrange_1d(x[idx, d], nodes[d], w) for d in range(3)]  # (count, p+1) each
    # L_k(x_j) for k = (k0, k1, k2) in C order: (count, (p+1)^3)
    Lk = (L[0][:, :, None, None] * L[1][:, None, :, None] * L[2][:, None, None, :]).reshape(idx.shape[0], -1)
    pos = np.stack(np.meshgrid(nodes[0], nodes[1], nodes[2], indexing="ij"), axis=-1).reshape(-1, 3)
    return pos, Lk.T @ a[idx], Lk.T @ m[idx]


def _record_sums(xt, nt, tid, ys, a, m, sid, eps, kappa, transpose=False):
    """Per target: [sum (K1 a + K2(m)), sum (K3 a + K4(m))] over the records
    (transpose: the phi and psi outputs of A^T, [sum (K2 w + K4(p)), sum (K1 w
    + K3(p))] with a = w, m = p), skipping a record whose id equals the
    target's (the self pair)."""
    xt, nt, ys, a, m = _c(xt), _c(nt), _c(ys), _c(a), _c(m)
    tid = np.ascontiguousarray(tid, dtype=np.int64)
    sid = np.ascontiguousarray(sid, dtype=np.int64)
    out = np.zeros((xt.shape[0], 2))
    f = lib().orc_record_sums_t if transpose else lib().orc_record_sums
    f(xt.shape[0], _p(xt), _p(nt), tid.ctypes.data_as(ctypes.c_void_p), ys.shape[0], _p(ys), _p(a), _p(m),
      sid.ctypes.data_as(ctypes.c_void_p), eps, kappa, _p(out))
    return out


def matvec(x, nrm, area, eps, kappa, u, theta, degree, leaf_size, rows=None, tree=None, lists=None,
           transpose=False):
    """Treecode approximation of A u (Eqs. 5-6), or of A^T u (``transpose``).
    ``rows``: indices into [0, 2N) to evaluate (default: all).  Returns the
    rows (or the full 2N vector).

    A^T u sums, for output element e, column e of A: the source records are
    (x_j, w_j = phi_j, p_j = psi_j n_j) -- the kernels K3 and K4 of row
    element j are linear in its normal, so p_j interpolates like a charge as
    m_j does for A u -- and the sums are multiplied by the output element's
    area.  The tree, the lists and the proxies are those of A u."""
    x, nrm, area, u = _c(x), _c(nrm), _c(area), _c(u)
    n = x.shape[0]
    phi, psi = u[:n], u[n:]
    if transpose:
        a = phi.copy()
        m = psi[:, None] * nrm
    else:
        a = area * psi
        m = (area * phi)[:, None] * nrm
    t = tree if tree is not None else build_tree(x, leaf_size)
    L = lists if lists is not None else interaction_lists(t, theta, degree)
    want = np.arange(2 * n) if rows is None else np.asarray(rows, dtype=np.int64)
    elems = np.unique(want % n)
    pos_of = np.empty(n, dtype=np.int64)
    pos_of[t.perm] = np.arange(n)
    leaf_of_pos = np.empty(n, dtype=np.int64)
    for li, b in enumerate(t.leaves):
        leaf_of_pos[t.start[b]:t.end[b]] = li
    sums = {}
    cache = {}
    by_leaf = {}
    for e in elems:
        by_leaf.setdefault(int(leaf_of_pos[pos_of[e]]), []).append(int(e))
    for li, es in by_leaf.items():
        ys, aa, mm, sid = [], [], [], []
        for ent in L[li]:
            if ent[0] == "direct":
                idx = t.perm[ent[1]:ent[2]]
                ys.append(x[idx])
                aa.append(a[idx])
                mm.append(m[idx])
                sid.append(idx)
            else:
                k = ent[1]
                if k not in cache:
                    cache[k] = proxies(t, k, x, a, m, degree)
                pp, pa, pm = cache[k]
                ys.append(pp)
                aa.append(pa)
                mm.append(pm)
                sid.append(np.full(pp.shape[0], -1, dtype=np.int64))
        es = np.array(es, dtype=np.int64)
        s = _record_sums(x[es], nrm[es], es, np.concatenate(ys), np.concatenate(aa), np.concatenate(mm),
                         np.concatenate(sid), eps, kappa, transpose)
        if transpose:
            s = s * area[es][:, None]
        for e, v in zip(es, s):
            sums[int(e)] = v
    out = np.empty(want.shape[0])
    for r, row in enumerate(want):
        e = int(row % n)
        if row < n:
            out[r] = 0.5 * (1.0 + eps) * phi[e] - sums[e][0]
        else:
            out[r] = 0.5 * (1.0 + 1.0 / eps) * psi[e] - sums[e][1]
    return out
