"""Block-diagonal leaf preconditioner of Sec. 2.2.4 (FP64 oracle).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

Sec. 2.2.4 takes M as the part of A that couples elements of the same tree
leaf: after a permutation M = diag(M_1, ..., M_n), M_i the rows and columns
of A (both unknowns phi and dphi/dnu of every element of leaf i), and solves
M y = z leaf by leaf with a direct method.  Here the leaves are those of the
treecode's tree (oracle.treecode.build_tree with N0 = n0; n0 = 1 gives one
element per leaf, whose block is diag(1/2 (1 + eps), 1/2 (1 + 1/eps)) since
the self pair is omitted), each block is solved by its inverse (numpy), and
GMRES runs on A M^-1 y = b with u = M^-1 y (right preconditioning, reading
P2: the GMRES residual is then the true residual).
"""
from __future__ import annotations

import numpy as np

from .gmres import gmres
from .treecode import build_tree


def leaves(x, n0):
    """Element index arrays of the leaves of at most n0 elements."""
    if n0 == 1:
        return [np.array([i]) for i in range(x.shape[0])]
    t = build_tree(x, n0)
    return [t.perm[t.start[k]:t.end[k]] for k in t.leaves]


def blocks(A, groups):
    """(unknown indices, inverse of A restricted to them) per leaf; A is the dense 2N x 2N matrix."""
    n = A.shape[0] // 2
    out = []
    for g in groups:
        idx = np.concatenate([g, g + n])
        out.append((idx, np.linalg.inv(A[np.ix_(idx, idx)])))
    return out


def apply(blks, v):
    """M^-1 v."""
    out = np.empty_like(v)
    for idx, B in blks:
        out[idx] = B @ v[idx]
    return out


def solve_right(A, b, blks, tol=1e-8, restart=10, max_iter=1000):
    """GMRES(restart) on A M^-1 y = b; returns (u = M^-1 y, info)."""
    y, info = gmres(lambda v: A @ apply(blks, v), b, tol=tol, restart=restart, max_iter=max_iter)
    return apply(blks, y), info
