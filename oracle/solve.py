"""End-to-end oracle solve: source, linear solve, energy, potential, gradient.

Test infrastructure only.  Follows the order of the paper's direct-sum
pipeline (Sec. 2.4): source terms, Krylov (or direct) solve of A u = b,
solvation energy; plus the adjoint solve A^T lam = c that the gradient of
the energy needs.

``prob`` is any object with ``centroids (N,3)``, ``normals (N,3)``,
``areas (N,)``, ``charge_pos (Nc,3)`` or ``(B,Nc,3)``, ``q (B,Nc)``,
``eps_in``, ``eps_out``, ``kappa``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import KCAL, assemble, energy, energy_row, gesv, grad, matvec, matvec_t, source
from .gmres import gmres

DIRECT_MAX_N = 1280  # Gaussian elimination up to 2N = 2560 unknowns


@dataclass
class Solution:
    u: np.ndarray  # (2N,) internal units
    b: np.ndarray
    energy_kcal: float
    phi_reac: np.ndarray  # (Nc,) internal units
    info: dict = field(default_factory=dict)

    def surface_potential(self):
        """(phi kcal/mol/e, dphi/dnu kcal/mol/e/A) on every element."""
        n = self.u.shape[0] // 2
        return KCAL * self.u[:n], KCAL * self.u[n:]


def _pos(prob, r):
    p = np.asarray(prob.charge_pos, dtype=np.float64)
    return p[r] if p.ndim == 3 else p


def _eps(prob):
    return prob.eps_out / prob.eps_in


def solve(prob, rhs=0, method="auto", tol=1e-12, restart=10, max_iter=3000):
    """Solve one right-hand side; ``method`` is 'direct', 'gmres' or 'auto'."""
    x, nrm, area = prob.centroids, prob.normals, prob.areas
    eps = _eps(prob)
    y = _pos(prob, rhs)
    q = np.asarray(prob.q, dtype=np.float64)[rhs]
    b = source(x, nrm, y, q, prob.eps_in)
    n = x.shape[0]
    if method == "auto":
        method = "direct" if n <= DIRECT_MAX_N else "gmres"
    if method == "direct":
        A = assemble(x, nrm, area, eps, prob.kappa)
        u = gesv(A, b)
        info = dict(method="direct", iters=0, converged=True,
                    rel_residual=float(np.linalg.norm(b - A @ u) / np.linalg.norm(b)))
    else:
        u, info = gmres(lambda v: matvec(x, nrm, area, eps, prob.kappa, v), b, tol=tol,
                        restart=restart, max_iter=max_iter)
        info = dict(info, method="gmres")
    e, pr = energy(x, nrm, area, eps, prob.kappa, y, q, u)
    return Solution(u=u, b=b, energy_kcal=KCAL * e, phi_reac=pr, info=info)


def solve_adjoint(prob, rhs=0, method="auto", tol=1e-12, restart=10, max_iter=3000):
    """lam with A^T lam = c, c the energy row (E = 1/2 c . u)."""
    x, nrm, area = prob.centroids, prob.normals, prob.areas
    eps = _eps(prob)
    y = _pos(prob, rhs)
    q = np.asarray(prob.q, dtype=np.float64)[rhs]
    c = energy_row(x, nrm, area, eps, prob.kappa, y, q)
    n = x.shape[0]
    if method == "auto":
        method = "direct" if n <= DIRECT_MAX_N else "gmres"
    if method == "direct":
        A = assemble(x, nrm, area, eps, prob.kappa)
        return gesv(A.T, c), c
    lam, _ = gmres(lambda v: matvec_t(x, nrm, area, eps, prob.kappa, v), c, tol=tol,
                   restart=restart, max_iter=max_iter)
    return lam, c


def energy_gradient(prob, rhs=0, method="auto", tol=1e-12):
    """(E kcal/mol, dE/dq kcal/mol/e, dE/dy kcal/mol/A) for one charge set."""
    sol = solve(prob, rhs, method, tol)
    lam, _ = solve_adjoint(prob, rhs, method, tol)
    y = _pos(prob, rhs)
    q = np.asarray(prob.q, dtype=np.float64)[rhs]
    dq, dy = grad(prob.centroids, prob.normals, prob.areas, _eps(prob), prob.kappa, prob.eps_in,
                  y, q, sol.u, lam)
    return sol.energy_kcal, KCAL * dq, KCAL * dy
