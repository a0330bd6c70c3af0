"""FP64 CPU oracle of the boundary-integral Poisson-Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The library (``paper_2312_10044_gb300``) never imports it, and this package
never imports the library: the two share no code.

Contents
--------
* ``bie_oracle.c`` (built into ``liboracle.so`` by :func:`build`): the pair
  Green's functions and kernels K1..K4, the source term, the matrix-free
  mat-vec and its transpose, the dense matrix, Gaussian elimination, the
  energy and the adjoint gradient, all plain FP64 (Sec. 2.2.1-2.2.2).
* :mod:`oracle.gmres`: textbook restarted GMRES (Saad & Schultz, the solver
  the paper cites in Sec. 2.2.2) with modified Gram-Schmidt and Givens
  rotations.
* :mod:`oracle.closed_forms`: Born ion and Kirkwood sphere energies and the
  Born surface potential, derived from the linearised PB equation.

Units: the unknowns are in the paper's internal units, in which G0 carries
1/(4 pi); ``KCAL`` = 4 pi * 332.0716 converts energies to kcal/mol and
surface potentials to kcal/mol/e (Sec. 2.1 gives the 332.0716 factor).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

KCAL = 4.0 * np.pi * 332.0716
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``bie_oracle.c`` with gcc + OpenMP into ``liboracle.so``."""
    src = os.path.join(_HERE, "bie_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        D = ctypes.c_double
        I = ctypes.c_int64
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_green.argtypes = [P, P, P, P, D, P]
        L.orc_kernels.argtypes = [P, P, P, P, D, D, P]
        L.orc_source.argtypes = [I, P, P, I, P, P, D, P]
        L.orc_matvec.argtypes = [I, P, P, P, D, D, P, P]
        L.orc_matvec_t.argtypes = [I, P, P, P, D, D, P, P]
        L.orc_matvec_rows.argtypes = [I, P, P, P, D, D, P, I, P, P]
        L.orc_matvec_t_rows.argtypes = [I, P, P, P, D, D, P, I, P, P]
        L.orc_record_sums.argtypes = [I, P, P, P, I, P, P, P, P, D, D, P]
        L.orc_record_sums_t.argtypes = [I, P, P, P, I, P, P, P, P, D, D, P]
        L.orc_assemble.argtypes = [I, P, P, P, D, D, P]
        L.orc_gesv.argtypes = [I, P, I, P]
        L.orc_gesv.restype = ctypes.c_int
        L.orc_energy_row.argtypes = [I, P, P, P, D, D, I, P, P, P]
        L.orc_energy.argtypes = [I, P, P, P, D, D, I, P, P, P, P]
        L.orc_energy.restype = D
        L.orc_grad.argtypes = [I, P, P, P, D, D, D, I, P, P, P, P, P, P]
        L.orc_potential.argtypes = [I, P, P, P, D, D, P, I, P, ctypes.c_int, I, P, P, D, P]
        L.orc_coulomb.argtypes = [I, P, P, D]
        L.orc_coulomb.restype = D
        _lib = L
    return _lib


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------- pair level
def green(x, nx, y, ny, kappa):
    """[G0, Gk, dG0/dnu_y, dGk/dnu_y, dG0/dnu_x, dGk/dnu_x, d2G0, d2Gk] at one pair."""
    out = np.zeros(8)
    x, nx, y, ny = _c(x), _c(nx), _c(y), _c(ny)
    lib().orc_green(_p(x), _p(nx), _p(y), _p(ny), kappa, _p(out))
    return out


def kernels(x, nx, y, ny, eps, kappa):
    """[K1, K2, K3, K4] at one pair (target x with normal nx, source y with ny)."""
    out = np.zeros(4)
    x, nx, y, ny = _c(x), _c(nx), _c(y), _c(ny)
    lib().orc_kernels(_p(x), _p(nx), _p(y), _p(ny), eps, kappa, _p(out))
    return out


# ---------------------------------------------------------------- passes
def source(x, nrm, y, q, eps_in):
    """b = [S1; S2] (length 2N) for one charge set."""
    x, nrm, y, q = _c(x), _c(nrm), _c(y), _c(q)
    n, nc = x.shape[0], q.shape[0]
    b = np.zeros(2 * n)
    lib().orc_source(n, _p(x), _p(nrm), nc, _p(y), _p(q), eps_in, _p(b))
    return b


def matvec(x, nrm, area, eps, kappa, u):
    x, nrm, area, u = _c(x), _c(nrm), _c(area), _c(u)
    n = x.shape[0]
    out = np.zeros(2 * n)
    lib().orc_matvec(n, _p(x), _p(nrm), _p(area), eps, kappa, _p(u), _p(out))
    return out


def matvec_rows(x, nrm, area, eps, kappa, u, rows):
    """Rows ``rows`` (indices into [0, 2N)) of A u, each summed on its own."""
    x, nrm, area, u = _c(x), _c(nrm), _c(area), _c(u)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(rows.shape[0])
    lib().orc_matvec_rows(x.shape[0], _p(x), _p(nrm), _p(area), eps, kappa, _p(u), rows.shape[0],
                          rows.ctypes.data_as(ctypes.c_void_p), _p(out))
    return out


def matvec_t_rows(x, nrm, area, eps, kappa, w, rows):
    """Rows ``rows`` (indices into [0, 2N)) of A^T w, each summed on its own."""
    x, nrm, area, w = _c(x), _c(nrm), _c(area), _c(w)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(rows.shape[0])
    lib().orc_matvec_t_rows(x.shape[0], _p(x), _p(nrm), _p(area), eps, kappa, _p(w), rows.shape[0],
                            rows.ctypes.data_as(ctypes.c_void_p), _p(out))
    return out


def matvec_t(x, nrm, area, eps, kappa, w):
    x, nrm, area, w = _c(x), _c(nrm), _c(area), _c(w)
    n = x.shape[0]
    out = np.zeros(2 * n)
    lib().orc_matvec_t(n, _p(x), _p(nrm), _p(area), eps, kappa, _p(w), _p(out))
    return out


def assemble(x, nrm, area, eps, kappa):
    x, nrm, area = _c(x), _c(nrm), _c(area)
    n = x.shape[0]
    A = np.zeros((2 * n, 2 * n))
    lib().orc_assemble(n, _p(x), _p(nrm), _p(area), eps, kappa, _p(A))
    return A


def gesv(A, B):
    """Solve A X = B by Gaussian elimination with partial pivoting (copies)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    B = np.array(B, dtype=np.float64, order="C", copy=True)
    vec = B.ndim == 1
    if vec:
        B = B[:, None].copy()
    rc = lib().orc_gesv(A.shape[0], _p(A), B.shape[1], _p(B))
    if rc != 0:
        raise np.linalg.LinAlgError(f"zero pivot in column {rc - 1}")
    return B[:, 0] if vec else B


def energy_row(x, nrm, area, eps, kappa, y, q):
    """c (length 2N) with E = 1/2 c . u in internal units."""
    x, nrm, area, y, q = _c(x), _c(nrm), _c(area), _c(y), _c(q)
    n, nc = x.shape[0], q.shape[0]
    c = np.zeros(2 * n)
    lib().orc_energy_row(n, _p(x), _p(nrm), _p(area), eps, kappa, nc, _p(y), _p(q), _p(c))
    return c


def energy(x, nrm, area, eps, kappa, y, q, u):
    """(E_sol in internal units, reaction potential at each charge)."""
    x, nrm, area, y, q, u = _c(x), _c(nrm), _c(area), _c(y), _c(q), _c(u)
    n, nc = x.shape[0], q.shape[0]
    pr = np.zeros(nc)
    e = lib().orc_energy(n, _p(x), _p(nrm), _p(area), eps, kappa, nc, _p(y), _p(q), _p(u), _p(pr))
    return e, pr


def potential(x, nrm, area, eps, kappa, u, pts, inside, y=None, q=None, eps_in=1.0):
    """Potential at points ``pts`` (internal units) from surface values u:
    Eq. eq_inside (with S1 of the charges y, q) when ``inside``, else the
    exterior representation Eq. eqbim_2 with dphi2/dnu = psi / eps."""
    x, nrm, area, u, pts = _c(x), _c(nrm), _c(area), _c(u), _c(pts, (-1, 3))
    if y is None:
        y, q = np.zeros((0, 3)), np.zeros(0)
    y, q = _c(y, (-1, 3)), _c(q)
    out = np.zeros(pts.shape[0])
    lib().orc_potential(x.shape[0], _p(x), _p(nrm), _p(area), eps, kappa, _p(u), pts.shape[0], _p(pts),
                        1 if inside else 0, q.shape[0], _p(y), _p(q), eps_in, _p(out))
    return out


def coulomb(y, q, eps_in):
    """1/2 (1/eps_in) sum over ordered pairs k != l of q_k q_l G0 (internal units)."""
    y, q = _c(y, (-1, 3)), _c(q)
    return lib().orc_coulomb(q.shape[0], _p(y), _p(q), eps_in)


def grad(x, nrm, area, eps, kappa, eps_in, y, q, u, lam):
    """(dE/dq, dE/dy) in internal units from the forward u and adjoint lam."""
    x, nrm, area, y, q, u, lam = _c(x), _c(nrm), _c(area), _c(y), _c(q), _c(u), _c(lam)
    n, nc = x.shape[0], q.shape[0]
    dq = np.zeros(nc)
    dy = np.zeros((nc, 3))
    lib().orc_grad(n, _p(x), _p(nrm), _p(area), eps, kappa, eps_in, nc, _p(y), _p(q), _p(u),
                   _p(lam), _p(dq), _p(dy))
    return dq, dy


from .gmres import gmres  # noqa: E402,F401
from . import closed_forms  # noqa: E402,F401
from . import treecode  # noqa: E402,F401
from . import precond  # noqa: E402,F401
from .solve import Solution, energy_gradient, solve, solve_adjoint  # noqa: E402,F401
