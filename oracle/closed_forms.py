"""Closed-form solutions of the linearised PB model for a spherical molecule.

Test infrastructure only.  These are the continuum answers that the
centroid-collocation discretisation (Sec. 2.2.2) converges to as the
icosphere is refined; they pin the oracle to the physics rather than to
itself.

Both follow from the model of Sec. 2.1: inside the sphere (radius a,
dielectric eps_in) the potential of the point charges plus a harmonic
reaction field; outside (eps_out) a screened solution of the linearised
equation; continuity of phi and of eps dphi/dnu on the sphere.  Energies use
the 332.0716 factor of Sec. 2.1 (kcal/mol with lengths in Angstrom).
"""
from __future__ import annotations

import math

import numpy as np

COULOMB = 332.0716


def born_energy(q, a, eps_in, eps_out, kappa):
    """Solvation energy of a charge q at the centre of a sphere of radius a.

    The reaction potential at the centre is q/(eps_out a (1 + kappa a)) -
    q/(eps_in a), so E = 1/2 q * that * 332.0716 kcal/mol.
    """
    return 0.5 * COULOMB * q * q * (1.0 / (eps_out * a * (1.0 + kappa * a)) - 1.0 / (eps_in * a))


def born_surface(q, a, eps_in, eps_out, kappa):
    """(phi, dphi/dnu inside) on the sphere, kcal/mol/e and kcal/mol/e/A.

    Outside, phi = q exp(-kappa (r - a)) / (eps_out r (1 + kappa a)), so the
    surface value is q/(eps_out a (1 + kappa a)); flux continuity with
    Gauss's law gives eps_in dphi/dnu = -q / a**2 on the inner side.
    """
    phi = COULOMB * q / (eps_out * a * (1.0 + kappa * a))
    dphi = -COULOMB * q / (eps_in * a * a)
    return phi, dphi


def born_potential(r, q, a, eps_in, eps_out, kappa):
    """Potential (kcal/mol/e) at distance r from a charge q at the centre of
    the sphere: inside, the charge's Coulomb potential plus the constant
    reaction potential of born_energy; outside, the screened field whose
    surface value born_surface gives."""
    r = np.asarray(r, dtype=np.float64)
    inside = q / (eps_in * r) + q * (1.0 / (eps_out * a * (1.0 + kappa * a)) - 1.0 / (eps_in * a))
    outside = q * np.exp(-kappa * (r - a)) / (eps_out * (1.0 + kappa * a) * r)
    return COULOMB * np.where(r < a, inside, outside)


def _log_deriv_k(nmax, z):
    """lambda_n = z k_n'(z) / k_n(z) for the modified spherical Bessel k_n.

    With rho_n = k_{n-1}/k_n (rho_0 = 1 since k_{-1} = k_0), the recurrence
    k_{n+1} = k_{n-1} + (2n+1)/z k_n gives rho_{n+1} = 1/(rho_n + (2n+1)/z),
    and k_n' = -k_{n-1} - (n+1)/z k_n gives lambda_n = -z rho_n - (n+1).
    For z = 0 (no salt) lambda_n = -(n+1).
    """
    lam = np.empty(nmax + 1)
    if z == 0.0:
        for n in range(nmax + 1):
            lam[n] = -(n + 1.0)
        return lam
    rho = 1.0
    for n in range(nmax + 1):
        lam[n] = -z * rho - (n + 1.0)
        rho = 1.0 / (rho + (2 * n + 1) / z)
    return lam


def kirkwood_energy(pos, q, a, eps_in, eps_out, kappa, nmax=60):
    """Solvation energy (kcal/mol) of point charges inside a sphere of radius a.

    Expanding the Coulomb field of charge k in Legendre polynomials and
    matching the interior reaction field B_n r^n P_n and the exterior
    screened field C_n k_n(kappa r) P_n at r = a gives, for each order n,

        B_n = (q_k / eps_in) r_k^n / a^(2n+1)
              * (eps_in (n+1) + eps_out lambda_n) / (eps_in n - eps_out lambda_n)

    and E = 1/2 * 332.0716 * sum_{k,l} q_l B_n(k) r_l^n P_n(cos gamma_kl),
    including k = l.  The n = 0 term of a centred charge is the Born energy.
    """
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    r = np.linalg.norm(pos, axis=1)
    lam = _log_deriv_k(nmax, kappa * a)
    fac = (eps_in * (np.arange(nmax + 1) + 1.0) + eps_out * lam) / (eps_in * np.arange(nmax + 1) - eps_out * lam)
    # cos of the angle between every pair (1 where either charge is at the centre)
    rr = np.outer(r, r)
    with np.errstate(invalid="ignore", divide="ignore"):
        cosg = np.where(rr > 0, (pos @ pos.T) / np.where(rr > 0, rr, 1.0), 1.0)
    cosg = np.clip(cosg, -1.0, 1.0)
    x = rr / (a * a)
    total = np.zeros_like(x)
    p_prev, p_n = None, np.ones_like(cosg)  # P_{n-1}, P_n (Legendre, 3-term recurrence)
    xn = np.ones_like(x)
    for n in range(nmax + 1):
        total += xn * (fac[n] / (eps_in * a)) * p_n
        xn = xn * x
        p_next = cosg.copy() if n == 0 else ((2 * n + 1) * cosg * p_n - n * p_prev) / (n + 1)
        p_prev, p_n = p_n, p_next
    return 0.5 * COULOMB * float(q @ total @ q)


def kirkwood_denergy_dr(r_k, a, eps_in, eps_out, kappa, nmax=60, q=1.0):
    """d E / d r for a single charge q at distance r from the centre (kcal/mol/A)."""
    lam = _log_deriv_k(nmax, kappa * a)
    s = 0.0
    for n in range(1, nmax + 1):
        fac = (eps_in * (n + 1.0) + eps_out * lam[n]) / (eps_in * n - eps_out * lam[n])
        s += fac * 2 * n * r_k ** (2 * n - 1) / a ** (2 * n + 1)
    return 0.5 * COULOMB * q * q * s / eps_in


def kirkwood_reaction_potential(pos, q, pts, a, eps_in, eps_out, kappa, nmax=60):
    """Reaction potential (kcal/mol/e) at points inside the sphere: the field
    sum_k sum_n B_n(k) r^n P_n(cos gamma) of kirkwood_energy evaluated at
    each point (gamma the angle between the point and charge k)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    rk = np.linalg.norm(pos, axis=1)
    rp = np.linalg.norm(pts, axis=1)
    lam = _log_deriv_k(nmax, kappa * a)
    fac = (eps_in * (np.arange(nmax + 1) + 1.0) + eps_out * lam) / (eps_in * np.arange(nmax + 1) - eps_out * lam)
    rr = np.outer(rp, rk)
    with np.errstate(invalid="ignore", divide="ignore"):
        cosg = np.where(rr > 0, (pts @ pos.T) / np.where(rr > 0, rr, 1.0), 1.0)
    cosg = np.clip(cosg, -1.0, 1.0)
    x = rr / (a * a)
    total = np.zeros_like(x)
    p_prev, p_n = None, np.ones_like(cosg)
    xn = np.ones_like(x)
    for n in range(nmax + 1):
        total += xn * (fac[n] / (eps_in * a)) * p_n
        xn = xn * x
        p_next = cosg.copy() if n == 0 else ((2 * n + 1) * cosg * p_n - n * p_prev) / (n + 1)
        p_prev, p_n = p_n, p_next
    return COULOMB * (total @ q)
