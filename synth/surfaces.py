"""Seeded triangulated surfaces and point charges (geometry only).

Recipes (all FP64, all seeded with ``numpy.random.default_rng``):

* ``icosphere(level, radius)``: the regular icosahedron (vertices on the three
  golden-ratio rectangles), each level splitting every triangle in four at its
  edge midpoints, re-projected to the sphere.  20 * 4**level triangles.
* ``displaced_icosphere(level, radius, seed)``: an icosphere whose vertices
  are moved radially to ``radius * (1 + 0.15 * S(theta, phi))`` where
  ``S = sum_{l<=8} sum_{|m|<=l} c_lm Y_lm`` with orthonormal real spherical
  harmonics and ``c_lm = N(0,1) / (l+1)**2`` drawn in (l, m) order first from
  ``default_rng(seed)``.
* ``triangle_geometry``: flat-face centroid (vertex mean), unit flat-face
  normal oriented away from the origin, and flat-face area.
* Charges: uniform in a ball, or uniform inside 80 % of a displaced surface
  (rejection sampling), values uniform in [-1, 1] e.

The surfaces replace the MSMS protein meshes of the paper's experiments
(Sec. 3, Tables 2 and 3), which need PDB structures not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS_IN = 1.0
EPS_OUT = 80.0
KAPPA = 0.1257  # 1/Angstrom, 0.15 M ionic strength (Sec. 3)
DISPLACE_AMP = 0.15
DISPLACE_LMAX = 8


# --------------------------------------------------------------------------
# icosphere
# --------------------------------------------------------------------------
def _icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [[-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0],
         [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
         [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    # orient every face so that its normal points away from the origin
    cr = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", cr, v[f].mean(axis=1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def _subdivide(v, f):
    m = f.shape[0]
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    edges = np.concatenate([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)])
    key = np.sort(edges, axis=1)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    mid = v[uniq[:, 0]] + v[uniq[:, 1]]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    nv = v.shape[0]
    ab = nv + inv[:m]
    bc = nv + inv[m:2 * m]
    ca = nv + inv[2 * m:]
    # children of face k are stored contiguously (4k .. 4k+3): the face order
    # stays spatially coherent, which keeps source tiles compact
    nf = np.stack([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                   np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], 1).reshape(-1, 3)
    return np.concatenate([v, mid]), nf


def icosphere(level: int, radius: float = 1.0):
    """Unit icosphere scaled to ``radius``; returns (vertices, faces)."""
    v, f = _icosahedron()
    for _ in range(level):
        v, f = _subdivide(v, f)
    return v * radius, f


# --------------------------------------------------------------------------
# real spherical harmonics (orthonormal), l <= lmax
# --------------------------------------------------------------------------
def _assoc_legendre(lmax, x):
    """P_l^m(x) for 0 <= m <= l <= lmax (no Condon-Shortley phase)."""
    x = np.asarray(x, dtype=np.float64)
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = {}
    pmm = np.ones_like(x)
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * sx
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = x * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def real_sph_harm_sum(coeffs, lmax, dirs):
    """S(dir) = sum_{l,m} coeffs[(l, m)] Y_lm(dir) for unit vectors ``dirs``."""
    dirs = np.asarray(dirs, dtype=np.float64)
    ct = np.clip(dirs[:, 2], -1.0, 1.0)
    ph = np.arctan2(dirs[:, 1], dirs[:, 0])
    P = _assoc_legendre(lmax, ct)
    out = np.zeros(dirs.shape[0])
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                y = norm * P[(l, 0)]
            elif m > 0:
                y = math.sqrt(2.0) * norm * P[(l, am)] * np.cos(am * ph)
            else:
                y = math.sqrt(2.0) * norm * P[(l, am)] * np.sin(am * ph)
            out += coeffs[(l, m)] * y
    return out


def _sh_coeffs(rng, lmax=DISPLACE_LMAX):
    c = {}
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            c[(l, m)] = rng.standard_normal() / (l + 1) ** 2
    return c


def _sh_bound(c, lmax=DISPLACE_LMAX):
    """Upper bound of |S| (|Y_lm| <= sqrt((2l+1)/(2 pi)) for real SH)."""
    return sum(abs(c[(l, m)]) * math.sqrt((2 * l + 1) / (2 * math.pi))
               for l in range(lmax + 1) for m in range(-l, l + 1))


def displaced_icosphere(level: int, radius: float, seed: int, amp: float = DISPLACE_AMP):
    """Returns (vertices, faces, radial_fn, rng) for the displaced sphere.

    ``radial_fn(dirs)`` gives the surface radius along unit directions; the
    returned ``rng`` has drawn only the SH coefficients, so the caller can go
    on drawing charges from the same stream.
    """
    rng = np.random.default_rng(seed)
    c = _sh_coeffs(rng)
    v, f = icosphere(level, 1.0)
    s = real_sph_harm_sum(c, DISPLACE_LMAX, v)
    fac = 1.0 + amp * s
    if fac.min() <= 0.3:
        raise ValueError("displacement too large: 1 + amp*S <= 0.3")

    def radial_fn(dirs):
        return radius * (1.0 + amp * real_sph_harm_sum(c, DISPLACE_LMAX, dirs))

    radial_fn.rmax = radius * (1.0 + amp * _sh_bound(c))
    return v * (radius * fac)[:, None], f, radial_fn, rng


# --------------------------------------------------------------------------
# per-triangle geometry
# --------------------------------------------------------------------------
def triangle_geometry(v, f):
    """Flat-face centroid, unit outward normal and area of every triangle."""
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    cen = (p0 + p1 + p2) / 3.0
    cr = np.cross(p1 - p0, p2 - p0)
    twice = np.linalg.norm(cr, axis=1)
    nrm = cr / twice[:, None]
    if np.any(np.einsum("ij,ij->i", nrm, cen) <= 0):
        raise ValueError("surface is not star-shaped about the origin")
    return np.ascontiguousarray(cen), np.ascontiguousarray(nrm), 0.5 * twice


# --------------------------------------------------------------------------
# charges
# --------------------------------------------------------------------------
def charges_in_ball(rng, n, radius):
    """Uniform in a ball: direction ~ isotropic, |p| = radius * U**(1/3)."""
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = radius * rng.random(n) ** (1.0 / 3.0)
    pos = d * rad[:, None]
    q = rng.uniform(-1.0, 1.0, n)
    return pos, q


def charges_inside_surface(rng, n, radial_fn, frac=0.8, batch=4096):
    """Uniform in {p : |p| < frac * r(p/|p|)} by rejection from a ball."""
    rb = frac * radial_fn.rmax
    out = []
    got = 0
    while got < n:
        cand = rng.uniform(-rb, rb, (batch, 3))
        rr = np.linalg.norm(cand, axis=1)
        ok = (rr < rb) & (rr > 0)
        cand, rr = cand[ok], rr[ok]
        keep = rr < frac * radial_fn(cand / rr[:, None])
        cand = cand[keep]
        out.append(cand)
        got += cand.shape[0]
    pos = np.concatenate(out)[:n]
    q = rng.uniform(-1.0, 1.0, n)
    return pos, q


# --------------------------------------------------------------------------
# named problems
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    centroids: np.ndarray  # (N, 3)
    normals: np.ndarray  # (N, 3)
    areas: np.ndarray  # (N,)
    charge_pos: np.ndarray  # (Nc, 3), or (B, Nc, 3) for one set per right-hand side
    q: np.ndarray  # (B, Nc)
    eps_in: float = EPS_IN
    eps_out: float = EPS_OUT
    kappa: float = KAPPA
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.centroids.shape[0]

    @property
    def nc(self):
        return self.charge_pos.shape[-2]

    @property
    def n_rhs(self):
        return self.q.shape[0]


def born_problem(level=3, radius=2.0, kappa=KAPPA, eps_in=EPS_IN, eps_out=EPS_OUT, charge=1.0):
    """Born ion: one charge at the centre of a sphere (icosphere level 3 -> 1280)."""
    v, f = icosphere(level, radius)
    c, n, a = triangle_geometry(v, f)
    return Problem("born", c, n, a, np.zeros((1, 3)), np.array([[charge]]),
                   eps_in, eps_out, kappa, dict(level=level, radius=radius))


def kirkwood_problem(level=5, radius=20.0, n_charges=50, charge_radius=16.0, seed=2):
    """Kirkwood sphere: charges uniform in a ball of radius 16 inside R=20."""
    v, f = icosphere(level, radius)
    c, n, a = triangle_geometry(v, f)
    rng = np.random.default_rng(seed)
    pos, q = charges_in_ball(rng, n_charges, charge_radius)
    return Problem("kirkwood", c, n, a, pos, q[None, :], meta=dict(level=level, radius=radius))


def protein_like_problem(level=6, radius=25.0, n_charges=2000, seed=3):
    """Displaced icosphere (level 6 -> 81920) with charges in its inner 80 %."""
    v, f, rfn, rng = displaced_icosphere(level, radius, seed)
    c, n, a = triangle_geometry(v, f)
    pos, q = charges_inside_surface(rng, n_charges, rfn)
    return Problem("protein_like", c, n, a, pos, q[None, :],
                   meta=dict(level=level, radius=radius, seed=seed))


def batched_charges(base: Problem, n_rhs=64, n_charges=2000, seed0=4000):
    """n_rhs charge configurations inside one surface.

    Configuration b draws its positions and then its values from
    ``default_rng(seed0 + b)``.  Returns a Problem whose ``charge_pos`` has
    shape (n_rhs, Nc, 3) and ``q`` shape (n_rhs, Nc).
    """
    seed = base.meta.get("seed", 3)
    _, _, rfn, _ = displaced_icosphere(base.meta["level"], base.meta["radius"], seed)
    pos, q = [], []
    for b in range(n_rhs):
        p, v = charges_inside_surface(np.random.default_rng(seed0 + b), n_charges, rfn)
        pos.append(p)
        q.append(v)
    return Problem("batched", base.centroids, base.normals, base.areas, np.stack(pos), np.stack(q),
                   base.eps_in, base.eps_out, base.kappa, dict(base.meta, n_rhs=n_rhs))


UNEVEN_LEVELS = (4, 4, 4, 5, 5, 5, 6, 6)


def uneven_batch_problems(levels=UNEVEN_LEVELS, seed0=4100):
    """Eight displaced spheres of 5120..81920 triangles, radii 12..25."""
    k = len(levels)
    radii = np.linspace(12.0, 25.0, k)
    ncs = np.rint(np.linspace(500, 2000, k)).astype(int)
    out = []
    for s in range(k):
        v, f, rfn, rng = displaced_icosphere(levels[s], float(radii[s]), seed0 + s)
        c, n, a = triangle_geometry(v, f)
        pos, q = charges_inside_surface(rng, int(ncs[s]), rfn)
        out.append(Problem(f"uneven{s}", c, n, a, pos, q[None, :],
                           meta=dict(level=levels[s], radius=float(radii[s]), seed=seed0 + s)))
    return out


def adjoint_problem(level=7, radius=45.0, n_charges=10000, seed=5):
    """Displaced icosphere level 7 (327680 triangles) with 10000 charges."""
    v, f, rfn, rng = displaced_icosphere(level, radius, seed)
    c, n, a = triangle_geometry(v, f)
    pos, q = charges_inside_surface(rng, n_charges, rfn)
    return Problem("adjoint", c, n, a, pos, q[None, :], meta=dict(level=level, radius=radius, seed=seed))


def two_spheres_problem(level=3, radius=5.0, gap=0.5):
    """Two icospheres of ``radius`` whose surfaces are ``gap`` apart along x,
    a +1 charge at the centre of one and a -1 charge at the centre of the
    other (near-touching surfaces, where the Krylov solve slows down)."""
    v, f = icosphere(level, radius)
    c, n, a = triangle_geometry(v, f)
    off = np.array([radius + 0.5 * gap, 0.0, 0.0])
    return Problem("two_spheres", np.concatenate([c - off, c + off]), np.concatenate([n, n]),
                   np.concatenate([a, a]), np.stack([-off, off]), np.array([[1.0, -1.0]]),
                   meta=dict(level=level, radius=radius, gap=gap))


def strongly_displaced_problem(level=3, radius=10.0, amp=0.3, seed=3, n_charges=20):
    """A displaced icosphere as in protein_like_problem with displacement
    amplitude ``amp`` (0.3 to 0.45: 30 to 45 % of the radius)."""
    v, f, rfn, rng = displaced_icosphere(level, radius, seed, amp=amp)
    c, n, a = triangle_geometry(v, f)
    pos, q = charges_inside_surface(rng, n_charges, rfn)
    return Problem("strongly_displaced", c, n, a, pos, q[None, :], meta=dict(level=level, radius=radius, amp=amp))


PROBLEM_NAMES = ("born", "kirkwood", "protein_like", "adjoint")


def problem_by_name(name: str, **kw) -> Problem:
    return {"born": born_problem, "kirkwood": kirkwood_problem,
            "protein_like": protein_like_problem, "adjoint": adjoint_problem}[name](**kw)
