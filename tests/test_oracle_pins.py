"""Pins of the FP64 CPU oracle to mathematics outside itself (no GPU).

Each test checks the oracle against something it does not compute the same
way: finite differences of the Green's functions, closed-form continuum
solutions (Born ion, Kirkwood sphere), library routines (LAPACK solve,
scipy's spherical Bessel functions), exact algebraic invariants of the
discrete system, and brute force on tiny meshes.  A dropped term, a wrong
sign or a transposed operand in the oracle breaks at least one of them.
"""
import math

import numpy as np
import pytest

import synth
from oracle import closed_forms as cf

EPS_IN, EPS_OUT, KAPPA = 1.0, 80.0, 0.1257


def _G0(x, y):
    return 1.0 / (4 * math.pi * np.linalg.norm(np.asarray(x) - np.asarray(y)))


def _Gk(x, y, kappa):
    r = np.linalg.norm(np.asarray(x) - np.asarray(y))
    return math.exp(-kappa * r) / (4 * math.pi * r)


def _unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


# ------------------------------------------------------------------ kernels
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_normal_derivatives_match_finite_differences(orc, seed):
    """d/dnu_x = +n_x.grad_x, d/dnu_y = +n_y.grad_y, mixed = +n_x n_y : grad grad.

    Central differences along the normals; this fixes the sign reading of
    the x-derivatives (Sec. 2.2.1 prints a leading minus there)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-2, 2, 3)
    y = x + _unit(rng.standard_normal(3)) * rng.uniform(0.5, 3.0)
    nx, ny = _unit(rng.standard_normal(3)), _unit(rng.standard_normal(3))
    g = orc.green(x, nx, y, ny, KAPPA)
    h = 1e-4
    for idx, G in ((0, lambda a, b: _G0(a, b)), (1, lambda a, b: _Gk(a, b, KAPPA))):
        assert g[idx] == pytest.approx(G(x, y), rel=1e-13)
        dy = (G(x, y + h * ny) - G(x, y - h * ny)) / (2 * h)
        dx = (G(x + h * nx, y) - G(x - h * nx, y)) / (2 * h)
        dxy = (G(x + h * nx, y + h * ny) - G(x + h * nx, y - h * ny)
               - G(x - h * nx, y + h * ny) + G(x - h * nx, y - h * ny)) / (4 * h * h)
        assert g[2 + idx] == pytest.approx(dy, rel=1e-6, abs=1e-12)
        assert g[4 + idx] == pytest.approx(dx, rel=1e-6, abs=1e-12)
        assert g[6 + idx] == pytest.approx(dxy, rel=1e-5, abs=1e-10)


def test_kernels_vanish_without_salt_and_contrast(orc):
    """kappa = 0 makes K1 = K4 = 0; additionally eps = 1 makes K2 = K3 = 0."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        x, y = rng.uniform(-3, 3, 3), rng.uniform(-3, 3, 3)
        nx, ny = _unit(rng.standard_normal(3)), _unit(rng.standard_normal(3))
        K = orc.kernels(x, nx, y, ny, 80.0, 0.0)
        assert abs(K[0]) < 1e-16 and abs(K[3]) < 1e-14
        assert abs(K[1]) > 0 and abs(K[2]) > 0
        K = orc.kernels(x, nx, y, ny, 1.0, 0.0)
        assert np.all(np.abs(K) < 1e-14)


def test_kernels_are_the_paper_combinations(orc):
    """K1 = G0-Gk, K2 = eps dGk/dnu_y - dG0/dnu_y, K3 = dG0/dnu_x - dGk/dnu_x/eps,
    K4 = d2Gk - d2G0 (Eqs. for K1-K4), built from the FD-pinned derivatives."""
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-3, 3, 3), rng.uniform(-3, 3, 3)
    nx, ny = _unit(rng.standard_normal(3)), _unit(rng.standard_normal(3))
    g = orc.green(x, nx, y, ny, KAPPA)
    K = orc.kernels(x, nx, y, ny, 80.0, KAPPA)
    np.testing.assert_allclose(K, [g[0] - g[1], 80 * g[3] - g[2], g[4] - g[5] / 80, g[7] - g[6]], rtol=1e-14)


# ------------------------------------------------------------------ linear algebra
@pytest.fixture(scope="module")
def small():
    p = synth.kirkwood_problem(level=1, radius=5.0, n_charges=4, charge_radius=3.0)
    return p


def test_dense_matches_matrix_free(orc, small):
    p = small
    eps = p.eps_out / p.eps_in
    A = orc.assemble(p.centroids, p.normals, p.areas, eps, p.kappa)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(2 * p.n)
    np.testing.assert_allclose(orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u), A @ u,
                               rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(orc.matvec_t(p.centroids, p.normals, p.areas, eps, p.kappa, u), A.T @ u,
                               rtol=1e-13, atol=1e-13)


def test_sampled_rows_match_full_matvec(orc, small):
    p = small
    eps = p.eps_out / p.eps_in
    u = np.random.default_rng(8).standard_normal(2 * p.n)
    full = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u)
    rows = np.array([0, 5, p.n - 1, p.n, 2 * p.n - 1])
    np.testing.assert_array_equal(orc.matvec_rows(p.centroids, p.normals, p.areas, eps, p.kappa, u, rows), full[rows])


def test_sampled_transpose_rows_match_dense_transpose(orc, small):
    """Rows of A^T w summed one by one equal the rows of the dense A^T w."""
    p = small
    eps = p.eps_out / p.eps_in
    A = orc.assemble(p.centroids, p.normals, p.areas, eps, p.kappa)
    w = np.random.default_rng(18).standard_normal(2 * p.n)
    rows = np.array([0, 7, p.n - 1, p.n, p.n + 3, 2 * p.n - 1])
    got = orc.matvec_t_rows(p.centroids, p.normals, p.areas, eps, p.kappa, w, rows)
    np.testing.assert_allclose(got, (A.T @ w)[rows], rtol=1e-13, atol=1e-13 * np.abs(A.T @ w).max())


def test_dense_entries_brute_force(orc, small):
    """Every entry of A rebuilt pair by pair from the kernels (Eqs. 5-6)."""
    p = small
    eps = p.eps_out / p.eps_in
    A = orc.assemble(p.centroids, p.normals, p.areas, eps, p.kappa)
    n = p.n
    for i in (0, 3, n - 1):
        for j in range(n):
            if i == j:
                assert A[i, j] == 0.5 * (1 + eps) and A[n + i, n + j] == 0.5 * (1 + 1 / eps)
                assert A[i, n + j] == 0 and A[n + i, j] == 0
                continue
            K = orc.kernels(p.centroids[i], p.normals[i], p.centroids[j], p.normals[j], eps, p.kappa)
            a = p.areas[j]
            assert A[i, j] == pytest.approx(-K[1] * a, rel=1e-15)
            assert A[i, n + j] == pytest.approx(-K[0] * a, rel=1e-15)
            assert A[n + i, j] == pytest.approx(-K[3] * a, rel=1e-15)
            assert A[n + i, n + j] == pytest.approx(-K[2] * a, rel=1e-15)


def test_gesv_matches_lapack(orc):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((60, 60)) + 10 * np.eye(60)
    B = rng.standard_normal((60, 3))
    np.testing.assert_allclose(orc.gesv(A, B), np.linalg.solve(A, B), rtol=1e-12, atol=1e-13)


def test_gmres_matches_direct_solve(orc):
    p = synth.born_problem(level=2)
    d = orc.solve(p, method="direct")
    g = orc.solve(p, method="gmres", tol=1e-13, max_iter=300)
    assert g.info["converged"]
    np.testing.assert_allclose(g.u, d.u, rtol=1e-11, atol=1e-12 * np.abs(d.u).max())
    assert g.energy_kcal == pytest.approx(d.energy_kcal, rel=1e-11)


def test_gmres_on_random_system_matches_lapack(orc):
    rng = np.random.default_rng(11)
    A = np.eye(200) + rng.standard_normal((200, 200)) / 40
    b = rng.standard_normal(200)
    x, info = orc.gmres(lambda v: A @ v, b, tol=1e-13, restart=10, max_iter=2000)
    assert info["converged"]
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-11)
    # history is the true residual of the iterate at each Arnoldi step within a cycle
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(info["history"], info["history"][1:]))


def test_identity_operator_when_no_contrast(orc):
    """eps_in = eps_out and kappa = 0: all kernels vanish, A = I, u = b,
    E_sol = 0 and GMRES stops after one step."""
    p = synth.born_problem(level=2, kappa=0.0, eps_in=2.0, eps_out=2.0)
    A = orc.assemble(p.centroids, p.normals, p.areas, 1.0, 0.0)
    np.testing.assert_allclose(A, np.eye(2 * p.n), atol=1e-15)
    s = orc.solve(p, method="gmres", tol=1e-12)
    assert s.info["iters"] == 1
    np.testing.assert_allclose(s.u, s.b, rtol=1e-14)
    assert abs(s.energy_kcal) < 1e-12


def test_adjoint_identity(orc):
    p = synth.protein_like_problem(level=2, n_charges=5)
    eps = p.eps_out / p.eps_in
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal(2 * p.n), rng.standard_normal(2 * p.n)
    Au = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u)
    ATv = orc.matvec_t(p.centroids, p.normals, p.areas, eps, p.kappa, v)
    assert np.dot(Au, v) == pytest.approx(np.dot(u, ATv), rel=1e-12)


def test_thread_count_invariance(orc):
    p = synth.protein_like_problem(level=2, n_charges=5)
    eps = p.eps_out / p.eps_in
    u = np.random.default_rng(4).standard_normal(2 * p.n)
    nt = orc.num_threads()
    try:
        orc.set_threads(1)
        a = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u)
        orc.set_threads(max(2, nt))
        b = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u)
    finally:
        orc.set_threads(nt)
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ closed forms
def test_born_value():
    """Config value: a = 2, q = +1, eps 1/80, kappa 0.1257."""
    assert cf.born_energy(1.0, 2.0, 1.0, 80.0, 0.1257) == pytest.approx(-82.18864976, abs=1e-7)


def test_kirkwood_reduces_to_born():
    for kappa in (0.0, 0.1257):
        assert cf.kirkwood_energy([[0, 0, 0]], [1.3], 3.0, 2.0, 80.0, kappa) == pytest.approx(
            cf.born_energy(1.3, 3.0, 2.0, 80.0, kappa), rel=1e-14)


def test_kirkwood_bessel_ratio_matches_scipy():
    special = pytest.importorskip("scipy.special")
    z = 0.1257 * 20.0
    lam = cf._log_deriv_k(30, z)
    for n in range(31):
        ref = z * special.spherical_kn(n, z, derivative=True) / special.spherical_kn(n, z)
        assert lam[n] == pytest.approx(ref, rel=1e-12)


def test_kirkwood_no_salt_textbook_form():
    """kappa = 0: the order-n factor is (n+1)(eps_in - eps_out)/(eps_in n + eps_out (n+1))."""
    rng = np.random.default_rng(9)
    pos = rng.uniform(-2, 2, (3, 3))
    q = rng.uniform(-1, 1, 3)
    a, ei, eo = 5.0, 2.0, 80.0
    r = np.linalg.norm(pos, axis=1)
    e = 0.0
    for k in range(3):
        for l in range(3):
            c = np.dot(pos[k], pos[l]) / (r[k] * r[l])
            P = np.polynomial.legendre.legval(c, np.eye(61))  # P_0..P_60
            for n in range(61):
                e += q[k] * q[l] * (r[k] * r[l]) ** n / a ** (2 * n + 1) * (n + 1) * (ei - eo) / (
                    ei * n + eo * (n + 1)) * P[n] / ei
    assert cf.kirkwood_energy(pos, q, a, ei, eo, 0.0) == pytest.approx(0.5 * 332.0716 * e, rel=1e-12)


def test_born_convergence_across_levels(orc):
    """Energy and surface phi / dphi/dnu converge to the Born closed form."""
    exact = cf.born_energy(1.0, 2.0, EPS_IN, EPS_OUT, KAPPA)
    phi_ex, dphi_ex = cf.born_surface(1.0, 2.0, EPS_IN, EPS_OUT, KAPPA)
    errs, perr, derr = [], [], []
    for lev in (1, 2, 3):
        s = orc.solve(synth.born_problem(level=lev), method="direct")
        errs.append(abs(s.energy_kcal / exact - 1))
        phi, dphi = s.surface_potential()
        perr.append(np.abs(phi / phi_ex - 1).max())
        derr.append(np.abs(dphi / dphi_ex - 1).max())
    assert errs[2] < 0.02
    for e in (errs, perr, derr):
        assert e[0] > 2.5 * e[1] > 2.5 * 2.5 * e[2] * 0.9


def test_kirkwood_convergence_across_levels(orc):
    p0 = synth.kirkwood_problem(level=2)
    exact = cf.kirkwood_energy(p0.charge_pos, p0.q[0], 20.0, EPS_IN, EPS_OUT, KAPPA)
    errs = []
    for lev in (2, 3, 4):
        s = orc.solve(synth.kirkwood_problem(level=lev), method="gmres", tol=1e-10, max_iter=300)
        assert s.info["converged"]
        errs.append(abs(s.energy_kcal / exact - 1))
    assert errs[0] > 2.5 * errs[1] and errs[1] > 2.5 * errs[2]
    assert errs[2] < 0.02


# ------------------------------------------------------------------ solute dielectric eps_in != 1
# S1 and S2 carry 1/eps_in (Sec. 2.2.1), and so do the source-column terms of
# the gradient.  With eps_in = 1 that factor is invisible; these pins fix it:
# without it b, and with it u and E, come out eps_in times too large.
@pytest.mark.parametrize("eps_in", [2.0, 4.0])
def test_born_convergence_with_solute_dielectric(orc, eps_in):
    """Born energy and surface values at eps_in = 2 and 4 converge to the
    closed form, whose reaction term carries 1/eps_in and whose inner normal
    derivative is -q / (eps_in a^2) (Gauss's law in the solute)."""
    exact = cf.born_energy(1.0, 2.0, eps_in, EPS_OUT, KAPPA)
    phi_ex, dphi_ex = cf.born_surface(1.0, 2.0, eps_in, EPS_OUT, KAPPA)
    errs, perr, derr = [], [], []
    for lev in (1, 2, 3):
        s = orc.solve(synth.born_problem(level=lev, eps_in=eps_in), method="direct")
        errs.append(abs(s.energy_kcal / exact - 1))
        phi, dphi = s.surface_potential()
        perr.append(np.abs(phi / phi_ex - 1).max())
        derr.append(np.abs(dphi / dphi_ex - 1).max())
    assert errs[2] < 0.03 and perr[2] < 0.03 and derr[2] < 0.03
    for e in (errs, perr, derr):
        assert e[0] > 2.5 * e[1] > 2.5 * 2.5 * e[2] * 0.9


def test_kirkwood_convergence_with_solute_dielectric(orc):
    """Kirkwood sphere with eps_in = 2: the series (every order carries
    1/eps_in) is approached level by level."""
    p0 = synth.kirkwood_problem(level=2)
    exact = cf.kirkwood_energy(p0.charge_pos, p0.q[0], 20.0, 2.0, EPS_OUT, KAPPA)
    errs = []
    for lev in (2, 3, 4):
        p = synth.kirkwood_problem(level=lev)
        p.eps_in = 2.0
        s = orc.solve(p, method="gmres", tol=1e-10, max_iter=300)
        assert s.info["converged"]
        errs.append(abs(s.energy_kcal / exact - 1))
    assert errs[0] > 2.5 * errs[1] and errs[1] > 2.5 * errs[2]
    assert errs[2] < 0.02


def test_gradient_matches_finite_differences_with_solute_dielectric(orc):
    """dE/dq and dE/dy at eps_in = 2 against central differences of solved
    energies: the adjoint's source-column term must carry 1/eps_in."""
    def prob():
        p = synth.kirkwood_problem(level=2, radius=8.0, n_charges=3, charge_radius=5.0)
        p.eps_in = 2.0
        return p

    p = prob()
    e, dq, dy = orc.energy_gradient(p, method="direct")
    h = 1e-4
    for k in range(3):
        for m in range(3):
            pp = prob()
            pp.charge_pos = p.charge_pos.copy()
            pp.charge_pos[k, m] += h
            ep = orc.solve(pp, method="direct").energy_kcal
            pp.charge_pos[k, m] -= 2 * h
            em = orc.solve(pp, method="direct").energy_kcal
            assert dy[k, m] == pytest.approx((ep - em) / (2 * h), rel=2e-6, abs=1e-7 * abs(e))
        pq = prob()
        pq.q = p.q.copy()
        pq.q[0, k] += 0.01
        ep = orc.solve(pq, method="direct").energy_kcal
        pq.q[0, k] -= 0.02
        em = orc.solve(pq, method="direct").energy_kcal
        assert dq[k] == pytest.approx((ep - em) / 0.02, rel=1e-9)


# ------------------------------------------------------------------ invariants of E
def test_energy_quadratic_in_charges(orc):
    p = synth.kirkwood_problem(level=2, n_charges=6)
    e1 = orc.solve(p, method="direct").energy_kcal
    p.q = 3.0 * p.q
    e3 = orc.solve(p, method="direct").energy_kcal
    assert e3 == pytest.approx(9.0 * e1, rel=1e-13)


def test_solution_linear_in_rhs(orc):
    p = synth.kirkwood_problem(level=2, n_charges=6)
    q = p.q[0].copy()
    qa, qb = q * 0.0, q * 0.0
    qa[:3], qb[3:] = q[:3], q[3:]
    p.q = np.stack([q, qa, qb])
    s, sa, sb = (orc.solve(p, rhs=r, method="direct") for r in range(3))
    np.testing.assert_allclose(s.u, sa.u + sb.u, rtol=1e-12, atol=1e-14 * np.abs(s.u).max())


def test_energy_rigid_motion_invariance(orc):
    p = synth.protein_like_problem(level=2, n_charges=8)
    e0 = orc.solve(p, method="direct").energy_kcal
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    R = Rz @ Rx
    t = np.array([3.0, -7.5, 12.25])
    p.centroids = p.centroids @ R.T + t
    p.normals = p.normals @ R.T
    p.charge_pos = p.charge_pos @ R.T + t
    e1 = orc.solve(p, method="direct").energy_kcal
    assert e1 == pytest.approx(e0, rel=1e-11)


def test_reaction_matrix_nearly_symmetric(orc):
    """R_kl = phi_reac(y_k; unit charge at l) is symmetric in the continuum;
    the discrete asymmetry shrinks with refinement (never tested at 1e-10)."""
    asym = []
    rng = np.random.default_rng(12)
    pos = rng.uniform(-6, 6, (4, 3))
    for lev in (2, 3):
        p = synth.kirkwood_problem(level=lev, radius=12.0, n_charges=4)
        p.charge_pos = pos
        p.q = np.eye(4)
        R = np.stack([orc.solve(p, rhs=l, method="direct").phi_reac for l in range(4)], axis=1)
        asym.append(np.linalg.norm(R - R.T) / np.linalg.norm(R))
    assert asym[1] < asym[0] < 0.05


# ------------------------------------------------------------------ gradient
def test_euler_identity(orc):
    """E is homogeneous of degree 2 in q: sum_k q_k dE/dq_k = 2E exactly."""
    p = synth.kirkwood_problem(level=2, n_charges=5)
    e, dq, _ = orc.energy_gradient(p, method="direct")
    assert np.dot(p.q[0], dq) == pytest.approx(2 * e, rel=1e-12)


def test_gradient_matches_finite_differences(orc):
    p = synth.kirkwood_problem(level=2, radius=8.0, n_charges=3, charge_radius=5.0)
    e, dq, dy = orc.energy_gradient(p, method="direct")
    h = 1e-4
    for k in range(3):
        for m in range(3):
            pp = synth.kirkwood_problem(level=2, radius=8.0, n_charges=3, charge_radius=5.0)
            pp.charge_pos = p.charge_pos.copy()
            pp.charge_pos[k, m] += h
            ep = orc.solve(pp, method="direct").energy_kcal
            pp.charge_pos[k, m] -= 2 * h
            em = orc.solve(pp, method="direct").energy_kcal
            assert dy[k, m] == pytest.approx((ep - em) / (2 * h), rel=2e-6, abs=1e-7 * abs(e))
        pq = synth.kirkwood_problem(level=2, radius=8.0, n_charges=3, charge_radius=5.0)
        pq.q = p.q.copy()
        pq.q[0, k] += 0.01
        ep = orc.solve(pq, method="direct").energy_kcal
        pq.q[0, k] -= 0.02
        em = orc.solve(pq, method="direct").energy_kcal
        assert dq[k] == pytest.approx((ep - em) / 0.02, rel=1e-9)


def test_born_centred_force_vanishes(orc):
    p = synth.born_problem(level=2)
    _, _, dy = orc.energy_gradient(p, method="direct")
    assert np.abs(dy).max() < 1e-10


def test_kirkwood_radial_force(orc):
    """One off-centre charge: dE/dr -> the derivative of the Kirkwood series."""
    a, rk = 6.0, 3.0
    exact = cf.kirkwood_denergy_dr(rk, a, EPS_IN, EPS_OUT, KAPPA)
    errs = []
    for lev in (2, 3):
        p = synth.born_problem(level=lev, radius=a)
        d = _unit([0.3, -0.5, 0.8])
        p.charge_pos = (rk * d)[None, :]
        _, _, dy = orc.energy_gradient(p, method="direct")
        errs.append(abs(np.dot(dy[0], d) / exact - 1))
    assert errs[1] < errs[0] < 0.3


# ------------------------------------------------------------------ potential off the surface, Coulomb energy
def _born_points(scale_in, scale_out):
    dirs = np.array([[1.0, 0.0, 0.0], [0.3, 0.5, 0.8], [-0.6, 0.2, -0.7]])
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    return np.concatenate([s * dirs for s in scale_in]), np.concatenate([s * dirs for s in scale_out])


def test_point_potential_born_exact_surface_data(orc):
    """With the exact Born surface values, Eq. eq_inside (inside, with the
    centre charge's S1) and the exterior representation reproduce the closed
    form up to the centroid-rule quadrature error, which falls 4x per level."""
    pin, pout = _born_points((0.5, 1.2), (3.0, 6.0))
    ein, eout = [], []
    for lev in (2, 3, 4):
        p = synth.born_problem(level=lev, eps_in=2.0)  # eps_in != 1 so that S1's 1/eps_in counts
        n = p.centroids.shape[0]
        phi, dphi = cf.born_surface(1.0, 2.0, p.eps_in, p.eps_out, p.kappa)
        u = np.concatenate([np.full(n, phi / orc.KCAL), np.full(n, dphi / orc.KCAL)])
        eps = p.eps_out / p.eps_in
        vi = orc.KCAL * orc.potential(p.centroids, p.normals, p.areas, eps, p.kappa, u, pin, True,
                                      np.zeros((1, 3)), np.array([1.0]), p.eps_in)
        vo = orc.KCAL * orc.potential(p.centroids, p.normals, p.areas, eps, p.kappa, u, pout, False)
        ri, ro = np.linalg.norm(pin, axis=1), np.linalg.norm(pout, axis=1)
        ein.append(np.abs(vi / cf.born_potential(ri, 1.0, 2.0, p.eps_in, p.eps_out, p.kappa) - 1).max())
        eout.append(np.abs(vo / cf.born_potential(ro, 1.0, 2.0, p.eps_in, p.eps_out, p.kappa) - 1).max())
    for e in (ein, eout):
        assert e[0] > 3.5 * e[1] > 3.5 * 3.5 * e[2]
    assert ein[2] < 1e-3 and eout[2] < 2e-3


def test_point_potential_kirkwood_reaction_field(orc):
    """The surface integral of Eq. eq_inside alone (no charges passed) is the
    reaction potential; from the oracle's own solve it converges to the
    Kirkwood series at interior points as the sphere is refined."""
    pts = np.array([[3.0, 1.0, -2.0], [-8.0, 4.0, 5.0], [0.0, -10.0, 2.0]])
    errs = []
    for lev in (2, 3, 4):
        p = synth.kirkwood_problem(level=lev, n_charges=5)
        y = p.charge_pos if p.charge_pos.ndim == 2 else p.charge_pos[0]
        s = orc.solve(p, method="gmres", tol=1e-11, max_iter=400)
        v = orc.KCAL * orc.potential(p.centroids, p.normals, p.areas, p.eps_out / p.eps_in, p.kappa, s.u, pts,
                                     True)
        ex = cf.kirkwood_reaction_potential(y, p.q[0], pts, 20.0, p.eps_in, p.eps_out, p.kappa)
        errs.append(np.abs(v - ex).max() / np.abs(ex).max())
    assert errs[0] > 2.0 * errs[1] > 2.0 * 2.0 * errs[2]
    assert errs[2] < 0.02


def test_exterior_potential_far_field_is_total_charge(orc):
    """Without salt the exterior potential far away is that of the total
    charge in the solvent dielectric, Q / (eps_out R) (Gauss's law), for
    the oracle's discrete solution of an off-centre charge set."""
    p = synth.kirkwood_problem(level=3, n_charges=4)
    p.kappa = 0.0
    s = orc.solve(p, method="gmres", tol=1e-11, max_iter=400)
    dirs = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [-0.5, 0.5, -0.7]])
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    R = 20000.0
    v = orc.KCAL * orc.potential(p.centroids, p.normals, p.areas, p.eps_out / p.eps_in, 0.0, s.u, R * dirs, False)
    Q = float(np.sum(p.q[0]))
    # the discrete solution's flux is off by its discretisation error (1.7 % at
    # level 3, 0.9 % at level 4); a dropped or flipped term is off by O(1)
    np.testing.assert_allclose(v, 332.0716 * Q / (p.eps_out * R), rtol=0.03)


def test_coulomb_energy_textbook_values(orc):
    """Two unit charges 1 A apart in vacuum: 332.0716 kcal/mol; charges
    (1, 1, -1) on an equilateral triangle of side 2 in eps_in = 4: the three
    pair terms sum to -1, so E = -332.0716 / (4 * 2).  Rigid motions and a
    permutation leave it unchanged; scaling the lengths by s scales it by 1/s."""
    e2 = orc.KCAL * orc.coulomb(np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]]), np.array([1.0, 1.0]), 1.0)
    assert e2 == pytest.approx(332.0716, rel=1e-14)
    tri = 2.0 * np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, math.sqrt(3) / 2, 0.0]])
    q = np.array([1.0, 1.0, -1.0])
    e3 = orc.KCAL * orc.coulomb(tri, q, 4.0)
    assert e3 == pytest.approx(-332.0716 / 8.0, rel=1e-13)
    rng = np.random.default_rng(9)
    y = rng.standard_normal((7, 3))
    qq = rng.standard_normal(7)
    e = orc.coulomb(y, qq, 2.0)
    c, sn = math.cos(0.7), math.sin(0.7)
    Rm = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
    perm = rng.permutation(7)
    assert orc.coulomb(y @ Rm.T + [3.0, -1.0, 2.0], qq, 2.0) == pytest.approx(e, rel=1e-12)
    assert orc.coulomb(y[perm], qq[perm], 2.0) == pytest.approx(e, rel=1e-12)
    assert orc.coulomb(2.5 * y, qq, 2.0) == pytest.approx(e / 2.5, rel=1e-12)


# ------------------------------------------------------------------ far-field treecode (Sec. 2.2.3)
@pytest.fixture(scope="module")
def tc_surface():
    return synth.protein_like_problem(level=4, n_charges=5)


def test_treecode_tree_and_lists_partition_every_pair(orc, tc_surface):
    """The tree splits at the median of the longest side, leaves hold at most
    N0 elements, and every leaf's list covers every source element exactly
    once (directly or inside one far cluster); every far cluster meets the
    particle-cluster MAC r_c / |x - x_c| <= theta for each target of the leaf."""
    tc = orc.treecode
    p = tc_surface
    theta, deg, leaf = 0.6, 4, 64
    t = tc.build_tree(p.centroids, leaf)
    n = p.n
    assert sorted(t.perm.tolist()) == list(range(n))
    for k, ch in enumerate(t.child):
        if ch is None:
            assert t.end[k] - t.start[k] <= leaf
            continue
        l, r = ch
        assert t.start[l] == t.start[k] and t.end[l] == t.start[r] and t.end[r] == t.end[k]
        assert t.end[l] - t.start[l] == (t.end[k] - t.start[k]) // 2
        d = int(np.argmax(t.hi[k] - t.lo[k]))
        assert p.centroids[t.perm[t.start[l]:t.end[l]], d].max() <= p.centroids[t.perm[t.start[r]:t.end[r]], d].min()
    lists = tc.interaction_lists(t, theta, deg)
    n_far = 0
    for li, b in enumerate(t.leaves):
        cover = np.zeros(n, dtype=int)
        tgt = p.centroids[t.perm[t.start[b]:t.end[b]]]
        for e in lists[li]:
            if e[0] == "direct":
                cover[e[1]:e[2]] += 1
            else:
                k = e[1]
                n_far += 1
                cover[t.start[k]:t.end[k]] += 1
                xc, rc = tc.geometry(t, k)
                assert t.end[k] - t.start[k] > (deg + 1) ** 3
                assert np.all(rc / np.linalg.norm(tgt - xc, axis=1) <= theta)
        assert np.all(cover == 1)
    assert n_far > 0


def test_treecode_proxies_reproduce_polynomial_moments(orc, tc_surface):
    """The proxy weights of a cluster are Lagrange interpolation at the
    Chebyshev points of its box: every moment sum_j a_j x^i y^j z^k with
    i, j, k <= p is reproduced exactly by the proxies (up to rounding)."""
    tc = orc.treecode
    p = tc_surface
    t = tc.build_tree(p.centroids, 64)
    k = t.child[t.child[0][0]][1]  # a cluster of a quarter of the surface
    rng = np.random.default_rng(3)
    a = rng.standard_normal(p.n)
    m = rng.standard_normal((p.n, 3))
    deg = 4
    pos, pa, pm = tc.proxies(t, k, p.centroids, a, m, deg)
    idx = t.perm[t.start[k]:t.end[k]]
    c = 0.5 * (t.lo[k] + t.hi[k])
    x, s = p.centroids[idx] - c, pos - c
    for i in range(deg + 1):
        for j in range(deg + 1):
            for l in (0, deg):
                mono_x = x[:, 0] ** i * x[:, 1] ** j * x[:, 2] ** l
                mono_s = s[:, 0] ** i * s[:, 1] ** j * s[:, 2] ** l
                ref = np.dot(mono_x, a[idx])
                assert np.dot(mono_s, pa) == pytest.approx(ref, rel=1e-9, abs=1e-9 * np.abs(mono_x * a[idx]).sum())
                refm = mono_x @ m[idx]
                np.testing.assert_allclose(mono_s @ pm, refm, rtol=1e-9, atol=1e-9 * np.abs(mono_x).sum())
    # a source on a node: its basis value is exactly 1 there and 0 at the other nodes
    nodes, w = tc.cheb_box(t.lo[k], t.hi[k], deg)
    assert tc.lagrange_1d(np.array([nodes[0][2]]), nodes[0], w)[0].tolist() == [0.0, 0.0, 1.0, 0.0, 0.0]


@pytest.mark.parametrize("transpose", [False, True])
def test_treecode_theta_zero_is_the_direct_matvec(orc, tc_surface, transpose):
    """theta = 0: no cluster is far, every pair is summed directly (A u, and
    A^T u against the oracle's transposed mat-vec)."""
    p = tc_surface
    eps = p.eps_out / p.eps_in
    u = np.random.default_rng(5).standard_normal(2 * p.n)
    f = orc.matvec_t if transpose else orc.matvec
    ref = f(p.centroids, p.normals, p.areas, eps, p.kappa, u)
    got = orc.treecode.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u, 0.0, 6, 64, transpose=transpose)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("transpose", [False, True])
def test_treecode_error_falls_with_degree(orc, tc_surface, transpose):
    """The far-field approximation error against the direct mat-vec (A u or
    A^T u) falls geometrically with the interpolation degree (2, 4, 6) at
    fixed theta, on a smooth field and a random one."""
    p = tc_surface
    eps = p.eps_out / p.eps_in
    x = p.centroids / 25.0
    f = orc.matvec_t if transpose else orc.matvec
    for u in (np.concatenate([1.0 + 0.3 * x[:, 2], 0.5 - 0.2 * x[:, 0]]),
              np.random.default_rng(6).standard_normal(2 * p.n)):
        ref = f(p.centroids, p.normals, p.areas, eps, p.kappa, u)
        errs = []
        for deg in (2, 4, 6):
            got = orc.treecode.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, u, 0.7, deg, 32,
                                      transpose=transpose)
            errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert errs[0] > 5 * errs[1] > 25 * errs[2] > 0, errs
