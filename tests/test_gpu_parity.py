"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (each derived from the arithmetic of the path it checks):
* FP64 passes (mat-vec, transpose, source, reaction): 1e-12 relative to the
  largest output (reordered FP64 sums over N <= 20480 terms).
* FP32 mat-vec: 3e-6 in the 2-norm and 2e-5 of the largest output per
  element (FP32 pair arithmetic with 2^-22 MUFU approximations, FP32 sums
  over one source split, FP64 across splits).
* Double-float mat-vec: 2e-12 of the largest output (pairs in ~48-bit
  arithmetic; measured 4e-14).
* Split-FP16 tensor-core mat-vec: the FP32 bounds.
* Solves: energies and potentials within 1e-10 (FP64, both sides solved to
  1e-12) and within 1e-7 (mixed, refined to 1e-8 ... 1e-10); potentials at
  points off the surface within 1e-9 of the largest value (the difference
  of two solves to 1e-12, carried through a kernel sum).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bipb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_10044_gb300.build import build

    build()
    import paper_2312_10044_gb300 as b

    b.load_library()
    return b


def _med(bipb, p):
    return bipb.medium(p.eps_in, p.eps_out, p.kappa)


def _ragged(level=3, drop=43, seed=6):
    """A displaced surface whose size is not a multiple of any tile."""
    p = synth.protein_like_problem(level=level, n_charges=7, seed=seed)
    keep = np.ones(p.n, bool)
    keep[np.random.default_rng(1).choice(p.n, drop, replace=False)] = False
    p.centroids, p.normals, p.areas = p.centroids[keep], p.normals[keep], p.areas[keep]
    return p


PROBLEMS = {
    "born_l2": lambda: synth.born_problem(level=2),
    "ragged_l3": lambda: _ragged(3),
    "kirkwood_l3": lambda: synth.kirkwood_problem(level=3),
}


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("transpose", [False, True])
def test_matvec_fp64_and_fp32(bipb, orc, name, transpose):
    p = PROBLEMS[name]()
    eps = p.eps_out / p.eps_in
    rng = np.random.default_rng(3)
    U = rng.standard_normal((2, 2 * p.n))
    f = orc.matvec_t if transpose else orc.matvec
    ref = np.stack([f(p.centroids, p.normals, p.areas, eps, p.kappa, u) for u in U])
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        cases = [(bipb.FP64, 0, sym) for sym in (True, False)] + [(bipb.DF64, 0, sym) for sym in (True, False)]
        cases += [(bipb.FP32, v, True) for v in range(bipb.MATVEC32_VARIANTS)]
        for prec, variant, sym in cases:
            s.set_variant(variant)
            s.symmetric_pairs(sym)
            yd = torch.full_like(ud, float("nan"))
            s.matvec(ud, yd, precision=prec, transpose=transpose, med=_med(bipb, p))
            y = yd.cpu().numpy()
            assert np.all(np.isfinite(y))
            scale = np.abs(ref).max()
            if prec == bipb.FP64:
                np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * scale)
            elif prec == bipb.DF64:
                np.testing.assert_allclose(y, ref, rtol=0, atol=2e-12 * scale)
            else:
                assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 3e-6, variant
                assert np.abs(y - ref).max() < 2e-5 * scale, variant


def test_degenerate_media(bipb, orc):
    """kappa = 0 (pure Coulomb kernels, the symmetric kernels' own form)
    against the oracle in every precision, both directions, and no
    dielectric contrast with kappa = 0, where every kernel vanishes
    exactly: A = I and the solve returns b after one iteration."""
    p = _ragged(3)
    rng = np.random.default_rng(8)
    U = rng.standard_normal((2, 2 * p.n))
    med0 = bipb.medium(1.0, 80.0, 0.0)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        for transpose in (False, True):
            f = orc.matvec_t if transpose else orc.matvec
            ref = np.stack([f(p.centroids, p.normals, p.areas, 80.0, 0.0, u) for u in U])
            for prec, variant, tol in ((bipb.FP64, 0, 1e-12), (bipb.DF64, 0, 2e-12), (bipb.FP32, 0, 2e-5),
                                       (bipb.FP32, 7, 2e-5), (bipb.FP32, 9, 2e-5), (bipb.TENSOR, 9, 2e-5)):
                s.set_variant(variant)
                yd = torch.full_like(ud, float("nan"))
                s.matvec(ud, yd, precision=prec, transpose=transpose, med=med0)
                err = np.abs(yd.cpu().numpy() - ref).max()
                assert err < tol * np.abs(ref).max(), (prec, variant, transpose)
        unit = bipb.medium(1.0, 1.0, 0.0)
        for prec in (bipb.FP64, bipb.DF64, bipb.FP32, bipb.TENSOR):
            yd = torch.full_like(ud, float("nan"))
            s.matvec(ud, yd, precision=prec, med=unit)
            assert torch.equal(yd, ud), prec
        s.set_charges(p.charge_pos, p.q)
        info = s.solve(eps_in=1.0, eps_out=1.0, kappa=0.0, tol=1e-12, precision=bipb.MIXED_DF64)[0]
        assert info["converged"] and info["iters"] <= 1
        assert s.energy()[0] == 0.0


@pytest.mark.parametrize("kappa", [1e-7, 2.5])
def test_matvec_kappa_range(bipb, orc, kappa):
    """The symmetric kernels work in kappa-scaled units; a Debye length
    above 1e6 A (kappa = 1e-7) takes the ordered kernels instead, and strong
    screening (kappa = 2.5 / A) makes e^{-kappa r} underflow for most pairs.
    Both directions against the oracle in every precision."""
    p = _ragged(3)
    rng = np.random.default_rng(12)
    U = rng.standard_normal((2, 2 * p.n))
    med = bipb.medium(1.0, 80.0, kappa)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        for transpose in (False, True):
            f = orc.matvec_t if transpose else orc.matvec
            ref = np.stack([f(p.centroids, p.normals, p.areas, 80.0, kappa, u) for u in U])
            scale = np.abs(ref).max()
            for prec, variant, tol in ((bipb.FP64, 0, 1e-12), (bipb.DF64, 0, 2e-12), (bipb.FP32, 9, 2e-5),
                                       (bipb.FP32, 7, 2e-5)):
                s.set_variant(variant)
                yd = torch.full_like(ud, float("nan"))
                s.matvec(ud, yd, precision=prec, transpose=transpose, med=med)
                err = np.abs(yd.cpu().numpy() - ref).max()
                assert err < tol * scale, (prec, variant, transpose, err / scale)


def test_autotune_picks_a_variant(bipb):
    p = synth.kirkwood_problem(level=3)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        v, ms = s.autotune(reps=2)
        assert 0 <= v < bipb.MATVEC32_VARIANTS and ms > 0


def test_matvec_is_deterministic(bipb):
    """Every mat-vec sums in a fixed order: repeated calls agree bit for bit
    (the tensor-core paths with several right-hand sides in both directions,
    the far-field one in both directions)."""
    p = _ragged(3)
    u = _dev(np.random.default_rng(0).standard_normal(2 * p.n))
    U = _dev(np.random.default_rng(1).standard_normal((5, 2 * p.n)))
    W = _dev(np.random.default_rng(2).standard_normal((16, 2 * p.n)))
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.treecode(0.7, 4, 64)
        for prec, v, tr in ((bipb.FP64, u, False), (bipb.FP32, u, False), (bipb.DF64, u, False),
                            (bipb.TENSOR, U, False), (bipb.TENSOR, U, True), (bipb.DF64, W, False),
                            (bipb.DF64, W, True), (bipb.TREE32, u, False), (bipb.TREE32, u, True)):
            a, b = torch.empty_like(v), torch.empty_like(v)
            s.matvec(v, a, precision=prec, transpose=tr)
            s.matvec(v, b, precision=prec, transpose=tr)
            assert torch.equal(a, b), (prec, tr)


def test_two_triangle_surface(bipb, orc):
    p = synth.born_problem(level=0)
    c, n, a = p.centroids[:2], p.normals[:2], p.areas[:2]
    u = np.array([0.3, -1.2, 0.7, 2.0])
    ref = orc.matvec(c, n, a, 80.0, 0.1257, u)
    with bipb.Surface(c, n, a) as s:
        ud = _dev(u)
        yd = torch.empty_like(ud)
        s.matvec(ud, yd, precision=bipb.FP64)
        np.testing.assert_allclose(yd.cpu().numpy(), ref, rtol=1e-13)


@pytest.mark.parametrize("name", ["ragged_l3", "kirkwood_l3"])
def test_source_and_reaction_fp64(bipb, orc, name):
    p = PROBLEMS[name]()
    eps = p.eps_out / p.eps_in
    b_ref = orc.source(p.centroids, p.normals, p.charge_pos, p.q[0], p.eps_in)
    u = np.random.default_rng(5).standard_normal(2 * p.n)
    e_ref, pr_ref = orc.energy(p.centroids, p.normals, p.areas, eps, p.kappa, p.charge_pos, p.q[0], u)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        bd = torch.full((2 * p.n,), float("nan"), dtype=torch.float64, device="cuda")
        s.source(bd, med=_med(bipb, p))
        np.testing.assert_allclose(bd.cpu().numpy(), b_ref, rtol=0, atol=1e-12 * np.abs(b_ref).max())
        pr = torch.empty(p.nc, dtype=torch.float64, device="cuda")
        e = torch.empty(1, dtype=torch.float64, device="cuda")
        s.reaction(_dev(u), pr, e, med=_med(bipb, p))
        np.testing.assert_allclose(pr.cpu().numpy(), pr_ref, rtol=0, atol=1e-12 * np.abs(pr_ref).max())
        assert e.item() == pytest.approx(orc.KCAL * e_ref, rel=1e-11)


def test_born_fp64_solve_matches_direct_solution(bipb, orc):
    p = synth.born_problem(level=3)
    ref = orc.solve(p, method="direct")
    phi_ref, dphi_ref = ref.surface_potential()
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        info = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=1e-12, precision=bipb.FP64)
        assert info[0]["converged"] and info[0]["rel_residual"] <= 1e-12
        e = s.energy()[0]
        phi, dphi = s.surface_potential()
    assert e == pytest.approx(ref.energy_kcal, rel=1e-10)
    np.testing.assert_allclose(phi[0], phi_ref, rtol=1e-10)
    np.testing.assert_allclose(dphi[0], dphi_ref, rtol=1e-10)


def test_born_iteration_count_matches_oracle_gmres(bipb, orc):
    p = synth.born_problem(level=3)
    ref = orc.solve(p, method="gmres", tol=1e-8)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        info = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=1e-8, precision=bipb.FP64)
    assert abs(info[0]["iters"] - ref.info["iters"]) <= 1
    assert info[0]["rel_residual"] <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed", "df64", "mixed_df64"])
def test_kirkwood_solve(bipb, orc, prec):
    p = synth.kirkwood_problem(level=4)
    ref = orc.solve(p, method="gmres", tol=1e-12)
    phi_ref, dphi_ref = ref.surface_potential()
    P = {"fp64": bipb.FP64, "mixed": bipb.MIXED, "df64": bipb.DF64, "mixed_df64": bipb.MIXED_DF64,
         "mixed_tensor": bipb.MIXED_TENSOR, "mixed_tree": bipb.MIXED_TREE}[prec]
    tol = 1e-12 if prec in ("fp64", "df64") else 1e-8
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        info = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=tol, precision=P)[0]
        e = s.energy()[0]
        phi, dphi = s.surface_potential()
    assert info["converged"] and info["rel_residual"] <= tol
    rt = 1e-10 if prec in ("fp64", "df64") else 1e-7
    assert e == pytest.approx(ref.energy_kcal, rel=rt)
    assert np.linalg.norm(phi[0] - phi_ref) / np.linalg.norm(phi_ref) < rt
    assert np.linalg.norm(dphi[0] - dphi_ref) / np.linalg.norm(dphi_ref) < rt
    if prec.startswith("mixed"):
        assert info["refine_steps"] >= 1 and info["matvecs32"] > info["matvecs64"]


def test_multiple_charge_sets_match_single_solves(bipb):
    base = synth.protein_like_problem(level=3, n_charges=20)
    batch = synth.batched_charges(base, n_rhs=3, n_charges=20)
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.set_charges(batch.charge_pos, batch.q)
        s.solve(tol=1e-11, precision=bipb.FP64)
        e_all = s.energy()
        phi_all, _ = s.surface_potential()
        for r in range(3):
            s.set_charges(batch.charge_pos[r], batch.q[r])
            s.solve(tol=1e-11, precision=bipb.FP64)
            assert s.energy()[0] == pytest.approx(e_all[r], rel=1e-9)
            np.testing.assert_allclose(s.surface_potential()[0][0], phi_all[r], rtol=1e-8, atol=1e-9)


def test_batched_mixed_df64_with_idle_systems(bipb):
    """20 charge sets solved together in MIXED_DF64; sets 3 and 7 carry no
    charge, so they are idle from the start and the batched double-float
    residual runs over a non-contiguous subset of the right-hand sides."""
    base = synth.protein_like_problem(level=3, n_charges=20)
    batch = synth.batched_charges(base, n_rhs=20, n_charges=20)
    q = batch.q.copy()
    q[3] = 0.0
    q[7] = 0.0
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.set_charges(batch.charge_pos, q)
        info = s.solve(tol=1e-10, precision=bipb.MIXED_DF64)
        assert all(i["converged"] for i in info)
        e_all = s.energy()
        phi_all, _ = s.surface_potential()
        assert e_all[3] == 0.0 and e_all[7] == 0.0
        assert not phi_all[3].any() and not phi_all[7].any()
        for r in (0, 8, 19):
            s.set_charges(batch.charge_pos[r], q[r])
            s.solve(tol=1e-10, precision=bipb.MIXED_DF64)
            assert s.energy()[0] == pytest.approx(e_all[r], rel=1e-8)
            np.testing.assert_allclose(s.surface_potential()[0][0], phi_all[r], rtol=1e-7, atol=1e-8)


def test_gradient_matches_oracle_adjoint(bipb, orc):
    p = synth.kirkwood_problem(level=3, radius=10.0, n_charges=6, charge_radius=7.0)
    e_ref, dq_ref, dy_ref = orc.energy_gradient(p, method="direct")
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=1e-12, precision=bipb.FP64)
        dq, dy = s.energy_grad(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=1e-12,
                               precision=bipb.FP64)
    np.testing.assert_allclose(dq[0], dq_ref, rtol=1e-8)
    np.testing.assert_allclose(dy[0], dy_ref, rtol=1e-7, atol=1e-8 * np.abs(dy_ref).max())


def test_kernel_timer_and_launch_count(bipb):
    p = synth.kirkwood_problem(level=3)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        for on in (True, False, True):
            bipb.timer_enable(s, on)
            n0 = bipb.launch_count(s)
            info = s.solve(tol=1e-8, precision=bipb.MIXED)[0]
            t = bipb.timer_read(s)
            assert bipb.launch_count(s) - n0 > info["matvecs32"] + info["matvecs64"]
            if on:
                # launches after convergence inside a recorded cycle return at once but still count
                assert info["matvecs32"] <= t["matvec32"][0] <= info["matvecs32"] + 9 * info["refine_steps"]
                assert t["matvec32"][1] > 0
                assert t["matvec64"][0] == info["matvecs64"] and t["matvec64"][1] > 0
                assert t["source"][0] == 1 and t["reaction"][0] == 1
            else:
                assert all(v == (0, 0.0) for v in t.values())


def test_energy_before_solve_is_a_state_error(bipb):
    p = synth.born_problem(level=1)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        with pytest.raises(bipb.BipbError) as ei:
            s.energy()
        assert ei.value.status == bipb.BIPB_ERR_STATE


def test_iteration_cap_reports_not_converged(bipb):
    p = synth.kirkwood_problem(level=3)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        info = s.solve(tol=1e-12, max_iter=3, precision=bipb.FP64, raise_on_not_converged=False)[0]
        assert not info["converged"] and info["iters"] == 3 and info["rel_residual"] > 1e-12
        with pytest.raises(bipb.BipbError) as ei:
            s.solve(tol=1e-12, max_iter=3, precision=bipb.FP64)
        assert ei.value.status == bipb.BIPB_ERR_NOT_CONVERGED
        assert np.isfinite(s.energy()[0])  # the best iterate is kept


def test_warm_start_from_solution_needs_no_iterations(bipb):
    p = synth.born_problem(level=2)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        s.solve(tol=1e-11, precision=bipb.FP64)
        phi, dphi = s.surface_potential()
        u = np.concatenate([phi[0], dphi[0]]) / bipb.KCAL
        info = s.solve(tol=1e-9, precision=bipb.FP64, x0=u[None, :])[0]
        assert info["iters"] == 0 and info["converged"]


# ---------------------------------------------------------------- full-size sampled checks
@pytest.mark.parametrize("cfg", ["kirkwood", "protein_like", "adjoint"])
@pytest.mark.parametrize("transpose", [False, True])
def test_full_size_matvec_sampled_rows(bipb, orc, cfg, transpose):
    """The benchmark's mat-vec launch at full size (up to level 7, N = 327680,
    where the symmetric work list spans 640 tile rows), forward and
    transposed, checked on sampled rows."""
    p = synth.problem_by_name(cfg)
    eps = p.eps_out / p.eps_in
    u = np.random.default_rng(9).standard_normal(2 * p.n)
    rows = np.sort(np.random.default_rng(10).choice(2 * p.n, 48, replace=False))
    rows = np.concatenate([rows, [0, p.n - 1, p.n, 2 * p.n - 1]])
    f = orc.matvec_t_rows if transpose else orc.matvec_rows
    ref = f(p.centroids, p.normals, p.areas, eps, p.kappa, u, rows)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(u)
        y64, y32, ydf = torch.empty_like(ud), torch.empty_like(ud), torch.empty_like(ud)
        s.matvec(ud, y64, precision=bipb.FP64, transpose=transpose, med=_med(bipb, p))
        s.matvec(ud, y32, precision=bipb.FP32, transpose=transpose, med=_med(bipb, p))
        s.matvec(ud, ydf, precision=bipb.DF64, transpose=transpose, med=_med(bipb, p))
        a64, a32, adf = y64.cpu().numpy(), y32.cpu().numpy(), ydf.cpu().numpy()
    scale = np.abs(ref).max()
    np.testing.assert_allclose(a64[rows], ref, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(adf[rows], ref, rtol=0, atol=2e-12 * scale)
    assert np.abs(a32[rows] - ref).max() < 2e-5 * scale


# ---------------------------------------------------------------- GMRES iterates (reading P1(i))
@pytest.mark.parametrize("name", ["born_l3", "kirkwood_l4"])
def test_gmres_iterates_match_oracle_at_equal_iteration_count(bipb, orc, name):
    """At equal iteration count k the FP64 GMRES(10) iterate is the same Krylov
    minimiser on both sides (CGS2 here, modified Gram-Schmidt in the oracle;
    Sec. 2.2.2): stopped after k = 5, 10 and 17 iterations (inside the first
    cycle, at the restart, inside the second), the iterates agree to 1e-10
    and so do the true residuals they leave."""
    p = synth.born_problem(level=3) if name == "born_l3" else synth.kirkwood_problem(level=4)
    eps = p.eps_out / p.eps_in
    b = orc.source(p.centroids, p.normals, p.charge_pos, p.q[0], p.eps_in)
    A = lambda v: orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, v)  # noqa: E731
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        for k in (5, 10, 17):
            x_ref, info_ref = orc.gmres(A, b, tol=1e-15, restart=10, max_iter=k)
            assert info_ref["iters"] == k and not info_ref["converged"]
            info = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=1e-15, max_iter=k,
                           precision=bipb.FP64, raise_on_not_converged=False)[0]
            assert info["iters"] == k and not info["converged"]
            phi, dphi = s.surface_potential()
            x = np.concatenate([phi[0], dphi[0]]) / bipb.KCAL
            assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-10, k
            # x differs from x_ref by rounding only (about 1e-13 relative), which moves a
            # residual of 1e-9 by a few 1e-12: compared to 5e-11 absolute
            assert info["rel_residual"] == pytest.approx(info_ref["rel_residual"], rel=1e-6, abs=5e-11), k


def test_long_restart_matches_oracle(bipb, orc):
    """GMRES(m) with m = 150 (the restart length may lie in [1, 200]): inside
    one long cycle, the iterates after k = 25 and 40 steps agree with the
    oracle's GMRES(150) to 1e-10 (tol 1e-300: neither side stops early)."""
    p = synth.kirkwood_problem(level=3)
    eps = p.eps_out / p.eps_in
    b = orc.source(p.centroids, p.normals, p.charge_pos, p.q[0], p.eps_in)
    A = lambda v: orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, v)  # noqa: E731
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        for k in (25, 40):
            x_ref, _ = orc.gmres(A, b, tol=1e-300, restart=150, max_iter=k)
            info = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=1e-300, max_iter=k, restart=150,
                           precision=bipb.FP64, raise_on_not_converged=False)[0]
            assert info["iters"] == k
            phi, dphi = s.surface_potential()
            x = np.concatenate([phi[0], dphi[0]]) / bipb.KCAL
            assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-10, k
        with pytest.raises(bipb.BipbError):
            s.solve(tol=1e-8, restart=201, precision=bipb.FP64)


# ---------------------------------------------------------------- solute dielectric eps_in != 1
def test_solute_dielectric_parity(bipb, orc):
    """eps_in = 2, eps_out = 80 (S1, S2 and the gradient's source column carry
    1/eps_in, Sec. 2.2.1): the source term, FP64 and mixed solves (double-float
    residual with CUDA-core, tensor-core and far-field Krylov mat-vecs),
    energy, surface potential, gradient and the potential at points inside
    and outside against the oracle."""
    p = synth.kirkwood_problem(level=3, radius=10.0, n_charges=6, charge_radius=7.0)
    p.eps_in = 2.0
    eps = p.eps_out / p.eps_in
    y, q = p.charge_pos, p.q[0]
    b_ref = orc.source(p.centroids, p.normals, y, q, p.eps_in)
    ref = orc.solve(p, method="direct")
    phi_ref, dphi_ref = ref.surface_potential()
    e_ref, dq_ref, dy_ref = orc.energy_gradient(p, method="direct")
    rng = np.random.default_rng(41)
    pin, pout = _ball(rng, 64, 0.0, 8.0), _ball(rng, 64, 12.0, 30.0)
    rin = orc.KCAL * orc.potential(p.centroids, p.normals, p.areas, eps, p.kappa, ref.u, pin, True, y, q, p.eps_in)
    rout = orc.KCAL * orc.potential(p.centroids, p.normals, p.areas, eps, p.kappa, ref.u, pout, False)
    kw = dict(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(y, p.q)
        bd = torch.full((2 * p.n,), float("nan"), dtype=torch.float64, device="cuda")
        s.source(bd, med=_med(bipb, p))
        np.testing.assert_allclose(bd.cpu().numpy(), b_ref, rtol=0, atol=1e-12 * np.abs(b_ref).max())
        s.treecode(0.7, 4, 64)  # far clusters on this small surface too
        for prec, tol, rt in ((bipb.FP64, 1e-12, 1e-10), (bipb.MIXED_DF64, 1e-10, 1e-7), (bipb.MIXED_TENSOR, 1e-10, 1e-7),
                              (bipb.MIXED_TREE, 1e-10, 1e-7)):
            info = s.solve(tol=tol, precision=prec, **kw)[0]
            assert info["converged"]
            assert s.energy()[0] == pytest.approx(ref.energy_kcal, rel=rt)
            phi, dphi = s.surface_potential()
            assert np.linalg.norm(phi[0] - phi_ref) / np.linalg.norm(phi_ref) < rt
            assert np.linalg.norm(dphi[0] - dphi_ref) / np.linalg.norm(dphi_ref) < rt
            dq, dy = s.energy_grad(tol=tol, precision=prec, **kw)
            np.testing.assert_allclose(dq[0], dq_ref, rtol=100 * rt)
            np.testing.assert_allclose(dy[0], dy_ref, rtol=0, atol=100 * rt * np.abs(dy_ref).max())
            vin, vout = s.potential_at(pin, inside=True), s.potential_at(pout, inside=False)
            np.testing.assert_allclose(vin[0], rin, rtol=0, atol=10 * rt * np.abs(rin).max())
            np.testing.assert_allclose(vout[0], rout, rtol=0, atol=10 * rt * np.abs(rout).max())


# ---------------------------------------------------------------- uneven batches
def _uneven():
    a = synth.born_problem(level=2, radius=4.0)
    a.charge_pos = np.array([[0.3, -0.2, 0.5], [-1.0, 0.4, 0.1]])
    a.q = np.array([[0.7, -0.4]])
    b = _ragged(3)
    c = synth.kirkwood_problem(level=3, radius=9.0, n_charges=5, charge_radius=6.0)
    return [a, b, c]


def test_uneven_batch_matvec_matches_oracle(bipb, orc):
    probs = _uneven()
    rng = np.random.default_rng(21)
    us = [rng.standard_normal(2 * p.n) for p in probs]
    with bipb.BatchSurface([(p.centroids, p.normals, p.areas) for p in probs]) as s:
        u = _dev(np.concatenate(us))
        cases = [(bipb.FP64, 1e-12, 0, True), (bipb.FP64, 1e-12, 0, False), (bipb.DF64, 2e-12, 0, True)]
        cases += [(bipb.FP32, 2e-5, v, True) for v in (0, 7, 8, 9)]
        for prec, tol, variant, sym in cases:
            s.set_variant(variant)
            s.symmetric_pairs(sym)
            for transpose in (False, True):
                y = torch.full_like(u, float("nan"))
                s.matvec(u, y, precision=prec, transpose=transpose)
                parts = np.split(y.cpu().numpy(), np.cumsum([2 * p.n for p in probs])[:-1])
                for p, uk, yk in zip(probs, us, parts):
                    f = orc.matvec_t if transpose else orc.matvec
                    ref = f(p.centroids, p.normals, p.areas, p.eps_out / p.eps_in, p.kappa, uk)
                    assert np.abs(yk - ref).max() < tol * np.abs(ref).max(), (prec, variant, sym, transpose)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uneven_batch_solve_matches_single_solves(bipb, prec):
    probs = _uneven()
    P = bipb.FP64 if prec == "fp64" else bipb.MIXED
    tol = 1e-11 if prec == "fp64" else 1e-9
    with bipb.BatchSurface([(p.centroids, p.normals, p.areas) for p in probs]) as s:
        s.set_charges([(p.charge_pos, p.q[0]) for p in probs])
        info = s.solve(tol=tol, precision=P)
        assert len(info) == 3 and all(i["converged"] for i in info)
        e = s.energy()
        phi, dphi = s.surface_potential()
        dq, dy = s.energy_grad(tol=1e-10, precision=P)
    for k, p in enumerate(probs):
        with bipb.Surface(p.centroids, p.normals, p.areas) as s1:
            s1.set_charges(p.charge_pos, p.q)
            s1.solve(tol=tol, precision=P)
            rt = 1e-9 if prec == "fp64" else 1e-7
            assert e[k] == pytest.approx(s1.energy()[0], rel=rt)
            ph1, dph1 = s1.surface_potential()
            assert np.linalg.norm(phi[k] - ph1[0]) < rt * 10 * np.linalg.norm(ph1[0])
            dq1, dy1 = s1.energy_grad(tol=1e-10, precision=P)
            np.testing.assert_allclose(dq[k], dq1[0], rtol=1e-6, atol=1e-9 * np.abs(dq1).max())
            np.testing.assert_allclose(dy[k], dy1[0], rtol=1e-6, atol=1e-9 * np.abs(dy1).max())


def test_uneven_batch_one_launch_per_pass(bipb):
    """A batched mat-vec is one pack, one pair-kernel and one reduction launch."""
    probs = _uneven()
    with bipb.BatchSurface([(p.centroids, p.normals, p.areas) for p in probs]) as s:
        u = _dev(np.ones(sum(2 * p.n for p in probs)))
        y = torch.empty_like(u)
        s.matvec(u, y, precision=bipb.FP32)
        n0 = bipb.launch_count(s)
        s.matvec(u, y, precision=bipb.FP32)
        assert bipb.launch_count(s) - n0 == 3


# ---------------------------------------------------------------- autograd
@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_autograd_energy_matches_oracle_and_finite_differences(bipb, orc, device):
    """CUDA tensors take the device entry points (charges, energy and gradient
    never pass through the host); CPU tensors the host ones."""
    from paper_2312_10044_gb300.torch_ops import SolvationEnergy

    p = synth.protein_like_problem(level=3, radius=12.0, n_charges=6, seed=8)
    e_ref, dq_ref, dy_ref = orc.energy_gradient(p, method="direct")
    model = SolvationEnergy(p.centroids, p.normals, p.areas, tol=1e-12, precision=bipb.FP64)
    q = torch.tensor(p.q[0], dtype=torch.float64, device=device, requires_grad=True)
    pos = torch.tensor(p.charge_pos, dtype=torch.float64, device=device, requires_grad=True)
    e = model(q, pos)
    assert e.device.type == device
    e.backward()
    assert q.grad.device.type == device and pos.grad.device.type == device
    assert e.item() == pytest.approx(e_ref, rel=1e-10)
    np.testing.assert_allclose(q.grad.cpu().numpy(), dq_ref, rtol=1e-8)
    np.testing.assert_allclose(pos.grad.cpu().numpy(), dy_ref, rtol=1e-7, atol=1e-9 * np.abs(dy_ref).max())
    # central differences, h = 1e-4 A, on two atoms
    h = 1e-4
    for k in (0, 3):
        for a in range(3):
            with torch.no_grad():
                pp = pos.detach().clone()
                pp[k, a] += h
                ep = model(q.detach(), pp).item()
                pp[k, a] -= 2 * h
                em = model(q.detach(), pp).item()
            fd = (ep - em) / (2 * h)
            assert pos.grad[k, a].item() == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(dy_ref).max())


def test_device_charges_are_checked_on_the_device(bipb):
    """bipb_charges_set_dev: the checks of bipb_charges_set run on the device
    and the next solve reports a failure (and forgets the charges)."""
    p = synth.born_problem(level=2)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        for bad in (p.centroids[17], np.array([np.nan, 0.0, 0.0])):
            s.set_charges_dev(_dev(np.stack([[0.0, 0.0, 0.0], bad])), _dev([[1.0, -1.0]]))
            with pytest.raises(bipb.BipbError) as ei:
                s.solve(tol=1e-8, precision=bipb.FP64)
            assert ei.value.status == bipb.BIPB_ERR_INVALID_ARG
            with pytest.raises(bipb.BipbError):  # the charges are gone
                s.solve(tol=1e-8, precision=bipb.FP64)
        # good charges, two configurations with their own positions, match the host path
        pos = np.array([[[0.1, 0.2, 0.0], [0.3, -0.2, 0.1]], [[0.0, 0.0, 0.5], [-0.4, 0.1, 0.0]]])
        q = np.array([[1.0, -0.5], [0.3, 0.7]])
        s.set_charges_dev(_dev(pos), _dev(q))
        s.solve(tol=1e-12, precision=bipb.FP64)
        e_dev = s.energy_dev().cpu().numpy()
        dq_d, dy_d = (t.cpu().numpy() for t in s.energy_grad_dev(tol=1e-12, precision=bipb.FP64))
        s.set_charges(pos, q)
        s.solve(tol=1e-12, precision=bipb.FP64)
        np.testing.assert_array_equal(s.energy(), e_dev)
        dq_h, dy_h = s.energy_grad(tol=1e-12, precision=bipb.FP64)
        np.testing.assert_array_equal(dq_h, dq_d)
        np.testing.assert_array_equal(dy_h, dy_d)


def test_autograd_batched_mixed(bipb):
    from paper_2312_10044_gb300.torch_ops import SolvationEnergy

    base = synth.protein_like_problem(level=3, n_charges=10)
    batch = synth.batched_charges(base, n_rhs=2, n_charges=10)
    model = SolvationEnergy(batch.centroids, batch.normals, batch.areas, tol=1e-9)
    q = torch.tensor(batch.q, dtype=torch.float64, requires_grad=True)
    pos = torch.tensor(batch.charge_pos, dtype=torch.float64, requires_grad=True)
    e = model(q, pos)
    (e * torch.tensor([1.0, -2.0], dtype=torch.float64)).sum().backward()
    # Euler identity per configuration: sum_k q_k dE/dq_k = 2 E (weights 1 and -2)
    assert torch.dot(q[0].detach(), q.grad[0]).item() == pytest.approx(2 * e[0].item(), rel=1e-6)
    assert torch.dot(q[1].detach(), q.grad[1]).item() == pytest.approx(-2 * 2 * e[1].item(), rel=1e-6)


# ---------------------------------------------------------------- tensor-core multi-RHS
@pytest.mark.parametrize("n_rhs", [5, 70])
def test_tensor_core_matvec_matches_oracle(bipb, orc, n_rhs):
    """Tensor-core mat-vec (kernel tile once per 64 right-hand sides, FP32
    operands scaled by powers of two and split into two FP16 parts, three
    products) vs the FP64 oracle: held to the FP32 mat-vec's bounds, 3e-6 in
    the 2-norm and 2e-5 of the largest output."""
    p = _ragged(3)
    eps = p.eps_out / p.eps_in
    U = np.random.default_rng(30 + n_rhs).standard_normal((n_rhs, 2 * p.n))
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        yd = torch.full_like(ud, float("nan"))
        s.matvec(ud, yd, precision=bipb.TENSOR, med=_med(bipb, p))
        Y = yd.cpu().numpy()
    for r in (0, n_rhs // 2, n_rhs - 1):
        ref = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, U[r])
        assert np.all(np.isfinite(Y[r]))
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) < 3e-6
        assert np.abs(Y[r] - ref).max() < 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("kappa", [1e-7, 1e-6, 2.5])
def test_tensor_core_matvec_kappa_range(bipb, orc, kappa):
    """Both forms of the tensor-core kernel at the ends of their kappa range:
    plain units below 1e-6 / A (1e-7), kappa-scaled positions from 1e-6 on
    (1e-6, where the scaled 1/r^3 is largest, and a short Debye length of
    0.4 A), held to the FP32 bounds against the oracle."""
    p = _ragged(3)
    eps = p.eps_out / p.eps_in
    U = np.random.default_rng(41).standard_normal((6, 2 * p.n))
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        yd = torch.full_like(ud, float("nan"))
        s.matvec(ud, yd, precision=bipb.TENSOR, med=bipb.medium(p.eps_in, p.eps_out, kappa))
        Y = yd.cpu().numpy()
    for r in (0, 3, 5):
        ref = orc.matvec(p.centroids, p.normals, p.areas, eps, kappa, U[r])
        assert np.all(np.isfinite(Y[r]))
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) < 3e-6
        assert np.abs(Y[r] - ref).max() < 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("geo_scale", [1e-3, 1.0, 1e3])
def test_tensor_core_matvec_scaled_inputs(bipb, orc, geo_scale):
    """The power-of-two row and column scaling of the tensor-core path:
    right-hand sides of magnitude 1e-25, 1 and 1e25 side by side, one zero
    right-hand side, and the surface in units 1e-3, 1 and 1e3 times as large
    (kernel values from about 1e-9 to 1e6 of the unscaled ones).  Each
    nonzero column is held to the FP32 bounds relative to its own size; the
    zero column gives exact zeros."""
    p = _ragged(3)
    c, a = p.centroids * geo_scale, p.areas * geo_scale**2
    eps = p.eps_out / p.eps_in
    rng = np.random.default_rng(41)
    mags = [1e-25, 1.0, 1e25]
    U = np.stack([m * rng.standard_normal(2 * p.n) for m in mags] + [np.zeros(2 * p.n)])
    with bipb.Surface(c, p.normals, a) as s:
        ud = _dev(U)
        yd = torch.full_like(ud, float("nan"))
        s.matvec(ud, yd, precision=bipb.TENSOR, med=_med(bipb, p))
        Y = yd.cpu().numpy()
    assert np.all(Y[3] == 0.0)
    for r in range(3):
        ref = orc.matvec(c, p.normals, a, eps, p.kappa, U[r])
        assert np.all(np.isfinite(Y[r]))
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) < 3e-6, r
        assert np.abs(Y[r] - ref).max() < 2e-5 * np.abs(ref).max(), r


@pytest.mark.parametrize("n_keep", [2, 7, 80, 200])
@pytest.mark.parametrize("transpose", [False, True])
def test_tensor_core_matvec_small_surfaces(bipb, orc, n_keep, transpose):
    """Surfaces smaller than one source chunk (32) and one target tile (128):
    two elements (the smallest surface the library takes), a ragged first chunk and
    a partly filled tile, against the FP64 oracle at the FP32 bounds (A U and
    A^T U); and the exact double-float pass of 16 right-hand sides on the same
    surfaces (steps of 16 sources, tiles of 64 targets) at 2e-12."""
    p = synth.protein_like_problem(level=2, n_charges=5, seed=8)  # 320 elements
    keep = np.sort(np.random.default_rng(n_keep).choice(p.n, n_keep, replace=False))
    c, nv, a = p.centroids[keep], p.normals[keep], p.areas[keep]
    eps = p.eps_out / p.eps_in
    U = np.random.default_rng(50 + n_keep).standard_normal((16, 2 * n_keep))
    with bipb.Surface(c, nv, a) as s:
        ud = _dev(U)
        yd, yx = torch.full_like(ud, float("nan")), torch.full_like(ud, float("nan"))
        s.matvec(ud[:3], yd[:3], precision=bipb.TENSOR, transpose=transpose, med=_med(bipb, p))
        s.matvec(ud, yx, precision=bipb.DF64, transpose=transpose, med=_med(bipb, p))
        Y, X = yd.cpu().numpy(), yx.cpu().numpy()
    f = orc.matvec_t if transpose else orc.matvec
    for r in range(3):
        ref = f(c, nv, a, eps, p.kappa, U[r])
        assert np.all(np.isfinite(Y[r]))
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) < 3e-6
        assert np.abs(Y[r] - ref).max() < 2e-5 * np.abs(ref).max()
        assert np.abs(X[r] - ref).max() < 2e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n_rhs,kappa", [(5, 0.1257), (70, 0.1257), (6, 1e-7), (6, 2.5)])
def test_tensor_core_transpose_matches_oracle(bipb, orc, n_rhs, kappa):
    """A^T U on the tensor cores (the transposed blocks generated in FP32 with
    the output's area applied to the sums; plain units below kappa = 1e-6,
    kappa-scaled above) vs the oracle's transpose, held to the FP32 bounds."""
    p = _ragged(3)
    eps = p.eps_out / p.eps_in
    U = np.random.default_rng(50 + n_rhs).standard_normal((n_rhs, 2 * p.n))
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        yd = torch.full_like(ud, float("nan"))
        s.matvec(ud, yd, precision=bipb.TENSOR, transpose=True, med=bipb.medium(p.eps_in, p.eps_out, kappa))
        Y = yd.cpu().numpy()
    for r in (0, n_rhs // 2, n_rhs - 1):
        ref = orc.matvec_t(p.centroids, p.normals, p.areas, eps, kappa, U[r])
        assert np.all(np.isfinite(Y[r]))
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) < 3e-6
        assert np.abs(Y[r] - ref).max() < 2e-5 * np.abs(ref).max()


def test_mixed_tensor_solve_matches_oracle(bipb, orc):
    """Three charge sets solved together with tensor-core Krylov mat-vecs and
    the double-float residual: energies, and the adjoint gradient (whose
    Krylov solve takes the tensor-core transpose), against the oracle."""
    base = synth.protein_like_problem(level=4, n_charges=30)
    batch = synth.batched_charges(base, n_rhs=3, n_charges=30)
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.set_charges(batch.charge_pos, batch.q)
        info = s.solve(tol=1e-9, precision=bipb.MIXED_TENSOR)
        e = s.energy()
        dq, dy = s.energy_grad(tol=1e-10, precision=bipb.MIXED_TENSOR)
    for r in range(3):
        assert info[r]["converged"] and info[r]["rel_residual"] <= 1e-9
        ref = orc.solve(batch, rhs=r, method="gmres", tol=1e-12)
        assert e[r] == pytest.approx(ref.energy_kcal, rel=1e-7)
        e_ref, dq_ref, dy_ref = orc.energy_gradient(batch, rhs=r, method="gmres", tol=1e-12)
        np.testing.assert_allclose(dq[r], dq_ref, rtol=0, atol=1e-7 * np.abs(dq_ref).max())
        np.testing.assert_allclose(dy[r], dy_ref, rtol=0, atol=1e-7 * np.abs(dy_ref).max())


def test_adjoint_config_level4_copy_matches_oracle(bipb, orc):
    """The adjoint configuration (R = 45 A, 10000 charges) on a level-4 copy of
    its surface: dE/dq and dE/dpos of 32 seeded atoms vs the oracle's FP64 adjoint."""
    p = synth.adjoint_problem(level=4)
    e_ref, dq_ref, dy_ref = orc.energy_gradient(p, method="gmres", tol=1e-12)
    atoms = np.random.default_rng(32).choice(p.nc, 32, replace=False)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        s.solve(tol=1e-12, precision=bipb.FP64)
        assert s.energy()[0] == pytest.approx(e_ref, rel=1e-10)
        dq, dy = s.energy_grad(tol=1e-12, precision=bipb.FP64)
        np.testing.assert_allclose(dq[0][atoms], dq_ref[atoms], rtol=1e-8)
        np.testing.assert_allclose(dy[0][atoms], dy_ref[atoms], rtol=1e-6, atol=1e-8 * np.abs(dy_ref).max())
        # the mixed path (FP32 Krylov, double-float residual), forward and adjoint at 1e-10
        s.solve(tol=1e-10, precision=bipb.MIXED_DF64)
        dqm, dym = s.energy_grad(tol=1e-10, precision=bipb.MIXED_DF64)
        np.testing.assert_allclose(dym[0][atoms], dy_ref[atoms], rtol=1e-5, atol=1e-7 * np.abs(dy_ref).max())


def test_central_differences_by_solution_differences(bipb, orc):
    """Central differences (h = 1e-4 A) of E in the positions and charges of 6
    atoms, formed from solution differences: moving charge k changes only its
    own source and energy-row terms, so E(y_k +- h e_d) - E = 1/2 [dc.u +
    c.du + dc.du] with A du = db for the charge pair {(y_k +- h e_d, q_k),
    (y_k, -q_k)}, each term a reaction-energy pass on the GPU.  The result is
    compared with the GPU adjoint gradient and with the oracle's."""
    p = synth.adjoint_problem(level=3, n_charges=200)
    e_ref, dq_ref, dy_ref = orc.energy_gradient(p, method="direct")
    n, y, q = p.n, p.charge_pos, p.q[0]
    med = _med(bipb, p)
    atoms = np.sort(np.random.default_rng(9).choice(p.nc, 6, replace=False))
    h = 1e-4
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(y, q)
        s.solve(tol=1e-12, precision=bipb.FP64)
        phi, dphi = s.surface_potential()
        u0 = np.concatenate([phi[0], dphi[0]]) / bipb.KCAL
        dq, dy = s.energy_grad(tol=1e-12, precision=bipb.FP64)
        pos_sets, q_sets = [], []
        for k in atoms:
            for d in range(3):
                for sg in (1.0, -1.0):
                    yp = y[k].copy()
                    yp[d] += sg * h
                    pos_sets.append([yp, y[k]])
                    q_sets.append([q[k], -q[k]])
        for k in atoms:
            pos_sets.append([y[k], y[k]])
            q_sets.append([1.0, 0.0])
        B = len(q_sets)
        s.set_charges(np.array(pos_sets), np.array(q_sets))
        info = s.solve(tol=1e-12, precision=bipb.MIXED_DF64)
        assert all(i["converged"] for i in info)
        phi, dphi = s.surface_potential()
        du = _dev(np.concatenate([phi, dphi], axis=1) / bipb.KCAL)
        e_a, e_b, e_c = (torch.empty(B, dtype=torch.float64, device="cuda") for _ in range(3))
        s.reaction(_dev(np.tile(u0, (B, 1))), None, e_a, med)
        s.reaction(du, None, e_b, med)
        s.set_charges(y[None], np.repeat(q[None], B, axis=0))
        s.reaction(du, None, e_c, med)
    m = len(atoms) * 6
    D = (e_a + e_b + e_c).cpu().numpy()
    g_fd = ((D[0:m:2] - D[1:m:2]) / (2 * h)).reshape(len(atoms), 3)
    dq_fd = (e_a + e_c).cpu().numpy()[m:]
    scale = np.abs(dy_ref[atoms]).max()
    np.testing.assert_allclose(g_fd, dy[0][atoms], rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(g_fd, dy_ref[atoms], rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(dq_fd, dq[0][atoms], rtol=1e-9)
    np.testing.assert_allclose(dq_fd, dq_ref[atoms], rtol=1e-9)


@pytest.mark.parametrize("n_rhs", [5, 70, 80])
def test_multi_rhs_df64_matvec_matches_oracle(bipb, orc, n_rhs):
    """The batched double-float mat-vec in blocks of up to 64 right-hand
    sides: 5 (df64 multiply-adds on the CUDA cores), 70 (a block of 64 on the
    tensor cores and one of 6 on the CUDA cores), 80 (blocks of 64 and 16,
    both on the tensor cores)."""
    p = _ragged(3)
    eps = p.eps_out / p.eps_in
    U = np.random.default_rng(40 + n_rhs).standard_normal((n_rhs, 2 * p.n))
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        yd = torch.full_like(ud, float("nan"))
        s.matvec(ud, yd, precision=bipb.DF64, med=_med(bipb, p))
        Y = yd.cpu().numpy()
    for r in (0, n_rhs // 2, n_rhs - 1):
        ref = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, U[r])
        np.testing.assert_allclose(Y[r], ref, rtol=0, atol=2e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n_rhs", [16, 40, 64])
def test_exact_tensor_residual_matches_cuda_core_df64(bipb, orc, n_rhs):
    """The double-float mat-vec of 16, 40 and 64 right-hand sides (the fewest
    the tensor-core form takes, a partly filled block of 64 columns, a full
    one) on the tensor cores (exact base-128 digits) against the same on the
    CUDA cores and against the oracle: right-hand sides of magnitude
    1e-20 .. 1e20 and one zero right-hand side."""
    p = _ragged(3)
    eps = p.eps_out / p.eps_in
    rng = np.random.default_rng(77)
    mags = 10.0 ** rng.uniform(-20, 20, n_rhs)
    U = rng.standard_normal((n_rhs, 2 * p.n)) * mags[:, None]
    U[11] = 0.0
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        yt, yc = torch.full_like(ud, float("nan")), torch.full_like(ud, float("nan"))
        s.matvec(ud, yt, precision=bipb.DF64, med=_med(bipb, p))
        s.exact_tensor_residual(False)
        s.matvec(ud, yc, precision=bipb.DF64, med=_med(bipb, p))
        Yt, Yc = yt.cpu().numpy(), yc.cpu().numpy()
    assert np.all(Yt[11] == 0.0)
    for r in range(n_rhs):
        if r == 11:
            continue
        scale = np.abs(Yc[r]).max()
        np.testing.assert_allclose(Yt[r], Yc[r], rtol=0, atol=1e-13 * scale, err_msg=str(r))
    for r in (0, n_rhs // 2 + 3, n_rhs - 1):
        ref = orc.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, U[r])
        np.testing.assert_allclose(Yt[r], ref, rtol=0, atol=2e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n_rhs", [4, 40])
def test_exact_tensor_residual_transpose_matches_oracle(bipb, orc, n_rhs):
    """The double-float A^T U of a batch of right-hand sides on the tensor cores
    (the transposed blocks as exact base-128 digits, the output's area on the
    sums) against the single-system double-float transpose on the CUDA cores
    and against the oracle's transpose: right-hand sides of magnitude
    1e-20 .. 1e20 and one zero right-hand side."""
    p = _ragged(3)
    eps = p.eps_out / p.eps_in
    rng = np.random.default_rng(88 + n_rhs)
    mags = 10.0 ** rng.uniform(-20, 20, n_rhs)
    U = rng.standard_normal((n_rhs, 2 * p.n)) * mags[:, None]
    U[1] = 0.0
    med = _med(bipb, p)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        ud = _dev(U)
        yt = torch.full_like(ud, float("nan"))
        s.matvec(ud, yt, precision=bipb.DF64, transpose=True, med=med)
        yc = torch.full_like(ud, float("nan"))
        for r in range(n_rhs):  # one system at a time: the symmetric double-float kernel
            s.matvec(ud[r], yc[r], precision=bipb.DF64, transpose=True, med=med)
        Yt, Yc = yt.cpu().numpy(), yc.cpu().numpy()
    assert np.all(Yt[1] == 0.0)
    for r in range(n_rhs):
        if r == 1:
            continue
        np.testing.assert_allclose(Yt[r], Yc[r], rtol=0, atol=1e-13 * np.abs(Yc[r]).max(), err_msg=str(r))
    for r in (0, n_rhs - 1):
        ref = orc.matvec_t(p.centroids, p.normals, p.areas, eps, p.kappa, U[r])
        np.testing.assert_allclose(Yt[r], ref, rtol=0, atol=2e-12 * np.abs(ref).max())


# ---------------------------------------------------------------- potential at points, free energy
def _ball(rng, n, r0, r1):
    """n points with radii uniform in [r0, r1) and uniform directions."""
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * rng.uniform(r0, r1, n)[:, None]


def test_potential_at_points_matches_oracle(bipb, orc):
    """Potential at 300 points inside the molecule (Eq. eq_inside, with S1 of
    the charges) and 257 points in the solvent (the exterior
    representation), for two charge sets, against the oracle's potential of
    its own solve (both FP64 to 1e-12): 1e-9 of the largest value."""
    base = synth.protein_like_problem(level=3, n_charges=12)
    batch = synth.batched_charges(base, n_rhs=2, n_charges=12)
    eps = batch.eps_out / batch.eps_in
    rng = np.random.default_rng(40)
    pin = _ball(rng, 300, 0.0, 20.0)   # the surface lies at r >= 25.5
    pout = _ball(rng, 257, 31.0, 80.0)  # ... and at r <= 29.3
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.set_charges(batch.charge_pos, batch.q)
        with pytest.raises(bipb.BipbError):
            s.potential_at(pin, inside=True)  # no solve yet
        s.solve(tol=1e-12, precision=bipb.FP64)
        vin = s.potential_at(pin, inside=True)
        vout = s.potential_at(pout, inside=False)
        assert s.potential_at(np.zeros((0, 3))).shape == (2, 0)
    for r in range(2):
        ref = orc.solve(batch, rhs=r, method="gmres", tol=1e-12)
        y, q = batch.charge_pos[r], batch.q[r]
        rin = orc.KCAL * orc.potential(batch.centroids, batch.normals, batch.areas, eps, batch.kappa, ref.u, pin,
                                       True, y, q, batch.eps_in)
        rout = orc.KCAL * orc.potential(batch.centroids, batch.normals, batch.areas, eps, batch.kappa, ref.u, pout,
                                        False)
        np.testing.assert_allclose(vin[r], rin, rtol=0, atol=1e-9 * np.abs(rin).max())
        np.testing.assert_allclose(vout[r], rout, rtol=0, atol=1e-9 * np.abs(rout).max())


def test_energy_free_matches_oracle(bipb, orc):
    """E_free = E_sol + E_coul per charge set (Eq. free_energy without the
    self terms) against the oracle; E_coul alone to 1e-12."""
    base = synth.protein_like_problem(level=3, n_charges=300)
    batch = synth.batched_charges(base, n_rhs=3, n_charges=300)
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.set_charges(batch.charge_pos, batch.q)
        s.solve(tol=1e-12, precision=bipb.FP64)
        e_sol = s.energy()
        e_free, e_coul = s.energy_free()
    for r in range(3):
        ec = orc.KCAL * orc.coulomb(batch.charge_pos[r], batch.q[r], batch.eps_in)
        assert e_coul[r] == pytest.approx(ec, rel=1e-12)
        ref = orc.solve(batch, rhs=r, method="gmres", tol=1e-12)
        assert e_free[r] == pytest.approx(ref.energy_kcal + ec, rel=1e-10)
        assert e_free[r] - e_sol[r] == pytest.approx(e_coul[r], rel=1e-12)


def test_potential_at_rejects_batch_handles(bipb):
    probs = [synth.born_problem(level=1), synth.born_problem(level=2)]
    with bipb.BatchSurface([(q.centroids, q.normals, q.areas) for q in probs]) as s:
        s.set_charges([(q.charge_pos, q.q[0]) for q in probs])
        s.solve(tol=1e-10, precision=bipb.FP64)
        with pytest.raises(bipb.BipbError):
            s.potential_at(np.zeros((3, 3)))
        ef, ec = s.energy_free()  # the free energy works per surface
        np.testing.assert_allclose(ec, 0.0)  # one charge per surface: no pairs
        np.testing.assert_allclose(ef, s.energy(), rtol=1e-14)


# ---------------------------------------------------------------- preconditioned solves
@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed", "mixed_df64", "mixed_tensor", "mixed_tree"])
def test_self_block_preconditioned_solve_matches_oracle(bipb, orc, prec):
    """GMRES with the element self-block preconditioner (Sec. 2.2.4, applied
    on the right) reaches the same solution as the oracle's unpreconditioned
    solve, in fewer iterations than without it."""
    p = synth.kirkwood_problem(level=4)
    ref = orc.solve(p, method="gmres", tol=1e-12)
    phi_ref, _ = ref.surface_potential()
    P = {"fp64": bipb.FP64, "mixed": bipb.MIXED, "df64": bipb.DF64, "mixed_df64": bipb.MIXED_DF64,
         "mixed_tensor": bipb.MIXED_TENSOR, "mixed_tree": bipb.MIXED_TREE}[prec]
    tol = 1e-12 if prec in ("fp64", "df64") else 1e-8
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        plain = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=tol, precision=P)[0]
        info = s.solve(eps_in=p.eps_in, eps_out=p.eps_out, kappa=p.kappa, tol=tol, precision=P,
                       precond=bipb.PRECOND_SELF)[0]
        e = s.energy()[0]
        phi, _ = s.surface_potential()
    assert info["converged"] and info["rel_residual"] <= tol
    assert info["iters"] < 0.6 * plain["iters"]
    rt = 1e-10 if prec in ("fp64", "df64") else 1e-7
    assert e == pytest.approx(ref.energy_kcal, rel=rt)
    assert np.linalg.norm(phi[0] - phi_ref) / np.linalg.norm(phi_ref) < rt


@pytest.mark.parametrize("prec", ["mixed_df64", "mixed_tensor"])
def test_self_block_preconditioned_batch_and_adjoint(bipb, orc, prec):
    """Charge sets solved together with the preconditioner (MIXED_DF64 with
    three sets; MIXED_TENSOR with five, so that the adjoint's residual takes
    the exact tensor-core transpose) and the adjoint gradient taken with it,
    against the unpreconditioned run."""
    n_rhs = 3 if prec == "mixed_df64" else 5
    precision = bipb.MIXED_DF64 if prec == "mixed_df64" else bipb.MIXED_TENSOR
    base = synth.protein_like_problem(level=3, n_charges=40)
    batch = synth.batched_charges(base, n_rhs=n_rhs, n_charges=40)
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.set_charges(batch.charge_pos, batch.q)
        prm = bipb.solve_params(batch.eps_in, batch.eps_out, batch.kappa, tol=1e-10, precision=precision)
        s.solve(prm)
        e0 = s.energy()
        dq0, dy0 = s.energy_grad(prm)
        prm.precond = bipb.PRECOND_SELF
        info = s.solve(prm)
        e1 = s.energy()
        dq1, dy1 = s.energy_grad(prm)
    assert all(i["converged"] and i["rel_residual"] <= 1e-10 for i in info)
    np.testing.assert_allclose(e1, e0, rtol=1e-8)
    np.testing.assert_allclose(dq1, dq0, rtol=0, atol=1e-7 * np.abs(dq0).max())
    np.testing.assert_allclose(dy1, dy0, rtol=0, atol=1e-7 * np.abs(dy0).max())


def test_new_entry_points_reject_bad_arguments(bipb):
    p = synth.born_problem(level=2)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=1e-8, precision=bipb.FP64)
        prm.precond = 7
        with pytest.raises(bipb.BipbError):
            s.solve(prm)
        prm.precond, prm.reserved = bipb.PRECOND_SELF, 1
        with pytest.raises(bipb.BipbError):
            s.solve(prm)
        prm.reserved = 0
        assert s.solve(prm)[0]["converged"]
        L = bipb.load_library()
        pts = np.array([[0.1, 0.2, 0.3]])
        out = np.zeros(1)
        st = L.bipb_potential_at(s.handle, 5, 1, pts.ctypes.data, out.ctypes.data)
        assert st == bipb.BIPB_ERR_INVALID_ARG
        with pytest.raises(bipb.BipbError):
            s.potential_at(np.array([[np.nan, 0.0, 0.0]]))
        # the inside potential at the centre's neighbourhood is finite and the outside one decays
        v_in = s.potential_at(np.array([[0.3, 0.0, 0.0]]), inside=True)
        v_out = s.potential_at(np.array([[10.0, 0.0, 0.0], [20.0, 0.0, 0.0]]), inside=False)
        assert np.isfinite(v_in).all() and v_out[0, 0] > v_out[0, 1] > 0


def test_charge_on_a_centroid_is_rejected(bipb):
    """A charge exactly on a centroid (FP64) is rejected; one that only rounds
    to the same FP32 point is accepted."""
    p = synth.born_problem(level=2)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        on = p.centroids[17].copy()
        with pytest.raises(bipb.BipbError, match="centroid"):
            s.set_charges(np.array([[0.0, 0.0, 0.0], on]), np.array([[1.0, -1.0]]))
        near = on + np.array([1e-12, 0.0, 0.0])
        s.set_charges(np.array([[0.0, 0.0, 0.0], near]), np.array([[1.0, -1.0]]))


# ---------------------------------------------------------------- far-field (treecode) mat-vec, Sec. 2.2.3
def _tc_vectors(p, seed):
    x = p.centroids / np.abs(p.centroids).max()
    rng = np.random.default_rng(seed)
    return np.stack([rng.standard_normal(2 * p.n), rng.standard_normal(2 * p.n),
                     np.concatenate([1.0 + 0.3 * x[:, 2], 0.5 - 0.2 * x[:, 0]])])


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("params", [(0.7, 4, 64), (0.8, 6, 64), (0.9, 8, 64), (0.8, 4, 256), (0.0, 6, 256)])
def test_treecode_matvec_matches_oracle_treecode(bipb, orc, params, transpose):
    """The far-field FP32 mat-vec (A u, or A^T u) against the oracle's
    treecode on the same tree (FP64, every row): the FP32 mat-vec's bounds,
    3e-6 in the 2-norm and 2e-5 of the largest output; theta = 0 is the
    direct mat-vec."""
    theta, deg, leaf = params
    p = _ragged(4)
    eps = p.eps_out / p.eps_in
    U = _tc_vectors(p, 70)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.treecode(theta, deg, leaf)
        ud = _dev(U)
        yd = torch.full_like(ud, float("nan"))
        s.matvec(ud, yd, precision=bipb.TREE32, transpose=transpose, med=_med(bipb, p))
        Y = yd.cpu().numpy()
        pairs, far, leaves = s.treecode_stats()
    assert (far > 0) == (theta > 0)
    assert leaves >= p.n // leaf and pairs <= p.n * p.n
    for r in range(U.shape[0]):
        ref = orc.treecode.matvec(p.centroids, p.normals, p.areas, eps, p.kappa, U[r], theta, deg, leaf,
                                  transpose=transpose)
        assert np.all(np.isfinite(Y[r]))
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) < 3e-6, (params, r)
        assert np.abs(Y[r] - ref).max() < 2e-5 * np.abs(ref).max(), (params, r)


def test_treecode_rejects_bad_use(bipb):
    p = synth.born_problem(level=2)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        for bad in ((1.0, 6, 256), (-0.1, 6, 256), (0.5, 5, 256), (0.5, 6, 16), (0.5, 6, 1024)):
            with pytest.raises(bipb.BipbError):
                s.treecode(*bad)
    probs = [synth.born_problem(level=1), synth.born_problem(level=2)]
    with bipb.BatchSurface([(q.centroids, q.normals, q.areas) for q in probs]) as s:
        u = _dev(np.ones(sum(2 * q.n for q in probs)))
        with pytest.raises(bipb.BipbError):
            s.matvec(u, torch.empty_like(u), precision=bipb.TREE32)


def test_mixed_tree_solve_matches_oracle(bipb, orc):
    """MIXED_TREE (far-field FP32 Krylov mat-vecs, direct double-float
    residual) reaches the exact discrete solution: energy and potentials of
    three charge sets against the oracle's GMRES to 1e-12 within 1e-7, and the
    adjoint gradient (far-field FP32 transpose inside, direct double-float
    transpose residual) within 1e-5."""
    base = synth.protein_like_problem(level=4, n_charges=30)
    batch = synth.batched_charges(base, n_rhs=3, n_charges=30)
    with bipb.Surface(batch.centroids, batch.normals, batch.areas) as s:
        s.treecode(0.7, 4, 64)
        s.set_charges(batch.charge_pos, batch.q)
        prm = bipb.solve_params(batch.eps_in, batch.eps_out, batch.kappa, tol=1e-9, precision=bipb.MIXED_TREE)
        info = s.solve(prm)
        e = s.energy()
        phi, _ = s.surface_potential()
        dq, dy = s.energy_grad(prm)
        assert s.treecode_stats()[1] > 0  # some clusters act through proxies
    for r in range(3):
        assert info[r]["converged"] and info[r]["rel_residual"] <= 1e-9
        assert info[r]["refine_steps"] <= 3 and info[r]["matvecs32"] > 0
        ref = orc.solve(batch, rhs=r, method="gmres", tol=1e-12)
        assert e[r] == pytest.approx(ref.energy_kcal, rel=1e-7)
        phi_ref, _ = ref.surface_potential()
        assert np.linalg.norm(phi[r] - phi_ref) / np.linalg.norm(phi_ref) < 1e-7
    e_ref, dq_ref, dy_ref = orc.energy_gradient(batch, rhs=1, method="gmres", tol=1e-12)
    np.testing.assert_allclose(dq[1], dq_ref, rtol=1e-5)
    np.testing.assert_allclose(dy[1], dy_ref, rtol=0, atol=1e-5 * np.abs(dy_ref).max())
