"""The seeded input generators shared by the oracle and the CUDA side: sizes,
geometry and charge placement of the benchmark's workloads."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_is_a_closed_triangulated_sphere(level):
    v, f = synth.icosphere(level, 1.0)
    assert f.shape == (20 * 4 ** level, 3)
    edges = {tuple(sorted(e)) for t in f for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    assert v.shape[0] - len(edges) + f.shape[0] == 2  # Euler characteristic of a sphere
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, rtol=1e-14)


def test_born_and_kirkwood_workloads():
    b = synth.born_problem(level=3)
    assert b.n == 1280 and b.nc == 1 and np.all(b.charge_pos == 0) and b.q[0, 0] == 1.0
    k = synth.kirkwood_problem(level=5)
    assert k.n == 20480 and k.nc == 50 and k.q.shape == (1, 50)
    assert np.all(np.linalg.norm(k.charge_pos, axis=1) < 16.0)
    assert np.all(np.abs(k.q) <= 1.0)
    for p, radius in ((b, 2.0), (k, 20.0)):
        np.testing.assert_allclose(np.linalg.norm(p.normals, axis=1), 1.0, rtol=1e-13)
        assert np.all(np.einsum("ij,ij->i", p.normals, p.centroids) > 0)  # outward
        # inscribed flat triangles: slightly less than the sphere's area, converging to it
        total = p.areas.sum() / (4 * np.pi * radius ** 2)
        assert 0.98 < total < 1.0
        assert np.unique(p.centroids, axis=0).shape[0] == p.n
    k2 = synth.kirkwood_problem(level=5)
    assert np.array_equal(k.charge_pos, k2.charge_pos) and np.array_equal(k.q, k2.q)


def test_displaced_surface_and_charges_inside():
    v, f, rfn, rng = synth.displaced_icosphere(4, 25.0, 3)
    c, n, a = synth.triangle_geometry(v, f)
    assert c.shape == (5120, 3) and np.all(a > 0)
    r = np.linalg.norm(v, axis=1)
    np.testing.assert_allclose(r, rfn(v / r[:, None]), rtol=1e-12)
    assert r.max() <= rfn.rmax * (1 + 1e-12) and r.min() > 0.3 * 25.0
    pos, q = synth.charges_inside_surface(rng, 500, rfn)
    rp = np.linalg.norm(pos, axis=1)
    assert pos.shape == (500, 3) and np.all(rp < 0.8 * rfn(pos / rp[:, None]))
    assert np.all(np.abs(q) <= 1.0)


def test_batched_charge_sets_are_seeded_per_set():
    base = synth.Problem("base", *synth.triangle_geometry(*synth.displaced_icosphere(3, 25.0, 3)[:2]),
                         np.zeros((1, 3)), np.ones((1, 1)), meta=dict(level=3, radius=25.0, seed=3))
    p = synth.batched_charges(base, n_rhs=3, n_charges=20)
    assert p.charge_pos.shape == (3, 20, 3) and p.q.shape == (3, 20)
    again = synth.batched_charges(base, n_rhs=2, n_charges=20)
    assert np.array_equal(p.charge_pos[:2], again.charge_pos) and np.array_equal(p.q[:2], again.q)
    assert not np.array_equal(p.charge_pos[0], p.charge_pos[1])
