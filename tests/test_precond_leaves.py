"""Leaf size of the block-diagonal preconditioner (Sec. 2.2.4), on the oracle.

The paper preconditions GMRES with the block diagonal of A over the leaves of
its tree.  The library applies it with one element per leaf
(BIPB_PRECOND_SELF), where the block is the diagonal of A and costs nothing
per iteration.  This test is the record of why larger leaves are not built:
on a sphere, on strongly displaced spheres and on two nearly touching
spheres, GMRES(10) to 1e-8 with leaves of 16 or 64 elements (the tree of the
far-field mat-vec) never takes fewer iterations than with single elements,
and on the 0.1 A gap it takes two to three times as many.  Every solve is
FP64 on the dense matrix, and every preconditioned solution is the solution
of A u = b.

Iteration counts measured with this test (GMRES(10), tol 1e-8):
    case                       plain   n0=1   n0=16   n0=64
    Kirkwood sphere, level 3     26       8       8       8
    displaced 30 %, level 3      37       9       9       9
    displaced 45 %, level 3      40       9       9       9
    two spheres, gap 0.5 A       34       9      10      10
    two spheres, gap 0.1 A      245      11      24      37
"""
import numpy as np
import pytest

import synth

CASES = {
    "kirkwood_l3": (lambda: synth.kirkwood_problem(level=3), (26, 8, 8, 8)),
    "displaced_30": (lambda: synth.strongly_displaced_problem(amp=0.3), (37, 9, 9, 9)),
    "displaced_45": (lambda: synth.strongly_displaced_problem(amp=0.45), (40, 9, 9, 9)),
    "gap_0.5": (lambda: synth.two_spheres_problem(gap=0.5), (34, 9, 10, 10)),
    "gap_0.1": (lambda: synth.two_spheres_problem(gap=0.1), (245, 11, 24, 37)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_larger_leaves_do_not_reduce_iterations(orc, case):
    make, expected = CASES[case]
    p = make()
    eps = p.eps_out / p.eps_in
    A = orc.assemble(p.centroids, p.normals, p.areas, eps, p.kappa)
    b = orc.source(p.centroids, p.normals, p.charge_pos, p.q[0], p.eps_in)
    u_ref = np.linalg.solve(A, b)
    _, info = orc.gmres(lambda v: A @ v, b, tol=1e-8, restart=10, max_iter=600)
    its = {"plain": info["iters"]}
    for n0 in (1, 16, 64):
        blks = orc.precond.blocks(A, orc.precond.leaves(p.centroids, n0))
        u, info = orc.precond.solve_right(A, b, blks, tol=1e-8, restart=10, max_iter=600)
        assert info["converged"]
        assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-6
        its[n0] = info["iters"]
    # the counts of the table above, within one iteration (BLAS summation order)
    for got, want in zip((its["plain"], its[1], its[16], its[64]), expected):
        assert abs(got - want) <= 1, (case, its)
    # single-element leaves cut the plain count at least in three; larger leaves never do better
    assert its[1] * 3 <= its["plain"]
    assert its[16] >= its[1] and its[64] >= its[1]


def test_single_element_block_is_the_diagonal(orc):
    """With the self pair omitted, an element's 2 x 2 block of A is
    diag(1/2 (1 + eps), 1/2 (1 + 1/eps)): what BIPB_PRECOND_SELF scales by."""
    p = synth.born_problem(level=1)
    eps = p.eps_out / p.eps_in
    A = orc.assemble(p.centroids, p.normals, p.areas, eps, p.kappa)
    for idx, B in orc.precond.blocks(A, orc.precond.leaves(p.centroids, 1))[:5]:
        np.testing.assert_allclose(B, np.diag([2 / (1 + eps), 2 / (1 + 1 / eps)]), rtol=1e-15)
