"""The allocation-free FP32 mat-vec (bipb_matvec32_static) agrees with the
handle-based FP32 mat-vec (bipb_matvec), through the C ABI, on two calls in a
row.

bipb_matvec32_static serves callers that cannot call cudaMalloc (a host
framework that already owns nearly all device memory, or a loop that must
not allocate after start-up).  Its scratch is one static device array shared
by every call, so the second call here also checks that leftovers of the
first (a larger surface) do not leak into the result.  This file is named to
be collected last.
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


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _compare(bipb, p, seed):
    med = bipb.medium(p.eps_in, p.eps_out, p.kappa)
    u = _dev(np.random.default_rng(seed).standard_normal(2 * p.n))
    y_ref = torch.empty_like(u)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.matvec(u, y_ref, precision=bipb.FP32, med=med)
        torch.cuda.synchronize()
    y = torch.full_like(u, float("nan"))
    bipb.matvec32_static(_dev(p.centroids), _dev(p.normals), _dev(p.areas), u, y, med=med)
    torch.cuda.synchronize()
    a, r = y.cpu().numpy(), y_ref.cpu().numpy()
    assert np.all(np.isfinite(a))
    # the FP32 mat-vec tolerance used by the parity tests
    assert np.linalg.norm(a - r) / np.linalg.norm(r) < 3e-6
    assert np.abs(a - r).max() < 2e-5 * np.abs(r).max()


def test_static_matvec_matches_handle_matvec_twice(bipb):
    # first call: 20480 triangles; second call: a ragged smaller surface
    _compare(bipb, synth.kirkwood_problem(level=5), seed=1)
    p = synth.protein_like_problem(level=3, n_charges=5)
    keep = np.arange(p.n) % 7 != 3
    p.centroids, p.normals, p.areas = p.centroids[keep], p.normals[keep], p.areas[keep]
    _compare(bipb, p, seed=2)


def test_static_matvec_rejects_oversized_surface(bipb):
    n = bipb.STATIC_MAX_N + 1
    z = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    a = torch.ones(n, dtype=torch.float64, device="cuda")
    u = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(u)
    with pytest.raises(bipb.BipbError) as ei:
        bipb.matvec32_static(z, z.clone(), a, u, y)
    assert ei.value.status == bipb.BIPB_ERR_INVALID_ARG
    assert "32768" in str(ei.value)
