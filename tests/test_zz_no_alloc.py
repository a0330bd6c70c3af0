"""The allocation-free FP32 mat-vec (bipb_matvec32_static) agrees with the
handle-based FP32 mat-vec (bipb_matvec) and with the FP64 oracle, through
the C ABI, on two calls in a row, with and without salt (kappa = 0 takes the
pair formula without the screened terms), on the current stream and on a
stream of its own.

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


def _compare(bipb, orc, p, seed, kappa, stream=None):
    med = bipb.medium(p.eps_in, p.eps_out, kappa)
    u_host = np.random.default_rng(seed).standard_normal(2 * p.n)
    u = _dev(u_host)
    y_ref = torch.empty_like(u)
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.matvec(u, y_ref, precision=bipb.FP32, med=med)
        torch.cuda.synchronize()
    y = torch.full_like(u, float("nan"))
    geo = (_dev(p.centroids), _dev(p.normals), _dev(p.areas))
    if stream is None:
        bipb.matvec32_static(*geo, u, y, med=med)
        torch.cuda.synchronize()
    else:
        stream.wait_stream(torch.cuda.current_stream())  # the inputs were written on the current stream
        with torch.cuda.stream(stream):
            bipb.matvec32_static(*geo, u, y, med=med, stream=stream.cuda_stream)
        stream.synchronize()
    a, r = y.cpu().numpy(), y_ref.cpu().numpy()
    exact = orc.matvec(p.centroids, p.normals, p.areas, p.eps_out / p.eps_in, kappa, u_host)
    assert np.all(np.isfinite(a))
    # the FP32 mat-vec tolerance used by the parity tests, against the handle
    # path and against the oracle
    for ref in (r, exact):
        assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 3e-6
        assert np.abs(a - ref).max() < 2e-5 * np.abs(ref).max()


def _ragged():
    p = synth.protein_like_problem(level=3, n_charges=5)
    keep = np.arange(p.n) % 7 != 3
    p.centroids, p.normals, p.areas = p.centroids[keep], p.normals[keep], p.areas[keep]
    return p


@pytest.mark.parametrize("kappa", [0.1257, 0.0])
def test_static_matvec_matches_handle_matvec_twice(bipb, orc, kappa):
    # first call: 20480 triangles; second call: a ragged smaller surface,
    # so leftovers of the first call sit in the shared scratch array
    _compare(bipb, orc, synth.kirkwood_problem(level=5), seed=1, kappa=kappa)
    _compare(bipb, orc, _ragged(), seed=2, kappa=kappa)


def test_static_matvec_on_its_own_stream(bipb, orc):
    s = torch.cuda.Stream()
    _compare(bipb, orc, _ragged(), seed=3, kappa=0.1257, stream=s)
    _compare(bipb, orc, synth.born_problem(level=3), seed=4, kappa=0.1257, stream=s)


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
