"""The C ABI library builds, loads and exports every declared symbol; host-side
argument validation rejects bad input before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bipb():
    from paper_2312_10044_gb300.build import build

    build()
    import paper_2312_10044_gb300 as b

    b.load_library()
    return b


def _declared():
    src = open(os.path.join(ROOT, "include", "bipb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bipb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_api():
    names = _declared()
    for must in ("bipb_surface_create", "bipb_charges_set", "bipb_solve", "bipb_energy",
                 "bipb_surface_potential", "bipb_energy_grad", "bipb_matvec", "bipb_surface_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(bipb):
    L = ctypes.CDLL(bipb.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(bipb.EXPORTED) == set(_declared())


def test_version_and_status_strings(bipb):
    L = bipb.load_library()
    assert b"sm_103a" in L.bipb_version()
    assert L.bipb_status_string(bipb.BIPB_ERR_NOT_CONVERGED) == b"not converged"


def _create(bipb, c, n, a):
    L = bipb.load_library()
    h = ctypes.c_void_p()
    c, n, a = (np.ascontiguousarray(v, dtype=np.float64) for v in (c, n, a))
    st = L.bipb_surface_create(a.shape[0], c.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                               a.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(h))
    return st, h, L.bipb_last_error().decode()


@pytest.fixture(scope="module")
def geom():
    p = synth.born_problem(level=1)
    return p.centroids.copy(), p.normals.copy(), p.areas.copy()


@pytest.mark.parametrize("case", ["nan_centroid", "zero_area", "neg_area", "bad_normal", "duplicate", "too_small",
                                  "empty", "inf_normal", "duplicate_fp32"])
def test_create_rejects_bad_geometry(bipb, geom, case):
    c, n, a = (v.copy() for v in geom)
    if case == "nan_centroid":
        c[3, 1] = np.nan
    elif case == "zero_area":
        a[7] = 0.0
    elif case == "neg_area":
        a[0] = -1.0
    elif case == "bad_normal":
        n[2] *= 1.01
    elif case == "duplicate":
        c[5] = c[9]
    elif case == "too_small":
        c, n, a = c[:1], n[:1], a[:1]
    elif case == "empty":
        c, n, a = c[:0], n[:0], a[:0]
    elif case == "inf_normal":
        n[4, 0] = np.inf
    elif case == "duplicate_fp32":
        # distinct in FP64, equal once rounded to the FP32 working copy
        c[5] = c[9] + 1e-9
    st, h, msg = _create(bipb, c, n, a)
    assert st == bipb.BIPB_ERR_INVALID_ARG, msg
    assert h.value is None
    assert msg
    if case == "duplicate_fp32":
        assert "FP32" in msg


def test_null_and_stale_handles_are_rejected(bipb):
    L = bipb.load_library()
    q = np.ones(1)
    pos = np.zeros((1, 3))
    st = L.bipb_charges_set(None, 1, pos.ctypes.data_as(ctypes.c_void_p), 1, 1, q.ctypes.data_as(ctypes.c_void_p))
    assert st == bipb.BIPB_ERR_STATE
    e = np.zeros(1)
    assert L.bipb_energy(ctypes.c_void_p(12345678), e.ctypes.data_as(ctypes.c_void_p)) == bipb.BIPB_ERR_STATE
    assert L.bipb_surface_size(None) == 0
    # the device-pointer and far-field entry points check the handle first as well
    stale = ctypes.c_void_p(12345678)
    assert L.bipb_charges_set_dev(None, 1, None, 1, 1, None) == bipb.BIPB_ERR_STATE
    assert L.bipb_energy_dev(stale, None) == bipb.BIPB_ERR_STATE
    assert L.bipb_energy_grad_dev(None, None, None, None) == bipb.BIPB_ERR_STATE
    assert L.bipb_treecode(stale, 0.5, 6, 256) == bipb.BIPB_ERR_STATE
    assert L.bipb_treecode_stats(None, None, None, None) == bipb.BIPB_ERR_STATE


def test_solve_params_layout_matches_header(bipb):
    # medium (3 doubles) + tol + 4 ints + inner_tol + pointer + precond + reserved
    assert ctypes.sizeof(bipb.bipb_solve_params) == 3 * 8 + 8 + 4 * 4 + 8 + 8 + 4 + 4
    assert ctypes.sizeof(bipb.bipb_solve_info) == 6 * 4 + 2 * 8


def test_static_matvec_binding_rejects_mismatched_sizes(bipb):
    """The allocation-free mat-vec trusts its sizes on the device, so the
    binding checks them (and the device) before any call into the library:
    CPU tensors stand in here, and every mismatch raises ValueError first."""
    torch = pytest.importorskip("torch")
    n = 10
    z = lambda k: torch.zeros(k, dtype=torch.float64)  # noqa: E731
    good = dict(centroids=z(3 * n), normals=z(3 * n), areas=z(n), u=z(2 * n), y=z(2 * n))
    bad = [dict(good, centroids=z(3 * n + 1)), dict(good, normals=z(3 * n - 3)), dict(good, areas=z(n + 1)),
           dict(good, u=z(2 * n - 1)), dict(good, y=z(4 * n))]
    for kw in bad:
        with pytest.raises(ValueError, match="expected centroids"):
            bipb.matvec32_static(**kw)
    # right sizes but not on a CUDA device: rejected before the library call as well
    with pytest.raises(ValueError, match="CUDA"):
        bipb.matvec32_static(**good)
