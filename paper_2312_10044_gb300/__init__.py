"""Python binding of libbipb, the GB300 direct-sum boundary-integral PB solver.

Argument marshalling only: every step of the path runs in the CUDA kernels
of ``libbipb.so`` (built in-tree by :func:`paper_2312_10044_gb300.build.build`).
There is no CPU fallback; importing this package fails if the library is
missing.  The names follow the C ABI in ``include/bipb.h``.

Host arrays are numpy FP64; device arrays are CUDA torch tensors (FP64,
contiguous), used only as device memory.
"""
from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbipb.so")

BIPB_OK = 0
BIPB_ERR_INVALID_ARG = 1
BIPB_ERR_CUDA = 2
BIPB_ERR_OOM = 3
BIPB_ERR_NOT_CONVERGED = 4
BIPB_ERR_STATE = 5

FP64 = 0
MIXED = 1
FP32 = 2
DF64 = 3
MIXED_DF64 = 4
TENSOR = 5
MIXED_TENSOR = 6
TF32, MIXED_TF32 = TENSOR, MIXED_TENSOR  # earlier names of the same values
TREE32 = 7
MIXED_TREE = 8

KCAL = 4.0 * np.pi * 332.0716  # internal units -> kcal/mol (per e)

EXPORTED = (
    "bipb_surface_create", "bipb_surface_destroy", "bipb_surface_size", "bipb_charges_set",
    "bipb_solve", "bipb_energy", "bipb_surface_potential", "bipb_energy_grad", "bipb_matvec",
    "bipb_source", "bipb_reaction", "bipb_last_error", "bipb_status_string", "bipb_version",
    "bipb_timer_enable", "bipb_timer_read", "bipb_launch_count", "bipb_matvec32_static",
    "bipb_autotune", "bipb_matvec_variant", "bipb_surface_create_batch", "bipb_charges_set_batch",
    "bipb_symmetric_pairs", "bipb_exact_tensor_residual", "bipb_potential_at", "bipb_energy_free", "bipb_treecode", "bipb_treecode_stats",
    "bipb_charges_set_dev", "bipb_energy_dev", "bipb_energy_grad_dev",
)
MATVEC32_VARIANTS = 10

KERNEL_KINDS = ("matvec64", "matvec32", "matvec64_t", "matvec32_t", "source", "reaction", "energy_row", "grad",
                "matvec_df", "matvec_df_t", "matvec_tc", "potential", "matvec_tree")
REGION_INSIDE = 0
REGION_OUTSIDE = 1
PRECOND_NONE = 0
PRECOND_SELF = 1


class bipb_medium(ctypes.Structure):
    _fields_ = [("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double), ("kappa", ctypes.c_double)]


class bipb_solve_params(ctypes.Structure):
    _fields_ = [
        ("medium", bipb_medium),
        ("tol", ctypes.c_double),
        ("restart", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("inner_max_iter", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("x0", ctypes.c_void_p),
        ("precond", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class bipb_solve_info(ctypes.Structure):
    _fields_ = [
        ("converged", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("refine_steps", ctypes.c_int),
        ("matvecs64", ctypes.c_int),
        ("matvecs32", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BipbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_charge_versions = itertools.count(1)


def load_library():
    """Load libbipb.so (ctypes); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbipb.so not found at {LIB_PATH}: run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = ctypes.CDLL(LIB_PATH)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "bipb_surface_create": ([I64, P, P, P, P, P], st),
        "bipb_surface_destroy": ([P], st),
        "bipb_surface_size": ([P], I64),
        "bipb_charges_set": ([P, I64, P, I, I, P], st),
        "bipb_solve": ([P, P, P], st),
        "bipb_energy": ([P, P], st),
        "bipb_surface_potential": ([P, P, P], st),
        "bipb_energy_grad": ([P, P, P, P], st),
        "bipb_matvec": ([P, P, I, I, I, P, P], st),
        "bipb_source": ([P, P, P], st),
        "bipb_reaction": ([P, P, P, P, P], st),
        "bipb_last_error": ([], ctypes.c_char_p),
        "bipb_status_string": ([I], ctypes.c_char_p),
        "bipb_version": ([], ctypes.c_char_p),
        "bipb_timer_enable": ([P, I], st),
        "bipb_timer_read": ([P, I, P, P], st),
        "bipb_launch_count": ([P, P], st),
        "bipb_matvec32_static": ([I64, P, P, P, P, P, P, P], st),
        "bipb_autotune": ([P, P, I, P, P], st),
        "bipb_surface_create_batch": ([I, P, P, P, P, P, P], st),
        "bipb_charges_set_batch": ([P, P, P, P], st),
        "bipb_matvec_variant": ([P, I], st),
        "bipb_symmetric_pairs": ([P, I], st),
        "bipb_exact_tensor_residual": ([P, I], st),
        "bipb_potential_at": ([P, I, I64, P, P], st),
        "bipb_energy_free": ([P, P, P], st),
        "bipb_treecode": ([P, D, I, I], st),
        "bipb_charges_set_dev": ([P, I64, P, I, I, P], st),
        "bipb_energy_dev": ([P, P], st),
        "bipb_energy_grad_dev": ([P, P, P, P], st),
        "bipb_treecode_stats": ([P, P, P, P], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status):
    if status != BIPB_OK:
        L = load_library()
        raise BipbError(status, L.bipb_last_error().decode())


def _host(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _hp(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _dp(t):
    """Device pointer of a CUDA FP64 contiguous torch tensor."""
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch

        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    except Exception:  # pragma: no cover - torch is optional for the host API
        return 0


def medium(eps_in=1.0, eps_out=80.0, kappa=0.1257):
    return bipb_medium(eps_in, eps_out, kappa)


def solve_params(eps_in=1.0, eps_out=80.0, kappa=0.1257, tol=1e-8, restart=10, max_iter=1000,
                 precision=MIXED, inner_max_iter=0, inner_tol=0.0, x0=None, precond=PRECOND_NONE):
    p = bipb_solve_params(bipb_medium(eps_in, eps_out, kappa), tol, restart, max_iter, precision,
                          inner_max_iter, inner_tol, None, precond, 0)
    return p


class Surface:
    """A triangulated surface on the GPU (one bipb_surface handle)."""

    def __init__(self, centroids, normals, areas, stream=None):
        self._L = load_library()
        c = _host(centroids, (-1, 3))
        n = _host(normals, (-1, 3))
        a = _host(areas, (-1,))
        if not (c.shape[0] == n.shape[0] == a.shape[0]):
            raise ValueError("centroids, normals and areas differ in length")
        h = ctypes.c_void_p()
        _check(self._L.bipb_surface_create(c.shape[0], _hp(c), _hp(n), _hp(a), ctypes.c_void_p(_stream(stream)),
                                           ctypes.byref(h)))
        self._h = h
        self.n = c.shape[0]
        self.sizes = [self.n]
        self.nc = 0
        self.n_rhs = 0
        self.n_charges_total = 0

    @property
    def n_systems(self):
        return self.n_rhs

    @property
    def unknowns(self):
        """Length of the batched unknown vector of the systems bipb_solve works on."""
        return 2 * self.n * self.n_rhs

    # -------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(self._L.bipb_surface_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -------------------------------------------------------------- charges
    def set_charges(self, pos, q):
        """pos: (Nc, 3) or (B, Nc, 3); q: (Nc,) or (B, Nc)."""
        q = _host(q)
        if q.ndim == 1:
            q = q[None, :]
        n_rhs, nc = q.shape
        pos = _host(pos)
        n_pos = 1 if pos.ndim == 2 else pos.shape[0]
        pos = _host(pos, (n_pos, nc, 3))
        _check(self._L.bipb_charges_set(self._h, nc, _hp(pos), n_pos, n_rhs, _hp(q)))
        self._charge_version = next(_charge_versions)
        self.nc, self.n_rhs = nc, n_rhs
        self.n_charges_total = nc * n_rhs

    def set_charges_dev(self, pos, q):
        """Charges from CUDA float64 tensors: pos (Nc, 3) or (B, Nc, 3), q (Nc,) or (B, Nc).
        Checked on the device; a bad charge is reported by the next solve."""
        if q.dim() == 1:
            q = q.reshape(1, -1)
        n_rhs, nc = q.shape
        n_pos = 1 if pos.dim() == 2 else pos.shape[0]
        if pos.numel() != n_pos * nc * 3 or n_pos not in (1, n_rhs):
            raise ValueError("pos must be (Nc, 3) or (B, Nc, 3) matching q")
        q, pos = q.contiguous(), pos.contiguous()
        _check(self._L.bipb_charges_set_dev(self._h, nc, _dp(pos), n_pos, n_rhs, _dp(q)))
        self._charge_version = next(_charge_versions)
        self._dev_charges = (pos, q)  # kept alive until the device has read them
        self.nc, self.n_rhs = nc, n_rhs
        self.n_charges_total = nc * n_rhs

    def energy_dev(self, out=None):
        """E_sol per configuration (kcal/mol) into a CUDA float64 tensor."""
        import torch

        out = out if out is not None else torch.empty(self.n_systems, dtype=torch.float64, device="cuda")
        _check(self._L.bipb_energy_dev(self._h, _dp(out)))
        return out

    def energy_grad_dev(self, params=None, **kw):
        """(dE/dq (B, Nc), dE/dpos (B, Nc, 3)) as CUDA float64 tensors."""
        import torch

        p = params if params is not None else solve_params(**kw)
        dq = torch.empty(self.n_charges_total, dtype=torch.float64, device="cuda")
        dy = torch.empty(self.n_charges_total, 3, dtype=torch.float64, device="cuda")
        _check(self._L.bipb_energy_grad_dev(self._h, ctypes.byref(p), _dp(dq), _dp(dy)))
        return dq.reshape(self.n_rhs, self.nc), dy.reshape(self.n_rhs, self.nc, 3)

    # -------------------------------------------------------------- solve / outputs
    def solve(self, params=None, x0=None, raise_on_not_converged=True, **kw):
        p = params if params is not None else solve_params(**kw)
        x0h = None
        if x0 is not None:
            x0h = _host(x0, (self.unknowns,))
            p.x0 = x0h.ctypes.data
        info = (bipb_solve_info * self.n_systems)()
        st = self._L.bipb_solve(self._h, ctypes.byref(p), info)
        p.x0 = None
        if st != BIPB_OK and not (st == BIPB_ERR_NOT_CONVERGED and not raise_on_not_converged):
            _check(st)
        return [i.as_dict() for i in info]

    def energy(self):
        e = np.zeros(self.n_systems)
        _check(self._L.bipb_energy(self._h, _hp(e)))
        return e

    def potential_at(self, pts, inside=True):
        """Potential (kcal/mol/e) at points (n, 3) A of the solute (inside) or
        the solvent (outside), shape (n_systems, n)."""
        p = _host(pts, (-1, 3))
        out = np.zeros((self.n_systems, p.shape[0]))
        region = REGION_INSIDE if inside else REGION_OUTSIDE
        _check(self._L.bipb_potential_at(self._h, region, p.shape[0], _hp(p), _hp(out)))
        return out

    def energy_free(self):
        """(E_free, E_coul) per system, kcal/mol: E_free = E_sol + E_coul."""
        ef = np.zeros(self.n_systems)
        ec = np.zeros(self.n_systems)
        _check(self._L.bipb_energy_free(self._h, _hp(ef), _hp(ec)))
        return ef, ec

    def surface_potential(self):
        """(phi, dphi/dnu): (n_rhs, N) arrays, or lists per surface for a batch handle."""
        phi = np.zeros(self.unknowns // 2)
        dphi = np.zeros(self.unknowns // 2)
        _check(self._L.bipb_surface_potential(self._h, _hp(phi), _hp(dphi)))
        return self._split_elems(phi), self._split_elems(dphi)

    def _split_elems(self, v):
        return v.reshape(self.n_rhs, self.n)

    def energy_grad(self, params=None, **kw):
        p = params if params is not None else solve_params(**kw)
        dq = np.zeros(self.n_charges_total)
        dy = np.zeros((self.n_charges_total, 3))
        _check(self._L.bipb_energy_grad(self._h, ctypes.byref(p), _hp(dq), _hp(dy)))
        return self._split_charges(dq), self._split_charges(dy)

    def _split_charges(self, v):
        return v.reshape((self.n_rhs, self.nc) + v.shape[1:])

    # -------------------------------------------------------------- device passes
    def matvec(self, u, y, precision=FP64, transpose=False, med=None):
        """y = A u (or A^T u); u, y CUDA float64 tensors of shape (k, 2N) or (2N,)."""
        m = med if med is not None else medium()
        n_vec = u.numel() // (2 * self.n)
        if u.numel() != n_vec * 2 * self.n or y.numel() != u.numel():
            raise ValueError("u and y must hold k * 2N values")
        _check(self._L.bipb_matvec(self._h, ctypes.byref(m), precision, int(transpose), n_vec, _dp(u), _dp(y)))
        return y

    def autotune(self, med=None, reps=3):
        """Pick the fastest FP32 mat-vec variant for this surface; returns (index, ms per mat-vec)."""
        m = med if med is not None else medium()
        v = ctypes.c_int()
        ms = ctypes.c_double()
        _check(self._L.bipb_autotune(self._h, ctypes.byref(m), reps, ctypes.byref(v), ctypes.byref(ms)))
        return v.value, ms.value

    def set_variant(self, variant):
        _check(self._L.bipb_matvec_variant(self._h, int(variant)))

    def treecode(self, theta=0.5, degree=6, leaf_size=256):
        """Parameters of the far-field mat-vec (TREE32, MIXED_TREE): MAC theta,
        interpolation degree per coordinate, largest leaf."""
        _check(self._L.bipb_treecode(self._h, float(theta), int(degree), int(leaf_size)))

    def treecode_stats(self):
        """(pairs per mat-vec and right-hand side, far clusters, leaves) of the far-field operator."""
        pairs, far, leaves = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(self._L.bipb_treecode_stats(self._h, ctypes.byref(pairs), ctypes.byref(far), ctypes.byref(leaves)))
        return pairs.value, far.value, leaves.value

    def exact_tensor_residual(self, on=True):
        """Double-float mat-vec of 16 or more right-hand sides on the tensor cores (exact digits) or not."""
        _check(self._L.bipb_exact_tensor_residual(self._h, int(bool(on))))

    def symmetric_pairs(self, on=True):
        """FP64 / double-float mat-vecs: visit every unordered pair once (True) or every ordered pair."""
        _check(self._L.bipb_symmetric_pairs(self._h, int(bool(on))))

    def source(self, b, med=None):
        m = med if med is not None else medium()
        _check(self._L.bipb_source(self._h, ctypes.byref(m), _dp(b)))
        return b

    def reaction(self, u, phi_reac=None, e_sol=None, med=None):
        m = med if med is not None else medium()
        _check(self._L.bipb_reaction(self._h, ctypes.byref(m), _dp(u),
                                     _dp(phi_reac) if phi_reac is not None else None,
                                     _dp(e_sol) if e_sol is not None else None))


def timer_enable(surface, on=True):
    _check(load_library().bipb_timer_enable(surface.handle, int(on)))


def timer_read(surface):
    """{kind: (launches, total_ms)} for every pair-kernel kind."""
    L = load_library()
    out = {}
    for k, name in enumerate(KERNEL_KINDS):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(L.bipb_timer_read(surface.handle, k, ctypes.byref(n), ctypes.byref(ms)))
        out[name] = (n.value, ms.value)
    return out


class BatchSurface(Surface):
    """Several surfaces of uneven size in one handle (bipb_surface_create_batch).

    One system per surface; every pass and every GMRES step covers all of
    them in one launch.  Outputs are lists with one entry per surface.
    """

    def __init__(self, surfaces, stream=None):
        self._L = load_library()
        geo = [(_host(c, (-1, 3)), _host(n, (-1, 3)), _host(a, (-1,))) for c, n, a in surfaces]
        k = len(geo)
        ns = (ctypes.c_int64 * k)(*[g[0].shape[0] for g in geo])
        arr = lambda i: (ctypes.c_void_p * k)(*[g[i].ctypes.data for g in geo])  # noqa: E731
        h = ctypes.c_void_p()
        _check(self._L.bipb_surface_create_batch(k, ns, arr(0), arr(1), arr(2), ctypes.c_void_p(_stream(stream)),
                                                 ctypes.byref(h)))
        self._h = h
        self._geo = geo
        self.sizes = [g[0].shape[0] for g in geo]
        self.n = sum(self.sizes)
        self.nc = 0
        self.n_rhs = 0
        self.ncs = []
        self.n_charges_total = 0

    @property
    def n_systems(self):
        return len(self.sizes)

    @property
    def unknowns(self):
        return 2 * self.n

    def set_charges(self, charges):
        """charges: one (pos (Nc_k, 3), q (Nc_k,)) pair per surface."""
        if len(charges) != self.n_systems:
            raise ValueError("one charge set per surface")
        pos = [_host(p, (-1, 3)) for p, _ in charges]
        q = [_host(v, (-1,)) for _, v in charges]
        k = self.n_systems
        nc = (ctypes.c_int64 * k)(*[v.shape[0] for v in q])
        _check(self._L.bipb_charges_set_batch(self._h, nc, (ctypes.c_void_p * k)(*[p.ctypes.data for p in pos]),
                                              (ctypes.c_void_p * k)(*[v.ctypes.data for v in q])))
        self._charge_version = next(_charge_versions)
        self.ncs = [v.shape[0] for v in q]
        self.n_charges_total = sum(self.ncs)
        self.n_rhs = k

    def _split_elems(self, v):
        return np.split(v, np.cumsum(self.sizes)[:-1])

    def _split_charges(self, v):
        return np.split(v, np.cumsum(self.ncs)[:-1])


STATIC_MAX_N = 32768


def matvec32_static(centroids, normals, areas, u, y, med=None, stream=None):
    """Allocation-free FP32 y = A u (bipb_matvec32_static); every argument a CUDA float64 tensor.

    For callers that cannot allocate device memory: the library's scratch is a
    static device array, so no cudaMalloc happens.  Calls that overlap on the
    GPU share that array and race; serialise them.
    """
    import torch

    m = med if med is not None else medium()
    # sizes first: the kernels trust them and would read or write past the end
    n, rem = divmod(centroids.numel(), 3)
    if rem or normals.numel() != 3 * n or areas.numel() != n or u.numel() != 2 * n or y.numel() != 2 * n:
        raise ValueError(f"matvec32_static: expected centroids and normals of 3n, areas of n, u and y of 2n "
                         f"values; got {centroids.numel()}, {normals.numel()}, {areas.numel()}, {u.numel()}, "
                         f"{y.numel()}")
    tensors = (centroids, normals, areas, u, y)
    if not all(isinstance(t, torch.Tensor) and t.is_cuda for t in tensors):
        raise ValueError("matvec32_static: every argument must be a CUDA tensor")
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in tensors):
        raise ValueError(f"matvec32_static: every tensor must be on the current device cuda:{dev} "
                         "(the scratch array used is that device's)")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ptrs = [_dp(t) for t in tensors]
    _check(load_library().bipb_matvec32_static(n, ptrs[0], ptrs[1], ptrs[2], ctypes.byref(m), ptrs[3], ptrs[4],
                                               ctypes.c_void_p(stream)))
    return y


def launch_count(surface):
    n = ctypes.c_int64()
    _check(load_library().bipb_launch_count(surface.handle, ctypes.byref(n)))
    return n.value


def version():
    return load_library().bipb_version().decode()
