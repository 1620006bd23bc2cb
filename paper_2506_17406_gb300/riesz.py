"""Thin ctypes binding of the C ABI declared in ``include/riesz.h``.

Argument marshalling only: every step of the solver runs in ``libriesz.so``
(host C++ for the reference element and mesh maps, sm_103a kernels for the
rest).  Device arrays are torch CUDA tensors (float64, contiguous); host
arrays are numpy.  If the library is missing, every call raises -- there is
no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

H1, HCURL, HDIV, L2, HCURL2, HDIV2 = 0, 1, 2, 3, 4, 5
# first kind (Eq. (2.5)): CG_p, Ned1_p, RT_p; second kind (Eq. (2.6)): NedTwo_p, BDM_p
SPACES = {"CG": H1, "H1": H1, "N1curl": HCURL, "HCURL": HCURL, "RT": HDIV, "HDIV": HDIV, "DG": L2, "L2": L2,
          "N2curl": HCURL2, "HCURL2": HCURL2, "BDM": HDIV2, "HDIV2": HDIV2}
PREC_FP64, PREC_FP32, PREC_BF16X3 = 0, 1, 2
APPLY_MATRIX_FREE, APPLY_ELEMENT = 0, 1
LOOP_HOST, LOOP_GRAPH = 0, 1
DECOMP_VERTEX_STAR, DECOMP_HT, DECOMP_EDGE_STAR = 0, 1, 2
FORM_ADDITIVE, FORM_HYBRID = 0, 1

KINDS = ["geom", "elem", "diag", "assemble", "cholesky", "to_f32", "apply", "gather", "patch_solve",
         "precond_gather", "dot", "scalar", "update", "load", "apply32", "coarse", "coarse_apply", "ht", "apply_tc"]

ERRORS = {1: "INVALID_ARG", 2: "BAD_MESH", 3: "OOM", 4: "NOT_CONVERGED", 5: "NONFINITE", 6: "CUDA",
          7: "INTERNAL", 8: "NO_DEVICE"}


class RieszError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("riesz error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precond_precision", ctypes.c_int), ("apply_mode", ctypes.c_int), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("nrhs_max", ctypes.c_int), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("apply_precision", ctypes.c_int), ("loop", ctypes.c_int),
                ("autotune", ctypes.c_int), ("coarse", ctypes.c_int), ("dirichlet", ctypes.c_int),
                ("decomposition", ctypes.c_int), ("form", ctypes.c_int), ("coarse_its", ctypes.c_int),
                ("dirichlet_vertices", ctypes.c_void_p), ("replace_digits", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int

_SIGS = {
    "riesz_default_opts": (None, [ctypes.POINTER(Opts)]),
    "riesz_last_error": (ctypes.c_char_p, []),
    "riesz_create": (_I, [_I, _I, _I64, _P, _I64, _P, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "riesz_num_dofs": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "riesz_num_cg_dofs": (_I, [_P, ctypes.POINTER(_I64)]),
    "riesz_ref_info": (_I, [_P, _P]),
    "riesz_dof_map": (_I, [_P, _P]),
    "riesz_patch_count": (_I, [_P, _P]),
    "riesz_patch_map": (_I, [_P, _P, _P]),
    "riesz_ht_gradient_map": (_I, [_P, _P, _P, _P]),
    "riesz_ref_tabulate": (_I, [_I, _I, _I64, _P, _P, _P]),
    "riesz_ref_mixed_tables": (_I, [_I, _I, _P]),
    "riesz_setup_device": (_I, [_P, _P]),
    "riesz_setup": (_I, [_I, _I, _I64, _P, _I64, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(_P)]),
    "riesz_apply": (_I, [_P, _P, _P, _I, _P]),
    "riesz_apply_noalloc": (_I, [_P, _P, _P, _P]),
    "riesz_precond": (_I, [_P, _P, _P, _I, _P]),
    "riesz_solve": (_I, [_P, _P, _P, _I, _P, _P, _P]),
    "riesz_solve_host": (_I, [_P, _P, _P, _I, _P, _P, _P]),
    "riesz_solve_batch": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "riesz_load": (_I, [_P, _P, _P, _P]),
    "riesz_stats": (_I, [_P, _P]),
    "riesz_tuning": (_I, [_P, _P]),
    "riesz_dirichlet_map": (_I, [_P, _P]),
    "riesz_update_geometry": (_I, [_P, _P, _P]),
    "riesz_profile": (_I, [_P, _I]),
    "riesz_profile_read": (_I, [_P, _P, _P]),
    "riesz_destroy": (_I, [_P]),
    "riesz_plan_bytes": (_I, [_P, _P, _P]),
    "riesz_hybrid_weights": (_I, [_P, _P, _I]),
    "riesz_apply_prec": (_I, [_P, _P, _P, _I, _I, _P]),
    "riesz_probe_fp64": (_I, [_I, _P, _P]),
    "riesz_hodge_setup": (_I, [_I, _I, _I64, _P, _I64, _P, ctypes.c_double, ctypes.POINTER(Opts), _P,
                               ctypes.POINTER(_P)]),
    "riesz_hodge_sizes": (_I, [_P, _P, _P, _P]),
    "riesz_hodge_apply": (_I, [_P, _P, _P, _P]),
    "riesz_hodge_precond": (_I, [_P, _P, _P, _P]),
    "riesz_hodge_load": (_I, [_P, _P, _P, _P]),
    "riesz_hodge_update_geometry": (_I, [_P, _P, _P]),
    "riesz_hodge_solve": (_I, [_P, _P, _P, _P, _P, _P]),
    "riesz_hodge_stats": (_I, [_P, _P]),
    "riesz_hodge_destroy": (_I, [_P]),
}


def library_path():
    return _build.LIB


def load_library(build_if_missing=False):
    """Load libriesz.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libriesz.so is not built (%s); run __graft_entry__.build()" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise RieszError(rc, _lib.riesz_last_error().decode())


def default_opts(**kw):
    lib = load_library()
    o = Opts()
    lib.riesz_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    """Address of a numpy array or torch tensor (device or host)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def riesz_ref_tabulate(space, p, pts):
    """Reference basis at points of the reference tetrahedron: (vals, dvals)."""
    lib = load_library()
    space = SPACES.get(space, space)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    ncomp = 1 if space in (H1, L2) else 3
    dcomp = 1 if space in (HDIV, HDIV2, L2) else 3
    nref = {H1: (p + 1) * (p + 2) * (p + 3) // 6, HCURL: p * (p + 2) * (p + 3) // 2,
            HDIV: p * (p + 1) * (p + 3) // 2, L2: p * (p + 1) * (p + 2) // 6,
            HCURL2: (p + 1) * (p + 2) * (p + 3) // 2, HDIV2: (p + 1) * (p + 2) * (p + 3) // 2}[space]
    vals = np.zeros((pts.shape[0], nref, ncomp))
    dvals = np.zeros((pts.shape[0], nref, dcomp))
    _check(lib.riesz_ref_tabulate(space, p, pts.shape[0], _ptr(pts), _ptr(vals), _ptr(dvals)))
    return vals, dvals


def riesz_ref_mixed_tables(k, p):
    """Reference coupling tables [6][n_{k-1}][n_k] of the Hodge-Laplace problem (host)."""
    lib = load_library()
    nref = {0: (p + 1) * (p + 2) * (p + 3) // 6, 1: p * (p + 2) * (p + 3) // 2, 2: p * (p + 1) * (p + 3) // 2,
            3: p * (p + 1) * (p + 2) // 6}
    out = np.zeros((1 if k == 3 else 6, nref[k - 1], nref[k]))
    _check(lib.riesz_ref_mixed_tables(k, p, _ptr(out)))
    return out


def probe_fp64(iters=16384, stream=None):
    """Measured FP64 FMA rate of the current device in TFLOP/s (riesz_probe_fp64)."""
    lib = load_library()
    out = np.zeros(1)
    _check(lib.riesz_probe_fp64(int(iters), _stream(stream), _ptr(out)))
    return float(out[0])


def update_geometry_batch(solvers, verts, stream=None):
    """Device setups of independent systems at once (riesz_update_geometry_batch); verts: device tensors."""
    lib = load_library()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
    vp = (ctypes.c_void_p * n)(*[v.data_ptr() for v in verts])
    _check(lib.riesz_update_geometry_batch(ctypes.cast(hs, _P), n, ctypes.cast(vp, _P), _stream(stream)))


def solve_batch(solvers, bs, xs, nrhs=None, stream=None):
    """Solve independent systems in one graph launch (riesz_solve_batch).

    solvers: list of Riesz handles; bs, xs: matching device tensors [nrhs_i][N_i].
    Returns (iters, relres, status) with iters/relres concatenated over the
    systems' right-hand sides and status per system."""
    lib = load_library()
    n = len(solvers)
    nr = [1] * n if nrhs is None else [int(k) for k in nrhs]
    hs = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    nra = np.asarray(nr, dtype=np.int32)
    iters = np.zeros(sum(nr), dtype=np.int32)
    relres = np.zeros(sum(nr))
    status = np.zeros(n, dtype=np.int32)
    rc = lib.riesz_solve_batch(ctypes.cast(hs, _P), n, ctypes.cast(bp, _P), ctypes.cast(xp, _P), _ptr(nra),
                               _stream(stream), _ptr(iters), _ptr(relres), _ptr(status))
    if rc not in (0, 4, 5):  # per-system convergence failures are reported in status
        _check(rc)
    return iters, relres, status


class Riesz:
    """A solver handle: ``Riesz(space, p, verts, cells, **opts)`` builds the host
    maps; ``setup_device()`` runs the device setup."""

    def __init__(self, space, p, verts, cells, device=True, stream=None, dirichlet_vertices=None, **opts):
        """dirichlet_vertices: optional flags (one per vertex) choosing Gamma_D with dirichlet=1."""
        self.lib = load_library()
        if dirichlet_vertices is not None:
            dv = np.ascontiguousarray(dirichlet_vertices, dtype=np.uint8)
            opts["dirichlet_vertices"] = dv.ctypes.data
        self.space = SPACES.get(space, space)
        self.p = p
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        self.ncells = cells.shape[0]
        self.nverts = verts.shape[0]
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(self.lib.riesz_create(self.space, p, verts.shape[0], _ptr(verts), cells.shape[0], _ptr(cells),
                                     ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h
        n, ni, ncg = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.riesz_num_dofs(self.h, ctypes.byref(n), ctypes.byref(ni)))
        _check(self.lib.riesz_num_cg_dofs(self.h, ctypes.byref(ncg)))
        self.N, self.n_interior, self.n_cg = n.value, ni.value, ncg.value
        info = np.zeros(8, dtype=np.int32)
        _check(self.lib.riesz_ref_info(self.h, _ptr(info)))
        self.nref, self.nint_cell, self.ncomp, self.dcomp = (int(x) for x in info[:4])
        self.per_entity = tuple(int(x) for x in info[4:])
        if device:
            self.setup_device(stream)

    # ----- host queries -----
    def dof_map(self):
        out = np.zeros((self.ncells, self.nref), dtype=np.int32)
        _check(self.lib.riesz_dof_map(self.h, _ptr(out)))
        return out

    def patch_map(self):
        """(offsets, dofs) of the patches: one per vertex (vertex stars) or per edge (edge stars)."""
        cnt = np.zeros(1, dtype=np.int64)
        _check(self.lib.riesz_patch_count(self.h, _ptr(cnt)))
        off = np.zeros(int(cnt[0]) + 1, dtype=np.int64)
        _check(self.lib.riesz_patch_map(self.h, _ptr(off), None))
        dofs = np.zeros(int(off[-1]), dtype=np.int32)
        _check(self.lib.riesz_patch_map(self.h, _ptr(off), _ptr(dofs)))
        return off, dofs

    def ht_gradient_map(self, n_interface):
        """(ptr, idx, sgn): the gradient map of a Hiptmair-Toselli handle as a signed CSR list over the
        Ned1_p interface DOFs (columns: CG_p interface DOFs)."""
        ptr = np.zeros(n_interface + 1, dtype=np.int64)
        _check(self.lib.riesz_ht_gradient_map(self.h, _ptr(ptr), None, None))
        idx = np.zeros(int(ptr[-1]), dtype=np.int32)
        sgn = np.zeros(int(ptr[-1]), dtype=np.float32)
        _check(self.lib.riesz_ht_gradient_map(self.h, _ptr(ptr), _ptr(idx), _ptr(sgn)))
        return ptr, idx, sgn

    def stats(self):
        out = np.zeros(8)
        _check(self.lib.riesz_stats(self.h, _ptr(out)))
        return {"setup_host_ms": out[0], "setup_device_ms": out[1], "device_bytes": out[2],
                "factor_bytes": out[3], "last_iters": int(out[4]), "launches": int(out[5]),
                "chol_flops": out[6], "precond_bytes": out[7]}

    def plan_bytes(self):
        """(bytes, allocations) that setup_device will allocate on the device (host-only)."""
        b = np.zeros(1)
        na = np.zeros(1, dtype=np.int64)
        _check(self.lib.riesz_plan_bytes(self.h, _ptr(b), _ptr(na)))
        return int(b[0]), int(na[0])

    def hybrid_weights(self, rho=None):
        """The hybrid form's weights (rho_1, rho_2, rho_3); with rho given, set them (kept from then on)."""
        out = np.zeros(3) if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        _check(self.lib.riesz_hybrid_weights(self.h, _ptr(out), 0 if rho is None else 1))
        return out

    def dirichlet_map(self):
        """Flags (uint8, [N]) of the DOFs fixed by the Dirichlet condition."""
        out = np.zeros(self.N, dtype=np.uint8)
        _check(self.lib.riesz_dirichlet_map(self.h, _ptr(out)))
        return out

    def tuning(self):
        out = np.zeros(5, dtype=np.int32)
        _check(self.lib.riesz_tuning(self.h, _ptr(out)))
        shape, timed = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.riesz_sweep_shape(self.h, ctypes.byref(shape), ctypes.byref(timed)))
        return {"cholesky_ctas_per_sm": int(out[0]), "candidates_timed": int(out[1]), "coarse_dofs": int(out[2]),
                "cholesky_ctas_per_patch": int(out[3]), "coarse_mode": int(out[4]),
                "sweep_shape": shape.value, "sweep_candidates_timed": timed.value}

    # ----- device calls -----
    def setup_device(self, stream=None):
        _check(self.lib.riesz_setup_device(self.h, _stream(stream)))

    def apply(self, x, y, nrhs=1, stream=None):
        _check(self.lib.riesz_apply(self.h, _ptr(x), _ptr(y), nrhs, _stream(stream)))
        return y

    def apply_prec(self, x, y, prec, nrhs=1, stream=None):
        """y = A x in the inner-product precision prec (PREC_FP64, PREC_FP32, PREC_BF16X3)."""
        _check(self.lib.riesz_apply_prec(self.h, _ptr(x), _ptr(y), nrhs, prec, _stream(stream)))
        return y

    def apply_noalloc(self, x, y, stream=None):
        _check(self.lib.riesz_apply_noalloc(self.h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def precond(self, r, z, nrhs=1, stream=None):
        _check(self.lib.riesz_precond(self.h, _ptr(r), _ptr(z), nrhs, _stream(stream)))
        return z

    def solve(self, b, x, nrhs=1, stream=None, check=True):
        iters = np.zeros(nrhs, dtype=np.int32)
        relres = np.zeros(nrhs)
        rc = self.lib.riesz_solve(self.h, _ptr(b), _ptr(x), nrhs, _stream(stream), _ptr(iters), _ptr(relres))
        if check:
            _check(rc)
        return iters, relres, rc

    def solve_host(self, b, x, nrhs=1, stream=None, check=True):
        iters = np.zeros(nrhs, dtype=np.int32)
        relres = np.zeros(nrhs)
        rc = self.lib.riesz_solve_host(self.h, _ptr(b), _ptr(x), nrhs, _stream(stream), _ptr(iters), _ptr(relres))
        if check:
            _check(rc)
        return iters, relres, rc

    def update_geometry(self, verts_dev, stream=None):
        _check(self.lib.riesz_update_geometry(self.h, _ptr(verts_dev), _stream(stream)))

    def profile(self, enable=True, kinds=None):
        """Turn the per-kernel CUDA-event profiler on (all kinds, or the named ones) or off."""
        mask = 0
        if enable:
            mask = -1 if kinds is None else sum(1 << KINDS.index(k) for k in kinds)
        _check(self.lib.riesz_profile(self.h, mask))

    def profile_read(self):
        ms = np.zeros(len(KINDS))
        cnt = np.zeros(len(KINDS), dtype=np.int64)
        _check(self.lib.riesz_profile_read(self.h, _ptr(ms), _ptr(cnt)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KINDS)}

    def load(self, fcg, b, stream=None):
        _check(self.lib.riesz_load(self.h, _ptr(fcg), _ptr(b), _stream(stream)))
        return b

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.riesz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hodge:
    """The mixed Hodge-Laplace problem of Section 7.2 for k = 1 (CG_p x Ned1_p), k = 2
    (Ned1_p x RT_p) or k = 3 (RT_p x DG_{p-1}): ``Hodge(k, p, verts, cells, gamma, **opts)``
    builds and sets up on the device; block vectors are [sigma (n0) | u (n1)]; the source of
    ``load`` is [3][n_cg] CG_p coefficients (k = 1, 2) or [n_cg] (k = 3)."""

    def __init__(self, k, p, verts, cells, gamma=1.0, stream=None, **opts):
        self.lib = load_library()
        self.k, self.p, self.gamma = k, p, gamma
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(self.lib.riesz_hodge_setup(k, p, verts.shape[0], _ptr(verts), cells.shape[0], _ptr(cells),
                                          float(gamma), ctypes.byref(self.opts), _stream(stream), ctypes.byref(h)))
        self.h = h
        sz = np.zeros(3, dtype=np.int64)
        _check(self.lib.riesz_hodge_sizes(self.h, _ptr(sz[0:1]), _ptr(sz[1:2]), _ptr(sz[2:3])))
        self.n0, self.n1, self.n_cg = (int(x) for x in sz)
        self.N = self.n0 + self.n1

    def apply(self, x, y, stream=None):
        _check(self.lib.riesz_hodge_apply(self.h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def precond(self, r, z, stream=None):
        _check(self.lib.riesz_hodge_precond(self.h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def load(self, fcg, b, stream=None):
        _check(self.lib.riesz_hodge_load(self.h, _ptr(fcg), _ptr(b), _stream(stream)))
        return b

    def update_geometry(self, verts_dev, stream=None):
        _check(self.lib.riesz_hodge_update_geometry(self.h, _ptr(verts_dev), _stream(stream)))

    def solve(self, b, x, stream=None, check=True):
        it = np.zeros(1, dtype=np.int32)
        rr = np.zeros(1)
        rc = self.lib.riesz_hodge_solve(self.h, _ptr(b), _ptr(x), _stream(stream), _ptr(it), _ptr(rr))
        if check:
            _check(rc)
        return int(it[0]), float(rr[0]), rc

    def stats(self):
        out = np.zeros(6)
        _check(self.lib.riesz_hodge_stats(self.h, _ptr(out)))
        return {"launches": int(out[0]), "last_iters": int(out[1]), "last_relres": out[2],
                "last_precond_residual_ratio": out[3], "n0": int(out[4]), "n1": int(out[5])}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.riesz_hodge_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
