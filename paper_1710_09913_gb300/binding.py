"""ctypes binding of the DoGIP C ABI (include/dogip.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libdogip.so``.  Device arrays are torch CUDA tensors (their data
pointers are passed through); host arrays are numpy arrays.  There is no CPU
fallback: if the shared library is missing this module raises at import.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdogip.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, EBREAKDOWN, ETIMEOUT, EUNSUPPORTED = range(8)
PROJECTION, ELLIPTIC = 0, 1
COEF_ELEM_SCALAR, COEF_ELEM_TENSOR = 0, 1
FP64, FP32, TF32 = 0, 1, 2
SCATTER_ATOMIC, SCATTER_COLOUR = 0, 1
SOLVE_FP64, SOLVE_MIXED, SOLVE_MIXED_RELIABLE = 0, 1, 2
FORMS = {"projection": PROJECTION, "elliptic": ELLIPTIC}
PRECS = {"fp64": FP64, "fp32": FP32, "tf32": TF32}
SCATTERS = {"atomic": SCATTER_ATOMIC, "colour": SCATTER_COLOUR, None: -1}
MODES = {"fp64": SOLVE_FP64, "mixed": SOLVE_MIXED, "mixed_reliable": SOLVE_MIXED_RELIABLE}
RECURRENCES = {"standard": 0, "fused_pq": 1, "single_reduction": 2}


class DogipError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dogip error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with paper_1710_09913_gb300.build.build() "
            "(the DoGIP path has no CPU fallback)")
    return C.CDLL(LIB_PATH)


lib = _load()


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_vertices", C.c_int64), ("coords", C.POINTER(C.c_double)),
                ("n_cells", C.c_int64), ("cells", C.POINTER(C.c_int32))]


class Opts(C.Structure):
    _fields_ = [("dirichlet", C.c_int), ("scatter", C.c_int), ("keep_fp32", C.c_int),
                ("device", C.c_int), ("factorized", C.c_int), ("global_w", C.c_int)]


class Info(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("form", C.c_int), ("coef_kind", C.c_int),
                ("dirichlet", C.c_int), ("scatter", C.c_int), ("n_cells", C.c_int64),
                ("n_dofs", C.c_int64), ("n_boundary", C.c_int64), ("v_loc", C.c_int),
                ("w_loc", C.c_int), ("n_sym", C.c_int), ("n_colours", C.c_int),
                ("nnz_b", C.c_int64), ("nnz_pm1_b", C.c_int64), ("bytes_ahat_fp64", C.c_int64),
                ("bytes_ahat_fp32", C.c_int64), ("bytes_conn", C.c_int64),
                ("kernel_launches", C.c_int64), ("n_wglobal", C.c_int64)]


class TuneInfo(C.Structure):
    _fields_ = [("variant", C.c_int * 2), ("block", C.c_int * 2)]


class SolveOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("tol", C.c_double), ("maxiter", C.c_int),
                ("inner_tol", C.c_double), ("inner_maxiter", C.c_int), ("max_outer", C.c_int),
                ("scatter", C.c_int), ("check_every", C.c_int), ("use_x0", C.c_int),
                ("timeout_ms", C.c_double), ("reliable_delta", C.c_double),
                ("inner_prec", C.c_int), ("inner_recurrence", C.c_int),
                ("single_launch", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("outer", C.c_int),
                ("rel_residual", C.c_double), ("seconds", C.c_double)]


_vp = C.c_void_p
_SIGS = {
    "dogip_opts_default": (C.c_int, [C.POINTER(Opts)]),
    "dogip_setup": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                              C.POINTER(Opts), C.POINTER(_vp)]),
    "dogip_destroy": (None, [_vp]),
    "dogip_set_coef": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "dogip_get_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "dogip_ndofs": (C.c_int64, [_vp]),
    "dogip_get_dofmap": (C.c_int, [_vp, _vp]),
    "dogip_get_colouring": (C.c_int, [_vp, _vp, C.POINTER(C.c_int)]),
    "dogip_get_boundary": (C.c_int, [_vp, _vp]),
    "dogip_get_ahat": (C.c_int, [_vp, _vp, _vp]),
    "dogip_get_diag": (C.c_int, [_vp, _vp, _vp]),
    "dogip_get_ahat_global": (C.c_int, [_vp, _vp, _vp]),
    "dogip_mesh_dofmap": (C.c_int, [C.c_int, C.c_int, C.c_int64, _vp, _vp, _vp]),
    "dogip_mesh_boundary": (C.c_int, [C.c_int, C.c_int, C.c_int64, _vp, _vp]),
    "dogip_mesh_colouring": (C.c_int, [C.c_int, C.c_int64, _vp, _vp, _vp]),
    "dogip_mesh_wdofmap": (C.c_int, [C.c_int, C.c_int, C.c_int64, _vp, _vp, _vp, _vp]),
    "dogip_get_wdofmap": (C.c_int, [_vp, _vp, _vp]),
    "dogip_get_tables": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, _vp, _vp]),
    "dogip_apply": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]),
    "dogip_apply_add": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]),
    "dogip_apply_qp": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "dogip_load": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dogip_solve_opts_default": (C.c_int, [C.POINTER(SolveOpts)]),
    "dogip_solve": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(SolveOpts), C.POINTER(SolveInfo),
                              _vp, _vp]),
    "dogip_solve_host": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(SolveOpts),
                                   C.POINTER(SolveInfo), _vp, _vp]),
    "dogip_grad_coef": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "dogip_check": (C.c_int, [_vp, _vp]),
    "dogip_set_coef_inclusions": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_double, C.c_double,
                                            C.c_int, _vp]),
    "dogip_autotune": (C.c_int, [_vp, C.c_int, C.POINTER(TuneInfo), _vp]),
    "dogip_batch_solve": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp),
                                    C.POINTER(SolveOpts), C.POINTER(SolveInfo), _vp]),
    "dogip_residual_norms_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int, _vp, _vp]),
    "dogip_last_error": (C.c_char_p, []),
    "dogip_version": (C.c_int, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(code, allow=()):
    if code != OK and code not in allow:
        raise DogipError(code, lib.dogip_last_error().decode())
    return code


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (checked)."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _hptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def residual_norms_noalloc(b, Ky, r=None, rel=None, stream=None):
    """||b - Ky|| / ||b|| per rhs on the device without any allocation by the
    library (b, Ky: float64 CUDA [n] or [n, R]); returns rel (float64 CUDA [R]).
    The C entry point has no context to check sizes against, so this wrapper
    checks them: Ky (and r) must have b's shape, rel at least R entries, and all
    tensors must live on one GPU; the call runs with that GPU current."""
    import torch
    if b.dim() not in (1, 2):
        raise ValueError("b must be [n] or [n, R]")
    R = 1 if b.dim() == 1 else b.shape[1]
    if tuple(Ky.shape) != tuple(b.shape):
        raise ValueError("Ky must have the shape of b")
    if r is not None and tuple(r.shape) != tuple(b.shape):
        raise ValueError("r must have the shape of b")
    devs = {t.device for t in (b, Ky, r, rel) if t is not None}
    if len(devs) != 1 or not b.is_cuda:
        raise ValueError("b, Ky, r and rel must be CUDA tensors on one device")
    with torch.cuda.device(b.device):
        if rel is None:
            rel = torch.empty(R, dtype=torch.float64, device=b.device)
        if rel.numel() < R:
            raise ValueError("rel must hold at least one entry per right-hand side")
        rp = _dptr(r, torch.float64) if r is not None else None
        _check(lib.dogip_residual_norms_noalloc(_dptr(b, torch.float64), _dptr(Ky, torch.float64),
                                                rp, b.shape[0], R, _dptr(rel, torch.float64),
                                                _stream(stream)))
    return rel


def batch_solve(ctxs, bs, us, *, mode="mixed", tol=1e-8, check_every=None, inner_tol=None,
                max_outer=None, maxiter=None, stream=None, single_launch=None):
    """Solve independent problems together (dogip_batch_solve); returns per-problem
    info dicts.  single_launch applies to the concurrent batch mode's solves."""
    import torch
    n = len(ctxs)
    hs = (_vp * n)(*[c._h.value for c in ctxs])
    bp = (_vp * n)(*[_dptr(x, torch.float64).value for x in bs])
    up = (_vp * n)(*[_dptr(x, torch.float64).value for x in us])
    o = ctxs[0]._solve_opts(mode, tol, maxiter, inner_tol, None, max_outer, None, check_every,
                            False, 0.0, single_launch=single_launch)
    infos = (SolveInfo * n)()
    code = lib.dogip_batch_solve(hs, n, bp, up, C.byref(o), infos, _stream(stream))
    _check(code, allow=(ENOTCONV,))
    return [dict(status=i.status, iterations=i.iterations, outer=i.outer,
                 rel_residual=i.rel_residual, seconds=i.seconds) for i in infos]


def _cells(cells):
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    return cells, cells.shape[1] - 1, cells.shape[0]


def mesh_dofmap(cells, p):
    """(ids [E, V_T] int32, n_dofs): first-appearance numbering (host, no GPU)."""
    cells, d, E = _cells(cells)
    n = C.c_int64()
    _check(lib.dogip_mesh_dofmap(d, int(p), E, cells.ctypes.data_as(_vp), None, C.byref(n)))
    V = len(_multi(d, p))
    ids = np.zeros((E, V), dtype=np.int32)
    _check(lib.dogip_mesh_dofmap(d, int(p), E, cells.ctypes.data_as(_vp), ids.ctypes.data_as(_vp),
                                 C.byref(n)))
    return ids, n.value


def mesh_boundary(cells, p):
    """Dirichlet boundary mask [n_dofs] bool (host, no GPU)."""
    cells, d, E = _cells(cells)
    _, n = mesh_dofmap(cells, p)
    mask = np.zeros(n, dtype=np.uint8)
    _check(lib.dogip_mesh_boundary(d, int(p), E, cells.ctypes.data_as(_vp), mask.ctypes.data_as(_vp)))
    return mask.astype(bool)


def mesh_colouring(cells):
    """(colour [E] int32, n_colours) of the greedy cell colouring (host, no GPU)."""
    cells, d, E = _cells(cells)
    col = np.zeros(E, dtype=np.int32)
    nc = C.c_int()
    _check(lib.dogip_mesh_colouring(d, E, cells.ctypes.data_as(_vp), col.ctypes.data_as(_vp),
                                    C.byref(nc)))
    return col, nc.value


def mesh_wdofmap(cells, p):
    """(W ids [E, W_T], owner flags [E, W_T] bool, n_W) of order 2p (host, no GPU)."""
    cells, d, E = _cells(cells)
    WT = len(_multi(d, 2 * p))
    ids = np.zeros((E, WT), dtype=np.int32)
    own = np.zeros((E, WT), dtype=np.uint8)
    n = C.c_int64()
    _check(lib.dogip_mesh_wdofmap(d, int(p), E, cells.ctypes.data_as(_vp), ids.ctypes.data_as(_vp),
                                  own.ctypes.data_as(_vp), C.byref(n)))
    return ids, own.astype(bool), n.value


def _multi(d, q):
    from math import comb
    return range(comb(q + d, d))


def get_tables(dim, p, form):
    """(B [NB, W, V], w [W]) reference tables as compiled into the kernels."""
    f = FORMS.get(form, form)
    sizes = (C.c_int * 3)()
    _check(lib.dogip_get_tables(dim, p, f, None, None, sizes))
    NB, W, V = sizes
    B = np.zeros((NB, W, V))
    w = np.zeros(W)
    _check(lib.dogip_get_tables(dim, p, f, B.ctypes.data_as(_vp), w.ctypes.data_as(_vp), None))
    return B, w


class Context:
    """A DoGIP operator on one mesh (wraps ``dogip_ctx``)."""

    def __init__(self, coords, cells, p, form, coef, *, dirichlet=None, scatter="atomic",
                 keep_fp32=True, device=None, factorized=False, global_w=False):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        d = coords.shape[1]
        self._h = None
        mesh = Mesh(d, coords.shape[0], _hptr(coords, C.c_double), cells.shape[0],
                    _hptr(cells, C.c_int32))
        o = Opts()
        lib.dogip_opts_default(C.byref(o))
        if dirichlet is not None:
            o.dirichlet = int(bool(dirichlet))
        o.scatter = SCATTERS[scatter]
        o.keep_fp32 = int(keep_fp32)
        if device is not None:
            o.device = int(device)
        o.factorized = int(bool(factorized))
        o.global_w = int(bool(global_w))
        kind = COEF_ELEM_TENSOR if coef.ndim == 3 else COEF_ELEM_SCALAR
        h = C.c_void_p()
        _check(lib.dogip_setup(C.byref(mesh), int(p), FORMS.get(form, form), kind,
                               _hptr(coef, C.c_double), C.byref(o), C.byref(h)))
        self._h = h
        self.info = Info()
        _check(lib.dogip_get_info(h, C.byref(self.info)))
        self.n = self.info.n_dofs
        self.E = self.info.n_cells
        self.d = d
        self.p = p
        self.form = form

    def __del__(self):
        if getattr(self, "_h", None):
            lib.dogip_destroy(self._h)
            self._h = None

    close = __del__

    # ------------------------------------------------------------ queries
    def launches(self):
        """Kernels this context has launched so far (graph nodes included)."""
        _check(lib.dogip_get_info(self._h, C.byref(self.info)))
        return self.info.kernel_launches

    def dofmap(self):
        out = np.zeros((self.E, self.info.v_loc), dtype=np.int32)
        _check(lib.dogip_get_dofmap(self._h, out.ctypes.data_as(_vp)))
        return out

    def colouring(self):
        out = np.zeros(self.E, dtype=np.int32)
        nc = C.c_int()
        _check(lib.dogip_get_colouring(self._h, out.ctypes.data_as(_vp), C.byref(nc)))
        return out, nc.value

    def boundary(self):
        out = np.zeros(self.n, dtype=np.uint8)
        _check(lib.dogip_get_boundary(self._h, out.ctypes.data_as(_vp)))
        return out.astype(bool)

    def ahat(self, stream=None):
        import torch
        out = torch.empty((self.E, self.info.w_loc, self.info.n_sym), dtype=torch.float64,
                          device="cuda")
        _check(lib.dogip_get_ahat(self._h, _dptr(out), _stream(stream)))
        return out

    def ahat_global(self, stream=None):
        """A_diag of the global double grid (global_w contexts): [n_W] float64."""
        import torch
        out = torch.empty(self.info.n_wglobal, dtype=torch.float64, device="cuda")
        _check(lib.dogip_get_ahat_global(self._h, _dptr(out), _stream(stream)))
        return out

    def wdofmap(self):
        """(W-node ids [E, W_T] int32, owner flags [E, W_T] bool) of a global_w context."""
        ids = np.zeros((self.E, self.info.w_loc), dtype=np.int32)
        own = np.zeros((self.E, self.info.w_loc), dtype=np.uint8)
        _check(lib.dogip_get_wdofmap(self._h, ids.ctypes.data_as(_vp), own.ctypes.data_as(_vp)))
        return ids, own.astype(bool)

    def diag(self, stream=None):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib.dogip_get_diag(self._h, _dptr(out), _stream(stream)))
        return out

    # ---------------------------------------------------------- operations
    def set_coef(self, coef, stream=None):
        import torch
        kind = COEF_ELEM_TENSOR if coef.dim() == 3 else COEF_ELEM_SCALAR
        _check(lib.dogip_set_coef(self._h, kind, _dptr(coef, torch.float64), _stream(stream)))
        _check(lib.dogip_get_info(self._h, C.byref(self.info)))

    def set_coef_inclusions(self, centres, radii, inside, outside, nq, stream=None):
        """Element factors of an inclusion field by sub-element quadrature."""
        centres = np.ascontiguousarray(centres, dtype=np.float64)
        radii = np.ascontiguousarray(radii, dtype=np.float64)
        _check(lib.dogip_set_coef_inclusions(self._h, len(radii), centres.ctypes.data_as(_vp),
                                             radii.ctypes.data_as(_vp), float(inside),
                                             float(outside), int(nq), _stream(stream)))
        _check(lib.dogip_get_info(self._h, C.byref(self.info)))

    def apply(self, u, y=None, prec="fp64", scatter=None, stream=None):
        """y = K u for u [n] or [n, R] (float64 for fp64, float32 for fp32 and tf32)."""
        import torch
        pr = PRECS.get(prec, prec)
        dt = torch.float64 if pr == FP64 else torch.float32
        R = 1 if u.dim() == 1 else u.shape[1]
        if u.shape[0] != self.n:
            raise ValueError("u has the wrong number of dofs")
        if y is None:
            y = torch.empty_like(u)
        if tuple(y.shape) != tuple(u.shape):
            raise ValueError("y must have the shape of u")
        _check(lib.dogip_apply(self._h, _dptr(u, dt), _dptr(y, dt), R, pr, SCATTERS[scatter],
                               _stream(stream)))
        return y

    def apply_add(self, u, y, prec="fp64", scatter=None, stream=None):
        """y += K u (dogip_apply_add): one kernel launch, y is not cleared."""
        import torch
        pr = PRECS.get(prec, prec)
        dt = torch.float64 if pr == FP64 else torch.float32
        R = 1 if u.dim() == 1 else u.shape[1]
        if u.shape[0] != self.n or tuple(y.shape) != tuple(u.shape):
            raise ValueError("u and y must both be [n] or [n, R]")
        _check(lib.dogip_apply_add(self._h, _dptr(u, dt), _dptr(y, dt), R, pr, SCATTERS[scatter],
                                   _stream(stream)))
        return y

    def apply_qp(self, u, y=None, prec="fp64", stream=None):
        """Comparator: the quadrature-point matrix-free apply (dogip_apply_qp), same
        result as ``apply`` up to rounding."""
        import torch
        pr = PRECS.get(prec, prec)
        dt = torch.float64 if pr == FP64 else torch.float32
        R = 1 if u.dim() == 1 else u.shape[1]
        if u.shape[0] != self.n:
            raise ValueError("u has the wrong number of dofs")
        if y is None:
            y = torch.empty_like(u)
        _check(lib.dogip_apply_qp(self._h, _dptr(u, dt), _dptr(y, dt), R, pr, _stream(stream)))
        return y

    def load(self, f=None, b=None, stream=None):
        import torch
        if b is None:
            b = torch.empty(self.n, dtype=torch.float64, device="cuda")
        fp = _dptr(f, torch.float64) if f is not None else None
        _check(lib.dogip_load(self._h, fp, _dptr(b, torch.float64), _stream(stream)))
        return b

    def _solve_opts(self, mode, tol, maxiter, inner_tol, inner_maxiter, max_outer, scatter,
                    check_every, x0, timeout_ms, reliable_delta=None, inner_prec=None,
                    inner_recurrence=None, single_launch=None):
        o = SolveOpts()
        lib.dogip_solve_opts_default(C.byref(o))
        o.mode = MODES.get(mode, mode)
        o.tol = tol
        if maxiter is not None:
            o.maxiter = maxiter
        if inner_tol is not None:
            o.inner_tol = inner_tol
        if inner_maxiter is not None:
            o.inner_maxiter = inner_maxiter
        if max_outer is not None:
            o.max_outer = max_outer
        o.scatter = SCATTERS[scatter]
        if check_every is not None:
            o.check_every = check_every
        o.use_x0 = int(x0)
        o.timeout_ms = timeout_ms
        if reliable_delta is not None:
            o.reliable_delta = reliable_delta
        if inner_prec is not None:
            o.inner_prec = PRECS.get(inner_prec, inner_prec)
        if inner_recurrence is not None:
            o.inner_recurrence = RECURRENCES.get(inner_recurrence, inner_recurrence)
        if single_launch is not None:
            o.single_launch = {"auto": -1, False: 0, True: 1}.get(single_launch, single_launch)
        return o

    def solve(self, b, u=None, *, mode="fp64", tol=1e-8, maxiter=None, inner_tol=None,
              inner_maxiter=None, max_outer=None, scatter=None, check_every=None, x0=False,
              timeout_ms=0.0, stream=None, allow_notconv=False, reliable_delta=None,
              inner_prec=None, inner_recurrence=None, single_launch=None):
        """Solve K u = b on the device; returns (u, info dict).  inner_prec ("fp32" or
        "tf32") selects the applies of the mixed modes' inner solves; single_launch
        ("auto", True, False) the one-kernel PCG iterations for problems that fit in L2."""
        import torch
        R = 1 if b.dim() == 1 else b.shape[1]
        if u is None:
            u = torch.zeros_like(b)
        o = self._solve_opts(mode, tol, maxiter, inner_tol, inner_maxiter, max_outer, scatter,
                             check_every, x0, timeout_ms, reliable_delta, inner_prec,
                             inner_recurrence, single_launch)
        inf = SolveInfo()
        rel = np.zeros(R)
        code = lib.dogip_solve(self._h, _dptr(b, torch.float64), _dptr(u, torch.float64), R,
                               C.byref(o), C.byref(inf), rel.ctypes.data_as(_vp), _stream(stream))
        _check(code, allow=(ENOTCONV,) if allow_notconv else ())
        return u, dict(status=inf.status, iterations=inf.iterations, outer=inf.outer,
                       rel_residual=inf.rel_residual, seconds=inf.seconds, rel_per_rhs=rel)

    def solve_host(self, b_host, u_host, *, mode="fp64", tol=1e-8, maxiter=None, inner_tol=None,
                   inner_maxiter=None, max_outer=None, scatter=None, check_every=None,
                   timeout_ms=0.0, stream=None):
        """Solve with host (numpy or pinned torch CPU) b and u; copies inside the call."""
        R = 1 if b_host.ndim == 1 else b_host.shape[1]
        bp = C.c_void_p(b_host.data_ptr() if hasattr(b_host, "data_ptr") else b_host.ctypes.data)
        up = C.c_void_p(u_host.data_ptr() if hasattr(u_host, "data_ptr") else u_host.ctypes.data)
        o = self._solve_opts(mode, tol, maxiter, inner_tol, inner_maxiter, max_outer, scatter,
                             check_every, False, timeout_ms)
        inf = SolveInfo()
        rel = np.zeros(R)
        _check(lib.dogip_solve_host(self._h, bp, up, R, C.byref(o), C.byref(inf),
                                    rel.ctypes.data_as(_vp), _stream(stream)))
        return dict(status=inf.status, iterations=inf.iterations, outer=inf.outer,
                    rel_residual=inf.rel_residual, seconds=inf.seconds)

    def autotune(self, force=False, stream=None):
        """Pick the apply kernel per precision by timing (dogip_autotune); returns
        {precision: (variant, cells per CTA)}."""
        t = TuneInfo()
        _check(lib.dogip_autotune(self._h, int(force), C.byref(t), _stream(stream)))
        return {"fp64": (t.variant[FP64], t.block[FP64]), "fp32": (t.variant[FP32], t.block[FP32])}

    def check(self, stream=None):
        """Synchronise and raise if a kernel-side bounded wait expired."""
        _check(lib.dogip_check(self._h, _stream(stream)))

    def grad_coef(self, u, lam, stream=None):
        import torch
        if self.form == "elliptic" and self.info.coef_kind == COEF_ELEM_TENSOR:
            dA = torch.empty((self.E, self.d, self.d), dtype=torch.float64, device="cuda")
        else:
            dA = torch.empty(self.E, dtype=torch.float64, device="cuda")
        _check(lib.dogip_grad_coef(self._h, _dptr(u, torch.float64), _dptr(lam, torch.float64),
                                   _dptr(dA), _stream(stream)))
        return dA
