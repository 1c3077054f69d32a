"""Thin ctypes binding of libhhg (include/hhg.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors / numpy arrays
into pointers and sizes, checks statuses and raises HHGError with the library's message.  It
fails loudly when the library has not been built (there is no CPU fallback).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhhg.so")

OK = 0
STATUS = {0: "HHG_OK", 1: "HHG_ERR_ARG", 2: "HHG_ERR_MESH", 3: "HHG_ERR_CUDA", 4: "HHG_ERR_OOM",
          5: "HHG_ERR_NOT_CONVERGED", 6: "HHG_ERR_DIVERGED", 7: "HHG_ERR_STATE", 8: "HHG_ERR_TIMEOUT"}


class HHGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class SolveParams(C.Structure):
    _fields_ = [("nu", C.c_int), ("pre", C.c_int), ("post", C.c_int), ("n_extra", C.c_int),
                ("precision", C.c_int), ("storage", C.c_int), ("ir_steps", C.c_int),
                ("ir_vcycles", C.c_int), ("rhs", C.c_int)]


class MeshInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("L", C.c_int), ("n_cells", C.c_int), ("n_verts", C.c_int),
                ("n_nodes", C.c_longlong * 16), ("n_unknowns", C.c_longlong),
                ("n_distinct", C.c_longlong), ("device_bytes", C.c_longlong), ("n_colours", C.c_int)]


class EstimateOut(C.Structure):
    _fields_ = [("eta_j", C.c_double), ("theta", C.c_double), ("err_l", C.c_double),
                ("err_lm1", C.c_double), ("err_Lm1", C.c_double)]


_lib = None


def lib():
    """Load libhhg.so (raises if it has not been built: no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhhg.so not built at %s; run python -m paper_2508_06049_gb300.build" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i, d, u8 = C.c_void_p, C.c_int, C.c_double, C.c_void_p
    sig = {
        "hhg_mesh_create": [i, i, vp, i, vp, vp, i, vp, C.POINTER(vp)],
        "hhg_mesh_destroy": [vp],
        "hhg_mesh_get_info": [vp, C.POINTER(MeshInfo)],
        "hhg_mesh_synchronize": [vp],
        "hhg_level_coords": [vp, i, vp],
        "hhg_set_coefficient": [vp, vp],
        "hhg_set_data": [vp, vp, vp],
        "hhg_fmg_solve": [vp, C.POINTER(SolveParams), vp],
        "hhg_estimate": [vp, i, vp, vp, C.POINTER(EstimateOut)],
        "hhg_estimate_norm": [vp, i, i, vp, vp, vp, C.POINTER(EstimateOut)],
        "hhg_get_vector": [vp, i, i, vp],
        "hhg_apply": [vp, i, i, vp, vp, i],
        "hhg_mark": [i, vp, d, u8, C.POINTER(i)],
        "hhg_rg2d_create": [i, vp, i, vp, C.POINTER(vp)],
        "hhg_rg2d_refine": [vp, u8],
        "hhg_rg2d_mesh": [vp, C.POINTER(i), vp, C.POINTER(i), vp],
        "hhg_rg2d_destroy": [vp],
        "hhg_mark_refine": [vp, vp, d, u8],
        "hhg_rg3d_create": [i, vp, i, vp, C.POINTER(vp)],
        "hhg_rg3d_refine": [vp, u8],
        "hhg_rg3d_mesh": [vp, C.POINTER(i), vp, C.POINTER(i), vp],
        "hhg_rg3d_destroy": [vp],
        "hhg_rg3d_mark_refine": [vp, vp, d, u8],
        "hhg_adjoint_l2": [vp, C.POINTER(SolveParams), u8, C.POINTER(d), vp, vp],
        "hhg_lattice_selfcheck": [i, i],
        "hhg_debug_check": [vp],
        "hhg_profile_kernel": [vp, i, i, i, C.POINTER(C.c_longlong), C.POINTER(d), C.POINTER(d)],
        "hhg_solve_launch_count": [vp, C.POINTER(SolveParams), C.POINTER(C.c_longlong)],
        "hhg_cell_mass_norms_noalloc": [vp, vp, vp, vp],
        "hhg_last_error": [],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name == "hhg_last_error" else C.c_int
    _lib = L
    return L


def _check(status):
    if status != OK:
        raise HHGError(status, lib().hhg_last_error().decode())


def _ptr(x):
    """Raw pointer of a torch tensor (host or device) or a numpy array; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return C.c_void_p(x.ctypes.data)
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(x.data_ptr())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def solve_params(nu=2, pre=2, post=1, n_extra=0, precision=0, storage=1, ir_steps=0, ir_vcycles=2, rhs=0):
    return SolveParams(nu, pre, post, n_extra, precision, storage, ir_steps, ir_vcycles, rhs)


class Mesh:
    """An HHG hierarchy on one GPU (hhg_mesh_create)."""

    def __init__(self, coords, cells, L, dirichlet=None, stream=None):
        coords = _f64(coords)
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
        dim = coords.shape[1]
        flags = None if dirichlet is None else np.ascontiguousarray(np.asarray(dirichlet, dtype=np.uint8))
        h = C.c_void_p()
        st = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(lib().hhg_mesh_create(dim, len(coords), _ptr(coords), len(cells), _ptr(cells),
                                     _ptr(flags), int(L), st, C.byref(h)))
        self._h = h
        self.dim, self.L, self.n_cells = dim, int(L), len(cells)
        self.info = self.get_info()

    def close(self):
        if getattr(self, "_h", None):
            lib().hhg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        """Wait for the work queued on the mesh's stream (hhg_mesh_synchronize)."""
        _check(lib().hhg_mesh_synchronize(self._h))

    def get_info(self):
        info = MeshInfo()
        _check(lib().hhg_mesh_get_info(self._h, C.byref(info)))
        return info

    def n_nodes(self, level):
        return int(self.info.n_nodes[level])

    def level_coords(self, level, out=None):
        if out is None:
            out = np.empty((self.n_nodes(level), self.dim), dtype=np.float64)
        _check(lib().hhg_level_coords(self._h, int(level), _ptr(out)))
        return out

    def set_coefficient(self, k):
        kk = None if k is None else _f64(k)
        _check(lib().hhg_set_coefficient(self._h, _ptr(kk)))

    def set_data(self, f, g):
        _check(lib().hhg_set_data(self._h, _ptr(f), _ptr(g)))

    def solve(self, params=None, out=None, **kw):
        p = params if params is not None else solve_params(**kw)
        if out is None:
            out = np.empty(self.n_nodes(self.L), dtype=np.float64)
        _check(lib().hhg_fmg_solve(self._h, C.byref(p), _ptr(out)))
        return out

    def estimate(self, j=1, want_local=True, norm=0, weights=None):
        """ErrorEstimate of the last solve; norm 0 L2, 1 energy, 2 L2 weighted per cell (weights)."""
        eta = np.empty(self.n_cells) if want_local else None
        etaj = np.empty(self.n_cells) if want_local else None
        out = EstimateOut()
        if norm == 0 and weights is None:
            _check(lib().hhg_estimate(self._h, int(j), _ptr(eta), _ptr(etaj), C.byref(out)))
        else:
            w = None if weights is None else _f64(weights)
            if w is not None and len(w) != self.n_cells:
                raise ValueError("weights must have one entry per macro cell")
            _check(lib().hhg_estimate_norm(self._h, int(j), int(norm), _ptr(w), _ptr(eta), _ptr(etaj),
                                           C.byref(out)))
        return dict(eta_j=out.eta_j, theta=out.theta, err_l=out.err_l, err_lm1=out.err_lm1,
                    err_Lm1=out.err_Lm1, eta_T=eta, eta_jT=etaj)

    def get_vector(self, which, level, out=None):
        n = self.n_nodes(level + 1 if which == 1 else level)
        if out is None:
            out = np.empty(n, dtype=np.float64)
        _check(lib().hhg_get_vector(self._h, int(which), int(level), _ptr(out)))
        return out

    def apply(self, level, op, x, out=None, nsweeps=0):
        if out is None:
            out = np.zeros(self.n_nodes(level), dtype=np.float64)
        _check(lib().hhg_apply(self._h, int(level), int(op), _ptr(x), _ptr(out), int(nsweeps)))
        return out

    def profile_kernel(self, kernel=0, precision=0, reps=1):
        """Enqueue `reps` launches of one solve kernel on the mesh stream (no sync); returns the
        per-launch model (units, algorithmic bytes, flops)."""
        u, b, f = C.c_longlong(), C.c_double(), C.c_double()
        _check(lib().hhg_profile_kernel(self._h, int(kernel), int(precision), int(reps), C.byref(u),
                                         C.byref(b), C.byref(f)))
        return u.value, b.value, f.value

    def cell_mass_norms_noalloc(self, a, b, out):
        """(a-b)^T M_T (a-b) per cell into the device tensor `out` without allocating (queued on the
        mesh stream, not synchronised).  a, b (b may be None): CUDA float64 contiguous tensors of N_L
        entries; out: CUDA float64 contiguous, one entry per macro cell; all on the mesh's device."""
        n = self.n_nodes(self.L)
        dev = None
        for name, t, size in (("a", a, n), ("b", b, n), ("out", out, self.n_cells)):
            if t is None and name == "b":
                continue
            if isinstance(t, np.ndarray) or not getattr(t, "is_cuda", False):
                raise ValueError("%s must be a CUDA tensor" % name)
            if str(t.dtype) != "torch.float64" or not t.is_contiguous() or t.numel() != size:
                raise ValueError("%s must be a contiguous float64 tensor of %d entries" % (name, size))
            if dev is None:
                dev = t.device
            elif t.device != dev:
                raise ValueError("a, b and out must be on the same device")
        _check(lib().hhg_cell_mass_norms_noalloc(self._h, _ptr(a), _ptr(b), _ptr(out)))
        return out

    def launch_count(self, params):
        n = C.c_longlong()
        _check(lib().hhg_solve_launch_count(self._h, C.byref(params), C.byref(n)))
        return n.value

    def adjoint_l2(self, in_S, params=None, grad_f=None, **kw):
        p = params if params is not None else solve_params(**kw)
        mask = np.ascontiguousarray(np.asarray(in_S, dtype=np.uint8))
        if grad_f is None:
            grad_f = np.empty(self.n_nodes(self.L), dtype=np.float64)
        grad_k = np.empty(self.n_cells, dtype=np.float64)
        J = C.c_double()
        _check(lib().hhg_adjoint_l2(self._h, C.byref(p), _ptr(mask), C.byref(J), _ptr(grad_f),
                                     _ptr(grad_k)))
        return J.value, grad_f, grad_k


def mark(eta, fraction):
    eta = _f64(eta)
    marked = np.zeros(len(eta), dtype=np.uint8)
    cnt = C.c_int()
    _check(lib().hhg_mark(len(eta), _ptr(eta), float(fraction), _ptr(marked), C.byref(cnt)))
    return marked.astype(bool)


class RG2D:
    """Host red-green refinement object (hhg_rg2d_*)."""

    def __init__(self, coords, cells):
        co = _f64(coords)
        ce = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
        h = C.c_void_p()
        _check(lib().hhg_rg2d_create(len(co), _ptr(co), len(ce), _ptr(ce), C.byref(h)))
        self._h = h

    def __del__(self):
        try:
            if self._h:
                lib().hhg_rg2d_destroy(self._h)
        except Exception:
            pass

    def mesh(self):
        nv, nc = C.c_int(), C.c_int()
        _check(lib().hhg_rg2d_mesh(self._h, C.byref(nv), None, C.byref(nc), None))
        co = np.empty((nv.value, 2), dtype=np.float64)
        ce = np.empty((nc.value, 3), dtype=np.int32)
        _check(lib().hhg_rg2d_mesh(self._h, C.byref(nv), _ptr(co), C.byref(nc), _ptr(ce)))
        return co, ce

    def refine(self, marked):
        m = np.ascontiguousarray(np.asarray(marked, dtype=np.uint8))
        _check(lib().hhg_rg2d_refine(self._h, _ptr(m)))

    def mark_refine(self, eta, fraction):
        eta = _f64(eta)
        marked = np.zeros(len(eta), dtype=np.uint8)
        _check(lib().hhg_mark_refine(self._h, _ptr(eta), float(fraction), _ptr(marked)))
        return marked.astype(bool)


class RG3D:
    """Host 3D red-green refinement object (hhg_rg3d_*)."""

    def __init__(self, coords, cells):
        co = _f64(coords)
        ce = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
        h = C.c_void_p()
        _check(lib().hhg_rg3d_create(len(co), _ptr(co), len(ce), _ptr(ce), C.byref(h)))
        self._h = h

    def __del__(self):
        try:
            if self._h:
                lib().hhg_rg3d_destroy(self._h)
        except Exception:
            pass

    def mesh(self):
        nv, nc = C.c_int(), C.c_int()
        _check(lib().hhg_rg3d_mesh(self._h, C.byref(nv), None, C.byref(nc), None))
        co = np.empty((nv.value, 3), dtype=np.float64)
        ce = np.empty((nc.value, 4), dtype=np.int32)
        _check(lib().hhg_rg3d_mesh(self._h, C.byref(nv), _ptr(co), C.byref(nc), _ptr(ce)))
        return co, ce

    def refine(self, marked):
        m = np.ascontiguousarray(np.asarray(marked, dtype=np.uint8))
        _check(lib().hhg_rg3d_refine(self._h, _ptr(m)))

    def mark_refine(self, eta, fraction):
        eta = _f64(eta)
        marked = np.zeros(len(eta), dtype=np.uint8)
        _check(lib().hhg_rg3d_mark_refine(self._h, _ptr(eta), float(fraction), _ptr(marked)))
        return marked.astype(bool)


def debug_check():
    out = np.zeros(8, dtype=np.int64)
    _check(lib().hhg_debug_check(_ptr(out)))
    return out


def lattice_selfcheck(dim, n):
    return lib().hhg_lattice_selfcheck(int(dim), int(n))
