"""Thin ctypes binding over libgw.so, the C ABI declared in include/gw.h.

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
their data pointers are handed to the library, which stages host arrays to
the device itself.  There is no CPU fallback: if the library is missing or
cannot be loaded, every call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgw.so")

GW_OK, GW_ERR_ARG, GW_ERR_CUDA, GW_ERR_OOM, GW_ERR_SETUP, GW_ERR_NOT_CONVERGED, GW_ERR_BREAKDOWN = range(7)
GW_NOFLOW, GW_DIRICHLET = 0, 1
GW_PREC_FP64, GW_PREC_MIXED32, GW_PREC_MIXED16, GW_PREC_MIXEDBF16 = 0, 1, 2, 3
GW_SMOOTH_JACOBI, GW_SMOOTH_CHEBYSHEV = 0, 1
GW_HALF_FINE, GW_HALF_FINE16 = 2, 4

EXPORTS = ("gw_amg_opts_default", "gw_assemble", "gw_matrix_size", "gw_matrix_export", "gw_amg_setup",
           "gw_pcg_solve", "gw_vcycle", "gw_hierarchy_info", "gw_hierarchy_export", "gw_matrix_free",
           "gw_hierarchy_free", "gw_status_str", "gw_last_error", "gw_profile_enable", "gw_profile_read",
           "gw_assemble_noalloc", "gw_adjoint_gradient", "gw_misfit", "gw_hierarchy_shift",
           "gw_pcg_solve_many", "gw_darcy_flux", "gw_hierarchy_prepare", "gw_device_allocations",
           "gw_batch_create", "gw_batch_add", "gw_batch_run", "gw_batch_state", "gw_batch_take", "gw_batch_free")

PK_NAMES = ("spmv", "update", "pre1", "pre2", "resid", "restrict", "l1down", "deep", "l1up", "prolong", "post1",
            "post2", "pupdate")


class gw_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class gw_bc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int * 6), ("value", ctypes.c_double * 6)]


class gw_amg_opts(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("smoother", ctypes.c_int), ("degree", ctypes.c_int),
                ("nu", ctypes.c_int), ("n_coarse", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int), ("delta", ctypes.c_double),
                ("half_storage", ctypes.c_int), ("mis_max_rounds", ctypes.c_int)]


class gw_level_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_longlong), ("nnz_p", ctypes.c_longlong),
                ("bytes", ctypes.c_longlong), ("naggregates", ctypes.c_int), ("mis_rounds", ctypes.c_int),
                ("omega_p", ctypes.c_double), ("jacobi_w", ctypes.c_double), ("lambda_max", ctypes.c_double)]


class gw_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 13), ("launches", ctypes.c_longlong * 13), ("bytes", ctypes.c_double * 13),
                ("kernel_launches", ctypes.c_longlong), ("solves", ctypes.c_longlong)]


class GwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_status_name(status), msg))
        self.status = status


_lib = None


def load():
    """Loads libgw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgw.so is not built (run paper_2001_05798_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    P = ctypes.POINTER
    sig = {
        "gw_amg_opts_default": (None, [P(gw_amg_opts)]),
        "gw_assemble": (i, [P(gw_grid), vp, vp, vp, P(gw_bc), vp, P(vp), vp, vp]),
        "gw_matrix_size": (i, [vp, P(i), P(ll)]),
        "gw_matrix_export": (i, [vp, vp, vp, vp, vp]),
        "gw_amg_setup": (i, [vp, P(gw_amg_opts), P(vp), vp]),
        "gw_pcg_solve": (i, [vp, vp, vp, d, i, P(i), P(d), vp]),
        "gw_vcycle": (i, [vp, vp, vp, vp]),
        "gw_hierarchy_info": (i, [vp, P(gw_level_info), i, P(i)]),
        "gw_hierarchy_export": (i, [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "gw_matrix_free": (None, [vp]),
        "gw_hierarchy_free": (None, [vp]),
        "gw_status_str": (ctypes.c_char_p, [i]),
        "gw_last_error": (ctypes.c_char_p, []),
        "gw_profile_enable": (i, [vp, i]),
        "gw_profile_read": (i, [vp, P(gw_profile), i]),
        "gw_assemble_noalloc": (i, [P(gw_grid), vp, vp, vp, P(gw_bc), vp, vp, vp, vp, vp, vp]),
        "gw_adjoint_gradient": (i, [P(gw_grid), vp, vp, vp, P(gw_bc), vp, vp, vp, vp]),
        "gw_misfit": (i, [i, vp, i, vp, vp, vp, vp, vp]),
        "gw_hierarchy_shift": (i, [vp, vp, d, P(i), vp]),
        "gw_pcg_solve_many": (i, [vp, i, vp, vp, d, i, vp, vp, vp]),
        "gw_hierarchy_prepare": (i, [vp]),
        "gw_darcy_flux": (i, [P(gw_grid), vp, vp, vp, P(gw_bc), vp, vp, vp, vp, vp]),
        "gw_device_allocations": (ll, []),
        "gw_batch_create": (i, [i, P(vp)]),
        "gw_batch_add": (i, [vp, vp, vp, d, i, P(i)]),
        "gw_batch_run": (i, [vp, i, P(i)]),
        "gw_batch_state": (i, [vp, i, P(i)]),
        "gw_batch_take": (i, [vp, i, vp, P(i), P(d)]),
        "gw_batch_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _status_name(s):
    try:
        return load().gw_status_str(s).decode()
    except Exception:
        return "status %d" % s


def _check(status):
    if status != GW_OK:
        raise GwError(status, load().gw_last_error().decode())
    return status


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (None for None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or a numpy array")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def gw_device_allocations():
    """Device allocations the library has made in this process so far."""
    return int(load().gw_device_allocations())


def amg_opts(**kw):
    o = gw_amg_opts()
    load().gw_amg_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Matrix:
    """Assembled FP64 matrix handle (CSR on the device)."""

    def __init__(self, handle):
        self.h = handle
        n, nnz = ctypes.c_int(), ctypes.c_longlong()
        _check(load().gw_matrix_size(self.h, ctypes.byref(n), ctypes.byref(nnz)))
        self.n, self.nnz = n.value, nnz.value

    def export(self, stream=None):
        rp = np.empty(self.n + 1, np.int32)
        ci = np.empty(self.nnz, np.int32)
        v = np.empty(self.nnz, np.float64)
        _check(load().gw_matrix_export(self.h, _ptr(rp), _ptr(ci), _ptr(v), _stream(stream)))
        return rp, ci, v

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gw_matrix_free(self.h)
            self.h = None


def gw_assemble(nx, ny, nz, Kx, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0), q=None,
                b_out=None, spacing=(1.0, 1.0, 1.0), stream=None):
    """Assembles C h = Q (include/gw.h: gw_assemble).  Returns (Matrix, b_out)."""
    L = load()
    g = gw_grid(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]))
    bc = gw_bc()
    for f in range(6):
        bc.type[f] = int(bct[f])
        bc.value[f] = float(bcv[f])
    if b_out is None:
        b_out = np.empty(nx * ny * nz, np.float64)
    h = ctypes.c_void_p()
    _check(L.gw_assemble(ctypes.byref(g), _ptr(Kx), _ptr(Ky if Ky is not None else Kx),
                         _ptr(Kz if Kz is not None else Kx), ctypes.byref(bc), _ptr(q), ctypes.byref(h),
                         _ptr(b_out), _stream(stream)))
    return Matrix(h), b_out


def gw_assemble_noalloc(nx, ny, nz, Kx, rowptr, col, val, b, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0),
                        bcv=(1.0, 0.0, 0, 0, 0, 0), q=None, spacing=(1.0, 1.0, 1.0), stream=None):
    """Assembly into caller-provided device arrays (include/gw.h: gw_assemble_noalloc)."""
    g = gw_grid(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]))
    bc = gw_bc()
    for f in range(6):
        bc.type[f] = int(bct[f])
        bc.value[f] = float(bcv[f])
    _check(load().gw_assemble_noalloc(ctypes.byref(g), _ptr(Kx), _ptr(Ky), _ptr(Kz), ctypes.byref(bc), _ptr(q),
                                      _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _stream(stream)))


def _grid_bc(nx, ny, nz, bct, bcv, spacing):
    g = gw_grid(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]))
    bc = gw_bc()
    for f in range(6):
        bc.type[f] = int(bct[f])
        bc.value[f] = float(bcv[f])
    return g, bc


def gw_adjoint_gradient(nx, ny, nz, Kx, h, lam, grad, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0),
                        bcv=(1.0, 0.0, 0, 0, 0, 0), spacing=(1.0, 1.0, 1.0), stream=None):
    """dJ/dlnK from heads and adjoint state (include/gw.h: gw_adjoint_gradient); device arrays."""
    g, bc = _grid_bc(nx, ny, nz, bct, bcv, spacing)
    _check(load().gw_adjoint_gradient(ctypes.byref(g), _ptr(Kx), _ptr(Ky), _ptr(Kz), ctypes.byref(bc), _ptr(h),
                                      _ptr(lam), _ptr(grad), _stream(stream)))
    return grad


def gw_misfit(h, obs, hobs, dJdh=None, stream=None):
    """J = sum (h[obs] - hobs)^2 and optionally dJ/dh (include/gw.h: gw_misfit)."""
    J = ctypes.c_double()
    _check(load().gw_misfit(int(h.numel() if hasattr(h, "numel") else h.size), _ptr(h), len(obs), _ptr(obs),
                            _ptr(hobs), ctypes.byref(J), _ptr(dJdh), _stream(stream)))
    return J.value


def gw_darcy_flux(nx, ny, nz, Kx, h, vx, vy, vz, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0),
                  bcv=(1.0, 0.0, 0, 0, 0, 0), spacing=(1.0, 1.0, 1.0), stream=None):
    """Darcy velocities on the staggered faces (include/gw.h: gw_darcy_flux); device arrays."""
    g, bc = _grid_bc(nx, ny, nz, bct, bcv, spacing)
    _check(load().gw_darcy_flux(ctypes.byref(g), _ptr(Kx), _ptr(Ky), _ptr(Kz), ctypes.byref(bc), _ptr(h), _ptr(vx),
                                _ptr(vy), _ptr(vz), _stream(stream)))
    return vx, vy, vz


class Hierarchy:
    """AMG hierarchy handle (include/gw.h: gw_amg_setup); keeps its matrix alive."""

    def __init__(self, A, stream=None, **opts):
        self.A = A
        self.opts = amg_opts(**opts)
        h = ctypes.c_void_p()
        _check(load().gw_amg_setup(A.h, ctypes.byref(self.opts), ctypes.byref(h), _stream(stream)))
        self.h = h

    def info(self):
        L = load()
        n = ctypes.c_int()
        _check(L.gw_hierarchy_info(self.h, None, 0, ctypes.byref(n)))
        arr = (gw_level_info * n.value)()
        _check(L.gw_hierarchy_info(self.h, arr, n.value, ctypes.byref(n)))
        return [{k: getattr(arr[l], k) for k, _ in gw_level_info._fields_} for l in range(n.value)]

    def export_level(self, level, stream=None):
        """(agg, root, (A rowptr, col, val), (P rowptr, col, val) or None) of one level."""
        inf = self.info()
        li = inf[level]
        n = li["n"]
        agg = np.empty(n, np.int32)
        root = np.empty(n, np.uint8)
        arp, aci, av = np.empty(n + 1, np.int32), np.empty(li["nnz"], np.int32), np.empty(li["nnz"], np.float64)
        last = level == len(inf) - 1
        if not last:
            prp, pci, pv = (np.empty(n + 1, np.int32), np.empty(li["nnz_p"], np.int32),
                            np.empty(li["nnz_p"], np.float64))
        else:
            prp = pci = pv = None
        _check(load().gw_hierarchy_export(self.h, level, _ptr(agg), _ptr(root), _ptr(arp), _ptr(aci), _ptr(av),
                                          _ptr(prp), _ptr(pci), _ptr(pv), _stream(stream)))
        return agg, root, (arp, aci, av), (None if last else (prp, pci, pv))

    def solve(self, b, h=None, tol=1e-8, maxit=500, stream=None, check=True):
        """gw_pcg_solve: returns (h, iters, relres, status)."""
        if h is None:
            h = np.empty_like(b) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
        it, rel = ctypes.c_int(), ctypes.c_double()
        st = load().gw_pcg_solve(self.h, _ptr(b), _ptr(h), float(tol), int(maxit), ctypes.byref(it),
                                 ctypes.byref(rel), _stream(stream))
        if check and st not in (GW_OK, GW_ERR_NOT_CONVERGED):
            _check(st)
        return h, it.value, rel.value, st

    def prepare(self):
        """Capture the solver's CUDA graphs now (include/gw.h: gw_hierarchy_prepare)."""
        _check(load().gw_hierarchy_prepare(self.h))

    def solve_many(self, B, X=None, tol=1e-8, maxit=500, stream=None):
        """k right-hand sides (columns of the n x k column-major B, i.e. rows of a (k, n) array)."""
        k = B.shape[0]
        if X is None:
            X = np.empty_like(B) if isinstance(B, np.ndarray) else B.new_empty(B.shape)
        its = (ctypes.c_int * k)()
        rels = (ctypes.c_double * k)()
        st = load().gw_pcg_solve_many(self.h, k, _ptr(B), _ptr(X), float(tol), int(maxit), its, rels,
                                      _stream(stream))
        if st not in (GW_OK, GW_ERR_NOT_CONVERGED):
            _check(st)
        return X, list(its), list(rels), st

    def shift(self, s, delta=0.01, stream=None):
        """Solve (C + diag(s)) from now on; returns 0 (hierarchy kept, level 0
        refreshed), 2 (coarse operators formed again) or 1 (rebuilt)."""
        rb = ctypes.c_int()
        _check(load().gw_hierarchy_shift(self.h, _ptr(s), float(delta), ctypes.byref(rb), _stream(stream)))
        return rb.value

    def profile(self, on=True):
        _check(load().gw_profile_enable(self.h, int(bool(on))))

    def profile_read(self, reset=True):
        """Per-kind level-0 kernel timing: {name: (ms_total, launches, bytes_per_launch)}, launches, solves."""
        p = gw_profile()
        _check(load().gw_profile_read(self.h, ctypes.byref(p), int(bool(reset))))
        kinds = {PK_NAMES[k]: (p.ms[k], p.launches[k], p.bytes[k]) for k in range(len(PK_NAMES))}
        return kinds, p.kernel_launches, p.solves

    def vcycle(self, r, z, stream=None):
        _check(load().gw_vcycle(self.h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gw_hierarchy_free(self.h)
            self.h = None


def solve(nx, ny, nz, Kx, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0), q=None,
          tol=1e-8, maxit=500, **opts):
    """Assemble, set up and solve in one call; returns (h, iters, relres)."""
    A, b = gw_assemble(nx, ny, nz, Kx, Ky, Kz, bct, bcv, q)
    H = Hierarchy(A, **opts)
    h, it, rel, st = H.solve(b, tol=tol, maxit=maxit)
    _check(st)
    return h, it, rel


class Batch:
    """Batched solves on resident hierarchies (include/gw.h: gw_batch_*).

    add() starts a solve in a free slot, run() replays the batched iteration
    graph, take() returns a finished solve's heads.  Hierarchies added are
    kept alive by the batch until their solve is taken."""

    def __init__(self, max_slots=8):
        h = ctypes.c_void_p()
        _check(load().gw_batch_create(int(max_slots), ctypes.byref(h)))
        self.h = h
        self.max_slots = max_slots
        self.held = {}

    def add(self, H, b, tol=1e-8, maxit=500):
        s = ctypes.c_int()
        _check(load().gw_batch_add(self.h, H.h, _ptr(b), float(tol), int(maxit), ctypes.byref(s)))
        self.held[s.value] = H
        return s.value

    def run(self, iterations=1):
        f = ctypes.c_int()
        _check(load().gw_batch_run(self.h, int(iterations), ctypes.byref(f)))
        return f.value

    def state(self, slot):
        st = ctypes.c_int()
        _check(load().gw_batch_state(self.h, int(slot), ctypes.byref(st)))
        return st.value

    def finished(self):
        return [s for s in list(self.held) if self.state(s) == 2]

    def take(self, slot, h=None):
        """Returns (h, iters, relres, status) of the finished solve in slot
        (h: a device or host array of n doubles)."""
        if self.state(slot) != 2:
            raise GwError(GW_ERR_ARG, "slot %d holds no finished solve" % slot)
        it, rel = ctypes.c_int(), ctypes.c_double()
        st = load().gw_batch_take(self.h, int(slot), _ptr(h), ctypes.byref(it), ctypes.byref(rel))
        self.held.pop(slot, None)
        if st not in (GW_OK, GW_ERR_NOT_CONVERGED):
            _check(st)
        return h, it.value, rel.value, st

    def close(self):
        if getattr(self, "h", None):
            load().gw_batch_free(self.h)
            self.h = None
        self.held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

