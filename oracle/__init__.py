"""FP64 CPU oracle for the AMG-PCG groundwater flow solve -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library and its binding) never imports, links or runs it, and shares no code
with it: ``gw_oracle.c`` is written separately from the same definitions.

Each wrapper below names the part of the paper (Sbai & Larabi) it follows; the
C source states the arithmetic order of every sum.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gw.so")
_lib = None

OK, ERR_ARG, ERR_SETUP, ERR_NOT_CONVERGED, ERR_BREAKDOWN = 0, 1, 4, 5, 6
NOFLOW, DIRICHLET = 0, 1

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p


def build(force=False):
    """Compile the oracle with gcc (FP contraction off, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    sig = {
        "or_csr_free": (None, [_vp]),
        "or_csr_info": (None, [_vp] + [ctypes.POINTER(ctypes.c_int)] * 3),
        "or_csr_copy": (None, [_vp, _vp, _vp, _vp]),
        "or_csr_from": (_vp, [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _f64p]),
        "or_spmv": (None, [_vp, _f64p, _f64p]),
        "or_nnz7": (ctypes.c_longlong, [ctypes.c_int] * 3),
        "or_assemble": (_vp, [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_f64p] * 3 +
                        [_i32p, _f64p, _vp, _f64p, ctypes.POINTER(ctypes.c_int)]),
        "or_strength": (None, [_vp, ctypes.c_double, _u8p]),
        "or_key": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int]),
        "or_mis2": (None, [_vp, _u8p, ctypes.c_uint64, ctypes.c_int, _u8p]),
        "or_aggregate": (ctypes.c_int, [_vp, _u8p, _u8p, ctypes.c_uint64, ctypes.c_int, _i32p]),
        "or_smooth_p": (_vp, [_vp, _u8p, _i32p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double)]),
        "or_transpose": (_vp, [_vp]),
        "or_spgemm": (_vp, [_vp, _vp]),
        "or_lu_factor": (ctypes.c_int, [ctypes.c_int, _f64p, _i32p]),
        "or_lu_solve": (None, [ctypes.c_int, _f64p, _i32p, _f64p, _f64p]),
        "or_setup": (_vp, [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
        "or_h_status": (ctypes.c_int, [_vp]),
        "or_h_nlevels": (ctypes.c_int, [_vp]),
        "or_h_A": (_vp, [_vp, ctypes.c_int]),
        "or_h_P": (_vp, [_vp, ctypes.c_int]),
        "or_h_R": (_vp, [_vp, ctypes.c_int]),
        "or_h_nagg": (ctypes.c_int, [_vp, ctypes.c_int]),
        "or_h_copy_level": (None, [_vp, ctypes.c_int, _vp, _vp, _vp]),
        "or_h_scalars": (None, [_vp, ctypes.c_int, _f64p]),
        "or_h_free": (None, [_vp]),
        "or_vcycle": (None, [_vp, _f64p, _f64p]),
        "or_h_smooth": (None, [_vp, ctypes.c_int, _f64p, _f64p, ctypes.c_int]),
        "or_pcg": (ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "or_adjoint_grad": (None, [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_f64p] * 3 +
                            [_i32p, _f64p, _f64p, _f64p, _f64p]),
        "or_misfit": (ctypes.c_double, [ctypes.c_int, _f64p, ctypes.c_int, _i32p, _f64p, _vp]),
        "or_shift_csr": (_vp, [_vp, _f64p]),
        "or_reuse_ok": (ctypes.c_int, [_vp, _f64p, _vp, ctypes.c_double]),
        "or_h_refresh_level0": (None, [_vp, _vp]),
        "or_h_refresh_numeric": (None, [_vp, _vp]),
        "or_darcy_flux": (None, [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_f64p] * 3 +
                          [_i32p, _f64p, _f64p, _f64p, _f64p, _f64p]),
        "or_cg_plain": (ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class CSR:
    """Owned (or borrowed) handle to an oracle CSR matrix."""

    def __init__(self, h, owned=True):
        self.h = h
        self.owned = owned
        nr, nc, nnz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _load().or_csr_info(h, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz))
        self.nr, self.nc, self.nnz = nr.value, nc.value, nnz.value
        self._arrays = None

    @classmethod
    def from_arrays(cls, rp, ci, v, nc=None):
        rp = np.ascontiguousarray(rp, dtype=np.int32)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.float64)
        nr = len(rp) - 1
        return cls(_load().or_csr_from(nr, nr if nc is None else nc, rp, ci, v))

    def arrays(self):
        """(rowptr int32, col int32, val float64) copies."""
        if self._arrays is None:
            rp = np.empty(self.nr + 1, np.int32)
            ci = np.empty(self.nnz, np.int32)
            v = np.empty(self.nnz, np.float64)
            _load().or_csr_copy(self.h, _ptr(rp), _ptr(ci), _ptr(v))
            self._arrays = (rp, ci, v)
        return self._arrays

    def dense(self):
        rp, ci, v = self.arrays()
        D = np.zeros((self.nr, self.nc))
        rows = np.repeat(np.arange(self.nr), np.diff(rp))
        D[rows, ci] = v
        return D

    def matvec(self, x):
        y = np.empty(self.nr)
        _load().or_spmv(self.h, np.ascontiguousarray(x, dtype=np.float64), y)
        return y

    def __del__(self):
        if self.owned and self.h and _lib is not None:
            _lib.or_csr_free(self.h)
            self.h = None


def nnz7(nx, ny, nz):
    """Structural nonzeros of the 7-point operator: 7n - 2(ny nz + nx nz + nx ny)."""
    return int(_load().or_nnz7(nx, ny, nz))


def assemble(nx, ny, nz, Kx, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0),
             q=None, spacing=(1.0, 1.0, 1.0)):
    """Cell-centred 5/7-point FV assembly of C h = Q (M-matrix, Benchmarking Examples;
    Eq. 2 with S = 0).  Returns (CSR A, b) or raises ValueError on a bad input."""
    L = _load()
    Kx = np.ascontiguousarray(Kx, dtype=np.float64).ravel()
    Ky = Kx if Ky is None else np.ascontiguousarray(Ky, dtype=np.float64).ravel()
    Kz = Kx if Kz is None else np.ascontiguousarray(Kz, dtype=np.float64).ravel()
    n = nx * ny * nz
    if Kx.size != n or Ky.size != n or Kz.size != n:
        raise ValueError("K has the wrong size")
    qq = None if q is None else np.ascontiguousarray(q, dtype=np.float64).ravel()
    b = np.empty(n)
    st = ctypes.c_int()
    h = L.or_assemble(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]),
                      Kx, Ky, Kz, np.asarray(bct, np.int32), np.asarray(bcv, np.float64),
                      _ptr(qq), b, ctypes.byref(st))
    if st.value != 0 or not h:
        raise ValueError("oracle assembly rejected the input (status %d)" % st.value)
    return CSR(h), b


def strength(A, theta2):
    S = np.empty(A.nnz, np.uint8)
    _load().or_strength(A.h, float(theta2), S)
    return S


def key(seed, level, i):
    return int(_load().or_key(seed, level, i))


def mis2(A, S, seed, level):
    root = np.empty(A.nr, np.uint8)
    _load().or_mis2(A.h, np.ascontiguousarray(S, np.uint8), seed, level, root)
    return root


def aggregate(A, S, root, seed, level):
    agg = np.empty(A.nr, np.int32)
    m = _load().or_aggregate(A.h, np.ascontiguousarray(S, np.uint8), np.ascontiguousarray(root, np.uint8),
                             seed, level, agg)
    return agg, m


def smooth_p(A, S, agg, nagg):
    om, rho = ctypes.c_double(), ctypes.c_double()
    h = _load().or_smooth_p(A.h, np.ascontiguousarray(S, np.uint8), np.ascontiguousarray(agg, np.int32),
                            int(nagg), ctypes.byref(om), ctypes.byref(rho))
    return CSR(h), om.value, rho.value


def transpose(P):
    return CSR(_load().or_transpose(P.h))


def spgemm(Lm, Rm):
    return CSR(_load().or_spgemm(Lm.h, Rm.h))


def lu_factor(M):
    a = np.ascontiguousarray(M, dtype=np.float64).copy()
    piv = np.empty(a.shape[0], np.int32)
    if _load().or_lu_factor(a.shape[0], a, piv) != 0:
        raise np.linalg.LinAlgError("singular")
    return a, piv


def lu_solve(lu, piv, b):
    x = np.empty(lu.shape[0])
    _load().or_lu_solve(lu.shape[0], lu, piv, np.ascontiguousarray(b, np.float64), x)
    return x


class Hierarchy:
    """Smoothed-aggregation hierarchy built by the oracle (AMG setup phase)."""

    def __init__(self, A, theta=0.04, smoother=1, degree=2, nu=1, n_coarse=1024, max_levels=12,
                 seed=0x5EED):
        L = _load()
        self.h = L.or_setup(A.h, float(theta), int(smoother), int(degree), int(nu), int(n_coarse),
                            int(max_levels), int(seed))
        self.status = L.or_h_status(self.h)
        self.nlevels = L.or_h_nlevels(self.h)

    def A(self, l):
        return CSR(_load().or_h_A(self.h, l), owned=False)

    def P(self, l):
        return CSR(_load().or_h_P(self.h, l), owned=False)

    def R(self, l):
        return CSR(_load().or_h_R(self.h, l), owned=False)

    def nagg(self, l):
        return int(_load().or_h_nagg(self.h, l))

    def level(self, l):
        """(agg int32, root uint8, S uint8) of level l (l < nlevels-1)."""
        A = self.A(l)
        agg = np.empty(A.nr, np.int32)
        root = np.empty(A.nr, np.uint8)
        S = np.empty(A.nnz, np.uint8)
        _load().or_h_copy_level(self.h, l, _ptr(agg), _ptr(root), _ptr(S))
        return agg, root, S

    def scalars(self, l):
        out = np.empty(6)
        _load().or_h_scalars(self.h, l, out)
        return dict(theta2=out[0], omegaP=out[1], rhoP=out[2], jacobi_w=out[3], rhoJ=out[4], lam=out[5])

    def refresh_level0(self, A):
        """Keep the coarse levels; level 0 becomes A (with its smoother data redone)."""
        _load().or_h_refresh_level0(self.h, A.h)
        self._A0 = A

    def refresh_numeric(self, A):
        """Keep the aggregates and prolongators; level 0 becomes A and every
        coarse operator is formed again as P^T A P (same patterns)."""
        _load().or_h_refresh_numeric(self.h, A.h)
        self._A0 = A

    def smooth(self, l, b, x, x0zero=False):
        """One application of the level-l smoother to A_l x = b; returns the new x."""
        x = np.array(x, dtype=np.float64, copy=True)
        _load().or_h_smooth(self.h, l, np.ascontiguousarray(b, np.float64), x, int(bool(x0zero)))
        return x

    def vcycle(self, r):
        z = np.empty(self.A(0).nr)
        _load().or_vcycle(self.h, np.ascontiguousarray(r, np.float64), z)
        return z

    def pcg(self, b, tol=1e-12, maxit=500):
        """AMG-preconditioned CG from x0 = 0 to true relative residual tol."""
        x = np.empty(self.A(0).nr)
        it, rel = ctypes.c_int(), ctypes.c_double()
        st = _load().or_pcg(self.h, np.ascontiguousarray(b, np.float64), x, float(tol), int(maxit),
                            ctypes.byref(it), ctypes.byref(rel))
        return x, it.value, rel.value, st

    def stats(self):
        """Table-1 style statistics: per level (n, nnz), operator/grid complexity."""
        ns = [self.A(l).nr for l in range(self.nlevels)]
        nz = [self.A(l).nnz for l in range(self.nlevels)]
        return complexities(ns, nz)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_h_free(self.h)
            self.h = None


def adjoint_grad(nx, ny, nz, Kx, h, lam, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0),
                 spacing=(1.0, 1.0, 1.0)):
    """dJ/dlnK per cell from the heads h and the adjoint state lam (C lam = dJ/dh)."""
    Kx = np.ascontiguousarray(Kx, dtype=np.float64).ravel()
    Ky = Kx if Ky is None else np.ascontiguousarray(Ky, dtype=np.float64).ravel()
    Kz = Kx if Kz is None else np.ascontiguousarray(Kz, dtype=np.float64).ravel()
    g = np.empty(nx * ny * nz)
    _load().or_adjoint_grad(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]), Kx, Ky, Kz,
                            np.asarray(bct, np.int32), np.asarray(bcv, np.float64),
                            np.ascontiguousarray(h, np.float64), np.ascontiguousarray(lam, np.float64), g)
    return g


def misfit(h, obs, hobs):
    """J = sum (h[obs] - hobs)^2 and dJ/dh."""
    h = np.ascontiguousarray(h, np.float64)
    d = np.empty_like(h)
    J = _load().or_misfit(h.size, h, len(obs), np.ascontiguousarray(obs, np.int32),
                          np.ascontiguousarray(hobs, np.float64), d.ctypes.data_as(ctypes.c_void_p))
    return J, d


def darcy_flux(nx, ny, nz, Kx, h, Ky=None, Kz=None, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0),
               spacing=(1.0, 1.0, 1.0)):
    """Darcy velocities on the x, y, z faces (staggered: (nx+1)*ny*nz, ...)."""
    Kx = np.ascontiguousarray(Kx, dtype=np.float64).ravel()
    Ky = Kx if Ky is None else np.ascontiguousarray(Ky, dtype=np.float64).ravel()
    Kz = Kx if Kz is None else np.ascontiguousarray(Kz, dtype=np.float64).ravel()
    vx = np.empty((nx + 1) * ny * nz)
    vy = np.empty(nx * (ny + 1) * nz)
    vz = np.empty(nx * ny * (nz + 1))
    _load().or_darcy_flux(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]), Kx, Ky, Kz,
                          np.asarray(bct, np.int32), np.asarray(bcv, np.float64),
                          np.ascontiguousarray(h, np.float64), vx, vy, vz)
    return vx, vy, vz


def shift(C, s):
    """C + diag(s) (Eq. 2: the transient operator with s_i = S_i V_i / dt)."""
    return CSR(_load().or_shift_csr(C.h, np.ascontiguousarray(s, np.float64)))


def reuse_ok(C, s, s_built=None, delta=0.01):
    """|s_i - s_built_i| < delta C_ii for every row (Discussion section criterion)."""
    sb = None if s_built is None else np.ascontiguousarray(s_built, np.float64)
    return bool(_load().or_reuse_ok(C.h, np.ascontiguousarray(s, np.float64), _ptr(sb), float(delta)))


def complexities(ns, nnzs):
    """Hierarchy statistics as the AMGCL report of Table 1 defines them:
    operator complexity = sum nnz_l / nnz_0, grid complexity = sum n_l / n_0,
    and each level's share of the total nonzeros in percent."""
    tot = float(sum(nnzs))
    return dict(n=list(ns), nnz=list(nnzs), op_complexity=tot / nnzs[0],
                grid_complexity=float(sum(ns)) / ns[0], nnz_percent=[100.0 * z / tot for z in nnzs])


def cg_plain(A, b, tol=1e-8, maxit=10000):
    x = np.empty(A.nr)
    it, rel = ctypes.c_int(), ctypes.c_double()
    st = _load().or_cg_plain(A.h, np.ascontiguousarray(b, np.float64), x, float(tol), int(maxit),
                             ctypes.byref(it), ctypes.byref(rel))
    return x, it.value, rel.value, st
