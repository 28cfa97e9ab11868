"""Plain CPU FP64 oracle for the HFAV hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_1710_08774_gb300``): the C part
(``oracle.c``) is compiled here by gcc with ``-O2 -ffp-contract=off`` and
loaded through ctypes; the MLP part is plain numpy.

Every function is the plain, unfused definition of what the fused pipelines
compute (HFAV Sec. 3.1: kernels are side-effect free and order agnostic, so
fusion and contraction do not change values).  Parity status per function is
listed in the module docstrings of ``tests/test_oracle_*.py``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


class GodunovStats(ctypes.Structure):
    _fields_ = [("floor_hits", ctypes.c_long), ("newton_nonconv", ctypes.c_long),
                ("newton_iters", ctypes.c_long), ("faces", ctypes.c_long),
                ("iters_hist", ctypes.c_long * 11)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_chain2d.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_int, dp, dp, dp]
        L.oracle_chain3d.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_int, dp]
        L.oracle_cosmo.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                   ctypes.c_int, ctypes.c_double, dp, dp, dp, dp]
        L.oracle_riemann.argtypes = [dp, dp, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_long)]
        L.oracle_trace.argtypes = [dp, ctypes.c_double, dp, ctypes.c_double, dp, dp]
        L.oracle_godunov.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, dp,
                                     ctypes.POINTER(GodunovStats)]
        L.oracle_godunov_cfl_dt.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double]
        L.oracle_godunov_cfl_dt.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def chain2d(u_padded, periodic=True):
    """Three-stage 2D chain over a (ny+4, nx+4) FP64 array with the interior at (2, 2).

    Returns (L, G, out): L on the halo-1 ring (ny+2, nx+2), G and out on the
    interior (ny, nx).  Periodic: the halo is the wrapped interior."""
    u = np.ascontiguousarray(u_padded, dtype=np.float64)
    ny, nx = u.shape[0] - 4, u.shape[1] - 4
    L = np.empty((ny + 2, nx + 2)); G = np.empty((ny, nx)); out = np.empty((ny, nx))
    rc = lib().oracle_chain2d(_p(u), nx, ny, u.shape[1], int(bool(periodic)), _p(L), _p(G), _p(out))
    if rc != 0:
        raise RuntimeError(f"oracle_chain2d failed: {rc}")
    return L, G, out


def chain3d(u_padded, periodic=True):
    """Four-stage 3D 7-point chain over a (nz+6, ny+6, nx+6) FP64 array, interior at (3,3,3)."""
    u = np.ascontiguousarray(u_padded, dtype=np.float64)
    nz, ny, nx = (s - 6 for s in u.shape)
    out = np.empty((nz, ny, nx))
    rc = lib().oracle_chain3d(_p(u), nx, ny, nz, int(bool(periodic)), _p(out))
    if rc != 0:
        raise RuntimeError(f"oracle_chain3d failed: {rc}")
    return out


def cosmo(u_padded, c, periodic=True):
    """COSMO horizontal diffusion (Sec. 5.3) over an (nz+4, ny+4, nx+4) FP64
    array, interior at (2, 2, 2); every k plane on its own.

    Returns (lap, flx, fly, out): lap on the halo-1 ring (nz, ny+2, nx+2),
    flx on faces i = -1 .. nx-1 (nz, ny, nx+1), fly on faces j = -1 .. ny-1
    (nz, ny+1, nx), out on the interior (nz, ny, nx)."""
    u = np.ascontiguousarray(u_padded, dtype=np.float64)
    nz, ny, nx = (s - 4 for s in u.shape)
    lap = np.empty((nz, ny + 2, nx + 2)); flx = np.empty((nz, ny, nx + 1)); fly = np.empty((nz, ny + 1, nx))
    out = np.empty((nz, ny, nx))
    rc = lib().oracle_cosmo(_p(u), nx, ny, nz, u.shape[2], u.shape[1] * u.shape[2], int(bool(periodic)), float(c),
                            _p(lap), _p(flx), _p(fly), _p(out))
    if rc != 0:
        raise RuntimeError(f"oracle_cosmo failed: {rc}")
    return lap, flx, fly, out


def riemann(qL, qR, gamma=1.4):
    """Two-shock Newton Riemann solver sampled at x/t = 0.

    Returns (state, iterations, nonconverged, floor_hits) with primitive
    states (rho, u_normal, u_transverse, p)."""
    a = np.ascontiguousarray(qL, dtype=np.float64); b = np.ascontiguousarray(qR, dtype=np.float64)
    g = np.empty(4); nc = ctypes.c_int(0); fh = ctypes.c_long(0)
    it = lib().oracle_riemann(_p(a), _p(b), gamma, _p(g), ctypes.byref(nc), ctypes.byref(fh))
    return g, it, bool(nc.value), fh.value


def trace(W, c, dW, dtdx):
    """Characteristic tracing of one cell: primitive state W = (rho, u_n, u_t, p),
    sound speed c, limited slopes dW, dt/dx.  Returns (qm, qp): the states at
    the cell's left and right faces."""
    a = np.ascontiguousarray(W, dtype=np.float64); d = np.ascontiguousarray(dW, dtype=np.float64)
    qm = np.empty(4); qp = np.empty(4)
    lib().oracle_trace(_p(a), float(c), _p(d), float(dtdx), _p(qm), _p(qp))
    return qm, qp


def godunov(U, nsteps, cfl=0.5, gamma=1.4, dt_fixed=0.0, sweeps=3):
    """nsteps of the split Godunov scheme on a periodic grid.

    U: (4, ny, nx) FP64 conserved state (rho, rho u, rho v, E), not modified.
    Returns (U_new, dt_history, stats)."""
    W = np.array(U, dtype=np.float64, order="C", copy=True)
    _, ny, nx = W.shape
    dts = np.zeros(max(nsteps, 1))
    st = GodunovStats()
    rc = lib().oracle_godunov(_p(W), nx, ny, nsteps, cfl, gamma, dt_fixed, sweeps, _p(dts), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"oracle_godunov failed: {rc}")
    return W, dts[:nsteps], st


def godunov_cfl_dt(U, cfl=0.5, gamma=1.4):
    W = np.ascontiguousarray(U, dtype=np.float64)
    _, ny, nx = W.shape
    return lib().oracle_godunov_cfl_dt(_p(W), nx, ny, cfl, gamma)
