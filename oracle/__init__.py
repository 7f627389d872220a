"""FP64 CPU oracle for the radiation-transfer step (arXiv:1403.6126, secs. 3-4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` (and the script there that
stores oracle values, ``tests/golden/make_stated_steps.py``),
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package.  It shares no
code with the GPU library (``paper_1403_6126_gb300``) and never imports it.

The arithmetic lives in ``rt_oracle.c`` (plain serial-per-cell C, double
precision, optional OpenMP over cells); this module compiles it with gcc and
marshals numpy arrays through ctypes.  Array conventions at this level:
cell fields (nz, ny, nx); vectors (3, nz, ny, nx); P (6, ...) ordered xx, yy,
zz, xy, xz, yz; intensities (M, nz, ny, nx).
"""
import ctypes
import os
import subprocess

import numpy as np

from . import angles  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
# RT_ORACLE_SRC / RT_ORACLE_LIB point the module at another copy of the C
# source and its library (tests/oracle_mutations.py builds altered copies
# there to check that the pins catch them); unset, the files beside this one
_SRC = os.environ.get("RT_ORACLE_SRC") or os.path.join(_HERE, "rt_oracle.c")
_LIB = os.environ.get("RT_ORACLE_LIB") or os.path.join(_HERE, "_liborc.so")

PERIODIC, VACUUM, COPY, INFLOW = 0, 1, 2, 3


def build(force=False):
    """Compile rt_oracle.c with gcc (-O2, no fast-math, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3), ("inflow", ctypes.POINTER(ctypes.c_double)),
        ("M", ctypes.c_int), ("mu", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
        ("C", ctypes.c_double), ("P", ctypes.c_double), ("gamma", ctypes.c_double), ("R", ctypes.c_double),
        ("hold_T", ctypes.c_int), ("estimate_v", ctypes.c_int), ("dense", ctypes.c_int),
        ("alpha_one", ctypes.c_int),
    ]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        lib.orc_step.restype = ctypes.c_long
        lib.orc_step.argtypes = [P, ctypes.c_double] + [_DP] * 9
        lib.orc_moments.argtypes = [P, _DP, _DP, _DP, _DP]
        lib.orc_transport.argtypes = [P, ctypes.c_double] + [_DP] * 5
        lib.orc_absorption_cell.restype = ctypes.c_int
        lib.orc_absorption_cell.argtypes = [P] + [ctypes.c_double] * 4 + [_DP] * 5
        lib.orc_scattering_cell.restype = ctypes.c_int
        lib.orc_scattering_cell.argtypes = [P, ctypes.c_double, ctypes.c_double, _DP, _DP, _DP]
        lib.orc_vtilde.argtypes = [P, ctypes.c_double, _DP, ctypes.c_double, ctypes.c_double, _DP, _DP,
                                   ctypes.c_double, _DP]
        lib.orc_alpha.restype = ctypes.c_double
        lib.orc_alpha.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_cfl_dt.restype = ctypes.c_double
        lib.orc_cfl_dt.argtypes = [P, ctypes.c_double]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Grid, angle set and dimensionless parameters of one radiation problem.

    shape: (nz, ny, nx) active cells (1 on inactive axes); dim: active axes.
    bc: ((x_lo, x_hi), (y_lo, y_hi), (z_lo, z_hi)) boundary kinds.
    inflow: optional dict {(axis, side): array[M]} for INFLOW faces.
    """

    def __init__(self, shape, dx, n, w, C, P, dim=None, bc=None, inflow=None, gamma=5.0 / 3.0, R=1.0,
                 hold_T=False, estimate_v=False, dense=False, alpha_one=False):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.dim = dim if dim is not None else (3 if nz > 1 else (2 if ny > 1 else 1))
        self.n_ang = _f64(n).reshape(-1, 3)
        self.w = _f64(w).reshape(-1)
        self.M = len(self.w)
        self.C, self.P, self.gamma, self.R = float(C), float(P), float(gamma), float(R)
        if np.isscalar(dx):
            dx = (dx, dx, dx)
        self.dx = tuple(float(x) for x in dx)
        self.bc = bc if bc is not None else ((PERIODIC, PERIODIC),) * 3
        self._inflow = np.zeros((3, 2, self.M))
        for (ax, side), val in (inflow or {}).items():
            self._inflow[ax, side] = val
        self.hold_T, self.estimate_v, self.dense = bool(hold_T), bool(estimate_v), bool(dense)
        self._s = _Problem()
        s = self._s
        s.dim = self.dim
        s.n[0], s.n[1], s.n[2] = nx, ny, nz
        for i in range(3):
            s.dx[i] = self.dx[i]
            s.bc[i][0], s.bc[i][1] = self.bc[i]
        s.inflow = _ptr(self._inflow)
        s.M = self.M
        s.mu, s.w = _ptr(self.n_ang), _ptr(self.w)
        s.C, s.P, s.gamma, s.R = self.C, self.P, self.gamma, self.R
        s.hold_T, s.estimate_v, s.dense = int(self.hold_T), int(self.estimate_v), int(self.dense)
        # alpha_one: alpha = 1 on every face (the plain upwinding the paper
        # improves on in sec. 4.2), a control for the tests only
        s.alpha_one = int(alpha_one)

    @property
    def N(self):
        nz, ny, nx = self.shape
        return nz * ny * nx

    def ref(self):
        return ctypes.byref(self._s)


def cfl_dt(prob, cfl):
    """Step 1 (sec. 4.1): dt = cfl * min(dx) / C over the active axes."""
    return _load().orc_cfl_dt(prob.ref(), cfl)


def alpha(dl, sigma_t):
    """Reduced transport-speed factor of sec. 4.2."""
    return _load().orc_alpha(float(dl), float(sigma_t))


def set_threads(k):
    _load().orc_set_threads(int(k))


def max_threads():
    return _load().orc_max_threads()


def _vec_to_c(v, N):
    return _f64(np.asarray(v, dtype=np.float64).reshape(3, N).T)


def moments(prob, I):
    """Sec. 3 quadrature: returns E (N), F (3, N), P (6, N), as float64."""
    N = prob.N
    I = _f64(I).reshape(prob.M, N)
    E, F, Pm = np.zeros(N), np.zeros((N, 3)), np.zeros((N, 6))
    _load().orc_moments(prob.ref(), _ptr(I), _ptr(E), _ptr(F), _ptr(Pm))
    return E, F.T.copy(), Pm.T.copy()


def transport(prob, dt, I, v, sa, ss):
    """Step 2 (sec. 4.2): Delta F (M, N)."""
    N = prob.N
    I = _f64(I).reshape(prob.M, N)
    dF = np.zeros((prob.M, N))
    _load().orc_transport(prob.ref(), dt, _ptr(I), _ptr(_vec_to_c(v, N)), _ptr(_f64(sa).reshape(N)),
                          _ptr(_f64(ss).reshape(N)), _ptr(dF))
    return dF


def step(prob, dt, I, T, rho, v, sa, ss, return_dF=False):
    """One full step (Steps 2-5 + quadrature).  Returns a dict with the new
    I (M, N), T (N), dEgas (N), dMom (3, N), E, F, P and the failure count."""
    N = prob.N
    I = _f64(I).reshape(prob.M, N).copy()
    T = _f64(T).reshape(N).copy()
    dE, dM = np.zeros(N), np.zeros((N, 3))
    dF = np.zeros((prob.M, N)) if return_dF else None
    fails = _load().orc_step(prob.ref(), dt, _ptr(I), _ptr(T), _ptr(_f64(rho).reshape(N)),
                             _ptr(_vec_to_c(v, N)), _ptr(_f64(sa).reshape(N)), _ptr(_f64(ss).reshape(N)),
                             _ptr(dE), _ptr(dM), _ptr(dF) if return_dF else ctypes.cast(None, _DP))
    E, F, Pm = moments(prob, I)
    out = dict(I=I, T=T, dEgas=dE, dMom=dM.T.copy(), E=E, F=F, P=Pm, failures=int(fails))
    if return_dF:
        out["dF"] = dF
    return out


def run(prob, dt, nsteps, I, T, rho, v, sa, ss):
    """nsteps steps from (I, T); returns the last step's dict."""
    out = None
    for _ in range(nsteps):
        out = step(prob, dt, I, T, rho, v, sa, ss)
        if out["failures"]:
            raise RuntimeError("oracle: %d cells failed to converge" % out["failures"])
        I, T = out["I"], out["T"]
    return out


def absorption_cell(prob, rho, T0, sa, dt, v, r, Istart=None):
    """Step 4 on one cell: returns (I_new[M], T_new, status)."""
    r = _f64(r)
    Istart = _f64(r if Istart is None else Istart)
    I = np.zeros(prob.M)
    T1 = ctypes.c_double(0.0)
    st = _load().orc_absorption_cell(prob.ref(), rho, T0, sa, dt, _ptr(_f64(v)), _ptr(r), _ptr(Istart),
                                     _ptr(I), ctypes.cast(ctypes.pointer(T1), _DP))
    return I, T1.value, st


def scattering_cell(prob, ss, dt, v, r):
    """Step 5 on one cell: returns (I_new[M], status)."""
    I = np.zeros(prob.M)
    st = _load().orc_scattering_cell(prob.ref(), ss, dt, _ptr(_f64(v)), _ptr(_f64(r)), _ptr(I))
    return I, st


def vtilde(prob, rho, v, st, E, F, Pd, dt):
    """Step 3 (sec. 4.5) on one cell."""
    out = np.zeros(3)
    _load().orc_vtilde(prob.ref(), rho, _ptr(_f64(v)), st, E, _ptr(_f64(F)), _ptr(_f64(Pd)), dt, _ptr(out))
    return out
