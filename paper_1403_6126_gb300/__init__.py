"""GB300 radiation-transfer step (Jiang, Stone & Davis 2014, arXiv:1403.6126).

Thin Python binding over the C ABI declared in ``include/rt.h``: the
functions below carry the C names and only marshal arguments (numpy arrays
for host memory, torch CUDA tensors for device memory).  Every step of the
method runs in the CUDA library ``librt_gb300.so`` built from ``csrc/``;
there is no CPU fallback, and importing the binding fails loudly when the
library has not been built.

Array conventions (as in rt.h): cell fields (nz, ny, nx) or flat N, x
fastest; vectors component-major (3, N); pressure (6, N) ordered xx, yy, zz,
xy, xz, yz; intensities angle-major (M, N).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt_gb300.so")

RT_OK, RT_PENDING = 0, 1
RT_E_INVALID, RT_E_NOMEM, RT_E_BUDGET, RT_E_CUDA, RT_E_NONFINITE, RT_E_TIMEOUT, RT_E_STATE = -1, -2, -3, -4, -5, -6, -7
RT_BC_PERIODIC, RT_BC_VACUUM, RT_BC_COPY, RT_BC_INFLOW = 0, 1, 2, 3
RT_FP64, RT_FP32, RT_BF16 = 0, 1, 2
RT_ANGLES_LEVEL_SYMMETRIC, RT_ANGLES_GAUSS_LEGENDRE, RT_ANGLES_PAPER_S4 = 0, 1, 2
RT_FAULT_NONE, RT_FAULT_ALLOC = 0, 1

_STATUS_NAMES = {0: "RT_OK", 1: "RT_PENDING", -1: "RT_E_INVALID", -2: "RT_E_NOMEM", -3: "RT_E_BUDGET",
                 -4: "RT_E_CUDA", -5: "RT_E_NONFINITE", -6: "RT_E_TIMEOUT", -7: "RT_E_STATE"}


class rt_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", (ctypes.c_int * 2) * 3)]


class rt_angles(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double))]


class rt_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cfl", ctypes.c_double), ("gamma", ctypes.c_double),
                ("r_ideal", ctypes.c_double), ("hold_T", ctypes.c_int), ("estimate_v", ctypes.c_int),
                ("device_ptrs", ctypes.c_int), ("stream", ctypes.c_void_p), ("newton_max_it", ctypes.c_int),
                ("newton_rtol", ctypes.c_double)]


class rt_noalloc_fields(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("I_in", "I_out", "rho", "sigma_a", "sigma_s", "v", "T", "mom_in",
                                               "mom_out", "dE_gas", "dMom", "inflow")]


class rt_tile_time(ctypes.Structure):
    _fields_ = [("tx", ctypes.c_int), ("ty", ctypes.c_int), ("tz", ctypes.c_int), ("ms", ctypes.c_double)]


class RTError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s: %s (%s)" % (where, _STATUS_NAMES.get(status, status), msg))
        self.status = status


_DP = ctypes.POINTER(ctypes.c_double)
_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librt_gb300.so is missing: run paper_1403_6126_gb300/build.py "
                              "(or __graft_entry__.build()) first; there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        V, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "rt_options_default": (I, [ctypes.POINTER(rt_options)]),
            "rt_angle_set": (I, [I, I, I, ctypes.POINTER(I), _DP, _DP]),
            "rt_create": (I, [ctypes.POINTER(rt_grid), ctypes.POINTER(rt_angles), D, D,
                              ctypes.POINTER(rt_options), ctypes.POINTER(V)]),
            "rt_set_material": (I, [V, V, V, V, V, V]),
            "rt_set_intensity": (I, [V, V]),
            "rt_set_inflow": (I, [V, I, I, _DP]),
            "rt_cfl_dt": (D, [V]),
            "rt_set_tile": (I, [V, I, I, I]),
            "rt_get_tile": (I, [V, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "rt_autotune": (I, [V, I, ctypes.POINTER(rt_tile_time), I, ctypes.POINTER(I)]),
            "rt_batch_autotune": (I, [V, I, _DP, ctypes.POINTER(I)]),
            "rt_state_bytes": (ctypes.c_size_t, [V]),
            "rt_save_state": (I, [V, V, ctypes.c_size_t]),
            "rt_load_state": (I, [V, V, ctypes.c_size_t]),
            "rt_step": (I, [V, D]),
            "rt_run": (I, [V, D, I]),
            "rt_sync": (I, [V]),
            "rt_moments": (I, [V, V, V, V]),
            "rt_sources": (I, [V, V, V, V]),
            "rt_eddington": (I, [V, V]),
            "rt_step_coupled": (I, [V, D, V, V, V, V, V, V, V, V]),
            "rt_get_intensity": (I, [V, V]),
            "rt_destroy": (None, [V]),
            "rt_batch_create": (I, [V, ctypes.POINTER(V)]),
            "rt_batch_add": (I, [V, V]),
            "rt_batch_remove": (I, [V, V]),
            "rt_batch_size": (I, [V]),
            "rt_batch_step": (I, [V, I]),
            "rt_batch_destroy": (None, [V]),
            "rt_server_create": (I, [ctypes.c_size_t, ctypes.POINTER(rt_options), ctypes.POINTER(V)]),
            "rt_submit": (I, [V, ctypes.POINTER(rt_grid), ctypes.POINTER(rt_angles), D, D, V, V, V, V, V, I,
                              ctypes.POINTER(ctypes.c_longlong)]),
            "rt_submit_inflow": (I, [V, ctypes.POINTER(rt_grid), ctypes.POINTER(rt_angles), D, D, V, V, V, V, V, V,
                                     I, ctypes.POINTER(ctypes.c_longlong)]),
            "rt_poll": (I, [V, ctypes.c_longlong, V, V, V, ctypes.POINTER(D)]),
            "rt_server_wait": (I, [V, ctypes.c_longlong, D]),
            "rt_server_stats": (I, [V, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I), ctypes.POINTER(I),
                                    ctypes.POINTER(ctypes.c_size_t)]),
            "rt_server_destroy": (None, [V]),
            "rt_step_noalloc": (I, [ctypes.POINTER(rt_grid), ctypes.POINTER(rt_angles), D, D, ctypes.POINTER(rt_options),
                                    D, ctypes.POINTER(rt_noalloc_fields), ctypes.POINTER(I)]),
            "rt_last_error": (ctypes.c_char_p, []),
            "rt_fault_inject": (I, [I, I]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != RT_OK:
        raise RTError(status, where, lib().rt_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    """Address of a C-contiguous float64 numpy array or torch tensor (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise ValueError("device arrays must be contiguous float64 tensors")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("host arrays must be C-contiguous float64 numpy arrays")
    return a.ctypes.data


# ---- the C ABI, one Python function per entry point ------------------------

def rt_options_default():
    o = rt_options()
    _check(lib().rt_options_default(ctypes.byref(o)), "rt_options_default")
    return o


def rt_angle_set(kind, order):
    """Returns (n [M,3], w [M]) from the library's generator."""
    cap = 512
    n = np.zeros((cap, 3))
    w = np.zeros(cap)
    m = ctypes.c_int(0)
    _check(lib().rt_angle_set(kind, order, cap, ctypes.byref(m), n.ctypes.data_as(_DP), w.ctypes.data_as(_DP)),
           "rt_angle_set")
    return n[: m.value].copy(), w[: m.value].copy()


def rt_create(grid, angles, Crat, Prat, opts):
    out = ctypes.c_void_p()
    _check(lib().rt_create(ctypes.byref(grid), ctypes.byref(angles), Crat, Prat, ctypes.byref(opts),
                           ctypes.byref(out)), "rt_create")
    return out


def rt_set_material(ctx, rho, T, v, sigma_a, sigma_s):
    _check(lib().rt_set_material(ctx, _ptr(rho), _ptr(T), _ptr(v), _ptr(sigma_a), _ptr(sigma_s)), "rt_set_material")


def rt_set_intensity(ctx, I):
    _check(lib().rt_set_intensity(ctx, _ptr(I)), "rt_set_intensity")


def rt_set_inflow(ctx, axis, side, I_ghost):
    I_ghost = np.ascontiguousarray(I_ghost, dtype=np.float64)
    _check(lib().rt_set_inflow(ctx, axis, side, I_ghost.ctypes.data_as(_DP)), "rt_set_inflow")


def rt_set_tile(ctx, tx, ty, tz):
    _check(lib().rt_set_tile(ctx, tx, ty, tz), "rt_set_tile")


def rt_get_tile(ctx):
    t = [ctypes.c_int(0) for _ in range(3)]
    _check(lib().rt_get_tile(ctx, *[ctypes.byref(x) for x in t]), "rt_get_tile")
    return tuple(x.value for x in t)


def rt_autotune(ctx, trial_steps=3):
    """Times every compiled tile that fits, keeps the fastest; returns
    [(tx, ty, tz, ms per step), ...]."""
    buf = (rt_tile_time * 8)()
    n = ctypes.c_int(0)
    _check(lib().rt_autotune(ctx, trial_steps, buf, 8, ctypes.byref(n)), "rt_autotune")
    return [(t.tx, t.ty, t.tz, t.ms) for t in buf[: n.value]]


def rt_state_bytes(ctx):
    return lib().rt_state_bytes(ctx)


def rt_save_state(ctx):
    """The context's restartable state as a uint8 numpy array."""
    buf = np.empty(rt_state_bytes(ctx), dtype=np.uint8)
    _check(lib().rt_save_state(ctx, buf.ctypes.data, buf.nbytes), "rt_save_state")
    return buf


def rt_load_state(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().rt_load_state(ctx, buf.ctypes.data, buf.nbytes), "rt_load_state")


def rt_cfl_dt(ctx):
    return lib().rt_cfl_dt(ctx)


def rt_step(ctx, dt):
    _check(lib().rt_step(ctx, dt), "rt_step")


def rt_run(ctx, dt, nsteps):
    _check(lib().rt_run(ctx, dt, nsteps), "rt_run")


def rt_sync(ctx):
    _check(lib().rt_sync(ctx), "rt_sync")


def rt_moments(ctx, E, F, P):
    _check(lib().rt_moments(ctx, _ptr(E), _ptr(F), _ptr(P)), "rt_moments")


def rt_eddington(ctx, f):
    _check(lib().rt_eddington(ctx, _ptr(f)), "rt_eddington")


def rt_sources(ctx, dE_gas, dMom, T_new):
    _check(lib().rt_sources(ctx, _ptr(dE_gas), _ptr(dMom), _ptr(T_new)), "rt_sources")


def rt_step_coupled(ctx, dt, rho, T, v, sigma_a, sigma_s, dE_gas, dMom, T_new):
    _check(lib().rt_step_coupled(ctx, float(dt), _ptr(rho), _ptr(T), _ptr(v), _ptr(sigma_a), _ptr(sigma_s),
                                 _ptr(dE_gas), _ptr(dMom), _ptr(T_new)), "rt_step_coupled")


def rt_get_intensity(ctx, I):
    _check(lib().rt_get_intensity(ctx, _ptr(I)), "rt_get_intensity")


def rt_destroy(ctx):
    lib().rt_destroy(ctx)


def rt_batch_create(stream=None):
    out = ctypes.c_void_p()
    _check(lib().rt_batch_create(stream, ctypes.byref(out)), "rt_batch_create")
    return out


def rt_batch_add(b, ctx):
    _check(lib().rt_batch_add(b, ctx), "rt_batch_add")


def rt_batch_remove(b, ctx):
    _check(lib().rt_batch_remove(b, ctx), "rt_batch_remove")


def rt_batch_size(b):
    return lib().rt_batch_size(b)


def rt_batch_step(b, nsteps):
    _check(lib().rt_batch_step(b, nsteps), "rt_batch_step")


def rt_batch_autotune(b, trial_steps=3):
    """Times the three compiled tile sets; returns (ms per step of each,
    -1 where a set does not fit, index kept)."""
    ms = np.zeros(3)
    chosen = ctypes.c_int(-1)
    _check(lib().rt_batch_autotune(b, trial_steps, ms.ctypes.data_as(_DP), ctypes.byref(chosen)),
           "rt_batch_autotune")
    return ms.tolist(), chosen.value


def rt_batch_destroy(b):
    lib().rt_batch_destroy(b)


def rt_server_create(hbm_budget_bytes, opts):
    out = ctypes.c_void_p()
    _check(lib().rt_server_create(hbm_budget_bytes, ctypes.byref(opts), ctypes.byref(out)), "rt_server_create")
    return out


def rt_submit(server, grid, angles, Crat, Prat, rho, T, v, sigma_a, sigma_s, nsteps):
    t = ctypes.c_longlong(0)
    _check(lib().rt_submit(server, ctypes.byref(grid), ctypes.byref(angles), Crat, Prat, _ptr(rho), _ptr(T), _ptr(v),
                           _ptr(sigma_a), _ptr(sigma_s), nsteps, ctypes.byref(t)), "rt_submit")
    return t.value


def rt_submit_inflow(server, grid, angles, Crat, Prat, rho, T, v, sigma_a, sigma_s, inflow, nsteps):
    """inflow: [3][2][M] float64 host array of incoming intensities per face, or None."""
    t = ctypes.c_longlong(0)
    _check(lib().rt_submit_inflow(server, ctypes.byref(grid), ctypes.byref(angles), Crat, Prat, _ptr(rho), _ptr(T),
                                  _ptr(v), _ptr(sigma_a), _ptr(sigma_s), _ptr(inflow),
                                  nsteps, ctypes.byref(t)), "rt_submit_inflow")
    return t.value


def rt_poll(server, ticket, E=None, F=None, P=None):
    """Returns None while pending, else the latency in seconds (E, F, P filled)."""
    lat = ctypes.c_double(0.0)
    st = lib().rt_poll(server, ticket, _ptr(E), _ptr(F), _ptr(P), ctypes.byref(lat))
    if st == RT_PENDING:
        return None
    _check(st, "rt_poll")
    return lat.value


def rt_server_wait(server, ticket, timeout_s=-1.0):
    _check(lib().rt_server_wait(server, ticket, timeout_s), "rt_server_wait")


def rt_server_stats(server):
    steps, q, r, b = ctypes.c_longlong(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_size_t(0)
    _check(lib().rt_server_stats(server, ctypes.byref(steps), ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)),
           "rt_server_stats")
    return dict(steps=steps.value, queued=q.value, running=r.value, bytes_in_use=b.value)


def rt_server_destroy(server):
    lib().rt_server_destroy(server)


def rt_step_noalloc(grid, angles, Crat, Prat, opts, dt, fields, want_failures=True):
    """fields: rt_noalloc_fields of device addresses.  Returns the Newton
    failure count when want_failures (the call then waits for the stream)."""
    nf = ctypes.c_int(0)
    _check(lib().rt_step_noalloc(ctypes.byref(grid), ctypes.byref(angles), Crat, Prat, ctypes.byref(opts), dt,
                                 ctypes.byref(fields), ctypes.byref(nf) if want_failures else None), "rt_step_noalloc")
    return nf.value


def rt_fault_inject(kind, after=0):
    _check(lib().rt_fault_inject(kind, after), "rt_fault_inject")


def rt_last_error():
    return lib().rt_last_error().decode(errors="replace")


# ---- convenience wrapper (argument marshalling only) ----------------------

class Context:
    """Owns one rt_ctx.  shape = (nz, ny, nx); lo/hi per axis (x, y, z);
    bc = ((x_lo, x_hi), (y_lo, y_hi), (z_lo, z_hi)); n, w the angle set."""

    def __init__(self, shape, n, w, Crat, Prat, dim=None, lo=(0, 0, 0), hi=(1, 1, 1), bc=None,
                 precision=RT_FP32, cfl=0.4, gamma=5.0 / 3.0, r_ideal=1.0, hold_T=False, estimate_v=True,
                 device_ptrs=False, stream=None):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.dim = dim if dim is not None else (3 if nz > 1 else (2 if ny > 1 else 1))
        g = rt_grid()
        g.dim = self.dim
        for d, nd in enumerate((nx, ny, nz)):
            g.n[d] = nd
            g.lo[d] = lo[d]
            g.hi[d] = hi[d]
        bc = bc or ((RT_BC_PERIODIC, RT_BC_PERIODIC),) * 3
        for d in range(3):
            g.bc[d][0], g.bc[d][1] = bc[d]
        self._n = np.ascontiguousarray(n, dtype=np.float64).reshape(-1, 3)
        self._w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        self.M = len(self._w)
        a = rt_angles()
        a.m = self.M
        a.n = self._n.ctypes.data_as(_DP)
        a.w = self._w.ctypes.data_as(_DP)
        o = rt_options_default()
        o.precision, o.cfl, o.gamma, o.r_ideal = precision, cfl, gamma, r_ideal
        o.hold_T, o.estimate_v, o.device_ptrs = int(hold_T), int(estimate_v), int(device_ptrs)
        o.stream = stream
        self.device_ptrs = bool(device_ptrs)
        self.ctx = rt_create(g, a, float(Crat), float(Prat), o)

    @property
    def N(self):
        nz, ny, nx = self.shape
        return nz * ny * nx

    def _host(self, a, count):
        if self.device_ptrs:
            return a
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if a.size != count:
            raise ValueError("expected %d values, got %d" % (count, a.size))
        return a

    def set_material(self, rho, T, v, sigma_a, sigma_s):
        N = self.N
        self._keep = [self._host(rho, N), self._host(T, N), self._host(v, 3 * N), self._host(sigma_a, N),
                      self._host(sigma_s, N)]
        rt_set_material(self.ctx, *self._keep)

    def set_intensity(self, I=None):
        rt_set_intensity(self.ctx, None if I is None else self._host(I, self.M * self.N))

    def set_inflow(self, axis, side, I_ghost):
        I_ghost = np.ascontiguousarray(I_ghost, dtype=np.float64).reshape(-1)
        if I_ghost.size != self.M:
            raise ValueError("expected %d incoming intensities, got %d" % (self.M, I_ghost.size))
        rt_set_inflow(self.ctx, axis, side, I_ghost)

    def cfl_dt(self):
        return rt_cfl_dt(self.ctx)

    def set_tile(self, tx, ty, tz):
        rt_set_tile(self.ctx, tx, ty, tz)

    def tile(self):
        return rt_get_tile(self.ctx)

    def autotune(self, trial_steps=3):
        return rt_autotune(self.ctx, trial_steps)

    def save_state(self):
        return rt_save_state(self.ctx)

    def load_state(self, buf):
        rt_load_state(self.ctx, buf)

    def step(self, dt=0.0):
        rt_step(self.ctx, dt)

    def run(self, dt, nsteps):
        rt_run(self.ctx, dt, nsteps)

    def sync(self):
        rt_sync(self.ctx)

    def moments(self):
        N = self.N
        E, F, P = np.zeros(N), np.zeros((3, N)), np.zeros((6, N))
        rt_moments(self.ctx, E, F, P)
        return E, F, P

    def eddington(self):
        """f = P_r / E_r (6, N): xx, yy, zz, xy, xz, yz."""
        f = np.zeros((6, self.N))
        rt_eddington(self.ctx, f)
        return f

    def sources(self):
        N = self.N
        dE, dM, T = np.zeros(N), np.zeros((3, N)), np.zeros(N)
        rt_sources(self.ctx, dE, dM, T)
        return dE, dM, T

    def step_coupled(self, dt, rho, T, v, sigma_a, sigma_s, dE_gas=None, dMom=None, T_new=None):
        """rt_step_coupled: the fields in, one step, the sources out (into the
        given float64 arrays, or new ones); returns (dE_gas, dMom, T_new)."""
        N = self.N
        fields = [self._host(rho, N), self._host(T, N), self._host(v, 3 * N), self._host(sigma_a, N),
                  self._host(sigma_s, N)]
        dE_gas = np.zeros(N) if dE_gas is None else dE_gas
        dMom = np.zeros((3, N)) if dMom is None else dMom
        T_new = np.zeros(N) if T_new is None else T_new
        rt_step_coupled(self.ctx, dt, *fields, dE_gas, dMom, T_new)
        return dE_gas, dMom, T_new

    def intensity(self):
        I = np.zeros((self.M, self.N))
        rt_get_intensity(self.ctx, I)
        return I

    def close(self):
        if getattr(self, "ctx", None):
            rt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
