"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the method: it only draws the gas fields
(density, temperature, velocity, attenuation coefficients), names the grid,
angle set and parameters, and says which faces get incoming beams.  Both the
GPU path and the CPU oracle take their inputs from here; each side builds
its own angle table from the set's name.

Workloads (the recipe of each is in its function's docstring):
  slab1d    1-D scattering slab, the shape of the sec. 5.3 atmosphere
  shadow2d  2-D shadow problem of sec. 5.8
  box3d     3-D periodic radiation-dominated box, the sec. 6 performance setup
            made radiation dominated, with turbulent velocity and opacity
"""
import numpy as np

PERIODIC, VACUUM, COPY, INFLOW = 0, 1, 2, 3


def _spectral_field(rng, shape, kmin, kmax, slope):
    """Unit-variance Gaussian random field on a periodic grid with power
    spectrum P(k) ~ k^slope for kmin <= |k| <= kmax (k in box units)."""
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    K = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    amp = np.zeros_like(K)
    band = (K >= kmin) & (K <= kmax)
    amp[band] = K[band] ** (slope / 2.0)
    noise = rng.normal(size=K.shape) + 1j * rng.normal(size=K.shape)
    f = np.fft.irfftn(noise * amp, s=shape, axes=(0, 1, 2))
    f -= f.mean()
    return f / f.std()


def slab1d(n=512, M=8, seed=0, steps=2000):
    """1-D slab on x in [0, 1]: rho = 1, T = 1 held, v = 0, sigma_a = 1e-2,
    sigma_s = 10^U(-1, 2) per cell (seed), I0 = 1/(4 pi); bottom (x = 0)
    copies all rays, top (x = 1) is vacuum (sec. 5.3 boundaries).  Crat = 10,
    Prat = 1, Courant 0.5, Gauss-Legendre angles, double precision."""
    rng = np.random.default_rng(seed)
    N = n
    return dict(
        name="slab1d", shape=(1, 1, n), dim=1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
        bc=((COPY, VACUUM), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC)),
        angles="gl%d" % M, C=10.0, P=1.0, gamma=5.0 / 3.0, R=1.0, cfl=0.5, hold_T=True, estimate_v=False,
        steps=steps, precision="fp64",
        rho=np.ones(N), T=np.ones(N), v=np.zeros((3, N)), sa=np.full(N, 1e-2),
        ss=10.0 ** rng.uniform(-1.0, 2.0, N), I0="isotropic_quarter_pi", inflow={},
    )


def shadow2d(nx=256, ny=128, angles="s8", steps=4000, precision="fp32"):
    """2-D shadow problem of sec. 5.8 on (-0.5, 0.5) x (-0.3, 0.3): rho = 1 +
    9 / (1 + exp(10 (r - 1))) with r = x^2/0.1^2 + y^2/0.06^2, T = 1/rho held,
    sigma_a = T^-3.5 rho^2, sigma_s = 0, v = 0.  Beam I = 10 enters through
    x = -0.5 on every ray with n_x > 0; x = 0.5 copies; y faces are vacuum.
    Crat = 10, Prat = 1, Courant 0.4."""
    x = -0.5 + (np.arange(nx) + 0.5) / nx
    y = -0.3 + (np.arange(ny) + 0.5) * 0.6 / ny
    X, Y = np.meshgrid(x, y)  # (ny, nx)
    r = X ** 2 / 0.1 ** 2 + Y ** 2 / 0.06 ** 2
    rho = 1.0 + 9.0 / (1.0 + np.exp(10.0 * (r - 1.0)))
    T = 1.0 / rho
    sa = T ** -3.5 * rho ** 2
    N = nx * ny
    return dict(
        name="shadow2d", shape=(1, ny, nx), dim=2, lo=(-0.5, -0.3, 0.0), hi=(0.5, 0.3, 1.0),
        bc=((INFLOW, COPY), (VACUUM, VACUUM), (PERIODIC, PERIODIC)),
        angles=angles, C=10.0, P=1.0, gamma=5.0 / 3.0, R=1.0, cfl=0.4, hold_T=True, estimate_v=False,
        steps=steps, precision=precision,
        rho=rho.reshape(N), T=T.reshape(N), v=np.zeros((3, N)), sa=sa.reshape(N), ss=np.zeros(N),
        I0="equilibrium", inflow={(0, 0): ("beam", 10.0, 0)},
    )


def _gas_fields(shape, C, seed, kmax):
    """rho, v, sigma_a, sigma_s of the box recipe on a periodic grid of the
    given shape: rho = exp(0.5 g - 1/8) with g a unit Gaussian random field,
    P(k) ~ k^-2 on 1 <= |k| <= kmax (seed); v a Gaussian random vector field
    (seed + 1) scaled to rms |v| = 0.05 Crat, then |v|/Crat clipped into
    [0.01, 0.1] keeping the direction; sigma_a, sigma_s = 10^U(0, 3) per cell
    (seed + 2)."""
    g = _spectral_field(np.random.default_rng(seed), shape, 1.0, kmax, -2.0)
    rho = np.exp(0.5 * g - 0.125)
    rv = np.random.default_rng(seed + 1)
    v = np.stack([_spectral_field(rv, shape, 1.0, kmax, -2.0) for _ in range(3)])
    speed = np.sqrt((v ** 2).sum(axis=0))
    v *= 0.05 * C / np.sqrt((speed ** 2).mean())
    speed = np.sqrt((v ** 2).sum(axis=0))
    target = np.clip(speed, 0.01 * C, 0.1 * C)
    v *= target / np.maximum(speed, 1e-300)
    ro = np.random.default_rng(seed + 2)
    N = int(np.prod(shape))
    sa = 10.0 ** ro.uniform(0.0, 3.0, N)
    ss = 10.0 ** ro.uniform(0.0, 3.0, N)
    return rho.reshape(N), v.reshape(3, N), sa, ss


def box3d(n=128, angles="s8", seed=2, steps=500, precision="fp32", kmax=None):
    """3-D periodic box [0, 1]^3 (the sec. 6 performance setup, radiation
    dominated), gas fields from _gas_fields with kmax = min(16, n/2) unless
    given; T0 = 1, I0 = 1/(4 pi); Crat = 100, Prat = 100, gamma = 5/3,
    R = 1, Courant 0.4; T live, velocity estimate on."""
    shape = (n, n, n)
    C = 100.0
    rho, v, sa, ss = _gas_fields(shape, C, seed, min(16.0, n / 2) if kmax is None else kmax)
    N = n ** 3
    return dict(
        name="box3d", shape=shape, dim=3, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
        bc=((PERIODIC, PERIODIC),) * 3,
        angles=angles, C=C, P=100.0, gamma=5.0 / 3.0, R=1.0, cfl=0.4, hold_T=False, estimate_v=True,
        steps=steps, precision=precision,
        rho=rho, T=np.ones(N), v=v, sa=sa, ss=ss,
        I0="isotropic_quarter_pi", inflow={},
    )


def box2d(n=256, angles="s8", seed=2, steps=500, precision="fp32", kmax=None):
    """The box recipe on a periodic square [0, 1]^2 (one cell in z): gas
    fields from _gas_fields on (1, n, n), kmax = min(16, n/2) unless given,
    the rest as in box3d."""
    wl = box3d(n=2, angles=angles, seed=seed, steps=steps, precision=precision, kmax=1.0)
    rho, v, sa, ss = _gas_fields((1, n, n), wl["C"], seed, min(16.0, n / 2) if kmax is None else kmax)
    wl.update(name="box2d", shape=(1, n, n), dim=2, rho=rho, T=np.ones(n * n), v=v, sa=sa, ss=ss)
    return wl


def batched(nprob=512, seed=5, steps=200):
    """Many independent problems of uneven size: half 1-D slabs (cells
    log-uniform in 64..4096, Gauss-Legendre M in {8,16,24,32,40,48}, copy /
    vacuum ends), half 2-D slabs (nx, ny log-uniform in 32..256
    independently, S2/S4/S6 = 8/24/48 angles) with the slab's boundaries
    along x (x = 0 copies all rays, x = 1 vacuum) and periodic in y.
    Opacities as in slab1d (sigma_a = 1e-2, sigma_s = 10^U(-1,2) per cell),
    rho = 1, T = 1 live, v = 0, Crat = 10, Prat = 1, float intensities."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        if i % 2 == 0:
            n = int(round(np.exp(rng.uniform(np.log(64), np.log(4096)))))
            M = int(rng.choice([8, 16, 24, 32, 40, 48]))
            wl = slab1d(n=n, M=M, seed=int(rng.integers(1 << 30)), steps=steps)
        else:
            nx = int(round(np.exp(rng.uniform(np.log(32), np.log(256)))))
            ny = int(round(np.exp(rng.uniform(np.log(32), np.log(256)))))
            ang = str(rng.choice(["s2", "s4", "s6"]))
            N = nx * ny
            r2 = np.random.default_rng(int(rng.integers(1 << 30)))
            wl = dict(name="slab2d", shape=(1, ny, nx), dim=2, lo=(0.0, 0.0, 0.0), hi=(1.0, ny / nx, 1.0),
                      bc=((COPY, VACUUM), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC)), angles=ang, C=10.0, P=1.0,
                      gamma=5.0 / 3.0, R=1.0, cfl=0.4,
                      estimate_v=False, steps=steps, rho=np.ones(N), T=np.ones(N), v=np.zeros((3, N)),
                      sa=np.full(N, 1e-2), ss=10.0 ** r2.uniform(-1.0, 2.0, N), I0="isotropic_quarter_pi",
                      inflow={})
        wl["hold_T"] = False
        wl["precision"] = "fp32"
        out.append(wl)
    return out


def _serving_specs(nreq, seed, scale):
    """(index, angle set, side, opacity seed) of each serving request, in
    the order the stream draws them."""
    rng = np.random.default_rng(seed)
    q = 32 if scale >= 1 else 8
    for i in range(nreq):
        ang = str(rng.choice(["s4", "s8"]))
        lo, hi = (64, 512) if i % 2 == 0 else (64, 192)
        side = max(q, int(round(np.exp(rng.uniform(np.log(lo * scale), np.log(hi * scale))) / q)) * q)
        yield i, ang, side, int(rng.integers(1 << 30))


def _serving_build(i, ang, side, ro_seed, steps, cache):
    make = box2d if i % 2 == 0 else box3d
    key = (make.__name__, side)
    if key not in cache:
        cache[key] = make(n=side, angles="s4", seed=1000 + side, steps=steps, kmax=max(1.0, side / 8))
    base = cache[key]
    ro = np.random.default_rng(ro_seed)
    N = int(np.prod(base["shape"]))
    return dict(base, angles=ang, steps=steps, sa=10.0 ** ro.uniform(0.0, 3.0, N), ss=10.0 ** ro.uniform(0.0, 3.0, N))


def serving(nreq=32, seed=6, steps=200, scale=1.0):
    """Requests for the serving loop: even ones 2-D (side log-uniform in
    64..512 x scale), odd ones 3-D (side log-uniform in 64..192 x scale),
    sides rounded to multiples of 32 (8 when scale < 1), 24 or 80 angles
    (S4 / S8), gas fields as in box3d with the velocity spectrum cut at
    side/8 (at least eight cells across its shortest wavelength), each
    `steps` steps.  Density and velocity are drawn once per (dimension,
    side); every request draws its own sigma_a, sigma_s (10^U(0, 3) per
    cell), so long streams stay cheap to generate.  The arrival gaps are
    drawn by the caller."""
    cache = {}
    return [_serving_build(i, ang, side, ro, steps, cache) for i, ang, side, ro in _serving_specs(nreq, seed, scale)]


def serving_request(index, seed=6, steps=200, scale=1.0):
    """Request `index` of the serving stream alone (the same fields as
    serving() gives it)."""
    for i, ang, side, ro in _serving_specs(index + 1, seed, scale):
        if i == index:
            return _serving_build(i, ang, side, ro, steps, {})


def initial_intensity(wl, M):
    """I0 as an (M, N) array: 1/(4 pi) everywhere, or the isotropic
    equilibrium T^4/(4 pi) of the given temperature."""
    N = int(np.prod(wl["shape"]))
    if wl["I0"] == "isotropic_quarter_pi":
        return np.full((M, N), 1.0 / (4.0 * np.pi))
    return np.repeat((wl["T"] ** 4 / (4.0 * np.pi))[None, :], M, axis=0)


def inflow_values(rule, n):
    """Per-angle incoming intensity for a face: ("beam", I, axis) gives I on
    every ray with n[axis] > 0 and 0 elsewhere."""
    kind, val, axis = rule
    assert kind == "beam"
    return np.where(n[:, axis] > 0, val, 0.0)


def rounded_to_float32(wl):
    """Copy of a workload whose fields are the float32-rounded values, so the
    double-precision oracle sees exactly what a float32 device copy holds."""
    out = dict(wl)
    for k in ("rho", "v", "sa", "ss"):
        out[k] = np.asarray(wl[k], dtype=np.float32).astype(np.float64)
    return out


def by_name(name, **kw):
    return {"slab1d": slab1d, "shadow2d": shadow2d, "box3d": box3d}[name](**kw)
