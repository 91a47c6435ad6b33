"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: models (sound speed, density), transducer
coordinates and source wavelets.  It holds none of the solver's arithmetic and
is shared by the tests, the benchmark, the CUDA path and the oracle alike.

The paper's datasets (the numerical breast database and MIDA head of Sec. 3.2
and 3.3, the PVA phantom recordings, the kWave/ITRUSST results of Sec. 3.1) are
not available; the phantoms below take their shapes, spacings and property
ranges instead:

  * ``config_homogeneous_2d``: the homogeneous accuracy setup of Sec. 3.1 on a
    256^2 grid at 0.2 mm with a Ricker source (the paper used a tone burst).
  * ``config_breast_2d``: a 2D breast-like slice (Sec. 3.2): water, an
    ellipse of fatty tissue holding 20-40 random inclusions, smoothed noise,
    a 256-element ring array; every second element fires.
  * ``config_skull_3d``: a 3D head-like model (Sec. 3.3): water, an
    ellipsoidal skull shell and soft-tissue interior, transducers on a
    Fibonacci sphere (the Fibonacci layout of Sec. 3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def ricker(f0: float, dt: float, nt: int, t0: float | None = None, amp: float = 1.0):
    """Ricker wavelet r(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0."""
    t0 = 1.5 / f0 if t0 is None else t0
    t = np.arange(nt) * dt - t0
    a = (np.pi * f0 * t) ** 2
    return amp * (1.0 - 2.0 * a) * np.exp(-a)


def ricker_fn(f0: float, t0: float | None = None, amp: float = 1.0):
    """The same wavelet as a function of continuous time (for analytic checks)."""
    t0 = 1.5 / f0 if t0 is None else t0

    def q(t):
        a = (np.pi * f0 * (np.asarray(t) - t0)) ** 2
        return amp * (1.0 - 2.0 * a) * np.exp(-a)
    return q


def ring(n: int, centre, radius: float, rotation: float = 0.0):
    """n points on a circle, turned by `rotation` element pitches; coordinates
    in axis order (y, x)."""
    th = 2.0 * np.pi * (np.arange(n) + rotation) / n
    return np.stack([centre[0] + radius * np.sin(th), centre[1] + radius * np.cos(th)], 1)


def fibonacci_sphere(n: int, centre, radius: float):
    """n nearly uniform points on a sphere (Fibonacci spiral); axis order (z, y, x)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    phi = np.pi * (1.0 + 5.0 ** 0.5) * k
    pts = np.stack([z, r * np.sin(phi), r * np.cos(phi)], 1)
    return np.asarray(centre)[None, :] + radius * pts


def cfl_dt(dx: float, c_max: float, cfl: float = 0.4) -> float:
    return cfl * dx / c_max


@dataclass
class Problem:
    """One synthetic problem: model, geometry, wavelets and time axis.

    vp, rho: float64 arrays of the grid shape (slowest axis first).
    src_xyz: [nshots][nsrc][ndim] metres; rec_xyz: [nrec][ndim] metres (shared).
    wavelet: [nshots][nsrc][nt]."""
    name: str
    shape: tuple
    spacing: float
    dt: float
    nt: int
    order: int
    nb: int
    vp: np.ndarray
    rho: np.ndarray | None
    src_xyz: np.ndarray
    rec_xyz: np.ndarray
    wavelet: np.ndarray
    c_ref: float = 1500.0
    vp_true: np.ndarray | None = None   # model that generates observed data
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def nshots(self):
        return self.src_xyz.shape[0]

    @property
    def npoints(self):
        return int(np.prod(self.shape))


def config_homogeneous_2d(n=256, dx=0.2e-3, nt=1000, nrec=64, radius=20e-3, f0=500e3,
                          c=1500.0, rho=1000.0, order=8, nb=20, variable_density=False):
    """Homogeneous 2D setup: on-node Ricker source at the centre node, a ring of
    receivers (default: 256^2, 0.2 mm, 64 receivers at 20 mm, 1000 steps)."""
    dt = cfl_dt(dx, c)
    shape = (n, n)
    vp = np.full(shape, c)
    rh = np.full(shape, rho) if variable_density else None
    ctr = (n // 2) * dx
    src = np.array([[[ctr, ctr]]])
    rec = ring(nrec, (ctr, ctr), radius)
    wav = ricker(f0, dt, nt)[None, None, :]
    return Problem("homogeneous_2d", shape, dx, dt, nt, order, nb, vp, rh, src, rec, wav,
                   c_ref=c)


def _ellipse_mask(Y, X, cy, cx, ay, ax, theta):
    ct, st = math.cos(theta), math.sin(theta)
    yy, xx = Y - cy, X - cx
    u = ct * xx + st * yy
    v = -st * xx + ct * yy
    return (u / ax) ** 2 + (v / ay) ** 2 <= 1.0


def _smooth(a, sigma_pts):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma_pts, mode="nearest")


def breast_model_2d(n: int, dx: float, seed: int, scale: float = 1.0, fat_vp=(1430.0, 1470.0),
                    incl_vp=(1400.0, 1600.0)):
    """Breast-like 2D slice: water (1500 m/s, 1000 kg/m^3); an ellipse of fatty
    tissue (semi-axes ~35-40 mm x scale, c ~ U[fat_vp]) holding 20-40 random
    inclusions with c ~ U[incl_vp] (default [1400, 1600]), rho ~ U[950, 1100];
    smoothed noise of std 5 m/s; clipped to [1400, 1600] / [950, 1100].
    Returns (vp, rho)."""
    rng = np.random.default_rng(seed)
    y = (np.arange(n) + 0.5 - n / 2) * dx
    Y, X = np.meshgrid(y, y, indexing="ij")
    vp = np.full((n, n), 1500.0)
    rho = np.full((n, n), 1000.0)
    ay, ax = rng.uniform(35e-3, 40e-3, 2) * scale
    breast = _ellipse_mask(Y, X, 0.0, 0.0, ay, ax, rng.uniform(0, np.pi))
    vp[breast] = rng.uniform(*fat_vp)
    rho[breast] = rng.uniform(950, 980)
    for _ in range(int(rng.integers(20, 41))):
        r = math.sqrt(rng.uniform(0.0, 1.0)) * 0.8
        ang = rng.uniform(0, 2 * np.pi)
        cy, cx = r * ay * math.sin(ang), r * ax * math.cos(ang)
        sy, sx = rng.uniform(2e-3, 15e-3, 2) * scale
        m = _ellipse_mask(Y, X, cy, cx, sy, sx, rng.uniform(0, np.pi)) & breast
        vp[m] = rng.uniform(*incl_vp)
        rho[m] = rng.uniform(950, 1100)
    noise = _smooth(rng.standard_normal((n, n)), 0.5e-3 / dx)
    noise *= 5.0 / max(noise.std(), 1e-12)
    vp = np.where(breast, vp + noise, vp)
    vp = np.clip(vp, 1400.0, 1600.0)
    rho = np.clip(rho, 950.0, 1100.0)
    return vp, rho


def gaussian_blobs(shape, dx, seed, n=3, amp=20.0, sigma=3e-3, extent=0.3):
    """Sum of n Gaussian blobs of amplitude +-amp m/s and width sigma, centres
    within +-extent of the domain size about the centre."""
    rng = np.random.default_rng(seed)
    axes = [(np.arange(s) + 0.5 - s / 2) * dx for s in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    out = np.zeros(shape)
    L = np.array(shape) * dx
    for _ in range(n):
        c = rng.uniform(-extent, extent, len(shape)) * L
        a = amp * rng.choice([-1.0, 1.0])
        r2 = sum((g - ci) ** 2 for g, ci in zip(grids, c))
        out += a * np.exp(-0.5 * r2 / sigma ** 2)
    return out


def breast_problem(shape, dx, nt, nelem=256, shots=None, order=8, nb=20, seed=2, f0=500e3,
                   c_max=1600.0, radius=None, perturb_seed=20, fat_vp=(1430.0, 1470.0),
                   incl_vp=(1400.0, 1600.0), rotation=0.0):
    """Breast-like 2D problem on a (possibly non-square) grid: the phantom of
    ``breast_model_2d`` scaled to the smaller side and centre-cropped, a ring of
    ``nelem`` elements about the centre (default radius: 0.4395 x the smaller
    side, i.e. 45 mm on a 1024 x 0.1 mm grid); shots fire the
    given elements (default every second one); all elements receive.  The
    observed-data model adds 3 Gaussian blobs (+-20 m/s, 3 mm x scale).
    rotation turns the whole array by that many element pitches (a rotated
    acquisition with the same phantom)."""
    ny, nx = (int(s) for s in shape)
    m, full = min(ny, nx), max(ny, nx)
    scale = m * dx / (1024 * 0.1e-3)
    vpf, rhof = breast_model_2d(full, dx, seed, scale=scale, fat_vp=fat_vp, incl_vp=incl_vp)
    oy, ox = (full - ny) // 2, (full - nx) // 2
    vp = vpf[oy:oy + ny, ox:ox + nx].copy()
    rho = rhof[oy:oy + ny, ox:ox + nx].copy()
    dt = cfl_dt(dx, c_max)
    ctr = ((ny / 2) * dx, (nx / 2) * dx)
    rad = 0.4395 * m * dx if radius is None else radius
    elems = ring(nelem, ctr, rad, rotation)
    fire = np.arange(0, nelem, 2) if shots is None else np.asarray(shots)
    src = elems[fire][:, None, :]
    w = ricker(f0, dt, nt)
    wav = np.broadcast_to(w, (len(fire), 1, nt)).copy()
    blobs = gaussian_blobs((full, full), dx, perturb_seed, sigma=3e-3 * scale)[oy:oy + ny, ox:ox + nx]
    vp_true = np.clip(vp + blobs, 1400.0, 1600.0)
    return Problem("breast_2d", (ny, nx), dx, dt, nt, order, nb, vp, rho, src, elems, wav,
                   c_ref=c_max, vp_true=vp_true)


def config_breast_2d(n=1024, dx=0.1e-3, nt=4000, nelem=256, radius=45e-3, f0=500e3,
                     order=8, nb=20, seed=2, shots=None, c_max=1600.0, rotation=0.0):
    """Breast-like 2D problem: n^2 grid, 256-element ring of radius 45 mm (scaled
    with n dx) about the centre; shots fire elements 0, 2, ..., all elements
    receive.  The observed-data model is the phantom plus 3 Gaussian blobs
    (+-20 m/s, 3 mm, seed 20).  Defaults are the full-size workload (1024^2,
    0.1 mm, 128 shots of 4000 steps, dt = 25 ns)."""
    scale = n * dx / (1024 * 0.1e-3)
    return breast_problem((n, n), dx, nt, nelem=nelem, shots=shots, order=order, nb=nb,
                          seed=seed, f0=f0, c_max=c_max, radius=radius * scale, rotation=rotation)


def skull_model_3d(n: int, dx: float, scale: float = 1.0):
    """Head-like 3D model: water; an ellipsoidal skull shell with outer
    semi-axes (20, 23, 19) mm x scale and 6 mm x scale thickness (2800 m/s,
    1900 kg/m^3) around soft tissue (1540 m/s, 1040 kg/m^3)."""
    z = (np.arange(n) + 0.5 - n / 2) * dx
    Z, Y, X = np.meshgrid(z, z, z, indexing="ij")
    a = np.array([20e-3, 23e-3, 19e-3]) * scale
    t = 6e-3 * scale
    outer = (Z / a[0]) ** 2 + (Y / a[1]) ** 2 + (X / a[2]) ** 2 <= 1.0
    inner = (Z / (a[0] - t)) ** 2 + (Y / (a[1] - t)) ** 2 + (X / (a[2] - t)) ** 2 <= 1.0
    vp = np.full((n, n, n), 1500.0)
    rho = np.full((n, n, n), 1000.0)
    vp[outer] = 2800.0
    rho[outer] = 1900.0
    vp[inner] = 1540.0
    rho[inner] = 1040.0
    return vp, rho


def skull_problem(shape, dx, nt, nrec=512, every=16, order=10, nb=20, f0=500e3, c_max=2800.0,
                  radius=None, shots=None, perturb_seed=30):
    """Head-like 3D problem on a (possibly non-cubic) grid: the model of
    ``skull_model_3d`` scaled to the smallest side and centre-cropped,
    ``nrec`` receivers on a Fibonacci sphere (default radius 25 mm x scale),
    shots firing every ``every``-th receiver.  Observed-data model: Gaussian
    blobs (+-20 m/s, 3 mm x scale) in the soft tissue."""
    shape = tuple(int(s) for s in shape)
    m, full = min(shape), max(shape)
    scale = m * dx / (256 * 0.25e-3)
    vpf, rhof = skull_model_3d(full, dx, scale)
    o = [(full - s) // 2 for s in shape]
    sl = tuple(slice(oi, oi + s) for oi, s in zip(o, shape))
    vp, rho = vpf[sl].copy(), rhof[sl].copy()
    dt = cfl_dt(dx, c_max)
    ctr = tuple((s / 2) * dx for s in shape)
    rad = 25e-3 * scale if radius is None else radius
    rec = fibonacci_sphere(nrec, ctr, rad)
    fire = np.arange(0, nrec, every) if shots is None else np.asarray(shots)
    src = rec[fire][:, None, :]
    w = ricker(f0, dt, nt)
    wav = np.broadcast_to(w, (len(fire), 1, nt)).copy()
    inner = (vp == 1540.0)
    blobs = gaussian_blobs((full,) * 3, dx, perturb_seed, sigma=3e-3 * scale)[sl]
    vp_true = np.where(inner, vp + blobs, vp)
    return Problem("skull_3d", shape, dx, dt, nt, order, nb, vp, rho, src, rec, wav,
                   c_ref=c_max, vp_true=vp_true)


def config_skull_3d(n=256, dx=0.25e-3, nt=2000, nrec=512, every=16, radius=25e-3,
                    f0=500e3, order=10, nb=20, c_max=2800.0, shots=None):
    """3D skull problem: n^3 grid, 512 receivers on a Fibonacci sphere of
    radius 25 mm (scaled with n dx); 32 shots fire every 16th receiver.
    Defaults are the full size (256^3, 0.25 mm, 2000 steps, dt = 35.71 ns)."""
    scale = n * dx / (256 * 0.25e-3)
    return skull_problem((n, n, n), dx, nt, nrec=nrec, every=every, order=order, nb=nb, f0=f0,
                         c_max=c_max, radius=radius * scale, shots=shots)


def config_uneven_batch(nprob=64, seed=4, side=(256, 1024), nt=(500, 4000), shots=(1, 16),
                        dx=0.1e-3, order=8, nb=20, nelem=64, f0=500e3):
    """Uneven set of independent 2D problems: square grids with side drawn
    uniformly from `side` (multiples of 4), time axes from `nt`, shot counts
    from `shots`; breast-like models as in ``breast_problem`` scaled to a ring
    of radius 0.42 x side x dx; dt at CFL 0.4 of 1600 m/s."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        n = 4 * int(rng.integers(side[0] // 4, side[1] // 4 + 1))
        steps = int(rng.integers(nt[0], nt[1] + 1))
        ns = int(rng.integers(shots[0], shots[1] + 1))
        fire = np.linspace(0, nelem, ns, endpoint=False).astype(int)
        p = breast_problem((n, n), dx, steps, nelem=nelem, shots=fire, order=order, nb=nb,
                           seed=seed * 1000 + i, f0=f0, radius=0.42 * n * dx)
        out.append(p)
    return out


def config_serving(nreq=650, seed=5, rate=20.0, frac_2d=0.75, frac_fwd=0.5,
                   side2d=(512, 1024), side3d=(128, 192), nt=(1000, 3000)):
    """Request stream for the serving pattern: Poisson arrivals (mean `rate`
    per second), 75% 2D (side ~ U[512, 1024], multiple of 4, dx 0.1 mm,
    breast-like) and 25% 3D (side ~ U[128, 192], dx 0.25 mm, skull-like),
    half forward and half gradient, one shot each, nt ~ U[1000, 3000].
    Returns a list of (arrival time in s, kind, Problem)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(nreq):
        t += rng.exponential(1.0 / rate)
        two_d = rng.uniform() < frac_2d
        kind = "forward" if rng.uniform() < frac_fwd else "gradient"
        steps = int(rng.integers(nt[0], nt[1] + 1))
        if two_d:
            n = 4 * int(rng.integers(side2d[0] // 4, side2d[1] // 4 + 1))
            shot = [int(rng.integers(0, 64))]
            p = breast_problem((n, n), 0.1e-3, steps, nelem=64, shots=shot, nb=20,
                               seed=5000 + (i % 8), radius=0.42 * n * 0.1e-3)
        else:
            n = 4 * int(rng.integers(side3d[0] // 4, side3d[1] // 4 + 1))
            p = skull_problem((n, n, n), 0.25e-3, steps, nrec=128, every=128,
                              shots=[int(rng.integers(0, 128))], nb=16)
        out.append((t, kind, p))
    return out


def random_smooth_model(shape, dx, seed, c_range=(1400.0, 1600.0), rho_range=(950.0, 1100.0),
                        sigma=1e-3):
    """Smooth random heterogeneous model (for parity tests on small grids)."""
    rng = np.random.default_rng(seed)
    sp = sigma / dx
    a = _smooth(rng.standard_normal(shape), sp)
    b = _smooth(rng.standard_normal(shape), sp)
    a = (a - a.min()) / max(a.max() - a.min(), 1e-12)
    b = (b - b.min()) / max(b.max() - b.min(), 1e-12)
    vp = c_range[0] + (c_range[1] - c_range[0]) * a
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * b
    return vp, rho


def random_points(n, shape, dx, seed, margin):
    """n random off-grid points at least `margin` grid points inside each edge."""
    rng = np.random.default_rng(seed)
    lo = margin * dx
    hi = (np.array(shape) - 1 - margin) * dx
    return rng.uniform(lo, hi, (n, len(shape)))


# ---------------------------------------------------------------------------
# Inversion workload (the 2D imaging experiment of Sec. 3.2)
# ---------------------------------------------------------------------------

def tone_burst(f0: float, dt: float, nt: int, cycles: int = 3, t0: float = 0.0,
               amp: float = 1.0):
    """`cycles`-cycle tone burst centred at f0 starting at t0: a sine of
    frequency f0 under a Hann envelope that spans the burst, zero elsewhere."""
    tau = np.arange(nt) * dt - t0
    T = cycles / f0
    on = (tau >= 0.0) & (tau <= T)
    env = 0.5 * (1.0 - np.cos(2.0 * np.pi * tau / T))
    return np.where(on, amp * np.sin(2.0 * np.pi * f0 * tau) * env, 0.0)


def shot_schedule(nshots: int, per_iter: int, nblocks: int, seed: int):
    """Random shot subsets without replacement (Sec. 3.2): for each block a
    fresh permutation of the shots, cut into iterations of `per_iter` shots
    (the last one shorter when per_iter does not divide nshots), so every
    shot is used once per block.  Returns [block][iteration] -> int64 ids."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nblocks):
        perm = rng.permutation(nshots).astype(np.int64)
        out.append([perm[i:i + per_iter] for i in range(0, nshots, per_iter)])
    return out


def disk_mask(shape, dx, centre, radius):
    """1 inside the disk (or ball) of the given centre and radius, 0 outside."""
    axes = [np.arange(s) * dx for s in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
    return (r2 <= radius * radius).astype(np.float64)


def config_inversion_2d(scale: float = 1.0, shape=(456, 485), dx=0.5e-3, dt=0.08e-6, nt=2500,
                        nelem=128, f0=500e3, freqs=(300e3, 400e3, 500e3, 600e3), per_iter=16,
                        c_start=1500.0, order=8, nb=20, seed=2, schedule_seed=7,
                        filter_cycles=3.0, fat_vp=(1480.0, 1495.0), incl_vp=(1440.0, 1560.0)):
    """The 2D breast imaging experiment of Sec. 3.2 with a synthetic phantom:
    456 x 485 grid at 0.5 mm, 128 ring transducers that all fire and receive,
    a 3-cycle tone burst at 500 kHz, 2500 steps of 0.08 us, constant density,
    a starting model of 1500 m/s, frequency blocks from 300 to 600 kHz with 16
    shots per iteration drawn without replacement (8 iterations per block).

    The phantom is ``breast_problem``'s with fatty tissue at U[fat_vp] =
    U[1480, 1495] m/s and inclusions at U[incl_vp] = U[1440, 1560] m/s, so
    that travel times through the breast from the 1500 m/s start stay within
    about half a period of the first (300 kHz) block, as the paper's start
    must have been for its first block to converge.

    ``scale`` > 1 keeps the domain and the phantom and divides the grid and
    the frequencies by `scale` (spacing, step and period x scale): the same
    points per wavelength and CFL number on a smaller grid, with the phantom
    `scale` times fewer wavelengths across (an easier, cheaper inversion).
    The record keeps its 200 us while the burst delay and a block filter's
    reach grow with `scale`, so beyond scale 4 they take most of it.
    The tone burst starts after filter_cycles periods of the lowest block
    frequency, so a zero-phase low-pass of that length sees the whole burst.
    ``extra`` holds freqs, schedule, mask (update region: the disk 5 points
    inside the ring) and filter_cycles."""
    s = float(scale)
    shp = tuple(int(round(n / s)) for n in shape)
    dx, dt, f0 = dx * s, dt * s, f0 / s
    freqs = tuple(f / s for f in freqs)
    nt = int(round(nt / s))
    base = breast_problem(shp, dx, nt, nelem=nelem, shots=np.arange(nelem), order=order, nb=nb,
                          seed=seed, f0=f0, c_max=1600.0, fat_vp=fat_vp, incl_vp=incl_vp)
    t0 = filter_cycles / min(freqs)
    w = tone_burst(f0, dt, nt, t0=t0)
    wav = np.broadcast_to(w, (nelem, 1, nt)).copy()
    ny, nx = shp
    ctr = ((ny / 2) * dx, (nx / 2) * dx)
    ring_r = float(np.hypot(*(base.rec_xyz[0] - np.array(ctr))))
    mask = disk_mask(shp, dx, ctr, ring_r - 5 * dx)
    sched = shot_schedule(nelem, per_iter, len(freqs), schedule_seed)
    return Problem("inversion_2d", shp, dx, dt, nt, order, nb, np.full(shp, float(c_start)),
                   None, base.src_xyz, base.rec_xyz, wav, c_ref=1600.0, vp_true=base.vp,
                   extra={"freqs": freqs, "schedule": sched, "mask": mask,
                          "filter_cycles": float(filter_cycles)})
