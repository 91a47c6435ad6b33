"""FP64 CPU oracle for the Stride acoustic FWI hot path (arXiv 2110.03345).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product library never
imports, links or runs it, and it imports nothing from the product package.

The discrete scheme lives in ``fwi_oracle.c`` (plain C, FP64, loops written
point by point; Sec. 2.4 Eq. 10 for the PDE, Sec. 2.2 Eqs. 5-9 for the
adjoint-state gradient).  This module is a thin ctypes shim around it plus the
closed-form homogeneous Green's functions used to pin the physics (Sec. 3.1).

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
  forward        pinned: analytic 2D/3D Green's function, 2nd-order time
                 convergence, reciprocity, linearity, superposition of
                 off-grid sources, energy conservation without sponge.
  adjoint        pinned: dot-product test (exact to rounding).
  gradient       pinned: Taylor test (second-order remainder), central
                 finite differences, checkpointed == full-history.
  apply_L/LT     pinned: smooth analytic fields, operator dot-product test.
  sponge         pinned only by invariants (energy decay, small reflection);
                 the profile itself is a reading of a citation-only passage.

Submodules: ``inversion`` (the inversion loop of Sec. 2.3 / 3.2), ``time4``
(a fourth-order-in-time scheme and its gradient), ``attenuation`` (the
power-law attenuation term of Eq. 10 and its gradient), ``sinc``
(Kaiser-windowed sinc interpolation of off-grid points) and ``pml`` (a
perfectly matched layer in 2D and 3D and its gradient), each with its own parity status
in its header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_liboracle.so (gcc, OpenMP, strict IEEE)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _CGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_long * 3),
                ("h", ctypes.c_double * 3), ("order", ctypes.c_int),
                ("nb", ctypes.c_int), ("c_ref", ctypes.c_double),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            d = P(ctypes.c_double)
            g = P(_CGrid)
            lib.orc_fd_weights.argtypes = [ctypes.c_int, d, d]
            lib.orc_sponge.argtypes = [g, d]
            lib.orc_apply_L.argtypes = [g, d, d, d]
            lib.orc_apply_LT.argtypes = [g, d, d, d]
            lib.orc_point_weights.argtypes = [g, d, P(ctypes.c_long), d]
            lib.orc_point_weights.restype = ctypes.c_int
            lib.orc_forward.argtypes = [g, d, d, ctypes.c_int, d, d, ctypes.c_int, d, d, d]
            lib.orc_adjoint_sources.argtypes = [g, d, d, ctypes.c_int, d, d,
                                                ctypes.c_int, d, d]
            lib.orc_gradient.argtypes = [g, d, d, ctypes.c_int, d, d, ctypes.c_int, d, d,
                                         d, d, d, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Grid:
    """Regular grid, time axis and solver options (Sec. 2.3 Listing 5, Sec. 2.4).

    shape/spacing list the axes slowest first (z, y, x or y, x)."""
    shape: tuple
    spacing: tuple
    dt: float
    nt: int
    order: int = 8
    nb: int = 20
    c_ref: float = 1500.0
    ndim: int = field(init=False)

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.ndim = len(self.shape)
        if isinstance(self.spacing, (int, float)):
            self.spacing = (float(self.spacing),) * self.ndim
        self.spacing = tuple(float(s) for s in self.spacing)
        assert self.ndim in (2, 3) and len(self.spacing) == self.ndim

    def c(self) -> _CGrid:
        cg = _CGrid()
        cg.ndim = self.ndim
        n = (1,) * (3 - self.ndim) + self.shape
        h = (1.0,) * (3 - self.ndim) + self.spacing
        for i in range(3):
            cg.n[i] = n[i]
            cg.h[i] = h[i]
        cg.order, cg.nb, cg.c_ref = self.order, self.nb, float(self.c_ref)
        cg.dt, cg.nt = float(self.dt), int(self.nt)
        return cg

    @property
    def npoints(self) -> int:
        return int(np.prod(self.shape))


def fd_weights(order: int):
    """(w2[0..R], w1[0..R]) used by the oracle's stencils."""
    lib = _load()
    w2 = np.zeros(6)
    w1 = np.zeros(6)
    lib.orc_fd_weights(order, _ptr(w2), _ptr(w1))
    R = order // 2
    return w2[:R + 1].copy(), w1[:R + 1].copy()


def sponge(grid: Grid) -> np.ndarray:
    lib = _load()
    out = np.zeros(grid.shape)
    lib.orc_sponge(ctypes.byref(grid.c()), _ptr(out))
    return out


def apply_L(grid: Grid, u, rho=None) -> np.ndarray:
    lib = _load()
    u = _f64(u)
    rho = _f64(rho)
    out = np.zeros(grid.shape)
    lib.orc_apply_L(ctypes.byref(grid.c()), _ptr(rho), _ptr(u), _ptr(out))
    return out


def apply_LT(grid: Grid, v, rho=None) -> np.ndarray:
    lib = _load()
    v = _f64(v)
    rho = _f64(rho)
    out = np.zeros(grid.shape)
    lib.orc_apply_LT(ctypes.byref(grid.c()), _ptr(rho), _ptr(v), _ptr(out))
    return out


def point_weights(grid: Grid, xyz):
    """Flat node indices and weights of the bi-/tri-linear stencil of one point."""
    lib = _load()
    xyz = _f64(np.asarray(xyz).reshape(grid.ndim))
    idx = np.zeros(8, dtype=np.int64)
    w = np.zeros(8)
    nc = lib.orc_point_weights(ctypes.byref(grid.c()), _ptr(xyz),
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _ptr(w))
    return idx[:nc].copy(), w[:nc].copy()


def _shot_arrays(grid, src_xyz, wavelet, nshots=None):
    src_xyz = _f64(src_xyz)
    wavelet = _f64(wavelet)
    if src_xyz.ndim == 2:       # one shot
        src_xyz = src_xyz[None]
        wavelet = wavelet[None]
    assert src_xyz.shape[-1] == grid.ndim
    assert wavelet.shape[:2] == src_xyz.shape[:2] and wavelet.shape[2] == grid.nt
    return src_xyz, wavelet


def forward(grid: Grid, vp, rho, src_xyz, wavelet, rec_xyz, acc_hist=False):
    """Traces [nshots][nrec][nt] for each shot (src_xyz [nshots][nsrc][ndim],
    wavelet [nshots][nsrc][nt], rec_xyz [nrec][ndim] shared by all shots).
    With acc_hist=True (one shot only) also returns a^n, shape [nt-1, *shape]."""
    lib = _load()
    vp, rho, rec_xyz = _f64(vp), _f64(rho), _f64(rec_xyz)
    src_xyz, wavelet = _shot_arrays(grid, src_xyz, wavelet)
    ns, nsrc = src_xyz.shape[:2]
    nrec = rec_xyz.shape[0]
    out = np.zeros((ns, nrec, grid.nt))
    hist = None
    if acc_hist:
        assert ns == 1
        hist = np.zeros((max(grid.nt - 1, 0),) + grid.shape)
    cg = grid.c()
    for s in range(ns):
        lib.orc_forward(ctypes.byref(cg), _ptr(vp), _ptr(rho), nsrc, _ptr(src_xyz[s]),
                        _ptr(wavelet[s]), nrec, _ptr(rec_xyz), _ptr(out[s]), _ptr(hist))
    return (out, hist) if acc_hist else out


def adjoint_sources(grid: Grid, vp, rho, rec_xyz, resid, src_xyz):
    """Adjoint of the linear map wavelet -> traces: resid [nrec][nt] -> [nsrc][nt]."""
    lib = _load()
    vp, rho, rec_xyz, resid, src_xyz = map(_f64, (vp, rho, rec_xyz, resid, src_xyz))
    out = np.zeros((src_xyz.shape[0], grid.nt))
    lib.orc_adjoint_sources(ctypes.byref(grid.c()), _ptr(vp), _ptr(rho), rec_xyz.shape[0],
                            _ptr(rec_xyz), _ptr(resid), src_xyz.shape[0], _ptr(src_xyz),
                            _ptr(out))
    return out


def gradient(grid: Grid, vp, rho, src_xyz, wavelet, rec_xyz, observed, ckpt_every=0,
             shots=None):
    """(J, g, traces): L2 misfit summed over shots, its gradient with respect to
    the squared slowness m = 1/vp^2 (shape of the grid) and the modelled traces.
    ckpt_every > 0 recomputes the forward history from checkpoints (same
    arithmetic, less memory).  `shots` restricts the sum to a subset."""
    lib = _load()
    vp, rho, rec_xyz, observed = map(_f64, (vp, rho, rec_xyz, observed))
    src_xyz, wavelet = _shot_arrays(grid, src_xyz, wavelet)
    if observed.ndim == 2:
        observed = observed[None]
    ns, nsrc = src_xyz.shape[:2]
    nrec = rec_xyz.shape[0]
    shots = range(ns) if shots is None else shots
    g = np.zeros(grid.shape)
    traces = np.zeros((ns, nrec, grid.nt))
    J = 0.0
    cg = grid.c()
    for s in shots:
        js = ctypes.c_double(0.0)
        lib.orc_gradient(ctypes.byref(cg), _ptr(vp), _ptr(rho), nsrc, _ptr(src_xyz[s]),
                         _ptr(wavelet[s]), nrec, _ptr(rec_xyz),
                         _ptr(np.ascontiguousarray(observed[s])), ctypes.byref(js), _ptr(g),
                         _ptr(traces[s]), int(ckpt_every))
        J += js.value
    return J, g, traces


# ---------------------------------------------------------------------------
# Closed-form homogeneous Green's functions (Sec. 3.1), for the operator
#     (1/c^2) p_tt - lap p = q(t) delta(x),  q(t) = 0 for t < 0.
# ---------------------------------------------------------------------------

def analytic_3d(q, r, t, c):
    """p(r, t) = q(t - r/c) / (4 pi r); q is a callable of time."""
    tau = np.asarray(t, dtype=np.float64) - r / c
    return np.where(tau >= 0.0, q(np.maximum(tau, 0.0)), 0.0) / (4.0 * np.pi * r)


def analytic_2d(q, r, t, c, nquad=2000):
    """p(r, t) = (1/2pi) int_0^inf q(t - (r/c) cosh xi) dxi  (singularity-free form
    of the 2D Green's function convolved with q).  Gauss-Legendre quadrature on
    [0, acosh(c t / r)] split into panels."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    xg, wg = np.polynomial.legendre.leggauss(16)
    for i, ti in enumerate(t):
        if ti * c <= r:
            continue
        xmax = np.arccosh(ti * c / r)
        npan = max(8, int(nquad // 16))
        edges = np.linspace(0.0, xmax, npan + 1)
        a, b = edges[:-1, None], edges[1:, None]
        xi = 0.5 * (b - a) * xg[None, :] + 0.5 * (b + a)
        tau = ti - (r / c) * np.cosh(xi)
        vals = np.where(tau >= 0.0, q(np.maximum(tau, 0.0)), 0.0)
        out[i] = np.sum(0.5 * (b - a) * wg[None, :] * vals) / (2.0 * np.pi)
    return out


def analytic_2d_freq(q_samples, dt, r, c, pad=8):
    """Frequency-domain 2D Green's function: P(w) = Q(w) (i/4) H0^(1)(w r / c) for
    the e^{-i w t} convention, evaluated by FFT of the sampled q (independent
    cross-check of analytic_2d)."""
    from scipy.special import hankel1
    n = len(q_samples) * pad
    Q = np.fft.rfft(q_samples, n) * dt              # int q(t) e^{+i w t} dt with numpy's sign
    w = 2.0 * np.pi * np.fft.rfftfreq(n, dt)
    G = np.zeros_like(Q)
    nz = w > 0
    # numpy's forward FFT uses e^{-i w t}; the causal Green's function in that
    # convention is the complex conjugate of (i/4) H0^(1).
    G[nz] = np.conj(0.25j * hankel1(0, w[nz] * r / c))
    p = np.fft.irfft(Q * G, n) / dt
    return p[:len(q_samples)]
