"""FP64 oracle of a fourth-order-in-time scheme for the acoustic equation of
Sec. 2.4, Eq. 10 (without attenuation), and of its exact discrete gradient.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
product never imports it.  The spatial operator L, its transpose, the sponge
profile and the point-interpolation weights are the C oracle's (pinned in
tests/test_oracle_pins.py); the time stepping and its reverse sweep are
written out here in numpy, one step at a time.

The paper states only that its scheme is fourth-order accurate in time and
cites its stability constants (Sec. 2.4).  The reading taken here is the
modified-equation (Lax-Wendroff) scheme, which adds one application of the
spatial operator per step.  With m = 1/vp^2, k = (vp dt)^2, the sponge term
alpha = sigma dt / 2, the source field s^n and w^n = L u^n + s^n:

    (1 + alpha) u^{n+1} = 2 u^n - (1 - alpha) u^{n-1} + F^n,
    F^n = k w^n + (1/12) k L(k w^n) + (1/12) k (s^{n+1} - 2 s^n + s^{n-1}),

i.e. dt^2 u_tt + (dt^4 / 12) u_tttt of u_tt = (L u + s) / m, with the source's
second time derivative taken as the centred second difference of its samples
(s^{-1} = 0).  Without the sponge it is fourth-order accurate in time; in the
sponge the damping term keeps the second-order central difference.  Its
stability limit is sqrt(3) times the leapfrog's (the amplification
polynomial 1 - z/2 + z^2/24 of z = -k x eigenvalue of L stays in [-1, 1] for
z <= 12, against z <= 4), where the paper cites 0.81 (2D) and 0.66 (3D) for
its own variant: that variant is not given, so parity with those constants is
unpinned.

The gradient is the reverse sweep of the recursion above (the discrete
Lagrangian): with c^n = ubar^{n+1} / (1 + alpha),
    ubar^n += 2 c^n + G^T c^n,     ubar^{n-1} -= (1 - alpha) c^n,
    G^T c = y + (1/12) L^T(k y),   y = L^T(k c),
    dJ/dk += c (w + (1/12)(L(k w) + s^{n+1} - 2 s^n + s^{n-1})) + (1/12) y w,
and dJ/dm = -(k^2 / dt^2) dJ/dk.

Parity status: forward pinned (reduces to the C leapfrog without the
correction; fourth-order self-convergence in dt; stability at sqrt(3) times
the leapfrog limit); gradient pinned (reduces to the C oracle's without the
correction; dot-product test of G; Taylor remainder; central differences).
"""
from __future__ import annotations

import numpy as np

from . import Grid, apply_L, apply_LT, sponge
from .points import point_list as _points, source_fields as _source_fields


def _model(grid: Grid, vp):
    vp = np.asarray(vp, dtype=np.float64).reshape(-1)
    k = (vp * grid.dt) ** 2
    alpha = sponge(grid).reshape(-1) * grid.dt / 2.0
    return k, alpha


def _L(grid, f, rho):
    return apply_L(grid, f.reshape(grid.shape), rho).reshape(-1)


def _LT(grid, f, rho):
    return apply_LT(grid, f.reshape(grid.shape), rho).reshape(-1)


def forward(grid: Grid, vp, rho, src_xyz, wavelet, rec_xyz, correction=True, keep=False,
            interp=None):
    """Traces [nrec][nt] of one shot (src_xyz [nsrc][ndim], wavelet
    [nsrc][nt]); u^0 = u^{-1} = 0, d^n = P u^n.  correction=False drops the
    fourth-order terms (the leapfrog of the C oracle).  keep=True also
    returns the states u^n, [nt][N].  interp: point weights (None:
    bi-/tri-linear; see oracle.sinc)."""
    N = grid.npoints
    k, alpha = _model(grid, vp)
    S = _source_fields(grid, src_xyz, wavelet, interp)
    recs = _points(grid, rec_xyz, interp)
    traces = np.zeros((len(recs), grid.nt))
    U = np.zeros((grid.nt, N)) if keep else None
    u_prev = np.zeros(N)
    u = np.zeros(N)
    for n in range(grid.nt):
        for r, (idx, w) in enumerate(recs):
            traces[r, n] = np.dot(w, u[idx])
        if keep:
            U[n] = u
        if n == grid.nt - 1:
            break
        w_n = _L(grid, u, rho) + S[n + 1]
        F = k * w_n
        if correction:
            F += (k * _L(grid, k * w_n, rho)) / 12.0
            F += k * (S[n + 2] - 2.0 * S[n + 1] + S[n]) / 12.0
        u_new = (2.0 * u - (1.0 - alpha) * u_prev + F) / (1.0 + alpha)
        u_prev, u = u, u_new
    return (traces, U) if keep else traces


def apply_G(grid: Grid, vp, rho, x, correction=True):
    """G x = k L x + (1/12) k L(k L x): the linear part of F in u."""
    k, _ = _model(grid, vp)
    y = k * _L(grid, np.asarray(x, dtype=np.float64).reshape(-1), rho)
    if correction:
        y = y + k * _L(grid, y, rho) / 12.0
    return y


def apply_GT(grid: Grid, vp, rho, c, correction=True):
    """G^T c = L^T(k c) + (1/12) L^T(k L^T(k c))."""
    k, _ = _model(grid, vp)
    y = _LT(grid, k * np.asarray(c, dtype=np.float64).reshape(-1), rho)
    if correction:
        y = y + _LT(grid, k * y, rho) / 12.0
    return y


def gradient(grid: Grid, vp, rho, src_xyz, wavelet, rec_xyz, observed, correction=True):
    """(J, dJ/dm, traces) of one shot, J = 1/2 sum (d - d_obs)^2, m = 1/vp^2,
    by the reverse sweep of the recursion (exact for the discrete scheme)."""
    N = grid.npoints
    nt = grid.nt
    k, alpha = _model(grid, vp)
    S = _source_fields(grid, src_xyz, wavelet)
    recs = _points(grid, rec_xyz)
    d, U = forward(grid, vp, rho, src_xyz, wavelet, rec_xyz, correction, keep=True)
    r = d - np.asarray(observed, dtype=np.float64).reshape(d.shape)
    J = 0.5 * float(np.sum(r * r))

    def receiver_adjoint(n):                 # P^T r^n (weights, no cell volume)
        f = np.zeros(N)
        for q, (idx, w) in enumerate(recs):
            f[idx] += w * r[q, n]
        return f

    kbar = np.zeros(N)
    ubar_next = receiver_adjoint(nt - 1)     # ubar^{n+1}, complete
    ubar = receiver_adjoint(nt - 2) if nt >= 2 else np.zeros(N)
    for n in range(nt - 2, -1, -1):
        c = ubar_next / (1.0 + alpha)
        w_n = _L(grid, U[n], rho) + S[n + 1]
        y = _LT(grid, k * c, rho)
        GTc = y + (_LT(grid, k * y, rho) / 12.0 if correction else 0.0)
        kbar += c * w_n
        if correction:
            kbar += c * (_L(grid, k * w_n, rho) + S[n + 2] - 2.0 * S[n + 1] + S[n]) / 12.0
            kbar += y * w_n / 12.0
        ubar = ubar + 2.0 * c + GTc
        ubar_prev = receiver_adjoint(n - 1) - (1.0 - alpha) * c if n >= 1 else None
        ubar_next, ubar = ubar, ubar_prev
    g = -(k * k / grid.dt ** 2) * kbar
    return J, g.reshape(grid.shape), d


def stability_limit(ndim: int, w2) -> float:
    """Largest c dt / h of this scheme on a uniform grid: sqrt(3) x the
    leapfrog's 2 / sqrt(ndim lambda), lambda = |w2_0 + 2 sum_j (-1)^j w2_j|."""
    lam = abs(w2[0] + 2.0 * sum((-1) ** j * w2[j] for j in range(1, len(w2))))
    return float(np.sqrt(3.0) * 2.0 / np.sqrt(ndim * lam))
