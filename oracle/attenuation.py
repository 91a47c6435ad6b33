"""FP64 oracle of the attenuating acoustic equation of Sec. 2.4, Eq. 10,

    (1/vp^2) p_tt = rho div(rho^-1 grad p) + eta d/dt (-lap)^(y/2) p + s,
    eta = -2 alpha0 vp^(y-1),  y in {0, 2},

on the leapfrog scheme of the rest of the oracle, and of its exact discrete
gradient with respect to m = 1/vp^2 (alpha0 held fixed).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
product never imports it.  The spatial operators, the sponge and the point
weights are the C oracle's; the time stepping and its reverse sweep are
written out here in numpy.

Readings (the paper gives the equation, not its discretisation):
  * y = 0: eta p_t = -(2 alpha0 / vp) p_t is a damping term and takes the
    sponge's central difference; dividing by m it adds a = alpha0 vp dt to
    the sponge's sigma dt / 2:
        (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} + k (L u^n + s^n).
  * y = 2: eta d/dt (-lap) p = 2 alpha0 vp d/dt lap p with the plain
    (constant-density) Laplacian of the same order, its time derivative
    taken backwards, (lap u^n - lap u^{n-1}) / dt, which keeps the step
    explicit (a central difference would couple u^{n+1} in space):
        (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1}
                          + k (L u^n + s^n + beta (lap u^n - lap u^{n-1}) / dt),
        beta = 2 alpha0 vp.
  With k = (vp dt)^2 and a = sigma dt / 2 (+ alpha0 vp dt for y = 0).  For a
  plane wave of angular frequency w both give the power-law attenuation
  alpha0 w^y (nepers per metre) when alpha0 vp / w and alpha0 vp w are small.

Parity status: forward pinned (alpha0 = 0 is the C leapfrog; the measured
decay of a narrowband wave is alpha0 w^y for y = 0 and 2); gradient pinned
(alpha0 = 0 is the C oracle's; Taylor remainder; central differences in m
for both y, with and without density, in the interior and in the sponge).
"""
from __future__ import annotations

import numpy as np

from . import Grid, apply_L, apply_LT, sponge
from .points import point_list as _points, source_fields as _source_fields


def _ops(grid: Grid, rho):
    def L(f):
        return apply_L(grid, f.reshape(grid.shape), rho).reshape(-1)

    def LT(f):
        return apply_LT(grid, f.reshape(grid.shape), rho).reshape(-1)

    def lap(f):                               # plain Laplacian: symmetric
        return apply_L(grid, f.reshape(grid.shape), None).reshape(-1)

    return L, LT, lap


def _coefficients(grid: Grid, vp, alpha0, y):
    vp = np.asarray(vp, dtype=np.float64).reshape(-1)
    al = np.broadcast_to(np.asarray(alpha0, dtype=np.float64), (grid.npoints,)).reshape(-1)
    k = (vp * grid.dt) ** 2
    a = sponge(grid).reshape(-1) * grid.dt / 2.0
    beta = np.zeros_like(vp)
    if y == 0:
        a = a + al * vp * grid.dt
    elif y == 2:
        beta = 2.0 * al * vp
    else:
        raise ValueError("y must be 0 or 2")
    return vp, al, k, a, beta


def forward(grid: Grid, vp, rho, alpha0, y, src_xyz, wavelet, rec_xyz, keep=False, interp=None):
    """Traces [nrec][nt] of one shot (src_xyz [nsrc][ndim], wavelet
    [nsrc][nt]); alpha0 is a scalar or a field (nepers per metre, at unit
    angular frequency for y = 2).  keep=True also returns u^n, [nt][N].
    interp: point weights (None: bi-/tri-linear; see oracle.sinc)."""
    N = grid.npoints
    _, _, k, a, beta = _coefficients(grid, vp, alpha0, y)
    L, _, lap = _ops(grid, rho)
    S = _source_fields(grid, src_xyz, wavelet, interp)
    recs = _points(grid, rec_xyz, interp)
    traces = np.zeros((len(recs), grid.nt))
    U = np.zeros((grid.nt, N)) if keep else None
    u_prev = np.zeros(N)
    u = np.zeros(N)
    lap_prev = np.zeros(N)
    for n in range(grid.nt):
        for r, (idx, w) in enumerate(recs):
            traces[r, n] = np.dot(w, u[idx])
        if keep:
            U[n] = u
        if n == grid.nt - 1:
            break
        E = L(u) + S[n + 1]
        if y == 2:
            lap_u = lap(u)
            E = E + beta * (lap_u - lap_prev) / grid.dt
            lap_prev = lap_u
        u_new = (2.0 * u - (1.0 - a) * u_prev + k * E) / (1.0 + a)
        u_prev, u = u, u_new
    return (traces, U) if keep else traces


def gradient(grid: Grid, vp, rho, alpha0, y, src_xyz, wavelet, rec_xyz, observed, interp=None):
    """(J, dJ/dm, traces) of one shot by the reverse sweep of the recursion:
    with c = ubar^{n+1} / (1 + a),
        ubar^n     += 2c + L^T(k c) + lap(beta k c) / dt,
        ubar^{n-1} -= (1 - a) c + lap(beta k c) / dt,
        kbar += c E^n,  abar += ubar^{n+1} (u^{n-1} - u^{n+1}) / (1 + a),
        betabar += c k (lap u^n - lap u^{n-1}) / dt,
    then dJ/dvp = 2 vp dt^2 kbar + (y = 0: alpha0 dt abar; y = 2: 2 alpha0 betabar)
    and dJ/dm = -(vp^3 / 2) dJ/dvp."""
    N = grid.npoints
    nt = grid.nt
    dt = grid.dt
    vpf, al, k, a, beta = _coefficients(grid, vp, alpha0, y)
    L, LT, lap = _ops(grid, rho)
    S = _source_fields(grid, src_xyz, wavelet, interp)
    recs = _points(grid, rec_xyz, interp)
    d, U = forward(grid, vp, rho, alpha0, y, src_xyz, wavelet, rec_xyz, keep=True, interp=interp)
    r = d - np.asarray(observed, dtype=np.float64).reshape(d.shape)
    J = 0.5 * float(np.sum(r * r))

    def receiver_adjoint(n):
        f = np.zeros(N)
        for q, (idx, w) in enumerate(recs):
            f[idx] += w * r[q, n]
        return f

    kbar = np.zeros(N)
    abar = np.zeros(N)
    bbar = np.zeros(N)
    ubar_next = receiver_adjoint(nt - 1)
    ubar = receiver_adjoint(nt - 2) if nt >= 2 else np.zeros(N)
    for n in range(nt - 2, -1, -1):
        u_prev = U[n - 1] if n >= 1 else np.zeros(N)
        u_next = U[n + 1]
        c = ubar_next / (1.0 + a)
        E = L(U[n]) + S[n + 1]
        ubar = ubar + 2.0 * c + LT(k * c)
        extra = np.zeros(N)
        if y == 2:
            dlap = (lap(U[n]) - lap(u_prev)) / dt
            E = E + beta * dlap
            bbar += c * k * dlap
            t = lap(beta * k * c) / dt
            ubar = ubar + t
            extra = -t
        kbar += c * E
        abar += ubar_next * (u_prev - u_next) / (1.0 + a)
        ubar_prev = receiver_adjoint(n - 1) - (1.0 - a) * c + extra if n >= 1 else None
        ubar_next, ubar = ubar, ubar_prev
    gvp = 2.0 * vpf * dt * dt * kbar
    if y == 0:
        gvp += al * dt * abar
    else:
        gvp += 2.0 * al * bbar
    g = -(vpf ** 3 / 2.0) * gvp
    return J, g.reshape(grid.shape), d
