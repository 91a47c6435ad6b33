"""FP64 oracle of a perfectly matched layer (PML) for the 2D acoustic
equation with constant density (Sec. 2.4 offers a PML next to the sponge,
citing an unsplit formulation), and of its exact discrete gradient with
respect to m = 1/vp^2.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
product never imports it.

Reading (the paper cites the PML without its equations): the unsplit
second-order form with one auxiliary field per axis,

    u_tt + (zx + zy) u_t + zx zy u = c^2 (lap u + div psi) + c^2 s / ...,
    psi_x,t = -zx psi_x + (zy - zx) d_x u,   psi_y,t = -zy psi_y + (zx - zy) d_y u,

with the damping profiles zx(x), zy(y) of the sponge (z = smax (delta/nb)^2,
smax = 3 c_ref ln(1000) / (2 nb h)), lap the solver's second-derivative
stencil and d_x, d_y its first-derivative stencils with zero extension.  In
time: the leapfrog with central u_t, and the auxiliary fields by the
trapezoidal rule driven by the new u:

    (1 + a) u^{n+1} = 2u^n - (1 - a) u^{n-1} - zx zy dt^2 u^n
                      + k (lap u^n + d_x psi_x^n + d_y psi_y^n + s^n),
    psi_x^{n+1} = [(1 - zx dt/2) psi_x^n + dt (zy - zx) d_x u^{n+1}] / (1 + zx dt/2),

a = (zx + zy) dt / 2, k = (vp dt)^2 (psi_y alike).  Outside the layer every
z is zero, psi stays zero and the step is the solver's leapfrog.  3D and
variable density are not covered.

Parity status: forward pinned (no layer: the C leapfrog; first-derivative
stencil antisymmetric; reflection far below the sponge's of the same width;
no late-time growth); gradient pinned (Taylor remainder; central
differences, inside the layer too).
"""
from __future__ import annotations

import numpy as np

from . import Grid, apply_L, fd_weights
from .time4 import _points, _source_fields


def profiles(grid: Grid):
    """zy, zx (1/s) on the grid: the sponge's quadratic profile per axis."""
    nb = grid.nb
    out = []
    for d in range(2):
        n, h = grid.shape[d], grid.spacing[d]
        z = np.zeros(n)
        if nb > 0:
            smax = 3.0 * grid.c_ref * np.log(1000.0) / (2.0 * nb * h)
            i = np.arange(n)
            delta = np.where(i < nb, nb - i, np.where(i > n - 1 - nb, i - (n - 1 - nb), 0))
            z = smax * (delta / nb) ** 2
        out.append(z)
    zy = np.broadcast_to(out[0][:, None], grid.shape).copy()
    zx = np.broadcast_to(out[1][None, :], grid.shape).copy()
    return zy, zx


def d1(grid: Grid, f, axis: int):
    """Central first derivative along `axis` with f = 0 outside the grid:
    (D f)_i = sum_j w1_j (f_{i+j} - f_{i-j}) / h."""
    _, w1 = fd_weights(grid.order)
    R = grid.order // 2
    h = grid.spacing[axis]
    f = np.asarray(f, dtype=np.float64).reshape(grid.shape)
    pad = [(0, 0), (0, 0)]
    pad[axis] = (R, R)
    fp = np.pad(f, pad)
    n = grid.shape[axis]
    out = np.zeros(grid.shape)
    for j in range(1, R + 1):
        up = np.take(fp, np.arange(R + j, R + j + n), axis=axis)
        dn = np.take(fp, np.arange(R - j, R - j + n), axis=axis)
        out += w1[j] * (up - dn)
    return out / h


def _setup(grid: Grid, vp):
    if grid.ndim != 2:
        raise ValueError("the PML oracle is 2D")
    zy, zx = profiles(grid)
    dt = grid.dt
    k = (np.asarray(vp, dtype=np.float64) * dt) ** 2
    a = (zx + zy) * dt / 2.0
    e = zx * zy * dt * dt
    px, qx = (1 - zx * dt / 2) / (1 + zx * dt / 2), dt * (zy - zx) / (1 + zx * dt / 2)
    py, qy = (1 - zy * dt / 2) / (1 + zy * dt / 2), dt * (zx - zy) / (1 + zy * dt / 2)
    return k, a, e, (px, qx), (py, qy)


def forward(grid: Grid, vp, src_xyz, wavelet, rec_xyz, keep=False):
    """Traces [nrec][nt] of one shot (constant density).  keep=True also
    returns the states (u, psi_x, psi_y) of every step."""
    k, a, e, (px, qx), (py, qy) = _setup(grid, vp)
    S = _source_fields(grid, src_xyz, wavelet)
    recs = _points(grid, rec_xyz)
    nt = grid.nt
    traces = np.zeros((len(recs), nt))
    hist = [] if keep else None
    u_prev = np.zeros(grid.shape)
    u = np.zeros(grid.shape)
    psx = np.zeros(grid.shape)
    psy = np.zeros(grid.shape)
    for n in range(nt):
        uf = u.reshape(-1)
        for r, (idx, w) in enumerate(recs):
            traces[r, n] = np.dot(w, uf[idx])
        if keep:
            hist.append((u, psx, psy))
        if n == nt - 1:
            break
        E = apply_L(grid, u, None) + d1(grid, psx, 1) + d1(grid, psy, 0) + S[n + 1].reshape(grid.shape)
        u_new = (2.0 * u - (1.0 - a) * u_prev - e * u + k * E) / (1.0 + a)
        psx = px * psx + qx * d1(grid, u_new, 1)
        psy = py * psy + qy * d1(grid, u_new, 0)
        u_prev, u = u, u_new
    return (traces, hist) if keep else traces


def gradient(grid: Grid, vp, src_xyz, wavelet, rec_xyz, observed):
    """(J, dJ/dm, traces) of one shot by the reverse sweep: undo the psi
    update of step n (into ubar^{n+1} and psibar^n), then the u update with
    c = ubar^{n+1} / (1 + a)."""
    k, a, e, (px, qx), (py, qy) = _setup(grid, vp)
    S = _source_fields(grid, src_xyz, wavelet)
    recs = _points(grid, rec_xyz)
    nt = grid.nt
    d, hist = forward(grid, vp, src_xyz, wavelet, rec_xyz, keep=True)
    r = d - np.asarray(observed, dtype=np.float64).reshape(d.shape)
    J = 0.5 * float(np.sum(r * r))

    def receiver_adjoint(n):
        f = np.zeros(grid.npoints)
        for q, (idx, w) in enumerate(recs):
            f[idx] += w * r[q, n]
        return f.reshape(grid.shape)

    kbar = np.zeros(grid.shape)
    ubar_next = receiver_adjoint(nt - 1)
    ubar = receiver_adjoint(nt - 2) if nt >= 2 else np.zeros(grid.shape)
    psx_bar = np.zeros(grid.shape)             # psibar^{n+1}
    psy_bar = np.zeros(grid.shape)
    for n in range(nt - 2, -1, -1):
        u_n, psx_n, psy_n = hist[n]
        u_prev = hist[n - 1][0] if n >= 1 else np.zeros(grid.shape)
        # psi^{n+1} = p psi^n + q d(u^{n+1}); d^T = -d
        ubar_next = ubar_next - d1(grid, qx * psx_bar, 1) - d1(grid, qy * psy_bar, 0)
        psx_bar, psy_bar = px * psx_bar, py * psy_bar
        # u^{n+1} = [2u^n - (1-a) u^{n-1} - e u^n + k E^n] / (1 + a)
        c = ubar_next / (1.0 + a)
        E = apply_L(grid, u_n, None) + d1(grid, psx_n, 1) + d1(grid, psy_n, 0) + S[n + 1].reshape(grid.shape)
        kbar += c * E
        kc = k * c
        ubar = ubar + (2.0 - e) * c + apply_L(grid, kc, None)     # the stencil is symmetric
        psx_bar = psx_bar - d1(grid, kc, 1)
        psy_bar = psy_bar - d1(grid, kc, 0)
        ubar_prev = receiver_adjoint(n - 1) - (1.0 - a) * c if n >= 1 else None
        ubar_next, ubar = ubar, ubar_prev
    g = -(k * k / grid.dt ** 2) * kbar
    return J, g, d
