"""FP64 oracle of a perfectly matched layer (PML) for the acoustic equation
in 2D and 3D (Sec. 2.4 offers a PML next to the sponge, citing an unsplit
formulation), and of its exact discrete gradient with respect to m = 1/vp^2.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
product never imports it.

Reading (the paper cites the PML without its equations): the unsplit
second-order form obtained from the coordinate stretching
d_j -> d_j / (1 + z_j / p) (p the time derivative), multiplied through by
the product of the stretchings.  With the per-axis damping profiles z_j (the
sponge's: z = smax (delta/nb)^2, smax = 3 c_ref ln(1000) / (2 nb h_j)), an
integral field q (q_t = u) and one auxiliary field phi_j per axis,

    u_tt + (sum z) u_t + (sum_{j<l} z_j z_l) u + (prod z) q = c^2 (lap u + sum_j d_j phi_j),
    phi_j,t = -z_j phi_j + (z_k + z_l - z_j) d_j u + z_k z_l d_j q,

k, l the other axes (in 2D z_l = 0: the q terms vanish), lap the solver's
second-derivative stencil, d_j its first-derivative stencil with zero
extension.  In time: the leapfrog with central u_t; q^{n+1} = q^n + dt u^{n+1};
phi by the trapezoidal rule driven by the new u and q:

    (1 + a) u^{n+1} = 2u^n - (1 - a) u^{n-1} - e u^n - f q^n
                      + k (lap u^n + sum_j d_j phi_j^n + s^n),
    phi_j^{n+1} = [(1 - z_j dt/2) phi_j^n
                   + dt ((z_k + z_l - z_j) d_j u^{n+1} + z_k z_l d_j q^{n+1})] / (1 + z_j dt/2),

a = (sum z) dt / 2, e = (sum_{j<l} z_j z_l) dt^2, f = (prod z) dt^2,
k = (vp dt)^2.  Outside the layer every z is zero, phi and the q term
vanish, and the step is the solver's leapfrog.  With variable density, lap
becomes the solver's rho div(rho^-1 grad): the density must be constant
over the layer and the stencil reach next to it (checked), where the two
operators coincide.

Parity status: forward pinned (no layer: the C leapfrog in 2D and 3D, with
and without density; first-derivative stencil antisymmetric; reflection far
below the sponge's of the same width in 2D and 3D; no late-time growth);
gradient pinned (Taylor remainder; central differences inside and outside
the layer, 2D and 3D, with and without density).
"""
from __future__ import annotations

import numpy as np

from . import Grid, apply_L, apply_LT, fd_weights
from .points import point_list as _points, source_fields as _source_fields


def profiles(grid: Grid):
    """[z_0, ..., z_{ndim-1}] (1/s) on the grid, axis order slowest first:
    the sponge's quadratic profile along each axis."""
    nb = grid.nb
    out = []
    for d in range(grid.ndim):
        n, h = grid.shape[d], grid.spacing[d]
        z = np.zeros(n)
        if nb > 0:
            smax = 3.0 * grid.c_ref * np.log(1000.0) / (2.0 * nb * h)
            i = np.arange(n)
            delta = np.where(i < nb, nb - i, np.where(i > n - 1 - nb, i - (n - 1 - nb), 0))
            z = smax * (delta / nb) ** 2
        shape = [1] * grid.ndim
        shape[d] = n
        out.append(np.broadcast_to(z.reshape(shape), grid.shape).copy())
    return out


def d1(grid: Grid, f, axis: int):
    """Central first derivative along `axis` with f = 0 outside the grid:
    (D f)_i = sum_j w1_j (f_{i+j} - f_{i-j}) / h."""
    _, w1 = fd_weights(grid.order)
    R = grid.order // 2
    h = grid.spacing[axis]
    f = np.asarray(f, dtype=np.float64).reshape(grid.shape)
    pad = [(0, 0)] * grid.ndim
    pad[axis] = (R, R)
    fp = np.pad(f, pad)
    n = grid.shape[axis]
    out = np.zeros(grid.shape)
    for j in range(1, R + 1):
        up = np.take(fp, np.arange(R + j, R + j + n), axis=axis)
        dn = np.take(fp, np.arange(R - j, R - j + n), axis=axis)
        out += w1[j] * (up - dn)
    return out / h


def _coefficients(grid: Grid, vp):
    z = profiles(grid)
    nd = grid.ndim
    dt = grid.dt
    zero = np.zeros(grid.shape)
    zs = z + [zero] * (3 - nd)                 # pad to three axes (2D: z_l = 0)
    k = (np.asarray(vp, dtype=np.float64).reshape(grid.shape) * dt) ** 2
    a = sum(z) * dt / 2.0
    e = (zs[0] * zs[1] + zs[0] * zs[2] + zs[1] * zs[2]) * dt * dt
    f = zs[0] * zs[1] * zs[2] * dt * dt
    axes = []
    for j in range(nd):
        o = [zs[i] for i in range(3) if i != j]
        den = 1.0 + z[j] * dt / 2.0
        axes.append(((1.0 - z[j] * dt / 2.0) / den,          # p_j
                     dt * (o[0] + o[1] - z[j]) / den,         # b_j: weight of d_j u
                     dt * o[0] * o[1] / den))                 # g_j: weight of d_j q
    return k, a, e, f, axes


def _check_density(grid: Grid, rho):
    """rho must be constant where any z is nonzero or within the stencil reach."""
    if rho is None or grid.nb == 0:
        return
    rho = np.asarray(rho, dtype=np.float64).reshape(grid.shape)
    reach = grid.nb + grid.order // 2
    inner = tuple(slice(reach, n - reach) for n in grid.shape)
    band = np.ones(grid.shape, dtype=bool)
    band[inner] = False
    vals = rho[band]
    if vals.size and np.ptp(vals) > 1e-12 * np.abs(vals).max():
        raise ValueError("the density must be constant over the PML and the stencil reach")


def _rhs(grid, u, phi, s, rho=None):
    E = apply_L(grid, u, rho) + s
    for j, ph in enumerate(phi):
        E = E + d1(grid, ph, j)
    return E


def forward(grid: Grid, vp, src_xyz, wavelet, rec_xyz, keep=False, rho=None):
    """Traces [nrec][nt] of one shot (rho None: constant density).  keep=True
    also returns the states (u, q, phi) of every step."""
    _check_density(grid, rho)
    k, a, e, f, axes = _coefficients(grid, vp)
    S = _source_fields(grid, src_xyz, wavelet)
    recs = _points(grid, rec_xyz)
    nt = grid.nt
    traces = np.zeros((len(recs), nt))
    hist = [] if keep else None
    u_prev = np.zeros(grid.shape)
    u = np.zeros(grid.shape)
    q = np.zeros(grid.shape)
    phi = [np.zeros(grid.shape) for _ in range(grid.ndim)]
    for n in range(nt):
        uf = u.reshape(-1)
        for r, (idx, w) in enumerate(recs):
            traces[r, n] = np.dot(w, uf[idx])
        if keep:
            hist.append((u, q, phi))
        if n == nt - 1:
            break
        E = _rhs(grid, u, phi, S[n + 1].reshape(grid.shape), rho)
        u_new = (2.0 * u - (1.0 - a) * u_prev - e * u - f * q + k * E) / (1.0 + a)
        q_new = q + grid.dt * u_new
        phi = [p * ph + b * d1(grid, u_new, j) + gq * d1(grid, q_new, j)
               for j, (ph, (p, b, gq)) in enumerate(zip(phi, axes))]
        u_prev, u, q = u, u_new, q_new
    return (traces, hist) if keep else traces


def gradient(grid: Grid, vp, src_xyz, wavelet, rec_xyz, observed, rho=None):
    """(J, dJ/dm, traces) of one shot by the reverse sweep.  For step n:
    undo phi^{n+1} (into ubar^{n+1}, qbar^{n+1}, phibar^n), then
    q^{n+1} = q^n + dt u^{n+1}, then the u update with c = ubar^{n+1}/(1 + a)
    (d_j^T = -d_j; the transpose of the solver's operator is the C oracle's
    L^T)."""
    k, a, e, f, axes = _coefficients(grid, vp)
    S = _source_fields(grid, src_xyz, wavelet)
    recs = _points(grid, rec_xyz)
    nt = grid.nt
    dt = grid.dt
    d, hist = forward(grid, vp, src_xyz, wavelet, rec_xyz, keep=True, rho=rho)
    r = d - np.asarray(observed, dtype=np.float64).reshape(d.shape)
    J = 0.5 * float(np.sum(r * r))

    def receiver_adjoint(n):
        out = np.zeros(grid.npoints)
        for i, (idx, w) in enumerate(recs):
            out[idx] += w * r[i, n]
        return out.reshape(grid.shape)

    zero = np.zeros(grid.shape)
    kbar = np.zeros(grid.shape)
    ubar_next = receiver_adjoint(nt - 1)
    ubar = receiver_adjoint(nt - 2) if nt >= 2 else zero.copy()
    qbar_next = zero.copy()                          # qbar^{n+1}
    phibar = [zero.copy() for _ in range(grid.ndim)]  # phibar^{n+1}
    for n in range(nt - 2, -1, -1):
        u_n, q_n, phi_n = hist[n]
        # phi_j^{n+1} = p_j phi_j^n + b_j d_j u^{n+1} + g_j d_j q^{n+1}
        for j, (p, b, gq) in enumerate(axes):
            ubar_next = ubar_next - d1(grid, b * phibar[j], j)
            qbar_next = qbar_next - d1(grid, gq * phibar[j], j)
            phibar[j] = p * phibar[j]
        # q^{n+1} = q^n + dt u^{n+1}
        ubar_next = ubar_next + dt * qbar_next
        qbar = qbar_next                             # becomes qbar^n below
        # u^{n+1} = [2u^n - (1-a) u^{n-1} - e u^n - f q^n + k E^n] / (1 + a)
        c = ubar_next / (1.0 + a)
        kbar += c * _rhs(grid, u_n, phi_n, S[n + 1].reshape(grid.shape), rho)
        kc = k * c
        ubar = ubar + (2.0 - e) * c + apply_LT(grid, kc, rho)
        qbar = qbar - f * c
        phibar = [pb - d1(grid, kc, j) for j, pb in enumerate(phibar)]
        ubar_prev = receiver_adjoint(n - 1) - (1.0 - a) * c if n >= 1 else None
        ubar_next, ubar, qbar_next = ubar, ubar_prev, qbar
    g = -(k * k / dt ** 2) * kbar
    return J, g, d
