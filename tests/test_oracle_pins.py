"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake in the oracle (a wrong stencil weight,
sign, index shift, transposed operand, dropped term or scaling):

  stencil weights      Fornberg's algorithm in exact rationals; polynomial exactness
  L and L^T            smooth analytic fields; operator dot-product test
  forward physics      closed-form homogeneous Green's functions in 2D and 3D
                       (Sec. 3.1), second-order convergence in dt
  source/receiver      superposition of on-node sources reproduces an off-grid one
  adjoint              dot-product test of wavelet -> traces (exact to rounding)
  gradient             Taylor remainder O(h^2); central finite differences
  reciprocity          constant density: exact; variable density: approximate
  stability            leapfrog limit 2/sqrt(d*lambda_max) of the stencil
  sponge               energy conservation without it, decay and weak
                       reflection with it
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2110_03345_gb300 import inputs


# ---------------------------------------------------------------- helpers

def fornberg(x0, xs, m):
    """Finite-difference weights for the m-th derivative at x0 on nodes xs (exact)."""
    n = len(xs)
    c = [[[Fraction(0)] * (m + 1) for _ in range(n)] for _ in range(n)]
    c[0][0][0] = Fraction(1)
    c1 = Fraction(1)
    c4 = xs[0] - x0
    for i in range(1, n):
        mn = min(i, m)
        c2 = Fraction(1)
        c5 = c4
        c4 = xs[i] - x0
        for j in range(i):
            c3 = xs[i] - xs[j]
            c2 *= c3
            if j == i - 1:
                for k in range(mn, 0, -1):
                    c[i][i][k] = c1 * (k * c[i - 1][i - 1][k - 1] - c5 * c[i - 1][i - 1][k]) / c2
                c[i][i][0] = -c1 * c5 * c[i - 1][i - 1][0] / c2
            for k in range(mn, 0, -1):
                c[i][j][k] = (c4 * c[i - 1][j][k] - k * c[i - 1][j][k - 1]) / c3
            c[i][j][0] = c4 * c[i - 1][j][0] / c3
        c1 = c2
    return [c[n - 1][j][m] for j in range(n)]


def small_problem(shape=(40, 48), nt=120, dx=0.5e-3, nb=8, order=8, seed=0, nsrc=2, nrec=5,
                  vd=True):
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    c_max = vp.max()
    dt = 0.4 * dx / c_max
    g = oracle.Grid(shape, dx, dt=dt, nt=nt, order=order, nb=nb, c_ref=1500.0)
    src = inputs.random_points(nsrc, shape, dx, seed + 1, margin=nb + 2)
    rec = inputs.random_points(nrec, shape, dx, seed + 2, margin=nb + 2)
    return g, vp, (rho if vd else None), src, rec


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ---------------------------------------------------------------- stencils

@pytest.mark.parametrize("order", [8, 10])
def test_fd_weights_match_fornberg(order):
    R = order // 2
    xs = [Fraction(j) for j in range(-R, R + 1)]
    d2 = fornberg(Fraction(0), xs, 2)
    d1 = fornberg(Fraction(0), xs, 1)
    w2, w1 = oracle.fd_weights(order)
    for j in range(R + 1):
        assert w2[j] == pytest.approx(float(d2[R + j]), rel=1e-15, abs=1e-16)
    for j in range(1, R + 1):
        assert w1[j] == pytest.approx(float(d1[R + j]), rel=1e-15, abs=1e-16)
    # exactness on monomials up to degree order+1 (second derivative) / order (first)
    for p in range(order + 2):
        s2 = sum(w2[abs(j)] * float(j) ** p for j in range(-R, R + 1))
        assert s2 == pytest.approx(p * (p - 1) if p == 2 else 0.0, abs=1e-9)
    for p in range(order + 1):
        s1 = sum(np.sign(j) * w1[abs(j)] * float(j) ** p for j in range(-R, R + 1))
        assert s1 == pytest.approx(1.0 if p == 1 else 0.0, abs=1e-9)


@pytest.mark.parametrize("order", [8, 10])
def test_leapfrog_stability_limit(order):
    """The scheme is stable just below 2/sqrt(d*lambda_max) and blows up just above
    (lambda_max = |sum_j (-1)^j w2_j|, the checkerboard eigenvalue of the stencil)."""
    w2, _ = oracle.fd_weights(order)
    R = order // 2
    lam = abs(w2[0] + 2 * sum((-1) ** j * w2[j] for j in range(1, R + 1)))
    limit = 2.0 / np.sqrt(2 * lam)
    n, dx, c = 24, 1e-3, 1500.0
    rng = np.random.default_rng(3)
    out = {}
    for fac in (0.98, 1.04):
        dt = fac * limit * dx / c
        g = oracle.Grid((n, n), dx, dt=dt, nt=600, order=order, nb=0)
        w = rng.standard_normal((1, 1, g.nt))
        src = np.array([[[10.3e-3, 11.7e-3]]])
        rec = np.array([[12e-3, 12e-3]])
        tr = oracle.forward(g, np.full((n, n), c), None, src, w, rec)
        out[fac] = np.abs(tr).max()
    assert np.isfinite(out[0.98]) and out[0.98] < 1e3
    assert not np.isfinite(out[1.04]) or out[1.04] > 1e12


def _smooth_fields(shape, h):
    axes = [np.arange(n) * h for n in shape]
    X = np.meshgrid(*axes, indexing="ij")
    L = [n * h for n in shape]
    k = [2 * np.pi * (1.3 + 0.4 * d) / Ld for d, Ld in enumerate(L)]
    u = np.ones(shape)
    for d in range(len(shape)):
        u = u * np.sin(k[d] * X[d] + 0.3 * d)
    lap = -sum(kd * kd for kd in k) * u
    grads = []
    for d in range(len(shape)):
        gd = np.ones(shape)
        for e in range(len(shape)):
            gd = gd * (k[e] * np.cos(k[e] * X[e] + 0.3 * e) if e == d else
                       np.sin(k[e] * X[e] + 0.3 * e))
        grads.append(gd)
    # ln rho = 0.2 * prod cos(q_d x_d): smooth density, analytic gradient
    q = [2 * np.pi * 0.7 / Ld for Ld in L]
    lr = 0.2 * np.ones(shape)
    for d in range(len(shape)):
        lr = lr * np.cos(q[d] * X[d])
    lr_grads = []
    for d in range(len(shape)):
        gd = 0.2 * np.ones(shape)
        for e in range(len(shape)):
            gd = gd * (-q[e] * np.sin(q[e] * X[e]) if e == d else np.cos(q[e] * X[e]))
        lr_grads.append(gd)
    return u, lap, grads, np.exp(lr), lr_grads


@pytest.mark.parametrize("shape", [(48, 56), (28, 30, 32)])
@pytest.mark.parametrize("order", [8, 10])
def test_apply_L_on_smooth_fields(shape, order):
    """L_rho u = lap u - grad ln rho . grad u on smooth fields, checked away from
    the edges (the zero extension there is a boundary condition, not the PDE)."""
    h = 1e-3
    g = oracle.Grid(shape, h, dt=1e-7, nt=2, order=order, nb=0)
    u, lap, grads, rho, lrg = _smooth_fields(shape, h)
    inner = tuple(slice(2 * (order // 2), n - 2 * (order // 2)) for n in shape)
    Lcd = oracle.apply_L(g, u)
    assert rel(Lcd[inner], lap[inner]) < 1e-6
    Lvd = oracle.apply_L(g, u, rho)
    expect = lap - sum(a * b for a, b in zip(lrg, grads))
    assert rel(Lvd[inner], expect[inner]) < 1e-6
    # a sign error on the advective term would be O(1) off
    wrong = lap + sum(a * b for a, b in zip(lrg, grads))
    assert rel(Lvd[inner], wrong[inner]) > 1e-2


@pytest.mark.parametrize("shape", [(17, 19), (9, 11, 13)])
@pytest.mark.parametrize("order", [8, 10])
def test_operator_transpose(shape, order):
    rng = np.random.default_rng(5)
    g = oracle.Grid(shape, (1e-3,) * len(shape), dt=1e-7, nt=2, order=order, nb=0)
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    rho = 1000 * np.exp(0.3 * rng.standard_normal(shape))
    for r in (None, rho):
        lhs = np.vdot(oracle.apply_L(g, u, r), v)
        rhs = np.vdot(u, oracle.apply_LT(g, v, r))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
    # variable density: L is not symmetric (L^T differs from L)
    assert rel(oracle.apply_L(g, v, rho), oracle.apply_LT(g, v, rho)) > 1e-3


# ---------------------------------------------------------------- physics

def _analytic_run_2d(cfl, n=200, r_cells=50, T=14e-6):
    c, dx, f0 = 1500.0, 0.2e-3, 500e3
    dt = cfl * dx / c
    nt = int(round(T / dt)) + 1
    g = oracle.Grid((n, n), dx, dt=dt, nt=nt, order=8, nb=20, c_ref=c)
    ctr = (n // 2) * dx
    src = np.array([[[ctr, ctr]]])
    rec = np.array([[ctr, ctr + r_cells * dx], [ctr - r_cells * dx, ctr]])
    w = inputs.ricker(f0, dt, nt)[None, None]
    tr = oracle.forward(g, np.full((n, n), c), None, src, w, rec)[0]
    t = np.arange(nt) * dt
    an = oracle.analytic_2d(inputs.ricker_fn(f0), r_cells * dx, t, c)
    return tr, an


def nrmse(x, ref):
    return float(np.sqrt(np.mean((x - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))


def test_analytic_2d_quadrature_matches_hankel():
    """The time-domain 2D Green's function equals the Hankel-function form."""
    c, dt, f0, r = 1500.0, 2e-8, 500e3, 10e-3
    nt = 800
    t = np.arange(nt) * dt
    a = oracle.analytic_2d(inputs.ricker_fn(f0), r, t, c)
    b = oracle.analytic_2d_freq(inputs.ricker(f0, dt, nt), dt, r, c)
    assert nrmse(b, a) < 1e-4


def test_analytic_2d_and_convergence():
    """Sec. 3.1: homogeneous medium vs the analytic solution; the error falls
    by ~4x per halving of dt (second order in time dominates)."""
    errs = []
    for cfl in (0.4, 0.2, 0.1):
        tr, an = _analytic_run_2d(cfl)
        errs.append(nrmse(tr[0], an))
        assert np.allclose(tr[0], tr[1], rtol=0, atol=1e-12 * np.abs(tr[0]).max())
    assert errs[0] < 5e-2
    for a, b in zip(errs[:-1], errs[1:]):
        assert 3.3 < a / b < 4.7


def test_analytic_3d_and_convergence():
    c, dx, f0 = 1500.0, 0.2e-3, 500e3
    n, nb, rc = 80, 10, 10
    errs = []
    for cfl in (0.4, 0.2):
        dt = cfl * dx / c
        nt = int(round(7e-6 / dt)) + 1
        g = oracle.Grid((n, n, n), dx, dt=dt, nt=nt, order=10, nb=nb, c_ref=c)
        ctr = (n // 2) * dx
        src = np.array([[[ctr, ctr, ctr]]])
        rec = np.array([[ctr, ctr, ctr + rc * dx], [ctr + rc * dx, ctr, ctr]])
        w = inputs.ricker(f0, dt, nt)[None, None]
        tr = oracle.forward(g, np.full((n, n, n), c), None, src, w, rec)[0]
        t = np.arange(nt) * dt
        an = oracle.analytic_3d(inputs.ricker_fn(f0), rc * dx, t, c)
        tref = (2 * (n // 2 - nb) * dx - rc * dx) / c   # first sponge echo
        m = t < tref
        errs.append(nrmse(tr[0][m], an[m]))
        assert np.allclose(tr[0], tr[1], rtol=0, atol=1e-12 * np.abs(tr[0]).max())
    assert errs[0] < 3e-2
    assert 3.3 < errs[0] / errs[1] < 4.7


def test_symmetry_centred_source():
    """Homogeneous model on an odd grid, on-node centred source: receivers related by the grid's
    symmetries (90-degree rotations, mirror) record identical traces."""
    p = inputs.config_homogeneous_2d(n=97, dx=0.2e-3, nt=200, nrec=16, radius=6e-3, nb=10)
    g = oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=8, nb=p.nb, c_ref=1500.0)
    tr = oracle.forward(g, p.vp, None, p.src_xyz, p.wavelet, p.rec_xyz)[0]
    scale = np.abs(tr).max()
    for k in range(1, 16):
        if k % 4 == 0:
            assert np.abs(tr[k] - tr[0]).max() < 1e-10 * scale
    assert np.abs(tr[1] - tr[15]).max() < 1e-10 * scale   # mirror y -> -y
    assert np.abs(tr[1] - tr[3]).max() < 1e-10 * scale    # mirror about the diagonal


def test_linearity():
    g, vp, rho, src, rec = small_problem()
    rng = np.random.default_rng(1)
    q = rng.standard_normal((1, len(src), g.nt))
    t1 = oracle.forward(g, vp, rho, src[None], q, rec)
    t2 = oracle.forward(g, vp, rho, src[None], 2.0 * q, rec)
    assert rel(t2, 2.0 * t1) < 1e-14
    t0 = oracle.forward(g, vp, rho, src[None], 0.0 * q, rec)
    assert np.all(t0 == 0.0)


def test_offgrid_source_superposition():
    """A source at fractional position (i+fy, j+fx) equals the bilinear
    combination of four on-node sources; the same for receivers."""
    g, vp, rho, _, _ = small_problem()
    h = g.spacing[0]
    fy, fx = 0.3, 0.8
    i, j = 20, 23
    w = inputs.ricker(2e5, g.dt, g.nt)[None, None]
    rec = np.array([[12.25 * h, 30.6 * h], [27.0 * h, 14.0 * h]])
    off = oracle.forward(g, vp, rho, np.array([[[(i + fy) * h, (j + fx) * h]]]), w, rec)[0]
    comb = np.zeros_like(off)
    for dy, wy in ((0, 1 - fy), (1, fy)):
        for dx_, wx in ((0, 1 - fx), (1, fx)):
            on = oracle.forward(g, vp, rho, np.array([[[(i + dy) * h, (j + dx_) * h]]]), w, rec)[0]
            comb += wy * wx * on
    assert rel(off, comb) < 1e-12
    # receivers: sampling at a fractional point = bilinear mix of on-node traces
    src = np.array([[[20.0 * h, 20.0 * h]]])
    r_off = np.array([[(i + fy) * h, (j + fx) * h]])
    r_on = np.array([[(i + a) * h, (j + b) * h] for a in (0, 1) for b in (0, 1)])
    t_off = oracle.forward(g, vp, rho, src, w, r_off)[0, 0]
    t_on = oracle.forward(g, vp, rho, src, w, r_on)[0]
    mix = ((1 - fy) * (1 - fx) * t_on[0] + (1 - fy) * fx * t_on[1]
           + fy * (1 - fx) * t_on[2] + fy * fx * t_on[3])
    assert rel(t_off, mix) < 1e-12


def test_point_weights_layout():
    g = oracle.Grid((10, 12, 14), 1.0, dt=1e-3, nt=2, nb=0)
    idx, w = oracle.point_weights(g, [2.25, 3.5, 4.75])
    assert w.sum() == pytest.approx(1.0)
    expect = {}
    for a, wa in ((2, 0.75), (3, 0.25)):
        for b, wb in ((3, 0.5), (4, 0.5)):
            for c, wc in ((4, 0.25), (5, 0.75)):
                expect[(a * 12 + b) * 14 + c] = wa * wb * wc
    got = dict(zip(idx.tolist(), w.tolist()))
    assert got == pytest.approx(expect)


# ---------------------------------------------------------------- reciprocity

def test_reciprocity_constant_density():
    g, vp, _, src, rec = small_problem(vd=False, nsrc=2)
    w = inputs.ricker(2e5, g.dt, g.nt)[None, None]
    A, B = src[0], src[1]
    ab = oracle.forward(g, vp, None, A[None, None], w, B[None])[0, 0]
    ba = oracle.forward(g, vp, None, B[None, None], w, A[None])[0, 0]
    assert rel(ab, ba) < 1e-12


def test_reciprocity_variable_density_approximate():
    """rho_A p_A(B) = rho_B p_B(A) (p_X(Y): field at Y from a source at X; the
    operator divided by rho is symmetric) holds only up to discretisation error
    for the expanded, non-symmetric density operator."""
    shape, dx = (64, 64), 0.5e-3
    vp, rho = inputs.random_smooth_model(shape, dx, 7, sigma=3e-3)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=260, order=8, nb=10)
    A = np.array([20 * dx, 22 * dx])
    B = np.array([44 * dx, 40 * dx])
    w = inputs.ricker(1.5e5, g.dt, g.nt)[None, None]
    ab = oracle.forward(g, vp, rho, A[None, None], w, B[None])[0, 0]
    ba = oracle.forward(g, vp, rho, B[None, None], w, A[None])[0, 0]
    rA, rB = rho[20, 22], rho[44, 40]
    assert rel(rA * ab, rB * ba) < 1e-2
    # the unweighted relation is visibly worse: the density weighting matters
    assert rel(ab, ba) > 2 * rel(rA * ab, rB * ba)


def test_variable_density_with_constant_rho_equals_constant_density():
    g, vp, _, src, rec = small_problem()
    w = inputs.ricker(2e5, g.dt, g.nt)[None, None].repeat(len(src), 1)
    a = oracle.forward(g, vp, None, src[None], w, rec)
    b = oracle.forward(g, vp, np.full(vp.shape, 1234.5), src[None], w, rec)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- adjoint & gradient

@pytest.mark.parametrize("shape,order", [((40, 48), 8), ((40, 48), 10), ((18, 20, 22), 10)])
@pytest.mark.parametrize("vd", [False, True])
def test_dot_product(shape, order, vd):
    nb = 6 if len(shape) == 3 else 8
    g, vp, rho, src, rec = small_problem(shape=shape, order=order, nb=nb, vd=vd,
                                         nt=80 if len(shape) == 3 else 120)
    rng = np.random.default_rng(11)
    q = rng.standard_normal((len(src), g.nt))
    y = rng.standard_normal((len(rec), g.nt))
    Fq = oracle.forward(g, vp, rho, src[None], q[None], rec)[0]
    Fty = oracle.adjoint_sources(g, vp, rho, rec, y, src)
    lhs, rhs = np.vdot(Fq, y), np.vdot(q, Fty)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def _misfit(g, vp, rho, src, w, rec, obs):
    d = oracle.forward(g, vp, rho, src, w, rec)
    return 0.5 * float(np.sum((d - obs) ** 2))


def _grad_setup(shape=(40, 48), vd=True, order=8, nt=140, nb=8):
    g, vp, rho, src, rec = small_problem(shape=shape, vd=vd, order=order, nt=nt,
                                         nsrc=2, nrec=6, nb=nb)
    w = np.stack([inputs.ricker(2.5e5, g.dt, g.nt)] * 2)[:, None, :]   # 2 shots, 1 source each
    src = src[:, None, :]
    idx = np.indices(shape).astype(float)
    ctr = (np.array(shape, dtype=float) / 2).reshape((-1,) + (1,) * len(shape))
    r2 = ((idx - ctr) ** 2).sum(0)
    vp_true = vp * (1.0 + 0.03 * np.exp(-r2 / 30.0))
    obs = oracle.forward(g, vp_true, rho, src, w, rec)
    return g, vp, rho, src, w, rec, obs


def test_misfit_definition():
    g, vp, rho, src, w, rec, obs = _grad_setup()
    J, grad, d = oracle.gradient(g, vp, rho, src, w, rec, obs)
    assert J == pytest.approx(0.5 * np.sum((d - obs) ** 2), rel=1e-14)
    assert J > 0


def test_taylor_second_order():
    """|J(m + h dm) - J(m) - h <g, dm>| = O(h^2) for the squared slowness m."""
    g, vp, rho, src, w, rec, obs = _grad_setup()
    J0, grad, _ = oracle.gradient(g, vp, rho, src, w, rec, obs)
    m = 1.0 / vp ** 2
    rng = np.random.default_rng(4)
    dm = m * rng.standard_normal(m.shape) * 0.1
    hs = np.array([1e-1, 5e-2, 2.5e-2, 1.25e-2])
    rem = []
    for h in hs:
        Jh = _misfit(g, 1.0 / np.sqrt(m + h * dm), rho, src, w, rec, obs)
        rem.append(abs(Jh - J0 - h * np.vdot(grad, dm)))
    slopes = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes
    # first-order remainder without the gradient term would have slope 1
    lin = [abs(_misfit(g, 1.0 / np.sqrt(m + h * dm), rho, src, w, rec, obs) - J0) for h in hs[:2]]
    assert abs(np.log(lin[0] / lin[1]) / np.log(2) - 1.0) < 0.2


@pytest.mark.parametrize("vd", [False, True])
def test_gradient_central_differences(vd):
    g, vp, rho, src, w, rec, obs = _grad_setup(vd=vd)
    J0, grad, _ = oracle.gradient(g, vp, rho, src, w, rec, obs)
    m = 1.0 / vp ** 2
    rng = np.random.default_rng(8)
    pts = [tuple(rng.integers(10, s - 10) for s in vp.shape) for _ in range(3)]
    pts.append((3, 4))   # inside the sponge: the gradient is defined there too
    for p in pts:
        h = 1e-4 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_misfit(g, 1 / np.sqrt(mp), rho, src, w, rec, obs)
              - _misfit(g, 1 / np.sqrt(mm), rho, src, w, rec, obs)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=1e-6, abs=1e-9 * np.abs(grad).max())


def test_gradient_3d_central_differences():
    g, vp, rho, src, w, rec, obs = _grad_setup(shape=(16, 18, 20), order=10, nt=70, nb=3)
    J0, grad, _ = oracle.gradient(g, vp, rho, src, w, rec, obs)
    m = 1.0 / vp ** 2
    p = (8, 9, 7)
    h = 1e-4 * m[p]
    mp, mm = m.copy(), m.copy()
    mp[p] += h
    mm[p] -= h
    fd = (_misfit(g, 1 / np.sqrt(mp), rho, src, w, rec, obs)
          - _misfit(g, 1 / np.sqrt(mm), rho, src, w, rec, obs)) / (2 * h)
    assert fd == pytest.approx(grad[p], rel=1e-6)


def test_checkpointed_gradient_equals_full_history():
    g, vp, rho, src, w, rec, obs = _grad_setup()
    J0, g0, d0 = oracle.gradient(g, vp, rho, src, w, rec, obs)
    for K in (7, 16, 139):
        J1, g1, d1 = oracle.gradient(g, vp, rho, src, w, rec, obs, ckpt_every=K)
        assert J1 == J0
        assert np.array_equal(g1, g0)
        assert np.array_equal(d1, d0)


# ---------------------------------------------------------------- sponge

def _states_from_acc(g, acc):
    """u^n from a^n when sigma = 0: u^{n+1} = 2u^n - u^{n-1} + dt^2 a^n."""
    u = [np.zeros(g.shape), np.zeros(g.shape)]   # u^{-1}, u^0
    for n in range(g.nt - 1):
        u.append(2 * u[-1] - u[-2] + g.dt ** 2 * acc[n])
    return u[1:]


def test_energy_conserved_without_sponge():
    """Discrete leapfrog energy E^{n+1/2} = <m du, du>/dt^2 - <u^{n+1}, L u^n>
    is constant once the source has stopped (nb = 0, rigid walls)."""
    n, dx, c = 48, 0.5e-3, 1500.0
    dt = 0.4 * dx / c
    g = oracle.Grid((n, n), dx, dt=dt, nt=300, order=8, nb=0)
    w = inputs.ricker(3e5, dt, g.nt)
    w[60:] = 0.0
    vp, _ = inputs.random_smooth_model((n, n), dx, 2)
    _, acc = oracle.forward(g, vp, None, np.array([[[20.3 * dx, 25.6 * dx]]]), w[None, None],
                            np.array([[10 * dx, 10 * dx]]), acc_hist=True)
    u = _states_from_acc(g, acc)
    m = 1.0 / vp ** 2
    E = []
    for k in range(80, g.nt - 1):
        du = (u[k + 1] - u[k]) / dt
        E.append(np.vdot(m * du, du) - np.vdot(u[k + 1], oracle.apply_L(g, u[k])))
    E = np.array(E)
    assert np.abs(E - E[0]).max() < 1e-9 * abs(E[0])


def test_sponge_absorbs():
    """With the sponge, a pulse leaves the box: the trace late in time is far
    weaker than with rigid walls (nb = 0), and the sponge-free interior sees
    exactly the rigid-wall solution until the wave reaches the layer."""
    n, dx, c = 120, 0.2e-3, 1500.0
    dt = 0.4 * dx / c
    nt = 900
    w = inputs.ricker(5e5, dt, nt)[None, None]
    ctr = 60 * dx
    src = np.array([[[ctr, ctr]]])
    rec = np.array([[ctr, ctr + 20 * dx]])
    out = {}
    for nb in (0, 20):
        g = oracle.Grid((n, n), dx, dt=dt, nt=nt, order=8, nb=nb, c_ref=c)
        out[nb] = oracle.forward(g, np.full((n, n), c), None, src, w, rec)[0, 0]
    t = np.arange(nt) * dt
    early = t < (60 * dx) / c       # before any echo from the layer's inner edge
    scale = np.abs(out[0]).max()
    assert np.abs(out[0][early] - out[20][early]).max() < 1e-4 * scale
    late = t > 2 * (60 * dx) / c + 8e-6
    assert np.abs(out[20][late]).max() < 0.05 * np.abs(out[0][late]).max()
