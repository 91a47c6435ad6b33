/*
 * FP64 CPU oracle for the acoustic FWI hot path of Stride (arXiv 2110.03345).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no source with the CUDA library.
 *
 * It is a plain, slow restatement of the discrete scheme, written point by
 * point with no blocking or fusion:
 *
 *  - PDE: the acoustic wave equation of Sec. 2.4, Eq. 10, without the
 *    attenuation term:  m p_tt = rho div(rho^-1 grad p) + s,  m = 1/v_p^2.
 *    The variable-density operator is taken in expanded form
 *        L_rho u = lap u - grad(ln rho) . grad u
 *    with central 8th/10th-order weights for the second and first
 *    derivatives (Sec. 2.4 gives the order only).  u = 0 outside the grid;
 *    ln rho is extended by edge replication.
 *  - Time: second-order leapfrog with a sponge term sigma(x) u_t:
 *        m [ (u+ - 2u + u-)/dt^2 + sigma (u+ - u-)/(2 dt) ] = L_rho u + s.
 *    The sponge follows the absorbing layer named in Sec. 2.4 with a
 *    quadratic profile sigma = sum_d smax_d (delta_d/nb)^2,
 *    smax_d = 3 c_ref ln(1000) / (2 nb h_d).
 *  - Sources and receivers (Sec. 2.4): bi-/tri-linear weights on the node
 *    grid.  Sources are spread with the transposed weights divided by the
 *    cell volume; receivers sample with the weights.
 *  - Objective: J = 1/2 sum (d - d_obs)^2 (the L2 trace misfit of Sec. 3.2).
 *  - Gradient with respect to m by the adjoint-state method of Sec. 2.2,
 *    Eqs. 5-9, applied to the discrete scheme (exact discrete adjoint):
 *        lambda^{k-1}: m[(l^{k-1} - 2 l^k + l^{k+1})/dt^2
 *                         + sigma (l^{k-1} - l^{k+1})/(2dt)] = L^T l^k + P^T r^k
 *        g = - sum_{n=0}^{nt-2} lambda^n * a^n,   a^n = (L u^n + s^n)/m.
 *
 * Index conventions: arrays are C order with the last axis fastest.  A 2D
 * grid is stored as shape {1, ny, nx}; only the last `ndim` axes carry
 * derivatives.  Time: u^0 = u^-1 = 0, step n (n = 0..nt-2) injects q^n and
 * produces u^{n+1}; traces d^n = P u^n for n = 0..nt-1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int ndim;        /* 2 or 3 */
    long n[3];       /* shape; for ndim == 2: {1, ny, nx} */
    double h[3];     /* spacing per axis (metres) */
    int order;       /* 8 or 10 */
    int nb;          /* sponge width in points */
    double c_ref;    /* sponge reference speed (m/s) */
    double dt;       /* time step (s) */
    int nt;          /* number of time samples */
} orc_grid;

/* ---- finite-difference weights (standard central Taylor weights) ---- */

static int radius_of(int order) { return order / 2; }

/* second derivative: w2[0] centre, w2[j] for offsets +-j */
static void d2_weights(int order, double *w2)
{
    if (order == 8) {
        w2[0] = -205.0 / 72.0; w2[1] = 8.0 / 5.0; w2[2] = -1.0 / 5.0;
        w2[3] = 8.0 / 315.0;   w2[4] = -1.0 / 560.0;
    } else {
        w2[0] = -5269.0 / 1800.0; w2[1] = 5.0 / 3.0; w2[2] = -5.0 / 21.0;
        w2[3] = 5.0 / 126.0;      w2[4] = -5.0 / 1008.0; w2[5] = 1.0 / 3150.0;
    }
}

/* first derivative: antisymmetric, w1[j] multiplies f(+j) - f(-j), j >= 1 */
static void d1_weights(int order, double *w1)
{
    w1[0] = 0.0;
    if (order == 8) {
        w1[1] = 4.0 / 5.0; w1[2] = -1.0 / 5.0; w1[3] = 4.0 / 105.0;
        w1[4] = -1.0 / 280.0;
    } else {
        w1[1] = 5.0 / 6.0; w1[2] = -5.0 / 21.0; w1[3] = 5.0 / 84.0;
        w1[4] = -5.0 / 504.0; w1[5] = 1.0 / 1260.0;
    }
}

void orc_fd_weights(int order, double *w2, double *w1)
{
    d2_weights(order, w2);
    d1_weights(order, w1);
}

/* ---- grid helpers ---- */

static long npoints(const orc_grid *g) { return g->n[0] * g->n[1] * g->n[2]; }

static int first_axis(const orc_grid *g) { return 3 - g->ndim; }

static long axis_stride(const orc_grid *g, int d)
{
    if (d == 2) return 1;
    if (d == 1) return g->n[2];
    return g->n[1] * g->n[2];
}

static void unflatten(const orc_grid *g, long p, long *i)
{
    i[2] = p % g->n[2];
    i[1] = (p / g->n[2]) % g->n[1];
    i[0] = p / (g->n[1] * g->n[2]);
}

/* value of f at p shifted by off along axis d, zero outside the grid */
static double at_zero(const orc_grid *g, const double *f, long p, const long *i,
                      int d, long off)
{
    long j = i[d] + off;
    if (j < 0 || j >= g->n[d]) return 0.0;
    return f[p + off * axis_stride(g, d)];
}

/* value of f at p shifted by off along axis d, clamped to the grid edge */
static double at_clamp(const orc_grid *g, const double *f, long p, const long *i,
                       int d, long off)
{
    long j = i[d] + off;
    if (j < 0) j = 0;
    if (j >= g->n[d]) j = g->n[d] - 1;
    return f[p + (j - i[d]) * axis_stride(g, d)];
}

/* sigma(x): quadratic sponge profile, summed over the active axes */
void orc_sponge(const orc_grid *g, double *sigma)
{
    long N = npoints(g);
    int nb = g->nb;
    for (long p = 0; p < N; ++p) {
        long i[3];
        unflatten(g, p, i);
        double s = 0.0;
        for (int d = first_axis(g); d < 3; ++d) {
            if (nb <= 0) continue;
            double smax = 3.0 * g->c_ref * log(1000.0) / (2.0 * nb * g->h[d]);
            long delta = 0;
            if (i[d] < nb) delta = nb - i[d];
            else if (i[d] > g->n[d] - 1 - nb) delta = i[d] - (g->n[d] - 1 - nb);
            double r = (double)delta / (double)nb;
            s += smax * r * r;
        }
        sigma[p] = s;
    }
}

/* b_d = D1_d ln(rho) (one field per active axis, stored [3][N]) */
static void density_gradient(const orc_grid *g, const double *rho, double *b)
{
    long N = npoints(g);
    int R = radius_of(g->order);
    double w1[6];
    d1_weights(g->order, w1);
    double *lr = (double *)malloc(sizeof(double) * N);
    for (long p = 0; p < N; ++p) lr[p] = log(rho[p]);
    for (int d = first_axis(g); d < 3; ++d) {
        for (long p = 0; p < N; ++p) {
            long i[3];
            unflatten(g, p, i);
            double acc = 0.0;
            for (int j = 1; j <= R; ++j)
                acc += w1[j] * (at_clamp(g, lr, p, i, d, j) - at_clamp(g, lr, p, i, d, -j));
            b[d * N + p] = acc / g->h[d];
        }
    }
    free(lr);
}

/* out = L_rho u.  b == NULL means constant density. */
static void apply_L(const orc_grid *g, const double *b, const double *u, double *out)
{
    long N = npoints(g);
    int R = radius_of(g->order);
    double w2[6], w1[6];
    d2_weights(g->order, w2);
    d1_weights(g->order, w1);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i[3];
        unflatten(g, p, i);
        double lap = 0.0, adv = 0.0;
        for (int d = first_axis(g); d < 3; ++d) {
            double s2 = w2[0] * u[p];
            for (int j = 1; j <= R; ++j)
                s2 += w2[j] * (at_zero(g, u, p, i, d, j) + at_zero(g, u, p, i, d, -j));
            lap += s2 / (g->h[d] * g->h[d]);
            if (b) {
                double s1 = 0.0;
                for (int j = 1; j <= R; ++j)
                    s1 += w1[j] * (at_zero(g, u, p, i, d, j) - at_zero(g, u, p, i, d, -j));
                adv += b[d * N + p] * s1 / g->h[d];
            }
        }
        out[p] = lap - adv;
    }
}

/* out = L_rho^T v = lap v + sum_d D1_d (b_d v)  (D2 symmetric, D1 antisymmetric) */
static void apply_LT(const orc_grid *g, const double *b, const double *v, double *out)
{
    long N = npoints(g);
    int R = radius_of(g->order);
    double w2[6], w1[6];
    d2_weights(g->order, w2);
    d1_weights(g->order, w1);
    double *bv = NULL;
    if (b) {
        bv = (double *)malloc(sizeof(double) * 3 * N);
        for (int d = first_axis(g); d < 3; ++d)
            for (long p = 0; p < N; ++p) bv[d * N + p] = b[d * N + p] * v[p];
    }
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i[3];
        unflatten(g, p, i);
        double lap = 0.0, div = 0.0;
        for (int d = first_axis(g); d < 3; ++d) {
            double s2 = w2[0] * v[p];
            for (int j = 1; j <= R; ++j)
                s2 += w2[j] * (at_zero(g, v, p, i, d, j) + at_zero(g, v, p, i, d, -j));
            lap += s2 / (g->h[d] * g->h[d]);
            if (b) {
                const double *f = bv + d * N;
                double s1 = 0.0;
                for (int j = 1; j <= R; ++j)
                    s1 += w1[j] * (at_zero(g, f, p, i, d, j) - at_zero(g, f, p, i, d, -j));
                div += s1 / g->h[d];
            }
        }
        out[p] = lap + div;
    }
    free(bv);
}

int orc_apply_L(const orc_grid *g, const double *rho, const double *u, double *out)
{
    long N = npoints(g);
    double *b = NULL;
    if (rho) {
        b = (double *)calloc(3 * N, sizeof(double));
        density_gradient(g, rho, b);
    }
    apply_L(g, b, u, out);
    free(b);
    return 0;
}

int orc_apply_LT(const orc_grid *g, const double *rho, const double *v, double *out)
{
    long N = npoints(g);
    double *b = NULL;
    if (rho) {
        b = (double *)calloc(3 * N, sizeof(double));
        density_gradient(g, rho, b);
    }
    apply_LT(g, b, v, out);
    free(b);
    return 0;
}

/* ---- off-grid points: bi-/tri-linear weights ---- */

/* For a point xyz (ndim coordinates, axis order), fill up to 8 node indices
 * and weights.  Along each axis: xi = x/h, i0 = floor(xi) clamped to n-2,
 * f = xi - i0, weights (1-f, f) at (i0, i0+1).  Returns the corner count. */
int orc_point_weights(const orc_grid *g, const double *xyz, long *idx, double *w)
{
    long base[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    int fa = first_axis(g);
    for (int d = fa; d < 3; ++d) {
        double xi = xyz[d - fa] / g->h[d];
        long i0 = (long)floor(xi);
        if (i0 > g->n[d] - 2) i0 = g->n[d] - 2;
        if (i0 < 0) i0 = 0;
        base[d] = i0;
        f[d] = xi - (double)i0;
    }
    int nc = 1 << g->ndim;
    for (int c = 0; c < nc; ++c) {
        long i[3] = {base[0], base[1], base[2]};
        double wt = 1.0;
        for (int k = 0; k < g->ndim; ++k) {
            int d = 2 - k;           /* bit k of c selects the upper node on axis 2-k */
            int up = (c >> k) & 1;
            i[d] += up;
            wt *= up ? f[d] : (1.0 - f[d]);
        }
        idx[c] = (i[0] * g->n[1] + i[1]) * g->n[2] + i[2];
        w[c] = wt;
    }
    return nc;
}

static double cell_volume(const orc_grid *g)
{
    double v = 1.0;
    for (int d = first_axis(g); d < 3; ++d) v *= g->h[d];
    return v;
}

/* s += spread of point values (weights / dV if scale_by_volume) */
static void spread(const orc_grid *g, int npt, const double *xyz, const double *vals,
                   int scale_by_volume, double *s)
{
    double inv_dv = scale_by_volume ? 1.0 / cell_volume(g) : 1.0;
    for (int k = 0; k < npt; ++k) {
        long idx[8];
        double w[8];
        int nc = orc_point_weights(g, xyz + (long)k * g->ndim, idx, w);
        for (int c = 0; c < nc; ++c) s[idx[c]] += w[c] * vals[k] * inv_dv;
    }
}

/* d_k = sum_c w_c f[idx_c] */
static double sample(const orc_grid *g, const double *xyz, const double *f)
{
    long idx[8];
    double w[8];
    int nc = orc_point_weights(g, xyz, idx, w);
    double acc = 0.0;
    for (int c = 0; c < nc; ++c) acc += w[c] * f[idx[c]];
    return acc;
}

/* ---- one leapfrog step ----
 * Given u (= u^n), uold (= u^{n-1}) and the source field s (= s^n),
 * compute a^n = (L u + s)/m into acc (if non-NULL) and u^{n+1} into unew.
 */
static void leapfrog(const orc_grid *g, const double *m, const double *sigma,
                     const double *Lu, const double *s, const double *u,
                     const double *uold, double *unew, double *acc)
{
    long N = npoints(g);
    double dt = g->dt;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        double a = (Lu[p] + s[p]) / m[p];
        if (acc) acc[p] = a;
        /* m[(u+ - 2u + u-)/dt^2 + sigma (u+ - u-)/(2dt)] = m a, solved for u+ */
        double lhs_coef = 1.0 / (dt * dt) + sigma[p] / (2.0 * dt);
        double rhs = a + (2.0 * u[p] - uold[p]) / (dt * dt) + sigma[p] * uold[p] / (2.0 * dt);
        unew[p] = rhs / lhs_coef;
    }
}

typedef struct {
    const orc_grid *g;
    double *m, *sigma, *b;
} orc_model;

static int model_init(orc_model *M, const orc_grid *g, const double *vp, const double *rho)
{
    long N = npoints(g);
    M->g = g;
    M->m = (double *)malloc(sizeof(double) * N);
    M->sigma = (double *)malloc(sizeof(double) * N);
    M->b = NULL;
    for (long p = 0; p < N; ++p) M->m[p] = 1.0 / (vp[p] * vp[p]);
    orc_sponge(g, M->sigma);
    if (rho) {
        M->b = (double *)calloc(3 * N, sizeof(double));
        density_gradient(g, rho, M->b);
    }
    return 0;
}

static void model_free(orc_model *M)
{
    free(M->m);
    free(M->sigma);
    free(M->b);
}

/* Forward modelling of one shot.
 *   wavelet [nsrc][nt], traces [nrec][nt] (output).
 *   acc_hist: optional [nt-1][N] output of a^n = (L u^n + s^n)/m.
 *   ckpt_every / ckpt: optional; if ckpt_every > 0, stores (u^n, u^{n-1}) for
 *   n = 0, K, 2K, ... (n <= nt-2) into ckpt[2*j][N], ckpt[2*j+1][N].
 */
static int forward_shot(const orc_model *M, int nsrc, const double *src_xyz,
                        const double *wavelet, int nrec, const double *rec_xyz,
                        double *traces, double *acc_hist, int ckpt_every, double *ckpt)
{
    const orc_grid *g = M->g;
    long N = npoints(g);
    int nt = g->nt;
    double *u = (double *)calloc(N, sizeof(double));
    double *uold = (double *)calloc(N, sizeof(double));
    double *unew = (double *)calloc(N, sizeof(double));
    double *Lu = (double *)malloc(sizeof(double) * N);
    double *s = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * (nsrc > 0 ? nsrc : 1));

    for (int n = 0; n < nt; ++n) {
        for (int r = 0; r < nrec; ++r)
            if (traces) traces[(long)r * nt + n] = sample(g, rec_xyz + (long)r * g->ndim, u);
        if (n == nt - 1) break;
        if (ckpt_every > 0 && n % ckpt_every == 0) {
            long j = n / ckpt_every;
            memcpy(ckpt + (2 * j) * N, u, sizeof(double) * N);
            memcpy(ckpt + (2 * j + 1) * N, uold, sizeof(double) * N);
        }
        memset(s, 0, sizeof(double) * N);
        for (int k = 0; k < nsrc; ++k) q[k] = wavelet[(long)k * nt + n];
        spread(g, nsrc, src_xyz, q, 1, s);
        apply_L(g, M->b, u, Lu);
        leapfrog(g, M->m, M->sigma, Lu, s, u, uold, unew,
                 acc_hist ? acc_hist + (long)n * N : NULL);
        double *t = uold; uold = u; u = unew; unew = t;
    }
    free(u); free(uold); free(unew); free(Lu); free(s); free(q);
    return 0;
}

/* Re-run forward steps n0 .. n1-1 from the state (u^{n0}, u^{n0-1}) and store
 * a^n for those steps into seg[(n - n0)][N]. */
static void recompute_segment(const orc_model *M, int nsrc, const double *src_xyz,
                              const double *wavelet, const double *u_n0,
                              const double *u_n0m1, int n0, int n1, double *seg)
{
    const orc_grid *g = M->g;
    long N = npoints(g);
    int nt = g->nt;
    double *u = (double *)malloc(sizeof(double) * N);
    double *uold = (double *)malloc(sizeof(double) * N);
    double *unew = (double *)calloc(N, sizeof(double));
    double *Lu = (double *)malloc(sizeof(double) * N);
    double *s = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * (nsrc > 0 ? nsrc : 1));
    memcpy(u, u_n0, sizeof(double) * N);
    memcpy(uold, u_n0m1, sizeof(double) * N);
    for (int n = n0; n < n1; ++n) {
        memset(s, 0, sizeof(double) * N);
        for (int k = 0; k < nsrc; ++k) q[k] = wavelet[(long)k * nt + n];
        spread(g, nsrc, src_xyz, q, 1, s);
        apply_L(g, M->b, u, Lu);
        leapfrog(g, M->m, M->sigma, Lu, s, u, uold, unew, seg + (long)(n - n0) * N);
        double *t = uold; uold = u; u = unew; unew = t;
    }
    free(u); free(uold); free(unew); free(Lu); free(s); free(q);
}

/* Adjoint sweep of one shot, backwards in time.
 *   resid [nrec][nt]: adjoint source r^k (for the L2 misfit, d - d_obs).
 *   For k = nt-1 .. 1 computes lambda^{k-1}.
 *   grad (optional, accumulated): grad -= lambda^n a^n for n = 0..nt-2, where
 *     a^n comes from acc_hist [nt-1][N] or, if acc_hist is NULL and
 *     ckpt_every > 0, from recomputation out of the checkpoints.
 *   src_adj (optional) [nsrc][nt]: (S lambda^n)/dV, the adjoint of the
 *     source-wavelet-to-trace map, with src_adj[., nt-1] = 0.
 */
static int adjoint_shot(const orc_model *M, int nrec, const double *rec_xyz,
                        const double *resid, const double *acc_hist, double *grad,
                        int nsrc, const double *src_xyz, double *src_adj,
                        const double *wavelet, int ckpt_every, const double *ckpt)
{
    const orc_grid *g = M->g;
    long N = npoints(g);
    int nt = g->nt;
    double dt = g->dt;
    double *lam = (double *)calloc(N, sizeof(double));      /* lambda^k */
    double *lam_next = (double *)calloc(N, sizeof(double)); /* lambda^{k+1} */
    double *lam_prev = (double *)calloc(N, sizeof(double)); /* lambda^{k-1} */
    double *LTl = (double *)malloc(sizeof(double) * N);
    double *pr = (double *)malloc(sizeof(double) * N);
    double *rv = (double *)malloc(sizeof(double) * (nrec > 0 ? nrec : 1));
    double *seg = NULL;
    int seg_lo = -1, seg_hi = -1;
    if (!acc_hist && grad && ckpt_every > 0)
        seg = (double *)malloc(sizeof(double) * (long)ckpt_every * N);
    double inv_dv = 1.0 / cell_volume(g);

    if (src_adj)
        for (int k = 0; k < nsrc; ++k) src_adj[(long)k * nt + (nt - 1)] = 0.0;

    /* lambda^{nt-1} = lambda^{nt} = 0; iterate k = nt-1 .. 1 to get lambda^{k-1} */
    for (int k = nt - 1; k >= 1; --k) {
        memset(pr, 0, sizeof(double) * N);
        for (int r = 0; r < nrec; ++r) rv[r] = resid[(long)r * nt + k];
        spread(g, nrec, rec_xyz, rv, 0, pr);
        apply_LT(g, M->b, lam, LTl);
        /* m[(l- - 2l + l+)/dt^2 + sigma (l- - l+)/(2dt)] = L^T l + P^T r, solved for l- */
#pragma omp parallel for schedule(static)
        for (long p = 0; p < N; ++p) {
            double a = (LTl[p] + pr[p]) / M->m[p];
            double coef = 1.0 / (dt * dt) + M->sigma[p] / (2.0 * dt);
            double rhs = a + (2.0 * lam[p] - lam_next[p]) / (dt * dt)
                         + M->sigma[p] * lam_next[p] / (2.0 * dt);
            lam_prev[p] = rhs / coef;
        }
        int n = k - 1; /* lam_prev holds lambda^n */
        if (grad) {
            const double *a_n;
            if (acc_hist) {
                a_n = acc_hist + (long)n * N;
            } else {
                if (n < seg_lo || n >= seg_hi) {
                    int j = n / ckpt_every;
                    seg_lo = j * ckpt_every;
                    seg_hi = seg_lo + ckpt_every;
                    if (seg_hi > nt - 1) seg_hi = nt - 1;
                    recompute_segment(M, nsrc, src_xyz, wavelet, ckpt + (2L * j) * N,
                                      ckpt + (2L * j + 1) * N, seg_lo, seg_hi, seg);
                }
                a_n = seg + (long)(n - seg_lo) * N;
            }
            for (long p = 0; p < N; ++p) grad[p] -= lam_prev[p] * a_n[p];
        }
        if (src_adj)
            for (int s = 0; s < nsrc; ++s)
                src_adj[(long)s * nt + n] = sample(g, src_xyz + (long)s * g->ndim, lam_prev) * inv_dv;
        double *t = lam_next; lam_next = lam; lam = lam_prev; lam_prev = t;
    }
    free(lam); free(lam_next); free(lam_prev); free(LTl); free(pr); free(rv); free(seg);
    return 0;
}

/* ---- exported entry points (one shot each; the caller loops over shots) ---- */

int orc_forward(const orc_grid *g, const double *vp, const double *rho,
                int nsrc, const double *src_xyz, const double *wavelet,
                int nrec, const double *rec_xyz, double *traces, double *acc_hist)
{
    orc_model M;
    model_init(&M, g, vp, rho);
    forward_shot(&M, nsrc, src_xyz, wavelet, nrec, rec_xyz, traces, acc_hist, 0, NULL);
    model_free(&M);
    return 0;
}

/* adjoint of the linear map wavelet -> traces, sampled at the sources */
int orc_adjoint_sources(const orc_grid *g, const double *vp, const double *rho,
                        int nrec, const double *rec_xyz, const double *resid,
                        int nsrc, const double *src_xyz, double *src_adj)
{
    orc_model M;
    model_init(&M, g, vp, rho);
    adjoint_shot(&M, nrec, rec_xyz, resid, NULL, NULL, nsrc, src_xyz, src_adj, NULL, 0, NULL);
    model_free(&M);
    return 0;
}

/* Misfit and gradient of one shot.  grad is ACCUMULATED (caller zeroes it);
 * misfit receives this shot's J.  traces (optional) receives d.
 * ckpt_every <= 0 or >= nt-1 stores the full a^n history; otherwise the
 * forward states are checkpointed every ckpt_every steps and a^n is
 * recomputed per segment (identical arithmetic, less memory). */
int orc_gradient(const orc_grid *g, const double *vp, const double *rho,
                 int nsrc, const double *src_xyz, const double *wavelet,
                 int nrec, const double *rec_xyz, const double *observed,
                 double *misfit, double *grad, double *traces, int ckpt_every)
{
    long N = npoints(g);
    int nt = g->nt;
    orc_model M;
    model_init(&M, g, vp, rho);
    double *d = (double *)malloc(sizeof(double) * (long)nrec * nt);
    int full = (ckpt_every <= 0 || ckpt_every >= nt - 1);
    double *acc = NULL, *ckpt = NULL;
    if (nt >= 2) {
        if (full) {
            acc = (double *)malloc(sizeof(double) * (long)(nt - 1) * N);
        } else {
            long nck = (nt - 2) / ckpt_every + 1;
            ckpt = (double *)malloc(sizeof(double) * 2 * nck * N);
        }
    }
    forward_shot(&M, nsrc, src_xyz, wavelet, nrec, rec_xyz, d, acc,
                 full ? 0 : ckpt_every, ckpt);
    double J = 0.0;
    for (long i = 0; i < (long)nrec * nt; ++i) {
        double r = d[i] - observed[i];
        J += 0.5 * r * r;
        if (traces) traces[i] = d[i];
        d[i] = r; /* d now holds the residual, the adjoint source */
    }
    *misfit = J;
    if (nt >= 2)
        adjoint_shot(&M, nrec, rec_xyz, d, acc, grad, nsrc, src_xyz, NULL, wavelet,
                     full ? 0 : ckpt_every, ckpt);
    free(d); free(acc); free(ckpt);
    model_free(&M);
    return 0;
}
