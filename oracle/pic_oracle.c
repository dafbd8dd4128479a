/*
 * pic_oracle.c -- plain FP64 CPU oracle for the particle loops of the
 * energy-conserving PIC scheme (1D reduced relativistic Vlasov--Maxwell)
 * of Li, "Energy conserving particle-in-cell methods for relativistic
 * Vlasov--Maxwell equations of laser-plasma interaction": the hbar = 0
 * scheme, and the spin terms (hbar != 0) at the end of the file.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only tests/, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or table with the CUDA
 * library.
 *
 * Everything here is written to be checked by eye against the paper:
 * one particle at a time, in double precision, no blocking, no fusion.
 * The grid-side linear algebra (mass matrices, solves) lives in oracle.py.
 *
 * Notation (Sec. 3.1): M cells of width dx = L/M, nodes x_j = j*dx.
 * Lambda^0_j = N^k_j (degree k), Lambda^1_j = N^{k-1}_j (degree k-1),
 * N^d_j has support [x_j, x_{j+d+1}).  A point with cell-unit coordinate
 * u = x/dx lies in cell c = floor(u) with local coordinate t = u - c, and
 * touches the basis functions j = c - r (mod M), r = 0..d, with value
 * N^d(r + t) where N^d is the cardinal B-spline on integer knots.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* B-splines (Sec. 3.1)                                                 */
/* ------------------------------------------------------------------ */

/* Cardinal B-spline N^d(s) of degree d on the integer knots 0..d+1, by
 * the Cox--de Boor recursion: N^0 = indicator of [0,1),
 * N^d(s) = ( s N^{d-1}(s) + (d+1-s) N^{d-1}(s-1) ) / d.                */
double orc_cardinal_bspline(int d, double s)
{
    if (d == 0) return (s >= 0.0 && s < 1.0) ? 1.0 : 0.0;
    return (s * orc_cardinal_bspline(d - 1, s)
            + ((double)(d + 1) - s) * orc_cardinal_bspline(d - 1, s - 1.0)) / (double)d;
}

/* Values vals[r] = N^d(r + t), r = 0..d, for the d+1 basis functions that
 * are nonzero in a cell at local coordinate t in [0,1).                 */
void orc_basis(int d, double t, double *vals)
{
    for (int r = 0; r <= d; ++r) vals[r] = orc_cardinal_bspline(d, (double)r + t);
}

static long wrap_index(long j, long M)
{
    long r = j % M;
    return r < 0 ? r + M : r;
}

/* Split a cell-unit coordinate u into (cell, local t).  A knot belongs to
 * the cell on its right (half-open cells).                             */
static void split_u(double u, long *c, double *t)
{
    double f = floor(u);
    *c = (long)f;
    *t = u - f;
}

/* Finite-element function value sum_j coef_j Lambda^d_j(x) at the point
 * x (physical units, any real: periodic).                               */
static double fe_value(int d, const double *coef, long M, double dx, double x)
{
    long c; double t;
    double v[8];
    split_u(x / dx, &c, &t);
    orc_basis(d, t, v);
    double s = 0.0;
    for (int r = 0; r <= d; ++r) s += coef[wrap_index(c - r, M)] * v[r];
    return s;
}

/* ------------------------------------------------------------------ */
/* Mass matrices (Sec. 3.1): first row of the circulant matrix          */
/* (M_d)_{0,j} = int_0^L Lambda^d_0 Lambda^d_j dx, by Gauss--Legendre   */
/* quadrature with d+1 nodes per cell (exact for degree 2d+1).          */
/* ------------------------------------------------------------------ */

/* Gauss--Legendre rule on [-1,1] with n nodes, 1 <= n <= 6, computed by
 * Newton's method on the Legendre polynomial P_n (three-term recurrence). */
int orc_gauss_legendre(int n, double *xi, double *w)
{
    if (n < 1 || n > 16) return 1;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            /* P_n(z) = p1, P_{n-1}(z) = p0 ; P_n'(z) = n (z P_n - P_{n-1})/(z^2-1) */
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int l = 2; l <= n; ++l) {
            double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
            p0 = p1; p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        xi[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

int orc_mass_row(int d, long M, double dx, double *row)
{
    double xi[16], w[16];
    int nq = d + 1;
    if (orc_gauss_legendre(nq, xi, w)) return 1;
    for (long j = 0; j < M; ++j) row[j] = 0.0;
    /* Lambda^d_0 is supported on cells 0..d (unwrapped). */
    for (int cell = 0; cell <= d; ++cell) {
        for (int q = 0; q < nq; ++q) {
            double t = 0.5 * (1.0 + xi[q]);
            double wq = 0.5 * w[q] * dx;
            double v[8];
            orc_basis(d, t, v);
            /* in this cell, Lambda^d_{cell-r} has value v[r]; Lambda^d_0 is r = cell */
            double phi0 = v[cell];
            for (int r = 0; r <= d; ++r)
                row[wrap_index((long)cell - r, M)] += wq * phi0 * v[r];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Path integral of the 1-form basis along a straight particle path     */
/* (Sec. 4.2, subsystem I: x(tau) linear from x^n to x^{n+1}).          */
/* The path is split at every knot it crosses; on each piece the        */
/* degree-(k-1) basis is a polynomial and q = ceil(k/2) Gauss--Legendre */
/* nodes integrate it exactly.                                          */
/* mean[i] += path mean of Lambda^1_i (1/|path| int Lambda^1_i dxi);    */
/* the signed integral is (x1 - x0) * mean[i].                          */
/* ------------------------------------------------------------------ */
static void path_mean_1form(int k, long M, double dx, double x0, double x1,
                            const double *xi, const double *w,
                            double *mean /* M, accumulated */,
                            long *touched_lo, long *touched_hi)
{
    int d = k - 1;
    int nq = (k + 1) / 2;
    double u0 = x0 / dx, u1 = x1 / dx;
    double len = u1 - u0;
    double dir = (len >= 0.0) ? 1.0 : -1.0;
    double ua = u0;
    long lo = 0, hi = 0;
    int first = 1;
    for (;;) {
        /* next knot strictly beyond ua in the direction of motion */
        double ub;
        if (dir > 0) { ub = floor(ua) + 1.0; if (ub > u1) ub = u1; }
        else         { ub = ceil(ua) - 1.0;  if (ub < u1) ub = u1; }
        if (len == 0.0) ub = u1;
        double seg_lo = ua < ub ? ua : ub;
        long c = (long)floor(seg_lo);
        double frac = (len == 0.0) ? 1.0 : (ub - ua) / len;
        for (int q = 0; q < nq; ++q) {
            double uq = ua + (ub - ua) * 0.5 * (1.0 + xi[q]);
            double t = uq - (double)c;
            double v[8];
            orc_basis(d, t, v);
            for (int r = 0; r <= d; ++r) {
                long j = wrap_index(c - r, M);
                mean[j] += frac * 0.5 * w[q] * v[r];
            }
        }
        if (first) { lo = c - d; hi = c; first = 0; }
        if (c - d < lo) lo = c - d;
        if (c > hi) hi = c;
        if (ub == u1) break;
        ua = ub;
    }
    if (touched_lo) *touched_lo = lo;
    if (touched_hi) *touched_hi = hi;
}

/* Exposed for tests: path mean and signed path integral of every
 * Lambda^1_i over x0 -> x1 (physical units, unwrapped).               */
void orc_path_integral(int k, long M, double dx, double x0, double x1,
                       double *mean, double *integral)
{
    double xi[16], w[16];
    orc_gauss_legendre((k + 1) / 2, xi, w);
    for (long i = 0; i < M; ++i) mean[i] = 0.0;
    path_mean_1form(k, M, dx, x0, x1, xi, w, mean, 0, 0);
    for (long i = 0; i < M; ++i) integral[i] = (x1 - x0) * mean[i];
}

/* ------------------------------------------------------------------ */
/* Gathers and deposits (Sec. 3.1, Eqs. fem_e, fem_a, f_dirac)          */
/* ------------------------------------------------------------------ */

/* out[a] = sum_j coef_j Lambda^d_j(x_a) */
void orc_gather(int d, long M, double dx, long np, const double *x,
                const double *coef, double *out)
{
    for (long a = 0; a < np; ++a) out[a] = fe_value(d, coef, M, dx, x[a]);
}

/* rho_j = sum_a w Lambda^k_j(x_a)  (the Lambda_0(X)^T W 1 of Sec. 4.2) */
void orc_charge(int k, long M, double dx, long np, const double *x,
                double w, double *rho)
{
    for (long j = 0; j < M; ++j) rho[j] = 0.0;
    for (long a = 0; a < np; ++a) {
        long c; double t; double v[8];
        split_u(x[a] / dx, &c, &t);
        orc_basis(k, t, v);
        for (int r = 0; r <= k; ++r) rho[wrap_index(c - r, M)] += w * v[r];
    }
}

/* sum_a w (gamma(p_a, A_perp(x_a)) - 1), gamma = sqrt(1 + p^2 + |A|^2)
 * (kinetic part of the discrete Hamiltonian, Eq. discrete_H).          */
double orc_kinetic(int k, long M, double dx, long np, const double *x,
                   const double *p, double w, const double *ay, const double *az)
{
    double s = 0.0;
    for (long a = 0; a < np; ++a) {
        double Ay = fe_value(k, ay, M, dx, x[a]);
        double Az = fe_value(k, az, M, dx, x[a]);
        double g = sqrt(1.0 + p[a] * p[a] + Ay * Ay + Az * Az);
        s += w * (g - 1.0);
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Subsystem I: one Picard sweep over all particles (Sec. 4.2).         */
/*                                                                      */
/* Given x^n, p^n, the current iterate x^(k) = x^n + delta^(k) and the   */
/* field average ebar = (e_x^n + e_x^(k))/2, each particle computes      */
/*   A1 = A_h^n(x^(k)), A0 = A_h^n(x^n),                                 */
/*   Ebar = path mean of E along x^n -> x^(k) = sum_i m_i ebar_i,        */
/*   D    = (A1 - A0)/(x^(k) - x^n) = sum_i m_i (G a)_i   (exact, since  */
/*          d/dx A_h = sum_i (G a)_i Lambda^1_i),                        */
/*   p^(k+1) = p^n + dt Ebar - dt (A1+A0).D / (g(p^n,A1) + g(p^n,A0)),   */
/*   delta^(k+1) = dt (p^n + p^(k+1)) / (g(p^n,A1) + g(p^(k+1),A1)),     */
/* and deposits j_i += w int_{x^n}^{x^n+delta^(k+1)} Lambda^1_i dxi.     */
/* Returns max |delta^(k+1)-delta^(k)| in dmax and max |p^(k+1)-p^(k)|.  */
/* ------------------------------------------------------------------ */
void orc_sweep1(int k, long M, double dx, double dt, double w, long np,
                const double *x, const double *p,
                double *delta /* in: delta^(k), out: delta^(k+1) */,
                double *pk    /* in: p^(k),     out: p^(k+1)     */,
                const double *ebar, const double *ga_y, const double *ga_z,
                const double *ay, const double *az,
                double *j /* M, accumulated */,
                double *dmax, double *pmax,
                double *mean_scratch /* M, all zero on entry and on return */)
{
    double dm = 0.0, pm = 0.0;
    double xi[16], wq[16];
    orc_gauss_legendre((k + 1) / 2, xi, wq);
    for (long a = 0; a < np; ++a) {
        double x0 = x[a];
        double x1 = x0 + delta[a];
        double A0y = fe_value(k, ay, M, dx, x0), A0z = fe_value(k, az, M, dx, x0);
        double A1y = fe_value(k, ay, M, dx, x1), A1z = fe_value(k, az, M, dx, x1);

        long lo, hi;
        path_mean_1form(k, M, dx, x0, x1, xi, wq, mean_scratch, &lo, &hi);
        double Ebar = 0.0, Dy = 0.0, Dz = 0.0;
        for (long jj = lo; jj <= hi && jj - lo < M; ++jj) {
            long i = wrap_index(jj, M);
            Ebar += mean_scratch[i] * ebar[i];
            Dy += mean_scratch[i] * ga_y[i];
            Dz += mean_scratch[i] * ga_z[i];
            mean_scratch[i] = 0.0;
        }
        double pn = p[a];
        double g1 = sqrt(1.0 + pn * pn + A1y * A1y + A1z * A1z);
        double g0 = sqrt(1.0 + pn * pn + A0y * A0y + A0z * A0z);
        double pnew = pn + dt * Ebar - dt * ((A1y + A0y) * Dy + (A1z + A0z) * Dz) / (g1 + g0);
        double g2 = sqrt(1.0 + pnew * pnew + A1y * A1y + A1z * A1z);
        double dnew = dt * (pn + pnew) / (g1 + g2);

        /* deposit along the new path x^n -> x^n + delta^(k+1) */
        path_mean_1form(k, M, dx, x0, x0 + dnew, xi, wq, mean_scratch, &lo, &hi);
        for (long jj = lo; jj <= hi && jj - lo < M; ++jj) {
            long i = wrap_index(jj, M);
            j[i] += w * dnew * mean_scratch[i];
            mean_scratch[i] = 0.0;
        }

        double dd = fabs(dnew - delta[a]);
        double dp = fabs(pnew - pk[a]);
        if (!(dd <= dm)) dm = dd;   /* NaN propagates as "not converged" */
        if (!(dp <= pm)) pm = dp;
        delta[a] = dnew;
        pk[a] = pnew;
    }
    *dmax = dm;
    *pmax = pm;
}

/* ------------------------------------------------------------------ */
/* Subsystem II: one fixed-point sweep over all particles (Sec. 4.2).   */
/* Particles are frozen at x; with A0 = A_h^n(x_a) and A1 = A_h^(k)(x_a) */
/* (a^(k) = a^n - dt/2 (e^n + e^(k))),                                   */
/*   s_i += w (A0 + A1) Lambda^0_i(x_a) / (g(p_a,A0) + g(p_a,A1))        */
/* for the y and z components.  The basis is Lambda^0 (e_y, a_y are     */
/* 0-forms, as in the subsystem's ODE).                                  */
/* ------------------------------------------------------------------ */
void orc_sweep2(int k, long M, double dx, double w, long np,
                const double *x, const double *p,
                const double *ay_n, const double *az_n,
                const double *ay_k, const double *az_k,
                double *s_y, double *s_z /* M, accumulated */)
{
    for (long a = 0; a < np; ++a) {
        long c; double t; double v[8];
        split_u(x[a] / dx, &c, &t);
        orc_basis(k, t, v);
        double A0y = 0, A0z = 0, A1y = 0, A1z = 0;
        for (int r = 0; r <= k; ++r) {
            long i = wrap_index(c - r, M);
            A0y += ay_n[i] * v[r]; A0z += az_n[i] * v[r];
            A1y += ay_k[i] * v[r]; A1z += az_k[i] * v[r];
        }
        double pa = p[a];
        double g0 = sqrt(1.0 + pa * pa + A0y * A0y + A0z * A0z);
        double g1 = sqrt(1.0 + pa * pa + A1y * A1y + A1z * A1z);
        double cf = w / (g0 + g1);
        for (int r = 0; r <= k; ++r) {
            long i = wrap_index(c - r, M);
            s_y[i] += cf * (A0y + A1y) * v[r];
            s_z[i] += cf * (A0z + A1z) * v[r];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Spin (hbar != 0): the terms of Sec. 4.2 that carry hbar.              */
/*                                                                      */
/* The Hamiltonian (Eq. discrete_H) adds                                 */
/*   hbar sum_a w (s_y,a dA_z/dx(x_a) - s_z,a dA_y/dx(x_a)),             */
/* with dA_h/dx = sum_i (G a)_i Lambda^1_i (Sec. 3.1).  Its second       */
/* derivative is the degree-(k-2) spline sum_i (G' G a)_i Lambda^2_i,    */
/* Lambda^2_i = N^{k-2}_i, (G' v)_i = (v_i - v_{i-1})/dx, by the same    */
/* derivative relation one degree lower.                                  */
/* ------------------------------------------------------------------ */

/* Path mean of every degree-d basis function N^d_i along x0 -> x1 (the
 * path split at every knot, q = ceil((d+1)/2) Gauss--Legendre nodes per
 * piece: exact for degree d).  mean[] must be zero on entry; the touched
 * node range is returned in [lo, hi] (unwrapped).                       */
static void path_mean_deg(int d, long M, double dx, double x0, double x1,
                          double *mean, long *touched_lo, long *touched_hi)
{
    double xi[16], w[16];
    int nq = (d + 2) / 2;
    orc_gauss_legendre(nq, xi, w);
    double u0 = x0 / dx, u1 = x1 / dx;
    double len = u1 - u0;
    double dir = (len >= 0.0) ? 1.0 : -1.0;
    double ua = u0;
    long lo = 0, hi = 0;
    int first = 1;
    for (;;) {
        double ub;
        if (dir > 0) { ub = floor(ua) + 1.0; if (ub > u1) ub = u1; }
        else         { ub = ceil(ua) - 1.0;  if (ub < u1) ub = u1; }
        if (len == 0.0) ub = u1;
        double seg_lo = ua < ub ? ua : ub;
        long c = (long)floor(seg_lo);
        double frac = (len == 0.0) ? 1.0 : (ub - ua) / len;
        for (int q = 0; q < nq; ++q) {
            double uq = ua + (ub - ua) * 0.5 * (1.0 + xi[q]);
            double v[8];
            orc_basis(d, uq - (double)c, v);
            for (int r = 0; r <= d; ++r) mean[wrap_index(c - r, M)] += frac * 0.5 * w[q] * v[r];
        }
        if (first) { lo = c - d; hi = c; first = 0; }
        if (c - d < lo) lo = c - d;
        if (c > hi) hi = c;
        if (ub == u1) break;
        ua = ub;
    }
    *touched_lo = lo;
    *touched_hi = hi;
}

/* Exposed for tests: path means of the degree-d basis along x0 -> x1. */
void orc_path_mean_deg(int d, long M, double dx, double x0, double x1, double *mean)
{
    long lo, hi;
    for (long i = 0; i < M; ++i) mean[i] = 0.0;
    path_mean_deg(d, M, dx, x0, x1, mean, &lo, &hi);
}

/* Subsystem I sweep with spin: orc_sweep1 plus, in the momentum update,
 *   - dt hbar ( s_y D2_z - s_z D2_y ),
 * D2 = (dA/dx(x^(k)) - dA/dx(x^n)) / (x^(k) - x^n) = the path mean of
 * d^2A/dx^2 = sum_i (G'Ga)_i m2_i, m2 = path means of Lambda^2 (exact, so
 * no 0/0 arises), the spin held at s^n (Sec. 4.2, subsystem I with the
 * discrete gradient of the Zeeman term).  gga_y, gga_z: G'G a_y, G'G a_z. */
void orc_sweep1_spin(int k, long M, double dx, double dt, double w, double hbar, long np,
                     const double *x, const double *p, const double *sy, const double *sz,
                     double *delta, double *pk,
                     const double *ebar, const double *ga_y, const double *ga_z,
                     const double *gga_y, const double *gga_z,
                     const double *ay, const double *az,
                     double *j, double *dmax, double *pmax,
                     double *mean_scratch, double *mean2_scratch)
{
    double dm = 0.0, pm = 0.0;
    double xi[16], wq[16];
    orc_gauss_legendre((k + 1) / 2, xi, wq);
    for (long a = 0; a < np; ++a) {
        double x0 = x[a];
        double x1 = x0 + delta[a];
        double A0y = fe_value(k, ay, M, dx, x0), A0z = fe_value(k, az, M, dx, x0);
        double A1y = fe_value(k, ay, M, dx, x1), A1z = fe_value(k, az, M, dx, x1);

        long lo, hi;
        path_mean_1form(k, M, dx, x0, x1, xi, wq, mean_scratch, &lo, &hi);
        double Ebar = 0.0, Dy = 0.0, Dz = 0.0;
        for (long jj = lo; jj <= hi && jj - lo < M; ++jj) {
            long i = wrap_index(jj, M);
            Ebar += mean_scratch[i] * ebar[i];
            Dy += mean_scratch[i] * ga_y[i];
            Dz += mean_scratch[i] * ga_z[i];
            mean_scratch[i] = 0.0;
        }
        double D2y = 0.0, D2z = 0.0;
        path_mean_deg(k - 2, M, dx, x0, x1, mean2_scratch, &lo, &hi);
        for (long jj = lo; jj <= hi && jj - lo < M; ++jj) {
            long i = wrap_index(jj, M);
            D2y += mean2_scratch[i] * gga_y[i];
            D2z += mean2_scratch[i] * gga_z[i];
            mean2_scratch[i] = 0.0;
        }
        double pn = p[a];
        double g1 = sqrt(1.0 + pn * pn + A1y * A1y + A1z * A1z);
        double g0 = sqrt(1.0 + pn * pn + A0y * A0y + A0z * A0z);
        double pnew = pn + dt * Ebar - dt * ((A1y + A0y) * Dy + (A1z + A0z) * Dz) / (g1 + g0)
                      - dt * hbar * (sy[a] * D2z - sz[a] * D2y);
        double g2 = sqrt(1.0 + pnew * pnew + A1y * A1y + A1z * A1z);
        double dnew = dt * (pn + pnew) / (g1 + g2);

        path_mean_1form(k, M, dx, x0, x0 + dnew, xi, wq, mean_scratch, &lo, &hi);
        for (long jj = lo; jj <= hi && jj - lo < M; ++jj) {
            long i = wrap_index(jj, M);
            j[i] += w * dnew * mean_scratch[i];
            mean_scratch[i] = 0.0;
        }

        double dd = fabs(dnew - delta[a]);
        double dp = fabs(pnew - pk[a]);
        if (!(dd <= dm)) dm = dd;
        if (!(dp <= pm)) pm = dp;
        delta[a] = dnew;
        pk[a] = pnew;
    }
    *dmax = dm;
    *pmax = pm;
}

/* d_i = sum_a w s_a Lambda^1_i(x_a): the Lambda_1(X)^T W S of the spin source
 * of subsystem II (applied with G^T on the grid side).                  */
void orc_spin_deposit(int k, long M, double dx, long np, const double *x, double w,
                      const double *s, double *d)
{
    for (long i = 0; i < M; ++i) d[i] = 0.0;
    for (long a = 0; a < np; ++a) {
        long c; double t; double v[8];
        split_u(x[a] / dx, &c, &t);
        orc_basis(k - 1, t, v);
        for (int r = 0; r <= k - 1; ++r) d[wrap_index(c - r, M)] += w * s[a] * v[r];
    }
}

/* Subsystem III (Sec. 4.2, Eq. spin_rodrigue): with Y = dA_y/dx(x_a),
 * Z = dA_z/dx(x_a) (V1 gathers of G a_y, G a_z), the spin obeys
 * ds/dt = r^ s, r^ s = r x s, r = (0, Z, -Y), and the exact step is the
 * Rodrigues rotation
 *   s^{n+1} = s + sin(dt|r|)/|r| (r x s) + (1/2) (sin(dt|r|/2)/(|r|/2))^2 r x (r x s). */
void orc_spin_rotate(int k, long M, double dx, double dt, long np, const double *x,
                     const double *ga_y, const double *ga_z,
                     double *sx, double *sy, double *sz)
{
    for (long a = 0; a < np; ++a) {
        double Y = fe_value(k - 1, ga_y, M, dx, x[a]);
        double Z = fe_value(k - 1, ga_z, M, dx, x[a]);
        double r0 = 0.0, r1 = Z, r2 = -Y;
        double nr = sqrt(r1 * r1 + r2 * r2);
        double s0 = sx[a], s1 = sy[a], s2 = sz[a];
        /* c1 = r x s, c2 = r x (r x s) */
        double c1x = r1 * s2 - r2 * s1, c1y = r2 * s0 - r0 * s2, c1z = r0 * s1 - r1 * s0;
        double c2x = r1 * c1z - r2 * c1y, c2y = r2 * c1x - r0 * c1z, c2z = r0 * c1y - r1 * c1x;
        double f1, f2;
        if (nr > 0.0) {
            f1 = sin(dt * nr) / nr;
            double h = sin(0.5 * dt * nr) / (0.5 * nr);
            f2 = 0.5 * h * h;
        } else {
            f1 = dt;
            f2 = 0.5 * dt * dt;
        }
        sx[a] = s0 + f1 * c1x + f2 * c2x;
        sy[a] = s1 + f1 * c1y + f2 * c2y;
        sz[a] = s2 + f1 * c1z + f2 * c2z;
    }
}

/* Zeeman part of the discrete Hamiltonian without hbar:
 * sum_a w (s_y,a dA_z/dx(x_a) - s_z,a dA_y/dx(x_a)).                   */
double orc_spin_energy(int k, long M, double dx, long np, const double *x, double w,
                       const double *sy, const double *sz, const double *ga_y, const double *ga_z)
{
    double e = 0.0;
    for (long a = 0; a < np; ++a) {
        double Y = fe_value(k - 1, ga_y, M, dx, x[a]);
        double Z = fe_value(k - 1, ga_z, M, dx, x[a]);
        e += w * (sy[a] * Z - sz[a] * Y);
    }
    return e;
}
