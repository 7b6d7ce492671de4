/*
 * Plain CPU FP64 oracle of the discretised HJM-SV pricing PDE.
 *
 * TEST INFRASTRUCTURE ONLY: the GPU library is checked against this file; the
 * product path never loads it. Everything here is unblocked and in the order
 * the paper states the method, so that it can be read against the paper line
 * by line. It is serial as built for the tests; the few OpenMP pragmas only
 * share independent lines (or planes) among threads in the separate OpenMP
 * build that times the oracle on all host cores, with the same results:
 *
 *   Model and PDE ............ Section 3.1 (SDEs, bond formula with G(s)),
 *                              Section 3.2 (Eq. (1) and its coefficient list)
 *   Stretched grid ........... Section 4.3 (sinh metric, derivative transforms
 *                              g1..g6), Section 7.1 (Jacobian, parameters)
 *   Discretisation ........... Section 5 (theta scheme, centred differences,
 *                              tridiagonal operators, delta form)
 *   Douglas ADI .............. Section 5.1
 *   Craig-Sneyd family ....... Section 5.1 (the paper names Craig-Sneyd as
 *                              the alternative it tried; the modified CS and
 *                              Hundsdorfer-Verwer schemes are those of the
 *                              In 't Hout-Welfert work it cites)
 *   Softened payoff .......... Section 7.2 (control-volume average)
 *   y faces .................. Section 7.3 (first/second order one-sided)
 *   Exact bond (pin) ......... Section 3.1 bond formula, Section 4.1
 *
 * Readings taken where the paper is silent, garbled or self-inconsistent
 * (each repeated where it is used):
 *   R1  zeta(t) in the coefficient list of Section 3.2 is gamma(t).
 *   R2  The Jacobian printed in Section 7.1 has sinh; it is the derivative
 *       of the metric of Section 4.3, i.e. cosh.
 *   R3  g5 divides h5 by J_v (Section 4.3 prints J_r).
 *   R4  The centred first difference divides by 2h and the mixed one by
 *       4 h_r h_v (Section 5 prints h and h_r h_v).
 *   R5  The Douglas stages of Section 5.1 carry theta:
 *       (I - theta dt A_d) dU_d = dU_{d-1}.
 *   R6  Implicit operators at t^{n+1/2}, explicit F at t^n (Section 5,
 *       delta-form equation). With time-dependent coefficients this makes
 *       the step first order in time; the grid option explicit_midpoint
 *       takes F at t^{n+1/2} too, which restores second order.
 *   R7  The reaction term -r belongs to A_r.
 *   R8  Boundary faces: r = r_max always, and r = r_min when gamma == 0, are
 *       Dirichlet with data g(t, r, y): the exact bond for a bond and
 *       max(P(t,T) - Delta_M P(t,T_M), 0) for a caplet. Every other face
 *       (v = 0, v = v_max, y = 0, y = y_max, r = 0 when gamma > 0) drops its
 *       own normal second derivative and takes the normal first derivative
 *       one-sided into the domain: second order in F (first order on y faces
 *       when y_boundary_order == 1), first order in the implicit operators so
 *       that they stay tridiagonal. The r-v mixed term is dropped only where
 *       its centred stencil leaves the grid, i.e. on the v faces and the
 *       non-Dirichlet r face; the y faces keep it, because y has no diffusion
 *       and no y-mixed term, so Eq. (1) of Section 3.2 holds unchanged in the
 *       r-v directions on y = 0 (the plane the price is read from) and on
 *       y = y_max. Dirichlet wins on edges.
 *   R9  Node counts include both boundaries; nodes xi_i = i/(n-1).
 *   R10 State at the readout: r = f(0,0), v = v0, y = 0; tensor-product
 *       cubic Lagrange interpolation in (xi_r, xi_v) on the y = 0 plane.
 *   R11 The softened payoff averages over the physical control volume
 *       [z(xi_i - h/2), z(xi_i + h/2)] clipped to the domain, in r and y; the
 *       r integral is closed form, the y integral 8-point Gauss-Legendre.
 *   R12 r^gamma is taken as 1 when gamma == 0 (any r), so negative rates are
 *       allowed in the Gaussian case only.
 *   R13 Craig-Sneyd family: a second explicit stage and a second sweep of
 *       the three line solves, as In 't Hout and Welfert define CS, modified
 *       CS and Hundsdorfer-Verwer. Every explicit operator of such a step is
 *       taken at t^{n+1/2} (the operator frozen over the step, whatever
 *       explicit_midpoint says), which keeps the schemes second order with
 *       the time-dependent drift; the implicit stages use the same line
 *       operators as the Douglas stages (R5, R6, R8).
 *   R14 Discrete initial curve (Section 6.1): the paper smooths the discount
 *       factors with splines so that df(0,T)/dT is continuous; here a natural
 *       cubic spline of ln P(0,t) through (0, 0) and the knots (zero second
 *       derivative at both ends), f = -(ln P)', df/dt = -(ln P)''; past the
 *       last knot ln P continues linearly (flat forward).
 */
#include "hjm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double ORC_PI = 3.14159265358979323846;

/* Natural cubic spline of ln P(0,t) of a discrete curve (R14). */
typedef struct {
    int m;                                 /* nodes: the origin and the knots */
    double tau[ORC_MAX_KNOTS + 1];         /* node times */
    double y[ORC_MAX_KNOTS + 1];           /* ln P(0, tau) */
    double M[ORC_MAX_KNOTS + 1];           /* second derivatives */
} orc_knot_spline;

struct orc_ctx {
    orc_curve c;
    orc_knot_spline sp;  /* the discrete curve's spline (kind 2) */
    orc_model m;
    orc_grid g;
    orc_inst in;
    double K;        /* absolute strike (caplet) */
    double DM;       /* Delta_M = 1 + (T_M - T) K, Section 3.2 */
    double dt;       /* T / n_steps */
    int n[3];        /* nodes on r, v, y */
    double h[3];     /* 1/(n-1) in the computational coordinate */
    double lo[3], hi[3], alpha[3], centre[3];
    double *z[3], *J[3], *J2[3];
    int r_lo_dirichlet;
};

/* ------------------------------------------------------------------ curve */

/* Natural cubic spline of ln P(0,t) through (0, 0) and the knots (R14):
 * nodes tau_0 = 0 < tau_1 < ... < tau_{m-1}, values y_i = ln P(0, tau_i),
 * second derivatives M_i with M_0 = M_{m-1} = 0 and, inside, continuity of
 * the first derivative:
 *   h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1}
 *       = 6 ((y_{i+1} - y_i) / h_i - (y_i - y_{i-1}) / h_{i-1}). */
static void knot_spline_build(const orc_curve* c, orc_knot_spline* sp)
{
    int m = c->n_knots + 1;
    sp->m = m;
    sp->tau[0] = 0.0;
    sp->y[0] = 0.0;
    for (int i = 1; i < m; ++i) {
        sp->tau[i] = c->knot_t[i - 1];
        sp->y[i] = log(c->knot_P[i - 1]);
    }
    for (int i = 0; i < m; ++i) sp->M[i] = 0.0;
    if (m < 3) return;
    /* Thomas on the interior unknowns M_1 .. M_{m-2} */
    double cp[ORC_MAX_KNOTS + 1], dp[ORC_MAX_KNOTS + 1];
    for (int i = 1; i <= m - 2; ++i) {
        double hl = sp->tau[i] - sp->tau[i - 1], hr = sp->tau[i + 1] - sp->tau[i];
        double a = hl, b = 2.0 * (hl + hr), cc = hr;
        double d = 6.0 * ((sp->y[i + 1] - sp->y[i]) / hr - (sp->y[i] - sp->y[i - 1]) / hl);
        if (i == 1) {
            cp[i] = cc / b;
            dp[i] = d / b;
        } else {
            double piv = b - a * cp[i - 1];
            cp[i] = cc / piv;
            dp[i] = (d - a * dp[i - 1]) / piv;
        }
    }
    sp->M[m - 2] = dp[m - 2];
    for (int i = m - 3; i >= 1; --i) sp->M[i] = dp[i] - cp[i] * sp->M[i + 1];
}

/* ln P(0,t) and its first two derivatives from the spline. */
static void knot_spline_eval(const orc_knot_spline* sp, double t, double* s, double* ds, double* d2s)
{
    int m = sp->m;
    if (t >= sp->tau[m - 1]) {
        /* slope at the last node from the last piece (b = 1, a = 0) */
        double h = sp->tau[m - 1] - sp->tau[m - 2];
        double slope = (sp->y[m - 1] - sp->y[m - 2]) / h + h / 6.0 * (sp->M[m - 2] + 2.0 * sp->M[m - 1]);
        *s = sp->y[m - 1] + slope * (t - sp->tau[m - 1]);
        *ds = slope;
        *d2s = 0.0;
        return;
    }
    int i = 0;
    while (i < m - 2 && t >= sp->tau[i + 1]) ++i;
    double h = sp->tau[i + 1] - sp->tau[i];
    double a = (sp->tau[i + 1] - t) / h, b = (t - sp->tau[i]) / h;
    *s = a * sp->y[i] + b * sp->y[i + 1] + ((a * a * a - a) * sp->M[i] + (b * b * b - b) * sp->M[i + 1]) * h * h / 6.0;
    *ds = (sp->y[i + 1] - sp->y[i]) / h + (-(3.0 * a * a - 1.0) * sp->M[i] + (3.0 * b * b - 1.0) * sp->M[i + 1]) * h / 6.0;
    *d2s = a * sp->M[i] + b * sp->M[i + 1];
}

static void knot_curve_at(const orc_curve* c, double t, double* s, double* ds, double* d2s)
{
    orc_knot_spline sp;
    knot_spline_build(c, &sp);
    knot_spline_eval(&sp, t, s, ds, d2s);
}

/* Initial forward curve f(0,t), Section 2 (f = -d ln p / dT). */
double orc_curve_f(const orc_curve* c, double t)
{
    if (c->kind == 0) return c->flat_rate;
    if (c->kind == 2) {
        double s, ds, d2s;
        knot_curve_at(c, t, &s, &ds, &d2s);
        return -ds;
    }
    double e = exp(-t / c->tau);
    return c->beta0 + c->beta1 * e + c->beta2 * (t / c->tau) * e;
}

double orc_curve_dfdt(const orc_curve* c, double t)
{
    if (c->kind == 0) return 0.0;
    if (c->kind == 2) {
        double s, ds, d2s;
        knot_curve_at(c, t, &s, &ds, &d2s);
        return -d2s;
    }
    double e = exp(-t / c->tau);
    return -c->beta1 / c->tau * e + c->beta2 / c->tau * e * (1.0 - t / c->tau);
}

/* P(0,t) = exp(-int_0^t f(0,s) ds), Section 2. */
double orc_curve_P(const orc_curve* c, double t)
{
    if (c->kind == 0) return exp(-c->flat_rate * t);
    if (c->kind == 2) {
        double s, ds, d2s;
        knot_curve_at(c, t, &s, &ds, &d2s);
        return exp(s);
    }
    double e = exp(-t / c->tau);
    double integral = c->beta0 * t + c->beta1 * c->tau * (1.0 - e)
                    + c->beta2 * (c->tau * (1.0 - e) - t * e);
    return exp(-integral);
}

/* G(s) = (1 - e^{-kappa s}) / kappa, Section 3.1; G(s) = s when kappa = 0. */
double orc_G(double kappa, double s)
{
    if (kappa == 0.0) return s;
    return -expm1(-kappa * s) / kappa;
}

/* Bond price p(t,S) at state (r, y), Section 3.1 with x = r - f(0,t). */
double orc_bond(const orc_curve* c, const orc_model* m, double t, double S,
                double r, double y)
{
    double G = orc_G(m->kappa, S - t);
    double x = r - orc_curve_f(c, t);
    return orc_curve_P(c, S) / orc_curve_P(c, t) * exp(-G * x - 0.5 * G * G * y);
}

static double norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Caplet paying max(1 - Delta_M p(T,T_M), 0) at T (Section 3.2) when the
 * volatility is deterministic (gamma = 0, epsilon = 0, v0 = 1, so eta = lambda):
 * ln p(T,T_M) is Gaussian with variance sigma_p^2 = G(T_M-T)^2 Var x(T),
 * Var x(T) = lambda^2 (1 - e^{-2 kappa T}) / (2 kappa), and the price is
 * Delta_M times a put on that bond with strike 1/Delta_M. */
double orc_gauss_caplet(const orc_curve* c, const orc_model* m, double T,
                        double TM, double K)
{
    double DM = 1.0 + (TM - T) * K;
    double P0T = orc_curve_P(c, T), P0M = orc_curve_P(c, TM);
    double var_x = m->kappa > 0.0
        ? m->lambda * m->lambda * (-expm1(-2.0 * m->kappa * T)) / (2.0 * m->kappa)
        : m->lambda * m->lambda * T;
    double sp = orc_G(m->kappa, TM - T) * sqrt(var_x);
    double h = log(DM * P0M / P0T) / sp + 0.5 * sp;
    return P0T * norm_cdf(-h + sp) - DM * P0M * norm_cdf(-h);
}

/* Simple forward rate over [T, T_M]: the strike that makes the caplet ATM. */
double orc_atm_strike(const orc_curve* c, double T, double TM)
{
    return (orc_curve_P(c, T) / orc_curve_P(c, TM) - 1.0) / (TM - T);
}

/* ------------------------------------------------------------------- grid */

/* Sinh metric of Section 4.3: z(xi) = K + alpha sinh(c2 xi + c1 (1 - xi)),
 * J = dz/dxi, J2 = d2z/dxi2 (cosh in J: reading R2). alpha <= 0: uniform. */
static void metric_at(double xi, double z0, double zinf, double alpha, double K,
                      double* z, double* J, double* J2)
{
    if (alpha <= 0.0) {
        *z = z0 + (zinf - z0) * xi;
        *J = zinf - z0;
        *J2 = 0.0;
        return;
    }
    double c1 = asinh((z0 - K) / alpha);
    double c2 = asinh((zinf - K) / alpha);
    double a = c2 * xi + c1 * (1.0 - xi);
    *z = K + alpha * sinh(a);
    *J = alpha * (c2 - c1) * cosh(a);
    *J2 = alpha * (c2 - c1) * (c2 - c1) * sinh(a);
    /* The end points are the domain bounds exactly (r = 0 must not round
     * below 0 when gamma > 0). */
    if (xi == 0.0) *z = z0;
    if (xi == 1.0) *z = zinf;
}

static double metric_z(const orc_ctx* x, int d, double xi)
{
    double z, J, J2;
    metric_at(xi, x->lo[d], x->hi[d], x->alpha[d], x->centre[d], &z, &J, &J2);
    return z;
}

/* Inverse of the metric: the computational coordinate of a physical z. */
static double metric_xi(const orc_ctx* x, int d, double z)
{
    double z0 = x->lo[d], zinf = x->hi[d], alpha = x->alpha[d], K = x->centre[d];
    if (alpha <= 0.0) return (z - z0) / (zinf - z0);
    double c1 = asinh((z0 - K) / alpha);
    double c2 = asinh((zinf - K) / alpha);
    return (asinh((z - K) / alpha) - c1) / (c2 - c1);
}

/* ------------------------------------------------------------ life cycle */

static int finite_all(const double* v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

int orc_ctx_create(const orc_curve* c, const orc_model* m, const orc_grid* g,
                   const orc_inst* in, orc_ctx** out)
{
    *out = NULL;
    double chk[] = {c->flat_rate, c->beta0, c->beta1, c->beta2, c->tau,
                    m->kappa, m->lambda, m->gamma, m->theta, m->epsilon, m->rho, m->v0,
                    g->r_min, g->r_max, g->y_max, g->v_max, g->alpha_r, g->alpha_y,
                    g->alpha_v, g->k_r, g->k_v, g->theta_adi, in->T, in->TM, in->K};
    if (!finite_all(chk, (int)(sizeof chk / sizeof chk[0]))) return 1;
    if (c->kind != 0 && c->kind != 1 && c->kind != 2) return 1;
    if (c->kind == 1 && !(c->tau > 0.0)) return 1;
    if (c->kind == 2) {
        if (c->n_knots < 1 || c->n_knots > ORC_MAX_KNOTS) return 1;
        for (int i = 0; i < c->n_knots; ++i) {
            if (!isfinite(c->knot_t[i]) || !isfinite(c->knot_P[i]) || !(c->knot_P[i] > 0.0)) return 1;
            if (!(c->knot_t[i] > (i ? c->knot_t[i - 1] : 0.0))) return 1;
        }
    }
    if (g->n_r < 5 || g->n_v < 5 || g->n_y < 5 || g->n_steps < 1) return 1;
    if (!(g->r_max > g->r_min) || !(g->y_max > 0.0) || !(g->v_max > 0.0)) return 1;
    if (m->gamma < 0.0 || m->gamma > 1.0) return 1;
    if (m->gamma > 0.0 && g->r_min != 0.0) return 1;
    if (m->rho < -1.0 || m->rho > 1.0) return 1;
    if (m->kappa < 0.0 || m->lambda < 0.0 || m->epsilon < 0.0 || m->theta < 0.0) return 1;
    if (m->v0 < 0.0 || m->v0 > g->v_max) return 1;
    if (g->theta_adi < 0.0 || g->theta_adi > 1.0) return 1;
    if (g->y_boundary_order != 1 && g->y_boundary_order != 2) return 1;
    if (g->explicit_midpoint != 0 && g->explicit_midpoint != 1) return 1;
    if (g->scheme < 0 || g->scheme > 3) return 1;
    if (!(in->T > 0.0)) return 1;
    if (in->kind != 0 && in->kind != 1 && in->kind != 2) return 1;
    double r0 = orc_curve_f(c, 0.0);
    if (r0 < g->r_min || r0 > g->r_max) return 1;

    orc_ctx* x = (orc_ctx*)calloc(1, sizeof *x);
    if (!x) return 1;
    x->c = *c;
    if (c->kind == 2) knot_spline_build(c, &x->sp);
    x->m = *m;
    x->g = *g;
    x->in = *in;
    x->K = 0.0;
    x->DM = 1.0;
    if (in->kind == 1 || in->kind == 2) {
        if (!(in->TM > in->T)) { free(x); return 1; }
        x->K = in->K + (in->strike_atm_relative ? orc_atm_strike(c, in->T, in->TM) : 0.0);
        x->DM = 1.0 + (in->TM - in->T) * x->K;
        if (!(x->DM > 0.0)) { free(x); return 1; }
    }
    x->dt = in->T / g->n_steps;
    x->n[0] = g->n_r; x->n[1] = g->n_v; x->n[2] = g->n_y;
    x->lo[0] = g->r_min; x->hi[0] = g->r_max; x->alpha[0] = g->alpha_r;
    x->centre[0] = g->center_r_on_strike ? (in->kind != 0 ? x->K : r0) : g->k_r;
    x->lo[1] = 0.0; x->hi[1] = g->v_max; x->alpha[1] = g->alpha_v; x->centre[1] = g->k_v;
    x->lo[2] = 0.0; x->hi[2] = g->y_max; x->alpha[2] = g->alpha_y; x->centre[2] = 0.0;
    for (int d = 0; d < 3; ++d) {
        int n = x->n[d];
        x->h[d] = 1.0 / (n - 1);
        x->z[d] = (double*)malloc(sizeof(double) * n);
        x->J[d] = (double*)malloc(sizeof(double) * n);
        x->J2[d] = (double*)malloc(sizeof(double) * n);
        for (int i = 0; i < n; ++i)
            metric_at(i * x->h[d], x->lo[d], x->hi[d], x->alpha[d], x->centre[d],
                      &x->z[d][i], &x->J[d][i], &x->J2[d][i]);
    }
    x->r_lo_dirichlet = (m->gamma == 0.0);
    *out = x;
    return 0;
}

void orc_ctx_destroy(orc_ctx* x)
{
    if (!x) return;
    for (int d = 0; d < 3; ++d) {
        free(x->z[d]);
        free(x->J[d]);
        free(x->J2[d]);
    }
    free(x);
}

long orc_n_points(const orc_ctx* x) { return (long)x->n[0] * x->n[1] * x->n[2]; }
double orc_strike(const orc_ctx* x) { return x->K; }
double orc_dt(const orc_ctx* x) { return x->dt; }

void orc_axis(const orc_ctx* x, int axis, double* z, double* J, double* J2)
{
    for (int i = 0; i < x->n[axis]; ++i) {
        z[i] = x->z[axis][i];
        J[i] = x->J[axis][i];
        J2[i] = x->J2[axis][i];
    }
}

/* Backward time tau = n dt runs from the payoff date; calendar t = T - tau. */
double orc_time(const orc_ctx* x, double n) { return x->in.T - n * x->dt; }

static long at(const orc_ctx* x, int i, int k, int j)
{
    return i + (long)x->n[0] * (k + (long)x->n[1] * j);
}

static int r_dirichlet(const orc_ctx* x, int i)
{
    return i == x->n[0] - 1 || (i == 0 && x->r_lo_dirichlet);
}

/* ---------------------------------------------------------- coefficients */

/* The PDE coefficients of Section 3.2 at a physical state (reading R1, R12). */
typedef struct { double zrr, zvv, zrv, mur, muv, muy, r; } coeffs;

static coeffs coeffs_at(const orc_ctx* x, int i, int k, int j, double t)
{
    const orc_model* m = &x->m;
    double r = x->z[0][i], v = x->z[1][k], y = x->z[2][j];
    double rg = (m->gamma == 0.0) ? 1.0 : pow(r, m->gamma);
    double r2g = (m->gamma == 0.0) ? 1.0 : pow(r, 2.0 * m->gamma);
    coeffs q;
    q.zrr = 0.5 * m->lambda * m->lambda * r2g * v;
    q.zvv = 0.5 * m->epsilon * m->epsilon * v;
    q.zrv = m->lambda * rg * m->epsilon * m->rho * v;
    double f0, df0;
    if (x->c.kind == 2) {
        double s, ds, d2s;
        knot_spline_eval(&x->sp, t, &s, &ds, &d2s);
        f0 = -ds;
        df0 = -d2s;
    } else {
        f0 = orc_curve_f(&x->c, t);
        df0 = orc_curve_dfdt(&x->c, t);
    }
    q.mur = df0 - m->kappa * (r - f0) + y;
    q.muv = m->theta * (1.0 - v);
    q.muy = m->lambda * m->lambda * r2g * v - 2.0 * m->kappa * y;
    q.r = r;
    return q;
}

/* Dirichlet data g(t, r, y) (reading R8). Section 4.1 proposes the exact
 * bond as boundary data; for the caplet and the floorlet the deep in/out-of-
 * the-money value, the positive part of the forward contract
 * p(t,T) - Delta_M p(t,T_M) (caplet) or of its negative (floorlet). */
double orc_dirichlet(const orc_ctx* x, double t, double r, double y)
{
    double pT = orc_bond(&x->c, &x->m, t, x->in.T, r, y);
    if (x->in.kind == 0) return pT;
    double pM = orc_bond(&x->c, &x->m, t, x->in.TM, r, y);
    double v = x->in.kind == 1 ? pT - x->DM * pM : x->DM * pM - pT;
    return v > 0.0 ? v : 0.0;
}

/* --------------------------------------------------- explicit operators */

/* One-sided first differences into the domain, Section 7.3. */
static double d1_fwd(double u0, double u1, double u2, double h, int order)
{
    return order == 1 ? (u1 - u0) / h : (-3.0 * u0 + 4.0 * u1 - u2) / (2.0 * h);
}
static double d1_bwd(double un, double un1, double un2, double h, int order)
{
    return order == 1 ? (un - un1) / h : (3.0 * un - 4.0 * un1 + un2) / (2.0 * h);
}

/* A_d applied at one non-Dirichlet node, with the centred differences of
 * Section 5 (reading R4) and the metric transforms of Section 4.3:
 *   A_r U = g1 d_rr U + g4 d_r U - r U,  g1 = zeta_rr/J_r^2,
 *           g4 = mu_r/J_r - zeta_rr J2_r/J_r^3
 *   A_v U = g2 d_vv U + g5 d_v U,        g2 = zeta_vv/J_v^2,
 *           g5 = mu_v/J_v - zeta_vv J2_v/J_v^3           (reading R3)
 *   A_y U = g6 d_y U,                    g6 = mu_y/J_y
 *   A_0 U = g3 d_rv U,                   g3 = zeta_rv/(J_r J_v)
 * On a degenerate face the physical second derivative (both its parts) and
 * the mixed term are dropped and the first derivative is one-sided. */
static double apply_node(const orc_ctx* x, int d, double t, const double* U,
                         int i, int k, int j)
{
    coeffs q = coeffs_at(x, i, k, j, t);
    int nr = x->n[0], nv = x->n[1], ny = x->n[2];
    double u = U[at(x, i, k, j)];
    if (d == 0) {
        double h = x->h[0], J = x->J[0][i], J2 = x->J2[0][i];
        double val;
        if (i > 0 && i < nr - 1) {
            double up = U[at(x, i + 1, k, j)], um = U[at(x, i - 1, k, j)];
            double g1 = q.zrr / (J * J);
            double g4 = q.mur / J - q.zrr * J2 / (J * J * J);
            val = g1 * (up - 2.0 * u + um) / (h * h) + g4 * (up - um) / (2.0 * h);
        } else { /* i == 0, degenerate face r = 0 (gamma > 0) */
            val = q.mur / J * d1_fwd(u, U[at(x, 1, k, j)], U[at(x, 2, k, j)], h, 2);
        }
        return val - q.r * u;
    }
    if (d == 1) {
        double h = x->h[1], J = x->J[1][k], J2 = x->J2[1][k];
        if (k > 0 && k < nv - 1) {
            double up = U[at(x, i, k + 1, j)], um = U[at(x, i, k - 1, j)];
            double g2 = q.zvv / (J * J);
            double g5 = q.muv / J - q.zvv * J2 / (J * J * J);
            return g2 * (up - 2.0 * u + um) / (h * h) + g5 * (up - um) / (2.0 * h);
        }
        if (k == 0)
            return q.muv / J * d1_fwd(u, U[at(x, i, 1, j)], U[at(x, i, 2, j)], h, 2);
        return q.muv / J * d1_bwd(u, U[at(x, i, nv - 2, j)], U[at(x, i, nv - 3, j)], h, 2);
    }
    if (d == 2) {
        double h = x->h[2], J = x->J[2][j];
        double g6 = q.muy / J;
        int ord = x->g.y_boundary_order;
        if (j > 0 && j < ny - 1)
            return g6 * (U[at(x, i, k, j + 1)] - U[at(x, i, k, j - 1)]) / (2.0 * h);
        if (j == 0)
            return g6 * d1_fwd(u, U[at(x, i, k, 1)], U[at(x, i, k, 2)], h, ord);
        return g6 * d1_bwd(u, U[at(x, i, k, ny - 2)], U[at(x, i, k, ny - 3)], h, ord);
    }
    /* d == 3: mixed r-v term, interior of both r and v only. */
    if (i > 0 && i < nr - 1 && k > 0 && k < nv - 1) {
        double g3 = q.zrv / (x->J[0][i] * x->J[1][k]);
        double s = U[at(x, i + 1, k + 1, j)] - U[at(x, i + 1, k - 1, j)]
                 - U[at(x, i - 1, k + 1, j)] + U[at(x, i - 1, k - 1, j)];
        return g3 * s / (4.0 * x->h[0] * x->h[1]);
    }
    return 0.0;
}

void orc_apply_dir(const orc_ctx* x, int d, double t, const double* U, double* AU)
{
#pragma omp parallel for
    for (int j = 0; j < x->n[2]; ++j)
        for (int k = 0; k < x->n[1]; ++k)
            for (int i = 0; i < x->n[0]; ++i)
                AU[at(x, i, k, j)] = r_dirichlet(x, i) ? 0.0 : apply_node(x, d, t, U, i, k, j);
}

/* F(U) of Section 5: the sum of all four split operators. */
void orc_apply_F(const orc_ctx* x, double t, const double* U, double* F)
{
#pragma omp parallel for
    for (int j = 0; j < x->n[2]; ++j)
        for (int k = 0; k < x->n[1]; ++k)
            for (int i = 0; i < x->n[0]; ++i) {
                double s = 0.0;
                if (!r_dirichlet(x, i))
                    for (int d = 0; d < 4; ++d) s += apply_node(x, d, t, U, i, k, j);
                F[at(x, i, k, j)] = s;
            }
}

/* Delta U^0 = dt F(U^n; t^n) (Section 5.1, first Douglas stage, reading R6);
 * on Dirichlet nodes the increment that lands on g(t^{n+1}) (reading R8).
 * With explicit_midpoint set, F is taken at t^{n+1/2} instead, the time at
 * which the implicit operators are taken (an option, not the paper's form);
 * the Craig-Sneyd family always takes it there (R13). */
void orc_explicit(const orc_ctx* x, int n, const double* U, double* dU0)
{
    int mid = x->g.explicit_midpoint || x->g.scheme != 0;
    double t = orc_time(x, mid ? n + 0.5 : n), t1 = orc_time(x, n + 1);
    orc_apply_F(x, t, U, dU0);
#pragma omp parallel for
    for (int j = 0; j < x->n[2]; ++j)
        for (int k = 0; k < x->n[1]; ++k)
            for (int i = 0; i < x->n[0]; ++i) {
                long p = at(x, i, k, j);
                if (r_dirichlet(x, i))
                    dU0[p] = orc_dirichlet(x, t1, x->z[0][i], x->z[2][j]) - U[p];
                else
                    dU0[p] *= x->dt;
            }
}

/* ---------------------------------------------------- implicit operators */

/* Row of A_d at one node of a line: the tridiagonal operators L_r, L_v, L_y
 * of Section 5, with first-order one-sided rows on degenerate faces and zero
 * rows on Dirichlet nodes (reading R8). */
static void row_A(const orc_ctx* x, int d, double t, int i, int k, int j,
                  double* lower, double* diag, double* upper)
{
    *lower = *diag = *upper = 0.0;
    if (r_dirichlet(x, i)) return;
    coeffs q = coeffs_at(x, i, k, j, t);
    if (d == 0) {
        double h = x->h[0], J = x->J[0][i], J2 = x->J2[0][i];
        if (i > 0) {
            double g1 = q.zrr / (J * J);
            double g4 = q.mur / J - q.zrr * J2 / (J * J * J);
            *lower = g1 / (h * h) - g4 / (2.0 * h);
            *diag = -2.0 * g1 / (h * h);
            *upper = g1 / (h * h) + g4 / (2.0 * h);
        } else {
            double b = q.mur / J / h;
            *diag = -b;
            *upper = b;
        }
        *diag -= q.r;
        return;
    }
    if (d == 1) {
        int nv = x->n[1];
        double h = x->h[1], J = x->J[1][k], J2 = x->J2[1][k];
        if (k > 0 && k < nv - 1) {
            double g2 = q.zvv / (J * J);
            double g5 = q.muv / J - q.zvv * J2 / (J * J * J);
            *lower = g2 / (h * h) - g5 / (2.0 * h);
            *diag = -2.0 * g2 / (h * h);
            *upper = g2 / (h * h) + g5 / (2.0 * h);
        } else if (k == 0) {
            double b = q.muv / J / h;
            *diag = -b;
            *upper = b;
        } else {
            double b = q.muv / J / h;
            *lower = -b;
            *diag = b;
        }
        return;
    }
    int ny = x->n[2];
    double h = x->h[2], g6 = q.muy / x->J[2][j];
    if (j > 0 && j < ny - 1) {
        *lower = -g6 / (2.0 * h);
        *upper = g6 / (2.0 * h);
    } else if (j == 0) {
        *diag = -g6 / h;
        *upper = g6 / h;
    } else {
        *lower = -g6 / h;
        *diag = g6 / h;
    }
}

/* Node coordinates of position p on line `line` of direction d. */
static void line_node(const orc_ctx* x, int d, long line, int p, int* i, int* k, int* j)
{
    if (d == 0) { *i = p; *k = (int)(line % x->n[1]); *j = (int)(line / x->n[1]); }
    else if (d == 1) { *i = (int)(line % x->n[0]); *k = p; *j = (int)(line / x->n[0]); }
    else { *i = (int)(line % x->n[0]); *k = (int)(line / x->n[0]); *j = p; }
}

static long n_lines(const orc_ctx* x, int d)
{
    return orc_n_points(x) / x->n[d];
}

void orc_line_matrix(const orc_ctx* x, int d, double t, long line,
                     double* sub, double* diag, double* sup)
{
    double w = x->g.theta_adi * x->dt;
    for (int p = 0; p < x->n[d]; ++p) {
        int i, k, j;
        double lo, di, up;
        line_node(x, d, line, p, &i, &k, &j);
        row_A(x, d, t, i, k, j, &lo, &di, &up);
        sub[p] = -w * lo;
        diag[p] = 1.0 - w * di;
        sup[p] = -w * up;
    }
}

/* Thomas algorithm (Section 5): forward elimination, back substitution. */
static void thomas(int n, const double* a, const double* b, const double* c,
                   const double* d, double* x, double* cp, double* dp)
{
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; ++i) {
        double m = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / m;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

long orc_solve_dir(const orc_ctx* x, int d, double t, const double* rhs, double* out)
{
    int n = x->n[d];
    long bad = 0;
    /* Lines are independent; the OpenMP build of this file (the multi-core
     * timing of the oracle) shares them among threads, each with its own
     * scratch, and gives the same results as the serial build. */
#pragma omp parallel reduction(+ : bad)
    {
    double* a = (double*)malloc(sizeof(double) * n * 7);
    double *b = a + n, *c = b + n, *r = c + n, *s = r + n, *cp = s + n, *dp = cp + n;
#pragma omp for
    for (long line = 0; line < n_lines(x, d); ++line) {
        orc_line_matrix(x, d, t, line, a, b, c);
        for (int p = 0; p < n; ++p) {
            int i, k, j;
            line_node(x, d, line, p, &i, &k, &j);
            r[p] = rhs[at(x, i, k, j)];
            if (fabs(b[p]) < fabs(a[p]) + fabs(c[p])) ++bad;
        }
        thomas(n, a, b, c, r, s, cp, dp);
        for (int p = 0; p < n; ++p) {
            int i, k, j;
            line_node(x, d, line, p, &i, &k, &j);
            out[at(x, i, k, j)] = s[p];
        }
    }
    free(a);
    }
    return bad;
}

/* ------------------------------------------------------------ Douglas */

/* One ADI step n -> n+1 in place. Douglas (Section 5.1, readings R5, R6):
 *   Y0 = U^n + dt F(U^n)                       (dU0 of orc_explicit)
 *   Yd = Y(d-1) + theta dt A_d (Yd - U^n),  d = r, v, y
 *        i.e. (I - theta dt A_d(t^{n+1/2})) (Yd - U^n) = Y(d-1) - U^n
 *   U^{n+1} = Yy.
 * The Craig-Sneyd family (R13) continues from Y0 and Yy (= Y3):
 *   CS:  Z0 = Y0 + 1/2 dt (A_0 Y3 - A_0 U^n)
 *   MCS: Z0 = Y0 + theta dt (A_0 Y3 - A_0 U^n)
 *               + (1/2 - theta) dt (F(Y3) - F(U^n))
 *   HV:  Z0 = Y0 + 1/2 dt (F(Y3) - F(U^n))
 *   Zd = Z(d-1) + theta dt A_d (Zd - B),  B = U^n (CS, MCS) or Y3 (HV)
 *   U^{n+1} = Zy.
 * A_0 is the mixed term, F the full explicit operator (both zero on
 * Dirichlet nodes, where Y0 = Y3 = Z0 = g(t^{n+1})). */
void orc_step(const orc_ctx* x, int n, double* U)
{
    long N = orc_n_points(x);
    int sch = x->g.scheme;
    double th = orc_time(x, n + 0.5), dt = x->dt, theta = x->g.theta_adi;
    double* w = (double*)malloc(sizeof(double) * N * 5);
    double *z = w, *a = w + N, *b = w + 2 * N, *y3 = w + 3 * N, *f = w + 4 * N;
    /* z = Y0 - U^n; a = Y3 - U^n after the three solves */
    orc_explicit(x, n, U, z);
    orc_solve_dir(x, 0, th, z, a);
    orc_solve_dir(x, 1, th, a, b);
    orc_solve_dir(x, 2, th, b, a);
    if (sch == 0) {
        for (long p = 0; p < N; ++p) U[p] += a[p];
        free(w);
        return;
    }
    for (long p = 0; p < N; ++p) y3[p] = U[p] + a[p];
    /* z = Z0 - U^n */
    if (sch == 1 || sch == 2) {
        double c = sch == 1 ? 0.5 : theta;
        orc_apply_dir(x, 3, th, y3, b);
        orc_apply_dir(x, 3, th, U, f);
        for (long p = 0; p < N; ++p) z[p] += c * dt * (b[p] - f[p]);
    }
    if (sch == 2 || sch == 3) {
        double c = sch == 2 ? 0.5 - theta : 0.5;
        orc_apply_F(x, th, y3, b);
        orc_apply_F(x, th, U, f);
        for (long p = 0; p < N; ++p) z[p] += c * dt * (b[p] - f[p]);
    }
    /* z = Z0 - B, then the three solves give Zy - B */
    if (sch == 3)
        for (long p = 0; p < N; ++p) z[p] -= a[p];
    orc_solve_dir(x, 0, th, z, b);
    orc_solve_dir(x, 1, th, b, f);
    orc_solve_dir(x, 2, th, f, b);
    for (long p = 0; p < N; ++p) U[p] = (sch == 3 ? y3[p] : U[p]) + b[p];
    free(w);
}

/* ------------------------------------------------------- terminal field */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on the
 * Legendre polynomial P_n (three-term recurrence). */
static void gauss_legendre(int n, double* xs, double* ws)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        xs[i] = z;
        ws[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Average over r in [ra, rb] of the floorlet payoff max(Delta_M p(T,T_M) - 1,
 * 0) at fixed y: with p(T,T_M) = A(y) e^{-G r} it is positive for r below
 * r* = ln(Delta_M A)/G, and its integral there is closed form. */
static double floor_avg_r(const orc_ctx* x, double ra, double rb, double y)
{
    double T = x->in.T, TM = x->in.TM;
    double G = orc_G(x->m.kappa, TM - T);
    double A = orc_curve_P(&x->c, TM) / orc_curve_P(&x->c, T)
             * exp(G * orc_curve_f(&x->c, T) - 0.5 * G * G * y);
    double DA = x->DM * A;
    if (!(rb > ra)) {
        double v = DA * exp(-G * ra) - 1.0;
        return v > 0.0 ? v : 0.0;
    }
    double rstar = log(DA) / G;
    double mhi = rb < rstar ? rb : rstar;
    if (mhi <= ra) return 0.0;
    /* int_ra^mhi (DA e^{-G r} - 1) dr */
    double integral = DA * exp(-G * ra) * (-expm1(-G * (mhi - ra))) / G - (mhi - ra);
    return integral / (rb - ra);
}

/* Average over r in [ra, rb] of the caplet payoff max(1 - Delta_M p(T,T_M), 0)
 * at fixed y (Section 3.2 payoff, Section 7.2 average). With p(T,T_M) =
 * A(y) e^{-G r} the payoff is positive for r above r* = ln(Delta_M A)/G and
 * its integral there is closed form. The floorlet pays the other side,
 * max(Delta_M p(T,T_M) - 1, 0), positive below r*. */
static double payoff_avg_r(const orc_ctx* x, double ra, double rb, double y)
{
    if (x->in.kind == 2) return floor_avg_r(x, ra, rb, y);
    double T = x->in.T, TM = x->in.TM;
    double G = orc_G(x->m.kappa, TM - T);
    double A = orc_curve_P(&x->c, TM) / orc_curve_P(&x->c, T)
             * exp(G * orc_curve_f(&x->c, T) - 0.5 * G * G * y);
    double DA = x->DM * A;
    if (!(rb > ra)) {
        double v = 1.0 - DA * exp(-G * ra);
        return v > 0.0 ? v : 0.0;
    }
    double rstar = log(DA) / G;
    double mlo = ra > rstar ? ra : rstar;
    if (mlo >= rb) return 0.0;
    /* int_mlo^rb (1 - DA e^{-G r}) dr */
    double integral = (rb - mlo) - DA * exp(-G * mlo) * (-expm1(-G * (rb - mlo))) / G;
    return integral / (rb - ra);
}

/* Terminal field U^0 at t = T: 1 for the bond (Section 3.2); the payoff
 * averaged over each node's control volume in r and y for the caplet and the
 * floorlet (Section 7.2, reading R11). v plays no role. */
void orc_terminal(const orc_ctx* x, double* U)
{
    long N = orc_n_points(x);
    if (x->in.kind == 0) {
        for (long p = 0; p < N; ++p) U[p] = 1.0;
        return;
    }
    double gx[8], gw[8];
    gauss_legendre(8, gx, gw);
    int nr = x->n[0], nv = x->n[1], ny = x->n[2];
    for (int j = 0; j < ny; ++j) {
        double xa = j * x->h[2] - 0.5 * x->h[2], xb = j * x->h[2] + 0.5 * x->h[2];
        double ya = metric_z(x, 2, xa < 0.0 ? 0.0 : xa);
        double yb = metric_z(x, 2, xb > 1.0 ? 1.0 : xb);
        for (int i = 0; i < nr; ++i) {
            double ra_ = i * x->h[0] - 0.5 * x->h[0], rb_ = i * x->h[0] + 0.5 * x->h[0];
            double ra = metric_z(x, 0, ra_ < 0.0 ? 0.0 : ra_);
            double rb = metric_z(x, 0, rb_ > 1.0 ? 1.0 : rb_);
            double avg = 0.0;
            for (int q = 0; q < 8; ++q) {
                double yq = 0.5 * (ya + yb) + 0.5 * (yb - ya) * gx[q];
                avg += 0.5 * gw[q] * payoff_avg_r(x, ra, rb, yq);
            }
            for (int k = 0; k < nv; ++k) U[at(x, i, k, j)] = avg;
        }
    }
}

void orc_march(const orc_ctx* x, double* U)
{
    orc_terminal(x, U);
    for (int n = 0; n < x->g.n_steps; ++n) orc_step(x, n, U);
}

/* ------------------------------------------------------------- readout */

/* Four-point Lagrange weights at s in node units from the stencil start. */
static void lagrange4(double s, double* w)
{
    for (int m = 0; m < 4; ++m) {
        double p = 1.0;
        for (int l = 0; l < 4; ++l)
            if (l != m) p *= (s - l) / (double)(m - l);
        w[m] = p;
    }
}

/* Reading R10: tensor-product cubic Lagrange interpolation in (xi_r, xi_v)
 * at r = f(0,0), v = v0 on the y = 0 plane, stencil of the 4 nodes nearest
 * in xi, shifted to stay inside the grid. */
double orc_readout(const orc_ctx* x, const double* U)
{
    double xr = metric_xi(x, 0, orc_curve_f(&x->c, 0.0)) / x->h[0];
    double xv = metric_xi(x, 1, x->m.v0) / x->h[1];
    int ir = (int)floor(xr) - 1, iv = (int)floor(xv) - 1;
    if (ir < 0) ir = 0;
    if (ir > x->n[0] - 4) ir = x->n[0] - 4;
    if (iv < 0) iv = 0;
    if (iv > x->n[1] - 4) iv = x->n[1] - 4;
    double wr[4], wv[4];
    lagrange4(xr - ir, wr);
    lagrange4(xv - iv, wv);
    double s = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a)
            s += wr[a] * wv[b] * U[at(x, ir + a, iv + b, 0)];
    return s;
}

/* Derivatives of the price in r and v at the read-out point (the Greeks
 * listed with the paper's figures: sensitivity to the short rate and to the
 * volatility level): the derivatives of the read-out interpolant of R10,
 * d/dz = (1 / (h J(xi))) d/ds with s = xi / h the node-unit coordinate and
 * J = dz/dxi the metric Jacobian at the read-out point. */
static void lagrange4_d(double s, double* dw)
{
    for (int m = 0; m < 4; ++m) {
        double sum = 0.0;
        for (int l = 0; l < 4; ++l) {
            if (l == m) continue;
            double p = 1.0 / (double)(m - l);
            for (int q = 0; q < 4; ++q)
                if (q != m && q != l) p *= (s - q) / (double)(m - q);
            sum += p;
        }
        dw[m] = sum;
    }
}

void orc_readout_greeks(const orc_ctx* x, const double* U, double* d_dr, double* d_dv)
{
    double xir = metric_xi(x, 0, orc_curve_f(&x->c, 0.0)), xiv = metric_xi(x, 1, x->m.v0);
    double xr = xir / x->h[0], xv = xiv / x->h[1];
    int ir = (int)floor(xr) - 1, iv = (int)floor(xv) - 1;
    if (ir < 0) ir = 0;
    if (ir > x->n[0] - 4) ir = x->n[0] - 4;
    if (iv < 0) iv = 0;
    if (iv > x->n[1] - 4) iv = x->n[1] - 4;
    double wr[4], wv[4], dwr[4], dwv[4];
    lagrange4(xr - ir, wr);
    lagrange4(xv - iv, wv);
    lagrange4_d(xr - ir, dwr);
    lagrange4_d(xv - iv, dwv);
    double sr = 0.0, sv = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
            sr += dwr[a] * wv[b] * U[at(x, ir + a, iv + b, 0)];
            sv += wr[a] * dwv[b] * U[at(x, ir + a, iv + b, 0)];
        }
    double z, Jr, Jv, J2;
    metric_at(xir, x->lo[0], x->hi[0], x->alpha[0], x->centre[0], &z, &Jr, &J2);
    metric_at(xiv, x->lo[1], x->hi[1], x->alpha[1], x->centre[1], &z, &Jv, &J2);
    *d_dr = sr / (x->h[0] * Jr);
    *d_dv = sv / (x->h[1] * Jv);
}

int orc_price(const orc_curve* c, const orc_model* m, const orc_grid* g,
              const orc_inst* in, double* price)
{
    orc_ctx* x;
    int st = orc_ctx_create(c, m, g, in, &x);
    if (st) return st;
    double* U = (double*)malloc(sizeof(double) * orc_n_points(x));
    orc_march(x, U);
    *price = orc_readout(x, U);
    free(U);
    orc_ctx_destroy(x);
    return 0;
}
