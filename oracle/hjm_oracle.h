/*
 * Plain CPU FP64 oracle of the discretised HJM-SV pricing PDE.
 *
 * TEST INFRASTRUCTURE ONLY. This header, hjm_oracle.c and the Python
 * wrapper beside them are the slow, obviously-correct reference that the
 * GPU library is checked against. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load them; the product path
 * never does. The oracle shares no code, header, table or constant with the
 * GPU library.
 *
 * What it computes (Valero, Torrealba, Lacasa, Fraysse, "Fast resolution of
 * a single factor HJM model with stochastic volatility"):
 *   - the model and its PDE, Sections 3.1-3.2;
 *   - the sinh stretched grid, Sections 4.3 and 7.1;
 *   - centred differences, the theta scheme in delta form and the Douglas
 *     ADI splitting, Sections 5 and 5.1;
 *   - the cell-averaged (softened) caplet payoff, Section 7.2;
 *   - one-sided differences on the y faces, Section 7.3;
 *   - the exact bond price (Section 3.1, bond formula; Section 4.1, exact
 *     solution) and the Gaussian-limit caplet as closed-form pins.
 * Where the paper is silent or garbled the readings are stated next to the
 * code that takes them.
 */
#ifndef HJM_ORACLE_H
#define HJM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Initial forward curve f(0,t). kind 0: flat f(0,t)=flat_rate.
 * kind 1: Nelson-Siegel in instantaneous-forward form
 *   f(0,t) = beta0 + beta1 e^{-t/tau} + beta2 (t/tau) e^{-t/tau}.
 * kind 2: discrete curve (Section 6.1): discount factors knot_P[i] at
 *   maturities knot_t[i] (0 < knot_t[0] < ... , 1 <= n_knots <= ORC_MAX_KNOTS),
 *   smoothed by a natural cubic spline of ln P(0,t) through (0, 0) and the
 *   knots; ln P continues linearly past the last knot. */
#define ORC_MAX_KNOTS 32
typedef struct {
    int kind;
    double flat_rate, beta0, beta1, beta2, tau;
    int n_knots;
    double knot_t[ORC_MAX_KNOTS];
    double knot_P[ORC_MAX_KNOTS];
} orc_curve;

/* Model parameters of Section 3.1, constant in time. */
typedef struct {
    double kappa, lambda, gamma, theta, epsilon, rho, v0;
} orc_model;

/* Grid: node counts per axis (boundaries included), the physical domain of
 * each axis, the sinh metric parameters (alpha <= 0 selects a uniform grid)
 * and the scheme parameters. r_min may be negative only when gamma == 0.
 * v and y start at 0. */
typedef struct {
    int n_r, n_y, n_v, n_steps;
    double r_min, r_max, y_max, v_max;
    double alpha_r, alpha_y, alpha_v;
    double k_r, k_v;
    int center_r_on_strike;   /* 1: metric centre in r is the strike (caplet)
                                 or f(0,0) (bond); 0: use k_r */
    double theta_adi;         /* theta of the theta scheme; 0.5 = CN */
    int y_boundary_order;     /* 1 or 2: one-sided order on the y faces in F */
    int explicit_midpoint;    /* 0: F at t^n (paper); 1: F at t^{n+1/2} */
    int scheme;               /* ADI scheme: 0 Douglas (Section 5.1), 1 Craig-Sneyd,
                                 2 modified Craig-Sneyd, 3 Hundsdorfer-Verwer */
} orc_grid;

/* Instrument: kind 0 zero-coupon bond maturing at T; kind 1 caplet with
 * expiry T, payment date TM and strike K (K is added to the ATM forward
 * rate when strike_atm_relative != 0), paying at T the put on the bond
 * max(1 - Delta_M p(T,T_M), 0), Delta_M = 1 + (TM - T) K (Section 3.2);
 * kind 2 the floorlet on the same period, max(Delta_M p(T,T_M) - 1, 0). */
typedef struct {
    int kind;
    double T, TM, K;
    int strike_atm_relative;
} orc_inst;

typedef struct orc_ctx orc_ctx;

/* Status: 0 ok, 1 invalid argument. */
int orc_ctx_create(const orc_curve* c, const orc_model* m, const orc_grid* g,
                   const orc_inst* in, orc_ctx** out);
void orc_ctx_destroy(orc_ctx* x);

/* Sizes and derived scalars. */
long orc_n_points(const orc_ctx* x);
double orc_strike(const orc_ctx* x);
double orc_dt(const orc_ctx* x);
/* Axis tables: axis 0 = r, 1 = v, 2 = y; arrays of length n. */
void orc_axis(const orc_ctx* x, int axis, double* z, double* J, double* J2);

/* Curve and closed forms. */
double orc_curve_f(const orc_curve* c, double t);
double orc_curve_dfdt(const orc_curve* c, double t);
double orc_curve_P(const orc_curve* c, double t);
double orc_G(double kappa, double s);
double orc_bond(const orc_curve* c, const orc_model* m, double t, double S,
                double r, double y);
double orc_gauss_caplet(const orc_curve* c, const orc_model* m, double T,
                        double TM, double K);
double orc_atm_strike(const orc_curve* c, double T, double TM);

/* Fields are n_r*n_v*n_y doubles, index i + n_r*(k + n_v*j) with i on r,
 * k on v, j on y. */
void orc_terminal(const orc_ctx* x, double* U);
/* Delta U^0 of step n: dt*F(U;t^n) off the Dirichlet faces, g(t^{n+1})-U on them. */
void orc_explicit(const orc_ctx* x, int n, const double* U, double* dU0);
/* Operator F(U;t) alone (no dt factor, zero on Dirichlet faces). */
void orc_apply_F(const orc_ctx* x, double t, const double* U, double* F);
/* One directional operator A_d(t) applied to U (d: 0 r, 1 v, 2 y, 3 mixed),
 * as used in F (second-order one-sided faces). Zero on Dirichlet faces. */
void orc_apply_dir(const orc_ctx* x, int d, double t, const double* U, double* AU);
/* Solve (I - theta dt A_d(t)) out = rhs along every line of direction d.
 * Returns the number of rows that were not diagonally dominant. */
long orc_solve_dir(const orc_ctx* x, int d, double t, const double* rhs, double* out);
/* The tridiagonal coefficients (sub, main, super) of (I - theta dt A_d(t))
 * along one line; line = index of the line (the two other coordinates,
 * lower axis fastest). len = n_d. */
void orc_line_matrix(const orc_ctx* x, int d, double t, long line,
                     double* sub, double* diag, double* sup);
/* One ADI step n -> n+1 in place (the grid's scheme). */
void orc_step(const orc_ctx* x, int n, double* U);
/* Terminal field followed by all n_steps steps. */
void orc_march(const orc_ctx* x, double* U);
/* Interpolated value at r = f(0,0), v = v0 on the y = 0 plane. */
double orc_readout(const orc_ctx* x, const double* U);
/* dC/dr and dC/dv at the read-out point: derivatives of the read-out
 * interpolant (divided by the metric Jacobian there). */
void orc_readout_greeks(const orc_ctx* x, const double* U, double* d_dr, double* d_dv);
/* Calendar time of step index n (n may be fractional). */
double orc_time(const orc_ctx* x, double n);
/* Dirichlet data g(t, r, y). */
double orc_dirichlet(const orc_ctx* x, double t, double r, double y);
/* Whole price: create, march, read out. Status as orc_ctx_create. */
int orc_price(const orc_curve* c, const orc_model* m, const orc_grid* g,
              const orc_inst* in, double* price);

#ifdef __cplusplus
}
#endif
#endif
