// The discrete initial curve of Section 6.1: discount factors at a set of
// maturities, smoothed by a cubic spline so that f(0,t) and df(0,t)/dt are
// continuous. The spline is the natural cubic spline of ln P(0,t) through
// (0, 0) and the knots (zero curvature at both ends), held in Hermite form:
// the node slopes k_i = (ln P)'(tau_i) solve the tridiagonal system
//   2 k_0 + k_1 = 3 d_0                                   (first node)
//   k_{i-1} / h_{i-1} + 2 (1/h_{i-1} + 1/h_i) k_i + k_{i+1} / h_i
//       = 3 (d_{i-1} / h_{i-1} + d_i / h_i)                (inside)
//   k_{m-2} + 2 k_{m-1} = 3 d_{m-2}                       (last node)
// with h_i = tau_{i+1} - tau_i and d_i = (y_{i+1} - y_i) / h_i, the
// conditions for continuous second derivatives and zero curvature at the
// ends. Past the last knot ln P continues linearly (flat forward). Built in
// FP64 by the set-up kernel (and on the host, for input validation only).
#pragma once

#include <math.h>

#include "hjm.h"

namespace hjm {

struct KnotCurve {
    int n;                           // knots (the origin not counted)
    double t[HJM_MAX_KNOTS];         // maturities, as given
    double P[HJM_MAX_KNOTS];         // discount factors, as given
    // spline nodes (origin first), ln P at the nodes, node slopes
    double tau[HJM_MAX_KNOTS + 1], y[HJM_MAX_KNOTS + 1], k[HJM_MAX_KNOTS + 1];
};

// Fills tau, y and k from t and P (idempotent: t and P are not touched).
__host__ __device__ inline void knot_build(KnotCurve& c)
{
    const int m = c.n + 1;
    c.tau[0] = 0.0;
    c.y[0] = 0.0;
    for (int i = 1; i < m; ++i) {
        c.tau[i] = c.t[i - 1];
        c.y[i] = log(c.P[i - 1]);
    }
    // Thomas: forward sweep keeps (c'_i, d'_i) in k[] and a local array.
    double cp[HJM_MAX_KNOTS + 1];
    for (int i = 0; i < m; ++i) {
        double a = 0.0, b, cc = 0.0, rhs;
        if (i == 0) {
            const double h = c.tau[1] - c.tau[0], d = (c.y[1] - c.y[0]) / h;
            b = 2.0 / h;
            cc = 1.0 / h;
            rhs = 3.0 * d / h;
        } else if (i == m - 1) {
            const double h = c.tau[i] - c.tau[i - 1], d = (c.y[i] - c.y[i - 1]) / h;
            a = 1.0 / h;
            b = 2.0 / h;
            rhs = 3.0 * d / h;
        } else {
            const double hl = c.tau[i] - c.tau[i - 1], hr = c.tau[i + 1] - c.tau[i];
            const double dl = (c.y[i] - c.y[i - 1]) / hl, dr = (c.y[i + 1] - c.y[i]) / hr;
            a = 1.0 / hl;
            b = 2.0 * (1.0 / hl + 1.0 / hr);
            cc = 1.0 / hr;
            rhs = 3.0 * (dl / hl + dr / hr);
        }
        const double piv = i == 0 ? b : b - a * cp[i - 1];
        cp[i] = cc / piv;
        c.k[i] = (i == 0 ? rhs : rhs - a * c.k[i - 1]) / piv;
    }
    for (int i = m - 2; i >= 0; --i) c.k[i] -= cp[i] * c.k[i + 1];
}

// ln P(0,t) (s) and its first two derivatives; t >= 0.
__host__ __device__ inline void knot_eval(const KnotCurve& c, double t, double& s, double& ds, double& d2s)
{
    const int last = c.n;  // index of the last node
    if (t >= c.tau[last]) {
        s = c.y[last] + c.k[last] * (t - c.tau[last]);
        ds = c.k[last];
        d2s = 0.0;
        return;
    }
    int i = 0;
    while (i + 1 < last && c.tau[i + 1] <= t) ++i;
    const double h = c.tau[i + 1] - c.tau[i], u = (t - c.tau[i]) / h;
    const double y0 = c.y[i], y1 = c.y[i + 1], m0 = h * c.k[i], m1 = h * c.k[i + 1];
    const double u2 = u * u, u3 = u2 * u;
    // cubic Hermite basis on [0, 1] and its derivatives
    s = (2.0 * u3 - 3.0 * u2 + 1.0) * y0 + (u3 - 2.0 * u2 + u) * m0 + (3.0 * u2 - 2.0 * u3) * y1 + (u3 - u2) * m1;
    ds = ((6.0 * u2 - 6.0 * u) * (y0 - y1) + (3.0 * u2 - 4.0 * u + 1.0) * m0 + (3.0 * u2 - 2.0 * u) * m1) / h;
    d2s = ((12.0 * u - 6.0) * (y0 - y1) + (6.0 * u - 4.0) * m0 + (6.0 * u - 2.0) * m1) / (h * h);
}

}  // namespace hjm
