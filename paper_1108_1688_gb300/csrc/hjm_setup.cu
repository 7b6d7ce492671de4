// FP64 set-up and read-out kernels of the ADI march.
//
// Everything here runs once per price (not per step): the curve and bond
// functions of Sections 2 and 3.1 (with the spline of a discrete curve,
// Section 6.1, built by k_setup), the sinh metric of Sections 4.3 / 7.1, the
// coefficient tables of the operator of Eq. (1) in the metric form of Section
// 4.3, the per-step scalars and Dirichlet data, the Thomas factors of the
// line-invariant v and y systems, the softened terminal field of Section 7.2
// and the cubic read-out at the model's initial state.
#include <math.h>

#include "hjm_kernels.cuh"

namespace hjm {

// ----------------------------------------------------------- curve, bonds

// f(0,t) of the initial curve (flat, Nelson-Siegel forward form, or the
// spline of a discrete curve, Section 6.1).
__device__ double fwd(const InstParams& p, double t)
{
    if (p.ckind == HJM_CURVE_FLAT) return p.flat;
    if (p.ckind == HJM_CURVE_KNOTS) {
        double s, ds, d2s;
        knot_eval(p.kc, t, s, ds, d2s);
        return -ds;
    }
    const double x = t / p.tau, e = exp(-x);
    return p.b0 + e * (p.b1 + p.b2 * x);
}

__device__ double fwd_slope(const InstParams& p, double t)
{
    if (p.ckind == HJM_CURVE_FLAT) return 0.0;
    if (p.ckind == HJM_CURVE_KNOTS) {
        double s, ds, d2s;
        knot_eval(p.kc, t, s, ds, d2s);
        return -d2s;
    }
    const double x = t / p.tau, e = exp(-x);
    return e * (p.b2 * (1.0 - x) - p.b1) / p.tau;
}

// P(0,t) = exp(-int_0^t f(0,s) ds).
__device__ double discount(const InstParams& p, double t)
{
    if (p.ckind == HJM_CURVE_FLAT) return exp(-p.flat * t);
    if (p.ckind == HJM_CURVE_KNOTS) {
        double s, ds, d2s;
        knot_eval(p.kc, t, s, ds, d2s);
        return exp(s);
    }
    const double x = t / p.tau, e = exp(-x), one_m_e = -expm1(-x);
    return exp(-(p.b0 * t + (p.b1 + p.b2) * p.tau * one_m_e - p.b2 * t * e));
}

// G(s) = (1 - e^{-kappa s}) / kappa, s when kappa = 0 (Section 3.1).
__device__ double Gfun(double kappa, double s)
{
    return kappa == 0.0 ? s : -expm1(-kappa * s) / kappa;
}

// --------------------------------------------------------------- metric

// z(xi) = K + alpha sinh(c2 xi + c1 (1 - xi)) with c1, c2 fixing the end
// points; J = dz/dxi, J2 = d2z/dxi2. alpha <= 0: uniform. End points exact.
__device__ void metric(double xi, double z0, double z1, double alpha, double K, double& z,
                       double& J, double& J2)
{
    if (alpha <= 0.0) {
        z = z0 + (z1 - z0) * xi;
        J = z1 - z0;
        J2 = 0.0;
    } else {
        const double c1 = asinh((z0 - K) / alpha), c2 = asinh((z1 - K) / alpha);
        const double a = c1 + (c2 - c1) * xi, span = c2 - c1;
        const double sh = sinh(a);
        z = K + alpha * sh;
        J = alpha * span * cosh(a);
        J2 = alpha * span * span * sh;
    }
    if (xi == 0.0) z = z0;
    if (xi == 1.0) z = z1;
}

__device__ double metric_inverse(double z, double z0, double z1, double alpha, double K)
{
    if (alpha <= 0.0) return (z - z0) / (z1 - z0);
    const double c1 = asinh((z0 - K) / alpha), c2 = asinh((z1 - K) / alpha);
    return (asinh((z - K) / alpha) - c1) / (c2 - c1);
}

__device__ double metric_z(double xi, double z0, double z1, double alpha, double K)
{
    double z, J, J2;
    metric(xi, z0, z1, alpha, K, z, J, J2);
    return z;
}

// Read-out point r = f(0,0), v = v0 in node units and the first node of the
// 4-point stencil in each direction, kept inside the grid.
__device__ void readout_stencil(const InstParams& p, const InstDerived& D, int nr, int nv, int& i0,
                                int& k0, double* sr = nullptr, double* sv = nullptr)
{
    const double r = metric_inverse(fwd(p, 0.0), p.rmin, p.rmax, p.ar, D.centre_r) * (nr - 1);
    const double v = metric_inverse(p.v0, 0.0, p.vmax, p.av, p.kv) * (nv - 1);
    i0 = min(max((int)floor(r) - 1, 0), nr - 4);
    k0 = min(max((int)floor(v) - 1, 0), nv - 4);
    if (sr) *sr = r;
    if (sv) *sv = v;
}

// ------------------------------------------------------------------ setup

template <typename T>
__global__ void __launch_bounds__(256) k_setup(GroupTables g)
{
    const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    const int nr = g.nr, nv = g.nv, ny = g.ny, ns = g.nsteps;
    // The discrete curve's spline, rebuilt from the knots at every set-up;
    // the later kernels read it from the parameters.
    if (tid == 0 && g.params[b].ckind == HJM_CURVE_KNOTS) knot_build(g.params[b].kc);
    __syncthreads();
    const InstParams& p = g.params[b];
    __shared__ InstDerived D;
    if (tid == 0) {
        double K = 0.0, DM = 1.0;
        if (p.kind != HJM_ZCB) {
            K = p.K;
            if (p.atm_rel) K += (discount(p, p.T) / discount(p, p.TM) - 1.0) / (p.TM - p.T);
            DM = 1.0 + (p.TM - p.T) * K;
        }
        D.K = K;
        D.DM = DM;
        D.dt = p.T / ns;
        D.centre_r = p.center_on_strike ? (p.kind != HJM_ZCB ? K : fwd(p, 0.0)) : p.kr;
        g.derived[b] = D;
    }
    __syncthreads();

    T* rt = (T*)g.rt + (size_t)b * RT_N * nr;
    T* vt = (T*)g.vt + (size_t)b * VT_N * nv;
    T* yt = (T*)g.yt + (size_t)b * YT_N * ny;
    double* axr = g.axr + (size_t)b * 3 * nr;
    double* axv = g.axv + (size_t)b * 3 * nv;
    double* axy = g.axy + (size_t)b * 3 * ny;
    const double lam2 = p.lambda * p.lambda, eps2 = p.eps * p.eps;
    const double w = p.theta_adi * D.dt;

    // r axis and r-operator factors: A_r = g1 d_rr + g4 d_r - r with
    // g1 = zeta_rr / J^2, g4 = mu_r / J - zeta_rr J2 / J^3 (Section 4.3),
    // zeta_rr = lambda^2 r^{2 gamma} v / 2, mu_r = a(t) - kappa r + y. The
    // grid spacings of the centred differences are folded in: the kernels
    // multiply the tables by v, a(t) + y and the undivided differences.
    const double ihr = nr - 1, ihv = nv - 1, ihy = ny - 1;
    for (int i = tid; i < nr; i += nth) {
        double z, J, J2;
        metric((double)i / (nr - 1), p.rmin, p.rmax, p.ar, D.centre_r, z, J, J2);
        axr[i] = z;
        axr[nr + i] = J;
        axr[2 * nr + i] = J2;
        const double rg = p.gamma == 0.0 ? 1.0 : pow(z, p.gamma);
        const double r2g = rg * rg;
        rt[RT_R * nr + i] = (T)z;
        rt[RT_IJ * nr + i] = (T)(0.5 * ihr / J);
        rt[RT_C1 * nr + i] = (T)(0.5 * lam2 * r2g / (J * J) * ihr * ihr);
        rt[RT_C4V * nr + i] = (T)(0.5 * lam2 * r2g * J2 / (J * J * J) * 0.5 * ihr);
        rt[RT_C4B * nr + i] = (T)(-p.kappa * z / J * 0.5 * ihr);
        rt[RT_C3 * nr + i] = (T)(p.lambda * rg * p.eps * p.rho / J * 0.25 * ihr * ihv);
        rt[RT_CY * nr + i] = (T)(lam2 * r2g);
        // folded tables (R2_P ..): zeros on the Dirichlet nodes, B = 1
        T* r2 = (T*)g.r2 + (size_t)b * R2_N * nr;
        const bool dir = i == nr - 1 || (i == 0 && p.gamma == 0.0);
        const double dt = D.dt, ith = p.theta_adi > 0.0 ? 1.0 / p.theta_adi : 0.0;
        const double c1 = 0.5 * lam2 * r2g / (J * J) * ihr * ihr;
        const double c4v = 0.5 * lam2 * r2g * J2 / (J * J * J) * 0.5 * ihr;
        const double ij = 0.5 * ihr / J, c4b = -p.kappa * z / J * 0.5 * ihr;
        const double f[R2_N] = {dt * ij, dt * c4b, ith + dt * z, dt * c1, dt * c4v, -dt * z * ith};
        for (int q = 0; q < R2_N; ++q) r2[q * nr + i] = (T)(dir ? (q == R2_B ? 1.0 : 0.0) : f[q]);
    }
    // v axis: A_v = g2 d_vv + g5 d_v, g2 = zeta_vv / J^2,
    // g5 = mu_v / J - zeta_vv J2 / J^3; on the v faces mu_v / J alone.
    for (int k = tid; k < nv; k += nth) {
        double z, J, J2;
        metric((double)k / (nv - 1), 0.0, p.vmax, p.av, p.kv, z, J, J2);
        axv[k] = z;
        axv[nv + k] = J;
        axv[2 * nv + k] = J2;
        const double zvv = 0.5 * eps2 * z, muv = p.theta * (1.0 - z);
        vt[VT_V * nv + k] = (T)z;
        vt[VT_IJ * nv + k] = (T)(1.0 / J);
        vt[VT_G2 * nv + k] = (T)(zvv / (J * J) * ihv * ihv);
        vt[VT_G5 * nv + k] = (T)((muv / J - zvv * J2 / (J * J * J)) * 0.5 * ihv);
        vt[VT_FV * nv + k] = (T)(muv / J * 0.5 * ihv);
    }
    // y axis: A_y = g6 d_y, g6 = (lambda^2 r^{2 gamma} v - 2 kappa y) / J.
    for (int j = tid; j < ny; j += nth) {
        double z, J, J2;
        metric((double)j / (ny - 1), 0.0, p.ymax, p.ay, 0.0, z, J, J2);
        axy[j] = z;
        axy[ny + j] = J;
        axy[2 * ny + j] = J2;
        yt[YT_Y * ny + j] = (T)z;
        yt[YT_IJ * ny + j] = (T)(0.5 * ihy / J);
        yt[YT_KY * ny + j] = (T)(-2.0 * p.kappa * z);
    }
    if (tid == 0) {
        T* sc = (T*)g.sc + (size_t)b * SC_N;
        sc[SC_DT] = (T)D.dt;
        sc[SC_W] = (T)w;
        sc[SC_IHR] = (T)(nr - 1);
        sc[SC_IHV] = (T)(nv - 1);
        sc[SC_IHY] = (T)(ny - 1);
        const double c1 = p.scheme == HJM_SCHEME_MCS ? 0.5 - p.theta_adi : (p.scheme == HJM_SCHEME_HV ? 0.5 : 0.0);
        const double he = p.scheme == HJM_SCHEME_HV ? 1.0 : 0.0;
        sc[SC_C1] = (T)c1;
        sc[SC_CX] = (T)(0.5 - c1);
        sc[SC_HE] = (T)he;
        sc[SC_KD] = (T)((1.0 - he) / (1.0 - c1));
        sc[SC_ITH] = (T)(p.theta_adi > 0.0 ? 1.0 / p.theta_adi : 0.0);
        sc[SC_XP] = (T)(p.lambda * p.eps * p.rho * 0.5 * (nv - 1));
        sc[SC_YL] = (T)(D.dt * p.lambda * p.lambda);
        int* fl = g.fl + (size_t)b * FL_N;
        fl[FL_RLO_DIR] = p.gamma == 0.0;
        fl[FL_YORDER] = p.yorder;
        fl[FL_YLU] = p.gamma == 0.0;
        int i0, k0;
        readout_stencil(p, D, nr, nv, i0, k0);
        fl[FL_RI0] = i0;
        fl[FL_RK0] = k0;
        fl[FL_PAD] = 0;
    }
    for (int n = tid; n < ns; n += nth) g.acc[(size_t)b * ns + n] = 0.0f;
    // a(t) = df(0,t)/dt + kappa f(0,t): F at t^n (or t^{n+1/2}, always for
    // the Craig-Sneyd family), implicit operators at t^{n+1/2} (Section 5,
    // delta form).
    T* st = (T*)g.st + (size_t)b * ns * 2;
    const bool mid = p.midpoint || p.scheme != HJM_SCHEME_DOUGLAS;
    for (int n = tid; n < ns; n += nth) {
        const double tF = p.T - (mid ? n + 0.5 : (double)n) * D.dt;
        const double tI = p.T - (n + 0.5) * D.dt;
        st[2 * n] = (T)(fwd_slope(p, tF) + p.kappa * fwd(p, tF));
        st[2 * n + 1] = (T)(fwd_slope(p, tI) + p.kappa * fwd(p, tI));
    }
    __syncthreads();  // y nodes above are read below by other threads

    // Thomas factors (sub, c', 1/m) of I - theta dt A_v: the same for every
    // v line (A_v depends on v only).
    if (tid == 0) {
        T* vf = (T*)g.vf + (size_t)b * 3 * nv;
        const double ih = nv - 1, ih2 = ih * ih;
        double cprev = 0.0;
        for (int k = 0; k < nv; ++k) {
            const double v = axv[k], J = axv[nv + k], J2 = axv[2 * nv + k];
            const double zvv = 0.5 * eps2 * v, muv = p.theta * (1.0 - v);
            double lo = 0.0, di = 0.0, up = 0.0;
            if (k > 0 && k < nv - 1) {
                const double g2 = zvv / (J * J), g5 = muv / J - zvv * J2 / (J * J * J);
                lo = g2 * ih2 - 0.5 * g5 * ih;
                di = -2.0 * g2 * ih2;
                up = g2 * ih2 + 0.5 * g5 * ih;
            } else if (k == 0) {
                di = -muv / J * ih;
                up = muv / J * ih;
            } else {
                lo = -muv / J * ih;
                di = muv / J * ih;
            }
            const double sub = -w * lo, mainv = 1.0 - w * di, sup = -w * up;
            const double m = mainv - sub * cprev;
            cprev = sup / m;
            vf[k] = (T)sub;
            vf[nv + k] = (T)cprev;
            vf[2 * nv + k] = (T)(1.0 / m);
        }
    }
    // Thomas factors of I - theta dt A_y per v node when gamma == 0 (then
    // g6 depends on v and y only, not on r).
    if (p.gamma == 0.0 && g.yf != nullptr) {
        const double ih = ny - 1;
        for (int k = tid; k < nv; k += nth) {
            T* yf = (T*)g.yf + ((size_t)b * nv + k) * 3 * ny;
            const double v = axv[k];
            double cprev = 0.0;
            for (int j = 0; j < ny; ++j) {
                const double g6 = (lam2 * v - 2.0 * p.kappa * axy[j]) / axy[ny + j];
                double lo = 0.0, di = 0.0, up = 0.0;
                if (j > 0 && j < ny - 1) {
                    lo = -0.5 * g6 * ih;
                    up = 0.5 * g6 * ih;
                } else if (j == 0) {
                    di = -g6 * ih;
                    up = g6 * ih;
                } else {
                    lo = -g6 * ih;
                    di = g6 * ih;
                }
                const double sub = -w * lo, mainv = 1.0 - w * di, sup = -w * up;
                const double m = mainv - sub * cprev;
                cprev = sup / m;
                yf[j] = (T)sub;
                yf[ny + j] = (T)cprev;
                yf[2 * ny + j] = (T)(1.0 / m);
            }
        }
    }
}

// Rows (sub, main, super) of I - theta dt A_v at v node k (Section 5.1, the
// one-sided first-order face rows of Section 7.3) and of I - theta dt A_y at
// y node j for the v node v (gamma = 0).
__device__ void v_row(const InstParams& p, const double* axv, int nv, double w, int k, double& sub,
                      double& mainv, double& sup)
{
    const double ih = nv - 1, ih2 = ih * ih;
    const double v = axv[k], J = axv[nv + k], J2 = axv[2 * nv + k];
    const double zvv = 0.5 * p.eps * p.eps * v, muv = p.theta * (1.0 - v);
    double lo = 0.0, di = 0.0, up = 0.0;
    if (k > 0 && k < nv - 1) {
        const double g2 = zvv / (J * J), g5 = muv / J - zvv * J2 / (J * J * J);
        lo = g2 * ih2 - 0.5 * g5 * ih;
        di = -2.0 * g2 * ih2;
        up = g2 * ih2 + 0.5 * g5 * ih;
    } else if (k == 0) {
        di = -muv / J * ih;
        up = muv / J * ih;
    } else {
        lo = -muv / J * ih;
        di = muv / J * ih;
    }
    sub = -w * lo;
    mainv = 1.0 - w * di;
    sup = -w * up;
}

__device__ void y_row(const InstParams& p, const double* axy, int ny, double w, double v, int j, double& sub,
                      double& mainv, double& sup)
{
    const double ih = ny - 1;
    const double g6 = (p.lambda * p.lambda * v - 2.0 * p.kappa * axy[j]) / axy[ny + j];
    double lo = 0.0, di = 0.0, up = 0.0;
    if (j > 0 && j < ny - 1) {
        lo = -0.5 * g6 * ih;
        up = 0.5 * g6 * ih;
    } else if (j == 0) {
        di = -g6 * ih;
        up = g6 * ih;
    } else {
        lo = -g6 * ih;
        di = g6 * ih;
    }
    sub = -w * lo;
    mainv = 1.0 - w * di;
    sup = -w * up;
}

// Factors of the v systems (axis 0: one per instrument) or y systems (axis 1:
// one per instrument and v node, gamma = 0 only) split into P chunks solved
// independently, one warp each, and joined through a small reduced system
// (layout in part_sys_size). For chunk p with rows [s, s + L):
//   the LU of the chunk's rows without their outside couplings;
//   V = A_p^{-1} (sub_s e_0) and W = A_p^{-1} (sup_{s+L-1} e_{L-1}), so
//   that x = A_p^{-1} d - x_{s-1} V - x_{s+L} W on the chunk;
//   evaluated at the chunks' end rows this gives the reduced system in
//   z = (last of chunk 0, first of chunk 1, last of chunk 1, ..., first of
//   chunk P-1), whose inverse yields, per chunk, the weights of the reduced
//   right-hand sides (the chunks' end values of A_p^{-1} d) in x_{s-1} and
//   x_{s+L}.
// One warp per system: lanes p < P factor the chunks, then the lanes run
// Gauss-Jordan with partial pivoting on [M | I] in shared memory. FP64
// throughout, stored in the march type.
template <typename T>
__global__ void __launch_bounds__(32) k_split(GroupTables g, int axis, int P)
{
    const int lane = threadIdx.x;
    const int nv = g.nv, ny = g.ny;
    const int b = axis == 0 ? blockIdx.x : blockIdx.x / nv;
    const int k = axis == 0 ? 0 : blockIdx.x % nv;
    const InstParams& p = g.params[b];
    if (axis == 1 && p.gamma != 0.0) return;
    const double w = p.theta_adi * g.derived[b].dt;
    const double* axv = g.axv + (size_t)b * 3 * nv;
    const double* axy = g.axy + (size_t)b * 3 * ny;
    const int n = axis == 0 ? nv : ny;
    T* out = axis == 0 ? (T*)g.vp + (size_t)b * part_sys_size(nv, kMaxSplit)
                       : (T*)g.yp + ((size_t)b * nv + k) * part_sys_size(ny, kMaxSplit);
    const int K = 2 * (P - 1);
    __shared__ double im[kMaxSplit][kMaxChunk], cp[kMaxSplit][kMaxChunk], lo[kMaxSplit][kMaxChunk],
        vv[kMaxSplit][kMaxChunk];
    __shared__ double Vend[2 * kMaxSplit], Wend[2 * kMaxSplit];
    __shared__ double A[2 * (kMaxSplit - 1)][4 * (kMaxSplit - 1)];
    __shared__ int piv_row;
    if (lane < P) {
        const int c = lane;
        int s, L;
        part_chunk(n, P, c, s, L);
        for (int m = 0; m < L; ++m) {
            double l, d, u;
            if (axis == 0)
                v_row(p, axv, nv, w, s + m, l, d, u);
            else
                y_row(p, axy, ny, w, axv[k], s + m, l, d, u);
            lo[c][m] = l;
            const double pv = m > 0 ? d - l * cp[c][m - 1] : d;
            im[c][m] = 1.0 / pv;
            cp[c][m] = u * im[c][m];
            out[2 * (s + m)] = (T)(m > 0 ? l : 0.0);
            out[2 * (s + m) + 1] = (T)im[c][m];
            out[4 * n + 2 * P * K + s + m] = (T)cp[c][m];
        }
        // V: forward with right-hand side sub_s e_0, then back substitution.
        vv[c][0] = lo[c][0] * im[c][0];
        for (int m = 1; m < L; ++m) vv[c][m] = -lo[c][m] * vv[c][m - 1] * im[c][m];
        for (int m = L - 2; m >= 0; --m) vv[c][m] -= cp[c][m] * vv[c][m + 1];
        // W: right-hand side sup_{s+L-1} e_{L-1}, whose forward value is c'.
        double wn = cp[c][L - 1];
        Wend[2 * c + 1] = wn;
        out[2 * n + 2 * (s + L - 1) + 1] = (T)wn;
        for (int m = L - 2; m >= 0; --m) {
            wn = -cp[c][m] * wn;
            out[2 * n + 2 * (s + m) + 1] = (T)wn;
        }
        Wend[2 * c] = wn;
        for (int m = 0; m < L; ++m) out[2 * n + 2 * (s + m)] = (T)vv[c][m];
        Vend[2 * c] = vv[c][0];
        Vend[2 * c + 1] = vv[c][L - 1];
    }
    __syncwarp();
    if (P == 1) return;
    // Reduced system M z = r: row 2q is chunk q's last row, row 2q + 1 is
    // chunk q+1's first row (q = 0..P-2). Lane j owns column j of [M | I].
    for (int i = 0; i < K; ++i)
        if (lane < 2 * K) A[i][lane] = (lane == i || lane == K + i) ? 1.0 : 0.0;
    __syncwarp();
    if (lane == 0)
        for (int q = 0; q + 1 < P; ++q) {
            if (q >= 1) A[2 * q][2 * q - 2] = Vend[2 * q + 1];
            A[2 * q][2 * q + 1] = Wend[2 * q + 1];
            A[2 * q + 1][2 * q] = Vend[2 * (q + 1)];
            if (q + 2 < P) A[2 * q + 1][2 * q + 3] = Wend[2 * (q + 1)];
        }
    __syncwarp();
    for (int c = 0; c < K; ++c) {
        if (lane == 0) {
            int r = c;
            for (int i = c + 1; i < K; ++i)
                if (fabs(A[i][c]) > fabs(A[r][c])) r = i;
            piv_row = r;
        }
        __syncwarp();
        const int r = piv_row;
        if (r != c && lane < 2 * K) {
            const double t = A[c][lane];
            A[c][lane] = A[r][lane];
            A[r][lane] = t;
        }
        __syncwarp();
        const double ip = 1.0 / A[c][c];
        __syncwarp();
        if (lane < 2 * K) A[c][lane] *= ip;
        __syncwarp();
        for (int i = 0; i < K; ++i) {
            const double f = A[i][c];
            __syncwarp();
            if (i != c && lane < 2 * K) A[i][lane] -= f * A[c][lane];
            __syncwarp();
        }
    }
    // Chunk c needs x_{s-1} = z_{2(c-1)} (c >= 1) and x_{s+L} = z_{2c+1}
    // (c <= P-2).
    for (int idx = lane; idx < P * K; idx += 32) {
        const int c = idx / K, q = idx % K;
        out[4 * n + 2 * idx] = (T)(c >= 1 ? A[2 * (c - 1)][K + q] : 0.0);
        out[4 * n + 2 * idx + 1] = (T)(c + 1 < P ? A[2 * c + 1][K + q] : 0.0);
    }
}

// Dirichlet data at t^{n+1} on r = r_min (face 0) and r = r_max (face 1):
// the exact bond p(t,S) = P(0,S)/P(0,t) exp(-G(S-t) x - G(S-t)^2 y / 2),
// x = r - f(0,t) (Section 3.1), for a bond, and the caplet's intrinsic
// forward value max(p(t,T) - Delta_M p(t,T_M), 0). One block per (step,
// instrument): the curve factors depend on t only and are formed once.
template <typename T>
__global__ void __launch_bounds__(128) k_faces(GroupTables g)
{
    const int n = blockIdx.x, b = blockIdx.y, ny = g.ny, ns = g.nsteps;
    const InstParams& p = g.params[b];
    __shared__ double sc[6];
    if (threadIdx.x == 0) {
        const InstDerived D = g.derived[b];
        const double t = p.T - (n + 1) * D.dt;
        const double Pt = discount(p, t);
        sc[0] = discount(p, p.T) / Pt;
        sc[1] = discount(p, p.TM) / Pt;
        sc[2] = fwd(p, t);
        sc[3] = Gfun(p.kappa, p.T - t);
        sc[4] = Gfun(p.kappa, p.TM - t);
        sc[5] = D.DM;
    }
    __syncthreads();
    const double* axy = g.axy + (size_t)b * 3 * ny;
    T* dir = (T*)g.dir + ((size_t)b * ns + n) * 2 * ny;
    for (int idx = threadIdx.x; idx < 2 * ny; idx += blockDim.x) {
        const int j = idx % ny, face = idx / ny;
        const double r = face ? p.rmax : p.rmin, y = axy[j], x = r - sc[2];
        const double pT = sc[0] * exp(-sc[3] * x - 0.5 * sc[3] * sc[3] * y);
        double v = pT;
        if (p.kind != HJM_ZCB) {
            const double pM = sc[1] * exp(-sc[4] * x - 0.5 * sc[4] * sc[4] * y);
            v = fmax(p.kind == HJM_CAPLET ? pT - sc[5] * pM : sc[5] * pM - pT, 0.0);
        }
        dir[idx] = (T)v;
    }
}

// ------------------------------------------------------- terminal field

// Gauss-Legendre rule of order 8 on [-1, 1] by Newton on the Legendre
// three-term recurrence (computed once per block).
__device__ void gauss_legendre8(double* x, double* wt, int q)
{
    const int n = 8;
    double z = cos(3.14159265358979323846 * (q + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 60; ++it) {
        double p0 = 1.0, p1 = z;
        for (int l = 2; l <= n; ++l) {
            const double p2 = ((2 * l - 1) * z * p1 - (l - 1) * p0) / l;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double step = p1 / dp;
        z -= step;
        if (fabs(step) < 1e-16) break;
    }
    x[q] = z;
    wt[q] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// Mean over r in [ra, rb] of the floorlet payoff max(Delta_M p(T,T_M; r, y) - 1,
// 0), Delta_M p = e^{lnDA - G r}: positive below r* = lnDA / G, its integral
// there closed form.
__device__ double floorlet_r_mean(double G, double lnDA, double ra, double rb)
{
    if (!(rb > ra)) {
        const double v = exp(lnDA - G * ra) - 1.0;
        return v > 0.0 ? v : 0.0;
    }
    const double hi = fmin(rb, lnDA / G);
    if (hi <= ra) return 0.0;
    // int_ra^hi e^{lnDA - G r} - 1 dr
    const double body = exp(lnDA - G * ra) * (-expm1(-G * (hi - ra))) / G;
    return (body - (hi - ra)) / (rb - ra);
}

// Mean over r in [ra, rb] of max(1 - Delta_M p(T,T_M; r, y), 0) where
// Delta_M p = e^{lnDA - G r}: the payoff is positive above r* = lnDA / G and
// its integral there is closed form.
__device__ double caplet_r_mean(double G, double lnDA, double ra, double rb)
{
    if (!(rb > ra)) {
        const double v = 1.0 - exp(lnDA - G * ra);
        return v > 0.0 ? v : 0.0;
    }
    const double lo = fmax(ra, lnDA / G);
    if (lo >= rb) return 0.0;
    // int_lo^rb 1 - e^{lnDA - G r} dr
    const double tail = exp(lnDA - G * lo) * (-expm1(-G * (rb - lo))) / G;
    return ((rb - lo) - tail) / (rb - ra);
}

// U^0 at t = T: 1 for a bond; for a caplet or floorlet the payoff averaged over each
// node's control volume in r and y (Section 7.2; closed form in r, 8-point
// Gauss-Legendre in y), the same for every v. One block per (y node,
// instrument); the y cell and the curve factors are formed once per block.
template <typename T>
__global__ void __launch_bounds__(128) k_terminal(GroupTables g, T* U)
{
    const int j = blockIdx.x, b = blockIdx.y;
    const int nr = g.nr, nv = g.nv, ny = g.ny;
    const InstParams& p = g.params[b];
    __shared__ double gx[8], gw[8], sc[4];
    if (threadIdx.x < 8) gauss_legendre8(gx, gw, threadIdx.x);
    if (p.kind != HJM_ZCB && threadIdx.x == 32) {
        const InstDerived D = g.derived[b];
        const double hy = 1.0 / (ny - 1);
        const double G = Gfun(p.kappa, p.TM - p.T);
        sc[0] = G;
        // ln(Delta_M p(T,T_M; r=0, y=0))
        sc[1] = log(D.DM) + log(discount(p, p.TM) / discount(p, p.T)) + G * fwd(p, p.T);
        sc[2] = metric_z(fmax(0.0, (j - 0.5) * hy), 0.0, p.ymax, p.ay, 0.0);
        sc[3] = metric_z(fmin(1.0, (j + 0.5) * hy), 0.0, p.ymax, p.ay, 0.0);
    }
    __syncthreads();
    const long long N = (long long)nr * nv * ny;
    const double hr = 1.0 / (nr - 1);
    const double centre = g.derived[b].centre_r;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        double val = 1.0;
        if (p.kind != HJM_ZCB) {
            const double ra = metric_z(fmax(0.0, (i - 0.5) * hr), p.rmin, p.rmax, p.ar, centre);
            const double rb = metric_z(fmin(1.0, (i + 0.5) * hr), p.rmin, p.rmax, p.ar, centre);
            const double G = sc[0], ya = sc[2], yb = sc[3];
            double s = 0.0;
            for (int q = 0; q < 8; ++q) {
                const double yq = 0.5 * (ya + yb) + 0.5 * (yb - ya) * gx[q];
                const double lnDA = sc[1] - 0.5 * G * G * yq;
                s += 0.5 * gw[q] * (p.kind == HJM_CAPLET ? caplet_r_mean(G, lnDA, ra, rb)
                                                         : floorlet_r_mean(G, lnDA, ra, rb));
            }
            val = s;
        }
        T* row = U + (long long)b * N + (long long)j * nv * nr + i;
        for (int k = 0; k < nv; ++k) row[(long long)k * nr] = (T)val;
    }
}

// ---------------------------------------------------------------- readout

// Price at r = f(0,0), v = v0 on the y = 0 plane: tensor-product cubic
// Lagrange interpolation in the computational coordinates on the 4 x 4
// nodes nearest the point, kept inside the grid.
template <typename T>
__global__ void k_readout(GroupTables g, const T* U, double* prices, double* indicators, double* greeks,
                          double u_op, double u_state, double u_incr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.B) return;
    const InstParams& p = g.params[b];
    const InstDerived D = g.derived[b];
    const int nr = g.nr, nv = g.nv;
    double sr, sv;
    int i0, k0;
    readout_stencil(p, D, nr, nv, i0, k0, &sr, &sv);
    double wr[4], wv[4];
    for (int a = 0; a < 4; ++a) {
        double pr = 1.0, pv = 1.0;
        for (int c = 0; c < 4; ++c) {
            if (c == a) continue;
            pr *= (sr - i0 - c) / (double)(a - c);
            pv *= (sv - k0 - c) / (double)(a - c);
        }
        wr[a] = pr;
        wv[a] = pv;
    }
    const T* Ub = U + (long long)b * nr * nv * g.ny;
    double s = 0.0;
    for (int c = 0; c < 4; ++c) {
        double row = 0.0;
        for (int a = 0; a < 4; ++a) row += wr[a] * (double)Ub[(long long)(k0 + c) * nr + i0 + a];
        s += wv[c] * row;
    }
    prices[b] = s;
    if (greeks) {
        // Derivatives of the interpolant in r and v, divided by the metric
        // Jacobian at the read-out point (d/dz = (n-1) / J d/ds).
        double dwr[4], dwv[4];
        for (int a = 0; a < 4; ++a) {
            double qr = 0.0, qv = 0.0;
            for (int l = 0; l < 4; ++l) {
                if (l == a) continue;
                double pr = 1.0 / (double)(a - l), pv = pr;
                for (int c = 0; c < 4; ++c) {
                    if (c == a || c == l) continue;
                    pr *= (sr - i0 - c) / (double)(a - c);
                    pv *= (sv - k0 - c) / (double)(a - c);
                }
                qr += pr;
                qv += pv;
            }
            dwr[a] = qr;
            dwv[a] = qv;
        }
        double gr = 0.0, gv = 0.0;
        for (int c = 0; c < 4; ++c)
            for (int a = 0; a < 4; ++a) {
                const double u = (double)Ub[(long long)(k0 + c) * nr + i0 + a];
                gr += dwr[a] * wv[c] * u;
                gv += wr[a] * dwv[c] * u;
            }
        double z, Jr, Jv, J2;
        metric(sr / (nr - 1), p.rmin, p.rmax, p.ar, D.centre_r, z, Jr, J2);
        metric(sv / (nv - 1), 0.0, p.vmax, p.av, p.kv, z, Jv, J2);
        greeks[2 * b] = gr * (nr - 1) / Jr;
        greeks[2 * b + 1] = gv * (nv - 1) / Jv;
    }
    if (indicators) {
        // A-posteriori rounding indicator of the march (reading of the
        // precision-control step): the unit roundoff of the operator's
        // coefficients times the price, that of the state times the
        // random-walk growth of the per-step rounding of U over the stencil,
        // and that of the increments times the summed per-step increments on
        // the stencil.
        double umax = 0.0, incr = 0.0;
        for (int c = 0; c < 4; ++c)
            for (int a = 0; a < 4; ++a) umax = fmax(umax, fabs((double)Ub[(long long)(k0 + c) * nr + i0 + a]));
        for (int n = 0; n < g.nsteps; ++n) incr += (double)g.acc[(size_t)b * g.nsteps + n];
        indicators[b] = kIndicatorC * (u_op * fabs(s) + u_state * sqrt((double)g.nsteps) * umax + u_incr * incr);
    }
}

// ------------------------------------------------------------- launchers

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t tables_bytes(int nr, int nv, int ny, int nsteps, int B, size_t elem)
{
    size_t s = 0;
    s += align_up((size_t)B * RT_N * nr * elem);
    s += align_up((size_t)B * R2_N * nr * elem);
    s += align_up((size_t)B * VT_N * nv * elem);
    s += align_up((size_t)B * YT_N * ny * elem);
    s += align_up((size_t)B * SC_N * elem);
    s += align_up((size_t)B * nsteps * 2 * elem);
    s += align_up((size_t)B * nsteps * 2 * ny * elem);
    s += align_up((size_t)B * 3 * nv * elem);
    s += align_up((size_t)B * nv * 3 * ny * elem);
    s += align_up((size_t)B * part_sys_size(nv, kMaxSplit) * elem);
    s += align_up((size_t)B * nv * part_sys_size(ny, kMaxSplit) * elem);
    s += align_up((size_t)B * FL_N * sizeof(int));
    s += align_up((size_t)B * nsteps * sizeof(float));
    s += align_up((size_t)B * 3 * (nr + nv + ny) * sizeof(double));
    s += align_up((size_t)B * sizeof(InstDerived));
    return s;
}

void tables_carve(GroupTables& g, void* block, size_t elem)
{
    char* p = (char*)block;
    const size_t B = g.B;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += align_up(bytes);
        return (void*)q;
    };
    g.rt = take(B * RT_N * g.nr * elem);
    g.r2 = take(B * R2_N * g.nr * elem);
    g.vt = take(B * VT_N * g.nv * elem);
    g.yt = take(B * YT_N * g.ny * elem);
    g.sc = take(B * SC_N * elem);
    g.st = take(B * g.nsteps * 2 * elem);
    g.dir = take(B * g.nsteps * 2 * g.ny * elem);
    g.vf = take(B * 3 * g.nv * elem);
    g.yf = take(B * g.nv * 3 * g.ny * elem);
    g.vp = take(B * part_sys_size(g.nv, kMaxSplit) * elem);
    g.yp = take(B * g.nv * part_sys_size(g.ny, kMaxSplit) * elem);
    g.fl = (int*)take(B * FL_N * sizeof(int));
    g.acc = (float*)take(B * g.nsteps * sizeof(float));
    double* ax = (double*)take(B * 3 * (g.nr + g.nv + g.ny) * sizeof(double));
    g.axr = ax;
    g.axv = ax + B * 3 * g.nr;
    g.axy = g.axv + B * 3 * g.nv;
    g.derived = (InstDerived*)take(B * sizeof(InstDerived));
}

cudaError_t launch_setup(const GroupTables& g, size_t elem, cudaStream_t s)
{
    const dim3 faces(g.nsteps, g.B);
    // p2P of 0 (passes 2 and 3 fused), 1 or kLinesTma needs no split factors
    auto ok = [](int P, int lo) { return (P >= lo && P <= kMaxSplit) || P == kLinesTma; };
    if (!ok(g.p2P, 0) || !ok(g.p3P, 1)) return cudaErrorInvalidValue;
    const bool sv = g.p2P > 1 && g.p2P <= kMaxSplit, sy = g.p3P > 1 && g.p3P <= kMaxSplit;
    if (elem == sizeof(float)) {
        k_setup<float><<<g.B, 256, 0, s>>>(g);
        k_faces<float><<<faces, 128, 0, s>>>(g);
        if (sv) k_split<float><<<g.B, 32, 0, s>>>(g, 0, g.p2P);
        if (sy) k_split<float><<<(unsigned)(g.B * g.nv), 32, 0, s>>>(g, 1, g.p3P);
    } else {
        k_setup<double><<<g.B, 256, 0, s>>>(g);
        k_faces<double><<<faces, 128, 0, s>>>(g);
        if (sv) k_split<double><<<g.B, 32, 0, s>>>(g, 0, g.p2P);
        if (sy) k_split<double><<<(unsigned)(g.B * g.nv), 32, 0, s>>>(g, 1, g.p3P);
    }
    return cudaGetLastError();
}

cudaError_t launch_terminal(const GroupTables& g, void* U, size_t elem, cudaStream_t s)
{
    const dim3 grid(g.ny, g.B);
    if (elem == sizeof(float))
        k_terminal<float><<<grid, 128, 0, s>>>(g, (float*)U);
    else
        k_terminal<double><<<grid, 128, 0, s>>>(g, (double*)U);
    return cudaGetLastError();
}

cudaError_t launch_faces64(const GroupTables& g, double* dir64, cudaStream_t s)
{
    GroupTables h = g;
    h.dir = dir64;
    k_faces<double><<<dim3(g.nsteps, g.B), 128, 0, s>>>(h);
    return cudaGetLastError();
}

cudaError_t launch_readout(const GroupTables& g, const void* U, size_t elem, double* prices,
                           double* indicators, double* greeks, cudaStream_t s, bool incr32)
{
    const int blocks = (g.B + 63) / 64;
    const double u32 = 5.9604644775390625e-08, u64 = 1.1102230246251565e-16;
    if (elem == sizeof(float))
        k_readout<float><<<blocks, 64, 0, s>>>(g, (const float*)U, prices, indicators, greeks, u32, u32, u32);
    else if (incr32)  // FP32 operator and increments on an FP64 state
        k_readout<double><<<blocks, 64, 0, s>>>(g, (const double*)U, prices, indicators, greeks, u32, u64, u32);
    else
        k_readout<double><<<blocks, 64, 0, s>>>(g, (const double*)U, prices, indicators, greeks, u64, u64, u64);
    return cudaGetLastError();
}

template <typename T>
March<T> march_args(const GroupTables& g)
{
    March<T> P;
    P.nr = g.nr;
    P.nv = g.nv;
    P.ny = g.ny;
    P.nsteps = g.nsteps;
    P.B = g.B;
    P.N = (long long)g.nr * g.nv * g.ny;
    P.rt = (const T*)g.rt;
    P.r2 = (const T*)g.r2;
    P.vt = (const T*)g.vt;
    P.yt = (const T*)g.yt;
    P.sc = (const T*)g.sc;
    P.st = (const T*)g.st;
    P.dir = (const T*)g.dir;
    P.vf = (const T*)g.vf;
    P.yf = (const T*)g.yf;
    P.fl = g.fl;
    P.acc = g.acc;
    P.vp = (const T*)g.vp;
    P.yp = (const T*)g.yp;
    P.p2P = g.p2P;
    P.p3P = g.p3P;
    P.tma_ok = g.tma_ok;
    return P;
}

template March<float> march_args<float>(const GroupTables&);
template March<double> march_args<double>(const GroupTables&);

}  // namespace hjm
