// Pass 1 of a Douglas ADI step (Section 5.1): the explicit operator
//   dU0 = dt F(U^n; t^n),  F = A_r U + A_v U + A_y U + A_0 U   (Eq. (1) in the
//   metric form of Section 4.3, centred differences of Section 5, the r-v
//   mixed term A_0 explicit only)
// fused with the r-line solve (I - theta dt A_r(t^{n+1/2})) dU1 = dU0.
//
// r lines are contiguous in memory. A line is owned by a segment of S lanes
// of a warp (S = 8, 16 or 32; 32/S lines per warp side by side); lane l of
// the segment holds M consecutive nodes e = l*M .. l*M+M-1, loaded with
// 16-byte vector loads. The per-node r factors of the operator (7 tables)
// are loaded once per CTA (a CTA never spans two instruments) into shared
// memory, laid out so every read is conflict-free (or, as a variant, into
// registers), and reused for every line the CTA processes. The line system is
// solved by a partition method: each lane eliminates its chunk down to
// equations in its first and last unknowns, the S interface equations are
// solved by parallel cyclic reduction over width-S warp shuffles, and each
// lane back-substitutes.
#include <stdio.h>
#include <stdlib.h>

#include "hjm_kernels.cuh"

namespace hjm {

template <typename T>
__device__ __forceinline__ T fast_rcp(T x)
{
    return T(1) / x;
}
// FP32 march: the hardware reciprocal (relative error of a few ulp) is
// ample for the FP32 tolerance and keeps the solver off the divide path.
template <>
__device__ __forceinline__ float fast_rcp<float>(float x)
{
    return __fdividef(1.0f, x);
}

template <typename T, int M>
__device__ __forceinline__ void p1_load(const T* __restrict__ row, int e0, int nr, T (&u)[M])
{
    constexpr int V = 16 / sizeof(T);
    if constexpr (M % V == 0) {
        if (e0 + M <= nr && (reinterpret_cast<uintptr_t>(row + e0) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < M / V; ++q) {
                if constexpr (sizeof(T) == 4) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(row + e0) + q);
                    u[4 * q] = x.x;
                    u[4 * q + 1] = x.y;
                    u[4 * q + 2] = x.z;
                    u[4 * q + 3] = x.w;
                } else {
                    const double2 x = __ldg(reinterpret_cast<const double2*>(row + e0) + q);
                    u[2 * q] = x.x;
                    u[2 * q + 1] = x.y;
                }
            }
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) u[m] = (e0 + m < nr) ? __ldg(row + e0 + m) : T(0);
}

template <typename T, int M>
__device__ __forceinline__ void p1_store(T* __restrict__ row, int e0, int nr, const T (&u)[M])
{
    constexpr int V = 16 / sizeof(T);
    if constexpr (M % V == 0) {
        if (e0 + M <= nr && (reinterpret_cast<uintptr_t>(row + e0) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < M / V; ++q) {
                if constexpr (sizeof(T) == 4)
                    reinterpret_cast<float4*>(row + e0)[q] =
                        make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
                else
                    reinterpret_cast<double2*>(row + e0)[q] = make_double2(u[2 * q], u[2 * q + 1]);
            }
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m)
        if (e0 + m < nr) row[e0 + m] = u[m];
}

// Partition solve of the tridiagonal system held by one S-lane segment
// (rows e = sl*M + m; a: sub-, b: main, c: super-diagonal, d: right-hand
// side; a of the first and c of the last row are 0, padding rows are
// identity rows). d returns the solution.
template <typename T, int S, int M>
__device__ __forceinline__ void seg_partition_solve(T (&a)[M], T (&b)[M], T (&c)[M], T (&d)[M],
                                                    int sl)
{
    static_assert(M >= 2, "chunk of at least two rows");
    // Forward elimination in the chunk: rows m >= 1 become
    //   a[m] x_s + x_m + c[m] x_{m+1} = d[m]   (x_s: the chunk's first unknown)
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const T r = fast_rcp(b[m]);
        a[m] *= r;
        c[m] *= r;
        d[m] *= r;
    }
#pragma unroll
    for (int m = 2; m < M; ++m) {
        const T r = fast_rcp(b[m] - a[m] * c[m - 1]);
        d[m] = r * (d[m] - a[m] * d[m - 1]);
        a[m] = -r * a[m] * a[m - 1];
        c[m] = r * c[m];
    }
    // Backward elimination: rows 1..M-2 become a[m] x_s + x_m + c[m] x_e = d[m].
#pragma unroll
    for (int m = M - 3; m >= 1; --m) {
        d[m] -= c[m] * d[m + 1];
        a[m] -= c[m] * a[m + 1];
        c[m] = -c[m] * c[m + 1];
    }
    // Row 0: a[0] x_{previous chunk's last} + x_s + c[0] x_e = d[0].
    if constexpr (M >= 3) {
        const T r = fast_rcp(T(1) - c[0] * a[1]);
        d[0] = r * (d[0] - c[0] * d[1]);
        a[0] = r * a[0];
        c[0] = -r * c[0] * c[1];
    }
    // Interface equations in the chunks' last unknowns.
    const T aS = a[0], cS = c[0], dS = d[0];
    const T aE = a[M - 1], cE = c[M - 1], dE = d[M - 1];
    T aSn = __shfl_down_sync(0xffffffffu, aS, 1, S);
    T cSn = __shfl_down_sync(0xffffffffu, cS, 1, S);
    T dSn = __shfl_down_sync(0xffffffffu, dS, 1, S);
    if (sl == S - 1) aSn = cSn = dSn = T(0);
    T al = -aE * aS;
    T be = T(1) - aE * cS - cE * aSn;
    T ga = -cE * cSn;
    T de = dE - aE * dS - cE * dSn;
#pragma unroll
    for (int s = 1; s < S; s <<= 1) {
        const T alm = __shfl_up_sync(0xffffffffu, al, s, S), bem = __shfl_up_sync(0xffffffffu, be, s, S);
        const T gam = __shfl_up_sync(0xffffffffu, ga, s, S), dem = __shfl_up_sync(0xffffffffu, de, s, S);
        const T alp = __shfl_down_sync(0xffffffffu, al, s, S), bep = __shfl_down_sync(0xffffffffu, be, s, S);
        const T gap = __shfl_down_sync(0xffffffffu, ga, s, S), dep = __shfl_down_sync(0xffffffffu, de, s, S);
        // Lanes with no partner s below (above) already have al = 0 (ga = 0):
        // the first row of the line has no sub-diagonal, the last no
        // super-diagonal, and each step doubles the zeroed span. The
        // out-of-range shuffles return the lane's own (finite) values, which
        // are then multiplied by k1 = 0 (k2 = 0).
        const T k1 = al * fast_rcp(bem), k2 = ga * fast_rcp(bep);
        const T nbe = be - gam * k1 - alp * k2;
        const T nde = de - dem * k1 - dep * k2;
        al = -alm * k1;
        ga = -gap * k2;
        be = nbe;
        de = nde;
    }
    const T xE = de * fast_rcp(be);
    T xEp = __shfl_up_sync(0xffffffffu, xE, 1, S);
    if (sl == 0) xEp = T(0);
    const T xS = dS - aS * xEp - cS * xE;
#pragma unroll
    for (int m = 1; m < M - 1; ++m) d[m] = d[m] - a[m] * xS - c[m] * xE;
    d[0] = xS;
    d[M - 1] = xE;
}

// One CTA = 4 warps = 4 * (32/S) segments; each segment processes R lines of
// one instrument (line index k + n_v j), all segments of a warp advancing
// together so the width-S shuffles always see full warps.
template <typename T, int S, int M, bool TS, bool PF>
__global__ void __launch_bounds__(128) k_pass1(const March<T> P, const T* __restrict__ U,
                                               T* __restrict__ out, const int n, const int R)
{
    constexpr int G = 32 / S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / S, sl = lane % S;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int L = nv * ny;
    const int lpc = 4 * G * R;
    const int bpi = (L + lpc - 1) / lpc;
    const int b = blockIdx.x / bpi, cb = blockIdx.x % bpi;

    const T* __restrict__ Ub = U + (long long)b * P.N;
    T* __restrict__ Ob = out + (long long)b * P.N;
    const T* __restrict__ rt = P.rt + (size_t)b * RT_N * nr;
    const T* __restrict__ vt = P.vt + (size_t)b * VT_N * nv;
    const T* __restrict__ yt = P.yt + (size_t)b * YT_N * ny;
    const T* __restrict__ sc = P.sc + (size_t)b * SC_N;
    const int* __restrict__ fl = P.fl + (size_t)b * FL_N;
    const T dt = sc[SC_DT], w = sc[SC_W];
    const T aF = P.st[((size_t)b * P.nsteps + n) * 2];
    const T aI = P.st[((size_t)b * P.nsteps + n) * 2 + 1];
    const T dA = aF - aI;
    const int rlo = fl[FL_RLO_DIR], yord = fl[FL_YORDER];
    const T* __restrict__ dir = P.dir + (((size_t)b * P.nsteps + n) * 2) * ny;

    // r-factor chunks of this lane, loaded once for all lines of the CTA:
    // in registers, or (TS) in shared memory laid out [table][m][lane in
    // segment] so each read is conflict-free.
    const int e0 = sl * M;
    __shared__ T tsm[TS ? RT_N * M * S : 1];
    T tR[TS ? 1 : M], tIJ[TS ? 1 : M], tC1[TS ? 1 : M], tC4V[TS ? 1 : M], tC4B[TS ? 1 : M],
        tC3[TS ? 1 : M], tCY[TS ? 1 : M];
    if constexpr (TS) {
        for (int idx = threadIdx.x; idx < RT_N * M * S; idx += blockDim.x) {
            const int q = idx / (M * S), e = idx % (M * S);
            tsm[(q * M + e % M) * S + e / M] = e < nr ? rt[q * nr + e] : T(0);
        }
        __syncthreads();
    } else {
        p1_load<T, M>(rt + RT_R * nr, e0, nr, tR);
        p1_load<T, M>(rt + RT_IJ * nr, e0, nr, tIJ);
        p1_load<T, M>(rt + RT_C1 * nr, e0, nr, tC1);
        p1_load<T, M>(rt + RT_C4V * nr, e0, nr, tC4V);
        p1_load<T, M>(rt + RT_C4B * nr, e0, nr, tC4B);
        p1_load<T, M>(rt + RT_C3 * nr, e0, nr, tC3);
        p1_load<T, M>(rt + RT_CY * nr, e0, nr, tCY);
    }
#define TAB(arr, q, m) (TS ? tsm[((q) * M + (m)) * S + sl] : arr[TS ? 0 : (m)])

    // Rows of the current line (and, with PF, of the next one, loaded while
    // the current line is computed).
    auto line_rows = [&](int it, int& k, int& j, bool& valid, int& ka, int& kb, int& ja, int& jb) {
        const int line = cb * lpc + (warp * R + it) * G + seg;
        valid = line < L;
        const int lc = valid ? line : L - 1;  // keep addresses in bounds
        k = lc % nv;
        j = lc / nv;
        const bool vin_ = k > 0 && k < nv - 1;
        ka = vin_ ? k - 1 : (k == 0 ? 1 : nv - 2);
        kb = vin_ ? k + 1 : (k == 0 ? 2 : nv - 3);
        const bool yin_ = j > 0 && j < ny - 1;
        ja = yin_ ? j - 1 : (j == 0 ? 1 : ny - 2);
        jb = yin_ ? j + 1 : (j == 0 ? 2 : ny - 3);
    };
    T uc[M], ua[M], ub[M], ya[M], yb[M];
    T nuc[PF ? M : 1], nua[PF ? M : 1], nub[PF ? M : 1], nya[PF ? M : 1], nyb[PF ? M : 1];
    int k, j, ka, kb, ja, jb;
    bool valid;
    line_rows(0, k, j, valid, ka, kb, ja, jb);
    auto load5 = [&](int k_, int j_, int ka_, int kb_, int ja_, int jb_, T (&c_)[M], T (&a_)[M],
                     T (&b_)[M], T (&ya_)[M], T (&yb_)[M]) {
        p1_load<T, M>(Ub + ((long long)j_ * nv + k_) * nr, e0, nr, c_);
        p1_load<T, M>(Ub + ((long long)j_ * nv + ka_) * nr, e0, nr, a_);
        p1_load<T, M>(Ub + ((long long)j_ * nv + kb_) * nr, e0, nr, b_);
        p1_load<T, M>(Ub + ((long long)ja_ * nv + k_) * nr, e0, nr, ya_);
        p1_load<T, M>(Ub + ((long long)jb_ * nv + k_) * nr, e0, nr, yb_);
    };
    load5(k, j, ka, kb, ja, jb, uc, ua, ub, ya, yb);

    for (int it = 0; it < R; ++it) {
        int nk = 0, nj = 0, nka = 0, nkb = 0, nja = 0, njb = 0;
        bool nvalid = false;
        if constexpr (PF) {
            if (it + 1 < R) {
                line_rows(it + 1, nk, nj, nvalid, nka, nkb, nja, njb);
                load5(nk, nj, nka, nkb, nja, njb, nuc, nua, nub, nya, nyb);
            }
        }

        const T v = vt[VT_V * nv + k];
        const T g2 = vt[VT_G2 * nv + k], g5 = vt[VT_G5 * nv + k], fv = vt[VT_FV * nv + k];
        const T vq = v * vt[VT_IJ * nv + k];
        const T y = yt[YT_Y * ny + j], iJy = yt[YT_IJ * ny + j], ky = yt[YT_KY * ny + j];
        const T aIy = aI + y, aFy = aF + y;
        const T vy = v * iJy, kyy = ky * iJy;  // g6 = cy * vy + kyy
        const T gLo = dir[j], gHi = dir[ny + j];

        const bool vin = k > 0 && k < nv - 1;
        const bool yin = j > 0 && j < ny - 1;
        T d[M];
        const T uc_prev = __shfl_up_sync(0xffffffffu, uc[M - 1], 1, S);
        const T uc_next = __shfl_down_sync(0xffffffffu, uc[0], 1, S);
        const T ua_prev = __shfl_up_sync(0xffffffffu, ua[M - 1], 1, S);
        const T ua_next = __shfl_down_sync(0xffffffffu, ua[0], 1, S);
        const T ub_prev = __shfl_up_sync(0xffffffffu, ub[M - 1], 1, S);
        const T ub_next = __shfl_down_sync(0xffffffffu, ub[0], 1, S);

        T a[M], bb[M], c[M];
        // r part, the r-v mixed term and the rows of I - theta dt A_r(t^{n+1/2}),
        // for every node as if interior in r (the r faces are patched below).
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const T u = uc[m];
            const T um = m > 0 ? uc[m - 1] : uc_prev;
            const T up = m < M - 1 ? uc[m + 1] : uc_next;
            const T g1 = TAB(tC1, RT_C1, m) * v;                                  // zeta_rr/(J^2 h^2)
            const T g4I = aIy * TAB(tIJ, RT_IJ, m) + (TAB(tC4B, RT_C4B, m) - v * TAB(tC4V, RT_C4V, m));     // g4/(2h) at t^{n+1/2}
            const T g4F = g4I + dA * TAB(tIJ, RT_IJ, m);                          // g4/(2h) at t^n
            T f = g1 * ((up - u) - (u - um)) + g4F * (up - um) - TAB(tR, RT_R, m) * u;
            const T bp = m < M - 1 ? ub[m + 1] : ub_next, bm = m > 0 ? ub[m - 1] : ub_prev;
            const T ap = m < M - 1 ? ua[m + 1] : ua_next, am = m > 0 ? ua[m - 1] : ua_prev;
            if (vin) f += TAB(tC3, RT_C3, m) * vq * ((bp - bm) - (ap - am));
            d[m] = f;
            a[m] = -w * (g1 - g4I);
            bb[m] = T(1) + w * (T(2) * g1 + TAB(tR, RT_R, m));
            c[m] = -w * (g1 + g4I);
        }
        // v and y parts (face lines use one-sided differences, Section 7.3).
        if (vin && yin) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const T u = uc[m];
                const T g6 = TAB(tCY, RT_CY, m) * vy + kyy;
                d[m] = dt * (d[m] + g2 * ((ub[m] - u) - (u - ua[m])) + g5 * (ub[m] - ua[m]) +
                             g6 * (yb[m] - ya[m]));
            }
        } else {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const T u = uc[m];
                T Av;
                if (vin)
                    Av = g2 * ((ub[m] - u) - (u - ua[m])) + g5 * (ub[m] - ua[m]);
                else if (k == 0)
                    Av = fv * (T(-3) * u + T(4) * ua[m] - ub[m]);
                else
                    Av = fv * (T(3) * u - T(4) * ua[m] + ub[m]);
                const T g6 = TAB(tCY, RT_CY, m) * vy + kyy;
                T Ay;
                if (yin)
                    Ay = g6 * (yb[m] - ya[m]);
                else if (j == 0)
                    Ay = yord == 1 ? T(2) * g6 * (ya[m] - u) : g6 * (T(-3) * u + T(4) * ya[m] - yb[m]);
                else
                    Ay = yord == 1 ? T(2) * g6 * (u - ya[m]) : g6 * (T(3) * u - T(4) * ya[m] + yb[m]);
                d[m] = dt * (d[m] + Av + Ay);
            }
        }
        // r faces: Dirichlet rows at r_max (and r_min when gamma = 0), the
        // degenerate r = 0 face when gamma > 0, identity padding rows.
        if (sl == 0) {
            if (rlo) {
                d[0] = gLo - uc[0];
                a[0] = T(0);
                bb[0] = T(1);
                c[0] = T(0);
            } else {
                // one-sided first derivative, zeta_rr = 0 and no mixed term at r = 0;
                // recompute the node's F without the centred r and mixed parts.
                const T u = uc[0], u1 = uc[1], u2 = M >= 3 ? uc[M >= 3 ? 2 : 1] : uc_next;
                const T fr = aFy * TAB(tIJ, RT_IJ, 0) + TAB(tC4B, RT_C4B, 0);  // mu_r / (2 h J) at t^n
                T Av;
                if (vin)
                    Av = g2 * ((ub[0] - u) - (u - ua[0])) + g5 * (ub[0] - ua[0]);
                else if (k == 0)
                    Av = fv * (T(-3) * u + T(4) * ua[0] - ub[0]);
                else
                    Av = fv * (T(3) * u - T(4) * ua[0] + ub[0]);
                const T g6 = TAB(tCY, RT_CY, 0) * vy + kyy;
                T Ay;
                if (yin)
                    Ay = g6 * (yb[0] - ya[0]);
                else if (j == 0)
                    Ay = yord == 1 ? T(2) * g6 * (ya[0] - u) : g6 * (T(-3) * u + T(4) * ya[0] - yb[0]);
                else
                    Ay = yord == 1 ? T(2) * g6 * (u - ya[0]) : g6 * (T(3) * u - T(4) * ya[0] + yb[0]);
                d[0] = dt * (fr * (T(-3) * u + T(4) * u1 - u2) - TAB(tR, RT_R, 0) * u + Av + Ay);
                const T frI = T(2) * (aIy * TAB(tIJ, RT_IJ, 0) + TAB(tC4B, RT_C4B, 0));  // mu_r / (h J) at t^{n+1/2}
                a[0] = T(0);
                bb[0] = T(1) + w * (frI + TAB(tR, RT_R, 0));
                c[0] = -w * frI;
            }
        }
        if (e0 + M > nr - 1) {  // only lanes holding r_max or padding
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int e = e0 + m;
                if (e >= nr - 1) {
                    d[m] = e == nr - 1 ? gHi - uc[m] : T(0);
                    a[m] = T(0);
                    bb[m] = T(1);
                    c[m] = T(0);
                }
            }
        }
        seg_partition_solve<T, S, M>(a, bb, c, d, sl);
        if (valid) p1_store<T, M>(Ob + ((long long)j * nv + k) * nr, e0, nr, d);
        if (it + 1 < R) {
            if constexpr (PF) {
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    uc[m] = nuc[m];
                    ua[m] = nua[m];
                    ub[m] = nub[m];
                    ya[m] = nya[m];
                    yb[m] = nyb[m];
                }
                k = nk;
                j = nj;
                valid = nvalid;
            } else {
                line_rows(it + 1, k, j, valid, ka, kb, ja, jb);
                load5(k, j, ka, kb, ja, jb, uc, ua, ub, ya, yb);
            }
        }
    }
#undef TAB
}

// (S, M, R) per r-line length: M nodes per lane, S lanes per line, R lines
// per segment per CTA.
struct P1Shape {
    int S, M, R, TS, PF;
};

// HJM_PASS1_SHAPE="S,M,R,TS,PF" overrides the table below (tuning experiments).
static bool p1_override(P1Shape& sh)
{
    static int state = -1;
    static P1Shape ov{0, 0, 0};
    if (state < 0) {
        const char* e = getenv("HJM_PASS1_SHAPE");
        state = e && sscanf(e, "%d,%d,%d,%d,%d", &ov.S, &ov.M, &ov.R, &ov.TS, &ov.PF) == 5 ? 1 : 0;
    }
    if (state) sh = ov;
    return state == 1;
}

static P1Shape p1_shape(int nr, size_t elem)
{
    P1Shape ov;
    if (p1_override(ov) && ov.S * ov.M >= nr) return ov;
    // Measured on GB300 (config-2-shaped batches): tables in shared memory
    // (128 registers, 16 warps per SM) beat tables in registers (173
    // registers) by 1.3-1.4x; prefetching the next line's rows costs more in
    // occupancy than it hides.
    if (elem == 4) {
        if (nr <= 64) return {8, 8, 4, 1, 0};
        if (nr <= 128) return {16, 8, 4, 1, 0};
        if (nr <= 256) return {32, 8, 4, 1, 0};
        return {32, 16, 4, 1, 0};
    }
    if (nr <= 32) return {16, 2, 4, 1, 0};
    if (nr <= 64) return {16, 4, 4, 1, 0};
    if (nr <= 128) return {32, 4, 4, 1, 0};
    if (nr <= 256) return {32, 8, 4, 1, 0};
    return {32, 16, 4, 1, 0};
}

int pass1_chunk(int nr)
{
    return nr <= 512 ? p1_shape(nr, 4).M : 0;
}

template <typename T, int S, int M, bool TS, bool PF>
static cudaError_t p1_launch(const March<T>& P, const T* U, T* out, int n, int R, cudaStream_t s)
{
    const int lpc = 4 * (32 / S) * R;
    const int bpi = (P.nv * P.ny + lpc - 1) / lpc;
    k_pass1<T, S, M, TS, PF><<<(unsigned)(bpi * P.B), 128, 0, s>>>(P, U, out, n, R);
    return cudaGetLastError();
}

template <typename T, int S, int M>
static cudaError_t p1_launch_v(const March<T>& P, const T* U, T* out, int n, const P1Shape& sh,
                               cudaStream_t s)
{
    if (sh.TS && sh.PF) return p1_launch<T, S, M, true, true>(P, U, out, n, sh.R, s);
    if (sh.TS) return p1_launch<T, S, M, true, false>(P, U, out, n, sh.R, s);
    if (sh.PF) return p1_launch<T, S, M, false, true>(P, U, out, n, sh.R, s);
    return p1_launch<T, S, M, false, false>(P, U, out, n, sh.R, s);
}

template <typename T>
cudaError_t launch_pass1(const March<T>& P, const T* U, T* out, int n, cudaStream_t s)
{
    const P1Shape sh = p1_shape(P.nr, sizeof(T));
    if (P.nr > 512) return cudaErrorInvalidValue;
    if constexpr (sizeof(T) == 4) {
        if (sh.S == 8 && sh.M == 8) return p1_launch_v<T, 8, 8>(P, U, out, n, sh, s);
        if (sh.S == 16 && sh.M == 8) return p1_launch_v<T, 16, 8>(P, U, out, n, sh, s);
        if (sh.S == 32 && sh.M == 8) return p1_launch_v<T, 32, 8>(P, U, out, n, sh, s);
        if (sh.S == 32 && sh.M == 4) return p1_launch_v<T, 32, 4>(P, U, out, n, sh, s);
        return p1_launch<T, 32, 16, true, false>(P, U, out, n, sh.R, s);
    } else {
        if (sh.S == 16 && sh.M == 2) return p1_launch<T, 16, 2, true, false>(P, U, out, n, sh.R, s);
        if (sh.S == 16 && sh.M == 4) return p1_launch<T, 16, 4, true, false>(P, U, out, n, sh.R, s);
        if (sh.S == 32 && sh.M == 4) return p1_launch<T, 32, 4, true, false>(P, U, out, n, sh.R, s);
        if (sh.S == 32 && sh.M == 8) return p1_launch<T, 32, 8, true, false>(P, U, out, n, sh.R, s);
        return p1_launch<T, 32, 16, true, false>(P, U, out, n, sh.R, s);
    }
}

template cudaError_t launch_pass1<float>(const March<float>&, const float*, float*, int, cudaStream_t);
template cudaError_t launch_pass1<double>(const March<double>&, const double*, double*, int, cudaStream_t);

}  // namespace hjm
