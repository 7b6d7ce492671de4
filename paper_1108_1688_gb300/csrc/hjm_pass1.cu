// Pass 1 of a Douglas ADI step (Section 5.1): the explicit operator
//   dU0 = dt F(U^n; t^n),  F = A_r U + A_v U + A_y U + A_0 U   (Eq. (1) in the
//   metric form of Section 4.3, centred differences of Section 5, the r-v
//   mixed term A_0 explicit only)
// fused with the r-line solve (I - theta dt A_r(t^{n+1/2})) dU1 = dU0.
// The same kernel, given the first stage's result Y3, forms the correction
// stage of the Craig-Sneyd family (right-hand side from U^n and Y3, the
// weights in the scalar table; see SC_C1 in hjm_kernels.cuh).
//
// r lines are contiguous in memory. A line is owned by a segment of S lanes
// of a warp (S = 8, 16 or 32; 32/S lines per warp side by side); lane l of
// the segment holds M consecutive nodes e = l*M .. l*M+M-1, loaded with
// 16-byte vector loads (k_pass1), or from a shared-memory ring of staged y
// planes (k_pass1s). The per-node r factors of the operator (7 tables) are
// loaded once per CTA (a CTA never spans two instruments) into shared
// memory, laid out so the lanes' 16-byte reads are conflict-free, and reused
// for every line the CTA processes. In FP32 the per-node arithmetic runs on
// node pairs with the paired FP32 instructions. The line system is solved by
// a partition method: each lane eliminates its chunk down to equations in
// its first and last unknowns, the S interface equations are solved by
// parallel cyclic reduction over width-S warp shuffles, and each lane
// back-substitutes.
#include "hjm_kernels.cuh"

namespace hjm {

template <typename T>
__device__ __forceinline__ T fast_rcp(T x);
// FP32 march: the hardware reciprocal (relative error of a few ulp) is
// ample for the FP32 tolerance and keeps the solver off the divide path.
template <>
__device__ __forceinline__ float fast_rcp<float>(float x)
{
    return __fdividef(1.0f, x);
}
// FP64 march: the IEEE division. A Newton-Raphson reciprocal from the FP32
// hardware seed (two steps of y + y (1 - x y), four FP64 fused multiply-adds
// and two conversions) was measured 4 % slower on the FP64-bound pass 1, and
// the correctly rounded reciprocal intrinsic equal to it.
template <>
__device__ __forceinline__ double fast_rcp<double>(double x)
{
    return 1.0 / x;
}

// 16-byte asynchronous global -> shared copies (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit16() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait16()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Loads nodes e0 .. e0+M-1 of a row (zero past n_r); vec: the row start is
// 16-byte aligned and n_r a multiple of the vector width (checked once per
// launch), so whole chunks use 16-byte loads.
template <typename T, int M>
__device__ __forceinline__ void p1_load(const T* __restrict__ row, int e0, int nr, T (&u)[M], bool vec = false)
{
    constexpr int V = 16 / sizeof(T);
    if constexpr (M % V == 0) {
        if (e0 + M <= nr && (vec || (reinterpret_cast<uintptr_t>(row + e0) & 15) == 0)) {
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
__device__ __forceinline__ void p1_store(T* __restrict__ row, int e0, int nr, const T (&u)[M], bool vec = false)
{
    constexpr int V = 16 / sizeof(T);
    if constexpr (M % V == 0) {
        if (e0 + M <= nr && (vec || (reinterpret_cast<uintptr_t>(row + e0) & 15) == 0)) {
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
    // interface row al x_{e-1} + x_e + ga x_{e+1} = de, divided by its
    // diagonal, so that every reduction level below takes one reciprocal
    T al, ga, de;
    {
        const T r = fast_rcp(T(1) - aE * cS - cE * aSn);
        al = -aE * aS * r;
        ga = -cE * cSn * r;
        de = (dE - aE * dS - cE * dSn) * r;
    }
#pragma unroll
    for (int s = 1; s < S; s <<= 1) {
        const T alm = __shfl_up_sync(0xffffffffu, al, s, S), gam = __shfl_up_sync(0xffffffffu, ga, s, S);
        const T dem = __shfl_up_sync(0xffffffffu, de, s, S);
        const T alp = __shfl_down_sync(0xffffffffu, al, s, S), gap = __shfl_down_sync(0xffffffffu, ga, s, S);
        const T dep = __shfl_down_sync(0xffffffffu, de, s, S);
        // Lanes with no partner s below (above) already have al = 0 (ga = 0):
        // the first row of the line has no sub-diagonal, the last no
        // super-diagonal, and each step doubles the zeroed span. The
        // out-of-range shuffles return the lane's own (finite) values, which
        // are then multiplied by al = 0 (ga = 0). Eliminating x_{e-s} and
        // x_{e+s} with the neighbours' unit-diagonal rows and dividing by the
        // new diagonal keeps the row at unit diagonal.
        const T r = fast_rcp(T(1) - al * gam - ga * alp);
        const T nde = (de - al * dem - ga * dep) * r;
        al = -al * alm * r;
        ga = -ga * gap * r;
        de = nde;
    }
    const T xE = de;
    T xEp = __shfl_up_sync(0xffffffffu, xE, 1, S);
    if (sl == 0) xEp = T(0);
    const T xS = dS - aS * xEp - cS * xE;
#pragma unroll
    for (int m = 1; m < M - 1; ++m) d[m] = d[m] - a[m] * xS - c[m] * xE;
    d[0] = xS;
    d[M - 1] = xE;
}

// Arithmetic on pairs of values: for FP32 the paired FP32 instructions of
// sm_100-class GPUs (one instruction for both lanes of a float2), for FP64
// two scalar operations. Every operation rounds each component exactly as
// its scalar counterpart (a - b is fma(b, -1, a)).
template <typename T>
struct Two;
template <>
struct Two<float> {
    using V = float2;
    static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ V splat(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ float x(V a) { return a.x; }
    static __device__ __forceinline__ float y(V a) { return a.y; }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
};
template <>
struct Two<double> {
    using V = double2;
    static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ V splat(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ double x(V a) { return a.x; }
    static __device__ __forceinline__ double y(V a) { return a.y; }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
    static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
};

// Shared-memory layout of the r tables: tsm[q][sl][MP], lane sl's M nodes
// contiguous, padded to MP so that 16-byte vector reads by consecutive lanes
// fall in distinct banks (MP * sizeof(T) / 16 odd).
template <typename T, int M>
struct P1Layout {
    static constexpr int W = (M * sizeof(T) >= 16) ? int(16 / sizeof(T)) : M;  // nodes per vector read
    static constexpr int MP = (M * sizeof(T) < 16 || ((M * sizeof(T) / 16) & 1)) ? M : M + int(16 / sizeof(T));
};

template <typename T, int W>
struct VecOf;
template <>
struct VecOf<float, 4> {
    using type = float4;
};
template <>
struct VecOf<float, 2> {
    using type = float2;
};
template <>
struct VecOf<double, 2> {
    using type = double2;
};

template <typename T, int W>
__device__ __forceinline__ void lds_vec(const T* p, T (&o)[W])
{
    const typename VecOf<T, W>::type x = *reinterpret_cast<const typename VecOf<T, W>::type*>(p);
    if constexpr (W == 4) {
        o[0] = x.x;
        o[1] = x.y;
        o[2] = x.z;
        o[3] = x.w;
    } else {
        o[0] = x.x;
        o[1] = x.y;
    }
}

// Per-instrument scalars of one pass-1 launch.
template <typename T>
struct P1Inst {
    int nr, nv, ny, rlo, yord;
    T dt, w, aF, aI, dA;
    const T* vt;
    const T* yt;
    const T* dir;  // Dirichlet data of this step: [2][n_y]
    // correction stage of the Craig-Sneyd family only (SC_C1 ..)
    T c1, cx, kd;
    bool hv;
};

template <typename T, bool ST2 = false>
__device__ __forceinline__ P1Inst<T> p1_inst(const March<T>& P, int b, int n)
{
    P1Inst<T> I;
    I.nr = P.nr;
    I.nv = P.nv;
    I.ny = P.ny;
    const T* sc = P.sc + (size_t)b * SC_N;
    const int* fl = P.fl + (size_t)b * FL_N;
    I.dt = sc[SC_DT];
    I.w = sc[SC_W];
    I.aF = P.st[((size_t)b * P.nsteps + n) * 2];
    I.aI = P.st[((size_t)b * P.nsteps + n) * 2 + 1];
    I.dA = I.aF - I.aI;
    I.rlo = fl[FL_RLO_DIR];
    I.yord = fl[FL_YORDER];
    I.vt = P.vt + (size_t)b * VT_N * P.nv;
    I.yt = P.yt + (size_t)b * YT_N * P.ny;
    I.dir = P.dir + (((size_t)b * P.nsteps + n) * 2) * P.ny;
    if constexpr (ST2) {
        I.c1 = sc[SC_C1];
        I.cx = sc[SC_CX];
        I.kd = sc[SC_KD];
        I.hv = sc[SC_HE] != T(0);
    } else {
        I.c1 = I.cx = I.kd = T(0);
        I.hv = false;
    }
    return I;
}

// One r line (v node k, y node j) on an S-lane segment, lane sl holding nodes
// e0 = sl M .. e0 + M - 1 (tables of this lane at tl, layout P1Layout):
//   1. the right-hand side dU0 = dt F(U^n) from the five rows (centre, v-a,
//      v-b, y-a, y-b; a, b the neighbours, one-sided on faces), face rows
//      patched;
//   2. the rows of I - theta dt A_r(t^{n+1/2}) from the r tables and the
//      line's (v, y) (the input rows are dead by then, which bounds the
//      registers at about 6 M + scalars);
//   3. the partition solve. d returns dU1 on the lane's nodes.
// ST2 (correction stage of the Craig-Sneyd family): the rows hold
// U + c1 E and xx the extra term: the mixed-term rows' weighted difference
// cx (E_{v,b} - E_{v,a}) (CS, MCS) or -E (HV, added to the right-hand
// side); Dirichlet nodes take kd (g - U - c1 E).
template <typename T, int S, int M, bool ST2 = false>
__device__ __forceinline__ void p1_line(const P1Inst<T>& I, const T* tl, int sl, int k, int j, const T (&uc)[M],
                                        const T (&ua)[M], const T (&ub)[M], const T (&ya)[M], const T (&yb)[M],
                                        const T (&xx)[M], T (&d)[M])
{
    constexpr int W = P1Layout<T, M>::W, MP = P1Layout<T, M>::MP;
    const int nr = I.nr, nv = I.nv, ny = I.ny, e0 = sl * M;
    const T* vt = I.vt;
    const T* yt = I.yt;
    const T v = vt[VT_V * nv + k];
    const T g2 = vt[VT_G2 * nv + k], g5 = vt[VT_G5 * nv + k], fv = vt[VT_FV * nv + k];
    const bool vin = k > 0 && k < nv - 1;
    const bool yin = j > 0 && j < ny - 1;
    const T vq = vin ? v * vt[VT_IJ * nv + k] : T(0);  // mixed term off on v faces
    const T y = yt[YT_Y * ny + j], iJy = yt[YT_IJ * ny + j], ky = yt[YT_KY * ny + j];
    const T aIy = I.aI + y, aFy = I.aF + y;
    const T vy = v * iJy, kyy = ky * iJy;  // g6 = cy * vy + kyy
    // v part A_v U = cA (U_{v,a} - U) + cB (U_{v,b} - U); centred inside,
    // one-sided on the v faces (Section 7.3).
    const T cA = vin ? g2 - g5 : (k == 0 ? T(4) * fv : T(-4) * fv);
    const T cB = vin ? g2 + g5 : (k == 0 ? -fv : fv);
    // y part A_y U = g6 (yA (U_{y,a} - U) + yB (U_{y,b} - U)).
    const int yord = I.yord;
    const T yA = yin ? T(-1) : (yord == 1 ? (j == 0 ? T(2) : T(-2)) : (j == 0 ? T(4) : T(-4)));
    const T yB = yin ? T(1) : (yord == 1 ? T(0) : (j == 0 ? T(-1) : T(1)));
    const T dt = I.dt, w = I.w;
    // FP64: dt rides on the per-line factors of the v and y parts, so the
    // first sweep yields dt (A_v + A_y) U directly and the second adds it in
    // one fused multiply-add (in FP32 the extra live scalars cost the
    // correction-stage shapes a CTA per SM)
    constexpr bool FOLD = sizeof(T) == 8;
    const T sd = FOLD ? dt : T(1);
    const T cAd = cA * sd, cBd = cB * sd, vyd = vy * sd, kyyd = kyy * sd;

#define TABV(q, m0, arr) lds_vec<T, W>(tl + (q) * S * MP + (m0), arr)
    // 1. right-hand side, every node as if interior in r, in two sweeps over
    // node pairs (m, m+1) (so the FP32 march runs on the paired FP32 pipe,
    // two lanes of arithmetic per instruction): (a) the v and y parts and the
    // mixed-term row differences wd = U_{v,b} - U_{v,a}, after which the four
    // neighbour rows are dead; (b) the r part, the reaction and the mixed
    // term from U and wd. Splitting the sweep keeps the registers of the
    // rows, the tables and the pair constants from being live together.
    using PV = typename Two<T>::V;
    constexpr int H = M / 2;
    // ST2: weights of xx in the mixed-term difference and in the right-hand side
    const PV xw2 = Two<T>::splat(ST2 && !I.hv ? T(1) : T(0)), xr2 = Two<T>::splat(ST2 && I.hv ? T(1) : T(0));
    T wd[M];
    {
        const PV cA2 = Two<T>::splat(cAd), cB2 = Two<T>::splat(cBd);
        const PV vy2 = Two<T>::splat(vyd), kyy2 = Two<T>::splat(kyyd), yA2 = Two<T>::splat(yA), yB2 = Two<T>::splat(yB);
#pragma unroll
        for (int m0 = 0; m0 < M; m0 += W) {
            T tCY[W];
            TABV(RT_CY, m0, tCY);
#pragma unroll
            for (int q = 0; q < W; q += 2) {
                const int m = m0 + q;
                const PV u = Two<T>::mk(uc[m], uc[m + 1]);
                const PV va = Two<T>::mk(ua[m], ua[m + 1]), vb = Two<T>::mk(ub[m], ub[m + 1]);
                const PV g6 = Two<T>::fma(Two<T>::mk(tCY[q], tCY[q + 1]), vy2, kyy2);
                const PV yy = Two<T>::fma(yA2, Two<T>::sub(Two<T>::mk(ya[m], ya[m + 1]), u),
                                          Two<T>::mul(yB2, Two<T>::sub(Two<T>::mk(yb[m], yb[m + 1]), u)));
                PV f = Two<T>::mul(g6, yy);
                f = Two<T>::fma(cA2, Two<T>::sub(va, u), f);
                f = Two<T>::fma(cB2, Two<T>::sub(vb, u), f);
                d[m] = Two<T>::x(f);
                d[m + 1] = Two<T>::y(f);
                PV wv = Two<T>::sub(vb, va);
                if constexpr (ST2) wv = Two<T>::fma(xw2, Two<T>::mk(xx[m], xx[m + 1]), wv);
                wd[m] = Two<T>::x(wv);
                wd[m + 1] = Two<T>::y(wv);
            }
        }
    }
    const T f1_0 = d[0];  // the v and y parts at the lane's first node (r = 0 face; FOLD: times dt)
    // Neighbours across lanes by shuffles: U and wd at the chunk's ends.
    const T uc_prev = __shfl_up_sync(0xffffffffu, uc[M - 1], 1, S);
    const T uc_next = __shfl_down_sync(0xffffffffu, uc[0], 1, S);
    const T wd_prev = __shfl_up_sync(0xffffffffu, wd[M - 1], 1, S);
    const T wd_next = __shfl_down_sync(0xffffffffu, wd[0], 1, S);
    {
        // shifted pairs sh = (U_{m-1}, U_m), tw = (wd_{m-1}, wd_m), rolled
        PV shc = Two<T>::mk(uc_prev, uc[0]);
        PV twc = Two<T>::mk(wd_prev, wd[0]);
        T dlast = uc[0] - uc_prev;  // FP64: U_m - U_{m-1} of the pair's first node, from the previous pair
        const PV v2 = Two<T>::splat(v), nv2 = Two<T>::splat(-v), aFy2 = Two<T>::splat(aFy);
        const PV vq2 = Two<T>::splat(vq), dt2 = Two<T>::splat(dt);
#pragma unroll
        for (int m0 = 0; m0 < M; m0 += W) {
            T tR[W], tIJ[W], tC1[W], tC4V[W], tC4B[W], tC3[W];
            TABV(RT_R, m0, tR);
            TABV(RT_IJ, m0, tIJ);
            TABV(RT_C1, m0, tC1);
            TABV(RT_C4V, m0, tC4V);
            TABV(RT_C4B, m0, tC4B);
            TABV(RT_C3, m0, tC3);
#pragma unroll
            for (int q = 0; q < W; q += 2) {
                const int m = m0 + q, h = m / 2;
                PV shn, twn;
                if (h + 1 < H) {
                    shn = Two<T>::mk(uc[m + 1], uc[m + 2]);
                    twn = Two<T>::mk(wd[m + 1], wd[m + 2]);
                } else {
                    shn = Two<T>::mk(uc[M - 1], uc_next);
                    twn = Two<T>::mk(wd[M - 1], wd_next);
                }
                const PV u = Two<T>::mk(uc[m], uc[m + 1]);
                const PV Dp = Two<T>::sub(shn, u);  // U_{m+1} - U_m
                PV Dm;                              // U_m - U_{m-1}
                if constexpr (sizeof(T) == 8) {     // the previous first differences (scalar FP64)
                    Dm = Two<T>::mk(dlast, Two<T>::x(Dp));
                    dlast = Two<T>::y(Dp);
                } else {                            // one paired instruction
                    Dm = Two<T>::sub(u, shc);
                }
                const PV g1 = Two<T>::mul(Two<T>::mk(tC1[q], tC1[q + 1]), v2);  // zeta_rr / (J^2 h^2)
                const PV g4F = Two<T>::fma(aFy2, Two<T>::mk(tIJ[q], tIJ[q + 1]),
                                           Two<T>::fma(nv2, Two<T>::mk(tC4V[q], tC4V[q + 1]),
                                                       Two<T>::mk(tC4B[q], tC4B[q + 1])));  // g4 / (2h) at t^n
                PV f = Two<T>::fma(g1, Two<T>::sub(Dp, Dm), Two<T>::mul(g4F, Two<T>::add(Dp, Dm)));
                if constexpr (sizeof(T) == 8)  // the reaction fused (FP64: a negated operand is free)
                    f = Two<T>::fma(Two<T>::mk(-tR[q], -tR[q + 1]), u, f);
                else
                    f = Two<T>::sub(f, Two<T>::mul(Two<T>::mk(tR[q], tR[q + 1]), u));
                f = Two<T>::fma(Two<T>::mul(Two<T>::mk(tC3[q], tC3[q + 1]), vq2), Two<T>::sub(twn, twc), f);
                PV r;
                if constexpr (FOLD) {
                    r = Two<T>::fma(dt2, f, Two<T>::mk(d[m], d[m + 1]));
                } else {
                    f = Two<T>::add(f, Two<T>::mk(d[m], d[m + 1]));
                    r = Two<T>::mul(dt2, f);
                }
                if constexpr (ST2) r = Two<T>::fma(xr2, Two<T>::mk(xx[m], xx[m + 1]), r);
                d[m] = Two<T>::x(r);
                d[m + 1] = Two<T>::y(r);
                shc = shn;
                twc = twn;
            }
        }
    }
    const T gLo = I.dir[j], gHi = I.dir[ny + j];
    if (sl == 0) {
        if (I.rlo) {
            d[0] = ST2 ? I.kd * (gLo - uc[0]) : gLo - uc[0];
        } else {
            // gamma > 0: r = 0 face, one-sided first derivative, zeta_rr = 0
            // and no mixed term (Section 7.3).
            const T u = uc[0], u1 = uc[1], u2 = M >= 3 ? uc[M >= 3 ? 2 : 1] : uc_next;
            const T fr = aFy * tl[RT_IJ * S * MP] + tl[RT_C4B * S * MP];  // mu_r / (2 h J) at t^n
            const T f = fr * (T(-3) * u + T(4) * u1 - u2) - tl[RT_R * S * MP] * u;
            d[0] = FOLD ? dt * f + f1_0 : dt * (f + f1_0);
            if constexpr (ST2) {
                if (I.hv) d[0] += xx[0];
            }
        }
    }
    if (e0 + M > nr - 1) {  // only lanes holding r_max or padding
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int e = e0 + m;
            if (e >= nr - 1) d[m] = e == nr - 1 ? (ST2 ? I.kd * (gHi - uc[m]) : gHi - uc[m]) : T(0);
        }
    }

    // 2. rows of I - theta dt A_r(t^{n+1/2}), node pairs as above.
    T a[M], bb[M], c[M];
    {
        const PV aIy2 = Two<T>::splat(aIy), nw2 = Two<T>::splat(-w), w2 = Two<T>::splat(w);
        const PV v2 = Two<T>::splat(v), nv2 = Two<T>::splat(-v);
        const PV one2 = Two<T>::splat(T(1)), two2 = Two<T>::splat(T(2));
#pragma unroll
        for (int m0 = 0; m0 < M; m0 += W) {
            T tR[W], tIJ[W], tC1[W], tC4V[W], tC4B[W];
            TABV(RT_R, m0, tR);
            TABV(RT_IJ, m0, tIJ);
            TABV(RT_C1, m0, tC1);
            TABV(RT_C4V, m0, tC4V);
            TABV(RT_C4B, m0, tC4B);
#pragma unroll
            for (int q = 0; q < W; q += 2) {
                const int m = m0 + q;
                const PV g1 = Two<T>::mul(Two<T>::mk(tC1[q], tC1[q + 1]), v2);
                const PV g4I = Two<T>::fma(aIy2, Two<T>::mk(tIJ[q], tIJ[q + 1]),
                                           Two<T>::fma(nv2, Two<T>::mk(tC4V[q], tC4V[q + 1]),
                                                       Two<T>::mk(tC4B[q], tC4B[q + 1])));
                const PV aa = Two<T>::mul(nw2, Two<T>::sub(g1, g4I));
                const PV bv = Two<T>::fma(w2, Two<T>::fma(two2, g1, Two<T>::mk(tR[q], tR[q + 1])), one2);
                const PV cc = Two<T>::mul(nw2, Two<T>::add(g1, g4I));
                a[m] = Two<T>::x(aa);
                a[m + 1] = Two<T>::y(aa);
                bb[m] = Two<T>::x(bv);
                bb[m + 1] = Two<T>::y(bv);
                c[m] = Two<T>::x(cc);
                c[m + 1] = Two<T>::y(cc);
            }
        }
    }
#undef TABV
    if (sl == 0) {
        if (I.rlo) {
            a[0] = T(0);
            bb[0] = T(1);
            c[0] = T(0);
        } else {
            const T frI = T(2) * (aIy * tl[RT_IJ * S * MP] + tl[RT_C4B * S * MP]);  // mu_r / (h J) at t^{n+1/2}
            a[0] = T(0);
            bb[0] = T(1) + w * (frI + tl[RT_R * S * MP]);
            c[0] = -w * frI;
        }
    }
    if (e0 + M > nr - 1) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            if (e0 + m >= nr - 1) {
                a[m] = T(0);
                bb[m] = T(1);
                c[m] = T(0);
            }
        }
    }
    // 3. solve.
    seg_partition_solve<T, S, M>(a, bb, c, d, sl);
}

// Loads the r tables of instrument b into shared memory (layout P1Layout).
template <typename T, int S, int M>
__device__ __forceinline__ void p1_tables(const March<T>& P, int b, T* tsm)
{
    constexpr int MP = P1Layout<T, M>::MP;
    const int nr = P.nr;
    const T* __restrict__ rt = P.rt + (size_t)b * RT_N * nr;
    for (int idx = threadIdx.x; idx < RT_N * S * M; idx += blockDim.x) {
        const int q = idx / (S * M), e = idx % (S * M);
        tsm[(q * S + e / M) * MP + e % M] = e < nr ? rt[q * nr + e] : T(0);
    }
}

// Neighbour rows of line (k, j): v-a, v-b, y-a, y-b (one-sided on faces).
__device__ __forceinline__ void p1_neighbours(int k, int j, int nv, int ny, int& ka, int& kb, int& ja, int& jb)
{
    const bool vin = k > 0 && k < nv - 1;
    ka = vin ? k - 1 : (k == 0 ? 1 : nv - 2);
    kb = vin ? k + 1 : (k == 0 ? 2 : nv - 3);
    const bool yin = j > 0 && j < ny - 1;
    ja = yin ? j - 1 : (j == 0 ? 1 : ny - 2);
    jb = yin ? j + 1 : (j == 0 ? 2 : ny - 3);
}

// Pass 1, rows from global memory: one CTA = 4 warps = 4 * (32/S) segments;
// each segment processes R lines of one instrument (line index k + n_v j),
// all segments of a warp advancing together so the width-S shuffles always
// see full warps. ST2: the correction stage of the Craig-Sneyd family, which
// also reads the rows of the first stage's result Y. The body of k_pass1 and
// k_pass1_r96 (which differ only in their register budget).
template <typename T, int S, int M, bool ST2>
__device__ __forceinline__ void pass1_rows(const March<T>& P, const T* __restrict__ U, const T* __restrict__ Y,
                                           T* __restrict__ out, const int n, const int R)
{
    constexpr int G = 32 / S;
    constexpr int MP = P1Layout<T, M>::MP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / S, sl = lane % S;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int L = nv * ny;
    const int lpc = 4 * G * R;
    const int bpi = (L + lpc - 1) / lpc;
    const int b = blockIdx.x / bpi, cb = blockIdx.x % bpi;
    const T* __restrict__ Ub = U + (long long)b * P.N;
    const T* __restrict__ Yb = ST2 ? Y + (long long)b * P.N : nullptr;
    T* __restrict__ Ob = out + (long long)b * P.N;
    const P1Inst<T> I = p1_inst<T, ST2>(P, b, n);
    const int e0 = sl * M;
    __shared__ __align__(16) T tsm[RT_N * S * MP];
    p1_tables<T, S, M>(P, b, tsm);
    __syncthreads();
    const T* tl = tsm + sl * MP;
    // 16-byte row access for every row when n_r is a multiple of the vector
    // width and the fields are 16-byte aligned (uniform, checked once).
    const bool vec = nr % (16 / (int)sizeof(T)) == 0 &&
                     ((reinterpret_cast<uintptr_t>(Ub) | reinterpret_cast<uintptr_t>(Ob) |
                       reinterpret_cast<uintptr_t>(Yb)) & 15) == 0;
    // Lines of this segment: line0, line0 + G, ...; (k, j) advanced without
    // divisions. Element offsets within an instrument fit in 32 bits.
    const int line0 = cb * lpc + warp * R * G + seg;
    int k = line0 % nv, j = line0 / nv;
    for (int it = 0; it < R; ++it) {
        const bool valid = line0 + it * G < L;
        const int kk = valid ? k : nv - 1, jj = valid ? j : ny - 1;  // keep addresses in bounds
        int ka, kb, ja, jb;
        p1_neighbours(kk, jj, nv, ny, ka, kb, ja, jb);
        const int off = (jj * nv + kk) * nr;
        T uc[M], ua[M], ub[M], ya[M], yb[M], d[M], xx[M];
        p1_load<T, M>(Ub + off, e0, nr, uc, vec);
        p1_load<T, M>(Ub + off + (ka - kk) * nr, e0, nr, ua, vec);
        p1_load<T, M>(Ub + off + (kb - kk) * nr, e0, nr, ub, vec);
        p1_load<T, M>(Ub + off + (ja - jj) * nv * nr, e0, nr, ya, vec);
        p1_load<T, M>(Ub + off + (jb - jj) * nv * nr, e0, nr, yb, vec);
        if constexpr (ST2) {
            // rows of U + c1 E with E = Y - U, and the extra term xx
            T e[M];
            p1_load<T, M>(Yb + off, e0, nr, e, vec);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                e[m] -= uc[m];
                xx[m] = I.hv ? -e[m] : T(0);
                uc[m] = fma(I.c1, e[m], uc[m]);
            }
            p1_load<T, M>(Yb + off + (ka - kk) * nr, e0, nr, e, vec);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                e[m] -= ua[m];
                if (!I.hv) xx[m] = -I.cx * e[m];
                ua[m] = fma(I.c1, e[m], ua[m]);
            }
            p1_load<T, M>(Yb + off + (kb - kk) * nr, e0, nr, e, vec);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                e[m] -= ub[m];
                if (!I.hv) xx[m] = fma(I.cx, e[m], xx[m]);
                ub[m] = fma(I.c1, e[m], ub[m]);
            }
            p1_load<T, M>(Yb + off + (ja - jj) * nv * nr, e0, nr, e, vec);
#pragma unroll
            for (int m = 0; m < M; ++m) ya[m] = fma(I.c1, e[m] - ya[m], ya[m]);
            p1_load<T, M>(Yb + off + (jb - jj) * nv * nr, e0, nr, e, vec);
#pragma unroll
            for (int m = 0; m < M; ++m) yb[m] = fma(I.c1, e[m] - yb[m], yb[m]);
        }
        p1_line<T, S, M, ST2>(I, tl, sl, kk, jj, uc, ua, ub, ya, yb, xx, d);
        if (valid) p1_store<T, M>(Ob + off, e0, nr, d, vec);
        k += G;
        while (k >= nv) {
            k -= nv;
            ++j;
        }
    }
}

template <typename T, int S, int M, bool ST2>
__global__ void __launch_bounds__(128) k_pass1(const March<T> P, const T* __restrict__ U,
                                               const T* __restrict__ Y, T* __restrict__ out, const int n,
                                               const int R)
{
    pass1_rows<T, S, M, ST2>(P, U, Y, out, n, R);
}

// The FP32 Douglas shapes with 8 nodes per lane, held to 96 registers so 5
// CTAs (5 warps per scheduler) fit on an SM: with the right-hand side in two
// sweeps they need no spills at that budget (measured 3 % faster on 128-node
// lines than at the compiler's 124 registers). The correction-stage variant
// spills there, and the shapes with fewer nodes per lane already fit more
// CTAs; they keep k_pass1.
template <typename T, int S, int M>
__global__ void __launch_bounds__(128, 5) k_pass1_r96(const March<T> P, const T* __restrict__ U,
                                                      T* __restrict__ out, const int n, const int R)
{
    pass1_rows<T, S, M, false>(P, U, nullptr, out, n, R);
}

// Pass 1 with staged planes: a CTA owns a strip of KB = 4 (32/S) RK
// consecutive v nodes and marches over a run of JC y nodes. The rows of the
// strip (plus two v neighbours each side) of y planes j-1, j, j+1 sit in a
// ring of four shared-memory slots; plane j+2 is copied in asynchronously
// (cp.async, 16 bytes per copy) while plane j is computed, so every row of
// U^n crosses L2 about once instead of five times. Rows are stored with the
// 16-byte chunk index XOR-swizzled so that the lanes' vector reads of their
// M-node chunks hit distinct banks. The y-face lines read their second y
// neighbour (a plane outside the ring) from global memory.
template <typename T, int M>
__device__ __forceinline__ int p1s_swz(int c)
{
    constexpr int CPL = (M * (int)sizeof(T)) / 16;  // 16-byte chunks per lane
    if constexpr (CPL >= 2)
        return c ^ ((c >> 3) & (CPL - 1));
    else
        return c;
}

template <typename T, int M>
__device__ __forceinline__ void p1s_row(const T* row, int e0, T (&u)[M])
{
    constexpr int V = 16 / sizeof(T);
    if constexpr (M * sizeof(T) >= 16) {
#pragma unroll
        for (int q = 0; q < M / V; ++q) {
            T x[V];
            lds_vec<T, V>(row + p1s_swz<T, M>(e0 / V + q) * V, x);
#pragma unroll
            for (int t = 0; t < V; ++t) u[q * V + t] = x[t];
        }
    } else {
        lds_vec<T, M>(row + e0, u);
    }
}

// Padded row stride of the ring (elements): whole groups of 8 chunks (the
// swizzle permutes within them) covering both the row and the lanes' reads.
__host__ __device__ inline int p1s_row_stride(int nr, int SM, int V)
{
    const int ch = (nr > SM ? nr : SM) / V + ((nr > SM ? nr : SM) % V != 0);
    return ((ch + 7) & ~7) * V;
}

// Body of k_pass1s and k_pass1s_r96 (which differ only in their register
// budget).
template <typename T, int S, int M>
__device__ __forceinline__ void pass1_staged(const March<T>& P, const T* __restrict__ U, T* __restrict__ out,
                                             const int n, const int RK, const int JC)
{
    constexpr int G = 32 / S;
    constexpr int MP = P1Layout<T, M>::MP;
    constexpr int V = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char p1s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / S, sl = lane % S;
    const int sg = warp * G + seg;  // segment index in the CTA
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int KB = 4 * G * RK;
    const int strips = (nv + KB - 1) / KB, runs = (ny + JC - 1) / JC;
    const int b = blockIdx.x / (strips * runs);
    const int st = (blockIdx.x / runs) % strips, rn = blockIdx.x % runs;
    const int k0 = st * KB, k1 = min(k0 + KB, nv);
    const int klo = max(k0 - 2, 0), khi = min(k1 + 1, nv - 1);
    const int nrows = khi - klo + 1;
    const int j0 = rn * JC, j1 = min(j0 + JC, ny);
    const int CPR = nr / V;  // 16-byte chunks per row
    const int RS = p1s_row_stride(nr, S * M, V);
    const int SLOT = (KB + 4) * RS;              // elements per ring slot
    const T* __restrict__ Ub = U + (long long)b * P.N;
    T* __restrict__ Ob = out + (long long)b * P.N;
    const P1Inst<T> I = p1_inst(P, b, n);
    const int e0 = sl * M;

    T* tsm = reinterpret_cast<T*>(p1s_raw);          // r tables
    T* ring = tsm + ((RT_N * S * MP + V - 1) / V) * V;  // 4 slots
    p1_tables<T, S, M>(P, b, tsm);
    for (int idx = threadIdx.x; idx < 4 * SLOT; idx += blockDim.x) ring[idx] = T(0);  // padding stays 0
    __syncthreads();
    const T* tl = tsm + sl * MP;

    auto load_plane = [&](int jp) {
        if (jp >= 0 && jp < ny && jp <= j1) {
            T* dst = ring + (jp & 3) * SLOT;
            const T* src = Ub + ((long long)jp * nv + klo) * nr;
            for (int c = threadIdx.x; c < nrows * CPR; c += blockDim.x) {
                const int r = c / CPR, ch = c % CPR;
                cp_async16(dst + r * RS + p1s_swz<T, M>(ch) * V, src + (long long)r * nr + ch * V);
            }
        }
        cp_async_commit16();
    };
    load_plane(j0 - 1);
    load_plane(j0);
    load_plane(j0 + 1);
    for (int j = j0; j < j1; ++j) {
        __syncthreads();  // every thread is done with plane j-2's slot
        load_plane(j + 2);
        cp_async_wait16<1>();  // this thread's copies of planes <= j+1 landed
        __syncthreads();       // and everyone's
        const T* pc = ring + (j & 3) * SLOT;
        for (int r = 0; r < RK; ++r) {
            const int kk = k0 + sg + 4 * G * r;
            const bool valid = kk < k1;
            const int k = valid ? kk : k1 - 1;
            int ka, kb, ja, jb;
            p1_neighbours(k, j, nv, ny, ka, kb, ja, jb);
            T uc[M], ua[M], ub[M], ya[M], yb[M], d[M];
            p1s_row<T, M>(pc + (k - klo) * RS, e0, uc);
            p1s_row<T, M>(pc + (ka - klo) * RS, e0, ua);
            p1s_row<T, M>(pc + (kb - klo) * RS, e0, ub);
            // y neighbours: in the ring unless two planes away (y faces)
            if (ja >= j - 1 && ja <= j + 1)
                p1s_row<T, M>(ring + (ja & 3) * SLOT + (k - klo) * RS, e0, ya);
            else
                p1_load<T, M>(Ub + ((long long)ja * nv + k) * nr, e0, nr, ya);
            if (jb >= j - 1 && jb <= j + 1)
                p1s_row<T, M>(ring + (jb & 3) * SLOT + (k - klo) * RS, e0, yb);
            else
                p1_load<T, M>(Ub + ((long long)jb * nv + k) * nr, e0, nr, yb);
            p1_line<T, S, M>(I, tl, sl, k, j, uc, ua, ub, ya, yb, uc, d);
            if (valid) p1_store<T, M>(Ob + ((long long)j * nv + k) * nr, e0, nr, d);
        }
    }
    cp_async_wait16<0>();
}

template <typename T, int S, int M>
__global__ void __launch_bounds__(128, 4) k_pass1s(const March<T> P, const T* __restrict__ U,
                                                T* __restrict__ out, const int n, const int RK, const int JC)
{
    pass1_staged<T, S, M>(P, U, out, n, RK, JC);
}

// The FP32 staged shapes with at most 8 nodes per lane, held to 96 registers
// (5 CTAs per SM) like k_pass1_r96; they fit without spills.
template <typename T, int S, int M>
__global__ void __launch_bounds__(128, 5) k_pass1s_r96(const March<T> P, const T* __restrict__ U,
                                                     T* __restrict__ out, const int n, const int RK,
                                                     const int JC)
{
    pass1_staged<T, S, M>(P, U, out, n, RK, JC);
}

// Pass-1 shapes compiled for each element type: (S, M) with S lanes per r
// line and M nodes per lane.
static bool p1_compiled(size_t elem, int S, int M)
{
    if (elem == 4)
        return (S == 8 && (M == 8 || M == 16)) || (S == 16 && (M == 4 || M == 8 || M == 16)) ||
               (S == 32 && (M == 2 || M == 4 || M == 8 || M == 16));
    return (S == 16 && (M == 2 || M == 4 || M == 8)) || (S == 32 && (M == 2 || M == 4 || M == 8 || M == 16));
}

static constexpr size_t kP1SmemLimit = 227 * 1024;

// Dynamic shared memory of the staged kernel (tables + four ring slots).
static size_t p1s_smem(int nr, int S, int M, int RK, size_t elem)
{
    const int V = (int)(16 / elem);
    const int Wt = (M * (int)elem >= 16) ? V : M;
    (void)Wt;
    const int MP = (M * (int)elem < 16 || (((M * (int)elem) / 16) & 1)) ? M : M + V;
    const size_t tab = (size_t)((RT_N * S * MP + V - 1) / V) * V;
    const int KB = 4 * (32 / S) * RK;
    const size_t slot = (size_t)(KB + 4) * p1s_row_stride(nr, S * M, V);
    return (tab + 4 * slot) * elem;
}

Tile default_tile(int nr, int nv, int ny, size_t elem)
{
    Tile t{32, 16, 4, 1, 1, 0, 0};
    // Heuristic table (the autotuner may replace it per grid shape); FP32
    // strided lines moved by TMA wherever that kernel covers them.
    if (elem == 4) {
        if (nr <= 64) t = {8, 8, 4, 1, 1, 0, 0};
        else if (nr <= 128) t = {16, 8, 4, 1, 1, 0, 0};
        else if (nr <= 256) t = {32, 8, 4, 1, 1, 0, 0};
        if (lines_t_valid(0, nr, nv, ny, elem)) t.p2_P = kLinesTma;
        if (lines_t_valid(1, nr, nv, ny, elem)) t.p3_P = kLinesTma;
    } else {
        if (nr <= 32) t = {16, 2, 4, 1, 1, 0, 0};
        else if (nr <= 64) t = {16, 4, 4, 1, 1, 0, 0};
        else if (nr <= 128) t = {32, 4, 4, 1, 1, 0, 0};
        else if (nr <= 256) t = {32, 8, 4, 1, 1, 0, 0};
    }
    return t;
}

bool tile_valid(const Tile& t, int nr, int nv, int ny, size_t elem)
{
    const bool p2ok = split_valid(nv, t.p2_P) || pass23_valid(nr, nv, ny, t.p2_P, elem) ||
                      (t.p2_P == kLinesTma && lines_t_valid(0, nr, nv, ny, elem));
    const bool p3ok = split_valid(ny, t.p3_P) || (t.p3_P == kLinesTma && lines_t_valid(1, nr, nv, ny, elem));
    if (!p2ok || !p3ok) return false;
    if (t.p1_stage == 2 || t.p1_stage == 3) return pass1t_valid(t, nr, nv, ny, elem);
    if (!p1_compiled(elem, t.p1_S, t.p1_M) || t.p1_S * t.p1_M < nr || t.p1_R < 1 || t.p1_R > 64) return false;
    if (t.p1_stage == 0) return t.p1_J == 0;
    // staged rows are copied in 16-byte pieces
    if ((nr * (int)elem) % 16 != 0) return false;
    if (t.p1_stage != 1 || t.p1_J < 1 || t.p1_J > 4096) return false;
    return p1s_smem(nr, t.p1_S, t.p1_M, t.p1_R, elem) <= kP1SmemLimit;
}

int pass1_chunk(int nr)
{
    return nr <= 512 ? default_tile(nr, 0, 0, 4).p1_M : 0;
}

template <typename T, int S, int M>
static cudaError_t p1_launch(const March<T>& P, const T* U, const T* Y, T* out, int n, const Tile& t,
                             cudaStream_t s)
{
    const bool aligned = ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (Y == nullptr && t.p1_stage == 1 && aligned) {
        const int KB = 4 * (32 / S) * t.p1_R;
        const int strips = (P.nv + KB - 1) / KB, runs = (P.ny + t.p1_J - 1) / t.p1_J;
        const size_t smem = p1s_smem(P.nr, S, M, t.p1_R, sizeof(T));
        const unsigned grid = (unsigned)((long long)P.B * strips * runs);
        if constexpr (sizeof(T) == 4 && M <= 8)
            k_pass1s_r96<T, S, M><<<grid, 128, smem, s>>>(P, U, out, n, t.p1_R, t.p1_J);
        else
            k_pass1s<T, S, M><<<grid, 128, smem, s>>>(P, U, out, n, t.p1_R, t.p1_J);
        return cudaGetLastError();
    }
    const int lpc = 4 * (32 / S) * t.p1_R;
    const int bpi = (P.nv * P.ny + lpc - 1) / lpc;
    if (Y)
        k_pass1<T, S, M, true><<<(unsigned)(bpi * P.B), 128, 0, s>>>(P, U, Y, out, n, t.p1_R);
    else if constexpr (sizeof(T) == 4 && M == 8)
        k_pass1_r96<T, S, M><<<(unsigned)(bpi * P.B), 128, 0, s>>>(P, U, out, n, t.p1_R);
    else
        k_pass1<T, S, M, false><<<(unsigned)(bpi * P.B), 128, 0, s>>>(P, U, nullptr, out, n, t.p1_R);
    return cudaGetLastError();
}

#define P1_SHAPES_F32(X) X(float, 8, 8) X(float, 8, 16) X(float, 16, 4) X(float, 16, 8) X(float, 16, 16) \
    X(float, 32, 2) X(float, 32, 4) X(float, 32, 8) X(float, 32, 16)
#define P1_SHAPES_F64(X) X(double, 16, 2) X(double, 16, 4) X(double, 16, 8) X(double, 32, 2) X(double, 32, 4) \
    X(double, 32, 8) X(double, 32, 16)

// The shared-memory limit of the register-capped staged kernel of a shape
// (only the FP32 shapes with at most 8 nodes per lane have one).
template <typename T, int S, int M>
static cudaError_t p1s_r96_attr()
{
    if constexpr (sizeof(T) == 4 && M <= 8)
        return cudaFuncSetAttribute(k_pass1s_r96<T, S, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kP1SmemLimit);
    else
        return cudaSuccess;
}

// Lets the staged kernels use up to kP1SmemLimit bytes of dynamic shared
// memory (once per device, before launches or captures).
cudaError_t init_pass1()
{
    cudaError_t e = cudaSuccess;
#define P1_ATTR(T_, S_, M_)                                                                                  \
    if (e == cudaSuccess)                                                                                    \
        e = cudaFuncSetAttribute(k_pass1s<T_, S_, M_>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                 (int)kP1SmemLimit);                                                         \
    if (e == cudaSuccess) e = p1s_r96_attr<T_, S_, M_>();                                                   \
                                                         \

    P1_SHAPES_F32(P1_ATTR)
    P1_SHAPES_F64(P1_ATTR)
#undef P1_ATTR
    if (e == cudaSuccess) e = init_pass1t();
    return e;
}

template <typename T>
cudaError_t launch_pass1(const March<T>& P, const T* U, const T* Y, T* out, int n, const Tile& t,
                         cudaStream_t s)
{
    if (!tile_valid(t, P.nr, P.nv, P.ny, sizeof(T))) return cudaErrorInvalidValue;
    if (t.p1_stage == 2 || t.p1_stage == 3) {
        // TMA-fed pass 1; the correction stage of the Craig-Sneyd family and
        // groups with gamma > 0 or theta = 0 run the default rows-from-memory
        // shape instead
        if constexpr (sizeof(T) == 4)
            if (Y == nullptr && P.tma_ok) return launch_pass1t(P, U, out, n, t, s);
        Tile t0 = default_tile(P.nr, P.nv, P.ny, sizeof(T));
        t0.p2_P = t.p2_P;
        t0.p3_P = t.p3_P;
        return launch_pass1<T>(P, U, Y, out, n, t0, s);
    }
    const int S = t.p1_S, M = t.p1_M;
#define P1_CASE(T_, S_, M_) \
    if (S == S_ && M == M_) return p1_launch<T, S_, M_>(P, U, Y, out, n, t, s);
    if constexpr (sizeof(T) == 4) {
        P1_SHAPES_F32(P1_CASE)
    } else {
        P1_SHAPES_F64(P1_CASE)
    }
#undef P1_CASE
    return cudaErrorInvalidValue;
}

template cudaError_t launch_pass1<float>(const March<float>&, const float*, const float*, float*, int,
                                         const Tile&, cudaStream_t);
template cudaError_t launch_pass1<double>(const March<double>&, const double*, const double*, double*, int,
                                          const Tile&, cudaStream_t);

}  // namespace hjm
