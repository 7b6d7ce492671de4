// Pass 1 of a Douglas ADI step (Section 5.1) for FP32 groups whose
// instruments all have gamma = 0 and theta > 0, with the rows of U^n moved
// into shared memory by the Tensor Memory Accelerator. It computes what
// k_pass1 (hjm_pass1.cu) computes,
//   dU0 = dt F(U^n; t^n)  (Eq. (1) in the metric form of Section 4.3, the
//                          centred differences of Section 5, the r-v mixed
//                          term explicit)
//   (I - theta dt A_r(t^{n+1/2})) dU1 = dU0,
// with less work per grid point:
//  - the r factors are recombined per node once per instrument (the R2_
//    tables: dt and 1/theta folded in, Dirichlet nodes as identity rows), so
//    each coefficient of a line is one fused multiply-add of a per-line
//    scalar and a table value, and the system is solved divided by theta;
//  - a CTA owns a strip of consecutive v lines and marches along y; each y
//    plane's strip (plus one halo line on each side) arrives by one
//    cp.async.bulk.tensor box copy issued by one thread into a ring of four
//    shared-memory slots with an mbarrier each, so the SM issues no load
//    instructions for the rows and every row crosses L2 about once;
//  - the tensor is viewed as 32-node chunks (x0, chunk, v, y plane) and the
//    box is 36 nodes wide in x0: the four nodes past each chunk are outside
//    the tensor and arrive as zeros, which pads every 128-byte chunk to 144
//    bytes in shared memory so that the lanes' 16-byte reads of their nodes
//    fall in distinct banks without any address swizzle;
//  - the forward elimination of the partition solve runs inside the
//    right-hand-side sweep, node pair by node pair, so only the eliminated
//    rows stay live, and the interface system is solved by parallel cyclic
//    reduction on rows normalised to a unit diagonal (three shuffles each
//    way per level, one reciprocal per level).
// An r line is owned by S lanes of a warp holding M consecutive nodes each
// (S M a multiple of 32, at least n_r; the nodes past n_r are identity rows
// fed with zeros). Every wait on a plane copy is bounded: a CTA whose wait
// runs out counts itself in a device counter (read by pass1t_timeouts),
// waits a bounded time for its other copies and leaves without writing.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "hjm_kernels.cuh"
#include "hjm_tma.cuh"

namespace hjm {
namespace {

constexpr int kSlots = 4;          // y planes in the ring
constexpr int kChunk = 32;         // nodes per chunk of the tensor view
constexpr int kChunkPad = 36;      // nodes per chunk in shared memory
constexpr int kChunkBytes = kChunkPad * 4;
constexpr unsigned kWaitPolls = 1u << 22;  // polls of a plane's barrier before giving up
constexpr int kPlaneBatch = 64;    // planes whose scalars are formed at once

template <int S, int M>
struct Shape1t {
    static constexpr int G = 32 / S;           // lines side by side in a warp
    static constexpr int BX = S * M;           // nodes per staged row
    static constexpr int NCH = BX / kChunk;    // chunks per staged row
    static constexpr int RSB = NCH * kChunkBytes;  // bytes per staged row
    // table row of a lane padded so that the lanes' 16-byte reads of one
    // table fall in distinct banks (M / 4 odd)
    static constexpr int MP = ((M / 4) & 1) ? M : M + 4;
    static_assert(M % 4 == 0 && BX % kChunk == 0, "whole 16-byte vectors and whole chunks");
};

__device__ unsigned g_p1t_timeouts;   // CTAs that gave up a wait
__device__ int g_p1t_drop = -1;       // test hook: plane never copied
__device__ unsigned g_p1t_limit = kWaitPolls;

__host__ __device__ inline int round128(int x) { return (x + 127) & ~127; }


// ----------------------------------------------------- PTX: TMA, mbarrier

using tma::su32;
using tma::mbar_init;
using tma::fence_barrier_init;
using tma::mbar_expect_tx;
using tma::mbar_try_wait;

// One box (36 x NCH x rows x 1) of the 4-D view into shared memory at dst;
// completion is signalled on bar. c0 is always 0 (16-byte aligned).
__device__ __forceinline__ void tma_box(unsigned dst, const CUtensorMap* tm, int c1, int c2, int c3, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;\n" : "=f"(y) : "f"(x));
    return y;
}

// Paired FP32 arithmetic (one instruction for both components, each rounded
// as its scalar counterpart).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ float4 lds4(const unsigned char* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 lds4f(const float* p) { return *reinterpret_cast<const float4*>(p); }

}  // namespace

namespace {

// Per-plane scalars, stored as pairs (both components equal) so that the
// paired instructions take them without a copy: (a(t^n) + y) / theta,
// a(t^{n+1/2}) + y, dt lambda^2 / (2 h_y J_y theta), -2 kappa y dt /
// (2 h_y J_y theta), the y-face weights yA, yB of the neighbour planes ja,
// jb (A_y U = g6 (yA (U_ja - U) + yB (U_jb - U))), the Dirichlet data (g at
// r_min, g at r_max) and 1/theta.
enum { PJ_AF = 0, PJ_AI = 2, PJ_IJY = 4, PJ_KYY = 6, PJ_YA = 8, PJ_YB = 10, PJ_G = 12, PJ_N = 16 };
// Per-line scalars, as pairs: v, v / theta, -v, -v / theta, 2 v, the weights
// of the v-neighbour rows' second difference (U_a - U) + (U_b - U) and
// difference U_b - U_a, (cA + cB) / 2 and (cB - cA) / 2 times dt / theta
// (cA, cB from the v tables, one-sided on the v faces), and the mixed-term
// weight v / (J_v theta) (0 on the v faces).
enum { LK_V = 0, LK_VT = 2, LK_NV = 4, LK_NVT = 6, LK_TV = 8, LK_CS = 10, LK_CD = 12, LK_VQ = 14, LK_N = 16 };

}  // namespace

namespace {

// Shared-memory bytes of one launch shape: barriers, tables, the scalars of
// kPlaneBatch planes, per-line scalars and the ring.
__host__ __device__ inline int p1t_smem(int S, int M, int RK)
{
    const int G = 32 / S, MP = ((M / 4) & 1) ? M : M + 4, KB = 4 * G * RK;
    const int slot = round128((KB + 2) * (S * M / kChunk) * kChunkBytes);
    // 128 bytes of slack to align the layout to 128 bytes (the box copies'
    // destinations) whatever the dynamic shared memory's base alignment
    return 128 + 128 + round128(R2_N * S * MP * 4) + round128(kPlaneBatch * PJ_N * 4) +
           round128(LK_N * KB * 4) + kSlots * slot;
}

// One r line on an S-lane segment; lane sl holds the line's nodes
// e0 = sl M .. e0 + M - 1 and vo[q] is the byte offset of its q-th 4-node
// vector in a staged row. rc, ra, rb: the staged rows of the line and of its
// v neighbours (one-sided on the v faces) in plane j; pa, pb: the line's rows
// in the y-neighbour planes ja, jb. tl: the lane's folded tables (table t at
// tl + t S MP). lk, pj: the line's and the plane's scalar pairs. YIN: j is
// not a y face (centred y difference). EXACT: n_r = S M, so the r_max node
// is the last lane's last node. Returns dU1 on the lane's nodes in x.
template <int S, int M, bool EXACT, bool YIN>
__device__ __forceinline__ void p1t_line(const float* __restrict__ tl, const unsigned char* rc,
                                         const unsigned char* ra, const unsigned char* rb,
                                         const unsigned char* pa, const unsigned char* pb, const int (&vo)[M / 4],
                                         const float* lk, const float* pj, int sl, int nr, float (&x)[M])
{
    using C = Shape1t<S, M>;
    constexpr int Q = M / 4;
    constexpr int TS = S * C::MP;  // floats per table
    constexpr unsigned FULL = 0xffffffffu;

    // line and plane scalars (pairs)
    const float4 k01 = lds4f(lk), k23 = lds4f(lk + 4), k45 = lds4f(lk + 8), k67 = lds4f(lk + 12);
    const float4 j01 = lds4f(pj), j23 = lds4f(pj + 4), j45 = lds4f(pj + 8), j67 = lds4f(pj + 12);
    const float2 v2 = f2(k01.x, k01.y), vt2 = f2(k01.z, k01.w), nv2 = f2(k23.x, k23.y);
    const float2 nvt2 = f2(k23.z, k23.w), tv2 = f2(k45.x, k45.y), cS2 = f2(k45.z, k45.w);
    const float2 cD2 = f2(k67.x, k67.y), vq2 = f2(k67.z, k67.w);
    const float2 aF2 = f2(j01.x, j01.y), aI2 = f2(j01.z, j01.w);
    const float2 vy2 = mul2(v2, f2(j23.x, j23.y)), ky2 = f2(j23.z, j23.w);
    const float2 yA2 = f2(j45.x, j45.y), yB2 = f2(j45.z, j45.w);
    const float gLo = j67.x, gHi = j67.y;
    const float2 ith2 = f2(j67.z, j67.w);  // 1/theta
    // y drift g6 = (dt lambda^2 v - 2 kappa y dt) / (2 h_y J_y theta): one pair
    // for the whole line (gamma = 0: no r dependence)
    const float2 g6 = add2(vy2, ky2);

    // The line's U^n, and of its v-neighbour rows the second difference
    // (U_a - U) + (U_b - U) and the difference U_b - U_a.
    float uc[M], ws[M], wd[M];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const float4 c = lds4(rc + vo[q]), a = lds4(ra + vo[q]), b = lds4(rb + vo[q]);
        uc[4 * q] = c.x;
        uc[4 * q + 1] = c.y;
        uc[4 * q + 2] = c.z;
        uc[4 * q + 3] = c.w;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 u = h ? f2(c.z, c.w) : f2(c.x, c.y);
            const float2 ua = h ? f2(a.z, a.w) : f2(a.x, a.y), ub = h ? f2(b.z, b.w) : f2(b.x, b.y);
            const float2 s2 = add2(sub2(ua, u), sub2(ub, u)), d2 = sub2(ub, ua);
            ws[4 * q + 2 * h] = s2.x;
            ws[4 * q + 2 * h + 1] = s2.y;
            wd[4 * q + 2 * h] = d2.x;
            wd[4 * q + 2 * h + 1] = d2.y;
        }
    }
    // r neighbours across lanes (at the line's ends the lane's own values:
    // finite, and multiplied by the zero tables of the Dirichlet or padding node)
    const float uL = __shfl_up_sync(FULL, uc[M - 1], 1, S), uR = __shfl_down_sync(FULL, uc[0], 1, S);
    const float wL = __shfl_up_sync(FULL, wd[M - 1], 1, S), wR = __shfl_down_sync(FULL, wd[0], 1, S);
    const float u0 = uc[0], uM = uc[M - 1];
    // first differences e[m] = U_{m+1} - U_m, m = -1 .. M-1 (stored at m + 1)
    float e[M + 1];
    e[0] = uc[0] - uL;
#pragma unroll
    for (int m = 0; m < M - 1; ++m) e[m + 1] = uc[m + 1] - uc[m];
    e[M] = uR - uc[M - 1];

    // Node pairs: the right-hand side dt F / theta and the row of the r
    // system divided by theta, a x_{m-1} + b x_m + c x_{m+1} = d (c = -up),
    // fused with a two-sided elimination of the lane's chunk: rows 1 .. H-1
    // (H = M/2) are eliminated downwards in terms of the chunk's first
    // unknown x_s = x_0,
    //   x_m + C[m] x_{m+1} + A[m] x_s = D[m],
    // rows M-2 .. H upwards in terms of its last unknown x_e = x_{M-1},
    //   x_m + C[m] x_{m-1} + A[m] x_e = D[m],
    // so the two recurrences (each a reciprocal per row) are independent and
    // half as long as one sweep. Pairs are visited from both ends inwards
    // (4-node blocks 0, Q-1, 1, Q-2, ...). Rows 0 and M-1 are kept as they
    // are for the interface equations.
    float A[M], Cc[M], D[M];
    float a0 = 0.f, b0 = 1.f, up0 = 0.f, d0 = 0.f, aN = 0.f, bN = 1.f, upN = 0.f, dN = 0.f;
    constexpr int H = M / 2;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        const int q = (s & 1) ? Q - 1 - (s >> 1) : (s >> 1);  // 0, Q-1, 1, Q-2, ...
        const float* t = tl + 4 * q;
        const float4 tP = lds4f(t + R2_P * TS), tQ = lds4f(t + R2_Q * TS), tB = lds4f(t + R2_B * TS);
        const float4 tE1 = lds4f(t + R2_E1 * TS), tE4 = lds4f(t + R2_E4 * TS), tRT = lds4f(t + R2_RT * TS);
        const float4 ya = lds4(pa + vo[q]), yb = lds4(pb + vo[q]);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            // pairs of a block below H ascend, pairs at or above H descend
            const int h = (4 * q + 2 < H + 1) ? hh : 1 - hh;
            const int m = 4 * q + 2 * h;
#define HJM_PR(v4) (h ? f2(v4.z, v4.w) : f2(v4.x, v4.y))
            const float2 Pp = HJM_PR(tP), E1 = HJM_PR(tE1), E4 = HJM_PR(tE4), Qq = HJM_PR(tQ);
            const float2 u = f2(uc[m], uc[m + 1]);
            // r part: g1 d2U + g4 d1U + RT U
            const float2 d2 = f2(e[m + 1] - e[m], e[m + 2] - e[m + 1]);
            const float2 d1 = f2(e[m + 1] + e[m], e[m + 2] + e[m + 1]);
            const float2 g4 = fma2(nvt2, E4, fma2(aF2, Pp, mul2(ith2, Qq)));
            float2 acc = mul2(HJM_PR(tRT), u);
            acc = fma2(mul2(vt2, E1), d2, acc);
            acc = fma2(g4, d1, acc);
            // v part: cA (U_{v,a} - U) + cB (U_{v,b} - U)
            acc = fma2(cS2, f2(ws[m], ws[m + 1]), acc);
            acc = fma2(cD2, f2(wd[m], wd[m + 1]), acc);
            // mixed r-v term: X vq (wd_{m+1} - wd_{m-1}), X = P SC_XP (in vq)
            const float wm1 = m > 0 ? wd[m - 1] : wL;
            const float wp2 = m + 2 < M ? wd[m + 2] : wR;
            acc = fma2(mul2(Pp, vq2), f2(wd[m + 1] - wm1, wp2 - wd[m]), acc);
            // y part: g6 (yA (U_{y,a} - U) + yB (U_{y,b} - U))
            float2 ty;
            if constexpr (YIN)
                ty = sub2(HJM_PR(yb), HJM_PR(ya));
            else
                ty = fma2(yB2, sub2(HJM_PR(yb), u), mul2(yA2, sub2(HJM_PR(ya), u)));
            acc = fma2(g6, ty, acc);
            // row of the r system at t^{n+1/2}, divided by theta
            const float2 sI = fma2(aI2, Pp, Qq);
            const float2 a = fma2(nv2, add2(E1, E4), sI);   // -lower
            const float2 up = fma2(v2, sub2(E1, E4), sI);   // upper (c = -up)
            const float2 b = fma2(tv2, E1, HJM_PR(tB));   // 1/theta - diag
#undef HJM_PR
#pragma unroll
            for (int zz = 0; zz < 2; ++zz) {
                const int z = m < H ? zz : 1 - zz;  // the bottom recurrence runs upwards
                const int mm = m + z;
                const float az = z ? a.y : a.x, bz = z ? b.y : b.x, uz = z ? up.y : up.x;
                float dz = z ? acc.y : acc.x;
                if constexpr (!EXACT)
                    if (sl * M + mm == nr - 1) dz = gHi - uc[mm];  // Dirichlet row inside the chunk
                if (mm == 0) {
                    a0 = az, b0 = bz, up0 = uz, d0 = dz;
                } else if (mm == M - 1) {
                    aN = az, bN = bz, upN = uz, dN = dz;
                } else if (mm < H) {  // downwards, reference x_s
                    if (mm == 1) {
                        const float r = rcp_approx(bz);
                        Cc[mm] = -uz * r;
                        D[mm] = dz * r;
                        A[mm] = az * r;
                    } else {
                        const float r = rcp_approx(fmaf(-az, Cc[mm - 1], bz));
                        Cc[mm] = -uz * r;
                        D[mm] = r * fmaf(-az, D[mm - 1], dz);
                        A[mm] = -r * (az * A[mm - 1]);
                    }
                } else {  // upwards, reference x_e
                    if (mm == M - 2) {
                        const float r = rcp_approx(bz);
                        Cc[mm] = az * r;
                        D[mm] = dz * r;
                        A[mm] = -uz * r;
                    } else {
                        const float r = rcp_approx(fmaf(uz, Cc[mm + 1], bz));
                        Cc[mm] = az * r;
                        D[mm] = r * fmaf(uz, D[mm + 1], dz);
                        A[mm] = r * (uz * A[mm + 1]);
                    }
                }
            }
        }
    }
    // Dirichlet rows (identity rows from the tables): r_min on the first
    // lane's first node, r_max on node n_r - 1.
    if (sl == 0) d0 = gLo - u0;
    if constexpr (EXACT)
        if (sl == S - 1) dN = gHi - uM;
    // Join the two recurrences at rows H-1 and H, then substitute outwards:
    // every row 1 .. M-2 becomes x_m = D[m] + A[m] x_s + Cc[m] x_e.
    {
        const float rho = rcp_approx(fmaf(-Cc[H], Cc[H - 1], 1.0f));
        const float fH = rho * fmaf(-Cc[H], D[H - 1], D[H]);
        const float gH = rho * (Cc[H] * A[H - 1]);
        const float kH = -rho * A[H];
        const float fL = fmaf(-Cc[H - 1], fH, D[H - 1]);
        const float gL = fmaf(-Cc[H - 1], gH, -A[H - 1]);
        const float kL = -Cc[H - 1] * kH;
        D[H] = fH, A[H] = gH, Cc[H] = kH;
        D[H - 1] = fL, A[H - 1] = gL, Cc[H - 1] = kL;
    }
#pragma unroll
    for (int t = 1; t < H - 1; ++t) {
        const int mt = H - 1 - t, mb = H + t;  // top row going up, bottom row going down
        const float ct = Cc[mt], cb = Cc[mb];
        D[mt] = fmaf(-ct, D[mt + 1], D[mt]);
        A[mt] = fmaf(-ct, A[mt + 1], -A[mt]);
        Cc[mt] = -ct * Cc[mt + 1];
        D[mb] = fmaf(-cb, D[mb - 1], D[mb]);
        const float kb = fmaf(-cb, Cc[mb - 1], -A[mb]);
        A[mb] = -cb * A[mb - 1];
        Cc[mb] = kb;
    }
    // Rows 0 and M-1 in the form of the interface equations:
    //   x_s = dS - aS x_prev - cS x_e,   aE x_s + x_e + cE x_next = dE.
    float aS, cS, dS, aE, cE, dE;
    {
        const float r0 = rcp_approx(fmaf(-up0, A[1], b0));
        dS = r0 * fmaf(up0, D[1], d0);
        aS = r0 * a0;
        cS = -r0 * (up0 * Cc[1]);
        const float rN = rcp_approx(fmaf(aN, Cc[M - 2], bN));
        aE = rN * (aN * A[M - 2]);
        cE = -rN * upN;
        dE = rN * fmaf(-aN, D[M - 2], dN);
    }
    // Interface equations in the lanes' last unknowns x_e, normalised to a
    // unit diagonal, solved by parallel cyclic reduction over width-S
    // shuffles. Lanes without a partner s below (above) have al = 0 (ga = 0)
    // already (the line's first row has no sub-diagonal, its last no
    // super-diagonal, and each level doubles the zeroed span), so the
    // out-of-range shuffles (which return the lane's own finite values) are
    // multiplied by zero.
    float aSn = __shfl_down_sync(FULL, aS, 1, S);
    float cSn = __shfl_down_sync(FULL, cS, 1, S);
    float dSn = __shfl_down_sync(FULL, dS, 1, S);
    if (sl == S - 1) aSn = cSn = dSn = 0.f;
    float al, ga, de;
    {
        const float be = fmaf(-aE, cS, fmaf(-cE, aSn, 1.0f));
        const float r = rcp_approx(be);
        al = -aE * aS * r;
        ga = -cE * cSn * r;
        de = fmaf(-aE, dS, fmaf(-cE, dSn, dE)) * r;
    }
#pragma unroll
    for (int s = 1; s < S; s <<= 1) {
        const float alm = __shfl_up_sync(FULL, al, s, S), gam = __shfl_up_sync(FULL, ga, s, S);
        const float dem = __shfl_up_sync(FULL, de, s, S);
        const float alp = __shfl_down_sync(FULL, al, s, S), gap = __shfl_down_sync(FULL, ga, s, S);
        const float dep = __shfl_down_sync(FULL, de, s, S);
        const float r = rcp_approx(fmaf(-al, gam, fmaf(-ga, alp, 1.0f)));
        const float nde = fmaf(-al, dem, fmaf(-ga, dep, de));
        al = -al * alm * r;
        ga = -ga * gap * r;
        de = nde * r;
    }
    const float xE = de;
    float xEp = __shfl_up_sync(FULL, xE, 1, S);
    if (sl == 0) xEp = 0.f;
    const float xS = fmaf(-aS, xEp, fmaf(-cS, xE, dS));
#pragma unroll
    for (int m = 1; m < M - 1; ++m) x[m] = fmaf(A[m], xS, fmaf(Cc[m], xE, D[m]));
    x[0] = xS;
    x[M - 1] = xE;
}

}  // namespace

namespace {

// Polls the barrier of the copy with sequence number seq (slot seq & 3,
// phase parity (seq >> 2) & 1) at most `limit` times.
__device__ __forceinline__ bool wait_slot(unsigned bar0, unsigned seq)
{
    const unsigned bar = bar0 + 8u * (seq & (kSlots - 1)), par = (seq >> 2) & 1u;
    if (mbar_try_wait(bar, par)) return true;  // the usual case: the copy has landed
    const unsigned limit = g_p1t_limit;
    for (unsigned it = 1; it < limit; ++it)
        if (mbar_try_wait(bar, par)) return true;
    return false;
}

// CTAs per SM the register budget is sized for: lanes of 12 or 16 nodes hold
// more live rows than 128 registers (four CTAs) allow without spills; 8-node
// lanes fit 96 registers (five CTAs).
template <int M>
struct P1tOcc {
    static constexpr int value = M >= 12 ? 3 : 5;
};

// Per-plane scalars of plane j of instrument b at step n (see PJ_).
__device__ __forceinline__ void plane_scalars(const March<float>& P, int b, int n, int j, float* o)
{
    const int ny = P.ny;
    const float* sc = P.sc + (size_t)b * SC_N;
    const float ith = sc[SC_ITH], dth = sc[SC_DT] * ith;
    const float aF = P.st[((size_t)b * P.nsteps + n) * 2], aI = P.st[((size_t)b * P.nsteps + n) * 2 + 1];
    const int yord = P.fl[(size_t)b * FL_N + FL_YORDER];
    const float* yt = P.yt + (size_t)b * YT_N * ny;
    const float* dir = P.dir + ((size_t)b * P.nsteps + n) * 2 * ny;
    const float y = yt[YT_Y * ny + j], iJy = yt[YT_IJ * ny + j], ky = yt[YT_KY * ny + j];
    const bool yin = j > 0 && j < ny - 1;
    const float yA = yin ? -1.f : (yord == 1 ? (j == 0 ? 2.f : -2.f) : (j == 0 ? 4.f : -4.f));
    const float yB = yin ? 1.f : (yord == 1 ? 0.f : (j == 0 ? -1.f : 1.f));
    // the y-drift factor dt lambda^2 (gamma = 0) folded into the v part of g6
    const float v[6] = {(aF + y) * ith, aI + y, sc[SC_YL] * iJy * ith, ky * iJy * dth, yA, yB};
    for (int q = 0; q < 6; ++q) o[2 * q] = o[2 * q + 1] = v[q];
    o[PJ_G] = dir[j];
    o[PJ_G + 1] = dir[ny + j];
    o[PJ_G + 2] = o[PJ_G + 3] = ith;
}

// Work: the units (instrument b, strip of KB = 4 (32/S) RK v lines, y plane
// j), ordered b, strip, j. JC > 0: CTA i takes the run of JC planes
// i mod runs of strip (i / runs) mod strips of instrument i / (strips runs).
// JC = 0 (persistent): the grid is one CTA per resident slot and CTA i takes
// units [T i / grid, T (i + 1) / grid) of the T = B strips n_y units, i.e.
// an equal share (to one plane) marched as runs of constant (b, strip).
// A CTA marches a run along y with the 4-slot ring; its 4 warps' segments
// take lines sg, sg + 4G, ... of the strip for every plane.
template <int S, int M, bool EXACT>
__global__ void __launch_bounds__(128, P1tOcc<M>::value) k_pass1t(const March<float> P,
                                                                   const __grid_constant__ CUtensorMap tm,
                                                                   float* __restrict__ out, const int n,
                                                                   const int RK, const int JC)
{
    using C = Shape1t<S, M>;
    constexpr int G = C::G, MP = C::MP, Q = M / 4;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((128u - (su32(sm_raw) & 127u)) & 127u);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int seg = lane / S, sl = lane % S, sg = warp * G + seg;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int KB = 4 * G * RK;
    const int strips = (nv + KB - 1) / KB;

    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm);
    int* abort_flag = reinterpret_cast<int*>(sm + 64);
    float* tsm = reinterpret_cast<float*>(sm + 128);
    float* pjs = tsm + round128(R2_N * S * MP * 4) / 4;
    float* lks = pjs + round128(kPlaneBatch * PJ_N * 4) / 4;
    unsigned char* ring = reinterpret_cast<unsigned char*>(lks) + round128(LK_N * KB * 4);
    const int slotB = round128((KB + 2) * C::RSB);
    const unsigned bar0 = su32(bar), ring0 = su32(ring);
    const unsigned boxB = (unsigned)((KB + 2) * C::RSB);

    // unit indices fit 32 bits (checked by the launcher)
    int u, uend;
    if (JC > 0) {
        const int runs = (ny + JC - 1) / JC;
        const int b = blockIdx.x / (strips * runs), st = (blockIdx.x / runs) % strips, rn = blockIdx.x % runs;
        u = (b * strips + st) * ny + rn * JC;
        uend = u + min(JC, ny - rn * JC);
    } else {
        const long long T = (long long)P.B * strips * ny;
        u = (int)(T * blockIdx.x / gridDim.x);
        uend = (int)(T * (blockIdx.x + 1) / gridDim.x);
    }
    if (tid == 0) {
        for (int i = 0; i < kSlots; ++i) mbar_init(bar0 + 8u * i, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    int vo[Q];  // the lane's 4-node vectors within a staged row (32-node chunks padded to 36)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int e = sl * M + 4 * q;
        vo[q] = (e >> 5) * kChunkBytes + (e & 31) * 4;
    }
    const float* tl = tsm + sl * MP;
    unsigned seq = 0;    // sequence number of the CTA's next plane copy (slot seq & 3)
    int cur_b = -1, cur_st = -1;
    int jf = 0, last = -1;  // the current run's first plane and last plane copied (thread 0)
    unsigned seq_run = 0;   // sequence number of the current run's first copy

    while (u < uend) {
        const int b = u / (strips * ny), rem = u % (strips * ny);
        const int st = rem / ny, j0 = rem % ny;
        const int j1 = min(ny, j0 + (uend - u));
        const int k0 = st * KB, k1 = min(k0 + KB, nv);
        // Planes in the ring: from the y-1 neighbour of j0 (two planes further
        // back for a run that ends on the y_max face, whose one-sided stencil
        // reaches plane n_y - 3) to the y+1 neighbour of the run's last plane
        // (at least plane 2 for a run starting on the y = 0 face).
        jf = max(0, min(j0 - 1, ny - 3));
        const int jl = min(max(j1, j0 == 0 ? 2 : 0), ny - 1);
        __syncthreads();  // the previous run is done with tables, scalars and slots
        if (b != cur_b) {
            // folded r tables (nodes past n_r: zeros, B = 1, i.e. identity rows)
            const float* __restrict__ r2 = P.r2 + (size_t)b * R2_N * nr;
            for (int idx = tid; idx < R2_N * C::BX; idx += blockDim.x) {
                const int t = idx / C::BX, e = idx % C::BX;
                tsm[(t * S + e / M) * MP + e % M] = e < nr ? r2[t * nr + e] : (t == R2_B ? 1.0f : 0.0f);
            }
        }
        if (b != cur_b || st != cur_st) {
            const float* sc = P.sc + (size_t)b * SC_N;
            const float ith = sc[SC_ITH], dth = sc[SC_DT] * ith, xp = sc[SC_XP];
            const float* vt = P.vt + (size_t)b * VT_N * nv;
            for (int li = tid; li < KB; li += blockDim.x) {
                const int k = min(k0 + li, k1 - 1);
                const float v = vt[VT_V * nv + k], g2 = vt[VT_G2 * nv + k], g5 = vt[VT_G5 * nv + k];
                const float fv = vt[VT_FV * nv + k];
                const bool vin = k > 0 && k < nv - 1;
                const float vq = vin ? v * vt[VT_IJ * nv + k] : 0.f;
                const float cA = vin ? g2 - g5 : (k == 0 ? 4.f * fv : -4.f * fv);
                const float cB = vin ? g2 + g5 : (k == 0 ? -fv : fv);
                // the mixed term's factor X = P SC_XP: SC_XP rides on vq
                const float w[8] = {v, v * ith, -v, -v * ith, 2.f * v, 0.5f * (cA + cB) * dth,
                                    0.5f * (cB - cA) * dth, vq * ith * xp};
                float* o = lks + li * LK_N;
                for (int q = 0; q < 8; ++q) o[2 * q] = o[2 * q + 1] = w[q];
            }
        }
        cur_b = b;
        cur_st = st;
        for (int jj = tid; jj < min(j1 - j0, kPlaneBatch); jj += blockDim.x)
            plane_scalars(P, b, n, j0 + jj, pjs + jj * PJ_N);
        __syncthreads();  // tables and scalars in place

        seq_run = seq;
        auto issue = [&](int p) {
            last = p;
            if (p == g_p1t_drop) return;  // test hook: the copy never starts, its waits run out
            const unsigned sq = seq_run + (unsigned)(p - jf), s = sq & (kSlots - 1);
            mbar_expect_tx(bar0 + 8u * s, boxB);
            tma_box(ring0 + s * (unsigned)slotB, &tm, 0, k0 - 1, b * ny + p, bar0 + 8u * s);
        };
        if (tid == 0)
            for (int p = jf; p <= min(j0 + 1, jl); ++p) issue(p);

        for (int j = j0; j < j1; ++j) {
            __syncthreads();  // every thread is done with plane j-2's slot
            if (*abort_flag) break;
            if (tid == 0 && j + 2 <= jl) issue(j + 2);  // into the slot of plane j-2
            if (j > j0 && (j - j0) % kPlaneBatch == 0) {  // the next batch of plane scalars
                for (int jj = tid; jj < min(j1 - j, kPlaneBatch); jj += blockDim.x)
                    plane_scalars(P, b, n, j + jj, pjs + jj * PJ_N);
                __syncthreads();
            }
            const bool yin = j > 0 && j < ny - 1;
            const int ja = yin ? j - 1 : (j == 0 ? 1 : ny - 2), jb = yin ? j + 1 : (j == 0 ? 2 : ny - 3);
            const unsigned sc_ = seq_run + (unsigned)(j - jf), sa = seq_run + (unsigned)(ja - jf),
                           sb = seq_run + (unsigned)(jb - jf);
            if (!(wait_slot(bar0, sc_) && wait_slot(bar0, sa) && wait_slot(bar0, sb))) {
                atomicExch(abort_flag, 1);
                continue;
            }
            const unsigned char* pc = ring + (sc_ & (kSlots - 1)) * slotB;
            const unsigned char* pa = ring + (sa & (kSlots - 1)) * slotB;
            const unsigned char* pb = ring + (sb & (kSlots - 1)) * slotB;
            const float* pjj = pjs + ((j - j0) % kPlaneBatch) * PJ_N;
            for (int r = 0; r < RK; ++r) {
                const int li = sg + 4 * G * r;
                const bool valid = k0 + li < k1;
                const int k = valid ? k0 + li : k1 - 1;  // segment-uniform; invalid lines are not stored
                const bool vin = k > 0 && k < nv - 1;
                const int ka = vin ? k - 1 : (k == 0 ? 1 : nv - 2), kb = vin ? k + 1 : (k == 0 ? 2 : nv - 3);
                const int rowc = (k - k0 + 1) * C::RSB;
                float xr[M];
                if (yin)
                    p1t_line<S, M, EXACT, true>(tl, pc + rowc, pc + (ka - k0 + 1) * C::RSB,
                                                pc + (kb - k0 + 1) * C::RSB, pa + rowc, pb + rowc, vo,
                                                lks + (k - k0) * LK_N, pjj, sl, nr, xr);
                else
                    p1t_line<S, M, EXACT, false>(tl, pc + rowc, pc + (ka - k0 + 1) * C::RSB,
                                                 pc + (kb - k0 + 1) * C::RSB, pa + rowc, pb + rowc, vo,
                                                 lks + (k - k0) * LK_N, pjj, sl, nr, xr);
                if (valid) {
                    float* o = out + ((size_t)(b * ny + j) * nv + k) * nr + sl * M;
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        if (EXACT || sl * M + 4 * q + 4 <= nr)
                            reinterpret_cast<float4*>(o)[q] =
                                make_float4(xr[4 * q], xr[4 * q + 1], xr[4 * q + 2], xr[4 * q + 3]);
                }
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        seq += (unsigned)(jl - jf + 1);
        u += j1 - j0;
    }
    __syncthreads();  // every thread has left the loops (a late timeout is seen below)
    if (tid == 0 && *abort_flag) {
        // leave no copy in flight into this CTA's shared memory: wait (bounded)
        // for the current run's last planes copied, one per slot
        for (int p = max(jf, last - kSlots + 1); p <= last; ++p)
            if (p != g_p1t_drop) wait_slot(bar0, seq_run + (unsigned)(p - jf));
        atomicAdd(&g_p1t_timeouts, 1u);
    }
    __syncthreads();
}

}  // namespace

// ------------------------------------------------------------------- host

namespace {

using tma::encoder;
using tma::EncodeTiled;

// 4-D view of a group's FP32 field U[b][j][k][i]: (i mod 32, i / 32, k,
// b n_y + j), box (36, chunks, rows, 1) starting at x0 = 0 (16-byte aligned).
cudaError_t field_map(CUtensorMap* m, const float* U, int nr, int nv, long long planes, int chunks, int rows)
{
    const EncodeTiled fn = encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)kChunk, (cuuint64_t)(nr / kChunk), (cuuint64_t)nv, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {(cuuint64_t)kChunk * 4, (cuuint64_t)nr * 4, (cuuint64_t)nr * nv * 4};
    const cuuint32_t box[4] = {(cuuint32_t)kChunkPad, (cuuint32_t)chunks, (cuuint32_t)rows, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(U), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kSmemLimit = 227 * 1024;

// (S, M) shapes compiled: n_r up to 64, 96, 128, 192, 256 and 512.
#define P1T_SHAPES(X) X(4, 16) X(8, 8) X(8, 12) X(8, 16) X(16, 8) X(16, 12) X(16, 16) X(32, 8) X(32, 16)

bool p1t_compiled(int S, int M)
{
#define P1T_IS(S_, M_) if (S == S_ && M == M_) return true;
    P1T_SHAPES(P1T_IS)
#undef P1T_IS
    return false;
}

// Resident CTAs of a kernel at this shared-memory size times the SM count
// of the current device (the persistent grid), cached per kernel.
template <typename K>
int resident_ctas(K kernel, size_t smem)
{
    static std::mutex mu;
    static int dev_cached = -1, sms = 0;
    static std::vector<std::pair<std::pair<const void*, size_t>, int>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (dev != dev_cached) {
        cache.clear();
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        dev_cached = dev;
    }
    const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), smem);
    for (const auto& c : cache)
        if (c.first == key) return c.second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 128, smem) != cudaSuccess) return 0;
    cache.emplace_back(key, nb * sms);
    return nb * sms;
}

template <int S, int M>
cudaError_t p1t_launch(const March<float>& P, const float* U, float* out, int n, const Tile& t, cudaStream_t s)
{
    using C = Shape1t<S, M>;
    const int KB = 4 * C::G * t.p1_R;
    CUtensorMap m;
    cudaError_t e = field_map(&m, U, P.nr, P.nv, (long long)P.B * P.ny, C::NCH, KB + 2);
    if (e != cudaSuccess) return e;
    const int strips = (P.nv + KB - 1) / KB;
    const size_t smem = (size_t)p1t_smem(S, M, t.p1_R);
    const bool exact = P.nr == C::BX;
    auto kern = exact ? k_pass1t<S, M, true> : k_pass1t<S, M, false>;
    long long grid;
    int JC = t.p1_J;
    const long long units = (long long)P.B * strips * P.ny;
    if (units >= (1ll << 31)) return cudaErrorInvalidValue;
    if (t.p1_stage == 3) {  // persistent: one CTA per resident slot, an equal share of the units each
        grid = std::min<long long>(units, resident_ctas(kern, smem));
        JC = 0;
        if (grid < 1) return cudaErrorInvalidConfiguration;
    } else {
        grid = (long long)P.B * strips * ((P.ny + JC - 1) / JC);
    }
    kern<<<(unsigned)grid, 128, smem, s>>>(P, m, out, n, t.p1_R, JC);
    return cudaGetLastError();
}

}  // namespace

bool pass1t_valid(const Tile& t, int nr, int nv, int ny, size_t elem)
{
    if (elem != sizeof(float) || (t.p1_stage != 2 && t.p1_stage != 3) || !p1t_compiled(t.p1_S, t.p1_M))
        return false;
    if (nr % kChunk != 0 || t.p1_S * t.p1_M < nr || nv < 4 || ny < 4) return false;
    if (t.p1_R < 1 || t.p1_R > 8) return false;
    // stage 2: runs of p1_J planes; stage 3: persistent, p1_J = 0
    if (t.p1_stage == 2 ? (t.p1_J < 1 || t.p1_J > 4096) : t.p1_J != 0) return false;
    const int KB = 4 * (32 / t.p1_S) * t.p1_R;
    // the one-sided v stencil of the last line reaches two lines back
    if (nv % KB != 0 && nv % KB < 3) return false;
    if (KB + 2 > 256) return false;
    return p1t_smem(t.p1_S, t.p1_M, t.p1_R) <= kSmemLimit;
}

cudaError_t launch_pass1t(const March<float>& P, const float* U, float* out, int n, const Tile& t, cudaStream_t s)
{
    if (!pass1t_valid(t, P.nr, P.nv, P.ny, sizeof(float)) || !P.tma_ok) return cudaErrorInvalidValue;
    if (((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(out)) & 15) != 0)
        return cudaErrorInvalidValue;
#define P1T_CASE(S_, M_) \
    if (t.p1_S == S_ && t.p1_M == M_) return p1t_launch<S_, M_>(P, U, out, n, t, s);
    P1T_SHAPES(P1T_CASE)
#undef P1T_CASE
    return cudaErrorInvalidValue;
}

cudaError_t init_pass1t()
{
    cudaError_t e = cudaSuccess;
#define P1T_ATTR(S_, M_)                                                                                 \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_pass1t<S_, M_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 kSmemLimit);                                                            \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_pass1t<S_, M_, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 kSmemLimit);
    P1T_SHAPES(P1T_ATTR)
#undef P1T_ATTR
    return e;
}

cudaError_t pass1t_timeouts(unsigned* count, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(count, g_p1t_timeouts, sizeof(unsigned));
    if (e == cudaSuccess && reset) {
        const unsigned z = 0;
        e = cudaMemcpyToSymbol(g_p1t_timeouts, &z, sizeof(unsigned));
    }
    return e;
}

cudaError_t pass1t_test_drop(int plane, unsigned limit)
{
    cudaError_t e = cudaMemcpyToSymbol(g_p1t_drop, &plane, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_p1t_limit, &limit, sizeof(unsigned));
    return e;
}

}  // namespace hjm
