// The three kernel passes of one Douglas ADI step (Section 5.1):
//
//   pass 1  dU0 = dt F(U^n; t^n)           explicit operator, Eq. (1) in the
//                                           metric form of Section 4.3, with
//                                           the r-v mixed term (Section 5)
//           (I - theta dt A_r) dU1 = dU0   fused: one warp per r line
//   pass 2  (I - theta dt A_v) dU2 = dU1   one thread per v line
//   pass 3  (I - theta dt A_y) dU3 = dU2   one thread per y line, fused
//           U^{n+1} = U^n + dU3            with the update
//
// Pass 1 keeps the r line in registers: lane p owns M consecutive nodes, the
// line is solved by a partition method (each lane eliminates its chunk down
// to two interface unknowns, the 32 interface equations are solved by
// parallel cyclic reduction with warp shuffles, then each lane back-
// substitutes). Passes 2 and 3 give each thread one strided line; the line is
// gathered into shared memory with asynchronous copies (one 4- or 8-byte copy
// per node, coalesced across the 32 consecutive r nodes of a warp) and solved
// by the Thomas algorithm (Section 5) in place, with the LU factors of the
// line-invariant systems precomputed by the set-up kernel.
#include "hjm_kernels.cuh"

namespace hjm {

template <typename T>
__device__ __forceinline__ T rcp(T x)
{
    return T(1) / x;
}
template <>
__device__ __forceinline__ float rcp<float>(float x)
{
    return __frcp_rn(x);
}

// ----------------------------------------------------------------- loads

template <typename T, int M>
__device__ __forceinline__ void load_chunk(const T* __restrict__ row, int e0, int nr, T (&u)[M])
{
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
    const bool full = e0 + M <= nr;
    if constexpr (M % V == 0) {
        if (full && (reinterpret_cast<uintptr_t>(row + e0) & 15) == 0) {
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
__device__ __forceinline__ void store_chunk(T* __restrict__ row, int e0, int nr, const T (&u)[M])
{
    constexpr int V = 16 / sizeof(T);
    const bool full = e0 + M <= nr;
    if constexpr (M % V == 0) {
        if (full && (reinterpret_cast<uintptr_t>(row + e0) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < M / V; ++q) {
                if constexpr (sizeof(T) == 4) {
                    reinterpret_cast<float4*>(row + e0)[q] =
                        make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
                } else {
                    reinterpret_cast<double2*>(row + e0)[q] = make_double2(u[2 * q], u[2 * q + 1]);
                }
            }
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m)
        if (e0 + m < nr) row[e0 + m] = u[m];
}

// ------------------------------------------------- partition line solver

// Solves the tridiagonal system whose rows e = lane*M + m are held by the
// warp (a: sub-diagonal, b: diagonal, c: super-diagonal, d: right-hand side;
// a of the first row and c of the last row must be 0, padding rows are
// identity rows). On return d holds the solution.
template <typename T, int M>
__device__ __forceinline__ void warp_partition_solve(T (&a)[M], T (&b)[M], T (&c)[M], T (&d)[M],
                                                     int lane)
{
    static_assert(M >= 2, "chunk of at least two rows");
    // Forward elimination inside the chunk: rows m >= 1 become
    //   a[m] x_s + x_m + c[m] x_{m+1} = d[m]       (x_s: chunk's first node)
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const T r = rcp(b[m]);
        a[m] *= r;
        c[m] *= r;
        d[m] *= r;
    }
#pragma unroll
    for (int m = 2; m < M; ++m) {
        const T r = rcp(b[m] - a[m] * c[m - 1]);
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
        const T r = rcp(T(1) - c[0] * a[1]);
        d[0] = r * (d[0] - c[0] * d[1]);
        a[0] = r * a[0];
        c[0] = -r * c[0] * c[1];
    }
    // Interface system in the chunks' last unknowns x_e: substitute x_s of
    // this chunk and of the next one.
    const T aS = a[0], cS = c[0], dS = d[0];
    const T aE = a[M - 1], cE = c[M - 1], dE = d[M - 1];
    T aSn = __shfl_down_sync(0xffffffffu, aS, 1);
    T cSn = __shfl_down_sync(0xffffffffu, cS, 1);
    T dSn = __shfl_down_sync(0xffffffffu, dS, 1);
    if (lane == 31) aSn = cSn = dSn = T(0);
    T al = -aE * aS;
    T be = T(1) - aE * cS - cE * aSn;
    T ga = -cE * cSn;
    T de = dE - aE * dS - cE * dSn;
    // Parallel cyclic reduction over the 32 lanes.
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        T alm = __shfl_up_sync(0xffffffffu, al, s), bem = __shfl_up_sync(0xffffffffu, be, s);
        T gam = __shfl_up_sync(0xffffffffu, ga, s), dem = __shfl_up_sync(0xffffffffu, de, s);
        T alp = __shfl_down_sync(0xffffffffu, al, s), bep = __shfl_down_sync(0xffffffffu, be, s);
        T gap = __shfl_down_sync(0xffffffffu, ga, s), dep = __shfl_down_sync(0xffffffffu, de, s);
        if (lane < s) {
            alm = T(0);
            bem = T(1);
            gam = T(0);
            dem = T(0);
        }
        if (lane + s >= 32) {
            alp = T(0);
            bep = T(1);
            gap = T(0);
            dep = T(0);
        }
        const T k1 = al * rcp(bem), k2 = ga * rcp(bep);
        const T nbe = be - gam * k1 - alp * k2;
        const T nde = de - dem * k1 - dep * k2;
        al = -alm * k1;
        ga = -gap * k2;
        be = nbe;
        de = nde;
    }
    const T xE = de * rcp(be);
    T xEp = __shfl_up_sync(0xffffffffu, xE, 1);
    if (lane == 0) xEp = T(0);
    const T xS = dS - aS * xEp - cS * xE;
#pragma unroll
    for (int m = 1; m < M - 1; ++m) d[m] = d[m] - a[m] * xS - c[m] * xE;
    d[0] = xS;
    d[M - 1] = xE;
}

// ------------------------------------------------------------------ pass 1

template <typename T, int M>
__global__ void __launch_bounds__(128) k_pass1(const March<T> P, const T* __restrict__ U,
                                               T* __restrict__ out, const int n)
{
    const int lane = threadIdx.x & 31;
    const long long line = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    if (line >= (long long)P.B * nv * ny) return;  // whole warps only
    const int k = (int)(line % nv);
    const int j = (int)((line / nv) % ny);
    const int b = (int)(line / ((long long)nv * ny));

    const T* __restrict__ Ub = U + (long long)b * P.N;
    const T* __restrict__ rt = P.rt + (size_t)b * RT_N * nr;
    const T* __restrict__ vt = P.vt + (size_t)b * VT_N * nv;
    const T* __restrict__ yt = P.yt + (size_t)b * YT_N * ny;
    const T* __restrict__ sc = P.sc + (size_t)b * SC_N;
    const int* __restrict__ fl = P.fl + (size_t)b * FL_N;
    const T dt = sc[SC_DT], w = sc[SC_W], ihr = sc[SC_IHR], ihv = sc[SC_IHV], ihy = sc[SC_IHY];
    const T hihr = T(0.5) * ihr, hihv = T(0.5) * ihv, hihy = T(0.5) * ihy, ihr2 = ihr * ihr,
            ihv2 = ihv * ihv;
    const T aF = P.st[((size_t)b * P.nsteps + n) * 2];
    const T aI = P.st[((size_t)b * P.nsteps + n) * 2 + 1];
    const int rlo = fl[FL_RLO_DIR], yord = fl[FL_YORDER];
    const T v = vt[VT_V * nv + k], iJv = vt[VT_IJ * nv + k], g2 = vt[VT_G2 * nv + k],
            g5 = vt[VT_G5 * nv + k], fv = vt[VT_FV * nv + k];
    const T y = yt[YT_Y * ny + j], iJy = yt[YT_IJ * ny + j], ky = yt[YT_KY * ny + j];
    const T* dir = P.dir + (((size_t)b * P.nsteps + n) * 2) * ny;
    const T gLo = dir[j], gHi = dir[ny + j];

    const bool vin = k > 0 && k < nv - 1;
    const int ka = vin ? k - 1 : (k == 0 ? 1 : nv - 2);
    const int kb = vin ? k + 1 : (k == 0 ? 2 : nv - 3);
    const bool yin = j > 0 && j < ny - 1;
    const int ja = yin ? j - 1 : (j == 0 ? 1 : ny - 2);
    const int jb = yin ? j + 1 : (j == 0 ? 2 : ny - 3);
    const int e0 = lane * M;

    T uc[M], ua[M], ub[M], d[M];
    load_chunk<T, M>(Ub + ((long long)j * nv + k) * nr, e0, nr, uc);
    load_chunk<T, M>(Ub + ((long long)j * nv + ka) * nr, e0, nr, ua);
    load_chunk<T, M>(Ub + ((long long)j * nv + kb) * nr, e0, nr, ub);
    const T uc_prev = __shfl_up_sync(0xffffffffu, uc[M - 1], 1);
    const T uc_next = __shfl_down_sync(0xffffffffu, uc[0], 1);
    const T ua_prev = __shfl_up_sync(0xffffffffu, ua[M - 1], 1);
    const T ua_next = __shfl_down_sync(0xffffffffu, ua[0], 1);
    const T ub_prev = __shfl_up_sync(0xffffffffu, ub[M - 1], 1);
    const T ub_next = __shfl_down_sync(0xffffffffu, ub[0], 1);

    // r, v and mixed parts of F.
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int e = e0 + m;
        const int ec = e < nr ? e : nr - 1;
        const T u = uc[m];
        const T um = m > 0 ? uc[m - 1] : uc_prev;
        const T up = m < M - 1 ? uc[m + 1] : uc_next;
        const T re = rt[RT_R * nr + ec], iJr = rt[RT_IJ * nr + ec];
        const T c4b = rt[RT_C4B * nr + ec];
        const bool rint = e > 0 && e < nr - 1;
        T Ar;
        if (rint) {
            const T g1 = rt[RT_C1 * nr + ec] * v;
            const T g4 = (aF + y) * iJr + c4b - v * rt[RT_C4V * nr + ec];
            Ar = g1 * (up - T(2) * u + um) * ihr2 + g4 * (up - um) * hihr;
        } else {
            // r = 0 face (gamma > 0): one-sided, zeta_rr vanishes there.
            const T u2 = M >= 3 ? uc[m + 2 < M ? m + 2 : M - 1] : uc_next;
            Ar = ((aF + y) * iJr + c4b) * (T(-3) * u + T(4) * up - u2) * hihr;
        }
        Ar -= re * u;
        T Av;
        if (vin)
            Av = g2 * (ub[m] - T(2) * u + ua[m]) * ihv2 + g5 * (ub[m] - ua[m]) * hihv;
        else if (k == 0)
            Av = fv * (T(-3) * u + T(4) * ua[m] - ub[m]) * hihv;
        else
            Av = fv * (T(3) * u - T(4) * ua[m] + ub[m]) * hihv;
        T A0 = T(0);
        if (vin && rint) {
            const T bp = m < M - 1 ? ub[m + 1] : ub_next, bm = m > 0 ? ub[m - 1] : ub_prev;
            const T ap = m < M - 1 ? ua[m + 1] : ua_next, am = m > 0 ? ua[m - 1] : ua_prev;
            A0 = rt[RT_C3 * nr + ec] * v * iJv * (bp - bm - ap + am) * (T(0.25) * ihr * ihv);
        }
        d[m] = Ar + Av + A0;
    }
    // y part of F (pure convection), then dt, then the Dirichlet rows.
    load_chunk<T, M>(Ub + ((long long)ja * nv + k) * nr, e0, nr, ua);
    load_chunk<T, M>(Ub + ((long long)jb * nv + k) * nr, e0, nr, ub);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int e = e0 + m;
        const int ec = e < nr ? e : nr - 1;
        const T u = uc[m];
        const T g6 = (rt[RT_CY * nr + ec] * v + ky) * iJy;
        T Ay;
        if (yin)
            Ay = g6 * (ub[m] - ua[m]) * hihy;
        else if (j == 0)
            Ay = yord == 1 ? g6 * (ua[m] - u) * ihy : g6 * (T(-3) * u + T(4) * ua[m] - ub[m]) * hihy;
        else
            Ay = yord == 1 ? g6 * (u - ua[m]) * ihy : g6 * (T(3) * u - T(4) * ua[m] + ub[m]) * hihy;
        T dv = dt * (d[m] + Ay);
        if (e == nr - 1) dv = gHi - u;
        if (e == 0 && rlo) dv = gLo - u;
        if (e >= nr) dv = T(0);
        d[m] = dv;
    }
    // Rows of I - theta dt A_r(t^{n+1/2}).
    T a[M], bb[M], c[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int e = e0 + m;
        const int ec = e < nr ? e : nr - 1;
        a[m] = T(0);
        bb[m] = T(1);
        c[m] = T(0);
        if (e >= nr || e == nr - 1 || (e == 0 && rlo)) continue;
        const T re = rt[RT_R * nr + ec], iJr = rt[RT_IJ * nr + ec], c4b = rt[RT_C4B * nr + ec];
        T lo = T(0), di, upc;
        if (e > 0) {
            const T g1 = rt[RT_C1 * nr + ec] * v;
            const T g4 = (aI + y) * iJr + c4b - v * rt[RT_C4V * nr + ec];
            lo = g1 * ihr2 - g4 * hihr;
            di = T(-2) * g1 * ihr2;
            upc = g1 * ihr2 + g4 * hihr;
        } else {
            const T fr = ((aI + y) * iJr + c4b) * ihr;
            di = -fr;
            upc = fr;
        }
        di -= re;
        a[m] = -w * lo;
        bb[m] = T(1) - w * di;
        c[m] = -w * upc;
    }
    warp_partition_solve<T, M>(a, bb, c, d, lane);
    store_chunk<T, M>(out + (long long)b * P.N + ((long long)j * nv + k) * nr, e0, nr, d);
}

// ---------------------------------------------------------- async gather

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ------------------------------------------------------------------ pass 2

template <typename T>
__global__ void __launch_bounds__(32) k_pass2(const March<T> P, const T* in, T* out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* col = reinterpret_cast<T*>(smem_raw);
    const int lane = threadIdx.x;
    const int nr = P.nr, nv = P.nv;
    const int tiles = (nr + 31) / 32;
    const long long blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int j = (int)((blk / tiles) % P.ny);
    const int b = (int)(blk / ((long long)tiles * P.ny));
    const int i = it * 32 + lane;
    if (i >= nr) return;
    const long long base = (long long)b * P.N + (long long)j * nv * nr + i;
    const T* src = in + base;
    T* dst = out + base;
    const int* fl = P.fl + (size_t)b * FL_N;
    if (i == nr - 1 || (i == 0 && fl[FL_RLO_DIR])) {  // Dirichlet line: identity system
        if (src != dst)
            for (int kk = 0; kk < nv; ++kk) dst[(long long)kk * nr] = src[(long long)kk * nr];
        return;
    }
    for (int kk = 0; kk < nv; ++kk) cp_async_elem(&col[kk * 32 + lane], src + (long long)kk * nr);
    cp_async_wait_all();
    const T* __restrict__ sub = P.vf + (size_t)b * 3 * nv;
    const T* __restrict__ cpr = sub + nv;
    const T* __restrict__ im = cpr + nv;
    T dp = col[lane] * __ldg(im);
    col[lane] = dp;
    for (int kk = 1; kk < nv; ++kk) {
        dp = (col[kk * 32 + lane] - __ldg(sub + kk) * dp) * __ldg(im + kk);
        col[kk * 32 + lane] = dp;
    }
    T x = dp;
    dst[(long long)(nv - 1) * nr] = x;
    for (int kk = nv - 2; kk >= 0; --kk) {
        x = col[kk * 32 + lane] - __ldg(cpr + kk) * x;
        dst[(long long)kk * nr] = x;
    }
}

// ------------------------------------------------------------------ pass 3

template <typename T>
__global__ void __launch_bounds__(32) k_pass3(const March<T> P, const T* in, const T* Un, T* out,
                                              const int gpos_smem)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    T* col = reinterpret_cast<T*>(smem_raw);  // dU2, then d', then x
    T* ucol = col + (size_t)ny * 32;          // U^n
    T* ccol = ucol + (size_t)ny * 32;         // c' (gamma > 0 only)
    const int tiles = (nr + 31) / 32;
    const long long blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int k = (int)((blk / tiles) % nv);
    const int b = (int)(blk / ((long long)tiles * nv));
    const int i = it * 32 + lane;
    if (i >= nr) return;
    const long long stride = (long long)nr * nv;
    const long long base = (long long)b * P.N + (long long)k * nr + i;
    const T* src = in + base;
    const T* usrc = Un + base;
    T* dst = out + base;
    const int* fl = P.fl + (size_t)b * FL_N;
    for (int jj = 0; jj < ny; ++jj) {
        cp_async_elem(&col[jj * 32 + lane], src + jj * stride);
        cp_async_elem(&ucol[jj * 32 + lane], usrc + jj * stride);
    }
    cp_async_wait_all();
    if (i == nr - 1 || (i == 0 && fl[FL_RLO_DIR])) {  // Dirichlet line: identity system
        for (int jj = 0; jj < ny; ++jj) dst[jj * stride] = ucol[jj * 32 + lane] + col[jj * 32 + lane];
        return;
    }
    if (fl[FL_YLU]) {
        const T* __restrict__ sub = P.yf + ((size_t)b * nv + k) * 3 * ny;
        const T* __restrict__ cpr = sub + ny;
        const T* __restrict__ im = cpr + ny;
        T dp = col[lane] * __ldg(im);
        col[lane] = dp;
        for (int jj = 1; jj < ny; ++jj) {
            dp = (col[jj * 32 + lane] - __ldg(sub + jj) * dp) * __ldg(im + jj);
            col[jj * 32 + lane] = dp;
        }
        T x = dp;
        dst[(ny - 1) * stride] = ucol[(ny - 1) * 32 + lane] + x;
        for (int jj = ny - 2; jj >= 0; --jj) {
            x = col[jj * 32 + lane] - __ldg(cpr + jj) * x;
            dst[jj * stride] = ucol[jj * 32 + lane] + x;
        }
        return;
    }
    if (!gpos_smem) return;  // host guarantees the c' column exists here
    // gamma > 0: the y line's coefficients depend on r too; factor on the fly.
    const T* __restrict__ yt = P.yt + (size_t)b * YT_N * ny;
    const T w = P.sc[(size_t)b * SC_N + SC_W], ihy = P.sc[(size_t)b * SC_N + SC_IHY];
    const T q = P.rt[(size_t)b * RT_N * nr + RT_CY * nr + i] * P.vt[(size_t)b * VT_N * nv + VT_V * nv + k];
    T cprev = T(0), dp = T(0);
    for (int jj = 0; jj < ny; ++jj) {
        const T g6 = (q + yt[YT_KY * ny + jj]) * yt[YT_IJ * ny + jj];
        T lo = T(0), di = T(0), up = T(0);
        if (jj > 0 && jj < ny - 1) {
            lo = T(-0.5) * g6 * ihy;
            up = T(0.5) * g6 * ihy;
        } else if (jj == 0) {
            di = -g6 * ihy;
            up = g6 * ihy;
        } else {
            lo = -g6 * ihy;
            di = g6 * ihy;
        }
        const T s = -w * lo, mn = T(1) - w * di, sp = -w * up;
        const T r = T(1) / (mn - s * cprev);
        cprev = sp * r;
        dp = (col[jj * 32 + lane] - s * dp) * r;
        col[jj * 32 + lane] = dp;
        ccol[jj * 32 + lane] = cprev;
    }
    T x = dp;
    dst[(ny - 1) * stride] = ucol[(ny - 1) * 32 + lane] + x;
    for (int jj = ny - 2; jj >= 0; --jj) {
        x = col[jj * 32 + lane] - ccol[jj * 32 + lane] * x;
        dst[jj * stride] = ucol[jj * 32 + lane] + x;
    }
}

// ------------------------------------------------------------- launchers

int pass1_chunk(int nr)
{
    const int per_lane = (nr + 31) / 32;
    if (per_lane <= 2) return 2;
    if (per_lane <= 4) return 4;
    if (per_lane <= 8) return 8;
    if (per_lane <= 16) return 16;
    return 0;
}

static const size_t kSmemLimit = 227 * 1024;

int max_strided_len(size_t elem, bool gamma_pos)
{
    const size_t cols = gamma_pos ? 3 : 2;  // pass 3 is the larger of the two
    return (int)(kSmemLimit / (cols * 32 * elem));
}

// Lets the strided-line kernels use up to kSmemLimit bytes of dynamic shared
// memory. Called once per device before any launch or stream capture.
cudaError_t init_kernels()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_pass2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    if ((e = cudaFuncSetAttribute(k_pass2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    if ((e = cudaFuncSetAttribute(k_pass3<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    return cudaFuncSetAttribute(k_pass3<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
}

template <typename T>
cudaError_t launch_pass1(const March<T>& P, const T* U, T* out, int n, cudaStream_t s)
{
    const long long lines = (long long)P.B * P.nv * P.ny;
    const unsigned blocks = (unsigned)((lines + 3) / 4);
    switch (pass1_chunk(P.nr)) {
    case 2: k_pass1<T, 2><<<blocks, 128, 0, s>>>(P, U, out, n); break;
    case 4: k_pass1<T, 4><<<blocks, 128, 0, s>>>(P, U, out, n); break;
    case 8: k_pass1<T, 8><<<blocks, 128, 0, s>>>(P, U, out, n); break;
    case 16: k_pass1<T, 16><<<blocks, 128, 0, s>>>(P, U, out, n); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass2(const March<T>& P, const T* in, T* out, cudaStream_t s)
{
    const size_t smem = (size_t)P.nv * 32 * sizeof(T);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    const long long tiles = (long long)P.B * P.ny * ((P.nr + 31) / 32);
    k_pass2<T><<<(unsigned)tiles, 32, smem, s>>>(P, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass3(const March<T>& P, const T* in, const T* Un, T* out, bool any_gamma_pos,
                         cudaStream_t s)
{
    const size_t smem = (size_t)P.ny * 32 * sizeof(T) * (any_gamma_pos ? 3 : 2);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    const long long tiles = (long long)P.B * P.nv * ((P.nr + 31) / 32);
    k_pass3<T><<<(unsigned)tiles, 32, smem, s>>>(P, in, Un, out, any_gamma_pos ? 1 : 0);
    return cudaGetLastError();
}

template cudaError_t launch_pass1<float>(const March<float>&, const float*, float*, int, cudaStream_t);
template cudaError_t launch_pass1<double>(const March<double>&, const double*, double*, int, cudaStream_t);
template cudaError_t launch_pass2<float>(const March<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_pass2<double>(const March<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_pass3<float>(const March<float>&, const float*, const float*, float*, bool,
                                         cudaStream_t);
template cudaError_t launch_pass3<double>(const March<double>&, const double*, const double*, double*,
                                          bool, cudaStream_t);

}  // namespace hjm
