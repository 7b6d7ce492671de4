// Passes 2 and 3 of one Douglas ADI step (Section 5.1; pass 1 is in
// hjm_pass1.cu). The three passes are:
//
//   pass 1  dU0 = dt F(U^n; t^n)           explicit operator, Eq. (1) in the
//                                           metric form of Section 4.3, with
//                                           the r-v mixed term (Section 5)
//           (I - theta dt A_r) dU1 = dU0   fused: one warp per r line
//   pass 2  (I - theta dt A_v) dU2 = dU1   one thread per v line
//   pass 3  (I - theta dt A_y) dU3 = dU2   one thread per y line, fused
//           U^{n+1} = U^n + dU3            with the update
//
// Passes 2 and 3 give each thread one strided line; the line is gathered
// into shared memory with asynchronous copies (one 4- or 8-byte copy per
// node, coalesced across the 32 consecutive r nodes of a warp, issued
// all at once, so a warp has its whole tile in flight) and solved by the
// Thomas algorithm (Section 5) in place, with the LU factors of the line-
// invariant systems precomputed by the set-up kernel. Pass 3 gathers U^n the
// same way for the update (measured faster than reading it a few rows ahead
// during the back substitution).
#include "hjm_kernels.cuh"

namespace hjm {

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

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Wait until at most `pending` of this thread's committed groups are in
// flight (the count must be an immediate, hence the switch).
__device__ __forceinline__ void cp_async_wait_pending(int pending)
{
    switch (pending) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
    }
}

// Gathers this thread's strided line (n nodes, `stride` elements apart) into
// its shared-memory column col[kk * 32 + lane] (every copy in flight at
// once) and runs the Thomas forward sweep d'_k = (d_k - sub_k d'_{k-1}) / m_k.
// The column then holds d'; returns d'_{n-1}.
template <typename T>
__device__ __forceinline__ T gather_forward(T* col, int lane, const T* src, long long stride, int n,
                                            const T* __restrict__ sub, const T* __restrict__ im)
{
    for (int kk = 0; kk < n; ++kk) cp_async_elem(&col[kk * 32 + lane], src + kk * stride);
    cp_async_commit();
    cp_async_wait_pending(0);
    T dp = T(0);
    for (int kk = 0; kk < n; ++kk) {
        dp = (col[kk * 32 + lane] - __ldg(sub + kk) * dp) * __ldg(im + kk);
        col[kk * 32 + lane] = dp;
    }
    return dp;
}

// Rounding indicator: the largest |dU3| of step n on the 4 x 4 read-out
// stencil of the y = 0 plane (non-negative floats order like their bits).
template <typename T>
__device__ __forceinline__ void note_increment(const March<T>& P, const int* fl, int b, int i, int k,
                                               int n, T x0)
{
    if (P.acc == nullptr) return;
    const int i0 = fl[FL_RI0], k0 = fl[FL_RK0];
    if (i < i0 || i >= i0 + 4 || k < k0 || k >= k0 + 4) return;
    atomicMax(reinterpret_cast<int*>(P.acc + (size_t)b * P.nsteps + n), __float_as_int(fabsf((float)x0)));
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
    const T* __restrict__ sub = P.vf + (size_t)b * 3 * nv;
    const T* __restrict__ cpr = sub + nv;
    const T* __restrict__ im = cpr + nv;
    T x = gather_forward<T>(col, lane, src, nr, nv, sub, im);
    dst[(long long)(nv - 1) * nr] = x;
    for (int kk = nv - 2; kk >= 0; --kk) {
        x = col[kk * 32 + lane] - __ldg(cpr + kk) * x;
        dst[(long long)kk * nr] = x;
    }
}

// ------------------------------------------------------------------ pass 3

template <typename T>
__global__ void __launch_bounds__(32) k_pass3(const March<T> P, const T* in, const T* Un, T* out,
                                              const int gpos_smem, const int n)
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
    // Both columns in flight at once (U^n is staged too: the update is in
    // place, so it cannot be read from global memory behind the stores).
    for (int jj = 0; jj < ny; ++jj) {
        cp_async_elem(&col[jj * 32 + lane], src + jj * stride);
        cp_async_elem(&ucol[jj * 32 + lane], usrc + jj * stride);
    }
    cp_async_commit();
    cp_async_wait_pending(0);
    if (i == nr - 1 || (i == 0 && fl[FL_RLO_DIR])) {  // Dirichlet line: identity system
        note_increment(P, fl, b, i, k, n, col[lane]);
        for (int jj = 0; jj < ny; ++jj) dst[jj * stride] = ucol[jj * 32 + lane] + col[jj * 32 + lane];
        return;
    }
    if (fl[FL_YLU]) {
        const T* __restrict__ sub = P.yf + ((size_t)b * nv + k) * 3 * ny;
        const T* __restrict__ cpr = sub + ny;
        const T* __restrict__ im = cpr + ny;
        T dp = T(0);
        for (int jj = 0; jj < ny; ++jj) {
            dp = (col[jj * 32 + lane] - __ldg(sub + jj) * dp) * __ldg(im + jj);
            col[jj * 32 + lane] = dp;
        }
        T x = dp;
        dst[(ny - 1) * stride] = ucol[(ny - 1) * 32 + lane] + x;
        for (int jj = ny - 2; jj >= 0; --jj) {
            x = col[jj * 32 + lane] - __ldg(cpr + jj) * x;
            dst[jj * stride] = ucol[jj * 32 + lane] + x;
        }
        note_increment(P, fl, b, i, k, n, x);
        return;
    }
    if (!gpos_smem) return;  // host guarantees the c' column exists here
    // gamma > 0: the y line's coefficients depend on r too; factor on the fly.
    const T* __restrict__ yt = P.yt + (size_t)b * YT_N * ny;
    const T w = P.sc[(size_t)b * SC_N + SC_W];
    const T q = P.rt[(size_t)b * RT_N * nr + RT_CY * nr + i] * P.vt[(size_t)b * VT_N * nv + VT_V * nv + k];
    T cprev = T(0), dp = T(0);
    for (int jj = 0; jj < ny; ++jj) {
        const T g6 = (q + yt[YT_KY * ny + jj]) * yt[YT_IJ * ny + jj];  // mu_y / (2 h_y J_y)
        T lo = T(0), di = T(0), up = T(0);
        if (jj > 0 && jj < ny - 1) {
            lo = -g6;
            up = g6;
        } else if (jj == 0) {
            di = T(-2) * g6;
            up = T(2) * g6;
        } else {
            lo = T(-2) * g6;
            di = T(2) * g6;
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
    note_increment(P, fl, b, i, k, n, x);
}

// ---------------------------------------------------- split line solves

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

// Passes 2 (AXIS 0: v lines) and 3 (AXIS 1: y lines, fused with the update
// U^{n+1} = U^n + dU3) with each line split into P chunks, one warp per
// chunk and one lane per line (32 consecutive r nodes per CTA, so every
// access is a 128-byte row):
//   1. gather the chunk of the right-hand side (and of U^n in pass 3) into
//      shared memory with asynchronous copies, all in flight at once;
//   2. y = A_p^{-1} d in registers with the chunk's precomputed LU;
//   3. publish the chunk's end values of y, barrier, and form the unknowns
//      just before and after the chunk as weighted sums of the published
//      values (weights: the inverse of the reduced system, precomputed);
//   4. x = y - x_before V - x_after W, store.
// Lines whose r node is a Dirichlet face keep the identity system.
template <typename T, int MC, int AXIS>
__global__ void __launch_bounds__(256) k_split_lines(const March<T> P, const T* in, const T* Un, T* out,
                                                     const int step_n)
{
    using T2 = typename Pair<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int n = AXIS == 0 ? nv : ny;
    const int other = AXIS == 0 ? ny : nv;
    const int K = 2 * (Pw - 1);
    T* red = reinterpret_cast<T*>(smem_raw);  // [K][32] reduced right-hand sides
    T* col = red + K * 32;                    // [n][32] right-hand side
    T* ucol = col + n * 32;                   // [n][32] U^n (pass 3)
    const int tiles = (nr + 31) / 32;
    const long long blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int o = (int)((blk / tiles) % other);
    const int b = (int)(blk / ((long long)tiles * other));
    const int i = it * 32 + lane;
    const bool live = i < nr;  // lanes past n_r only join the barrier
    const int ic = live ? i : nr - 1;
    const long long stride = AXIS == 0 ? (long long)nr : (long long)nr * nv;
    const long long base = (long long)b * P.N + (AXIS == 0 ? (long long)o * nv * nr : (long long)o * nr) + ic;
    int s, L;
    part_chunk(n, Pw, c, s, L);
    const T* F = AXIS == 0 ? P.vp + (size_t)b * part_sys_size(nv, kMaxSplit)
                           : P.yp + ((size_t)b * nv + o) * part_sys_size(ny, kMaxSplit);
    const T2* AB = reinterpret_cast<const T2*>(F) + s;          // (sub, 1/pivot)
    const T2* VW = reinterpret_cast<const T2*>(F + 2 * n) + s;  // (V, W)
    const T2* CF = reinterpret_cast<const T2*>(F + 4 * n) + c * K;
    const T* CP = F + 4 * n + 2 * Pw * K + s;

    // 1. gather.
    const T* src = in + base + s * stride;
    for (int m = 0; m < L; ++m) cp_async_elem(&col[(s + m) * 32 + lane], src + m * stride);
    if constexpr (AXIS == 1) {
        const T* usrc = Un + base + s * stride;
        for (int m = 0; m < L; ++m) cp_async_elem(&ucol[(s + m) * 32 + lane], usrc + m * stride);
    }
    cp_async_commit();
    cp_async_wait_pending(0);
    T d[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m)
        if (m < L) d[m] = col[(s + m) * 32 + lane];
    // 2. chunk solve with the local LU.
    {
        const T2 f = __ldg(AB);
        d[0] *= f.y;
    }
#pragma unroll
    for (int m = 1; m < MC; ++m)
        if (m < L) {
            const T2 f = __ldg(AB + m);
            d[m] = (d[m] - f.x * d[m - 1]) * f.y;
        }
    T nxt = T(0), ylast = T(0);
#pragma unroll
    for (int m = MC - 1; m >= 0; --m)
        if (m < L) {
            const T cpm = m < L - 1 ? __ldg(CP + m) : T(0);
            d[m] -= cpm * nxt;
            nxt = d[m];
            if (m == L - 1) ylast = nxt;
        }
    // 3. reduced system across the chunks of each line.
    if (Pw > 1) {
        if (c >= 1) red[(2 * c - 1) * 32 + lane] = d[0];
        if (c + 1 < Pw) red[(2 * c) * 32 + lane] = ylast;
        __syncthreads();
        T xb = T(0), xa = T(0);
        for (int q = 0; q < K; ++q) {
            const T r = red[q * 32 + lane];
            const T2 w = __ldg(CF + q);
            xb += w.x * r;
            xa += w.y * r;
        }
#pragma unroll
        for (int m = 0; m < MC; ++m)
            if (m < L) {
                const T2 f = __ldg(VW + m);
                d[m] -= f.x * xb + f.y * xa;
            }
    }
    if (!live) return;
    const int* fl = P.fl + (size_t)b * FL_N;
    if (i == nr - 1 || (i == 0 && fl[FL_RLO_DIR])) {  // Dirichlet line: identity system
#pragma unroll
        for (int m = 0; m < MC; ++m)
            if (m < L) d[m] = col[(s + m) * 32 + lane];
    }
    if constexpr (AXIS == 1)
        if (c == 0) note_increment(P, fl, b, i, o, step_n, d[0]);  // dU3 at j = 0
    T* dst = out + base + s * stride;
#pragma unroll
    for (int m = 0; m < MC; ++m)
        if (m < L) {
            if constexpr (AXIS == 1)
                dst[m * stride] = ucol[(s + m) * 32 + lane] + d[m];
            else
                dst[m * stride] = d[m];
        }
}

static size_t split_smem(int n, int Pw, int axis, size_t elem)
{
    return (size_t)(2 * (Pw - 1) + n * (axis == 1 ? 2 : 1)) * 32 * elem;
}

template <typename T, int AXIS>
static cudaError_t split_launch(const March<T>& P, const T* in, const T* Un, T* out, int Pw, int step_n,
                                cudaStream_t s)
{
    const int n = AXIS == 0 ? P.nv : P.ny;
    const int other = AXIS == 0 ? P.ny : P.nv;
    const int chunk = (n + Pw - 1) / Pw;
    const long long blocks = (long long)P.B * other * ((P.nr + 31) / 32);
    const size_t smem = split_smem(n, Pw, AXIS, sizeof(T));
    const dim3 grid((unsigned)blocks), block(32 * Pw);
    if (chunk <= 4) k_split_lines<T, 4, AXIS><<<grid, block, smem, s>>>(P, in, Un, out, step_n);
    else if (chunk <= 8) k_split_lines<T, 8, AXIS><<<grid, block, smem, s>>>(P, in, Un, out, step_n);
    else if (chunk <= 16) k_split_lines<T, 16, AXIS><<<grid, block, smem, s>>>(P, in, Un, out, step_n);
    else if (chunk <= 32) k_split_lines<T, 32, AXIS><<<grid, block, smem, s>>>(P, in, Un, out, step_n);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

bool split_valid(int n, int Pw)
{
    return Pw == 1 || ((Pw == 2 || Pw == 4 || Pw == 8) && n >= 2 * Pw && (n + Pw - 1) / Pw <= kMaxChunk &&
                       split_smem(n, Pw, 1, sizeof(double)) <= 227 * 1024);
}

// ------------------------------------------------------- wide line solves

// Copies of 8 or 16 bytes (VL consecutive r nodes) global -> shared.
template <int BYTES>
__device__ __forceinline__ void cp_async_vec(void* smem_dst, const void* gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}

template <typename T, int VL>
struct Lanes {
    T v[VL];
};

template <typename T, int VL>
__device__ __forceinline__ Lanes<T, VL> ld_lanes(const T* p)
{
    Lanes<T, VL> r;
    if constexpr (VL * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 4) {
            const float4 x = *reinterpret_cast<const float4*>(p);
            r.v[0] = x.x;
            r.v[1] = x.y;
            r.v[2] = x.z;
            r.v[3] = x.w;
        } else {
            const double2 x = *reinterpret_cast<const double2*>(p);
            r.v[0] = x.x;
            r.v[1] = x.y;
        }
    } else {
        const float2 x = *reinterpret_cast<const float2*>(p);
        r.v[0] = x.x;
        r.v[1] = x.y;
    }
    return r;
}

template <typename T, int VL>
__device__ __forceinline__ void st_lanes(T* p, const Lanes<T, VL>& r)
{
    if constexpr (VL * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 4)
            *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
        else
            *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
    } else {
        *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
    }
}

// Passes 2 (AXIS 0) and 3 (AXIS 1, gamma = 0 groups) with VL consecutive
// lines per lane (32 VL lines per warp): the lines are gathered with 8- or
// 16-byte asynchronous copies (VL r nodes each, a warp reads 32 VL
// contiguous nodes of a row) into shared memory and solved by Thomas with
// the precomputed LU factors, the VL recurrences of a lane side by side.
// Pass 3 stages U^n the same way. Needs n_r a multiple of VL and 8/16-byte
// aligned fields (checked by the launcher).
template <typename T, int VL, int AXIS>
__global__ void __launch_bounds__(32) k_wide_lines(const March<T> P, const T* in, const T* Un, T* out,
                                                   const int step_n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int n = AXIS == 0 ? nv : ny;
    const int other = AXIS == 0 ? ny : nv;
    T* col = reinterpret_cast<T*>(smem_raw);  // [n][32 VL] right-hand side, then d'
    T* ucol = col + (size_t)n * 32 * VL;      // [n][32 VL] U^n (pass 3)
    const int tiles = (nr + 32 * VL - 1) / (32 * VL);
    const long long blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int o = (int)((blk / tiles) % other);
    const int b = (int)(blk / ((long long)tiles * other));
    const int i0 = (it * 32 + lane) * VL;
    if (i0 >= nr) return;
    const long long stride = AXIS == 0 ? (long long)nr : (long long)nr * nv;
    const long long base = (long long)b * P.N + (AXIS == 0 ? (long long)o * nv * nr : (long long)o * nr) + i0;
    const T* src = in + base;
    T* dst = out + base;
    T* cl = col + lane * VL;
    T* ul = ucol + lane * VL;
    for (int kk = 0; kk < n; ++kk) cp_async_vec<VL * sizeof(T)>(cl + kk * 32 * VL, src + kk * stride);
    if constexpr (AXIS == 1)
        for (int kk = 0; kk < n; ++kk) cp_async_vec<VL * sizeof(T)>(ul + kk * 32 * VL, Un + base + kk * stride);
    cp_async_commit();
    cp_async_wait_pending(0);
    const T* __restrict__ sub = AXIS == 0 ? P.vf + (size_t)b * 3 * nv : P.yf + ((size_t)b * nv + o) * 3 * ny;
    const T* __restrict__ cpr = sub + n;
    const T* __restrict__ im = cpr + n;
    Lanes<T, VL> dp;
#pragma unroll
    for (int c = 0; c < VL; ++c) dp.v[c] = T(0);
    for (int kk = 0; kk < n; ++kk) {
        const T sk = __ldg(sub + kk), ik = __ldg(im + kk);
        Lanes<T, VL> x = ld_lanes<T, VL>(cl + kk * 32 * VL);
#pragma unroll
        for (int c = 0; c < VL; ++c) dp.v[c] = (x.v[c] - sk * dp.v[c]) * ik;
        st_lanes<T, VL>(cl + kk * 32 * VL, dp);
    }
    // Dirichlet lines (r faces) keep the identity system: their components
    // take the right-hand side as it came in.
    const int* fl = P.fl + (size_t)b * FL_N;
    bool dirc[VL];
    bool anyd = false;
#pragma unroll
    for (int c = 0; c < VL; ++c) {
        const int i = i0 + c;
        dirc[c] = i == nr - 1 || (i == 0 && fl[FL_RLO_DIR]);
        anyd = anyd || dirc[c];
    }
    Lanes<T, VL> x = dp;
    for (int kk = n - 1; kk >= 0; --kk) {
        if (kk < n - 1) {
            const T ck = __ldg(cpr + kk);
            const Lanes<T, VL> y = ld_lanes<T, VL>(cl + kk * 32 * VL);
#pragma unroll
            for (int c = 0; c < VL; ++c) x.v[c] = y.v[c] - ck * x.v[c];
        }
        Lanes<T, VL> r = x;
        if (anyd) {
            const Lanes<T, VL> orig = ld_lanes<T, VL>(src + kk * stride);  // read before this lane's store
#pragma unroll
            for (int c = 0; c < VL; ++c)
                if (dirc[c]) r.v[c] = orig.v[c];
        }
        if constexpr (AXIS == 1) {
            const Lanes<T, VL> u = ld_lanes<T, VL>(ul + kk * 32 * VL);
            if (kk == 0)
#pragma unroll
                for (int c = 0; c < VL; ++c) note_increment(P, fl, b, i0 + c, o, step_n, r.v[c]);  // dU3, j = 0
#pragma unroll
            for (int c = 0; c < VL; ++c) r.v[c] += u.v[c];
        }
        st_lanes<T, VL>(dst + kk * stride, r);
    }
}

template <typename T, int AXIS>
static cudaError_t wide_launch(const March<T>& P, const T* in, const T* Un, T* out, int VL, int step_n,
                               cudaStream_t s)
{
    const int n = AXIS == 0 ? P.nv : P.ny;
    const int other = AXIS == 0 ? P.ny : P.nv;
    const long long blocks = (long long)P.B * other * ((P.nr + 32 * VL - 1) / (32 * VL));
    const size_t smem = (size_t)n * 32 * VL * sizeof(T) * (AXIS == 1 ? 2 : 1);
    if (smem > 227 * 1024 || P.nr % VL != 0) return cudaErrorInvalidValue;
    if (VL * sizeof(T) == 16)
        k_wide_lines<T, 16 / sizeof(T), AXIS><<<(unsigned)blocks, 32, smem, s>>>(P, in, Un, out, step_n);
    else if (sizeof(T) == 4 && VL == 2)
        k_wide_lines<T, 2, AXIS><<<(unsigned)blocks, 32, smem, s>>>(P, in, Un, out, step_n);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// Lines per lane of a wide tile value (0: 16-byte lanes, -1: 8-byte lanes,
// FP32 only), 0 when the value does not select the wide kernels.
int wide_lanes(int p, size_t elem)
{
    if (p == 0) return (int)(16 / elem);
    if (p == -1 && elem == 4) return 2;
    return 0;
}

bool wide_valid(int n, int nr, int p, size_t elem)
{
    const int VL = wide_lanes(p, elem);
    return VL > 0 && nr % VL == 0 && (size_t)n * 32 * VL * elem * 2 <= 227 * 1024;
}

// ------------------------------------------------------------- launchers

static const size_t kSmemLimit = 227 * 1024;

int max_strided_len(size_t elem, bool gamma_pos)
{
    const size_t cols = gamma_pos ? 3 : 2;
    return (int)(kSmemLimit / (cols * 32 * elem));
}

// Lets the strided-line kernels use up to kSmemLimit bytes of dynamic shared
// memory. Called once per device before any launch or stream capture.
cudaError_t init_kernels()
{
    cudaError_t e;
    if ((e = init_pass1())) return e;
#define SPLIT_ATTR(T_, MC_, AX_)                                                                             \
    if ((e = cudaFuncSetAttribute(k_split_lines<T_, MC_, AX_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)kSmemLimit)))                                                        \
        return e;
    SPLIT_ATTR(float, 4, 0) SPLIT_ATTR(float, 8, 0) SPLIT_ATTR(float, 16, 0) SPLIT_ATTR(float, 32, 0)
    SPLIT_ATTR(float, 4, 1) SPLIT_ATTR(float, 8, 1) SPLIT_ATTR(float, 16, 1) SPLIT_ATTR(float, 32, 1)
    SPLIT_ATTR(double, 4, 0) SPLIT_ATTR(double, 8, 0) SPLIT_ATTR(double, 16, 0) SPLIT_ATTR(double, 32, 0)
    SPLIT_ATTR(double, 4, 1) SPLIT_ATTR(double, 8, 1) SPLIT_ATTR(double, 16, 1) SPLIT_ATTR(double, 32, 1)
#undef SPLIT_ATTR
#define WIDE_ATTR(T_, VL_, AX_)                                                                              \
    if ((e = cudaFuncSetAttribute(k_wide_lines<T_, VL_, AX_>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                  (int)kSmemLimit)))                                                        \
        return e;
    WIDE_ATTR(float, 4, 0) WIDE_ATTR(float, 4, 1) WIDE_ATTR(float, 2, 0) WIDE_ATTR(float, 2, 1)
    WIDE_ATTR(double, 2, 0) WIDE_ATTR(double, 2, 1)
#undef WIDE_ATTR
    if ((e = cudaFuncSetAttribute(k_pass2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    if ((e = cudaFuncSetAttribute(k_pass2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    if ((e = cudaFuncSetAttribute(k_pass3<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    return cudaFuncSetAttribute(k_pass3<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
}

template <typename T>
cudaError_t launch_pass2(const March<T>& P, const T* in, T* out, cudaStream_t s)
{
    const int vl2 = wide_lanes(P.p2P, sizeof(T));
    if (vl2 > 0 && (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & (vl2 * sizeof(T) - 1)) == 0))
        return wide_launch<T, 0>(P, in, nullptr, out, vl2, 0, s);
    if (P.p2P > 1) {
        if (!split_valid(P.nv, P.p2P)) return cudaErrorInvalidValue;
        return split_launch<T, 0>(P, in, nullptr, out, P.p2P, 0, s);
    }
    const size_t smem = (size_t)P.nv * 32 * sizeof(T);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    const long long tiles = (long long)P.B * P.ny * ((P.nr + 31) / 32);
    k_pass2<T><<<(unsigned)tiles, 32, smem, s>>>(P, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass3(const March<T>& P, const T* in, const T* Un, T* out, bool any_gamma_pos,
                         int n, cudaStream_t s)
{
    // Split and wide y lines need line-invariant y systems (gamma = 0 in the group).
    const int vl3 = wide_lanes(P.p3P, sizeof(T));
    if (vl3 > 0 && !any_gamma_pos &&
        (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(Un) | reinterpret_cast<uintptr_t>(out)) &
          (vl3 * sizeof(T) - 1)) == 0))
        return wide_launch<T, 1>(P, in, Un, out, vl3, n, s);
    if (P.p3P > 1 && !any_gamma_pos) {
        if (!split_valid(P.ny, P.p3P)) return cudaErrorInvalidValue;
        return split_launch<T, 1>(P, in, Un, out, P.p3P, n, s);
    }
    const size_t smem = (size_t)P.ny * 32 * sizeof(T) * (any_gamma_pos ? 3 : 2);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    const long long tiles = (long long)P.B * P.nv * ((P.nr + 31) / 32);
    k_pass3<T><<<(unsigned)tiles, 32, smem, s>>>(P, in, Un, out, any_gamma_pos ? 1 : 0, n);
    return cudaGetLastError();
}

template cudaError_t launch_pass2<float>(const March<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_pass2<double>(const March<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_pass3<float>(const March<float>&, const float*, const float*, float*, bool,
                                         int, cudaStream_t);
template cudaError_t launch_pass3<double>(const March<double>&, const double*, const double*, double*,
                                          bool, int, cudaStream_t);

}  // namespace hjm
