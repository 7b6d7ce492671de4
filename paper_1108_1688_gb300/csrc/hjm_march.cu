// Passes 2 and 3 of one Douglas ADI step (Section 5.1; pass 1 is in
// hjm_pass1.cu). The three passes are:
//
//   pass 1  dU0 = dt F(U^n; t^n)           explicit operator, Eq. (1) in the
//                                           metric form of Section 4.3, with
//                                           the r-v mixed term (Section 5)
//           (I - theta dt A_r) dU1 = dU0   fused: lane segments per r line
//   pass 2  (I - theta dt A_v) dU2 = dU1   strided v lines
//   pass 3  (I - theta dt A_y) dU3 = dU2   strided y lines, fused with
//           U^{n+1} = U^n + dU3            the update
//
// The strided lines run in one of three ways (chosen per grid shape):
//   k_pass2 / k_pass3   one lane per line: the line is gathered into shared
//                       memory with asynchronous copies (coalesced across
//                       the 32 consecutive r nodes of a warp, all in flight
//                       at once) and solved by Thomas (Section 5) with the
//                       precomputed LU factors of the line-invariant systems
//                       (pass 3 stages U^n the same way);
//   k_split_lines       2-8 warps per line, one chunk each, joined through a
//                       precomputed reduced system (spike partition);
//   k_pass23            passes 2 and 3 together on a shared-memory slab of
//                       8 r nodes when its (v, y) plane fits;
//   k_lines_t           one lane per line, 32-line tiles moved in and out by
//                       the Tensor Memory Accelerator (hjm_lines_t.cu).
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
__device__ __forceinline__ T gather_forward(T* col, int lane, const T* src, int stride, int n,
                                            const T* __restrict__ sub, const T* __restrict__ im)
{
    {
        const T* p = src;
        T* c = col + lane;
#pragma unroll 8
        for (int kk = 0; kk < n; ++kk) {
            cp_async_elem(c, p);
            c += 32;
            p += stride;
        }
    }
    cp_async_commit();
    cp_async_wait_pending(0);
    T dp = T(0);
    T* c = col + lane;
#pragma unroll 4
    for (int kk = 0; kk < n; ++kk) {
        dp = (c[kk * 32] - __ldg(sub + kk) * dp) * __ldg(im + kk);
        c[kk * 32] = dp;
    }
    return dp;
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
    const unsigned blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int j = (int)((blk / tiles) % P.ny);
    const int b = (int)(blk / (unsigned)(tiles * P.ny));
    const int i = it * 32 + lane;
    if (i >= nr) return;
    const long long base = (long long)b * P.N + (long long)j * nv * nr + i;
    const T* src = in + base;
    T* dst = out + base;
    const int* fl = P.fl + (size_t)b * FL_N;
    if (i == nr - 1 || (i == 0 && fl[FL_RLO_DIR])) {  // Dirichlet line: identity system
        if (src != dst)
            for (int kk = 0; kk < nv; ++kk) dst[kk * nr] = src[kk * nr];
        return;
    }
    const T* __restrict__ sub = P.vf + (size_t)b * 3 * nv;
    const T* __restrict__ cpr = sub + nv;
    const T* __restrict__ im = cpr + nv;
    T x = gather_forward<T>(col, lane, src, nr, nv, sub, im);
    T* p = dst + (nv - 1) * nr;
    *p = x;
    const T* c = col + lane;
#pragma unroll 4
    for (int kk = nv - 2; kk >= 0; --kk) {
        x = c[kk * 32] - __ldg(cpr + kk) * x;
        p -= nr;
        *p = x;
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
    const unsigned blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int k = (int)((blk / tiles) % nv);
    const int b = (int)(blk / (unsigned)(tiles * nv));
    const int i = it * 32 + lane;
    if (i >= nr) return;
    const int stride = nr * nv;  // element offsets within an instrument fit in 32 bits
    const long long base = (long long)b * P.N + (long long)k * nr + i;
    const T* src = in + base;
    const T* usrc = Un + base;
    T* dst = out + base;
    const int* fl = P.fl + (size_t)b * FL_N;
    // Both columns in flight at once (U^n is staged too: the update is in
    // place, so it cannot be read from global memory behind the stores).
    {
        const T* p = src;
        const T* q = usrc;
        T* c = col + lane;
        T* u = ucol + lane;
#pragma unroll 8
        for (int jj = 0; jj < ny; ++jj) {
            cp_async_elem(c, p);
            cp_async_elem(u, q);
            c += 32;
            u += 32;
            p += stride;
            q += stride;
        }
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
        T* c = col + lane;
        const T* u = ucol + lane;
#pragma unroll 4
        for (int jj = 0; jj < ny; ++jj) {
            dp = (c[jj * 32] - __ldg(sub + jj) * dp) * __ldg(im + jj);
            c[jj * 32] = dp;
        }
        T x = dp;
        T* p = dst + (ny - 1) * stride;
        *p = u[(ny - 1) * 32] + x;
#pragma unroll 4
        for (int jj = ny - 2; jj >= 0; --jj) {
            x = c[jj * 32] - __ldg(cpr + jj) * x;
            p -= stride;
            *p = u[jj * 32] + x;
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
// The per-thread work of k_split_lines on a chunk of L nodes (FULL: L = MC,
// every loop unpredicated). cl / ul point at the chunk's first node of this
// lane's column in shared memory (node stride 32).
template <typename T, int MC, int AXIS, bool FULL>
__device__ __forceinline__ T split_body(const T* src, const T* usrc, T* dst, int stride, T* cl, T* ul, T* red,
                                           int lane, int c, int Pw, int L, const typename Pair<T>::type* AB,
                                           const typename Pair<T>::type* VW, const typename Pair<T>::type* CF,
                                           const T* CP, bool live, bool dirl)
{
    using T2 = typename Pair<T>::type;
    const int K = 2 * (Pw - 1);
    // 1. gather (all copies in flight at once)
    {
        const T* p = src;
#pragma unroll
        for (int m = 0; m < MC; ++m) {
            if (FULL || m < L) cp_async_elem(cl + m * 32, p);
            p += stride;
        }
        if constexpr (AXIS == 1) {
            const T* q = usrc;
#pragma unroll
            for (int m = 0; m < MC; ++m) {
                if (FULL || m < L) cp_async_elem(ul + m * 32, q);
                q += stride;
            }
        }
    }
    cp_async_commit();
    cp_async_wait_pending(0);
    T d[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m)
        if (FULL || m < L) d[m] = cl[m * 32];
    // 2. chunk solve with the local LU
    {
        const T2 f = __ldg(AB);
        d[0] *= f.y;
    }
#pragma unroll
    for (int m = 1; m < MC; ++m)
        if (FULL || m < L) {
            const T2 f = __ldg(AB + m);
            d[m] = (d[m] - f.x * d[m - 1]) * f.y;
        }
    T ylast;
    if constexpr (FULL) {
        ylast = d[MC - 1];
#pragma unroll
        for (int m = MC - 2; m >= 0; --m) d[m] -= __ldg(CP + m) * d[m + 1];
    } else {
        T nxt = T(0);
        ylast = T(0);
#pragma unroll
        for (int m = MC - 1; m >= 0; --m)
            if (m < L) {
                const T cpm = m < L - 1 ? __ldg(CP + m) : T(0);
                d[m] -= cpm * nxt;
                nxt = d[m];
                if (m == L - 1) ylast = nxt;
            }
    }
    // 3. reduced system across the chunks of each line
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
            if (FULL || m < L) {
                const T2 f = __ldg(VW + m);
                d[m] -= f.x * xb + f.y * xa;
            }
    }
    if (!live) return T(0);
    if (dirl) {
#pragma unroll
        for (int m = 0; m < MC; ++m)
            if (FULL || m < L) d[m] = cl[m * 32];
    }
    const T x0 = d[0];  // dU3 at the chunk's first node
    // 4. store (pass 3: U^n + dU3)
    T* p = dst;
#pragma unroll
    for (int m = 0; m < MC; ++m) {
        if (FULL || m < L) {
            if constexpr (AXIS == 1)
                *p = ul[m * 32] + d[m];
            else
                *p = d[m];
        }
        p += stride;
    }
    return x0;
}

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
    const unsigned blk = blockIdx.x;
    const int it = (int)(blk % tiles);
    const int o = (int)((blk / tiles) % other);
    const int b = (int)(blk / (unsigned)(tiles * other));
    const int i = it * 32 + lane;
    const bool live = i < nr;  // lanes past n_r only join the barrier
    const int ic = live ? i : nr - 1;
    const int stride = AXIS == 0 ? nr : nr * nv;  // 32-bit offsets within an instrument
    const long long base = (long long)b * P.N + (AXIS == 0 ? (long long)o * nv * nr : (long long)o * nr) + ic;
    int s, L;
    part_chunk(n, Pw, c, s, L);
    const T* F = AXIS == 0 ? P.vp + (size_t)b * part_sys_size(nv, kMaxSplit)
                           : P.yp + ((size_t)b * nv + o) * part_sys_size(ny, kMaxSplit);
    const T2* AB = reinterpret_cast<const T2*>(F) + s;          // (sub, 1/pivot)
    const T2* VW = reinterpret_cast<const T2*>(F + 2 * n) + s;  // (V, W)
    const T2* CF = reinterpret_cast<const T2*>(F + 4 * n) + c * K;
    const T* CP = F + 4 * n + 2 * Pw * K + s;

    const int* fl = P.fl + (size_t)b * FL_N;
    const bool dirl = i == nr - 1 || (i == 0 && fl[FL_RLO_DIR]);  // Dirichlet line: identity system
    const T* src = in + base + s * stride;
    T* dst = out + base + s * stride;
    const T* usrc = AXIS == 1 ? Un + base + s * stride : nullptr;
    // every chunk holds exactly MC nodes: unpredicated body (uniform in the
    // CTA, which matters for the barrier inside)
    const bool full = n % Pw == 0 && n / Pw == MC;
    T x0;
    if (full)
        x0 = split_body<T, MC, AXIS, true>(src, usrc, dst, stride, col + s * 32 + lane, ucol + s * 32 + lane, red,
                                           lane, c, Pw, MC, AB, VW, CF, CP, live, dirl);
    else
        x0 = split_body<T, MC, AXIS, false>(src, usrc, dst, stride, col + s * 32 + lane, ucol + s * 32 + lane, red,
                                            lane, c, Pw, L, AB, VW, CF, CP, live, dirl);
    if constexpr (AXIS == 1)
        if (live && c == 0) note_increment(P, fl, b, i, o, step_n, x0);  // dU3 at j = 0
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

// ------------------------------------------------- fused passes 2 and 3

template <typename T, int V>
struct Vec16;
template <>
struct Vec16<float, 4> {
    using type = float4;
};
template <>
struct Vec16<double, 2> {
    using type = double2;
};

// 16-byte shared read of V elements.
template <typename T, int V>
__device__ __forceinline__ void lds_pair(const T* p, T (&x)[V])
{
    const typename Vec16<T, V>::type v = *reinterpret_cast<const typename Vec16<T, V>::type*>(p);
    if constexpr (V == 4) {
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    } else {
        x[0] = v.x;
        x[1] = v.y;
    }
}

// 16-byte global store of u + x.
template <typename T, int V>
__device__ __forceinline__ void add_store(T* p, const typename Vec16<T, V>::type& u, const T (&x)[V])
{
    if constexpr (V == 4)
        *reinterpret_cast<float4*>(p) = make_float4(u.x + x[0], u.y + x[1], u.z + x[2], u.w + x[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(u.x + x[0], u.y + x[1]);
}

// Passes 2 and 3 of a step in one kernel when the (v, y) plane of a slab of
// SL = 8 consecutive r nodes (32-byte rows) fits in shared memory (gamma = 0
// groups): the CTA
// gathers dU1 of its slab (16-byte copies, SL r nodes of every (k, j) row),
// solves every v line of the slab in place, then every y line, then writes
// U^{n+1} = U^n + dU3. The same Thomas sweeps with the same factors as the
// separate passes, so the results are the same; dU2 never goes to global
// memory (12 bytes per point instead of 8 + 12).
// Shared layout S[j][k SL + ii], row stride RJ = n_v SL + pad with RJ = SL
// (mod 32): lanes (ii fastest) of a v line sweep or a y line sweep hit
// distinct banks.
template <typename T, int SL>
__global__ void __launch_bounds__(1024) k_pass23(const March<T> P, const T* in, const T* Un, T* out, const int n,
                                                 const int RJ)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte piece
    constexpr int H = SL / V;          // 16-byte pieces per row of the slab
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int slabs = (nr + SL - 1) / SL;
    const int b = blockIdx.x / slabs;
    const int i0 = (blockIdx.x % slabs) * SL;
    const int sw = min(SL, nr - i0);  // live r nodes of this slab
    const long long base = (long long)b * P.N + i0;
    const T* src = in + base;
    const int* fl = P.fl + (size_t)b * FL_N;
    const int rows = nv * ny;
    // Work items are (row, piece); (j, k) of item q = tid + t nth advanced
    // without divisions.
    const int qn = rows * H;
    const int dq = nth / H, dk0 = dq % nv, dj0 = dq / nv;
    // 1. gather dU1 of the slab (a ragged last slab copies element-wise)
    if (sw == SL) {
        int h = tid % H, r = tid / H, k = r % nv, j = r / nv;
        for (int q = tid; q < qn; q += nth) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(S + j * RJ + k * SL + h * V);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src + (j * nv + k) * nr + h * V)
                         : "memory");
            k += dk0;
            j += dj0;
            if (k >= nv) {
                k -= nv;
                ++j;
            }
        }
    } else {
        for (int q = tid; q < rows * SL; q += nth) {
            const int r = q / SL, ii = q % SL;
            if (ii < sw) cp_async_elem(S + (r / nv) * RJ + (r % nv) * SL + ii, src + r * nr + ii);
        }
    }
    cp_async_commit();
    cp_async_wait_pending(0);
    __syncthreads();
    const int rlo = fl[FL_RLO_DIR];
    // 2. v lines (ii, j) and 3. y lines (ii, k): Thomas with the precomputed
    // factors, four nodes loaded ahead of the recurrence.
    auto thomas = [&](T* line, int len, int st, const T* __restrict__ sub, const T* __restrict__ cpr,
                      const T* __restrict__ im) {
        T dp = T(0);
        int k = 0;
        for (; k + 4 <= len; k += 4) {
            const T x0 = line[k * st], x1 = line[(k + 1) * st], x2 = line[(k + 2) * st], x3 = line[(k + 3) * st];
            dp = (x0 - __ldg(sub + k) * dp) * __ldg(im + k);
            line[k * st] = dp;
            dp = (x1 - __ldg(sub + k + 1) * dp) * __ldg(im + k + 1);
            line[(k + 1) * st] = dp;
            dp = (x2 - __ldg(sub + k + 2) * dp) * __ldg(im + k + 2);
            line[(k + 2) * st] = dp;
            dp = (x3 - __ldg(sub + k + 3) * dp) * __ldg(im + k + 3);
            line[(k + 3) * st] = dp;
        }
        for (; k < len; ++k) {
            dp = (line[k * st] - __ldg(sub + k) * dp) * __ldg(im + k);
            line[k * st] = dp;
        }
        T x = dp;
        int m = len - 2;
        for (; m - 3 >= 0; m -= 4) {
            const T y0 = line[m * st], y1 = line[(m - 1) * st], y2 = line[(m - 2) * st], y3 = line[(m - 3) * st];
            x = y0 - __ldg(cpr + m) * x;
            line[m * st] = x;
            x = y1 - __ldg(cpr + m - 1) * x;
            line[(m - 1) * st] = x;
            x = y2 - __ldg(cpr + m - 2) * x;
            line[(m - 2) * st] = x;
            x = y3 - __ldg(cpr + m - 3) * x;
            line[(m - 3) * st] = x;
        }
        for (; m >= 0; --m) {
            x = line[m * st] - __ldg(cpr + m) * x;
            line[m * st] = x;
        }
    };
    {
        const T* sub = P.vf + (size_t)b * 3 * nv;
        for (int q = tid; q < SL * ny; q += nth) {
            const int ii = q % SL, j = q / SL, i = i0 + ii;
            if (ii >= sw || i == nr - 1 || (i == 0 && rlo)) continue;  // Dirichlet lines: identity
            thomas(S + j * RJ + ii, nv, SL, sub, sub + nv, sub + 2 * nv);
        }
    }
    __syncthreads();
    for (int q = tid; q < SL * nv; q += nth) {
        const int ii = q % SL, k = q / SL, i = i0 + ii;
        if (ii >= sw || i == nr - 1 || (i == 0 && rlo)) continue;
        const T* sub = P.yf + ((size_t)b * nv + k) * 3 * ny;
        thomas(S + k * SL + ii, ny, RJ, sub, sub + ny, sub + 2 * ny);
    }
    __syncthreads();
    // 4. U^{n+1} = U^n + dU3 in 16-byte pieces, four loads ahead of the
    // stores (each piece is read before it is written, by the same thread),
    // and the rounding indicator on j = 0.
    const T* ub = Un + base;
    T* ob = out + base;
    if (sw == SL) {
        int h = tid % H, r = tid / H, k = r % nv, j = r / nv;
        for (int q0 = tid; q0 < qn; q0 += 4 * nth) {
            typename Vec16<T, V>::type u[4];
            int jj[4], kk[4], hh[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                jj[t] = j;
                kk[t] = k;
                hh[t] = h;
                if (q0 + t * nth < qn)
                    u[t] = *reinterpret_cast<const typename Vec16<T, V>::type*>(ub + (j * nv + k) * nr + h * V);
                k += dk0;
                j += dj0;
                if (k >= nv) {
                    k -= nv;
                    ++j;
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (q0 + t * nth >= qn) break;
                const T* sp = S + jj[t] * RJ + kk[t] * SL + hh[t] * V;
                T x[V];
                lds_pair<T, V>(sp, x);
                if (jj[t] == 0)
#pragma unroll
                    for (int c = 0; c < V; ++c) note_increment(P, fl, b, i0 + hh[t] * V + c, kk[t], n, x[c]);
                add_store<T, V>(ob + (jj[t] * nv + kk[t]) * nr + hh[t] * V, u[t], x);
            }
        }
    } else {
        for (int q = tid; q < rows * SL; q += nth) {
            const int r = q / SL, ii = q % SL;
            if (ii >= sw) continue;
            const int j = r / nv, k = r % nv;
            const T x = S[j * RJ + k * SL + ii];
            if (j == 0) note_increment(P, fl, b, i0 + ii, k, n, x);
            ob[r * nr + ii] = ub[r * nr + ii] + x;
        }
    }
}

// Row stride (elements) of the fused kernel's shared plane: RJ = SL (mod 32).
static int p23_row_stride(int nv, int SL)
{
    const int base = nv * SL;
    return base + ((SL - base % 32) % 32 + 32) % 32;
}

size_t pass23_smem(int nv, int ny, int SL, size_t elem)
{
    return (size_t)ny * p23_row_stride(nv, SL) * elem;
}

bool pass23_valid(int nr, int nv, int ny, int p2, size_t elem)
{
    constexpr int SL = 8;
    if (p2 != 0 || (nr * (int)elem) % 16 != 0) return false;
    if (SL * (nv > ny ? nv : ny) > 1024 * 8) return false;
    return pass23_smem(nv, ny, SL, elem) <= 227 * 1024;
}

template <typename T>
cudaError_t launch_pass23(const March<T>& P, const T* in, const T* Un, T* out, int n, cudaStream_t s)
{
    constexpr int SL = 8;
    if (!pass23_valid(P.nr, P.nv, P.ny, P.p2P, sizeof(T))) return cudaErrorInvalidValue;
    if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(Un) | reinterpret_cast<uintptr_t>(out)) &
         15) != 0)
        return cudaErrorInvalidValue;
    const int RJ = p23_row_stride(P.nv, SL);
    const size_t smem = pass23_smem(P.nv, P.ny, SL, sizeof(T));
    const int lines = SL * (P.nv > P.ny ? P.nv : P.ny);
    const int threads = lines < 1024 ? ((lines + 31) / 32) * 32 : 1024;
    const unsigned blocks = (unsigned)(P.B * ((P.nr + SL - 1) / SL));
    k_pass23<T, SL><<<blocks, threads, smem, s>>>(P, in, Un, out, n, RJ);
    return cudaGetLastError();
}

// ------------------------------------- MIXED: FP32 increments, FP64 state

// U = hi + lo with hi = fl32(U) and lo = fl32(U - hi): the FP32 march of hi
// sees its neighbour differences exactly (they are FP32 numbers), and the
// march of lo carries the part of the state FP32 cannot hold.
__global__ void k_split64(const double* __restrict__ U, float* __restrict__ hi, float* __restrict__ lo,
                          long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double u = U[i];
        const float h = (float)u;
        hi[i] = h;
        lo[i] = (float)(u - (double)h);
    }
}

// U^{n+1} = U^n + (x1 + x2) in FP64.
__global__ void k_update64(double* __restrict__ U, const float* __restrict__ x1, const float* __restrict__ x2,
                           long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        U[i] += (double)x1[i] + (double)x2[i];
}

static unsigned elementwise_grid(long long n)
{
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_split64(const double* U, float* hi, float* lo, long long count, cudaStream_t s)
{
    k_split64<<<elementwise_grid(count), 256, 0, s>>>(U, hi, lo, count);
    return cudaGetLastError();
}

cudaError_t launch_update64(double* U, const float* x1, const float* x2, long long count, cudaStream_t s)
{
    k_update64<<<elementwise_grid(count), 256, 0, s>>>(U, x1, x2, count);
    return cudaGetLastError();
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
    if ((e = init_lines_t())) return e;
#define SPLIT_ATTR(T_, MC_, AX_)                                                                             \
    if ((e = cudaFuncSetAttribute(k_split_lines<T_, MC_, AX_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)kSmemLimit)))                                                        \
        return e;
    SPLIT_ATTR(float, 4, 0) SPLIT_ATTR(float, 8, 0) SPLIT_ATTR(float, 16, 0) SPLIT_ATTR(float, 32, 0)
    SPLIT_ATTR(float, 4, 1) SPLIT_ATTR(float, 8, 1) SPLIT_ATTR(float, 16, 1) SPLIT_ATTR(float, 32, 1)
    SPLIT_ATTR(double, 4, 0) SPLIT_ATTR(double, 8, 0) SPLIT_ATTR(double, 16, 0) SPLIT_ATTR(double, 32, 0)
    SPLIT_ATTR(double, 4, 1) SPLIT_ATTR(double, 8, 1) SPLIT_ATTR(double, 16, 1) SPLIT_ATTR(double, 32, 1)
#undef SPLIT_ATTR
    if ((e = cudaFuncSetAttribute(k_pass23<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;
    if ((e = cudaFuncSetAttribute(k_pass23<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)))
        return e;

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
    if (P.p2P == kLinesTma) {
        if constexpr (sizeof(T) == sizeof(float)) {
            const cudaError_t e = launch_lines_t(0, P, in, nullptr, out, 0, s);
            if (e != cudaErrorNotSupported) return e;
        }
        // FP64 or a field not 16-byte aligned: one lane per line
    } else if (P.p2P > 1) {
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
    // Split and TMA-fed y lines need line-invariant y systems (gamma = 0 in
    // the group); otherwise one lane per line.
    if (P.p3P == kLinesTma) {
        if constexpr (sizeof(T) == sizeof(float)) {
            if (!any_gamma_pos) {
                const cudaError_t e = launch_lines_t(1, P, in, Un, out, n, s);
                if (e != cudaErrorNotSupported) return e;
            }
        }
    } else if (P.p3P > 1 && !any_gamma_pos) {
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

template cudaError_t launch_pass23<float>(const March<float>&, const float*, const float*, float*, int,
                                          cudaStream_t);
template cudaError_t launch_pass23<double>(const March<double>&, const double*, const double*, double*, int,
                                           cudaStream_t);

}  // namespace hjm
