// Passes 2 and 3 of a Douglas ADI step (Section 5.1) on FP32 groups with
// the strided lines moved by the Tensor Memory Accelerator:
//
//   pass 2  (I - theta dt A_v) dU2 = dU1          v lines (stride n_r)
//   pass 3  (I - theta dt A_y) dU3 = dU2,         y lines (stride n_r n_v),
//           U^{n+1} = U^n + dU3                   fused with the update
//
// A tile is 32 consecutive r nodes times one whole line: for pass 2 the
// (32 x n_v) block of one y plane, for pass 3 the (32 x n_y) block of one v
// node (and the same block of U^n). One cp.async.bulk.tensor box copy brings
// a tile into shared memory as n rows of 128 bytes, lane i of the warp owns
// column i (one line; the columns fall in distinct banks), solves its line
// in place by the Thomas algorithm (Section 5) with the precomputed LU
// factors of the line-invariant systems (the v system is the same for every
// v line of an instrument; with gamma = 0 the y system depends on v only),
// and one box store writes the tile back. Nodes past n_r arrive as zeros
// and are not stored (the box is clipped at the tensor's edge).
//
// The grid is persistent: every warp marches its own tiles (tile g, g + NW,
// g + 2 NW, ... for global warp g of NW) through a ring of R shared-memory
// slots (R = 1 in use, see lines_shape): R copies are started at once, and as
// soon as the box store of tile q has read its slot, the copy of tile q + R
// goes into it; the copies in and out of the many warps resident on an SM
// overlap one another's line solves. Each tile's LU factors are copied into
// shared memory (cp.async) while the previous tile is solved. Warps
// never wait on one another. Every wait on a copy is bounded: a warp whose
// wait runs out counts itself in a device counter (read by
// lines_t_timeouts), waits a bounded time for its other copies and leaves
// without writing the rest of its tiles. The arithmetic, and so the
// rounding, is that of k_pass2 / k_pass3 (hjm_march.cu).
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "hjm_kernels.cuh"
#include "hjm_tma.cuh"

namespace hjm {
namespace {

constexpr unsigned kLinePolls = 1u << 22;  // polls of a tile's barrier before giving up
constexpr int kHeader = 256;               // barriers: up to 4 per warp, 8 warps
constexpr int kRowB = 32 * 4;              // one row of a tile: 32 FP32 values
constexpr int kSmemLimit = 227 * 1024;

// Bytes of one factor buffer of a line of L nodes (3 L floats, 128-byte
// multiple so that every slot stays aligned for the box copies).
__host__ __device__ inline int fac_bytes(int L) { return (3 * L * 4 + 127) & ~127; }

__device__ unsigned g_lt_timeouts;          // warps that gave up a wait
__device__ long long g_lt_drop = -1;        // test hook: tile never copied
__device__ unsigned g_lt_limit = kLinePolls;

// 4-byte asynchronous copy global -> shared (the factor tables of a tile).
__device__ __forceinline__ void cp4(unsigned dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Thomas solve of one column (stride 32 floats) of L nodes in place with the
// LU factors fp[k] = (l_k, 1/pivot_k) and fc[k] = c'_k (Section 5):
//   forward  d'_k = (d_k - l_k d'_{k-1}) / pivot_k,
//   backward x_k = d'_k - c'_k x_{k+1};
// UPD: the column receives u_k + x_k instead of x_k (pass 3's update).
// Eight nodes at a time: the next eight nodes' operands are read into
// registers before the current eight are eliminated and stored, so the
// shared-memory latency is paid once per eight nodes and not on every link
// of the recurrence. Returns x_0.
template <bool UPD>
__device__ __forceinline__ float line_solve(float* col, const float* u, const float2* fp, const float* fc, int L)
{
    constexpr int C = 8;
    float dp = 0.f;
    int kk = 0;
    if (L >= C) {
        float c[C];
        float2 f[C];
#pragma unroll
        for (int e = 0; e < C; ++e) {
            c[e] = col[e * 32];
            f[e] = fp[e];
        }
        for (; kk + C <= L; kk += C) {
            float cn[C];
            float2 fn[C];
#pragma unroll
            for (int e = 0; e < C; ++e) {  // the next eight (clamped: always inside the column)
                const int q = min(kk + C + e, L - 1);
                cn[e] = col[q * 32];
                fn[e] = fp[q];
            }
#pragma unroll
            for (int e = 0; e < C; ++e) {
                dp = (c[e] - f[e].x * dp) * f[e].y;
                c[e] = dp;
            }
#pragma unroll
            for (int e = 0; e < C; ++e) col[(kk + e) * 32] = c[e];
#pragma unroll
            for (int e = 0; e < C; ++e) {
                c[e] = cn[e];
                f[e] = fn[e];
            }
        }
    }
    for (; kk < L; ++kk) {
        const float2 f = fp[kk];
        dp = (col[kk * 32] - f.x * dp) * f.y;
        col[kk * 32] = dp;
    }
    float x = dp;
    if (UPD) col[(L - 1) * 32] = u[(L - 1) * 32] + x;
    kk = L - 2;
    if (kk + 1 >= C) {
        float c[C], g[C], w[C];
#pragma unroll
        for (int e = 0; e < C; ++e) {
            c[e] = col[(kk - e) * 32];
            g[e] = fc[kk - e];
            w[e] = UPD ? u[(kk - e) * 32] : 0.f;
        }
        for (; kk + 1 >= C; kk -= C) {  // nodes kk .. kk - 7
            float cn[C], gn[C], wn[C];
#pragma unroll
            for (int e = 0; e < C; ++e) {
                const int q = max(kk - C - e, 0);
                cn[e] = col[q * 32];
                gn[e] = fc[q];
                wn[e] = UPD ? u[q * 32] : 0.f;
            }
#pragma unroll
            for (int e = 0; e < C; ++e) {
                x = c[e] - g[e] * x;
                c[e] = UPD ? w[e] + x : x;
            }
#pragma unroll
            for (int e = 0; e < C; ++e) col[(kk - e) * 32] = c[e];
#pragma unroll
            for (int e = 0; e < C; ++e) {
                c[e] = cn[e];
                g[e] = gn[e];
                w[e] = wn[e];
            }
        }
    }
    for (; kk >= 0; --kk) {
        x = col[kk * 32] - fc[kk] * x;
        col[kk * 32] = UPD ? u[kk * 32] + x : x;
    }
    return x;
}

// Bounded wait of the whole warp on the copy with parity par of barrier
// bar: true when every lane saw it complete.
__device__ __forceinline__ bool warp_wait(unsigned bar, unsigned par)
{
    bool ok = tma::mbar_try_wait(bar, par);
    if (!ok) {
        const unsigned limit = g_lt_limit;
        for (unsigned it = 1; it < limit && !ok; ++it) ok = tma::mbar_try_wait(bar, par);
    }
    return __all_sync(0xffffffffu, ok);
}

// AXIS 0: pass 2 (in: dU1 as a 3-D view (n_r, n_v, B n_y), out: dU2, the
// same view); AXIS 1: pass 3 (in: dU2 and un: U^n as 4-D views (n_r, n_v,
// n_y, B), out: U^{n+1}); AXIS 2: pass 3 in place (out = un = U): the tile
// of dU3 is added to U by the box store itself (a reduction store), so U^n
// is never staged and a warp needs half the shared memory. R slots per
// warp, blockDim.x / 32 warps per CTA.
template <int AXIS>
__global__ void __launch_bounds__(128) k_lines_t(const March<float> P, const __grid_constant__ CUtensorMap tin,
                                                  const __grid_constant__ CUtensorMap tun,
                                                  const __grid_constant__ CUtensorMap tout, const int n,
                                                  const int R)
{
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((128u - (tma::su32(sm_raw) & 127u)) & 127u);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int nr = P.nr, nv = P.nv, ny = P.ny;
    const int L = AXIS == 0 ? nv : ny;   // nodes per line
    const int colB = L * kRowB;          // one block of 32 lines
    const int slotB = AXIS == 1 ? 2 * colB : colB;
    const int facB = fac_bytes(L);       // one factor buffer: (sub, 1/pivot) pairs, then c'
    const unsigned bar0 = tma::su32(sm) + 32u * (unsigned)warp;
    unsigned char* slots = sm + kHeader + (size_t)warp * (R * slotB + 2 * facB);
    const unsigned slots0 = tma::su32(slots);
    float* const facs = reinterpret_cast<float*>(slots + R * slotB);  // two buffers, tile q in q & 1
    const int rt = (nr + 31) >> 5;       // tiles across r
    const int mid = AXIS == 0 ? ny : nv; // tiles across the other transverse axis
    const long long ntile = (long long)P.B * mid * rt;
    const long long gw = (long long)blockIdx.x * W + warp, NW = (long long)gridDim.x * W;
    const int cnt = gw < ntile ? (int)((ntile - 1 - gw) / NW + 1) : 0;
    if (cnt == 0) return;
    if (lane == 0) {
        for (int s = 0; s < R; ++s) tma::mbar_init(bar0 + 8u * s, 1);
        tma::fence_barrier_init();
    }
    __syncwarp();
    const long long drop = g_lt_drop;

    // lane 0: start the copy of the warp's q-th tile into slot q mod R
    auto issue = [&](int q) {
        const long long t = gw + (long long)q * NW;
        if (t == drop) return;  // test hook: the copy never starts, its wait runs out
        const unsigned s = (unsigned)(q % R), bar = bar0 + 8u * s, dst = slots0 + s * (unsigned)slotB;
        const int x0 = (int)(t % rt) * 32;
        const long long r = t / rt;
        if constexpr (AXIS == 0) {
            tma::mbar_expect_tx(bar, (unsigned)colB);
            tma::load3(dst, &tin, x0, 0, (int)r, bar);
        } else if constexpr (AXIS == 2) {
            tma::mbar_expect_tx(bar, (unsigned)colB);
            tma::load4(dst, &tin, x0, (int)(r % nv), 0, (int)(r / nv), bar);
        } else {
            tma::mbar_expect_tx(bar, 2u * (unsigned)colB);
            tma::load4(dst, &tin, x0, (int)(r % nv), 0, (int)(r / nv), bar);
            tma::load4(dst + (unsigned)colB, &tun, x0, (int)(r % nv), 0, (int)(r / nv), bar);
        }
    };
    // every lane: start the copies of the q-th tile's LU factors (sub-diagonal
    // l, c' and 1/pivot of the line system, contiguous in the tables) into
    // factor buffer q & 1, as pairs (l, 1/pivot) followed by c'
    auto issue_factors = [&](int q) {
        const long long r = (gw + (long long)q * NW) / rt;
        const int b = (int)(r / mid), m = (int)(r % mid);
        const float* src = AXIS == 0 ? P.vf + (size_t)b * 3 * nv : P.yf + ((size_t)b * nv + m) * 3 * ny;
        const unsigned dst = tma::su32(facs + (q & 1) * (facB / 4));
        for (int e = lane; e < 3 * L; e += 32) {
            const int w = e / L, kk = e - w * L;
            const int o = w == 0 ? 2 * kk : (w == 2 ? 2 * kk + 1 : 2 * L + kk);
            cp4(dst + 4u * (unsigned)o, src + e);
        }
        cp_commit();
    };
    // the q-th tile's instrument flags (r_min Dirichlet, read-out corner),
    // read a tile ahead so that the load's latency hides behind a solve
    auto flags = [&](int q) {
        const int* f = P.fl + (size_t)((gw + (long long)q * NW) / rt / mid) * FL_N;
        return make_int3(f[FL_RLO_DIR], f[FL_RI0], f[FL_RK0]);
    };
    int issued = min(R, cnt);  // tiles whose copy has been started (0 .. issued - 1)
    if (lane == 0)
        for (int q = 0; q < issued; ++q) issue(q);
    issue_factors(0);
    int3 fnext = flags(0);

    for (int q = 0; q < cnt; ++q) {
        const unsigned s = (unsigned)(q % R);
        if (!warp_wait(bar0 + 8u * s, (unsigned)(q / R) & 1u)) {
            // leave no copy in flight into this warp's slots: wait (bounded)
            // for the tiles started after this one, and for the stores
            if (lane == 0) {
                const unsigned limit = g_lt_limit;
                for (int p = q + 1; p < issued; ++p) {
                    if (gw + (long long)p * NW == drop) continue;
                    const unsigned bar = bar0 + 8u * (unsigned)(p % R), par = (unsigned)(p / R) & 1u;
                    bool ok = false;
                    for (unsigned it = 0; it < limit && !ok; ++it) ok = tma::mbar_try_wait(bar, par);
                }
                tma::bulk_wait_all();
                atomicAdd(&g_lt_timeouts, 1u);
            }
            cp_wait_all();
            __syncwarp();
            return;
        }
        cp_wait_all();  // this tile's factors (the only group in flight)
        __syncwarp();
        if (q + 1 < cnt) issue_factors(q + 1);  // the other buffer: tile q - 1 is done with it
        const int3 fl = fnext;  // (r_min Dirichlet, FL_RI0, FL_RK0) of this tile's instrument
        if (q + 1 < cnt) fnext = flags(q + 1);
        const float2* fp = reinterpret_cast<const float2*>(facs + (q & 1) * (facB / 4));
        const float* fc = facs + (q & 1) * (facB / 4) + 2 * L;
        const long long t = gw + (long long)q * NW;
        const int i = (int)(t % rt) * 32 + lane;
        const long long r = t / rt;
        const int b = (int)(r / mid), m = (int)(r % mid);  // m: y plane (pass 2) or v node (pass 3)
        float* col = reinterpret_cast<float*>(slots + s * slotB) + lane;
        if (i < nr) {
            const bool dir = i == nr - 1 || (i == 0 && fl.x);  // identity system
            if constexpr (AXIS == 0) {
                if (!dir) line_solve<false>(col, nullptr, fp, fc, nv);
            } else if constexpr (AXIS == 2) {  // dU3 (dU2 itself on an identity line), added by the store
                if (!dir) line_solve<false>(col, nullptr, fp, fc, ny);
                note_increment_at(P, fl.y, fl.z, b, i, m, n, col[0]);
            } else {
                const float* u = col + ny * 32;
                if (dir) {
                    note_increment_at(P, fl.y, fl.z, b, i, m, n, col[0]);
                    for (int jj = 0; jj < ny; ++jj) col[jj * 32] = u[jj * 32] + col[jj * 32];
                } else {
                    const float x0 = line_solve<true>(col, u, fp, fc, ny);
                    note_increment_at(P, fl.y, fl.z, b, i, m, n, x0);
                }
            }
        }
        tma::fence_proxy_async_smem();  // the solved column before the store reads it
        __syncwarp();
        if (lane == 0) {
            const unsigned src = slots0 + s * (unsigned)slotB;
            const int x0 = (int)(t % rt) * 32;
            if constexpr (AXIS == 0)
                tma::store3(&tout, x0, 0, (int)r, src);
            else if constexpr (AXIS == 2)
                tma::reduce_add4(&tout, x0, m, 0, b, src);
            else
                tma::store4(&tout, x0, m, 0, b, src);
            tma::bulk_commit();
            if (issued < cnt) {  // tile q + R into this slot, once the store has read it
                tma::bulk_wait_read_0();
                issue(issued);
                ++issued;
            }
        }
        issued = __shfl_sync(0xffffffffu, issued, 0);
    }
    if (lane == 0) tma::bulk_wait_all();
}

// ------------------------------------------------------------------- host

// Tensor map of a group's FP32 field U[b][j][k][i]: AXIS 0 the 3-D view
// (i, k, b n_y + j) with box (32, n_v, 1); AXIS 1 the 4-D view (i, k, j, b)
// with box (32, 1, n_y, 1). n_r a multiple of 4 (16-byte row strides).
cudaError_t lines_map(CUtensorMap* m, const float* U, const March<float>& P, int axis)
{
    const tma::EncodeTiled fn = tma::encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t nr = (cuuint64_t)P.nr, nv = (cuuint64_t)P.nv, ny = (cuuint64_t)P.ny, B = (cuuint64_t)P.B;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r;
    if (axis == 0) {
        const cuuint64_t dims[3] = {nr, nv, B * ny};
        const cuuint64_t strides[2] = {nr * 4, nr * nv * 4};
        const cuuint32_t box[3] = {32, (cuuint32_t)nv, 1};
        r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(U), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[4] = {nr, nv, ny, B};
        const cuuint64_t strides[3] = {nr * 4, nr * nv * 4, nr * nv * ny * 4};
        const cuuint32_t box[4] = {32, 1, (cuuint32_t)ny, 1};
        r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(U), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Warps per CTA and slots per warp for a line of L nodes: three slots, as
// many warps (4, 2, 1) as fit; two slots when one warp of three does not fit.
size_t lines_smem(int axis, int L, int W, int R)
{
    const size_t per_warp = (size_t)R * L * kRowB * (axis == 1 ? 2 : 1) + 2 * (size_t)fac_bytes(L);
    return (size_t)kHeader + (size_t)W * per_warp + 128;  // + alignment slack
}

// One slot per warp (a deeper ring costs resident warps, and the strided
// passes are bound by the number of lines in flight per SM: measured on the
// 128 x 64 x 64 batch, two slots per warp made pass 3 35 % slower and three
// slots 80 % slower; pass 2 was equal with two slots, slower with three),
// and the warps per CTA (4, 2, 1) that put the most warps on an SM (228 KB
// of shared memory, 1 KB of it reserved per CTA).
bool lines_shape(int axis, int L, int& W, int& R)
{
    R = 1;
    int best = 0;
    for (int w = 4; w >= 1; w /= 2) {
        const size_t sm = lines_smem(axis, L, w, R);
        if (sm > (size_t)kSmemLimit) continue;
        const int warps = w * (int)(228 * 1024 / (sm + 1024));
        if (warps > best) {
            best = warps;
            W = w;
        }
    }
    return best > 0;
}

// Resident CTAs of the kernel (kind 0, 1, 2 as the template argument) at
// this shape times the SM count, cached.
int lines_grid(int axis, int W, size_t smem)
{
    static std::mutex mu;
    static int dev_cached = -1, sms = 0;
    static std::vector<std::pair<std::pair<int, size_t>, int>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (dev != dev_cached) {
        cache.clear();
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        dev_cached = dev;
    }
    const auto key = std::make_pair(axis * 16 + W, smem);
    for (const auto& c : cache)
        if (c.first == key) return c.second;
    int nb = 0;
    const cudaError_t e =
        axis == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lines_t<0>, 32 * W, smem)
        : axis == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lines_t<1>, 32 * W, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lines_t<2>, 32 * W, smem);
    if (e != cudaSuccess) return 0;
    cache.emplace_back(key, nb * sms);
    return nb * sms;
}

}  // namespace

bool lines_t_valid(int axis, int nr, int nv, int ny, size_t elem)
{
    const int L = axis == 0 ? nv : ny;
    int W, R;
    return elem == sizeof(float) && nr >= 1 && nr % 4 == 0 && L >= 2 && L <= 256 && nv >= 1 && ny >= 1 &&
           lines_shape(axis, L, W, R);
}

cudaError_t launch_lines_t(int axis, const March<float>& P, const float* in, const float* Un, float* out, int n,
                           cudaStream_t s)
{
    if (!lines_t_valid(axis, P.nr, P.nv, P.ny, sizeof(float))) return cudaErrorInvalidValue;
    if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) |
          reinterpret_cast<uintptr_t>(axis == 0 ? in : Un)) & 15) != 0)
        return cudaErrorNotSupported;  // the caller falls back to the lane-per-line kernels
    CUtensorMap mi, mu, mo;
    cudaError_t e = lines_map(&mi, in, P, axis);
    if (e == cudaSuccess) e = lines_map(&mu, axis == 0 ? in : Un, P, axis);
    if (e == cudaSuccess) e = lines_map(&mo, out, P, axis);
    if (e != cudaSuccess) return e;
    // pass 3 in place (the Douglas stage: U^{n+1} over U^n) adds dU3 to U by
    // the reduction store; otherwise U^n is staged next to dU2
    const int kind = axis == 0 ? 0 : (Un == out ? 2 : 1);
    int W, R;
    lines_shape(kind, axis == 0 ? P.nv : P.ny, W, R);
    const size_t smem = lines_smem(kind, axis == 0 ? P.nv : P.ny, W, R);
    const long long ntile = (long long)P.B * (axis == 0 ? P.ny : P.nv) * ((P.nr + 31) / 32);
    const long long grid = std::min<long long>((ntile + W - 1) / W, lines_grid(kind, W, smem));
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (kind == 0)
        k_lines_t<0><<<(unsigned)grid, 32 * W, smem, s>>>(P, mi, mu, mo, n, R);
    else if (kind == 1)
        k_lines_t<1><<<(unsigned)grid, 32 * W, smem, s>>>(P, mi, mu, mo, n, R);
    else
        k_lines_t<2><<<(unsigned)grid, 32 * W, smem, s>>>(P, mi, mu, mo, n, R);
    return cudaGetLastError();
}

cudaError_t init_lines_t()
{
    cudaError_t e = cudaFuncSetAttribute(k_lines_t<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lines_t<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lines_t<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    return e;
}

cudaError_t lines_t_timeouts(unsigned* count, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(count, g_lt_timeouts, sizeof(unsigned));
    if (e == cudaSuccess && reset) {
        const unsigned z = 0;
        e = cudaMemcpyToSymbol(g_lt_timeouts, &z, sizeof(unsigned));
    }
    return e;
}

cudaError_t lines_t_test_drop(long long tile, unsigned limit)
{
    cudaError_t e = cudaMemcpyToSymbol(g_lt_drop, &tile, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_lt_limit, &limit, sizeof(unsigned));
    return e;
}

}  // namespace hjm
