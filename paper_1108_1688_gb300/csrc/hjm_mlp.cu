// Kernels of the pricing surrogate's network: a 9 -> 256 -> 256 -> 256 -> 256
// -> 1 multilayer perceptron with SiLU activations (not a part of the paper's
// method; it is trained on prices the Douglas ADI march produces).
//
// The three 256 x 256 layers run on the tensor cores: bfloat16 operands
// (weights and input activations rounded to nearest even), FP32 accumulation,
// mma.sync m16n8k16 issued per warp from shared-memory tiles. One tiled GEMM
// kernel covers the forward products and both backward products (operands
// read transposed while they are staged), with fused epilogues: bias + SiLU
// (forward), SiLU' (backward). The 9-wide input layer and the 1-wide output
// layer are too thin for the tensor cores and run in FP32.
#include <cuda_bf16.h>
#include <stdint.h>

#include "hjm_mlp.cuh"

namespace hjm {
namespace mlp {

__device__ __forceinline__ float sigm(float u) { return 1.0f / (1.0f + __expf(-u)); }
__device__ __forceinline__ float silu(float u) { return u * sigm(u); }
__device__ __forceinline__ float silu_grad(float u)
{
    const float s = sigm(u);
    return s * (1.0f + u * (1.0f - s));
}

__device__ __forceinline__ float as_float(float x) { return x; }
__device__ __forceinline__ float as_float(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M x N] = op(A) op(B), op(A) M x K, op(B) K x N. A(m, k) = A[m lda + k], or
// A[k lda + m] when TA; B(k, n) = B[k ldb + n], or B[n ldb + k] when TB.
// CTA tile 64 x 64 x 32, four warps of 32 x 32, each 2 x 4 mma tiles.
template <typename TA_, typename TB_, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const TA_* __restrict__ A, int lda,
                                              const TB_* __restrict__ B, int ldb, Epi e)
{
    constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;

    for (int k0 = 0; k0 < K; k0 += BK) {
        // Stage both tiles as [row][k] in bfloat16, reading along the
        // operand's contiguous dimension.
        for (int idx = tid; idx < BM * BK; idx += 128) {
            int mm, kk;
            if (TA) {
                kk = idx / BM;
                mm = idx % BM;
            } else {
                mm = idx / BK;
                kk = idx % BK;
            }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.0f;
            if (m < M && k < K) v = as_float(TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]);
            As[mm][kk] = __float2bfloat16_rn(v);
        }
        for (int idx = tid; idx < BN * BK; idx += 128) {
            int nn, kk;
            if (TB) {
                nn = idx / BK;
                kk = idx % BK;
            } else {
                kk = idx / BN;
                nn = idx % BN;
            }
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.0f;
            if (n < N && k < K) v = as_float(TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n]);
            Bs[nn][kk] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = wm * 32 + mt * 16;
                a[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r0 + g][ks + 2 * t]);
                a[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + g + 8][ks + 2 * t]);
                a[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r0 + g][ks + 8 + 2 * t]);
                a[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + g + 8][ks + 8 + 2 * t]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c0 = wn * 32 + nt * 8;
                b[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[c0 + g][ks + 2 * t]);
                b[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[c0 + g][ks + 8 + 2 * t]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt], b[nt]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = m0 + wm * 32 + mt * 16 + g + (q >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + nt * 8 + 2 * t + (q & 1);
                if (row >= M || col >= N) continue;
                const size_t o = (size_t)row * e.ldc + col;
                const float v = acc[mt][nt][q];
                if (EPI == EPI_STORE) {
                    e.C[o] = v;
                } else if (EPI == EPI_FWD) {
                    const float z = v + e.bias[col];
                    if (e.Z) e.Z[o] = z;
                    e.H[o] = __float2bfloat16_rn(silu(z));
                } else {  // EPI_BWD: dz = dh * SiLU'(z)
                    const float dz = v * silu_grad(e.Zin[o]);
                    e.C[o] = dz;
                    e.H[o] = __float2bfloat16_rn(dz);
                }
            }
}

template <typename TA_, typename TB_, bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const TA_* A, int lda, const TB_* B, int ldb, const Epi& e,
                 cudaStream_t s)
{
    const dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<TA_, TB_, TA, TB, EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, e);
    return cudaGetLastError();
}

// Forward layer l = 1..3: Z = H_{l-1} W_l^T + b_l, H_l = SiLU(Z).
cudaError_t gemm_forward(int rows, const __nv_bfloat16* Hin, const __nv_bfloat16* Wl, const float* bl,
                         float* Z, __nv_bfloat16* Hout, cudaStream_t s)
{
    Epi e{};
    e.ldc = kWidth;
    e.bias = bl;
    e.Z = Z;
    e.H = Hout;
    return gemm<__nv_bfloat16, __nv_bfloat16, false, true, EPI_FWD>(rows, kWidth, kWidth, Hin, kWidth, Wl,
                                                                     kWidth, e, s);
}

// Backward through layer l: gW_l = dZ_l^T H_{l-1} (reduction over the rows).
cudaError_t gemm_weight_grad(int rows, const __nv_bfloat16* dZ, const __nv_bfloat16* Hin, float* gW,
                             cudaStream_t s)
{
    Epi e{};
    e.ldc = kWidth;
    e.C = gW;
    return gemm<__nv_bfloat16, __nv_bfloat16, true, false, EPI_STORE>(kWidth, kWidth, rows, dZ, kWidth, Hin,
                                                                       kWidth, e, s);
}

// Backward through layer l: dZ_{l-1} = (dZ_l W_l) * SiLU'(Z_{l-1}).
cudaError_t gemm_input_grad(int rows, const __nv_bfloat16* dZ, const __nv_bfloat16* Wl, const float* Zprev,
                            float* dZprev, __nv_bfloat16* dZprev16, cudaStream_t s)
{
    Epi e{};
    e.ldc = kWidth;
    e.Zin = Zprev;
    e.C = dZprev;
    e.H = dZprev16;
    return gemm<__nv_bfloat16, __nv_bfloat16, false, false, EPI_BWD>(rows, kWidth, kWidth, dZ, kWidth, Wl,
                                                                      kWidth, e, s);
}

// Plain product used by the tests of the tensor-core path.
cudaError_t gemm_plain(int M, int N, int K, const __nv_bfloat16* A, int lda, bool ta, const __nv_bfloat16* B,
                       int ldb, bool tb, float* C, int ldc, cudaStream_t s)
{
    Epi e{};
    e.ldc = ldc;
    e.C = C;
    if (!ta && !tb) return gemm<__nv_bfloat16, __nv_bfloat16, false, false, EPI_STORE>(M, N, K, A, lda, B, ldb, e, s);
    if (!ta && tb) return gemm<__nv_bfloat16, __nv_bfloat16, false, true, EPI_STORE>(M, N, K, A, lda, B, ldb, e, s);
    if (ta && !tb) return gemm<__nv_bfloat16, __nv_bfloat16, true, false, EPI_STORE>(M, N, K, A, lda, B, ldb, e, s);
    return gemm<__nv_bfloat16, __nv_bfloat16, true, true, EPI_STORE>(M, N, K, A, lda, B, ldb, e, s);
}

// ------------------------------------------------------------ thin layers

// Features f = (kappa, lambda, theta, epsilon, rho, T, delta, K - F, F) of
// raw inputs x = (kappa, lambda, theta, epsilon, rho, T, delta, K, F), mapped
// to [-1, 1] by the box; layer 0: Z0 = W0 f + b0, H0 = SiLU(Z0).
__global__ void k_layer0(int rows, const float* __restrict__ x, const float* __restrict__ lo,
                         const float* __restrict__ hi, const float* __restrict__ W0,
                         const float* __restrict__ b0, float* __restrict__ Xn, float* __restrict__ Z0,
                         __nv_bfloat16* __restrict__ H0)
{
    const int n = blockIdx.x;
    const int o = threadIdx.x;  // 256 threads
    if (n >= rows) return;
    __shared__ float f[kIn];
    if (o < kIn) {
        float v = x[(size_t)n * kIn + o];
        if (o == 7) v -= x[(size_t)n * kIn + 8];
        f[o] = 2.0f * (v - lo[o]) / (hi[o] - lo[o]) - 1.0f;
        if (Xn) Xn[(size_t)n * kIn + o] = f[o];
    }
    __syncthreads();
    float z = b0[o];
#pragma unroll
    for (int k = 0; k < kIn; ++k) z += W0[o * kIn + k] * f[k];
    if (Z0) Z0[(size_t)n * kWidth + o] = z;
    H0[(size_t)n * kWidth + o] = __float2bfloat16_rn(silu(z));
}

// Output layer: y = W4 . H3 + b4, one warp per row.
__global__ void k_layer4(int rows, const __nv_bfloat16* __restrict__ H3, const float* __restrict__ W4,
                         const float* __restrict__ b4, float* __restrict__ y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    float s = 0.0f;
    for (int k = lane; k < kWidth; k += 32) s += W4[k] * __bfloat162float(H3[(size_t)warp * kWidth + k]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) y[warp] = s + b4[0];
}

// Mean squared error: dy = 2 (y - t) / rows; loss accumulated into *loss.
__global__ void k_loss(int rows, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                       float* __restrict__ loss)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (n < rows) {
        const float r = y[n] - t[n];
        dy[n] = 2.0f * r / rows;
        l = r * r / rows;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) l += __shfl_down_sync(0xffffffffu, l, d);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// Back through the output layer: dZ3 = dy W4 * SiLU'(Z3).
__global__ void k_layer4_back(int rows, const float* __restrict__ dy, const float* __restrict__ W4,
                              const float* __restrict__ Z3, float* __restrict__ dZ3,
                              __nv_bfloat16* __restrict__ dZ3h)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)rows * kWidth) return;
    const int n = (int)(i / kWidth), k = (int)(i % kWidth);
    const float dz = dy[n] * W4[k] * silu_grad(Z3[i]);
    dZ3[i] = dz;
    dZ3h[i] = __float2bfloat16_rn(dz);
}

// Column sums g[c] = sum_n w[n] M[n][c] (w = 1 when null), M FP32 or BF16.
template <typename TM>
__global__ void k_colsum(int rows, int cols, const TM* __restrict__ Mx, const float* __restrict__ w,
                         float* __restrict__ g)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int n = 0; n < rows; ++n) s += (w ? w[n] : 1.0f) * as_float(Mx[(size_t)n * cols + c]);
    g[c] = s;
}

// Back through layer 0: gW0 = dZ0^T Xn, gb0 = sum dZ0 (one thread per unit).
__global__ void k_layer0_back(int rows, const float* __restrict__ dZ0, const float* __restrict__ Xn,
                              float* __restrict__ gW0, float* __restrict__ gb0)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= kWidth) return;
    float s[kIn], sb = 0.0f;
#pragma unroll
    for (int k = 0; k < kIn; ++k) s[k] = 0.0f;
    for (int n = 0; n < rows; ++n) {
        const float d = dZ0[(size_t)n * kWidth + o];
        sb += d;
#pragma unroll
        for (int k = 0; k < kIn; ++k) s[k] += d * Xn[(size_t)n * kIn + k];
    }
#pragma unroll
    for (int k = 0; k < kIn; ++k) gW0[o * kIn + k] = s[k];
    gb0[o] = sb;
}

// AdamW on the FP32 master weights; refreshes the bfloat16 copies of the
// three 256 x 256 weight matrices.
__global__ void k_adamw(size_t n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                        const float* __restrict__ g, float lr, float b1, float b2, float eps, float wd,
                        float c1, float c2, __nv_bfloat16* __restrict__ w16)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i];
    wi -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * wi);
    w[i] = wi;
    w16[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(size_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

cudaError_t layer0(int rows, const float* x, const float* lo, const float* hi, const float* W0, const float* b0,
                   float* Xn, float* Z0, __nv_bfloat16* H0, cudaStream_t s)
{
    if (rows == 0) return cudaSuccess;
    k_layer0<<<rows, kWidth, 0, s>>>(rows, x, lo, hi, W0, b0, Xn, Z0, H0);
    return cudaGetLastError();
}

cudaError_t layer4(int rows, const __nv_bfloat16* H3, const float* W4, const float* b4, float* y, cudaStream_t s)
{
    if (rows == 0) return cudaSuccess;
    k_layer4<<<(rows * 32 + 255) / 256, 256, 0, s>>>(rows, H3, W4, b4, y);
    return cudaGetLastError();
}

cudaError_t loss(int rows, const float* y, const float* t, float* dy, float* l, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(l, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    k_loss<<<(rows + 255) / 256, 256, 0, s>>>(rows, y, t, dy, l);
    return cudaGetLastError();
}

cudaError_t layer4_back(int rows, const float* dy, const float* W4, const float* Z3, float* dZ3,
                        __nv_bfloat16* dZ3h, const __nv_bfloat16* H3, float* gW4, float* gb4, cudaStream_t s)
{
    const size_t n = (size_t)rows * kWidth;
    k_layer4_back<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rows, dy, W4, Z3, dZ3, dZ3h);
    k_colsum<__nv_bfloat16><<<1, kWidth, 0, s>>>(rows, kWidth, H3, dy, gW4);
    k_colsum<float><<<1, 1, 0, s>>>(rows, 1, dy, nullptr, gb4);
    return cudaGetLastError();
}

cudaError_t bias_grad(int rows, const float* dZ, float* gb, cudaStream_t s)
{
    k_colsum<float><<<1, kWidth, 0, s>>>(rows, kWidth, dZ, nullptr, gb);
    return cudaGetLastError();
}

cudaError_t layer0_back(int rows, const float* dZ0, const float* Xn, float* gW0, float* gb0, cudaStream_t s)
{
    k_layer0_back<<<1, kWidth, 0, s>>>(rows, dZ0, Xn, gW0, gb0);
    return cudaGetLastError();
}

cudaError_t adamw(size_t n, float* w, float* m, float* v, const float* g, float lr, float b1, float b2, float eps,
                  float wd, long long step, __nv_bfloat16* w16, cudaStream_t s)
{
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adamw<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, w, m, v, g, lr, b1, b2, eps, wd, c1, c2, w16);
    return cudaGetLastError();
}

cudaError_t to_bf16(size_t n, const float* a, __nv_bfloat16* b, cudaStream_t s)
{
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace hjm
