// Declarations of the surrogate network's kernels (hjm_mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace hjm {
namespace mlp {

constexpr int kWidth = 256;  // hidden width
constexpr int kIn = 9;       // raw inputs / features

// Flat parameter layout: W0 [256 x 9], b0, W1 [256 x 256], b1, W2, b2, W3, b3,
// W4 [256], b4 [1].
constexpr size_t kOffW0 = 0;
constexpr size_t kOffB0 = kOffW0 + (size_t)kWidth * kIn;
constexpr size_t kOffW1 = kOffB0 + kWidth;
constexpr size_t kOffB1 = kOffW1 + (size_t)kWidth * kWidth;
constexpr size_t kOffW2 = kOffB1 + kWidth;
constexpr size_t kOffB2 = kOffW2 + (size_t)kWidth * kWidth;
constexpr size_t kOffW3 = kOffB2 + kWidth;
constexpr size_t kOffB3 = kOffW3 + (size_t)kWidth * kWidth;
constexpr size_t kOffW4 = kOffB3 + kWidth;
constexpr size_t kOffB4 = kOffW4 + kWidth;
constexpr size_t kParams = kOffB4 + 1;  // 200,193

enum { EPI_STORE = 0, EPI_FWD = 1, EPI_BWD = 2 };

struct Epi {
    int ldc;
    const float* bias;   // EPI_FWD
    float* Z;            // EPI_FWD: pre-activation out (may be null)
    __nv_bfloat16* H;    // EPI_FWD: SiLU(Z) out; EPI_BWD: dz out (bfloat16)
    const float* Zin;    // EPI_BWD: pre-activation of the previous layer
    float* C;            // EPI_STORE / EPI_BWD: FP32 out
};

cudaError_t gemm_forward(int rows, const __nv_bfloat16* Hin, const __nv_bfloat16* Wl, const float* bl, float* Z,
                         __nv_bfloat16* Hout, cudaStream_t s);
cudaError_t gemm_weight_grad(int rows, const __nv_bfloat16* dZ, const __nv_bfloat16* Hin, float* gW,
                             cudaStream_t s);
cudaError_t gemm_input_grad(int rows, const __nv_bfloat16* dZ, const __nv_bfloat16* Wl, const float* Zprev,
                            float* dZprev, __nv_bfloat16* dZprev16, cudaStream_t s);
cudaError_t gemm_plain(int M, int N, int K, const __nv_bfloat16* A, int lda, bool ta, const __nv_bfloat16* B,
                       int ldb, bool tb, float* C, int ldc, cudaStream_t s);
cudaError_t layer0(int rows, const float* x, const float* lo, const float* hi, const float* W0, const float* b0,
                   float* Xn, float* Z0, __nv_bfloat16* H0, cudaStream_t s);
cudaError_t layer4(int rows, const __nv_bfloat16* H3, const float* W4, const float* b4, float* y, cudaStream_t s);
cudaError_t loss(int rows, const float* y, const float* t, float* dy, float* l, cudaStream_t s);
cudaError_t layer4_back(int rows, const float* dy, const float* W4, const float* Z3, float* dZ3,
                        __nv_bfloat16* dZ3h, const __nv_bfloat16* H3, float* gW4, float* gb4, cudaStream_t s);
cudaError_t bias_grad(int rows, const float* dZ, float* gb, cudaStream_t s);
cudaError_t layer0_back(int rows, const float* dZ0, const float* Xn, float* gW0, float* gb0, cudaStream_t s);
cudaError_t adamw(size_t n, float* w, float* m, float* v, const float* g, float lr, float b1, float b2, float eps,
                  float wd, long long step, __nv_bfloat16* w16, cudaStream_t s);
cudaError_t to_bf16(size_t n, const float* a, __nv_bfloat16* b, cudaStream_t s);
// Inference forward of the whole network in one tcgen05 kernel
// (hjm_mlp_tc.cu): y [rows] from raw inputs x [rows][9], the box [2][9], the
// FP32 parameters P (biases, W0, W4) and their bfloat16 copy P16 (W1..W3);
// packed: scratch of 3 x 256 x 256 bfloat16 values (the three layers'
// weights re-ordered for bulk copies, rewritten by every call).
cudaError_t forward_fused(int rows, const float* x, const float* box, const float* P, const __nv_bfloat16* P16,
                          __nv_bfloat16* packed, float* y, cudaStream_t s);
// CTAs of forward_fused whose bounded wait on the tensor cores ran out.
cudaError_t forward_fused_timeouts(unsigned* count, bool reset);

}  // namespace mlp
}  // namespace hjm
