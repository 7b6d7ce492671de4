// Inference of the surrogate network (hjm_surrogate.cu) fused into one kernel
// on the fifth-generation tensor cores. A CTA takes tiles of 128 rows through
// every layer: the FP32 input layer writes the tile's bfloat16 activations to
// shared memory; each 256 x 256 layer is 16 tcgen05.mma (M 128, N 256, K 16,
// bfloat16 operands from shared memory, FP32 accumulator in tensor memory)
// issued by one thread, with completion signalled on an mbarrier; the
// epilogue reads the accumulator back with tcgen05.ld, adds the bias, applies
// SiLU, rounds to bfloat16 and writes the next layer's operand over the
// previous one (or, after the last hidden layer, the FP32 output dot
// product). Rounding is the unfused path's: bfloat16 weights and hidden
// activations, FP32 accumulation and biases, FP32 thin layers.
//
// Operands are laid out in the canonical K-major form without swizzle: 8 x 8
// bfloat16 "core matrices" of 128 contiguous bytes (8 rows of 16 bytes),
// core matrices adjacent in K 128 bytes apart (the descriptor's leading
// byte offset) and groups of 8 rows 4096 bytes apart (its stride byte
// offset, the 32 core matrices of a 256-wide row group). Every wait on the
// mbarrier is bounded; a CTA whose wait runs out writes NaN outputs for its
// tile, counts itself (mlp_tc_timeouts), releases its tensor memory and stops.
#include <cuda_bf16.h>
#include <stdint.h>

#include "hjm_mlp.cuh"

namespace hjm {
namespace mlp {
namespace {

constexpr int kTM = 128;                              // rows per tile: the MMA's M
constexpr int kThr = 512;                             // 16 warps
constexpr uint32_t kLBO = 128;                        // bytes between core matrices along K
constexpr uint32_t kSBO = (kWidth / 8) * 128;         // bytes between 8-row groups
constexpr uint32_t kABytes = kTM * kWidth * 2;        // activations: 64 KB
constexpr uint32_t kWBytes = kWidth * kWidth * 2;     // one layer's weights: 128 KB
constexpr int kAux = 3 * kWidth + kWidth * kIn + kWidth + kWidth + 1 + 2 * kIn + 3 * kTM;  // floats
constexpr uint32_t kSmem = 1024 + kABytes + kWBytes + kAux * 4 + 64;
constexpr unsigned kPolls = 1u << 24;                 // bounded wait on an MMA batch
constexpr uint32_t kTmemCols = 256;                   // the accumulator: 128 lanes x 256 FP32 columns

__device__ unsigned g_tc_timeouts;

// Byte offset of element (row r, column k) of a 128- or 256-row operand.
__device__ __forceinline__ uint32_t op_off(int r, int k)
{
    return (uint32_t)(r >> 3) * kSBO + (uint32_t)(k >> 3) * kLBO + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2;
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed
// descriptor version 1 (46-47), base offset 0, layout type 0 = no swizzle
// (61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((kLBO >> 4) & 0x3fff) << 16) |
           ((uint64_t)((kSBO >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// bfloat16 A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28), dense, no negation.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kWidth >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// The same load split in two: the request, and the wait, which names the
// registers the request fills (so that no use of them moves above it).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// 8 floats from 32-byte-aligned shared memory.
__device__ __forceinline__ void ld8(const float* p, float (&v)[8])
{
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}

// SiLU with the hardware exponential and an approximate division (a few
// instructions; its error, a few FP32 units, is far below the bfloat16
// rounding that follows).
__device__ __forceinline__ float silu_f(float u) { return __fdividef(u, 1.0f + __expf(-u)); }

__device__ __forceinline__ void st16(unsigned char* p, const float (&v)[8])
{
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<uint4*>(h);
}

// Chunk d (16 bytes) of a layer's weights in the canonical layout holds
// W[n][8c .. 8c + 7], n = 8 (d >> 8) + (d & 7), c = (d >> 3) & 31: the
// order of the copy below (and of the packed weights, k_pack_weights).
__device__ __forceinline__ void chunk_source(int d, int& n, int& c)
{
    n = (d >> 8) * 8 + (d & 7);
    c = (d >> 3) & 31;
}

// One layer's packed weights (128 KB, already in the shared-memory order)
// into sW by four bulk copies of 32 KB, completion (bytes) on the mbarrier.
__device__ __forceinline__ void load_weights(uint32_t sW_a, const __nv_bfloat16* __restrict__ Wp, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(kWBytes) : "memory");
    for (int i = 0; i < 4; ++i)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                sW_a + (uint32_t)i * (kWBytes / 4)),
            "l"(Wp + (size_t)i * (kWidth * kWidth / 4)), "r"(kWBytes / 4), "r"(bar)
            : "memory");
}


__device__ __forceinline__ const __nv_bfloat16* layer_weights(const __nv_bfloat16* P16, int l)
{
    return P16 + (l == 0 ? kOffW1 : (l == 1 ? kOffW2 : kOffW3));
}

// The three 256 x 256 layers' bfloat16 weights into the shared-memory
// order of the MMA operand (packed[l] = 8192 chunks of 16 bytes), so that
// a layer arrives by a few bulk copies instead of 8192 per-thread copies.
__global__ void k_pack_weights(const __nv_bfloat16* __restrict__ P16, __nv_bfloat16* __restrict__ packed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * kWidth * kWidth / 8) return;
    const int l = i / (kWidth * kWidth / 8), d = i % (kWidth * kWidth / 8);
    int n, c;
    chunk_source(d, n, c);
    const uint4 v = *reinterpret_cast<const uint4*>(layer_weights(P16, l) + (size_t)n * kWidth + c * 8);
    *reinterpret_cast<uint4*>(packed + (size_t)l * kWidth * kWidth + (size_t)d * 8) = v;
}

__global__ void __launch_bounds__(kThr, 1) k_mlp_fused(int rows, const float* __restrict__ x,
                                                      const float* __restrict__ box, const float* __restrict__ P,
                                                      const __nv_bfloat16* __restrict__ P16p,
                                                      float* __restrict__ y)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA = sm;
    unsigned char* sW = sm + kABytes;
    float* aux = reinterpret_cast<float*>(sm + kABytes + kWBytes);
    float* sB = aux;                         // b1, b2, b3
    float* sW0 = sB + 3 * kWidth;            // W0 transposed, [9][256]: 8 outputs' weights of an input in 32 bytes
    float* sb0 = sW0 + kWidth * kIn;
    float* sW4 = sb0 + kWidth;
    float* sb4 = sW4 + kWidth;
    float* slo = sb4 + 1;                    // box lo, hi
    float* shi = slo + kIn;
    float* ypart = shi + kIn;                // [3][128] partial output dot products
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(ypart + 3 * kTM) + 15) & ~(uintptr_t)15);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);  // bar[0]: MMAs done, bar[1]: weights landed
    int* stop = reinterpret_cast<int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_a = su32(bar), wbar_a = bar_a + 8u;
    for (int i = tid; i < kWidth; i += kThr) {
        sB[i] = P[kOffB1 + i];
        sB[kWidth + i] = P[kOffB2 + i];
        sB[2 * kWidth + i] = P[kOffB3 + i];
        sb0[i] = P[kOffB0 + i];
        sW4[i] = P[kOffW4 + i];
    }
    for (int i = tid; i < kWidth * kIn; i += kThr) sW0[(i % kIn) * kWidth + i / kIn] = P[kOffW0 + i];
    if (tid < kIn) {
        slo[tid] = box[tid];
        shi[tid] = box[kIn + tid];
    }
    if (tid == 0) {
        sb4[0] = P[kOffB4];
        *stop = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(wbar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {  // the accumulator's tensor memory (one warp allocates)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t sA_a = su32(sA), sW_a = su32(sW);
    uint32_t phase = 0;

    // epilogue mapping: warp w reads accumulator lanes (rows) 32 (w % 4) ..
    // and the 64 columns 64 (w / 4) .. of them
    const int r_ep = 32 * (warp & 3) + lane, cq = warp >> 2;
    const uint32_t t_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * cq);

    const int tiles = (rows + kTM - 1) / kTM;
    // thread 0: weight loads issued and completions seen (parity of the next)
    unsigned w_issued = 0, w_seen = 0;
    if (tid == 0 && blockIdx.x < tiles) {  // the first tile's first layer
        load_weights(sW_a, P16p, wbar_a);
        ++w_issued;
    }
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int row0 = tile * kTM;
        // input layer (FP32): row r = tid % 128, the 64 outputs 64 (tid / 128) ..
        {
            const int r = tid & (kTM - 1), qt = tid >> 7;
            float f[kIn];
            const int gr = row0 + r;
#pragma unroll
            for (int k = 0; k < kIn; ++k) f[k] = gr < rows ? x[(size_t)gr * kIn + k] : 0.0f;
            f[7] -= f[8];
#pragma unroll
            for (int k = 0; k < kIn; ++k) f[k] = 2.0f * (f[k] - slo[k]) / (shi[k] - slo[k]) - 1.0f;
            for (int c8 = 0; c8 < 8; ++c8) {
                // 8 outputs: bias and weights as 16-byte vectors (the same
                // addresses across the warp), the sums in the order b + sum_k
                const int o0 = qt * 64 + c8 * 8;
                float h[8];
                ld8(sb0 + o0, h);
#pragma unroll
                for (int k = 0; k < kIn; ++k) {
                    float w[8];
                    ld8(sW0 + k * kWidth + o0, w);
#pragma unroll
                    for (int q = 0; q < 8; ++q) h[q] += w[q] * f[k];
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) h[q] = silu_f(h[q]);
                st16(sA + op_off(r, o0), h);
            }
        }
        for (int l = 0; l < 3; ++l) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // operands visible to the MMA
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                // this layer's weights have landed (bounded wait)
                bool wok = false;
                for (unsigned it = 0; it < kPolls && !wok; ++it) wok = bar_try(wbar_a, w_seen & 1u);
                if (wok) {
                    ++w_seen;
#pragma unroll
                    for (int kk = 0; kk < kWidth / 16; ++kk)
                        mma_f16(tmem, smem_desc(sA_a + kk * 2 * kLBO), smem_desc(sW_a + kk * 2 * kLBO), kk > 0);
                } else {
                    atomicExch(stop, 1);
                }
                mma_commit(bar_a);  // (with no MMA after a failed wait: completes at once)
            }
            // one warp watches the barrier (bounded), the others wait at the
            // CTA barrier instead of polling shared memory beside the MMAs
            if (warp == 0) {
                bool ok = false;
                for (unsigned it = 0; it < kPolls && !ok; ++it) ok = bar_try(bar_a, phase);
                if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicExch(stop, 1);
            }
            phase ^= 1u;
            __syncthreads();
            if (*stop) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // the weight buffer is free: the next layer's weights (the next
            // tile's first layer after the last) travel during the epilogue
            if (tid == 0 && (l < 2 || tile + (int)gridDim.x < tiles)) {
                load_weights(sW_a, P16p + (size_t)(l == 2 ? 0 : l + 1) * kWidth * kWidth, wbar_a);
                ++w_issued;
            }
            const float* bias = sB + l * kWidth;
            float part = 0.0f;
            // accumulator columns 16 at a time; the next 16 are requested
            // before the current 16 are processed (one wait per block)
            uint32_t v[2][16];
            tmem_ld16_issue(t_row, v[0]);
            tmem_ld_wait(v[0]);
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                if (cb + 1 < 4) tmem_ld16_issue(t_row + 16 * (cb + 1), v[(cb + 1) & 1]);
                const int col0 = 64 * cq + 16 * cb;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    float h[8], bb[8];
                    ld8(bias + col0 + 8 * hh, bb);
#pragma unroll
                    for (int q = 0; q < 8; ++q) h[q] = silu_f(__uint_as_float(v[cb & 1][8 * hh + q]) + bb[q]);
                    if (l < 2) {
                        st16(sA + op_off(r_ep, col0 + 8 * hh), h);
                    } else {  // output layer: FP32 dot with the bfloat16-rounded activations
                        float w4[8];
                        ld8(sW4 + col0 + 8 * hh, w4);
#pragma unroll
                        for (int q = 0; q < 8; ++q) part += w4[q] * __bfloat162float(__float2bfloat16_rn(h[q]));
                    }
                }
                if (cb + 1 < 4) tmem_ld_wait(v[(cb + 1) & 1]);
            }
            if (l == 2) {
                if (cq > 0) ypart[(cq - 1) * kTM + r_ep] = part;
                __syncthreads();
                if (cq == 0 && row0 + r_ep < rows)
                    y[row0 + r_ep] = part + ypart[r_ep] + ypart[kTM + r_ep] + ypart[2 * kTM + r_ep] + sb4[0];
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();  // accumulator read and operands written before the next MMA
        }
        if (*stop) {
            for (int r = tid; r < kTM; r += kThr)
                if (row0 + r < rows) y[row0 + r] = __int_as_float(0x7fc00000);
            if (tid == 0) atomicAdd(&g_tc_timeouts, 1u);
            break;
        }
    }
    if (tid == 0 && w_issued > w_seen) {  // no copy left in flight into this CTA's shared memory
        bool wok = false;
        for (unsigned it = 0; it < kPolls && !wok; ++it) wok = bar_try(wbar_a, w_seen & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

}  // namespace

cudaError_t forward_fused(int rows, const float* x, const float* box, const float* P, const __nv_bfloat16* P16,
                          __nv_bfloat16* packed, float* y, cudaStream_t s)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) {
            sms = 0;
            return e;
        }
    }
    if (rows <= 0) return cudaSuccess;
    const int tiles = (rows + kTM - 1) / kTM;
    k_pack_weights<<<(3 * kWidth * kWidth / 8 + 255) / 256, 256, 0, s>>>(P16, packed);
    k_mlp_fused<<<tiles < sms ? tiles : sms, kThr, kSmem, s>>>(rows, x, box, P, packed, y);
    return cudaGetLastError();
}

cudaError_t forward_fused_timeouts(unsigned* count, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(count, g_tc_timeouts, sizeof(unsigned));
    if (e == cudaSuccess && reset) {
        const unsigned z = 0;
        e = cudaMemcpyToSymbol(g_tc_timeouts, &z, sizeof(unsigned));
    }
    return e;
}

}  // namespace mlp
}  // namespace hjm
