// The pricing surrogate (not a part of the paper's method): a multilayer
// perceptron trained on caplet prices produced by this library's own FP32
// Douglas ADI march, used for fast repeated pricing (calibration loops),
// with the march as its fallback and as the reference that measures its error.
//
// Inputs x = (kappa, lambda, theta, epsilon, rho, T, delta, K, F): the model
// parameters (gamma = 0, v0 = 1), expiry T, accrual delta = T_M - T, strike
// K and the simple forward F of the curve over [T, T_M]. With gamma = 0 the
// caplet price divided by P(0,T) depends on the curve only through F. The
// forward premium C / P(0,T) splits into the Gaussian-HJM caplet (epsilon = 0:
// v stays at v0 = 1 and the model is the Gaussian one of Section 3.1, whose
// caplet is a put on the log-normal bond p(T,T_M), in closed form) and the
// stochastic-volatility correction; the network learns only the correction,
// q = (C - C_gauss) / (P(0,T) delta s_r), s_r = 1e-4, which carries the
// epsilon, rho and theta dependence at order one, and reports the forward
// premium C_gauss / P(0,T) + q delta s_r; callers multiply by their P(0,T).
// Labels and fallback prices come from the march on a flat curve with that
// forward (continuous rate c = ln(1 + F delta) / delta).
//
// Host code here draws inputs, lays out batches and drives the kernels of
// hjm_mlp.cu and the pricing path; every arithmetic step on the data runs on
// the device.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "hjm.h"
#include "hjm_mlp.cuh"

using namespace hjm::mlp;

extern "C" hjm_status hjm_price_batch(const hjm_batch_item*, size_t, hjm_precision, double, double*,
                                      hjm_price_info*, void*);
hjm_status hjm_internal_fail(hjm_status s, const char* msg);

namespace {

constexpr double kResidScale = 1e-4;  // s_r: the correction per unit accrual is at most a few 1e-4
constexpr int kBinsT = 9, kBinsK = 8, kBins = kBinsT * kBinsK;
constexpr double kGateTol = 1e-4;     // PDE-judged error accepted on C / P(0,T)
constexpr double kGateSafety = 0.5;   // a bin answers when its held-out maximum is below half of it
constexpr uint32_t kFileMagic = 0x484a4d52;  // "HJMR": a network of the residual target

hjm_status fail(hjm_status s, const char* msg) { return hjm_internal_fail(s, msg); }

#define SCU(expr)                                                              \
    do {                                                                       \
        cudaError_t e_ = (expr);                                               \
        if (e_ != cudaSuccess) {                                               \
            char b_[256];                                                      \
            snprintf(b_, sizeof b_, "%s: %s", #expr, cudaGetErrorString(e_)); \
            return fail(e_ == cudaErrorMemoryAllocation ? HJM_ENOMEM : HJM_ECUDA, b_); \
        }                                                                      \
    } while (0)

// Counter-based uniform generator (splitmix64 finaliser of seed + counter).
struct Rng {
    uint64_t seed, ctr = 0;
    double uniform()
    {
        uint64_t z = seed + 0x9e3779b97f4a7c15ULL * (++ctr);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        return (z >> 11) * (1.0 / 9007199254740992.0);
    }
};

template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t m)
    {
        if (m <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, m * sizeof(T));
        if (e == cudaSuccess) n = m;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

__global__ void k_gather_rows(int rows, const int* __restrict__ idx, const float* __restrict__ x,
                              const float* __restrict__ t, float* __restrict__ xb, float* __restrict__ tb)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int s = idx[r];
    for (int k = 0; k < kIn; ++k) xb[(size_t)r * kIn + k] = x[(size_t)s * kIn + k];
    tb[r] = t[s];
}

// Forward premium C_gauss / P(0,T) of the Gaussian-HJM caplet (gamma = 0,
// epsilon = 0, v = 1): ln p(T,T_M) is normal with standard deviation
// sp = G(delta) sqrt(Var x(T)), G(s) = (1 - e^{-kappa s}) / kappa (the bond
// formula of Section 3.1), Var x(T) = lambda^2 (1 - e^{-2 kappa T}) / (2 kappa),
// and the caplet is Delta_M = 1 + delta K times a put on p(T,T_M) with strike
// 1 / Delta_M; with P(0,T_M) / P(0,T) = 1 / (1 + F delta),
//   C_gauss / P(0,T) = N(sp - h) - Delta_M / (1 + F delta) N(-h),
//   h = ln(Delta_M / (1 + F delta)) / sp + sp / 2.
__device__ double gauss_premium(double kap, double lam, double T, double dl, double K, double F)
{
    const double G = kap > 0.0 ? -expm1(-kap * dl) / kap : dl;
    const double var = kap > 0.0 ? lam * lam * (-expm1(-2.0 * kap * T)) / (2.0 * kap) : lam * lam * T;
    const double sp = G * sqrt(var);
    const double a = (1.0 + dl * K) / (1.0 + F * dl);
    const double h = log(a) / sp + 0.5 * sp;
    return normcdf(sp - h) - a * normcdf(-h);
}

__global__ void k_gauss_premium(int rows, const float* __restrict__ x, double* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* f = x + (size_t)r * kIn;
    out[r] = gauss_premium(f[0], f[1], f[5], f[6], f[7], f[8]);
}

// Forward premium of a flat-curve caplet price: C / P(0,T), P(0,T) = e^{-cT},
// c = ln(1 + F delta) / delta; `scaled` gives the network's target instead,
// (C / P(0,T) - C_gauss / P(0,T)) / (delta s_r).
__global__ void k_forward_premium(int rows, const float* __restrict__ x, const double* __restrict__ C,
                                  float* __restrict__ qf, double* __restrict__ qd, int scaled)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* f = x + (size_t)r * kIn;
    const double T = f[5], dl = f[6], F = f[8];
    const double c = log1p(F * dl) / dl;
    double q = C[r] * exp(c * T);
    if (scaled) q = (q - gauss_premium(f[0], f[1], T, dl, f[7], F)) / (dl * kResidScale);
    if (qf) qf[r] = (float)q;
    if (qd) qd[r] = q;
}

// Network output q -> forward premium C_gauss / P(0,T) + q delta s_r (double).
__global__ void k_unscale(int rows, const float* __restrict__ x, const float* __restrict__ y,
                          double* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* f = x + (size_t)r * kIn;
    out[r] = gauss_premium(f[0], f[1], f[5], f[6], f[7], f[8]) + (double)y[r] * f[6] * kResidScale;
}

__device__ int bin_of(const float* f, const float* lo, const float* hi)
{
    // T bins over [lo5, hi5], moneyness (K - F) bins over [lo7, hi7]
    int bt = (int)floorf((f[5] - lo[5]) / (hi[5] - lo[5]) * kBinsT);
    int bk = (int)floorf((f[7] - lo[7]) / (hi[7] - lo[7]) * kBinsK);
    bt = min(max(bt, 0), kBinsT - 1);
    bk = min(max(bk, 0), kBinsK - 1);
    return bt * kBinsK + bk;
}

// Gate of one row: inside the training box, and its (T, K - F) bin's held-out
// PDE-judged error below half the tolerance (a margin for unseen rows).
__global__ void k_gate(int rows, const float* __restrict__ x, const float* __restrict__ lo,
                       const float* __restrict__ hi, const float* __restrict__ table, unsigned char* __restrict__ rej)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float f[kIn];
    for (int k = 0; k < kIn; ++k) f[k] = x[(size_t)r * kIn + k];
    f[7] -= f[8];
    bool ok = true;
    for (int k = 0; k < kIn; ++k) ok = ok && f[k] >= lo[k] && f[k] <= hi[k];
    if (ok) ok = table[bin_of(f, lo, hi)] <= (float)(kGateSafety * kGateTol);
    rej[r] = ok ? 0 : 1;
}

// Held-out errors per bin: table[bin] = max |q_net - q_pde| in C / P(0,T) units.
__global__ void k_bin_errors(int rows, const float* __restrict__ x, const float* __restrict__ lo,
                             const float* __restrict__ hi, const float* __restrict__ y, const float* __restrict__ t,
                             float* __restrict__ table, unsigned* __restrict__ count)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float f[kIn];
    for (int k = 0; k < kIn; ++k) f[k] = x[(size_t)r * kIn + k];
    f[7] -= f[8];
    const int b = bin_of(f, lo, hi);
    const float err = fabsf(y[r] - t[r]) * f[6] * (float)kResidScale;
    atomicMax(reinterpret_cast<int*>(table + b), __float_as_int(err));
    atomicAdd(count + b, 1u);
}

__global__ void k_scatter_d(int n, const int* __restrict__ idx, const double* __restrict__ src,
                            double* __restrict__ dst, unsigned char* __restrict__ flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[idx[i]] = src[i];
    if (flag) flag[idx[i]] = 1;
}

__global__ void k_empty_bins(float* table, const unsigned* count)
{
    const int b = threadIdx.x;
    if (b < kBins && count[b] == 0) table[b] = __int_as_float(0x7f800000);  // +inf: no evidence, gate off
}

}  // namespace

struct hjm_surrogate {
    hjm_surrogate_cfg cfg;
    std::string ckpt;
    std::vector<float> lo, hi;  // feature box (float)
    DBuf<float> w, m, v, g, box, table, loss;
    DBuf<__nv_bfloat16> w16;
    DBuf<__nv_bfloat16> w16p;  // W1..W3 packed for the fused inference kernel's bulk copies
    long long step = 0;
    int epoch = 0;
    Rng rng{0};
    // activations
    DBuf<float> xb, tb, Xn, Z[4], dZa, dZb, y, dy;
    DBuf<__nv_bfloat16> H[4], dZha, dZhb;
    DBuf<int> idx;
    DBuf<unsigned> cnt;
    DBuf<double> dtmp;
    DBuf<unsigned char> rej;
    // march fallback of hjm_surrogate_infer (grow-only, kept between calls)
    DBuf<float> fb_x;
    DBuf<double> fb_q;
    DBuf<int> fb_idx;
    std::mutex mu;
};

namespace {

cudaError_t ensure_acts(hjm_surrogate* s, int rows, bool train)
{
    cudaError_t e;
    const size_t R = rows;
    if ((e = s->xb.ensure(R * kIn)) || (e = s->tb.ensure(R)) || (e = s->Xn.ensure(R * kIn)) ||
        (e = s->y.ensure(R)) || (e = s->dy.ensure(R)))
        return e;
    for (int l = 0; l < 4; ++l) {
        if ((e = s->H[l].ensure(R * kWidth))) return e;
        if (train && (e = s->Z[l].ensure(R * kWidth))) return e;
    }
    if (train) {
        if ((e = s->dZa.ensure(R * kWidth)) || (e = s->dZb.ensure(R * kWidth)) || (e = s->dZha.ensure(R * kWidth)) ||
            (e = s->dZhb.ensure(R * kWidth)))
            return e;
    }
    return cudaSuccess;
}

// Network forward on `rows` raw input rows x (device) into s->y. Inference
// (keep = false) runs the fused tensor-core kernel; training keeps the
// per-layer kernels, whose pre-activations the backward pass needs.
hjm_status forward(hjm_surrogate* s, const float* x, int rows, bool keep, cudaStream_t st)
{
    if (!keep) {
        SCU(s->w16p.ensure((size_t)3 * kWidth * kWidth));
        SCU(forward_fused(rows, x, s->box.p, s->w.p, s->w16.p, s->w16p.p, s->y.p, st));
        return HJM_OK;
    }
    const float* W = s->w.p;
    const __nv_bfloat16* W16 = s->w16.p;
    const float* lo = s->box.p;
    const float* hi = s->box.p + kIn;
    SCU(layer0(rows, x, lo, hi, W + kOffW0, W + kOffB0, s->Xn.p, keep ? s->Z[0].p : nullptr, s->H[0].p, st));
    const size_t offW[3] = {kOffW1, kOffW2, kOffW3}, offB[3] = {kOffB1, kOffB2, kOffB3};
    for (int l = 1; l <= 3; ++l)
        SCU(gemm_forward(rows, s->H[l - 1].p, W16 + offW[l - 1], W + offB[l - 1], keep ? s->Z[l].p : nullptr,
                         s->H[l].p, st));
    SCU(layer4(rows, s->H[3].p, W + kOffW4, W + kOffB4, s->y.p, st));
    return HJM_OK;
}

// Loss and gradient (into s->g) of a batch already in s->xb / s->tb.
hjm_status loss_grad(hjm_surrogate* s, int rows, cudaStream_t st)
{
    hjm_status r = forward(s, s->xb.p, rows, true, st);
    if (r != HJM_OK) return r;
    float* G = s->g.p;
    const float* W = s->w.p;
    const __nv_bfloat16* W16 = s->w16.p;
    SCU(loss(rows, s->y.p, s->tb.p, s->dy.p, s->loss.p, st));
    SCU(layer4_back(rows, s->dy.p, W + kOffW4, s->Z[3].p, s->dZa.p, s->dZha.p, s->H[3].p, G + kOffW4, G + kOffB4, st));
    const size_t offW[3] = {kOffW1, kOffW2, kOffW3}, offB[3] = {kOffB1, kOffB2, kOffB3};
    float* dz = s->dZa.p;
    __nv_bfloat16* dzh = s->dZha.p;
    float* dzn = s->dZb.p;
    __nv_bfloat16* dznh = s->dZhb.p;
    for (int l = 3; l >= 1; --l) {
        SCU(gemm_weight_grad(rows, dzh, s->H[l - 1].p, G + offW[l - 1], st));
        SCU(bias_grad(rows, dz, G + offB[l - 1], st));
        SCU(gemm_input_grad(rows, dzh, W16 + offW[l - 1], s->Z[l - 1].p, dzn, dznh, st));
        std::swap(dz, dzn);
        std::swap(dzh, dznh);
    }
    SCU(layer0_back(rows, dz, s->Xn.p, G + kOffW0, G + kOffB0, st));
    return HJM_OK;
}

hjm_status valid_cfg(const hjm_surrogate_cfg* c)
{
    if (!c) return fail(HJM_EINVAL, "null surrogate configuration");
    if (c->hidden != kWidth || c->depth != 4)
        return fail(HJM_EINVAL, "the surrogate network is 4 hidden layers of width 256");
    if (c->batch < 1 || c->epochs < 0 || !(c->lr > 0.0f)) return fail(HJM_EINVAL, "batch, epochs or lr out of range");
    for (int k = 0; k < kIn; ++k)
        if (!(c->box_hi[k] > c->box_lo[k])) return fail(HJM_EINVAL, "empty input box");
    if (c->box_lo[0] < 0 || c->box_lo[1] < 0 || c->box_lo[2] < 0 || c->box_lo[3] < 0 || c->box_lo[4] < -1 ||
        c->box_hi[4] > 1 || c->box_lo[5] <= 0 || c->box_lo[6] <= 0)
        return fail(HJM_EINVAL, "input box outside the model's parameter ranges");
    return HJM_OK;
}

// Grid of one label: counts and scheme from the configuration, domain from
// the draw (r: +- 7 lambda sqrt(v_max T) around F, v: [0, max(5, 1 + 10
// epsilon / sqrt(2 theta))], y: [0, 4 lambda^2 v_max (1 - e^{-2 kappa T}) /
// (2 kappa)], sinh widths a quarter of each axis).
hjm_batch_item label_item(const hjm_surrogate_cfg& cfg, const float* x)
{
    const double kap = x[0], lam = x[1], th = x[2], eps = x[3], rho = x[4], T = x[5], dl = x[6], K = x[7],
                 F = x[8];
    hjm_batch_item it;
    memset(&it, 0, sizeof it);
    const double c = log1p(F * dl) / dl;
    it.curve.kind = HJM_CURVE_FLAT;
    it.curve.flat_rate = c;
    it.curve.tau = 1.0;
    it.model.kappa = kap;
    it.model.lambda = lam;
    it.model.gamma = 0.0;
    it.model.theta = th;
    it.model.epsilon = eps;
    it.model.rho = rho;
    it.model.v0 = 1.0;
    hjm_grid_spec g = cfg.label_grid;
    const double vmax = fmax(5.0, 1.0 + 10.0 * eps / sqrt(2.0 * fmax(th, 1e-12)));
    const double fb = fabs(c);
    const double w = 7.0 * lam * sqrt(vmax * T);
    g.r_min = fmin(0.0, -fb - w);
    g.r_max = fb + w;
    g.v_max = vmax;
    g.y_max = kap > 0 ? 4.0 * lam * lam * vmax * (-expm1(-2.0 * kap * T)) / (2.0 * kap) : 4.0 * lam * lam * vmax * T;
    g.alpha_r = 0.25 * (g.r_max - g.r_min);
    g.alpha_v = 0.25 * vmax;
    g.alpha_y = 0.25 * g.y_max;
    g.k_v = 1.0;
    g.center_r_on_strike = 1;
    it.grid = g;
    it.inst.kind = HJM_CAPLET;
    it.inst.expiry_T = T;
    it.inst.pay_TM = T + dl;
    it.inst.strike_K = K;
    it.inst.strike_atm_relative = 0;
    return it;
}

// PDE forward premia (C / P(0,T), or scaled targets) of `rows` raw inputs on
// the host, into device arrays; chunked to bound the march's memory.
hjm_status pde_targets(hjm_surrogate* s, const std::vector<float>& hx, int rows, float* d_x, float* qf, double* qd,
                       int scaled, cudaStream_t st)
{
    const int chunk = 1024;
    std::vector<hjm_batch_item> items;
    SCU(s->dtmp.ensure(chunk));
    for (int r0 = 0; r0 < rows; r0 += chunk) {
        const int n = std::min(chunk, rows - r0);
        items.clear();
        for (int i = 0; i < n; ++i) items.push_back(label_item(s->cfg, &hx[(size_t)(r0 + i) * kIn]));
        hjm_status r = hjm_price_batch(items.data(), n, HJM_FP32, 0.0, s->dtmp.p, nullptr, st);
        if (r != HJM_OK) return r;
        k_forward_premium<<<(n + 127) / 128, 128, 0, st>>>(n, d_x + (size_t)r0 * kIn, s->dtmp.p,
                                                            qf ? qf + r0 : nullptr, qd ? qd + r0 : nullptr, scaled);
        SCU(cudaGetLastError());
    }
    return HJM_OK;
}

hjm_status init_weights(hjm_surrogate* s, cudaStream_t st)
{
    // Uniform(-a, a), a = sqrt(6 / (fan_in + fan_out)); biases 0.
    std::vector<float> w(kParams, 0.0f);
    Rng r{s->cfg.seed ^ 0x5eedULL};
    auto fill = [&](size_t off, int fo, int fi) {
        const double a = sqrt(6.0 / (fi + fo));
        for (size_t i = 0; i < (size_t)fo * fi; ++i) w[off + i] = (float)((2.0 * r.uniform() - 1.0) * a);
    };
    fill(kOffW0, kWidth, kIn);
    fill(kOffW1, kWidth, kWidth);
    fill(kOffW2, kWidth, kWidth);
    fill(kOffW3, kWidth, kWidth);
    fill(kOffW4, 1, kWidth);
    SCU(cudaMemcpyAsync(s->w.p, w.data(), kParams * sizeof(float), cudaMemcpyHostToDevice, st));
    SCU(cudaMemsetAsync(s->m.p, 0, kParams * sizeof(float), st));
    SCU(cudaMemsetAsync(s->v.p, 0, kParams * sizeof(float), st));
    SCU(to_bf16(kParams, s->w.p, s->w16.p, st));
    return HJM_OK;
}

hjm_status alloc_state(hjm_surrogate* s)
{
    SCU(s->w.ensure(kParams));
    SCU(s->m.ensure(kParams));
    SCU(s->v.ensure(kParams));
    SCU(s->g.ensure(kParams));
    SCU(s->w16.ensure(kParams));
    SCU(s->box.ensure(2 * kIn));
    SCU(s->table.ensure(kBins));
    SCU(s->loss.ensure(1));
    SCU(s->cnt.ensure(kBins));
    return HJM_OK;
}

hjm_status upload_box_and_table(hjm_surrogate* s, cudaStream_t st, const float* table_host)
{
    std::vector<float> b(2 * kIn);
    for (int k = 0; k < kIn; ++k) {
        b[k] = (float)s->cfg.box_lo[k];
        b[kIn + k] = (float)s->cfg.box_hi[k];
    }
    s->lo.assign(b.begin(), b.begin() + kIn);
    s->hi.assign(b.begin() + kIn, b.end());
    SCU(cudaMemcpyAsync(s->box.p, b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    std::vector<float> t(kBins, INFINITY);
    if (table_host) t.assign(table_host, table_host + kBins);
    SCU(cudaMemcpyAsync(s->table.p, t.data(), kBins * sizeof(float), cudaMemcpyHostToDevice, st));
    SCU(cudaStreamSynchronize(st));
    return HJM_OK;
}

// One pass of minibatch AdamW over rows [0, n) of device (x, t).
hjm_status train_epochs(hjm_surrogate* s, const float* d_x, const float* d_t, int n, int epochs, long long total_steps,
                        cudaStream_t st, float* last_loss)
{
    const int B = std::min(s->cfg.batch, n);
    if (ensure_acts(s, B, true)) return fail(HJM_ENOMEM, "surrogate activations");
    std::vector<int> perm(n);
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int)(s->rng.uniform() * (i + 1)) % (i + 1)]);
        SCU(s->idx.ensure(n));
        SCU(cudaMemcpyAsync(s->idx.p, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        for (int b0 = 0; b0 + B <= n; b0 += B) {
            k_gather_rows<<<(B + 127) / 128, 128, 0, st>>>(B, s->idx.p + b0, d_x, d_t, s->xb.p, s->tb.p);
            SCU(cudaGetLastError());
            hjm_status r = loss_grad(s, B, st);
            if (r != HJM_OK) return r;
            ++s->step;
            const double frac = total_steps > 0 ? std::min(1.0, (double)s->step / total_steps) : 1.0;
            const float lr = (float)(s->cfg.lr * (0.05 + 0.95 * 0.5 * (1.0 + cos(3.14159265358979323846 * frac))));
            SCU(adamw(kParams, s->w.p, s->m.p, s->v.p, s->g.p, lr, 0.9f, 0.999f, 1e-8f, 1e-5f, s->step, s->w16.p, st));
        }
        ++s->epoch;
        float l = 0.0f;
        SCU(cudaMemcpyAsync(&l, s->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st));
        SCU(cudaStreamSynchronize(st));
        if (!isfinite(l)) return fail(HJM_ENUMERIC, "surrogate training loss is not finite");
        if (last_loss) *last_loss = l;
        if (!s->ckpt.empty()) {
            hjm_status r = hjm_surrogate_save(s, s->ckpt.c_str());
            if (r != HJM_OK) return r;
        }
    }
    return HJM_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI

extern "C" hjm_status hjm_surrogate_create(const hjm_surrogate_cfg* cfg, void* cuda_stream, hjm_surrogate** out)
{
    if (!out) return fail(HJM_EINVAL, "null argument");
    *out = nullptr;
    hjm_status r = valid_cfg(cfg);
    if (r != HJM_OK) return r;
    hjm_surrogate* s = new (std::nothrow) hjm_surrogate();
    if (!s) return fail(HJM_ENOMEM, "host allocation");
    s->cfg = *cfg;
    s->ckpt = cfg->checkpoint_path ? cfg->checkpoint_path : "";
    s->cfg.checkpoint_path = nullptr;
    s->rng.seed = cfg->seed;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if ((r = alloc_state(s)) != HJM_OK || (r = init_weights(s, st)) != HJM_OK ||
        (r = upload_box_and_table(s, st, nullptr)) != HJM_OK) {
        hjm_surrogate_destroy(s);
        return r;
    }
    *out = s;
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_destroy(hjm_surrogate* s)
{
    if (!s) return HJM_OK;
    cudaDeviceSynchronize();
    for (auto* b : {&s->w, &s->m, &s->v, &s->g, &s->box, &s->table, &s->loss, &s->xb, &s->tb, &s->Xn, &s->dZa,
                    &s->dZb, &s->y, &s->dy})
        b->release();
    for (int l = 0; l < 4; ++l) {
        s->Z[l].release();
        s->H[l].release();
    }
    s->w16.release();
    s->w16p.release();
    s->dZha.release();
    s->dZhb.release();
    s->idx.release();
    s->cnt.release();
    s->dtmp.release();
    s->rej.release();
    s->fb_x.release();
    s->fb_q.release();
    s->fb_idx.release();
    delete s;
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_get_params(const hjm_surrogate* s, float* out)
{
    if (!s || !out) return fail(HJM_EINVAL, "null argument");
    SCU(cudaMemcpy(out, s->w.p, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_set_params(hjm_surrogate* s, const float* in)
{
    if (!s || !in) return fail(HJM_EINVAL, "null argument");
    SCU(cudaMemcpy(s->w.p, in, kParams * sizeof(float), cudaMemcpyHostToDevice));
    SCU(to_bf16(kParams, s->w.p, s->w16.p, 0));
    SCU(cudaDeviceSynchronize());
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_forward(hjm_surrogate* s, const float* x, size_t n, float* y_out,
                                            void* cuda_stream)
{
    if (!s || !x || !y_out) return fail(HJM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int chunk = 65536;
    if (ensure_acts(s, (int)std::min<size_t>(n, chunk), false)) return fail(HJM_ENOMEM, "surrogate activations");
    for (size_t r0 = 0; r0 < n; r0 += chunk) {
        const int rows = (int)std::min<size_t>(chunk, n - r0);
        hjm_status r = forward(s, x + r0 * kIn, rows, false, st);
        if (r != HJM_OK) return r;
        SCU(cudaMemcpyAsync(y_out + r0, s->y.p, rows * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_premium(hjm_surrogate* s, const float* x, size_t n, double* premium_out,
                                            void* cuda_stream)
{
    if (!s || !x || !premium_out) return fail(HJM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int chunk = 65536;
    if (ensure_acts(s, (int)std::min<size_t>(n, chunk), false)) return fail(HJM_ENOMEM, "surrogate activations");
    for (size_t r0 = 0; r0 < n; r0 += chunk) {
        const int rows = (int)std::min<size_t>(chunk, n - r0);
        hjm_status r = forward(s, x + r0 * kIn, rows, false, st);
        if (r != HJM_OK) return r;
        k_unscale<<<(rows + 255) / 256, 256, 0, st>>>(rows, x + r0 * kIn, s->y.p, premium_out + r0);
        SCU(cudaGetLastError());
    }
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_gauss_premium(const float* x, size_t n, double* premium_out, void* cuda_stream)
{
    if (!x || !premium_out) return fail(HJM_EINVAL, "null argument");
    if (n == 0) return HJM_OK;
    k_gauss_premium<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>((int)n, x, premium_out);
    SCU(cudaGetLastError());
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_loss_grad(hjm_surrogate* s, const float* x, const float* t, size_t n,
                                              float* loss_out, float* grad_out, void* cuda_stream)
{
    if (!s || !x || !t || !grad_out || n == 0) return fail(HJM_EINVAL, "null argument or empty batch");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (ensure_acts(s, (int)n, true)) return fail(HJM_ENOMEM, "surrogate activations");
    SCU(cudaMemcpyAsync(s->xb.p, x, n * kIn * sizeof(float), cudaMemcpyDeviceToDevice, st));
    SCU(cudaMemcpyAsync(s->tb.p, t, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    hjm_status r = loss_grad(s, (int)n, st);
    if (r != HJM_OK) return r;
    SCU(cudaMemcpyAsync(grad_out, s->g.p, kParams * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (loss_out) {
        SCU(cudaMemcpyAsync(loss_out, s->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st));
        SCU(cudaStreamSynchronize(st));
    }
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_fit(hjm_surrogate* s, const float* x, const float* t, size_t n, int epochs,
                                        void* cuda_stream, float* final_loss)
{
    if (!s || !x || !t || n == 0 || epochs < 0) return fail(HJM_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    const long long per_epoch = (long long)(n / std::max(1, std::min(s->cfg.batch, (int)n)));
    return train_epochs(s, x, t, (int)n, epochs, s->step + per_epoch * epochs, (cudaStream_t)cuda_stream,
                        final_loss);
}

extern "C" hjm_status hjm_surrogate_train(const hjm_surrogate_cfg* cfg, void* cuda_stream, hjm_surrogate** out)
{
    if (!out) return fail(HJM_EINVAL, "null argument");
    *out = nullptr;
    hjm_status r = valid_cfg(cfg);
    if (r != HJM_OK) return r;
    if (cfg->n_train < 64) return fail(HJM_EINVAL, "n_train must be >= 64");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    hjm_surrogate* s = nullptr;
    // Resume from a checkpoint when one exists.
    if (cfg->checkpoint_path) {
        FILE* f = fopen(cfg->checkpoint_path, "rb");
        if (f) {
            fclose(f);
            r = hjm_surrogate_load(cfg->checkpoint_path, &s);
            if (r != HJM_OK) return r;
            s->ckpt = cfg->checkpoint_path;
        }
    }
    if (!s && (r = hjm_surrogate_create(cfg, cuda_stream, &s)) != HJM_OK) return r;
    const int n = (int)cfg->n_train;
    const int nhold = std::max(16, n / 16);
    const int ntr = n - nhold;
    // Draws over the box (features -> raw inputs: K = (K - F) + F). The
    // generator is counter based, so a resumed run draws the same set.
    Rng dr{cfg->seed};
    std::vector<float> hx((size_t)n * kIn);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < kIn; ++k)
            hx[(size_t)i * kIn + k] = (float)(cfg->box_lo[k] + (cfg->box_hi[k] - cfg->box_lo[k]) * dr.uniform());
        hx[(size_t)i * kIn + 7] += hx[(size_t)i * kIn + 8];
    }
    DBuf<float> dx, dt;
    if (dx.ensure((size_t)n * kIn) || dt.ensure(n)) {
        hjm_surrogate_destroy(s);
        return fail(HJM_ENOMEM, "training set");
    }
    auto cleanup = [&](hjm_status rr) {
        dx.release();
        dt.release();
        if (rr != HJM_OK) hjm_surrogate_destroy(s);
        return rr;
    };
    if (cudaMemcpyAsync(dx.p, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, st))
        return cleanup(fail(HJM_ECUDA, "upload of the training inputs"));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r = pde_targets(s, hx, n, dx.p, dt.p, nullptr, 1, st);
        if (r != HJM_OK) return cleanup(r);
        const int remaining = std::max(0, cfg->epochs - s->epoch);
        const long long total = (long long)(ntr / std::max(1, std::min(cfg->batch, ntr))) * cfg->epochs;
        r = train_epochs(s, dx.p, dt.p, ntr, remaining, total, st, nullptr);
        if (r != HJM_OK) return cleanup(r);
        // Held-out PDE-judged error table.
        if (ensure_acts(s, nhold, false)) return cleanup(fail(HJM_ENOMEM, "surrogate activations"));
        r = forward(s, dx.p + (size_t)ntr * kIn, nhold, false, st);
        if (r != HJM_OK) return cleanup(r);
        if (cudaMemsetAsync(s->table.p, 0, kBins * sizeof(float), st) ||
            cudaMemsetAsync(s->cnt.p, 0, kBins * sizeof(unsigned), st))
            return cleanup(fail(HJM_ECUDA, "error table"));
        k_bin_errors<<<(nhold + 127) / 128, 128, 0, st>>>(nhold, dx.p + (size_t)ntr * kIn, s->box.p, s->box.p + kIn,
                                                          s->y.p, dt.p + ntr, s->table.p, s->cnt.p);
        k_empty_bins<<<1, kBins, 0, st>>>(s->table.p, s->cnt.p);
        if (cudaGetLastError() || cudaStreamSynchronize(st)) return cleanup(fail(HJM_ECUDA, "error table"));
    }
    if (!s->ckpt.empty() && (r = hjm_surrogate_save(s, s->ckpt.c_str())) != HJM_OK) return cleanup(r);
    cleanup(HJM_OK);
    *out = s;
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_error_table(const hjm_surrogate* s, float* out)
{
    if (!s || !out) return fail(HJM_EINVAL, "null argument");
    SCU(cudaMemcpy(out, s->table.p, kBins * sizeof(float), cudaMemcpyDeviceToHost));
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_infer(hjm_surrogate* s, const float* x, size_t n, double* price_out,
                                          uint8_t* used_pde, void* cuda_stream)
{
    if (!s || !x || !price_out) return fail(HJM_EINVAL, "null argument");
    if (n == 0) return HJM_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int chunk = 65536;
    if (ensure_acts(s, (int)std::min<size_t>(n, chunk), false)) return fail(HJM_ENOMEM, "surrogate activations");
    SCU(s->rej.ensure(n));
    for (size_t r0 = 0; r0 < n; r0 += chunk) {
        const int rows = (int)std::min<size_t>(chunk, n - r0);
        hjm_status r = forward(s, x + r0 * kIn, rows, false, st);
        if (r != HJM_OK) return r;
        k_unscale<<<(rows + 255) / 256, 256, 0, st>>>(rows, x + r0 * kIn, s->y.p, price_out + r0);
        k_gate<<<(rows + 255) / 256, 256, 0, st>>>(rows, x + r0 * kIn, s->box.p, s->box.p + kIn, s->table.p,
                                                    s->rej.p + r0);
        SCU(cudaGetLastError());
    }
    if (used_pde) SCU(cudaMemcpyAsync(used_pde, s->rej.p, n, cudaMemcpyDeviceToDevice, st));
    // Fallback: rows outside the box or in a bin whose held-out error misses
    // the tolerance are priced by the march.
    std::vector<unsigned char> rej(n);
    SCU(cudaMemcpyAsync(rej.data(), s->rej.p, n, cudaMemcpyDeviceToHost, st));
    SCU(cudaStreamSynchronize(st));
    std::vector<int> idx;
    for (size_t i = 0; i < n; ++i)
        if (rej[i]) idx.push_back((int)i);
    if (idx.empty()) return HJM_OK;
    const int m = (int)idx.size();
    std::vector<float> hx((size_t)n * kIn);
    SCU(cudaMemcpyAsync(hx.data(), x, (size_t)n * kIn * sizeof(float), cudaMemcpyDeviceToHost, st));
    SCU(cudaStreamSynchronize(st));
    std::vector<float> sx((size_t)m * kIn);
    for (int q = 0; q < m; ++q)
        for (int k = 0; k < kIn; ++k) sx[(size_t)q * kIn + k] = hx[(size_t)idx[q] * kIn + k];
    if (s->fb_x.ensure((size_t)m * kIn) || s->fb_q.ensure(m) || s->fb_idx.ensure(m))
        return fail(HJM_ENOMEM, "fallback buffers");
    hjm_status r = HJM_OK;
    if (cudaMemcpyAsync(s->fb_x.p, sx.data(), sx.size() * sizeof(float), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(s->fb_idx.p, idx.data(), m * sizeof(int), cudaMemcpyHostToDevice, st))
        r = fail(HJM_ECUDA, "fallback upload");
    if (r == HJM_OK) r = pde_targets(s, sx, m, s->fb_x.p, nullptr, s->fb_q.p, 0, st);
    if (r == HJM_OK) {
        k_scatter_d<<<(m + 127) / 128, 128, 0, st>>>(m, s->fb_idx.p, s->fb_q.p, price_out, nullptr);
        if (cudaGetLastError() || cudaStreamSynchronize(st)) r = fail(HJM_ECUDA, "fallback scatter");
    }
    return r;
}

// File: magic, version, config (without the path), step, epoch, rng counter,
// box, table, then w, m, v (FP32).
extern "C" hjm_status hjm_surrogate_save(const hjm_surrogate* s, const char* path)
{
    if (!s || !path) return fail(HJM_EINVAL, "null argument");
    std::vector<float> w(kParams), m(kParams), v(kParams), t(kBins);
    SCU(cudaDeviceSynchronize());
    SCU(cudaMemcpy(w.data(), s->w.p, kParams * 4, cudaMemcpyDeviceToHost));
    SCU(cudaMemcpy(m.data(), s->m.p, kParams * 4, cudaMemcpyDeviceToHost));
    SCU(cudaMemcpy(v.data(), s->v.p, kParams * 4, cudaMemcpyDeviceToHost));
    SCU(cudaMemcpy(t.data(), s->table.p, kBins * 4, cudaMemcpyDeviceToHost));
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(HJM_EINVAL, "cannot open the checkpoint file for writing");
    const uint32_t magic = kFileMagic, version = 1;
    hjm_surrogate_cfg c = s->cfg;
    c.checkpoint_path = nullptr;
    bool ok = fwrite(&magic, 4, 1, f) == 1 && fwrite(&version, 4, 1, f) == 1 && fwrite(&c, sizeof c, 1, f) == 1 &&
              fwrite(&s->step, sizeof s->step, 1, f) == 1 && fwrite(&s->epoch, sizeof s->epoch, 1, f) == 1 &&
              fwrite(&s->rng.ctr, sizeof s->rng.ctr, 1, f) == 1 && fwrite(t.data(), 4, kBins, f) == (size_t)kBins &&
              fwrite(w.data(), 4, kParams, f) == kParams && fwrite(m.data(), 4, kParams, f) == kParams &&
              fwrite(v.data(), 4, kParams, f) == kParams;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) return fail(HJM_EINVAL, "writing the checkpoint failed");
    return HJM_OK;
}

extern "C" hjm_status hjm_surrogate_load(const char* path, hjm_surrogate** out)
{
    if (!path || !out) return fail(HJM_EINVAL, "null argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(HJM_EINVAL, "cannot open the checkpoint file");
    uint32_t magic = 0, version = 0;
    hjm_surrogate_cfg c;
    long long step = 0;
    int epoch = 0;
    uint64_t ctr = 0;
    std::vector<float> w(kParams), m(kParams), v(kParams), t(kBins);
    bool ok = fread(&magic, 4, 1, f) == 1 && fread(&version, 4, 1, f) == 1 && magic == kFileMagic && version == 1 &&
              fread(&c, sizeof c, 1, f) == 1 && fread(&step, sizeof step, 1, f) == 1 &&
              fread(&epoch, sizeof epoch, 1, f) == 1 && fread(&ctr, sizeof ctr, 1, f) == 1 &&
              fread(t.data(), 4, kBins, f) == (size_t)kBins && fread(w.data(), 4, kParams, f) == kParams &&
              fread(m.data(), 4, kParams, f) == kParams && fread(v.data(), 4, kParams, f) == kParams;
    fclose(f);
    if (!ok) return fail(HJM_EINVAL, "not a surrogate checkpoint (or truncated)");
    c.checkpoint_path = nullptr;
    hjm_surrogate* s = nullptr;
    hjm_status r = hjm_surrogate_create(&c, nullptr, &s);
    if (r != HJM_OK) return r;
    s->step = step;
    s->epoch = epoch;
    s->rng.ctr = ctr;
    if (cudaMemcpy(s->w.p, w.data(), kParams * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(s->m.p, m.data(), kParams * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(s->v.p, v.data(), kParams * 4, cudaMemcpyHostToDevice) ||
        to_bf16(kParams, s->w.p, s->w16.p, 0) || upload_box_and_table(s, 0, t.data())) {
        hjm_surrogate_destroy(s);
        return fail(HJM_ECUDA, "uploading the checkpoint");
    }
    *out = s;
    return HJM_OK;
}

// Tensor-core GEMM of bfloat16 operands with FP32 accumulation, exposed for
// testing the surrogate's matrix products directly.
extern "C" hjm_status hjm_mlp_gemm(int M, int N, int K, const void* A, int lda, int trans_a, const void* B, int ldb,
                                   int trans_b, float* C, int ldc, void* cuda_stream)
{
    if (!A || !B || !C || M < 0 || N < 0 || K < 0) return fail(HJM_EINVAL, "bad GEMM arguments");
    SCU(gemm_plain(M, N, K, (const __nv_bfloat16*)A, lda, trans_a != 0, (const __nv_bfloat16*)B, ldb, trans_b != 0, C,
                   ldc, (cudaStream_t)cuda_stream));
    return HJM_OK;
}
