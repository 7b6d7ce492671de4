// C ABI of libhjm (declared in include/hjm.h): argument validation, grouping
// of batch items by grid shape and scheme, device workspaces, the step
// sequence of each scheme (Douglas; the Craig-Sneyd family's two stages),
// CUDA-graph capture of the time march, read-out and error reporting.
//
// Host code here validates and marshals only; every arithmetic step of the
// method (set-up tables, terminal field, the march, the read-out) runs in the
// kernels of hjm_setup.cu and hjm_march.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hjm_kernels.cuh"
#include "hjm_mlp.cuh"

using namespace hjm;

// ----------------------------------------------------------------- errors

static thread_local std::string g_last_error;

static hjm_status fail(hjm_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define CU_TRY(expr)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? HJM_ENOMEM : HJM_ECUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

extern "C" const char* hjm_status_string(hjm_status s)
{
    switch (s) {
    case HJM_OK: return "ok";
    case HJM_EINVAL: return "invalid argument";
    case HJM_ENOMEM: return "out of memory";
    case HJM_ECUDA: return "CUDA error";
    case HJM_ETOL: return "tolerance missed";
    case HJM_ETIMEOUT: return "device wait timed out";
    case HJM_ENUMERIC: return "non-finite result";
    case HJM_ERANGE: return "size out of supported range";
    }
    return "unknown status";
}

extern "C" const char* hjm_last_error(void) { return g_last_error.c_str(); }

// Error reporting for the other translation units of the library.
hjm_status hjm_internal_fail(hjm_status s, const char* msg) { return fail(s, "%s", msg); }

// ------------------------------------------------------------- validation

static bool finite_all(std::initializer_list<double> xs)
{
    for (double x : xs)
        if (!isfinite(x)) return false;
    return true;
}

static hjm_status validate(const hjm_curve& c, const hjm_model_params& m, const hjm_grid_spec& g,
                           const hjm_instrument* in, size_t elem)
{
    if (!finite_all({c.flat_rate, c.beta0, c.beta1, c.beta2, c.tau, m.kappa, m.lambda, m.gamma,
                     m.theta, m.epsilon, m.rho, m.v0, g.r_min, g.r_max, g.y_max, g.v_max, g.alpha_r,
                     g.alpha_y, g.alpha_v, g.k_r, g.k_v, g.theta_adi}))
        return fail(HJM_EINVAL, "non-finite curve, model or grid parameter");
    if (c.kind != HJM_CURVE_FLAT && c.kind != HJM_CURVE_NELSON_SIEGEL && c.kind != HJM_CURVE_KNOTS)
        return fail(HJM_EINVAL, "unknown curve kind %d", c.kind);
    if (c.kind == HJM_CURVE_NELSON_SIEGEL && !(c.tau > 0.0))
        return fail(HJM_EINVAL, "Nelson-Siegel tau must be > 0");
    double r00 = c.kind == HJM_CURVE_FLAT ? c.flat_rate : c.beta0 + c.beta1;  // f(0,0)
    if (c.kind == HJM_CURVE_KNOTS) {
        if (c.n_knots < 1 || c.n_knots > HJM_MAX_KNOTS)
            return fail(HJM_EINVAL, "n_knots must be in [1, %d]", HJM_MAX_KNOTS);
        for (int i = 0; i < c.n_knots; ++i) {
            if (!isfinite(c.knot_t[i]) || !isfinite(c.knot_P[i]) || !(c.knot_P[i] > 0.0))
                return fail(HJM_EINVAL, "knot %d: non-finite maturity or non-positive discount factor", i);
            if (!(c.knot_t[i] > (i ? c.knot_t[i - 1] : 0.0)))
                return fail(HJM_EINVAL, "knot maturities must be positive and increasing");
        }
        KnotCurve kc;
        kc.n = c.n_knots;
        memcpy(kc.t, c.knot_t, sizeof kc.t);
        memcpy(kc.P, c.knot_P, sizeof kc.P);
        knot_build(kc);
        double s0, ds0, d2s0;
        knot_eval(kc, 0.0, s0, ds0, d2s0);
        r00 = -ds0;
    }
    if (g.n_r < 5 || g.n_v < 5 || g.n_y < 5) return fail(HJM_EINVAL, "each axis needs >= 5 nodes");
    if ((long long)g.n_r * g.n_v * g.n_y > 0x7fffffffLL)
        return fail(HJM_ERANGE, "n_r * n_v * n_y above 2^31 - 1 nodes");  // 32-bit offsets in the kernels
    if (g.n_steps < 1) return fail(HJM_EINVAL, "n_steps must be >= 1");
    if (!(g.r_max > g.r_min) || !(g.y_max > 0.0) || !(g.v_max > 0.0))
        return fail(HJM_EINVAL, "empty domain");
    if (m.gamma < 0.0 || m.gamma > 1.0) return fail(HJM_EINVAL, "gamma must be in [0,1]");
    if (m.gamma > 0.0 && g.r_min != 0.0) return fail(HJM_EINVAL, "gamma > 0 needs r_min = 0");
    if (m.rho < -1.0 || m.rho > 1.0) return fail(HJM_EINVAL, "rho must be in [-1,1]");
    if (m.kappa < 0.0 || m.lambda < 0.0 || m.epsilon < 0.0 || m.theta < 0.0)
        return fail(HJM_EINVAL, "kappa, lambda, epsilon, theta must be >= 0");
    if (m.v0 < 0.0 || m.v0 > g.v_max) return fail(HJM_EINVAL, "v0 outside [0, v_max]");
    if (g.theta_adi < 0.0 || g.theta_adi > 1.0) return fail(HJM_EINVAL, "theta_adi outside [0,1]");
    if (g.y_boundary_order != 1 && g.y_boundary_order != 2)
        return fail(HJM_EINVAL, "y_boundary_order must be 1 or 2");
    if (g.explicit_midpoint != 0 && g.explicit_midpoint != 1)
        return fail(HJM_EINVAL, "explicit_midpoint must be 0 or 1");
    if (g.scheme < HJM_SCHEME_DOUGLAS || g.scheme > HJM_SCHEME_HV)
        return fail(HJM_EINVAL, "unknown scheme %d", g.scheme);
    if (!(r00 >= g.r_min && r00 <= g.r_max)) return fail(HJM_EINVAL, "f(0,0) outside [r_min, r_max]");
    if (pass1_chunk(g.n_r) == 0) return fail(HJM_ERANGE, "n_r = %d above 512", g.n_r);
    if (elem) {
        const int lim = max_strided_len(elem, m.gamma > 0.0);
        if (g.n_v > lim || g.n_y > lim)
            return fail(HJM_ERANGE, "n_v, n_y must be <= %d for this precision", lim);
    }
    if (in) {
        if (!finite_all({in->expiry_T, in->pay_TM, in->strike_K}))
            return fail(HJM_EINVAL, "non-finite instrument field");
        if (in->kind != HJM_ZCB && in->kind != HJM_CAPLET && in->kind != HJM_FLOORLET)
            return fail(HJM_EINVAL, "unknown instrument kind %d", in->kind);
        if (!(in->expiry_T > 0.0)) return fail(HJM_EINVAL, "expiry must be > 0");
        if (in->kind != HJM_ZCB && !(in->pay_TM > in->expiry_T))
            return fail(HJM_EINVAL, "caplet and floorlet need pay_TM > expiry_T");
    }
    return HJM_OK;
}

static InstParams to_params(const hjm_batch_item& it)
{
    InstParams p;
    memset(&p, 0, sizeof p);
    p.ckind = it.curve.kind;
    p.flat = it.curve.flat_rate;
    p.b0 = it.curve.beta0;
    p.b1 = it.curve.beta1;
    p.b2 = it.curve.beta2;
    p.tau = it.curve.tau;
    p.kc.n = it.curve.kind == HJM_CURVE_KNOTS ? it.curve.n_knots : 0;
    memcpy(p.kc.t, it.curve.knot_t, sizeof p.kc.t);
    memcpy(p.kc.P, it.curve.knot_P, sizeof p.kc.P);
    p.kappa = it.model.kappa;
    p.lambda = it.model.lambda;
    p.gamma = it.model.gamma;
    p.theta = it.model.theta;
    p.eps = it.model.epsilon;
    p.rho = it.model.rho;
    p.v0 = it.model.v0;
    p.nr = it.grid.n_r;
    p.nv = it.grid.n_v;
    p.ny = it.grid.n_y;
    p.nsteps = it.grid.n_steps;
    p.rmin = it.grid.r_min;
    p.rmax = it.grid.r_max;
    p.ymax = it.grid.y_max;
    p.vmax = it.grid.v_max;
    p.ar = it.grid.alpha_r;
    p.ay = it.grid.alpha_y;
    p.av = it.grid.alpha_v;
    p.kr = it.grid.k_r;
    p.kv = it.grid.k_v;
    p.center_on_strike = it.grid.center_r_on_strike;
    p.theta_adi = it.grid.theta_adi;
    p.yorder = it.grid.y_boundary_order;
    p.midpoint = it.grid.explicit_midpoint;
    p.scheme = it.grid.scheme;
    p.kind = it.inst.kind;
    p.T = it.inst.expiry_T;
    p.TM = it.inst.kind != HJM_ZCB ? it.inst.pay_TM : it.inst.expiry_T;
    p.K = it.inst.strike_K;
    p.atm_rel = it.inst.strike_atm_relative != 0;
    return p;
}

// ---------------------------------------------------------- device context

namespace {

struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need)
    {
        if (need <= bytes) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&ptr, need);
        if (e == cudaSuccess) bytes = need;
        return e;
    }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

// Cached batch graphs, keyed by precision, shapes and buffer addresses.

struct Workspace {
    Buffer block;                     // fields + tables of all groups
    std::map<std::string, cudaGraphExec_t> graphs;
    std::set<std::string> seen;       // batch keys launched once without a graph
    void drop_graphs()
    {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
        seen.clear();
    }
    void release()
    {
        drop_graphs();
        block.release();
    }
};

std::mutex g_mu;
std::map<cudaStream_t, Workspace*> g_ws;  // batch workspaces, one per stream
bool g_init_done = false;
cudaStream_t g_capture_stream = nullptr;
constexpr int kBranches = 8;  // streams the shape groups of a batch graph fork onto
cudaStream_t g_branch[kBranches];
std::vector<cudaEvent_t> g_events;

// Launch shapes per grid shape (n_r, n_v, n_y, element size), set by
// hjm_tile_set or hjm_autotune; shapes without an entry use default_tile.
std::map<std::tuple<int, int, int, size_t>, Tile> g_tiles;

Tile tile_for(int nr, int nv, int ny, size_t elem)
{
    auto it = g_tiles.find(std::make_tuple(nr, nv, ny, elem));
    return it != g_tiles.end() ? it->second : default_tile(nr, nv, ny, elem);
}

hjm_status ensure_init()
{
    if (g_init_done) return HJM_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(HJM_ECUDA, "no CUDA device");
    CU_TRY(init_kernels());
    CU_TRY(cudaStreamCreateWithFlags(&g_capture_stream, cudaStreamNonBlocking));
    for (int q = 0; q < kBranches; ++q) CU_TRY(cudaStreamCreateWithFlags(&g_branch[q], cudaStreamNonBlocking));
    g_init_done = true;
    return HJM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Group {
    int nr, nv, ny, nsteps;
    int scheme = HJM_SCHEME_DOUGLAS;  // the same for every instrument of the group
    std::vector<size_t> idx;  // positions in the caller's item array
    bool gpos = false;
    bool theta0 = false;  // some instrument has theta = 0 (no TMA-fed pass 1)
    Tile tile{};
    GroupTables t{};
    void* U = nullptr;
    void* A = nullptr;
    void* Y = nullptr;  // Craig-Sneyd family: the first stage's result Y3
    // MIXED's escalation march (FP32 increments on an FP64 state): the FP64
    // state, the FP32 remainder field, a zero field, and the Dirichlet data
    // in FP64 and as their FP32 remainder
    void* U64 = nullptr;
    void* D = nullptr;
    void* Z = nullptr;
    void* dir64 = nullptr;
    void* dirlo = nullptr;
    double* prices = nullptr;
    double* ind = nullptr;     // rounding indicators
    double* greeks = nullptr;  // [2 B]: dC/dr, dC/dv at the read-out point
};

// ------------------------------------------------------------ tracing

bool g_trace_on = false;
hjm_trace g_trace;
std::vector<cudaEvent_t> g_ev_pool;
std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> g_ev_pending;

// Event pair around one launch of kind `kind` (only while tracing).
struct TraceScope {
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    static cudaEvent_t take()
    {
        if (!g_ev_pool.empty()) {
            cudaEvent_t e = g_ev_pool.back();
            g_ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    TraceScope(int k, cudaStream_t st) : kind(k), s(st)
    {
        if (!g_trace_on || k < 0) return;  // k < 0: never traced
        a = take();
        b = take();
        cudaEventRecord(a, s);
    }
    ~TraceScope()
    {
        if (!a) return;
        cudaEventRecord(b, s);
        g_ev_pending.push_back({kind, {a, b}});
    }
};

// Called after the stream is synchronised: fold pending event pairs in.
void trace_collect()
{
    for (auto& p : g_ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
            g_trace.launches[p.first] += 1;
            g_trace.total_ms[p.first] += ms;
        }
        g_ev_pool.push_back(p.second.first);
        g_ev_pool.push_back(p.second.second);
    }
    g_ev_pending.clear();
}

// One stage of step n: pass 1 from U (and, for a correction stage, the first
// stage's result Y) into A, then out = base + the v and y solves of A.
template <typename T>
hjm_status adi_stage(const March<T>& P, const T* U, const T* Y, T* A, const T* base, T* out, bool gpos,
                     const Tile& tile, int n, cudaStream_t s, bool trace)
{
    {
        TraceScope ts(trace ? 2 : -1, s);
        CU_TRY(launch_pass1<T>(P, U, Y, A, n, tile, s));
    }
    if (tile.p2_P == 0 && !gpos) {  // passes 2 and 3 fused (traced as pass 3)
        TraceScope ts(trace ? 4 : -1, s);
        CU_TRY(launch_pass23<T>(P, A, base, out, n, s));
        return HJM_OK;
    }
    {
        TraceScope ts(trace ? 3 : -1, s);
        CU_TRY(launch_pass2<T>(P, A, A, s));
    }
    {
        TraceScope ts(trace ? 4 : -1, s);
        CU_TRY(launch_pass3<T>(P, A, base, out, gpos, n, s));
    }
    return HJM_OK;
}

// One ADI step n in place on U (scheme as in hjm.h): Douglas is one stage
// into U; the Craig-Sneyd family runs the Douglas stage into Y (Y3), then
// the correction stage from U and Y into U (base U for CS and MCS, Y3 for
// HV). trace: event pairs around the launches while tracing is enabled.
template <typename T>
hjm_status adi_step(const March<T>& P, int scheme, T* U, T* A, T* Y, bool gpos, const Tile& tile, int n,
                    cudaStream_t s, bool trace)
{
    if (scheme == HJM_SCHEME_DOUGLAS) return adi_stage<T>(P, U, nullptr, A, U, U, gpos, tile, n, s, trace);
    hjm_status st = adi_stage<T>(P, U, nullptr, A, U, Y, gpos, tile, n, s, trace);
    if (st != HJM_OK) return st;
    return adi_stage<T>(P, U, Y, A, scheme == HJM_SCHEME_HV ? Y : U, U, gpos, tile, n, s, trace);
}

template <typename T>
hjm_status run_steps(const Group& g, int n_from, int n_to, cudaStream_t s)
{
    const March<T> P = march_args<T>(g.t);
    for (int n = n_from; n < n_to; ++n) {
        hjm_status st = adi_step<T>(P, g.scheme, (T*)g.U, (T*)g.A, (T*)g.Y, g.gpos, g.tile, n, s, true);
        if (st != HJM_OK) return st;
    }
    return HJM_OK;
}

hjm_status run_steps_any(const Group& g, size_t elem, int n_from, int n_to, cudaStream_t s)
{
    return elem == sizeof(float) ? run_steps<float>(g, n_from, n_to, s)
                                 : run_steps<double>(g, n_from, n_to, s);
}

// Set-up, terminal field, the n_steps x 3 passes and the read-out of one
// group, in order on stream s.
hjm_status group_sequence(const Group& g, size_t elem, cudaStream_t s)
{
    {
        TraceScope ts(0, s);
        CU_TRY(launch_setup(g.t, elem, s));
    }
    {
        TraceScope ts(1, s);
        CU_TRY(launch_terminal(g.t, g.U, elem, s));
    }
    hjm_status st = run_steps_any(g, elem, 0, g.nsteps, s);
    if (st != HJM_OK) return st;
    TraceScope ts(5, s);
    CU_TRY(launch_readout(g.t, g.U, elem, g.prices, g.ind, g.greeks, s));
    return HJM_OK;
}

// MIXED's escalation march of one Douglas group, FP32 increments on an FP64
// state: each step splits U^n = hi + lo (hi its FP32 rounding, lo the FP32
// remainder), runs the FP32 Douglas step on hi (with the FP32 Dirichlet
// data) and on lo (with the data's FP32 remainder), each increment written
// on its own (added to a zero field), and adds both to U^n in FP64. The step
// is linear in (U^n, data), so hi + lo gives the step of U^n; the FP32
// kernels see hi's neighbour differences exactly, and the state no longer
// carries an FP32 rounding per step. About three FP32 steps of traffic.
hjm_status group_sequence_x64(const Group& g, cudaStream_t s)
{
    const long long N = (long long)g.nr * g.nv * g.ny * g.t.B;
    const long long F = (long long)g.t.B * g.nsteps * 2 * g.ny;
    CU_TRY(launch_setup(g.t, sizeof(float), s));
    CU_TRY(launch_faces64(g.t, (double*)g.dir64, s));
    CU_TRY(launch_split64((const double*)g.dir64, (float*)g.t.dir, (float*)g.dirlo, F, s));
    CU_TRY(launch_terminal(g.t, g.U64, sizeof(double), s));
    CU_TRY(cudaMemsetAsync(g.Z, 0, (size_t)N * sizeof(float), s));
    const March<float> P = march_args<float>(g.t);
    March<float> Plo = P;
    Plo.dir = (const float*)g.dirlo;
    float* hi = (float*)g.U;
    float* lo = (float*)g.D;
    float* A = (float*)g.A;
    const float* Z = (const float*)g.Z;
    for (int n = 0; n < g.nsteps; ++n) {
        CU_TRY(launch_split64((const double*)g.U64, hi, lo, N, s));
        hjm_status st = adi_stage<float>(P, hi, nullptr, A, Z, hi, g.gpos, g.tile, n, s, true);
        if (st != HJM_OK) return st;
        st = adi_stage<float>(Plo, lo, nullptr, A, Z, lo, g.gpos, g.tile, n, s, true);
        if (st != HJM_OK) return st;
        CU_TRY(launch_update64((double*)g.U64, hi, lo, N, s));
    }
    CU_TRY(launch_readout(g.t, g.U64, sizeof(double), g.prices, g.ind, g.greeks, s, true));
    return HJM_OK;
}

// The whole batch as one CUDA-graph launch: every shape group is a branch of
// the graph (fork from one node, join into one), so groups of different
// sizes run concurrently and fill the GPU together. Captured the second time
// a set of shapes, launch shapes and buffers is seen, then replayed (the
// first time the launches go straight to the stream).
hjm_status batch_graph(Workspace& ws, const std::vector<Group>& groups, size_t elem, cudaStream_t s)
{
    std::string key = std::to_string(elem);
    for (const auto& g : groups) {
        char buf[240];
        snprintf(buf, sizeof buf, "|%d,%d,%d,%d,%d,%d,%d,%p,%p,%p,%p,%d.%d.%d.%d.%d.%d.%d", g.nr, g.nv, g.ny,
                 g.nsteps, g.t.B, (int)g.gpos, g.scheme, g.U, g.A, g.Y, g.t.rt, g.tile.p1_S, g.tile.p1_M,
                 g.tile.p1_R, g.tile.p2_P, g.tile.p3_P, g.tile.p1_stage, g.tile.p1_J);
        key += buf;
    }
    auto it = ws.graphs.find(key);
    if (it == ws.graphs.end() && ws.seen.insert(key).second) {
        // First sighting of this batch: launch it directly (groups one after
        // another on s). Capturing and instantiating a graph costs more than
        // one launch sequence, and a batch whose make-up changes on every
        // call (the surrogate's fallback rows, calibration loops) would pay
        // that each time; a batch seen again is captured and replayed.
        if (ws.seen.size() > 1024) ws.seen.clear();
        for (const auto& g : groups) {
            hjm_status st = group_sequence(g, elem, s);
            if (st != HJM_OK) return st;
        }
        return HJM_OK;
    }
    if (it == ws.graphs.end()) {
        if (ws.graphs.size() > 64) ws.drop_graphs();
        while (g_events.size() < groups.size() + 1) {
            cudaEvent_t e;
            CU_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            g_events.push_back(e);
        }
        cudaGraph_t graph = nullptr;
        cudaStream_t cs = g_capture_stream;
        CU_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        hjm_status st = HJM_OK;
        cudaError_t e = cudaEventRecord(g_events[0], cs);
        for (size_t q = 0; q < groups.size() && st == HJM_OK && e == cudaSuccess; ++q) {
            cudaStream_t bs = g_branch[q % kBranches];
            e = cudaStreamWaitEvent(bs, g_events[0], 0);
            if (e != cudaSuccess) break;
            st = group_sequence(groups[q], elem, bs);
            if (st != HJM_OK) break;
            e = cudaEventRecord(g_events[q + 1], bs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, g_events[q + 1], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st != HJM_OK || e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (st != HJM_OK) return st;
            CU_TRY(e != cudaSuccess ? e : e2);
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CU_TRY(e);
        it = ws.graphs.emplace(key, exec).first;
    }
    CU_TRY(cudaGraphLaunch(it->second, s));
    return HJM_OK;
}

__global__ void k_scatter(const double* src, const long long* idx, int n, double* dst)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[idx[t]] = src[t];
}

// Pairs: dst[2 idx[t] + c] = src[2 t + c].
__global__ void k_scatter2(const double* src, const long long* idx, int n, double* dst)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        dst[2 * idx[t]] = src[2 * t];
        dst[2 * idx[t] + 1] = src[2 * t + 1];
    }
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Plan the groups of a batch and carve their buffers out of the workspace.
hjm_status plan(Workspace& ws, const hjm_batch_item* items, size_t n, size_t elem,
                std::vector<Group>& groups, InstParams** d_params, long long** d_idx,
                double** d_prices_all, double** d_ind_all = nullptr, double** d_greeks_all = nullptr,
                bool x64 = false)
{
    // Groups hold at most kMaxGroup instruments (the set-up kernels index
    // instruments with the grid's y dimension).
    constexpr size_t kMaxGroup = 65535;
    std::map<std::tuple<int, int, int, int, int>, size_t> where;
    for (size_t i = 0; i < n; ++i) {
        const hjm_grid_spec& g = items[i].grid;
        auto key = std::make_tuple(g.n_r, g.n_v, g.n_y, g.n_steps, g.scheme);
        auto f = where.find(key);
        if (f != where.end() && groups[f->second].idx.size() >= kMaxGroup) {
            where.erase(f);
            f = where.end();
        }
        if (f == where.end()) {
            Group gr;
            gr.nr = g.n_r;
            gr.nv = g.n_v;
            gr.ny = g.n_y;
            gr.nsteps = g.n_steps;
            gr.scheme = g.scheme;
            f = where.emplace(key, groups.size()).first;
            groups.push_back(gr);
        }
        Group& gr = groups[f->second];
        if (gr.idx.empty()) gr.tile = tile_for(gr.nr, gr.nv, gr.ny, elem);
        gr.idx.push_back(i);
        gr.gpos = gr.gpos || items[i].model.gamma > 0.0;
        gr.theta0 = gr.theta0 || !(items[i].grid.theta_adi > 0.0);
    }
    size_t bytes = align256(n * sizeof(InstParams)) + align256(n * sizeof(long long)) +
                   4 * align256(n * sizeof(double)) + 2 * align256(2 * n * sizeof(double));
    for (auto& g : groups) {
        const size_t B = g.idx.size();
        const size_t N = (size_t)g.nr * g.nv * g.ny;
        bytes += (g.scheme != HJM_SCHEME_DOUGLAS ? 3 : 2) * align256(B * N * elem) +
                 tables_bytes(g.nr, g.nv, g.ny, g.nsteps, (int)B, elem);
        if (x64) {
            const size_t F = B * g.nsteps * 2 * g.ny;
            bytes += align256(B * N * 8) + 2 * align256(B * N * 4) + align256(F * 8) + align256(F * 4);
        }
    }
    const void* old = ws.block.ptr;
    cudaError_t e = ws.block.ensure(bytes);
    if (e != cudaSuccess)
        return fail(HJM_ENOMEM, "device workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    if (ws.block.ptr != old) ws.drop_graphs();
    char* p = (char*)ws.block.ptr;
    *d_params = (InstParams*)p;
    p += align256(n * sizeof(InstParams));
    *d_idx = (long long*)p;
    p += align256(n * sizeof(long long));
    *d_prices_all = (double*)p;
    p += align256(n * sizeof(double));
    double* group_prices = (double*)p;
    p += align256(n * sizeof(double));
    if (d_ind_all) *d_ind_all = (double*)p;
    p += align256(n * sizeof(double));
    double* group_ind = (double*)p;
    p += align256(n * sizeof(double));
    if (d_greeks_all) *d_greeks_all = (double*)p;
    p += align256(2 * n * sizeof(double));
    double* group_greeks = (double*)p;
    p += align256(2 * n * sizeof(double));
    size_t off = 0;
    for (auto& g : groups) {
        const size_t B = g.idx.size();
        const size_t N = (size_t)g.nr * g.nv * g.ny;
        g.U = p;
        p += align256(B * N * elem);
        g.A = p;
        p += align256(B * N * elem);
        g.Y = nullptr;
        if (g.scheme != HJM_SCHEME_DOUGLAS) {
            g.Y = p;
            p += align256(B * N * elem);
        }
        g.U64 = g.D = g.Z = g.dir64 = g.dirlo = nullptr;
        if (x64) {
            const size_t F = B * g.nsteps * 2 * g.ny;
            g.U64 = p;
            p += align256(B * N * 8);
            g.D = p;
            p += align256(B * N * 4);
            g.Z = p;
            p += align256(B * N * 4);
            g.dir64 = p;
            p += align256(F * 8);
            g.dirlo = p;
            p += align256(F * 4);
        }
        g.t.nr = g.nr;
        g.t.nv = g.nv;
        g.t.ny = g.ny;
        g.t.nsteps = g.nsteps;
        g.t.B = (int)B;
        g.t.p2P = g.tile.p2_P;
        g.t.p3P = g.tile.p3_P;
        g.t.tma_ok = !g.gpos && !g.theta0;
        g.t.params = *d_params + off;
        g.prices = group_prices + off;
        g.ind = group_ind + off;
        g.greeks = group_greeks + 2 * off;
        tables_carve(g.t, p, elem);
        p += tables_bytes(g.nr, g.nv, g.ny, g.nsteps, (int)B, elem);
        off += B;
    }
    return HJM_OK;
}

Workspace* stream_workspace(cudaStream_t s)
{
    auto it = g_ws.find(s);
    if (it != g_ws.end()) return it->second;
    Workspace* w = new Workspace();
    g_ws[s] = w;
    return w;
}

// Enqueue set-up, march and read-out of a whole batch in one precision on
// stream s. On return *d_prices and *d_ind (device, caller order, inside the
// workspace) will hold the prices and rounding indicators once the stream
// reaches them. Caller holds g_mu and has validated the items.
// x64: MIXED's escalation march (FP32 increments on an FP64 state, Douglas
// items only; elem is then sizeof(float)), groups in turn, no graph.
hjm_status march_batch(Workspace& ws, const hjm_batch_item* items, size_t n, size_t elem,
                       cudaStream_t s, double** d_prices_out, double** d_ind_out, double** d_greeks_out = nullptr,
                       bool x64 = false)
{
    std::vector<Group> groups;
    InstParams* d_params;
    long long* d_idx;
    double* d_prices;
    double* d_ind;
    double* d_greeks;
    hjm_status st = plan(ws, items, n, elem, groups, &d_params, &d_idx, &d_prices, &d_ind, &d_greeks, x64);
    if (st != HJM_OK) return st;
    // Parameters in group order, and the scatter map back to caller order.
    std::vector<InstParams> hp;
    std::vector<long long> order;
    hp.reserve(n);
    order.reserve(n);
    for (auto& g : groups)
        for (size_t i : g.idx) {
            hp.push_back(to_params(items[i]));
            order.push_back((long long)i);
        }
    CU_TRY(cudaMemcpyAsync(d_params, hp.data(), n * sizeof(InstParams), cudaMemcpyHostToDevice, s));
    CU_TRY(cudaMemcpyAsync(d_idx, order.data(), n * sizeof(long long), cudaMemcpyHostToDevice, s));
    if (x64) {
        for (auto& g : groups) {
            st = group_sequence_x64(g, s);
            if (st != HJM_OK) return st;
        }
    } else if (g_trace_on) {
        for (auto& g : groups) {
            st = group_sequence(g, elem, s);
            if (st != HJM_OK) return st;
        }
    } else {
        st = batch_graph(ws, groups, elem, s);
        if (st != HJM_OK) return st;
    }
    // group order -> caller order
    k_scatter<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(groups[0].prices, d_idx, (int)n, d_prices);
    CU_TRY(cudaGetLastError());
    k_scatter<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(groups[0].ind, d_idx, (int)n, d_ind);
    CU_TRY(cudaGetLastError());
    if (d_greeks_out) {
        k_scatter2<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(groups[0].greeks, d_idx, (int)n, d_greeks);
        CU_TRY(cudaGetLastError());
        *d_greeks_out = d_greeks;
    }
    *d_prices_out = d_prices;
    *d_ind_out = d_ind;
    return HJM_OK;
}

// HJM_ETIMEOUT (and the count cleared) when a bounded device-side wait of
// the march gave up since the last check.
static hjm_status check_waits()
{
    unsigned n = 0, l = 0;
    CU_TRY(pass1t_timeouts(&n, false));
    CU_TRY(lines_t_timeouts(&l, false));
    if (n == 0 && l == 0) return HJM_OK;
    CU_TRY(pass1t_timeouts(&n, true));
    CU_TRY(lines_t_timeouts(&l, true));
    if (n) return fail(HJM_ETIMEOUT, "%u CTA(s) of the TMA-fed pass 1 gave up waiting for a plane copy", n);
    return fail(HJM_ETIMEOUT, "%u warp(s) of the TMA-fed strided passes gave up waiting for a line tile", l);
}

// Core of hjm_price_batch (caller holds g_mu, items validated).
//  FP32 / FP64: one march in that precision.
//  MIXED: the FP32 march; every instrument whose rounding indicator exceeds
//  max(tol_rel |p|, 1e-6) (or whose price is not finite; every instrument
//  when tol_rel = 0) is priced again, Douglas items first by the escalation
//  march (FP32 increments on an FP64 state) and, where that bound still
//  misses, like the Craig-Sneyd family, in FP64; they are reported as
//  escalated. MIXED synchronises the stream.
hjm_status price_batch(Workspace& ws, const hjm_batch_item* items, size_t n, hjm_precision prec,
                       double tol_rel, double* prices_out, hjm_price_info* infos, cudaStream_t s)
{
    const size_t elem = prec == HJM_FP64 ? sizeof(double) : sizeof(float);
    const bool dev_out = is_device_ptr(prices_out);
    const bool sync = !dev_out || infos != nullptr || prec == HJM_MIXED || g_trace_on;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (infos) {
        CU_TRY(cudaEventCreate(&ev0));
        CU_TRY(cudaEventCreate(&ev1));
        CU_TRY(cudaEventRecord(ev0, s));
    }
    double *d_prices, *d_ind, *d_greeks = nullptr;
    hjm_status st = march_batch(ws, items, n, elem, s, &d_prices, &d_ind, infos ? &d_greeks : nullptr);
    if (st != HJM_OK) return st;
    std::vector<double> hp, hi, hg;
    if (infos) {
        hg.resize(2 * n);
        CU_TRY(cudaMemcpyAsync(hg.data(), d_greeks, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    std::vector<int> used(n, prec == HJM_FP64 ? HJM_FP64 : HJM_FP32), esc(n, 0);
    if (sync) {
        hp.resize(n);
        hi.resize(n);
        CU_TRY(cudaMemcpyAsync(hp.data(), d_prices, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaMemcpyAsync(hi.data(), d_ind, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        if (g_trace_on) trace_collect();
        st = check_waits();
        if (st != HJM_OK) return st;
    }
    if (prec == HJM_MIXED) {
        auto misses = [&](double p, double ind) { return !isfinite(p) || !(ind <= fmax(tol_rel * fabs(p), 1e-6)); };
        // first the escalation march for the Douglas items that miss
        std::vector<hjm_batch_item> mid;
        std::vector<size_t> at;
        for (size_t i = 0; i < n; ++i)
            if ((tol_rel == 0.0 || misses(hp[i], hi[i])) && items[i].grid.scheme == HJM_SCHEME_DOUGLAS) {
                mid.push_back(items[i]);
                at.push_back(i);
            }
        if (!mid.empty()) {
            double* d_gm = nullptr;
            st = march_batch(ws, mid.data(), mid.size(), sizeof(float), s, &d_prices, &d_ind, infos ? &d_gm : nullptr,
                             true);
            if (st != HJM_OK) return st;
            std::vector<double> pm(mid.size()), im(mid.size()), gm(infos ? 2 * mid.size() : 0);
            CU_TRY(cudaMemcpyAsync(pm.data(), d_prices, mid.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaMemcpyAsync(im.data(), d_ind, mid.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            if (infos)
                CU_TRY(cudaMemcpyAsync(gm.data(), d_gm, 2 * mid.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaStreamSynchronize(s));
            if (g_trace_on) trace_collect();
            st = check_waits();
            if (st != HJM_OK) return st;
            for (size_t q = 0; q < mid.size(); ++q) {
                const size_t i = at[q];
                hp[i] = pm[q];
                hi[i] = im[q];
                used[i] = HJM_MIXED;
                esc[i] = 1;
                if (infos) {
                    hg[2 * i] = gm[2 * q];
                    hg[2 * i + 1] = gm[2 * q + 1];
                }
            }
        }
        // then FP64 for what still misses (and the Craig-Sneyd family)
        std::vector<hjm_batch_item> redo;
        std::vector<size_t> where;
        for (size_t i = 0; i < n; ++i) {
            const bool first = !(used[i] == HJM_MIXED);
            if (first ? (tol_rel == 0.0 || misses(hp[i], hi[i])) : misses(hp[i], hi[i])) {
                redo.push_back(items[i]);
                where.push_back(i);
            }
        }
        if (!redo.empty()) {
            double* d_g64 = nullptr;
            st = march_batch(ws, redo.data(), redo.size(), sizeof(double), s, &d_prices, &d_ind,
                             infos ? &d_g64 : nullptr);
            if (st != HJM_OK) return st;
            std::vector<double> p64(redo.size()), i64(redo.size()), g64(infos ? 2 * redo.size() : 0);
            CU_TRY(cudaMemcpyAsync(p64.data(), d_prices, redo.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaMemcpyAsync(i64.data(), d_ind, redo.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            if (infos)
                CU_TRY(cudaMemcpyAsync(g64.data(), d_g64, 2 * redo.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                       s));
            CU_TRY(cudaStreamSynchronize(s));
            if (g_trace_on) trace_collect();
            for (size_t q = 0; q < redo.size(); ++q) {
                hp[where[q]] = p64[q];
                hi[where[q]] = i64[q];
                used[where[q]] = HJM_FP64;
                esc[where[q]] = 1;
                if (infos) {
                    hg[2 * where[q]] = g64[2 * q];
                    hg[2 * where[q] + 1] = g64[2 * q + 1];
                }
            }
        }
    }
    if (infos) CU_TRY(cudaEventRecord(ev1, s));
    if (sync) {
        if (dev_out)
            CU_TRY(cudaMemcpyAsync(prices_out, hp.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        else
            memcpy(prices_out, hp.data(), n * sizeof(double));
    } else {
        CU_TRY(cudaMemcpyAsync(prices_out, d_prices, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (infos) {
        CU_TRY(cudaEventSynchronize(ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        for (size_t i = 0; i < n; ++i) {
            infos[i].precision_used = used[i];
            infos[i].escalated = esc[i];
            infos[i].err_estimate = hi[i];
            infos[i].n_steps = items[i].grid.n_steps;
            infos[i].time_us = ms * 1000.f;
            infos[i].d_dr = hg[2 * i];
            infos[i].d_dv = hg[2 * i + 1];
            {
                const hjm_grid_spec& gs = items[i].grid;
                const Tile t = tile_for(gs.n_r, gs.n_v, gs.n_y, used[i] == HJM_FP64 ? sizeof(double) : sizeof(float));
                infos[i].tile_cfg =
                    t.p1_S | t.p1_M << 8 | t.p1_R << 14 | t.p2_P << 21 | t.p3_P << 25 | t.p1_stage << 29;
            }
        }
    }
    if (sync) {
        if (dev_out) CU_TRY(cudaStreamSynchronize(s));  // hp is a local buffer
        for (size_t i = 0; i < n; ++i)
            if (!isfinite(hp[i])) return fail(HJM_ENUMERIC, "item %zu: price is not finite", i);
        if (prec == HJM_MIXED)
            for (size_t i = 0; i < n; ++i)
                if (!(hi[i] <= fmax(tol_rel * fabs(hp[i]), 1e-6)))
                    return fail(HJM_ETOL, "item %zu: indicator %.3g above tolerance after escalation", i, hi[i]);
    }
    return HJM_OK;
}

}  // namespace

// ------------------------------------------------------------------- grids

struct hjm_grid {
    hjm_curve curve;
    hjm_model_params model;
    hjm_grid_spec spec;
    cudaStream_t stream;
    Workspace ws;
};

extern "C" hjm_status hjm_grid_create(const hjm_curve* curve, const hjm_model_params* model,
                                      const hjm_grid_spec* spec, void* cuda_stream, hjm_grid** out)
{
    if (!curve || !model || !spec || !out) return fail(HJM_EINVAL, "null argument");
    *out = nullptr;
    hjm_status st = validate(*curve, *model, *spec, nullptr, 0);
    if (st != HJM_OK) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    st = ensure_init();
    if (st != HJM_OK) return st;
    hjm_grid* g = new (std::nothrow) hjm_grid();
    if (!g) return fail(HJM_ENOMEM, "host allocation");
    g->curve = *curve;
    g->model = *model;
    g->spec = *spec;
    g->stream = (cudaStream_t)cuda_stream;
    *out = g;
    return HJM_OK;
}

extern "C" hjm_status hjm_grid_destroy(hjm_grid* grid)
{
    if (!grid) return HJM_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStreamSynchronize(grid->stream);
    grid->ws.release();
    delete grid;
    return HJM_OK;
}

static hjm_batch_item grid_item(const hjm_grid* g, const hjm_instrument* inst)
{
    hjm_batch_item it;
    it.curve = g->curve;
    it.model = g->model;
    it.grid = g->spec;
    it.inst = *inst;
    return it;
}

extern "C" hjm_status hjm_price(hjm_grid* grid, const hjm_instrument* inst, hjm_precision precision,
                                double tol_rel, double* price_out, hjm_price_info* info_out)
{
    if (!grid || !inst || !price_out) return fail(HJM_EINVAL, "null argument");
    if (precision != HJM_FP64 && precision != HJM_FP32 && precision != HJM_MIXED)
        return fail(HJM_EINVAL, "unknown precision %d", (int)precision);
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    const hjm_batch_item it = grid_item(grid, inst);
    st = validate(it.curve, it.model, it.grid, &it.inst,
                  precision == HJM_FP64 ? sizeof(double) : sizeof(float));
    if (st != HJM_OK) return st;
    if (precision == HJM_MIXED) {
        st = validate(it.curve, it.model, it.grid, &it.inst, sizeof(double));
        if (st != HJM_OK) return st;
    }
    double p = 0.0;
    st = price_batch(grid->ws, &it, 1, precision, tol_rel, &p, info_out, grid->stream);
    if (st != HJM_OK) return st;
    *price_out = p;
    return HJM_OK;
}

extern "C" hjm_status hjm_price_batch(const hjm_batch_item* items, size_t n, hjm_precision precision,
                                      double tol_rel, double* prices_out, hjm_price_info* infos_out,
                                      void* cuda_stream)
{
    if (n == 0) return HJM_OK;
    if (!items || !prices_out) return fail(HJM_EINVAL, "null argument");
    if (precision != HJM_FP64 && precision != HJM_FP32 && precision != HJM_MIXED)
        return fail(HJM_EINVAL, "unknown precision %d", (int)precision);
    if (!(tol_rel >= 0.0)) return fail(HJM_EINVAL, "tol_rel must be >= 0");
    // MIXED may re-run any item in FP64, so it must fit the FP64 kernels too.
    const size_t elem = precision == HJM_FP32 ? sizeof(float) : sizeof(double);
    for (size_t i = 0; i < n; ++i) {
        hjm_status st = validate(items[i].curve, items[i].model, items[i].grid, &items[i].inst, elem);
        if (st != HJM_OK) {
            std::string why = g_last_error;
            return fail(st, "item %zu: %s", i, why.c_str());
        }
    }
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    return price_batch(*stream_workspace(s), items, n, precision, tol_rel, prices_out, infos_out, s);
}

// ------------------------------------------------------- caps and floors

// Field by field (the struct has padding after its ints).
static bool same_curve(const hjm_curve& a, const hjm_curve& b)
{
    if (a.kind != b.kind || a.flat_rate != b.flat_rate || a.beta0 != b.beta0 || a.beta1 != b.beta1 ||
        a.beta2 != b.beta2 || a.tau != b.tau || a.n_knots != b.n_knots)
        return false;
    for (int k = 0; k < a.n_knots && k < HJM_MAX_KNOTS; ++k)
        if (a.knot_t[k] != b.knot_t[k] || a.knot_P[k] != b.knot_P[k]) return false;
    return true;
}

extern "C" hjm_status hjm_price_strip(const hjm_batch_item* items, size_t n, hjm_precision precision,
                                      double tol_rel, double* strip_price, double* item_prices,
                                      void* cuda_stream)
{
    if (!items || !strip_price || n == 0) return fail(HJM_EINVAL, "null argument or empty strip");
    const hjm_instrument& f = items[0].inst;
    if (f.kind != HJM_CAPLET && f.kind != HJM_FLOORLET)
        return fail(HJM_EINVAL, "a strip holds caplets (a cap) or floorlets (a floor)");
    const double tenor = f.pay_TM - f.expiry_T;
    for (size_t i = 0; i < n; ++i) {
        const hjm_batch_item& it = items[i];
        if (it.inst.kind != f.kind || it.inst.strike_atm_relative != 0 || it.inst.strike_K != f.strike_K)
            return fail(HJM_EINVAL, "strip item %zu: one kind and one absolute strike", i);
        if (!same_curve(it.curve, items[0].curve) || memcmp(&it.model, &items[0].model, sizeof it.model) != 0)
            return fail(HJM_EINVAL, "strip item %zu: the curve and the model of the strip", i);
        const double ti = it.inst.pay_TM - it.inst.expiry_T;
        if (fabs(ti - tenor) > 1e-12 * fmax(1.0, tenor))
            return fail(HJM_EINVAL, "strip item %zu: the tenor of the strip", i);
        if (i > 0 && fabs(it.inst.expiry_T - items[i - 1].inst.pay_TM) > 1e-12 * fmax(1.0, it.inst.expiry_T))
            return fail(HJM_EINVAL, "strip item %zu does not start where item %zu ends", i, i - 1);
    }
    std::vector<double> p(n);
    hjm_status st = hjm_price_batch(items, n, precision, tol_rel, p.data(), nullptr, cuda_stream);
    if (st != HJM_OK) return st;
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) {
        s += p[i];
        if (item_prices) item_prices[i] = p[i];
    }
    *strip_price = s;
    return HJM_OK;
}

// ---------------------------------------------------------- launch shapes

static bool tile_precision(hjm_precision precision, size_t& elem)
{
    if (precision != HJM_FP64 && precision != HJM_FP32 && precision != HJM_MIXED) return false;
    elem = precision == HJM_FP64 ? sizeof(double) : sizeof(float);
    return true;
}

static Tile from_abi(const hjm_tile& t)
{
    return Tile{t.p1_lanes, t.p1_nodes, t.p1_lines, t.p2_warps, t.p3_warps, t.p1_staged, t.p1_planes};
}

extern "C" hjm_status hjm_tile_get(int n_r, int n_v, int n_y, hjm_precision precision, hjm_tile* out)
{
    size_t elem;
    if (!out) return fail(HJM_EINVAL, "null argument");
    if (!tile_precision(precision, elem)) return fail(HJM_EINVAL, "unknown precision %d", (int)precision);
    if (n_r < 4 || n_v < 4 || n_y < 4) return fail(HJM_EINVAL, "node counts must be >= 4");
    std::lock_guard<std::mutex> lk(g_mu);
    const Tile t = tile_for(n_r, n_v, n_y, elem);
    *out = hjm_tile{t.p1_S, t.p1_M, t.p1_R, t.p2_P, t.p3_P, t.p1_stage, t.p1_J};
    return HJM_OK;
}

extern "C" hjm_status hjm_tile_set(int n_r, int n_v, int n_y, hjm_precision precision, const hjm_tile* tile)
{
    size_t elem;
    if (!tile_precision(precision, elem)) return fail(HJM_EINVAL, "unknown precision %d", (int)precision);
    if (n_r < 4 || n_v < 4 || n_y < 4) return fail(HJM_EINVAL, "node counts must be >= 4");
    std::lock_guard<std::mutex> lk(g_mu);
    const auto key = std::make_tuple(n_r, n_v, n_y, elem);
    if (!tile) {
        g_tiles.erase(key);
        return HJM_OK;
    }
    const Tile t = from_abi(*tile);
    if (!tile_valid(t, n_r, n_v, n_y, elem))
        return fail(HJM_EINVAL, "tile (%d, %d, %d, %d, %d, %d, %d) is not available for %d x %d x %d", t.p1_S,
                    t.p1_M, t.p1_R, t.p2_P, t.p3_P, t.p1_stage, t.p1_J, n_r, n_v, n_y);
    g_tiles[key] = t;
    return HJM_OK;
}

// Pass-1 shapes to try: every compiled shape that covers the r line without
// more than doubling it (padding rows are identity rows, wasted work).
static std::vector<Tile> pass1_candidates(int nr, int nv, int ny, size_t elem, const Tile& base)
{
    std::vector<Tile> out;
    int cover = 1 << 30;  // fewest nodes of a compiled shape that covers n_r
    for (int S : {8, 16, 32})
        for (int M : {2, 4, 8, 16}) {
            Tile t = base;
            t.p1_S = S;
            t.p1_M = M;
            if (tile_valid(t, nr, nv, ny, elem)) cover = std::min(cover, S * M);
        }
    for (int S : {8, 16, 32})
        for (int M : {2, 4, 8, 16}) {
            if (S * M > std::max(2 * nr + 32, cover)) continue;
            for (int R : {2, 4, 8}) {  // rows from global memory
                Tile t = base;
                t.p1_S = S;
                t.p1_M = M;
                t.p1_R = R;
                t.p1_stage = 0;
                t.p1_J = 0;
                if (tile_valid(t, nr, nv, ny, elem)) out.push_back(t);
            }
            for (int R : {1, 2})  // staged y planes
                for (int J : {8, 16, 32}) {
                    Tile t = base;
                    t.p1_S = S;
                    t.p1_M = M;
                    t.p1_R = R;
                    t.p1_stage = 1;
                    t.p1_J = J;
                    if (tile_valid(t, nr, nv, ny, elem)) out.push_back(t);
                }
        }
    // y planes staged by TMA (FP32; the launcher falls back to the default
    // rows-from-memory shape for groups the kernel does not cover)
    int cover2 = 1 << 30;
    for (int S : {4, 8, 16, 32})
        for (int M : {8, 12, 16}) {
            Tile t = base;
            t.p1_S = S;
            t.p1_M = M;
            t.p1_R = 1;
            t.p1_stage = 3;
            t.p1_J = 0;
            if (tile_valid(t, nr, nv, ny, elem)) cover2 = std::min(cover2, S * M);
        }
    for (int S : {4, 8, 16, 32})
        for (int M : {8, 12, 16}) {
            if (S * M > std::max(nr + nr / 4, cover2)) continue;
            for (int R : {1, 2}) {
                for (int J : {0, 16}) {  // persistent balanced grid, runs of 16 planes
                    Tile t = base;
                    t.p1_S = S;
                    t.p1_M = M;
                    t.p1_R = R;
                    t.p1_stage = J == 0 ? 3 : 2;
                    t.p1_J = J;
                    if (tile_valid(t, nr, nv, ny, elem)) out.push_back(t);
                }
            }
        }
    return out;
}

// Device time of each pass over `ns` Douglas steps of group g with its
// current tile (set-up and terminal field re-run first: the split factors
// depend on the tile).
template <typename T>
static hjm_status time_passes(Group& g, int ns, cudaStream_t s, cudaEvent_t* ev, float ms[3])
{
    const size_t elem = sizeof(T);
    g.t.p2P = g.tile.p2_P;
    g.t.p3P = g.tile.p3_P;
    CU_TRY(launch_setup(g.t, elem, s));
    CU_TRY(launch_terminal(g.t, g.U, elem, s));
    const March<T> P = march_args<T>(g.t);
    T* U = (T*)g.U;
    T* A = (T*)g.A;
    // A Craig-Sneyd-family group also runs the correction-stage pass 1 (from
    // U^n and Y3; Y3 = U^n here, the values do not change the timing), so
    // its pass-1 time is that of both kinds of launch.
    T* Y = g.scheme != HJM_SCHEME_DOUGLAS ? (T*)g.Y : nullptr;
    if (Y)
        CU_TRY(cudaMemcpyAsync(Y, U, (size_t)g.t.B * g.nr * g.nv * g.ny * sizeof(T), cudaMemcpyDeviceToDevice,
                               s));
    ms[0] = ms[1] = ms[2] = 0.f;
    for (int n = -1; n < ns; ++n) {  // n = -1: untimed warm-up step
        const int sn = n < 0 ? 0 : n;
        CU_TRY(cudaEventRecord(ev[0], s));
        CU_TRY(launch_pass1<T>(P, U, nullptr, A, sn, g.tile, s));
        if (Y) CU_TRY(launch_pass1<T>(P, U, Y, A, sn, g.tile, s));
        CU_TRY(cudaEventRecord(ev[1], s));
        if (g.tile.p2_P == 0 && !g.gpos) {
            CU_TRY(cudaEventRecord(ev[2], s));
            CU_TRY(launch_pass23<T>(P, A, U, U, sn, s));
        } else {
            CU_TRY(launch_pass2<T>(P, A, A, s));
            CU_TRY(cudaEventRecord(ev[2], s));
            CU_TRY(launch_pass3<T>(P, A, U, U, g.gpos, sn, s));
        }
        CU_TRY(cudaEventRecord(ev[3], s));
        CU_TRY(cudaEventSynchronize(ev[3]));
        if (n < 0) continue;
        for (int q = 0; q < 3; ++q) {
            float t = 0.f;
            CU_TRY(cudaEventElapsedTime(&t, ev[q], ev[q + 1]));
            ms[q] += t;
        }
    }
    return HJM_OK;
}

extern "C" hjm_status hjm_autotune(const hjm_batch_item* items, size_t n, hjm_precision precision, int steps,
                                   void* cuda_stream)
{
    size_t elem;
    if (n == 0) return HJM_OK;
    if (!items) return fail(HJM_EINVAL, "null argument");
    if (!tile_precision(precision, elem)) return fail(HJM_EINVAL, "unknown precision %d", (int)precision);
    if (steps < 1 || steps > 1000) return fail(HJM_EINVAL, "steps must be in [1, 1000]");
    for (size_t i = 0; i < n; ++i) {
        hjm_status st = validate(items[i].curve, items[i].model, items[i].grid, &items[i].inst, elem);
        if (st != HJM_OK) {
            std::string why = g_last_error;
            return fail(st, "item %zu: %s", i, why.c_str());
        }
    }
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Workspace& ws = *stream_workspace(s);
    // The batch's instruments by grid shape; each shape is timed on its own
    // instruments, all marching with the first one's step count.
    std::map<std::tuple<int, int, int>, std::vector<hjm_batch_item>> shapes;
    for (size_t i = 0; i < n; ++i)
        shapes[std::make_tuple(items[i].grid.n_r, items[i].grid.n_v, items[i].grid.n_y)].push_back(items[i]);
    struct Events {
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events()
        {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evs;
    for (auto& e : evs.e) CU_TRY(cudaEventCreate(&e));
    for (auto& kv : shapes) {
        std::vector<hjm_batch_item>& v = kv.second;
        for (auto& it : v) it.grid.n_steps = v[0].grid.n_steps;
        const int ns = std::min(steps, v[0].grid.n_steps);
        const int nr = std::get<0>(kv.first), nv = std::get<1>(kv.first), ny = std::get<2>(kv.first);
        std::vector<Group> groups;
        InstParams* d_params;
        long long* d_idx;
        double* d_prices;
        st = plan(ws, v.data(), v.size(), elem, groups, &d_params, &d_idx, &d_prices);
        if (st != HJM_OK) return st;
        std::vector<InstParams> hp;
        for (auto& g : groups)
            for (size_t i : g.idx) hp.push_back(to_params(v[i]));
        CU_TRY(cudaMemcpyAsync(d_params, hp.data(), hp.size() * sizeof(InstParams), cudaMemcpyHostToDevice, s));
        Group& g = groups[0];
        Tile best = default_tile(nr, nv, ny, elem);
        // Pass 1 shapes (passes 2 and 3 at their defaults), then the line
        // splits of passes 2 and 3 (pass 1 at its best): each pass keeps the
        // fastest of its own options, best of two timings; last, passes 2
        // and 3 fused, kept when faster than the two best separate passes.
        std::vector<Tile> cands = pass1_candidates(nr, nv, ny, elem, best);
        float best_ms[3] = {3.0e38f, 3.0e38f, 3.0e38f};
        for (int phase = 0; phase < 3; ++phase) {
            if (phase == 1) {
                cands.clear();
                for (int Pw : {1, 2, 4, 8}) {
                    Tile t = best;
                    t.p2_P = split_valid(nv, Pw) ? Pw : 1;
                    t.p3_P = split_valid(ny, Pw) && !g.gpos ? Pw : 1;
                    cands.push_back(t);
                }
                {  // lines moved by TMA (FP32)
                    Tile t = best;
                    t.p2_P = lines_t_valid(0, nr, nv, ny, elem) ? kLinesTma : 1;
                    t.p3_P = lines_t_valid(1, nr, nv, ny, elem) && !g.gpos ? kLinesTma : 1;
                    if (t.p2_P == kLinesTma || t.p3_P == kLinesTma) cands.push_back(t);
                }
                best_ms[1] = best_ms[2] = 3.0e38f;
            }
            if (phase == 2) {
                cands.clear();
                for (int F : {0}) {
                    Tile t = best;
                    t.p2_P = F;
                    t.p3_P = 1;
                    if (!g.gpos && tile_valid(t, nr, nv, ny, elem)) cands.push_back(t);
                }
            }
            for (const Tile& cand : cands) {
                g.tile = cand;
                float ms[3], mn[3] = {3.0e38f, 3.0e38f, 3.0e38f};
                for (int rep = 0; rep < 2; ++rep) {
                    st = elem == sizeof(float) ? time_passes<float>(g, ns, s, evs.e, ms)
                                               : time_passes<double>(g, ns, s, evs.e, ms);
                    if (st != HJM_OK) return st;
                    for (int q = 0; q < 3; ++q) mn[q] = std::min(mn[q], ms[q]);
                }
                if (phase == 0 && mn[0] < best_ms[0]) {
                    best_ms[0] = mn[0];
                    best.p1_S = cand.p1_S;
                    best.p1_M = cand.p1_M;
                    best.p1_R = cand.p1_R;
                    best.p1_stage = cand.p1_stage;
                    best.p1_J = cand.p1_J;
                }
                if (phase == 1) {
                    if (mn[1] < best_ms[1]) {
                        best_ms[1] = mn[1];
                        best.p2_P = cand.p2_P;
                    }
                    if (mn[2] < best_ms[2]) {
                        best_ms[2] = mn[2];
                        best.p3_P = cand.p3_P;
                    }
                }
                if (phase == 2 && mn[1] + mn[2] < best_ms[1] + best_ms[2]) {
                    best_ms[1] = mn[1];
                    best_ms[2] = mn[2];
                    best.p2_P = cand.p2_P;
                    best.p3_P = 1;
                }
            }
        }
        g_tiles[std::make_tuple(nr, nv, ny, elem)] = best;
    }
    return HJM_OK;
}

// ---------------------------------------------------------- stepwise access

// Set up one instrument on the grid's workspace (tables + terminal field).
static hjm_status setup_one(hjm_grid* grid, const hjm_instrument* inst, hjm_precision prec,
                            std::vector<Group>& groups, size_t& elem)
{
    if (prec == HJM_MIXED) return fail(HJM_EINVAL, "stepwise access needs FP32 or FP64");
    elem = prec == HJM_FP32 ? sizeof(float) : sizeof(double);
    hjm_status st = validate(grid->curve, grid->model, grid->spec, inst, elem);
    if (st != HJM_OK) return st;
    const hjm_batch_item it = grid_item(grid, inst);
    InstParams* d_params;
    long long* d_idx;
    double* d_prices;
    st = plan(grid->ws, &it, 1, elem, groups, &d_params, &d_idx, &d_prices);
    if (st != HJM_OK) return st;
    const InstParams hp = to_params(it);
    CU_TRY(cudaMemcpyAsync(d_params, &hp, sizeof hp, cudaMemcpyHostToDevice, grid->stream));
    CU_TRY(launch_setup(groups[0].t, elem, grid->stream));
    return HJM_OK;
}

extern "C" hjm_status hjm_field(hjm_grid* grid, const hjm_instrument* inst, hjm_precision precision,
                                int n_run, void* field_out)
{
    if (!grid || !inst || !field_out) return fail(HJM_EINVAL, "null argument");
    if (n_run < 0 || n_run > grid->spec.n_steps) return fail(HJM_EINVAL, "n_run outside [0, n_steps]");
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    std::vector<Group> groups;
    size_t elem;
    st = setup_one(grid, inst, precision, groups, elem);
    if (st != HJM_OK) return st;
    const Group& g = groups[0];
    CU_TRY(launch_terminal(g.t, g.U, elem, grid->stream));
    st = run_steps_any(g, elem, 0, n_run, grid->stream);
    if (st != HJM_OK) return st;
    const size_t bytes = (size_t)g.nr * g.nv * g.ny * elem;
    CU_TRY(cudaMemcpyAsync(field_out, g.U, bytes, cudaMemcpyDefault, grid->stream));
    CU_TRY(cudaStreamSynchronize(grid->stream));
    return HJM_OK;
}

extern "C" hjm_status hjm_axis(hjm_grid* grid, const hjm_instrument* inst, int axis, double* z_out,
                               double* J_out, double* J2_out)
{
    if (!grid || !inst || !z_out || !J_out || !J2_out) return fail(HJM_EINVAL, "null argument");
    if (axis < 0 || axis > 2) return fail(HJM_EINVAL, "axis must be 0, 1 or 2");
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    std::vector<Group> groups;
    size_t elem;
    st = setup_one(grid, inst, HJM_FP64, groups, elem);
    if (st != HJM_OK) return st;
    const Group& g = groups[0];
    const int n = axis == 0 ? g.nr : (axis == 1 ? g.nv : g.ny);
    const double* src = axis == 0 ? g.t.axr : (axis == 1 ? g.t.axv : g.t.axy);
    CU_TRY(cudaMemcpyAsync(z_out, src, n * sizeof(double), cudaMemcpyDeviceToHost, grid->stream));
    CU_TRY(cudaMemcpyAsync(J_out, src + n, n * sizeof(double), cudaMemcpyDeviceToHost, grid->stream));
    CU_TRY(cudaMemcpyAsync(J2_out, src + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, grid->stream));
    CU_TRY(cudaStreamSynchronize(grid->stream));
    return HJM_OK;
}

extern "C" hjm_status hjm_douglas_pass(hjm_grid* grid, const hjm_instrument* inst,
                                       hjm_precision precision, int pass, int step_n, const void* in,
                                       const void* in2, void* out)
{
    if (!grid || !inst || !in || !out) return fail(HJM_EINVAL, "null argument");
    if (pass < 1 || pass > 4) return fail(HJM_EINVAL, "pass must be 1, 2, 3 or 4");
    if (pass == 3 && !in2) return fail(HJM_EINVAL, "pass 3 needs U^n");
    if (pass == 4 && (!in2 || grid->spec.scheme == HJM_SCHEME_DOUGLAS))
        return fail(HJM_EINVAL, "pass 4 needs Y3 and a Craig-Sneyd-family scheme");
    if (step_n < 0 || step_n >= grid->spec.n_steps) return fail(HJM_EINVAL, "step outside [0, n_steps)");
    if ((pass == 1 || pass == 4) && (in == out || in2 == out))
        return fail(HJM_EINVAL, "pass %d cannot run in place", pass);
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    std::vector<Group> groups;
    size_t elem;
    st = setup_one(grid, inst, precision, groups, elem);
    if (st != HJM_OK) return st;
    const Group& g = groups[0];
    cudaStream_t s = grid->stream;
    if (elem == sizeof(float)) {
        const March<float> P = march_args<float>(g.t);
        if (pass == 1 || pass == 4)
            CU_TRY(launch_pass1<float>(P, (const float*)in, pass == 4 ? (const float*)in2 : nullptr, (float*)out,
                                       step_n, g.tile, s));
        if (pass == 2) CU_TRY(launch_pass2<float>(P, (const float*)in, (float*)out, s));
        if (pass == 3)
            CU_TRY(launch_pass3<float>(P, (const float*)in, (const float*)in2, (float*)out, g.gpos, step_n, s));
    } else {
        const March<double> P = march_args<double>(g.t);
        if (pass == 1 || pass == 4)
            CU_TRY(launch_pass1<double>(P, (const double*)in, pass == 4 ? (const double*)in2 : nullptr,
                                        (double*)out, step_n, g.tile, s));
        if (pass == 2) CU_TRY(launch_pass2<double>(P, (const double*)in, (double*)out, s));
        if (pass == 3)
            CU_TRY(launch_pass3<double>(P, (const double*)in, (const double*)in2, (double*)out, g.gpos, step_n, s));
    }
    CU_TRY(cudaStreamSynchronize(s));
    return HJM_OK;
}

extern "C" hjm_status hjm_wait_status(int reset)
{
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    CU_TRY(cudaDeviceSynchronize());
    unsigned n = 0, l = 0, m = 0;
    CU_TRY(pass1t_timeouts(&n, reset != 0));
    CU_TRY(lines_t_timeouts(&l, reset != 0));
    CU_TRY(mlp::forward_fused_timeouts(&m, reset != 0));
    if (n) return fail(HJM_ETIMEOUT, "%u CTA(s) of the TMA-fed pass 1 gave up waiting for a plane copy", n);
    if (l) return fail(HJM_ETIMEOUT, "%u warp(s) of the TMA-fed strided passes gave up waiting for a line tile", l);
    if (m) return fail(HJM_ETIMEOUT, "%u CTA(s) of the fused surrogate forward gave up waiting for the tensor cores", m);
    return HJM_OK;
}

extern "C" hjm_status hjm_test_drop_plane(int plane, unsigned polls)
{
    if (plane < -1) return fail(HJM_EINVAL, "plane must be >= -1");
    std::lock_guard<std::mutex> lk(g_mu);
    hjm_status st = ensure_init();
    if (st != HJM_OK) return st;
    CU_TRY(cudaDeviceSynchronize());
    const unsigned lim = plane < 0 || polls == 0 ? (1u << 22) : polls;
    CU_TRY(pass1t_test_drop(plane, lim));
    CU_TRY(lines_t_test_drop(plane, lim));
    return HJM_OK;
}

extern "C" hjm_status hjm_trace_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_trace_on = on != 0;
    return HJM_OK;
}

extern "C" hjm_status hjm_trace_read(hjm_trace* out, int reset)
{
    if (!out) return fail(HJM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(g_mu);
    *out = g_trace;
    if (reset) memset(&g_trace, 0, sizeof g_trace);
    return HJM_OK;
}

// ------------------------------------------------- allocation-free pricing
//
// hjm_price_static (declared in hjm.h): the whole march of one instrument in
// a file-scope device array, for callers that cannot allocate device memory
// (device memory owned by another allocator or a fixed pool, latency-critical
// loops that cannot take cudaMalloc's implicit synchronisation). Nothing here allocates; the array is reserved when the library's
// module is loaded on a device and lives until the process exits.

static __device__ __align__(256) unsigned char g_static_scratch[HJM_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kStaticMaxDevices = 64;
void* g_static_addr[kStaticMaxDevices];  // device address of g_static_scratch, per device
std::mutex g_static_mu;

template <typename T>
hjm_status static_march(const GroupTables& t, int scheme, void* U, void* A, void* Y, int nsteps, bool gpos,
                        const Tile& tile, cudaStream_t s)
{
    const March<T> P = march_args<T>(t);
    for (int n = 0; n < nsteps; ++n) {
        hjm_status st = adi_step<T>(P, scheme, (T*)U, (T*)A, (T*)Y, gpos, tile, n, s, false);
        if (st != HJM_OK) return st;
    }
    return HJM_OK;
}
}  // namespace

extern "C" hjm_status hjm_price_static(const hjm_batch_item* item, hjm_precision precision,
                                       double* price_out, void* cuda_stream)
{
    if (!item || !price_out) return fail(HJM_EINVAL, "null argument");
    if (precision != HJM_FP32 && precision != HJM_FP64)
        return fail(HJM_EINVAL, "hjm_price_static takes HJM_FP32 or HJM_FP64");
    const size_t elem = precision == HJM_FP32 ? sizeof(float) : sizeof(double);
    hjm_status st = validate(item->curve, item->model, item->grid, &item->inst, elem);
    if (st != HJM_OK) return st;
    const hjm_grid_spec& g = item->grid;
    const size_t N = (size_t)g.n_r * g.n_v * g.n_y;
    const int fields = g.scheme != HJM_SCHEME_DOUGLAS ? 3 : 2;
    const size_t need = align256(sizeof(InstParams)) + fields * align256(N * elem) +
                        tables_bytes(g.n_r, g.n_v, g.n_y, g.n_steps, 1, elem) + align256(sizeof(double));
    if (need > HJM_STATIC_SCRATCH_BYTES)
        return fail(HJM_ERANGE, "item needs %zu bytes of scratch, the static array holds %u", need,
                    (unsigned)HJM_STATIC_SCRATCH_BYTES);
    if (!is_device_ptr(price_out)) return fail(HJM_EINVAL, "price_out must be device memory");
    int dev = 0;
    CU_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(HJM_ERANGE, "device ordinal %d not supported", dev);
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            // Once per device, with that device current: the host-side name
            // of the array is not a device address, so look the address up.
            void* addr = nullptr;
            CU_TRY(cudaGetSymbolAddress(&addr, g_static_scratch));
            CU_TRY(init_kernels());
            g_static_addr[dev] = addr;
        }
        base = g_static_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    char* p = (char*)base;
    GroupTables t{};
    t.nr = g.n_r;
    t.nv = g.n_v;
    t.ny = g.n_y;
    t.nsteps = g.n_steps;
    t.B = 1;
    t.params = (InstParams*)p;
    p += align256(sizeof(InstParams));
    void* U = p;
    p += align256(N * elem);
    void* A = p;
    p += align256(N * elem);
    void* Y = nullptr;
    if (fields == 3) {
        Y = p;
        p += align256(N * elem);
    }
    tables_carve(t, p, elem);
    p += tables_bytes(g.n_r, g.n_v, g.n_y, g.n_steps, 1, elem);
    double* ind = (double*)p;
    Tile tile;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        tile = tile_for(g.n_r, g.n_v, g.n_y, elem);
    }
    t.p2P = tile.p2_P;
    t.p3P = tile.p3_P;
    t.tma_ok = item->model.gamma == 0.0 && item->grid.theta_adi > 0.0;
    // Every region above is fully rewritten by the kernels below before it
    // is read (the set-up kernel also zeroes the rounding indicator), so no
    // clearing is needed between calls.
    const InstParams hp = to_params(*item);
    CU_TRY(cudaMemcpyAsync(t.params, &hp, sizeof hp, cudaMemcpyHostToDevice, s));
    CU_TRY(launch_setup(t, elem, s));
    CU_TRY(launch_terminal(t, U, elem, s));
    const bool gpos = item->model.gamma > 0.0;
    st = elem == sizeof(float) ? static_march<float>(t, g.scheme, U, A, Y, g.n_steps, gpos, tile, s)
                               : static_march<double>(t, g.scheme, U, A, Y, g.n_steps, gpos, tile, s);
    if (st != HJM_OK) return st;
    CU_TRY(launch_readout(t, U, elem, price_out, ind, nullptr, s));
    return HJM_OK;
}
