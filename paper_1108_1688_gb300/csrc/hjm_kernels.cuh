// Internal declarations shared by the CUDA translation units of libhjm.
//
// Data layout in device memory (one "group" = instruments of equal grid
// shape that march together in the same launches; b indexes the group):
//   field    U[b][j][k][i]            i on r (fastest), k on v, j on y
//   r tables rt[b][RT_N][n_r]         per-node factors of the r operator,
//   v tables vt[b][VT_N][n_v]         with the grid spacings of the centred
//   y tables yt[b][YT_N][n_y]         differences folded in (see k_setup)
//   scalars  sc[b][SC_N]              dt, theta*dt, 1/h per axis, and the
//                                     weights of the Craig-Sneyd correction
//                                     stage (see SC_C1 ..)
//   steps    st[b][n_steps][2]        a(t) = df(0,t)/dt + kappa f(0,t) for
//                                     the explicit and the implicit stage
//   faces    dir[b][n_steps][2][n_y]  Dirichlet data at t^{n+1}, r_min/r_max
//   v LU     vf[b][3][n_v]            Thomas factors of I - theta dt A_v
//   y LU     yf[b][n_v][3][n_y]       Thomas factors of I - theta dt A_y
//                                     (gamma == 0 instruments only)
//   v split  vp[b][sys]               factors of the v system split into
//   y split  yp[b][n_v][sys]          p2P (p3P) chunks, one warp per chunk
//                                     (see part_sys_size; y: gamma == 0)
//   r folded r2[b][R2_N][n_r]         the r tables recombined for the TMA-fed
//                                     pass 1 (dt and 1/theta folded in, the
//                                     Dirichlet nodes zeroed; see R2_L ..)
//   flags    fl[b][FL_N]              r_min Dirichlet, y face order, y LU
//                                     present, read-out stencil corner (i, k)
//   indicator acc[b][n_steps] (float) max |dU3| of each step over the 4 x 4
//                                     read-out stencil on y = 0
// All tables are built in FP64 on the device and stored in the march type.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hjm.h"
#include "hjm_curve.cuh"

namespace hjm {

// Host-validated parameters of one instrument, as uploaded to the device.
struct InstParams {
    int ckind;
    double flat, b0, b1, b2, tau;
    KnotCurve kc;  // HJM_CURVE_KNOTS: knots as given, spline built by the set-up
    double kappa, lambda, gamma, theta, eps, rho, v0;
    int nr, nv, ny, nsteps;
    double rmin, rmax, ymax, vmax, ar, ay, av, kr, kv;
    int center_on_strike;
    double theta_adi;
    int yorder, midpoint;
    int scheme;  // hjm_scheme
    int kind;
    double T, TM, K;
    int atm_rel;
};

// Scalars derived on the device by the setup kernel (FP64).
struct InstDerived {
    double K;        // absolute strike
    double DM;       // Delta_M = 1 + (T_M - T) K
    double dt;       // T / n_steps
    double centre_r; // metric centre in r
};

// Safety factor of the a-posteriori rounding indicator, calibrated against
// the oracle by the precision-control tests (it must bound the measured
// FP32-march error of every tested instrument).
constexpr double kIndicatorC = 8.0;

enum { RT_R, RT_IJ, RT_C1, RT_C4V, RT_C4B, RT_C3, RT_CY, RT_N };
// Folded r tables of the TMA-fed pass 1 (gamma = 0 groups). With C1, C4V,
// IJ, C4B the RT_ factors above, z the node's rate, dt the step and theta
// the ADI weight, the kernel solves the r system divided by theta,
//   a x_{i-1} + b x_i + c x_{i+1} = dt F / theta,
//   a = s_I - v (E1 + E4),  c = -(v (E1 - E4) + s_I),  b = B + 2 v E1,
//   s_I = (a_I + y) P + Q   (a_I = a(t^{n+1/2})),
// and forms the explicit r part from the undivided second and first
// differences of U^n (no cancelling sums of large terms):
//   (dt/theta) A_r U = g1 d2U + g4 d1U + RT U,
//   g1 = (v/theta) E1,  g4 = (a_F + y)/theta P + Q/theta - (v/theta) E4.
// So P = dt IJ, Q = dt C4B, B = 1/theta + dt z, E1 = dt C1, E4 = dt C4V,
// RT = -dt z / theta (a table of its own: 1/theta - B would cancel). With
// gamma = 0 the mixed-term factor is P times the per-instrument SC_XP and
// the y-drift factor the per-instrument SC_YL, so neither is a table. The
// Dirichlet nodes (i = 0 and i = n_r - 1 when gamma = 0) carry zeros and
// B = 1, so their rows are identity rows without a branch per node.
enum { R2_P, R2_Q, R2_B, R2_E1, R2_E4, R2_RT, R2_N };
enum { VT_V, VT_IJ, VT_G2, VT_G5, VT_FV, VT_N };
enum { YT_Y, YT_IJ, YT_KY, YT_N };
// Correction stage of the Craig-Sneyd family (all explicit operators at
// t^{n+1/2}, E = Y3 - U^n the first stage's increment):
//   Z0 - B = dt (A_0 (U + E/2) + A_dir (U + c1 E)) - he E,
// with A_dir = A_r + A_v + A_y; c1 = 0 (CS), 1/2 - theta (MCS), 1/2 (HV);
// he = 1 for HV (B = Y3), 0 otherwise (B = U^n). SC_CX = 1/2 - c1 is the
// extra weight of the mixed term; on Dirichlet nodes Z0 - B = kd (g - U -
// c1 E) with kd = (1 - he) / (1 - c1) (there E = g - U^n).
// SC_ITH = 1 / theta (0 when theta = 0). SC_XP = lambda eps rho (n_v - 1) / 2
// and SC_YL = dt lambda^2: the mixed-term factor over the r table P and the
// y-drift factor of the TMA-fed pass 1 (gamma = 0).
enum { SC_DT, SC_W, SC_IHR, SC_IHV, SC_IHY, SC_C1, SC_CX, SC_HE, SC_KD, SC_ITH, SC_XP, SC_YL, SC_N };
enum { FL_RLO_DIR, FL_YORDER, FL_YLU, FL_RI0, FL_RK0, FL_PAD, FL_N };

template <typename T>
struct March {
    int nr, nv, ny, nsteps, B;
    long long N;  // nr * nv * ny
    const T* rt;
    const T* r2;
    const T* vt;
    const T* yt;
    const T* sc;
    const T* st;
    const T* dir;
    const T* vf;
    const T* yf;
    const int* fl;
    float* acc;  // [B][nsteps], rounding indicator of the FP32 march
    const T* vp;
    const T* yp;
    int p2P, p3P;  // chunks per v line / y line (1: one thread per line)
    int tma_ok;    // every instrument has gamma = 0 and theta > 0 (the TMA-fed
                   // pass 1 applies)
};

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

// The same with the instrument's read-out corner (FL_RI0, FL_RK0) given.
template <typename T>
__device__ __forceinline__ void note_increment_at(const March<T>& P, int i0, int k0, int b, int i, int k, int n,
                                                  T x0)
{
    if (P.acc == nullptr || i < i0 || i >= i0 + 4 || k < k0 || k >= k0 + 4) return;
    atomicMax(reinterpret_cast<int*>(P.acc + (size_t)b * P.nsteps + n), __float_as_int(fabsf((float)x0)));
}

// Largest number of chunks a strided line is split into, and the largest
// chunk a thread holds in registers.
constexpr int kMaxSplit = 8;
constexpr int kMaxChunk = 32;

// Elements of one split system of n rows in P chunks (layout, all offsets
// even so pairs are aligned):
//   [0, 2n)        (sub-diagonal, 1 / pivot) of each row, chunk-local LU
//   [2n, 4n)       (V, W): the chunk's solution for a unit value of the
//                  unknown before (V) and after (W) the chunk
//   [4n, 4n+2PK)   per chunk p and reduced row q (K = 2 (P - 1)): the
//                  coefficients of the reduced right-hand side q in the
//                  unknowns just before and just after chunk p
//   [4n+2PK, 5n+2PK)  c' of each row (chunk-local LU)
__host__ __device__ inline size_t part_sys_size(int n, int P)
{
    const size_t K = 2 * (size_t)(P - 1);
    return ((5 * (size_t)n + 2 * (size_t)P * K) + 3) & ~(size_t)3;
}
// Rows [s, s + L) of chunk p of a line of n nodes split in P chunks.
__host__ __device__ inline void part_chunk(int n, int P, int p, int& s, int& L)
{
    const int q = n / P, r = n % P;
    L = q + (p < r ? 1 : 0);
    s = p * q + (p < r ? p : r);
}

// Group buffers produced by setup (all device pointers).
struct GroupTables {
    int nr, nv, ny, nsteps, B;
    InstParams* params;   // [B]
    InstDerived* derived; // [B]
    double* axr;          // [B][3][nr] z, J, J2 (FP64)
    double* axv;          // [B][3][nv]
    double* axy;          // [B][3][ny]
    void* rt;
    void* r2;
    void* vt;
    void* yt;
    void* sc;
    void* st;
    void* dir;
    void* vf;
    void* yf;
    int* fl;
    float* acc;           // [B][nsteps]
    void* vp;             // split factors (sized for kMaxSplit chunks)
    void* yp;
    int p2P, p3P;         // chunks per v / y line used by set-up and march
    int tma_ok = 0;       // gamma = 0 and theta > 0 for every instrument
};

// Bytes of the march-type tables of a group.
size_t tables_bytes(int nr, int nv, int ny, int nsteps, int B, size_t elem);
// Carve the table pointers out of one device block of tables_bytes().
void tables_carve(GroupTables& g, void* block, size_t elem);

// Setup (FP64) of all tables for a group; elem = sizeof(float|double).
cudaError_t launch_setup(const GroupTables& g, size_t elem, cudaStream_t s);
// Terminal field U^0 (Section 7.2 cell average for caplets, 1 for bonds).
cudaError_t launch_terminal(const GroupTables& g, void* U, size_t elem, cudaStream_t s);
// FP64 readout of every instrument's price into prices[B]; when indicators
// is not null also the a-posteriori rounding indicator of the march; when
// greeks is not null also dC/dr and dC/dv at the read-out point ([B][2]).
cudaError_t launch_readout(const GroupTables& g, const void* U, size_t elem, double* prices,
                           double* indicators, double* greeks, cudaStream_t s, bool incr32 = false);
// The escalation march of MIXED (FP32 increments on an FP64 state): the state
// split into its FP32 rounding and the FP32 remainder, U = hi + lo, and the
// FP64 update U += x1 + x2 (count values each).
cudaError_t launch_split64(const double* U, float* hi, float* lo, long long count, cudaStream_t s);
// Dirichlet data of every step (the faces table) in FP64 into dir64.
cudaError_t launch_faces64(const GroupTables& g, double* dir64, cudaStream_t s);
cudaError_t launch_update64(double* U, const float* x1, const float* x2, long long count, cudaStream_t s);

// Launch shapes of the three passes for one grid shape (heuristic default or
// picked by the autotuner).
struct Tile {
    int p1_S;  // pass 1: lanes per r line (8, 16, 32)
    int p1_M;  // pass 1: r nodes per lane; p1_S * p1_M >= n_r
    int p1_R;  // pass 1: lines per lane segment per CTA
    int p2_P;  // pass 2: warps sharing each v line (1, 2, 4, 8); 0: passes 2 and 3
               // fused; kLinesTma: lines moved by TMA (k_lines_t)
    int p3_P;  // pass 3: warps sharing each y line (1, 2, 4, 8); kLinesTma
    int p1_stage;  // pass 1: 0 rows from global memory, 1 staged y planes,
                   // 2 y planes staged by TMA (k_pass1t, FP32, gamma = 0)
    int p1_J;      // pass 1 staged: y planes marched per CTA (0 when not staged)
};
Tile default_tile(int nr, int nv, int ny, size_t elem);
// Whether the kernels are compiled for t and it covers the grid shape.
bool tile_valid(const Tile& t, int nr, int nv, int ny, size_t elem);
// Whether a line of n nodes can be split into Pw chunks (Pw = 1: unsplit).
bool split_valid(int n, int Pw);
// Passes 2 and 3 fused over slabs of 8 r nodes (tile p2 = 0) when the
// slab's (v, y) plane fits in shared memory; gamma = 0 groups.
bool pass23_valid(int nr, int nv, int ny, int p2, size_t elem);
template <typename T>
cudaError_t launch_pass23(const March<T>& P, const T* in, const T* Un, T* out, int n, cudaStream_t s);

// The three Douglas passes of step n (in/out as documented in hjm.h). Pass 1
// with Y == nullptr: dU1 from dt F(U^n); with Y = Y3 of a Craig-Sneyd-family
// step: Z1 - B of its correction stage (never the staged kernel).
template <typename T>
cudaError_t launch_pass1(const March<T>& P, const T* U, const T* Y, T* out, int n, const Tile& t,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_pass2(const March<T>& P, const T* in, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_pass3(const March<T>& P, const T* in, const T* Un, T* out, bool any_gamma_pos,
                         int n, cudaStream_t s);
// Raises the dynamic shared-memory limit of the strided-line kernels; call
// once per device before launching or capturing.
cudaError_t init_kernels();
// The same for the staged pass-1 kernels (called by init_kernels).
cudaError_t init_pass1();
// Chunk size per lane used by pass 1 for this n_r (0 if unsupported).
int pass1_chunk(int nr);
// Largest line length pass 2 / pass 3 accept for this element size.
int max_strided_len(size_t elem, bool gamma_pos);

// TMA-fed pass 1 (hjm_pass1t.cu): whether it covers the shape (FP32, gamma =
// 0, n_r a multiple of 32, a compiled (S, M)), its launch, the one-time
// attribute set-up and the count of its bounded waits that ran out.
bool pass1t_valid(const Tile& t, int nr, int nv, int ny, size_t elem);
cudaError_t launch_pass1t(const March<float>& P, const float* U, float* out, int n, const Tile& t,
                          cudaStream_t s);
cudaError_t init_pass1t();
// Strided passes fed by the Tensor Memory Accelerator (hjm_lines_t.cu), the
// launch-shape code kLinesTma of p2_P / p3_P: FP32, n_r a multiple of 4,
// lines of 2..256 nodes; pass 3 only for groups with gamma = 0 (the caller
// falls back to the lane-per-line kernels otherwise, and when
// launch_lines_t returns cudaErrorNotSupported: a field not 16-byte
// aligned). axis 0: pass 2 (Un unused), axis 1: pass 3.
constexpr int kLinesTma = 15;
bool lines_t_valid(int axis, int nr, int nv, int ny, size_t elem);
cudaError_t launch_lines_t(int axis, const March<float>& P, const float* in, const float* Un, float* out, int n,
                           cudaStream_t s);
cudaError_t init_lines_t();
// Warps of the TMA-fed strided passes that gave up a wait (reset clears).
cudaError_t lines_t_timeouts(unsigned* count, bool reset);
// Test hook: from the next launch on, tile `tile` (-1: none) is never copied
// and the waits give up after `limit` polls.
cudaError_t lines_t_test_drop(long long tile, unsigned limit);
// Reads (and with reset clears) the number of CTAs of the TMA-fed pass 1 that
// gave up a wait on a plane copy; synchronises the device.
cudaError_t pass1t_timeouts(unsigned* count, bool reset);
// Test hook: plane index that the next launches never copy (-1: off), so
// the waits for it run out; wait limit in polls.
cudaError_t pass1t_test_drop(int plane, unsigned limit);

template <typename T>
March<T> march_args(const GroupTables& g);

}  // namespace hjm
