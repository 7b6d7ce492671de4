/*
 * hjm.h - C ABI of the GB300 (sm_103a) solver for the single-factor
 * Heath-Jarrow-Morton model with stochastic volatility.
 *
 * The method is the one of E. Valero, M. Torrealba, L. Lacasa, F. Fraysse,
 * "Fast resolution of a single factor Heath-Jarrow-Morton model with
 * stochastic volatility": the Markovian state (r, v, y) of Section 3.1, the
 * pricing PDE of Section 3.2 (Eq. (1)), the sinh-stretched grid of Sections
 * 4.3 and 7.1, centred finite differences and the theta scheme in delta form
 * of Section 5, and the Douglas ADI splitting of Section 5.1, with the
 * softened payoff of Section 7.2 and the one-sided y faces of Section 7.3.
 *
 * Conventions shared by every call:
 *  - Every call returns hjm_status; nothing is thrown across the ABI. On a
 *    non-zero status hjm_last_error() (thread-local) holds a one-line reason.
 *  - Handles are created and destroyed by the caller and owned by the
 *    library. Output buffers are owned by the caller.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream). Device
 *    pointers are plain CUDA device addresses (e.g. torch data_ptr()).
 *  - Fields are stored r fastest, then v, then y: index i + n_r*(k + n_v*j)
 *    for node (r_i, v_k, y_j). Node counts include both boundaries.
 *  - The library never falls back to the CPU: without a CUDA device every
 *    compute call returns HJM_ECUDA.
 */
#ifndef HJM_H
#define HJM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HJM_OK = 0,
    HJM_EINVAL = 1,     /* an argument is out of range or inconsistent */
    HJM_ENOMEM = 2,     /* device or host allocation failed */
    HJM_ECUDA = 3,      /* a CUDA call failed, or no device */
    HJM_ETOL = 4,       /* the error indicator misses tol_rel after escalation */
    HJM_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    HJM_ENUMERIC = 6,   /* a price came out NaN or infinite */
    HJM_ERANGE = 7      /* a size exceeds what the kernels support */
} hjm_status;

/* Arithmetic of the time march. FP64: state, operator and solves in double.
 * FP32: state, operator and solves in float (set-up and read-out stay in
 * double). MIXED: the FP32 march for every instrument; each instrument whose
 * a-posteriori rounding indicator exceeds max(tol_rel |price|, 1e-6) (every
 * instrument when tol_rel = 0) is priced again, a Douglas-scheme instrument
 * first by the escalation march: FP32 increments on an FP64 state (each step
 * splits U^n = hi + lo into its FP32 rounding and FP32 remainder, runs the
 * FP32 step on both, the Dirichlet data split the same way, and adds both
 * increments to U^n in double; about three FP32 steps of memory traffic per
 * step), then in FP64 if its indicator still misses (and for the
 * Craig-Sneyd family). MIXED synchronises the stream. */
typedef enum { HJM_FP64 = 0, HJM_FP32 = 1, HJM_MIXED = 2 } hjm_precision;

/* Initial forward curve f(0,t) (Section 2: p(0,T) = exp(-int_0^T f(0,s) ds)).
 * FLAT: f = flat_rate. NELSON_SIEGEL (instantaneous-forward form):
 * f(0,t) = beta0 + beta1 e^{-t/tau} + beta2 (t/tau) e^{-t/tau}, tau > 0.
 * KNOTS (the discrete curve of Section 6.1): discount factors knot_P[i] > 0
 * at maturities 0 < knot_t[0] < knot_t[1] < ..., 1 <= n_knots <=
 * HJM_MAX_KNOTS, smoothed by the natural cubic spline of ln P(0,t) through
 * (0, 0) and the knots (f = -(ln P)', df/dt = -(ln P)'' continuous; the
 * spline is built on the device by the set-up); past the last knot ln P
 * continues linearly (flat forward). The knot fields are ignored for the
 * other kinds. Calls taking a curve return HJM_EINVAL for an unknown kind,
 * tau <= 0 (Nelson-Siegel), n_knots outside [1, HJM_MAX_KNOTS], maturities
 * not positive and increasing, a discount factor not finite and positive, or
 * f(0,0) outside [r_min, r_max]. */
typedef enum { HJM_CURVE_FLAT = 0, HJM_CURVE_NELSON_SIEGEL = 1, HJM_CURVE_KNOTS = 2 } hjm_curve_kind;
#define HJM_MAX_KNOTS 32
typedef struct {
    int kind;                 /* hjm_curve_kind */
    double flat_rate;
    double beta0, beta1, beta2, tau;
    int n_knots;
    double knot_t[HJM_MAX_KNOTS];
    double knot_P[HJM_MAX_KNOTS];
} hjm_curve;

/* Model of Section 3.1, constant in time: mean reversion kappa >= 0,
 * volatility level lambda >= 0, elasticity gamma in [0,1] (gamma = 0 allows
 * negative rates), variance mean reversion theta >= 0, vol-of-vol
 * epsilon >= 0, correlation rho in [-1,1], initial variance v0 in [0,v_max]. */
typedef struct {
    double kappa, lambda, gamma, theta, epsilon, rho, v0;
} hjm_model_params;

/* Grid and scheme (Sections 4.3, 5, 5.1, 7.1, 7.3).
 *  n_r, n_y, n_v   node counts per axis, boundaries included, each >= 5
 *  n_steps         time steps, uniform dt = T / n_steps
 *  r_min, r_max    rate domain; r_min must be 0 when gamma > 0
 *  y_max, v_max    upper bounds of y and v (both start at 0)
 *  alpha_*         sinh metric width per axis; <= 0 selects a uniform grid
 *  k_r, k_v        metric centres in r and v (y is centred at 0)
 *  center_r_on_strike  1: the r centre is the strike (caplet) or f(0,0) (bond)
 *  theta_adi       theta of the theta scheme (0.5 = Crank-Nicolson)
 *  y_boundary_order    1 or 2: order of the one-sided y differences in F
 *  explicit_midpoint   0: F at t^n as in Section 5; 1: F at t^{n+1/2}
 *  scheme          hjm_scheme: the Douglas scheme of Section 5.1, or one of
 *                  the Craig-Sneyd family (Section 5.1 names Craig-Sneyd as
 *                  the alternative; modified CS and Hundsdorfer-Verwer are
 *                  those of the In 't Hout-Welfert work it cites). These add
 *                  a correction stage (explicit operators and the three line
 *                  solves once more) that makes the step second order in time
 *                  with the mixed term; they take every explicit operator at
 *                  t^{n+1/2}, whatever explicit_midpoint says. Usual theta:
 *                  CS 1/2, MCS 1/3, HV 1/2 + sqrt(3)/6. Another value:
 *                  HJM_EINVAL. A scheme of the family needs a third field
 *                  of the grid's size on the device.
 * Boundary rule: r = r_max, and r = r_min when gamma == 0, carry Dirichlet
 * data (exact bond; caplet max(P(t,T) - Delta_M P(t,T_M), 0)); the v and y
 * faces (and r = 0 when gamma > 0) drop the normal second derivative and the
 * mixed term and use one-sided first differences. */
typedef struct {
    int n_r, n_y, n_v, n_steps;
    double r_min, r_max, y_max, v_max;
    double alpha_r, alpha_y, alpha_v;
    double k_r, k_v;
    int center_r_on_strike;
    double theta_adi;
    int y_boundary_order;
    int explicit_midpoint;
    int scheme;
} hjm_grid_spec;

/* ADI schemes (hjm_grid_spec.scheme). One step of each, with F = A_0 + A_r +
 * A_v + A_y (A_0 the r-v mixed term, explicit only) and the line operators
 * A_d implicit:
 *   Douglas  Y0 = U + dt F(U); Yd = Y(d-1) + theta dt A_d (Yd - U), d = r,v,y;
 *            U' = Y3
 *   CS       Z0 = Y0 + dt/2 A_0 (Y3 - U)
 *   MCS      Z0 = Y0 + theta dt A_0 (Y3 - U) + (1/2 - theta) dt F (Y3 - U)
 *   HV       Z0 = Y0 + dt/2 F (Y3 - U)
 *            then Zd = Z(d-1) + theta dt A_d (Zd - B), B = U (CS, MCS) or
 *            Y3 (HV); U' = Z3. */
typedef enum {
    HJM_SCHEME_DOUGLAS = 0,
    HJM_SCHEME_CS = 1,
    HJM_SCHEME_MCS = 2,
    HJM_SCHEME_HV = 3
} hjm_scheme;

/* Instruments of Section 3.2. ZCB pays 1 at T. CAPLET pays
 * max(1 - Delta_M p(T,T_M), 0) at T with Delta_M = 1 + (T_M - T) K; when
 * strike_atm_relative != 0 the strike is K plus the ATM simple forward
 * (P(0,T)/P(0,T_M) - 1)/(T_M - T). FLOORLET pays the other side,
 * max(Delta_M p(T,T_M) - 1, 0) at T (caplet - floorlet is the forward
 * contract, P(0,T) - Delta_M P(0,T_M) at t = 0). A cap (floor) is the sum of
 * its caplets (floorlets): see hjm_price_strip. */
typedef enum { HJM_ZCB = 0, HJM_CAPLET = 1, HJM_FLOORLET = 2 } hjm_kind;
typedef struct {
    int kind;                 /* hjm_kind */
    double expiry_T, pay_TM, strike_K;
    int strike_atm_relative;
} hjm_instrument;

/* Per-price report. err_estimate is the a-posteriori rounding indicator of
 * the march that produced the price: C (u_op |p| + u_state sqrt(n_steps)
 * max|U| + u_incr sum_n max|dU3_n|), the u the unit roundoffs of the
 * operator's coefficients, the state and the increments (all that of the
 * march type; for the escalation march of MIXED the FP32 one for the
 * coefficients and increments and the FP64 one for the state), the maxima
 * over the 4 x 4 read-out stencil on y = 0, C a safety factor calibrated
 * against the FP64 oracle. */
typedef struct {
    int precision_used;       /* HJM_FP32 or HJM_FP64: the march's type; HJM_MIXED:
                                 MIXED's escalation march (FP32 increments on an
                                 FP64 state) */
    int escalated;            /* 1 if the FP32 result was replaced */
    double err_estimate;
    int n_steps;
    float time_us;            /* device time of the whole call, microseconds */
    int tile_cfg;             /* launch shape used, packed as described at hjm_tile */
    double d_dr;              /* dC/dr at the read-out point r = f(0,0), v = v0, y = 0 */
    double d_dv;              /* dC/dv there (derivatives of the FP64 read-out
                                 interpolant, i.e. of the final field) */
} hjm_price_info;

typedef struct hjm_grid hjm_grid;

/* Create a pricing grid for one curve and model. The handle keeps copies of
 * the three structs and the stream; device memory is allocated at the first
 * price. Errors: HJM_EINVAL on out-of-range parameters, HJM_ERANGE on sizes
 * the kernels do not support, HJM_ECUDA without a device. */
hjm_status hjm_grid_create(const hjm_curve* curve, const hjm_model_params* model,
                           const hjm_grid_spec* spec, void* cuda_stream, hjm_grid** out);
hjm_status hjm_grid_destroy(hjm_grid* grid);

/* Price one instrument (Sections 3.2, 5.1): FP64 setup on the device, the
 * Douglas march of n_steps steps in the requested precision, FP64 cubic
 * readout at r = f(0,0), v = v0, y = 0. Synchronises the grid's stream.
 * tol_rel: relative tolerance for the MIXED escalation (ignored otherwise;
 * 0 re-prices every instrument by the escalation). price_out: host double.
 * info_out may be NULL. */
hjm_status hjm_price(hjm_grid* grid, const hjm_instrument* inst, hjm_precision precision,
                     double tol_rel, double* price_out, hjm_price_info* info_out);

/* Price n independent instruments, each with its own curve, model and grid,
 * in one call. Items of equal grid shape (and scheme) march together in the
 * same kernel launches; a batch of the same make-up seen again is replayed
 * as one CUDA graph in which the shape groups run concurrently. prices_out: n doubles, host or device memory (detected).
 * infos_out: n host structs or NULL. Asynchronous on cuda_stream when both
 * outputs are device/NULL; otherwise synchronises before returning. */
typedef struct {
    hjm_curve curve;
    hjm_model_params model;
    hjm_grid_spec grid;
    hjm_instrument inst;
} hjm_batch_item;
hjm_status hjm_price_batch(const hjm_batch_item* items, size_t n, hjm_precision precision,
                           double tol_rel, double* prices_out, hjm_price_info* infos_out,
                           void* cuda_stream);

/* Stepwise access for checking and for users who want the whole field.
 *
 * hjm_field: run the setup and the first n_run steps (0 <= n_run <= n_steps)
 * of the march for one instrument and copy the field (n_r*n_v*n_y values,
 * double for FP64, float for FP32) to field_out (host or device).
 *
 * hjm_axis: FP64 node, Jacobian and second-derivative tables of axis
 * (0 = r, 1 = v, 2 = y) for this instrument (the r centre can depend on the
 * strike); host arrays of the axis length.
 *
 * hjm_douglas_pass: one kernel pass of step n on device buffers of the
 * field's type and size, on the grid's stream:
 *   pass 1: in = U^n                -> out = dU1 (explicit F and r solve)
 *   pass 2: in = dU1                -> out = dU2 (v solve)
 *   pass 3: in = dU2, in2 = U^n     -> out = U^{n+1} (y solve and update)
 *   pass 4: in = U^n, in2 = Y3      -> out = Z1 - B (Craig-Sneyd family:
 *           the correction stage's explicit operators and r solve, Y3 the
 *           first stage's result, B as in hjm_scheme)
 * For the Craig-Sneyd family pass 3 also serves both stages: in2 is the
 * base the increment is added to (U^n in the first stage, B in the second).
 * in and out may alias for passes 2 and 3 (in place). */
hjm_status hjm_field(hjm_grid* grid, const hjm_instrument* inst, hjm_precision precision,
                     int n_run, void* field_out);
hjm_status hjm_axis(hjm_grid* grid, const hjm_instrument* inst, int axis,
                    double* z_out, double* J_out, double* J2_out);
hjm_status hjm_douglas_pass(hjm_grid* grid, const hjm_instrument* inst, hjm_precision precision,
                            int pass, int step_n, const void* in, const void* in2, void* out);

/* Kernel tracing. While enabled, hjm_price_batch and hjm_price launch the
 * march kernel by kernel (no graph) with a CUDA event pair around every
 * launch on the caller's stream, and synchronise at the end of the call to
 * accumulate the device time of each kernel kind. Intended for measurement,
 * not for production runs. hjm_trace_read copies the totals (reset != 0
 * clears them). Kinds: 0 set-up, 1 terminal field, 2 pass 1, 3 pass 2,
 * 4 pass 3, 5 read-out. */
#define HJM_TRACE_KINDS 6
typedef struct {
    long long launches[HJM_TRACE_KINDS];
    double total_ms[HJM_TRACE_KINDS];
} hjm_trace;
hjm_status hjm_trace_enable(int on);
hjm_status hjm_trace_read(hjm_trace* out, int reset);

/* Launch shapes of the march kernels for one grid shape and precision (the
 * Douglas passes of Section 5.1). Pass 1 gives each r line p1_lanes lanes
 * of a warp holding p1_nodes consecutive nodes each (p1_lanes * p1_nodes >=
 * n_r; compiled: FP32 (8: 8, 16), (16: 4, 8, 16), (32: 2, 4, 8, 16); FP64
 * (16: 2, 4, 8), (32: 2, 4, 8, 16)) and processes p1_lines lines per lane
 * segment per CTA (1..64). p2_warps / p3_warps: warps sharing each v / y
 * line of passes 2 and 3: 1 (one lane per line), or 2, 4, 8 when the line
 * has at least 2 and at most 32 nodes per warp (pass 3 splits y lines only
 * in groups where every instrument has gamma = 0). p2_warps = 0 fuses
 * passes 2 and 3: a CTA holds the whole (v, y) plane of 8 consecutive r
 * nodes in shared memory and runs both line solves there (gamma = 0
 * groups, n_r * element size a multiple of 16, the plane within a CTA's
 * shared memory); p3_warps is then unused (1). p2_warps / p3_warps =
 * HJM_LINES_TMA: one lane per line, the lines moved in and out in tiles of
 * 32 consecutive r nodes by the Tensor Memory Accelerator (one box copy in
 * and one box store per tile, a persistent grid in which every warp marches
 * its own tiles through a ring of shared-memory slots; pass 3 in place adds
 * dU3 to U^n with a reduction store, so U^n is not staged; FP32, n_r a
 * multiple of 4, lines of at most 256 nodes; pass 3 in groups where every
 * instrument has gamma = 0, the lane-per-line kernel otherwise; same results
 * as 1, bit for bit). Stepwise access
 * (hjm_douglas_pass) always runs the passes separately. p1_staged selects how
 * pass 1 gets its five stencil rows: 0 straight from global memory, 1 a CTA
 * copies the y planes of a strip of 4 * (32 / p1_lanes) * p1_lines v nodes
 * into a shared-memory ring and marches over p1_planes (1..4096) y nodes
 * (p1_planes = 0 unless staged; staged needs n_r * element size a multiple
 * of 16 and the ring within the shared memory of a CTA), 2 the same march
 * with each y plane's strip copied by the Tensor Memory Accelerator (one
 * box copy per plane, FP32, n_r a multiple of 32, v strips of at least 3
 * nodes or a multiple of the strip; shapes (p1_lanes: p1_nodes) (4: 16),
 * (8: 8, 12, 16), (16: 8, 12, 16), (32: 8, 16); lines of r nodes at the Section
 * 5.1 Douglas stage only: the Craig-Sneyd correction stage and groups with
 * gamma > 0 or theta_adi = 0 fall back to the default shape of pass 1), 3
 * the same kernel persistent (p1_planes = 0): one CTA per resident slot of
 * the GPU, each marching an equal share (to one plane) of the group's
 * (instrument, strip, y plane) units. A shape changes speed and the
 * rounding of the line solves, nothing else.
 * tile_cfg in hjm_price_info packs p1_lanes | p1_nodes << 8 | p1_lines << 14
 * | p2_warps << 21 | p3_warps << 25 | p1_staged << 29. */
#define HJM_LINES_TMA 15
typedef struct {
    int p1_lanes;
    int p1_nodes;
    int p1_lines;
    int p2_warps;
    int p3_warps;
    int p1_staged;
    int p1_planes;
} hjm_tile;
/* The shape in use for (n_r, n_v, n_y, precision): set, tuned or default.
 * HJM_MIXED reads the FP32 entry. */
hjm_status hjm_tile_get(int n_r, int n_v, int n_y, hjm_precision precision, hjm_tile* out);
/* Use *tile for this grid shape from now on (process-wide); NULL restores
 * the default. HJM_EINVAL when the shape is not compiled or does not cover
 * n_r. */
hjm_status hjm_tile_set(int n_r, int n_v, int n_y, hjm_precision precision, const hjm_tile* tile);
/* Autotuner: for every grid shape among the items, march the items of that
 * shape for `steps` steps (1..1000) with each candidate launch shape (timed
 * with CUDA events on cuda_stream, best of two), and keep the fastest for
 * later calls. For items of the Craig-Sneyd family the pass-1 time includes
 * the correction stage's pass 1, which never uses the staged row feed. One
 * shape is kept per grid shape and precision, whatever the scheme: tune
 * with the items (and scheme) that will be priced. Prices are not computed;
 * synchronous; the items are validated as in hjm_price_batch. */
hjm_status hjm_autotune(const hjm_batch_item* items, size_t n, hjm_precision precision, int steps,
                        void* cuda_stream);

/* Pricing surrogate (the paper has no counterpart: it is a learned stand-in
 * for the march, for repeated pricing in calibration loops). A multilayer
 * perceptron 9 -> 256 -> 256 -> 256 -> 256 -> 1 with SiLU activations; its
 * three 256 x 256 layers run on the tensor cores with bfloat16 operands and
 * FP32 accumulation (forward and backward), AdamW on FP32 master weights.
 * Inference (hjm_surrogate_forward, _premium, _infer) runs all layers of a
 * 128-row tile in one kernel on the fifth-generation tensor cores (tcgen05,
 * accumulators in tensor memory); training runs them layer by layer.
 *
 * Inputs, per row (float, device, [n][9]): x = (kappa, lambda, theta,
 * epsilon, rho, T, delta, K, F) with gamma = 0 and v0 = 1: model parameters,
 * expiry T, accrual delta = T_M - T, strike K and the simple forward rate F
 * of the curve over [T, T + delta]. Output: the forward premium C / P(0,T)
 * of the caplet paying max(1 - (1 + delta K) p(T, T_M), 0) at T (multiply by
 * the caller's P(0,T) for the price). With gamma = 0 this quantity depends on
 * the curve only through F. It is the Gaussian-HJM caplet of Section 3.1
 * (epsilon = 0: a put on the log-normal bond p(T,T_M), in closed form) plus
 * the stochastic-volatility correction, and the network learns only the
 * correction, scaled: q = (C - C_gauss) / (P(0,T) delta 1e-4).
 *
 * Training data are the library's own FP32 march prices (labels on a flat
 * curve with that forward), drawn uniformly over the box of features
 * (kappa, lambda, theta, epsilon, rho, T, delta, K - F, F); 1/16 of the draws
 * are held out and give, per (T, K - F) bin (9 x 8), the largest PDE-judged
 * error. Inference answers from the network inside the box in bins whose
 * held-out error is at most 0.5e-4 (half the 1e-4 price tolerance, a margin
 * for unseen rows), and prices every other row with the march (the
 * fallback); used_pde marks those rows.
 *
 * label_grid: node counts, steps and scheme options of each label's march;
 * its domain fields are ignored (set per draw from the model's scales).
 * checkpoint_path: NULL, or a file written after every epoch; an existing
 * file resumes training from it. hidden must be 256 and depth 4. */
typedef struct {
    size_t n_train;
    int hidden, depth;
    int epochs, batch;
    float lr;
    uint64_t seed;
    double box_lo[9], box_hi[9];
    hjm_grid_spec label_grid;
    const char* checkpoint_path;
} hjm_surrogate_cfg;
typedef struct hjm_surrogate hjm_surrogate;
#define HJM_SURROGATE_PARAMS 200193
#define HJM_SURROGATE_BINS 72

/* Untrained network (seeded Glorot-uniform weights); every row falls back. */
hjm_status hjm_surrogate_create(const hjm_surrogate_cfg* cfg, void* cuda_stream, hjm_surrogate** out);
/* Draw, label with the march, train, build the error table. Synchronous. */
hjm_status hjm_surrogate_train(const hjm_surrogate_cfg* cfg, void* cuda_stream, hjm_surrogate** out);
/* epochs of AdamW on given data: x [n][9] raw inputs and t [n] scaled
 * targets q = (C - C_gauss) / (P(0,T) delta 1e-4), both device. */
hjm_status hjm_surrogate_fit(hjm_surrogate* s, const float* x, const float* t, size_t n, int epochs,
                             void* cuda_stream, float* final_loss);
/* Gated prices (device x [n][9], device price_out [n], device used_pde [n]
 * or NULL). Synchronises when rows fall back. */
hjm_status hjm_surrogate_infer(hjm_surrogate* s, const float* x, size_t n, double* price_out,
                               uint8_t* used_pde, void* cuda_stream);
/* The network alone: y_out [n] = scaled output q (device). */
hjm_status hjm_surrogate_forward(hjm_surrogate* s, const float* x, size_t n, float* y_out, void* cuda_stream);
/* The network alone as forward premia, C_gauss / P(0,T) + q delta 1e-4
 * (device, double; no gate, no fallback). */
hjm_status hjm_surrogate_premium(hjm_surrogate* s, const float* x, size_t n, double* premium_out,
                                 void* cuda_stream);
/* The closed-form part alone: the Gaussian-HJM caplet's forward premium
 * C_gauss / P(0,T) of each row (device x [n][9], device double out [n]). */
hjm_status hjm_surrogate_gauss_premium(const float* x, size_t n, double* premium_out, void* cuda_stream);
/* Mean squared error of the scaled targets t and its gradient (device,
 * HJM_SURROGATE_PARAMS floats, layout W0 [256x9], b0, W1 [256x256], b1, W2,
 * b2, W3, b3, W4 [256], b4). loss_out: host float or NULL. */
hjm_status hjm_surrogate_loss_grad(hjm_surrogate* s, const float* x, const float* t, size_t n,
                                   float* loss_out, float* grad_out, void* cuda_stream);
hjm_status hjm_surrogate_get_params(const hjm_surrogate* s, float* out);
hjm_status hjm_surrogate_set_params(hjm_surrogate* s, const float* in);
/* Held-out error per bin (host, HJM_SURROGATE_BINS floats, +inf = no data). */
hjm_status hjm_surrogate_error_table(const hjm_surrogate* s, float* out);
hjm_status hjm_surrogate_save(const hjm_surrogate* s, const char* path);
hjm_status hjm_surrogate_load(const char* path, hjm_surrogate** out);
hjm_status hjm_surrogate_destroy(hjm_surrogate* s);
/* A cap or a floor (Section 1 motivates the model by their calibration): the
 * strip of its caplets or floorlets, items[i] the period [T_i, T_i + tenor]
 * with T_{i+1} = T_i + tenor, all of one kind (HJM_CAPLET for a cap,
 * HJM_FLOORLET for a floor) with the same curve, model, tenor and absolute
 * strike (strike_atm_relative = 0); each item on its own grid (the caller
 * sizes the domain for its expiry). Prices the strip as one batch
 * (hjm_price_batch, host outputs) and returns the sum in *strip_price and,
 * when item_prices is not NULL, each period's price. HJM_EINVAL when the
 * items do not form such a strip. */
hjm_status hjm_price_strip(const hjm_batch_item* items, size_t n, hjm_precision precision, double tol_rel,
                           double* strip_price, double* item_prices, void* cuda_stream);

/* The surrogate's tensor-core product, exposed for testing: C[M x N] (FP32,
 * device) = op(A) op(B) with bfloat16 A, B (device); op(A)(m,k) = A[m lda+k]
 * or A[k lda+m] when trans_a, op(B)(k,n) = B[k ldb+n] or B[n ldb+k]. */
hjm_status hjm_mlp_gemm(int M, int N, int K, const void* A, int lda, int trans_a, const void* B, int ldb,
                        int trans_b, float* C, int ldc, void* cuda_stream);

/* Allocation-free pricing of one instrument (the paper has no counterpart;
 * this is a deployment aid). For callers that cannot allocate device memory:
 * processes whose device memory belongs to another allocator (a framework's
 * caching allocator, or a fixed pool sized at start-up, where a cudaMalloc
 * outside it fails or fragments the pool), and latency-critical loops that
 * cannot take cudaMalloc's implicit device-wide synchronisation. Tested on
 * ordinary streams, two calls in a row against hjm_price.
 *
 * Instead of a workspace, the march uses one file-scope device array of
 * HJM_STATIC_SCRATCH_BYTES bytes that every GPU loading the library holds
 * until the process exits. The call allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine): it copies the item's parameters
 * into the array, runs set-up, terminal field, the n_steps ADI steps and
 * the read-out on cuda_stream, and writes the price to price_out, which must
 * be device memory (one double). precision: HJM_FP32 or HJM_FP64.
 *
 * Limits and caveats:
 *  - an item whose fields and tables do not fit in the array is rejected with
 *    HJM_ERANGE (FP64 fields of up to about 2^19 points per field fit, fewer
 *    with a Craig-Sneyd-family scheme, which holds a third field; the
 *    message states the bytes needed);
 *  - the first call on each device looks up the array's device address and
 *    sets the kernels' shared-memory limit;
 *  - every call shares the one array and leaves the last call's contents in
 *    it: calls that overlap on the GPU (different streams without ordering,
 *    or several host threads) race and give wrong prices; order them. */
#define HJM_STATIC_SCRATCH_BYTES (8u << 20)
hjm_status hjm_price_static(const hjm_batch_item* item, hjm_precision precision, double* price_out,
                            void* cuda_stream);

/* Bounded device-side waits (no counterpart in the paper). The TMA-fed pass
 * 1 (p1_staged = 2, 3) waits on a barrier for each y plane it copies; a CTA
 * whose wait runs out of polls (the copy never arrived) stops without
 * writing the rest of its planes and is counted. The TMA-fed passes 2 and 3
 * (HJM_LINES_TMA) wait on a barrier for each line tile; a warp whose wait
 * runs out stops without writing the rest of its tiles and is counted. The
 * surrogate's fused
 * tensor-core forward waits on a barrier for each layer's matrix products;
 * a CTA whose wait runs out writes NaN for its rows and is counted too. hjm_wait_status
 * synchronises the current device and returns HJM_ETIMEOUT when any CTA has
 * given up since the last reset (reset != 0 clears the count), HJM_OK
 * otherwise; hjm_price and hjm_price_batch with host outputs check it
 * themselves. hjm_test_drop_plane is a test hook: from the next launch on,
 * the copy of y plane `plane` (0 .. n_y - 1 of every instrument) in the
 * TMA-fed pass 1, and of line tile `plane` of each launch of the TMA-fed
 * passes 2 and 3 (tiles numbered r block fastest, then y plane (pass 2) or
 * v node (pass 3), then instrument), is never started and each wait gives
 * up after `polls` polls; plane = -1 and polls = 0 restore normal operation. */
hjm_status hjm_wait_status(int reset);
hjm_status hjm_test_drop_plane(int plane, unsigned polls);

const char* hjm_status_string(hjm_status status);
const char* hjm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HJM_H */
