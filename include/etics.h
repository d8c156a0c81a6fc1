/*
 * etics.h -- C ABI of the GB300 (sm_103a) SCF and MEX expansion force library.
 *
 * Method: Meiron, Li, Holley-Bockelmann & Spurzem, "Expansion Techniques for
 * Collisionless Stellar Dynamical Simulations" (the ETICS code).  The problem
 * (Sec. 2.1, eqs. 1-3) is the Poisson equation of N point masses with G = 1;
 * the library returns the acceleration a = -grad(Phi) and the potential Phi at
 * every particle by one of two expansions:
 *   SCF (Sec. 2.4 eq. 18, Sec. 2.5, Sec. 3.3): coefficients of the
 *       Hernquist-Ostriker basis, then a field pass over the coefficients;
 *   MEX (Sec. 2.4 eqs. 15-17, Sec. 2.2, Sec. 3.2): radial sort, then inner and
 *       outer cumulative multipole sums along radius.
 *
 * Conventions shared by every entry point
 *   - Expansion centre at the origin, Hernquist scale length a = 1 (Sec. 5.1).
 *   - precision = ETICS_MIXED: particle arrays are float4 (16 B per particle),
 *     basis recursions and field sums in FP32, coefficient reductions and the
 *     MEX cross-tile carries in FP64.  precision = ETICS_FP64: arrays are 4
 *     doubles per particle (32 B) and everything is FP64.
 *   - posm  [N] = (x, y, z, m);  vel [N] = (vx, vy, vz, unused);
 *     accpot[N] = (ax, ay, az, Phi), in the caller's particle order.
 *   - Real orthonormal spherical harmonics without the Condon-Shortley phase:
 *     Y_l0 = N_l0 P_l^0(cos t), Y_lm = sqrt2 N_lm P_l^m cos(m phi),
 *     Y_l-m = sqrt2 N_lm P_l^m sin(m phi) (m > 0), so Y_11 = +sqrt(3/4pi) x/r.
 *     SCF coefficients are doubles c[n*(l_max+1)^2 + l*l + l + m] with
 *     Phi(x) = sum c * phi_nl(r) Y_lm, phi_nl = -r^l (1+r)^-(2l+1) C_n^(2l+3/2)(xi),
 *     xi = (r-1)/(r+1).  A_000 = c[0]/sqrt(4 pi) equals the mass of a
 *     Hernquist system.
 *   - All pointers except those named "host" are DEVICE pointers owned by the
 *     caller; the library never frees them and allocates no device memory.
 *     posm/vel/accpot must be 16-byte aligned; ws 256-byte aligned.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Every call is
 *     asynchronous on it and returns a status: argument errors are reported
 *     synchronously (nothing is launched); data errors (non-finite input,
 *     FP32 overflow, a lookback wait that timed out) set a device error word
 *     that etics_get_error() reads.
 *   - Limits: 0 <= n_max <= ETICS_NMAX_LIMIT, 0 <= l_max <= ETICS_LMAX_LIMIT
 *     (SCF); 0 <= l_max <= ETICS_MEX_LMAX_LIMIT (MEX); 0 <= N < 2^30.
 *   - Results are deterministic: the same inputs on the same device give
 *     bitwise identical outputs.
 */
#ifndef ETICS_H
#define ETICS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ETICS_VERSION 100

enum etics_status {
    ETICS_OK = 0,
    ETICS_ERR_ARG = -1,         /* invalid argument (null/misaligned pointer, bad size)   */
    ETICS_ERR_CUDA = -2,        /* a CUDA runtime call failed                             */
    ETICS_ERR_WORKSPACE = -3,   /* ws_bytes smaller than etics_workspace_bytes()          */
    ETICS_ERR_NONFINITE = -4,   /* device: NaN/Inf input or FP32 overflow in a sum        */
    ETICS_ERR_TIMEOUT = -5,     /* device: a bounded inter-block wait gave up             */
    ETICS_ERR_UNSUPPORTED = -6  /* parameters beyond the compiled limits                  */
};

enum etics_precision { ETICS_FP64 = 0, ETICS_MIXED = 1 };
enum etics_method { ETICS_SCF = 0, ETICS_MEX = 1 };
enum etics_out { ETICS_OUT_ACC = 1, ETICS_OUT_POT = 2 };   /* force/potential/both */

#define ETICS_NMAX_LIMIT 16
#define ETICS_LMAX_LIMIT 14
#define ETICS_MEX_LMAX_LIMIT 10

/* Bytes of device workspace a call of `method` (ETICS_SCF: etics_scf_coeffs
 * and etics_leapfrog_step with SCF; ETICS_MEX: etics_mex_field,
 * etics_radial_sort and etics_leapfrog_step with MEX) needs on the current
 * device.  Returns 0 for invalid arguments. */
size_t etics_workspace_bytes(int64_t N, int n_max, int l_max, int method, int precision);

/* SCF coefficient pass (Sec. 3.3, first part; eq. 18):
 *   c[n][l,m] = (1/J_nl) sum_k m_k phi_nl(r_k) Y_lm(x_k),
 *   J_nl = int rho_nl phi_nl r^2 dr.
 * coeffs: device double[(n_max+1)*(l_max+1)^2], overwritten.  ws: device
 * workspace of at least etics_workspace_bytes(N, n_max, l_max, ETICS_SCF, p).
 * N = 0 writes zeros. */
int etics_scf_coeffs(const void *posm, int64_t N, int n_max, int l_max, int precision,
                     double *coeffs, void *ws, size_t ws_bytes, void *stream);

/* SCF field pass (Sec. 3.3, second part): Phi = sum c phi_nl Y_lm and
 * a = -grad Phi at each particle of posm (the masses are ignored).
 * out_mask: ETICS_OUT_ACC | ETICS_OUT_POT (at least one); components not
 * requested are written as 0.  Needs no workspace. */
int etics_scf_field(const void *posm, int64_t N, int n_max, int l_max, int precision,
                    const double *coeffs, void *accpot, int out_mask, void *stream);

/* The two SCF passes with a chosen radial basis (Sec. 2.5 describes both):
 *   ETICS_BASIS_HO: Hernquist-Ostriker, the Hernquist model as zeroth term
 *     (what etics_scf_coeffs / etics_scf_field use);
 *   ETICS_BASIS_CB: Clutton-Brock, the Plummer model as zeroth term,
 *     phi_nl = -r^l (1+r^2)^-(l+1/2) C_n^(l+1)(xi), xi = (r^2-1)/(r^2+1),
 *     J_nl = -K_nl 2^-(4l+6) (n+2l+1)! / (n! (n+l+1) (l!)^2),
 *     K_nl = 4n(n+2l+2) + (2l+1)(2l+3).
 * Arguments, layouts, workspace and errors as etics_scf_coeffs /
 * etics_scf_field; an unknown basis is ETICS_ERR_ARG.  Coefficients of one
 * basis are meaningless in the other. */
#define ETICS_BASIS_HO 0
#define ETICS_BASIS_CB 1
int etics_scf_coeffs_basis(const void *posm, int64_t N, int n_max, int l_max, int basis,
                           int precision, double *coeffs, void *ws, size_t ws_bytes,
                           void *stream);
int etics_scf_field_basis(const void *posm, int64_t N, int n_max, int l_max, int basis,
                          int precision, const double *coeffs, void *accpot, int out_mask,
                          void *stream);

/* MEX force calculation (Sec. 2.4 eqs. 15-17, Sec. 3.2): radial sort, inner
 * and outer exclusive cumulative sums of m r^l Y_lm and m r^-(l+1) Y_lm, and
 * Phi_i = -sum_l 4pi/(2l+1) sum_m [q_lm(i) r^-(l+1) + p_lm(i) r^l] Y_lm(x_i).
 * The order is by r^2 = (x*x + y*y) + z*z evaluated in FP64 (bitwise as a
 * CPU evaluates it), ties by particle index, with no limit on how many
 * particles share a radius (a shell).  A particle at the origin sorts first,
 * contributes no outer moment, and feels only the outer l <= 1 field.
 * 0 <= l_max <= ETICS_MEX_LMAX_LIMIT; levels above 6 run in level groups
 * (more time, the same registers).
 * ws: at least etics_workspace_bytes(N, 0, l_max, ETICS_MEX, p) (it grows
 * with (l_max+1)^2 above l_max = 6). */
int etics_mex_field(const void *posm, int64_t N, int l_max, int precision, void *accpot,
                    int out_mask, void *ws, size_t ws_bytes, void *stream);

/* The radial order MEX uses (Sec. 3.2, the sort): order[k] = index of the
 * particle of rank k.  order: device uint32[N].  ws as for etics_mex_field. */
int etics_radial_sort(const void *posm, int64_t N, int precision, uint32_t *order,
                      void *ws, size_t ws_bytes, void *stream);

/* The radial sort key of every particle (the first step of the MEX sort):
 * keys[i] = high 32 bits of the IEEE-754 FP64 bit pattern of
 * r^2 = (x*x + y*y) + z*z evaluated in FP64 (as a CPU rounds it), for the
 * particle's own coordinates (float4 coordinates are widened exactly).
 * keys: device uint32[N].  Needs no workspace. */
int etics_radial_keys(const void *posm, int64_t N, int precision, uint32_t *keys, void *stream);

/* ---- batches of independent systems ------------------------------------
 * Many independent systems of uneven size and expansion order in one SCF pass
 * (the paper notes the GPU is under-loaded at small N, Sec. 3.4): the
 * particles of all systems are concatenated in posm, system i owning
 * items[i].n consecutive particles; its coefficients are packed one system
 * after another (n_max+1)(l_max+1)^2 each, in the layout of etics_scf_coeffs. */
typedef struct { int64_t n; int n_max; int l_max; } etics_batch_item;
/* Launch shape (0 = default): particles per coefficient tile -- mixed
 * precision: 8..512, rounded up to a multiple of 64 (default 512); FP64:
 * multiple of 4, 8..128 (default 32; tiles > 64 exceed one block's shared
 * memory and are rejected with ETICS_ERR_UNSUPPORTED) -- coefficient blocks
 * per SM (1..8), field threads per block (multiple of 32, <= 256), particles
 * per field work item (>= 1). */
typedef struct { int tile; int blocks_per_sm; int field_threads; int field_chunk; } etics_batch_tuning;

/* Builds the batch plan in HOST memory.  With plan == NULL only the sizes are
 * returned: *plan_bytes_needed (plan size), *ws_bytes (device workspace) and
 * *coeff_count (doubles of packed coefficients).  Limits per system:
 * n_max <= 14, l_max <= 8.  The caller copies the plan to device memory and
 * passes both copies to etics_scf_batch. */
int etics_scf_batch_plan(const etics_batch_item *items, int ninst,
                         const etics_batch_tuning *tuning, int precision, void *plan,
                         size_t plan_bytes, size_t *plan_bytes_needed, size_t *ws_bytes,
                         int64_t *coeff_count);

/* SCF coefficients and field of every system of the plan: three kernels
 * (coefficients, ordered finalize, field), no host synchronisation, so the
 * call can be captured into a CUDA graph.  accpot may be NULL (coefficients
 * only).  ws: at least the plan's ws_bytes. */
int etics_scf_batch(const void *posm, const void *plan_host, const void *plan_dev, int precision,
                    double *coeffs, void *accpot, int out_mask, void *ws, size_t ws_bytes,
                    void *stream);

/* One kick-drift-kick leapfrog step (Sec. 3.4, Sec. 5.4), in place:
 *   v += dt/2 a;  x += dt v;  (a, Phi) = force(x) by `method`;  v += dt/2 a.
 * accpot holds a(x) on entry and (a, Phi) at the new positions on exit.
 * coeffs_out (nullable, SCF only): receives the new coefficients.
 * ws: etics_workspace_bytes(N, n_max, l_max, method, precision) bytes. */
int etics_leapfrog_step(void *posm, void *vel, void *accpot, int64_t N, double dt,
                        int method, int n_max, int l_max, int precision, double *coeffs_out,
                        void *ws, size_t ws_bytes, void *stream);

/* Size of the fixed scratch array behind etics_scf_coeffs_noalloc. */
#define ETICS_STATIC_SCRATCH_BYTES (4u << 20)

/* The SCF coefficient pass without a caller workspace (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory or
 * pass a device buffer, e.g. a hard real-time loop where an allocation could
 * block or fail, or a host application that owns all device memory and gives
 * plug-in code no allocation rights).  Same arguments and result as
 * etics_scf_coeffs minus ws/ws_bytes; allocates nothing.  Its scratch is a
 * fixed array of ETICS_STATIC_SCRATCH_BYTES that every GPU loading the library
 * holds until process exit; it returns ETICS_ERR_WORKSPACE when
 * etics_workspace_bytes(N, n_max, l_max, ETICS_SCF, precision) exceeds it
 * (e.g. n_max = 16, l_max = 14 on a 152-SM GB300).  The first call on a device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture.  All calls share the one array:
 * calls that overlap on the GPU (different streams, or different host
 * threads) race and give wrong coefficients. */
int etics_scf_coeffs_noalloc(const void *posm, int64_t N, int n_max, int l_max, int precision,
                             double *coeffs, void *stream);

/* One kick-drift-kick step like etics_leapfrog_step with method SCF, but the
 * force at the new positions uses the given coefficients (c[n][l*l+l+m],
 * device, (n_max+1)(l_max+1)^2 doubles) instead of a coefficient pass: the
 * step that a coefficient forecast drives.  Needs no workspace. */
int etics_leapfrog_step_coeffs(void *posm, void *vel, void *accpot, int64_t N, double dt,
                               int n_max, int l_max, int precision, const double *coeffs,
                               void *stream);

/* ---- coefficient-forecasting MLP ----------------------------------------
 * Not in the paper.  It extends the reuse of coefficients over several steps
 * (temporal softening, end of Sec. 4.1) to a forecast: a multilayer
 * perceptron maps the last 8 coefficient vectors to the next one, so that the
 * coefficient pass can be skipped on most steps.
 *
 * Network: dims[0] -> dims[1] -> ... -> dims[nlayers]; tanh after every layer
 * but the last.  params: device FP32, for each layer i W_i (dims[i] x
 * dims[i+1], row-major, input index first) then b_i (dims[i+1]);
 * params_bf16: device bf16 codes (uint16) of the same vector, the operands of
 * the tensor-core products (bf16 x bf16, FP32 accumulation).  x: device bf16
 * codes, batch x dims[0] row-major; y / target: device FP32, batch x
 * dims[nlayers].  All results are deterministic (fixed summation orders). */
#define ETICS_MLP_MAX_LAYERS 4
typedef struct { int nlayers; int dims[ETICS_MLP_MAX_LAYERS + 1]; } etics_mlp_shape;

/* Floats in params (-1 for an invalid shape: nlayers outside 1..4 or a
 * width outside 1..2^20). */
int64_t etics_mlp_param_count(const etics_mlp_shape *shape);
/* Device workspace of etics_mlp_forward / etics_mlp_loss_grad for `batch` rows
 * (0 for an invalid shape). */
size_t etics_mlp_workspace_bytes(const etics_mlp_shape *shape, int batch);
/* y = network(x). */
int etics_mlp_forward(const etics_mlp_shape *shape, const float *params,
                      const uint16_t *params_bf16, const uint16_t *x, int batch, float *y,
                      void *ws, size_t ws_bytes, void *stream);
/* *loss (device double) = mean over batch x dims[nlayers] of (y - target)^2
 * and grads (device FP32, the layout of params) = its gradient by
 * back-propagation.  batch >= 1. */
int etics_mlp_loss_grad(const etics_mlp_shape *shape, const float *params,
                        const uint16_t *params_bf16, const uint16_t *x, const float *target,
                        int batch, float *grads, double *loss, void *ws, size_t ws_bytes,
                        void *stream);
/* One Adam step (t >= 1: the step count, for the bias corrections) on params
 * with moment buffers m, v (device FP32, zero before the first step); also
 * refreshes params_bf16. */
int etics_mlp_adam(const etics_mlp_shape *shape, float *params, const float *grads, float *m,
                   float *v, int64_t t, float lr, float beta1, float beta2, float eps,
                   uint16_t *params_bf16, void *stream);
/* params_bf16 = bf16(params) (round to nearest even). */
int etics_mlp_to_bf16(const etics_mlp_shape *shape, const float *params, uint16_t *params_bf16,
                      void *stream);

/* Coefficient forecasting glue.  A forecast works on a history of eight true
 * coefficient vectors c_0..c_7 (oldest first) spaced `stride` steps apart
 * (1 <= stride <= 4) and predicts the vector k steps after c_7 for each
 * horizon k = 1..stride: the cubic through c_4..c_7 evaluated at
 * s = k/stride of a spacing after c_7, ((c_7 + s d1) + s(s+1)/2 d2) +
 * s(s+1)(s+2)/6 d3 (backward differences of the history at c_7), plus a
 * per-coefficient linear correction fitted to the trajectory, plus the
 * network's correction.
 *
 * Normalisers and fitted predictors of a trajectory traj (device, T x D
 * doubles, T >= 5) into norm (device, (7 + 9 stride) x D doubles): rows 0-6
 * the mean, 1/standard deviation, 1/RMS of the k-th backward differences at
 * spacing `stride` (k = 1..4) and their RMS s4 (a reciprocal is 0 where its
 * scale is 0); then per horizon k, from row 7 + 9(k-1): beta_k[0..6], the RMS
 * q_k of its residual and 1/q_k.  The predictor of horizon k regresses
 * t_k = (c_{t+k} - cubic_k) / s4 by least squares on the regressors u of the
 * history (the seven feature blocks 1-7 of etics_coeff_features before their
 * bf16 rounding) over every history of traj whose horizons lie inside it,
 * with a 1e-12 relative ridge; beta = 0 and q = 1 where there is none.  Two
 * kernels. */
int etics_coeff_stats(const double *traj, int T, int D, int stride, double *norm, void *stream);
/* Network inputs x (bf16 codes) of the histories store[rows[b][0..7]]
 * (device int32, oldest first; store: device, rows of D doubles), eight
 * blocks per coefficient from the backward differences d1..d4 of the history:
 * block 0 the normalised state, blocks 1-3 the newest d1, d2, d3, blocks 4-7
 * the four newest d4, newest first, each over its RMS.  layout
 * ETICS_FEAT_JOINT: x is batch x 8D, element [b][blk*D + j] (one network row
 * sees every coefficient); ETICS_FEAT_PER_COEFF: x is (batch*D) x 8, element
 * [b*D + j][blk] (one row per coefficient, a network shared by all
 * coefficients).  With next_rows (nullable, device int32[batch][stride]: the
 * vectors 1..stride steps after each history) also the training targets
 * (FP32): for horizon k, (t_k - beta_k . u) / q_k, what the fitted predictor
 * misses, at [(b*D + j)*stride + k-1] (per coefficient) or
 * [(b*stride + k-1)*D + j] (joint). */
#define ETICS_FEAT_JOINT 0
#define ETICS_FEAT_PER_COEFF 1
int etics_coeff_features(const double *store, const int32_t *rows, const int32_t *next_rows,
                         int batch, int D, int stride, const double *norm, int layout,
                         uint16_t *x, float *target, void *stream);
/* A forecast or a push on a ring of 8 vectors (ring: device 8 x D doubles;
 * order: device int32[8], slots oldest..newest).  Forecast (y non-NULL,
 * 1 <= horizon <= stride): cubic_k + s4 (beta_k . u + q_k y[j*y_stride]) for
 * the network output y (device FP32).  Push (coeffs_in non-NULL): coeffs_in.
 * Exactly one of coeffs_in, y.  With commit != 0 the vector is written into
 * the oldest slot and order rotated in place; coeffs_out (nullable when
 * commit != 0) receives it.  One block; graph-capturable. */
int etics_coeff_advance(double *ring, int32_t *order, int D, int stride, int horizon,
                        const double *coeffs_in, const float *y, int y_stride,
                        const double *norm, double *coeffs_out, int commit, void *stream);

/* Relative acceleration error e_i = |a_i - r_i| / |r_i| (Sec. 4.2) of
 * accpot a against accpot r (device (N,4) arrays of the given precision):
 * out (device uint64[3], overwritten) = { #(e_i > tol_a), #(e_i > tol_b),
 * bit pattern of max e_i as an IEEE double }.  A zero reference acceleration
 * counts as e_i = inf unless a_i is zero too.  Budgets on the median and the
 * maximum follow from the counts: median <= tol_a iff 2 #(e > tol_a) <= N. */
int etics_force_error(const void *a, const void *r, int64_t N, int precision, double tol_a,
                      double tol_b, uint64_t *out, void *stream);

/* Waits for `stream`, then returns and clears the device error word
 * (ETICS_OK if no kernel reported a data error since the last call). */
int etics_get_error(void *stream);

/* ---- failure detection ---------------------------------------------------
 * The paper has no counterpart; these exist so that the error path of the
 * bounded device waits can be exercised without faulting or hanging a GPU.
 *
 * Bound, in polls, of the waits of the MEX radial sort's decoupled lookback
 * (a tile waiting for an earlier tile to publish its digit counts) in later
 * calls on any stream; 0 restores the default (2^22 polls of >= 32 ns).
 * When a wait runs out, the error word records ETICS_ERR_TIMEOUT, the tile
 * goes on with a partial prefix, and every later kernel of the call keeps its
 * reads and writes inside the caller's buffers (an order entry >= N is
 * skipped), so the call returns with undefined outputs instead of faulting.
 * A negative bound is ETICS_ERR_ARG.  Process-wide, not thread-safe. */
int etics_set_wait_limit(int64_t spins);

/* Makes one bounded wait run out on purpose and returns like the library's
 * own kernels do when that happens (ETICS_ERR_TIMEOUT in the error word, no
 * fault, the context stays usable):
 *   ETICS_WAIT_LOOKBACK: one radix pass over 8192 keys whose single block
 *     waits for a predecessor tile that never publishes, giving up after
 *     `spins` polls.  ws: device workspace of at least
 *     etics_workspace_bytes(8192, 0, 0, ETICS_MEX, ETICS_MIXED) bytes
 *     (its contents are overwritten); a smaller ws_bytes is
 *     ETICS_ERR_WORKSPACE.
 *   ETICS_WAIT_MBARRIER: a block that holds tensor memory waits `spins`
 *     tries on an mbarrier nothing arrives on (the wait of the tcgen05
 *     products of the MLP), then frees the tensor memory.  ws is unused.
 * spins < 0 or an unknown `which` is ETICS_ERR_ARG.  Asynchronous on stream;
 * read the outcome with etics_get_error(). */
#define ETICS_WAIT_LOOKBACK 0
#define ETICS_WAIT_MBARRIER 1
int etics_test_wait_timeout(int which, int64_t spins, void *ws, size_t ws_bytes, void *stream);

/* ---- measurement aid -------------------------------------------------------
 * The arithmetic rates behind the roofline fractions of the benchmark (the
 * paper compares single- and double-precision speed, Sec. 3.4; it has no
 * such entry point).  Launches `blocks` blocks of 256 threads, each thread
 * running `iters` rounds of 256 fused multiply-adds on 16 independent
 * accumulator chains:
 *   ETICS_PEAK_FFMA:  FP32 fmaf;
 *   ETICS_PEAK_FFMA2: the paired FP32 FMA (two FMAs per instruction);
 *   ETICS_PEAK_DFMA:  FP64 fma.
 * sink: device float[blocks * 256], overwritten with one value per thread (so
 * that the work cannot be elided).  *flops_host (host) receives the
 * floating-point operations of the launch (2 per FMA); time the launch with
 * events on `stream`.  Bad arguments are ETICS_ERR_ARG. */
#define ETICS_PEAK_FFMA 0
#define ETICS_PEAK_FFMA2 1
#define ETICS_PEAK_DFMA 2
int etics_fma_peak(int kind, int blocks, int64_t iters, float *sink, double *flops_host,
                   void *stream);

/* Static description of a status code. */
const char *etics_strerror(int status);

/* Number of kernels this library has launched in this process. */
uint64_t etics_launch_count(void);

/* Profiling aid: when events is non-NULL, later calls record
 * events[k] (cudaEvent_t) at stage boundaries on their stream:
 *   SCF coeffs: 0 start, 1 after the coefficient kernel, 2 end;
 *   SCF field : 0 start, 1 end;
 *   MEX       : 0 start, 1 keys, 2 sorted, 3 tile sums, 4 carries, 5 end;
 *   MLP       : per product 0 start, 1 after the product, 2 after its epilogue
 *               (a multi-layer call keeps the last product's events).
 * n_events is the array length (recording stops at it).  NULL disables.
 * Not thread-safe: for single-threaded benchmarking. */
int etics_set_stage_events(void **events, int n_events);

#ifdef __cplusplus
}
#endif
#endif
