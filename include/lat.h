/*
 * lat.h - C ABI of the GB300 phase-space lattice library.
 *
 * The library advances the discretised phase-space density f(x, v, t) of heavy inertial
 * particles (Laenen, Krstulovic & Bec, arXiv:1508.02899) by the lattice method of Section 2:
 * an exact streaming shift in x by the lattice velocity index (dx = dv dt), a first-order
 * upwind finite-volume step of the Stokes drag a = -(v - u(x,t))/tau_p of Eq. (stokes_drag),
 * and a finite-volume velocity diffusion with coefficient kappa (Eq. conslaw), with zero flux
 * through the walls of the velocity box.  Every step runs in this library's CUDA kernels on
 * one GPU; there is no CPU fallback.
 *
 * Conventions shared by every call:
 *  - Every call returns an int status (LAT_OK = 0 or one of the LAT_E* codes below) except
 *    lat_strerror, lat_free and the small getters.  A failed call leaves the context as it
 *    was unless the code is LAT_ECUDA (the CUDA context may then be unusable).
 *  - Velocity lattice: N_v odd, J = (N_v - 1)/2, v_j = j dv for j = -J..J, dv = dx / dt,
 *    dx = L / N_x (Section 2; the cell centres span [-V_max, V_max] with V_max = J dv).
 *  - Layout of f in device memory, element type given by dtype, densely packed:
 *        d = 1: f[j][x]          (x fastest), N_v * N_x elements per instance;
 *               ensemble instances are concatenated in instance order.
 *        d = 2: f[jy][jx][y][x]  (x fastest), N_v^2 * N_y * N_x elements.
 *    f is a density: the mass of a cell is f dx^d dv^d (Section 3.2 normalisation).
 *  - Ownership: the caller owns the two device buffers f_a and f_b passed to lat_init /
 *    lat_ensemble_init and any device field passed to lat_set_flow; they must outlive the
 *    context.  Each step reads the current buffer and writes the other one; lat_current
 *    tells which one holds the state.  The context owns only its own scratch (flow state,
 *    noise table, reduction partials, CUDA graphs) and frees it in lat_free.
 *  - All work is enqueued on the stream given at init (NULL = legacy default stream);
 *    lat_step is asynchronous, lat_moments and lat_status synchronise that stream.
 *  - Device-side conditions (CFL exceeded by the evolving flow, exhausted noise table,
 *    non-finite values, FP16 scale overflow) are recorded in a device status word and
 *    reported by the next synchronising call (lat_moments, lat_status).
 */
#ifndef LAT_H
#define LAT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LAT_OK 0
#define LAT_EINVAL 1     /* bad argument (null pointer, size, layout, unsupported N_v) */
#define LAT_ECFL 2       /* Eq. (cfl) or Eq. (stabLapl) violated (host check or device flag) */
#define LAT_ENOMEM 3     /* device allocation of context scratch failed */
#define LAT_ECUDA 4      /* a CUDA runtime call failed */
#define LAT_ENUMERIC 5   /* non-finite value met in f (found by lat_moments) */
#define LAT_ETIMEOUT 6   /* a bounded device wait gave up */
#define LAT_EOVERFLOW 7  /* a reduced-precision value exceeded its line scale */
#define LAT_ENOISE 8     /* a step ran past the end of the noise table (flow frozen then) */

/* ---- storage types of f ---- */
#define LAT_F64 0
#define LAT_F32 1
#define LAT_F16 2
#define LAT_BF16 3

/* ---- flow kinds (lat_flow.kind) ---- */
#define LAT_FLOW_NONE 0   /* u = 0 */
#define LAT_FLOW_FIELD 1  /* caller's device field, frozen until the next lat_set_flow */
#define LAT_FLOW_MODES 2  /* synthetic random flow evolved on the device every step */

/* ---- drag schemes (lat_set_scheme) ---- */
#define LAT_SCHEME_UPWIND 0  /* first-order upwind flux, forward Euler (Sec. 2) */
#define LAT_SCHEME_KOREN 1   /* flux-limited, Heun's method (Sec. 2, flux limiter) */

typedef struct lat_ctx lat_ctx;

/* One lattice (Section 2).  d = 1: ny must be 1.  d = 2: the domain is nx*dx by ny*dx. */
typedef struct {
    int d;          /* spatial dimension, 1 or 2 */
    int nx, ny;     /* spatial cells */
    int nv;         /* velocity cells per component, odd, 1..129 */
    int dtype;      /* LAT_F64, LAT_F32 (d = 1, 2); LAT_F16, LAT_BF16 (d = 2) */
    double L;       /* period along x: dx = L / nx */
    double tau_p;   /* Stokes time of Eq. (stokes_drag); +inf switches the drag off */
    double kappa;   /* velocity diffusion coefficient of Eq. (conslaw), >= 0 */
    double dt;      /* time step; dv = dx / dt */
} lat_grid;

/* One member of a 1D ensemble (independent realisation, own size and parameters). */
typedef struct {
    int nx;
    double L, tau_p, kappa, dt;
} lat_instance;

/*
 * Carrier flow u(x, t).
 *  FIELD: `field` is a device array of d * ny * nx values (component-major: all u_x, then
 *    all u_y), double for LAT_F64 contexts and float otherwise.  For an ensemble it holds the
 *    instances' fields concatenated.  Not copied: it must stay valid while steps run.
 *  MODES, d = 1 (Sec. 3.1 Eq. u1d/A1d with M modes):
 *    u(x_i) = sum_m A_m cos(2 pi k_m i / N_x) + B_m sin(2 pi k_m i / N_x), with amplitudes
 *    that are Ornstein-Uhlenbeck processes of correlation time tau_f and stationary standard
 *    deviation sigma, updated exactly after every step:
 *        A <- A e^{-dt/tau_f} + sigma sqrt(1 - e^{-2 dt/tau_f}) xi,  xi ~ N(0,1) from the
 *    noise table (lat_set_noise).  k: host [M] wavenumbers; amp0: host [n_inst][2M] initial
 *    (A_0..A_{M-1}, B_0..B_{M-1}).  M <= 16.
 *  MODES, d = 2 (incompressible random-phase flow): psi = sum_m a_m cos(theta_m),
 *    theta_m = 2 pi (kx_m i / N_x + ky_m l / N_y) + phi_m, u = (d_y psi, -d_x psi); phases
 *    walk as phi <- phi + sqrt(2 dt / tau_f) xi.  k: host [M][2]; amp0: host [M] amplitudes
 *    a_m; phase0: host [M] initial phases.  M <= 512.
 *  tau_f <= 0 or infinite freezes the flow (no noise is consumed).
 * Step n uses the flow at t_n, then the flow state advances to t_{n+1}.
 */
typedef struct {
    int kind;
    const void* field;
    int nmodes;
    const int* k;
    const double* amp0;
    const double* phase0;
    double tau_f;
    double sigma;
} lat_flow;

/* Create a context for one lattice.  f_a holds the initial state; f_b is the other ping-pong
 * buffer (same size).  stream: a cudaStream_t or NULL.  Returns LAT_ECFL if the lattice is
 * unstable at rest: (dt/dv) J dv / tau_p > 1 (Eq. cfl with u = 0) or 2 d kappa dt/dv^2 > 1
 * (Eq. stabLapl generalised to d dimensions). */
int lat_init(lat_ctx** out, const lat_grid* g, void* f_a, void* f_b, void* stream);

/* Create a context for n_inst independent 1D lattices sharing N_v and dtype (F64 or F32),
 * advanced together by one persistent launch per step (captured in a CUDA graph). */
int lat_ensemble_init(lat_ctx** out, int n_inst, const lat_instance* inst, int nv, int dtype,
                      void* f_a, void* f_b, void* stream);

/* Set the carrier flow (see lat_flow).  Resets the noise table. */
int lat_set_flow(lat_ctx* c, const lat_flow* flow);

/* Copy `rows` steps of standard normal draws from host memory into the context's noise table;
 * row r feeds the flow update after the r-th following step.  Layout: d = 1 [rows][n_inst][2M],
 * d = 2 [rows][M].  Pinned host memory makes the copy asynchronous. */
int lat_set_noise(lat_ctx* c, const double* noise, long long rows);

/* Enqueue n time steps (Section 2: stream, drag, diffuse) on the context's stream.  In the
 * default launch mode the n steps are one CUDA-graph launch; the graph is captured on first use
 * of that n and cached (see lat_prepare). */
int lat_step(lat_ctx* c, int n);

/* Capture and instantiate the graph for n steps now, without running it, so that a later
 * lat_step(c, n) does no capture work. */
int lat_prepare(lat_ctx* c, int n);

/* Velocity moments of the current state (Sec. 3.2 normalisation; Sec. 4.2 density by summing
 * over v).  Per-cell outputs are DEVICE arrays of doubles (any may be NULL):
 *   rho = sum_j f dv^d;  mean_v = sum_j v_j f / sum_j f (d arrays of cells, component-major);
 *   mean_v2 = sum_j |v_j|^2 f / sum_j f; mean values are 0 where rho = 0.
 * `globals` is a HOST array (may be NULL): per instance [M, P_1..P_d, E] = sum f dx^d dv^d
 * times [1, v_1..v_d, |v|^2], formed with compensated (Neumaier) FP64 sums in a fixed order.
 * Synchronises; returns the pending device status (LAT_ECFL, LAT_ENUMERIC, ...) if any. */
int lat_moments(lat_ctx* c, double* rho, double* mean_v, double* mean_v2, double* globals);

/* lat_step(c, n) followed by lat_moments(c, ...), with the moments of the final state computed
 * inside the last step (no second pass over f) when the 1D producer/consumer kernel is in use,
 * or, in 2D, FP32 storage with the upwind drag on launch kernel 4, 5 or 8-10; otherwise exactly
 * the two calls.  Same arguments, outputs, synchronisation and status as
 * lat_moments.  The per-cell outputs equal lat_moments' bit for bit; the globals agree to the
 * rounding order of the compensated sums. */
int lat_step_moments(lat_ctx* c, int n, double* rho, double* mean_v, double* mean_v2,
                     double* globals);

/* lat_step_moments without the synchronisation, for a caller that reads each step's globals while
 * later steps run: enqueues the n steps, the reduction of the final state's global moments and
 * their copy into `globals` (HOST memory, pinned or registered, per instance [M, P_1..P_d, E] as
 * for lat_moments; not NULL) on the context's stream, and returns.  The values are in `globals`
 * once the stream has passed that point (the caller's cudaStreamSynchronize or event, or the
 * next synchronising call); `globals` must stay valid until then.  The device status of these
 * steps is reported by the next lat_status (or any synchronising call).  LAT_EINVAL for a NULL
 * `globals` or n < 1. */
int lat_step_moments_async(lat_ctx* c, int n, double* globals);

/* Synchronise, return and clear the pending device status. */
int lat_status(lat_ctx* c);

/* 0 if f_a holds the current state, 1 if f_b does. */
int lat_current(const lat_ctx* c);
/*
 * Reduced-precision storage (d = 2, dtype LAT_F16 or LAT_BF16).  The paper computes in double
 * precision; this storage form is this library's own (it halves the bytes a step moves).
 * Values are stored as 16-bit numbers h with one power-of-two scale S per x-line (velocity plane
 * (jx, jy) and row y): f = h * S.  The context owns the scales (two sets, one per buffer).
 * Each step decodes f*, computes in FP32 exactly like the FP32 path, and encodes with output
 * scales chosen from a bound of the step's growth (at most 3 times the largest input on the
 * 13-cell velocity diamond) so that encoded values stay below 2^15; the rounding residual of
 * every value is carried into the next value of the same cell's velocity column, so the stored
 * mass of a cell equals its FP32 mass up to one residual of the corner velocity cell.  A value
 * that still leaves the format's range (the CFL condition broken) raises LAT_EOVERFLOW.
 * The caller's f_a is taken at lat_init as 16-bit values with scale 1; lat_encode replaces the
 * current state.  FIELD flows are float arrays.
 */
/* Encode the FP32 DEVICE array src (layout of f, N_v^2 N_y N_x floats, caller-owned) into the
 * current buffer with fresh scales: S = 2^(ilogb(line max) - 12), residuals carried along each
 * cell's velocity column in (jy, jx) order.  Synchronises; LAT_EINVAL for other contexts. */
int lat_encode(lat_ctx* c, const float* src);
/* Decode the current state into the FP32 DEVICE array dst (may be NULL) and copy its line
 * scales, [jy][jx][y] floats, to the DEVICE array scales (may be NULL).  Synchronises. */
int lat_decode(lat_ctx* c, float* dst, float* scales);
/*
 * Learned flux closure on a coarse 2D lattice (d = 2, LAT_F32, N_v in {3, 5, 9, 13, 17},
 * N_x and N_y > (N_v + 1)/2, N_v^2 N_x N_y < 2^32; LAT_EINVAL otherwise).  The
 * paper proposes large-eddy closures for the lattice (Section 5); this library's closure adds
 * learned fluxes to the upwind drag fluxes of every interior velocity face, so mass is kept
 * exactly.  Per phase-space cell (x, j) after streaming, 16 features: f*(x, j + d)/rho*(x) for
 * the 3 x 3 velocity neighbourhood d = (dy, dx) (row-major, 0 outside the box; rho* the streamed
 * density), dt du_x/dx, dt du_x/dy, dt du_y/dx, dt du_y/dy (centred differences), the Courant
 * numbers g (u_x/dv - jx + J) and g (u_y/dv - jy + J), and 1; then h1 = relu(X W1 + b1),
 * h2 = relu(h1 W2 + b2), y = b tanh(z), z = h2 W3 + b3, with b = 1/4 for z <= 0 (extra
 * diffusion) and b = 0.9 |ca| (1 - |ca|) / 2 for z > 0 (anti-diffusion: at most 0.9 of the
 * upwind flux's numerical diffusivity; ca = the cell's drag Courant number - g/2).  Then
 * y_0 (f*_{jx+1} - f*_{jx}) and y_1 (f*_{jy+1} - f*_{jy}) join the drag fluxes through faces
 * jx + 1/2 and jy + 1/2 (a learned face diffusivity in lattice units).
 * params: HOST array of LAT_LEARN_NPARAM floats, W1 [16][64], b1 [64], W2 [64][64], b2 [64],
 *         W3 [64][2], b3 [2] (row-major, copied).
 * mode:   0 off (plain step), 1 FP32 network on CUDA cores, 2 BF16 network on the tensor cores
 *         (FP32 accumulation).  Every lat_step then runs the learned step.
 */
#define LAT_LEARN_NPARAM 5378
int lat_learn(lat_ctx* c, const float* params, int mode);
/* Enqueue the learned correction fluxes of the current state at the current step (the flow, the
 * streamed density, the network and G; the state and the flow do not advance) and, when G is not
 * NULL, copy them to the DEVICE array G of 2 N_v^2 N_y N_x floats: G[0] through faces jx + 1/2,
 * G[1] through faces jy + 1/2, zero on the walls.  reuse_inputs != 0 keeps the flow and the
 * streamed density of the previous call and runs the network alone (same state and step).
 * Asynchronous; LAT_EINVAL without lat_learn. */
int lat_learn_corrections(lat_ctx* c, float* G, int reuse_inputs);
/* Training loss after nsteps learned steps (the network of the lat_learn mode: FP32 on CUDA cores,
 * or BF16 on the tensor cores, whose backward and weight-gradient sums then run as tcgen05 MMAs
 * as well) from the current state against the
 * DEVICE array target (layout of f):
 *     loss = mean over all values of (f - target)^2 + rho_weight * mean over the spatial cells
 *            of (sum_j (f - target))^2,
 * and its exact gradient with respect to the parameters (HOST array grad of LAT_LEARN_NPARAM
 * floats), by the adjoint of every step; loss: HOST double.  The state, the flow and the step
 * count are left as they were (the flow's noise rows of the following nsteps steps are read).
 * Needs lat_learn with mode 1 or 2, a flow, nsteps <= 64 and rho_weight >= 0.  Synchronises. */
int lat_learn_grad(lat_ctx* c, int nsteps, const float* target, double rho_weight, double* loss,
                   float* grad);
/* Restriction of a fine 2D FP32 state (N_v = nv_fine = 4 m + 1 >= 5, layout of f, DEVICE) to the
 * coarse lattice of N_v = m + 1 velocities per axis with four times the velocity step (same dx and
 * V_max, so dt four times smaller): coarse cell k collects fine cells 4k - 2 .. 4k + 2 with weights
 * (1/2, 1, 1, 1, 1/2) per axis, divided by 16, which keeps the mass sum f dx^2 dv^2.  coarse:
 * DEVICE array of (m + 1)^2 ny nx floats.  Asynchronous on `stream`. */
int lat_restrict(const float* fine, int nv_fine, int nx, int ny, float* coarse, void* stream);

/* One Adam step (Kingma and Ba) of the learned closure's training, on DEVICE arrays of n floats
 * (caller-owned): g = grad_scale * grad; m <- beta1 m + (1 - beta1) g; v <- beta2 v +
 * (1 - beta2) g^2; params <- params - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps),
 * t >= 1 the step number.  FP32 arithmetic.  The paper has no counterpart (it trains nothing);
 * the closure's training is this library's.  Asynchronous on `stream`. */
int lat_adam(float* params, float* m, float* v, const float* grad, int n, int t, double lr,
             double beta1, double beta2, double eps, double grad_scale, void* stream);

/* Steps taken since init. */
long long lat_steps_done(const lat_ctx* c);

/* Launch shape of the step kernel.  Every variant gives the same bits.
 *  kernel: 0 keep; 1 plain coalesced loads (any size, FP32 or FP64).  The others bring the
 *          shifted plane windows into shared memory with bulk asynchronous copies (FP32; every
 *          N_x a multiple of 4 and >= 132):
 *          d = 1: 2..4 ring of that many item slots refilled after a block barrier;
 *                 5..7 producer warp + consumer warps on a ring of 2..4 slots (no barrier).
 *          d = 2: 2 ring refilled after a block barrier (block = 128 C threads splits each
 *                 cell's jx range over C = 1..4 warp groups);
 *                 3..7 producer warp + consumer warps (3: vy-drag flux row in registers,
 *                 4 slots; 4: in shared memory, 4 slots; 5: in shared memory, 3 slots; 6: the
 *                 vy-diffusion flux row in shared memory too, 3 slots; 7: as 6, 2 slots;
 *                 8..10 the sweep of two half-rows per thread in FP32 register pairs, the
 *                 vy-drag flux row in registers with 3 slots (8), in shared memory with 3 (9)
 *                 or 2 slots (10)).
 *          d = 2 with 16-bit storage: 1 plain loads (any size); 4..7 as above (N_x a
 *                 multiple of 8 and >= 136, N_v >= 9).
 *          d = 2 with the flux-limited scheme (lat_set_scheme): 1 three passes over the state
 *                 (any N_v); 2 one fused kernel per step (N_v >= 5; the default where it
 *                 exists).  Same bits up to the sign of zero values.
 *          d = 2 with the learned closure on the tensor cores (lat_learn mode 2): with a copy
 *                 pipeline and N_x a multiple of 128 the network takes all velocity planes of
 *                 128 x of one grid row in turn; with kernel 1 it takes tiles of 128 phase cells
 *                 in storage order.  Same bits.
 *  block:  threads per block (= x cells per tile) for kernel 1; the copy pipelines fix a 128-cell
 *          tile (2D kernel 2: 128 C threads); 0 keeps.
 *  blocks_per_sm: resident blocks per SM of the persistent grid; 0 keeps.  The fused
 *          flux-limited kernel takes 1 or 2 (FP32, N_v = 17 and 19: the register budget it is
 *          compiled for; 2 by default) and ignores it otherwise.
 *  mode:   -1 keep; 0 one persistent launch per step, n steps captured in one CUDA graph;
 *          1 one launch per instance per step (the unbatched baseline, 1D); 2 persistent
 *          launches issued directly (no graph).
 * Returns LAT_EINVAL for a shape the lattice does not support. */
int lat_set_launch(lat_ctx* c, int kernel, int block, int blocks_per_sm, int mode);

/* Drag sub-step scheme (Section 2 offers the first-order upwind flux and a flux-limiter scheme
 * after Hundsdorfer et al. with Koren's limiter, "parameter 2/3").
 *  scheme: LAT_SCHEME_UPWIND (default) or LAT_SCHEME_KOREN.  KOREN: the flux through interface
 *          j+1/2 is, for each split flux P = a^+ f and M = a^- f (cell-centre force) taken from
 *          its upwind side, q_j + psi(theta_j)(q_{j+1} - q_j) with theta_j = (q_j - q_{j-1}) /
 *          (q_{j+1} - q_j) and psi(theta) = max(0, min(1, 1/3 + theta/6, mu theta)); cells
 *          beyond the walls count as empty and the wall fluxes stay zero.  The sub-step is
 *          integrated by Heun's method: f1 = f + dt L(f), f_new = (f + f1 + dt L(f1)) / 2.
 *  mu:     limiter bound, 0 < mu <= 2 (2/3 reads the paper's parameter; 1 is the limiter's
 *          usual form); ignored for UPWIND.
 * Each Heun stage keeps f >= 0 when (dt/dv) max|a| (1 + mu) <= 1 (2D, unsplit: the sum of both
 * axes' maxima); lat_set_scheme checks the at-rest bound (dt/tau_p) J d (1 + mu) <= 1 of every
 * instance (LAT_ECFL otherwise) and the step kernels flag the local bound at run time.
 * 1D lattices and ensembles, FP32 or FP64, with N_v in {3, 5, 9, 17, 33, 65}: the limited sweep
 * runs inside every 1D step kernel.  2D lattices, FP32 or FP64, N_v^2 N_x N_y < 2^32 and
 * N_x, N_y > (N_v - 1) / 2: three
 * passes (two Heun stages, the diffusion) with a scratch copy of the state allocated here.  The
 * 16-bit and learned 2D paths keep the upwind scheme (LAT_EINVAL). */
int lat_set_scheme(lat_ctx* c, int scheme, double mu);

/* ---- observables (Section 3.2, Eqs. def_coarse and def_eulS1) ---- */

/* Second moment of the coarse-grained density.  rho_r(x) is the mass in a window of width r
 * around x (Eq. def_coarse); here r = w dx for whole numbers w of cells, the window of cell i
 * covering cells i .. i + w - 1, periodic (2D: the w x w square of cells from (y, x)).
 *   widths: host array of nw window widths in cells, 1 <= w <= N_x (2D: min(N_x, N_y)).
 *   out:    host array, out[k nw + q] = (1 / N_x) sum_i rho_r(x_i)^2 for instance k and width
 *           widths[q] (one instance for a single lattice or a 2D lattice; 2D divides by
 *           N_x N_y).  rho = sum_j f dv (dv^2 in 2D); rho_r in units of mass.
 * Window sums come from compensated FP64 prefix sums (a summed-area table in 2D) of the per-cell
 * density, the average from a compensated FP64 sum.  Synchronises; returns the pending device
 * status, LAT_EINVAL for nw outside 1..256 or a width out of range. */
int lat_coarse_moment(lat_ctx* c, int nw, const int* widths, double* out);

/* Eulerian first-order velocity structure function of 1D lattices (Eq. def_eulS1):
 *   num[k ns + q] = (1 / N_x) sum_i sum_j sum_j' f_j(x_i) f_j'(x_{i+s}) |v_j - v_j'| dv^2,
 *   den[k ns + q] = (1 / N_x) sum_i rho(x_i) rho(x_{i+s}),   S1(s dx) = num / den,
 * for instance k and separation s = seps[q] in cells (0 <= s < N_x, periodic).  The velocity
 * double sum runs in the state's precision by two running sums without cancellation (about
 * N_v u of its positive terms); sums over cells are compensated FP64.  FP32 or FP64 state.
 * Synchronises; LAT_EINVAL for 2D, ns outside 1..256 or a separation out of range. */
int lat_s1(lat_ctx* c, int ns, const int* seps, double* num, double* den);

/* Time candidate launch shapes on the current state without advancing it (reads the current
 * buffer, writes the other; the flow state is not advanced) and keep the fastest.  best[4]
 * (host, may be NULL) receives {kernel, block, blocks_per_sm, microseconds per step}. */
int lat_autotune(lat_ctx* c, int reps, double* best);

/* ---- host density I/O and checkpoints ------------------------------------------------------ */

/* Copy the current state to HOST memory as FP64 values, in the layout of f (N_v^d values per
 * spatial cell, instances concatenated; see the conventions above).  f_host: caller-owned host
 * array of N_v^d * (sum of the instances' N_x, or N_x N_y) doubles.  FP32 and 16-bit states
 * are widened exactly (16-bit values are decoded as h * S with their line scales).  Uses a
 * temporary device buffer (at most 512 MiB for FP32 states; 12 bytes per value for 16-bit
 * states).  Synchronises; returns the pending device status. */
int lat_get_density(lat_ctx* c, double* f_host);

/* Replace the current state by the FP64 HOST array f_host (layout as lat_get_density).  FP32
 * storage rounds each value to nearest; 16-bit storage encodes the FP32-rounded values with
 * fresh line scales, as lat_encode does.  The step count, the flow and the noise table are not
 * touched.  Synchronises; returns the pending device status (LAT_EOVERFLOW if a value does not
 * fit the 16-bit format). */
int lat_set_density(lat_ctx* c, const double* f_host);

/*
 * Checkpoints.  The image holds everything of a context that evolves with the steps, so that a
 * run resumed from it continues bit for bit (Section 2's scheme is a deterministic map of this
 * state and the noise draws):
 *   - the current density buffer in its storage type, and for 16-bit storage its line scales
 *     and line maxima;
 *   - the step count;
 *   - the flow state at that step: the Ornstein-Uhlenbeck amplitudes of a 1D modal flow (FP64
 *     and the FP32 copy the FP32 kernels read) or the phases of a 2D modal flow;
 *   - the noise rows the context holds for this and later steps, with where they start.
 * It does not hold what the caller sets once: the geometry, the flow's kind, wave vectors and
 * constants, a FIELD flow's array, the drag scheme, the launch shape and the learned closure's
 * parameters.  To resume, create a context with the same lat_grid (or instances), call
 * lat_set_flow with the same flow (and lat_learn / lat_set_scheme as before), then
 * lat_set_state.  The image is a flat byte array in host byte order, starting with a header
 * that identifies the context's geometry and flow; it is not meant to move between hosts of
 * different byte order.
 */
/* Size in bytes of the image of the context's present state (HOST long long).  Synchronises. */
int lat_state_bytes(lat_ctx* c, long long* bytes);
/* Write the image into the HOST buffer `image` of `bytes` bytes (at least lat_state_bytes).
 * Synchronises; LAT_EINVAL if the buffer is too small.  The context is not changed. */
int lat_get_state(lat_ctx* c, void* image, long long bytes);
/* Restore the state from an image made by lat_get_state of a context with the same geometry,
 * instances, dtype and flow kind / mode count (LAT_EINVAL otherwise, the context unchanged).
 * Writes the density into the buffer that the image's step count selects (lat_current), the
 * scales, the flow state into both parities and the noise rows into the noise table (grown if
 * needed); clears the pending status.  Synchronises. */
int lat_set_state(lat_ctx* c, const void* image, long long bytes);

/* Test hook of the timeout path (the paper has no counterpart; the waits are this library's
 * bulk-copy pipelines).  While on != 0, the producer warp of every producer/consumer step
 * kernel (1D launch kernels 5..7, 2D kernels 3..7, 16-bit kernels 4..7: the defaults where the
 * sizes allow them) issues no copies, so each consumer warp's bounded wait on its first row
 * gives up after about one second; the step then writes no output and the next synchronising
 * call returns LAT_ETIMEOUT.  No copy is in flight when a wait gives up, and the context stays
 * usable: turn the hook off and step again.  Kernels without a pipeline ignore it.
 * Asynchronous (ordered on the context's stream). */
int lat_debug_stall(lat_ctx* c, int on);

/* Human-readable text of a status code. */
const char* lat_strerror(int status);

/* Release the context's scratch.  Does not touch f_a, f_b or a caller's field. */
void lat_free(lat_ctx* c);

/* ---- allocation-free entry point ---------------------------------------------------------- */

/* Largest number of 128-column tiles lat_moments1d_noalloc accepts: N_x <= 8192 * 128. */
#define LAT_NOALLOC_MAX_TILES 8192

/*
 * Global moments [M, P, E] = sum f dx dv * [1, v, v^2] of one 1D FP32 lattice, computed without
 * allocating anything.  It gives the same result as the globals of lat_moments on the same
 * state, to rounding order.  The paper has no counterpart; this call exists for callers that
 * must not allocate device memory, for example:
 *  - code running inside another runtime that has reserved the GPU's memory for its own pool;
 *  - latency-critical loops in which cudaMalloc or cudaFree would synchronise the device.
 * Such callers cannot create a lat_ctx, whose scratch is allocated with cudaMalloc.
 *
 *   f        DEVICE array f[j][x] of nv * nx floats (layout of include/lat.h), caller-owned.
 *   nv, nx   odd N_v >= 1; 1 <= N_x <= LAT_NOALLOC_MAX_TILES * 128, else LAT_EINVAL with a
 *            message on stderr, before anything is launched.
 *   dx, dv   lattice spacings (> 0).
 *   globals  DEVICE array of 3 doubles, caller-owned, written asynchronously.
 *   stream   cudaStream_t or NULL.
 *
 * The scratch is a fixed static device array of LAT_NOALLOC_MAX_TILES * 6 doubles (384 KiB).
 * Every GPU that loads this library holds it until the process exits.  The function calls no
 * cudaMalloc, cudaFree or any other allocating routine.
 *
 * The first call on each device looks up that array's device address (cudaGetSymbolAddress,
 * with the device current).  Make that first call before any stream capture on the device.
 *
 * Every call shares the one array and overwrites the slots it uses, so nothing needs clearing.
 * Calls that overlap on the GPU (on different streams, or from several threads without
 * ordering) race on the array and give wrong results.  Returns LAT_OK, LAT_EINVAL or LAT_ECUDA.
 */
int lat_moments1d_noalloc(const float* f, int nv, int nx, double dx, double dv, double* globals,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LAT_H */
