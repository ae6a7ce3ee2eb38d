/*
 * turret.h -- C ABI of libturret.so, the GB300 (sm_103a) hot path of one time
 * step of the Palabos Turret method (Bhowmick, Latt, Wang, Bagheri,
 * arXiv 2408.15115): recursive-regularized D3Q27 lattice Boltzmann
 * collide+stream over a window that follows a settling particle, immersed-
 * boundary multi-direct forcing on the particle's surface markers, the
 * stress-based surface force and torque, and the rigid-body (6DOF) update.
 *
 * Conventions shared by every call
 *   - Lattice units: dx = dt = 1, rho_0 = 1, c_s^2 = 1/3 (Sec. 2.1).
 *   - Window coordinates: cell centres at integer (x, y, z), 0 <= x < nx, ...;
 *     x is the fastest index of every field; z is "up" (gravity along -z).
 *   - Device memory is owned by the caller.  lbm_init and ibm_load_surface
 *     borrow a caller-allocated device workspace (sizes from the *_bytes
 *     queries) until lbm_destroy; host arrays are copied during the call.
 *   - Every call enqueues its GPU work on the caller's CUDA stream given to
 *     lbm_init.  Only query_particle_state, lbm_copy_* and lbm_set_fields wait
 *     for the stream.
 *   - Errors: every call returns a turret_status; nothing aborts or throws
 *     across the ABI.  turret_last_error() holds a message for the last
 *     failure.  Conditions detected on the device during step() (a marker
 *     stencil leaving the window, a non-finite force) are latched in a device
 *     status word and returned by the next query_particle_state().
 */
#ifndef TURRET_H
#define TURRET_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TURRET_API __attribute__((visibility("default")))
#else
#define TURRET_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct turret_ctx turret_ctx;

typedef enum {
    TURRET_OK = 0,
    TURRET_EINVAL = 1,    /* invalid argument (sizes, tau <= 1/2, bad mesh, ...)      */
    TURRET_ENOMEM = 2,    /* workspace too small                                       */
    TURRET_ECUDA = 3,     /* a CUDA runtime call failed                                */
    TURRET_ESTATE = 4,    /* call out of order (e.g. step before ibm_load_surface)     */
    TURRET_EDIVERGED = 5, /* non-finite force or torque                                */
    TURRET_ETIMEOUT = 6,  /* a bounded device wait gave up                             */
    TURRET_EDOMAIN = 7,   /* a marker stencil left the window along a closed axis      */
    TURRET_EOVERFLOW = 8  /* more markers touch one 4^3 support tile than its list holds */
} turret_status;

typedef enum { TURRET_D3Q27 = 27 } turret_lattice;

/* Population storage.  Populations are stored as deviations q_i = f_i - w_i
 * from the rest equilibrium: FP32 as is; FP16 as q_i * 16 / w_i; BF16 as
 * q_i / w_i (round to nearest even).  Arithmetic is FP32 in every case.     */
typedef enum { TURRET_F32 = 0, TURRET_F16 = 1, TURRET_BF16 = 2 } turret_storage;

enum { TURRET_BC_PERIODIC = 0, TURRET_BC_NOSLIP = 1, TURRET_BC_PRESSURE = 2, TURRET_BC_MOVING = 3 };

/* Simulation window (Sec. 2.5, Fig. 1).  bc_x, bc_y: periodic or no-slip
 * (halfway bounce-back).  bc_bottom: periodic, no-slip or moving wall.
 * bc_top: periodic, no-slip, constant pressure (ghost plane at rest density
 * with the velocity of the top plane) or moving wall.  A moving wall is a
 * no-slip wall sliding in its plane with the velocity set by
 * lbm_set_wall_velocity (shear flows; not with slide = 1).  sponge_cells: planes below the top over which tau rises
 * linearly to 1 on the top plane.  slide = 1: the window follows the particle
 * vertically as a ring buffer (replaces the re-injection copy of Sec. 2.5);
 * the particle centre is kept within one cell of z = anchor_frac * nz.      */
typedef struct {
    int32_t nx, ny, nz;
    int32_t bc_x, bc_y;
    int32_t bc_bottom, bc_top;
    int32_t sponge_cells;
    int32_t slide;
    int32_t pad0;
    double anchor_frac;
} turret_window;

/* Readings of points the paper leaves open (all default 0):
 *   force_scheme 0: f* = (1-1/tau) f0(u) + (1/tau) f0(u + tau h) + (1-1/tau) f1
 *                   (adds rho h per step); 1: Eq. 15 as printed.
 *   rot_form     0: angular momentum L advanced by T, omega = M^T J^-1 M L;
 *                1: omega advanced by M^T J^-1 M T as printed (Sec. 2.3).
 *   gravity      0: g_eff = (1 - 1/kappa) g (buoyancy); 1: g as printed.
 *   renorm_orientation 1: modified Gram-Schmidt of d_0, d_1, d_2 each step.
 *   ibm_cycles: number n of IBM cycles (Sec. 2.2: n = 4).
 *   no_graph 1: launch every kernel of a step directly instead of replaying a
 *               captured CUDA graph (same results; for debugging).
 *   fixed_position 1: the particle's centre is held (v = 0) while its
 *               rotation stays free (a sphere spun up by a shear flow).
 *   force_eval 0: the surface stress is taken on the surface offset by two
 *               cells along the marker normals (areas and arms of that
 *               surface), whose interpolation stencils lie in the fluid
 *               outside the diffuse interface; 1: at the markers, as printed
 *               in Sec. 2.2 (which averages in the fluid inside the body and
 *               gives 2-3 times too small a drag and torque).
 *   stochastic_rounding 1 (BF16 storage only): the collide+stream stores
 *               round each stored value up or down with probability equal to
 *               its distance from the other neighbour (unbiased rounding),
 *               the random bits a hash of (element pair, time step), one hash
 *               per pair of elements 2k, 2k + 1 of a population array:
 *               results stay deterministic and independent of the kernel.
 *               0: round to nearest even.
 *   staged_loads 1 (FP16 / BF16 storage): the bulk collide+stream moves its
 *               tiles' sources and results through shared memory with bulk
 *               tensor copies (a producer warp and four computing warps per
 *               block) instead of the default x-adjacent cell pairs with
 *               4-byte global loads and stores (0, the default, measured
 *               faster).  Results are identical.                           */
typedef struct {
    int32_t force_scheme;
    int32_t rot_form;
    int32_t gravity;
    int32_t renorm_orientation;
    int32_t ibm_cycles;
    int32_t no_graph;
    int32_t stochastic_rounding;
    int32_t fixed_position;
    int32_t force_eval;
    int32_t staged_loads;
} turret_flags;

/* Particle state (Sec. 2.3): r = centre of mass in global lattice coordinates
 * (window origin included), d = rows d_0, d_1, d_2 of the orientation matrix M,
 * v, w at t - 1/2 (leap-frog), F, T = hydrodynamic force and torque at t
 * (rho_f = 1; the stress integrated over the surface that flags.force_eval
 * selects: by default the surface offset two cells along the normals, torque
 * about the centre of mass), L = angular momentum at t - 1/2, origin = global
 * coordinates of window cell (0, 0, 0), step = t, status = latched device
 * status.                                                                    */
typedef struct {
    double r[3], d[9], v[3], w[3], F[3], T[3], L[3];
    int64_t origin[3];
    int64_t step;
    int32_t status;
    int32_t n_markers;
    double volume;   /* particle volume V                                  */
    double area;     /* surface area, sum of the marker areas dS_k          */
    int32_t kernels_per_step;  /* kernel launches one step() enqueues      */
    int32_t pad0;
    double Fp[3];    /* pressure part of F: sum_k dA_k (-p(Y_k)) n_k over the
                      * same surface (Y_k = X_k + 2 n_k, dA_k its areas, by
                      * default; X_k, dS_k with force_eval 1), with
                      * p = c_s^2 (rho - 1) the isotropic part of Eq. 10;
                      * F - Fp is the viscous (shear) part                 */
} turret_particle_state;

/* ---- fluid ------------------------------------------------------------- */

/* Bytes of device workspace lbm_init needs for this window and storage.     */
TURRET_API size_t lbm_workspace_bytes(const turret_window *win, turret_storage st);

/* Creates a context.  nu: kinematic viscosity, tau = 3 nu + 1/2 (Eq. 9), must
 * give tau > 1/2.  rho_ratio: kappa = rho_p / rho_f.  g: gravity (3 doubles).
 * device_workspace: >= lbm_workspace_bytes bytes of device memory, 256-byte
 * aligned.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * The fluid starts at rest (all deviations zero).  *out receives the context. */
TURRET_API turret_status lbm_init(turret_ctx **out, const turret_window *win, turret_lattice lat, double nu,
                       double rho_ratio, const double g[3], turret_storage st, void *device_workspace,
                       size_t workspace_bytes, void *cuda_stream);

/* Replaces the reading flags (before ibm_load_surface). */
TURRET_API turret_status lbm_set_flags(turret_ctx *c, const turret_flags *flags);

/* Velocities (3 doubles each, the normal component must be 0) of the bottom
 * and top walls of bc TURRET_BC_MOVING.  The halfway bounce-back of a moving
 * wall adds the momentum it imparts, f_i(x) = f*_{opp i}(x) + 2 w_i (xi_i .
 * u_w) / c_s^2 (reference density 1), for every population whose source lies
 * beyond that face.  EINVAL for a normal component or a speed above 0.3.    */
TURRET_API turret_status lbm_set_wall_velocity(turret_ctx *c, const double u_bottom[3], const double u_top[3]);

/* Sets the state to the equilibrium of the given host fields, as the
 * post-collision populations at t = -1: rho (nz*ny*nx doubles, NULL = 1) and
 * u (nz*ny*nx*3 doubles, (x,y,z) per cell, NULL = 0), z-major then y then x.
 * The pressure-ghost velocity is the u of the top plane.  Synchronous.      */
TURRET_API turret_status lbm_set_fields(turret_ctx *c, const double *rho, const double *u);

/* ---- particle ------------------------------------------------------------ */

/* Bytes of device workspace ibm_load_surface needs for this surface.        */
TURRET_API size_t ibm_workspace_bytes(const turret_ctx *c, const double *verts_body, int64_t n_verts, const int32_t *tris,
                           int64_t n_tris);

/* Loads the particle surface (Sec. 2.2: the mesh vertices are the Lagrangian
 * markers; dS_k is one third of the area of the triangles sharing vertex k).
 * verts_body: n_verts x 3 doubles; tris: n_tris x 3 int32, counter-clockwise
 * seen from outside; the mesh must be closed.  The body is re-centred on its
 * centre of mass; body frame = lab frame at t = 0.  r0: centre of mass in
 * window coordinates; v0, w0: v(-1/2), omega(-1/2).  Computes F(0), T(0) and
 * h_imm(0) (Table 1 events 3 and 4 at t = 0).  device_workspace: >=
 * ibm_workspace_bytes bytes, 256-byte aligned.                               */
TURRET_API turret_status ibm_load_surface(turret_ctx *c, const double *verts_body, int64_t n_verts, const int32_t *tris,
                               int64_t n_tris, const double r0[3], const double v0[3], const double w0[3],
                               void *device_workspace, size_t workspace_bytes);

/* ---- time stepping ---------------------------------------------------------- */

/* Advances n coupled time steps in the order of Table 1: collide+stream with
 * h_imm(t), particle update with F(t), T(t), window slide, stress and velocity
 * at t+1 on the support box, F(t+1), T(t+1), IBM cycles -> h_imm(t+1).
 * Without a particle, advances the fluid alone.  Asynchronous; replays CUDA
 * graphs: groups of 8 steps as one graph in which the immersed-boundary chain
 * of a step overlaps the bulk collide+stream of the next (same results as
 * one graph per step), the remaining steps one graph each.                  */
TURRET_API turret_status step(turret_ctx *c, int64_t n);

/* Advances the fluid alone by n collide+stream steps (Eq. 7 / Eq. 15 with
 * h_imm held at its current value; the particle does not move).  Launches
 * only the fused collide+stream kernels a coupled step uses for the window:
 * with a particle whose support box is small against the window, the
 * far-cell launch on the context's stream and the near-region launch beside
 * it on the context's internal stream (the two write disjoint cells), joined
 * before the next step, as in the coupled step; otherwise one launch over the
 * whole window.  Asynchronous: ordered after earlier work on the context's
 * stream, and later work on it is ordered after both launches.             */
TURRET_API turret_status lbm_fluid_step(turret_ctx *c, int64_t n);

/* Copies the particle state to the host (waits for the stream); returns the
 * latched device status (TURRET_EDOMAIN, TURRET_EDIVERGED) if one was set.   */
TURRET_API turret_status query_particle_state(turret_ctx *c, turret_particle_state *out);

/* Density and unforced velocity u = sum xi f / sum f of f(t) at every cell
 * (Eqs. 5-6), written to caller device memory dev_out as 4 planes
 * [rho, u_x, u_y, u_z][nz][ny][nx] of floats in window order.  Waits.        */
TURRET_API turret_status lbm_copy_macro(turret_ctx *c, float *dev_out);

/* Deviations q_i = f_i(t) - w_i of the pre-collision populations at every
 * cell, written as float [27][nz][ny][nx] in window order, population index
 * i = (xi_x+1) + 3 (xi_y+1) + 9 (xi_z+1).  Waits.                           */
TURRET_API turret_status lbm_copy_populations(turret_ctx *c, float *dev_out);

/* ---- standalone operator ------------------------------------------------------ */

/* Bytes of device workspace ibm_spread needs (0 for invalid sizes).         */
TURRET_API size_t ibm_spread_workspace_bytes(int32_t nx, int32_t ny, int32_t nz, int64_t n_markers);

/* The spreading step of the immersed-boundary method (Sec. 2.2, step l = 1)
 * on an nx x ny x nz grid with cell centres at integer coordinates:
 *   field(x) = sum_k h_k W(x - X_k) dS_k,  W the 3-D Peskin 4-point kernel.
 * X: device [3][n_markers] floats (all x, then all y, then all z); h: device
 * [3][n_markers] floats; dS: device [n_markers] floats; field: device
 * [3][nz][ny][nx] floats, overwritten.  Every marker's 4x4x4 stencil
 * (floor(X) - 1 .. floor(X) + 2 per axis) must lie inside the grid
 * (TURRET_EDOMAIN otherwise; such markers contribute nothing).  Grid sides
 * 4..1023.  workspace: >= ibm_spread_workspace_bytes, 256-byte aligned.
 * Enqueued on `stream`; waits for it and returns the status.  Bitwise
 * reproducible (fixed summation order, no atomics).                        */
TURRET_API turret_status ibm_spread(const float *X, const float *h, const float *dS, int64_t n_markers, int32_t nx,
                                    int32_t ny, int32_t nz, float *field, void *workspace, size_t workspace_bytes,
                                    void *stream);

/* ibm_spread without a workspace, for callers that cannot allocate device
 * memory (a host framework whose pool owns the device, a plugin given no
 * allocator, a real-time loop that forbids allocation after start-up).  The
 * paper has no counterpart; this is a deployment variant of ibm_spread with
 * the same arguments minus the workspace and the same results.  Scratch comes
 * from a fixed 8 MiB array in the library's device image, held by every GPU
 * that loads the library until the process exits; sizes whose
 * ibm_spread_workspace_bytes exceed it return TURRET_ENOMEM.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make it before any stream capture.  All calls on a device
 * share the one array: calls whose GPU work overlaps (other streams, other
 * threads) race and must be serialised by the caller.  The looked-up address
 * is kept for the life of the process: after cudaDeviceReset on a device
 * (which unloads the library's device image there) this entry point must not
 * be called on that device again.  Waits for `stream`.                      */
TURRET_API turret_status ibm_spread_noalloc(const float *X, const float *h, const float *dS, int64_t n_markers,
                                            int32_t nx, int32_t ny, int32_t nz, float *field, void *stream);

/* ---- batched ensemble ------------------------------------------------------ */

/* Many independent settling runs advanced together.  The paper has no
 * counterpart (it simulates one particle at a time); a batch is a throughput
 * form of step() over runs of different shapes, windows, viscosities and
 * storage types.  Each turret_step of a batch launches every phase of the
 * step (collide+stream, particle + markers, support moments, interpolation,
 * IBM cycles, spreading, F/T reduction) ONCE for all runs, over a table of
 * (run, block) pairs, and replays it as one CUDA graph per step parity.  The
 * per-cell and per-marker arithmetic is the single-run arithmetic, so every
 * run of a batch evolves bit for bit as it does alone under step().          */
typedef struct turret_batch turret_batch;

/* Bytes of device workspace a batch of n_runs runs needs (descriptors and
 * per-phase block tables); 0 for n_runs < 1.                                */
TURRET_API size_t turret_batch_workspace_bytes(int32_t n_runs);

/* Groups n_runs contexts into a batch.  Every context must hold a particle
 * (ibm_load_surface done), be at a time level of the same parity and use the
 * same ibm_cycles; a context appears once.  The contexts stay owned by the
 * caller and must outlive the batch.  GPU work of the batch is
 * enqueued on `stream` (the caller's); turret_batch_step orders it after the
 * work already enqueued on each context's stream and makes each context's
 * stream wait for it, so query_particle_state on a context sees the batched
 * steps.  device_workspace: >= turret_batch_workspace_bytes, 256-byte
 * aligned.  Initial tiles: 128 threads per block, tile width 32, register
 * budget variant 2 (see turret_batch_set_tiles).                           */
TURRET_API turret_status turret_batch_init(turret_batch **out, turret_ctx *const *ctxs, int32_t n_runs,
                                           void *device_workspace, size_t workspace_bytes, void *stream);

/* Collide+stream launch shape of a batch: threads per block (64, 128, 256),
 * register-budget variant minb (2: <= 128 registers per thread, 3: <= 85, the
 * number of resident 256-thread blocks per SM the compiler plans for) and per
 * run the tile width tx[r] in {16, 32, 64, 128} (<= threads; the tile covers
 * tx cells along x and threads / tx rows along y of a pair of planes, two
 * cells per thread).  Results do not depend on these.  Waits.              */
TURRET_API turret_status turret_batch_set_tiles(turret_batch *b, int32_t threads, int32_t minb, const int32_t *tx);

/* Advances every run of the batch by n coupled steps (the order of step()).
 * Runs may be stepped alone between calls; every run must then still be at a
 * time level of the same parity (TURRET_ESTATE otherwise).                  */
TURRET_API turret_status turret_batch_step(turret_batch *b, int64_t n);

/* Releases the batch (not the contexts or the workspace); waits for it.     */
TURRET_API turret_status turret_batch_destroy(turret_batch *b);

/* Message of the last failure on this batch (or of the last failed
 * turret_batch_init when b is NULL).                                        */
TURRET_API const char *turret_batch_last_error(const turret_batch *b);

/* Times `reps` launches of the collide+stream kernel of one context with the
 * given launch shape (as turret_batch_set_tiles), from the current time level
 * into the idle population buffer, so the context's state is unchanged; the
 * mean duration in microseconds goes to *us_out.  Used by the tile
 * autotuner.  Waits for the context's stream.                               */
TURRET_API turret_status turret_time_collide(turret_ctx *c, int32_t threads, int32_t tx, int32_t minb, int32_t reps,
                                             float *us_out);

/* ---- force/torque surrogate network ------------------------------------------ */

/* A small multilayer perceptron that predicts the particle's next
 * hydrodynamic force and torque from its recent state; the paper has no
 * counterpart (its only predictor is the orientation predictor-corrector of
 * Sec. 2.3).  Architecture: TURRET_MLP_IN = 34 inputs -> three hidden layers
 * of 128 units with the exact GELU x Phi(x) -> TURRET_MLP_OUT = 6 outputs,
 * applied to standardised inputs (x - mean_x) / std_x; outputs are
 * standardised targets, returned de-standardised.  Parameters are a flat
 * float array of TURRET_MLP_NPARAM values: W1 [128][34], b1 [128],
 * W2 [128][128], b2 [128], W3 [128][128], b3 [128], W4 [6][128], b4 [6]
 * (row-major, y = W x + b per layer).  precision 0: matrix products on BF16
 * tensor cores (weights and activations rounded to BF16, FP32 accumulation);
 * precision 1: FP32 throughout (a check mode).  Training: mean squared error
 * of the standardised outputs, AdamW with decoupled weight decay on the
 * weight matrices.  All calls run on the stream given to mlp_init.         */
#define TURRET_MLP_IN 34
#define TURRET_MLP_OUT 6
#define TURRET_MLP_NPARAM 38278
typedef struct turret_mlp turret_mlp;
typedef struct {
    float lr, beta1, beta2, eps, weight_decay;
} turret_adamw;

/* Device workspace for a network trained on batches of up to batch_cap rows
 * (0 for batch_cap outside 1 .. 16384).                                     */
TURRET_API size_t mlp_workspace_bytes(int32_t batch_cap);
/* Creates a network with the host parameters `params` [TURRET_MLP_NPARAM],
 * identity standardisation and zero optimiser moments; waits.               */
TURRET_API turret_status mlp_init(turret_mlp **out, int32_t batch_cap, int32_t precision, const float *params,
                                  void *device_workspace, size_t workspace_bytes, void *stream);
/* Copies parameters from / to the host; wait.                               */
TURRET_API turret_status mlp_set_params(turret_mlp *m, const float *params);
TURRET_API turret_status mlp_get_params(turret_mlp *m, float *params);
/* Sets the standardisation (host arrays of 34, 34, 6, 6 floats; std > 0).   */
TURRET_API turret_status mlp_set_norm(turret_mlp *m, const float *mean_x, const float *std_x, const float *mean_y,
                                      const float *std_y);
/* y [n][6] = network(x [n][34]), device arrays, 1 <= n <= batch_cap, with the
 * training kernels (batched matrix products).  Asynchronous.               */
TURRET_API turret_status mlp_forward(turret_mlp *m, const float *x, int32_t n, float *y);
/* The same outputs from the fused inference kernel (16 rows per block, any
 * n >= 1), as used by the particle predictor.  Asynchronous.               */
TURRET_API turret_status mlp_infer(turret_mlp *m, const float *x, int32_t n, float *y);
/* Loss of raw targets y [n][6] and, if grad is not NULL, its gradient with
 * respect to the parameters into device memory grad [TURRET_MLP_NPARAM].
 * Waits.                                                                    */
TURRET_API turret_status mlp_loss_grad(turret_mlp *m, const float *x, const float *y, int32_t n, float *loss,
                                       float *grad);
/* One AdamW step on the batch (x, y); the loss before the step to *loss if
 * loss is not NULL (then waits).                                            */
TURRET_API turret_status mlp_train_step(turret_mlp *m, const float *x, const float *y, int32_t n,
                                        const turret_adamw *opt, float *loss);
/* Releases the network (not the workspace).                                 */
TURRET_API turret_status mlp_destroy(turret_mlp *m);
TURRET_API const char *mlp_last_error(const turret_mlp *m);

/* ---- force/torque predictor (surrogate modes) -------------------------------- */

/* The paper's step (mode 0, the default) forms the marker target velocities
 * U_k from v, w at t + 1/2 and runs ibm_cycles IBM cycles from h = 0.  The
 * predictor modes, which the paper does not have, predict the force and
 * torque of the next time level -- mode 1 by linear extrapolation
 * 2 F(t) - F(t-1), mode 2 by the network `net` (kept by the caller; it
 * corrects the linear extrapolation, see mlp_build_samples) with linear
 * extrapolation as its fallback: in mode 2 the network runs at every step
 * once four time levels of history exist, and its prediction is used unless
 * its previous one missed the force by |F - F^| / |F| > resid_theta.
 * options (bits):
 *   TURRET_PRED_VEL:  form U_k from the estimates
 *       v(t+1) = v(t+1/2) + (g_eff + F^/m) / 2 and L(t+1) = L(t+1/2) + T^/2
 *       (w(t+1) = w(t+1/2) + (J/m)^-1 T^/(2m) in the literal rotation form);
 *   TURRET_PRED_WARM: start the IBM cycles from the previous step's
 *       Lagrangian force and run at most ibm_cycles of them, skipping the
 *       rest once the slip max_k |U_k - I[u* + S h](X_k)| is below slip_eps;
 *   TURRET_PRED_REL: resid_theta is a ratio: the network's prediction is used
 *       while the running mean (weight 1/8 per time level) of its error is at
 *       most resid_theta times the running mean of linear extrapolation's
 *       error on the same time levels.
 * Takes effect for the following steps (a batch copies it when created).    */
#define TURRET_PRED_WARM 1
#define TURRET_PRED_VEL 2
#define TURRET_PRED_REL 4
TURRET_API turret_status turret_set_predictor(turret_ctx *c, int32_t mode, const turret_mlp *net, int32_t options,
                                              double slip_eps, double resid_theta);

/* The re-injection copy of Sec. 2.5 instead of a sliding window (windows
 * with slide = 0; trigger 0 switches it off): once the particle centre's
 * window z falls below the plane `trigger`, the post-collision planes
 * [zf - below, zf + above) around it (zf = floor of that z, clipped to the
 * window; planes that would leave the top are dropped) are copied up by
 * target - zf and the window origin moves down by as much, so the particle
 * keeps its global position and lands at plane `target`; the rest of the
 * fluid is left as it was.  Steps then run without the far/near split (one
 * collide+stream launch over the window).  EINVAL unless
 * 0 < trigger < target < nz and below + above <= nz.                       */
TURRET_API turret_status turret_set_reinjection(turret_ctx *c, int32_t trigger, int32_t target, int32_t below,
                                                int32_t above);

/* Trajectory log: after the force of each time level j is known, record
 * (n mod capacity), n the count of records written so far, of the caller's
 * device array records [capacity][TURRET_LOG_REC] doubles receives d(j) [9]
 * (rows of the orientation matrix), v(j - 1/2) [3], w(j - 1/2) [3], F(j)
 * [3], T(j) [3], j, the relative error |F - F^| / |F| of the prediction made
 * for j (or -1), F^ [3], T^ [3], 1 if the network made it (0 linear, -1 no
 * prediction), the relative error of the network's prediction for j (or -1:
 * the network did not run), 0.  capacity 0 detaches the log.               */
#define TURRET_LOG_REC 32
TURRET_API turret_status turret_set_log(turret_ctx *c, double *records, int64_t capacity);

typedef struct {
    int64_t steps;      /* predictions made                                   */
    int64_t net_steps;  /* ... of them by the network                          */
    int64_t fallbacks;  /* linear predictions made in network mode             */
    int64_t cycles;     /* IBM cycles run in the predictor modes               */
    int64_t logged;     /* trajectory records written                          */
    double resid;       /* |F - F^| / |F| of the last checked prediction       */
    double slip[8];     /* slip seen by each IBM cycle of the last step        */
    int32_t hist_n, fallback;
} turret_predictor_stats;

/* Counters of the predictor (waits for the stream).                        */
TURRET_API turret_status turret_query_predictor(turret_ctx *c, turret_predictor_stats *out);

/* Training pairs of the network from n_records consecutive records of a
 * trajectory log (device): sample j (0 <= j < n_records - 4) is built at
 * t = record j + 3, in the body frame M of t.  Inputs x [j][34]: quaternion
 * (w >= 0) of M, M v, M w, then M F / sF, M T / sT of records t, t - 1,
 * t - 2, t - 3, with sF, sT the largest of those four force and torque
 * magnitudes.  Targets y [j][6]: M (F(t+1) - 2 F(t) + F(t-1)) / sF and the
 * torque alike -- the departure from linear extrapolation, which the
 * predictor adds back (F^ = 2 F(t) - F(t-1) + sF M^T y).  Records whose time
 * levels are not consecutive give NaN inputs and are counted in the device
 * integer *bad.  Asynchronous on `stream`.                                 */
TURRET_API turret_status mlp_build_samples(const double *records, int64_t n_records, float *x, float *y, int32_t *bad,
                                           void *stream);

/* ---- checkpoints --------------------------------------------------------------- */

/* Writes the state of the context at its current time level to a file:
 * post-collision populations (storage precision as is), the top-plane ghost
 * velocity, the rigid-body and window state (ring offset, origin, slots,
 * step count, F, T, predictor history), h_imm on the support box and the
 * Lagrangian IBM force.  Waits for the stream.                              */
TURRET_API turret_status turret_save(turret_ctx *c, const char *path);
/* Restores a checkpoint into a context created with the same window,
 * storage, viscosity, density ratio, gravity and flags and loaded with the
 * same surface (TURRET_ESTATE otherwise); stepping then continues bit for
 * bit as from the saved context.  Waits.                                   */
TURRET_API turret_status turret_load(turret_ctx *c, const char *path);

/* Releases the context (not the caller's workspaces).                       */
TURRET_API turret_status lbm_destroy(turret_ctx *c);

/* Message of the last failure on this context (or of the last failed
 * lbm_init when c is NULL).                                                 */
TURRET_API const char *turret_last_error(const turret_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* TURRET_H */
