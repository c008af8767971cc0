/*
 * lbmfno — GB300 (sm_103a) hot path of the hybrid Fourier Neural Operator -
 * Lattice Boltzmann Method (arXiv 2604.27158).  Plain C ABI.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status (enum lbm_status).  Nothing throws.  On
 *    failure lbm_last_error() returns a message (thread-local, valid until the
 *    next failing call on the same thread).
 *  - Pointers with a `_d` suffix are device pointers (cudaMalloc / torch CUDA
 *    memory) owned by the caller; `_h` pointers are host memory owned by the
 *    caller.  The library owns only its opaque handles and small tables.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated otherwise.
 *  - Lattice: D2Q9, i = 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1)
 *    6:(-1,1) 7:(-1,-1) 8:(1,-1); weights 4/9, 1/9 (i=1..4), 1/36 (i=5..8);
 *    c_s^2 = 1/3; lattice units dx = dt = 1.
 *  - Canonical population layout ("canonical" below): for grid g with
 *    cells_before(g) = sum of nx*ny of the grids before it, population i of
 *    cell (x, y) sits at 9 * cells_before(g) + (i * ny + y) * nx + x.  Values
 *    are *shifted*: g_i = f_i - w_i (FP32), the quantity the kernels carry.
 *  - Dense field layout ("dense"): value of cell (x, y) of grid g at
 *    cells_before(g) + y * nx + x.
 *  - Packed mask: for grid g, words_before(g) = sum of ny * ceil(nx/32) of the
 *    grids before it; bit (x % 32) of word words_before(g) + y*ceil(nx/32) + x/32
 *    is 1 iff cell (x, y) is solid.
 */
#ifndef LBMFNO_H
#define LBMFNO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum lbm_status {
  LBM_OK = 0,
  LBM_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or configuration */
  LBM_ERR_CUDA = 2,        /* a CUDA runtime / driver call failed */
  LBM_ERR_UNSTABLE = 3,    /* NaN/Inf or |u| > u_max detected in a reduction */
  LBM_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired */
  LBM_ERR_UNSUPPORTED = 5  /* valid request this build does not implement */
};

/* x-end boundary kinds.  y is always periodic; walls are solid mask rows. */
enum lbm_bc {
  LBM_BC_PERIODIC = 0, /* both x ends periodic */
  LBM_BC_PRESSURE = 1, /* Zou-He, prescribed density (value = rho) */
  LBM_BC_VELOCITY = 2  /* Zou-He, prescribed normal velocity (value = u_x), u_y = 0 */
};

/* One lattice of a batch.  Sec. 2.1 (D2Q9 SRT); porous-media boundary set-up of
 * the appendix table (fixed inflow, periodic sides, fixed outlet pressure). */
typedef struct lbm_grid {
  int32_t nx, ny;     /* lattice size, nx >= 2, ny >= 2 */
  double tau;         /* BGK relaxation time, > 0.5 */
  double fx, fy;      /* constant body-force density (Guo forcing), lattice units */
  int32_t bc_west;    /* enum lbm_bc at x = 0 */
  int32_t bc_east;    /* enum lbm_bc at x = nx-1 (periodic iff bc_west periodic) */
  double west_value;  /* rho or u_x imposed at x = 0 */
  double east_value;  /* rho or u_x imposed at x = nx-1 */
} lbm_grid;

/* Sizes a caller allocates for a batch of grids (lbm_query_layout). */
typedef struct lbm_layout {
  size_t f_elems;    /* floats in EACH of the two population buffers */
  size_t mask_words; /* uint32 words of the packed mask */
  size_t cells;      /* total cells: length of a dense field */
  size_t ws_bytes;   /* device workspace bytes for lbm_init */
} lbm_layout;

/* Per-grid statistics returned by lbm_residual, LBM_NSTAT doubles per grid. */
#define LBM_NSTAT 8
enum lbm_stat_index {
  LBM_STAT_RESIDUAL = 0, /* ||u^n - u^prev||_2 / ||u^n||_2 over fluid cells */
  LBM_STAT_UNORM = 1,    /* ||u^n||_2 over fluid cells */
  LBM_STAT_DP = 2,       /* c_s^2 (mean rho at x=0 - mean rho at x=nx-1), fluid cells */
  LBM_STAT_MASS = 3,     /* sum of rho over fluid cells */
  LBM_STAT_MOMX = 4,     /* sum of rho u_x over fluid cells */
  LBM_STAT_MOMY = 5,     /* sum of rho u_y over fluid cells */
  LBM_STAT_BAD = 6,      /* cells with non-finite values or |u| > u_max */
  LBM_STAT_FLUID = 7     /* fluid cells */
};

typedef struct lbm_handle lbm_handle;

const char* lbm_last_error(void);

/* Layout of a batch of `ngrids` grids (host only, no GPU work). */
int lbm_query_layout(const lbm_grid* grids_h, int ngrids, lbm_layout* out_h);

/*
 * Create a solver for a batch of grids and set the rest state rho = 1, u = 0
 * (the default initialisation of Fig. 1).  mask_d: packed mask (read, must
 * stay valid and unchanged for the handle's life).  f_a_d, f_b_d: two
 * population buffers of layout.f_elems floats, 16-byte aligned, owned by the
 * caller, used as ping-pong state.  ws_d: layout.ws_bytes of workspace.
 * u_max: |u| above which reductions flag a cell as unstable.
 */
int lbm_init(const lbm_grid* grids_h, int ngrids, const uint32_t* mask_d, float* f_a_d,
             float* f_b_d, void* ws_d, double u_max, void* stream, lbm_handle** out);

/* Advance every grid by nsteps fused collide+stream steps (Sec. 2.1 loop:
 * equilibrium, SRT collision, streaming with halfway bounce-back, moments).
 * One kernel launch per step. */
int lbm_step(lbm_handle* h, int nsteps, void* stream);

/*
 * Persistent multi-step execution (the super-time-stepping loop of Sec. 2.3 advances
 * many trajectories of uneven size for k steps between FNO calls).  With on != 0,
 * lbm_step(h, nsteps > 1) runs all nsteps time steps of the batch in ONE cooperative
 * launch of the step kernel: its CTAs stay resident and meet at a grid-wide barrier
 * between steps instead of ending the grid; results are bitwise identical to one launch
 * per step.  Every barrier wait is bounded (2 s): an expired wait records
 * LBM_ERR_TIMEOUT (reported by the next lbm_residual) and every CTA returns.
 * Default off.  Host only.
 */
int lbm_set_persistent(lbm_handle* h, int on);

/*
 * Self-test of the multi-step launch's bounded grid barrier (the paper has no
 * counterpart).  Runs two persistent steps whose barrier waits for every CTA
 * (arrive_all != 0: completes, the state advances by two steps) or for one CTA more than
 * the launch has (arrive_all == 0: the wait expires after limit_ms, 0 < limit_ms <= 2000,
 * every CTA returns after the first step's stores, which go to the other buffer, so the
 * state is unchanged).  status_d: one caller-owned device word (overwritten).
 * Synchronises `stream`.  Returns LBM_ERR_TIMEOUT when the wait expired, LBM_OK when it
 * completed; the context stays usable either way.
 */
int lbm_barrier_selftest(lbm_handle* h, unsigned* status_d, int arrive_all, double limit_ms,
                         void* stream);

/* Macroscopic fields (Sec. 2.1 moments) of the current state, dense layout.
 * Solid cells report rho = 1, u = 0.  Any output pointer may be NULL. */
int lbm_macro(lbm_handle* h, float* rho_d, float* ux_d, float* uy_d, void* stream);

/*
 * Steady-state statistics of the current state (FP64 reductions on the GPU,
 * deterministic order): LBM_NSTAT doubles per grid into out_h.  The residual
 * compares u with the velocity stored by the previous lbm_residual call with
 * update_prev != 0 (or by lbm_init / lbm_reinit_from_macro); with
 * update_prev != 0 the current velocity is stored for the next call.
 * Synchronises `stream`.  Returns LBM_ERR_UNSTABLE if any grid has BAD > 0.
 */
int lbm_residual(lbm_handle* h, double* out_h, int update_prev, void* stream);

/*
 * lbm_residual of the current time level followed by one lbm_step, in one launch of
 * the step kernel (the statistics are taken from the populations the step pulls, so a
 * convergence check costs about one step instead of a step and a separate pass; the
 * steady driver of the hybrid framework, Sec. 2.3, checks this way).  out_h and
 * update_prev as for lbm_residual: the statistics are those of the level BEFORE the
 * step.  The step is taken (and counted) also when LBM_ERR_UNSTABLE is returned; not
 * on LBM_ERR_CUDA or LBM_ERR_TIMEOUT.  Synchronises `stream`.
 */
int lbm_step_residual(lbm_handle* h, double* out_h, int update_prev, void* stream);

/*
 * lbm_residual without caller-provided scratch memory (the paper has no
 * counterpart: this is a library convenience).  Same statistics, same output
 * layout and same update_prev behaviour as lbm_residual; the FP32 row-segment
 * partials, FP64 block sums and per-grid sums live in a 4 MiB array compiled into
 * the library instead of the lbm_init workspace, for callers that cannot allocate
 * device memory when they need the statistics (their device memory is owned by
 * another allocator, or their runtime forbids allocation after start-up).
 * Allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *  - Limit: batches whose statistics need more than 4 MiB of scratch (about 87,000
 *    row segments of 128 cells, roughly 11 million lattice cells; each grid rounds
 *    its segment count up to a multiple of 1024) are rejected with
 *    LBM_ERR_INVALID_ARG; use lbm_residual for them.
 *  - Every call looks up the array's device address for the current device
 *    (cudaGetSymbolAddress, which allocates nothing), so the address stays right
 *    after the device's context has been destroyed and created again.
 *  - Every GPU that loads the library holds the array until the process exits.
 *    All calls share it and it keeps the last call's contents (every slot a call
 *    reads is rewritten by that call first, so nothing needs clearing).  Calls
 *    whose kernels overlap on the GPU race on it.
 * Synchronises `stream`.
 */
int lbm_residual_static(lbm_handle* h, double* out_h, int update_prev, void* stream);

/*
 * Re-initialise the populations from macroscopic fields (hybrid framework,
 * Sec. 2.3): fluid cells get f^eq(rho, u) (Sec. 2.1) plus, if neq_mode != 0,
 * the first-order non-equilibrium estimate
 *   f_i^neq = -(tau w_i rho / c_s^2) Q_iab d_a u_b,  Q_iab = c_ia c_ib - c_s^2 d_ab,
 * with central differences (one-sided next to solid cells and open ends).
 * Inputs are dense fields.  The stored velocity used by lbm_residual is reset
 * to the given u.
 */
int lbm_reinit_from_macro(lbm_handle* h, const float* rho_d, const float* ux_d,
                          const float* uy_d, int neq_mode, void* stream);

/* Vorticity omega = d_x u_y - d_y u_x of dense velocity fields (the unsteady
 * accuracy metric, Sec. 3.2.2: normalised vorticity error), with the difference
 * stencils of lbm_reinit_from_macro (central; one-sided next to solid cells and open
 * ends; periodic wrap).  Dense layout; solid cells get 0. */
int lbm_vorticity(lbm_handle* h, const float* ux_d, const float* uy_d, float* omega_d,
                  void* stream);

/* Post-stream shifted populations g_i = f_i - w_i of the current time level
 * (after bounce-back and Zou-He completion), canonical layout, 9*cells floats.
 * Solid cells export 0. */
int lbm_export_f(lbm_handle* h, float* g_d, void* stream);

/* Overwrite / read the raw stored state: the shifted post-collision
 * populations of the previous time level, canonical layout.  Streaming them
 * (lbm_export_f) gives the current time level. */
int lbm_set_state(lbm_handle* h, const float* gstar_d, void* stream);
int lbm_get_state(lbm_handle* h, float* gstar_d, void* stream);

/* Streaming alone, through the step kernel's own gather (Sec. 2.1 streaming with
 * halfway bounce-back on solid cells, then the Zou-He completion of open end
 * columns): one launch of tile shape `variant` (0 .. LBM_STEP_VARIANTS-1) with the
 * BGK collision replaced by the identity, so the stored state becomes its streamed
 * populations (solid cells 0).  Not a time step of the method: it exists so that the
 * index map of the kernel that advances the lattice can be compared bit for bit with
 * a reference streaming (values are moved, never combined, except the Zou-He
 * unknowns).  The step counter is unchanged.  Asynchronous on `stream`. */
int lbm_stream_probe(lbm_handle* h, int variant, void* stream);

/*
 * Step-kernel tile shapes.  The fused step runs as a persistent kernel whose
 * tile shape (rows per tile, shared-memory stages, CTAs per SM) is one of
 * LBM_STEP_VARIANTS compiled shapes; all shapes give bitwise identical results.
 * lbm_autotune times every shape `reps` times on this batch (reading the
 * current state, writing only the scratch buffer: the state is unchanged),
 * selects the fastest, and optionally returns the per-shape milliseconds per
 * step (ms_h, LBM_STEP_VARIANTS entries, INFINITY for shapes that do not fit)
 * and the chosen index.  Synchronises `stream`.
 */
#define LBM_STEP_VARIANTS 6
int lbm_autotune(lbm_handle* h, int reps, float* ms_h, int* chosen_h, void* stream);
int lbm_set_step_variant(lbm_handle* h, int variant);
int lbm_get_step_variant(const lbm_handle* h, int* variant_h, int* rows_per_tile_h, int* stages_h,
                         int* ctas_per_sm_h);

/* Number of lbm_step time steps taken since lbm_init / the last reinit. */
int lbm_steps_done(const lbm_handle* h, long long* out_h);

int lbm_destroy(lbm_handle* h);

/* Self-test of failure detection (the paper has no counterpart).  The step kernel and
 * the tensor-core FNO kernels never wait without a limit: a device-side wait that does
 * not complete in time sets a status bit, the kernel returns, and the next call that
 * reads the status (lbm_residual, fno_check) reports LBM_ERR_TIMEOUT with the context
 * still usable.  This call runs the same kind of bounded mbarrier wait in a one-warp
 * kernel, on a barrier that nothing arrives on (arrive = 0) or on one that completes
 * (arrive != 0), with a limit of limit_ms (0 < limit_ms <= 2000).  status_d: one
 * caller-owned device word (overwritten).  Synchronises `stream`.  Returns
 * LBM_ERR_TIMEOUT when the wait expired, LBM_OK when it completed. */
int lbm_wait_selftest(unsigned* status_d, int arrive, double limit_ms, void* stream);

/* ----------------------------------------------------------------------
 * Adjoint (reverse mode) of the LBM part of the hybrid pipeline, for training
 * the FNO on a loss taken after LBM steps that follow its prediction (Sec. 2.3).
 * The paper trains its networks offline on data and differentiates nothing
 * through the LBM; these calls are this library's extension of its method.
 *
 * Let s_n be the stored state at time level n (what lbm_get_state returns),
 * P the pull (streaming with halfway bounce-back of Sec. 2.1, then the Zou-He
 * completion of the open end columns), C the BGK collision with the Guo source
 * and M the moments:  lbm_step: s_{n+1} = C(P(s_n));  lbm_macro: M(P(s_n)).
 * The adjoint variable mu_n (canonical layout, FP32) is the gradient of the loss
 * with respect to the populations of level n as the pull gathers them, before
 * the Zou-He completion: solid cells and the Zou-He unknowns of open end cells
 * (i = 1, 5, 8 at x = 0; 3, 6, 7 at x = nx-1) hold 0.  A loss on
 * (rho, u) of level N and initial fields (rho, u)_0 give:
 *   mu_N = lbm_adjoint_macro(s_N, dL/drho_N, dL/du_N);
 *   mu_{n-1} = lbm_adjoint_step(s_{n-1}, mu_n), n = N .. 1;
 *   dL/d(rho, u)_0 = lbm_adjoint_reinit(mu_0, (rho, u)_0).
 * States s_n come from lbm_get_state (checkpoints, recomputed in between with
 * lbm_set_state + lbm_step); none of these calls changes the handle's state.
 * All are asynchronous on `stream`, per-cell, deterministic (no atomics).
 * ------------------------------------------------------------------- */

/* mu_d (canonical) = adjoint seed of the moments of P(gstar_d): for fluid cells
 * mu_j = drho + (dux (c_jx - u_x) + duy (c_jy - u_y)) / rho, then the transpose
 * of the Zou-He completion.  gstar_d: canonical state s_N; drho_d, dux_d, duy_d:
 * dense gradients of the loss with respect to lbm_macro's outputs (their values
 * at solid cells are ignored). */
int lbm_adjoint_macro(lbm_handle* h, const float* gstar_d, const float* drho_d,
                      const float* dux_d, const float* duy_d, float* mu_d, void* stream);

/* mu_prev_d (canonical) = adjoint of one time step: the transpose of the pull's
 * gather applied to mu_d (slot (j, x) of s_n is read by cell x + c_j if that is a
 * fluid cell of the domain, by population opp(j) of x if it is solid),
 * times the transposed collision Jacobian at P(gstar_prev_d), then the transpose
 * of the Zou-He completion.  gstar_prev_d: canonical state s_{n-1}.  mu_d and
 * mu_prev_d must not alias. */
int lbm_adjoint_step(lbm_handle* h, const float* gstar_prev_d, const float* mu_d,
                     float* mu_prev_d, void* stream);

/* Gradients with respect to the fields given to lbm_reinit_from_macro: the
 * populations that the pull gathers after a reinit are f^eq(rho, u) + f^neq
 * (f^neq = -(tau w_i rho / c_s^2) Q_iab d_a u_b with the library's
 * central/one-sided differences), so dL/d(rho, u) is the transpose of that map
 * applied to mu_d = mu_0, including the transposed difference stencils when
 * neq_mode != 0.  rho_d, ux_d, uy_d: the dense fields the reinit was given.
 * scratch_d: 3 * cells floats.  Outputs drho_d, dux_d, duy_d: dense (0 at solid
 * cells).  The outputs must not alias the inputs. */
int lbm_adjoint_reinit(lbm_handle* h, const float* mu_d, const float* rho_d, const float* ux_d,
                       const float* uy_d, int neq_mode, float* scratch_d, float* drho_d,
                       float* dux_d, float* duy_d, void* stream);


/* ======================================================================
 * Fourier Neural Operator (Sec. 2.2, Fig. 2):
 *   theta_0 = P(phi);  theta_{n+1} = sigma(W theta_n + F^-1(R . F(theta_n))), n < N;
 *   out = Q(theta_N).
 * P: 1x1 network (c_in + 2 coordinate channels x/(W-1), y/(H-1)) -> C/2 -> sigma
 *    -> C.  F keeps ky in [0, m) U [H-m, H), kx in [0, m) (unnormalised forward
 *    DFT); R: per kept mode a complex C x C matrix (one [C, C, m, m] block per
 *    ky half); F^-1 is the real-input inverse (1/(H W), kx > 0 counted twice).
 *    W: 1x1 convolution with bias.  sigma: GELU (exact erf form) or ReLU.
 *    Q: dec_layers hidden 1x1 layers of dec_size with sigma, then a linear
 *    output layer.
 * Precision: parameters and inputs are bfloat16 values, activations are stored
 * as bfloat16 between layers, every sum accumulates in FP32.
 * Parameter pack (bfloat16 bits, this order, row-major shapes):
 *   lift0.w [C/2][c_in+2], lift0.b [C/2], lift1.w [C][C/2], lift1.b [C],
 *   per layer n: r1.re, r1.im, r2.re, r2.im [C_in][C_out][m][m], w [C][C], b [C],
 *   per decoder layer l: w [S][fan_in], b [S];  out.w [c_out][S], out.b [c_out].
 * ====================================================================== */
enum fno_activation { FNO_ACT_GELU = 0, FNO_ACT_RELU = 1 };

typedef struct fno_config {
  int32_t c_in;       /* physical input channels */
  int32_t c_out;      /* output channels */
  int32_t width;      /* latent channels C (even, <= 64) */
  int32_t layers;     /* Fourier layers N */
  int32_t modes;      /* kept modes m per corner block */
  int32_t dec_layers; /* hidden decoder layers (>= 1) */
  int32_t dec_size;   /* decoder width S (<= 64) */
  int32_t activation; /* enum fno_activation */
  int32_t padding;    /* zero padding of the latent field after lifting, at the high
                         end of both axes; cropped after the last Fourier layer
                         (appendix tables: "Padding: 9"); 0 <= padding <= 64 */
} fno_config;

typedef struct fno_sizes {
  size_t n_params;     /* parameters in the bfloat16 pack */
  size_t packed_bytes; /* device bytes of the repacked parameters (fno_create) */
  size_t ws_bytes;     /* device workspace bytes of fno_forward for (B, H, W) */
} fno_sizes;

typedef struct fno_handle fno_handle;

/* Sizes for a configuration and a forward shape B x H x W (host only).
 * Requires 2m <= H + padding and m < (W + padding)/2. */
int fno_query(const fno_config* cfg_h, int B, int H, int W, fno_sizes* out_h);

/* Repack the bfloat16 parameter pack params_d (n_params values, device) into
 * packed_d (packed_bytes, caller-owned, 256-byte aligned).  The handle keeps
 * pointers to packed_d only. */
int fno_create(const fno_config* cfg_h, const uint16_t* params_d, void* packed_d, void* stream,
               fno_handle** out);

/* Forward pass.  in_d: [B][c_in][H][W] FP32 (rounded to bfloat16 on entry);
 * out_d: [B][c_out][H][W] FP32; ws_d: ws_bytes from fno_query(B, H, W). */
int fno_forward(fno_handle* h, const float* in_d, float* out_d, int B, int H, int W, void* ws_d,
                size_t ws_bytes, void* stream);

/* Configuration the handle was created with. */
int fno_get_config(const fno_handle* h, fno_config* out_h);

/* Kernel path.  FNO_PATH_AUTO (default): tcgen05 tensor-core kernels where the
 * shape allows (C in {16, 32, 64}, m <= 16, H a multiple of 8, W a multiple of 128,
 * W <= 2048, no padding),
 * CUDA-core kernels otherwise.  FNO_PATH_CUDA_CORES: always the CUDA-core
 * kernels (same results up to rounding). */
enum fno_path { FNO_PATH_AUTO = 0, FNO_PATH_CUDA_CORES = 1 };
int fno_set_path(fno_handle* h, int path);
/* *out_h = 1 when fno_forward(B, H, W) runs the tensor-core kernels. */
int fno_uses_tensor_cores(const fno_handle* h, int H, int W, int* out_h);
/* Synchronise `stream` and report a device-side wait that expired during the
 * last fno_forward(B, H, W) on workspace ws_d (LBM_ERR_TIMEOUT), else LBM_OK. */
int fno_check(const fno_handle* h, const void* ws_d, int B, int H, int W, void* stream);
/* The activation between Fourier layers (Sec. 2.2; GELU or ReLU) exactly as the
 * inference kernels (tensor-core and CUDA-core paths) evaluate it, applied
 * element-wise: y_d[i] = act(x_d[i]) for i < n, on `stream` (asynchronous).  x_d, y_d:
 * caller-owned device FP32 arrays (may alias).  GELU is within 5e-6 (1 + |x|) of the exact x Phi(x).  For tests; returns
 * LBM_ERR_INVALID_ARG for an unknown act or a null buffer with n > 0. */
int fno_activation_eval(int act, const float* x_d, float* y_d, size_t n, void* stream);

int fno_destroy(fno_handle* h);

/* ----------------------------------------------------------------------
 * FNO training path: forward with saved activations and its exact reverse mode
 * (Sec. 2.2 network; the training objective itself is the caller's).  FP32 master
 * parameters in the packing order of the bfloat16 pack (n_params floats), FP32
 * activations, FP32 accumulation; no handle: every call takes the configuration
 * and the current parameters.  Spectral-layer adjoint, per layer:
 *   dz = dtheta' sigma'(z);  dW = sum_pixels dz theta^T;  db = sum_pixels dz;
 *   dY = (c_kx / (H W)) F(dz);  dR = sum_batch conj(X) dY;  dX = dY conj(R)^T;
 *   dtheta = W^T dz + Re sum_k dX e^{+i phi_k}
 * (F the truncated forward DFT, X = F(theta) saved by the forward pass).  Limits:
 * m <= 32, 2m <= H <= 8192, m <= W/2, W <= 2048.  Deterministic (fixed-order
 * reductions, no atomics).
 * ------------------------------------------------------------------- */
typedef struct fno_train_sizes {
  size_t n_params;    /* FP32 parameters (same order as the bfloat16 pack) */
  size_t saved_bytes; /* activations kept from forward to backward */
  size_t ws_bytes;    /* scratch of either call */
} fno_train_sizes;

int fno_train_query(const fno_config* cfg_h, int B, int H, int W, fno_train_sizes* out_h);

/* out_d [B][c_out][H][W] = FNO(in_d [B][c_in][H][W]); the input is used as given
 * (no bfloat16 rounding), the coordinate channels as in fno_forward.  saved_d:
 * saved_bytes, kept unchanged until the matching backward; ws_d: ws_bytes,
 * 256-byte aligned.  Parameters are read, not kept. */
int fno_train_forward(const fno_config* cfg_h, const float* params_d, const float* in_d,
                      float* out_d, int B, int H, int W, float* saved_d, void* ws_d,
                      void* stream);

/* Given dout_d = dL/dout, writes dparams_d (n_params, overwritten) = dL/dparams and,
 * if din_d is not NULL, din_d [B][c_in][H][W] = dL/din.  params_d and saved_d must
 * be those of the forward call. */
int fno_train_backward(const fno_config* cfg_h, const float* params_d, const float* dout_d,
                       const float* saved_d, float* dparams_d, float* din_d, int B, int H, int W,
                       void* ws_d, void* stream);

/* ======================================================================
 * Hybrid FNO-LBM framework (Sec. 2.3, Fig. 3)
 *   steady   (Fig. 3a): FNO prediction of (rho - 1, u) from the mask and the
 *            default fields -> clamp -> re-initialisation of f -> LBM until the
 *            residual of every grid is below tol (checked every check_every
 *            steps) or max_steps.  use_fno = 0 runs the plain rest-state start.
 *   unsteady (Fig. 3b): per cycle k_lbm LBM steps, then m_fno FNO steps on the
 *            macroscopic fields, then re-initialisation of f.
 * FNO input planes are chosen from (rho - 1, u_x, u_y, mask) per cell (a bit mask,
 * bit 0 = rho - 1, bit 1 = u_x, bit 2 = u_y, bit 3 = mask; 0 means all four, in that
 * order).  One network maps its planes to (rho - 1, u_x, u_y); or, as the paper's
 * model groups are built (appendix tables), a density network (one output, rho - 1)
 * and a velocity network (two outputs, u_x and u_y), both reading the fields of the
 * same time level.  Grids of equal size share one FNO call per network.
 * ====================================================================== */
enum hybrid_mode { HYBRID_STEADY = 0, HYBRID_UNSTEADY = 1 };

typedef struct hybrid_config {
  int32_t mode;        /* enum hybrid_mode */
  int32_t use_fno;     /* steady: 1 = FNO initialisation, 0 = rest state */
  int32_t neq_mode;    /* re-initialisation: 1 = f^eq + f^neq, 0 = f^eq */
  int32_t check_every; /* steady: residual interval (steps) */
  double tol;          /* steady: residual tolerance */
  int64_t max_steps;   /* steady: step cap */
  int32_t k_lbm;       /* unsteady: LBM steps per cycle */
  int32_t m_fno;       /* unsteady: FNO steps per cycle */
  double rho_lo, rho_hi; /* clamp of the predicted density before re-initialisation */
  double u_clamp;        /* clamp of the predicted speed */
  int32_t in_channels;   /* input planes of the (density) network, 0 = all four */
  int32_t in_channels_u; /* input planes of the velocity network, 0 = all four */
} hybrid_config;

typedef struct hybrid_stats {
  int64_t steps;       /* LBM steps taken by this call */
  int32_t converged;   /* steady: all grids below tol */
  int32_t fno_calls;   /* fno_forward calls made (per size group and network) */
  double max_residual; /* steady: largest final residual over grids */
} hybrid_stats;

typedef struct hybrid_handle hybrid_handle;

/* Device workspace bytes of a hybrid over the LBM batch `grids_h` with the network
 * `cfg_h` and, if cfg_u_h is not NULL, the velocity network cfg_u_h.  The grids are
 * predicted in size groups (one FNO call per network and group); every group and network
 * has its own FNO buffers, because an FNO step runs them as parallel branches on streams
 * the hybrid handle owns (forked from and joined back into the caller's stream). */
int hybrid_query_ws(const lbm_grid* grids_h, int ngrids, const fno_config* cfg_h,
                    const fno_config* cfg_u_h, size_t* ws_h);

/* Couple an LBM handle with one FNO (fno_u NULL: c_out = 3) or with a density network
 * `fno` (c_out = 1) and a velocity network `fno_u` (c_out = 2).  Each network's c_in
 * must equal the number of planes its in_channels selects.  All handles stay owned by
 * the caller. */
int hybrid_create(lbm_handle* lbm, fno_handle* fno, fno_handle* fno_u, const hybrid_config* cfg_h,
                  void* ws_d, size_t ws_bytes, hybrid_handle** out);

/*
 * Steady mode: cycles is ignored; runs to convergence or max_steps.
 * grid_steps_h (ngrids, may be NULL): step count at which each grid first met
 * tol (-1 if never); grid_residual_h (ngrids, may be NULL): final residuals.
 * Unsteady mode: runs `cycles` cycles, enqueued on `stream` without host
 * synchronisation (replayed from a CUDA graph after the first cycle).
 */
int hybrid_advance(hybrid_handle* h, int cycles, hybrid_stats* out_h, int64_t* grid_steps_h,
                   double* grid_residual_h, void* stream);

int hybrid_destroy(hybrid_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* LBMFNO_H */
