/*
 * lbm.h -- C ABI of the GB300 free-energy D3Q27 lattice Boltzmann library.
 *
 * The library advances the chemical-potential-based free-energy LB model with
 * generalized (sixth-order Hermite) equilibria and central-moment collision of
 * Saito, Baba & Takada, "A thermodynamically consistent free-energy lattice
 * Boltzmann model" (arXiv 2504.03819), one time step per call of the hot path.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice units, delta_t = c = 1, c_s^2 = 1/3 (Sec. II B).
 *  - Grid of nx * ny * nz nodes, periodic in x, y and z.  Node index
 *    n = x + nx * (y + ny * z) (x fastest).  Walls are nodes of the solid mask.
 *  - Field arrays are structure-of-arrays: a scalar field is N = nx*ny*nz
 *    floats; a vector field is 3*N floats, component a at offset a*N.
 *  - Population q (0..26) has velocity c_q = (q%3 - 1, (q/3)%3 - 1, q/9 - 1);
 *    q = 13 is the rest population and 26 - q is the opposite of q.
 *    Population arrays are 27*N elements, population q at offset q*N.
 *  - Memory: the caller owns every buffer.  Device pointers are plain CUDA
 *    device addresses on the current device; host pointers are ordinary host
 *    memory.  The library allocates no device buffers: all of its device
 *    state lives in the caller's workspace, and the context keeps views of it
 *    (and of the solid mask) until lbm_destroy.  The CUDA graphs that
 *    lbm_step and lbm_adjoint_segment capture hold driver-managed resources,
 *    and one private stream is created to capture them; lbm_destroy releases
 *    both.
 *  - Streams: all device work of a context is enqueued on the stream given at
 *    lbm_init_domain (NULL = legacy default stream).  Entry points return after
 *    enqueueing unless documented otherwise.
 *  - Errors: every function returning int returns LBM_OK (0) or a negative
 *    LBM_ERR_* code and never aborts, throws or traps on the device.  Arguments
 *    are validated before any launch; lbm_last_error gives a message.
 *  - Arithmetic: FP32 on the device with IEEE division and logf (no fast
 *    math); FP64 only in the mass / energy reductions.
 *
 * Equation numbers follow the paper's numbered displays in order.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,        /* invalid argument (value, size, null pointer) */
  LBM_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  LBM_ERR_STATE = -3,      /* call out of order (no params / no state yet) */
  LBM_ERR_NONFINITE = -4,  /* a NaN/Inf density or momentum was detected */
  LBM_ERR_DOMAIN = -5,     /* a fluid density left (0, 1/b), the EOS domain */
  LBM_ERR_SIZE = -6,       /* workspace too small or grid too large */
  LBM_ERR_TIMEOUT = -7     /* a bounded wait inside a kernel gave up (an
                              asynchronous copy did not complete in 2 s) */
};

/* Population storage type.  Compute is always FP32. */
enum { LBM_F32 = 0, LBM_F16 = 1 };

/* How stored populations are shifted (see lbm_params.shift_mode). */
enum { LBM_SHIFT_CONST = 0, LBM_SHIFT_REST = 1 };

/* Wetting modes of the improved wetting boundary (Sec. III C, Eq. 38). */
enum { LBM_WET_NEUTRAL = 0, LBM_WET_PHI = 1, LBM_WET_DELTA = 2 };

typedef struct lbm_ctx lbm_ctx;

/*
 * Model parameters.
 *  a, b, R, T   van der Waals EOS p0 = rho R T/(1 - b rho) - a rho^2 (Eq. 29)
 *               and its chemical potential (Eq. 32); T is absolute.
 *               Requires a >= 0, b > 0, R > 0, T > 0.
 *  kappa        interfacial coefficient of mu = mu0 - kappa lap(rho) (Eq. 2),
 *               kappa >= 0.
 *  omega[11]    relaxation rates omega_0..omega_10 of Eqs. 21-26, each in
 *               [0, 2].
 *  nu           if > 0, omega_1 is set per node from 1/omega_1 =
 *               rho nu / p_m + 1/2 (Sec. II B) and omega[1] is ignored.
 *  q4_correction 1 applies the fourth-order correction of Eq. 28, 0 omits it.
 *  wetting_mode LBM_WET_NEUTRAL: rho_s = rho_ave;  LBM_WET_PHI: rho_s =
 *               phi * rho_ave;  LBM_WET_DELTA: rho_s = rho_ave - delta_rho,
 *               inside the contact-line band and limited to it (Eqs. 37-38).
 *  wetting_value phi (> 0) or delta_rho (>= 0); ignored when neutral.
 *  rho_l, rho_v liquid / vapour densities that define the contact-line band
 *               [0.05 rho_l + 0.95 rho_v, 0.95 rho_l + 0.05 rho_v]; needed
 *               (rho_l > rho_v > 0) only for the non-neutral modes.
 *  shift_mode   LBM_SHIFT_CONST: populations are stored as f_i - w_i rho_0
 *               with rho_0 = rho_shift.  LBM_SHIFT_REST: f_i(x) is stored
 *               minus the rest equilibrium of x at the previous step,
 *               w_i rho + (p_m - rho/3) E_i with E_i the isotropic operator of
 *               Eq. 16 at u = 0 (-19/9, 2/9, 1/18, 1/72 by speed class); the
 *               shift bases (rho, p_m - rho/3) are part of the raw state.
 *               Keeps FP16 storage accurate in dense liquid.
 *  rho_shift    rho_0 of LBM_SHIFT_CONST.
 *  check_interval  unused by the step (the non-finite / domain check runs in
 *               every step at no extra cost); kept for forward compatibility,
 *               must be >= 0.
 */
typedef struct {
  double a, b, R, T;
  double kappa;
  double omega[11];
  double nu;
  int q4_correction;
  int wetting_mode;
  double wetting_value;
  double rho_l, rho_v;
  double rho_shift;
  int shift_mode;
  int check_interval;
} lbm_params;

/* Device workspace (bytes) a domain of this size and storage type needs.
 * Pure host function.  Returns 0 for invalid sizes. */
size_t lbm_workspace_bytes(int nx, int ny, int nz, int storage);

/*
 * Create a context for an nx*ny*nz periodic domain (each >= 1, N < 2^31).
 *  storage       LBM_F32 or LBM_F16 (populations stored as f_i - w_i rho_0).
 *  solid_mask    device array of N bytes, nonzero = solid node, or NULL for
 *                an all-fluid domain.  Halfway bounce-back (Sec. III C) acts
 *                on fluid-solid links; solid nodes next to fluid get rho, mu
 *                from the wetting scheme (Eqs. 36-38).  Read at init (to list
 *                boundary nodes) and at every step; must stay valid and
 *                unchanged until lbm_destroy.
 *  workspace     device buffer of at least lbm_workspace_bytes(...) bytes,
 *                256-byte aligned; owned by the caller.
 *  cuda_stream   cudaStream_t to enqueue on (NULL = default stream).
 * Synchronises the stream once (to count boundary nodes).  *out is set only
 * on success.
 */
int lbm_init_domain(lbm_ctx **out, int nx, int ny, int nz, int storage,
                    const uint8_t *solid_mask, void *workspace, size_t ws_bytes,
                    void *cuda_stream);

/* Validate and store the model parameters (host struct, copied). */
int lbm_set_params(lbm_ctx *ctx, const lbm_params *params);

/*
 * Moving walls (Sec. III B drives its Galilean test with walls moving at a
 * constant velocity; the paper gives no boundary formula).  wall_u: device,
 * 3*N floats SoA (x, y, z planes), the velocity of each solid node (values on
 * fluid nodes are ignored), or NULL for walls at rest (the default).  A
 * population bounced back from a solid node moving with U gains the part of
 * the generalized equilibrium (Eq. 13) odd in the velocity, at U to first
 * order and at the rho and p_m of the fluid node: 2 w_i (c_i . U) / c_s^2 * A
 * with A = p_m / c_s^2 (edge and corner velocities) or p_m / c_s^2 +
 * (9/4)(rho - p_m / c_s^2) (face velocities).  The library keeps the pointer
 * (caller-owned: it must stay valid while steps and adjoint steps that use it
 * are enqueued).  Applies to lbm_step, lbm_adjoint_step and
 * lbm_adjoint_segment.  LBM_ERR_STATE for a domain without walls.
 */
int lbm_set_wall_velocity(lbm_ctx *ctx, const float *wall_u);

/*
 * Initial state: populations at the equilibrium whose central moments are
 * those of Eq. 20 about u0, with rho = rho0 and p_m = (1 + mu(rho0))/3
 * (mu from Eqs. 2, 32 and the wetting values of Eqs. 36-38 on solid nodes).
 *  rho0  device, N floats (values on solid nodes are ignored).
 *  u0    device, 3*N floats SoA, or NULL for u0 = 0.
 * Requires lbm_set_params.
 */
int lbm_set_state(lbm_ctx *ctx, const float *rho0, const float *u0);

/*
 * Advance n >= 0 time steps (Sec. II B): moments (Eq. 11), wetting density
 * (Eqs. 37-38), chemical potential (Eqs. 2, 32), wetting chemical potential
 * (Eq. 36), force (Eq. 12), corrections (Eqs. 27-28), central-moment
 * collision (Eqs. 19-26) and streaming (Eq. 10) with halfway bounce-back.
 * Enqueues only; a density that is non-finite or outside (0, 1/b) at the
 * start of any step sets a status flag read by lbm_sync_status.  Groups of
 * 16 steps run as one CUDA graph, captured on the context's own stream at
 * the first such call from each buffer (and again after lbm_set_params or
 * lbm_set_wall_velocity) and launched into the context's stream; results
 * are bitwise those of single steps.  Not while per-kernel profiling is on.
 */
int lbm_step(lbm_ctx *ctx, int n);

/*
 * Step variant (off by default): with on = 1 the fused collision kernel also
 * forms the moments of Eq. 11 (rho, j) and mu0(rho) of the state it writes,
 * so the next step needs no separate pass over the 27 populations.  Blocks
 * run in thread-block clusters spanning the x range and up to 16 blocks;
 * after each plane a cluster barrier lets every block sum its nodes of the
 * plane two behind (read back from L2), and a small pass completes the
 * first and last row of each cluster and the first and last plane of each
 * block's z range.  The moments are the bits of the separate pass, so the
 * trajectory is bitwise the same either way.  It applies to domains whose
 * population rows are whole multiples of 16 bytes (the tensor-copy path);
 * others keep the separate pass.  On GB300 it is slower than the default
 * (the 16-block clusters leave SMs of each GPC unused and the per-plane
 * cluster barrier holds the blocks in step), so it is kept for measurement.
 * on = 0 or 1, else LBM_ERR_ARG.
 */
int lbm_set_fused_moments(lbm_ctx *ctx, int on);

/* Synchronise the context's stream and return LBM_OK, LBM_ERR_NONFINITE,
 * LBM_ERR_DOMAIN or LBM_ERR_TIMEOUT from the device status word (the flags
 * stay set until lbm_set_state / lbm_set_raw_state / lbm_set_populations). */
int lbm_sync_status(lbm_ctx *ctx);

/*
 * Failure-path test hook (the paper has no counterpart).  In the next time
 * step enqueued, one block of the fused collision kernel makes its first
 * wait for a population tensor copy on a barrier that no thread arrives at,
 * bounded by 1 ms instead of 2 s, so the wait runs out: the block then
 * waits (with the full bound) for its own copy in flight, records
 * LBM_ERR_TIMEOUT in the status word and returns, as a real late copy would
 * make it do.  That step's populations are therefore incomplete.  One-shot;
 * acts only on domains whose population rows are whole multiples of 16 bytes
 * (nx a multiple of 4 with FP32 storage, of 8 with FP16), the ones staged by
 * tensor copies.  Nothing faults, traps or hangs: lbm_sync_status returns
 * LBM_ERR_TIMEOUT and lbm_set_state / lbm_set_raw_state clear it.
 */
int lbm_inject_wait_timeout(lbm_ctx *ctx);

/* Enqueue a copy of the device status word into host memory *dst (pinned
 * memory for an asynchronous copy) and return without waiting: after the
 * stream reaches it, *dst is 0 when no flag is set and nonzero otherwise
 * (lbm_sync_status then returns the error code).  Lets a caller read each
 * step's status while the next step runs.  LBM_ERR_ARG for a null pointer. */
int lbm_status_async(lbm_ctx *ctx, int *dst);

/*
 * Macroscopic fields of the current state (Eq. 11 and Eq. 2): rho (N floats,
 * wetting value on solid nodes next to fluid), u (3*N floats, force-corrected
 * velocity, 0 on solid nodes), mu (N floats) and mass_energy (2 doubles:
 * sum of fluid rho and 1/2 sum of fluid rho |u|^2, FP64 reductions with a
 * fixed summation order).  All pointers are device pointers and each may be
 * NULL.
 */
int lbm_moments(lbm_ctx *ctx, float *rho, float *u, float *mu, double *mass_energy);

/* Bytes of the raw state: 27*N elements of the storage type (shifted
 * populations, population q at offset q*N) followed, in LBM_SHIFT_REST mode,
 * by 2*N floats of shift bases.  Depends on the parameters (call after
 * lbm_set_params); 0 on error. */
size_t lbm_state_bytes(const lbm_ctx *ctx);

/* Raw state copy (lbm_state_bytes bytes), device to device.  Bitwise round
 * trip: lbm_set_raw_state of a saved state reproduces the same trajectory.
 * Population slots of solid nodes are never read. */
int lbm_get_state(lbm_ctx *ctx, void *f);
int lbm_set_raw_state(lbm_ctx *ctx, const void *f);

/* Unshifted FP32 populations f_i (27*N floats, device), zero on solid nodes;
 * and the inverse (stored shifted and rounded to the storage type). */
int lbm_get_populations(lbm_ctx *ctx, float *f);
int lbm_set_populations(lbm_ctx *ctx, const float *f);

/* Message for the last error on this context (never NULL). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Free the host-side context (no device memory is owned). */
void lbm_destroy(lbm_ctx *ctx);

/* ---- discrete adjoint ---------------------------------------------------
 *
 * The paper has no adjoint; these entry points give the exact reverse-mode
 * derivative of the discrete step above (the transpose of its linearisation
 * at the given state), so that gradients of a scalar objective J of the
 * state after T steps can be taken with respect to the parameters and the
 * initial density.  Adjoint fields lambda = dJ/df are unshifted FP32 arrays
 * of 27*N floats (population layout as above), zero on solid nodes.
 * Parameter gradients are LBM_NGRAD doubles in the order
 * [kappa, omega_0 .. omega_10, wetting_value], summed in FP64 in a fixed
 * order and ADDED to the caller's device array.  Derivatives through the
 * contact-line band test and limiter (Eq. 38) are those of the branch taken
 * at the given state (a clamped density passes no gradient).
 */
#define LBM_NGRAD 13

/* Objectives (of the current state), J[0] = value:
 *  LBM_OBJ_ENERGY          1/2 sum_fluid rho |u|^2 (u force-corrected, Eq. 11)
 *  LBM_OBJ_CENTROID_X      sum x (rho - rho_v) / sum (rho - rho_v), fluid nodes
 *                          (J[1] = the denominator)
 *  LBM_OBJ_CONTACT_RADIUS  sqrt(A/pi), A = sum over the fluid layer z = wall_z+1
 *                          of (rho - rho_v)/(rho_l - rho_v)
 */
enum { LBM_OBJ_ENERGY = 0, LBM_OBJ_CENTROID_X = 1, LBM_OBJ_CONTACT_RADIUS = 2 };

/* Value of objective `kind` of the current state into J (device, 2 doubles)
 * and its seed lambda = dJ/df into lam (device, 27*N floats, overwritten).
 * grad_params (device, LBM_NGRAD doubles, or NULL) receives the objective's
 * direct dependence on the parameters at fixed populations (the kinetic
 * energy depends on kappa and the wetting value through F), accumulated. */
int lbm_objective(lbm_ctx *ctx, int kind, int wall_z, double *J, float *lam, double *grad_params);

/*
 * One adjoint step.  state_t: raw state at time t (lbm_state_bytes bytes,
 * device, as from lbm_get_state); lam_next: dJ/df(t+1) (device, 27*N
 * floats); lam_t: output dJ/df(t) (device, 27*N floats, must not alias
 * lam_next); grad_params: device, LBM_NGRAD doubles, accumulated.  The
 * context's current state becomes state_t (the forward fields of f(t) are
 * recomputed from it).  Enqueues only.
 */
int lbm_adjoint_step(lbm_ctx *ctx, const void *state_t, const float *lam_next, float *lam_t,
                     double *grad_params);

/*
 * Adjoint of lbm_set_state: given lam0 = dJ/df(0) (device, 27*N floats),
 * writes dJ/drho0 into grad_rho0 (device, N floats, 0 on solid nodes) and
 * adds the parameter contributions of the initialisation (kappa, wetting
 * value) to grad_params.  rho0, u0 as passed to lbm_set_state (u0 may be
 * NULL).  The context's current state becomes the initial state of rho0, u0.
 */
int lbm_adjoint_init(lbm_ctx *ctx, const float *rho0, const float *u0, const float *lam0,
                     double *grad_params, float *grad_rho0);

/*
 * Bytes per step of the pool of lbm_adjoint_segment: one raw state
 * (lbm_state_bytes) plus the fields the recompute captures for the adjoint
 * (rho, mu, u, F, Q: 11*N floats), 256-byte aligned.  0 before
 * lbm_set_params.
 */
size_t lbm_adjoint_pool_bytes(const lbm_ctx *ctx);

/*
 * Adjoint sweep over one checkpoint segment of n >= 1 steps, enqueued from
 * the library (no per-step host round trip).  ckpt: raw state at t0
 * (device, lbm_state_bytes bytes); state_pool: device buffer of
 * n * lbm_adjoint_pool_bytes bytes that receives the recomputed states t0 ..
 * t0+n-1 and, for t0 .. t0+n-2, the fields the fused step computed from them
 * (the step writes into it directly, so the adjoint does not recompute
 * them); lam: device, 27*N floats, on entry dJ/df(t0+n), on return
 * dJ/df(t0); lam_tmp: device, 27*N floats of scratch; grad_params:
 * accumulated as in lbm_adjoint_step.  The context's current state becomes
 * ckpt.  Equivalent to n calls of lbm_adjoint_step on the recomputed states
 * (up to FP32 rounding of the fields).  The status word is cleared at the
 * start, as by lbm_set_raw_state, and keeps every flag the recompute raises,
 * so lbm_sync_status after the sweep reports a segment that left the EOS
 * domain.  The sweep between the checkpoint
 * copy-in and the restore runs as one CUDA graph, captured at the first call
 * with a given n, state_pool, lam, lam_tmp and grad_params (the two most
 * recent are kept; lbm_set_params and lbm_set_wall_velocity discard them);
 * results are bitwise those of the direct launches, which run instead while
 * per-kernel profiling is on.
 */
int lbm_adjoint_segment(lbm_ctx *ctx, const void *ckpt, int n, void *state_pool, float *lam, float *lam_tmp,
                        double *grad_params);

/* ---- instrumentation ---------------------------------------------------- */

/* Copy of the moments the next time step starts from, as stored (no
 * recomputation): rho (N floats, fluid nodes; solid boundary nodes hold the
 * last wetting value), j (3*N floats, sum f c, Eq. 11) and mu0 (N floats,
 * mu0(rho) - mu_ref of the bulk chemical potential, Eq. 32), device
 * pointers, each may be NULL.  A step whose fused kernel also produced the
 * moments of its output leaves them stored; LBM_ERR_STATE when no valid
 * moments are stored (after lbm_set_state, lbm_set_raw_state,
 * lbm_set_populations or lbm_set_params, until the next step, and after
 * steps that do not produce them).  For checking that path against a fresh
 * moments pass (lbm_moments). */
int lbm_stored_moments(lbm_ctx *ctx, float *rho, float *j, float *mu0);

/* Number of kernels this context has launched since init. */
long long lbm_launch_count(const lbm_ctx *ctx);

/* Enable (1) / disable (0) per-kernel CUDA-event timing of lbm_step launches
 * on the context's stream; enabling clears the accumulators. */
int lbm_profile_enable(lbm_ctx *ctx, int on);

/* Accumulated device time (ms) and launch count of kernel `id` (0-based, see
 * lbm_kernel_name) over the profiled lbm_step calls.  Synchronises the
 * stream.  Returns LBM_ERR_ARG for an unknown id. */
int lbm_profile_read(lbm_ctx *ctx, int id, double *total_ms, long long *launches);

/* Name of kernel `id` of the step, or NULL past the last one. */
const char *lbm_kernel_name(int id);

/* ---- a step without device allocation ----------------------------------- */

/* Largest domain (nx*ny*nz) lbm_step_noalloc accepts. */
#define LBM_NOALLOC_MAX_NODES 32768

/*
 * One time step for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a packaging of lbm_step for code that is not
 * allowed to call cudaMalloc or a caching allocator (for example a plugin or
 * solver kernel embedded in a host application that owns every device
 * allocation, or code running under a fixed memory budget), so it cannot
 * provide the workspace of lbm_init_domain.
 *
 * Runs the same kernels as lbm_step with LBM_F32 storage on unshifted
 * populations (params->shift_mode and rho_shift are ignored).  The step's
 * scratch (the macroscopic fields and the wall bookkeeping, about 2.9 MB) lives
 * in one static device array of the library, sized for
 * LBM_NOALLOC_MAX_NODES nodes; every GPU that loads the library holds it
 * until the process exits.
 *  f_in        device, 27*N floats: populations f_i at time t (layout as in
 *              the conventions above); read only.
 *  f_out       device, 27*N floats, must not alias f_in: populations at
 *              t + 1; solid-node slots are set to 0.
 *  solid_mask  device, N bytes, or NULL for an all-fluid domain.
 *  params      host; validated as by lbm_set_params.
 *  cuda_stream stream to enqueue on (NULL = default stream).
 * Returns LBM_ERR_SIZE if nx*ny*nz > LBM_NOALLOC_MAX_NODES, LBM_ERR_ARG for
 * invalid arguments (no message: there is no context), LBM_ERR_CUDA if a
 * CUDA call fails, and otherwise the step's status as lbm_sync_status
 * reports it: LBM_ERR_NONFINITE / LBM_ERR_DOMAIN when a fluid density or
 * momentum of f_in is non-finite or a density lies outside (0, 1/b) (f_out is
 * then meaningless), else LBM_OK.  To read that status it synchronises the
 * stream before returning, so the call is blocking (with a solid mask it
 * also synchronises once earlier, to count boundary nodes).  Calls no
 * cudaMalloc, cudaFree or allocating library routine.
 * The first call on each device looks up the device address of the static
 * array (cudaGetSymbolAddress, with that device current) and keeps it for
 * the process.  That address does not survive cudaDeviceReset or another
 * teardown of the device's primary context: after one, do not call this
 * entry point again in the same process.  Every call shares the one array,
 * so calls whose work overlaps on the GPU (different streams, threads or
 * processes sharing a context) race and give wrong results: serialise them.
 */
int lbm_step_noalloc(const float *f_in, float *f_out, const uint8_t *solid_mask, int nx, int ny, int nz,
                     const lbm_params *params, void *cuda_stream);

/* ---- host helpers ------------------------------------------------------- */

/*
 * Coexistence densities of the van der Waals EOS (Eq. 29) at temperature T
 * below T_c = 8a/(27 R b) (Eq. 30) from Maxwell's equal-area rule (Sec. III):
 * mu0(rho_l) = mu0(rho_v) and p0(rho_l) = p0(rho_v).  Pure host function.
 * Returns LBM_ERR_ARG if T >= T_c or a parameter is out of range.
 */
int lbm_maxwell(double a, double b, double R, double T, double *rho_l, double *rho_v);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
