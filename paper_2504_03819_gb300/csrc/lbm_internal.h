// Internal declarations shared by the C-ABI layer (lbm_api.cu) and the
// kernels (lbm_forward.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// Kernel-side model parameters, FP32 (the device arithmetic type).
struct KParams {
  int nx, ny, nz, N;
  float RT, a, b, kappa;
  float om[11];
  float om_c[11], om_h[11];  // 1 - omega_i and 1 - omega_i / 2 (collision factors)
  float g3, g5, o10e;        // 2 (1 - omega_3/2) / 3, (1 - omega_9/2) / 9, omega_10 / 9
  // the factors above that multiply a post-collision moment directly, scaled
  // for the halved moments of from_central_h (exact powers of two):
  // om_c[0]/2, om_h[0]/2, om_c[5]/8, om_c[8]/8, om_c[9]/8, g5/8, om_c[10]/8, o10e/8
  float hs[8];
  float nu;        // > 0: omega_1 per node from 1/omega_1 = rho nu / p_m + 1/2
  int q4;          // fourth-order correction on/off
  float rho_shift; // rho_0 of the stored populations f_i - w_i rho_0
  int shift_mode;  // LBM_SHIFT_CONST or LBM_SHIFT_REST
  int wet_mode;
  float wet_value, band_lo, band_hi;
  // Chemical potential is carried as mu' = mu - mu_ref.  mu0(rho) - mu_ref
  // is evaluated about the reference density of the node's phase (rho_l
  // above rho_split, rho_v below) so that FP32 does not cancel large terms.
  float mu_ref, pm_ref;             // pm_ref = (1 + mu_ref) / 3
  float rho_split;
  float ref_rho[2], ref_omb[2], ref_dmu[2];  // [0] vapour, [1] liquid: rho_r, 1 - b rho_r, mu0(rho_r) - mu_ref
  float ref_inv[2], ref_bomb[2];             // 1 / rho_r, b / (1 - b rho_r)
  float ref_bomb2[2];                        // b / (1 - b rho_r)^2
  int inject_wait;  // failure-path test: block 0's first bounded wait waits on a barrier nothing completes
};

// Device views carved out of the caller's workspace.
struct Fields {
  float *rho;  // N     density (fluid: sum f; solid: wetting value)
  float *j;    // 3N    sum f c
  float *mu;   // N     chemical potential minus mu_ref
  float *u;    // 3N    force-corrected velocity
  float *F;    // 3N    force (1/3 - rho) grad mu
  float *phi;  // 3N    (p_m - rho/3) u
  float *Q;    // 3N    Q_200, Q_020, Q_002
  float *sb;   // 2N    shift bases of LBM_SHIFT_REST: rho, then p_m - rho/3
  float *mu0;  // N     mu0(rho) - mu_ref of the fluid nodes, handed from the
               //       moments kernel to the chemical-potential kernel
};

// Moments of a population state: rho, j and mu0(rho) - mu_ref of the fluid
// nodes.  Two sets, one per population buffer (set k belongs to the state in
// f[k]); the fused step writes the moments of the state it produces into the
// other set, and Fields.rho / .j / .mu0 view the set of the current state.
struct Moments {
  float *rho, *j, *mu0;
};

// Adjoint scratch (reused between the stages of one adjoint step).
struct AdjFields {
  float *u, *F, *Q, *phi;  // 3N each
  float *pm, *om1, *rho, *mu;  // N each
};

enum KernelId {
  K_MOMENTS = 0,
  K_WET_RHO,
  K_MU,
  K_WET_MU,
  K_UPHI,
  K_Q,
  K_COLLIDE,
  K_MOM_EDGE,
  K_COUNT
};

// Tensor map of one population buffer for the TMA-staged step, cached by
// buffer address (the adjoint's segment sweep steps through pool buffers).
struct TmapEntry {
  const void *ptr;
  int ok;  // 1: map encoded; 0: this buffer cannot be described (fallback)
  CUtensorMap map;  // 64-byte aligned by its own declaration
};
constexpr int TMAP_CACHE = 4;

// A captured adjoint segment sweep and the buffers it was captured with.
struct SegmentGraph {
  int n;
  void *pool;
  float *lam, *lam_tmp;
  double *grad;
  cudaGraphExec_t exec;
  long long launches;
};
constexpr int SEG_GRAPHS = 2;

struct ProfEvent {
  int id;
  cudaEvent_t start, stop;
};

}  // namespace lbm

struct lbm_ctx {
  int nx, ny, nz, N, storage;
  cudaStream_t stream;
  const uint8_t *mask;  // device, may be null
  int n_bnd;
  int *bnd;             // solid nodes with at least one fluid neighbour, in node order; then, from
                        // bnd + n_bnd, the n_fw fluid nodes with a solid neighbour (adjoint only)
  int n_fw;
  uint32_t *nbr;        // per node: bit q set when node + c_q is solid (walls only)
  float *inv_den;       // per solid boundary node: 1 / sum of w_q over fluid neighbours, else 0
  int *scan;            // per-block counts of the boundary-list compaction
  void *f[2];
  int cur;
  float *capture;       // when set, the fused step writes rho, mu', u, F, Q of its input state here (11 N floats)
  float *sb_out;        // when set, the fused step writes the new shift bases here instead of over fld.sb
  const float *wall_u;  // caller's 3 N wall velocities (read at solid nodes), or null: walls at rest
  lbm::Fields fld;
  lbm::Moments mom[2];  // moments of the state in f[0] / f[1] (fld views mom[cur])
  int mom_valid;        // mom[cur] holds the moments of f[cur]
  int no_mom;           // the step never produces the next moments itself (lbm_step_noalloc)
  int fuse_mom;         // opt-in (lbm_set_fused_moments): the fused kernel produces the next moments
  int mom_cfg;          // cluster launch of the fused step: 0 not chosen yet, 1 chosen, -1 unavailable
  int mom_cx, mom_cy, mom_tz;  // its cluster shape (blocks) and planes per block
  double *red_partial;  // RED_BLOCKS * 2
  lbm::AdjFields adj;   // adjoint scratch
  double *adj_partial;  // per-block FP64 parameter-gradient partials
  int *status;          // [0] status bits, [1] counter scratch
  lbm_params params;
  lbm::KParams kp;
  int have_params, have_state;
  long long launches;
  int prof_on;
  std::vector<lbm::ProfEvent> prof_pending;
  std::vector<cudaEvent_t> prof_free;
  double prof_ms[lbm::K_COUNT];
  long long prof_n[lbm::K_COUNT];
  lbm::TmapEntry tmaps[lbm::TMAP_CACHE];
  int tmap_next;
  // CUDA graphs of lbm::GRAPH_STEPS steps, one per starting buffer, captured
  // on a private stream and launched into `stream`; rebuilt after any change
  // of the parameters or wall velocities the kernels take by value
  cudaStream_t capture_stream;
  cudaGraphExec_t step_graph[2];
  long long graph_launches;  // kernel launches one graph replays
  lbm::SegmentGraph seg_graphs[lbm::SEG_GRAPHS];
  int seg_next;
  std::string err;
};

namespace lbm {

constexpr int RED_BLOCKS = 1024;
constexpr int GRAPH_STEPS = 16;  // steps per captured graph (even: the buffers return to their start)

// Node-parallel adjoint kernels run on 3-D grids of 32 x ADJ_BY x 1 blocks
// (x fastest); the number of blocks sizes their per-block partial sums.
constexpr int ADJ_BY = 4;
inline size_t adj_blocks(int nx, int ny, int nz) {
  return (size_t)((nx + 31) / 32) * (size_t)((ny + ADJ_BY - 1) / ADJ_BY) * (size_t)nz;
}
constexpr int STATUS_NONFINITE = 1;
constexpr int STATUS_DOMAIN = 2;
constexpr int STATUS_TIMEOUT = 4;

// Launchers (lbm_forward.cu).  Each enqueues on ctx->stream and counts its
// launches; they do not check errors (the caller does).
void launch_mark_boundary(lbm_ctx *ctx);
void launch_mark_fluid_wall(lbm_ctx *ctx);  // after n_bnd is known; total into status[1]
void launch_step(lbm_ctx *ctx);                 // one full time step, swaps buffers
void launch_step_fused(lbm_ctx *ctx);           // the three-kernel step (lbm_step_fused.cu)
void launch_wet_rho(lbm_ctx *ctx);
void launch_wet_mu(lbm_ctx *ctx);
void launch_fields(lbm_ctx *ctx, bool with_u);  // moments .. (u, F, phi) of current state
void launch_init(lbm_ctx *ctx, const float *rho0, const float *u0);
void launch_reduce(lbm_ctx *ctx, double *out);
void launch_get_populations(lbm_ctx *ctx, float *out);
void launch_copy_mu(lbm_ctx *ctx, float *out);       // mu' + mu_ref
void launch_fields_full(lbm_ctx *ctx);               // rho, j, mu', u, F, phi, Q of the current state
void launch_moments_mu(lbm_ctx *ctx);                // rho, j, mu' (+ wetting) of the current state
// One adjoint step; its parameter-gradient partials are added to
// ctx->adj_partial (zeroed and reduced into the gradient by the two calls
// below, once per step or once per checkpoint segment).  captured: fields of
// f_state as written by the fused step (rho, mu', u, F, Q; 11 N floats) with
// sb_state its shift bases, or null to recompute them.
void launch_adjoint_step(lbm_ctx *ctx, const void *f_state, const float *lam_next, float *lam_t,
                         const float *captured = nullptr, const float *sb_state = nullptr);
void launch_adjoint_partials_zero(lbm_ctx *ctx);
void launch_adjoint_partials_reduce(lbm_ctx *ctx, double *grad);
void launch_adjoint_init(lbm_ctx *ctx, const float *u0, const float *lam0, double *grad, float *grad_rho0);
void launch_objective(lbm_ctx *ctx, int kind, int wall_z, double *J, float *lam, double *grad);
void launch_set_populations(lbm_ctx *ctx, const float *in);
void drop_step_graphs(lbm_ctx *ctx);  // after a change the captured step graphs would miss (lbm_api.cu)
void launch_moments_current(lbm_ctx *ctx);  // moments of f[cur] into mom[cur] (lbm_step_fused.cu)
bool step_produces_moments(lbm_ctx *ctx);    // a step from f[cur] writes the moments of its output

// Points the field views at the moment set of the current state.
inline void view_moments(lbm_ctx *ctx) {
  ctx->fld.rho = ctx->mom[ctx->cur].rho;
  ctx->fld.j = ctx->mom[ctx->cur].j;
  ctx->fld.mu0 = ctx->mom[ctx->cur].mu0;
}
const char *kernel_name(int id);

// Counts a kernel launch of the context and, when per-kernel profiling is on,
// brackets it with CUDA events on the context stream (events are recycled).
struct TimedLaunch {
  lbm_ctx *ctx;
  ProfEvent ev;
  TimedLaunch(lbm_ctx *c, int id) : ctx(c) {
    ev.id = id;
    if (ctx->prof_on) {
      ev.start = take();
      ev.stop = take();
      cudaEventRecord(ev.start, ctx->stream);
    }
    ctx->launches++;
  }
  ~TimedLaunch() {
    if (ctx->prof_on) {
      cudaEventRecord(ev.stop, ctx->stream);
      ctx->prof_pending.push_back(ev);
    }
  }
  cudaEvent_t take() {
    if (ctx->prof_free.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = ctx->prof_free.back();
    ctx->prof_free.pop_back();
    return e;
  }
};

}  // namespace lbm
