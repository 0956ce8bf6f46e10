// C ABI of the library (include/lbm.h): argument validation, workspace
// layout, context state and the host-side Maxwell construction.  Every device
// operation is a kernel from lbm_forward.cu enqueued on the context stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// Workspace layout (each region 256-byte aligned):
//   f[0], f[1]      27 N elements of the storage type each
//   fields          rho N, j 3N, mu N, u 3N, F 3N, phi 3N, Q 3N, sb 2N, mu0 N floats,
//                   then the second moment set: rho N, j 3N, mu0 N floats
//   boundary list   N ints
//   neighbours      N uint32 solid-neighbour bitmasks, N floats of inverse
//                   fluid-weight sums, N/256 + 2 ints of compaction counts
//   reduction       RED_BLOCKS * 2 doubles
//   status          2 ints
//   adjoint         16 N floats, then 2 regions of adj_blocks() blocks x
//                   LBM_NGRAD doubles of gradient partials
struct Layout {
  size_t f0, f1, fields, bnd, nbr, inv_den, scan, red, status, adj, adj_partial, total;
};

bool layout(int nx, int ny, int nz, int storage, Layout *L) {
  if (nx < 1 || ny < 1 || nz < 1) return false;
  if (storage != LBM_F32 && storage != LBM_F16) return false;
  long long N = (long long)nx * ny * nz;
  if (N >= (1LL << 31)) return false;
  size_t elem = storage == LBM_F16 ? 2 : 4;
  size_t off = 0;
  L->f0 = off; off = align_up(off + 27 * (size_t)N * elem);
  L->f1 = off; off = align_up(off + 27 * (size_t)N * elem);
  L->fields = off; off = align_up(off + 25 * (size_t)N * sizeof(float));
  L->bnd = off; off = align_up(off + (size_t)N * sizeof(int));
  L->nbr = off; off = align_up(off + (size_t)N * sizeof(uint32_t));
  L->inv_den = off; off = align_up(off + (size_t)N * sizeof(float));
  L->scan = off; off = align_up(off + (size_t)(N / 256 + 2) * sizeof(int));
  L->red = off; off = align_up(off + (size_t)RED_BLOCKS * 2 * sizeof(double));
  L->status = off; off = align_up(off + 2 * sizeof(int));
  L->adj = off; off = align_up(off + 16 * (size_t)N * sizeof(float));
  L->adj_partial = off; off = align_up(off + 2 * adj_blocks(nx, ny, nz) * LBM_NGRAD * sizeof(double));
  L->total = off;
  return true;
}

int fail(lbm_ctx *ctx, int code, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int check_cuda(lbm_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return LBM_OK;
}

bool finite(double v) { return std::isfinite(v); }

int validate(lbm_ctx *ctx, const lbm_params *p) {
  if (!p) return fail(ctx, LBM_ERR_ARG, "params is NULL");
  if (!finite(p->a) || p->a < 0) return fail(ctx, LBM_ERR_ARG, "a must be finite and >= 0");
  if (!finite(p->b) || p->b <= 0) return fail(ctx, LBM_ERR_ARG, "b must be > 0");
  if (!finite(p->R) || p->R <= 0) return fail(ctx, LBM_ERR_ARG, "R must be > 0");
  if (!finite(p->T) || p->T <= 0) return fail(ctx, LBM_ERR_ARG, "T must be > 0");
  if (!finite(p->kappa) || p->kappa < 0) return fail(ctx, LBM_ERR_ARG, "kappa must be >= 0");
  for (int i = 0; i < 11; ++i)
    if (!finite(p->omega[i]) || p->omega[i] < 0 || p->omega[i] > 2)
      return fail(ctx, LBM_ERR_ARG, "omega[%d] must lie in [0, 2]", i);
  if (!finite(p->nu) || p->nu < 0) return fail(ctx, LBM_ERR_ARG, "nu must be >= 0");
  if (p->q4_correction != 0 && p->q4_correction != 1) return fail(ctx, LBM_ERR_ARG, "q4_correction must be 0 or 1");
  if (p->wetting_mode < LBM_WET_NEUTRAL || p->wetting_mode > LBM_WET_DELTA)
    return fail(ctx, LBM_ERR_ARG, "unknown wetting_mode %d", p->wetting_mode);
  if (p->wetting_mode != LBM_WET_NEUTRAL) {
    if (!finite(p->wetting_value) || (p->wetting_mode == LBM_WET_PHI ? p->wetting_value <= 0 : p->wetting_value < 0))
      return fail(ctx, LBM_ERR_ARG, "wetting_value out of range for the wetting mode");
    if (!finite(p->rho_l) || !finite(p->rho_v) || !(p->rho_l > p->rho_v && p->rho_v > 0))
      return fail(ctx, LBM_ERR_ARG, "wetting needs rho_l > rho_v > 0");
  }
  if (!finite(p->rho_shift)) return fail(ctx, LBM_ERR_ARG, "rho_shift must be finite");
  if (p->shift_mode != LBM_SHIFT_CONST && p->shift_mode != LBM_SHIFT_REST)
    return fail(ctx, LBM_ERR_ARG, "unknown shift_mode %d", p->shift_mode);
  if (p->check_interval < 0) return fail(ctx, LBM_ERR_ARG, "check_interval must be >= 0");
  return LBM_OK;
}

void harvest_profile(lbm_ctx *ctx) {
  for (auto &e : ctx->prof_pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e.start, e.stop) == cudaSuccess) {
      ctx->prof_ms[e.id] += ms;
      ctx->prof_n[e.id] += 1;
    }
    ctx->prof_free.push_back(e.start);
    ctx->prof_free.push_back(e.stop);
  }
  ctx->prof_pending.clear();
  cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_maxwell(double a, double b, double R, double T, double *rho_l, double *rho_v);

size_t lbm_workspace_bytes(int nx, int ny, int nz, int storage) {
  Layout L;
  return layout(nx, ny, nz, storage, &L) ? L.total : 0;
}

int lbm_init_domain(lbm_ctx **out, int nx, int ny, int nz, int storage, const uint8_t *solid_mask,
                    void *workspace, size_t ws_bytes, void *cuda_stream) {
  if (!out) return LBM_ERR_ARG;
  Layout L;
  if (nx < 1 || ny < 1 || nz < 1 || (storage != LBM_F32 && storage != LBM_F16)) return LBM_ERR_ARG;
  if (!layout(nx, ny, nz, storage, &L)) return LBM_ERR_SIZE;
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0) return LBM_ERR_ARG;
  if (ws_bytes < L.total) return LBM_ERR_SIZE;
  lbm_ctx *ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) return LBM_ERR_ARG;
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->nz = nz;
  ctx->N = nx * ny * nz;
  ctx->storage = storage;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->mask = solid_mask;
  char *base = (char *)workspace;
  ctx->f[0] = base + L.f0;
  ctx->f[1] = base + L.f1;
  ctx->cur = 0;
  float *fl = (float *)(base + L.fields);
  size_t N = ctx->N;
  ctx->fld.rho = fl;
  ctx->fld.j = fl + N;
  ctx->fld.mu = fl + 4 * N;
  ctx->fld.u = fl + 5 * N;
  ctx->fld.F = fl + 8 * N;
  ctx->fld.phi = fl + 11 * N;
  ctx->fld.Q = fl + 14 * N;
  ctx->fld.sb = fl + 17 * N;
  ctx->fld.mu0 = fl + 19 * N;
  ctx->mom[0] = lbm::Moments{fl, fl + N, fl + 19 * N};
  ctx->mom[1] = lbm::Moments{fl + 20 * N, fl + 21 * N, fl + 24 * N};
  view_moments(ctx);
  ctx->bnd = (int *)(base + L.bnd);
  ctx->nbr = (uint32_t *)(base + L.nbr);
  ctx->inv_den = (float *)(base + L.inv_den);
  ctx->scan = (int *)(base + L.scan);
  ctx->red_partial = (double *)(base + L.red);
  ctx->status = (int *)(base + L.status);
  float *ad = (float *)(base + L.adj);
  ctx->adj.u = ad;
  ctx->adj.F = ad + 3 * N;
  ctx->adj.Q = ad + 6 * N;
  ctx->adj.phi = ad + 9 * N;
  ctx->adj.pm = ad + 12 * N;
  ctx->adj.om1 = ad + 13 * N;
  ctx->adj.rho = ad + 14 * N;
  ctx->adj.mu = ad + 15 * N;
  ctx->adj_partial = (double *)(base + L.adj_partial);
  ctx->kp.nx = nx;
  ctx->kp.ny = ny;
  ctx->kp.nz = nz;
  ctx->kp.N = ctx->N;
  cudaGetLastError();
  cudaMemsetAsync(fl, 0, 25 * N * sizeof(float), ctx->stream);
  // solid-node population slots are never written by the step: start them at 0
  cudaMemsetAsync(ctx->f[0], 0, L.f1 - L.f0, ctx->stream);
  cudaMemsetAsync(ctx->f[1], 0, L.f1 - L.f0, ctx->stream);
  cudaMemsetAsync(ctx->status, 0, 2 * sizeof(int), ctx->stream);
  ctx->n_bnd = 0;
  ctx->n_fw = 0;
  if (solid_mask) {
    launch_mark_boundary(ctx);
    int cnt = 0;
    cudaMemcpyAsync(&cnt, ctx->status + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
      int rc = check_cuda(ctx, "boundary list");
      delete ctx;
      return rc == LBM_OK ? LBM_ERR_CUDA : rc;
    }
    ctx->n_bnd = cnt;
    if (cnt) {  // the adjoint's list of fluid nodes next to walls, after the solid one
      launch_mark_fluid_wall(ctx);
      cudaMemcpyAsync(&cnt, ctx->status + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
      if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        int rc = check_cuda(ctx, "fluid wall list");
        delete ctx;
        return rc == LBM_OK ? LBM_ERR_CUDA : rc;
      }
      ctx->n_fw = cnt;
    }
  }
  if (check_cuda(ctx, "lbm_init_domain") != LBM_OK) {
    delete ctx;
    return LBM_ERR_CUDA;
  }
  *out = ctx;
  return LBM_OK;
}

int lbm_set_params(lbm_ctx *ctx, const lbm_params *p) {
  if (!ctx) return LBM_ERR_ARG;
  int rc = validate(ctx, p);
  if (rc != LBM_OK) return rc;
  drop_step_graphs(ctx);  // the kernels take the parameters by value
  ctx->mom_valid = 0;     // the stored moments depend on the shift and the EOS
  ctx->params = *p;
  KParams &k = ctx->kp;
  k.RT = (float)(p->R * p->T);
  k.a = (float)p->a;
  k.b = (float)p->b;
  k.kappa = (float)p->kappa;
  for (int i = 0; i < 11; ++i) {
    k.om[i] = (float)p->omega[i];
    k.om_c[i] = 1.0f - k.om[i];
    k.om_h[i] = 1.0f - 0.5f * k.om[i];
  }
  k.g3 = 2.0f * k.om_h[3] * (1.0f / 3.0f);
  k.g5 = k.om_h[9] * (1.0f / 3.0f) * (1.0f / 3.0f);
  k.o10e = k.om[10] * (1.0f / 3.0f) * (1.0f / 3.0f);
  const float hs[8] = {k.om_c[0], k.om_h[0], k.om_c[5], k.om_c[8], k.om_c[9], k.g5, k.om_c[10], k.o10e};
  for (int i = 0; i < 8; ++i) k.hs[i] = hs[i] * (i < 2 ? 0.5f : 0.125f);
  k.nu = (float)p->nu;
  k.q4 = p->q4_correction;
  k.rho_shift = (float)p->rho_shift;
  k.shift_mode = p->shift_mode;
  k.wet_mode = p->wetting_mode;
  k.wet_value = (float)p->wetting_value;
  k.band_lo = (float)(0.05 * p->rho_l + 0.95 * p->rho_v);
  k.band_hi = (float)(0.95 * p->rho_l + 0.05 * p->rho_v);
  // references of the mu' = mu - mu_ref form: the coexistence densities below
  // T_c (where mu0(rho_l) = mu0(rho_v) = mu_ref), the critical density above
  double rl = 1.0 / (3.0 * p->b), rv = rl;
  if (!(p->a > 0 && p->T < 8.0 * p->a / (27.0 * p->R * p->b) &&
        lbm_maxwell(p->a, p->b, p->R, p->T, &rl, &rv) == LBM_OK)) {
    rl = rv = 1.0 / (3.0 * p->b);
  }
  const double RT = p->R * p->T;
  auto mu0 = [&](double r) {
    return RT * (std::log(r / (1 - p->b * r)) + 1 / (1 - p->b * r)) - 2 * p->a * r;
  };
  const double mu_ref = 0.5 * (mu0(rl) + mu0(rv));
  k.mu_ref = (float)mu_ref;
  k.pm_ref = (float)((1.0 + mu_ref) / 3.0);
  k.rho_split = (float)(0.5 * (rl + rv));
  const double refs[2] = {rv, rl};
  for (int i = 0; i < 2; ++i) {
    k.ref_rho[i] = (float)refs[i];
    k.ref_omb[i] = (float)(1.0 - p->b * (double)(float)refs[i]);
    k.ref_dmu[i] = (float)(mu0((double)(float)refs[i]) - mu_ref);
    k.ref_inv[i] = (float)(1.0 / (double)(float)refs[i]);
    k.ref_bomb[i] = (float)(p->b / (1.0 - p->b * (double)(float)refs[i]));
    k.ref_bomb2[i] = (float)(p->b / ((1.0 - p->b * (double)(float)refs[i]) * (1.0 - p->b * (double)(float)refs[i])));
  }
  ctx->have_params = 1;
  return LBM_OK;
}

int lbm_set_wall_velocity(lbm_ctx *ctx, const float *wall_u) {
  if (!ctx) return LBM_ERR_ARG;
  if (wall_u && !ctx->mask) return fail(ctx, LBM_ERR_STATE, "wall velocities need a domain with a solid mask");
  if (wall_u != ctx->wall_u) drop_step_graphs(ctx);
  ctx->wall_u = wall_u;
  return LBM_OK;
}

int lbm_set_state(lbm_ctx *ctx, const float *rho0, const float *u0) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->have_params) return fail(ctx, LBM_ERR_STATE, "lbm_set_params must come first");
  if (!rho0) return fail(ctx, LBM_ERR_ARG, "rho0 is NULL");
  cudaGetLastError();
  cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
  launch_init(ctx, rho0, u0);
  ctx->mom_valid = 0;
  int rc = check_cuda(ctx, "lbm_set_state");
  if (rc == LBM_OK) ctx->have_state = 1;
  return rc;
}

}  // extern "C"

namespace {

// Graph of GRAPH_STEPS steps from the current buffer, captured once on the
// context's private stream (the kernels and their arguments are recorded,
// not run); null when capture is not possible, so the caller launches
// directly.
cudaGraphExec_t step_graph(lbm_ctx *ctx) {
  const int parity = ctx->cur;
  if (ctx->step_graph[parity]) return ctx->step_graph[parity];
  if (!ctx->capture_stream && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->capture_stream = nullptr;
    return nullptr;
  }
  cudaStream_t user = ctx->stream;
  const long long l0 = ctx->launches;
  if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->stream = ctx->capture_stream;
  for (int i = 0; i < GRAPH_STEPS; ++i) launch_step(ctx);
  ctx->stream = user;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  const bool ok = cudaStreamEndCapture(ctx->capture_stream, &g) == cudaSuccess && g &&
                  cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  ctx->graph_launches = ctx->launches - l0;
  ctx->launches = l0;  // counted when the graph runs
  if (!ok) return nullptr;
  ctx->step_graph[parity] = exec;
  return exec;
}

}  // namespace

namespace lbm {
void drop_step_graphs(lbm_ctx *ctx) {
  for (cudaGraphExec_t &e : ctx->step_graph) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  for (SegmentGraph &g : ctx->seg_graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = SegmentGraph{};
  }
}
}  // namespace lbm

extern "C" {

int lbm_step(lbm_ctx *ctx, int n) {
  if (!ctx) return LBM_ERR_ARG;
  if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
  if (!ctx->have_state) return fail(ctx, LBM_ERR_STATE, "no state: call lbm_set_state first");
  cudaGetLastError();
  // whole groups of GRAPH_STEPS steps replay a captured graph (one launch
  // instead of three to five per step); per-kernel profiling needs the
  // individual launches
  // a captured group starts from valid moments when its steps produce them
  if (n >= GRAPH_STEPS && !ctx->prof_on && !ctx->kp.inject_wait && !ctx->mom_valid &&
      step_produces_moments(ctx))
    launch_moments_current(ctx);
  while (n >= GRAPH_STEPS && !ctx->prof_on && !ctx->kp.inject_wait) {
    cudaGraphExec_t g = step_graph(ctx);
    if (!g || cudaGraphLaunch(g, ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    ctx->launches += ctx->graph_launches;
    n -= GRAPH_STEPS;
  }
  for (int i = 0; i < n; ++i) launch_step(ctx);
  return check_cuda(ctx, "lbm_step");
}

int lbm_set_fused_moments(lbm_ctx *ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return LBM_ERR_ARG;
  if (on != ctx->fuse_mom) {
    drop_step_graphs(ctx);  // the captured steps take one path or the other
    ctx->fuse_mom = on;
    ctx->mom_valid = 0;
  }
  return LBM_OK;
}

int lbm_inject_wait_timeout(lbm_ctx *ctx) {
  if (!ctx) return LBM_ERR_ARG;
  ctx->kp.inject_wait = 1;
  return LBM_OK;
}

int lbm_sync_status(lbm_ctx *ctx) {
  if (!ctx) return LBM_ERR_ARG;
  int st = 0;
  cudaGetLastError();
  cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return check_cuda(ctx, "lbm_sync_status");
  if (st & STATUS_NONFINITE) return fail(ctx, LBM_ERR_NONFINITE, "non-finite density or momentum");
  if (st & STATUS_DOMAIN) return fail(ctx, LBM_ERR_DOMAIN, "density outside (0, 1/b)");
  if (st & STATUS_TIMEOUT) return fail(ctx, LBM_ERR_TIMEOUT, "a kernel's bounded wait for a tensor copy gave up");
  return LBM_OK;
}

int lbm_status_async(lbm_ctx *ctx, int *dst) {
  if (!ctx || !dst) return LBM_ERR_ARG;
  cudaGetLastError();
  cudaMemcpyAsync(dst, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  return check_cuda(ctx, "lbm_status_async");
}

int lbm_moments(lbm_ctx *ctx, float *rho, float *u, float *mu, double *mass_energy) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->have_state) return fail(ctx, LBM_ERR_STATE, "no state");
  cudaGetLastError();
  const bool need_u = u || mass_energy;
  launch_fields(ctx, need_u);
  size_t N = ctx->N;
  if (rho) cudaMemcpyAsync(rho, ctx->fld.rho, N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  if (mu) launch_copy_mu(ctx, mu);
  if (u) cudaMemcpyAsync(u, ctx->fld.u, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  if (mass_energy) launch_reduce(ctx, mass_energy);
  return check_cuda(ctx, "lbm_moments");
}

size_t lbm_state_bytes(const lbm_ctx *ctx) {
  if (!ctx || !ctx->have_params) return 0;
  size_t pops = 27 * (size_t)ctx->N * (ctx->storage == LBM_F16 ? 2 : 4);
  return pops + (ctx->kp.shift_mode == LBM_SHIFT_REST ? 2 * (size_t)ctx->N * sizeof(float) : 0);
}

int lbm_get_state(lbm_ctx *ctx, void *f) {
  if (!ctx || !f) return LBM_ERR_ARG;
  if (!ctx->have_state) return fail(ctx, LBM_ERR_STATE, "no state");
  size_t pops = 27 * (size_t)ctx->N * (ctx->storage == LBM_F16 ? 2 : 4);
  cudaGetLastError();
  cudaMemcpyAsync(f, ctx->f[ctx->cur], pops, cudaMemcpyDeviceToDevice, ctx->stream);
  if (ctx->kp.shift_mode == LBM_SHIFT_REST)
    cudaMemcpyAsync((char *)f + pops, ctx->fld.sb, 2 * (size_t)ctx->N * sizeof(float), cudaMemcpyDeviceToDevice,
                    ctx->stream);
  return check_cuda(ctx, "lbm_get_state");
}

int lbm_set_raw_state(lbm_ctx *ctx, const void *f) {
  if (!ctx || !f) return LBM_ERR_ARG;
  if (!ctx->have_params) return fail(ctx, LBM_ERR_STATE, "lbm_set_params must come first");
  size_t pops = 27 * (size_t)ctx->N * (ctx->storage == LBM_F16 ? 2 : 4);
  cudaGetLastError();
  cudaMemcpyAsync(ctx->f[ctx->cur], f, pops, cudaMemcpyDeviceToDevice, ctx->stream);
  if (ctx->kp.shift_mode == LBM_SHIFT_REST)
    cudaMemcpyAsync(ctx->fld.sb, (const char *)f + pops, 2 * (size_t)ctx->N * sizeof(float),
                    cudaMemcpyDeviceToDevice, ctx->stream);
  cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
  ctx->mom_valid = 0;
  int rc = check_cuda(ctx, "lbm_set_raw_state");
  if (rc == LBM_OK) ctx->have_state = 1;
  return rc;
}

int lbm_get_populations(lbm_ctx *ctx, float *f) {
  if (!ctx || !f) return LBM_ERR_ARG;
  if (!ctx->have_state) return fail(ctx, LBM_ERR_STATE, "no state");
  cudaGetLastError();
  launch_get_populations(ctx, f);
  return check_cuda(ctx, "lbm_get_populations");
}

int lbm_set_populations(lbm_ctx *ctx, const float *f) {
  if (!ctx || !f) return LBM_ERR_ARG;
  if (!ctx->have_params) return fail(ctx, LBM_ERR_STATE, "lbm_set_params must come first");
  cudaGetLastError();
  launch_set_populations(ctx, f);
  cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
  ctx->mom_valid = 0;
  int rc = check_cuda(ctx, "lbm_set_populations");
  if (rc == LBM_OK) ctx->have_state = 1;
  return rc;
}

int lbm_objective(lbm_ctx *ctx, int kind, int wall_z, double *J, float *lam, double *grad_params) {
  if (!ctx || !J || !lam) return LBM_ERR_ARG;
  if (!ctx->have_state) return fail(ctx, LBM_ERR_STATE, "no state");
  if (kind < LBM_OBJ_ENERGY || kind > LBM_OBJ_CONTACT_RADIUS) return fail(ctx, LBM_ERR_ARG, "unknown objective");
  if (kind == LBM_OBJ_CONTACT_RADIUS && (wall_z < 0 || wall_z + 1 >= ctx->nz))
    return fail(ctx, LBM_ERR_ARG, "wall_z + 1 must be a plane of the domain");
  if (kind != LBM_OBJ_ENERGY && !(ctx->params.rho_l > ctx->params.rho_v))
    return fail(ctx, LBM_ERR_ARG, "objective needs rho_l > rho_v in the parameters");
  cudaGetLastError();
  launch_objective(ctx, kind, wall_z, J, lam, grad_params);
  return check_cuda(ctx, "lbm_objective");
}

int lbm_adjoint_step(lbm_ctx *ctx, const void *state_t, const float *lam_next, float *lam_t, double *grad_params) {
  if (!ctx || !state_t || !lam_next || !lam_t || !grad_params || (const void *)lam_next == (const void *)lam_t)
    return LBM_ERR_ARG;
  int rc = lbm_set_raw_state(ctx, state_t);
  if (rc != LBM_OK) return rc;
  launch_adjoint_partials_zero(ctx);
  launch_adjoint_step(ctx, ctx->f[ctx->cur], lam_next, lam_t);
  launch_adjoint_partials_reduce(ctx, grad_params);
  return check_cuda(ctx, "lbm_adjoint_step");
}

size_t lbm_adjoint_pool_bytes(const lbm_ctx *ctx) {
  if (!ctx || !ctx->have_params) return 0;
  return align_up(align_up(lbm_state_bytes(ctx)) + 11 * (size_t)ctx->N * sizeof(float));
}

}  // extern "C"

namespace {

struct SegmentLayout {
  size_t pops, sbb, sbytes, stride, cap_off;
  bool rest;
};

SegmentLayout segment_layout(const lbm_ctx *ctx) {
  SegmentLayout L;
  L.pops = 27 * (size_t)ctx->N * (ctx->storage == LBM_F16 ? 2 : 4);
  L.rest = ctx->kp.shift_mode == LBM_SHIFT_REST;
  L.sbb = L.rest ? 2 * (size_t)ctx->N * sizeof(float) : 0;
  L.sbytes = L.pops + L.sbb;
  L.stride = lbm_adjoint_pool_bytes(ctx);
  L.cap_off = align_up(L.sbytes);
  return L;
}

// The sweep of one segment after its checkpoint is in pool slot 0 (and its
// shift bases in fld.sb): recompute of the states and their fields, the
// adjoint steps from the last state down to the first, the gradient
// reduction.  Enqueued on ctx->stream; leaves ctx->f / ctx->cur pointing
// into the pool (the caller restores them).
void enqueue_segment(lbm_ctx *ctx, int n, char *pool, float *lam, float *lam_tmp, double *grad) {
  const SegmentLayout L = segment_layout(ctx);
  auto slot = [&](int i) { return pool + (size_t)i * L.stride; };
  cudaStream_t s = ctx->stream;
  // with the rest shift the shift bases of state i live in slot i: step i
  // reads them from slot i-1 and writes them into slot i
  float *const own_sb = ctx->fld.sb;
  auto bases = [&](int i) { return (float *)(slot(i) + L.pops); };
  ctx->mom_valid = 0;  // slot 0 holds the checkpoint just copied in
  // recompute: step i reads slot i-1, writes slot i and captures the fields
  // of state i-1 into slot i-1
  for (int i = 1; i < n; ++i) {
    ctx->f[ctx->cur] = slot(i - 1);
    ctx->f[1 - ctx->cur] = slot(i);
    ctx->capture = (float *)(slot(i - 1) + L.cap_off);
    if (L.rest) {
      ctx->fld.sb = bases(i - 1);
      ctx->sb_out = bases(i);
    }
    launch_step(ctx);
    ctx->capture = nullptr;
    ctx->sb_out = nullptr;
  }
  // adjoint steps from t0+n-1 down to t0, lambda ping-pong; the last state
  // of the segment was not stepped, so its fields are recomputed
  float *lin = lam, *lout = lam_tmp;
  launch_adjoint_partials_zero(ctx);  // the segment's gradient partials accumulate over its steps
  for (int k = n - 1; k >= 0; --k) {
    ctx->f[ctx->cur] = slot(k);
    if (k == n - 1) {
      if (L.rest) ctx->fld.sb = bases(k);
      launch_adjoint_step(ctx, ctx->f[ctx->cur], lin, lout);
      ctx->fld.sb = own_sb;
    } else {
      launch_adjoint_step(ctx, ctx->f[ctx->cur], lin, lout, (const float *)(slot(k) + L.cap_off),
                          L.rest ? (const float *)(slot(k) + L.pops) : ctx->fld.sb);
    }
    float *t = lin;
    lin = lout;
    lout = t;
  }
  launch_adjoint_partials_reduce(ctx, grad);
  if (lin != lam) cudaMemcpyAsync(lam, lin, 27 * (size_t)ctx->N * sizeof(float), cudaMemcpyDeviceToDevice, s);
  ctx->mom_valid = 0;
}

// The segment sweep as a CUDA graph, captured once per (length, buffers) on
// the context's private stream; null when capture is not possible.
cudaGraphExec_t segment_graph(lbm_ctx *ctx, int n, char *pool, float *lam, float *lam_tmp, double *grad) {
  for (const SegmentGraph &g : ctx->seg_graphs)
    if (g.exec && g.n == n && g.pool == pool && g.lam == lam && g.lam_tmp == lam_tmp && g.grad == grad) {
      ctx->launches += g.launches;
      return g.exec;
    }
  if (!ctx->capture_stream && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->capture_stream = nullptr;
    return nullptr;
  }
  void *own0 = ctx->f[0], *own1 = ctx->f[1];
  const int own_cur = ctx->cur;
  cudaStream_t user = ctx->stream;
  const long long l0 = ctx->launches;
  if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->stream = ctx->capture_stream;
  enqueue_segment(ctx, n, pool, lam, lam_tmp, grad);
  ctx->stream = user;
  ctx->f[0] = own0;
  ctx->f[1] = own1;
  ctx->cur = own_cur;
  view_moments(ctx);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const bool ok = cudaStreamEndCapture(ctx->capture_stream, &graph) == cudaSuccess && graph &&
                  cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  const long long counted = ctx->launches - l0;
  if (!ok) {
    ctx->launches = l0;
    return nullptr;
  }
  SegmentGraph &g = ctx->seg_graphs[ctx->seg_next];
  ctx->seg_next = (ctx->seg_next + 1) % SEG_GRAPHS;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g = SegmentGraph{n, pool, lam, lam_tmp, grad, exec, counted};
  return exec;  // the capture's launch count stands for this first replay
}

}  // namespace

extern "C" {

int lbm_adjoint_segment(lbm_ctx *ctx, const void *ckpt, int n, void *state_pool, float *lam, float *lam_tmp,
                        double *grad_params) {
  if (!ctx || !ckpt || n < 1 || !state_pool || !lam || !lam_tmp || !grad_params || lam == lam_tmp)
    return LBM_ERR_ARG;
  if (!ctx->have_params) return fail(ctx, LBM_ERR_STATE, "lbm_set_params must come first");
  const SegmentLayout L = segment_layout(ctx);
  char *pool = (char *)state_pool;
  cudaStream_t s = ctx->stream;
  cudaGetLastError();
  cudaMemcpyAsync(pool, ckpt, L.sbytes, cudaMemcpyDeviceToDevice, s);  // state and shift bases into slot 0
  // the status word starts clear, as after lbm_set_raw_state, and keeps any
  // flag the recompute raises for lbm_sync_status after the sweep
  cudaMemsetAsync(ctx->status, 0, sizeof(int), s);
  void *own0 = ctx->f[0], *own1 = ctx->f[1];
  const int own_cur = ctx->cur;
  // one graph launch per segment (per-kernel profiling needs the launches)
  cudaGraphExec_t g = ctx->prof_on ? nullptr : segment_graph(ctx, n, pool, lam, lam_tmp, grad_params);
  if (!g || cudaGraphLaunch(g, s) != cudaSuccess) {
    cudaGetLastError();
    enqueue_segment(ctx, n, pool, lam, lam_tmp, grad_params);
  }
  // the context's own buffers hold ckpt afterwards
  ctx->f[0] = own0;
  ctx->f[1] = own1;
  ctx->cur = own_cur;
  view_moments(ctx);
  ctx->mom_valid = 0;
  cudaMemcpyAsync(ctx->f[ctx->cur], ckpt, L.pops, cudaMemcpyDeviceToDevice, s);
  if (L.rest) cudaMemcpyAsync(ctx->fld.sb, (const char *)ckpt + L.pops, L.sbb, cudaMemcpyDeviceToDevice, s);
  ctx->have_state = 1;
  return check_cuda(ctx, "lbm_adjoint_segment");
}

int lbm_adjoint_init(lbm_ctx *ctx, const float *rho0, const float *u0, const float *lam0, double *grad_params,
                     float *grad_rho0) {
  if (!ctx || !rho0 || !lam0 || !grad_params || !grad_rho0) return LBM_ERR_ARG;
  int rc = lbm_set_state(ctx, rho0, u0);  // fields of rho0 in the workspace
  if (rc != LBM_OK) return rc;
  launch_adjoint_init(ctx, u0, lam0, grad_params, grad_rho0);
  return check_cuda(ctx, "lbm_adjoint_init");
}

const char *lbm_last_error(const lbm_ctx *ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void lbm_destroy(lbm_ctx *ctx) {
  if (!ctx) return;
  if (!ctx->prof_pending.empty()) {
    cudaStreamSynchronize(ctx->stream);
    harvest_profile(ctx);
  }
  for (cudaEvent_t e : ctx->prof_free) cudaEventDestroy(e);
  drop_step_graphs(ctx);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  cudaGetLastError();
  delete ctx;
}

long long lbm_launch_count(const lbm_ctx *ctx) { return ctx ? ctx->launches : -1; }

int lbm_stored_moments(lbm_ctx *ctx, float *rho, float *j, float *mu0) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->have_state || !ctx->mom_valid) return fail(ctx, LBM_ERR_STATE, "no stored moments of the current state");
  const size_t N = ctx->N;
  const lbm::Moments &m = ctx->mom[ctx->cur];
  cudaGetLastError();
  if (rho) cudaMemcpyAsync(rho, m.rho, N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  if (j) cudaMemcpyAsync(j, m.j, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  if (mu0) cudaMemcpyAsync(mu0, m.mu0, N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  return check_cuda(ctx, "lbm_stored_moments");
}

int lbm_profile_enable(lbm_ctx *ctx, int on) {
  if (!ctx) return LBM_ERR_ARG;
  if (on) {
    if (!ctx->prof_pending.empty()) {
      cudaStreamSynchronize(ctx->stream);
      harvest_profile(ctx);
    }
    for (int i = 0; i < K_COUNT; ++i) {
      ctx->prof_ms[i] = 0.0;
      ctx->prof_n[i] = 0;
    }
  }
  ctx->prof_on = on ? 1 : 0;
  return LBM_OK;
}

int lbm_profile_read(lbm_ctx *ctx, int id, double *total_ms, long long *launches) {
  if (!ctx || id < 0 || id >= K_COUNT) return LBM_ERR_ARG;
  if (!ctx->prof_pending.empty()) {
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return check_cuda(ctx, "lbm_profile_read");
    harvest_profile(ctx);
  }
  if (total_ms) *total_ms = ctx->prof_ms[id];
  if (launches) *launches = ctx->prof_n[id];
  return LBM_OK;
}

const char *lbm_kernel_name(int id) { return kernel_name(id); }

}  // extern "C"

// Maxwell equal-area construction for the vdW EOS (Sec. III, Eqs. 29-32):
// find the coexistence pressure by bisection between the spinodal pressures;
// at each trial pressure the outer roots of p0(rho) = p are the two phases and
// mu0(rho_l) - mu0(rho_v) changes sign at coexistence.
namespace {
struct Eos {
  double a, b, RT;
  double p0(double r) const { return r * RT / (1 - b * r) - a * r * r; }
  double dp0(double r) const { return RT / ((1 - b * r) * (1 - b * r)) - 2 * a * r; }
  double mu0(double r) const { return RT * (std::log(r / (1 - b * r)) + 1 / (1 - b * r)) - 2 * a * r; }
};

template <typename Fn>
double bisect(Fn fn, double lo, double hi) {
  double flo = fn(lo);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double fm = fn(mid);
    if ((fm < 0) == (flo < 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
    if (hi - lo <= 1e-16 * std::fabs(mid)) break;
  }
  return 0.5 * (lo + hi);
}
}  // namespace

extern "C" int lbm_maxwell(double a, double b, double R, double T, double *rho_l, double *rho_v) {
  if (!rho_l || !rho_v || !(a > 0) || !(b > 0) || !(R > 0) || !(T > 0)) return LBM_ERR_ARG;
  const double Tc = 8 * a / (27 * R * b);
  if (!(T < Tc)) return LBM_ERR_ARG;
  Eos e{a, b, R * T};
  const double rc = 1 / (3 * b), rmax = (1 - 1e-13) / b;
  const double s_lo = bisect([&](double r) { return e.dp0(r); }, 1e-12, rc);
  const double s_hi = bisect([&](double r) { return -e.dp0(r); }, rc, rmax);
  double p_lo = e.p0(s_hi), p_hi = e.p0(s_lo);
  if (p_lo < 1e-300) p_lo = 1e-300;
  auto phases = [&](double p, double *rl, double *rv) {
    *rv = bisect([&](double r) { return e.p0(r) - p; }, 1e-300, s_lo);
    *rl = bisect([&](double r) { return e.p0(r) - p; }, s_hi, rmax);
  };
  double pc = bisect(
      [&](double p) {
        double rl, rv;
        phases(p, &rl, &rv);
        return e.mu0(rl) - e.mu0(rv);
      },
      p_lo, p_hi);
  phases(pc, rho_l, rho_v);
  return LBM_OK;
}
