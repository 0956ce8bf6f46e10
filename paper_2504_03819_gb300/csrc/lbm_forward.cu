// Staged kernels of the free-energy D3Q27 LB model (Sec. II B, Sec. III C)
// over structure-of-arrays fields, plus initialisation, boundary marking,
// population import/export and the FP64 diagnostics:
//
//   wet_rho   solid-node density from the wetting scheme (Eqs. 37-38)
//   mu        mu = mu0(rho) - kappa lap rho on fluid nodes (Eqs. 2, 32)
//   wet_mu    solid-node chemical potential (Eq. 36)
//   uphi      F = (1/3 - rho) grad mu (Eq. 12), u = (j + F/2)/rho,
//             phi = (p_m - rho/3) u with p_m = (1 + mu)/3
//   q         Q_aa = -3 d_a phi_a (Eq. 27)
//
// The time step itself (collision and streaming) is the fused kernel chain
// of lbm_step_fused.cu; these kernels produce the stored fields that
// lbm_moments and the adjoint read.
//
// Stencils: lap g = 6 sum_i w_i (g(x+c_i) - g(x)), d_a g = 3 sum_i w_i c_ia
// (g(x+c_i) - g(x)) (the subtracted centre value does not change the sum
// because sum_i w_i c_ia = 0; it keeps FP32 cancellation small).
#include "lbm_lattice.cuh"

namespace lbm {

namespace {

constexpr int BLOCK = 256;

inline int blocks_for(long long n) { return (int)((n + BLOCK - 1) / BLOCK); }

// ---------------------------------------------------------------------------
// wetting boundary (Eqs. 36-38) on the listed solid nodes
// ---------------------------------------------------------------------------
// weighted mean of g over the fluid neighbours of solid node n; `solid` has
// bit q set when n + c_q is solid
__device__ __forceinline__ float fluid_average(const float *__restrict__ g, uint32_t solid, int n,
                                               const KParams &kp) {
  const Node p = decode(n, kp.nx, kp.ny);
  const int ox[3] = {p.x == 0 ? kp.nx - 1 : -1, 0, p.x == kp.nx - 1 ? -(kp.nx - 1) : 1};
  const int oy[3] = {p.y == 0 ? (kp.ny - 1) * kp.nx : -kp.nx, 0, p.y == kp.ny - 1 ? -(kp.ny - 1) * kp.nx : kp.nx};
  const int nxy = kp.nx * kp.ny;
  const int oz[3] = {p.z == 0 ? (kp.nz - 1) * nxy : -nxy, 0, p.z == kp.nz - 1 ? -(kp.nz - 1) * nxy : nxy};
  float num = 0.0f, den = 0.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (q == 13) continue;
    if (!((solid >> q) & 1u)) {
      num += weight_of(q) * g[n + ox[cx_of(q) + 1] + oy[cy_of(q) + 1] + oz[cz_of(q) + 1]];
      den += weight_of(q);
    }
  }
  return num / den;  // listed nodes have at least one fluid neighbour
}

__global__ void __launch_bounds__(BLOCK) k_wet_rho(const int *__restrict__ bnd, int nb,
                                                   const uint32_t *__restrict__ nbr, float *rho, KParams kp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb) return;
  int n = bnd[t];
  float ave = fluid_average(rho, nbr[n], n, kp);
  float rs = ave;
  if (kp.wet_mode != LBM_WET_NEUTRAL && ave >= kp.band_lo && ave <= kp.band_hi) {
    float m = kp.wet_mode == LBM_WET_PHI ? kp.wet_value * ave : ave - kp.wet_value;
    rs = fminf(fmaxf(m, kp.band_lo), kp.band_hi);
  }
  rho[n] = rs;
}

__global__ void __launch_bounds__(BLOCK) k_wet_mu(const int *__restrict__ bnd, int nb,
                                                  const uint32_t *__restrict__ nbr, float *mu, KParams kp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb) return;
  int n = bnd[t];
  mu[n] = fluid_average(mu, nbr[n], n, kp);
}

// ---------------------------------------------------------------------------
// chemical potential (Eqs. 2, 32)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BLOCK) k_mu(const float *__restrict__ rho, const uint8_t *__restrict__ mask,
                                              float *__restrict__ mu, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N || (mask && mask[n])) return;
  Node p = decode(n, kp.nx, kp.ny);
  float r = rho[n];
  float lap = 0.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (q == 13) continue;
    lap += weight_of(q) * (__ldg(rho + neighbour(p, cx_of(q), cy_of(q), cz_of(q), kp)) - r);
  }
  mu[n] = mu0_vdw(r, kp) - kp.kappa * (6.0f * lap);
}

// ---------------------------------------------------------------------------
// force, velocity and the flux of the third-order correction
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BLOCK) k_uphi(const float *__restrict__ rho, const float *__restrict__ j,
                                                const float *__restrict__ mu, const uint8_t *__restrict__ mask,
                                                float *__restrict__ u, float *__restrict__ F,
                                                float *__restrict__ phi, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  if (mask && mask[n]) {
    for (int a = 0; a < 3; ++a) u[a * N + n] = F[a * N + n] = phi[a * N + n] = 0.0f;
    return;
  }
  Node p = decode(n, kp.nx, kp.ny);
  float m = mu[n];
  float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (q == 13) continue;
    float d = weight_of(q) * (__ldg(mu + neighbour(p, cx_of(q), cy_of(q), cz_of(q), kp)) - m);
    if (cx_of(q)) gx += cx_of(q) * d;
    if (cy_of(q)) gy += cy_of(q) * d;
    if (cz_of(q)) gz += cz_of(q) * d;
  }
  float r = rho[n];
  float c = (1.0f / 3.0f - r) * 3.0f;
  float Fx = c * gx, Fy = c * gy, Fz = c * gz;
  float ux = (j[n] + 0.5f * Fx) / r, uy = (j[N + n] + 0.5f * Fy) / r, uz = (j[2 * N + n] + 0.5f * Fz) / r;
  float e = basis_c(r, m, kp);  // p_m - rho/3
  u[n] = ux;
  u[N + n] = uy;
  u[2 * N + n] = uz;
  F[n] = Fx;
  F[N + n] = Fy;
  F[2 * N + n] = Fz;
  phi[n] = e * ux;
  phi[N + n] = e * uy;
  phi[2 * N + n] = e * uz;
}

// ---------------------------------------------------------------------------
// third-order diagonal correction Q_aa = -3 d_a phi_a (Eq. 27)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BLOCK) k_q(const float *__restrict__ phi, const uint8_t *__restrict__ mask,
                                             float *__restrict__ Q, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  if (mask && mask[n]) {
    Q[n] = Q[N + n] = Q[2 * N + n] = 0.0f;
    return;
  }
  Node p = decode(n, kp.nx, kp.ny);
  float cx0 = phi[n], cy0 = phi[N + n], cz0 = phi[2 * N + n];
  float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (q == 13) continue;
    int m = neighbour(p, cx_of(q), cy_of(q), cz_of(q), kp);
    if (cx_of(q)) sx += cx_of(q) * weight_of(q) * (__ldg(phi + m) - cx0);
    if (cy_of(q)) sy += cy_of(q) * weight_of(q) * (__ldg(phi + N + m) - cy0);
    if (cz_of(q)) sz += cz_of(q) * weight_of(q) * (__ldg(phi + 2 * N + m) - cz0);
  }
  Q[n] = -9.0f * sx;
  Q[N + n] = -9.0f * sy;
  Q[2 * N + n] = -9.0f * sz;
}

// ---------------------------------------------------------------------------
// initialisation: equilibrium central moments (Eq. 20) about u0
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BLOCK) k_init_rho(const float *__restrict__ rho0, const uint8_t *__restrict__ mask,
                                                    float *__restrict__ rho, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  rho[n] = (mask && mask[n]) ? 0.0f : rho0[n];
}

template <typename T>
__global__ void __launch_bounds__(BLOCK) k_init_f(const float *__restrict__ rho, const float *__restrict__ mu,
                                                  const float *__restrict__ u0, const uint8_t *__restrict__ mask,
                                                  T *__restrict__ f, float *__restrict__ sb, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  if (mask && mask[n]) {
#pragma unroll
    for (int q = 0; q < 27; ++q) store_pop<T>(f + q * N + n, 0.0f);
    return;
  }
  const float cs2 = 1.0f / 3.0f;
  float pm = pm_of(mu[n], kp);
  float k[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) k[q] = 0.0f;
  KM(0, 0, 0) = rho[n];
  KM(2, 0, 0) = KM(0, 2, 0) = KM(0, 0, 2) = pm;
  KM(2, 2, 0) = KM(2, 0, 2) = KM(0, 2, 2) = pm * cs2;
  KM(2, 2, 2) = pm * cs2 * cs2;
  float ux = 0.0f, uy = 0.0f, uz = 0.0f;
  if (u0) {
    ux = u0[n];
    uy = u0[N + n];
    uz = u0[2 * N + n];
  }
  from_central(k, ux, uy, uz);
  const bool rest = kp.shift_mode == LBM_SHIFT_REST;
  const float rb = rho[n], cb = basis_c(rb, mu[n], kp);
#pragma unroll
  for (int q = 0; q < 27; ++q)
    store_pop<T>(f + q * N + n, k[q] - (rest ? shift_rest(q, rb, cb) : weight_of(q) * kp.rho_shift));
  if (rest) {
    sb[n] = rb;
    sb[N + n] = cb;
  }
}

// ---------------------------------------------------------------------------
// boundary list, population copies, FP64 reductions
// ---------------------------------------------------------------------------
// Boundary bookkeeping of a domain with walls, computed once: per node the
// solid-neighbour bitmask and, for solid nodes with fluid neighbours, the
// inverse fluid-weight sum of Eqs. 36-37 and a per-block count; then the
// list of those nodes in node order (a deterministic compaction).
__global__ void __launch_bounds__(BLOCK) k_mark_nbr(const uint8_t *__restrict__ mask, uint32_t *__restrict__ nbr,
                                                    float *__restrict__ inv_den, int *__restrict__ counts,
                                                    KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  bool boundary = false;
  if (n < kp.N) {
    const Node p = decode(n, kp.nx, kp.ny);
    uint32_t bits = 0;
    float den = 0.0f;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      if (q == 13) continue;
      if (mask[neighbour(p, cx_of(q), cy_of(q), cz_of(q), kp)])
        bits |= 1u << q;
      else
        den += weight_of(q);
    }
    nbr[n] = bits;
    boundary = mask[n] && den > 0.0f;
    inv_den[n] = boundary ? 1.0f / den : 0.0f;
  }
  const int c = __syncthreads_count(boundary);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// exclusive prefix sum of the per-block counts in place (one block of
// SCAN_T threads, each a contiguous chunk); the total goes to *total
constexpr int SCAN_T = 1024;
__global__ void __launch_bounds__(SCAN_T) k_scan_counts(int *__restrict__ counts, int nblocks, int *__restrict__ total) {
  __shared__ int part[SCAN_T];
  const int t = threadIdx.x;
  const int chunk = (nblocks + SCAN_T - 1) / SCAN_T;
  const int b0 = min(t * chunk, nblocks), b1 = min(b0 + chunk, nblocks);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += counts[b];
  part[t] = sum;
  __syncthreads();
  for (int w = 1; w < SCAN_T; w <<= 1) {  // inclusive scan of the chunk sums
    const int v = t >= w ? part[t - w] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - sum;
  for (int b = b0; b < b1; ++b) {
    const int c = counts[b];
    counts[b] = run;
    run += c;
  }
  if (t == SCAN_T - 1) *total = part[t];
}

// per-block counts of fluid nodes with a solid neighbour (second list)
__global__ void __launch_bounds__(BLOCK) k_count_fw(const uint8_t *__restrict__ mask, const uint32_t *__restrict__ nbr,
                                                    int *__restrict__ counts, KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const bool fw = n < kp.N && !mask[n] && nbr[n] != 0u;
  const int c = __syncthreads_count(fw);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// writes the nodes of a block that satisfy `in` at out[offsets[block] + rank]
__device__ __forceinline__ void compact_block(bool in, int n, const int *__restrict__ offsets, int *__restrict__ out) {
  __shared__ int warp_base[BLOCK / 32];
  const unsigned ball = __ballot_sync(0xffffffffu, in);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_base[w] = __popc(ball);
  __syncthreads();
  int base = offsets[blockIdx.x];
  for (int i = 0; i < w; ++i) base += warp_base[i];
  if (in) out[base + __popc(ball & ((1u << lane) - 1u))] = n;
}

__global__ void __launch_bounds__(BLOCK) k_write_fw(const uint8_t *__restrict__ mask, const uint32_t *__restrict__ nbr,
                                                    const int *__restrict__ offsets, int *__restrict__ list,
                                                    KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  compact_block(n < kp.N && !mask[n] && nbr[n] != 0u, n, offsets, list);
}

__global__ void __launch_bounds__(BLOCK) k_write_bnd(const float *__restrict__ inv_den, const int *__restrict__ offsets,
                                                     int *__restrict__ bnd, KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  compact_block(n < kp.N && inv_den[n] > 0.0f, n, offsets, bnd);
}


template <typename T>
__global__ void __launch_bounds__(BLOCK) k_get_pop(const T *__restrict__ f, const uint8_t *__restrict__ mask,
                                                   const float *__restrict__ sb, float *__restrict__ out,
                                                   KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  bool solid = mask && mask[n];
  const bool rest = kp.shift_mode == LBM_SHIFT_REST;
  float rb = kp.rho_shift, cb = 0.0f;
  if (rest && !solid) {
    rb = sb[n];
    cb = sb[N + n];
  }
#pragma unroll
  for (int q = 0; q < 27; ++q)
    out[q * N + n] = solid ? 0.0f
                           : load_pop<T>(f + q * N + n) + (rest ? shift_rest(q, rb, cb) : weight_of(q) * rb);
}

// In LBM_SHIFT_REST mode the basis of a set state is (sum_i f_i, 0).
template <typename T>
__global__ void __launch_bounds__(BLOCK) k_set_pop(const float *__restrict__ in, const uint8_t *__restrict__ mask,
                                                   T *__restrict__ f, float *__restrict__ sb, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  bool solid = mask && mask[n];
  const bool rest = kp.shift_mode == LBM_SHIFT_REST;
  float rb = kp.rho_shift;
  if (rest) {
    rb = 0.0f;
    if (!solid)
      for (int q = 0; q < 27; ++q) rb += in[q * N + n];
    sb[n] = rb;
    sb[N + n] = 0.0f;
  }
#pragma unroll
  for (int q = 0; q < 27; ++q) store_pop<T>(f + q * N + n, solid ? 0.0f : in[q * N + n] - weight_of(q) * rb);
}

// Mass sum rho and energy 1/2 sum rho |u|^2 over fluid nodes in FP64.  Each
// block walks a fixed node subset in a fixed order and reduces in a fixed
// tree; the final kernel sums the block partials in order.  Deterministic.
__global__ void __launch_bounds__(BLOCK) k_reduce_partial(const float *__restrict__ rho, const float *__restrict__ u,
                                                          const uint8_t *__restrict__ mask,
                                                          double *__restrict__ partial, KParams kp) {
  __shared__ double sm[2][BLOCK];
  const size_t N = (size_t)kp.N;
  double m = 0.0, e = 0.0;
  for (int n = blockIdx.x * BLOCK + threadIdx.x; n < kp.N; n += gridDim.x * BLOCK) {
    if (mask && mask[n]) continue;
    double r = rho[n], ux = u[n], uy = u[N + n], uz = u[2 * N + n];
    m += r;
    e += 0.5 * r * (ux * ux + uy * uy + uz * uz);
  }
  sm[0][threadIdx.x] = m;
  sm[1][threadIdx.x] = e;
  __syncthreads();
  for (int s = BLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sm[0][0];
    partial[2 * blockIdx.x + 1] = sm[1][0];
  }
}

__global__ void __launch_bounds__(RED_BLOCKS) k_reduce_final(const double *__restrict__ partial, double *out) {
  __shared__ double sm[2][RED_BLOCKS];
  sm[0][threadIdx.x] = partial[2 * threadIdx.x];
  sm[1][threadIdx.x] = partial[2 * threadIdx.x + 1];
  __syncthreads();
  for (int s = RED_BLOCKS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sm[0][0];
    out[1] = sm[1][0];
  }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
void fields_impl(lbm_ctx *ctx, bool with_u) {
  const KParams &kp = ctx->kp;
  const Fields &d = ctx->fld;
  const int g = blocks_for(kp.N);
  cudaStream_t s = ctx->stream;
  launch_moments_current(ctx);  // the step's own moments pass: the same bits
  if (ctx->n_bnd) { k_wet_rho<<<blocks_for(ctx->n_bnd), BLOCK, 0, s>>>(ctx->bnd, ctx->n_bnd, ctx->nbr, d.rho, kp); ctx->launches++; }
  k_mu<<<g, BLOCK, 0, s>>>(d.rho, ctx->mask, d.mu, kp);
  ctx->launches++;
  if (ctx->n_bnd) { k_wet_mu<<<blocks_for(ctx->n_bnd), BLOCK, 0, s>>>(ctx->bnd, ctx->n_bnd, ctx->nbr, d.mu, kp); ctx->launches++; }
  if (with_u) {
    k_uphi<<<g, BLOCK, 0, s>>>(d.rho, d.j, d.mu, ctx->mask, d.u, d.F, d.phi, kp);
    ctx->launches++;
  }
}

}  // namespace

void launch_mark_boundary(lbm_ctx *ctx) {
  const int g = blocks_for(ctx->N);
  k_mark_nbr<<<g, BLOCK, 0, ctx->stream>>>(ctx->mask, ctx->nbr, ctx->inv_den, ctx->scan, ctx->kp);
  k_scan_counts<<<1, SCAN_T, 0, ctx->stream>>>(ctx->scan, g, ctx->status + 1);
  k_write_bnd<<<g, BLOCK, 0, ctx->stream>>>(ctx->inv_den, ctx->scan, ctx->bnd, ctx->kp);
  ctx->launches += 3;
}

void launch_mark_fluid_wall(lbm_ctx *ctx) {
  const int g = blocks_for(ctx->N);
  k_count_fw<<<g, BLOCK, 0, ctx->stream>>>(ctx->mask, ctx->nbr, ctx->scan, ctx->kp);
  k_scan_counts<<<1, SCAN_T, 0, ctx->stream>>>(ctx->scan, g, ctx->status + 1);
  k_write_fw<<<g, BLOCK, 0, ctx->stream>>>(ctx->mask, ctx->nbr, ctx->scan, ctx->bnd + ctx->n_bnd, ctx->kp);
  ctx->launches += 3;
}

void launch_step(lbm_ctx *ctx) { launch_step_fused(ctx); }

void launch_fields_full(lbm_ctx *ctx) {
  launch_moments_mu(ctx);
  const Fields &d = ctx->fld;
  const int g = blocks_for(ctx->N);
  k_uphi<<<g, BLOCK, 0, ctx->stream>>>(d.rho, d.j, d.mu, ctx->mask, d.u, d.F, d.phi, ctx->kp);
  k_q<<<g, BLOCK, 0, ctx->stream>>>(d.phi, ctx->mask, d.Q, ctx->kp);
  ctx->launches += 2;
}

void launch_wet_rho(lbm_ctx *ctx) {
  TimedLaunch t(ctx, K_WET_RHO);
  k_wet_rho<<<blocks_for(ctx->n_bnd), BLOCK, 0, ctx->stream>>>(ctx->bnd, ctx->n_bnd, ctx->nbr, ctx->fld.rho, ctx->kp);
}

void launch_wet_mu(lbm_ctx *ctx) {
  TimedLaunch t(ctx, K_WET_MU);
  k_wet_mu<<<blocks_for(ctx->n_bnd), BLOCK, 0, ctx->stream>>>(ctx->bnd, ctx->n_bnd, ctx->nbr, ctx->fld.mu, ctx->kp);
}

void launch_fields(lbm_ctx *ctx, bool with_u) { fields_impl(ctx, with_u); }

void launch_init(lbm_ctx *ctx, const float *rho0, const float *u0) {
  const KParams &kp = ctx->kp;
  const Fields &d = ctx->fld;
  const int g = blocks_for(kp.N);
  cudaStream_t s = ctx->stream;
  k_init_rho<<<g, BLOCK, 0, s>>>(rho0, ctx->mask, d.rho, kp);
  ctx->launches++;
  if (ctx->n_bnd) { k_wet_rho<<<blocks_for(ctx->n_bnd), BLOCK, 0, s>>>(ctx->bnd, ctx->n_bnd, ctx->nbr, d.rho, kp); ctx->launches++; }
  k_mu<<<g, BLOCK, 0, s>>>(d.rho, ctx->mask, d.mu, kp);
  ctx->launches++;
  if (ctx->n_bnd) { k_wet_mu<<<blocks_for(ctx->n_bnd), BLOCK, 0, s>>>(ctx->bnd, ctx->n_bnd, ctx->nbr, d.mu, kp); ctx->launches++; }
  if (ctx->storage == LBM_F16)
    k_init_f<__half><<<g, BLOCK, 0, s>>>(d.rho, d.mu, u0, ctx->mask, (__half *)ctx->f[ctx->cur], d.sb, kp);
  else
    k_init_f<float><<<g, BLOCK, 0, s>>>(d.rho, d.mu, u0, ctx->mask, (float *)ctx->f[ctx->cur], d.sb, kp);
  ctx->launches++;
}

void launch_reduce(lbm_ctx *ctx, double *out) {
  k_reduce_partial<<<RED_BLOCKS, BLOCK, 0, ctx->stream>>>(ctx->fld.rho, ctx->fld.u, ctx->mask, ctx->red_partial, ctx->kp);
  k_reduce_final<<<1, RED_BLOCKS, 0, ctx->stream>>>(ctx->red_partial, out);
  ctx->launches += 2;
}

__global__ void __launch_bounds__(BLOCK) k_copy_mu(const float *__restrict__ mu, float *__restrict__ out, KParams kp) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < kp.N) out[n] = mu[n] + kp.mu_ref;
}

void launch_copy_mu(lbm_ctx *ctx, float *out) {
  k_copy_mu<<<blocks_for(ctx->N), BLOCK, 0, ctx->stream>>>(ctx->fld.mu, out, ctx->kp);
  ctx->launches++;
}

void launch_get_populations(lbm_ctx *ctx, float *out) {
  const int g = blocks_for(ctx->N);
  if (ctx->storage == LBM_F16)
    k_get_pop<__half><<<g, BLOCK, 0, ctx->stream>>>((const __half *)ctx->f[ctx->cur], ctx->mask, ctx->fld.sb, out, ctx->kp);
  else
    k_get_pop<float><<<g, BLOCK, 0, ctx->stream>>>((const float *)ctx->f[ctx->cur], ctx->mask, ctx->fld.sb, out, ctx->kp);
  ctx->launches++;
}

void launch_set_populations(lbm_ctx *ctx, const float *in) {
  const int g = blocks_for(ctx->N);
  if (ctx->storage == LBM_F16)
    k_set_pop<__half><<<g, BLOCK, 0, ctx->stream>>>(in, ctx->mask, (__half *)ctx->f[ctx->cur], ctx->fld.sb, ctx->kp);
  else
    k_set_pop<float><<<g, BLOCK, 0, ctx->stream>>>(in, ctx->mask, (float *)ctx->f[ctx->cur], ctx->fld.sb, ctx->kp);
  ctx->launches++;
}

const char *kernel_name(int id) {
  static const char *names[K_COUNT] = {"moments", "wet_rho", "mu", "wet_mu", "uphi", "q", "collide", "moments_edge"};
  return (id >= 0 && id < K_COUNT) ? names[id] : nullptr;
}

}  // namespace lbm
