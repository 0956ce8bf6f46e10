// Fused time step (Sec. II B): three kernels per step instead of seven.
//
//   k_moments_v   rho, j from the populations (Eq. 11), mu0(rho) - mu_ref,
//                 status check
//   k_mu_z        mu' = mu0(rho) - mu_ref - kappa lap rho on fluid nodes
//                 (Eqs. 2, 32), marching in z with the rho planes in shared
//                 memory and the separable 27-point Laplacian
//   k_fused       per (x, y) column tile, marching in z: F = (1/3 - rho) grad
//                 mu, u = (j + F/2)/rho and phi = (p_m - rho/3) u on the tile
//                 plus a one-node ring (shared-memory planes), Q_aa = -3
//                 d_a phi_a (Eq. 27) on the tile, then the central-moment
//                 collision (Eqs. 19-26, 28) and push streaming with halfway
//                 bounce-back (Eq. 10, Sec. III C)
//
// The wetting kernels of lbm_forward.cu run between them when the domain has
// solid nodes.  Everything is FP32; shared-memory rings hold the planes a
// stencil needs so each field value is read from global memory about once.
#include "lbm_lattice.cuh"
#include "lbm_tma.cuh"

#include <atomic>
#include <mutex>

namespace lbm {

namespace {

// one-dimensional factor of the D3Q27 weights: w_q = w1(cx) w1(cy) w1(cz)
__device__ __forceinline__ constexpr float w1(int c) { return c == 0 ? 2.0f / 3.0f : 1.0f / 6.0f; }

// ---------------------------------------------------------------------------
// moments (Eq. 11)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_moments_v(const T *__restrict__ f, const uint8_t *__restrict__ mask,
                                                   const float *__restrict__ sb, float *__restrict__ rho,
                                                   float *__restrict__ j, float *__restrict__ mu0,
                                                   int *__restrict__ status, KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad_nf = false, bad_dom = false;
  if (n < kp.N && !(mask && mask[n])) {
    const size_t N = (size_t)kp.N;
    float v[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) v[q] = load_pop<T>(f + q * N + n);
    float s, sx, sy, sz;
    node_sums(v, s, sx, sy, sz);
    const float r = s + (kp.shift_mode == LBM_SHIFT_REST ? sb[n] : kp.rho_shift);
    rho[n] = r;
    j[n] = sx;
    j[N + n] = sy;
    j[2 * N + n] = sz;
    // the bulk chemical potential here, where the issue slots are idle (this
    // kernel waits on HBM), rather than in the issue-bound stencil kernel
    mu0[n] = mu0_vdw(r, kp);
    bad_nf = !(isfinite(r) && isfinite(sx) && isfinite(sy) && isfinite(sz));
    bad_dom = !bad_nf && !(r > 0.0f && kp.b * r < 1.0f);
  }
  const unsigned nf = __ballot_sync(0xffffffffu, bad_nf), dm = __ballot_sync(0xffffffffu, bad_dom);
  if ((threadIdx.x & 31) == 0) {
    if (nf) atomicOr(status, STATUS_NONFINITE);
    if (dm) atomicOr(status, STATUS_DOMAIN);
  }
}

// FP16 storage: two neighbouring nodes per thread through __half2 loads (N
// even, so every pair is 4-byte aligned); the same sums per node
__global__ void __launch_bounds__(256) k_moments_h2(const __half *__restrict__ f, const uint8_t *__restrict__ mask,
                                                    const float *__restrict__ sb, float *__restrict__ rho,
                                                    float *__restrict__ j, float *__restrict__ mu0,
                                                    int *__restrict__ status, KParams kp) {
  const int n0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  bool bad_nf = false, bad_dom = false;
  if (n0 < kp.N) {
    const size_t N = (size_t)kp.N;
    float v0[27], v1[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const float2 p = __half22float2(__ldg(reinterpret_cast<const __half2 *>(f + q * N + n0)));
      v0[q] = p.x;
      v1[q] = p.y;
    }
    auto finish = [&](const float (&v)[27], int n) {
      if (mask && mask[n]) return;
      float s, sx, sy, sz;
      node_sums(v, s, sx, sy, sz);
      const float r = s + (kp.shift_mode == LBM_SHIFT_REST ? sb[n] : kp.rho_shift);
      rho[n] = r;
      j[n] = sx;
      j[N + n] = sy;
      j[2 * N + n] = sz;
      mu0[n] = mu0_vdw(r, kp);
      const bool nf = !(isfinite(r) && isfinite(sx) && isfinite(sy) && isfinite(sz));
      bad_nf |= nf;
      bad_dom |= !nf && !(r > 0.0f && kp.b * r < 1.0f);
    };
    finish(v0, n0);
    finish(v1, n0 + 1);
  }
  const unsigned nf = __ballot_sync(0xffffffffu, bad_nf), dm = __ballot_sync(0xffffffffu, bad_dom);
  if ((threadIdx.x & 31) == 0) {
    if (nf) atomicOr(status, STATUS_NONFINITE);
    if (dm) atomicOr(status, STATUS_DOMAIN);
  }
}

// ---------------------------------------------------------------------------
// chemical potential, z-marching (Eqs. 2, 32)
// ---------------------------------------------------------------------------
constexpr int MX = 32, MY = 8;   // tile of k_mu_z
constexpr int MU_DEPTH = 4;      // rho planes in flight ahead of the stencil

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Each block marches a 32 x 8 column through z.  The rho planes (with a
// one-node periodic ring) stream into a shared-memory ring by asynchronous
// copies issued MU_DEPTH planes ahead, so several planes per block are in
// flight while the stencil works on planes z-1, z, z+1.
__global__ void __launch_bounds__(MX *MY) k_mu_z(const float *__restrict__ rho, const float *__restrict__ mu0,
                                                 const uint8_t *__restrict__ mask, float *__restrict__ mu,
                                                 KParams kp, int MZ) {
  constexpr int HX = MX + 2, HY = MY + 2, HP = HX * HY;
  constexpr int NR = MU_DEPTH + 3;  // planes z-1 .. z+1 being read, MU_DEPTH in flight, one being refilled
  __shared__ float s_r[NR][HP];
  __shared__ float s_m0[NR][MX * MY];  // mu0 of the tile, copied with its plane
  const int tx = threadIdx.x % MX, ty = threadIdx.x / MX;
  const int x0 = blockIdx.x * MX, y0 = blockIdx.y * MY, z0 = blockIdx.z * MZ;
  const int z1 = min(z0 + MZ, kp.nz);
  const int nxy = kp.nx * kp.ny;
  // xy offsets of this thread's halo-plane slots (periodic wrap), fixed over z
  constexpr int SLOTS = (HP + MX * MY - 1) / (MX * MY);
  int slot_xy[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int k = threadIdx.x + s * MX * MY;
    const int hx = k % HX, hy = k / HX;
    slot_xy[s] = k < HP ? pmod(x0 + hx - 1, kp.nx) + kp.nx * pmod(y0 + hy - 1, kp.ny) : 0;
  }
  auto ring = [&](int z) { return (z - z0 + 1 + NR) % NR; };  // z >= z0 - 1
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < kp.nx && y < kp.ny;
  const int nxy0 = x + kp.nx * y;
  // asynchronous copy of plane z into its ring slot, with mu0 of the tile
  // nodes of the planes the block updates (one commit group per plane,
  // empty past the end of the column)
  auto issue = [&](int z, int slot) {
    if (z <= z1) {
      // z in [z0 - 1, z1]: one period of wrap (no division) once nz >= 2
      const float *src = rho + (size_t)nxy * (kp.nz >= 2 ? wrap(z, kp.nz) : pmod(z, kp.nz));
      float *dst = s_r[slot];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int k = threadIdx.x + s * MX * MY;
        if (k < HP) cp_async4(dst + k, src + slot_xy[s]);
      }
      if (inside && z >= z0 && z < z1) cp_async4(&s_m0[slot][threadIdx.x], mu0 + (size_t)nxy * z + nxy0);
    }
    cp_async_commit();
  };
  // D(z') = sum_{cx,cy} w1 w1 (rho(x+cx, y+cy, z') - rho(x, y, z')) about
  // each plane's own centre: small numbers, accurate in FP32
  auto plane_sum = [&](int slot, float &centre) {
    const float *p = s_r[slot];
    const int c = (ty + 1) * HX + tx + 1;
    centre = p[c];
    const float row_m = w1(1) * (p[c - HX - 1] - centre) + w1(0) * (p[c - HX] - centre) + w1(1) * (p[c - HX + 1] - centre);
    const float row_0 = w1(1) * (p[c - 1] - centre) + w1(1) * (p[c + 1] - centre);
    const float row_p = w1(1) * (p[c + HX - 1] - centre) + w1(0) * (p[c + HX] - centre) + w1(1) * (p[c + HX + 1] - centre);
    return w1(1) * row_m + w1(0) * row_0 + w1(1) * row_p;
  };
  // prologue: planes z0-1 .. z0+MU_DEPTH in flight, the first three waited for
  for (int z = z0 - 1; z <= z0 + MU_DEPTH; ++z) issue(z, ring(z));
  cp_async_wait<MU_DEPTH - 1>();
  __syncthreads();
  float dm, cm, d0, c0, dp, cp;
  dm = plane_sum(ring(z0 - 1), cm);
  d0 = plane_sum(ring(z0), c0);
  int slot_in = ring(z0 + MU_DEPTH + 1), slot_next = ring(z0 + 1), slot_cur = ring(z0);  // rotate with z
  auto advance = [](int s) { return s + 1 == NR ? 0 : s + 1; };
  for (int z = z0; z < z1; ++z) {
    // plane z+1 has landed for every thread; the slot of plane z-2 is free
    cp_async_wait<MU_DEPTH - 1>();
    __syncthreads();
    issue(z + MU_DEPTH + 1, slot_in);
    dp = plane_sum(slot_next, cp);
    const float m0 = s_m0[slot_cur][threadIdx.x];
    slot_in = advance(slot_in);
    slot_next = advance(slot_next);
    slot_cur = advance(slot_cur);
    if (inside) {
      const int n = nxy0 + nxy * z;
      if (!(mask && mask[n])) {
        // lap = 6 sum_q w_q (rho(x + c_q) - rho(x)), split by planes
        const float lap = 6.0f * (w1(1) * (dm + (cm - c0)) + w1(0) * d0 + w1(1) * (dp + (cp - c0)));
        mu[n] = m0 - kp.kappa * lap;
      }
    }
    dm = d0;
    cm = c0;
    d0 = dp;
    c0 = cp;
  }
  cp_async_wait<0>();  // no copy outlives the block
}

// ---------------------------------------------------------------------------
// fused force / correction / collision / streaming
// ---------------------------------------------------------------------------
// column tile: one thread per (x, y); the launch bounds ask for FUSED_MINB
// blocks per SM (32 x 4 tiles measured fastest on GB300; four blocks fill
// the shared memory and cap the registers at 128, with no spills)
#ifndef LBM_FUSED_TX
#define LBM_FUSED_TX 32
#endif
#ifndef LBM_FUSED_TY
#define LBM_FUSED_TY 4
#endif
#ifndef LBM_FUSED_MINB
#define LBM_FUSED_MINB 4
#endif
constexpr int TX = LBM_FUSED_TX, TY = LBM_FUSED_TY;
constexpr int NT = TX * TY;
constexpr int H1X = TX + 2, H1Y = TY + 2, H1P = H1X * H1Y;  // one-node ring
constexpr int H2X = TX + 4, H2Y = TY + 4, H2P = H2X * H2Y;  // two-node ring
constexpr int S1 = (H1P + NT - 1) / NT;
constexpr int S2 = (H2P + NT - 1) / NT;

struct FusedSmem {
  float mu[4][H2P];       // mu' planes z-1 .. z+2 (two-node ring)
  float rho[4][H1P];      // rho planes z-2 .. z+1 (one-node ring)
  float j[3][3][H1P];     // j planes
  float gp[2][3][H1P];    // per ring position: the mu' partial sums of the gradient (two planes)
  float phi[3][H1P];      // (p_m - rho/3) u of the newest plane
  float qp[2][3][NT];     // per tile node: the phi partial sums of Q (planes z-1, z)
  float shift[3][4][H1P]; // storage shift by speed class, planes z-1 .. z+1
  float uF[2][6][NT];     // u, F of the tile for planes z, z+1
  uint8_t solid[4][H1P];  // mask planes
  alignas(8) uint64_t bar;  // completion barrier of the population tile copy
  uint64_t never;           // barrier no thread arrives at (failure-path test)
};
// the population tile of one plane, [q][y][x], staged by a tensor copy
// behind FusedSmem at a 128-byte boundary
constexpr size_t FBUF_OFFSET = (sizeof(FusedSmem) + 127) / 128 * 128;
template <typename T> constexpr size_t fused_smem_size(bool tma) {
  return tma ? FBUF_OFFSET + 27 * NT * sizeof(T) : sizeof(FusedSmem);
}

__device__ __forceinline__ int r4(int z) { return (z + 8) & 3; }
__device__ __forceinline__ int r3(int z) { return (z + 6) % 3; }
__device__ __forceinline__ int r2(int z) { return (z + 4) & 1; }

// Split barrier of a thread-block cluster: arrive (release at cluster scope)
// and wait (acquire at cluster scope), each executed by every thread of
// every block of the cluster, alternately.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait;" ::: "memory"); }

// population load through L2 only (values other blocks of the cluster wrote)
template <typename T> __device__ __forceinline__ float load_cg(const T *p);
template <> __device__ __forceinline__ float load_cg<float>(const float *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float load_cg<__half>(const __half *p) { return __half2float(__ldcg(p)); }

// Where the fused step writes the moments of the state it produces (rho,
// j, mu0 of the other moment set); rho == nullptr: it does not.
struct MomArgs {
  float *rho, *j, *mu0;
  int crows;  // rows of one cluster of blocks (cluster height x TY); >= ny: it spans y
  int zspan;  // one block's z range is the whole domain
};

// Base address of each population's plane of the output state (fout + q N):
// kernel parameters, so every push store is one constant-bank base plus the
// 32-bit node index of its destination.
template <typename T> struct PopPlanes {
  T *p[27];
};

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

// MASK: the domain has solid nodes (bounce-back and solid checks compiled
// in).  TMA: the populations of each plane arrive in shared memory by one
// tensor copy issued a plane ahead (tmap describes fin as [27][nz][ny][nx]);
// otherwise each thread loads its node's populations directly.  WALLV: the
// walls move (wall_u holds the solid nodes' velocities); compiled out of the
// resting-wall instantiations, whose registers it would raise.  UNIT: every
// rate but omega_1 is 1, so the collision reads only seven central moments
// (to_central_unit, collide_cm_unit).  REST: the populations are stored with
// the destination-keyed rest shift (otherwise with the constant one), fixed
// per launch so the shift choice costs no branches.  sb holds the shift bases of the input
// state, sb_out receives those of the output state; they may be one array
// (each node reads its own bases before it writes them).
template <typename T, bool MASK, bool TMA, bool WALLV, bool UNIT, bool REST>
__global__ void __launch_bounds__(NT, LBM_FUSED_MINB)
    k_fused(const T *__restrict__ fin, T *__restrict__ fout, const uint8_t *__restrict__ mask,
            const float *__restrict__ rho, const float *__restrict__ jv, const float *__restrict__ mu,
            const float *sb, float *sb_out, int *__restrict__ status, float *__restrict__ cap,
            const float *__restrict__ wall_u, MomArgs mo, const PopPlanes<T> op, KParams kp, int TZ,
            const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FusedSmem &S = *reinterpret_cast<FusedSmem *>(smem_raw);
  const T *fbuf = reinterpret_cast<const T *>(smem_raw + FBUF_OFFSET);
  constexpr uint32_t FBYTES = 27 * NT * sizeof(T);
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int z1 = min(z0 + TZ, kp.nz);
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const int nxy = nx * ny;
  const size_t N = (size_t)kp.N;
  constexpr bool rest = REST;

  // failure-path test: block 0 makes its first wait on a barrier that no
  // thread arrives at, so that bounded wait runs out
  const bool inject = TMA && kp.inject_wait && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  if (TMA) {
    // the first plane's copy is in flight while the field planes load
    if (tid == 0) {
      tma_prefetch_map(&tmap);
      mbar_init(&S.bar, 1);
      if (inject) mbar_init(&S.never, 1);
      mbar_fence_init();
      mbar_arrive_expect_tx(&S.bar, FBYTES);
      tma_load_4d(smem_raw + FBUF_OFFSET, &tmap, &S.bar, x0, y0, z0, 0);
    }
  }

  // xy offsets (periodic) of this thread's slots in the two-node and the
  // one-node rings; fixed for the whole column
  int xy2[S2], xy1[S1];
#pragma unroll
  for (int s = 0; s < S2; ++s) {
    const int k = tid + s * NT;
    xy2[s] = k < H2P ? pmod(x0 + k % H2X - 2, nx) + nx * pmod(y0 + k / H2X - 2, ny) : 0;
  }
#pragma unroll
  for (int s = 0; s < S1; ++s) {
    const int k = tid + s * NT;
    xy1[s] = k < H1P ? pmod(x0 + k % H1X - 1, nx) + nx * pmod(y0 + k / H1X - 1, ny) : 0;
  }
  // z runs over [z0 - 2, z1 + 1]: one period of wrap once nz >= 3 (no
  // division in the loop); thinner domains take the general modulus
  auto zoff = [&](int z) { return (size_t)nxy * (nz >= 3 ? wrap(z, nz) : pmod(z, nz)); };

  // planes are fetched into registers one iteration before they are stored
  // to shared memory, so their DRAM latency overlaps a whole plane of work
  float pmu[S2], prho[S1], pj[3][S1];
  uint8_t psolid[S1];
  auto fetch = [&](int zm, int zr) {  // mu' plane zm, rho/j/mask plane zr
    const size_t om = zoff(zm), orr = zoff(zr);
#pragma unroll
    for (int s = 0; s < S2; ++s) pmu[s] = (tid + s * NT < H2P) ? __ldg(mu + om + xy2[s]) : 0.0f;
#pragma unroll
    for (int s = 0; s < S1; ++s) {
      const bool ok = tid + s * NT < H1P;
      const size_t g = orr + xy1[s];
      prho[s] = ok ? __ldg(rho + g) : 0.0f;
      pj[0][s] = ok ? __ldg(jv + g) : 0.0f;
      pj[1][s] = ok ? __ldg(jv + N + g) : 0.0f;
      pj[2][s] = ok ? __ldg(jv + 2 * N + g) : 0.0f;
      if (MASK) psolid[s] = (ok && mask) ? mask[g] : (uint8_t)0;
    }
  };
  auto store = [&](int s4, int zr) {  // s4: ring slot of the mu' plane
    float *dm = S.mu[s4];
#pragma unroll
    for (int s = 0; s < S2; ++s)
      if (tid + s * NT < H2P) dm[tid + s * NT] = pmu[s];
    const int rg = r4(zr), jg = r3(zr);
#pragma unroll
    for (int s = 0; s < S1; ++s) {
      const int k = tid + s * NT;
      if (k < H1P) {
        S.rho[rg][k] = prho[s];
        S.j[jg][0][k] = pj[0][s];
        S.j[jg][1][k] = pj[1][s];
        S.j[jg][2][k] = pj[2][s];
        if (MASK) S.solid[rg][k] = psolid[s];
      }
    }
  };
  // F, u, phi at every one-node-ring position of plane z (u, F kept for the
  // tile positions)
  // this thread's one-node-ring positions k = tid, tid + NT: position in the
  // two-node ring and tile index (-1 off the tile), fixed for the column
  static_assert(S1 == 2, "two ring slots per thread");
  int fc[2], ft[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int k = tid + s * NT, hx = k % H1X, hy = k / H1X;
    fc[s] = (hy + 1) * H2X + hx + 1;
    ft[s] = (hx >= 1 && hx <= TX && hy >= 1 && hy <= TY) ? (hy - 1) * TX + hx - 1 : -1;
  }
  // The gradient of Eq. 12, sum_q w_q c_q mu'(x + c_q), factored like Q
  // (w_q = w1(cx) w1(cy) w1(cz)): with the in-plane partial sums of plane z'
  //   dx(z') = sum_cy w1(cy) [mu'(x+1, y+cy) - mu'(x-1, y+cy)],
  //   dy(z') likewise along y, pp(z') = sum_cx,cy w1(cx) w1(cy) mu',
  // its components are w1(1) sum_cz w1(cz) dx(z+cz), likewise for y, and
  // w1(1) (pp(z+1) - pp(z-1)).  Each thread forms the partial sums of its
  // own ring positions once per plane, when the plane arrives, and keeps two
  // older planes in its slots of gp.
  auto gpart = [&](const float *mp, int c, float &dx, float &dy, float &pp) {
    const float a = mp[c - H2X - 1], b = mp[c - H2X], e = mp[c - H2X + 1];
    const float d = mp[c - 1], m = mp[c], g = mp[c + 1];
    const float h = mp[c + H2X - 1], i = mp[c + H2X], l = mp[c + H2X + 1];
    dx = fmaf(w1(0), g - d, w1(1) * ((e - a) + (l - h)));
    dy = fmaf(w1(0), i - b, w1(1) * ((h - a) + (l - e)));
    pp = fmaf(w1(0), fmaf(w1(0), m, w1(1) * (d + g)),
              w1(1) * (fmaf(w1(0), b, w1(1) * (a + e)) + fmaf(w1(0), i, w1(1) * (h + l))));
  };
  auto gpart_store = [&](const float *mp, int zp) {
    for (int k = tid, s = 0; k < H1P; k += NT, ++s) {
      float dx, dy, pp;
      gpart(mp, s ? fc[1] : fc[0], dx, dy, pp);
      S.gp[zp & 1][0][k] = dx;
      S.gp[zp & 1][1][k] = dy;
      S.gp[zp & 1][2][k] = pp;
    }
  };
  // (a4, a4p: ring slots of mu' planes z and z+1; rp: slot of plane z in the
  // three-plane rings)
  auto fields = [&](int z, bool keep_uF, int a4, int a4p, int rp) {
    const int rg = r4(z), jg = r3(z);
    const float *m1 = S.mu[a4], *m2 = S.mu[a4p];
    float *gm = S.gp[(z - 1) & 1][0];  // plane z-1, then z+1
    const float *g0 = S.gp[z & 1][0];
#pragma unroll 1
    for (int k = tid, s = 0; k < H1P; k += NT, ++s) {
      const int fcs = s ? fc[1] : fc[0], fts = s ? ft[1] : ft[0];
      float phx = 0.0f, phy = 0.0f, phz = 0.0f, ux = 0.0f, uy = 0.0f, uz = 0.0f, Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
      float sh0 = 0.0f, sh1 = 0.0f, sh2 = 0.0f, sh3 = 0.0f;
      // partial sums of plane z+1 (every position: a solid one here may be
      // fluid in the next planes), those of z-1 replaced by them
      float dxn, dyn, ppn;
      gpart(m2, fcs, dxn, dyn, ppn);
      const float dxm = gm[k], dym = gm[H1P + k], ppm = gm[2 * H1P + k];
      gm[k] = dxn;
      gm[H1P + k] = dyn;
      gm[2 * H1P + k] = ppn;
      if (!MASK || !S.solid[rg][k]) {
        const float mc = m1[fcs];
        const float gx = w1(1) * fmaf(w1(0), g0[k], w1(1) * (dxm + dxn));
        const float gy = w1(1) * fmaf(w1(0), g0[H1P + k], w1(1) * (dym + dyn));
        const float gz = w1(1) * (ppn - ppm);
        const float r = S.rho[rg][k];
        const float cf = 3.0f * (1.0f / 3.0f - r);
        Fx = cf * gx;
        Fy = cf * gy;
        Fz = cf * gz;
        const float ir = 1.0f / r;
        ux = (S.j[jg][0][k] + 0.5f * Fx) * ir;
        uy = (S.j[jg][1][k] + 0.5f * Fy) * ir;
        uz = (S.j[jg][2][k] + 0.5f * Fz) * ir;
        const float e = basis_c(r, mc, kp);
        phx = e * ux;
        phy = e * uy;
        phz = e * uz;
        if (rest) {  // destination-keyed shifts of the four speed classes
          sh0 = shift_rest(13, r, e);
          sh1 = shift_rest(12, r, e);
          sh2 = shift_rest(9, r, e);
          sh3 = shift_rest(0, r, e);
        }
      }
      S.phi[0][k] = phx;
      S.phi[1][k] = phy;
      S.phi[2][k] = phz;
      if (rest) {
        S.shift[rp][0][k] = sh0;
        S.shift[rp][1][k] = sh1;
        S.shift[rp][2][k] = sh2;
        S.shift[rp][3][k] = sh3;
      }
      if (keep_uF && fts >= 0) {
        const int t = fts;
        float *o = S.uF[r2(z)][0];
        o[t] = ux;
        o[NT + t] = uy;
        o[2 * NT + t] = uz;
        o[3 * NT + t] = Fx;
        o[4 * NT + t] = Fy;
        o[5 * NT + t] = Fz;
      }
    }
  };

  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < nx && y < ny;
  // destination offsets in the node index for c = -1, 0, +1 per axis
  const int ox[3] = {x == 0 ? nx - 1 : -1, 0, x == nx - 1 ? -(nx - 1) : 1};
  const int oy[3] = {y == 0 ? (ny - 1) * nx : -nx, 0, y == ny - 1 ? -(ny - 1) * nx : nx};

  // prologue: mu' planes z0-2 .. z0+1 and rho/j planes z0-1 .. z0 in shared
  // memory, mu'(z0+2) and rho/j(z0+1) in registers; the gradient partial
  // sums of z0-2 .. z0+1, phi of z0-1 and z0, u/F of z0.  mu'(z0-2) takes the
  // slot of z0+2: its partial sums are formed before that plane is stored.
  fetch(z0 - 2, z0 - 1);
  store(r4(z0 - 2), z0 - 1);
  fetch(z0 - 1, z0);
  store(r4(z0 - 1), z0);
  fetch(z0, z0);
  store(r4(z0), z0);
  fetch(z0 + 1, z0);
  store(r4(z0 + 1), z0);
  __syncthreads();
  gpart_store(S.mu[r4(z0 - 2)], z0 - 2);
  gpart_store(S.mu[r4(z0 - 1)], z0 - 1);
  fetch(z0 + 2, z0 + 1);
  const int c1 = (ty + 1) * H1X + tx + 1;
  const int t = ty * TX + tx;
  // Q_aa = -3 d_a phi_a = -9 sum_q w_q c_qa phi_a(x + c_q) (Eq. 27).  The
  // weights factor, w_q = w1(cx) w1(cy) w1(cz), so with the in-plane partial
  // sums of plane z'
  //   ex(z') = sum_cy w1(cy) [phi_x(x+1, y+cy) - phi_x(x-1, y+cy)],
  //   ey(z') likewise along y, pz(z') = sum_cx,cy w1(cx) w1(cy) phi_z,
  // Q_x = -9/6 sum_cz w1(cz) ex(z+cz), Q_y likewise, Q_z = -9/6 (pz(z+1) -
  // pz(z-1)).  Each thread forms the partial sums of its own node once per
  // plane, right after the plane's phi, and keeps the two older planes in
  // its slots of qp.
  auto qpartials = [&](int zp, float &ex_out, float &ey_out, float &pz_out) {
    const float *px = S.phi[0], *py = S.phi[1], *pz = S.phi[2];
    const float ex = fmaf(w1(0), px[c1 + 1] - px[c1 - 1],
                          w1(1) * ((px[c1 + 1 - H1X] - px[c1 - 1 - H1X]) + (px[c1 + 1 + H1X] - px[c1 - 1 + H1X])));
    const float ey = fmaf(w1(0), py[c1 + H1X] - py[c1 - H1X],
                          w1(1) * ((py[c1 + H1X - 1] - py[c1 - H1X - 1]) + (py[c1 + H1X + 1] - py[c1 - H1X + 1])));
    float row[3];
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy) {
      const int o = c1 + cy * H1X;
      row[cy + 1] = fmaf(w1(0), pz[o], w1(1) * (pz[o - 1] + pz[o + 1]));
    }
    const float pzs = fmaf(w1(0), row[1], w1(1) * (row[0] + row[2]));
    float *dst = S.qp[zp & 1][0];
    dst[t] = ex;
    dst[NT + t] = ey;
    dst[2 * NT + t] = pzs;
    ex_out = ex;
    ey_out = ey;
    pz_out = pzs;
  };
  float qdummy[3];

  __syncthreads();
  fields(z0 - 1, false, r4(z0 - 1), r4(z0), r3(z0 - 1));
  __syncthreads();
  qpartials(z0 - 1, qdummy[0], qdummy[1], qdummy[2]);
  __syncthreads();  // the phi plane is rewritten next
  fields(z0, true, r4(z0), r4(z0 + 1), r3(z0));
  __syncthreads();
  qpartials(z0, qdummy[0], qdummy[1], qdummy[2]);
  // ring slots of planes z, z+1, z+2 (mu') and z-1, z, z+1 (shift),
  // carried from plane to plane instead of recomputed (no division)
  int i4a = r4(z0), i4b = r4(z0 + 1), i4c = r4(z0 + 2);
  int i3m = r3(z0 - 1), i3a = r3(z0), i3b = r3(z0 + 1);
  auto advance = [&]() {
    i4a = i4b;
    i4b = i4c;
    i4c = (i4c + 1) & 3;
    const int t = i3m;
    i3m = i3a;
    i3a = i3b;
    i3b = t;
  };

  // corrections, collision and push of fluid node n of plane z (its
  // populations in f, the shift basis of its stored state in rb, cb)
  auto update = [&](int z, int n, float (&f)[27], float rb, float cb, float Qx, float Qy, float Qz) {
    const float *uF = S.uF[r2(z)][0];
    const float ux = uF[t], uy = uF[NT + t], uz = uF[2 * NT + t];
    const float Fx = uF[3 * NT + t], Fy = uF[4 * NT + t], Fz = uF[5 * NT + t];
    const float r_own = S.rho[r4(z)][c1];
    const float mu_own = S.mu[i4a][(ty + 2) * H2X + tx + 2];
    if (cap) {  // fields of this state for the adjoint: rho, mu', u, F, Q
      cap[n] = r_own;
      cap[N + n] = mu_own;
      cap[2 * N + n] = ux;
      cap[3 * N + n] = uy;
      cap[4 * N + n] = uz;
      cap[5 * N + n] = Fx;
      cap[6 * N + n] = Fy;
      cap[7 * N + n] = Fz;
      cap[8 * N + n] = Qx;
      cap[9 * N + n] = Qy;
      cap[10 * N + n] = Qz;
    }
    const float pm = pm_of(mu_own, kp);
    float om1 = kp.om[1];
    if (kp.nu > 0.0f) om1 = 1.0f / (r_own * kp.nu / pm + 0.5f);

    // the storage shift (basis rb, cb; rho_0 and 0 for the constant shift)
    // added back: f* - s rounded on the store and + s here restore f* exactly
    // wherever f* is within a factor two of s, which is why the shift is
    // added per population and not to the moments
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q] += shift_rest(q, rb, cb);
    // post-collision moments halved as from_central_h takes them
    if (UNIT) {
      to_central_unit(f, ux, uy, uz);
      collide_cm_unit<true>(f, pm, Fx, Fy, Fz, Qx, Qy, Qz, om1, kp);
    } else {
      to_central(f, ux, uy, uz);
      collide_cm<true>(f, pm, Fx, Fy, Fz, Qx, Qy, Qz, om1, kp);
    }
    from_central_h(f, ux, uy, uz);

    // push with bounce-back; shifts keyed by the destination's fields
    const int oz[3] = {z == 0 ? (nz - 1) * nxy : -nxy, 0, z == nz - 1 ? -(nz - 1) * nxy : nxy};
    const float c_own = rest ? basis_c(r_own, mu_own, kp) : 0.0f;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int cx = cx_of(q), cy = cy_of(q), cz = cz_of(q);
      float sh = weight_of(q) * kp.rho_shift;
      if (q == 13) {
        if (rest) sh = shift_rest(q, r_own, c_own);
        store_pop<T>(op.p[q] + n, f[q] - sh);
        continue;
      }
      const int hk = c1 + cx + cy * H1X;
      if (MASK && S.solid[r4(z + cz)][hk]) {
        if (rest) sh = shift_rest(q, r_own, c_own);
        if (WALLV) {  // moving wall: the velocity of the solid node x + c_q
          const int b = n + ox[cx + 1] + oy[cy + 1] + oz[cz + 1];
          sh += wall_odd(q, r_own, pm, wall_u[b], wall_u[N + b], wall_u[2 * N + b]);
        }
        store_pop<T>(op.p[26 - q] + n, f[q] - sh);
      } else {
        if (rest) sh = S.shift[cz < 0 ? i3m : (cz == 0 ? i3a : i3b)][cx * cx + cy * cy + cz * cz][hk];
        const int m = n + ox[cx + 1] + oy[cy + 1] + oz[cz + 1];
        store_pop<T>(op.p[q] + m, f[q] - sh);
      }
    }
    if (rest) {
      sb_out[n] = r_own;
      sb_out[N + n] = c_own;
    }
  };

  // Moments of the output state (Eq. 11), when mo.rho is set: once every
  // block of the cluster has pushed planes up to d + 1, plane d of fout holds
  // all of its populations at the nodes whose 27 sources lie in the
  // cluster's columns and this block's z range, and this thread sums its
  // node there (from L2: the planes were just written).  The first and last
  // rows of the cluster (unless it spans y) and the first and last plane of
  // the z range (unless it spans z) take populations from other clusters or
  // blocks: the edge pass completes them after the kernel.
  const bool mom = mo.rho != nullptr;
  bool yedge = false;
  if (mom && mo.crows < ny) {
    const int lo = (y0 / mo.crows) * mo.crows, hi = min(lo + mo.crows, ny) - 1;
    yedge = y == lo || y == hi;
  }
  auto readback = [&](int d) {
    bool nf = false, dm = false;
    const int nd = x + nx * y + nxy * d;
    if (inside && !yedge && !(MASK && mask[nd])) {
      float v[27];
#pragma unroll
      for (int q = 0; q < 27; ++q) v[q] = load_cg<T>(fout + q * N + nd);
      float sr, sx, sy, sz;
      node_sums(v, sr, sx, sy, sz);
      const float r = sr + (rest ? sb_out[nd] : kp.rho_shift);
      mo.rho[nd] = r;
      mo.j[nd] = sx;
      mo.j[N + nd] = sy;
      mo.j[2 * N + nd] = sz;
      mo.mu0[nd] = mu0_vdw(r, kp);
      nf = !(isfinite(r) && isfinite(sx) && isfinite(sy) && isfinite(sz));
      dm = !nf && !(r > 0.0f && kp.b * r < 1.0f);
    }
    const unsigned bn = __ballot_sync(0xffffffffu, nf), bd = __ballot_sync(0xffffffffu, dm);
    if ((tid & 31) == 0) {
      if (bn) atomicOr(status, STATUS_NONFINITE);
      if (bd) atomicOr(status, STATUS_DOMAIN);
    }
  };

  // A block whose bounded wait gave up stops its work; in a cluster launch it
  // keeps taking part in the cluster barriers so that no other block waits
  // for it forever.
  bool dead = false;
  if (mom) cluster_arrive();
  for (int z = z0; z < z1; ++z, advance()) {
    if (!dead) {
      // publish mu'(z+2), rho/j(z+1); prefetch mu'(z+3), rho/j(z+2)
      store(i4c, z + 1);
      if (z + 1 < z1) fetch(z + 3, z + 2);
      // populations of this node
      const int n = x + nx * y + nxy * z;
      const bool active = inside && (!MASK || !S.solid[r4(z)][c1]);
      float f[27];
      float rb = kp.rho_shift, cb = 0.0f;
      if (rest && active) {
        rb = sb[n];
        cb = sb[N + n];
      }
      if (TMA) {
        const bool ok = (inject && z == z0) ? mbar_wait_bounded(&S.never, 0u, INJECTED_WAIT_NS)
                                            : mbar_wait_bounded(&S.bar, (uint32_t)(z - z0) & 1u);
        if (active) {
#pragma unroll
          for (int q = 0; q < 27; ++q) f[q] = to_f32<T>(fbuf[q * NT + tid]);
        }
        // every thread has its populations: the buffer takes the next plane
        if (__syncthreads_or(!ok)) {
          if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            mbar_wait_bounded(&S.bar, (uint32_t)(z - z0) & 1u);  // let the late copy land before exit
          }
          if (!mom) return;
          dead = true;
        } else if (tid == 0 && z + 1 < z1) {
          // the block's reads of this plane's tile (ordered before this point
          // by the barrier) complete before the copy of the next plane lands
          // in the same buffer
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&S.bar, FBYTES);
          tma_load_4d(smem_raw + FBUF_OFFSET, &tmap, &S.bar, x0, y0, z + 1, 0);
        }
      } else {
        if (active) {
#pragma unroll
          for (int q = 0; q < 27; ++q) f[q] = load_pop<T>(fin + q * N + n);
        }
        __syncthreads();
      }
      if (!dead) {
        fields(z + 1, true, i4b, i4c, i3b);
        __syncthreads();
        // Q of plane z from the partial sums of planes z-1, z (kept) and
        // z+1 (formed now, into the slot of z-1)
        const float *qm = S.qp[(z - 1) & 1][0], *q0 = S.qp[z & 1][0];
        const float exm = qm[t], eym = qm[NT + t], pzm = qm[2 * NT + t];
        const float ex0 = q0[t], ey0 = q0[NT + t];
        float exn, eyn, pzn;
        qpartials(z + 1, exn, eyn, pzn);
        const float Qx = -1.5f * fmaf(w1(0), ex0, w1(1) * (exm + exn));
        const float Qy = -1.5f * fmaf(w1(0), ey0, w1(1) * (eym + eyn));
        const float Qz = -1.5f * (pzn - pzm);
        if (active) {
          update(z, n, f, rb, cb, Qx, Qy, Qz);
        } else if (cap && inside) {  // solid node: its wetting rho and mu', no flow
          cap[n] = S.rho[r4(z)][c1];
          cap[N + n] = S.mu[i4a][(ty + 2) * H2X + tx + 2];
#pragma unroll
          for (int c = 0; c < 9; ++c) cap[(2 + c) * N + n] = 0.0f;
        }
      }
    }
    if (mom) {
      cluster_wait();  // every block of the cluster has pushed plane z - 1
      if (!dead && z - 2 >= z0 + 1) readback(z - 2);
      cluster_arrive();
    }
  }
  if (mom) {
    cluster_wait();  // ... and every plane of its z range
    if (!dead) {
      if (z1 - 2 >= z0 + 1) readback(z1 - 2);
      if (mo.zspan) {  // the z range wraps onto itself: its end planes are complete too
        readback(z1 - 1);
        readback(z0);
      }
    }
  }
}

// Planes per block of a z-marching kernel.  Blocks run in waves of `slots`
// (SMs x resident blocks per SM) and a block of tz planes costs about
// tz + pro plane-times (pro: its prologue of halo planes), so the choice
// minimises waves x (tz + pro): long columns amortise the prologue, short
// ones fill the last wave.
int z_chunk(int xy_blocks, int nz, int slots, int pro) {
  int best = 1;
  long long best_cost = -1;
  for (int tz = 1; tz <= 64; tz *= 2) {
    const long long blocks = (long long)xy_blocks * ((nz + tz - 1) / tz);
    const long long cost = (blocks + slots - 1) / slots * (tz + pro);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = tz;
    }
    if (tz >= nz) break;
  }
  return best;
}

// The dynamic shared-memory limit is a per-device attribute of each kernel:
// raised once per device for every instantiation that is launched.
template <auto K> void ensure_smem(size_t bytes) {
  static std::atomic<unsigned long long> done{0};  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(K, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);  // clusters of up to 16 blocks
    cudaGetLastError();
    done.fetch_or(bit);
  }
}

// SMs x resident blocks per SM of kernel K at this block size and dynamic
// shared memory, once per device
template <auto K> int resident_slots(int threads, size_t smem) {
  static int cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  dev &= 63;
  if (cached[dev] <= 0) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K, threads, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    cached[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 152);
  }
  return cached[dev];
}

// the chemical-potential kernel: z-chunks sized by the same wave model
void launch_mu_z(lbm_ctx *ctx) {
  const KParams &kp = ctx->kp;
  const int xyb = ((kp.nx + MX - 1) / MX) * ((kp.ny + MY - 1) / MY);
  const int mz = z_chunk(xyb, kp.nz, resident_slots<k_mu_z>(MX * MY, 0), 2);
  const dim3 grid((kp.nx + MX - 1) / MX, (kp.ny + MY - 1) / MY, (kp.nz + mz - 1) / mz);
  k_mu_z<<<grid, MX * MY, 0, ctx->stream>>>(ctx->fld.rho, ctx->fld.mu0, ctx->mask, ctx->fld.mu, kp, mz);
}

void launch_moments(lbm_ctx *ctx) {
  const KParams &kp = ctx->kp;
  const Fields &d = ctx->fld;
  const int g = (kp.N + 255) / 256;
  const void *fin = ctx->f[ctx->cur];
  if (ctx->storage == LBM_F16 && kp.N % 2 == 0)
    k_moments_h2<<<(kp.N / 2 + 255) / 256, 256, 0, ctx->stream>>>((const __half *)fin, ctx->mask, d.sb, d.rho, d.j,
                                                                  d.mu0, ctx->status, kp);
  else if (ctx->storage == LBM_F16)
    k_moments_v<__half><<<g, 256, 0, ctx->stream>>>((const __half *)fin, ctx->mask, d.sb, d.rho, d.j, d.mu0,
                                                    ctx->status, kp);
  else
    k_moments_v<float><<<g, 256, 0, ctx->stream>>>((const float *)fin, ctx->mask, d.sb, d.rho, d.j, d.mu0,
                                                   ctx->status, kp);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled of the CUDA driver API, resolved once through the runtime
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// Tensor map of population buffer p as [27][nz][ny][nx] with a box of one
// tile plane (TX x TY x 1 x 27), or nullptr when p cannot be described: the
// rows must be multiples of 16 bytes (nx a multiple of 4 in FP32, 8 in FP16)
// and p 16-byte aligned.  Encoded maps are cached in the context by address.
const CUtensorMap *population_tmap(lbm_ctx *ctx, const void *p) {
  for (const TmapEntry &e : ctx->tmaps)
    if (e.ptr == p) return e.ok ? &e.map : nullptr;
  TmapEntry &e = ctx->tmaps[ctx->tmap_next];
  ctx->tmap_next = (ctx->tmap_next + 1) % TMAP_CACHE;
  e.ptr = p;
  e.ok = 0;
  const size_t es = ctx->storage == LBM_F16 ? 2 : 4;
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || reinterpret_cast<uintptr_t>(p) % 16 != 0 || ((size_t)ctx->nx * es) % 16 != 0) return nullptr;
  const cuuint64_t dims[4] = {(cuuint64_t)ctx->nx, (cuuint64_t)ctx->ny, (cuuint64_t)ctx->nz, 27};
  const cuuint64_t strides[3] = {ctx->nx * es, (cuuint64_t)ctx->nx * ctx->ny * es, (cuuint64_t)ctx->N * es};
  const cuuint32_t box[4] = {TX, TY, 1, 27};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(&e.map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        const_cast<void *>(p), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  e.ok = r == CUDA_SUCCESS;
  return e.ok ? &e.map : nullptr;
}

// Moments of the output state at the nodes the fused step's read-back
// leaves out (Eq. 11), summed like every other moments kernel: mode 0 takes
// the first and last row of each cluster of blocks (crows rows) in every
// plane, mode 1 the other rows of the first and last plane of each block's
// z range (tz planes).  Grids: (ceil(nx / 256), 2 ceil(ny / crows), nz) and
// (ceil(nx / 256), ny, 2 ceil(nz / tz)).
template <typename T>
__global__ void __launch_bounds__(256) k_moments_edge(const T *__restrict__ f, const uint8_t *__restrict__ mask,
                                                      const float *__restrict__ sb, float *__restrict__ rho,
                                                      float *__restrict__ j, float *__restrict__ mu0,
                                                      int *__restrict__ status, KParams kp, int crows, int tz,
                                                      int mode) {
  const int x = blockIdx.x * 256 + threadIdx.x;
  int y, z;
  if (mode == 0) {
    const int e = blockIdx.y, lo = (e >> 1) * crows, hi = min(lo + crows, kp.ny) - 1;
    if ((e & 1) && hi == lo) return;  // a one-row cluster has one edge row (whole block)
    y = (e & 1) ? hi : lo;
    z = blockIdx.z;
  } else {
    const int e = blockIdx.z, lo = (e >> 1) * tz, hi = min(lo + tz, kp.nz) - 1;
    if ((e & 1) && hi == lo) return;
    z = (e & 1) ? hi : lo;
    y = blockIdx.y;
    if (crows < kp.ny) {  // edge rows are mode 0's
      const int ylo = (y / crows) * crows, yhi = min(ylo + crows, kp.ny) - 1;
      if (y == ylo || y == yhi) return;
    }
  }
  bool bad_nf = false, bad_dom = false;
  const int n = x + kp.nx * (y + kp.ny * z);
  if (x < kp.nx && !(mask && mask[n])) {
    const size_t N = (size_t)kp.N;
    float v[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) v[q] = load_pop<T>(f + q * N + n);
    float s, sx, sy, sz;
    node_sums(v, s, sx, sy, sz);
    const float r = s + (kp.shift_mode == LBM_SHIFT_REST ? sb[n] : kp.rho_shift);
    rho[n] = r;
    j[n] = sx;
    j[N + n] = sy;
    j[2 * N + n] = sz;
    mu0[n] = mu0_vdw(r, kp);
    bad_nf = !(isfinite(r) && isfinite(sx) && isfinite(sy) && isfinite(sz));
    bad_dom = !bad_nf && !(r > 0.0f && kp.b * r < 1.0f);
  }
  const unsigned nf = __ballot_sync(0xffffffffu, bad_nf), dm = __ballot_sync(0xffffffffu, bad_dom);
  if ((threadIdx.x & 31) == 0) {
    if (nf) atomicOr(status, STATUS_NONFINITE);
    if (dm) atomicOr(status, STATUS_DOMAIN);
  }
}

// Cluster launch of the fused step that also produces the next moments:
// the cluster spans every block column in x (so no population crosses its x
// edges) and as many block rows as fit in 16 blocks; z ranges of at least 4
// planes.  Chosen once per context from the occupancy of the kernel K.
template <auto K>
bool mom_config(lbm_ctx *ctx, size_t smem) {
  if (ctx->mom_cfg) return ctx->mom_cfg > 0;
  ctx->mom_cfg = -1;
  const KParams &kp = ctx->kp;
  const int gx = (kp.nx + TX - 1) / TX, gy = (kp.ny + TY - 1) / TY;
  if (ctx->no_mom || gx > 16 || kp.nz < 3) return false;
  for (int cy = 16 / gx; cy >= 1; --cy) {
    if (gy % cy) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(gx, gy, 1);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = gx;
    at.val.clusterDim.y = cy;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, K, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      continue;
    }
    int tz = z_chunk(gx * gy, kp.nz, clusters * gx * cy, 2);
    if (tz < kp.nz) tz = max(tz, 4);
    if (tz >= kp.nz) tz = kp.nz;
    ctx->mom_cx = gx;
    ctx->mom_cy = cy;
    ctx->mom_tz = tz;
    ctx->mom_cfg = 1;
    return true;
  }
  return false;
}

// Launches k_fused; with the tensor-copy path and a usable cluster shape it
// also writes the moments of the output state into the other moment set
// (returns true: the edge pass must follow).
// The cluster shape from a representative instantiation: every k_fused
// instantiation has the same launch bounds and shared memory, so the same
// occupancy.
template <typename T>
bool mom_config_t(lbm_ctx *ctx) {
  constexpr auto K = k_fused<T, false, true, false, true, true>;
  constexpr size_t sm = fused_smem_size<T>(true);
  ensure_smem<K>(sm);
  return mom_config<K>(ctx, sm);
}

template <typename T, bool MASK, bool TMA, bool WALLV, bool UNIT, bool REST>
bool launch_fused_u(lbm_ctx *ctx, const T *fin, T *fout, const CUtensorMap &map, bool produce) {
  const KParams &kp = ctx->kp;
  const Fields &d = ctx->fld;
  constexpr size_t sm = fused_smem_size<T>(TMA);
  constexpr auto K = k_fused<T, MASK, TMA, WALLV, UNIT, REST>;
  ensure_smem<K>(sm);
  const int gx = (kp.nx + TX - 1) / TX, gy = (kp.ny + TY - 1) / TY;
  float *sb_out = ctx->sb_out ? ctx->sb_out : d.sb;
  const uint8_t *mask = MASK ? ctx->mask : nullptr;
  const float *wall_u = WALLV ? ctx->wall_u : nullptr;
  PopPlanes<T> op;
  for (int q = 0; q < 27; ++q) op.p[q] = fout + (size_t)q * kp.N;
  if (TMA && produce) {
    const Moments &m = ctx->mom[1 - ctx->cur];
    MomArgs mo{m.rho, m.j, m.mu0, ctx->mom_cy * TY, ctx->mom_tz >= kp.nz ? 1 : 0};
    const int tz = ctx->mom_tz;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(gx, gy, (kp.nz + tz - 1) / tz);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = ctx->mom_cx;
    at.val.clusterDim.y = ctx->mom_cy;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, K, fin, fout, mask, (const float *)d.rho, (const float *)d.j, (const float *)d.mu,
                       (const float *)d.sb, sb_out, ctx->status, ctx->capture, wall_u, mo, op, kp, tz, map);
    return true;
  }
  const int tz = z_chunk(gx * gy, kp.nz, resident_slots<K>(NT, sm), 2);
  const dim3 grid(gx, gy, (kp.nz + tz - 1) / tz);
  const MomArgs none{nullptr, nullptr, nullptr, 0, 0};
  K<<<grid, NT, sm, ctx->stream>>>(fin, fout, mask, d.rho, d.j, d.mu, d.sb, sb_out, ctx->status, ctx->capture,
                                   wall_u, none, op, kp, tz, map);
  return false;
}

// every rate but omega_1 equal to 1 (exactly: each 1 - omega_i is 0)
bool unit_rates(const KParams &kp) {
  for (int i = 0; i < 11; ++i)
    if (i != 1 && kp.om_c[i] != 0.0f) return false;
  return true;
}

template <typename T, bool MASK, bool TMA, bool WALLV>
bool launch_fused_k(lbm_ctx *ctx, const T *fin, T *fout, const CUtensorMap &map, bool produce) {
  const bool unit = unit_rates(ctx->kp), rest = ctx->kp.shift_mode == LBM_SHIFT_REST;
  if (unit && rest) return launch_fused_u<T, MASK, TMA, WALLV, true, true>(ctx, fin, fout, map, produce);
  if (unit) return launch_fused_u<T, MASK, TMA, WALLV, true, false>(ctx, fin, fout, map, produce);
  if (rest) return launch_fused_u<T, MASK, TMA, WALLV, false, true>(ctx, fin, fout, map, produce);
  return launch_fused_u<T, MASK, TMA, WALLV, false, false>(ctx, fin, fout, map, produce);
}

template <typename T>
bool launch_fused(lbm_ctx *ctx, const void *fin_v, void *fout_v, bool produce) {
  const T *fin = static_cast<const T *>(fin_v);
  T *fout = static_cast<T *>(fout_v);
  const CUtensorMap *map = population_tmap(ctx, fin_v);
  const bool moving = ctx->mask && ctx->wall_u;
  if (map) {
    if (moving) return launch_fused_k<T, true, true, true>(ctx, fin, fout, *map, produce);
    if (ctx->mask) return launch_fused_k<T, true, true, false>(ctx, fin, fout, *map, produce);
    return launch_fused_k<T, false, true, false>(ctx, fin, fout, *map, produce);
  }
  // rows that a tensor copy cannot describe: per-thread loads, the mask
  // checks compiled in (an all-fluid domain has an all-zero solid plane)
  static const CUtensorMap unused{};
  if (moving) return launch_fused_k<T, true, false, true>(ctx, fin, fout, unused, false);
  return launch_fused_k<T, true, false, false>(ctx, fin, fout, unused, false);
}

// the edge pass after a fused step that produced the next moments
template <typename T>
void launch_edge(lbm_ctx *ctx, const void *fout) {
  const KParams &kp = ctx->kp;
  const Moments &m = ctx->mom[1 - ctx->cur];
  const float *sb = ctx->sb_out ? ctx->sb_out : ctx->fld.sb;
  const int crows = ctx->mom_cy * TY, tz = ctx->mom_tz;
  const int gx = (kp.nx + 255) / 256;
  if (crows < kp.ny) {
    const dim3 g(gx, 2 * ((kp.ny + crows - 1) / crows), kp.nz);
    k_moments_edge<T><<<g, 256, 0, ctx->stream>>>((const T *)fout, ctx->mask, sb, m.rho, m.j, m.mu0, ctx->status,
                                                  kp, crows, tz, 0);
    ctx->launches++;
  }
  if (tz < kp.nz) {
    const dim3 g(gx, kp.ny, 2 * ((kp.nz + tz - 1) / tz));
    k_moments_edge<T><<<g, 256, 0, ctx->stream>>>((const T *)fout, ctx->mask, sb, m.rho, m.j, m.mu0, ctx->status,
                                                  kp, crows, tz, 1);
    ctx->launches++;
  }
}

}  // namespace

void launch_moments_mu(lbm_ctx *ctx) {
  launch_moments(ctx);
  ctx->launches++;
  if (ctx->n_bnd) launch_wet_rho(ctx);
  launch_mu_z(ctx);
  ctx->launches++;
  if (ctx->n_bnd) launch_wet_mu(ctx);
}

void launch_moments_current(lbm_ctx *ctx) {
  {
    TimedLaunch t(ctx, K_MOMENTS);
    launch_moments(ctx);
  }
  ctx->mom_valid = 1;
}

// Whether a step from the current state also produces the next state's
// moments: the tensor-copy instantiations with a usable cluster shape.
bool step_produces_moments(lbm_ctx *ctx) {
  if (!ctx->fuse_mom || ctx->no_mom || !population_tmap(ctx, ctx->f[ctx->cur])) return false;
  return ctx->storage == LBM_F16 ? mom_config_t<__half>(ctx) : mom_config_t<float>(ctx);
}

void launch_step_fused(lbm_ctx *ctx) {
  const void *fin = ctx->f[ctx->cur];
  void *fout = ctx->f[1 - ctx->cur];
  // the separate moments pass, unless the previous fused step produced them
  const bool produce = step_produces_moments(ctx);
  if (!produce || !ctx->mom_valid) launch_moments_current(ctx);
  if (ctx->n_bnd) launch_wet_rho(ctx);
  {
    TimedLaunch t(ctx, K_MU);
    launch_mu_z(ctx);
  }
  if (ctx->n_bnd) launch_wet_mu(ctx);
  bool produced;
  {
    TimedLaunch t(ctx, K_COLLIDE);
    produced = ctx->storage == LBM_F16 ? launch_fused<__half>(ctx, fin, fout, produce)
                                       : launch_fused<float>(ctx, fin, fout, produce);
  }
  if (produced) {
    TimedLaunch t(ctx, K_MOM_EDGE);
    ctx->launches--;  // launch_edge counts its launches (zero to two)
    if (ctx->storage == LBM_F16)
      launch_edge<__half>(ctx, fout);
    else
      launch_edge<float>(ctx, fout);
  }
  ctx->kp.inject_wait = 0;  // the injected wait is one-shot
  ctx->cur = 1 - ctx->cur;
  view_moments(ctx);
  ctx->mom_valid = produced ? 1 : 0;
}

}  // namespace lbm
