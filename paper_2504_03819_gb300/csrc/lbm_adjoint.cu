// Discrete adjoint of one time step (reverse mode of the step in
// lbm_forward.cu / lbm_step_fused.cu).  The paper has no adjoint; this is the
// exact transpose of the linearised discrete map f(t) -> f(t+1).
//
// Given the state f(t) and lambda(t+1) = dJ/df(t+1), the kernels compute
// lambda(t) = (df(t+1)/df(t))^T lambda(t+1) and add the step's contribution
// to dJ/d{kappa, omega_0..10, wetting value}:
//
//   forward recompute   rho, j, mu', u, F, phi, Q of f(t) (staged kernels)
//   k_adj_collide       pull of lambda(t+1) (transpose of push + bounce-back),
//                       transpose of the inverse CM transform, of the
//                       collision (Eqs. 21-26, 28) and of the forward CM
//                       transform (Eq. 19), with the u-derivatives of both
//                       transforms; adjoint sources for u, F, Q, p_m, omega_1
//   k_adj_fields        Q_aa = -3 d_a phi_a (Eq. 27) transposed (a gather),
//                       phi = (p_m - rho/3) u, u = (j + F/2)/rho,
//                       F = (1/3 - rho) grad mu (Eq. 12), p_m = (1 + mu)/3,
//                       per-node omega_1 (Sec. II B) transposed
//   k_adj_mu            grad mu transposed (a gather) + the local p_m term
//   k_adj_wet_mu        Eq. 36 transposed (solid -> fluid neighbours)
//   k_adj_rho           mu = mu0(rho) - kappa lap rho (Eqs. 2, 32) transposed,
//                       Eqs. 37-38 transposed at solid boundary nodes (branch
//                       of the forward pass: clamped densities pass no
//                       gradient), and lambda_q(t) = local part + lambda_rho
//                       + c_q . lambda_j at fluid nodes away from walls
//   k_adj_out_wall      the same output at fluid nodes next to walls, with
//                       the wetting gather
//
// Parameter gradients are summed per block in FP64 and reduced in a fixed
// order (deterministic).
#include "lbm_lattice.cuh"

namespace lbm {

namespace {

constexpr int BLK = 128;
// parameter slots: 0 kappa, 1..11 omega_0..omega_10, 12 wetting value
constexpr int NPAR = 13;

// ---------------------------------------------------------------------------
// one axis of the CM transform: forward A(u), inverse B(u) and transposes
// ---------------------------------------------------------------------------
// forward: M0 = a+b+c, M1 = (c-a) - u M0, M2 = (a+c) - 2u(c-a) + u^2 M0
__device__ __forceinline__ void fwd_T(float &a, float &b, float &c, float u) {
  // (a, b, c) <- A(u)^T (l0, l1, l2) with (l0, l1, l2) = (a, b, c) on entry
  const float l0 = a, l1 = b, l2 = c;
  a = l0 + (-1.0f - u) * l1 + (1.0f + u) * (1.0f + u) * l2;
  b = l0 - u * l1 + u * u * l2;
  c = l0 + (1.0f - u) * l1 + (1.0f - u) * (1.0f - u) * l2;
}
// d/du of the forward outputs given the inputs (a, b, c), dotted with the
// adjoints (l1, l2) of (M1, M2)
__device__ __forceinline__ float fwd_du(float a, float b, float c, float u, float l1, float l2) {
  const float m0 = a + b + c, d = c - a;
  return -m0 * l1 + (-2.0f * d + 2.0f * u * m0) * l2;
}
// inverse: a = ((u^2-u) M0 + (2u-1) M1 + M2)/2, b = (1-u^2) M0 - 2u M1 - M2,
//          c = ((u^2+u) M0 + (2u+1) M1 + M2)/2
__device__ __forceinline__ void inv_T(float &m0, float &m1, float &m2, float u) {
  const float la = m0, lb = m1, lc = m2;
  m0 = 0.5f * (u * u - u) * la + (1.0f - u * u) * lb + 0.5f * (u * u + u) * lc;
  m1 = 0.5f * (2.0f * u - 1.0f) * la - 2.0f * u * lb + 0.5f * (2.0f * u + 1.0f) * lc;
  m2 = 0.5f * la - lb + 0.5f * lc;
}
__device__ __forceinline__ float inv_du(float m0, float m1, float la, float lb, float lc, float u) {
  return la * (0.5f * (2.0f * u - 1.0f) * m0 + m1) + lb * (-2.0f * u * m0 - 2.0f * m1) +
         lc * (0.5f * (2.0f * u + 1.0f) * m0 + m1);
}

// copy helpers for 27-arrays
__device__ __forceinline__ void cp27(float *d, const float *s) {
#pragma unroll
  for (int q = 0; q < 27; ++q) d[q] = s[q];
}

// pass indices (same order as to_central / from_central)
// z-pass triples: (p, p+9, p+18), p = 0..8;  y-pass: (a+9g, a+3+9g, a+6+9g);
// x-pass: (q, q+1, q+2), q = 0, 3, ..., 24.

// lam <- (d from_central / d k)^T lam, accumulating d/du into gu.  kin are the
// post-collision moments (input of from_central).  The intermediate stages of
// from_central are recomputed from kin one at a time (one scratch array).
__device__ __forceinline__ void from_central_vjp(float lam[27], const float kin[27], float ux, float uy, float uz,
                                                 float &gux, float &guy, float &guz) {
  float K[27];
  // z-pass (last) transposed; its inputs are Y(X(kin))
  cp27(K, kin);
#pragma unroll
  for (int q = 0; q < 27; q += 3) cm_axis_inv(K[q], K[q + 1], K[q + 2], ux);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) cm_axis_inv(K[a + 9 * g], K[a + 3 + 9 * g], K[a + 6 + 9 * g], uy);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    guz += inv_du(K[p], K[p + 9], lam[p], lam[p + 9], lam[p + 18], uz);
    inv_T(lam[p], lam[p + 9], lam[p + 18], uz);
  }
  // y-pass transposed; its inputs are X(kin)
  cp27(K, kin);
#pragma unroll
  for (int q = 0; q < 27; q += 3) cm_axis_inv(K[q], K[q + 1], K[q + 2], ux);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int i0 = a + 9 * g, i1 = a + 3 + 9 * g, i2 = a + 6 + 9 * g;
      guy += inv_du(K[i0], K[i1], lam[i0], lam[i1], lam[i2], uy);
      inv_T(lam[i0], lam[i1], lam[i2], uy);
    }
  // x-pass transposed; its inputs are kin
#pragma unroll
  for (int q = 0; q < 27; q += 3) {
    gux += inv_du(kin[q], kin[q + 1], lam[q], lam[q + 1], lam[q + 2], ux);
    inv_T(lam[q], lam[q + 1], lam[q + 2], ux);
  }
}

// lam <- (d to_central / d f)^T lam, accumulating d/du.  f are the populations
// (input of to_central); stages are recomputed from f one at a time.
__device__ __forceinline__ void to_central_vjp(float lam[27], const float f[27], float ux, float uy, float uz,
                                               float &gux, float &guy, float &guz) {
  float G[27];
  // x-pass (last) transposed; its inputs are Y(Z(f))
  cp27(G, f);
#pragma unroll
  for (int p = 0; p < 9; ++p) cm_axis(G[p], G[p + 9], G[p + 18], uz);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) cm_axis(G[a + 9 * g], G[a + 3 + 9 * g], G[a + 6 + 9 * g], uy);
#pragma unroll
  for (int q = 0; q < 27; q += 3) {
    gux += fwd_du(G[q], G[q + 1], G[q + 2], ux, lam[q + 1], lam[q + 2]);
    fwd_T(lam[q], lam[q + 1], lam[q + 2], ux);
  }
  // y-pass transposed; its inputs are Z(f)
  cp27(G, f);
#pragma unroll
  for (int p = 0; p < 9; ++p) cm_axis(G[p], G[p + 9], G[p + 18], uz);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int i0 = a + 9 * g, i1 = a + 3 + 9 * g, i2 = a + 6 + 9 * g;
      guy += fwd_du(G[i0], G[i1], G[i2], uy, lam[i1], lam[i2]);
      fwd_T(lam[i0], lam[i1], lam[i2], uy);
    }
  // z-pass transposed; its inputs are f
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    guz += fwd_du(f[p], f[p + 9], f[p + 18], uz, lam[p + 9], lam[p + 18]);
    fwd_T(lam[p], lam[p + 9], lam[p + 18], uz);
  }
}

// to_central_vjp when every rate but omega_1 is 1: the collision then reads
// only k000 and the six second-order central moments (its transpose leaves
// every other entry of lam exactly zero), and the transpose of the transform
// has a closed form per population.  With X = c_x - u_x, Y, Z likewise,
//   lam_q = l000 + l200 X^2 + l020 Y^2 + l002 Z^2 + l110 X Y + l101 X Z + l011 Y Z,
// and since d k200 / d u_x = -2 k100, d k110 / d u_x = -k010, ..., the
// u-derivatives need only the first central moments k of the recompute.
__device__ __forceinline__ void to_central_vjp_unit(float lam[27], const float k[27], float ux, float uy, float uz,
                                                    float &gux, float &guy, float &guz) {
  const float l000 = lam[0], l200 = lam[2], l020 = lam[6], l002 = lam[18];
  const float l110 = lam[4], l101 = lam[10], l011 = lam[12];
  const float k100 = k[1], k010 = k[3], k001 = k[9];
  gux += -2.0f * l200 * k100 - l110 * k010 - l101 * k001;
  guy += -2.0f * l020 * k010 - l110 * k100 - l011 * k001;
  guz += -2.0f * l002 * k001 - l101 * k100 - l011 * k010;
  float X[3], Y[3], Z[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    X[c] = (float)(c - 1) - ux;
    Y[c] = (float)(c - 1) - uy;
    Z[c] = (float)(c - 1) - uz;
  }
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int i = q % 3, j = (q / 3) % 3, m = q / 9;
    const float ax = fmaf(l200, X[i], fmaf(l110, Y[j], l101 * Z[m]));  // multiplies X
    const float ay = fmaf(l020, Y[j], l011 * Z[m]);                     // multiplies Y
    lam[q] = fmaf(ax, X[i], fmaf(ay, Y[j], fmaf(l002 * Z[m], Z[m], l000)));
  }
}

#define LK(a, b, c) lk[(a) + 3 * (b) + 9 * (c)]
#define LS(a, b, c) ls[(a) + 3 * (b) + 9 * (c)]

// Transpose of collide_cm (Eqs. 21-26, 28).  k: pre-collision moments;
// ls: adjoint of the post-collision moments (consumed); lk: adjoint of k
// (output).  Accumulates the adjoints of p_m, F, Q, omega_1 (om1) and of
// the global rates (gom[0..10], gom[1] unused here).
__device__ __forceinline__ void collide_vjp(const float *k, float *ls, float *lk, float pm, float Fx, float Fy,
                                            float Fz, float Qx, float Qy, float Qz, float om1, const KParams &kp,
                                            float &lpm, float &lFx, float &lFy, float &lFz, float &lQx, float &lQy,
                                            float &lQz, float &lom1, float gom[11]) {
  const float o0 = kp.om[0], o2 = kp.om[2], o3 = kp.om[3], o4 = kp.om[4], o5 = kp.om[5];
  const float o6 = kp.om[6], o7 = kp.om[7], o8 = kp.om[8], o9 = kp.om[9], o10 = kp.om[10];
  const float cs2 = 1.0f / 3.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) lk[q] = 0.0f;
  LK(0, 0, 0) = LS(0, 0, 0);
  // first order
  {
    const float Fa[3] = {Fx, Fy, Fz};
    const int ids[3] = {1, 3, 9};
    float *lF[3] = {&lFx, &lFy, &lFz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float l = ls[ids[a]];
      lk[ids[a]] = (1.0f - o0) * l;
      *lF[a] += (1.0f - 0.5f * o0) * l;
      gom[0] += (-k[ids[a]] - 0.5f * Fa[a]) * l;
    }
  }
  // second order off-diagonal
  {
    const int ids[3] = {4, 12, 10};  // k110, k011, k101
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lk[ids[a]] = (1.0f - om1) * ls[ids[a]];
      lom1 += -k[ids[a]] * ls[ids[a]];
    }
  }
  // second order diagonal
  {
    const float l200 = LS(2, 0, 0), l020 = LS(0, 2, 0), l002 = LS(0, 0, 2);
    const float lS = (l200 + l020 + l002) * (1.0f / 3.0f);
    const float lA = (l200 - 2.0f * l020 + l002) * (1.0f / 3.0f);
    const float lB = (l200 + l020 - 2.0f * l002) * (1.0f / 3.0f);
    const float k200 = k[2], k020 = k[6], k002 = k[18];
    LK(2, 0, 0) += (1.0f - om1) * (lA + lB) + (1.0f - o2) * lS;
    LK(0, 2, 0) += -(1.0f - om1) * lA + (1.0f - o2) * lS;
    LK(0, 0, 2) += -(1.0f - om1) * lB + (1.0f - o2) * lS;
    const float h1 = 1.0f - 0.5f * om1, h2 = 1.0f - 0.5f * o2;
    lQx += h1 * (lA + lB) + h2 * lS;
    lQy += -h1 * lA + h2 * lS;
    lQz += -h1 * lB + h2 * lS;
    lpm += 3.0f * o2 * lS;
    lom1 += (-(k200 - k020) - 0.5f * (Qx - Qy)) * lA + (-(k200 - k002) - 0.5f * (Qx - Qz)) * lB;
    gom[2] += (-(k200 + k020 + k002) + 3.0f * pm - 0.5f * (Qx + Qy + Qz)) * lS;
  }
  // third order
  {
    // pairs (k120, k102) with F_x, (k210, k012) with F_y, (k201, k021) with F_z
    const int P0[3] = {7, 5, 11}, P1[3] = {19, 21, 15};
    const float Fa[3] = {Fx, Fy, Fz};
    float *lF[3] = {&lFx, &lFy, &lFz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float lP = 0.5f * (ls[P0[a]] + ls[P1[a]]);
      const float lD = 0.5f * (ls[P0[a]] - ls[P1[a]]);
      lk[P0[a]] = (1.0f - o3) * lP + (1.0f - o4) * lD;
      lk[P1[a]] = (1.0f - o3) * lP - (1.0f - o4) * lD;
      *lF[a] += 2.0f * (1.0f - 0.5f * o3) * cs2 * lP;
      gom[3] += (-(k[P0[a]] + k[P1[a]]) - Fa[a] * cs2) * lP;
      gom[4] += -(k[P0[a]] - k[P1[a]]) * lD;
    }
    LK(1, 1, 1) = (1.0f - o5) * LS(1, 1, 1);
    gom[5] += -KM(1, 1, 1) * LS(1, 1, 1);
  }
  // fourth order
  {
    const float a = KM(2, 2, 0), b = KM(2, 0, 2), c = KM(0, 2, 2);
    const float lT = (LS(2, 2, 0) + LS(2, 0, 2) + LS(0, 2, 2)) * (1.0f / 3.0f);
    const float lD1 = (LS(2, 2, 0) - LS(2, 0, 2)) * (1.0f / 3.0f);
    const float lD2 = (LS(2, 2, 0) - LS(0, 2, 2)) * (1.0f / 3.0f);
    LK(2, 2, 0) = (1.0f - o6) * (lD1 + lD2) + (1.0f - o7) * lT;
    LK(2, 0, 2) = (1.0f - o6) * (-2.0f * lD1 + lD2) + (1.0f - o7) * lT;
    LK(0, 2, 2) = (1.0f - o6) * (lD1 - 2.0f * lD2) + (1.0f - o7) * lT;
    float Q220 = 0.0f, Q202 = 0.0f, Q022 = 0.0f;
    if (kp.q4) {
      Q220 = (Qx + Qy) * cs2;
      Q202 = (Qx + Qz) * cs2;
      Q022 = (Qy + Qz) * cs2;
      const float h6 = 1.0f - 0.5f * o6, h7 = 1.0f - 0.5f * o7;
      const float l220 = h6 * (lD1 + lD2) + h7 * lT;
      const float l202 = h6 * (-2.0f * lD1 + lD2) + h7 * lT;
      const float l022 = h6 * (lD1 - 2.0f * lD2) + h7 * lT;
      lQx += (l220 + l202) * cs2;
      lQy += (l220 + l022) * cs2;
      lQz += (l202 + l022) * cs2;
    }
    lpm += o7 * lT;
    gom[6] += (-(a - 2.0f * b + c) - 0.5f * (Q220 - 2.0f * Q202 + Q022)) * lD1 +
              (-(a + b - 2.0f * c) - 0.5f * (Q220 + Q202 - 2.0f * Q022)) * lD2;
    gom[7] += (-(a + b + c) + pm - 0.5f * (Q220 + Q202 + Q022)) * lT;
    const int ids[3] = {14, 16, 22};  // k211, k121, k112
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lk[ids[i]] = (1.0f - o8) * ls[ids[i]];
      gom[8] += -k[ids[i]] * ls[ids[i]];
    }
  }
  // fifth order
  {
    const int i122 = 1 + 6 + 18, i212 = 2 + 3 + 18, i221 = 2 + 6 + 9;
    const int id5[3] = {i122, i212, i221};
    const float Fa[3] = {Fx, Fy, Fz};
    float *lF[3] = {&lFx, &lFy, &lFz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float l = ls[id5[a]];
      lk[id5[a]] = (1.0f - o9) * l;
      *lF[a] += (1.0f - 0.5f * o9) * cs2 * cs2 * l;
      gom[9] += (-k[id5[a]] - 0.5f * Fa[a] * cs2 * cs2) * l;
    }
  }
  // sixth order
  LK(2, 2, 2) = (1.0f - o10) * LS(2, 2, 2);
  lpm += o10 * cs2 * cs2 * LS(2, 2, 2);
  gom[10] += (-KM(2, 2, 2) + pm * cs2 * cs2) * LS(2, 2, 2);
}

// every rate but omega_1 equal to 1 (each 1 - omega_i exactly 0): the rate
// setting for which the forward step takes its unit-rate collision
bool adj_unit_rates(const KParams &kp) {
  for (int i = 0; i < 11; ++i)
    if (i != 1 && kp.om_c[i] != 0.0f) return false;
  return true;
}

// A node of a 3-D launch: blocks of 32 x blockDim.y threads over (x, y), one
// z-plane per block row of the grid; neighbour indices by periodic offsets.
struct Site {
  int n;
  bool in;
  int ox[3], oy[3], oz[3];
  __device__ __forceinline__ int at(int cx, int cy, int cz) const { return n + ox[cx + 1] + oy[cy + 1] + oz[cz + 1]; }
};

__device__ __forceinline__ Site site_of(const KParams &kp) {
  Site s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz, nxy = nx * ny;
  s.in = x < nx && y < ny;
  s.n = x + nx * (y + ny * z);
  s.ox[0] = x == 0 ? nx - 1 : -1;
  s.ox[1] = 0;
  s.ox[2] = x == nx - 1 ? -(nx - 1) : 1;
  s.oy[0] = y == 0 ? (ny - 1) * nx : -nx;
  s.oy[1] = 0;
  s.oy[2] = y == ny - 1 ? -(ny - 1) * nx : nx;
  s.oz[0] = z == 0 ? (nz - 1) * nxy : -nxy;
  s.oz[1] = 0;
  s.oz[2] = z == nz - 1 ? -(nz - 1) * nxy : nxy;
  return s;
}

// Site of node n (for kernels over node lists)
__device__ __forceinline__ Site site_at(int n, const KParams &kp) {
  Site s;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz, nxy = nx * ny;
  const int x = n % nx, t = n / nx, y = t % ny, z = t / ny;
  s.in = true;
  s.n = n;
  s.ox[0] = x == 0 ? nx - 1 : -1;
  s.ox[1] = 0;
  s.ox[2] = x == nx - 1 ? -(nx - 1) : 1;
  s.oy[0] = y == 0 ? (ny - 1) * nx : -nx;
  s.oy[1] = 0;
  s.oy[2] = y == ny - 1 ? -(ny - 1) * nx : nx;
  s.oz[0] = z == 0 ? (nz - 1) * nxy : -nxy;
  s.oz[1] = 0;
  s.oz[2] = z == nz - 1 ? -(nz - 1) * nxy : nxy;
  return s;
}

__device__ __forceinline__ int block_id() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }

// Block sums of M FP32 per-node values, added to the parameter slots
// slot[0..M) of partial[block_id() * NPAR + ...]: a fixed FP32 shuffle tree
// per warp (the per-node contributions are FP32), then the warp sums in FP64
// in warp order.  Deterministic; the partials accumulate over launches until
// the caller reduces them.
template <int M>
__device__ void block_partials(float (&v)[M], const int (&slot)[M], double *partial) {
  constexpr int MAXW = 8;
  __shared__ float sm[M][MAXW];
  const int t = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y) / 32;
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  if ((t & 31) == 0)
#pragma unroll
    for (int i = 0; i < M; ++i) sm[i][t >> 5] = v[i];
  __syncthreads();
  if (t < M) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += (double)sm[t][w];
    partial[(size_t)block_id() * NPAR + slot[t]] += acc;
  }
}

// the same with FP64 per-node values in every slot (objective sums)
__device__ void block_partials_f64(double (&v)[NPAR], double *partial) {
  constexpr int MAXW = 8;
  __shared__ double sm[NPAR][MAXW];
  const int t = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y) / 32;
#pragma unroll
  for (int i = 0; i < NPAR; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  if ((t & 31) == 0)
#pragma unroll
    for (int i = 0; i < NPAR; ++i) sm[i][t >> 5] = v[i];
  __syncthreads();
  if (t < NPAR) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += sm[t][w];
    partial[(size_t)block_id() * NPAR + t] += acc;
  }
}

// ---------------------------------------------------------------------------
// collision + streaming adjoint, per fluid node
// ---------------------------------------------------------------------------
// four blocks per SM for FP32 storage (128 registers: about 200 bytes per
// thread spill to L1, and the extra warps hide more of the kernel's load
// latency than the spills cost: 1.5% faster than three blocks without
// spills); the FP16 conversions need the register budget of two.  UNIT:
// every rate but omega_1 is 1 (to_central_vjp_unit; the populations are
// loaded once).
template <typename T, bool UNIT>
__global__ void __launch_bounds__(BLK, sizeof(T) == 4 ? 4 : 2) k_adj_collide(const T *__restrict__ fstate, const float *__restrict__ sb,
                                                     const uint8_t *__restrict__ mask, const uint32_t *__restrict__ nbr,
                                                     const float *__restrict__ lam_next, float *__restrict__ lam_t,
                                                     Fields d, AdjFields a, const float *__restrict__ wall_u,
                                                     double *__restrict__ partial, KParams kp) {
  const Site st = site_of(kp);
  const int n = st.n;
  float pg[11];  // dJ/d omega_0..omega_10 of this node
#pragma unroll
  for (int i = 0; i < 11; ++i) pg[i] = 0.0f;
  const size_t N = (size_t)kp.N;
  if (st.in) {
    if (mask && mask[n]) {
#pragma unroll
      for (int q = 0; q < 27; ++q) lam_t[q * N + n] = 0.0f;
      for (int c = 0; c < 3; ++c) a.u[c * N + n] = a.F[c * N + n] = a.Q[c * N + n] = 0.0f;
      a.pm[n] = 0.0f;
      a.om1[n] = 0.0f;
      a.rho[n] = 0.0f;
    } else {
      const bool rest = kp.shift_mode == LBM_SHIFT_REST;
      const float rb = rest ? sb[n] : kp.rho_shift, cb = rest ? sb[N + n] : 0.0f;
      auto load_f = [&](float f[27]) {
#pragma unroll
        for (int q = 0; q < 27; ++q)
          f[q] = load_pop<T>(fstate + q * N + n) + (rest ? shift_rest(q, rb, cb) : weight_of(q) * rb);
      };
      // pull of lambda(t+1): transpose of push with bounce-back
      const uint32_t solid = mask ? nbr[n] : 0u;
      float lam[27];
#pragma unroll
      for (int q = 0; q < 27; ++q) {
        if (q == 13) {
          lam[q] = lam_next[q * N + n];
          continue;
        }
        lam[q] = ((solid >> q) & 1u) ? lam_next[(size_t)(26 - q) * N + n]
                                     : lam_next[q * N + st.at(cx_of(q), cy_of(q), cz_of(q))];
      }
      // moving walls: the bounced population carries -wall_odd(q, rho, p_m,
      // U(x + c_q)); its rho and p_m derivatives
      float lr_wall = 0.0f, lpm_wall = 0.0f;
      if (wall_u && solid) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
          if (q == 13 || !((solid >> q) & 1u)) continue;
          const int b = st.at(cx_of(q), cy_of(q), cz_of(q));
          const float cu = cx_of(q) * wall_u[b] + cy_of(q) * wall_u[N + b] + cz_of(q) * wall_u[2 * N + b];
          const float g = -6.0f * weight_of(q) * cu * lam[q];
          lr_wall += g * wall_coef_rho(q);
          lpm_wall += g * wall_coef_pm(q);
        }
      }
      const float ux = d.u[n], uy = d.u[N + n], uz = d.u[2 * N + n];
      const float Fx = d.F[n], Fy = d.F[N + n], Fz = d.F[2 * N + n];
      const float Qx = d.Q[n], Qy = d.Q[N + n], Qz = d.Q[2 * N + n];
      const float r = d.rho[n];
      const float pm = pm_of(d.mu[n], kp);
      float om1 = kp.om[1];
      if (kp.nu > 0.0f) om1 = 1.0f / (r * kp.nu / pm + 0.5f);
      // forward recompute of the moments
      float k[27], ks[27];
      load_f(k);
      to_central(k, ux, uy, uz);
      cp27(ks, k);
      collide_cm(ks, pm, Fx, Fy, Fz, Qx, Qy, Qz, om1, kp);
      float gux = 0.0f, guy = 0.0f, guz = 0.0f;
      from_central_vjp(lam, ks, ux, uy, uz, gux, guy, guz);
      float lk[27];
      float lpm = 0.0f, lFx = 0.0f, lFy = 0.0f, lFz = 0.0f, lQx = 0.0f, lQy = 0.0f, lQz = 0.0f, lom1 = 0.0f;
      float gom[11];
#pragma unroll
      for (int i = 0; i < 11; ++i) gom[i] = 0.0f;
      collide_vjp(k, lam, lk, pm, Fx, Fy, Fz, Qx, Qy, Qz, om1, kp, lpm, lFx, lFy, lFz, lQx, lQy, lQz, lom1, gom);
      if (UNIT) {
        to_central_vjp_unit(lk, k, ux, uy, uz, gux, guy, guz);
      } else {
        float f[27];  // populations reloaded (L2) rather than kept live
        load_f(f);
        to_central_vjp(lk, f, ux, uy, uz, gux, guy, guz);
      }
#pragma unroll
      for (int q = 0; q < 27; ++q) lam_t[q * N + n] = lk[q];
      a.u[n] = gux;
      a.u[N + n] = guy;
      a.u[2 * N + n] = guz;
      a.F[n] = lFx;
      a.F[N + n] = lFy;
      a.F[2 * N + n] = lFz;
      a.Q[n] = lQx;
      a.Q[N + n] = lQy;
      a.Q[2 * N + n] = lQz;
      a.pm[n] = lpm + lpm_wall;
      a.rho[n] = lr_wall;  // direct density adjoint: only from moving walls
      if (kp.nu > 0.0f) {
        a.om1[n] = lom1;
      } else {
        a.om1[n] = 0.0f;
        gom[1] = lom1;
      }
#pragma unroll
      for (int i = 0; i < 11; ++i) pg[i] = gom[i];
    }
  }
  const int slots[11] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11};
  block_partials(pg, slots, partial);
}

// local field adjoints at a fluid node.  First lphi(x) by the transposed
// Q stencil, lphi_a(x) = -9 sum_q w_q c_qa lQ_a(x - c_q) (a gather of a.Q,
// zero on solid nodes); then phi = (p_m - rho/3) u, omega_1(rho, p_m),
// u = (j + F/2)/rho, F = (1/3 - rho) g and p_m = (1 + mu)/3 transposed.
// Writes lrho (added to a.rho), lj (into a.u), lg = adjoint of grad mu (into
// a.phi) and the local lmu (into a.mu).
__global__ void __launch_bounds__(256) k_adj_fields(const uint8_t *__restrict__ mask, Fields d, AdjFields a,
                                                    KParams kp) {
  const Site st = site_of(kp);
  if (!st.in) return;
  const int n = st.n;
  const size_t N = (size_t)kp.N;
  if (mask && mask[n]) {
    a.rho[n] = 0.0f;
    a.mu[n] = 0.0f;
    for (int c = 0; c < 3; ++c) a.u[c * N + n] = a.phi[c * N + n] = 0.0f;
    return;
  }
  float lph[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (q == 13) continue;
    const int m = st.at(-cx_of(q), -cy_of(q), -cz_of(q));
    if (cx_of(q)) lph[0] += cx_of(q) * weight_of(q) * a.Q[m];
    if (cy_of(q)) lph[1] += cy_of(q) * weight_of(q) * a.Q[N + m];
    if (cz_of(q)) lph[2] += cz_of(q) * weight_of(q) * a.Q[2 * N + m];
  }
  const float r = d.rho[n];
  const float mup = d.mu[n];
  const float pm = pm_of(mup, kp);
  const float e = basis_c(r, mup, kp);
  const float u[3] = {d.u[n], d.u[N + n], d.u[2 * N + n]};
  const float F[3] = {d.F[n], d.F[N + n], d.F[2 * N + n]};
  const float c3 = 1.0f / 3.0f - r;
  float lrho = 0.0f, lpm = a.pm[n];
  // phi = e u
  float lu[3], le = 0.0f;
  for (int c = 0; c < 3; ++c) {
    lph[c] *= -9.0f;
    le += lph[c] * u[c];
    lu[c] = a.u[c * N + n] + e * lph[c];
  }
  lpm += le;
  lrho += -le * (1.0f / 3.0f);
  // omega_1 = 1 / (rho nu / p_m + 1/2)
  if (kp.nu > 0.0f) {
    const float om1 = 1.0f / (r * kp.nu / pm + 0.5f);
    const float lo = a.om1[n];
    lrho += lo * (-om1 * om1 * kp.nu / pm);
    lpm += lo * (om1 * om1 * r * kp.nu / (pm * pm));
  }
  // u = (j + F/2)/rho, F = (1/3 - rho) g; every input is read before the
  // first store (the adjoint arrays share no restrict guarantee)
  const float ir = 1.0f / r;
  const float lFin[3] = {a.F[n], a.F[N + n], a.F[2 * N + n]};
  const float lrho0 = a.rho[n];
  float udot = 0.0f, Fdotg = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float lF = lFin[c] + 0.5f * lu[c] * ir;
    udot += lu[c] * u[c];
    const float g = F[c] / c3;  // grad mu recovered from F (rho != 1/3 on fluid nodes)
    Fdotg += lF * g;
    a.phi[c * N + n] = c3 * lF;   // lg
    a.u[c * N + n] = lu[c] * ir;  // lj
  }
  lrho += -udot * ir - Fdotg;
  a.rho[n] = lrho0 + lrho;  // adds to any direct seed
  a.mu[n] = lpm * (1.0f / 3.0f);
}

// lmu(y) = local(y) + 3 sum_q w_q sum_a c_qa lg_a(y - c_q)
__global__ void __launch_bounds__(256) k_adj_mu(const uint8_t *__restrict__ mask, AdjFields a, KParams kp) {
  const Site st = site_of(kp);
  if (!st.in) return;
  const int n = st.n;
  const size_t N = (size_t)kp.N;
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (q == 13) continue;
    const int m = st.at(-cx_of(q), -cy_of(q), -cz_of(q));
    float v = 0.0f;
    if (cx_of(q)) v += cx_of(q) * a.phi[m];
    if (cy_of(q)) v += cy_of(q) * a.phi[N + m];
    if (cz_of(q)) v += cz_of(q) * a.phi[2 * N + m];
    s += weight_of(q) * v;
  }
  // total lmu: in place in a.mu on fluid nodes (each thread reads only its
  // own entry), into a.pm on solid nodes for the wetting gather
  if (mask && mask[n])
    a.pm[n] = 3.0f * s;
  else
    a.mu[n] = a.mu[n] + 3.0f * s;
}

// Eq. 36 transposed: mu(b) = sum_q w_q s(b+c_q) mu(b+c_q) / den(b) on solid
// boundary nodes b.  Gathered at the fluid nodes y next to walls (list fw of
// n_fw nodes): sum over the solid neighbours b = y + c_p of (w_p / den(b))
// lmu(b), with 1/den(b) stored per node and the solid neighbours read from
// y's bitmask; added to y's lmu in a.mu.
__global__ void __launch_bounds__(256) k_adj_wet_mu(const int *__restrict__ fw, int n_fw,
                                                    const uint32_t *__restrict__ nbr,
                                                    const float *__restrict__ inv_den, AdjFields a, KParams kp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_fw) return;
  const int n = fw[i];
  const Site st = site_at(n, kp);
  const uint32_t solid = nbr[n];
  float add = 0.0f;
#pragma unroll
  for (int p = 0; p < 27; ++p) {
    if (p == 13 || !((solid >> p) & 1u)) continue;
    const int b = st.at(cx_of(p), cy_of(p), cz_of(p));
    add += weight_of(p) * inv_den[b] * a.pm[b];
  }
  a.mu[n] = a.mu[n] + add;  // final lmu
}

// lambda_q(t)(n) += lrho + c_q . lj with lj = a.u(n): all 27 loads are
// issued before the first store (stores to one plane could otherwise alias
// the loads of the next and serialise them)
__device__ __forceinline__ void add_output(float *__restrict__ lam_t, int n, size_t N, float lr, const AdjFields &a) {
  const float jx = a.u[n], jy = a.u[N + n], jz = a.u[2 * N + n];
  float v[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) v[q] = lam_t[q * N + n];
#pragma unroll
  for (int q = 0; q < 27; ++q) lam_t[q * N + n] = v[q] + (lr + cx_of(q) * jx + cy_of(q) * jy + cz_of(q) * jz);
}

// mu(x) = mu0(rho(x)) - kappa 6 (sum_q w_q rho(x+c_q) - rho(x)) on fluid x:
// lrho(y) += [fluid y] (mu0'(rho) + 6 kappa) lmu(y) - 6 kappa sum_q w_q lmu(y+c_q)
// and dJ/dkappa += -sum_fluid lmu(x) 6 (sum_q w_q rho(x+c_q) - rho(x)).
// lrho goes to a.phi.  Then, per node:
//  - solid boundary node b: Eqs. 37-38 transposed, part 1: the derivative of
//    the solid density with respect to rho_ave (1, phi, or 0 when clamped)
//    and to the wetting value; dJ/d value += lrho(b) d rho_s / d value, and
//    a.F[b] = (d rho_s / d rho_ave) lrho(b) / den(b) for the fluid gather;
//  - fluid node with no solid neighbour, when lam_t is given: the output
//    lambda_q(t) += lrho + c_q . lj (nodes next to walls finish in
//    k_adj_out_wall, once every a.F[b] exists).
__global__ void __launch_bounds__(BLK) k_adj_rho(const uint8_t *__restrict__ mask, const uint32_t *__restrict__ nbr,
                                                 const float *__restrict__ inv_den, Fields d, AdjFields a,
                                                 const float *__restrict__ lmu, float *__restrict__ lam_t,
                                                 double *__restrict__ partial, KParams kp) {
  const Site st = site_of(kp);
  const int n = st.n;
  float pg[2] = {0.0f, 0.0f};  // dJ/d kappa, dJ/d wetting value of this node
  if (st.in) {
    const bool solid = mask && mask[n];  // lmu: final lmu on fluid nodes; solid entries are not read
    const uint32_t sn = mask ? nbr[n] : 0u;
    float s = 0.0f, lap = 0.0f;
    const float r = d.rho[n];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      if (q == 13) continue;
      const int m = st.at(cx_of(q), cy_of(q), cz_of(q));
      if (!((sn >> q) & 1u)) s += weight_of(q) * lmu[m];
      lap += weight_of(q) * (d.rho[m] - r);
    }
    float lr;
    if (solid) {
      lr = -6.0f * kp.kappa * s;
    } else {
      const float l0 = lmu[n];
      const float om = 1.0f - kp.b * r;
      const float dmu0 = kp.RT * (1.0f / r + kp.b / om + kp.b / (om * om)) - 2.0f * kp.a;
      lr = a.rho[n] + dmu0 * l0 - 6.0f * kp.kappa * (s + weight_of(13) * l0 - l0);
      pg[0] = -6.0f * l0 * lap;
    }
    if (solid && inv_den[n] > 0.0f) {
      // rho_ave formed exactly as the forward k_wet_rho forms it
      float num = 0.0f, den = 0.0f;
#pragma unroll
      for (int q = 0; q < 27; ++q) {
        if (q == 13 || ((sn >> q) & 1u)) continue;
        num += weight_of(q) * d.rho[st.at(cx_of(q), cy_of(q), cz_of(q))];
        den += weight_of(q);
      }
      const float ave = num / den;
      float dave = 1.0f, dval = 0.0f;
      if (kp.wet_mode != LBM_WET_NEUTRAL && ave >= kp.band_lo && ave <= kp.band_hi) {
        const float mv = kp.wet_mode == LBM_WET_PHI ? kp.wet_value * ave : ave - kp.wet_value;
        if (mv < kp.band_lo || mv > kp.band_hi) {
          dave = 0.0f;
        } else if (kp.wet_mode == LBM_WET_PHI) {
          dave = kp.wet_value;
          dval = ave;
        } else {
          dave = 1.0f;
          dval = -1.0f;
        }
      }
      pg[1] = lr * dval;
      a.F[n] = dave / den * lr;  // scaled adjoint handed to the fluid neighbours
    } else if (!solid && sn == 0u && lam_t) {
      add_output(lam_t, n, (size_t)kp.N, lr, a);
    }
    a.phi[n] = lr;  // total lrho into a.phi[0..N)
  }
  const int slots[2] = {0, 12};
  block_partials(pg, slots, partial);
}

// lambda_q(t)(x) += lrho(x) + c_q . lj(x) at the fluid nodes next to walls
// (list fw), with part 2 of Eqs. 37-38 transposed: lrho(y) += sum over solid
// neighbours b of w_q (dave(b)/den(b)) lrho(b) (stored in a.F by k_adj_rho)
__global__ void __launch_bounds__(256) k_adj_out_wall(const int *__restrict__ fw, int n_fw,
                                                      const uint32_t *__restrict__ nbr, AdjFields a,
                                                      float *__restrict__ lam_t, KParams kp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_fw) return;
  const int n = fw[i];
  const Site st = site_at(n, kp);
  const uint32_t solid = nbr[n];
  const size_t N = (size_t)kp.N;
  float lr = a.phi[n];
#pragma unroll
  for (int p = 0; p < 27; ++p) {
    if (p == 13 || !((solid >> p) & 1u)) continue;
    lr += weight_of(p) * a.F[st.at(cx_of(p), cy_of(p), cz_of(p))];
  }
  add_output(lam_t, n, N, lr, a);
}

// adds the NPAR block partials of `blocks` blocks into out[0..NPAR): one
// block per parameter, each thread a fixed strided subset, then a fixed tree
// (deterministic)
constexpr int RB = 256;
__global__ void __launch_bounds__(RB) k_adj_reduce(const double *__restrict__ partial, int blocks,
                                                   double *__restrict__ out) {
  __shared__ double sm[RB];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < blocks; b += RB) s += partial[(size_t)b * NPAR + i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] += sm[0];
}

// ---------------------------------------------------------------------------
// adjoint of the initialisation: f(0) = equilibrium (Eq. 20) about u0 at
// rho = rho0 and p_m = (1 + mu(rho0))/3
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_init(const uint8_t *__restrict__ mask, const float *__restrict__ u0,
                                                  const float *__restrict__ lam0, Fields d, AdjFields a, KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  if (mask && mask[n]) {
    a.rho[n] = 0.0f;
    a.mu[n] = 0.0f;
    return;
  }
  float lam[27], keq[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    lam[q] = lam0[q * N + n];
    keq[q] = 0.0f;
  }
  const float cs2 = 1.0f / 3.0f, pm = pm_of(d.mu[n], kp);
  float *k = keq;
  KM(0, 0, 0) = d.rho[n];
  KM(2, 0, 0) = KM(0, 2, 0) = KM(0, 0, 2) = pm;
  KM(2, 2, 0) = KM(2, 0, 2) = KM(0, 2, 2) = pm * cs2;
  KM(2, 2, 2) = pm * cs2 * cs2;
  float ux = 0.0f, uy = 0.0f, uz = 0.0f;
  if (u0) {
    ux = u0[n];
    uy = u0[N + n];
    uz = u0[2 * N + n];
  }
  float gx = 0.0f, gy = 0.0f, gz = 0.0f;  // u0 is not differentiated
  from_central_vjp(lam, keq, ux, uy, uz, gx, gy, gz);
  float *ls = lam;
  const float lpm = LS(2, 0, 0) + LS(0, 2, 0) + LS(0, 0, 2) + (LS(2, 2, 0) + LS(2, 0, 2) + LS(0, 2, 2)) * cs2 +
                    LS(2, 2, 2) * cs2 * cs2;
  a.rho[n] = LS(0, 0, 0);
  a.mu[n] = lpm * (1.0f / 3.0f);
}

// lrho (fluid nodes, with the wetting part gathered from solid neighbours)
// into the caller's gradient array
__global__ void __launch_bounds__(256) k_adj_grad_rho0(const uint8_t *__restrict__ mask, int wet, AdjFields a,
                                                       float *__restrict__ g, KParams kp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  if (mask && mask[n]) {
    g[n] = 0.0f;
    return;
  }
  float lr = a.phi[n];
  if (wet) {
    Node p = decode(n, kp.nx, kp.ny);
    for (int q = 0; q < 27; ++q) {
      if (q == 13) continue;
      const int b = neighbour(p, -cx_of(q), -cy_of(q), -cz_of(q), kp);
      if (mask[b]) lr += weight_of(q) * a.F[b];
    }
  }
  g[n] = lr;
}

// ---------------------------------------------------------------------------
// objectives of the current state and their seeds dJ/df
// ---------------------------------------------------------------------------
// per-block FP64 partials of the sums an objective needs (into slots 0..2)
__global__ void __launch_bounds__(BLK) k_obj_sums(int kind, int wall_z, const uint8_t *__restrict__ mask, Fields d,
                                                  double *__restrict__ partial, KParams kp, float rho_v) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double par[NPAR];
#pragma unroll
  for (int i = 0; i < NPAR; ++i) par[i] = 0.0;
  if (n < kp.N && !(mask && mask[n])) {
    const size_t N = (size_t)kp.N;
    const float r = d.rho[n];
    Node p = decode(n, kp.nx, kp.ny);
    if (kind == LBM_OBJ_ENERGY) {
      const float ux = d.u[n], uy = d.u[N + n], uz = d.u[2 * N + n];
      par[0] = 0.5 * (double)r * ((double)ux * ux + (double)uy * uy + (double)uz * uz);
    } else if (kind == LBM_OBJ_CENTROID_X) {
      par[0] = (double)p.x * (r - rho_v);
      par[1] = (double)(r - rho_v);
    } else if (p.z == wall_z + 1) {
      par[0] = (double)(r - rho_v);
    }
  }
  block_partials_f64(par, partial);
}

__global__ void __launch_bounds__(RB) k_obj_finish(int kind, const double *__restrict__ partial, int blocks,
                                                   double *__restrict__ out, float rho_l, float rho_v) {
  __shared__ double sm[2][RB];
  double a0 = 0.0, a1 = 0.0;
  for (int b = threadIdx.x; b < blocks; b += RB) {
    a0 += partial[(size_t)b * NPAR];
    a1 += partial[(size_t)b * NPAR + 1];
  }
  sm[0][threadIdx.x] = a0;
  sm[1][threadIdx.x] = a1;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + w];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double s0 = sm[0][0], s1 = sm[1][0];
  if (kind == LBM_OBJ_ENERGY) {
    out[0] = s0;
  } else if (kind == LBM_OBJ_CENTROID_X) {
    out[0] = s0 / s1;
    out[1] = s1;
  } else {
    const double area = s0 / ((double)rho_l - rho_v);
    out[0] = sqrt(area / 3.14159265358979323846);
  }
}

// seeds of the field adjoints: energy -> lu = rho u, lrho = |u|^2/2 (added
// after k_adj_fields); centroid -> lrho = (x - J)/W; contact radius ->
// lrho = 1/(2 pi J (rho_l - rho_v)) on the first fluid layer
__global__ void __launch_bounds__(256) k_obj_seed(int kind, int wall_z, const uint8_t *__restrict__ mask, Fields d,
                                                  AdjFields a, const double *__restrict__ Jv, KParams kp,
                                                  float rho_l, float rho_v) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kp.N) return;
  const size_t N = (size_t)kp.N;
  for (int c = 0; c < 3; ++c) a.u[c * N + n] = a.F[c * N + n] = a.phi[c * N + n] = a.Q[c * N + n] = 0.0f;
  a.pm[n] = 0.0f;
  a.om1[n] = 0.0f;
  a.rho[n] = 0.0f;
  if (mask && mask[n]) return;
  Node p = decode(n, kp.nx, kp.ny);
  if (kind == LBM_OBJ_ENERGY) {
    const float r = d.rho[n];
    const float ux = d.u[n], uy = d.u[N + n], uz = d.u[2 * N + n];
    a.u[n] = r * ux;
    a.u[N + n] = r * uy;
    a.u[2 * N + n] = r * uz;
    a.rho[n] = 0.5f * (ux * ux + uy * uy + uz * uz);
  } else if (kind == LBM_OBJ_CENTROID_X) {
    a.rho[n] = (float)(((double)p.x - Jv[0]) / Jv[1]);
  } else if (p.z == wall_z + 1) {
    a.rho[n] = (float)(1.0 / (2.0 * 3.14159265358979323846 * Jv[0] * ((double)rho_l - rho_v)));
  }
}

// Parameter partials: region 0 (collision) and region 1 (mu -> rho, with the
// wetting transpose) lie back to back in ctx->adj_partial.  Kernels add to
// them; launch_adjoint_partials_reduce sums both regions into the gradient.
struct Regions {
  double *collide, *rho;
  int gb;
};

// 3-D launch shape of the node-parallel kernels: 32 x by threads per block
dim3 grid3(const lbm_ctx *ctx, int by) { return dim3((ctx->nx + 31) / 32, (ctx->ny + by - 1) / by, ctx->nz); }

Regions regions(lbm_ctx *ctx) {
  Regions r;
  r.gb = (int)adj_blocks(ctx->nx, ctx->ny, ctx->nz);
  r.collide = ctx->adj_partial;
  r.rho = ctx->adj_partial + (size_t)r.gb * NPAR;
  return r;
}

// mu -> rho transpose with the wetting transpose and, when lam_t is given,
// the output lambda(t) (bulk nodes in k_adj_rho, nodes next to walls after)
void adj_tail(lbm_ctx *ctx, const float *lmu, const Regions &R, const Fields &d, float *lam_t) {
  const KParams &kp = ctx->kp;
  cudaStream_t s = ctx->stream;
  k_adj_rho<<<grid3(ctx, ADJ_BY), dim3(32, ADJ_BY), 0, s>>>(ctx->mask, ctx->nbr, ctx->inv_den, d, ctx->adj, lmu,
                                                            lam_t, R.rho, kp);
  ctx->launches++;
  if (lam_t && ctx->n_fw) {
    k_adj_out_wall<<<(ctx->n_fw + 255) / 256, 256, 0, s>>>(ctx->bnd + ctx->n_bnd, ctx->n_fw, ctx->nbr, ctx->adj,
                                                          lam_t, kp);
    ctx->launches++;
  }
}

// lmu: gather of lg (+ the local part), and Eq. 36 transposed with walls
const float *adj_mu(lbm_ctx *ctx) {
  const KParams &kp = ctx->kp;
  k_adj_mu<<<grid3(ctx, 8), dim3(32, 8), 0, ctx->stream>>>(ctx->mask, ctx->adj, kp);
  ctx->launches++;
  if (ctx->n_fw) {
    k_adj_wet_mu<<<(ctx->n_fw + 255) / 256, 256, 0, ctx->stream>>>(ctx->bnd + ctx->n_bnd, ctx->n_fw, ctx->nbr,
                                                                  ctx->inv_den, ctx->adj, kp);
    ctx->launches++;
  }
  return ctx->adj.mu;
}

}  // namespace

void launch_adjoint_partials_zero(lbm_ctx *ctx) {
  const Regions R = regions(ctx);
  cudaMemsetAsync(ctx->adj_partial, 0, (size_t)2 * R.gb * NPAR * sizeof(double), ctx->stream);
}

void launch_adjoint_partials_reduce(lbm_ctx *ctx, double *grad) {
  const Regions R = regions(ctx);
  k_adj_reduce<<<NPAR, RB, 0, ctx->stream>>>(ctx->adj_partial, 2 * R.gb, grad);
  ctx->launches++;
}

void launch_adjoint_init(lbm_ctx *ctx, const float *u0, const float *lam0, double *grad, float *grad_rho0) {
  const KParams &kp = ctx->kp;
  cudaStream_t s = ctx->stream;
  const int g = (kp.N + 255) / 256;
  const Regions R = regions(ctx);
  // fields of the initial density are in ctx->fld (lbm_set_state ran before)
  k_adj_init<<<g, 256, 0, s>>>(ctx->mask, u0, lam0, ctx->fld, ctx->adj, kp);
  ctx->launches++;
  launch_adjoint_partials_zero(ctx);
  adj_tail(ctx, ctx->adj.mu, R, ctx->fld, nullptr);
  launch_adjoint_partials_reduce(ctx, grad);
  k_adj_grad_rho0<<<g, 256, 0, s>>>(ctx->mask, ctx->n_bnd ? 1 : 0, ctx->adj, grad_rho0, kp);
  ctx->launches++;
}

void launch_objective(lbm_ctx *ctx, int kind, int wall_z, double *J, float *lam, double *grad) {
  const KParams &kp = ctx->kp;
  cudaStream_t s = ctx->stream;
  const int g = (kp.N + 255) / 256;
  const Regions R = regions(ctx);
  const float rl = (float)ctx->params.rho_l, rv = (float)ctx->params.rho_v;
  launch_fields_full(ctx);
  launch_adjoint_partials_zero(ctx);
  k_obj_sums<<<R.gb, BLK, 0, s>>>(kind, wall_z, ctx->mask, ctx->fld, ctx->adj_partial, kp, rv);
  k_obj_finish<<<1, RB, 0, s>>>(kind, ctx->adj_partial, R.gb, J, rl, rv);
  k_obj_seed<<<g, 256, 0, s>>>(kind, wall_z, ctx->mask, ctx->fld, ctx->adj, J, kp, rl, rv);
  ctx->launches += 3;
  cudaMemsetAsync(lam, 0, 27 * (size_t)kp.N * sizeof(float), s);
  k_adj_fields<<<grid3(ctx, 8), dim3(32, 8), 0, s>>>(ctx->mask, ctx->fld, ctx->adj, kp);
  ctx->launches++;
  const float *lmu = adj_mu(ctx);
  // the objective's direct dependence on kappa and on the wetting value
  launch_adjoint_partials_zero(ctx);
  adj_tail(ctx, lmu, R, ctx->fld, lam);
  if (grad) launch_adjoint_partials_reduce(ctx, grad);
}

void launch_adjoint_step(lbm_ctx *ctx, const void *f_state, const float *lam_next, float *lam_t,
                         const float *captured, const float *sb_state) {
  const KParams &kp = ctx->kp;
  cudaStream_t s = ctx->stream;
  const Regions R = regions(ctx);
  const dim3 g4 = grid3(ctx, ADJ_BY), b4(32, ADJ_BY), g8 = grid3(ctx, 8), b8(32, 8);
  Fields d = ctx->fld;
  const float *sb = ctx->fld.sb;
  if (captured) {  // fields of f(t) from the recompute: rho, mu', u, F, Q
    const size_t N = (size_t)kp.N;
    d.rho = const_cast<float *>(captured);
    d.mu = d.rho + N;
    d.u = d.rho + 2 * N;
    d.F = d.rho + 5 * N;
    d.Q = d.rho + 8 * N;
    sb = sb_state;
  } else {
    launch_fields_full(ctx);  // forward recompute of the fields of f(t) (the state is in ctx->f[cur])
  }
  const float *wu = ctx->mask ? ctx->wall_u : nullptr;
  const bool unit = adj_unit_rates(kp);
  if (ctx->storage == LBM_F16) {
    const __half *fs = (const __half *)f_state;
    if (unit)
      k_adj_collide<__half, true><<<g4, b4, 0, s>>>(fs, sb, ctx->mask, ctx->nbr, lam_next, lam_t, d, ctx->adj, wu,
                                                    R.collide, kp);
    else
      k_adj_collide<__half, false><<<g4, b4, 0, s>>>(fs, sb, ctx->mask, ctx->nbr, lam_next, lam_t, d, ctx->adj, wu,
                                                     R.collide, kp);
  } else {
    const float *fs = (const float *)f_state;
    if (unit)
      k_adj_collide<float, true><<<g4, b4, 0, s>>>(fs, sb, ctx->mask, ctx->nbr, lam_next, lam_t, d, ctx->adj, wu,
                                                   R.collide, kp);
    else
      k_adj_collide<float, false><<<g4, b4, 0, s>>>(fs, sb, ctx->mask, ctx->nbr, lam_next, lam_t, d, ctx->adj, wu,
                                                    R.collide, kp);
  }
  k_adj_fields<<<g8, b8, 0, s>>>(ctx->mask, d, ctx->adj, kp);
  ctx->launches += 2;
  const float *lmu = adj_mu(ctx);
  adj_tail(ctx, lmu, R, d, lam_t);
}

}  // namespace lbm
