// Device-side D3Q27 lattice helpers: weights, periodic neighbour indexing,
// storage conversion, the central-moment transform factorised into three
// 1-D passes, and the central-moment collision of Sec. II B (Eqs. 21-26).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "lbm_internal.h"

namespace lbm {

// Population q has velocity (q%3 - 1, (q/3)%3 - 1, q/9 - 1); rest is q = 13.
__host__ __device__ constexpr int cx_of(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int cy_of(int q) { return (q / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int q) { return q / 9 - 1; }

// Lattice weights by |c|^2 = 0, 1, 2, 3 (Eq. 17).
__host__ __device__ constexpr float weight_of(int q) {
  return (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 0   ? 8.0f / 27.0f
         : (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 1 ? 2.0f / 27.0f
         : (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 2 ? 1.0f / 54.0f
                                                                                 : 1.0f / 216.0f;
}

// E_i of Eq. 16 at u = 0 by speed class: -19/9, 2/9, 1/18, 1/72.
__host__ __device__ constexpr float iso_rest_of(int q) {
  return (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 0   ? -19.0f / 9.0f
         : (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 1 ? 2.0f / 9.0f
         : (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 2 ? 1.0f / 18.0f
                                                                                 : 1.0f / 72.0f;
}

// Storage shift of population q.  LBM_SHIFT_CONST: w_q rho_0.
// LBM_SHIFT_REST: the rest equilibrium w_q rho_b + c_b E_q of a basis
// (rho_b, c_b = p_m - rho/3); basis_c gives c_b from rho and mu, and every
// writer and reader of a population computes it with this same function.
__device__ __forceinline__ float basis_c(float rho, float mup, const KParams &kp) {
  return fmaf(mup - rho, 1.0f / 3.0f, kp.pm_ref);
}
__device__ __forceinline__ float shift_rest(int q, float rb, float cb) {
  return fmaf(weight_of(q), rb, cb * iso_rest_of(q));
}

// Periodic index for v in [-n, 2n) (one period of wrap).
__device__ __forceinline__ int wrap(int v, int n) {
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// Periodic index for any v (tiles and halos of domains smaller than a tile
// reach more than one period away).
__device__ __forceinline__ int pmod(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

struct Node {
  int x, y, z;
};

__device__ __forceinline__ Node decode(int n, int nx, int ny) {
  Node p;
  p.x = n % nx;
  int t = n / nx;
  p.y = t % ny;
  p.z = t / ny;
  return p;
}

__device__ __forceinline__ int neighbour(const Node &p, int dx, int dy, int dz, const KParams &kp) {
  return wrap(p.x + dx, kp.nx) + kp.nx * (wrap(p.y + dy, kp.ny) + kp.ny * wrap(p.z + dz, kp.nz));
}

// ---- storage type conversion ----------------------------------------------
template <typename T> __device__ __forceinline__ float load_pop(const T *p);
template <> __device__ __forceinline__ float load_pop<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_pop<__half>(const __half *p) {
  return __half2float(__ldg(p));
}
template <typename T> __device__ __forceinline__ void store_pop(T *p, float v);
template <> __device__ __forceinline__ void store_pop<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void store_pop<__half>(__half *p, float v) {
  *p = __float2half_rn(v);
}

// ---- moments of one node (Eq. 11) ----------------------------------------
// Sums of a node's 27 stored populations v[q]: s = sum_q v_q and the
// momentum sums per axis as (+1 class) - (-1 class), grouped to keep FP32
// rounding small.  Every kernel that forms moments (the moments passes, the
// fused step's read-back of the state it wrote, the edge pass) uses this one
// order, so the moments of a state are the same bits whichever path made
// them.
__device__ __forceinline__ void node_sums(const float (&v)[27], float &s, float &sx, float &sy, float &sz) {
  s = 0.0f;
  sx = 0.0f;
  sy = 0.0f;
  sz = 0.0f;
#pragma unroll
  for (int q = 0; q < 27; ++q) s += v[q];
#pragma unroll
  for (int q = 0; q < 27; q += 3) sx += v[q + 2] - v[q];
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) sy += v[a + 6 + 9 * g] - v[a + 9 * g];
#pragma unroll
  for (int p = 0; p < 9; ++p) sz += v[p + 18] - v[p];
}

// ---- central-moment transform (Eq. 19) ----------------------------------
// One axis: values (a, b, c) of the velocities -1, 0, +1 become the central
// moments of order 0, 1, 2 about u.  With s = a + c, d = c - a:
//   M0 = s + b,  M1 = d - u M0,  M2 = s - 2 u d + u^2 M0.
__device__ __forceinline__ void cm_axis(float &a, float &b, float &c, float u) {
  float s = a + c, d = c - a;
  float m0 = s + b;
  float m1 = fmaf(-u, m0, d);
  float m2 = fmaf(u * u, m0, fmaf(-2.0f * u, d, s));
  a = m0;
  b = m1;
  c = m2;
}

// Inverse of cm_axis: d = M1 + u M0, s = M2 + 2 u d - u^2 M0, then
// a = (s - d)/2, b = M0 - s, c = (s + d)/2.
__device__ __forceinline__ void cm_axis_inv(float &a, float &b, float &c, float u) {
  float m0 = a, m1 = b, m2 = c;
  float d = fmaf(u, m0, m1);
  float s = fmaf(-u * u, m0, fmaf(2.0f * u, d, m2));
  a = 0.5f * (s - d);
  b = m0 - s;
  c = 0.5f * (s + d);
}

// cm_axis_inv for inputs whose first- and second-order entries are halved,
// (M0, M1/2, M2/2).  With delta = d/2 and sigma = s/2:
//   delta = M1/2 + (u/2) M0,  sigma = M2/2 + 2 u delta - (u^2/2) M0,
//   a = sigma - delta,  b = M0 - 2 sigma,  c = sigma + delta,
// six operations instead of eight.  Halving is exact in binary floating
// point, so every intermediate is exactly half of its cm_axis_inv
// counterpart and the outputs are the same values.
__device__ __forceinline__ void cm_axis_inv_h(float &a, float &b, float &c, float u) {
  const float m0 = a, h1 = b, h2 = c;
  const float dl = fmaf(0.5f * u, m0, h1);
  const float sg = fmaf(-0.5f * (u * u), m0, fmaf(2.0f * u, dl, h2));
  a = sg - dl;
  b = fmaf(-2.0f, sg, m0);
  c = sg + dl;
}

// f[q] (q = (cx+1) + 3(cy+1) + 9(cz+1)) -> k[a + 3b + 9c] in place: the
// triple sum over (cz, cy, cx) of Eq. 19 done one axis at a time.
__device__ __forceinline__ void to_central(float f[27], float ux, float uy, float uz) {
#pragma unroll
  for (int p = 0; p < 9; ++p) cm_axis(f[p], f[p + 9], f[p + 18], uz);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) cm_axis(f[a + 9 * g], f[a + 3 + 9 * g], f[a + 6 + 9 * g], uy);
#pragma unroll
  for (int q = 0; q < 27; q += 3) cm_axis(f[q], f[q + 1], f[q + 2], ux);
}

// to_central restricted to the moments the collision reads when every rate
// but omega_1 is 1 (collide_cm_unit): k000, the three mixed and the three
// diagonal second-order moments.  The z pass is complete; the y and x
// passes form only what those seven need, with the operations of cm_axis,
// so the seven values are those of to_central.  The other entries of k are
// left unspecified.
__device__ __forceinline__ void to_central_unit(float f[27], float ux, float uy, float uz) {
#pragma unroll
  for (int p = 0; p < 9; ++p) cm_axis(f[p], f[p + 9], f[p + 18], uz);
  // y pass: z order 0 complete, z order 1 up to y order 1, z order 2 order 0
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cm_axis(f[a], f[a + 3], f[a + 6], uy);
    {
      const float s = f[a + 9] + f[a + 15], d = f[a + 15] - f[a + 9];
      const float m0 = s + f[a + 12];
      f[a + 9] = m0;
      f[a + 12] = fmaf(-uy, m0, d);
    }
    f[a + 18] = (f[a + 18] + f[a + 24]) + f[a + 21];
  }
  // x pass: k000 and k200 (group 0), k110, k101 (first order of groups 3
  // and 9), k020, k011, k002 (zeroth order of groups 6, 12, 18)
  {
    const float s = f[0] + f[2], d = f[2] - f[0];
    const float m0 = s + f[1];
    f[0] = m0;
    f[2] = fmaf(ux * ux, m0, fmaf(-2.0f * ux, d, s));
  }
#pragma unroll
  for (int q = 3; q <= 9; q += 6) {
    const float s = f[q] + f[q + 2], d = f[q + 2] - f[q];
    f[q + 1] = fmaf(-ux, s + f[q + 1], d);
  }
#pragma unroll
  for (int q = 6; q <= 18; q += 6) f[q] = (f[q] + f[q + 2]) + f[q + 1];
}

__device__ __forceinline__ void from_central(float k[27], float ux, float uy, float uz) {
#pragma unroll
  for (int q = 0; q < 27; q += 3) cm_axis_inv(k[q], k[q + 1], k[q + 2], ux);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) cm_axis_inv(k[a + 9 * g], k[a + 3 + 9 * g], k[a + 6 + 9 * g], uy);
#pragma unroll
  for (int p = 0; p < 9; ++p) cm_axis_inv(k[p], k[p + 9], k[p + 18], uz);
}

// from_central for moments stored with k[a + 3b + 9c] scaled by
// 2^-(number of nonzero a, b, c): every pass then sees halved first- and
// second-order entries (cm_axis_inv_h) and the populations come out
// unscaled, equal to those of from_central on the unscaled moments.
__device__ __forceinline__ void from_central_h(float k[27], float ux, float uy, float uz) {
#pragma unroll
  for (int q = 0; q < 27; q += 3) cm_axis_inv_h(k[q], k[q + 1], k[q + 2], ux);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) cm_axis_inv_h(k[a + 9 * g], k[a + 3 + 9 * g], k[a + 6 + 9 * g], uy);
#pragma unroll
  for (int p = 0; p < 9; ++p) cm_axis_inv_h(k[p], k[p + 9], k[p + 18], uz);
}

#define KM(a, b, c) k[(a) + 3 * (b) + 9 * (c)]

// Post-collision central moments, Eqs. 21-26, in place.  k000 is unchanged.
// om1 is omega_1 of this node; the other rates enter through the factors
// 1 - omega_i, 1 - omega_i/2 and the forcing / equilibrium coefficients
// precomputed in kp.  HALVED: every output except k000 is written scaled by
// 2^-(number of nonzero indices), the input scaling of from_central_h; each
// output's last multiplication takes the power of two (exact), so the
// values are those of the unscaled form divided by it.
template <bool HALVED = false>
__device__ __forceinline__ void collide_cm(float k[27], float pm, float Fx, float Fy, float Fz,
                                           float Qx, float Qy, float Qz, float om1,
                                           const KParams &kp) {
  constexpr float s1 = HALVED ? 0.5f : 1.0f, s2 = HALVED ? 0.25f : 1.0f, s3 = HALVED ? 0.125f : 1.0f;
  // per-output factors: the scaled copies in kp.hs where a factor is a parameter
  const float f1c = HALVED ? kp.hs[0] : kp.om_c[0], f1h = HALVED ? kp.hs[1] : kp.om_h[0];
  const float f5 = HALVED ? kp.hs[2] : kp.om_c[5], f8 = HALVED ? kp.hs[3] : kp.om_c[8];
  const float f9 = HALVED ? kp.hs[4] : kp.om_c[9], f9g = HALVED ? kp.hs[5] : kp.g5;
  const float f10 = HALVED ? kp.hs[6] : kp.om_c[10], f10e = HALVED ? kp.hs[7] : kp.o10e;
  const float c1 = 1.0f - om1, h1 = 1.0f - 0.5f * om1;
  // c1 for the mixed second-order moments, with their scale (exact)
  const float c1m = HALVED ? fmaf(-0.25f, om1, 0.25f) : c1;
  // first order (Eq. 21)
  KM(1, 0, 0) = f1c * KM(1, 0, 0) + f1h * Fx;
  KM(0, 1, 0) = f1c * KM(0, 1, 0) + f1h * Fy;
  KM(0, 0, 1) = f1c * KM(0, 0, 1) + f1h * Fz;
  // second order (Eq. 22)
  KM(1, 1, 0) *= c1m;
  KM(0, 1, 1) *= c1m;
  KM(1, 0, 1) *= c1m;
  {
    float A = c1 * (KM(2, 0, 0) - KM(0, 2, 0)) + h1 * (Qx - Qy);
    float B = c1 * (KM(2, 0, 0) - KM(0, 0, 2)) + h1 * (Qx - Qz);
    float S = kp.om_c[2] * (KM(2, 0, 0) + KM(0, 2, 0) + KM(0, 0, 2)) + 3.0f * kp.om[2] * pm +
              kp.om_h[2] * (Qx + Qy + Qz);
    KM(2, 0, 0) = (S + A + B) * (s1 / 3.0f);
    KM(0, 2, 0) = (S - 2.0f * A + B) * (s1 / 3.0f);
    KM(0, 0, 2) = (S + A - 2.0f * B) * (s1 / 3.0f);
  }
  // third order (Eq. 23)
  {
    float P, D;
    P = kp.om_c[3] * (KM(1, 2, 0) + KM(1, 0, 2)) + kp.g3 * Fx;
    D = kp.om_c[4] * (KM(1, 2, 0) - KM(1, 0, 2));
    KM(1, 2, 0) = (0.5f * s2) * (P + D);
    KM(1, 0, 2) = (0.5f * s2) * (P - D);
    P = kp.om_c[3] * (KM(2, 1, 0) + KM(0, 1, 2)) + kp.g3 * Fy;
    D = kp.om_c[4] * (KM(2, 1, 0) - KM(0, 1, 2));
    KM(2, 1, 0) = (0.5f * s2) * (P + D);
    KM(0, 1, 2) = (0.5f * s2) * (P - D);
    P = kp.om_c[3] * (KM(2, 0, 1) + KM(0, 2, 1)) + kp.g3 * Fz;
    D = kp.om_c[4] * (KM(2, 0, 1) - KM(0, 2, 1));
    KM(2, 0, 1) = (0.5f * s2) * (P + D);
    KM(0, 2, 1) = (0.5f * s2) * (P - D);
    KM(1, 1, 1) *= f5;
  }
  // fourth order (Eq. 24) with the approximate correction of Eq. 28
  {
    float Q220 = 0.0f, Q202 = 0.0f, Q022 = 0.0f;
    if (kp.q4) {
      Q220 = (Qx + Qy) * (1.0f / 3.0f);
      Q202 = (Qx + Qz) * (1.0f / 3.0f);
      Q022 = (Qy + Qz) * (1.0f / 3.0f);
    }
    float a = KM(2, 2, 0), b = KM(2, 0, 2), c = KM(0, 2, 2);
    float D1 = kp.om_c[6] * (a - 2.0f * b + c) + kp.om_h[6] * (Q220 - 2.0f * Q202 + Q022);
    float D2 = kp.om_c[6] * (a + b - 2.0f * c) + kp.om_h[6] * (Q220 + Q202 - 2.0f * Q022);
    float T = kp.om_c[7] * (a + b + c) + kp.om[7] * pm + kp.om_h[7] * (Q220 + Q202 + Q022);
    KM(2, 2, 0) = (T + D1 + D2) * (s2 / 3.0f);
    KM(2, 0, 2) = (T - D1) * (s2 / 3.0f);
    KM(0, 2, 2) = (T - D2) * (s2 / 3.0f);
    KM(2, 1, 1) *= f8;
    KM(1, 2, 1) *= f8;
    KM(1, 1, 2) *= f8;
  }
  // fifth order (Eq. 25)
  KM(1, 2, 2) = f9 * KM(1, 2, 2) + f9g * Fx;
  KM(2, 1, 2) = f9 * KM(2, 1, 2) + f9g * Fy;
  KM(2, 2, 1) = f9 * KM(2, 2, 1) + f9g * Fz;
  // sixth order (Eq. 26)
  KM(2, 2, 2) = f10 * KM(2, 2, 2) + f10e * pm;
}

// collide_cm when omega_0 and omega_2 .. omega_10 are 1 (the paper's runs
// relax only the shear moments at another rate): each term 1 - omega_i of
// Eqs. 21-26 vanishes, so a post-collision moment is its equilibrium and
// forcing part alone, except the mixed and deviatoric second-order moments
// relaxed by omega_1.  Reads k000 and the six second-order moments of
// to_central_unit; writes all 26 others, scaled as collide_cm<HALVED>.
template <bool HALVED>
__device__ __forceinline__ void collide_cm_unit(float k[27], float pm, float Fx, float Fy, float Fz,
                                                float Qx, float Qy, float Qz, float om1, const KParams &kp) {
  constexpr float s1 = HALVED ? 0.5f : 1.0f, s2 = HALVED ? 0.25f : 1.0f, s3 = HALVED ? 0.125f : 1.0f;
  const float c1 = 1.0f - om1, h1 = 1.0f - 0.5f * om1;
  const float c1m = HALVED ? fmaf(-0.25f, om1, 0.25f) : c1;
  // first order: (1 - omega_0/2) F
  KM(1, 0, 0) = (0.5f * s1) * Fx;
  KM(0, 1, 0) = (0.5f * s1) * Fy;
  KM(0, 0, 1) = (0.5f * s1) * Fz;
  // second order
  KM(1, 1, 0) *= c1m;
  KM(0, 1, 1) *= c1m;
  KM(1, 0, 1) *= c1m;
  {
    const float A = c1 * (KM(2, 0, 0) - KM(0, 2, 0)) + h1 * (Qx - Qy);
    const float B = c1 * (KM(2, 0, 0) - KM(0, 0, 2)) + h1 * (Qx - Qz);
    const float S = 3.0f * pm + 0.5f * (Qx + Qy + Qz);
    KM(2, 0, 0) = (S + A + B) * (s1 / 3.0f);
    KM(0, 2, 0) = (S - 2.0f * A + B) * (s1 / 3.0f);
    KM(0, 0, 2) = (S + A - 2.0f * B) * (s1 / 3.0f);
  }
  // third order: the forcing part g3 F of the symmetric combination P
  {
    const float gx = (0.5f * s2) * kp.g3 * Fx, gy = (0.5f * s2) * kp.g3 * Fy, gz = (0.5f * s2) * kp.g3 * Fz;
    KM(1, 2, 0) = gx;
    KM(1, 0, 2) = gx;
    KM(2, 1, 0) = gy;
    KM(0, 1, 2) = gy;
    KM(2, 0, 1) = gz;
    KM(0, 2, 1) = gz;
    KM(1, 1, 1) = 0.0f;
  }
  // fourth order: pm and the corrections of Eq. 28
  {
    float Q220 = 0.0f, Q202 = 0.0f, Q022 = 0.0f;
    if (kp.q4) {
      Q220 = (Qx + Qy) * (1.0f / 3.0f);
      Q202 = (Qx + Qz) * (1.0f / 3.0f);
      Q022 = (Qy + Qz) * (1.0f / 3.0f);
    }
    const float D1 = 0.5f * (Q220 - 2.0f * Q202 + Q022);
    const float D2 = 0.5f * (Q220 + Q202 - 2.0f * Q022);
    const float T = pm + 0.5f * (Q220 + Q202 + Q022);
    KM(2, 2, 0) = (T + D1 + D2) * (s2 / 3.0f);
    KM(2, 0, 2) = (T - D1) * (s2 / 3.0f);
    KM(0, 2, 2) = (T - D2) * (s2 / 3.0f);
    KM(2, 1, 1) = 0.0f;
    KM(1, 2, 1) = 0.0f;
    KM(1, 1, 2) = 0.0f;
  }
  // fifth and sixth order
  KM(1, 2, 2) = (s3 * kp.g5) * Fx;
  KM(2, 1, 2) = (s3 * kp.g5) * Fy;
  KM(2, 2, 1) = (s3 * kp.g5) * Fz;
  KM(2, 2, 2) = (s3 * kp.o10e) * pm;
}

// Bulk chemical potential of the van der Waals EOS (bulk part of Eq. 32),
// returned as mu0(rho) - mu_ref.  With d = rho - rho_r about the reference
// density of the node's phase, A = d/rho_r and C = b d/(1 - b rho_r), the
// identity
//   mu0(rho) = mu0(rho_r) + RT [ln((1 + A)/(1 - C)) + C/(1 - b rho)] - 2 a d,
//   ln((1 + A)/(1 - C)) = log1p((A + C)/(1 - C)),
// holds exactly; every term is O(d), so FP32 keeps its relative precision
// where the direct form cancels (liquid: RT(...) ~ 2.5 against 2 a rho ~ 2.3).
// Both quotients share 1/(1 - C): 1 - b rho = (1 - b rho_r)(1 - C), so
// C/(1 - b rho) = d b/(1 - b rho_r)^2 / (1 - C); one correctly rounded
// reciprocal replaces the two divisions.
__device__ __forceinline__ float mu0_vdw(float r, const KParams &kp) {
  const bool liq = r > kp.rho_split;
  const float d = r - (liq ? kp.ref_rho[1] : kp.ref_rho[0]);
  const float A = d * (liq ? kp.ref_inv[1] : kp.ref_inv[0]);
  const float Cc = d * (liq ? kp.ref_bomb[1] : kp.ref_bomb[0]);
  const float rc = __frcp_rn(1.0f - Cc);
  const float t = log1pf((A + Cc) * rc) + d * (liq ? kp.ref_bomb2[1] : kp.ref_bomb2[0]) * rc;
  return (liq ? kp.ref_dmu[1] : kp.ref_dmu[0]) + kp.RT * t - 2.0f * kp.a * d;
}

// Moving halfway wall: f^eq_q - f^eq_-q of the generalized equilibrium
// (Eq. 13) at the wall velocity U to first order, at the fluid node's rho and
// p_m: 2 w_q (c_q . U) / c_s^2 * A with A = p_m / c_s^2 for edge and corner
// velocities and A = p_m / c_s^2 + (9/4)(rho - p_m / c_s^2) for faces.  Sec.
// III B uses moving walls without giving the term; for p_m = rho c_s^2 it is
// the usual 2 w_q rho (c_q . U) / c_s^2.
__device__ __forceinline__ float wall_coef_rho(int q) {  // dA/drho
  return (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 1 ? 2.25f : 0.0f;
}
__device__ __forceinline__ float wall_coef_pm(int q) {  // dA/dp_m
  return (cx_of(q) * cx_of(q) + cy_of(q) * cy_of(q) + cz_of(q) * cz_of(q)) == 1 ? 3.0f - 6.75f : 3.0f;
}
__device__ __forceinline__ float wall_odd(int q, float rho, float pm, float ux, float uy, float uz) {
  const float cu = cx_of(q) * ux + cy_of(q) * uy + cz_of(q) * uz;
  return 6.0f * weight_of(q) * cu * (wall_coef_pm(q) * pm + wall_coef_rho(q) * rho);
}

// p_m = (1 + mu)/3 from mu' = mu - mu_ref.
__device__ __forceinline__ float pm_of(float mup, const KParams &kp) {
  return fmaf(mup, 1.0f / 3.0f, kp.pm_ref);
}

}  // namespace lbm
