// Per-cell collision operators and equilibria (device code).
//
// Every function works on the shifted values g_i held in registers:
//   D3Q19 (incompressible, Section 2): g_i = f_i, the fluctuation with sum delta rho;
//   D3Q27 (compressible, Section 2):   g_i = f_i - w_i, with sum rho - 1.
// Keeping the weights out of the registers keeps float32 arithmetic accurate
// relative to the small non-equilibrium parts.
#pragma once
#include <cuda_fp16.h>

#include "lattice.cuh"

namespace lbm {

// ------------------------------------------------------------------ storage
// Storage types: double / float hold g_i; __half holds g_i / w_i.
template <class S>
struct Store;
template <>
struct Store<double> {
  using T = double;
  template <int Q, int i>
  __device__ static __forceinline__ T get(const double* p) { return *p; }
  template <int Q, int i>
  __device__ static __forceinline__ void put(double* p, T v) { *p = v; }
};
template <>
struct Store<float> {
  using T = float;
  template <int Q, int i>
  __device__ static __forceinline__ T get(const float* p) { return __ldg(p); }
  template <int Q, int i>
  __device__ static __forceinline__ void put(float* p, T v) { *p = v; }
};
template <>
struct Store<__half> {
  using T = float;
  template <int Q, int i>
  __device__ static __forceinline__ T get(const __half* p) {
    return __half2float(__ldg(p)) * float(Lattice<Q>::w(i));
  }
  template <int Q, int i>
  __device__ static __forceinline__ void put(__half* p, T v) {
    *p = __float2half_rn(v * float(1.0 / Lattice<Q>::w(i)));
  }
};

// runtime-index variants for the small interface / utility kernels
template <class S, int Q>
__device__ __forceinline__ typename Store<S>::T load_rt(const S* p, int i);
template <class S, int Q>
__device__ __forceinline__ void store_rt(S* p, int i, typename Store<S>::T v);

template <int Q>
__device__ __forceinline__ double weight_rt(int i) {
  double w = 0.0;
  static_for<Q>([&](auto c) {
    if (i == c) w = Lattice<Q>::w(c);
  });
  return w;
}

template <>
__device__ __forceinline__ double load_rt<double, 19>(const double* p, int) { return *p; }
template <>
__device__ __forceinline__ double load_rt<double, 27>(const double* p, int) { return *p; }
template <>
__device__ __forceinline__ float load_rt<float, 19>(const float* p, int) { return *p; }
template <>
__device__ __forceinline__ float load_rt<float, 27>(const float* p, int) { return *p; }
template <>
__device__ __forceinline__ float load_rt<__half, 19>(const __half* p, int i) {
  return __half2float(*p) * float(weight_rt<19>(i));
}
template <>
__device__ __forceinline__ float load_rt<__half, 27>(const __half* p, int i) {
  return __half2float(*p) * float(weight_rt<27>(i));
}
template <>
__device__ __forceinline__ void store_rt<double, 19>(double* p, int, double v) { *p = v; }
template <>
__device__ __forceinline__ void store_rt<double, 27>(double* p, int, double v) { *p = v; }
template <>
__device__ __forceinline__ void store_rt<float, 19>(float* p, int, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_rt<float, 27>(float* p, int, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_rt<__half, 19>(__half* p, int i, float v) {
  *p = __float2half_rn(v / float(weight_rt<19>(i)));
}
template <>
__device__ __forceinline__ void store_rt<__half, 27>(__half* p, int i, float v) {
  *p = __float2half_rn(v / float(weight_rt<27>(i)));
}

// ------------------------------------------------------------------ D3Q19 MRT-LES
// Incompressible equilibrium (Section 2, c = 1): w (drho + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2).
template <class T>
__device__ __forceinline__ void feq19(T drho, T ux, T uy, T uz, T* out) {
  const T uu = T(1.5) * (ux * ux + uy * uy + uz * uz);
  static_for<19>([&](auto i) {
    constexpr int x = D3Q19::ex(i), y = D3Q19::ey(i), z = D3Q19::ez(i);
    const T eu = T(x) * ux + T(y) * uy + T(z) * uz;
    out[i] = T(D3Q19::w(i)) * (drho + T(3) * eu + T(4.5) * eu * eu - uu);
  });
}

template <class T>
__device__ __forceinline__ void moments19(const T* g, T& drho, T& ux, T& uy, T& uz) {
  drho = T(0);
  ux = uy = uz = T(0);
  static_for<19>([&](auto i) {
    drho += g[i];
    if constexpr (D3Q19::ex(i) != 0) ux += T(D3Q19::ex(i)) * g[i];
    if constexpr (D3Q19::ey(i) != 0) uy += T(D3Q19::ey(i)) * g[i];
    if constexpr (D3Q19::ez(i) != 0) uz += T(D3Q19::ez(i)) * g[i];
  });
}

// MRT with every non-shear rate 1 (the paper's choice, Section 2) written in
// closed form: f* = f_eq + (1 - s1) P (f - f_eq).  P keeps the five shear
// moments of Table 1 (s1 group) of the non-equilibrium part and drops all
// others: axis links receive 1/2 (Pi_aa - tr Pi / 3), the diagonal links of
// plane ab receive 1/4 e_a e_b Pi_ab, the rest link 0.  s1 = 1/tau_total with
// tau_total from Eq. eqTauTotFinal and Q from Eq. EqnQ.
// Opposite links (2k-1, 2k) are handled as pairs: their sums carry the even
// moments and their differences the odd ones, and since the D3Q19 set is
// isotropic to fourth order, sum_i e_a e_b f_eq_i = drho/3 delta_ab + u_a u_b,
// so Pi^neq = sum e e f - drho/3 I - u u without forming f - f_eq per link.
// Returns |S| = 3 Q / (2 tau_total) (Eq. eqStrainRate, lattice units).
// Scaled: g holds g_i / w_i on entry and exit (the FP16 storage form); the
// weights then enter as constant factors of the sums and of the output
// terms instead of one multiply per population each way.
template <class T, bool Scaled = false>
__device__ __forceinline__ T collide19(T* g, T tau0, T cs2_18) {
  T sp[9], dp[9];
  static_for<9>([&](auto p) {
    sp[p] = g[2 * p + 1] + g[2 * p + 2];
    dp[p] = g[2 * p + 1] - g[2 * p + 2];
  });
  T drho = Scaled ? T(D3Q19::w(0)) * g[0] : g[0];
  T ux = T(0), uy = T(0), uz = T(0);
  T sxx = T(0), syy = T(0), szz = T(0), sxy = T(0), sxz = T(0), syz = T(0);
  static_for<9>([&](auto p) {
    constexpr int i = 2 * p + 1;
    constexpr int x = D3Q19::ex(i), y = D3Q19::ey(i), z = D3Q19::ez(i);
    constexpr double ws = Scaled ? D3Q19::w(i) : 1.0;
    drho += T(ws) * sp[p];
    if constexpr (x != 0) { ux += T(x * ws) * dp[p]; sxx += T(ws) * sp[p]; }
    if constexpr (y != 0) { uy += T(y * ws) * dp[p]; syy += T(ws) * sp[p]; }
    if constexpr (z != 0) { uz += T(z * ws) * dp[p]; szz += T(ws) * sp[p]; }
    if constexpr (x * y != 0) sxy += T(x * y * ws) * sp[p];
    if constexpr (x * z != 0) sxz += T(x * z * ws) * sp[p];
    if constexpr (y * z != 0) syz += T(y * z * ws) * sp[p];
  });
  const T d3 = drho * T(1.0 / 3.0);
  const T pxx = sxx - d3 - ux * ux, pyy = syy - d3 - uy * uy, pzz = szz - d3 - uz * uz;
  const T pxy = sxy - ux * uy, pxz = sxz - ux * uz, pyz = syz - uy * uz;
  const T qq = T(2) * (pxx * pxx + pyy * pyy + pzz * pzz + T(2) * (pxy * pxy + pxz * pxz + pyz * pyz));
  const T Qn = sqrt(qq);
  const T tau = T(0.5) * (tau0 + sqrt(tau0 * tau0 + cs2_18 * Qn));
  const T k = T(1) - T(1) / tau;
  const T tr3 = (pxx + pyy + pzz) * T(1.0 / 3.0);
  // shear projections 1/2 (axis links) and 1/4 (diagonal links), divided by
  // the link weights 1/18 and 1/36 when scaled
  const T cA = Scaled ? T(9) : T(0.5), cD = Scaled ? T(9) : T(0.25);
  const T ax = cA * k * (pxx - tr3), ay = cA * k * (pyy - tr3), az = cA * k * (pzz - tr3);
  const T dxy = cD * k * pxy, dxz = cD * k * pxz, dyz = cD * k * pyz;
  const T base = drho - T(1.5) * (ux * ux + uy * uy + uz * uz);
  g[0] = Scaled ? base : T(D3Q19::w(0)) * base;
  static_for<9>([&](auto p) {
    constexpr int i = 2 * p + 1;
    constexpr int x = D3Q19::ex(i), y = D3Q19::ey(i), z = D3Q19::ez(i);
    constexpr int nz = (x != 0) + (y != 0) + (z != 0);
    T eu = T(0);
    if constexpr (x != 0) eu += T(x) * ux;
    if constexpr (y != 0) eu += T(y) * uy;
    if constexpr (z != 0) eu += T(z) * uz;
    constexpr T w = T(D3Q19::w(i));
    T proj;
    if constexpr (nz == 1) proj = (x != 0) ? ax : (y != 0) ? ay : az;
    else if constexpr (z == 0) proj = T(x * y) * dxy;
    else if constexpr (y == 0) proj = T(x * z) * dxz;
    else proj = T(y * z) * dyz;
    T sym, asym;
    if constexpr (Scaled) {
      sym = base + T(4.5) * eu * eu + proj;
      asym = T(3) * eu;
    } else {
      sym = w * (base + T(4.5) * eu * eu) + proj;
      asym = (T(3) * w) * eu;
    }
    g[i] = sym + asym;
    g[i + 1] = sym - asym;
  });
  return T(1.5) * Qn / tau;
}

// ------------------------------------------------------------------ D3Q27 FCLB
// Central moments by three one-dimensional passes (z, then y, then x): the
// D3Q27 velocity set is the product {-1,0,1}^3 and the central-moment
// matrix of Section 2 factorises into 3x3 per-axis transforms.  Each pass is
// written for deviations from the weight part: a line whose weight part is
// K (w1(-1), w1(0), w1(+1)) = K (1/6, 2/3, 1/6) has moments K (1, 0, 1/3) at
// rest, and the pass outputs the deviations from those.  After three passes
// v[a][b][c] = rho kappa_abc - C_abc with C_abc = c_a c_b c_c, c = (1, 0, 1/3).
// (Index 0/1/2 means velocity -1/0/+1 before a pass and order 0/1/2 after.)
__host__ __device__ constexpr double w1(int k) { return k == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double c1(int k) { return k == 0 ? 1.0 : k == 1 ? 0.0 : 1.0 / 3.0; }

template <class T>
__device__ __forceinline__ void fwd_line(T& a, T& b, T& c, T u, T uu, T K) {
  const T m0 = a + b + c;
  const T d = c - a;
  const T s = c + a;
  const T m0k = m0 + K;
  a = m0;
  b = d - u * m0k;
  c = s - T(2) * u * d + uu * m0k;
}
template <class T>
__device__ __forceinline__ void inv_line(T& a, T& b, T& c, T u, T uu, T K) {
  const T m0 = a, m1 = b, m2 = c;
  const T m0k = m0 + K;
  const T gm = T(0.5) * ((uu - u) * m0k + (T(2) * u - T(1)) * m1 + m2);
  const T gp = T(0.5) * ((uu + u) * m0k + (T(2) * u + T(1)) * m1 + m2);
  const T g0 = m0 * (T(1) - uu) - T(2) * u * m1 - m2 - K * uu;
  a = gm;
  b = g0;
  c = gp;
}

template <class T>
__device__ __forceinline__ void forward27(T (&v)[3][3][3], T ux, T uy, T uz) {
  const T ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) fwd_line(v[i][j][0], v[i][j][1], v[i][j][2], uz, uz2, T(w1(i) * w1(j)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) fwd_line(v[i][0][k], v[i][1][k], v[i][2][k], uy, uy2, T(w1(i) * c1(k)));
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) fwd_line(v[0][j][k], v[1][j][k], v[2][j][k], ux, ux2, T(c1(j) * c1(k)));
}

template <class T>
__device__ __forceinline__ void inverse27(T (&v)[3][3][3], T ux, T uy, T uz) {
  const T ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) inv_line(v[0][j][k], v[1][j][k], v[2][j][k], ux, ux2, T(c1(j) * c1(k)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) inv_line(v[i][0][k], v[i][1][k], v[i][2][k], uy, uy2, T(w1(i) * c1(k)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) inv_line(v[i][j][0], v[i][j][1], v[i][j][2], uz, uz2, T(w1(i) * w1(j)));
}

template <class T>
__device__ __forceinline__ void to_cube(const T* g, T (&v)[3][3][3]) {
  static_for<27>([&](auto i) { v[D3Q27::ex(i) + 1][D3Q27::ey(i) + 1][D3Q27::ez(i) + 1] = g[i]; });
}
template <class T>
__device__ __forceinline__ void from_cube(const T (&v)[3][3][3], T* g) {
  static_for<27>([&](auto i) { g[i] = v[D3Q27::ex(i) + 1][D3Q27::ey(i) + 1][D3Q27::ez(i) + 1]; });
}

template <class T>
__device__ __forceinline__ void moments27(const T* g, T& drho, T& jx, T& jy, T& jz) {
  drho = jx = jy = jz = T(0);
  static_for<27>([&](auto i) {
    drho += g[i];
    if constexpr (D3Q27::ex(i) != 0) jx += T(D3Q27::ex(i)) * g[i];
    if constexpr (D3Q27::ey(i) != 0) jy += T(D3Q27::ey(i)) * g[i];
    if constexpr (D3Q27::ez(i) != 0) jz += T(D3Q27::ez(i)) * g[i];
  });
}

// Factorized cascaded collision (Section 2, Table 2; whole moments recomputed):
// the normal-stress differences and shear moments relax with omega, the
// trace and every higher moment with rate 1 to the Table 2 equilibria built
// from the post-collision second-order moments (third and fifth order 0,
// fourth M_aa M_bb and M_aa M_bc, sixth M11 M22 M33).  With a body force F,
// u = (j + F/2)/rho and the first central moments leave as F/(2 rho).
template <class T>
__device__ __forceinline__ void collide27(T* g, T omega, T Fx, T Fy, T Fz) {
  T drho, jx, jy, jz;
  moments27(g, drho, jx, jy, jz);
  const T rho = T(1) + drho;
  const T irho = T(1) / rho;
  const T ux = (jx + T(0.5) * Fx) * irho, uy = (jy + T(0.5) * Fy) * irho, uz = (jz + T(0.5) * Fz) * irho;
  T v[3][3][3];
  to_cube(g, v);
  forward27(v, ux, uy, uz);
  const T om1 = T(1) - omega;
  const T mean = (v[2][0][0] + v[0][2][0] + v[0][0][2]) * T(1.0 / 3.0);
  const T Dx = om1 * (v[2][0][0] - mean) * irho;
  const T Dy = om1 * (v[0][2][0] - mean) * irho;
  const T Dz = om1 * (v[0][0][2] - mean) * irho;
  const T kxy = om1 * v[1][1][0], kxz = om1 * v[1][0][1], kyz = om1 * v[0][1][1];  // rho kappa'
  const T third = T(1.0 / 3.0);
  const T Xx = third + Dx, Yy = third + Dy, Zz = third + Dz;  // kappa'_200 ...
  // zeroth and first order
  v[0][0][0] = drho;
  v[1][0][0] = T(0.5) * Fx;
  v[0][1][0] = T(0.5) * Fy;
  v[0][0][1] = T(0.5) * Fz;
  // second order
  v[2][0][0] = drho * third + rho * Dx;
  v[0][2][0] = drho * third + rho * Dy;
  v[0][0][2] = drho * third + rho * Dz;
  v[1][1][0] = kxy;
  v[1][0][1] = kxz;
  v[0][1][1] = kyz;
  // third order
  v[2][1][0] = v[2][0][1] = v[1][2][0] = v[0][2][1] = v[1][0][2] = v[0][1][2] = v[1][1][1] = T(0);
  // fourth order
  const T ninth = T(1.0 / 9.0);
  v[2][2][0] = drho * ninth + rho * ((Dx + Dy) * third + Dx * Dy);
  v[2][0][2] = drho * ninth + rho * ((Dx + Dz) * third + Dx * Dz);
  v[0][2][2] = drho * ninth + rho * ((Dy + Dz) * third + Dy * Dz);
  v[2][1][1] = Xx * kyz;
  v[1][2][1] = Yy * kxz;
  v[1][1][2] = Zz * kxy;
  // fifth order
  v[2][2][1] = v[2][1][2] = v[1][2][2] = T(0);
  // sixth order
  v[2][2][2] = drho * T(1.0 / 27.0) +
               rho * ((Dx + Dy + Dz) * ninth + (Dx * Dy + Dx * Dz + Dy * Dz) * third + Dx * Dy * Dz);
  inverse27(v, ux, uy, uz);
  from_cube(v, g);
}

// The same collision in closed form, used by the stream-collide kernel.
// Because every moment above second order is relaxed with rate 1, only the
// six pre-collision second-order central moments matter; they follow from
// raw sums: rho kappa_aa = S_aa - 2 u_a j_a + u_a^2 rho (+ const), rho kappa_ab =
// S_ab - u_a j_b - u_b j_a + u_a u_b rho.  The post-collision normalised
// central moments are then a sum of per-axis products: prod_a (1, 0, X_a)
// for the diagonal part (X_a = 1/3 + D_a), plus kappa'_xy (0,1,0)(0,1,0)(1,0,Z)
// and its two permutations, plus F/(2 rho) in the first order.  The 1-D
// inverse transform of (1, 0, X) is phi(0) = 1 - u^2 - X, phi(+-1) =
// (u^2 +- u + X)/2; of (0, 1, 0) psi(0) = -2u, psi(+-1) = u +- 1/2; of
// (1, 0, 0) chi(0) = 1 - u^2, chi(+-1) = (u^2 +- u)/2.  Writing phi = w1 + delta
// keeps f* - w free of cancellation:
//   f*_i - w_i = drho W_i + rho (dx Py Pz... expanded) + k_xy psi_x psi_y phi_z + ...
// (the paper notes that fixed rates remove most of the FCLB flops).
// Scaled: g holds g_i / w_i on entry and exit (the FP16 storage form); the
// product weights w_i = w1_x w1_y w1_z then enter once per z-line on input
// and once per (e_y, e_z) pair and per e_x factor on output.
template <class T, bool Force, bool Scaled = false>
__device__ __forceinline__ void collide27_closed(T* g, T omega, T Fx, T Fy, T Fz) {
  // ---- zeroth, first and second raw moments of g by a z, y, x collapse
  T m0[3][3], dz[3][3], sz[3][3];  // per (ex, ey): sum, difference, sum of ends along z
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T lo = g[D3Q27::index(a - 1, b - 1, -1)];
      const T mi = g[D3Q27::index(a - 1, b - 1, 0)];
      const T hi = g[D3Q27::index(a - 1, b - 1, 1)];
      if constexpr (Scaled) {
        const T ce = T(w1(a) * w1(b) * w1(0)), cm = T(w1(a) * w1(b) * w1(1));
        sz[a][b] = ce * (hi + lo);
        dz[a][b] = ce * (hi - lo);
        m0[a][b] = sz[a][b] + cm * mi;
      } else {
        sz[a][b] = hi + lo;
        dz[a][b] = hi - lo;
        m0[a][b] = sz[a][b] + mi;
      }
    }
  T M0[3], My[3], Myy[3], Dz[3], Dyz[3], Szz[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T e = m0[a][2] + m0[a][0];
    Myy[a] = e;
    My[a] = m0[a][2] - m0[a][0];
    M0[a] = e + m0[a][1];
    Dz[a] = dz[a][0] + dz[a][1] + dz[a][2];
    Dyz[a] = dz[a][2] - dz[a][0];
    Szz[a] = sz[a][0] + sz[a][1] + sz[a][2];
  }
  const T Sxx = M0[2] + M0[0];
  const T drho = Sxx + M0[1];
  const T jx = M0[2] - M0[0];
  const T jy = My[0] + My[1] + My[2];
  const T Sxy = My[2] - My[0];
  const T Syy = Myy[0] + Myy[1] + Myy[2];
  const T jz = Dz[0] + Dz[1] + Dz[2];
  const T Sxz = Dz[2] - Dz[0];
  const T Syz = Dyz[0] + Dyz[1] + Dyz[2];
  const T Szzt = Szz[0] + Szz[1] + Szz[2];
  // ---- velocity and second-order central moments (deviations from rho/3)
  const T rho = T(1) + drho;
  const T r = T(1) / rho;
  T px = jx, py = jy, pz = jz;
  if constexpr (Force) {
    px += T(0.5) * Fx;
    py += T(0.5) * Fy;
    pz += T(0.5) * Fz;
  }
  const T ux = px * r, uy = py * r, uz = pz * r;
  // rho u_a u_a - 2 u_a j_a = u_a (rho u_a - 2 j_a) = u_a (p_a - 2 j_a)
  const T vxx = Sxx + ux * (px - T(2) * jx);
  const T vyy = Syy + uy * (py - T(2) * jy);
  const T vzz = Szzt + uz * (pz - T(2) * jz);
  const T vxy = Sxy + ux * py - ux * jy - uy * jx;
  const T vxz = Sxz + ux * pz - ux * jz - uz * jx;
  const T vyz = Syz + uy * pz - uy * jz - uz * jy;
  // ---- relaxation: deviatoric part with omega, trace to equilibrium
  const T om1 = T(1) - omega;
  const T mean = (vxx + vyy + vzz) * T(1.0 / 3.0);
  const T Dx = om1 * (vxx - mean) * r, Dy = om1 * (vyy - mean) * r, Dz_ = om1 * (vzz - mean) * r;
  const T kxy = om1 * vxy, kxz = om1 * vxz, kyz = om1 * vyz;  // rho kappa'
  // ---- per-axis factors, index 0/1/2 = velocity -1/0/+1
  T dl[3][3], ph[3][3], ps[3][3], ch[3][3];
  const T uu[3] = {ux, uy, uz};
  const T DD[3] = {Dx, Dy, Dz_};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T u = uu[a], u2 = u * u, D = DD[a];
    dl[a][1] = -u2 - D;
    dl[a][0] = T(0.5) * (u2 - u + D);
    dl[a][2] = T(0.5) * (u2 + u + D);
    ph[a][1] = T(2.0 / 3.0) + dl[a][1];
    ph[a][0] = T(1.0 / 6.0) + dl[a][0];
    ph[a][2] = T(1.0 / 6.0) + dl[a][2];
    ps[a][1] = T(-2) * u;
    ps[a][0] = u - T(0.5);
    ps[a][2] = u + T(0.5);
    if constexpr (Force) {
      ch[a][1] = T(1) - u2;
      ch[a][0] = T(0.5) * (u2 - u);
      ch[a][2] = T(0.5) * (u2 + u);
    }
  }
  // ---- per (e_y, e_z) pair, then per e_x
  if constexpr (Scaled) {
    // the x factors divided by w1_x once
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dl[0][a] *= T(1.0 / w1(a));
      ps[0][a] *= T(1.0 / w1(a));
      ph[0][a] *= T(1.0 / w1(a));
      if constexpr (Force) ch[0][a] *= T(1.0 / w1(a));
    }
  }
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T P = ph[1][b] * ph[2][c];                            // phi_y phi_z
      const T Qd = T(w1(b)) * dl[2][c] + dl[1][b] * ph[2][c];     // phi_y phi_z - w1_y w1_z
      T rP = rho * P, rQ = rho * Qd;
      T R = kxy * ps[1][b] * ph[2][c] + kxz * ph[1][b] * ps[2][c];
      T Sy = kyz * ps[1][b] * ps[2][c];
      T Fp = T(0), Gp = T(0);
      if constexpr (Force) {
        Fp = T(0.5) * Fx * ch[1][b] * ch[2][c];
        Gp = T(0.5) * Fy * ps[1][b] * ch[2][c] + T(0.5) * Fz * ch[1][b] * ps[2][c];
      }
      if constexpr (Scaled) {
        const T ibc = T(1.0 / (w1(b) * w1(c)));
        rP *= ibc;
        R *= ibc;
        Sy *= ibc;
        if constexpr (Force) {
          Fp *= ibc;
          Gp *= ibc;
        }
        const T base = drho + ibc * rQ;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          T v = base + dl[0][a] * rP + ps[0][a] * R + ph[0][a] * Sy;
          if constexpr (Force) v += ps[0][a] * Fp + ch[0][a] * Gp;
          g[D3Q27::index(a - 1, b - 1, c - 1)] = v;
        }
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T W = T(w1(a) * w1(b) * w1(c));
          T v = drho * W + dl[0][a] * rP + T(w1(a)) * rQ + ps[0][a] * R + ph[0][a] * Sy;
          if constexpr (Force) v += ps[0][a] * Fp + ch[0][a] * Gp;
          g[D3Q27::index(a - 1, b - 1, c - 1)] = v;
        }
      }
    }
}

// Product-form D3Q27 equilibrium minus the weights: the distribution whose
// normalised central moments are the Table 2 equilibria at rest shape is
// rho prod_a phi(e_a, u_a), phi(0) = 2/3 - u^2, phi(+-1) = (1/3 + u^2 +- u)/2.
// With phi = w1 + delta it is evaluated without cancellation as
// drho W + rho (delta_x phi_y phi_z + w1_x (delta_y phi_z + w1_y delta_z)).
template <class T>
__device__ __forceinline__ void feq27(T drho, T ux, T uy, T uz, T* out) {
  const T rho = T(1) + drho;
  T dl[3][3], ph[3][3];
  const T uu[3] = {ux, uy, uz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T u = uu[a], u2 = u * u;
    dl[a][1] = -u2;
    dl[a][0] = T(0.5) * (u2 - u);
    dl[a][2] = T(0.5) * (u2 + u);
    ph[a][1] = T(2.0 / 3.0) + dl[a][1];
    ph[a][0] = T(1.0 / 6.0) + dl[a][0];
    ph[a][2] = T(1.0 / 6.0) + dl[a][2];
  }
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T rP = rho * ph[1][b] * ph[2][c];
      const T rQ = rho * (T(w1(b)) * dl[2][c] + dl[1][b] * ph[2][c]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        out[D3Q27::index(a - 1, b - 1, c - 1)] = drho * T(w1(a) * w1(b) * w1(c)) + dl[0][a] * rP + T(w1(a)) * rQ;
    }
}

// ------------------------------------------------------------------ model traits
struct MrtLes {
  static constexpr int Q = 19;
  template <class T>
  __device__ static __forceinline__ void moments(const T* g, T& rl, T& ux, T& uy, T& uz) {
    moments19(g, rl, ux, uy, uz);  // rho_0 = 1
  }
  template <class T>
  __device__ static __forceinline__ void feq(T rl, T ux, T uy, T uz, T* out) {
    feq19(rl, ux, uy, uz, out);
  }
};
struct Fclb {
  static constexpr int Q = 27;
  template <class T>
  __device__ static __forceinline__ void moments(const T* g, T& rl, T& ux, T& uy, T& uz) {
    T jx, jy, jz;
    moments27(g, rl, jx, jy, jz);
    const T ir = T(1) / (T(1) + rl);
    ux = jx * ir;
    uy = jy * ir;
    uz = jz * ir;
  }
  template <class T>
  __device__ static __forceinline__ void feq(T rl, T ux, T uy, T uz, T* out) {
    feq27(rl, ux, uy, uz, out);
  }
};

}  // namespace lbm
