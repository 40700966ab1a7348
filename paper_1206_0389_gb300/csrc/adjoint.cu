// Discrete adjoint of one D3Q27 FCLB stream-collide step with a body force.
//
// Forward step (single periodic level): f~_{t+1}(x) = C(p(x), F(x)) with the
// pulled pre-collision vector p(x)_i = f~_t(x - e_i)_i.  For a loss L of the
// final state, lambda_t = dL/df~_t obeys
//   mu(x) = J_C(p(x), F(x))^T lambda_{t+1}(x),   lambda_t(x - e_i)_i = mu(x)_i,
// and dL/dF(x) += (dC/dF(p(x), F(x)))^T lambda_{t+1}(x).
// So the adjoint kernel reads f~_t at exactly the addresses the forward pull
// reads, reads lambda_{t+1} at its own cell, and writes mu_i to lambda_t at
// the forward pull addresses (each written once: no races).
//
// J_C^T is hand-derived reverse mode of collide27 (collide.cuh): the three
// forward one-dimensional passes, the relaxation with its products of
// post-collision second-order moments, and the three inverse passes, each
// reversed with its own pass inputs recomputed instead of stored.
#include "collide.cuh"
#include "kernels.cuh"

namespace lbm {

// adjoint of fwd_line: (a, b, c) are the pass inputs; (l0, l1, l2) the
// adjoints of the outputs on entry and of (a, b, c) on exit; returns du.
template <class T>
__device__ __forceinline__ T fwd_line_adj(T a, T b, T c, T& l0, T& l1, T& l2, T u, T uu, T K) {
  const T m0k = a + b + c + K;
  const T d = c - a;
  const T lm0 = l0 - u * l1 + uu * l2;
  const T ld = l1 - T(2) * u * l2;
  const T ls = l2;
  const T du = -l1 * m0k + l2 * (T(2) * u * m0k - T(2) * d);
  l0 = lm0 - ld + ls;
  l1 = lm0;
  l2 = lm0 + ld + ls;
  return du;
}

// adjoint of inv_line: (m0, m1, m2) are the pass inputs; (la, lb, lc) the
// adjoints of (g-, g0, g+) on entry and of (m0, m1, m2) on exit; returns du.
template <class T>
__device__ __forceinline__ T inv_line_adj(T m0, T m1, T m2, T& la, T& lb, T& lc, T u, T uu, T K) {
  (void)m2;
  const T lm = la, l0 = lb, lp = lc;
  const T m0k = m0 + K;
  const T du = T(0.5) * lm * ((T(2) * u - T(1)) * m0k + T(2) * m1) -
               T(2) * l0 * (u * m0k + m1) + T(0.5) * lp * ((T(2) * u + T(1)) * m0k + T(2) * m1);
  la = T(0.5) * (uu - u) * lm + (T(1) - uu) * l0 + T(0.5) * (uu + u) * lp;
  lb = (u - T(0.5)) * lm - T(2) * u * l0 + (u + T(0.5)) * lp;
  lc = T(0.5) * lm - l0 + T(0.5) * lp;
  return du;
}

template <class T>
struct RelaxState {
  T drho, r, A, B, C, kxy, kxz, kyz, Fx, Fy, Fz;
};

// post-collision moments (deviation form) from the relaxation scalars; the
// same values collide27 builds
template <class T>
__device__ __forceinline__ void build_vprime(T (&v)[3][3][3], const RelaxState<T>& s) {
  const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0);
  const T A = s.A, B = s.B, C = s.C, r = s.r, d = s.drho;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[a][b][c] = T(0);
  v[0][0][0] = d;
  v[1][0][0] = T(0.5) * s.Fx;
  v[0][1][0] = T(0.5) * s.Fy;
  v[0][0][1] = T(0.5) * s.Fz;
  v[2][0][0] = d * third + A;
  v[0][2][0] = d * third + B;
  v[0][0][2] = d * third + C;
  v[1][1][0] = s.kxy;
  v[1][0][1] = s.kxz;
  v[0][1][1] = s.kyz;
  v[2][2][0] = d * ninth + (A + B) * third + A * B * r;
  v[2][0][2] = d * ninth + (A + C) * third + A * C * r;
  v[0][2][2] = d * ninth + (B + C) * third + B * C * r;
  v[2][1][1] = (third + A * r) * s.kyz;
  v[1][2][1] = (third + B * r) * s.kxz;
  v[1][1][2] = (third + C * r) * s.kxy;
  v[2][2][2] = d * T(1.0 / 27.0) + (A + B + C) * ninth + (A * B + A * C + B * C) * r * third + A * B * C * r * r;
}

template <class T>
__device__ __forceinline__ void inv_x(T (&v)[3][3][3], T u, T uu) {
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) inv_line(v[0][j][k], v[1][j][k], v[2][j][k], u, uu, T(c1(j) * c1(k)));
}
template <class T>
__device__ __forceinline__ void inv_y(T (&v)[3][3][3], T u, T uu) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) inv_line(v[i][0][k], v[i][1][k], v[i][2][k], u, uu, T(w1(i) * c1(k)));
}
template <class T>
__device__ __forceinline__ void fwd_z(T (&v)[3][3][3], T u, T uu) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) fwd_line(v[i][j][0], v[i][j][1], v[i][j][2], u, uu, T(w1(i) * w1(j)));
}
template <class T>
__device__ __forceinline__ void fwd_y(T (&v)[3][3][3], T u, T uu) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) fwd_line(v[i][0][k], v[i][1][k], v[i][2][k], u, uu, T(w1(i) * c1(k)));
}
template <class T>
__device__ __forceinline__ void fwd_x(T (&v)[3][3][3], T u, T uu) {
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) fwd_line(v[0][j][k], v[1][j][k], v[2][j][k], u, uu, T(c1(j) * c1(k)));
}

// mu = J_C^T lambda for the pre-collision shifted values g; lam holds lambda
// on entry and mu on exit; F-bar (dL/dF of this step) is added to Fb.
// The relaxation only reads the six second-order central moments of the
// incoming populations, v_aa = S_aa + u_a (p_a - 2 j_a) and
// v_ab = S_ab + u_a p_b - u_a j_b - u_b j_a (S = raw second moments of g,
// j = first moments, p = j + F/2 = rho u), so the forward transform is
// reversed through those closed forms; the inverse passes and the relaxation
// are reversed pass by pass.
template <class T>
__device__ __forceinline__ void collide27_adjoint(const T* g, T* lam, T omega, T Fx, T Fy, T Fz, T& Fbx,
                                                  T& Fby, T& Fbz) {
  // ---- forward recomputation: raw moments, velocity, second-order central moments
  T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
  T Sxx = T(0), Syy = T(0), Szz = T(0), Sxy = T(0), Sxz = T(0), Syz = T(0);
  static_for<27>([&](auto i) {
    constexpr int x = D3Q27::ex(i), y = D3Q27::ey(i), z = D3Q27::ez(i);
    const T v = g[i];
    drho += v;
    if constexpr (x != 0) { jx += T(x) * v; Sxx += v; }
    if constexpr (y != 0) { jy += T(y) * v; Syy += v; }
    if constexpr (z != 0) { jz += T(z) * v; Szz += v; }
    if constexpr (x * y != 0) Sxy += T(x * y) * v;
    if constexpr (x * z != 0) Sxz += T(x * z) * v;
    if constexpr (y * z != 0) Syz += T(y * z) * v;
  });
  const T r = T(1) / (T(1) + drho);
  const T px = jx + T(0.5) * Fx, py = jy + T(0.5) * Fy, pz = jz + T(0.5) * Fz;
  const T ux = px * r, uy = py * r, uz = pz * r;
  const T ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const T vxx = Sxx + ux * (px - T(2) * jx), vyy = Syy + uy * (py - T(2) * jy), vzz = Szz + uz * (pz - T(2) * jz);
  const T vxy = Sxy + ux * py - ux * jy - uy * jx;
  const T vxz = Sxz + ux * pz - ux * jz - uz * jx;
  const T vyz = Syz + uy * pz - uy * jz - uz * jy;
  const T om1 = T(1) - omega;
  const T mean = (vxx + vyy + vzz) * T(1.0 / 3.0);
  RelaxState<T> s;
  s.drho = drho;
  s.r = r;
  s.A = om1 * (vxx - mean);
  s.B = om1 * (vyy - mean);
  s.C = om1 * (vzz - mean);
  s.kxy = om1 * vxy;
  s.kxz = om1 * vxz;
  s.kyz = om1 * vyz;
  s.Fx = Fx;
  s.Fy = Fy;
  s.Fz = Fz;
  T W[3][3][3], L[3][3][3];
  to_cube(lam, L);
  T ubx = T(0), uby = T(0), ubz = T(0);
  // ---- inverse z pass (input = yinv(xinv(V')))
  build_vprime(W, s);
  inv_x(W, ux, ux2);
  inv_y(W, uy, uy2);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      ubz += inv_line_adj(W[i][j][0], W[i][j][1], W[i][j][2], L[i][j][0], L[i][j][1], L[i][j][2], uz, uz2,
                          T(w1(i) * w1(j)));
  // ---- inverse y pass (input = xinv(V'))
  build_vprime(W, s);
  inv_x(W, ux, ux2);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      uby += inv_line_adj(W[i][0][k], W[i][1][k], W[i][2][k], L[i][0][k], L[i][1][k], L[i][2][k], uy, uy2,
                          T(w1(i) * c1(k)));
  // ---- inverse x pass (input = V')
  build_vprime(W, s);
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      ubx += inv_line_adj(W[0][j][k], W[1][j][k], W[2][j][k], L[0][j][k], L[1][j][k], L[2][j][k], ux, ux2,
                          T(c1(j) * c1(k)));
  // ---- relaxation
  const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0);
  const T A = s.A, B = s.B, C = s.C;
  T drb = L[0][0][0] + (L[2][0][0] + L[0][2][0] + L[0][0][2]) * third +
          (L[2][2][0] + L[2][0][2] + L[0][2][2]) * ninth + L[2][2][2] * T(1.0 / 27.0);
  Fbx += T(0.5) * L[1][0][0];
  Fby += T(0.5) * L[0][1][0];
  Fbz += T(0.5) * L[0][0][1];
  const T Ab = L[2][0][0] + L[2][2][0] * (third + B * r) + L[2][0][2] * (third + C * r) + L[2][1][1] * r * s.kyz +
               L[2][2][2] * (ninth + (B + C) * r * third + B * C * r * r);
  const T Bb = L[0][2][0] + L[2][2][0] * (third + A * r) + L[0][2][2] * (third + C * r) + L[1][2][1] * r * s.kxz +
               L[2][2][2] * (ninth + (A + C) * r * third + A * C * r * r);
  const T Cb = L[0][0][2] + L[2][0][2] * (third + A * r) + L[0][2][2] * (third + B * r) + L[1][1][2] * r * s.kxy +
               L[2][2][2] * (ninth + (A + B) * r * third + A * B * r * r);
  const T kxyb = L[1][1][0] + L[1][1][2] * (third + C * r);
  const T kxzb = L[1][0][1] + L[1][2][1] * (third + B * r);
  const T kyzb = L[0][1][1] + L[2][1][1] * (third + A * r);
  T rb = L[2][2][0] * A * B + L[2][0][2] * A * C + L[0][2][2] * B * C + L[2][1][1] * A * s.kyz +
         L[1][2][1] * B * s.kxz + L[1][1][2] * C * s.kxy +
         L[2][2][2] * ((A * B + A * C + B * C) * third + T(2) * A * B * C * r);
  const T Sb = (Ab + Bb + Cb) * third;
  const T vxxb = om1 * (Ab - Sb), vyyb = om1 * (Bb - Sb), vzzb = om1 * (Cb - Sb);
  const T vxyb = om1 * kxyb, vxzb = om1 * kxzb, vyzb = om1 * kyzb;
  // ---- second-order central moments from raw moments
  T jbx = T(-2) * vxxb * ux - vxyb * uy - vxzb * uz;
  T jby = T(-2) * vyyb * uy - vxyb * ux - vyzb * uz;
  T jbz = T(-2) * vzzb * uz - vxzb * ux - vyzb * uy;
  // (v_ab is written with u_a p_b, so p_x enters only v_xx and p_y only v_yy, v_xy)
  T pbx = vxxb * ux;
  T pby = vyyb * uy + vxyb * ux;
  T pbz = vzzb * uz + vxzb * ux + vyzb * uy;
  ubx += vxxb * (px - T(2) * jx) + vxyb * (py - jy) + vxzb * (pz - jz);
  uby += vyyb * (py - T(2) * jy) + vxyb * (-jx) + vyzb * (pz - jz);
  ubz += vzzb * (pz - T(2) * jz) + vxzb * (-jx) + vyzb * (-jy);
  // ---- u = p r, p = j + F/2, r = 1/(1 + drho)
  pbx += ubx * r;
  pby += uby * r;
  pbz += ubz * r;
  rb += ubx * px + uby * py + ubz * pz;
  jbx += pbx;
  jby += pby;
  jbz += pbz;
  Fbx += T(0.5) * pbx;
  Fby += T(0.5) * pby;
  Fbz += T(0.5) * pbz;
  drb -= rb * r * r;
  // ---- back to the populations: d/dg_i of (drho, j, S)
  static_for<27>([&](auto i) {
    constexpr int x = D3Q27::ex(i), y = D3Q27::ey(i), z = D3Q27::ez(i);
    T m = drb;
    if constexpr (x != 0) m += T(x) * jbx + vxxb;
    if constexpr (y != 0) m += T(y) * jby + vyyb;
    if constexpr (z != 0) m += T(z) * jbz + vzzb;
    if constexpr (x * y != 0) m += T(x * y) * vxyb;
    if constexpr (x * z != 0) m += T(x * z) * vxzb;
    if constexpr (y * z != 0) m += T(y * z) * vyzb;
    lam[i] = m;
  });
}

// One adjoint step over all blocks of a periodic single level (CTA = block).
template <class T, int TPB>
__global__ void __launch_bounds__(TPB, sizeof(T) == 4 ? 4 : 1) k_adjoint(const AdjointArgs a) {
  constexpr int Q = 27;
  constexpr int QS = Q * kCells;
  const T* __restrict__ fsrc = reinterpret_cast<const T*>(a.f_t);
  const T* __restrict__ lin = reinterpret_cast<const T*>(a.lam_in);
  T* __restrict__ lout = reinterpret_cast<T*>(a.lam_out);
  T* __restrict__ gF = reinterpret_cast<T*>(a.dLdF);
  const int64_t ncell = int64_t(a.BX) * a.BY * a.BZ * kCells;
  for (int b = blockIdx.x; b < a.nblocks; b += gridDim.x) {
    const int bx = b % a.BX, by = (b / a.BX) % a.BY, bz = b / (a.BX * a.BY);
    const int BXY = a.BX * a.BY;
    // x / y block offsets fit an int (the planner keeps BX * BY * 27 * 512
    // below 2^31); a periodic z wrap moves by up to nblocks * 27 * 512
    // elements, so the z neighbours enter through 64-bit base indices
    const int dxm = bx == 0 ? a.BX - 1 : -1, dxp = bx == a.BX - 1 ? -(a.BX - 1) : 1;
    const int dym = by == 0 ? a.BX * (a.BY - 1) : -a.BX, dyp = by == a.BY - 1 ? -a.BX * (a.BY - 1) : a.BX;
    const int64_t dzm = bz == 0 ? int64_t(BXY) * (a.BZ - 1) : -int64_t(BXY);
    const int64_t dzp = bz == a.BZ - 1 ? -int64_t(BXY) * (a.BZ - 1) : int64_t(BXY);
#pragma unroll 1
    for (int c = threadIdx.x; c < kCells; c += TPB) {
      const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
      const int Xm = (x == 0) ? dxm * QS + 8 : 0, Xp = (x == 7) ? dxp * QS - 8 : 0;
      const int Ym = (y == 0) ? dym * QS + 64 : 0, Yp = (y == 7) ? dyp * QS - 64 : 0;
      const int64_t own = int64_t(b) * QS + c;
      const int64_t B1 = z == 0 ? own + dzm * QS + 512 : own;   // base of e_z = +1 pulls
      const int64_t Bm = z == 7 ? own + dzp * QS - 512 : own;   // base of e_z = -1 pulls
      // element index of population i's pull source (= its adjoint target)
      auto pull = [&](auto i) {
        constexpr int ex = D3Q27::ex(i), ey = D3Q27::ey(i), ez = D3Q27::ez(i);
        int o = int(i) * kCells - (ex + 8 * ey + 64 * ez);
        if constexpr (ex == 1) o += Xm;
        if constexpr (ex == -1) o += Xp;
        if constexpr (ey == 1) o += Ym;
        if constexpr (ey == -1) o += Yp;
        return (ez == 1 ? B1 : ez == -1 ? Bm : own) + o;
      };
      T g[Q], lam[Q];
      static_for<Q>([&](auto i) {
        g[i] = fsrc[pull(i)];
        lam[i] = lin[own + int(i) * kCells];
      });
      const int64_t j = int64_t(b) * kCells + c;
      T Fx = T(0), Fy = T(0), Fz = T(0);
      if (a.force != nullptr) {
        const T* F = reinterpret_cast<const T*>(a.force);
        Fx = F[j];
        Fy = F[ncell + j];
        Fz = F[2 * ncell + j];
      }
      T Fbx = T(0), Fby = T(0), Fbz = T(0);
      collide27_adjoint<T>(g, lam, T(a.omega), Fx, Fy, Fz, Fbx, Fby, Fbz);
      static_for<Q>([&](auto i) { lout[pull(i)] = lam[i]; });
      gF[j] += Fbx;
      gF[ncell + j] += Fby;
      gF[2 * ncell + j] += Fbz;
    }
  }
}

cudaError_t launch_adjoint(int storage, const AdjointArgs& a, cudaStream_t st) {
  if (a.nblocks == 0) return cudaSuccess;
  if (storage == LBM_F64)
    k_adjoint<double, 128><<<a.nblocks, 128, 0, st>>>(a);
  else if (storage == LBM_F32)
    k_adjoint<float, 128><<<a.nblocks, 128, 0, st>>>(a);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lbm
