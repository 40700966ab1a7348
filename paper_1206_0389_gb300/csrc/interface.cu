// Level-interface and boundary kernels of the time-nested grid.
//
// Coarse-to-fine (Yu et al., cited in Sections 1 and 3.2; reading fixed by
// this library): each fine ghost cell receives the trilinear interpolation F^
// of the coarse post-collision values (at t for fine substep 0, the mean of t
// and t+1 for substep 1), then f~_f = f_eq(F^) + r_cf (F^ - f_eq(F^)),
// r_cf = (tau_f - 1) / (2 (tau_c - 1)), with the Smagorinsky |S| carried by
// the same interpolation (tau_c = tau0_c + 3 Cs^2 |S|, tau_f = tau0_f + 3 Cs^2 |S|/2).
// Fine-to-coarse: hidden coarse cells take the mean over their 8 children of
// f_eq + r_fc (f~ - f_eq), r_fc = 2 (tau_c - 1) / (tau_f - 1), with tau_f the
// child's own and tau_c = tau0_c + 3 Cs^2 (2 |S|_child).
// Inflow: ghost = f_eq(rho of the adjacent cell, u_bc) with the top-hat disc
// velocity (Section 3.2 names a constant inflow velocity).  The zero-gradient
// outflow (ghost = copy of the adjacent cell) has no kernel here: the
// stream-collide kernel pulls those populations from the adjacent cell.
// Streaming only pulls, so a ghost cell is read only through the populations
// that point from it into an updated cell; the kernels write just those (the
// planner's per-item mask; e_x = +1 at the inflow) and leave the others as
// they were.
#include <type_traits>

#include "collide.cuh"
#include "kernels.cuh"

namespace lbm {

// ---------------------------------------------------------------- lane-per-population helpers
// The inflow kernel gives each population of a ghost cell to a lane (the
// x-face cells it serves are 8 elements apart, so a thread-per-cell kernel
// serialises 27 sector loads per thread).  Each lane reads its velocity and
// weight through L1 (the lanes of a warp read different entries, which
// constant memory would serialise) and keeps them in registers.
__device__ const int8_t g_ex[32] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, 1, -1, -1, 1, -1};
__device__ const int8_t g_ey[32] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, 1, -1, 1, -1, -1};
__device__ const int8_t g_ez[32] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, 1, -1, -1, -1};

// velocity and weight of the lane's population (lanes >= Q get zeros)
template <class T, int Q>
struct Lane {
  int x, y, z;
  bool act;
  T w;
  __device__ __forceinline__ explicit Lane(int q) {
    act = q < Q;
    x = act ? int(__ldg(g_ex + q)) : 0;
    y = act ? int(__ldg(g_ey + q)) : 0;
    z = act ? int(__ldg(g_ez + q)) : 0;
    const int n = x * x + y * y + z * z;
    if (Q == 19) w = T(n == 0 ? 1.0 / 3.0 : n == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    else w = T(n == 0 ? 8.0 / 27.0 : n == 1 ? 2.0 / 27.0 : n == 2 ? 1.0 / 54.0 : 1.0 / 216.0);
  }
};

// one population of storage <-> shifted value g
template <class S, class T, int Q>
__device__ __forceinline__ T lane_load(const S* p, const Lane<T, Q>& ln) {
  if constexpr (std::is_same<S, __half>::value) return __half2float(*p) * ln.w;
  else return *p;
}
template <class S, class T, int Q>
__device__ __forceinline__ void lane_store(S* p, const Lane<T, Q>& ln, T v) {
  if constexpr (std::is_same<S, __half>::value) *p = __float2half_rn(v / ln.w);
  else *p = v;
}

// equilibrium of the lane's population, shifted like the storage
template <class M, class T, int Q>
__device__ __forceinline__ T lane_feq(T rl, T ux, T uy, T uz, const Lane<T, Q>& ln) {
  if constexpr (M::Q == 19) {
    const T eu = T(ln.x) * ux + T(ln.y) * uy + T(ln.z) * uz;
    return ln.w * (rl + T(3) * eu + T(4.5) * eu * eu - T(1.5) * (ux * ux + uy * uy + uz * uz));
  } else {
    // rho prod_a phi(e_a, u_a) - prod_a w1(e_a), phi = w1 + delta
    auto delta = [](int e, T u) { return e == 0 ? -u * u : T(0.5) * (u * u + T(e) * u); };
    auto wone = [](int e) { return e == 0 ? T(2.0 / 3.0) : T(1.0 / 6.0); };
    const T dx = delta(ln.x, ux), dy = delta(ln.y, uy), dz = delta(ln.z, uz);
    const T wx = wone(ln.x), wy = wone(ln.y), wz = wone(ln.z);
    const T py = wy + dy, pz = wz + dz;
    const T rho = T(1) + rl;
    return rl * wx * wy * wz + rho * (dx * py * pz + wx * (dy * pz + wy * dz));
  }
}

// Fine-to-coarse: four lanes serve one item; lane r loads the child pair
// p = r (one aligned two-element load per population), the partial sums meet
// by two xor shuffles, and lane r stores the populations i with i % 4 == r.
constexpr int kLanes = 4;

// SplitMix64 (Steele, Lea & Flood 2014): advance by the golden gamma, then mix.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// xi in [-1, 1) for one boundary value: chain over (seed, coarse step,
// level << 32 | substep, cell, component)
__device__ __forceinline__ double inflow_xi(unsigned long long seed, long long step, int level,
                                            int substep, long long cell, int comp) {
  unsigned long long h = splitmix64(seed);
  h = splitmix64(h ^ (unsigned long long)step);
  h = splitmix64(h ^ (((unsigned long long)level << 32) | (unsigned long long)substep));
  h = splitmix64(h ^ (unsigned long long)cell);
  h = splitmix64(h ^ (unsigned long long)comp);
  return 2.0 * double(h >> 11) * 0x1.0p-53 - 1.0;
}

// inflow velocity component c (0, 1, 2) of face cell (y, z) of a level at
// (coarse step, level, substep): the disc velocity with its perturbation,
// zero outside the disc (double: the disc test decides a bit)
__device__ __forceinline__ double inflow_u(const long long* step, double y0, double z0, double r2,
                                           double u_in, double perturb, unsigned long long seed,
                                           int level, int substep, int NY, double inv_scale, int y,
                                           int z, int c) {
  const double yc = (double(y) + 0.5) * inv_scale;
  const double zc = (double(z) + 0.5) * inv_scale;
  const double dy = yc - y0, dz = zc - z0;
  if (!(dy * dy + dz * dz < r2)) return 0.0;
  const long long cell = (long long)y + (long long)NY * z;
  const double xi = inflow_xi(seed, *step, level, substep, cell, c);
  return c == 0 ? u_in * (1.0 + perturb * xi) : u_in * perturb * xi;
}

// the level that owns global item g of a multi-level launch (a register
// copy: the unrolled selects keep the launch parameters in the constant
// bank); g becomes the level-local index
template <class Lv, class Args>
__device__ __forceinline__ Lv pick_level(const Args& a, int& g) {
  Lv L = a.lv[0];
#pragma unroll
  for (int k = 1; k < kMaxL; ++k)
    if (k < a.nlv && g >= L.n) {
      g -= L.n;
      L = a.lv[k];
    }
  return L;
}

template <class T>
__device__ __forceinline__ T quad_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// One CTA per chunk (kC2FMaxItems threads): stage the chunk's distinct
// coarse stencil cells in shared memory (for substep 1 already averaged over
// t and t+1), one thread per cell with all Q loads in flight (consecutive
// threads read consecutive cells of the address-sorted list); then one thread
// per ghost cell interpolates from shared memory.  The distinct cells of a
// chunk number about a quarter of its 8 x items stencil references.
template <class M, class S>
__global__ void __launch_bounds__(kC2FMaxItems) k_c2f(const C2FArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int Q = M::Q;
  constexpr int QS = Q * kCells;
  constexpr int MC = c2f_max_cells(std::is_same<S, double>::value ? LBM_F64 : LBM_F32);
  // one row of Q values per staged cell, padded to whole 16-byte vectors:
  // rows are written and read with 16-byte shared accesses (the row stride
  // of 20 or 28 words keeps the lanes of a quarter warp on distinct banks)
  constexpr int VW = 16 / int(sizeof(T));
  constexpr int QP = (Q + VW - 1) / VW * VW;
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  __shared__ __align__(16) T sv[MC * QP];
  __shared__ T sS[MC];
  int g = blockIdx.x;
  const C2FLevel L = pick_level<C2FLevel>(a, g);
  const C2FChunk ch = L.chunks[g];
  const int nc = ch.ncells;
  const S* co = reinterpret_cast<const S*>(L.c_old);
  const S* cn = reinterpret_cast<const S*>(L.c_new);
  // each thread stages whole cells (MC / blockDim of them at most), all Q
  // loads of a cell issued before the first is used
#pragma unroll 1
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    const C2FCell cl = L.cells[ch.first_cell + j];
    const int64_t o = int64_t(cl.cblock) * QS + cl.ccell;
    T v[Q];
    static_for<Q>([&](auto i) { v[i] = St::template get<Q, i>(co + o + int(i) * kCells); });
    if (L.s == 1) {
      static_for<Q>([&](auto i) { v[i] = T(0.5) * (v[i] + St::template get<Q, i>(cn + o + int(i) * kCells)); });
    }
    static_for<QP / VW>([&](auto b) {
      T t[VW];
      static_for<VW>([&](auto e) {
        constexpr int i = int(b) * VW + int(e);
        if constexpr (i < Q) t[e] = v[i];
        else t[e] = T(0);
      });
      V vec;
      if constexpr (VW == 4) vec = make_float4(t[0], t[1], t[2], t[3]);
      else vec = make_double2(t[0], t[1]);
      *reinterpret_cast<V*>(sv + j * QP + int(b) * VW) = vec;
    });
    if (L.a_old != nullptr) {
      const int64_t jj = int64_t(cl.cblock) * kCells + cl.ccell;
      T sj = reinterpret_cast<const T*>(L.a_old)[jj];
      if (L.s == 1) sj = T(0.5) * (sj + reinterpret_cast<const T*>(L.a_new)[jj]);
      sS[j] = sj;
    }
  }
  __syncthreads();
  if (int(threadIdx.x) >= ch.nitems) return;
  const C2FItem it = L.items[ch.first_item + threadIdx.x];
  const T tx = (it.tbits & 1) ? T(0.75) : T(0.25);
  const T ty = (it.tbits & 2) ? T(0.75) : T(0.25);
  const T tz = (it.tbits & 4) ? T(0.75) : T(0.25);
  T F[Q];
  static_for<Q>([&](auto i) { F[i] = T(0); });
  T Sh = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const T W = ((k & 4) ? tz : T(1) - tz) * ((k & 2) ? ty : T(1) - ty) * ((k & 1) ? tx : T(1) - tx);
    const T* row = sv + int(it.slot[k]) * QP;
    static_for<QP / VW>([&](auto b) {
      const V vec = *reinterpret_cast<const V*>(row + int(b) * VW);
      const T* t = reinterpret_cast<const T*>(&vec);
      static_for<VW>([&](auto e) {
        constexpr int i = int(b) * VW + int(e);
        if constexpr (i < Q) F[i] += W * t[e];
      });
    });
    if (L.a_old != nullptr) Sh += W * sS[it.slot[k]];
  }
  T rl, ux, uy, uz;
  M::moments(F, rl, ux, uy, uz);
  T feq[Q];
  M::feq(rl, ux, uy, uz, feq);
  const T tc = T(L.tau0_c) + T(a.cs2_3) * Sh;
  const T tf = T(L.tau0_f) + T(a.cs2_3) * Sh / T(2);
  const T rr = (tf - T(1)) / (T(2) * (tc - T(1)));
  S* fd = reinterpret_cast<S*>(L.f_dst) + int64_t(it.fblock) * QS + it.fcell;
  static_for<Q>([&](auto i) {
    if ((it.need >> int(i)) & 1u) St::template put<Q, i>(fd + int(i) * kCells, feq[i] + rr * (F[i] - feq[i]));
  });
  if (L.fa_dst != nullptr) reinterpret_cast<T*>(L.fa_dst)[int64_t(it.fblock) * kCells + it.fcell] = Sh / T(2);
  if (it.bc >= 0) {
    // the inflow ghost fed by this ghost cell: f_eq(rho of the cell, u_bc);
    // the cell's density is that of F^ (f_eq and F^ - f_eq carry rho^, 0)
    const BCItem b = L.bc[it.bc];
    T ub[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      ub[c] = a.closed ? T(0)
                       : T(inflow_u(a.step, a.y0, a.z0, a.r2, a.u_in, a.perturb, a.seed, L.level, L.substep,
                                    L.NY, L.inv_scale, b.y, b.z, c));
    T fb[Q];
    M::feq(rl, ub[0], ub[1], ub[2], fb);
    S* gd = reinterpret_cast<S*>(L.f_dst) + int64_t(b.gblock) * QS + b.gcell;
    static_for<Q>([&](auto i) {
      if constexpr (Lattice<Q>::ex(i) == 1) St::template put<Q, i>(gd + int(i) * kCells, fb[i]);
    });
  }
}

// two adjacent stored values starting at an even index: one aligned load
template <class S, int Q, int i>
__device__ __forceinline__ void get_pair(const S* p, typename Store<S>::T& a, typename Store<S>::T& b) {
  if constexpr (std::is_same<S, double>::value) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
  } else if constexpr (std::is_same<S, float>::value) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    a = v.x;
    b = v.y;
  } else {
    const __half2 v = __ldg(reinterpret_cast<const __half2*>(p));
    a = __low2float(v) * float(Lattice<Q>::w(i));
    b = __high2float(v) * float(Lattice<Q>::w(i));
  }
}

template <class M, class S>
__global__ void __launch_bounds__(128) k_f2c(const F2CArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int Q = M::Q;
  constexpr int QS = Q * kCells;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = t & (kLanes - 1);
  const bool valid = (t / kLanes) < a.n;
  int g = valid ? t / kLanes : a.n - 1;
  const F2CLevel L = pick_level<F2CLevel>(a, g);
  const F2CItem& it = L.items[g];
  const int64_t base = int64_t(it.fblock[r]) * QS + it.fcell[r];
  const S* fs = reinterpret_cast<const S*>(L.f_src);
  T acc[Q];
  static_for<Q>([&](auto i) { acc[i] = T(0); });
  T accS = T(0);
  // add f_eq + r_fc (f - f_eq) of one child
  auto child = [&](const T (&g)[Q], T Sk) {
    T rl, ux, uy, uz;
    M::moments(g, rl, ux, uy, uz);
    T feq[Q];
    M::feq(rl, ux, uy, uz, feq);
    const T tf = T(L.tau0_f) + T(a.cs2_3) * Sk;
    const T tc = T(L.tau0_c) + T(a.cs2_3) * T(2) * Sk;
    const T rr = T(2) * (tc - T(1)) / (tf - T(1));
    static_for<Q>([&](auto i) { acc[i] += feq[i] + rr * (g[i] - feq[i]); });
    accS += T(2) * Sk;
  };
  {
    T g0[Q], g1[Q];
    static_for<Q>([&](auto i) { get_pair<S, Q, i>(fs + base + int(i) * kCells, g0[i], g1[i]); });
    T S0 = T(0), S1 = T(0);
    if (L.fa_src != nullptr) {
      const T* fa = reinterpret_cast<const T*>(L.fa_src) + int64_t(it.fblock[r]) * kCells + it.fcell[r];
      S0 = fa[0];
      S1 = fa[1];
    }
    child(g0, S0);
    child(g1, S1);
  }
  static_for<Q>([&](auto i) { acc[i] = quad_sum(acc[i]); });
  accS = quad_sum(accS);
  if (!valid) return;
  S* cd = reinterpret_cast<S*>(L.c_dst) + int64_t(it.cblock) * QS + it.ccell;
  static_for<Q>([&](auto i) {
    if ((int(i) & (kLanes - 1)) == r) St::template put<Q, i>(cd + int(i) * kCells, acc[i] / T(8));
  });
  if (L.ca_dst != nullptr && r == 0) reinterpret_cast<T*>(L.ca_dst)[int64_t(it.cblock) * kCells + it.ccell] = accS / T(8);
}

// Inflow: eight lanes per ghost cell, four cells per warp; lane r loads the
// source cell's populations r, r + 8, r + 16, r + 24 (the x-face cells are 8
// elements apart, so every value costs a sector however the lanes are laid
// out), the density is a sum over the eight lanes, and each lane writes its
// populations with e_x = +1.
constexpr int kBCLanes = 8;

template <class M, class S>
__global__ void __launch_bounds__(128) k_bc(const BCArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int Q = M::Q;
  constexpr int QS = Q * kCells;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = t & (kBCLanes - 1);
  const bool valid = (t / kBCLanes) < a.n;
  int n = valid ? t / kBCLanes : a.n - 1;  // tail lanes mirror the last cell
  const BCLevel L = pick_level<BCLevel>(a, n);
  const BCItem& it = L.items[n];
  S* f = reinterpret_cast<S*>(L.f);
  const S* src = f + int64_t(it.sblock) * QS + it.scell;
  S* dst = f + int64_t(it.gblock) * QS + it.gcell;
  constexpr int NJ = (Q + kBCLanes - 1) / kBCLanes;
  // density-like sum and momentum of the source cell (the momentum serves
  // the pressure outlet only)
  T part = T(0), jx = T(0), jy = T(0), jz = T(0);
  T gs[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int q = r + kBCLanes * j;
    const Lane<T, Q> ln(q);
    gs[j] = q < Q ? lane_load(src + q * kCells, ln) : T(0);
    part += gs[j];
    jx += T(ln.x) * gs[j];
    jy += T(ln.y) * gs[j];
    jz += T(ln.z) * gs[j];
  }
#pragma unroll
  for (int m = 1; m < kBCLanes; m <<= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, m);
    jx += __shfl_xor_sync(0xffffffffu, jx, m);
    jy += __shfl_xor_sync(0xffffffffu, jy, m);
    jz += __shfl_xor_sync(0xffffffffu, jz, m);
  }
  const T rl = part;
  // inflow: the disc test and the draws run in double on lanes 0..2 of the
  // group only (lane c computes velocity component c): FP64 throughput is
  // scarce on this part.  Every lane takes part in the shuffles (groups of
  // both item types may share a warp).
  T uc = T(0);
  if (it.type == 0 && r < 3 && !a.closed)
    uc = T(inflow_u(a.step, a.y0, a.z0, a.r2, a.u_in, a.perturb, a.seed, L.level, L.substep, L.NY, L.inv_scale,
                    it.y, it.z, r));
  const int g0 = int(threadIdx.x & 31) & ~(kBCLanes - 1);
  T ux = __shfl_sync(0xffffffffu, uc, g0);
  T uy = __shfl_sync(0xffffffffu, uc, g0 + 1);
  T uz = __shfl_sync(0xffffffffu, uc, g0 + 2);
  const bool outlet = it.type == 1;
  if (outlet) {
    // pressure outlet: the source cell's velocity, u_N = j / rho for the
    // compressible D3Q27 model, j for the incompressible D3Q19 model
    const T inv = M::Q == 19 ? T(1) : T(1) / (T(1) + rl);
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
  }
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int q = r + kBCLanes * j;
    if (q >= Q) continue;
    const Lane<T, Q> ln(q);
    if (!outlet && ln.x == 1) lane_store(dst + q * kCells, ln, lane_feq<M>(rl, ux, uy, uz, ln));
    // f_eq(rho_out, u_N) + f_N - f_eq(rho_N, u_N) for the populations pulled
    // into the domain (e_x = -1)
    if (outlet && ln.x == -1)
      lane_store(dst + q * kCells, ln,
                 gs[j] + (lane_feq<M>(T(a.rl_out), ux, uy, uz, ln) - lane_feq<M>(rl, ux, uy, uz, ln)));
  }
}

// Nozzle links (LinkItem): one thread per link.  The value is written into
// population ib of the solid cell, where the pull of the fluid cell takes it.
// Bouzidi linear interpolation (no-slip at fraction q of the link):
//   q <  1/2: 2q f~_i(f) + (1 - 2q) f~_i(f - e_i)   (f~_i(f) if f - e_i is solid)
//   q >= 1/2: f~_i(f) / (2q) + (2q - 1)/(2q) f~_ib(f)
// Both are affine with weights summing to 1 and w_i = w_ib, so they apply to
// the shifted storage values unchanged.  On the downstream cap: the inflow
// equilibrium with the density of the fluid cell straight downstream.
template <class M, class S>
__global__ void __launch_bounds__(128) k_links(const LinkArgs a) {
  using T = typename Store<S>::T;
  constexpr int Q = M::Q;
  constexpr int QS = Q * kCells;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n) return;
  const LinkItem it = a.items[t];
  S* f = reinterpret_cast<S*>(a.f);
  const int i = it.i, ib = it.ib;
  T v;
  if (it.type == 0) {
    const T q = T(it.q);
    const T fi = load_rt<S, Q>(f + int64_t(it.fblock) * QS + i * kCells + it.fcell, i);
    if (it.q < 0.5) {
      v = fi;
      if (it.sblock >= 0) {
        const T si = load_rt<S, Q>(f + int64_t(it.sblock) * QS + i * kCells + it.scell, i);
        v = T(2) * q * fi + (T(1) - T(2) * q) * si;
      }
    } else {
      const T fb = load_rt<S, Q>(f + int64_t(it.fblock) * QS + ib * kCells + it.fcell, ib);
      v = fi / (T(2) * q) + (T(2) * q - T(1)) / (T(2) * q) * fb;
    }
  } else {
    const S* s = f + int64_t(it.sblock) * QS + it.scell;
    T rl = T(0);
    for (int k = 0; k < Q; ++k) rl += load_rt<S, Q>(s + k * kCells, k);
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      u[c] = T(inflow_u(a.step, a.y0, a.z0, a.r2, a.u_in, a.perturb, a.seed, a.level, a.substep, a.NY, a.inv_scale,
                        it.y, it.z, c));
    v = lane_feq<M>(rl, u[0], u[1], u[2], Lane<T, Q>(ib));
  }
  store_rt<S, Q>(f + int64_t(it.bblock) * QS + ib * kCells + it.bcell, ib, v);
}

__global__ void k_step_inc(long long* step) { *step += 1; }

// coarse-to-fine: one CTA per chunk; fine-to-coarse: four lanes per item, 32
// items per CTA; inflow: eight lanes per item, 16 items per CTA
template <class M, class S>
static cudaError_t c2f_ms(const C2FArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_c2f<M, S><<<a.n, kC2FMaxItems, 0, st>>>(a);
  return cudaGetLastError();
}
template <class M, class S>
static cudaError_t f2c_ms(const F2CArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_f2c<M, S><<<(a.n + 31) / 32, 128, 0, st>>>(a);
  return cudaGetLastError();
}
template <class M, class S>
static cudaError_t links_ms(const LinkArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_links<M, S><<<(a.n + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}
template <class M, class S>
static cudaError_t bc_ms(const BCArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_bc<M, S><<<(a.n + 128 / kBCLanes - 1) / (128 / kBCLanes), 128, 0, st>>>(a);
  return cudaGetLastError();
}

#define LBM_DISPATCH(FN, ...)                                              \
  if (model == LBM_D3Q19_MRT_LES) {                                        \
    if (storage == LBM_F64) return FN<MrtLes, double>(__VA_ARGS__);        \
    if (storage == LBM_F32) return FN<MrtLes, float>(__VA_ARGS__);         \
    return FN<MrtLes, __half>(__VA_ARGS__);                                \
  }                                                                        \
  if (storage == LBM_F64) return FN<Fclb, double>(__VA_ARGS__);            \
  if (storage == LBM_F32) return FN<Fclb, float>(__VA_ARGS__);             \
  return FN<Fclb, __half>(__VA_ARGS__);

cudaError_t launch_c2f(int model, int storage, const C2FArgs& a, cudaStream_t st) { LBM_DISPATCH(c2f_ms, a, st) }
cudaError_t launch_f2c(int model, int storage, const F2CArgs& a, cudaStream_t st) { LBM_DISPATCH(f2c_ms, a, st) }
cudaError_t launch_bc(int model, int storage, const BCArgs& a, cudaStream_t st) { LBM_DISPATCH(bc_ms, a, st) }
cudaError_t launch_links(int model, int storage, const LinkArgs& a, cudaStream_t st) { LBM_DISPATCH(links_ms, a, st) }

cudaError_t launch_step_inc(long long* step, cudaStream_t st) {
  k_step_inc<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

}  // namespace lbm
