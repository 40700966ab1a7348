// Utility kernels: dense <-> block staging (state, equilibrium initialisation,
// macroscopic fields, body force), sampled gathers and the float64
// mass/momentum audit.
#include <cmath>

#include "collide.cuh"
#include "kernels.cuh"

namespace lbm {

template <int Q>
__device__ __forceinline__ double shift_of(int i) {
  return Q == 27 ? weight_rt<27>(i) : 0.0;  // D3Q19 stores the incompressible f itself
}

// locate dense level cell (x, y, z) in the level box; -1 if outside
__device__ __forceinline__ int64_t box_index(int x, int y, int z, int ox, int oy, int oz, int BX,
                                             int BY, int BZ) {
  const int bx = (x >> 3) - ox, by = (y >> 3) - oy, bz = (z >> 3) - oz;
  if (bx < 0 || bx >= BX || by < 0 || by >= BY || bz < 0 || bz >= BZ) return -1;
  return (int64_t(bx) + int64_t(BX) * (by + int64_t(BY) * bz)) * kCells + (x & 7) + 8 * (y & 7) +
         64 * (z & 7);
}

template <class M, class S>
__global__ void k_slab(const SlabArgs a) {
  using T = typename Store<S>::T;
  constexpr int Q = M::Q;
  const int64_t n = int64_t(a.NX) * a.NY * a.nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int x = int(t % a.NX), y = int((t / a.NX) % a.NY), z = a.z0 + int(t / (int64_t(a.NX) * a.NY));
  const int64_t j = box_index(x, y, z, a.ox, a.oy, a.oz, a.BX, a.BY, a.BZ);
  const int64_t blk = j >= 0 ? j / kCells : 0, cell = j >= 0 ? j % kCells : 0;
  S* f = reinterpret_cast<S*>(a.f) + blk * Q * kCells + cell;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  switch (a.mode) {
    case SLAB_SET_STATE: {
      if (j < 0) return;
      for (int i = 0; i < Q; ++i) {
        const double v = a.in[int64_t(i) * n + t];
        if (isnan(v)) continue;
        store_rt<S, Q>(f + i * kCells, i, T(v - shift_of<Q>(i)));
      }
      return;
    }
    case SLAB_GET_STATE: {
      for (int i = 0; i < Q; ++i)
        a.out[int64_t(i) * n + t] = j < 0 ? nan : double(load_rt<S, Q>(f + i * kCells, i)) + shift_of<Q>(i);
      return;
    }
    case SLAB_INIT_EQ: {
      if (j < 0) return;
      const T rl = T(a.in[t] - 1.0);  // delta rho for both shifted models
      const T ux = T(a.in[n + t]), uy = T(a.in[2 * n + t]), uz = T(a.in[3 * n + t]);
      T feq[Q];
      M::feq(rl, ux, uy, uz, feq);
      for (int i = 0; i < Q; ++i) store_rt<S, Q>(f + i * kCells, i, feq[i]);
      return;
    }
    case SLAB_MACRO: {
      const uint8_t k = j < 0 ? uint8_t(K_NONE) : a.kind[j];
      if (k != K_ACTIVE && k != K_HIDDEN1 && k != K_HIDDEN2) {
        for (int c = 0; c < 4; ++c) a.out[c * n + t] = nan;
        return;
      }
      double g[Q];
      for (int i = 0; i < Q; ++i) g[i] = double(load_rt<S, Q>(f + i * kCells, i));
      double rl = 0, jx = 0, jy = 0, jz = 0;
      static_for<Q>([&](auto i) {
        rl += g[i];
        jx += Lattice<Q>::ex(i) * g[i];
        jy += Lattice<Q>::ey(i) * g[i];
        jz += Lattice<Q>::ez(i) * g[i];
      });
      const double rho = 1.0 + rl;
      double ux = jx, uy = jy, uz = jz;
      if (Q == 27) {
        if (a.force != nullptr) {
          const int64_t nn = int64_t(a.BX) * a.BY * a.BZ * kCells;
          jx += 0.5 * a.force[j];
          jy += 0.5 * a.force[nn + j];
          jz += 0.5 * a.force[2 * nn + j];
        }
        ux = jx / rho;
        uy = jy / rho;
        uz = jz / rho;
      }
      a.out[t] = rho;
      a.out[n + t] = ux;
      a.out[2 * n + t] = uy;
      a.out[3 * n + t] = uz;
      return;
    }
    case SLAB_SET_LAMBDA: {
      if (j < 0) return;
      T* r = reinterpret_cast<T*>(a.raw) + blk * Q * kCells + cell;
      for (int i = 0; i < Q; ++i) r[i * kCells] = T(a.in[int64_t(i) * n + t]);
      return;
    }
    case SLAB_GET_FIELD3: {
      const int64_t nn = int64_t(a.BX) * a.BY * a.BZ * kCells;
      const T* r = reinterpret_cast<const T*>(a.raw);
      for (int c = 0; c < 3; ++c) a.out[c * n + t] = j < 0 ? nan : double(r[c * nn + j]);
      return;
    }
    case SLAB_GET_STATS: {
      // mean rho, u_x, u_y, u_z, then the variances <u_a^2> - <u_a>^2
      const uint8_t k = j < 0 ? uint8_t(K_NONE) : a.kind[j];
      const bool ok = k == K_ACTIVE || k == K_HIDDEN1 || k == K_HIDDEN2;
      const int64_t nn = int64_t(a.BX) * a.BY * a.BZ * kCells;
      const double* r = reinterpret_cast<const double*>(a.raw);
      for (int c = 0; c < 4; ++c) a.out[c * n + t] = ok ? r[c * nn + j] * a.scale : nan;
      for (int c = 0; c < 3; ++c) {
        const double m = ok ? r[(1 + c) * nn + j] * a.scale : 0.0;
        a.out[(4 + c) * n + t] = ok ? r[(4 + c) * nn + j] * a.scale - m * m : nan;
      }
      return;
    }
    case SLAB_GET_AUX: {
      a.out[t] = j < 0 ? nan : double(reinterpret_cast<const T*>(a.raw)[j]);
      return;
    }
    case SLAB_SET_AUX: {
      if (j < 0 || isnan(a.in[t])) return;
      reinterpret_cast<T*>(a.raw)[j] = T(a.in[t]);
      return;
    }
    case SLAB_SET_FORCE: {
      if (j < 0) return;
      const int64_t nn = int64_t(a.BX) * a.BY * a.BZ * kCells;
      for (int c = 0; c < 3; ++c) a.force[c * nn + j] = a.in[c * n + t];
      return;
    }
  }
}

template <class M, class S>
__global__ void k_gather(const GatherArgs a) {
  constexpr int Q = M::Q;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= a.n) return;
  const long long c = a.cells[t];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const long long ncell = (long long)a.NX * a.NY * a.NZ;
  int64_t j = -1;
  if (c >= 0 && c < ncell) {
    const int x = int(c % a.NX), y = int((c / a.NX) % a.NY), z = int(c / ((long long)a.NX * a.NY));
    j = box_index(x, y, z, a.ox, a.oy, a.oz, a.BX, a.BY, a.BZ);
  }
  const S* f = reinterpret_cast<const S*>(a.f) + (j >= 0 ? (j / kCells) * Q * kCells + j % kCells : 0);
  for (int i = 0; i < Q; ++i)
    a.out[t * Q + i] = j < 0 ? nan : double(load_rt<S, Q>(f + i * kCells, i)) + shift_of<Q>(i);
}

// Float64 sums over active cells: (delta rho, j_x, j_y, j_z) times vol.
//
// Each thread first sums every population separately over its cells,
// S_i = sum_cells g_i, and forms delta rho = sum_i S_i and j_a = sum_i e_ia S_i
// only at the end: Q float64 additions per cell instead of one per non-zero
// term of the four sums (81 for D3Q27), which matters on a part whose
// float64 rate is a small fraction of its float32 rate.  For float32 and
// float16 storage the per-population sums run in float32 pairs (s, e) by
// Knuth's TwoSum, s + e being the sum of up to kFlush values with the
// rounding of each addition kept in e, and every kFlush cells (inactive
// ones adding zeros) both are added to the float64 sum.  The pair's error
// over m values is below about m^2 u^2 sum |g| (u = 2^-24), 4e-12 of sum |g|
// for m = 32, the order of the bound of plain float64 recursive summation
// over a thread's values; the float64 work (two conversions and two
// additions per population and flush) is what limits the kernel on GB300.
// The populations are taken in chunks (registers), each chunk one pass over
// the thread's cells.
constexpr int kFlush = 32;
constexpr int kReduceUnroll = 4;  // cells per iteration, their loads issued together

template <class M, class S>
__global__ void __launch_bounds__(256, reduce_ctas_per_sm(std::is_same<S, __half>::value ? LBM_F16 : LBM_F32))
    k_reduce(const ReduceArgs a) {
  constexpr int Q = M::Q;
  constexpr int P = Q == 19 ? 10 : 9;  // populations per pass
  constexpr int NP = (Q + P - 1) / P;
  constexpr int U = kReduceUnroll;
  constexpr bool kPair = !std::is_same<S, double>::value;
  using V = typename std::conditional<kPair, float, double>::type;
  double s[4] = {0, 0, 0, 0};
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  static_for<NP>([&](auto pass) {
    constexpr int i0 = int(pass) * P;
    constexpr int n = (Q - i0) < P ? (Q - i0) : P;
    double D[n];
    float hs[n], he[n];
    static_for<n>([&](auto k) {
      D[k] = 0.0;
      hs[k] = 0.f;
      he[k] = 0.f;
    });
    [[maybe_unused]] int m = 0;  // cells since the last flush (float pairs only)
    for (int64_t t = t0; t < a.ncells; t += U * stride) {
      // U cells t, t + stride, ...: every value and kind loaded at once (the
      // values unconditionally: every cell of the box has storage, so no
      // load waits for a kind), then inactive cells select zeros
      S raw[U][n];
      bool on[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t tt = t + u * stride;
        const int64_t tc = tt < a.ncells ? tt : a.ncells - 1;
        const S* f = reinterpret_cast<const S*>(a.f) + (tc / kCells) * Q * kCells + tc % kCells;
        static_for<n>([&](auto k) { raw[u][k] = f[(i0 + int(k)) * kCells]; });
        on[u] = tt < a.ncells && a.kind[tc] == K_ACTIVE;
      }
      V v[U][n];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        static_for<n>([&](auto k) {
          [[maybe_unused]] constexpr int i = i0 + int(k);
          if constexpr (std::is_same<S, __half>::value)
            // the stored value as the collision sees it: the product h w
            // rounded to float (__fmul_rn keeps it from being fused into
            // the addition below, which would sum unrounded products)
            v[u][k] = on[u] ? __fmul_rn(__half2float(raw[u][k]), float(Lattice<Q>::w(i))) : 0.f;
          else
            v[u][k] = on[u] ? V(raw[u][k]) : V(0);
        });
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        static_for<n>([&](auto k) {
          if constexpr (!kPair) {
            D[k] += v[u][k];
          } else {
            // TwoSum: x = hs + g exactly equals x + r
            const float g = v[u][k];
            const float x = hs[k] + g;
            const float b = x - hs[k];
            const float r = (hs[k] - (x - b)) + (g - b);
            hs[k] = x;
            he[k] += r;
          }
        });
      }
      if constexpr (kPair) {
        m += U;
        if (m >= kFlush) {
          static_for<n>([&](auto k) {
            D[k] += double(hs[k]);
            D[k] += double(he[k]);
            hs[k] = 0.f;
            he[k] = 0.f;
          });
          m = 0;
        }
      }
    }
    static_for<n>([&](auto k) {
      constexpr int i = i0 + int(k);
      const double Si = kPair ? (D[k] + double(hs[k])) + double(he[k]) : D[k];
      s[0] += Si;
      if constexpr (Lattice<Q>::ex(i) != 0) s[1] += Lattice<Q>::ex(i) > 0 ? Si : -Si;
      if constexpr (Lattice<Q>::ey(i) != 0) s[2] += Lattice<Q>::ey(i) > 0 ? Si : -Si;
      if constexpr (Lattice<Q>::ez(i) != 0) s[3] += Lattice<Q>::ez(i) > 0 ? Si : -Si;
    });
  });
  __shared__ double sh[4][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double v = s[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    a.partial[blockIdx.x * 4 + threadIdx.x] = v * a.vol;
  }
}

__global__ void k_reduce_final(const double* partial, int n, double* out, int* nonfinite) {
  if (threadIdx.x < 4) {
    double v = 0;
    for (int i = 0; i < n; ++i) v += partial[i * 4 + threadIdx.x];
    out[threadIdx.x] = v;
    if (!isfinite(v)) atomicExch(nonfinite, 1);
  }
}

template <class M, class S>
static cudaError_t slab_ms(const SlabArgs& a, cudaStream_t st) {
  const int64_t n = int64_t(a.NX) * a.NY * a.nz;
  if (n == 0) return cudaSuccess;
  k_slab<M, S><<<unsigned((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}
template <class M, class S>
static cudaError_t gather_ms(const GatherArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_gather<M, S><<<unsigned((a.n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}
template <class M, class S>
static cudaError_t reduce_ms(const ReduceArgs& a, int ctas, cudaStream_t st) {
  k_reduce<M, S><<<ctas, 256, 0, st>>>(a);
  return cudaGetLastError();
}

#define LBM_DISPATCH(FN, ...)                                       \
  if (model == LBM_D3Q19_MRT_LES) {                                 \
    if (storage == LBM_F64) return FN<MrtLes, double>(__VA_ARGS__); \
    if (storage == LBM_F32) return FN<MrtLes, float>(__VA_ARGS__);  \
    return FN<MrtLes, __half>(__VA_ARGS__);                         \
  }                                                                 \
  if (storage == LBM_F64) return FN<Fclb, double>(__VA_ARGS__);     \
  if (storage == LBM_F32) return FN<Fclb, float>(__VA_ARGS__);      \
  return FN<Fclb, __half>(__VA_ARGS__);

cudaError_t launch_slab(int model, int storage, const SlabArgs& a, cudaStream_t st) { LBM_DISPATCH(slab_ms, a, st) }
cudaError_t launch_gather(int model, int storage, const GatherArgs& a, cudaStream_t st) { LBM_DISPATCH(gather_ms, a, st) }
cudaError_t launch_reduce(int model, int storage, const ReduceArgs& a, int ctas, cudaStream_t st) {
  LBM_DISPATCH(reduce_ms, a, ctas, st)
}
__global__ void k_fill(double* p, long long n, double v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p[t] = v;
}
// one sample of the time statistics: rho and u of every cell holding a value
// of the level (the same moments as the macroscopic output), accumulated in
// float64
template <class M, class S>
__global__ void k_stats(const StatsArgs a) {
  constexpr int Q = M::Q;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= a.ncells) return;
  const uint8_t k = a.kind[j];
  if (k != K_ACTIVE && k != K_HIDDEN1 && k != K_HIDDEN2) return;
  const S* f = reinterpret_cast<const S*>(a.f) + (j / kCells) * Q * kCells + (j % kCells);
  double g[Q];
  for (int i = 0; i < Q; ++i) g[i] = double(load_rt<S, Q>(f + i * kCells, i));
  double rl = 0, jx = 0, jy = 0, jz = 0;
  static_for<Q>([&](auto i) {
    rl += g[i];
    jx += Lattice<Q>::ex(i) * g[i];
    jy += Lattice<Q>::ey(i) * g[i];
    jz += Lattice<Q>::ez(i) * g[i];
  });
  const double rho = 1.0 + rl;
  double ux = jx, uy = jy, uz = jz;
  if (Q == 27) {
    ux = jx / rho;
    uy = jy / rho;
    uz = jz / rho;
  }
  const double v[7] = {rho, ux, uy, uz, ux * ux, uy * uy, uz * uz};
  for (int c = 0; c < 7; ++c) a.sums[c * a.ncells + j] += v[c];
}

__global__ void k_radial(const RadialArgs a) {
  const int64_t per = int64_t(a.NY) * a.NZ;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= per * a.nst) return;
  const int s = int(t / per);
  const int y = int(t % a.NY), z = int((t % per) / a.NY);
  const int64_t j = box_index(a.xs[s], y, z, a.ox, a.oy, a.oz, a.BX, a.BY, a.BZ);
  if (j < 0) return;
  const uint8_t k = a.kind[j];
  if (k != K_ACTIVE && (a.active_only || (k != K_HIDDEN1 && k != K_HIDDEN2))) return;
  const double dy = (y + 0.5) * a.inv_scale - a.y0, dz = (z + 0.5) * a.inv_scale - a.z0;
  const double r = sqrt(__dadd_rn(__dmul_rn(dy, dy), __dmul_rn(dz, dz)));
  // compare before converting: r / dr may exceed the int range (tiny dr)
  const double rb = floor(r / a.dr);
  if (!(rb < double(a.nbins))) return;
  const int b = int(rb);
  const int64_t nn = int64_t(a.BX) * a.BY * a.BZ * kCells;
  const double m = a.sums[nn + j] * a.scale;
  const double v = a.sums[4 * nn + j] * a.scale - m * m;
  const int64_t o = int64_t(s) * a.nbins + b;
  atomicAdd(a.acc + 3 * o, a.weight * m);
  atomicAdd(a.acc + 3 * o + 1, a.weight * v);
  atomicAdd(a.acc + 3 * o + 2, a.weight);
  atomicAdd(a.cnt + o, 1ull);
}

cudaError_t launch_radial(const RadialArgs& a, cudaStream_t st) {
  const int64_t n = int64_t(a.NY) * a.NZ * a.nst;
  if (n == 0) return cudaSuccess;
  k_radial<<<unsigned((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <class M, class S>
static cudaError_t stats_ms(const StatsArgs& a, cudaStream_t st) {
  if (a.ncells == 0) return cudaSuccess;
  k_stats<M, S><<<unsigned((a.ncells + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stats(int model, int storage, const StatsArgs& a, cudaStream_t st) {
  if (model == LBM_D3Q19_MRT_LES) {
    if (storage == LBM_F64) return stats_ms<MrtLes, double>(a, st);
    if (storage == LBM_F32) return stats_ms<MrtLes, float>(a, st);
    return stats_ms<MrtLes, __half>(a, st);
  }
  if (storage == LBM_F64) return stats_ms<Fclb, double>(a, st);
  if (storage == LBM_F32) return stats_ms<Fclb, float>(a, st);
  return stats_ms<Fclb, __half>(a, st);
}

__global__ void k_to_float(const double* in, float* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = float(in[i]);
}

cudaError_t launch_to_float(const double* in, float* out, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_to_float<<<unsigned((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_fill<<<unsigned((n + 255) / 256), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_reduce_final(const double* partial, int n, double* out, int* nonfinite, cudaStream_t st) {
  k_reduce_final<<<1, 32, 0, st>>>(partial, n, out, nonfinite);
  return cudaGetLastError();
}

}  // namespace lbm
