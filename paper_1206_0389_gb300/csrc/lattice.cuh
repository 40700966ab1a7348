// Lattice tables for the device code: D3Q19 and D3Q27 velocity sets in the
// column order of the paper's Section 2 tables, and their weights
// (1/3, 1/18, 1/36 and 8/27, 2/27, 1/54, 1/216 by |e|^2).  Every accessor is
// constexpr so the kernels see compile-time constants after unrolling.
#pragma once
#include <cstdint>
#include <utility>

namespace lbm {

// D3Q27 table (Section 2, parts i = 0..15 and i = 16..26); D3Q19 is its
// first 19 columns.
__host__ __device__ constexpr int ex27(int i) {
  constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0,
                         0, 0, 0, 1, -1, 1, 1, -1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int ey27(int i) {
  constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1,
                         -1, 1, -1, 1, 1, -1, 1, -1, 1, -1, -1};
  return t[i];
}
__host__ __device__ constexpr int ez27(int i) {
  constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1,
                         -1, -1, 1, 1, 1, 1, -1, 1, -1, -1, -1};
  return t[i];
}

template <int Q_>
struct Lattice {
  static constexpr int Q = Q_;
  __host__ __device__ static constexpr int ex(int i) { return ex27(i); }
  __host__ __device__ static constexpr int ey(int i) { return ey27(i); }
  __host__ __device__ static constexpr int ez(int i) { return ez27(i); }
  __host__ __device__ static constexpr int norm2(int i) {
    return ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i);
  }
  __host__ __device__ static constexpr double w(int i) {
    return Q == 19 ? (norm2(i) == 0 ? 1.0 / 3.0 : norm2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0)
                   : (norm2(i) == 0   ? 8.0 / 27.0
                      : norm2(i) == 1 ? 2.0 / 27.0
                      : norm2(i) == 2 ? 1.0 / 54.0
                                      : 1.0 / 216.0);
  }
  // index of the velocity (x, y, z), -1 if absent
  __host__ __device__ static constexpr int index(int x, int y, int z) {
    for (int i = 0; i < Q; ++i)
      if (ex(i) == x && ey(i) == y && ez(i) == z) return i;
    return -1;
  }
};

using D3Q19 = Lattice<19>;
using D3Q27 = Lattice<27>;

// compile-time integer usable as a constant expression in device code
template <int I>
struct Int {
  static constexpr int value = I;
  __host__ __device__ constexpr operator int() const { return I; }
};

// compile-time loop: f(Int<i>) for i = 0..N-1
template <class F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(Int<Is>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

}  // namespace lbm
