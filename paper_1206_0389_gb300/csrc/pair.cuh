// Two-cell arithmetic for the FP16-storage stream-collide kernel.
//
// V2 holds one float per cell of an x-adjacent cell pair.  Its operators map
// onto Blackwell's packed FP32x2 instructions (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: one instruction for both cells), so the collision of two cells
// issues about as many FP32 instructions as that of one.  A product is kept
// unevaluated (P2) until it meets an addition, which then becomes one fused
// multiply-add rounded once, as the compiler would contract a*b + c in
// scalar code.  Division and square root act per component.
#pragma once
#include <cuda_fp16.h>

namespace lbm {

struct V2 {
  float x, y;
  __host__ __device__ constexpr V2() : x(0.f), y(0.f) {}
  __host__ __device__ constexpr V2(double d) : x(float(d)), y(float(d)) {}
  __host__ __device__ constexpr V2(float a, float b) : x(a), y(b) {}
  __device__ __forceinline__ float2 f2() const { return make_float2(x, y); }
  __device__ __forceinline__ static V2 of(float2 v) { return V2(v.x, v.y); }
};

// a pending product a * b
struct P2 {
  V2 a, b;
  __device__ __forceinline__ operator V2() const { return V2::of(__fmul2_rn(a.f2(), b.f2())); }
};

__device__ __forceinline__ V2 operator-(V2 a) { return V2(-a.x, -a.y); }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2::of(__fadd2_rn(a.f2(), b.f2())); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2::of(__fadd2_rn(a.f2(), (-b).f2())); }
__device__ __forceinline__ P2 operator*(V2 a, V2 b) { return P2{a, b}; }
__device__ __forceinline__ P2 operator*(P2 a, V2 b) { return P2{V2(a), b}; }
__device__ __forceinline__ P2 operator*(V2 a, P2 b) { return P2{a, V2(b)}; }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2{V2(a), V2(b)}; }
__device__ __forceinline__ P2 operator-(P2 a) { return P2{-a.a, a.b}; }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return V2::of(__ffma2_rn(a.f2(), b.f2(), c.f2())); }
__device__ __forceinline__ V2 operator+(P2 p, V2 c) { return fma2(p.a, p.b, c); }
__device__ __forceinline__ V2 operator+(V2 c, P2 p) { return fma2(p.a, p.b, c); }
__device__ __forceinline__ V2 operator-(P2 p, V2 c) { return fma2(p.a, p.b, -c); }
__device__ __forceinline__ V2 operator-(V2 c, P2 p) { return fma2(-p.a, p.b, c); }
__device__ __forceinline__ V2 operator+(P2 p, P2 q) { return fma2(p.a, p.b, V2(q)); }
__device__ __forceinline__ V2 operator-(P2 p, P2 q) { return fma2(p.a, p.b, -V2(q)); }
__device__ __forceinline__ V2 operator/(V2 a, V2 b) { return V2(a.x / b.x, a.y / b.y); }
__device__ __forceinline__ V2 operator/(P2 a, V2 b) { return V2(a) / b; }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) { return a = a + b; }
__device__ __forceinline__ V2& operator+=(V2& a, P2 b) { return a = b + a; }
__device__ __forceinline__ V2& operator-=(V2& a, V2 b) { return a = a - b; }
__device__ __forceinline__ V2& operator*=(V2& a, V2 b) { return a = V2(a * b); }
__device__ __forceinline__ V2 sqrt(V2 a) { return V2(sqrtf(a.x), sqrtf(a.y)); }

}  // namespace lbm
