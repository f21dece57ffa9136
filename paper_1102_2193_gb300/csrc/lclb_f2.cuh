// lclb_f2.cuh -- two FP32 values (two neighbouring lattice nodes) computed
// together by the packed FP32x2 instructions of sm_100+ (add, multiply and
// fused multiply-add on a register pair: one issue slot for two results).
//
// A product is kept unrounded (f2mul) until it is added to or subtracted from
// another value, where it becomes one fused multiply-add, so that expressions
// written as a * b + c compile to the packed FMA as scalar FP32 code compiles
// to FFMA.  Every result is rounded as the corresponding scalar operation
// (fused multiply-add: one rounding).
#pragma once
#include <cuda_runtime.h>

namespace lclb {

struct f2 {
  float2 v;
  f2() = default;
  __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit f2(float2 w) : v(w) {}
};

struct f2mul {
  float2 a, b;
  __device__ __forceinline__ operator f2() const { return f2(__fmul2_rn(a, b)); }
};

__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }

__device__ __forceinline__ f2mul operator*(f2 a, f2 b) { return {a.v, b.v}; }
__device__ __forceinline__ f2mul operator*(float a, f2 b) { return {make_float2(a, a), b.v}; }
__device__ __forceinline__ f2mul operator*(f2 a, float b) { return {a.v, make_float2(b, b)}; }
__device__ __forceinline__ f2mul operator*(f2mul a, f2 b) { return {__fmul2_rn(a.a, a.b), b.v}; }
__device__ __forceinline__ f2mul operator*(f2 a, f2mul b) { return {a.v, __fmul2_rn(b.a, b.b)}; }
__device__ __forceinline__ f2mul operator*(f2mul a, float b) { return {__fmul2_rn(a.a, a.b), make_float2(b, b)}; }
__device__ __forceinline__ f2mul operator*(float a, f2mul b) { return {make_float2(a, a), __fmul2_rn(b.a, b.b)}; }
__device__ __forceinline__ f2mul operator*(f2mul a, f2mul b) { return {__fmul2_rn(a.a, a.b), __fmul2_rn(b.a, b.b)}; }

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator+(f2mul m, f2 c) { return f2(__ffma2_rn(m.a, m.b, c.v)); }
__device__ __forceinline__ f2 operator+(f2 c, f2mul m) { return f2(__ffma2_rn(m.a, m.b, c.v)); }
__device__ __forceinline__ f2 operator+(f2mul m, f2mul n) { return f2(__ffma2_rn(m.a, m.b, __fmul2_rn(n.a, n.b))); }
__device__ __forceinline__ f2 operator+(f2 a, float b) { return a + f2(b); }
__device__ __forceinline__ f2 operator+(float a, f2 b) { return f2(a) + b; }
__device__ __forceinline__ f2 operator+(f2mul m, float c) { return m + f2(c); }
__device__ __forceinline__ f2 operator+(float c, f2mul m) { return m + f2(c); }

__device__ __forceinline__ f2 operator-(f2 a) { return f2(neg2(a.v)); }
__device__ __forceinline__ f2mul operator-(f2mul m) { return {neg2(m.a), m.b}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ f2 operator-(f2mul m, f2 c) { return f2(__ffma2_rn(m.a, m.b, neg2(c.v))); }
__device__ __forceinline__ f2 operator-(f2 c, f2mul m) { return f2(__ffma2_rn(neg2(m.a), m.b, c.v)); }
__device__ __forceinline__ f2 operator-(f2mul m, f2mul n) { return f2(__ffma2_rn(m.a, m.b, neg2(__fmul2_rn(n.a, n.b)))); }
__device__ __forceinline__ f2 operator-(f2 a, float b) { return a - f2(b); }
__device__ __forceinline__ f2 operator-(float a, f2 b) { return f2(a) - b; }
__device__ __forceinline__ f2 operator-(f2mul m, float c) { return m - f2(c); }
__device__ __forceinline__ f2 operator-(float c, f2mul m) { return f2(c) - m; }

}  // namespace lclb
