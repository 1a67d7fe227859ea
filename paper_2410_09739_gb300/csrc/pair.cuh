// pair.cuh -- two cells per thread on the packed fp32 pipe.
//
// sm_100-class GPUs execute fma/add/mul on a pair of fp32 values as one
// instruction (fma.rn.f32x2 and friends).  The collision of two cells is the
// same instruction stream on different data, so a thread that collides two
// cells at once with `f2` arithmetic issues about half the floating-point
// instructions per cell.  Every operation is the IEEE round-to-nearest fp32
// operation on each lane: results equal two scalar collisions up to
// contraction choices (a*b+c written with fma on one side and not the other).
//
// f2 supplies what collide_cell needs from its arithmetic type R: + - * and
// unary minus, fmaR, construction from a constant, 1/x, and a comparison that
// is true only when it holds on both lanes (collide_cell's validity check).
#pragma once
#include <cuda_runtime.h>

namespace fpc {

struct f2 {
    float2 v;
    f2() = default;
    __host__ __device__ constexpr f2(float2 a) : v(a) {}
    __host__ __device__ constexpr f2(double c) : v{(float)c, (float)c} {}
    __host__ __device__ constexpr f2(float x, float y) : v{x, y} {}
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2 operator/(f2 a, f2 b) { return f2(make_float2(a.v.x / b.v.x, a.v.y / b.v.y)); }
__device__ __forceinline__ bool operator>(f2 a, f2 b) { return a.v.x > b.v.x && a.v.y > b.v.y; }
__device__ __forceinline__ bool operator<(f2 a, f2 b) { return a.v.x < b.v.x && a.v.y < b.v.y; }
// overloads of collide.cuh's fmaR, fminR, fmaxR (a non-template exact match wins for f2)
__device__ __forceinline__ f2 fminR(f2 a, f2 b) { return f2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ f2 fmaxR(f2 a, f2 b) { return f2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
__device__ __forceinline__ f2 fmaR(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }

}  // namespace fpc
