// A pair of FP32 values, one per node of a two-node thread, computed with
// the packed FP32 instructions of sm_100 and later (add, mul and fma on
// .f32x2): one instruction updates both nodes, which halves the issue slots
// of the per-node arithmetic. The per-node code (moment transforms,
// equilibria, collision) is written once, templated on its compute type, and
// runs unchanged on F2.
//
// A product a * b is kept pending (P2) until it is used: added to or
// subtracted from a value it becomes one fused multiply-add, as the scalar
// compiler contracts a * b + c; used any other way it becomes a multiply.
// Each lane rounds exactly as the scalar FP32 code with the same
// contractions would.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct P2;

struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float2 x) : v(x) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ F2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ F2(double a) : F2((float)a) {}
    __device__ __forceinline__ F2(int a) : F2((float)a) {}
    __device__ __forceinline__ F2(const P2& p);
};

struct P2 {
    float2 a, b;
};

__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ F2::F2(const P2& p) : v(__fmul2_rn(p.a, p.b)) {}

__device__ __forceinline__ P2 operator*(F2 a, F2 b) { return {a.v, b.v}; }
__device__ __forceinline__ P2 operator*(const P2& a, F2 b) { return {F2(a).v, b.v}; }
__device__ __forceinline__ P2 operator*(F2 a, const P2& b) { return {a.v, F2(b).v}; }
__device__ __forceinline__ P2 operator*(const P2& a, const P2& b) { return {F2(a).v, F2(b).v}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return __fadd2_rn(a.v, b.v); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return __fadd2_rn(a.v, neg2(b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return neg2(a.v); }
__device__ __forceinline__ P2 operator-(const P2& p) { return {neg2(p.a), p.b}; }

__device__ __forceinline__ F2 operator+(const P2& p, F2 c) { return __ffma2_rn(p.a, p.b, c.v); }
__device__ __forceinline__ F2 operator+(F2 c, const P2& p) { return __ffma2_rn(p.a, p.b, c.v); }
__device__ __forceinline__ F2 operator+(const P2& p, const P2& q) { return __ffma2_rn(p.a, p.b, F2(q).v); }
__device__ __forceinline__ F2 operator-(const P2& p, F2 c) { return __ffma2_rn(p.a, p.b, neg2(c.v)); }
__device__ __forceinline__ F2 operator-(F2 c, const P2& p) { return __ffma2_rn(neg2(p.a), p.b, c.v); }
__device__ __forceinline__ F2 operator-(const P2& p, const P2& q) { return __ffma2_rn(p.a, p.b, neg2(F2(q).v)); }

__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator+=(F2& a, const P2& p) { return a = a + p; }
__device__ __forceinline__ F2& operator-=(F2& a, const P2& p) { return a = a - p; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = F2(a * b); }

// the scalar helpers of the per-node code, lane by lane
__device__ __forceinline__ F2 recip(F2 x) { return F2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y)); }
__device__ __forceinline__ F2 clamp01(F2 w) {
    const float a = w.v.x, b = w.v.y;
    return F2(a < 0.f ? 0.f : (a > 1.f ? 1.f : a), b < 0.f ? 0.f : (b > 1.f ? 1.f : b));
}
// m / 9 with the constant split into its FP32 rounding and the remainder
// (the pair form of the scalar ninth())
__device__ __forceinline__ F2 ninth(F2 m) {
    constexpr float hi = (float)(1.0 / 9.0);
    constexpr float lo = (float)(1.0 / 9.0 - (double)(float)(1.0 / 9.0));
    return __ffma2_rn(m.v, make_float2(hi, hi), __fmul2_rn(m.v, make_float2(lo, lo)));
}

}  // namespace lbm
