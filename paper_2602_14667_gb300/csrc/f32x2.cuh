// f32x2.cuh -- two FP32 lanes as one value, for the collision of a pair of
// nodes on the packed FP32 instructions of sm_100 and later (one FFMA2 /
// FADD2 / FMUL2 does the work of two scalar instructions).
//
// F2 carries node k in .x and node k+1 in .y.  Products are kept unevaluated
// (F2Mul) until they meet an addition or a subtraction, where they become
// one fused multiply-add, so that `a * b + c` costs one packed instruction
// as it costs one FFMA per node in scalar code.  Every lane is rounded as
// IEEE single precision (round to nearest even); the pairing changes which
// products are fused, so results may differ from the scalar evaluation in
// the last bit.  F1 below is the one-lane form with the same rounding.
#pragma once

#include <cuda_runtime.h>

namespace mhd {

struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ explicit F2(float2 a) : v(a) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    // broadcast of a constant or a per-lattice parameter
    __device__ __forceinline__ explicit F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit F2(double s) : F2((float)s) {}
    __device__ __forceinline__ explicit F2(int s) : F2((float)s) {}
};

struct F2Mul {
    F2 a, b;
    __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a.v, b.v)); }
};

__device__ __forceinline__ F2 neg(F2 x) { return F2(-x.v.x, -x.v.y); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

__device__ __forceinline__ F2Mul operator*(F2 a, F2 b) { return F2Mul{a, b}; }
__device__ __forceinline__ F2Mul operator*(F2Mul m, F2 b) { return F2Mul{F2(m), b}; }
__device__ __forceinline__ F2Mul operator*(F2 a, F2Mul m) { return F2Mul{a, F2(m)}; }
__device__ __forceinline__ F2Mul operator*(F2Mul m, F2Mul n) { return F2Mul{F2(m), F2(n)}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
// a - b as b * (-1) + a: exact negation, one rounding, i.e. IEEE subtraction
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return fma2(b, F2(-1.0f), a); }
__device__ __forceinline__ F2 operator-(F2 a) { return neg(a); }

__device__ __forceinline__ F2 operator+(F2Mul m, F2 c) { return fma2(m.a, m.b, c); }
__device__ __forceinline__ F2 operator+(F2 c, F2Mul m) { return fma2(m.a, m.b, c); }
__device__ __forceinline__ F2 operator+(F2Mul m, F2Mul n) { return fma2(m.a, m.b, F2(n)); }
__device__ __forceinline__ F2 operator-(F2Mul m, F2 c) { return fma2(m.a, m.b, neg(c)); }
__device__ __forceinline__ F2 operator-(F2 c, F2Mul m) { return fma2(neg(m.a), m.b, c); }
__device__ __forceinline__ F2 operator-(F2Mul m, F2Mul n) { return fma2(m.a, m.b, neg(F2(n))); }
__device__ __forceinline__ F2Mul operator-(F2Mul m) { return F2Mul{neg(m.a), m.b}; }

__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator+=(F2& a, F2Mul m) { return a = a + m; }
__device__ __forceinline__ F2& operator-=(F2& a, F2Mul m) { return a = a - m; }

// lane by lane, IEEE division as in scalar code
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }

// One FP32 lane with exactly the fusion rules of F2: a product fuses into
// the addition or subtraction it meets (__fmaf_rn) and is otherwise rounded
// on its own (__fmul_rn / __fadd_rn are never contracted by the compiler).
// A collision evaluated on F1 is therefore bitwise that of the same node in
// an F2 pair, at the register cost of scalar code.
struct F1 {
    float v;
    F1() = default;
    __device__ __forceinline__ explicit F1(float s) : v(s) {}
    __device__ __forceinline__ explicit F1(double s) : v((float)s) {}
    __device__ __forceinline__ explicit F1(int s) : v((float)s) {}
};

struct F1Mul {
    F1 a, b;
    __device__ __forceinline__ operator F1() const { return F1(__fmul_rn(a.v, b.v)); }
};

__device__ __forceinline__ F1 neg(F1 x) { return F1(-x.v); }
__device__ __forceinline__ F1 fma1(F1 a, F1 b, F1 c) { return F1(__fmaf_rn(a.v, b.v, c.v)); }

__device__ __forceinline__ F1Mul operator*(F1 a, F1 b) { return F1Mul{a, b}; }
__device__ __forceinline__ F1Mul operator*(F1Mul m, F1 b) { return F1Mul{F1(m), b}; }
__device__ __forceinline__ F1Mul operator*(F1 a, F1Mul m) { return F1Mul{a, F1(m)}; }
__device__ __forceinline__ F1Mul operator*(F1Mul m, F1Mul n) { return F1Mul{F1(m), F1(n)}; }

__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return fma1(b, F1(-1.0f), a); }
__device__ __forceinline__ F1 operator-(F1 a) { return neg(a); }

__device__ __forceinline__ F1 operator+(F1Mul m, F1 c) { return fma1(m.a, m.b, c); }
__device__ __forceinline__ F1 operator+(F1 c, F1Mul m) { return fma1(m.a, m.b, c); }
__device__ __forceinline__ F1 operator+(F1Mul m, F1Mul n) { return fma1(m.a, m.b, F1(n)); }
__device__ __forceinline__ F1 operator-(F1Mul m, F1 c) { return fma1(m.a, m.b, neg(c)); }
__device__ __forceinline__ F1 operator-(F1 c, F1Mul m) { return fma1(neg(m.a), m.b, c); }
__device__ __forceinline__ F1 operator-(F1Mul m, F1Mul n) { return fma1(m.a, m.b, neg(F1(n))); }
__device__ __forceinline__ F1Mul operator-(F1Mul m) { return F1Mul{neg(m.a), m.b}; }

__device__ __forceinline__ F1& operator+=(F1& a, F1 b) { return a = a + b; }
__device__ __forceinline__ F1& operator-=(F1& a, F1 b) { return a = a - b; }
__device__ __forceinline__ F1& operator+=(F1& a, F1Mul m) { return a = a + m; }
__device__ __forceinline__ F1& operator-=(F1& a, F1Mul m) { return a = a - m; }

__device__ __forceinline__ F1 operator/(F1 a, F1 b) { return F1(a.v / b.v); }

}  // namespace mhd
