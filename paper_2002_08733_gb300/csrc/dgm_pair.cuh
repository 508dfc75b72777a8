// Column-pair arithmetic for the paired stage kernel (dgm_stage2.cuh): each
// thread advances two columns at once, so that every coefficient of the
// generated reference operators and every piece of control flow and address
// arithmetic serves two elements.
//   F2x: the pair in a float2, arithmetic with the packed FP32x2 instructions
//        of sm_100+ (__ffma2_rn, __fadd2_rn, __fmul2_rn);
//   P2:  the pair as two floats with scalar arithmetic.
#pragma once

#include <cuda_runtime.h>

namespace dgm {

struct F2x {
    float2 v;
    __device__ __forceinline__ F2x() {}
    __device__ __forceinline__ F2x(double a) : v(make_float2(float(a), float(a))) {}
    __device__ __forceinline__ F2x(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ float a() const { return v.x; }
    __device__ __forceinline__ float b() const { return v.y; }
};
__device__ __forceinline__ F2x operator+(F2x x, F2x y) { F2x r; r.v = __fadd2_rn(x.v, y.v); return r; }
__device__ __forceinline__ F2x operator*(F2x x, F2x y) { F2x r; r.v = __fmul2_rn(x.v, y.v); return r; }
__device__ __forceinline__ F2x operator-(F2x x, F2x y) {
    F2x r;
    r.v = __ffma2_rn(y.v, make_float2(-1.f, -1.f), x.v);
    return r;
}
__device__ __forceinline__ F2x operator-(F2x x) { F2x r; r.v = __fmul2_rn(x.v, make_float2(-1.f, -1.f)); return r; }
__device__ __forceinline__ F2x& operator+=(F2x& x, F2x y) { x = x + y; return x; }
__device__ __forceinline__ F2x& operator-=(F2x& x, F2x y) { x = x - y; return x; }
__device__ __forceinline__ F2x& operator*=(F2x& x, F2x y) { x = x * y; return x; }
__device__ __forceinline__ F2x fmaa(F2x a, F2x b, F2x c) { F2x r; r.v = __ffma2_rn(a.v, b.v, c.v); return r; }

struct P2 {
    float x, y;
    __device__ __forceinline__ P2() {}
    __device__ __forceinline__ P2(double a) : x(float(a)), y(float(a)) {}
    __device__ __forceinline__ P2(float a, float b) : x(a), y(b) {}
    __device__ __forceinline__ float a() const { return x; }
    __device__ __forceinline__ float b() const { return y; }
};
__device__ __forceinline__ P2 operator+(P2 p, P2 q) { return P2(p.x + q.x, p.y + q.y); }
__device__ __forceinline__ P2 operator-(P2 p, P2 q) { return P2(p.x - q.x, p.y - q.y); }
__device__ __forceinline__ P2 operator*(P2 p, P2 q) { return P2(p.x * q.x, p.y * q.y); }
__device__ __forceinline__ P2 operator-(P2 p) { return P2(-p.x, -p.y); }
__device__ __forceinline__ P2& operator+=(P2& p, P2 q) { p = p + q; return p; }
__device__ __forceinline__ P2& operator-=(P2& p, P2 q) { p = p - q; return p; }
__device__ __forceinline__ P2& operator*=(P2& p, P2 q) { p = p * q; return p; }
__device__ __forceinline__ P2 fmaa(P2 p, P2 q, P2 r) { return P2(fmaf(p.x, q.x, r.x), fmaf(p.y, q.y, r.y)); }

// per-half helpers
template <typename T> __device__ __forceinline__ T psqrt(T v) { return T(sqrtf(v.a()), sqrtf(v.b())); }
template <typename T> __device__ __forceinline__ T prcp(T v) { return T(1.0f / v.a(), 1.0f / v.b()); }
template <typename T> __device__ __forceinline__ T pabs(T v) { return T(fabsf(v.a()), fabsf(v.b())); }
template <typename T> __device__ __forceinline__ T psel(bool ca, bool cb, T x, T y) {
    return T(ca ? x.a() : y.a(), cb ? x.b() : y.b());
}

}  // namespace dgm
