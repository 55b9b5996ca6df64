// Complex arithmetic on CUDA vector types (double2 = complex FP64, float2 = complex FP32).
#pragma once
#include <cuda_runtime.h>

namespace hm {

template <class T> struct Real;
template <> struct Real<double2> { typedef double type; };
template <> struct Real<float2> { typedef float type; };

__device__ __forceinline__ double2 czero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 czero(float2) { return make_float2(0.f, 0.f); }

// c + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c)
{
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
    return c;
}
// c - a*b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c)
{
    c.x = fma(-a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(-a.x, b.y, c.y);
    c.y = fma(-a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c)
{
    c.x = fmaf(-a.x, b.x, c.x);
    c.x = fmaf(a.y, b.y, c.x);
    c.y = fmaf(-a.x, b.y, c.y);
    c.y = fmaf(-a.y, b.x, c.y);
    return c;
}
// c + conj(a)*b
__device__ __forceinline__ double2 cjfma(double2 a, double2 b, double2 c)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(-a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <class T> __device__ __forceinline__ T cconv(double2 v);
template <> __device__ __forceinline__ double2 cconv<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cconv<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 cwiden(double2 v) { return v; }
__device__ __forceinline__ double2 cwiden(float2 v) { return make_double2((double)v.x, (double)v.y); }

// L2-only load (the sweeps read blocks other CTAs have just published)
__device__ __forceinline__ double2 ldcg(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ float2 ldcg(const float2 *p) { return __ldcg(p); }

}  // namespace hm
