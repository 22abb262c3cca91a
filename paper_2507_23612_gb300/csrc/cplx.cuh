// Scalar helpers shared by the kernels: one code path for real and complex elements.
#pragma once
#include <cuda_runtime.h>

namespace hub {

template <typename R, bool CPLX> struct VT;
template <> struct VT<double, false> { using T = double; };
template <> struct VT<float, false> { using T = float; };
template <> struct VT<double, true> { using T = double2; };
template <> struct VT<float, true> { using T = float2; };

__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ float zero_of(float) { return 0.0f; }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 zero_of(float2) { return make_float2(0.f, 0.f); }

// a + b
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// acc + w * a, w real
__device__ __forceinline__ double fmar(double w, double a, double acc) { return fma(w, a, acc); }
__device__ __forceinline__ float fmar(float w, float a, float acc) { return fmaf(w, a, acc); }
__device__ __forceinline__ double2 fmar(double w, double2 a, double2 acc) {
    return make_double2(fma(w, a.x, acc.x), fma(w, a.y, acc.y));
}
__device__ __forceinline__ float2 fmar(float w, float2 a, float2 acc) {
    return make_float2(fmaf(w, a.x, acc.x), fmaf(w, a.y, acc.y));
}

// w * a, w real
__device__ __forceinline__ double mulr(double w, double a) { return w * a; }
__device__ __forceinline__ float mulr(float w, float a) { return w * a; }
__device__ __forceinline__ double2 mulr(double w, double2 a) { return make_double2(w * a.x, w * a.y); }
__device__ __forceinline__ float2 mulr(float w, float2 a) { return make_float2(w * a.x, w * a.y); }

// complex product a * b (real: plain product)
__device__ __forceinline__ double cmul(double a, double b) { return a * b; }
__device__ __forceinline__ float cmul(float a, float b) { return a * b; }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + conj(a) * b
__device__ __forceinline__ double cfma_conj(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ float cfma_conj(float a, float b, float acc) { return fmaf(a, b, acc); }
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
// acc + a * b
__device__ __forceinline__ double cfma(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ float cfma(float a, float b, float acc) { return fmaf(a, b, acc); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

// conj(a); real part; modulus; a - b; a / r for real r; a real value in T
__device__ __forceinline__ double cconj(double a) { return a; }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double re_of(double a) { return a; }
__device__ __forceinline__ double re_of(double2 a) { return a.x; }
__device__ __forceinline__ double cabs_of(double a) { return fabs(a); }
__device__ __forceinline__ double cabs_of(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double csub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double divr(double a, double r) { return a / r; }
__device__ __forceinline__ double2 divr(double2 a, double r) { return make_double2(a.x / r, a.y / r); }
template <typename T> __device__ __forceinline__ T from_real(double v);
template <> __device__ __forceinline__ double from_real<double>(double v) { return v; }
template <> __device__ __forceinline__ double2 from_real<double2>(double v) { return make_double2(v, 0.0); }
// shuffle-down of a real or complex value
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 shfl_down(double2 v, int o) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}

__device__ __forceinline__ bool finite_val(double a) { return isfinite(a); }
__device__ __forceinline__ bool finite_val(float a) { return isfinite(a); }
__device__ __forceinline__ bool finite_val(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ bool finite_val(float2 a) { return isfinite(a.x) && isfinite(a.y); }

// phase^w for a unit complex phase and a small integer w (real: 1)
template <typename T> __device__ __forceinline__ T phase_pow(double pr, double pi, int w);
template <> __device__ __forceinline__ double phase_pow<double>(double, double, int) { return 1.0; }
template <> __device__ __forceinline__ float phase_pow<float>(double, double, int) { return 1.0f; }
template <> __device__ __forceinline__ double2 phase_pow<double2>(double pr, double pi, int w) {
    double2 r = make_double2(1.0, 0.0);
    double2 b = w >= 0 ? make_double2(pr, pi) : make_double2(pr, -pi);
    int k = w >= 0 ? w : -w;
    for (int i = 0; i < k; ++i) r = cmul(r, b);
    return r;
}
template <> __device__ __forceinline__ float2 phase_pow<float2>(double pr, double pi, int w) {
    double2 r = phase_pow<double2>(pr, pi, w);
    return make_float2((float)r.x, (float)r.y);
}

}  // namespace hub
