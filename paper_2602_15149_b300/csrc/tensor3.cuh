// Small 3x3 tensor helpers for the TLSPH kernels (row-major, register resident).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

// Host + device so that the same code can be checked on the CPU.
#ifndef TL_HD
#define TL_HD __host__ __device__ __forceinline__
#endif

namespace tl {

template <typename T> struct M3 {
    T a[9];
    TL_HD T &operator()(int r, int c) { return a[3 * r + c]; }
    TL_HD T operator()(int r, int c) const { return a[3 * r + c]; }
};

template <typename T> TL_HD M3<T> m3_zero() {
    M3<T> m;
#pragma unroll
    for (int k = 0; k < 9; k++) m.a[k] = T(0);
    return m;
}
template <typename T> TL_HD M3<T> m3_eye() {
    M3<T> m = m3_zero<T>();
    m.a[0] = m.a[4] = m.a[8] = T(1);
    return m;
}
template <typename T> TL_HD M3<T> mul(const M3<T> &x, const M3<T> &y) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.a[3 * i + j] = x.a[3 * i] * y.a[j] + x.a[3 * i + 1] * y.a[3 + j] + x.a[3 * i + 2] * y.a[6 + j];
    return r;
}
// x^T y
template <typename T> TL_HD M3<T> mul_tn(const M3<T> &x, const M3<T> &y) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.a[3 * i + j] = x.a[i] * y.a[j] + x.a[3 + i] * y.a[3 + j] + x.a[6 + i] * y.a[6 + j];
    return r;
}
template <typename T> TL_HD M3<T> transpose(const M3<T> &x) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.a[3 * i + j] = x.a[3 * j + i];
    return r;
}
template <typename T> TL_HD T trace(const M3<T> &x) { return x.a[0] + x.a[4] + x.a[8]; }
// tr(x y) for general x, y
template <typename T> TL_HD T trace_mul(const M3<T> &x, const M3<T> &y) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) s += x.a[3 * i + k] * y.a[3 * k + i];
    return s;
}
template <typename T> TL_HD T det(const M3<T> &m) {
    return m.a[0] * (m.a[4] * m.a[8] - m.a[5] * m.a[7]) - m.a[1] * (m.a[3] * m.a[8] - m.a[5] * m.a[6]) +
           m.a[2] * (m.a[3] * m.a[7] - m.a[4] * m.a[6]);
}
// det(I + x) - 1 without cancellation: tr x + (principal 2x2 minors) + det x
template <typename T> TL_HD T det_eye_plus_m1(const M3<T> &x) {
    T tr = trace(x);
    T m2 = (x.a[0] * x.a[4] - x.a[1] * x.a[3]) + (x.a[0] * x.a[8] - x.a[2] * x.a[6]) +
           (x.a[4] * x.a[8] - x.a[5] * x.a[7]);
    return tr + m2 + det(x);
}
// adjugate-based inverse; returns det
template <typename T> TL_HD T inverse(const M3<T> &m, M3<T> &r) {
    T c00 = m.a[4] * m.a[8] - m.a[5] * m.a[7];
    T c01 = m.a[5] * m.a[6] - m.a[3] * m.a[8];
    T c02 = m.a[3] * m.a[7] - m.a[4] * m.a[6];
    T d = m.a[0] * c00 + m.a[1] * c01 + m.a[2] * c02;
    T id = T(1) / d;
    r.a[0] = c00 * id;
    r.a[1] = (m.a[2] * m.a[7] - m.a[1] * m.a[8]) * id;
    r.a[2] = (m.a[1] * m.a[5] - m.a[2] * m.a[4]) * id;
    r.a[3] = c01 * id;
    r.a[4] = (m.a[0] * m.a[8] - m.a[2] * m.a[6]) * id;
    r.a[5] = (m.a[2] * m.a[3] - m.a[0] * m.a[5]) * id;
    r.a[6] = c02 * id;
    r.a[7] = (m.a[1] * m.a[6] - m.a[0] * m.a[7]) * id;
    r.a[8] = (m.a[0] * m.a[4] - m.a[1] * m.a[3]) * id;
    return d;
}
template <typename T> TL_HD M3<T> sym_part(const M3<T> &x) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.a[3 * i + j] = T(0.5) * (x.a[3 * i + j] + x.a[3 * j + i]);
    return r;
}

// precision helpers
TL_HD float t_sqrt(float x) { return sqrtf(x); }
TL_HD double t_sqrt(double x) { return sqrt(x); }
TL_HD float t_log1p(float x) { return log1pf(x); }
TL_HD double t_log1p(double x) { return log1p(x); }
TL_HD float t_expm1(float x) { return expm1f(x); }
TL_HD double t_expm1(double x) { return expm1(x); }
TL_HD float t_exp(float x) { return expf(x); }
TL_HD double t_exp(double x) { return exp(x); }
TL_HD float t_acos(float x) { return acosf(x); }
TL_HD double t_acos(double x) { return acos(x); }
TL_HD float t_cos(float x) { return cosf(x); }
TL_HD double t_cos(double x) { return cos(x); }
TL_HD float t_abs(float x) { return fabsf(x); }
TL_HD double t_abs(double x) { return fabs(x); }
// a b + c with one rounding (the library is compiled without implicit contraction, so
// every fused multiply-add is written out and rounds the same in every kernel)
TL_HD float t_fma(float a, float b, float c) { return fmaf(a, b, c); }
TL_HD double t_fma(double a, double b, double c) { return fma(a, b, c); }
TL_HD float t_max(float a, float b) { return fmaxf(a, b); }
TL_HD double t_max(double a, double b) { return fmax(a, b); }
TL_HD float t_min(float a, float b) { return fminf(a, b); }
TL_HD double t_min(double a, double b) { return fmin(a, b); }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float v = 1.1920929e-7f; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

}  // namespace tl
