// Shared device helpers: interleaved complex arithmetic on float2 / double2,
// atomics on non-negative doubles, error plumbing for the launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef RSRR_DEV
#define RSRR_DEV __device__ __forceinline__
#endif
#ifndef RSRR_HD
#define RSRR_HD __host__ __device__ inline
#endif

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

RSRR_DEV float2 cmake(float re, float im) { return make_float2(re, im); }
RSRR_DEV double2 cmake(double re, double im) { return make_double2(re, im); }

template <typename C> RSRR_DEV C czero();
template <> RSRR_DEV float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> RSRR_DEV double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <typename C> RSRR_DEV C cone();
template <> RSRR_DEV float2 cone<float2>() { return make_float2(1.f, 0.f); }
template <> RSRR_DEV double2 cone<double2>() { return make_double2(1.0, 0.0); }

RSRR_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
RSRR_DEV double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
RSRR_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
RSRR_DEV double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
RSRR_DEV float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
RSRR_DEV double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
RSRR_DEV float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
RSRR_DEV double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// acc - a*b
RSRR_DEV float2 cfms(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(-a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}
RSRR_DEV double2 cfms(double2 acc, double2 a, double2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
// acc + a*b
RSRR_DEV float2 cfma(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
RSRR_DEV double2 cfma(double2 acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a)*b
RSRR_DEV double2 cfmac(double2 acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
RSRR_DEV float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
RSRR_DEV double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
RSRR_DEV float cabsv(float2 a) { return hypotf(a.x, a.y); }
RSRR_DEV double cabsv(double2 a) { return hypot(a.x, a.y); }
RSRR_DEV bool cnonzero(float2 a) { return a.x != 0.f || a.y != 0.f; }
RSRR_DEV bool cnonzero(double2 a) { return a.x != 0.0 || a.y != 0.0; }
// 1/b with Smith's scaling (avoids overflow of |b|^2)
RSRR_DEV float2 crecip(float2 b) {
    if (fabsf(b.x) >= fabsf(b.y)) {
        float r = b.y / b.x, d = b.x + b.y * r;
        return make_float2(1.f / d, -r / d);
    } else {
        float r = b.x / b.y, d = b.y + b.x * r;
        return make_float2(r / d, -1.f / d);
    }
}
RSRR_DEV double2 crecip(double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2(1.0 / d, -r / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return make_double2(r / d, -1.0 / d);
    }
}
RSRR_DEV float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
RSRR_DEV double2 to_c128(float2 a) { return make_double2((double)a.x, (double)a.y); }

// Real overloads of the same helpers: the band LU and solves instantiated for
// float / double factor real NEPs at real sampling points (real arithmetic
// at a quarter of the multiplies and half the storage of the complex path).
template <> struct real_of<float> { using type = float; };
template <> struct real_of<double> { using type = double; };
template <> RSRR_DEV float czero<float>() { return 0.f; }
template <> RSRR_DEV double czero<double>() { return 0.0; }
template <> RSRR_DEV float cone<float>() { return 1.f; }
template <> RSRR_DEV double cone<double>() { return 1.0; }
RSRR_DEV float cadd(float a, float b) { return a + b; }
RSRR_DEV double cadd(double a, double b) { return a + b; }
RSRR_DEV float csub(float a, float b) { return a - b; }
RSRR_DEV double csub(double a, double b) { return a - b; }
RSRR_DEV float cmul(float a, float b) { return a * b; }
RSRR_DEV double cmul(double a, double b) { return a * b; }
RSRR_DEV float cmulc(float a, float b) { return a * b; }
RSRR_DEV double cmulc(double a, double b) { return a * b; }
RSRR_DEV float cfms(float acc, float a, float b) { return fmaf(-a, b, acc); }
RSRR_DEV double cfms(double acc, double a, double b) { return fma(-a, b, acc); }
RSRR_DEV float cfma(float acc, float a, float b) { return fmaf(a, b, acc); }
RSRR_DEV double cfma(double acc, double a, double b) { return fma(a, b, acc); }
RSRR_DEV float cabs1(float a) { return fabsf(a); }
RSRR_DEV double cabs1(double a) { return fabs(a); }
RSRR_DEV float cabsv(float a) { return fabsf(a); }
RSRR_DEV double cabsv(double a) { return fabs(a); }
RSRR_DEV bool cnonzero(float a) { return a != 0.f; }
RSRR_DEV bool cnonzero(double a) { return a != 0.0; }
RSRR_DEV float crecip(float b) { return 1.f / b; }
RSRR_DEV double crecip(double b) { return 1.0 / b; }

template <typename T> RSRR_DEV T shfl_down(T v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }

// max of non-negative doubles through their ordered bit patterns
RSRR_DEV void atomic_max_nonneg(double *addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}
