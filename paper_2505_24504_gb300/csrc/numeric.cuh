// Scalar types of the device physics.
//
//  D64   IEEE double whose operators are the round-to-nearest intrinsics, so the
//        compiler never contracts or reorders them.  The same expression on the
//        same inputs gives the same bits in every kernel; this is what keeps
//        U' = 0 at an exact zero residual when background fluxes computed once at
//        set-up are subtracted from fluxes computed inside the residual kernels.
//  TL32  FP32 value with an FP32 tangent (forward-mode dual number).  Running the
//        flux code on TL32 gives the exact directional derivative J(u) x of the
//        operator in FP32, the product the FP32 preconditioner smooths with.
//
// Both carry a power x^gamma:
//  D64: table-driven reduction x = 2^e m_i (1+t), |t| < 2^-8, with 2^(e gamma),
//       m_i^gamma and 1/m_i from tables built on the host in long double and the
//       binomial series of (1+t)^gamma to t^6 (truncation < 1e-18); about 10
//       FP64 pipe operations against ~100 for the library pow on this GPU.
//       Inputs outside the table range fall back to pow().
//  TL32: value by the fast exp2/log2 power, tangent gamma p / x.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define JF_HD __host__ __device__ __forceinline__
#define JF_D __device__ __forceinline__

// ---------------------------------------------------------------------------
struct PowTab {
    double gamma;
    double pe[64];      // 2^(e gamma), e = -32 .. 31
    double mg[256];     // (1 + i/256)^gamma
    double minv[256];   // 1 / (1 + i/256)
    double c[7];        // binomial coefficients C(gamma, n), n = 1..6 (c[0] unused)
};

JF_D double pow_gamma_tab(double x, const PowTab *T) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (!(x > 0.0) || e < -32 || e > 31) return pow(x, T->gamma);
    const int i = (int)((b >> 44) & 0xff);
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double mi = __longlong_as_double((b & 0x000ff00000000000LL) | 0x3ff0000000000000LL);
    const double t = __dmul_rn(__dsub_rn(m, mi), T->minv[i]);
    double q = T->c[6];
    q = __fma_rn(q, t, T->c[5]);
    q = __fma_rn(q, t, T->c[4]);
    q = __fma_rn(q, t, T->c[3]);
    q = __fma_rn(q, t, T->c[2]);
    q = __fma_rn(q, t, T->c[1]);
    q = __dmul_rn(q, t);                      // (1+t)^gamma - 1
    const double s = __dmul_rn(T->pe[e + 32], T->mg[i]);
    return __fma_rn(s, q, s);
}

// ---------------------------------------------------------------------------
struct D64 {
    double x;
};
JF_D D64 mk(double v, D64) { return D64{v}; }
JF_D D64 operator+(D64 a, D64 b) { return D64{__dadd_rn(a.x, b.x)}; }
JF_D D64 operator-(D64 a, D64 b) { return D64{__dsub_rn(a.x, b.x)}; }
JF_D D64 operator*(D64 a, D64 b) { return D64{__dmul_rn(a.x, b.x)}; }
JF_D D64 operator/(D64 a, D64 b) { return D64{__ddiv_rn(a.x, b.x)}; }
JF_D D64 operator-(D64 a) { return D64{-a.x}; }
JF_D D64 jsqrt(D64 a) { return D64{__dsqrt_rn(a.x)}; }
JF_D double val(D64 a) { return a.x; }
JF_D D64 jfma(D64 a, D64 b, D64 c) { return D64{__fma_rn(a.x, b.x, c.x)}; }

// ---------------------------------------------------------------------------
struct TL32 {
    float v, d;
};
JF_D TL32 mk(double v, TL32) { return TL32{(float)v, 0.0f}; }
JF_D TL32 operator+(TL32 a, TL32 b) { return TL32{a.v + b.v, a.d + b.d}; }
JF_D TL32 operator-(TL32 a, TL32 b) { return TL32{a.v - b.v, a.d - b.d}; }
JF_D TL32 operator*(TL32 a, TL32 b) { return TL32{a.v * b.v, fmaf(a.v, b.d, a.d * b.v)}; }
// The tangent feeds only the preconditioner: quotients and square roots use the
// hardware approximations (reciprocal, reciprocal square root; a few ulp)
// instead of the correctly rounded FP32 sequences.
JF_D float frcp(float x) { return __fdividef(1.0f, x); }
JF_D TL32 operator/(TL32 a, TL32 b) {
    const float ib = frcp(b.v);
    const float q = a.v * ib;
    return TL32{q, (a.d - q * b.d) * ib};
}
JF_D TL32 operator-(TL32 a) { return TL32{-a.v, -a.d}; }
JF_D TL32 jsqrt(TL32 a) {
    if (!(a.v > 0.0f)) return TL32{0.0f, 0.0f};
    const float r = rsqrtf(a.v);
    return TL32{a.v * r, 0.5f * a.d * r};
}
JF_D float val(TL32 a) { return a.v; }   // compared in FP32: no FP64-pipe conversion
JF_D TL32 jfma(TL32 a, TL32 b, TL32 c) { return a * b + c; }

// An FP32 constant in tangent-linear arithmetic (its tangent is zero): products,
// sums and quotients with a TL32 drop the tangent terms that are known to vanish
// (a TL32 with a zero tangent would still multiply and add them).  Converts to
// TL32 where a dual number is needed.
struct TLc {
    float v;
    JF_D operator TL32() const { return TL32{v, 0.0f}; }
};
JF_D TL32 operator*(TLc a, TL32 b) { return TL32{a.v * b.v, a.v * b.d}; }
JF_D TL32 operator*(TL32 a, TLc b) { return TL32{a.v * b.v, a.d * b.v}; }
JF_D TL32 operator+(TL32 a, TLc b) { return TL32{a.v + b.v, a.d}; }
JF_D TL32 operator+(TLc a, TL32 b) { return TL32{a.v + b.v, b.d}; }
JF_D TL32 operator-(TL32 a, TLc b) { return TL32{a.v - b.v, a.d}; }
JF_D TL32 operator-(TLc a, TL32 b) { return TL32{a.v - b.v, -b.d}; }
JF_D TL32 operator/(TLc a, TL32 b) {
    const float ib = frcp(b.v);
    const float q = a.v * ib;
    return TL32{q, -(q * b.d) * ib};
}
JF_D TL32 jfma(TLc a, TL32 b, TL32 c) { return TL32{fmaf(a.v, b.v, c.v), fmaf(a.v, b.d, c.d)}; }

// Constants held in both precisions: the FP32 tangent takes the float copy, so
// no double-to-float conversion (an FP64-pipe instruction) runs per use.
JF_D D64 mkc(double d, float, D64) { return D64{d}; }
JF_D TLc mkc(double, float f, TL32) { return TLc{f}; }
template <class S> JF_D S pick(double d, float f);
template <> JF_D double pick<double>(double d, float) { return d; }
template <> JF_D float pick<float>(double, float f) { return f; }
