// ul_math.cuh — per-precision arithmetic for the link updates.
//
// FP64 path: sin/cos/exp/atan2 with a fixed IEEE operation sequence.  The update is
// chaotic (a one-ulp change in a cos/sin grows to ~1e-4 rad within one compound
// sweep), so the FP64 path is only comparable link by link with an independent FP64
// program if both evaluate the same operations.  The functions follow published
// methods:
//   sincos: additive range reduction by pi/2 with a three-part constant (Cody & Waite,
//           "Software Manual for the Elementary Functions", 1980) and the Taylor
//           series of sin and cos on [-pi/4, pi/4] evaluated by Horner's rule;
//   exp:    reduction by ln 2 (same method), Taylor series on [-ln2/2, ln2/2], 2^k scale;
//   atan2:  octant reduction to t in [0,1], the addition formula
//           atan(t) = atan(j/8) + atan((t - j/8)/(1 + t j/8)) with j = rint(8t), and
//           the Taylor series of atan for |u| <= 1/16.
// Every fused multiply-add is an explicit fma(); the FP64 translation unit is compiled
// with -fmad=false so no other multiply-add is fused.  All results are within 1 ulp.
//
// FP32 path: CUDA's single-precision sincosf/expf/atan2f.  The FP32 translation unit is
// also compiled with -fmad=false and its complex products are fused explicitly, so a link's
// new value does not depend on the kernel that computes it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ul_device.cuh"

namespace ul {

struct c64 {
    double re, im;
};
struct c32 {
    float re, im;
};

// ---------------------------------------------------------------------------
// FP64 elementary functions
// ---------------------------------------------------------------------------
namespace dm {
// pi/2 = P1 + P2 + P3 (P1 = pi/2 rounded to double, P2 and P3 the next two roundings)
constexpr double P1 = 0x1.921fb54442d18p+0;
constexpr double P2 = 0x1.1a62633145c07p-54;
constexpr double P3 = -0x1.f1976b7ed8fbcp-110;
constexpr double TWO_OVER_PI = 0x1.45f306dc9c883p-1;
constexpr double LN2_A = 0x1.62e42fefa39efp-1;  // ln 2 rounded to double
constexpr double LN2_B = 0x1.abc9e3b39803fp-56; // ln 2 - LN2_A rounded
constexpr double LOG2_E = 0x1.71547652b82fep+0; // 1/ln 2
constexpr double PI = 0x1.921fb54442d18p+1;     // pi rounded to double

// Exact integer forms of some FP64 steps (the FP64 pipe is the update's bottleneck; the
// integer pipes are idle).  For doubles that are not NaN:
//   order_key(x) is monotonic in x and equal for +0 and -0, so x < y <=> key(x) < key(y);
//   for x >= +0 the bit patterns themselves are ordered;
//   multiplying a normal double by 2^n is adding n to its exponent field, exact as long as
//   the result is normal.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double from_bits(long long b) { return __longlong_as_double(b); }
__device__ __forceinline__ long long order_key(double x)
{
    const long long b = dbits(x);
    return b >= 0 ? b : -(b & 0x7fffffffffffffffLL);
}
constexpr long long kExpUnit = 1LL << 52;                      // one step of the exponent field
constexpr long long kBitsTwoPi = 0x401921fb54442d18LL;         // 2 pi (= 2 PI below)
constexpr long long kBitsFourPi = 0x402921fb54442d18LL;        // 4 pi
constexpr long long kBits700 = 0x4085e00000000000LL;           // 700.0
constexpr long long kBitsInf = 0x7ff0000000000000LL;           // +infinity

static __device__ const double kAtanJ8[2][9] = {
    // atan(j/8) rounded to double, j = 0..8
    {0.0, 0x1.fd5ba9aac2f6ep-4, 0x1.f5b75f92c80ddp-3, 0x1.6f61941e4def1p-2, 0x1.dac670561bb4fp-2,
     0x1.1e00babdefeb4p-1, 0x1.4978fa3269ee1p-1, 0x1.700a7c5784634p-1, 0x1.921fb54442d18p-1},
    // the rounding remainder atan(j/8) - first row
    {0.0, -0x1.cd37686760c17p-59, 0x1.8ab6e3cf7afbdp-57, -0x1.c63aae6f6e918p-56, 0x1.a2b7f222f65e2p-56,
     -0x1.928df287a668fp-58, 0x1.2419a87f2a458p-56, -0x1.8c34d25aadef6p-56, 0x1.1a62633145c07p-55}};

__device__ __forceinline__ void sincos_det(double x, double* sp, double* cp)
{
    const double k = rint(x * TWO_OVER_PI);
    double r = fma(-k, P1, x);
    r = fma(-k, P2, r);
    r = fma(-k, P3, r);
    const double r2 = r * r;
    // odd series, highest term 1/17!
    double a = 1.0 / 355687428096000.0;
    a = fma(a, r2, -1.0 / 1307674368000.0);
    a = fma(a, r2, 1.0 / 6227020800.0);
    a = fma(a, r2, -1.0 / 39916800.0);
    a = fma(a, r2, 1.0 / 362880.0);
    a = fma(a, r2, -1.0 / 5040.0);
    a = fma(a, r2, 1.0 / 120.0);
    a = fma(a, r2, -1.0 / 6.0);
    const double sr = fma(r * r2, a, r);
    // even series, highest term 1/16!
    double b = 1.0 / 20922789888000.0;
    b = fma(b, r2, -1.0 / 87178291200.0);
    b = fma(b, r2, 1.0 / 479001600.0);
    b = fma(b, r2, -1.0 / 3628800.0);
    b = fma(b, r2, 1.0 / 40320.0);
    b = fma(b, r2, -1.0 / 720.0);
    b = fma(b, r2, 1.0 / 24.0);
    b = fma(b, r2, -0.5);
    const double cr = fma(r2, b, 1.0);
    const int quadrant = static_cast<int>(static_cast<long long>(k) & 3);
    switch (quadrant) {
    case 0: *sp = sr; *cp = cr; break;
    case 1: *sp = cr; *cp = -sr; break;
    case 2: *sp = -sr; *cp = -cr; break;
    default: *sp = -cr; *cp = sr; break;
    }
}

__device__ __forceinline__ double exp_det(double x)
{
    // x > 700: +inf, x < -700: 0 (as floating-point comparisons; NaN falls through)
    const long long xb = dbits(x), ab = xb & 0x7fffffffffffffffLL;
    if (ab > kBits700 && ab <= kBitsInf) return xb < 0 ? 0.0 : from_bits(kBitsInf);
    const double k = rint(x * LOG2_E);
    double r = fma(-k, LN2_A, x);
    r = fma(-k, LN2_B, r);
    double e = 1.0 / 6227020800.0;
    e = fma(e, r, 1.0 / 479001600.0);
    e = fma(e, r, 1.0 / 39916800.0);
    e = fma(e, r, 1.0 / 3628800.0);
    e = fma(e, r, 1.0 / 362880.0);
    e = fma(e, r, 1.0 / 40320.0);
    e = fma(e, r, 1.0 / 5040.0);
    e = fma(e, r, 1.0 / 720.0);
    e = fma(e, r, 1.0 / 120.0);
    e = fma(e, r, 1.0 / 24.0);
    e = fma(e, r, 1.0 / 6.0);
    e = fma(e, r, 0.5);
    e = fma(e, r, 1.0);
    e = fma(e, r, 1.0);
    // ldexp(e, k): e is within (0.7, 1.5) and |k| <= 1010, so e 2^k is normal and exact
    return from_bits(dbits(e) + static_cast<long long>(k) * kExpUnit);
}

__device__ __forceinline__ double atan_small(double u)
{
    const double u2 = u * u;
    double q = -1.0 / 15.0;
    q = fma(q, u2, 1.0 / 13.0);
    q = fma(q, u2, -1.0 / 11.0);
    q = fma(q, u2, 1.0 / 9.0);
    q = fma(q, u2, -1.0 / 7.0);
    q = fma(q, u2, 1.0 / 5.0);
    q = fma(q, u2, -1.0 / 3.0);
    return fma(u * u2, q, u);
}

// atan2 with signed zeros treated as +0 and atan2(0, 0) = 0.
__device__ __forceinline__ double atan2_det(double y, double x)
{
    const double ax = fabs(x), ay = fabs(y);
    const long long bx = dbits(ax), by = dbits(ay);
    if ((bx | by) == 0) return 0.0;          // ax == 0 and ay == 0
    const bool steep = by > bx;              // ay > ax (both >= +0)
    const double t = steep ? ax / ay : ay / ax;
    // t 8: an exponent change where t is normal (t = 0 or subnormal: the multiplication)
    const long long tb = dbits(t);
    const double jd = rint(tb >= kExpUnit ? from_bits(tb + 3 * kExpUnit) : t * 8.0);
    const int j = static_cast<int>(jd);
    double a;
    if (j == 0) {
        a = atan_small(t);
    } else {
        const double cj = from_bits(dbits(jd) - 3 * kExpUnit); // j * 0.125, exact (j >= 1)
        const double u = (t - cj) / (1.0 + t * cj);
        a = kAtanJ8[0][j] + (kAtanJ8[1][j] + atan_small(u));
    }
    if (steep) a = (P1 - a) + P2;
    if (dbits(x) < 0 && bx != 0) a = (2.0 * P1 - a) + 2.0 * P2; // x < 0.0
    return (dbits(y) < 0 && by != 0) ? -a : a;                  // y < 0.0
}
} // namespace dm

// ---------------------------------------------------------------------------
// Precision traits used by the templated kernels
// ---------------------------------------------------------------------------
template <typename R>
struct Prec;

template <>
struct Prec<double> {
    using real = double;
    using cs_t = double2; // (cos, sin) of a link angle
    static constexpr double PI = dm::PI;
    static __device__ __forceinline__ void sincos(double x, double* s, double* c) { dm::sincos_det(x, s, c); }
    static __device__ __forceinline__ double exp(double x) { return dm::exp_det(x); }
    static __device__ __forceinline__ double atan2(double y, double x) { return dm::atan2_det(y, x); }
    // uniform in [0,1) from a 64-bit word
    // (w >> 11) 2^-53: the conversion is exact (< 2^53) and the scaling an exponent change
    static __device__ __forceinline__ double uniform(uint64_t w)
    {
        const uint64_t m = w >> 11;
        const double d = static_cast<double>(m);
        return m ? dm::from_bits(dm::dbits(d) - 53 * dm::kExpUnit) : 0.0;
    }
    // 2 u - 1 for a uniform u (0 or >= 2^-53): the doubling is an exponent change
    static __device__ __forceinline__ double two_u_minus_one(double u)
    {
        const double twice = dm::dbits(u) ? dm::from_bits(dm::dbits(u) + dm::kExpUnit) : 0.0;
        return twice - 1.0;
    }
    // a < b for doubles >= +0 that are not NaN (the Metropolis test u2 < exp(-dS))
    static __device__ __forceinline__ bool less_nonneg(double a, double b) { return dm::dbits(a) < dm::dbits(b); }
    // Metropolis uniforms of link link_id in pass `pass`: words 0 and 1 of
    // Philox4x64-10(counter (link_id, pass, 0, 0), key (seed, 1))
    static __device__ __forceinline__ void metro_uniforms(uint64_t link_id, uint64_t pass, uint64_t seed, double* u1,
                                                          double* u2)
    {
        const Philox4 w = philox4x64_10(link_id, pass, 0, 0, seed, kStreamMetropolis);
        *u1 = uniform(w.w[0]);
        *u2 = uniform(w.w[1]);
    }
    // th - 2pi floor((th + pi) / 2pi).  For a = th + pi in [-2pi, 4pi) the floor of the
    // correctly rounded quotient a / 2pi is -1, 0 or 1 exactly where a < 0, a < 2pi,
    // a < 4pi (no quotient in that range rounds across an integer: the double nearest
    // below 2pi (4pi) divided by 2pi lies more than half an ulp below 1 (2)), so the
    // comparisons reproduce the division's result bit for bit; other a take the division.
    // (The comparisons run on integer keys of a: the same decisions, off the FP64 pipe.)
    static __device__ __forceinline__ double wrap(double th)
    {
        const double two_pi = 2.0 * PI;
        const double a = th + PI;
        const long long ka = dm::order_key(a);
        if (ka >= -dm::kBitsTwoPi && ka < dm::kBitsFourPi) {
            // two_pi k for k = -1, 0, 1 is exact: select it instead of multiplying
            const double shift = ka < 0 ? -two_pi : (ka < dm::kBitsTwoPi ? 0.0 : two_pi);
            return th - shift;
        }
        return th - two_pi * floor(a / two_pi);
    }
    // -2 a: an exponent change and a sign flip where a is normal (else the multiplication)
    static __device__ __forceinline__ double minus_twice(double a)
    {
        const long long b = dm::dbits(a);
        const long long m = b & 0x7fffffffffffffffLL;
        if (m >= dm::kExpUnit && m < dm::kBitsInf - dm::kExpUnit)
            return dm::from_bits((b ^ static_cast<long long>(0x8000000000000000ULL)) + dm::kExpUnit);
        return -2.0 * a;
    }
};

template <>
struct Prec<float> {
    using real = float;
    using cs_t = float2;
    static constexpr float PI = 3.14159265358979323846f;
    static __device__ __forceinline__ void sincos(float x, float* s, float* c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
    static __device__ __forceinline__ float atan2(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float uniform(uint64_t w)
    {
        return static_cast<float>(static_cast<uint32_t>(w >> 40)) * 0x1.0p-24f;
    }
    // Metropolis uniforms: words 0 and 1 of Philox4x32-10(counter (link_id, pass low, pass
    // high, 1), key (seed low, seed high)), 24 bits each: u = (w >> 8) 2^-24
    static __device__ __forceinline__ void metro_uniforms(uint64_t link_id, uint64_t pass, uint64_t seed, float* u1,
                                                          float* u2)
    {
        const Philox4x32 w = philox4x32_10(static_cast<uint32_t>(link_id), static_cast<uint32_t>(pass),
                                           static_cast<uint32_t>(pass >> 32), static_cast<uint32_t>(kStreamMetropolis),
                                           static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
        *u1 = static_cast<float>(w.w[0] >> 8) * 0x1.0p-24f;
        *u2 = static_cast<float>(w.w[1] >> 8) * 0x1.0p-24f;
    }
    static __device__ __forceinline__ float two_u_minus_one(float u) { return 2.0f * u - 1.0f; }
    static __device__ __forceinline__ float minus_twice(float a) { return -2.0f * a; }
    static __device__ __forceinline__ bool less_nonneg(float a, float b) { return a < b; }
    static __device__ __forceinline__ float wrap(float th)
    {
        const float two_pi = 2.0f * PI;
        return th - two_pi * floorf((th + PI) / two_pi);
    }
};

// ---------------------------------------------------------------------------
// Complex helpers (FP32 products may be contracted by the compiler; FP64 products below)
// ---------------------------------------------------------------------------
template <typename T>
struct Cx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ Cx<T> cx(T re, T im)
{
    return Cx<T>{re, im};
}
template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b)
{
    return Cx<T>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// FP64 complex product: each component one fused multiply-add of an exact and a rounded
// product, re = fma(a.re, b.re, -(a.im b.im)), im = fma(a.re, b.im, a.im b.re) (four FP64
// instructions; the FP64 oracle forms its products the same way).
template <>
__device__ __forceinline__ Cx<double> cmul<double>(Cx<double> a, Cx<double> b)
{
    return Cx<double>{fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
}
// FP32 complex product, fused the same way (two FFMA and two FMUL).
template <>
__device__ __forceinline__ Cx<float> cmul<float>(Cx<float> a, Cx<float> b)
{
    return Cx<float>{__fmaf_rn(a.re, b.re, -__fmul_rn(a.im, b.im)), __fmaf_rn(a.re, b.im, __fmul_rn(a.im, b.re))};
}
// Complex products with a fixed rounding sequence in every compilation context (FP32: every
// operation rounded separately; FP64: one explicit fused multiply-add per component), used
// by the measurements so that they do not depend on how a kernel inlines them.
__device__ __forceinline__ Cx<float> cmul_rn(Cx<float> a, Cx<float> b)
{
    return Cx<float>{__fsub_rn(__fmul_rn(a.re, b.re), __fmul_rn(a.im, b.im)),
                     __fadd_rn(__fmul_rn(a.re, b.im), __fmul_rn(a.im, b.re))};
}
__device__ __forceinline__ Cx<double> cmul_rn(Cx<double> a, Cx<double> b)
{
    // explicit fused form: as deterministic as separate roundings, two FP64 instructions fewer
    return Cx<double>{__fma_rn(a.re, b.re, -__dmul_rn(a.im, b.im)), __fma_rn(a.re, b.im, __dmul_rn(a.im, b.re))};
}
// Explicitly fused multiply-add in precision R.
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// A += p q, both components accumulated by fused multiply-adds:
//   Re: fma(p.re, q.re, fma(-p.im, q.im, A.re)),  Im: fma(p.re, q.im, fma(p.im, q.re, A.im))
// (the FP64 oracle accumulates its staple terms the same way).
template <typename T>
__device__ __forceinline__ void cmul_acc(Cx<T>& A, Cx<T> p, Cx<T> q)
{
    A.re = fma_r(p.re, q.re, fma_r(-p.im, q.im, A.re));
    A.im = fma_r(p.re, q.im, fma_r(p.im, q.re, A.im));
}

template <typename T>
__device__ __forceinline__ Cx<T> cconj(Cx<T> a)
{
    return Cx<T>{a.re, -a.im};
}
template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b)
{
    return Cx<T>{a.re + b.re, a.im + b.im};
}

} // namespace ul
