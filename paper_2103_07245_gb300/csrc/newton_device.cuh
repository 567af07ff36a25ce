// 1/d and 1/sqrt(d) in FP64 without FP64 division or square root, for the
// sequential pivot chains of the Cholesky and QR kernels: a dependent FP64
// FMA takes 64 cycles on GB300, an FP64 square root ~670 and a division ~430.
#pragma once
#include <cmath>
#include <cstdint>

namespace pbq {

// 1/d for a positive normal double: d = m 2^k with m in [1, 2), an FP32 seed
// for 1/m refined by two Newton-Raphson steps y += y (1 - m y) (each doubles
// the correct bits: ~24 -> ~48 -> 53), scaled by 2^-k.  The scale 2^-k is a
// normal double only for k <= 1022; d >= 2^1023 (biased exponent 2046, a
// subnormal result), subnormal, zero, negative and non-finite d take the
// library division.  Within 2 ulp of the correctly rounded 1/d.
__device__ __forceinline__ double rcp_nr(double d) {
    const long long b = __double_as_longlong(d);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb == 0 || eb >= 0x7FE || b < 0) return 1.0 / d;
    const int k = eb - 1023;
    const double m = __longlong_as_double(b - (long long)k * (1LL << 52));
    double y = (double)__frcp_rn((float)m);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double e = fma(-m, y, 1.0);
        y = fma(y, e, y);
    }
    return y * __longlong_as_double((long long)(1023 - k) << 52);
}

// 1/sqrt(d) for a positive normal double: d = m 4^k with m in [1, 4), an FP32
// seed for 1/sqrt(m) refined by two Newton-Raphson steps y += y (1 - m y^2) / 2,
// scaled by 2^-k (k in [-511, 511], always a normal scale).  Subnormal, zero,
// negative and non-finite d take the library operations.  Within 2 ulp of
// the correctly rounded 1/sqrt(d).
__device__ __forceinline__ double rsqrt_nr(double d) {
    const long long b = __double_as_longlong(d);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb == 0 || eb == 0x7FF || b < 0) return 1.0 / sqrt(d);
    const int k = (eb - 1023) >> 1;   // floor((eb - 1023) / 2)
    const double m = __longlong_as_double(b - (long long)(2 * k) * (1LL << 52));
    double y = (double)rsqrtf((float)m);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double e = fma(-m, y * y, 1.0);
        y = fma(0.5 * y, e, y);
    }
    return y * __longlong_as_double((long long)(1023 - k) << 52);
}

// 1/d for a positive normal double in one Goldschmidt step: d = m 2^k with m
// in [1, 2), y0 an FP32 seed for 1/m (relative error e0 < 2^-22), e = 1 - m y0,
// 1/m = y0 (1 + e + e^2 + ...) truncated after e^2 (error e^3 < 2^-66, below
// FP64 rounding).  The scale 2^-k goes into the seed's exponent field with an
// integer subtraction (exact while the result is normal, i.e. k <= 1021, since
// y0 lies in (1/2, 1]), so the chain holds three FP64 instructions; d >= 2^1022
// takes two FP64 multiplications by normal factors instead.  No checks: zero,
// subnormal, negative and non-finite d give meaningless (but finite or NaN)
// results, so callers check d themselves.  Within 2 ulp of the correctly
// rounded 1/d for normal d.
__device__ __forceinline__ double rcp_gs(double d) {
    const long long b = __double_as_longlong(d);
    const int k = (int)((b >> 52) & 0x7FF) - 1023;
    const double m = __longlong_as_double((b & 0x800FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double y0 = (double)__frcp_rn((float)m);
    double ys;
    if (k <= 1021) {
        ys = __longlong_as_double(__double_as_longlong(y0) - ((long long)k << 52));
    } else {
        const int k1 = k >> 1, k2 = k - k1;
        ys = (y0 * __longlong_as_double((long long)(1023 - k1) << 52)) *
             __longlong_as_double((long long)(1023 - k2) << 52);
    }
    const double e = fma(-m, y0, 1.0);
    const double t = fma(e, e, e);
    return fma(ys, t, ys);
}

}  // namespace pbq
