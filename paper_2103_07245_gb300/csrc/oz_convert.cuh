// Exact integer sums of the FP64-accurate digit products to FP64: the value
// (hi 2^28 + lo) 2^e, hi and lo 64-bit two's complement integers, rounded
// once to the nearest double (ties to even).  oz_to_double is the reference
// form (92-bit magnitude normalised with a leading-zero count and rounded on
// its dropped bits, integer operations only); oz_to_double_fast reaches the
// same double with 64-bit operations and one hardware conversion.
#pragma once
#include <cstdint>

namespace pbq {

__device__ __forceinline__ double pow2i(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// (hi 2^28 + lo) 2^e as the nearest double (ties to even), with integer
// operations only (FP64 arithmetic runs at 2 lanes per clock per SM on GB300):
// the 92-bit magnitude is normalised with a leading-zero count and rounded on
// its dropped bits.  Results outside the normal range take the FP64 route
// (x 2^k in exact power-of-two factors).
__device__ __forceinline__ double oz_to_double(int64_t hi, int64_t lo, int e) {
    const __int128 N = ((__int128)hi << 28) + (__int128)lo;
    if (N == 0) return 0.0;
    const bool neg = N < 0;
    const unsigned __int128 U = neg ? (unsigned __int128)(-N) : (unsigned __int128)N;
    const uint64_t uh = (uint64_t)(U >> 64), ul = (uint64_t)U;
    const int p = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);   // leading 1 at bit p
    uint64_t m;
    int pe = p;
    if (p <= 52) {
        m = ul << (52 - p);
    } else {
        const int sh = p - 52;
        m = (uint64_t)(U >> sh);
        const unsigned __int128 rem = U & ((((unsigned __int128)1) << sh) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
        if (rem > half || (rem == half && (m & 1))) {
            ++m;
            if (m >> 53) { m >>= 1; ++pe; }
        }
    }
    const int biased = pe + e + 1023;
    if (biased <= 0 || biased >= 2047) {
        // subnormal or overflowing result: m 2^(pe - 52 + e) in exact power-of-two factors
        const double v = neg ? -(double)m : (double)m;   // m < 2^53: exact
        int k = pe - 52 + e;
        const int k1 = k > 900 ? 900 : (k < -900 ? -900 : k);
        k -= k1;
        const int k2 = k > 900 ? 900 : (k < -900 ? -900 : k);
        return v * pow2i(k1) * pow2i(k2) * pow2i(k - k2);
    }
    const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)biased << 52) | (m & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}


// The same double from 64-bit operations: N = H 2^28 + L with 0 <= L < 2^28
// (H = hi + floor(lo / 2^28)) has the sign of H; its magnitude, shifted right
// by s >= 0 so that it fits in 63 bits with every shifted-out bit folded into
// bit 0, converts to double with one round-to-nearest-even.  When s > 0 the
// shifted value has its leading bit at bit 62, so the folded bit lies ten
// places below the last place of the 53-bit result and acts only as the
// sticky bit of that rounding: the result is N correctly rounded.  The scale
// 2^(s + e) enters through the exponent field; results outside the normal
// range take oz_to_double.  |hi| < 2^62 (the sums never come near).
__device__ __forceinline__ double oz_to_double_fast(int64_t hi, int64_t lo, int e) {
    const int64_t H0 = hi + (lo >> 28);
    const uint64_t L0 = (uint64_t)lo & ((1ull << 28) - 1);
    const bool neg = H0 < 0;
    uint64_t H, L;
    if (!neg) {
        H = (uint64_t)H0;
        L = L0;
    } else if (L0) {   // -(H0 2^28 + L0) = (-H0 - 1) 2^28 + (2^28 - L0)
        H = (uint64_t)(-(H0 + 1));
        L = (1ull << 28) - L0;
    } else {
        H = (uint64_t)(-H0);
        L = 0;
    }
    int s = 0;
    uint64_t M;
    if (H < (1ull << 35)) {
        M = (H << 28) | L;
    } else {
        s = 63 - __clzll((long long)H) - 34;   // 1 .. 28: the leading bit of H 2^(28 - s) at 62
        M = (H << (28 - s)) | (L >> s) | ((L & ((1ull << s) - 1)) ? 1ull : 0ull);
    }
    if (M == 0) return 0.0;
    const long long bits = __double_as_longlong(__ull2double_rn(M));
    const int be = (int)((bits >> 52) & 0x7FF) + s + e;
    if (be <= 0 || be >= 2047) return oz_to_double(hi, lo, e);
    const long long scaled = bits + (long long)((unsigned long long)(long long)(s + e) << 52);
    return __longlong_as_double(neg ? (scaled | (long long)0x8000000000000000ull) : scaled);
}

}  // namespace pbq
