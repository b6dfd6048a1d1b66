// FP64 fused multiply-add on the integer pipe.
//
// GB300 executes FP64 arithmetic at 1/64 of its FP32 rate, while its integer
// pipe idles during the FP64-bound solver loop. fma64_int(a, b, c) computes
// the IEEE 754 result of a*b + c -- the exact value rounded once to nearest,
// ties to even -- with 32/64-bit integer instructions only, so it can take
// part of the FP64 work off the FP64 pipe without changing a single result
// bit. It is written from the definition of the operation:
//
//   a = ma 2^Ea, b = mb 2^Eb, c = mc 2^Ec with 53-bit integer significands;
//   the product P = ma mb (106 bits) is exact in 128 bits; P and mc are
//   placed in a 128-bit window (P << 21, mc << 74: leading bits at 125-126),
//   the one with the smaller exponent is shifted right with the shifted-out
//   bits OR-ed into bit 0 ("sticky"), the two are added or subtracted, the
//   sum is normalised and rounded to 53 bits from its guard and sticky bits.
//
// The window keeps every product bit, and a shifted operand only loses bits
// when it is at least two binades below the other, so at most one leading
// bit cancels and the sticky bit stays far below the rounding position: the
// rounding is correct (the usual argument for a jammed right shift).
// Normal and zero operands with a normal result take the integer path;
// subnormal, infinite or NaN operands and results that overflow or are
// subnormal use the hardware fma, so the function always equals fma(a, b, c).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace bbs {

struct U128 {
    uint64_t hi, lo;
};

// x >> k (k >= 0) with every shifted-out bit OR-ed into bit 0
__device__ __forceinline__ U128 shr_jam(U128 x, int k) {
    if (k == 0) return x;
    U128 r;
    uint64_t lost;
    if (k < 64) {
        lost = x.lo << (64 - k);
        r.lo = (x.lo >> k) | (x.hi << (64 - k));
        r.hi = x.hi >> k;
    } else if (k == 64) {
        lost = x.lo;
        r.lo = x.hi;
        r.hi = 0;
    } else if (k < 128) {
        lost = x.lo | (x.hi << (128 - k));
        r.lo = x.hi >> (k - 64);
        r.hi = 0;
    } else {
        lost = x.lo | x.hi;
        r.lo = 0;
        r.hi = 0;
    }
    r.lo |= (lost != 0) ? 1ull : 0ull;
    return r;
}

__device__ __forceinline__ double fma64_int(double a, double b, double c) {
    const uint64_t A = (uint64_t)__double_as_longlong(a);
    const uint64_t B = (uint64_t)__double_as_longlong(b);
    const uint64_t Cb = (uint64_t)__double_as_longlong(c);
    constexpr uint64_t kM52 = (1ull << 52) - 1;
    const int ea = (int)((A >> 52) & 0x7ff), eb = (int)((B >> 52) & 0x7ff), ec = (int)((Cb >> 52) & 0x7ff);
    const uint64_t sp = (A ^ B) >> 63, sc = Cb >> 63;
    const bool a_zero = (A << 1) == 0, b_zero = (B << 1) == 0, c_zero = (Cb << 1) == 0;
    const bool a_norm = (unsigned)(ea - 1) < 2046u, b_norm = (unsigned)(eb - 1) < 2046u;
    const bool c_norm = (unsigned)(ec - 1) < 2046u;
    if ((a_zero && (b_norm || b_zero)) || (b_zero && a_norm)) {  // exact zero product
        if (c_norm) return c;
        if (c_zero) return __longlong_as_double((long long)((sp & sc) << 63));
        return fma(a, b, c);
    }
    if (!(a_norm && b_norm && (c_norm || c_zero))) return fma(a, b, c);

    const uint64_t ma = (A & kM52) | (1ull << 52), mb = (B & kM52) | (1ull << 52);
    const uint64_t plo = ma * mb, phi = __umul64hi(ma, mb);  // P < 2^106
    U128 X{(phi << 21) | (plo >> 43), plo << 21};
    int Ex = ea + eb - 2150 - 21;  // value = X 2^Ex
    U128 Y{0, 0};
    int Ey = Ex;
    if (!c_zero) {
        Y.hi = ((Cb & kM52) | (1ull << 52)) << 10;  // mc << 74
        Ey = ec - 1075 - 74;
    }
    int E;
    if (Ex >= Ey) {
        Y = shr_jam(Y, Ex - Ey);
        E = Ex;
    } else {
        X = shr_jam(X, Ey - Ex);
        E = Ey;
    }
    U128 S;
    uint64_t sign;
    if (sp == sc) {
        S.lo = X.lo + Y.lo;
        S.hi = X.hi + Y.hi + (S.lo < X.lo ? 1ull : 0ull);
        sign = sp;
    } else {
        const bool x_ge = (X.hi > Y.hi) || (X.hi == Y.hi && X.lo >= Y.lo);
        const U128 G = x_ge ? X : Y, Lw = x_ge ? Y : X;
        S.lo = G.lo - Lw.lo;
        S.hi = G.hi - Lw.hi - (G.lo < Lw.lo ? 1ull : 0ull);
        sign = x_ge ? sp : sc;
    }
    if ((S.hi | S.lo) == 0) return 0.0;  // exact cancellation rounds to +0
    const int L = S.hi ? 127 - __clzll((long long)S.hi) : 63 - __clzll((long long)S.lo);
    int be = E + L + 1023;  // biased exponent of the leading bit
    if (be <= 0) return fma(a, b, c);  // subnormal result
    const int sh = L - 52;
    uint64_t mant;
    bool guard = false, sticky = false;
    if (sh <= 0) {
        mant = S.lo << (-sh);  // exact (S < 2^53)
    } else {
        if (sh < 64)
            mant = (S.lo >> sh) | (sh > 0 ? (S.hi << (64 - sh)) : 0ull);
        else
            mant = S.hi >> (sh - 64);
        const int g = sh - 1;  // guard bit index
        if (g < 64) {
            guard = (S.lo >> g) & 1ull;
            sticky = g > 0 && (S.lo << (64 - g)) != 0;
        } else {
            guard = (S.hi >> (g - 64)) & 1ull;
            sticky = S.lo != 0 || (g > 64 && (S.hi << (128 - g)) != 0);
        }
    }
    if (guard && (sticky || (mant & 1ull))) {
        mant += 1;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            be += 1;
        }
    }
    if (be >= 2047) return fma(a, b, c);  // overflow
    return __longlong_as_double((long long)((sign << 63) | ((uint64_t)be << 52) | (mant & kM52)));
}

}  // namespace bbs
