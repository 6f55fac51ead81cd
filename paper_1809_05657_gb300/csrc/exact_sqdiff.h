// exact_sqdiff.h -- (x - y)^2 of two binary32 numbers in binary64, by integer arithmetic.
//
// The residual kernel stores q = RN64(d * d) with d = RN64(x - y) for binary32 (or bfloat16)
// fields x, y, exactly as binary64 instructions would.  On this GPU the binary64 pipe is narrow,
// so the common case is done with integer operations, which give the same bits:
//
//   * x = sx * Mx * 2^(ex - 150), y = sy * My * 2^(ey - 150) with 24-bit significands Mx, My
//     (normal numbers; a zero has M = 0).  With g = |ex - ey| <= 28 the operand with the larger
//     exponent is shifted left by g, and D = (+-Mx << g) - (+-My) is the exact difference as an
//     integer times 2^(min(ex, ey) - 150), |D| < 2^53: binary64 holds d exactly.
//   * d * d = D^2 * 2^(2 (min(ex, ey) - 150)), with D^2 < 2^106 formed as a 128-bit product; its
//     top 53 bits are rounded to nearest, ties to even, as the binary64 multiply does.  The
//     exponent always lies in binary64's normal range (the operands are normal binary32 numbers).
//
// Anything else -- subnormal, infinite or NaN operands, exponents more than 28 apart -- returns
// false and the caller takes the binary64 instructions.  The same source compiles for the host,
// where a test compares it with IEEE binary64 arithmetic.
//
// sqdiff_f32_exact serves the common case of a residual, two close values, with fewer integer
// operations: s = RN32(x - y) and its rounding error by the error-free transformation TwoSum
// (Knuth, TAOCP vol. 2, 4.2.2; six binary32 additions).  When the error is zero, s is the exact
// difference d, its 24-bit significand M squares exactly in 48 bits, and d * d = M^2 * 2^(2 e)
// needs no rounding in binary64: the bits come from one 32 x 32 -> 64-bit product.  A nonzero
// error, a subnormal, infinite or NaN s returns false (the caller takes sqdiff_f32_bits).
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define HDA_HD __host__ __device__ __forceinline__
#else
#define HDA_HD inline
#endif

namespace hda {

HDA_HD int hda_clz64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return __builtin_clzll(v);
#endif
}

HDA_HD uint64_t hda_mulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// bits of RN64((x - y)^2) for the binary32 bit patterns ux, uy; false when outside the integer path
HDA_HD bool sqdiff_f32_bits(uint32_t ux, uint32_t uy, uint64_t &qbits)
{
    const uint32_t ex = (ux >> 23) & 0xffu, ey = (uy >> 23) & 0xffu;
    const uint32_t mx = ux & 0x7fffffu, my = uy & 0x7fffffu;
    const bool zx = (ux & 0x7fffffffu) == 0, zy = (uy & 0x7fffffffu) == 0;
    // normal or zero operands only
    if ((!zx && (ex - 1u) >= 254u) || (!zy && (ey - 1u) >= 254u)) return false;
    int64_t X = zx ? 0 : (int64_t)(mx | 0x800000u), Y = zy ? 0 : (int64_t)(my | 0x800000u);
    // exponent of the unit of the smaller operand; a zero takes the other operand's exponent
    int e_hi = (int)(zx ? ey : ex), e_lo = (int)(zy ? ex : ey);
    int e;
    if (e_hi >= e_lo) {
        const int g = e_hi - e_lo;
        if (g > 28) return false;
        X <<= g;
        e = e_lo;
    } else {
        const int g = e_lo - e_hi;
        if (g > 28) return false;
        Y <<= g;
        e = e_hi;
    }
    if (ux >> 31) X = -X;
    if (uy >> 31) Y = -Y;
    const int64_t D = X - Y;  // d = D * 2^(e - 150), |D| < 2^53
    if (D == 0) {             // x - y = +0 in round to nearest; its square is +0
        qbits = 0;
        return true;
    }
    const uint64_t A = (uint64_t)(D < 0 ? -D : D);
    const uint64_t lo = A * A, hi = hda_mulhi64(A, A);
    const int P = hi ? 127 - hda_clz64(hi) : 63 - hda_clz64(lo);  // top bit of D^2
    const int E2 = 2 * (e - 150);                                 // D^2 * 2^E2
    uint64_t M;
    int top = P;
    if (P <= 52) {
        M = lo << (52 - P);  // exact
    } else {
        const int s = P - 52;  // 1 .. 53: bits shifted out, all in lo
        M = (lo >> s) | (s < 64 ? (hi << (64 - s)) : 0);
        const uint64_t rbit = (lo >> (s - 1)) & 1u;
        const uint64_t sticky = lo & ((((uint64_t)1) << (s - 1)) - 1u);
        if (rbit && (sticky || (M & 1u))) {
            M += 1;
            if (M >> 53) {  // carried into a new top bit
                M >>= 1;
                top += 1;
            }
        }
    }
    qbits = ((uint64_t)(top + E2 + 1023) << 52) | (M & 0x000fffffffffffffull);
    return true;
}

#ifdef __CUDA_ARCH__
#define HDA_FADD(a, b) __fadd_rn((a), (b))
#else
#define HDA_FADD(a, b) ((a) + (b))  // the host build compiles without contraction (-ffp-contract=off)
#endif

// bits of RN64((x - y)^2) when RN32(x - y) is exact and normal or zero; false otherwise
HDA_HD bool sqdiff_f32_exact(float x, float y, uint64_t &qbits)
{
    const float a = x, b = -y;
    const float s = HDA_FADD(a, b);
    const float bb = HDA_FADD(s, -a);
    const float err = HDA_FADD(HDA_FADD(a, -HDA_FADD(s, -bb)), HDA_FADD(b, -bb));
    if (!(err == 0.0f)) return false;  // inexact, or infinite / NaN operands
    uint32_t u;
    memcpy(&u, &s, 4);
    if ((u & 0x7fffffffu) == 0) {  // x - y = 0: the square is +0
        qbits = 0;
        return true;
    }
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0 || e == 0xffu) return false;  // subnormal or not finite
    const uint64_t M = (uint64_t)((u & 0x7fffffu) | 0x800000u);
    const uint64_t P = M * M;                  // 2^46 <= P < 2^48: d^2 = P * 2^(2 (e - 150)), exact
    const int top = (P >> 47) ? 47 : 46;       // leading bit of P
    const uint64_t mant = (P << (52 - top)) & 0x000fffffffffffffull;
    qbits = ((uint64_t)(2 * ((int)e - 150) + top + 1023) << 52) | mant;
    return true;
}

#undef HDA_FADD

}  // namespace hda
