// Integer arithmetic of the emulated-FP64 products (HTS_GEMM_EMU_BF16), shared by the
// mma.sync kernel (emu.cu) and the tcgen05 kernel (emu_tc.cu).
//
// Every operand is written as a fixed-point integer with a shared scale, x = round(v 2^-unit),
// split into 8 balanced base-256 digits d_1..d_8 in [-128, 127] (x = sum d_i 256^(8-i)); each
// digit is exact in BF16.  A product of a line window with U_k is the sum over digit pairs
// (i, t) of (digits_i of the lines) (digits_t of U_k), weighted by 256^-(i+t); pairs with the
// same level i + t share an FP32 accumulator, in which every partial sum is an integer below
// 2^22 in magnitude and hence exact.  Levels 2..9 are formed and summed in 64-bit integer
// arithmetic.  FP64 values enter and leave through integer manipulation of their IEEE-754
// encoding, so no FP64 instruction runs in the update loop.
#pragma once

#include "hts_internal.cuh"

namespace hts {
namespace emu {

constexpr int kDigits = 8;                 // balanced base-256 digits per operand
constexpr int kTopLevel = 9;               // digit pairs with i + t <= 9 are formed
constexpr int kPlaneWords = kDigits * 2 * 4 * 32;   // uint2 words of one U_k (16 KiB)
constexpr int kUnitU = -61;                // U_k entries as integers round(u 2^61)
constexpr int kZeroExp = -4000;            // "exponent" of a zero value

// Operand K index of window position p (0..31) in the tcgen05 kernel.  A product sums over K,
// so any order of the positions serves as long as both operands use it; this one puts the
// positions 2j, 2j+1, 16+2j, 17+2j (the four a thread of that kernel holds) at K = 4j .. 4j+3,
// next to each other in a core-matrix row, so that a thread writes them with one 8-byte store.
__host__ __device__ __forceinline__ int tc_kidx(int p) { return 4 * ((p & 15) >> 1) + (p & 1) + 2 * (p >> 4); }

// ---- IEEE-754 double <-> fixed point (integer arithmetic only) --------------------------

// Smallest e with |v| < 2^e, or kZeroExp for zero and subnormal v (treated as zero).
__device__ __forceinline__ int exp_of_f64(double v)
{
    const int eb = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
    return eb == 0 ? kZeroExp : eb - 1022;
}

// Smallest e with |x 2^unit| < 2^e, or kZeroExp.
__device__ __forceinline__ int exp_of_fixed(long long x, int unit)
{
    if (x == 0) return kZeroExp;
    const unsigned long long m = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
    return 64 - __clzll(m) + unit;
}

// round(v 2^-unit) for |v| < 2^(unit + 62); zero and subnormal v give 0.
__device__ __forceinline__ long long f64_to_fixed(double v, int unit)
{
    const long long b = __double_as_longlong(v);
    const int eb = (int)((b >> 52) & 0x7ff);
    if (eb == 0) return 0;
    const long long mant = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;   // v = +-mant 2^(eb-1075)
    const int sh = eb - 1075 - unit;
    long long x;
    if (sh >= 0) x = mant << sh;
    else if (sh > -63) x = (mant + (1LL << (-sh - 1))) >> (-sh);
    else x = 0;
    return b < 0 ? -x : x;
}

// x 2^unit rounded to the nearest double (ties to even); results below the normal range
// become signed zero.
__device__ __forceinline__ double fixed_to_f64(long long x, int unit)
{
    if (x == 0) return 0.0;
    const unsigned long long sgn = x < 0 ? 0x8000000000000000ULL : 0ULL;
    unsigned long long m = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
    const int lz = __clzll(m);
    m <<= lz;                                    // leading one at bit 63
    const int eb = 63 - lz + unit + 1023;        // biased exponent of the result
    if (eb <= 0) return __longlong_as_double((long long)sgn);
    unsigned long long mant = m >> 11;           // 53 bits including the leading one
    const unsigned long long rem = m & 0x7ffULL;
    if (rem > 0x400ULL || (rem == 0x400ULL && (mant & 1ULL))) ++mant;
    // the leading one of mant adds 1 to the exponent field; a rounding carry adds one more
    const unsigned long long bits = ((unsigned long long)(eb - 1) << 52) + mant;
    return __longlong_as_double((long long)(sgn | bits));
}

// x 2^su expressed in units 2^du (rounded), for values known to fit.
__device__ __forceinline__ long long refix(long long x, int su, int du)
{
    const int s = su - du;
    if (s >= 0) return x << s;
    if (s > -63) return (x + (1LL << (-s - 1))) >> (-s);
    return 0;
}

// ---- balanced digits --------------------------------------------------------------------

// BF16 bit patterns of the 8 balanced base-256 digits of x (|x| < 2^62), most significant
// first, in the upper halves of FP32 words: with u = x + 0x8080808080808080 (no wrap-around
// in that range), digit i is byte (8 - i) of u minus 128.  One byte permute places the byte
// under the exponent of 2^23 and one subtraction removes 2^23 + 128; a digit in [-128, 127]
// has 16 trailing zero bits in FP32, so the upper half of its encoding is its exact BF16.
__device__ __forceinline__ void digits_bf16(long long x, unsigned (&bf)[kDigits])
{
    const unsigned long long u = (unsigned long long)x + 0x8080808080808080ULL;
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
#pragma unroll
    for (int i = 0; i < kDigits; ++i) {
        const unsigned word = (i < 4) ? hi : lo;
        const unsigned sel = 0x7650u | (unsigned)(3 - (i & 3));   // bytes {b, 0, 0, 0x4B}
        bf[i] = __float_as_uint(__uint_as_float(__byte_perm(word, 0x4B000000u, sel)) - 8388736.0f);
    }
}

// Two BF16 values (the upper halves of the FP32 words lo and hi) in one register, lo in the
// low half.
__device__ __forceinline__ unsigned pack_bf16(unsigned lo, unsigned hi) { return __byte_perm(lo, hi, 0x7632u); }

// An FP32 value holding an integer of magnitude below 2^22, as int (exact).
__device__ __forceinline__ int f32_exact_int(float c) { return __float_as_int(c + 12582912.0f) - 0x4B400000; }


// Levels 2..9 of one product (c[0] = level 2 .. c[7] = level 9, FP32 sums of exact integers)
// as one integer in units 2^(ua + 3) when the line's unit is ua and U's is 2^-61: level L
// weighs 2^(8 (8 - L)); level 9 is rounded into level 8's unit.
__device__ __forceinline__ long long combine_levels(float c2f, float c3f, float c4f, float c5f, float c6f, float c7f,
                                                    float c8f, float c9f)
{
    const int c2 = f32_exact_int(c2f), c3 = f32_exact_int(c3f);
    const int c4 = f32_exact_int(c4f), c5 = f32_exact_int(c5f);
    const int c6 = f32_exact_int(c6f), c7 = f32_exact_int(c7f);
    const int c8 = f32_exact_int(c8f), c9 = f32_exact_int(c9f);
    const int lo = (c7 << 8) + c8 + ((c9 + 128) >> 8);
    const int mid = (c5 << 8) + c6;
    const long long hi = ((long long)c2 << 16) + (long long)((c3 << 8) + c4);
    return (hi << 32) + ((long long)mid << 16) + (long long)lo;
}

// ---- FP16 digit pairs (the tcgen05 kernel's operands) --------------------------------------

// FP16 bit patterns of the 8 balanced base-256 digits of two values x0, x1 (|x| < 2^62), most
// significant first, packed in pairs: word i holds digit i of x0 in its low half and of x1 in
// its high half.  With u = x + 0x8080808080808080, digit i is byte 7-i of u minus 128.  One byte
// permute places the two bytes under the FP16 exponent of 2^10 (the halves read 1024 + byte,
// exactly, since FP16 steps by 1 in [1024, 2048)), one AND/OR clears the other bytes and sets
// that exponent, and one packed FP16 subtraction of 1024 + 128 leaves the digits, exact because
// they are integers of magnitude at most 128.
__device__ __forceinline__ void digit_pairs_f16(long long x0, long long x1, unsigned (&w)[kDigits])
{
    const unsigned long long u0 = (unsigned long long)x0 + 0x8080808080808080ULL;
    const unsigned long long u1 = (unsigned long long)x1 + 0x8080808080808080ULL;
    const unsigned h0 = (unsigned)(u0 >> 32), l0 = (unsigned)u0, h1 = (unsigned)(u1 >> 32), l1 = (unsigned)u1;
#pragma unroll
    for (int i = 0; i < kDigits; ++i) {
        const unsigned by = 3u - (unsigned)(i & 3);   // byte of the word holding digit i
        const unsigned sel = by | (by << 4) | ((by + 4u) << 8) | ((by + 4u) << 12);
        const unsigned t = (__byte_perm(i < 4 ? h0 : l0, i < 4 ? h1 : l1, sel) & 0x00FF00FFu) | 0x64006400u;
        unsigned d;
        asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(t), "r"(0x64806480u));
        w[i] = d;
    }
}

// Two FP16 values (the low halves of the words lo and hi) in one register, lo in the low half.
__device__ __forceinline__ unsigned pack_f16(unsigned lo, unsigned hi) { return __byte_perm(lo, hi, 0x5410u); }

// combine_levels with the FP32-to-integer bias of the levels removed once per group of levels
// instead of once per level: bits(c + 1.5 2^23) = 0x4B400000 + c for the exact integers c, and
// the sums below are taken modulo 2^32 (lo, mid) or 2^64 (hi), where the biases cancel exactly.
__device__ __forceinline__ long long combine_levels_folded(float c2f, float c3f, float c4f, float c5f, float c6f,
                                                           float c7f, float c8f, float c9f)
{
    constexpr unsigned K = 0x4B400000u;
    const float m = 12582912.0f;
    const unsigned b2 = __float_as_uint(c2f + m), b3 = __float_as_uint(c3f + m), b4 = __float_as_uint(c4f + m);
    const unsigned b5 = __float_as_uint(c5f + m), b6 = __float_as_uint(c6f + m), b7 = __float_as_uint(c7f + m);
    const unsigned b8 = __float_as_uint(c8f + m), b9 = __float_as_uint(c9f + m);
    const int lo = (int)((b7 << 8) + b8 - K * 257u) + ((int)(b9 - (K - 128u)) >> 8);
    const int mid = (int)((b5 << 8) + b6 - K * 257u);
    const long long hi = (long long)(((unsigned long long)b2 << 16) + ((unsigned long long)b3 << 8) + b4 -
                                     (unsigned long long)K * 65793ull);
    return (hi << 32) + ((long long)mid << 16) + (long long)lo;
}

}  // namespace emu
}  // namespace hts
