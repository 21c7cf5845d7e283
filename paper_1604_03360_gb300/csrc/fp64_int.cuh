// fp64_int.cuh -- IEEE 754 binary64 multiplication carried out with 32-bit
// integer instructions.
//
// Why: on this part the FP64 pipe retires 2 operations per clock per SM while
// the integer pipes retire about 64, and the WENO stage kernels keep the FP64
// pipe busy with the issue slots mostly idle.  A product computed on the
// integer pipe frees one FP64 slot (64 clocks of a scheduler's FP64 unit per
// warp instruction) for about 40 integer instructions (fewer for a constant
// factor).  The stage kernels use it for the products with constants, which
// sit early in each reconstruction's dependency chain; products on the
// critical path (the nonlinear weights) and the stencil differences stay on
// the FP64 unit, where moving them measured slower.
//
// What: dmul_int(x, y) returns exactly the round-to-nearest-even product that
// IEEE 754-2008 defines (Sec. 4.3.1, 5.4.1), the value the FP64 unit returns
// for x * y; dmul_pow2_bits / dmul_small_bits are cheaper forms for factors
// 2^k and small odd integers times 2^k.  The integer path covers finite normal operands and zeros whose
// product is a normal number or zero; subnormal, infinite and NaN operands, and
// products that overflow or fall below the normal range, are handed to the
// FP64 unit.  The method is the textbook one (e.g. Muller et al., Handbook of
// Floating-Point Arithmetic, Ch. 7): multiply the 53-bit significands exactly
// (106 bits from four 32 x 32 -> 64-bit products), normalise by at most one
// bit, and round with a guard bit and a sticky bit.
//
// The header also compiles as plain C++ (host), so the same source is tested
// against the host's IEEE multiplication.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define HYDRO_HD __host__ __device__ __forceinline__
#else
#define HYDRO_HD inline
#endif

namespace hydro {

HYDRO_HD uint64_t f64_to_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

HYDRO_HD double f64_from_bits(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, sizeof x);
    return x;
#endif
}

// Integer-path product; false when the operands or the result need the FP64
// unit (see above).
HYDRO_HD bool dmul_int_bits(uint64_t a, uint64_t b, uint64_t& r)
{
    const uint32_t ah = (uint32_t)(a >> 32), bh = (uint32_t)(b >> 32);
    const uint32_t al = (uint32_t)a, bl = (uint32_t)b;
    const uint32_t ea = (ah >> 20) & 0x7ffu, eb = (bh >> 20) & 0x7ffu;
    const uint64_t sign = (uint64_t)((ah ^ bh) & 0x80000000u) << 32;
    if (ea - 1u >= 0x7feu || eb - 1u >= 0x7feu) {
        // a zero or subnormal (exponent 0), or an infinity or NaN (0x7ff)
        if (ea == 0x7ffu || eb == 0x7ffu) return false;
        const bool za = ((a << 1) == 0), zb = ((b << 1) == 0);
        if (!(za || zb)) return false;          // subnormal operand
        r = sign;                               // finite x 0 = signed zero
        return true;
    }
    // significands with the hidden bit: (mh << 32) | l, mh < 2^21
    const uint32_t mah = (ah & 0xfffffu) | 0x100000u, mbh = (bh & 0xfffffu) | 0x100000u;
    // p = ma mb = hh 2^64 + mid 2^32 + ll, in [2^104, 2^106)
    const uint64_t ll = (uint64_t)al * bl;
    const uint64_t mid = (uint64_t)mah * bl + (uint64_t)al * mbh + (ll >> 32);   // < 2^55
    const uint64_t hh = (uint64_t)mah * mbh + (mid >> 32);                       // p >> 64, < 2^42
    // x = p >> 42 (leading bit 63 or 62); the bits below it only decide stickiness
    const uint64_t x = (hh << 22) | ((uint32_t)mid >> 10);
    const bool below = (((uint32_t)mid & 0x3ffu) | (uint32_t)ll) != 0u;
    const uint32_t t = (uint32_t)(x >> 63);                  // 1: product of significands >= 2
    const uint64_t y = x << (1u - t);                        // leading bit at 63
    uint64_t m = y >> 11;                                    // 53-bit significand
    const uint64_t guard = (y >> 10) & 1u;
    const uint64_t sticky = ((y & 0x3ffu) != 0u || below) ? 1u : 0u;
    m += guard & (sticky | (m & 1u));                        // round to nearest, ties to even
    int e = (int)ea + (int)eb - 1023 + (int)t;               // biased exponent of the result
    if (m >> 53) {                                           // rounding carried out: m = 2^53
        m >>= 1;
        e += 1;
    }
    if (e < 1 || e > 2046) return false;                     // subnormal or overflowing result
    r = sign | (((uint64_t)(e - 1) << 52) + m);              // the hidden bit adds the last 1
    return true;
}

HYDRO_HD double dmul_int(double x, double y)
{
    uint64_t r;
    if (dmul_int_bits(f64_to_bits(x), f64_to_bits(y), r)) return f64_from_bits(r);
    return x * y;
}

// x * 2^k on the integer path: an exponent shift, exact for normal x whose
// result stays normal, and zeros keep their sign.
HYDRO_HD bool dmul_pow2_bits(uint64_t a, int k, uint64_t& r)
{
    const uint32_t ea = (uint32_t)(a >> 52) & 0x7ffu;
    if (ea - 1u >= 0x7feu) {
        if ((a << 1) != 0) return false;        // subnormal, infinity or NaN
        r = a;
        return true;
    }
    const int e = (int)ea + k;
    if (e < 1 || e > 2046) return false;
    r = a + ((uint64_t)(int64_t)k << 52);
    return true;
}

// x * (c 2^k) for an odd integer 1 < c < 2^CB, 2^(CB-1) <= c: the product of
// the 53-bit significand and c fits in 64 bits, so one integer product, a
// one-bit normalisation and the rounding give the IEEE result.
template <int CB>
HYDRO_HD bool dmul_small_bits(uint64_t a, uint32_t c, int k, uint64_t& r)
{
    static_assert(CB >= 2 && CB <= 10, "small odd factor");
    const uint32_t ea = (uint32_t)(a >> 52) & 0x7ffu;
    const uint64_t sign = a & 0x8000000000000000ull;
    if (ea - 1u >= 0x7feu) {
        if ((a << 1) != 0) return false;
        r = sign;                               // zero times a positive factor
        return true;
    }
    const uint64_t p = ((a & 0xfffffffffffffull) | 0x10000000000000ull) * c;   // [2^(51+CB), 2^(53+CB))
    const uint32_t t = (uint32_t)(p >> (52 + CB));                          // 1: leading bit at 52 + CB
    const uint64_t y = p << (1u - t);                                       // leading bit at 52 + CB
    uint64_t m = y >> CB;
    const uint64_t guard = (y >> (CB - 1)) & 1u;
    const uint64_t sticky = (y & ((1ull << (CB - 1)) - 1u)) != 0u ? 1u : 0u;
    m += guard & (sticky | (m & 1u));
    int e = (int)ea + k + (CB - 1) + (int)t;
    if (m >> 53) {
        m >>= 1;
        e += 1;
    }
    if (e < 1 || e > 2046) return false;
    r = sign | (((uint64_t)(e - 1) << 52) + m);
    return true;
}

// Which products of a kernel run on the integer pipe (bit flags of a kernel's
// EMU template argument): the products with constants, the squares and
// products of the nonlinear weights, the last products of the weighted sums
// and of the face combination.
constexpr int kEmuConst = 1, kEmuWeights = 2, kEmuFace = 4;

// Operations on the integer pipe (E) or the FP64 unit; both give the same bits.
template <bool E>
HYDRO_HD double xmul(double x, double y)
{
    if constexpr (E) return dmul_int(x, y);
    else return x * y;
}

// x * 2^K
template <bool E, int K>
HYDRO_HD double xmul_pow2(double x)
{
    constexpr double f = K >= 0 ? (double)(1ull << (K >= 0 ? K : 0)) : 1.0 / (double)(1ull << (K < 0 ? -K : 0));
    if constexpr (E) {
        uint64_t r;
        if (dmul_pow2_bits(f64_to_bits(x), K, r)) return f64_from_bits(r);
    }
    return x * f;
}

// x * (C 2^K), C odd with CB bits
template <bool E, int C, int CB, int K>
HYDRO_HD double xmul_small(double x)
{
    static_assert((C & 1) && C < (1 << CB) && C >= (1 << (CB - 1)), "C must be odd with CB bits");
    constexpr double f = K >= 0 ? (double)C * (double)(1ull << (K >= 0 ? K : 0))
                                : (double)C / (double)(1ull << (K < 0 ? -K : 0));
    if constexpr (E) {
        uint64_t r;
        if (dmul_small_bits<CB>(f64_to_bits(x), (uint32_t)C, K, r)) return f64_from_bits(r);
    }
    return x * f;
}

}  // namespace hydro
