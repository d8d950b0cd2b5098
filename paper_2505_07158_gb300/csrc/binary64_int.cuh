// Binary64 multiply and add on the integer pipes, bit-identical to IEEE 754 round-to-nearest-even.
//
// On this GPU a binary64 instruction holds its sub-partition's binary64 pipe for ~76 cycles, while the
// integer pipes beside it stay nearly idle: a warp of integer work slows binary64 warps on the same
// sub-partitions by ~7 % (and itself by ~1 %).  These routines let part of the worker chains run their RK4
// steps on the integer pipes.
//
// Method (the textbook one, e.g. Goldberg, "What every computer scientist should know about floating-point
// arithmetic", 1991, and the Handbook of Floating-Point Arithmetic, ch. 7-8): unpack sign, biased exponent and
// the 53-bit significand with its hidden bit; multiply exactly (106-bit product from four 32 x 32 -> 64-bit
// partial products) or add exactly after aligning the smaller operand with three extra low bits (guard,
// round, sticky); normalise; round to nearest, ties to even; repack.  The fast path takes two normal
// operands, or a zero addend, whose result is normal.  Everything else -- zeros in a product, two zero
// addends, subnormal, infinite or NaN operands, a result that overflows or falls below the normal range --
// sets `special`, and the caller computes that lane with the binary64 instruction instead.
#pragma once
#include <cstdint>

namespace fhd {
namespace {

constexpr uint64_t kMant = (1ull << 52) - 1;
constexpr uint64_t kHidden = 1ull << 52;
constexpr uint64_t kSign = 1ull << 63;

// a * b, rounded to nearest even; `special` when the fast path does not apply (the result is then garbage).
__device__ __forceinline__ uint64_t b64_mul(uint64_t A, uint64_t B, bool &special) {
    const uint32_t ea = (uint32_t)(A >> 52) & 0x7ff, eb = (uint32_t)(B >> 52) & 0x7ff;
    special = ea - 1 >= 0x7fe || eb - 1 >= 0x7fe;   // zero, subnormal, infinite or NaN operand
    const uint64_t ma = (A & kMant) | kHidden, mb = (B & kMant) | kHidden;
    const uint32_t al = (uint32_t)ma, ah = (uint32_t)(ma >> 32), bl = (uint32_t)mb, bh = (uint32_t)(mb >> 32);
    // 106-bit product P = hh 2^64 + mid 2^32 + ll (ah, bh < 2^21)
    const uint64_t ll = (uint64_t)al * bl;
    const uint64_t mid = (uint64_t)al * bh + (uint64_t)ah * bl;   // < 2^54
    const uint64_t hh = (uint64_t)ah * bh;                        // < 2^42
    const uint64_t lo = ll + (mid << 32);
    const uint64_t hi = hh + (mid >> 32) + (lo < ll ? 1 : 0);     // P = hi 2^64 + lo, P in [2^104, 2^106)
    const uint32_t n = (uint32_t)(hi >> 41) & 1;                  // P >= 2^105: one more bit above the point
    // 53-bit significand P >> (52 + n), guard bit and sticky bits below it
    uint64_t M = n ? (hi << 11) | (lo >> 53) : (hi << 12) | (lo >> 52);
    const uint64_t rest = n ? lo & ((1ull << 53) - 1) : lo & ((1ull << 52) - 1);
    const uint64_t half = n ? 1ull << 52 : 1ull << 51;
    const bool up = rest > half || (rest == half && (M & 1));
    M += up ? 1 : 0;
    int e = (int)ea + (int)eb - 1023 + (int)n;
    if (M >> 53) {   // rounding carried into a new bit
        M >>= 1;
        ++e;
    }
    special = special || e < 1 || e > 2046;
    return ((A ^ B) & kSign) | ((uint64_t)e << 52) | (M & kMant);
}

// a + b, rounded to nearest even; `special` when the fast path does not apply (the result is then garbage).
__device__ __forceinline__ uint64_t b64_add(uint64_t A, uint64_t B, bool &special) {
    // order by magnitude: |a| >= |b|
    const uint64_t MA = A & ~kSign, MB = B & ~kSign;
    if (MA < MB) {
        const uint64_t t = A;
        A = B;
        B = t;
    }
    const uint32_t ea = (uint32_t)(A >> 52) & 0x7ff, eb = (uint32_t)(B >> 52) & 0x7ff;
    const bool bzero = (B & ~kSign) == 0;
    // the larger operand must be normal; the smaller one normal or a zero (then the sum is a, exactly)
    special = ea - 1 >= 0x7fe || (!bzero && eb - 1 >= 0x7fe);
    if (bzero) return A;   // |a| >= |b| = 0: a + (+-0) = a for a != 0 (a zero a is special above)
    const uint64_t ma = ((A & kMant) | kHidden) << 3;   // 56 bits: significand, guard, round, sticky
    uint64_t mb = ((B & kMant) | kHidden) << 3;
    const uint32_t d = ea - eb;
    if (d >= 56) {
        mb = 1;   // only sticky survives
    } else if (d) {
        const uint64_t lost = mb & ((1ull << d) - 1);
        mb = (mb >> d) | (lost ? 1 : 0);
    }
    int e = (int)ea;
    uint64_t S;
    if (((A ^ B) & kSign) == 0) {
        S = ma + mb;                 // < 2^57
        if (S >> 56) {               // carry: one bit right, keeping the sticky bit
            S = (S >> 1) | (S & 1);
            ++e;
        }
    } else {
        S = ma - mb;                 // >= 0: |a| >= |b|
        if (S == 0) return 0;        // exact cancellation: +0 under round to nearest
        const int lz = __clzll(S) - 8;   // leading zeros below bit 55
        S <<= lz;
        e -= lz;
    }
    // S: bits 55..3 the significand, bit 2 guard, bits 1..0 round and sticky
    const uint32_t low = (uint32_t)S & 7;
    uint64_t M = S >> 3;
    const bool up = low > 4 || (low == 4 && (M & 1));
    M += up ? 1 : 0;
    if (M >> 53) {
        M >>= 1;
        ++e;
    }
    special = special || e < 1 || e > 2046;
    return (A & kSign) | ((uint64_t)e << 52) | (M & kMant);
}

// Warp-level wrappers: the fast path on every lane, and the binary64 instruction on the lanes it does not
// cover (the warp takes that branch only when some lane needs it).  All 32 lanes must call them together.
__device__ __forceinline__ double i64_mul(double a, double b) {
    bool sp;
    uint64_t r = b64_mul((uint64_t)__double_as_longlong(a), (uint64_t)__double_as_longlong(b), sp);
    if (__any_sync(0xffffffffu, sp) && sp) r = (uint64_t)__double_as_longlong(__dmul_rn(a, b));
    return __longlong_as_double((long long)r);
}

__device__ __forceinline__ double i64_add(double a, double b) {
    bool sp;
    uint64_t r = b64_add((uint64_t)__double_as_longlong(a), (uint64_t)__double_as_longlong(b), sp);
    if (__any_sync(0xffffffffu, sp) && sp) r = (uint64_t)__double_as_longlong(__dadd_rn(a, b));
    return __longlong_as_double((long long)r);
}

}  // namespace
}  // namespace fhd
