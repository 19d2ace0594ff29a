// hww_device.cuh -- device numerics of the HWW library (sm_103a).
//
// The library and its CPU checker agree on a written numerics contract, and
// each implements it on its own:
//   * counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
//     SC'11) with key (seed_lo, seed_hi ^ n) and counter
//     (id, lineage_lo, lineage_hi, 2 e + s) for event e of a track, word s = 0
//     giving the flight and absorption uniforms, s = 1 the new direction and
//     the roulette uniform;
//   * uniform on (0,1): top 52 bits of a 64-bit word plus one half, times
//     2^-52 (FP64); top 23 bits plus one half times 2^-23 (FP32 tracking);
//   * log: table-driven reduction (128 entries by the top mantissa bits),
//     r = m IC_j - 1, log1p(r) by a degree-9 Horner polynomial with fused
//     multiply-adds, plus (e + K_j) ln 2 (ln 2 split in a 32-bit head and a
//     tail) and the table's T_j; see hw_log;
//   * tallies: contributions rounded to 64-bit integers at a power-of-two
//     scale, summed as 128-bit integers, so that any order of summation
//     gives the same bits.
// FP64 translation units are built with contraction off, so every a*b+c
// below is two roundings unless fma() is written.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hww {

// A 128-bit sum kept in split form so that every update is a pair of
// fire-and-forget reductions (no returned value, no carry test):
//   lo = sum of the low 32-bit halves of the addends (unsigned),
//   hi = sum of the high 32-bit halves (signed, arithmetic shift),
// value = hi 2^32 + lo exactly, as long as fewer than 2^32 addends reach one
// accumulator (each low half is below 2^32).
struct Acc128 {
    unsigned long long lo;
    long long hi;
};

// exact 128-bit value (high word, low word) of a split accumulator
struct I128 {
    long long hi;
    unsigned long long lo;
};

__host__ __device__ __forceinline__ I128 acc_value(Acc128 a) {
    const unsigned long long shifted = (unsigned long long)a.hi << 32;
    const unsigned long long low = shifted + a.lo;
    const long long carry = (low < a.lo) ? 1 : 0;
    return I128{(a.hi >> 32) + carry, low};
}

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// ((x >> 12) + 1/2) 2^-52 of the 64-bit word x: the 52 bits are placed in
// the mantissa of a double m in [1, 2), then 1 is subtracted and 2^-53 added;
// both steps are exact, so the value equals the definition, without an
// integer-to-FP64 conversion (GB300's FP64 pipe is narrow)
__device__ __forceinline__ double u01(uint32_t lo, uint32_t hi) {
    const uint64_t x = ((uint64_t)hi << 32) | lo;
    const double m = __longlong_as_double((long long)(0x3FF0000000000000ull | (x >> 12)));
    return (m - 1.0) + 0x1p-53;
}

// ((hi >> 9) + 1/2) 2^-23, the same way in FP32
__device__ __forceinline__ float u01f(uint32_t hi) {
    const float m = __int_as_float((int)(0x3F800000u | (hi >> 9)));
    return (m - 1.0f) + 0x1p-24f;
}

// Natural logarithm of u in (0, 1), the numerics contract's steps:
// u = 2^e m with m in [1, 2); j = the top 7 bits of m's mantissa; from the
// table (log_table.inc) IC_j ~ 1/c_j and T_j = -log(IC_j 2^K_j), K_j = [j >= 64];
// r = m IC_j - 1 in one fused multiply-add (|r| < 2^-7);
// log1p(r) = r + r^2 (-1/2 + r/3 - r^2/4 + ... + r^7/9) by Horner's rule;
// log u = (e + K_j) (ln2_hi + ln2_lo) + T_j + log1p(r), ln 2 split into a
// 32-bit head and a tail.  No division (an FP64 divide is about ten
// instructions on GB300's narrow FP64 pipe); within 2 ulp.
#include "log_table.inc"

__device__ __forceinline__ double hw_log(double u) {
    const long long b = __double_as_longlong(u);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const long long mant = b & 0x000fffffffffffffLL;
    const double m = __longlong_as_double(mant | 0x3ff0000000000000LL);
    const int j = (int)(mant >> 45);
    const double r = fma(m, __ldg(&LOG_IC[j]), -1.0);
    double q = 1.0 / 9.0;
    q = fma(q, r, -1.0 / 8.0);
    q = fma(q, r, 1.0 / 7.0);
    q = fma(q, r, -1.0 / 6.0);
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -1.0 / 4.0);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -1.0 / 2.0);
    const double r2 = r * r;
    const double p = fma(r2, q, r);
    const double kd = (double)(e + (j >> 6));
    const double hi = fma(kd, 0x1.62e42fee00000p-1, __ldg(&LOG_T[j]));
    const double lo = fma(kd, 0x1.a39ef35793c76p-33, p);
    return hi + lo;
}

// lineage key of daughter j of a split at event e of a track with key `lin`
__host__ __device__ __forceinline__ uint64_t lineage_hash(uint64_t lin, uint32_t e, uint32_t j) {
    uint32_t c[4] = {(uint32_t)lin, (uint32_t)(lin >> 32), e, j};
    philox4x32_10(c, 0x4C494E45u, 0x41474521u);
    return ((uint64_t)c[1] << 32) | c[0];
}

// x * scale rounded to the nearest 64-bit integer (ties to even); scale is a
// power of two, so the product is exact
__device__ __forceinline__ long long to_fixed(double x, double scale) {
    return __double2ll_rn(x * scale);
}

// The same value, x 2^S rounded to the nearest integer (ties to even), from
// the bits of x in integer arithmetic: the hot loops' FP64 pipe (two
// instructions here) is the scarce unit on GB300, the integer ALU is not.
// |x| 2^S must stay below 2^63 (the tally scales are chosen so).
__device__ __forceinline__ long long fixed_bits(double x, int S) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FFu);
    if (ex == 0) return 0;  // zero or subnormal: far below one unit
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = ex - 1075 + S;  // |x| 2^S = m 2^sh
    unsigned long long v;
    if (sh >= 0) {
        v = m << sh;
    } else if (sh > -64) {
        const int s = -sh;
        const unsigned long long q = m >> s, rem = m & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        v = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    } else {
        v = 0;
    }
    return (b >> 63) ? -(long long)v : (long long)v;
}

// add a signed 64-bit value to a split accumulator
__device__ __forceinline__ void add128(Acc128* a, long long v) {
    if (v == 0) return;
    atomicAdd(&a->lo, (unsigned long long)(unsigned)(v & 0xFFFFFFFFll));
    const long long h = v >> 32;
    if (h != 0) atomicAdd((unsigned long long*)&a->hi, (unsigned long long)h);
}

// 128-bit value to double: one rounding when it fits a signed 64-bit
// integer, else hi*2^64 + lo
__host__ __device__ __forceinline__ double i128_to_double(I128 v) {
    const bool fits = (v.hi == 0 && (long long)v.lo >= 0) || (v.hi == -1 && (long long)v.lo < 0);
    if (fits) return (double)(long long)v.lo;
    return (double)v.hi * 0x1p64 + (double)v.lo;
}

__host__ __device__ __forceinline__ double acc_to_double(Acc128 a) { return i128_to_double(acc_value(a)); }

// 2^e as a double for -1022 <= e <= 1023
__host__ __device__ __forceinline__ double pow2(int e) {
    union {
        unsigned long long u;
        double d;
    } v;
    v.u = (unsigned long long)(e + 1023) << 52;
    return v.d;
}

// FP32 path: a weight at the tally scale rounded to FP32, a = fl32(w 2^S)
// (the scaling by 2^S is exact in FP64, so this is one rounding of w's
// significand to 24 bits)
__device__ __forceinline__ float tally_weight(double w, double scale) { return __double2float_rn(w * scale); }

// fl32(x 2^k) for x > 0 (nearest, ties to even) from the bits of x, in
// integer arithmetic: the 53-bit significand rounded to 24 bits, the
// exponent moved by k (a carry out of the significand moves into the
// exponent field by itself).  Where the result would not be a normal FP32
// number, the FP64 conversion gives it (the same value).  The hot loops use
// this instead of FP64 instructions (GB300's FP64 pipe is narrow).
__device__ __forceinline__ float fl32_scaled(double x, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ed = (int)(b >> 52);  // x > 0: no sign bit
    const int e = ed - 1023 + k + 127;
    if (ed == 0 || ed == 0x7FF || e < 1 || e > 254) return __double2float_rn(x * pow2(k));
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned long long q = m >> 29, r = m & 0x1FFFFFFFull;
    const unsigned long long f = q + ((r > 0x10000000ull || (r == 0x10000000ull && (q & 1ull))) ? 1ull : 0ull);
    return __uint_as_float(((unsigned)e << 23) + (unsigned)(f - 0x800000ull));
}

// the tally weight of the FP32 path, fl32(w 2^S), without FP64 instructions
__device__ __forceinline__ float tally_weight_bits(double w, int S) { return fl32_scaled(w, S); }

// FP32 path: the tally contribution round(a f) of an FP32 factor f to an FP32
// weight a > 0 at the tally scale, rounded half up, from the exact 48-bit
// product P of the two 24-bit significands (one 32 x 32 -> 64-bit multiply):
// a f = P 2^(ea + ef - 300) with ea, ef the biased exponents.  A zero or
// subnormal operand counts as 0.
__device__ __forceinline__ long long fx_mul24(float a, float f) {
    const unsigned ua = __float_as_uint(a), uf = __float_as_uint(f);
    const int ea = (int)((ua >> 23) & 0xFFu), ef = (int)((uf >> 23) & 0xFFu);
    const unsigned long long P =
        (unsigned long long)((ua & 0x7FFFFFu) | 0x800000u) * (unsigned long long)((uf & 0x7FFFFFu) | 0x800000u);
    const int s = 300 - ea - ef;  // a f = P 2^-s
    unsigned long long r;
    if (s > 0) {
        // P < 2^48, so the rounding increment never carries out of 64 bits,
        // and s >= 49 leaves 0 (the shift is capped at 63)
        const int t = s < 63 ? s : 63;
        r = (P + (1ull << (t - 1))) >> t;
    } else {
        r = P << (-s < 15 ? -s : 15);  // a f >= 2^48, far above any tally scale's contributions
    }
    if (ea == 0 || ef == 0) r = 0;
    return (uf >> 31) ? -(long long)r : (long long)r;
}

}  // namespace hww
