// Integer arithmetic for the backward phase on GB300's integer pipes.
//
// GB300 executes FP64 at a small fraction of its integer rate, so the
// dependency accumulation of Eq. 2 is done in fixed point:
//
//   for (v, lane) at level l with sigma_v = N * 2^(E - 63) (N normalised,
//   top bit set; E = floor(log2 sigma_v)):
//     A     = sum over successors w of  psi_w * 2^(E + 64)     (u128, exact
//             integer sum of terms truncated below 2^-64 of 2^E)
//     delta = sigma_v * psi_sum = N * A / 2^63 * 2^-64          (u128, units 2^-64)
//     psi_v = (1 + delta) / sigma_v = (R + A) * 2^(-64 - E),  R = floor(2^127 / N)
//
// where psi_w = (1 + delta_w) / sigma_w is stored per (w, lane) as a double
// (its mantissa and exponent are read as integers), with an extra int32
// exponent in the wide format.  Integer sums do not depend on the order of
// their terms, so delta, psi and BC are identical for every schedule.
#pragma once
#include <stdint.h>

namespace gbbc {

typedef unsigned long long u64;

struct u128 {
    u64 lo, hi;
};

__device__ __forceinline__ u128 add128(u128 a, u128 b) {
    u128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

__device__ __forceinline__ u128 mul64(u64 a, u64 b) {
    u128 r;
    r.lo = a * b;
    r.hi = __umul64hi(a, b);
    return r;
}

__device__ __forceinline__ int clz128(u128 a) { return a.hi ? __clzll(a.hi) : 64 + __clzll(a.lo); }

// x * 2^s for s in [-127, 63], as u128 (x < 2^64); bits shifted out below
// 2^0 are dropped.
__device__ __forceinline__ u128 shl_term(u64 x, int s) {
    u128 t;
    if (s >= 0) {
        s = s > 63 ? 63 : s;
        t.lo = x << s;
        t.hi = s ? (x >> (64 - s)) : 0ull;
    } else {
        int r = -s;
        t.lo = r < 64 ? (x >> r) : 0ull;
        t.hi = 0ull;
    }
    return t;
}

// floor(N * A / 2^63) for N < 2^64 and A < 2^127 whose result fits u128.
__device__ __forceinline__ u128 mul_shift63(u64 N, u128 A) {
    u128 p0 = mul64(N, A.lo);  // bits 0..127
    u128 p1 = mul64(N, A.hi);  // bits 64..191
    // 192-bit product (w0, w1, w2)
    u64 w0 = p0.lo;
    u64 w1 = p0.hi + p1.lo;
    u64 c = w1 < p0.hi ? 1ull : 0ull;
    u64 w2 = p1.hi + c;
    u128 r;
    r.lo = (w1 << 1) | (w0 >> 63);
    r.hi = (w2 << 1) | (w1 >> 63);
    return r;
}

// R = floor(2^127 / N) for normalised N in [2^63, 2^64), as u128 (R = 2^64
// exactly when N = 2^63).  A single-precision reciprocal of the top 24 bits,
// reduced by a 2^-20 margin, is a guaranteed under-estimate; two Newton steps
// x <- x + floor(x * (2^127 - N x) / 2^127) approach 2^127/N from below (each
// step's error is N * err^2, so 2^-20 -> 2^-40 -> 2^-80), and a final
// correction makes the remainder 2^127 - N R lie in [0, N).
__device__ __forceinline__ u128 recip127(u64 N) {
    u128 R;
    if (N == 0x8000000000000000ull) {
        R.lo = 0ull;
        R.hi = 1ull;
        return R;
    }
    float nf = __ull2float_rz(N >> 40);           // in [2^23, 2^24)
    float r = __frcp_rn(nf);                      // ~2^-24 relative error
    u64 x = __float2ull_rz(r * 0x1p87f);          // ~ 2^127 / N
    x -= (x >> 20) + 2ull;                        // under-estimate
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        u128 p = mul64(N, x);                     // N x <= 2^127
        u128 e;                                   // 2^127 - N x  (>= 0)
        e.lo = 0ull - p.lo;
        e.hi = 0x8000000000000000ull - p.hi - (p.lo != 0ull ? 1ull : 0ull);
        // floor(x * e / 2^127): 64 x 128 -> 192 bits, take bits 127..190
        u128 q0 = mul64(x, e.lo);
        u128 q1 = mul64(x, e.hi);
        u64 w1 = q0.hi + q1.lo;
        u64 c = w1 < q0.hi ? 1ull : 0ull;
        u64 w2 = q1.hi + c;
        u64 inc = (w2 << 1) | (w1 >> 63);
        x += inc;
    }
    // correction: make 0 <= 2^127 - N x < N
    u128 p = mul64(N, x);
    u128 rem;
    rem.lo = 0ull - p.lo;
    rem.hi = 0x8000000000000000ull - p.hi - (p.lo != 0ull ? 1ull : 0ull);
#pragma unroll 1
    for (int it = 0; it < 4 && (rem.hi != 0ull || rem.lo >= N); ++it) {
        x += 1ull;
        u64 b = rem.lo < N ? 1ull : 0ull;
        rem.lo -= N;
        rem.hi -= b;
    }
    R.lo = x;
    R.hi = 0ull;
    return R;
}

// Round a u128 value times 2^scale to 53 bits (ties to even).  Returns the
// 53-bit integer mantissa M (2^52 <= M < 2^53) and the exponent e with value
// = M * 2^(e - 52); for zero returns M = 0.
__device__ __forceinline__ void round128(u128 a, int scale, u64& M, int& e) {
    if (a.hi == 0ull && a.lo == 0ull) {
        M = 0ull;
        e = 0;
        return;
    }
    int lz = clz128(a);
    int bits = 128 - lz;
    // normalise so that bit 127 is set
    u64 h, l;
    if (lz >= 64) {
        h = a.lo << (lz - 64);
        l = 0ull;
    } else if (lz > 0) {
        h = (a.hi << lz) | (a.lo >> (64 - lz));
        l = a.lo << lz;
    } else {
        h = a.hi;
        l = a.lo;
    }
    u64 keep = h >> 11;
    u64 rem = h & 0x7FFull;
    bool sticky = l != 0ull;
    if (rem > 0x400ull || (rem == 0x400ull && (sticky || (keep & 1ull)))) {
        keep += 1ull;
        if (keep == (1ull << 53)) {
            keep = 1ull << 52;
            bits += 1;
        }
    }
    M = keep;
    e = bits - 1 + scale;
}

// IEEE double bits of M * 2^(e - 52) (normal range: -1022 <= e <= 1023).
__device__ __forceinline__ u64 double_bits(u64 M, int e) {
    if (M == 0ull) return 0ull;
    return ((u64)(e + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull);
}

// Mantissa of the double bits in [1, 2) with the true exponent moved out:
// returns bits with biased exponent 1023.
__device__ __forceinline__ u64 unit_bits(u64 M) {
    return M == 0ull ? 0ull : ((u64)1023 << 52) | (M & 0xFFFFFFFFFFFFFull);
}

// Correctly rounded double of a u128 fixed-point value in units of 2^-64.
__device__ __forceinline__ double fixed_to_double(u128 a) {
    u64 M;
    int e;
    round128(a, -64, M, e);
    return __longlong_as_double((long long)double_bits(M, e));
}

}  // namespace gbbc
