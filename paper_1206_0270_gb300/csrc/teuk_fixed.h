// teuk_fixed.h -- sums of products of FP64 numbers in 64-bit fixed point.
//
// The Pi rows of the predictor (Eq. 3) and corrector (Eq. 4) are short sums
// sum_k f_k c_k x_k (f_k = +-1, 6 to 10 terms) of FP64 coefficients and
// fields.  GB300 issues FP64 FMAs at under 2 per clock per SM but 32-bit
// integer multiply-adds at about 60, so these sums are evaluated on the
// integer pipe:
//
//   * each operand is split into its 53-bit significand m and exponent e,
//     value = m 2^(e - 1075) (subnormals and zero fields: no hidden bit,
//     e = 1, which is exact; a zero coefficient never sets the frame);
//   * each product m_c m_x (at most 106 bits) is formed exactly with four
//     32 x 32 -> 64-bit multiply-adds;
//   * all products are aligned to the largest product exponent E and
//     truncated to units of 2^(E - 2103): the largest product keeps at least
//     57 bits (2^104 <= m_c m_x), every product is below 2^59 units, and up
//     to 16 of them sum without overflow in a signed 64-bit integer;
//   * the integer sum is rounded once to FP64, to nearest, ties to even (on
//     the device by the hardware int64 -> FP64 conversion, the frame's power
//     of two added to the exponent field; on the host by integer rounding,
//     with the same bits).
//
// Error: |result - exact| <= n 2^-57 max_k |c_k x_k| + 2^-53 |exact|
// (truncation of n products, then one rounding), which is at or below the
// error of the same sum formed by FP64 fused multiply-adds (each of its n
// roundings is relative to a partial sum).  Integer addition is exact and
// associative, so the result does not depend on the order of the terms, and
// terms whose coefficient or field is zero add nothing; a zero coefficient
// does not take part in the choice of the frame either.
//
// The sum reports failure, and the caller evaluates it with FP64 FMAs
// instead, when an input is not finite or the result is below 2^-823 (there
// a product with a subnormal or zero field, counted at the exponent of the
// smallest subnormal, could have set the frame; coefficients of the scheme
// are far below the 2^170 this bound allows) or would overflow.
//
// Everything here is plain integer arithmetic on host and device, so the
// same code is tested on the CPU against exact rational arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define TEUK_FX_HD __host__ __device__ __forceinline__
#else
#define TEUK_FX_HD static inline
#endif

namespace teuk {

TEUK_FX_HD uint64_t fx_bits(double v)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t u;
    memcpy(&u, &v, sizeof u);
    return u;
#endif
}

TEUK_FX_HD double fx_double(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double v;
    memcpy(&v, &u, sizeof v);
    return v;
#endif
}

TEUK_FX_HD int fx_clz64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// p >> s for any s >= 0 (0 once s >= 64; PTX shr clamps the shift count)
TEUK_FX_HD uint64_t fx_shr(uint64_t p, uint32_t s)
{
#ifdef __CUDA_ARCH__
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(p), "r"(s));
    return r;
#else
    return s >= 64 ? 0 : p >> s;
#endif
}

// floor(v / 2^s) for any s >= 0 (PTX shr.s64 clamps the count at 64)
TEUK_FX_HD long long fx_sar(long long v, uint32_t s)
{
#ifdef __CUDA_ARCH__
    long long r;
    asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(s));
    return r;
#else
    return v >> (s > 63u ? 63u : s);
#endif
}

// An FP64 number split for the fixed-point sums.
struct Fx {
    uint32_t mhi, mlo;  // significand: high 21 bits (hidden bit included for normal numbers), low 32 bits
    int e;              // max(biased exponent, 1); -4096 for +-0
    uint32_t neg;       // sign bit
    uint32_t braw;      // biased exponent field (2047: not finite)
};

TEUK_FX_HD Fx fx_unpack(double v)
{
    const uint64_t u = fx_bits(v);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t eraw = (hi >> 20) & 0x7FFu;
    Fx o;
    o.mhi = (hi & 0xFFFFFu) | (eraw ? 0x100000u : 0u);
    o.mlo = lo;
    o.e = eraw ? (int)eraw : 1;
    o.neg = hi >> 31;
    o.braw = eraw;
    return o;
}

// Split of a coefficient that is known to be finite and either normal or
// exactly zero (the step kernels' coefficient planes guarantee it): no
// subnormal case and no finiteness flag.  A zero gets e = -4096, so its
// product is shifted out entirely; for every such input the term contributes
// exactly what fx_unpack's split gives.
TEUK_FX_HD Fx fx_unpack_coef(double v)
{
    const uint64_t u = fx_bits(v);
    const uint32_t hi = (uint32_t)(u >> 32);
    const int eraw = (int)((hi >> 20) & 0x7FFu);
    Fx o;
    o.mhi = (hi & 0xFFFFFu) | 0x100000u;
    o.mlo = (uint32_t)u;
    o.e = eraw ? eraw : -4096;
    o.neg = hi >> 31;
    o.braw = 0;
    return o;
}

// floor(m_c m_x / 2^47) of the exact 106-bit product
TEUK_FX_HD uint64_t fx_prod47(const Fx &c, const Fx &x)
{
    const uint64_t t0 = (uint64_t)c.mlo * x.mlo;
    const uint64_t t1 = (uint64_t)c.mlo * x.mhi + (t0 >> 32);
    const uint64_t t2 = (uint64_t)c.mhi * x.mlo + t1;
    const uint64_t t3 = (uint64_t)c.mhi * x.mhi + (t2 >> 32);
    // m_c m_x = t3 2^64 + (t2 mod 2^32) 2^32 + (t0 mod 2^32)
    return (t3 << 17) | ((t2 & 0xFFFFFFFFu) >> 15);
}

// *out = sum_k (-1)^flip[k] c[k] x[k] for N <= 16 terms.  Returns false
// (with *out unspecified) when the caller must use FP64 arithmetic instead.
// With EXTRA, one more term enters already formed: P 2^(TP - 2103), |P| <
// 2^59 like a truncated product, P = 0 with a very negative TP when it is
// zero (at most 15 product terms then).
template <int N, bool EXTRA = false>
TEUK_FX_HD bool fx_dot(const Fx *c, const Fx *x, const uint32_t *flip, double *out, long long P = 0,
                       int TP = -100000)
{
    static_assert(N >= 1 && N + (EXTRA ? 1 : 0) <= 16, "at most 16 terms fit the 64-bit accumulator");
    int T[N];
    int E = EXTRA && TP > 0 ? TP : 0;
    uint32_t braw = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        T[k] = c[k].e + x[k].e;  // negative when either factor is zero
        E = T[k] > E ? T[k] : E;
        braw = c[k].braw > braw ? c[k].braw : braw;
        braw = x[k].braw > braw ? x[k].braw : braw;
    }
    uint64_t acc = EXTRA ? (uint64_t)fx_sar(P, (uint32_t)(E - TP)) : 0;  // two's complement, units of 2^(E - 2103)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const uint64_t v = fx_shr(fx_prod47(c[k], x[k]), (uint32_t)(E - T[k]));
        acc += (c[k].neg ^ x[k].neg ^ flip[k]) ? (uint64_t)0 - v : v;
    }
    // One rounding to nearest (ties to even) of the exact sum acc 2^(E - 2103);
    // the sum applies when the rounded result's biased exponent ef lies in
    // [200, 2045] (2^-823 <= |result| < 2^1023).
#ifdef __CUDA_ARCH__
    // the hardware int64 -> FP64 conversion rounds like the integer path
    // below; the frame's power of two then goes onto the exponent field
    if (acc == 0) {
        *out = 0.0;
        return braw < 0x7FFu;
    }
    const uint64_t cb = fx_bits(__ll2double_rn((long long)acc));
    const int ef = (int)((cb >> 52) & 0x7FFu) + (E - 2103);
    *out = fx_double(cb + ((uint64_t)(long long)(E - 2103) << 52));
    return braw < 0x7FFu && ef >= 200 && ef <= 2045;
#else
    const uint32_t neg = (uint32_t)(acc >> 63);
    const uint64_t mag = neg ? (uint64_t)0 - acc : acc;
    const int lz = fx_clz64(mag);
    const uint64_t nrm = mag << (lz & 63);  // leading one at bit 63
    uint64_t m = nrm >> 11;                 // 53-bit significand
    const uint32_t guard = (uint32_t)(nrm >> 10) & 1u;
    const uint32_t sticky = (nrm & 0x3FFu) != 0;
    m += guard & (sticky | (uint32_t)(m & 1u));
    const int eb = E - 1017 - lz;  // biased exponent of the leading one
    // (eb - 1) 2^52 + m: the hidden bit lifts the exponent field to eb, and a
    // significand that rounds up to 2^53 carries into it
    const uint64_t r = (((uint64_t)(eb - 1) << 52) + m) | ((uint64_t)neg << 63);
    const int ef = (int)((r >> 52) & 0x7FFu);
    *out = mag == 0 ? 0.0 : fx_double(r);
    return braw < 0x7FFu && (mag == 0 || (ef >= 200 && ef <= 2045));
#endif
}

// ---------------------------------------------------------------------------
// The sixth difference of the angular dissipation,
//   D6 = 20 u_3 - 15 (u_2 + u_4) + 6 (u_1 + u_5) - (u_0 + u_6),
// of seven FP64 values, as an exact integer sum rounded once.
//
//   * each value is prepared once: v = +-m 2^4 (|v| < 2^57) and its exponent
//     e = max(biased exponent, 1) (2047: not finite);
//   * with F the largest e of the seven, every v is shifted right by F - e
//     (floor), so each is truncated to units of 2^(F - 1079) by less than one
//     unit and the largest keeps all 53 bits of its significand;
//   * the weighted sum is exact in a signed 64-bit integer (|sum| < 64 2^57)
//     and is rounded once to FP64, to nearest, ties to even.
//
// Error: |result - D6| <= 64 2^(F - 1079) + 2^-53 |D6| <= 2^-50 max|u_q|
// + 2^-53 |D6|; scaled by the dissipation strength eps/64 this is at most
// eps 2^-56 max|u_q| + 2^-53 |eps D6 / 64|, below one FP64 rounding of the
// largest value of the window.  A non-finite input gives NaN.
// ---------------------------------------------------------------------------

// A value prepared for fx_d6.
struct alignas(16) FxP {
    long long v;  // +-m 2^4
    int e;        // max(biased exponent, 1); 2047 if not finite
};

TEUK_FX_HD FxP fx_prep(double x)
{
    const uint64_t u = fx_bits(x);
    const uint32_t hi = (uint32_t)(u >> 32);
    const int eraw = (int)((hi >> 20) & 0x7FFu);
    const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (eraw ? (1ull << 52) : 0ull);
    const long long v = (long long)(m << 4);
    FxP o;
    o.v = (hi >> 31) ? -v : v;
    o.e = eraw ? eraw : 1;
    return o;
}


// RN(D 2^k) for |D| < 2^63 and D 2^k below the FP64 overflow threshold,
// subnormal results included.  For a sixth difference (D from fx_d6_int,
// k = F - 1079) a subnormal result is always exact: F <= 4 there, and every
// aligned term is a multiple of 2^(5 - F), the subnormal branch's shift.
TEUK_FX_HD double fx_ldexp_rn(long long D, int k)
{
    if (D == 0) return 0.0;
#ifdef __CUDA_ARCH__
    // the hardware conversion rounds D to nearest (ties to even) like the
    // integer path below; scaling by 2^k is then exact on the exponent field
    // wherever the result is a normal number
    {
        const uint64_t cb = fx_bits(__ll2double_rn(D));
        const int ef = (int)((cb >> 52) & 0x7FFu) + k;
        if (ef >= 1 && ef <= 2046) return fx_double(cb + ((uint64_t)(long long)k << 52));
    }
#endif
    const uint64_t neg = D < 0 ? 1u : 0u;
    const uint64_t mag = neg ? (uint64_t)0 - (uint64_t)D : (uint64_t)D;
    const int lz = fx_clz64(mag);
    const int eb = 63 - lz + k + 1023;  // biased exponent of the leading one
    uint64_t r;
    if (eb >= 1) {
        const uint64_t nrm = mag << lz;  // leading one at bit 63
        uint64_t m = nrm >> 11;
        const uint64_t guard = (nrm >> 10) & 1u;
        const uint64_t sticky = (nrm & 0x3FFu) != 0;
        m += guard & (sticky | (m & 1u));
        r = ((uint64_t)(eb - 1) << 52) + m;  // a significand rounded up to 2^53 carries into the exponent
    } else {
        // subnormal: units of 2^-1074; mag 2^k = mag 2^(k + 1074) units, k + 1074 < 52
        const int sh = -(k + 1074);
        if (sh <= 0) {
            r = mag << (-sh);
        } else if (sh >= 64) {
            r = 0;  // mag < 2^63 <= half a unit
        } else {
            const uint64_t q = mag >> sh, rem = mag & ((1ull << sh) - 1), half = 1ull << (sh - 1);
            r = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
        }
    }
    return fx_double(r | (neg << 63));
}

// The exact integer sum of D6 before its rounding: D6 = D 2^(F - 1079)
// (F = 2047: an input was not finite).
struct FxI {
    long long D;
    int F;
};

TEUK_FX_HD FxI fx_d6_int(const FxP *p)
{
    int F = p[0].e;
#pragma unroll
    for (int q = 1; q < 7; ++q) F = p[q].e > F ? p[q].e : F;
    long long w[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) w[q] = fx_sar(p[q].v, (uint32_t)(F - p[q].e));
    FxI r;
    r.D = 20 * w[3] - 15 * (w[2] + w[4]) + 6 * (w[1] + w[5]) - (w[0] + w[6]);
    r.F = F;
    return r;
}

TEUK_FX_HD double fx_d6_round(const FxI &r)
{
    return r.F >= 2047 ? fx_double(0x7FF8000000000000ull) : fx_ldexp_rn(r.D, r.F - 1079);
}

// D6 of seven prepared values p[0..6] (p[3] the centre).
TEUK_FX_HD double fx_d6(const FxP *p) { return fx_d6_round(fx_d6_int(p)); }

// D6 of seven FP64 values u[0], u[stride], ..., u[6 stride].
TEUK_FX_HD double fx_d6_values(const double *u, int stride)
{
    FxP p[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) p[q] = fx_prep(u[q * stride]);
    return fx_d6(p);
}



}  // namespace teuk
