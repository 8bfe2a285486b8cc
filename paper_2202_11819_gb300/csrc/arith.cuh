// Device arithmetic of the 7-point Jacobi update and of the residual term.
//
// The paper (Section II-A, Figs. 1 and 3) updates every cell of a block from
// its six face neighbours each iteration but does not print the formula; the
// update here is the mean of the cell and its six face neighbours.
//
//  mean7_seq      binary64: c + xm + xp + ym + yp + zm + zp left to right,
//                 every addition rounded to nearest even, then a correctly
//                 rounded division by 7 (the GPU's binary64 units).
//  mean7_seq_f32  the same in binary32.
//  mean7_exact    the exact sum of the seven values divided by 7, rounded
//                 once to nearest even. Computed in integer arithmetic: on
//                 this GPU the binary64 pipe issues about two operations per
//                 SM per clock, while the integer pipes issue 64-128, so the
//                 exact mean in integers is both more accurate and faster than
//                 six binary64 additions and a binary64 division.
//  laplacian_exact xm + xp + ym + yp + zm + zp - 6c, exact, rounded once.
//
// Fast paths cover values of one sign whose exponents lie within 72 bits of
// the largest and whose result is a normal number; everything else takes an
// exact wide-accumulator path (rare: mixed signs, subnormals, huge spreads).
#pragma once
#include <cmath>

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define JAC_HD __host__ __device__
#else
#define JAC_HD
#endif

namespace jac {

// bit casts and leading-zero counts that also compile for the host, so the
// integer arithmetic below can be checked on a CPU
JAC_HD inline uint64_t dbits(double v)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t b;
    memcpy(&b, &v, 8);
    return b;
#endif
}

JAC_HD inline double bitsd(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double v;
    memcpy(&v, &b, 8);
    return v;
#endif
}

JAC_HD inline int clz64(uint64_t x)  // x != 0
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

JAC_HD inline int clz32(uint32_t x)  // 32 for x == 0
{
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

JAC_HD inline int imax(int a, int b) { return a > b ? a : b; }

JAC_HD inline uint32_t umulhi32(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

JAC_HD inline uint64_t mulhi_u64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// RN(s / 7) for a binary64 s whose exponent field e is in [4, 2046] (so s
// and the quotient are normal), in integer arithmetic only (no binary64
// instruction: the sequential rule's six additions already fill that pipe).
// N = significand << 11 lies in [2^63, 2^64); Qa, the
// high word of N * floor(2^64/7), is floor(N/7) or one less, and has 61 or 62
// bits, so converting it rounds away its d = 8 or 9 low bits. That rounding
// equals the rounding of the exact quotient N/7: the two could differ only
// if a rounding midpoint lay in [Qa, N/7], i.e. if floor(N/7) had its d low
// bits equal to 2^(d-1). As N is a multiple of 2^11, 7 floor(N/7) + r = N
// (r < 7) forces floor(N/7) mod 2^d to be 0 modulo 2^(d-1) only together
// with r = 128 (d = 8) or r = 256 (d = 9), which cannot be; and Qa one less
// happens only for r <= 1 and steps over no midpoint either. The exponent is
// then rescaled by e - 1086 and the sign copied. Returns false (out unset)
// outside that range: zero, subnormals, infinities and NaN. Checked against
// correctly rounded division on the host (tests/test_arith_host.py).
JAC_HD inline bool div7d(double s, double& out)
{
    const uint64_t b = dbits(s);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
    const uint64_t N = (((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11);
    const uint64_t Qa = mulhi_u64(N, 0x2492492492492492ull);
    // RN(Qa) to 53 bits, ties to even, by adding 2^(k-1) - 1 plus bit k and
    // dropping the k low bits (k = 8 or 9): R in [2^52, 2^53], RN(Qa) = R 2^k.
    // Then RN(Qa) has exponent field 1074 + k + (R's hidden bit), so adding R
    // to (1074 + k + e - 1086) << 52 both encodes it and applies the rescale
    // (a carry of R into 2^53 moves to the next binade by itself).
    const int k = (uint32_t)(Qa >> 32) >= (1u << 29) ? 9 : 8;
    const uint64_t R = (Qa + (((1ull << (k - 1)) - 1u) + ((Qa >> k) & 1u))) >> k;
    out = bitsd((R + ((uint64_t)((int)e + k - 12) << 52)) | (b & 0x8000000000000000ull));
    return e >= 4u && e <= 2046u;
}

// RN(a + b) for binary64 a, b >= 0 in integer arithmetic. Returns false
// (out unset) unless the larger has exponent field in [1, 2044] and the
// smaller is normal in that range or +0; then the sum is normal and finite.
// With hi >= lo (nonnegative doubles order like their bits) and d the
// difference of their exponent fields, the significands shifted left by 10
// are mh in [2^62, 2^63) and ml; ml >> min(d, 63) is added to mh, and the
// bits it drops become a sticky bit in bit 0 (below the rounding point, which
// is bit 10, or bit 11 when the sum reaches 2^63). For d >= 54 the result is
// hi, as lo is then below half an ulp of hi: the sticky bit alone gives
// that. Rounding to nearest, ties to even, adds 2^(k-1) - 1 plus bit k and
// drops k bits; R in [2^52, 2^53] then encodes with exponent field
// eh - 11 + k + (R's hidden bit), a carry into 2^53 moving up a binade.
JAC_HD inline bool dadd_nonneg(double a, double b, double& out)
{
    const uint64_t x = dbits(a), y = dbits(b);
    const uint64_t hi = x > y ? x : y, lo = x > y ? y : x;
    const uint32_t eh = (uint32_t)(hi >> 52), el = (uint32_t)(lo >> 52);  // >= 2048 with the sign bit
    const bool lo_zero = lo == 0u;
    const bool ok = eh - 1u < 2044u && (el - 1u < 2044u || lo_zero);
    const uint32_t dd = eh - el;
    const int d = (int)(dd < 63u ? dd : 63u);
    const uint64_t mh = ((hi & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    const uint64_t ml = ((lo & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    const uint64_t sh = ml >> d;
    const uint64_t S = (mh + sh) | ((sh << d) != ml ? 1u : 0u);
    const int k = (S >> 63) != 0u ? 11 : 10;
    const uint64_t R = (S + (((1ull << (k - 1)) - 1u) + ((S >> k) & 1u))) >> k;
    const uint64_t r = R + ((uint64_t)((int)eh - 11 + k) << 52);
    out = bitsd(lo_zero ? hi : r);
    return ok;
}

__device__ __forceinline__ double mean7_seq(double c, double xm, double xp, double ym, double yp,
                                            double zm, double zp)
{
    // the first two additions in integer arithmetic (this rule is bound by
    // the binary64 pipe); a lane whose values do not qualify takes the pipe
    double s;
    const bool ok1 = dadd_nonneg(c, xm, s);
    if (!ok1) s = __dadd_rn(c, xm);
    s = __dadd_rn(s, xp);
    s = __dadd_rn(s, ym);
    s = __dadd_rn(s, yp);
    s = __dadd_rn(s, zm);
    s = __dadd_rn(s, zp);
    double q;
    if (!div7d(s, q)) q = __ddiv_rn(s, 7.0);
    return q;
}

// RN(s / 7) in binary32 without a division routine (so without the call its
// rare slow path makes, which costs registers in a loop). For |s| >= 2^-100
// one product and one fused multiply-add with a two-word reciprocal of 7
// (zh = RN(1/7), zl = RN(1/7 - zh); the method of Brisebarre, Muller and
// Raina, "Accelerating correctly rounded floating-point division when the
// divisor is known in advance", IEEE Trans. Computers 53(8), 2004). Below
// that, and for zero, exact integer division in units of 2^-149. Checked
// bit for bit against the correctly rounded quotient for every finite
// binary32 value (tests/test_div7f_exhaustive.py).
// The common case of div7f (|s| >= 2^-100, s finite), without the branch.
JAC_HD inline float div7f_fast(float s)
{
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(s, 0x1.24924ap-3f, __fmul_rn(s, -0x1.b6db6ep-28f));
#else
    return fmaf(s, 0x1.24924ap-3f, s * -0x1.b6db6ep-28f);
#endif
}

// True when div7f_fast(s) may differ from div7f(s).
JAC_HD inline bool div7f_needs_exact(float s) { return !(fabsf(s) >= 0x1p-100f); }

JAC_HD inline float div7f(float s)
{
    const float zh = 0x1.24924ap-3f;
    const float zl = -0x1.b6db6ep-28f;
    if (fabsf(s) >= 0x1p-100f) {
#if defined(__CUDA_ARCH__)
        return __fmaf_rn(s, zh, __fmul_rn(s, zl));
#else
        return fmaf(s, zh, s * zl);
#endif
    }
    if (s == 0.0f) return s;
    uint32_t b;
    memcpy(&b, &s, 4);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t e = (b >> 23) & 0xFFu;  // <= 27 here
    const uint32_t f = b & 0x7FFFFFu;
    const uint64_t S = e ? ((uint64_t)(f | 0x800000u) << (e - 1)) : (uint64_t)f;  // s / 2^-149, < 2^50
    uint64_t Q = S / 7u;
    const uint64_t R = S - 7u * Q;
    uint32_t out;
    if (Q < (1ull << 23)) {
        // subnormal (or the smallest normal after rounding): units of 2^-149,
        // the fraction R/7 is never exactly one half
        out = (uint32_t)(Q + (R >= 4u ? 1u : 0u));
    } else {
        int L = 0;
        for (uint64_t t = Q; t; t >>= 1) ++L;  // 24 .. 47
        const int sh = L - 24;
        uint64_t mant = Q >> sh;
        bool up;
        if (sh == 0) {
            up = R >= 4u;
        } else {
            const bool rbit = (Q >> (sh - 1)) & 1u;
            const bool sticky = (Q & ((1ull << (sh - 1)) - 1ull)) != 0ull || R != 0u;
            up = rbit && (sticky || (mant & 1u));
        }
        mant += up ? 1u : 0u;
        out = ((uint32_t)sh << 23) + (uint32_t)mant;  // the implicit bit lifts the exponent to sh + 1
    }
    out |= sign;
    float r;
    memcpy(&r, &out, 4);
    return r;
}

__device__ __forceinline__ float mean7_seq_f32(float c, float xm, float xp, float ym, float yp,
                                               float zm, float zp)
{
    float s = __fadd_rn(c, xm);
    s = __fadd_rn(s, xp);
    s = __fadd_rn(s, ym);
    s = __fadd_rn(s, yp);
    s = __fadd_rn(s, zm);
    s = __fadd_rn(s, zp);
    return div7f(s);
}

// ------------------------------------------------------------------------
// Wide exact accumulator (slow path). Bit q of the accumulator weighs
// 2^(q - 1074), so every finite binary64 is an integer number of units.
// ------------------------------------------------------------------------
constexpr int kWideWords = 72;  // 2304 bits

JAC_HD inline __noinline__ double exact_weighted_sum_round(const double* v, const int* w, int n,
                                                        uint32_t divisor)
{
    uint32_t P[kWideWords], N[kWideWords];
    for (int t = 0; t < kWideWords; ++t) {
        P[t] = 0u;
        N[t] = 0u;
    }
    for (int t = 0; t < n; ++t) {
        uint64_t bits = dbits(v[t]);
        int neg = (int)(bits >> 63);
        int e = (int)((bits >> 52) & 0x7FF);
        uint64_t m = bits & ((1ull << 52) - 1);
        int pos = 0;
        if (e != 0) {
            m |= (1ull << 52);
            pos = e - 1;
        }
        if (m == 0) continue;
        int wt = w[t];
        if (wt < 0) {
            neg = !neg;
            wt = -wt;
        }
        m *= (uint64_t)wt;
        uint32_t* A = neg ? N : P;
        int q = pos >> 5, sh = pos & 31;
        uint64_t lo = m << sh;
        uint64_t hi = sh ? (m >> (64 - sh)) : 0ull;
        uint32_t part[3] = {(uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi};
        uint64_t carry = 0;
        for (int u = 0; u < 3; ++u) {
            uint64_t s = (uint64_t)A[q + u] + part[u] + carry;
            A[q + u] = (uint32_t)s;
            carry = s >> 32;
        }
        for (int u = q + 3; carry && u < kWideWords; ++u) {
            uint64_t s = (uint64_t)A[u] + carry;
            A[u] = (uint32_t)s;
            carry = s >> 32;
        }
    }
    // magnitude and sign of P - N
    int cmp = 0;
    for (int t = kWideWords - 1; t >= 0 && cmp == 0; --t) {
        if (P[t] != N[t]) cmp = P[t] > N[t] ? 1 : -1;
    }
    if (cmp == 0) return 0.0;
    const uint32_t* big = cmp > 0 ? P : N;
    const uint32_t* small = cmp > 0 ? N : P;
    uint32_t S[kWideWords];
    int64_t borrow = 0;
    for (int t = 0; t < kWideWords; ++t) {
        int64_t d = (int64_t)big[t] - (int64_t)small[t] - borrow;
        borrow = d < 0;
        S[t] = (uint32_t)(d + (borrow ? (1ll << 32) : 0));
    }
    // long division by the divisor
    uint64_t r = 0;
    for (int t = kWideWords - 1; t >= 0; --t) {
        uint64_t cur = (r << 32) | S[t];
        uint64_t qt = cur / divisor;
        S[t] = (uint32_t)qt;
        r = cur - qt * divisor;
    }
    int top = -1;
    for (int t = kWideWords - 1; t >= 0 && top < 0; --t)
        if (S[t]) top = t * 32 + 31 - clz32(S[t]);
    uint64_t mant = 0;
    int shift = 0;
    bool up;
    if (top < 0) {
        up = 2 * r > divisor;
    } else {
        shift = top > 52 ? top - 52 : 0;
        for (int q = top; q >= shift; --q) mant = (mant << 1) | ((S[q >> 5] >> (q & 31)) & 1u);
        if (shift > 0) {
            bool rbit = (S[(shift - 1) >> 5] >> ((shift - 1) & 31)) & 1u;
            bool sticky = r != 0;
            int below = shift - 1;
            int wf = below >> 5;
            for (int t = 0; t < wf && !sticky; ++t) sticky = S[t] != 0;
            if (!sticky && (below & 31)) sticky = (S[wf] & ((1u << (below & 31)) - 1u)) != 0;
            up = rbit && (sticky || (mant & 1));
        } else {
            up = (2 * r > divisor) || (2 * r == divisor && (mant & 1));
        }
    }
    mant += up ? 1 : 0;
    if (mant == 0ull) return 0.0;
    // mant * 2^(shift - 1074): with mant < 2^52 (only when shift == 0) this is
    // the subnormal encoding; otherwise the significand's leading bit adds one
    // to the exponent field, so the same expression covers both.
    uint64_t out = ((uint64_t)shift << 52) + mant;
    if (cmp < 0) out |= (1ull << 63);
    return bitsd(out);
}

// ------------------------------------------------------------------------
// 128-bit helpers
// ------------------------------------------------------------------------
JAC_HD inline void add128(uint64_t& lo, uint64_t& hi, uint64_t alo, uint64_t ahi)
{
    uint64_t nlo = lo + alo;
    hi = hi + ahi + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
}

// m (< 2^57) shifted left by s (0 <= s <= 71+) as a 128-bit value
JAC_HD inline void shl128(uint64_t m, int s, uint64_t& lo, uint64_t& hi)
{
    if (s >= 64) {
        lo = 0ull;
        hi = m << (s - 64);
    } else if (s == 0) {
        lo = m;
        hi = 0ull;
    } else {
        lo = m << s;
        hi = m >> (64 - s);
    }
}

// ------------------------------------------------------------------------
// Correctly rounded mean of seven binary64 values.
// Fast path: all values of one sign, each either zero or a normal number
// within 72 binades of the largest, the largest at least 2^-959. The values
// are placed in a 128-bit fixed-point frame whose unit is
// 2^(emax - 1147) (the largest significand lands on bits 72..124), summed
// exactly, and the top 64 bits are divided by 7; the remaining bits only
// feed the sticky bit.
// ------------------------------------------------------------------------
JAC_HD inline double mean7_exact(double c, double xm, double xp, double ym, double yp,
                                              double zm, double zp)
{
    const double v[7] = {c, xm, xp, ym, yp, zm, zp};
    uint64_t b[7];
    uint64_t sor = 0ull, sand = ~0ull;
    int emax = 0;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        b[t] = dbits(v[t]);
        sor |= b[t];
        sand &= b[t];
        int e = (int)((b[t] >> 52) & 0x7FF);
        emax = imax(emax, e);
    }
    const bool neg = (sand >> 63) != 0;
    bool ok = neg || (sor >> 63) == 0;  // one sign only
    if (emax == 0 && ok && ((sor << 1) == 0)) return 0.0;  // all zeros
    ok = ok && emax >= 64;
    uint64_t lo = 0ull, hi = 0ull;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        int e = (int)((b[t] >> 52) & 0x7FF);
        uint64_t frac = b[t] & ((1ull << 52) - 1);
        int d = emax - e;
        if (e == 0) {
            ok = ok && frac == 0;  // zero adds nothing; a subnormal goes the slow way
        } else {
            ok = ok && d <= 72;
            uint64_t plo, phi;
            shl128(frac | (1ull << 52), imax(72 - d, 0), plo, phi);
            add128(lo, hi, plo, phi);
        }
    }
    if (!ok) {
        const int w[7] = {1, 1, 1, 1, 1, 1, 1};
        return exact_weighted_sum_round(v, w, 7, 7u);
    }
    // S = hi:lo in [2^124, 7 * 2^125); S/7 = Q1 * 2^64 + (R1 * 2^64 + lo)/7
    const uint64_t Q1 = hi / 7ull;
    const uint64_t R1 = hi - Q1 * 7ull;
    const int L = 64 - clz64(Q1);  // 58 .. 61
    const int shift = L - 53;                  // 5 .. 8
    uint64_t mant = Q1 >> shift;
    const uint64_t rbit = (Q1 >> (shift - 1)) & 1ull;
    const bool sticky = (Q1 & ((1ull << (shift - 1)) - 1ull)) != 0ull || R1 != 0ull || lo != 0ull;
    mant += rbit & ((sticky ? 1ull : 0ull) | (mant & 1ull));
    // value = mant * 2^(emax - 1083 + shift); biased exponent emax - 8 + shift
    uint64_t out = ((uint64_t)(emax - 8 + shift - 1) << 52) + mant;
    if (neg) out |= (1ull << 63);
    return bitsd(out);
}

// ------------------------------------------------------------------------
// Exact Laplacian term xm + xp + ym + yp + zm + zp - 6c, rounded once.
// Fast path: all seven values >= 0, normal or zero, within 71 binades of
// the largest (largest >= 2^-959), result normal. Frame unit 2^(emax - 1146):
// the largest significand lands on bits 71..123, so both the neighbour sum
// and 6c stay below 2^127 and the difference fits a signed 128-bit word.
// ------------------------------------------------------------------------
JAC_HD inline double laplacian_exact(double c, double xm, double xp, double ym,
                                                  double yp, double zm, double zp)
{
    const double v[7] = {xm, xp, ym, yp, zm, zp, c};
    uint64_t b[7];
    uint64_t sor = 0ull;
    int emax = 0;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        b[t] = dbits(v[t]);
        sor |= b[t];
        emax = imax(emax, (int)((b[t] >> 52) & 0x7FF));
    }
    bool ok = (sor >> 63) == 0;
    if (ok && (sor << 1) == 0) return 0.0;
    ok = ok && emax >= 64;
    uint64_t plo = 0ull, phi = 0ull, clo = 0ull, chi = 0ull;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        int e = (int)((b[t] >> 52) & 0x7FF);
        uint64_t frac = b[t] & ((1ull << 52) - 1);
        if (e == 0) {
            ok = ok && frac == 0;
        } else {
            int d = emax - e;
            ok = ok && d <= 71;
            uint64_t m = frac | (1ull << 52);
            if (t == 6) m *= 6ull;
            uint64_t alo, ahi;
            shl128(m, imax(71 - d, 0), alo, ahi);
            if (t == 6) {
                clo = alo;
                chi = ahi;
            } else {
                add128(plo, phi, alo, ahi);
            }
        }
    }
    if (ok) {
        // L = P - C (two's complement), then magnitude
        uint64_t llo = plo - clo;
        uint64_t lhi = phi - chi - (plo < clo ? 1ull : 0ull);
        const bool lneg = (int64_t)lhi < 0;
        if (lneg) {
            llo = ~llo + 1ull;
            lhi = ~lhi + (llo == 0ull ? 1ull : 0ull);
        }
        if ((llo | lhi) == 0ull) return 0.0;
        const int t = lhi ? 127 - clz64(lhi) : 63 - clz64(llo);
        const int bexp = t + emax - 123;  // biased exponent of the result
        if (bexp >= 1) {
            uint64_t mant;
            uint64_t rbit = 0ull;
            bool sticky = false;
            if (t <= 52) {
                mant = llo << (52 - t);  // exact
            } else {
                const int sh = t - 52;  // 1 .. 74
                if (sh >= 64) {
                    mant = lhi >> (sh - 64);
                } else {
                    mant = (llo >> sh) | (lhi << (64 - sh));
                }
                const int rb = sh - 1;  // round-bit position
                rbit = rb >= 64 ? (lhi >> (rb - 64)) & 1ull : (llo >> rb) & 1ull;
                if (rb >= 64) {
                    sticky = llo != 0ull || (rb > 64 && (lhi & ((1ull << (rb - 64)) - 1ull)) != 0ull);
                } else {
                    sticky = rb > 0 && (llo & ((1ull << rb) - 1ull)) != 0ull;
                }
            }
            mant += rbit & ((sticky ? 1ull : 0ull) | (mant & 1ull));
            uint64_t out = ((uint64_t)(bexp - 1) << 52) + mant;
            if (lneg) out |= (1ull << 63);
            return bitsd(out);
        }
    }
    const int w[7] = {1, 1, 1, 1, 1, 1, -6};
    return exact_weighted_sum_round(v, w, 7, 1u);
}

// ========================================================================
// Grid-frame arithmetic.
//
// One fixed-point frame per grid: with E the largest exponent field of any
// value of the grid and its boundary (the maximum principle keeps every
// later iterate at or below that maximum), the frame's unit is
// 2^(Eref - 1106), Eref = E + 1. A normal binary64 value v >= 0 with
// exponent field e is (1.f) 2^(e-1023) = m * 2^(e-1075), m < 2^53, i.e.
// m << s units with s = e - Eref + 31 in [0, 31] when e >= Eref - 31. That
// fits 96 bits as three 32-bit words (w < 2^84). Each cell converts only its
// own value; the seven-term sum is then exact in 96-bit integer arithmetic
// (< 2^87). A value outside the frame (negative, subnormal, or more than 31
// binades below the maximum) becomes a marker 2^93, which a sum detects as
// its top word reaching 2^29; such a cell takes the exact per-cell path.
// ========================================================================
namespace frame {

constexpr uint32_t kMarker = 1u << 29;  // w2 of an unrepresentable value (2^93)

struct __align__(16) W96 {
    uint32_t w0, w1, w2, w3;  // w3 is padding (one 16-byte load per value)
};

JAC_HD inline uint32_t fsl(uint32_t lo, uint32_t hi, int s)  // ((hi:lo) << s) >> 32, 0 <= s <= 31
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, s);
#else
    return (uint32_t)(((((uint64_t)hi << 32) | lo) << (s & 31)) >> 32);
#endif
}

JAC_HD inline uint32_t fsr(uint32_t lo, uint32_t hi, int s)  // ((hi:lo) >> s) & 0xffffffff, 0 <= s <= 31
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, s);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> s);
#endif
}

JAC_HD inline uint32_t fsrc(uint32_t lo, uint32_t hi, int s)  // ((hi:lo) >> min(s, 32)) & 0xffffffff, s >= 0
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_rc(lo, hi, s);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> (s < 32 ? s : 32));
#endif
}

JAC_HD inline uint32_t shlc(uint32_t x, int s)  // x << min(s, 32) (0 for s >= 32), s >= 0
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_lc(0u, x, s);
#else
    return s < 32 ? x << s : 0u;
#endif
}

JAC_HD inline uint64_t umulhi64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

JAC_HD inline W96 of(double v, int eref)
{
    // in the frame: sign 0 and exponent field e in [max(eref - 31, 1), eref - 1];
    // the sign bit makes (hi >> 20) at least 2048, outside every window
    const uint64_t b = dbits(v);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int lo_e = eref - 31 > 1 ? eref - 31 : 1;
    const int wn = eref - 1 - lo_e;  // window width - 1 (negative: empty)
    const uint32_t se = hi >> 20;
    const bool ok = wn >= 0 && se - (uint32_t)lo_e <= (uint32_t)wn;
    const bool zero = ((hi & 0x7FFFFFFFu) | lo) == 0u;
    const int sc = (int)se - (eref - 31);  // 0 .. 30 when ok
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    W96 w;
    w.w0 = ok ? fsl(0u, lo, sc) : 0u;
    w.w1 = ok ? fsl(lo, mh, sc) : 0u;
    w.w2 = ok ? fsl(mh, 0u, sc) : (zero ? 0u : kMarker);
    w.w3 = 0u;
    return w;
}

JAC_HD inline W96 add(W96 a, const W96& b)
{
#if defined(__CUDA_ARCH__)
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, %5;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2)
        : "r"(b.w0), "r"(b.w1), "r"(b.w2));
    return a;
#else
    const uint64_t l = (uint64_t)a.w0 + b.w0;
    const uint64_t m = (uint64_t)a.w1 + b.w1 + (l >> 32);
    a.w0 = (uint32_t)l;
    a.w1 = (uint32_t)m;
    a.w2 = a.w2 + b.w2 + (uint32_t)(m >> 32);
    return a;
#endif
}

// Correctly rounded conversion of an integer below 2^63 to binary64.
JAC_HD inline double u64_to_double_rn(uint64_t q)
{
#if defined(__CUDA_ARCH__)
    return __ull2double_rn(q);
#else
    return (double)(int64_t)q;
#endif
}

// S = a + b + c + d + e + f + g over 96 bits, in one carry chain.
JAC_HD inline void sum7(const W96& a, const W96& b, const W96& c, const W96& d, const W96& e, const W96& f,
                        const W96& g, uint32_t& s0, uint32_t& s1, uint32_t& s2)
{
#if defined(__CUDA_ARCH__)
    asm("add.cc.u32 %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32 %2, %5, %8;\n\t"
        "add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.u32 %2, %2, %11;\n\t"
        "add.cc.u32 %0, %0, %12;\n\t"
        "addc.cc.u32 %1, %1, %13;\n\t"
        "addc.u32 %2, %2, %14;\n\t"
        "add.cc.u32 %0, %0, %15;\n\t"
        "addc.cc.u32 %1, %1, %16;\n\t"
        "addc.u32 %2, %2, %17;\n\t"
        "add.cc.u32 %0, %0, %18;\n\t"
        "addc.cc.u32 %1, %1, %19;\n\t"
        "addc.u32 %2, %2, %20;\n\t"
        "add.cc.u32 %0, %0, %21;\n\t"
        "addc.cc.u32 %1, %1, %22;\n\t"
        "addc.u32 %2, %2, %23;"
        : "=&r"(s0), "=&r"(s1), "=&r"(s2)
        : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(b.w0), "r"(b.w1), "r"(b.w2), "r"(c.w0), "r"(c.w1), "r"(c.w2),
          "r"(d.w0), "r"(d.w1), "r"(d.w2), "r"(e.w0), "r"(e.w1), "r"(e.w2), "r"(f.w0), "r"(f.w1), "r"(f.w2),
          "r"(g.w0), "r"(g.w1), "r"(g.w2));
#else
    uint64_t lo = 0;
    uint32_t hi = 0;
    const W96* v[7] = {&a, &b, &c, &d, &e, &f, &g};
    for (const W96* w : v) {
        const uint64_t x = ((uint64_t)w->w1 << 32) | w->w0;
        lo += x;
        hi += w->w2 + (lo < x ? 1u : 0u);
    }
    s0 = (uint32_t)lo;
    s1 = (uint32_t)(lo >> 32);
    s2 = hi;
#endif
}

// S = a + b + c + d + e + f over 96 bits, in one carry chain.
JAC_HD inline void sum6(const W96& a, const W96& b, const W96& c, const W96& d, const W96& e, const W96& f,
                        uint32_t& s0, uint32_t& s1, uint32_t& s2)
{
#if defined(__CUDA_ARCH__)
    asm("add.cc.u32 %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32 %2, %5, %8;\n\t"
        "add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.u32 %2, %2, %11;\n\t"
        "add.cc.u32 %0, %0, %12;\n\t"
        "addc.cc.u32 %1, %1, %13;\n\t"
        "addc.u32 %2, %2, %14;\n\t"
        "add.cc.u32 %0, %0, %15;\n\t"
        "addc.cc.u32 %1, %1, %16;\n\t"
        "addc.u32 %2, %2, %17;\n\t"
        "add.cc.u32 %0, %0, %18;\n\t"
        "addc.cc.u32 %1, %1, %19;\n\t"
        "addc.u32 %2, %2, %20;"
        : "=&r"(s0), "=&r"(s1), "=&r"(s2)
        : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(b.w0), "r"(b.w1), "r"(b.w2), "r"(c.w0), "r"(c.w1), "r"(c.w2),
          "r"(d.w0), "r"(d.w1), "r"(d.w2), "r"(e.w0), "r"(e.w1), "r"(e.w2), "r"(f.w0), "r"(f.w1), "r"(f.w2));
#else
    const W96 t = add(add(add(a, b), add(c, d)), add(e, f));
    s0 = t.w0;
    s1 = t.w1;
    s2 = t.w2;
#endif
}

// RN(S / 7) for the frame sum S = s2:s1:s0 of seven values, without
// branches. Returns false when the exact per-cell path must be taken (a
// marker, or a subnormal result).
//   S (96 bits, below 2^87 unless a marker is present) is normalised so its
//   top bit is bit 63 of N (a sum below 2^64 is first moved up 32 bits; a
//   nonzero in-frame value is at least 2^52, so S is then zero or has a
//   nonzero top word); the bits shifted out become a sticky flag.
//   Q = floor(N / 7) from a multiply-high by floor(2^64/7), which is exact
//   or one short, and the remainder against it; Q in [2^60.2, 2^61.2). Q
//   has 61 or 62 bits and is rounded to 53: its last bit lies below the
//   rounding position, so OR-ing the sticky
//   information (nonzero remainder or dropped bits) into it lets one correctly
//   rounded integer -> binary64 conversion round the exact quotient.
//   S/7 = (Q + fraction) * 2^(L-64) units of 2^(eref-1106): that scale is
//   added to the exponent field of the converted value.
JAC_HD inline bool mean7_of_sum(uint32_t s0, uint32_t s1, uint32_t s2, int eref, double& out)
{
    const bool marker = s2 >= kMarker;
    const bool z2 = s2 == 0u;
    const uint32_t t2 = z2 ? s1 : s2, t1 = z2 ? s0 : s1, t0 = z2 ? 0u : s0;
    const bool zero = t2 == 0u;                 // S == 0
    const int r = 32 - clz32(t2);               // 1 .. 32 (0 when S == 0)
    const uint64_t Nn = ((uint64_t)fsrc(t1, t2, r) << 32) | fsrc(t0, t1, r);
    const bool st0 = shlc(t0, 32 - r) != 0u;
    const int L = r + (z2 ? 32 : 64);
    // Qa = floor(Nn * floor(2^64/7) / 2^64) is Q or Q - 1; the remainder
    // against it, R' in [0, 13], fixes both Q and the true remainder
    const uint64_t Qa = umulhi64(Nn, 0x2492492492492492ull);
    const uint32_t Ra = (uint32_t)Nn - 7u * (uint32_t)Qa;
    const uint32_t fix = Ra >= 7u ? 1u : 0u;
    const uint64_t Q = Qa + fix;
    const uint32_t R = Ra - 7u * fix;
    const uint64_t qj = Q | ((R != 0u || st0) ? 1ull : 0ull);
    const uint64_t qb = dbits(u64_to_double_rn(qj));
    const int adj = L - 64 + eref - 1106;
    const int biased = (int)(qb >> 52) + adj;
    out = zero ? 0.0 : bitsd(qb + ((uint64_t)(int64_t)adj << 52));
    return !marker && (zero || biased >= 1);
}

// mean7 on frame values: the sum, then mean7_of_sum.
JAC_HD inline bool mean7(const W96& c, const W96& xm, const W96& xp, const W96& ym, const W96& yp, const W96& zm,
                         const W96& zp, int eref, double& out)
{
    uint32_t s0, s1, s2;
    sum7(c, xm, xp, ym, yp, zm, zp, s0, s1, s2);
    return mean7_of_sum(s0, s1, s2, eref, out);
}

// The mean from a sum in the top binades of the frame: 2^82 <= S < 2^86
// (top word in [2^18, 2^22); a sum of in-frame values is below 7 * 2^83), for
// eref >= 7. Then N = S >> 25 lies in [2^57, 2^61) and Q = floor(N / 7) in
// [2^54.19, 2^58.2), so Q has two bits or more below the binary64 rounding
// position: one correctly rounded conversion of Q with the sticky bit (bits
// of S below 2^25, or a remainder) jammed into its last bit rounds the exact
// mean. The result's exponent field is at least eref - 4 >= 1 (a normal
// number) and S is not zero, so no per-cell checks remain.
//   Q is the high half of N * C with C = ceil(2^64 / 7) = (2^64 + 5) / 7:
//   N C / 2^64 = N / 7 + 5 N / (7 2^64), and for N < 2^61 the excess is below
//   5 / 56 < 1 / 7, so it never carries past the next integer (N / 7 has
//   fractional part at most 6 / 7). The remainder N - 7 Q is then in [0, 6].
// The scale 2^(25 + eref - 1106) is the constant scale_hi =
// (uint32_t)(eref - 1081) << 20 added to the high word of the conversion.
JAC_HD inline bool sum_in_top(uint32_t s2) { return s2 - (1u << 18) < (1u << 22) - (1u << 18); }

JAC_HD inline double mean7_top(uint32_t s0, uint32_t s1, uint32_t s2, uint32_t scale_hi)
{
    const uint32_t nl = fsr(s0, s1, 25), nh = fsr(s1, s2, 25);  // N = S >> 25, nh < 2^29
    uint32_t ql, qh;
#if defined(__CUDA_ARCH__)
    // high half of N * C over 32-bit limbs; the middle column
    // lo(nl cl) carry + nl ch + nh cl stays below 2^62 (no carry out)
    asm("{\n\t.reg .u32 t, m0, m1;\n\t"
        "mul.hi.u32 t, %2, 0x92492493;\n\t"
        "mad.lo.cc.u32 m0, %2, 0x24924924, t;\n\t"
        "madc.hi.u32 m1, %2, 0x24924924, 0;\n\t"
        "mad.lo.cc.u32 m0, %3, 0x92492493, m0;\n\t"
        "madc.hi.u32 m1, %3, 0x92492493, m1;\n\t"
        "mad.lo.cc.u32 %0, %3, 0x24924924, m1;\n\t"
        "madc.hi.u32 %1, %3, 0x24924924, 0;\n\t"
        "}"
        : "=r"(ql), "=r"(qh)
        : "r"(nl), "r"(nh));
#else
    const uint64_t q = umulhi64(((uint64_t)nh << 32) | nl, 0x2492492492492493ull);
    ql = (uint32_t)q;
    qh = (uint32_t)(q >> 32);
#endif
    const uint32_t sticky = (nl - 7u * ql) | (s0 & 0x1FFFFFFu);  // remainder, dropped bits
    const uint64_t qj = ((uint64_t)qh << 32) | (ql | (sticky != 0u ? 1u : 0u));
    return bitsd(dbits(u64_to_double_rn(qj)) + ((uint64_t)scale_hi << 32));
}

// RN(xm + xp + ym + yp + zm + zp - 6c) from frame values. Returns false for
// the exact per-cell path (a marker, or a subnormal result).
JAC_HD inline bool laplacian(const W96& c, const W96& xm, const W96& xp, const W96& ym, const W96& yp,
                             const W96& zm, const W96& zp, int eref, double& out)
{
    const W96 S = add(add(add(c, xm), add(xp, ym)), add(add(yp, zm), zp));
    if (S.w2 >= kMarker) return false;
    // T = 7c = 8c - c; L = S - T, two's complement over 96 bits
    const uint64_t c64 = ((uint64_t)c.w1 << 32) | c.w0;
    const uint64_t c8lo = c64 << 3;
    const uint32_t c8hi = (c.w2 << 3) | (c.w1 >> 29);
    const uint64_t tlo = c8lo - c64;
    const uint32_t thi = c8hi - c.w2 - (c8lo < c64 ? 1u : 0u);
    const uint64_t slo = ((uint64_t)S.w1 << 32) | S.w0;
    uint64_t llo = slo - tlo;
    uint32_t lhi = S.w2 - thi - (slo < tlo ? 1u : 0u);
    const bool neg = (lhi >> 31) != 0u;
    if (neg) {
        llo = ~llo + 1ull;
        lhi = ~lhi + (llo == 0ull ? 1u : 0u);
    }
    if ((llo | lhi) == 0ull) {
        out = 0.0;
        return true;
    }
    const int t = lhi ? 64 + 31 - clz32(lhi) : 63 - clz64(llo);  // top bit index
    const int biased = t + eref - 83;
    if (biased < 1) return false;
    uint64_t mant;
    if (t <= 52) {
        mant = llo << (52 - t);
    } else {
        const int sh = t - 52;  // 1 .. 34
        mant = (llo >> sh) | ((uint64_t)lhi << (64 - sh));
        const uint64_t rbit = (llo >> (sh - 1)) & 1ull;
        const bool sticky = (llo & ((1ull << (sh - 1)) - 1ull)) != 0ull;
        mant += rbit & ((sticky ? 1ull : 0ull) | (mant & 1ull));
    }
    uint64_t out_bits = ((uint64_t)(biased - 1) << 52) + mant;
    if (neg) out_bits |= (1ull << 63);
    out = bitsd(out_bits);
    return true;
}

// ---- binary32 residual in a 64-bit frame
// A binary32 grid's Laplacian term L = xm + xp + ym + yp + zm + zp - 6c is
// exact in a signed 64-bit frame of 2^(eref32 - 186) per unit (eref32 = the
// grid's largest binary32 exponent field + 1): a value of exponent field e
// in [eref32 - 36, eref32 - 1] is its 24-bit significand shifted left by
// e - eref32 + 36 (at most 35), below 2^59 in magnitude, so |L| < 12 * 2^59.
// Zero is 0; other values (tiny or subnormal) are outside the window (ok is
// set false) and the tile is redone with the exact per-cell routines.
JAC_HD inline int64_t of32(float v, int eref32, bool& ok)
{
    uint32_t b;
    memcpy(&b, &v, 4);
    const int e = (int)((b >> 23) & 0xFFu);
    const int sh = e - eref32 + 36;
    const bool zero = (b & 0x7FFFFFFFu) == 0u;
    ok = zero || (e != 0 && sh >= 0);
    const int64_t m = (int64_t)((b & 0x7FFFFFu) | 0x800000u);
    const int64_t w = (zero || sh < 0) ? 0 : (m << (sh & 63));
    return (b >> 31) ? -w : w;
}

// a += L^2 over 192 bits (|L| < 2^63)
JAC_HD inline void add_square(int64_t L, uint64_t& a0, uint64_t& a1, uint64_t& a2)
{
    const uint64_t u = L < 0 ? (uint64_t)(-L) : (uint64_t)L;
    const uint64_t lo = u * u, hi = umulhi64(u, u);
    const uint64_t s0 = a0 + lo;
    const uint64_t c0 = s0 < lo ? 1u : 0u;
    const uint64_t t1 = a1 + hi;
    const uint64_t c1 = t1 < hi ? 1u : 0u;
    const uint64_t s1 = t1 + c0;
    const uint64_t c2 = s1 < t1 ? 1u : 0u;
    a0 = s0;
    a1 = s1;
    a2 += c1 + c2;
}

// The 192-bit a2:a1:a0 rounded once to binary64, times 2^scale (the caller
// keeps the result in the normal range).
JAC_HD inline double u192_to_double_scaled(uint64_t a0, uint64_t a1, uint64_t a2, int scale)
{
    uint64_t top, rest;
    int below;  // bits below `top`
    if (a2) {
        const int lz = clz64(a2);
        top = lz ? (a2 << lz) | (a1 >> (64 - lz)) : a2;
        rest = (lz ? a1 << lz : a1) | a0;
        below = 128 - lz;
    } else if (a1) {
        const int lz = clz64(a1);
        top = lz ? (a1 << lz) | (a0 >> (64 - lz)) : a1;
        rest = lz ? a0 << lz : a0;
        below = 64 - lz;
    } else {
        top = a0;
        rest = 0;
        below = 0;
    }
    // top has its leading bit at bit 63 (or is a0 itself): jam the sticky bit
    const uint64_t tj = top | (rest != 0u ? 1u : 0u);
#if defined(__CUDA_ARCH__)
    const double t = __ull2double_rn(tj);
    return scalbn(t, below + scale);
#else
    const double t = (double)tj;  // correctly rounded on the host (the oracle's platform)
    return std::ldexp(t, below + scale);
#endif
}

}  // namespace frame

// ------------------------------------------------------------------------
// The 64-bit frame of the correctly rounded mean.
// A grid whose largest value has exponent field eref - 1 places every value
// of exponent field e in [eref - 9, eref - 1] at its 53-bit significand
// shifted left by e - (eref - 9) <= 8: an integer below 2^61 in units of
// 2^(eref - 1084). Seven such values sum to less than 7 * 2^61 < 2^64, so the
// sum of a cell and its six neighbours is one exact 64-bit integer, and the
// exchange plane holds 8 bytes per value instead of the 96-bit frame's 16.
// Values outside those nine binades (negative, zero or subnormal where the
// caller does not accept them, tiny) are flagged: the engine then takes the
// 96-bit frame for that step.
// ------------------------------------------------------------------------
namespace nframe {

constexpr int kWindow = 9;  // exponent fields eref - 9 .. eref - 1

// elo_hi = (eref - 9) << 20: the window's lowest exponent field placed
// where it sits in the high word of a binary64.
JAC_HD inline uint32_t elo_hi(int eref) { return (uint32_t)(eref - kWindow) << 20; }

// A value as a frame integer; ok is false unless it is a positive normal
// number inside the window. t = hi - elo_hi is below 9 * 2^20 exactly for
// those (a sign bit, a smaller exponent or a zero wrap it far above).
JAC_HD inline uint64_t of(double v, uint32_t elo_hi, bool& ok)
{
    const uint64_t b = dbits(v);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t t = hi - elo_hi;
    ok = t < ((uint32_t)kWindow << 20);
    const int sh = (int)(t >> 20);  // 0 .. 8 when ok
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    return ((uint64_t)frame::fsl(lo, mh, sh) << 32) | frame::fsl(0u, lo, sh);
}

// As `of`, and +0 is accepted as the frame integer 0 (the implicit bit is
// dropped when both words are zero, so any shift of it stays 0).
JAC_HD inline uint64_t of0(double v, uint32_t elo_hi, bool& ok)
{
    const uint64_t b = dbits(v);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const bool zero = (hi | lo) == 0u;
    const uint32_t t = hi - elo_hi;
    ok = zero || t < ((uint32_t)kWindow << 20);
    const int sh = (int)(t >> 20);
    const uint32_t mh = (hi & 0xFFFFFu) | (zero ? 0u : 0x100000u);
    return ((uint64_t)frame::fsl(lo, mh, sh) << 32) | frame::fsl(0u, lo, sh);
}

// The frame integer as a 96-bit frame value (units of 2^(eref - 1106)):
// the same number shifted left by 22.
JAC_HD inline frame::W96 widen(uint64_t w)
{
    frame::W96 r;
    const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
    r.w0 = lo << 22;
    r.w1 = frame::fsl(lo, hi, 22);
    r.w2 = hi >> 10;
    r.w3 = 0u;
    return r;
}

// scale_hi = (eref - 1081) << 20, the exponent offset mean7 adds.
JAC_HD inline uint32_t scale_hi(int eref) { return (uint32_t)(eref - 1081) << 20; }

// RN(S / 7) in units of 2^(eref - 1084), for a frame sum S with
// 2^52 <= S < 7 * 2^61 (the cell's own value is in the window, so S is at
// least its significand) and eref >= 13 (so the result is normal).
//   S has a nonzero high word (S >= 2^52), whose leading zeros lz <= 11
//   normalise it: N = S << lz lies in [2^63, 2^64). M = N >> 3 lies in
//   [2^60, 2^61), below 2^64 / 5, so the high half of M * ceil(2^64 / 7) is
//   floor(M / 7) exactly (its excess 5 M / (7 2^64) stays below 1/7, and the
//   fraction of M / 7 is at most 6/7). Q = floor(M / 7) lies in
//   [2^57.19, 2^58.19): 58 or 59 bits, so its three lowest bits lie below the
//   binary64 round bit. OR-ing the sticky information (the remainder
//   M - 7Q, below 7, and the three bits N drops) into them therefore lets
//   one correctly rounded integer -> binary64 conversion round the exact
//   quotient S / 7 = (Q + f) 2^(3 - lz). The scale 2^(3 - lz + eref - 1084)
//   is added to the exponent field: the result's field is at least
//   eref - 12 >= 1.
//   The high half of M * C, C = ch 2^32 + cl, is mh ch + floor(t / 2^32) with
//   t = mh cl + ml ch + floor(ml cl / 2^32) < 2^62.2 (the low partial
//   product's own low word cannot carry into it): four multiplies with
//   64-bit accumulation and no carry chain.
JAC_HD inline double mean7(uint64_t S, uint32_t scale_hi)
{
    constexpr uint32_t ch = 0x24924924u, cl = 0x92492493u;  // ceil(2^64 / 7)
    const uint32_t hi = (uint32_t)(S >> 32), lo = (uint32_t)S;
    const int lz = clz32(hi);
    const uint32_t nh = frame::fsl(lo, hi, lz), nl = frame::fsl(0u, lo, lz);
    const uint32_t mh = nh >> 3, ml = frame::fsr(nl, nh, 3);
    const uint64_t t = (uint64_t)mh * cl + (uint64_t)ml * ch + (uint64_t)umulhi32(ml, cl);
    const uint64_t q = (uint64_t)mh * ch + (t >> 32);
    const uint32_t sticky = (ml - 7u * (uint32_t)q) | (nl & 7u);
    const uint64_t d = dbits(frame::u64_to_double_rn(q | sticky));
    return bitsd(d + ((uint64_t)(scale_hi - ((uint32_t)lz << 20)) << 32));
}

// q += L^2 over 192 bits for the Laplacian term L = S - 7c of a cell whose
// frame sum is S and whose own frame integer is c. Both S and 7c lie below
// 7 * 2^61 < 2^64, so |L| fits 64 bits unsigned (the signed difference, up to
// 6 * 2^61 in magnitude, would not fit 64 bits signed) and L^2 < 2^128.
JAC_HD inline void add_laplacian_square(uint64_t S, uint64_t c, uint64_t& q0, uint64_t& q1, uint64_t& q2)
{
    const uint64_t c7 = 7u * c;
    const uint64_t u = S >= c7 ? S - c7 : c7 - S;
    const uint64_t lo = u * u, hi = frame::umulhi64(u, u);
    const uint64_t s0 = q0 + lo;
    const uint64_t k0 = s0 < lo ? 1u : 0u;
    const uint64_t t1 = q1 + hi;
    const uint64_t k1 = t1 < hi ? 1u : 0u;
    const uint64_t s1 = t1 + k0;
    const uint64_t k2 = s1 < t1 ? 1u : 0u;
    q0 = s0;
    q1 = s1;
    q2 += k1 + k2;
}

}  // namespace nframe

// ------------------------------------------------------------------------
// The binary32 residual in 32-bit words (the residual term of the update
// launch, kernel fusion of Section III-D1).
// Let every value of a binary32 grid satisfy |v| < 2^(E - 1) (E = the grid's
// largest binary32 exponent field - 125). Two additions of constants split v
// exactly into v = H q1 + r, q1 = 2^(E - 22), and r = G q2 when r is a
// multiple of q2 = 2^(E - 45):
//   t1 = RN(v + C1), C1 = 1.5 * 2^(E + 1): t1 lies in [2^(E + 1), 2^(E + 2)],
//        where the binary32 numbers are spaced q1 apart, so t1 - C1 = H q1 is
//        v rounded to a multiple of q1 (|H| <= 2^21) and the bit pattern of t1
//        is bits(C1) + H (the patterns of one binade are consecutive
//        integers, and 2^(E + 2) continues the count).
//   r  = v - (t1 - C1), exact (|r| <= q1 / 2, a multiple of v's spacing).
//   t2 = RN(r + C2), C2 = 1.5 * 2^(E - 22): t2 lies in [q1, 2 q1], spaced q2
//        apart, and its bit pattern is bits(C2) + G, G = r rounded to a
//        multiple of q2 (|G| <= 2^22). G q2 = r exactly iff RN(t2 - C2) == r
//        (a subtraction that is itself exact): true for 0 and for every
//        |v| >= 2^(E - 22), whose spacing is at least q2.
// In a sum of bit patterns whose integer weights add up to zero the offsets
// bits(C1), bits(C2) cancel, so the Laplacian term's two parts are 32-bit
// integer sums of the raw patterns (wrapping arithmetic, exact results):
//   LH = sum_6 bits(t1_n) - 6 bits(t1_c),  |LH| <= 12 * 2^21,
//   LG = sum_6 bits(t2_n) - 6 bits(t2_c),  |LG| <= 12 * 2^22,
// and L = (LH 2^23 + LG) q2 exactly. L^2 / q2^2 = LH^2 2^46 + 2 LH LG 2^23 +
// LG^2: three 64-bit sums of 32 x 32-bit products, each term below 2^51.2,
// so up to 2^11 cells per sum stay below 2^63; their combination
// S = A 2^46 + B 2^24 + C is exact in 128 bits, and the sum of squares is
// S q2^2 = S 2^(2 E - 90).
// ------------------------------------------------------------------------
namespace r32 {

JAC_HD inline float fadd(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;  // binary32 arithmetic on the host (SSE / NEON): rounded to nearest even
#endif
}

JAC_HD inline float fsub(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}

JAC_HD inline uint32_t fbits(float v)
{
    uint32_t b;
    memcpy(&b, &v, 4);
    return b;
}

// 1.5 * 2^e as a binary32 number (e in [-126, 127]).
JAC_HD inline float c15(int e)
{
    const uint32_t b = ((uint32_t)(e + 127) << 23) | 0x400000u;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

// E for a grid whose largest binary32 exponent field is f (|v| < 2^(f - 126)).
JAC_HD inline int frame_E(int f) { return f - 125; }

// C1 and C2 are normal binary32 numbers and the result's scale is a normal
// binary64 one.
JAC_HD inline bool frame_ok(int E) { return E >= -100 && E <= 125; }

struct Split {
    uint32_t h, g;  // bit patterns of t1 and t2
};

// The split of v (c1 = C1, c2 = C2); `inexact` is set when r is not a
// multiple of q2.
JAC_HD inline Split split(float v, float c1, float c2, bool& inexact)
{
    const float t1 = fadd(v, c1);
    const float r = fsub(v, fsub(t1, c1));
    const float t2 = fadd(r, c2);
    inexact |= fsub(t2, c2) != r;
    return {fbits(t1), fbits(t2)};
}

// The split without the check (for a value another lane checks).
JAC_HD inline Split split_nc(float v, float c1, float c2)
{
    const float t1 = fadd(v, c1);
    const float r = fsub(v, fsub(t1, c1));
    return {fbits(t1), fbits(fadd(r, c2))};
}

// One part of L: n0 + ... + n5 - 6 c over bit patterns.
JAC_HD inline int32_t lpart(uint32_t c, uint32_t n0, uint32_t n1, uint32_t n2, uint32_t n3, uint32_t n4, uint32_t n5)
{
    return (int32_t)(n0 + n1 + n2 + n3 + n4 + n5 - 6u * c);
}

struct Acc {
    int64_t a, b, c;  // sums of LH^2, LH LG, LG^2
};

JAC_HD inline void add_square(int32_t lh, int32_t lg, Acc& s)
{
    s.a += (int64_t)lh * lh;
    s.b += (int64_t)lh * lg;
    s.c += (int64_t)lg * lg;
}

// (lo, hi) += x 2^sh as 128-bit two's complement (0 <= sh < 64).
JAC_HD inline void add_i128(uint64_t& lo, uint64_t& hi, int64_t x, int sh)
{
    const uint64_t xl = (uint64_t)x << sh;
    const uint64_t xh = sh ? (uint64_t)(x >> (64 - sh)) : (x < 0 ? ~0ull : 0ull);
    const uint64_t nl = lo + xl;
    hi += xh + (nl < xl ? 1u : 0u);
    lo = nl;
}

// S = a 2^46 + b 2^24 + c (nonnegative: a sum of squares) as 128 bits.
JAC_HD inline void combine(const Acc& s, uint64_t& lo, uint64_t& hi)
{
    lo = 0u;
    hi = 0u;
    add_i128(lo, hi, s.c, 0);
    add_i128(lo, hi, s.b, 24);
    add_i128(lo, hi, s.a, 46);
}

}  // namespace r32

}  // namespace jac
