// Device arithmetic of the Jacobi step (Shao & Nakatsukasa, Sec. 2, Eq. (1.1)).
//
// Every FP64 operation below is written with an explicit rounding intrinsic
// (__dadd_rn, __dmul_rn, __fma_rn, __dsqrt_rn, __ddiv_rn), so the result does
// not depend on compiler contraction: the rotation, the updated entries and
// the gap score are the IEEE-rounded values of the stated expressions.
//
// Expressions (the paper gives the rotation only as "compute c and s such
// that G_ij^T A_ij G_ij is diagonal"; the standard symmetric 2x2 Schur form
// with |theta| <= pi/4 is used):
//   d   = a_ii - a_jj,  q = a_ij,  q2 = q*q
//   den = |d| + sqrt(d*d + 4*q2)
//   L   = (2*q2) / den                                  (Eq. (1.1))
//   t   = (2|q|) / den, negated when d != 0 and sign(d) != sign(q)
//   c   = den / sqrt(den*den + 4*q2)   (= 1/sqrt(1+t^2)),  s = t*c
//   a_ii' = fma(t, q, a_ii),  a_jj' = fma(-t, q, a_jj),  a_ij' = 0
//   x' = fma(c, x, s*y),  y' = fma(c, y, -(s*x))   for (a_ki, a_kj), (v_ki, v_kj)
// When max(|d|,|q|) lies outside [2^-500, 2^500] both are first scaled by the
// exact power of two 2^-ilogb(max) (L is homogeneous of degree 1, t and c of
// degree 0).
#pragma once
#include <cstdint>
#include <climits>

namespace pjac {

// The GPU's global nanosecond timer (wall time, independent of the SM clock).
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The scaling exponent: ilogb(m) when m = max(|d|, |q|) > 2^500 or
// m < 2^-500, else 0.  Non-negative doubles order as their bit patterns, so
// the maximum and both tests are integer operations (an FP64 compare waits
// on the FP64 pipe's long latency).
__device__ __forceinline__ int scale_exp(double d, double q) {
    const unsigned long long ud = (unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffULL;
    const unsigned long long uq = (unsigned long long)__double_as_longlong(q) & 0x7fffffffffffffffULL;
    const unsigned long long um = ud > uq ? ud : uq;
    if (um > 0x5F30000000000000ULL || um < 0x20B0000000000000ULL)   // 2^500, 2^-500
        return ilogb(__longlong_as_double((long long)um));
    return 0;
}

// t negated when d != 0 and sign(d) != sign(q), tested on the sign bits
__device__ __forceinline__ bool opposite_nonzero(double d, double q) {
    const unsigned long long bd = (unsigned long long)__double_as_longlong(d);
    const unsigned long long bq = (unsigned long long)__double_as_longlong(q);
    return (bd & 0x7fffffffffffffffULL) != 0 && ((bd ^ bq) >> 63) != 0;
}

// Eq. (1.1) for diagonal entries dii, djj and off-diagonal q.
__device__ __forceinline__ double gap_exact(double dii, double djj, double q) {
    if ((__double_as_longlong(q) & 0x7fffffffffffffffLL) == 0) return 0.0;
    double d = __dadd_rn(dii, -djj);
    int e = scale_exp(d, q);
    if (e != 0) { d = ldexp(d, -e); q = ldexp(q, -e); }
    double q2 = __dmul_rn(q, q);
    double r = __dsqrt_rn(__dadd_rn(__dmul_rn(d, d), __dmul_rn(4.0, q2)));
    double den = __dadd_rn(fabs(d), r);
    double l = __ddiv_rn(__dmul_rn(2.0, q2), den);
    if (e != 0) l = ldexp(l, e);
    return l;
}

struct Rot { double c, s, t; };

__device__ __forceinline__ Rot rot_params(double dii, double djj, double q) {
    Rot r;
    if ((__double_as_longlong(q) & 0x7fffffffffffffffLL) == 0) { r.c = 1.0; r.s = 0.0; r.t = 0.0; return r; }
    double d = __dadd_rn(dii, -djj);
    int e = scale_exp(d, q);
    if (e != 0) { d = ldexp(d, -e); q = ldexp(q, -e); }
    double q2 = __dmul_rn(q, q);
    double q4 = __dmul_rn(4.0, q2);
    double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(d, d), q4));
    double den = __dadd_rn(fabs(d), rr);
    double t = __ddiv_rn(__dmul_rn(2.0, fabs(q)), den);
    if (opposite_nonzero(d, q)) t = -t;
    double c = __ddiv_rn(den, __dsqrt_rn(__dadd_rn(__dmul_rn(den, den), q4)));
    r.t = t;
    r.c = c;
    r.s = __dmul_rn(t, c);
    return r;
}

// Exact Eq. (1.1) score and the rotation of pivot (i, j), i < j, from one
// shared denominator: l equals gap_exact(dii, djj, q) and (c, s, t) equal
// rot_params(dii, djj, q), bit for bit (the score depends on |d| only).
struct Eval { double l, c, s, t; };

__device__ __forceinline__ Eval eval_pair(double dii, double djj, double q) {
    Eval r;
    if ((__double_as_longlong(q) & 0x7fffffffffffffffLL) == 0) { r.l = 0.0; r.c = 1.0; r.s = 0.0; r.t = 0.0; return r; }
    double d = __dadd_rn(dii, -djj);
    int e = scale_exp(d, q);
    if (e != 0) { d = ldexp(d, -e); q = ldexp(q, -e); }
    double q2 = __dmul_rn(q, q);
    double q4 = __dmul_rn(4.0, q2);
    double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(d, d), q4));
    double den = __dadd_rn(fabs(d), rr);
    double l = __ddiv_rn(__dmul_rn(2.0, q2), den);
    if (e != 0) l = ldexp(l, e);
    double t = __ddiv_rn(__dmul_rn(2.0, fabs(q)), den);
    if (opposite_nonzero(d, q)) t = -t;
    double c = __ddiv_rn(den, __dsqrt_rn(__dadd_rn(__dmul_rn(den, den), q4)));
    r.l = l;
    r.t = t;
    r.c = c;
    r.s = __dmul_rn(t, c);
    return r;
}

// The same evaluation in two halves, so that the score can be published
// before the cosine is known: the head gives l and t (as eval_pair) and the
// scaled den and 4q^2; rot_cs then gives c and s from them, bit for bit as
// eval_pair (c is a ratio of scaled quantities, so the scaling drops out).
struct EvalHead { double l, t, den, q4; };

__device__ __forceinline__ EvalHead eval_pair_head(double dii, double djj, double q) {
    EvalHead r;
    if ((__double_as_longlong(q) & 0x7fffffffffffffffLL) == 0) {   // q == 0 (rot_cs: c = 1, s = 0)
        r.l = 0.0; r.t = 0.0; r.den = 1.0; r.q4 = 0.0;
        return r;
    }
    double d = __dadd_rn(dii, -djj);
    int e = scale_exp(d, q);
    if (e != 0) { d = ldexp(d, -e); q = ldexp(q, -e); }
    double q2 = __dmul_rn(q, q);
    double q4 = __dmul_rn(4.0, q2);
    double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(d, d), q4));
    double den = __dadd_rn(fabs(d), rr);
    double l = __ddiv_rn(__dmul_rn(2.0, q2), den);
    if (e != 0) l = ldexp(l, e);
    double t = __ddiv_rn(__dmul_rn(2.0, fabs(q)), den);
    if (opposite_nonzero(d, q)) t = -t;
    r.l = l;
    r.t = t;
    r.den = den;
    r.q4 = q4;
    return r;
}

__device__ __forceinline__ void rot_cs(double den, double q4, double t, double& c, double& s) {
    c = __ddiv_rn(den, __dsqrt_rn(__dadd_rn(__dmul_rn(den, den), q4)));
    s = __dmul_rn(t, c);
}

// ---------------------------------------------------------------------------
// Screen keys.  Selecting the pivot needs the exact argmax of the FP64
// scores (ties to the smallest index), but an FP64 square root and division
// per entry are expensive.  Entries are first ranked by a 32-bit integer key
// computed with integer and FP32 instructions; only entries whose key lies
// within KEY_TIE of the best key are evaluated exactly.
//
// Gap rule: key = floor(2^20 * log2(L~)).  Error budget of log2 L~:
// mantissas truncated to 23 bits (2^-23 relative each), the FP32 quotient,
// square root and reciprocal taken from the fast approximations (__fdividef
// and rsqrtf, each within 2 ulp) plus a few correctly rounded FP32
// operations -- about 12 ulp = 12 * 2^-24 relative in all, 2^-19.5 in log2
// -- and __log2f, within 2 ulp of a result of magnitude <= 64 (<= 2^-17
// absolute).  The key is therefore within 12 units of 2^20 log2 L, and
// KEY_GAP_TIE = 64 units keeps more than a 2x margin over twice that: an
// entry whose key is more than KEY_GAP_TIE below another's has a strictly
// smaller FP64 score.  The asymptotic forms below are exact to 2^-118.
// Greedy rule: key = high 32 bits of |x| (monotone in |x|); entries with the
// same key are compared on the full |x|.
// ---------------------------------------------------------------------------
constexpr int KEY_NONE = INT_MIN;          // no candidate
constexpr int KEY_ZERO = INT_MIN + 1;      // x == 0: score exactly 0
constexpr int KEY_GAP_TIE = 64;
// Below 2^-500 every candidate is compared exactly: an unscaled FP64 score
// 2*q2/den loses accuracy only when q*q underflows, which (with
// max(|d|,|q|) >= 2^-500, else the operands are rescaled) needs
// L < 2^-1022/2^-500 = 2^-522.
constexpr int KEY_SUB = -500 * (1 << 20);

__device__ __forceinline__ float mant23(unsigned long long b) {
    return __int_as_float(0x3f800000u | (unsigned)((b >> 29) & 0x7fffffu));
}

// Unbiased exponent and the top 23 mantissa bits of a non-negative double
// (magnitude bit pattern b != 0), subnormals normalised with integer shifts
// (the leading one moved to the implicit bit).
__device__ __forceinline__ void split_bits(unsigned long long b, int& e, float& m23) {
    const int ef = (int)(b >> 52);
    unsigned long long mb = b & 0x000fffffffffffffULL;
    if (ef == 0) {
        const int lz = __clzll((long long)mb);      // >= 12
        mb = (mb << (lz - 11)) & 0x000fffffffffffffULL;
        e = -1011 - lz;
    } else {
        e = ef - 1023;
    }
    m23 = mant23(mb);
}

// Branch-free: every case's operands are formed and the argument of the one
// logarithm is selected, so that two keys of one thread interleave.
__device__ __forceinline__ int gap_key(double x, double dd) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    const unsigned long long bd = (unsigned long long)__double_as_longlong(dd) & 0x7fffffffffffffffULL;
    int exu, edu;
    float mx, md;
    split_bits(bx | (bx == 0), exu, mx);            // (x == 0 is answered at the end)
    split_bits(bd | (bd == 0), edu, md);
    const int e = edu - exu;
    // |d| far below |x| (or d == 0): L ~ |x|
    float arg = mx;
    int ip = exu;
    if (bd != 0 && e >= 60) {                        // |d| far above |x|: L ~ x^2/|d|
        arg = __fdividef(mx * mx, md);
        ip = 2 * exu - edu;
    } else if (bd != 0 && e > -60) {
        const float rho = __fdividef(md, mx) * __int_as_float((e + 127) << 23);
        const float v = __fmaf_rn(rho, rho, 4.0f);
        const float g = __fdividef(2.0f, rho + v * rsqrtf(v));
        arg = mx * g;
    }
    const float f = __log2f(arg);
    if (ip < -2040) ip = -2040;
    const int key = ip * (1 << 20) + __float2int_rd(f * 1048576.0f);
    return bx == 0 ? KEY_ZERO : key;
}

__device__ __forceinline__ int greedy_key(double x) {
    unsigned long long bx = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    return (int)(bx >> 32);
}

// The randomized pivot rule's pair of step k (Sec. 4.2's comparator: every
// pair equally likely).  The draw is the output function of Steele, Lea and
// Flood's SplitMix64 generator applied to the counter seed + (k+1) gamma;
// its low word picks i among n, its high word j among the other n-1.
__device__ __forceinline__ void random_pair(unsigned long long seed, long long k, int n, int& i, int& j) {
    unsigned long long z = seed + (unsigned long long)(k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    const int a = (int)((unsigned)z % (unsigned)n);
    int b = (int)((unsigned)(z >> 32) % (unsigned)(n - 1));
    if (b >= a) b++;
    i = min(a, b);
    j = max(a, b);
}

// Order-preserving 64-bit integer image of a double (for sorting W).
__device__ __forceinline__ unsigned long long order_key(double w) {
    unsigned long long b = (unsigned long long)__double_as_longlong(w);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

}  // namespace pjac
