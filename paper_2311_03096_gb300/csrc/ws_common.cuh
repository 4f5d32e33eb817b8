// ws_common.cuh -- shared device helpers of the GB300 prox_R path.
//
// Notation (arXiv 2311.03096): a segment of d weights is sorted ascending into
// x_0..x_{d-1} (0-based here); the shift of Alg. 2 for sorted position j is
// lambda*(d - 1 - 2j)/(d - 1) (the paper's lambda(d+1-2k)/(d-1) with k = j+1).
// Points P_p = (p, S_p), p = 0..d, S_p = sum_{j<p} y_j: the isotonic
// regression of y (Sec. 3) is the slope sequence of the lower convex hull of
// these points, pooled on >= (Sec. 4.1).  Two facts make the hull exact and
// cheap:
//   * S_p = X_p + lambda p (d - p)/(d - 1) with X_p = sum_{j<p} x_j, so
//     slope(a, b) = mean(x_a..x_{b-1}) + lambda (d - a - b)/(d - 1): the shift
//     never has to be stored;
//   * X is carried in 128-bit fixed point (q_j = x_j * 2^L, |q_j| <= 2^58, L
//     the smallest scale at which every value is an integer when that fits,
//     exact for every input whose values span < ~2^(58-24) of dynamic range),
//     and the "is b a strict hull vertex between a and c" test is decided
//     with exact integer arithmetic (below), so merge decisions never round.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// status bits OR-ed into the context's device status word
// ---------------------------------------------------------------------------
enum : uint32_t {
    WS_STATUS_NONFINITE = 1u,
    WS_STATUS_TIMEOUT = 2u,
    WS_STATUS_INTERNAL = 4u,
    WS_STATUS_BAD_LAMBDA = 8u,
    WS_STATUS_INEXACT = 16u,   // information, not an error (ws_note_scale)
};

__device__ __forceinline__ void ws_flag(uint32_t* status, uint32_t bit) {
    if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------------------
// IEEE total-order keys (-0 < +0), as unsigned integers
// ---------------------------------------------------------------------------
template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
    typedef uint32_t K;
    static constexpr int BITS = 32;
    static constexpr int MANT = 23;   // stored mantissa bits
    static constexpr int EXPMASK = 0xff;
    static constexpr int FIX_OFS = 34;   // 58 - (MANT + 1)
    static constexpr int L_BASE = 184;   // L = L_BASE - emax  (150 + FIX_OFS)
    __device__ __forceinline__ static K to_key(float v) {
        uint32_t b = __float_as_uint(v);
        return b ^ ((b >> 31) ? 0xffffffffu : 0x80000000u);
    }
    __device__ __forceinline__ static float from_key(K k) {
        return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xffffffffu));
    }
    __device__ __forceinline__ static uint32_t bits(float v) { return __float_as_uint(v); }
};
template <> struct KeyOf<double> {
    typedef uint64_t K;
    static constexpr int BITS = 64;
    static constexpr int MANT = 52;
    static constexpr int EXPMASK = 0x7ff;
    static constexpr int FIX_OFS = 5;     // 58 - (MANT + 1)
    static constexpr int L_BASE = 1080;   // 1075 + FIX_OFS
    __device__ __forceinline__ static K to_key(double v) {
        uint64_t b = (uint64_t)__double_as_longlong(v);
        return b ^ ((b >> 63) ? 0xffffffffffffffffull : 0x8000000000000000ull);
    }
    __device__ __forceinline__ static double from_key(K k) {
        return __longlong_as_double((long long)(k ^ ((k >> 63) ? 0x8000000000000000ull : 0xffffffffffffffffull)));
    }
    __device__ __forceinline__ static uint64_t bits(double v) { return (uint64_t)__double_as_longlong(v); }
};

template <typename T> __device__ __forceinline__ bool ws_isfinite(T v) {
    typedef KeyOf<T> KO;
    uint64_t b = (uint64_t)KO::bits(v);
    int e = (int)((b >> KO::MANT) & KO::EXPMASK);
    return e != KO::EXPMASK;
}

// Effective biased exponent (denormals count as exponent 1).
template <typename T> __device__ __forceinline__ int ws_eff_exp(T v) {
    typedef KeyOf<T> KO;
    uint64_t b = (uint64_t)KO::bits(v);
    int e = (int)((b >> KO::MANT) & KO::EXPMASK);
    return e == 0 ? 1 : e;
}

// Fixed-point image q = x * 2^L, L = L_BASE - emax (emax: the scale parameter
// E of ws_fix_scale), truncated toward zero when x has bits below 2^-L
// (monotone, so sorted order is preserved).  |q| <= 2^58 whenever the
// effective exponent of x is <= E.
template <typename T> __device__ __forceinline__ int64_t ws_fixed(T v, int emax) {
    typedef KeyOf<T> KO;
    uint64_t b = (uint64_t)KO::bits(v);
    int e = (int)((b >> KO::MANT) & KO::EXPMASK);
    uint64_t m = b & ((1ull << KO::MANT) - 1ull);
    if (e == 0) e = 1; else m |= (1ull << KO::MANT);
    int sh = e - emax + KO::FIX_OFS;
    uint64_t mag;
    if (sh >= 0) mag = m << sh;            // sh <= FIX_OFS, so m << sh < 2^58
    else mag = (sh > -64) ? (m >> (-sh)) : 0ull;
    bool neg = (b >> (KO::BITS - 1)) & 1ull;
    return neg ? -(int64_t)mag : (int64_t)mag;
}

// Scale parameter E of a segment's fixed point (L = L_BASE - E): the largest
// E at which every value is still an exact integer, E = emin + FIX_OFS, as
// long as the largest value then stays within 2^58 (E >= emax); otherwise
// E = emax and values more than FIX_OFS binades below the largest lose their
// lowest bits (toward zero).  emin / emax: smallest / largest effective
// exponent of the segment's nonzero values (emin > emax when there are none).
// Small q keeps tiles that cross binades (zero crossings) in 64-bit
// deviations instead of 128-bit sums.
template <typename T> __device__ __forceinline__ int ws_fix_scale(int emax, int emin) {
    return (emin <= emax && emax - emin <= KeyOf<T>::FIX_OFS) ? emin + KeyOf<T>::FIX_OFS : emax;
}

// Records in the status word that a segment's nonzero values span more than
// FIX_OFS binades (ws_fix_scale then returns emax and the smallest values lose
// their lowest bits in the fixed point; the partition is exact for the
// truncated values).  Information for ws_get_inexact, not an error.
template <typename T> __device__ __forceinline__ void ws_note_scale(int emax, int emin, uint32_t* status) {
    if (emin <= emax && emax - emin > KeyOf<T>::FIX_OFS) ws_flag(status, WS_STATUS_INEXACT);
}

// ---------------------------------------------------------------------------
// Per-segment constants of the exact hull test
// ---------------------------------------------------------------------------
struct SegConst {
    int64_t d;        // segment length
    int L;            // fixed-point scale: q = x * 2^L
    int s;            // e_lambda + L  (lambda = mlam * 2^e_lambda exactly)
    uint64_t mlam;    // integer mantissa of lambda (0 iff lambda == 0)
    uint64_t dm1;     // d - 1 (>= 1 when used)
    float mu_f;       // lambda / (d - 1) rounded to float
    double mu_d;      // lambda / (d - 1) in double
};

// lambda = mlam * 2^elam exactly (lambda >= 0, finite).
__device__ __forceinline__ void ws_split_lambda(double lam, uint64_t& mlam, int& elam) {
    uint64_t b = (uint64_t)__double_as_longlong(lam);
    int e = (int)((b >> 52) & 0x7ff);
    uint64_t m = b & ((1ull << 52) - 1ull);
    if (e == 0) e = 1; else m |= (1ull << 52);
    mlam = m;
    elam = e - 1075;
    if (m == 0) elam = 0;
}

// Constants for fixed-point scale 2^L (q = x * 2^L).
__device__ __forceinline__ SegConst ws_seg_const_L(int64_t d, double lam, int L) {
    SegConst c;
    c.d = d;
    c.L = L;
    int elam;
    ws_split_lambda(lam, c.mlam, elam);
    c.s = elam + c.L;
    c.dm1 = d > 1 ? (uint64_t)(d - 1) : 1ull;
    c.mu_d = d > 1 ? lam / (double)(d - 1) : 0.0;
    c.mu_f = (float)c.mu_d;
    return c;
}

// The same constants without FP64 arithmetic (GB300 runs FP64 at a small
// fraction of the FP32 rate, and a CTA's set-up is on its critical path):
// the integer fields come from lambda's bits; mu_f = mlam 2^elam / (d - 1)
// in FP32 (two roundings); mu_d (FP64 values only) on request.
__device__ __forceinline__ float ws_u64_to_float(uint64_t v);
__device__ __forceinline__ SegConst ws_seg_const_f(int64_t d, double lam, int L, bool with_mu_d) {
    SegConst c;
    c.d = d;
    c.L = L;
    int elam;
    ws_split_lambda(lam, c.mlam, elam);
    c.s = elam + L;
    c.dm1 = d > 1 ? (uint64_t)(d - 1) : 1ull;
    c.mu_f = d > 1 ? ldexpf(ws_u64_to_float(c.mlam), elam) / ws_u64_to_float(c.dm1) : 0.0f;
    c.mu_d = (with_mu_d && d > 1) ? lam / (double)(d - 1) : 0.0;
    return c;
}

template <typename T>
__device__ __forceinline__ SegConst ws_seg_const(int64_t d, double lam, int emax) {
    SegConst c;
    c.d = d;
    c.L = KeyOf<T>::L_BASE - emax;
    int elam;
    ws_split_lambda(lam, c.mlam, elam);
    c.s = elam + c.L;
    c.dm1 = d > 1 ? (uint64_t)(d - 1) : 1ull;
    c.mu_d = d > 1 ? lam / (double)(d - 1) : 0.0;
    c.mu_f = (float)c.mu_d;
    return c;
}

// ---------------------------------------------------------------------------
// 192-bit unsigned helpers for the exact comparison
// ---------------------------------------------------------------------------
struct U192 { uint64_t w0, w1, w2; };   // value = w0 + w1 2^64 + w2 2^128

__device__ __forceinline__ int ws_bitlen64(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }
__device__ __forceinline__ int ws_bitlen128(u128 v) {
    uint64_t hi = (uint64_t)(v >> 64);
    return hi ? 64 + ws_bitlen64(hi) : ws_bitlen64((uint64_t)v);
}
__device__ __forceinline__ int ws_bitlen192(const U192& v) {
    if (v.w2) return 128 + ws_bitlen64(v.w2);
    if (v.w1) return 64 + ws_bitlen64(v.w1);
    return ws_bitlen64(v.w0);
}
__device__ __forceinline__ U192 ws_mul128x64(u128 a, uint64_t b) {
    u128 lo = (u128)(uint64_t)a * b;
    u128 hi = (u128)(uint64_t)(a >> 64) * b;
    U192 r;
    r.w0 = (uint64_t)lo;
    u128 mid = (lo >> 64) + (u128)(uint64_t)hi;
    r.w1 = (uint64_t)mid;
    r.w2 = (uint64_t)(mid >> 64) + (uint64_t)(hi >> 64);
    return r;
}
__device__ __forceinline__ U192 ws_shl192(const U192& v, int k) {   // 0 <= k < 192
    U192 r = v;
    while (k >= 64) { r.w2 = r.w1; r.w1 = r.w0; r.w0 = 0; k -= 64; }
    if (k > 0) {
        r.w2 = (r.w2 << k) | (r.w1 >> (64 - k));
        r.w1 = (r.w1 << k) | (r.w0 >> (64 - k));
        r.w0 = r.w0 << k;
    }
    return r;
}
__device__ __forceinline__ int ws_cmp192(const U192& a, const U192& b) {
    if (a.w2 != b.w2) return a.w2 > b.w2 ? 1 : -1;
    if (a.w1 != b.w1) return a.w1 > b.w1 ? 1 : -1;
    if (a.w0 != b.w0) return a.w0 > b.w0 ? 1 : -1;
    return 0;
}

// ---------------------------------------------------------------------------
// The exact hull test.
//   convex(a, b, c)  <=>  slope(a, b) < slope(b, c)  <=>  P_b is a strict
//   vertex of the lower hull of {P_a, P_b, P_c}; pooling on >= means a point
//   on the chord is NOT a vertex.
// With A = X_b - X_a, B = X_c - X_b (fixed point), n1 = b - a, n2 = c - b:
//   slope(b,c) - slope(a,b) = B/n2 - A/n1 - mu (c - a),   mu = lambda/(d-1)
// so convex <=> (B n1 - A n2) (d - 1) > lambda 2^L (c - a) n1 n2, and with
// lambda = mlam 2^elam every quantity is an integer: compare
//   LHS = (B n1 - A n2) (d - 1)   vs   RHS = mlam (c - a) n1 n2 2^(elam + L).
// Sorted x gives B n1 - A n2 >= 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ws_convex(i128 Xa, i128 Xb, i128 Xc, int64_t a, int64_t b, int64_t c,
                                          const SegConst& sc) {
    i128 A = Xb - Xa, B = Xc - Xb;
    uint64_t n1 = (uint64_t)(b - a), n2 = (uint64_t)(c - b);
    i128 D = B * (i128)n1 - A * (i128)n2;
    if (D <= 0) return false;
    if (sc.mlam == 0) return true;
    u128 Du = (u128)D;
    u128 P = (u128)((uint64_t)(c - a) * n1) * (u128)n2;
    int blD = ws_bitlen128(Du), blm = ws_bitlen64(sc.dm1);
    int blP = ws_bitlen128(P), blL = ws_bitlen64(sc.mlam);
    int lhs_lo = blD + blm - 1, lhs_hi = blD + blm;
    int rhs_lo = blP + blL - 1 + sc.s, rhs_hi = blP + blL + sc.s;
    if (lhs_lo > rhs_hi) return true;
    if (lhs_hi < rhs_lo) return false;
    U192 Lv = ws_mul128x64(Du, sc.dm1);
    U192 Rv = ws_mul128x64(P, sc.mlam);
    int bl = ws_bitlen192(Lv), brr = ws_bitlen192(Rv);
    int br = brr + sc.s;
    if (bl != br) return bl > br;
    Lv = ws_shl192(Lv, 192 - bl);
    Rv = ws_shl192(Rv, 192 - brr);
    return ws_cmp192(Lv, Rv) > 0;
}

// ---------------------------------------------------------------------------
// Cluster values.  A cluster covers sorted positions [a, b) with exact
// fixed-point sum SX; its value is mean(x_a..x_{b-1}) + mu (d - a - b).
// ---------------------------------------------------------------------------
// v * 2^-neg_exp, rounded to float (high and low 64-bit halves converted
// separately, so all significant bits take part in the rounding).
// Positive 64-bit integer to float from its two 32-bit halves (no 64-bit
// conversion instruction, which GB300 runs at its FP64 rate): the halves
// round once each and the fused add once more, <= 3 * 2^-24 relative.
__device__ __forceinline__ float ws_u64_to_float(uint64_t v) {
    return fmaf((float)(uint32_t)(v >> 32), 4294967296.0f, (float)(uint32_t)v);
}
__device__ __forceinline__ float ws_i128_to_float_scaled(i128 v, int neg_exp) {
    // keep the top 62 significant bits (exact shift), then convert (<= 3 roundings)
    u128 mag = v < 0 ? (u128)(-v) : (u128)v;
    int sh = ws_bitlen128(mag) - 62;
    if (sh < 0) sh = 0;
    const float f = ws_u64_to_float((uint64_t)(mag >> sh));
    return ldexpf(v < 0 ? -f : f, sh - neg_exp);
}
// Magnitude first, sign last: the halves of a negative two's-complement value
// would cancel (hi = -1, lo ~ 2^64 - |v|) and lose the low bits of |v|.
// hi converts exactly while |v| < 2^117; lo rounds once and the fused add
// once more: <= 2 roundings relative to |v|.
__device__ __forceinline__ double ws_i128_to_double(i128 v) {
    const bool neg = v < 0;
    const u128 m = neg ? (u128)0 - (u128)v : (u128)v;
    const double r = fma(__ull2double_rn((uint64_t)(m >> 64)), 18446744073709551616.0, __ull2double_rn((uint64_t)m));
    return neg ? -r : r;
}

// S / n in FP64 arithmetic for an exact 128-bit sum S and a count n >= 1,
// without an FP64 division (GB300 runs FP64 at a small fraction of the FP32
// rate): q = the FP32 quotient (<= 4 roundings: |q - S/n| <= 2^-21 |S/n|),
// truncated to an integer Q; the remainder R = S - Q n is exact in 128 bits
// and |R / n| <= 2^-21 |S/n| + 1, so S/n = Q + R/n with R/n taken in FP32 has
// an error below 2^-42 |S/n| + 2^-21 (in the units of S).
__device__ __forceinline__ double ws_div_i128_n(i128 S, int64_t n) {
    const float q = ws_i128_to_float_scaled(S, 0) / (float)n;
    const uint32_t bits = __float_as_uint(q);
    const int e = (int)((bits >> 23) & 0xffu) - 150;   // q = m 2^e, m the 24-bit significand
    const uint32_t m = (bits & 0x7fffffu) | 0x800000u;
    u128 mag = 0;
    float qt = 0.0f;   // trunc(q), exactly Q
    if (((bits >> 23) & 0xffu) >= 127u) {   // |q| >= 1
        mag = e >= 0 ? ((u128)m << e) : (u128)(m >> (-e));
        qt = truncf(q);
    }
    const i128 Q = (bits >> 31) ? -(i128)mag : (i128)mag;
    const i128 R = S - Q * (i128)n;
    const float corr = ws_i128_to_float_scaled(R, 0) / (float)n;
    return (double)qt + (double)corr;
}

// Weight sharing + l1 with rewinding (Rewinding section, Alg. 2): a cluster
// with mean position x and mean velocity v (its shift) ends at
//   0                                  if |x + v| < beta,
//   x + gamma (v - beta sign(x + v))   otherwise, gamma = v_scale (1 - rho);
// with the epilogue off it ends at x + v (the prox of lambda R alone).
struct WsEpi {
    double beta, gamma;
    float beta_f, gamma_f;
    int on;
};

template <typename V>
__device__ __forceinline__ V ws_epilogue(V x, V v, V beta, V gamma, bool on) {
    const V s = x + v;
    if (!on) return s;
    if ((s < (V)0 ? -s : s) < beta) return (V)0;
    return x + gamma * (v - (s > (V)0 ? beta : -beta));
}

template <typename T> struct ValueOut;
template <> struct ValueOut<float> {
    __device__ __forceinline__ static float value(i128 SX, int64_t a, int64_t b, float xsingle, const SegConst& sc,
                                                  bool fp64, const WsEpi& ep) {
        int64_t n = b - a;
        int64_t t = sc.d - a - b;
        if (fp64) {
            double mean = (n == 1) ? (double)xsingle : ldexp(ws_div_i128_n(SX, n), -sc.L);
            return (float)ws_epilogue<double>(mean, sc.mu_d * (double)t, ep.beta, ep.gamma, ep.on != 0);
        }
        float mean = (n == 1) ? xsingle : ldexpf(ws_i128_to_float_scaled(SX, 0) / (float)n, -sc.L);
        return ws_epilogue<float>(mean, sc.mu_f * (float)t, ep.beta_f, ep.gamma_f, ep.on != 0);
    }
};
template <> struct ValueOut<double> {
    __device__ __forceinline__ static double value(i128 SX, int64_t a, int64_t b, double xsingle,
                                                   const SegConst& sc, bool fp64, const WsEpi& ep) {
        int64_t n = b - a;
        int64_t t = sc.d - a - b;
        if (!fp64) {
            // FP32 arithmetic on the exact sum, widened to the output type
            float mean = (n == 1) ? (float)xsingle : ldexpf(ws_i128_to_float_scaled(SX, 0) / (float)n, -sc.L);
            return (double)ws_epilogue<float>(mean, sc.mu_f * (float)t, ep.beta_f, ep.gamma_f, ep.on != 0);
        }
        double mean = (n == 1) ? xsingle : ldexp(ws_div_i128_n(SX, n), -sc.L);
        return ws_epilogue<double>(mean, sc.mu_d * (double)t, ep.beta, ep.gamma, ep.on != 0);
    }
};

// ---------------------------------------------------------------------------
// Bounded spin-wait helper: every device-side wait has an iteration limit.
// ---------------------------------------------------------------------------
// L2 eviction priorities.  The lookup directory is re-read at random by every
// weight while the weights and outputs stream through L2 once, so the
// directory is loaded and stored with evict_last and the streams with
// evict_first (.cs).
__device__ __forceinline__ uint64_t ws_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint2 ws_ld_u2_last(const void* ptr, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void ws_st_u2_last(void* ptr, uint2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(ptr), "r"(v.x), "r"(v.y), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void ws_backoff(int it) {
    if (it > 64) __nanosleep(it > 4096 ? 256 : 32);
}
