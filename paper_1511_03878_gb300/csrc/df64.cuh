// Double-word ("double-float") arithmetic: a value hi + lo held in two FP32 numbers
// with |lo| <= ulp(hi)/2, about 48 significant bits, computed with FP32 operations
// only. GB300 executes FP64 at 1/64 of its FP32 rate; this type lets the particle
// kernel reach FP64-class accuracy (relative errors of a few 2^-48) on the FP32 pipes.
//
// Building blocks (published error-free transformations):
//   TwoSum            Knuth, TAOCP vol. 2, 4.2.2 (6 flops, exact sum)
//   Fast2Sum          Dekker 1971 (3 flops, exact when |a| >= |b|)
//   TwoProd           product with FMA (exact product)
// Operations: DWPlusDW (accurate), DWTimesDW and DWTimesFP with FMA, following Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44 (2017); division and reciprocal square root by
// Newton corrections of the FP32 result.
// Intrinsics with explicit rounding (__fadd_rn, __fmul_rn) keep the compiler from
// contracting or reassociating inside the transformations.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace pic {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit df64(float h) : hi(h), lo(0.0f) {}
    __host__ __device__ constexpr explicit df64(int i) : hi((float)i), lo(0.0f) {}
    // exact split of a double (48 of its 53 bits); compile-time for literals
    __host__ __device__ constexpr explicit df64(double d)
        : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

template <typename T>
struct is_f64 : std::false_type {};
template <>
struct is_f64<double> : std::true_type {};
// particle positions: FP64 keeps global cell-unit coordinates, the others a cell
// index plus an offset in [0, 1)
template <typename T>
__host__ __device__ constexpr bool uses_cell() {
    return !is_f64<T>::value;
}

#ifdef __CUDACC__

__device__ __forceinline__ df64 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return df64(s, e);
}

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df64(s, __fadd_rn(b, -__fadd_rn(s, -a)));
}

__device__ __forceinline__ df64 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return df64(p, __fmaf_rn(a, b, -p));
}

// DWPlusDW, accurate variant (relative error below 3u^2 + 13u^3, u = 2^-24)
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
    const df64 s = two_sum(x.hi, y.hi);
    const df64 t = two_sum(x.lo, y.lo);
    const float c = __fadd_rn(s.lo, t.hi);
    const df64 v = fast_two_sum(s.hi, c);
    const float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }

// DWPlusFP: x + b for an FP32 number b (relative error below 2u^2)
__device__ __forceinline__ df64 add_f(df64 x, float b) {
    const df64 s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

// DWTimesDW with FMA (relative error below 4u^2)
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
    const df64 c = two_prod(x.hi, y.hi);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    const float cl3 = __fadd_rn(c.lo, cl2);
    return fast_two_sum(c.hi, cl3);
}

// DWTimesFP with FMA (x times an FP32 number)
__device__ __forceinline__ df64 mul_f(df64 x, float b) {
    const df64 c = two_prod(x.hi, b);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, b, c.lo));
}

// quotient: FP32 quotient q, remainder r = x - y q in double-word, one correction
__device__ __forceinline__ df64 operator/(df64 x, df64 y) {
    const float q = __fdiv_rn(x.hi, y.hi);
    const df64 r = x - mul_f(y, q);
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q, q2);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool operator<(df64 a, df64 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

// exact scaling by a power of two
__device__ __forceinline__ df64 scale2(df64 x, float p2) {
    return df64(__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2));
}

// 1/sqrt(x): FP32 estimate (within 2 ulp), one Newton step y <- y + y (1 - x y^2) / 2
// in double-word: relative error about 2^-43
__device__ __forceinline__ df64 rsqrt_t(df64 x) {
    df64 y(rsqrtf(x.hi));
    const df64 e = add_f(-(x * (y * y)), 1.0f);
    return y + scale2(y, 0.5f) * e;
}

// Compensated dot product accumulator (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), Dot2 extended to double-word inputs):
// exact hi*hi products by TwoProd, cross terms by FMA, the running sum by TwoSum with
// the errors gathered in FP32; absolute error about 2^-48 sum |a_i b_i|.
struct Dot2 {
    float s = 0.0f, c = 0.0f;
    Dot2() = default;
    __device__ __forceinline__ explicit Dot2(float s0) : s(s0), c(0.0f) {}
    // a plain double-word term
    __device__ __forceinline__ void add(df64 v) {
        const df64 t = two_sum(s, v.hi);
        s = t.hi;
        c = __fadd_rn(c, __fadd_rn(t.lo, v.lo));
    }
    __device__ __forceinline__ void add(df64 a, df64 b) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
        const df64 t = two_sum(s, p);
        s = t.hi;
        c = __fadd_rn(c, __fadd_rn(t.lo, e));
    }
    __device__ __forceinline__ df64 result() const { return fast_two_sum(s, c); }
};

// Fixed-point conversions for an int64 current accumulator: v * 2^k rounded to an
// integer with integer operations only (|v| 2^k < 2^62), and back.
__device__ __forceinline__ long long f32_to_fixed(float x) {
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu);
    if (e == 0) return 0;  // zero or below the quantum
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 150;
    long long r;
    if (sh >= 0)
        r = m << sh;
    else if (sh > -25)
        r = (m + (1LL << (-sh - 1))) >> (-sh);
    else
        r = 0;
    return (b >> 31) ? -r : r;
}

// fixed-point value of a product a*b, a already carrying the fixed-point factor 2^k:
// the rounded product of the high parts and its exact error (FMA) plus the cross terms,
// each FP32 part converted on its own (no renormalisation needed before an integer sum)
__device__ __forceinline__ long long fixed_prod(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float t = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.lo)));
    const float e = __fadd_rn(__fmaf_rn(a.hi, b.hi, -p), t);
    return f32_to_fixed(p) + f32_to_fixed(e);
}

// int64 -> double times 2^-k built with integer operations (exact below 2^53,
// rounded to nearest above)
__device__ __forceinline__ double fixed_to_f64(long long q, int k) {
    if (q == 0) return 0.0;
    const unsigned long long sign = q < 0 ? 0x8000000000000000ULL : 0ULL;
    const unsigned long long a = q < 0 ? (unsigned long long)(-q) : (unsigned long long)q;
    int msb = 63 - __clzll((long long)a);
    unsigned long long mant;
    if (msb > 52) {
        const int sh = msb - 52;
        mant = (a + (1ULL << (sh - 1))) >> sh;
        if (mant >> 53) {  // the rounding carried into a new leading bit
            mant >>= 1;
            msb += 1;
        }
    } else {
        mant = a << (52 - msb);
    }
    const long long ex = (long long)msb - k + 1023;
    if (ex <= 0) return 0.0;
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)ex << 52) | (mant & 0xFFFFFFFFFFFFFULL)));
}

// 2^e as an FP32 number (-126 <= e <= 127)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

#endif  // __CUDACC__

}  // namespace pic
