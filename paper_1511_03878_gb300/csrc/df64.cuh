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

// 1/sqrt(x): FP32 estimate, two Newton steps y <- y + y (1 - x y^2) / 2 in double-word
__device__ __forceinline__ df64 rsqrt_t(df64 x) {
    df64 y(rsqrtf(x.hi));
    for (int i = 0; i < 2; i++) {
        const df64 e = df64(1.0f) - x * (y * y);
        y = y + mul_f(y, 0.5f) * e;
    }
    return y;
}

#endif  // __CUDACC__

}  // namespace pic
