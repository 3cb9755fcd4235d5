// Device-side building blocks: mbarrier + TMA inline PTX (sm_103a), order-2
// B-spline shapes, relativistic Boris rotation, block-level scans.
#pragma once
#include <stdint.h>

#include "df64.cuh"
#include "pic_internal.h"

namespace pic {

// Runs `body` with T bound to the storage/arithmetic type of a precision code:
// 0 = FP64, 1 = FP32, 2 = double-word FP32 pairs.
#define PIC_DISPATCH(prec, body)           \
    do {                                   \
        if ((prec) == 0) {                 \
            using T = double;              \
            body;                          \
        } else if ((prec) == 1) {          \
            using T = float;               \
            body;                          \
        } else {                           \
            using T = ::pic::df64;         \
            body;                          \
        }                                  \
    } while (0)

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order earlier generic-proxy accesses of shared memory before async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~2^31 SM clocks (about a
// second) so that a lost transfer turns into a status flag, never a hang.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    return true;
}

// TMA tiled load of a 3D box (x, y, component) into shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// TMA tiled load of a 4D box (x, y, z, component) into shared memory.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- numerics

// Quadratic B-spline weights of nodes (i-1, i, i+1) for delta = xi - i in [-1/2, 1/2].
template <typename T>
__device__ __forceinline__ void shape3(T delta, T S[3]) {
    const T a = T(0.5) - delta, b = T(0.5) + delta;
    S[0] = T(0.5) * a * a;
    S[1] = T(0.75) - delta * delta;
    S[2] = T(0.5) * b * b;
}

// FP64 shapes in five FP64-pipe operations instead of seven: with h = delta/2 (exact)
// and q = delta^2/2 + 1/8, the outer weights are q -/+ h (their sum is 1/4 + delta^2 and
// their difference delta), the middle one 3/4 - delta^2
__device__ __forceinline__ void shape3(double delta, double S[3]) {
    const double h = 0.5 * delta;
    const double q = fma(h, delta, 0.125);
    S[0] = q - h;
    S[1] = fma(-delta, delta, 0.75);
    S[2] = q + h;
}

// double-word shapes: FP32 constants added with DWPlusFP, exact halving
__device__ __forceinline__ void shape3(df64 delta, df64 S[3]) {
    const df64 a = add_f(-delta, 0.5f), b = add_f(delta, 0.5f);
    S[0] = scale2(a * a, 0.5f);
    S[1] = add_f(-(delta * delta), 0.75f);
    S[2] = scale2(b * b, 0.5f);
}

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
// 2/x. FP64: twice the correctly rounded reciprocal, the same value as the correctly
// rounded quotient (doubling is exact) wherever 1/x is a normal number, here for x >= 1,
// in fewer FP64-pipe instructions than the division. FP32 keeps the division, which
// measured no slower.
__device__ __forceinline__ double two_over_t(double x) { return 2.0 * __drcp_rn(x); }
__device__ __forceinline__ float two_over_t(float x) { return 2.0f / x; }

// Relativistic Boris rotation (Boris 1970): u^{n-1/2} -> u^{n+1/2}; eps = q dt/(2m).
// Returns 1/gamma^{n+1/2}.
template <typename T>
__device__ __forceinline__ T boris(T eps, const T E[3], const T B[3], T u[3]) {
    T um0 = u[0] + eps * E[0], um1 = u[1] + eps * E[1], um2 = u[2] + eps * E[2];
    const T ig = rsqrt_t(T(1) + um0 * um0 + um1 * um1 + um2 * um2);
    const T ei = eps * ig;
    const T t0 = ei * B[0], t1 = ei * B[1], t2 = ei * B[2];
    const T f = two_over_t(T(1) + t0 * t0 + t1 * t1 + t2 * t2);
    const T s0 = f * t0, s1 = f * t1, s2 = f * t2;
    // each component of both cross-product updates as two fused multiply-adds into the
    // running value (two roundings instead of the three of product, difference, sum)
    const T up0 = fma_t(um1, t2, fma_t(-um2, t1, um0));
    const T up1 = fma_t(um2, t0, fma_t(-um0, t2, um1));
    const T up2 = fma_t(um0, t1, fma_t(-um1, t0, um2));
    um0 = fma_t(up1, s2, fma_t(-up2, s1, um0));
    um1 = fma_t(up2, s0, fma_t(-up0, s2, um1));
    um2 = fma_t(up0, s1, fma_t(-up1, s0, um2));
    u[0] = um0 + eps * E[0];
    u[1] = um1 + eps * E[1];
    u[2] = um2 + eps * E[2];
    return rsqrt_t(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// Double-word Boris: the same steps, with every sum of products (|u|^2, |t|^2 and the
// two cross-product updates) as one compensated dot product.
__device__ __forceinline__ df64 boris(df64 eps, const df64 E[3], const df64 B[3], df64 u[3]) {
    const df64 h0 = eps * E[0], h1 = eps * E[1], h2 = eps * E[2];
    const df64 um0 = u[0] + h0, um1 = u[1] + h1, um2 = u[2] + h2;
    Dot2 g(1.0f);
    g.add(um0, um0), g.add(um1, um1), g.add(um2, um2);
    const df64 ei = eps * rsqrt_t(g.result());
    const df64 t0 = ei * B[0], t1 = ei * B[1], t2 = ei * B[2];
    Dot2 n(1.0f);
    n.add(t0, t0), n.add(t1, t1), n.add(t2, t2);
    const df64 f = df64(2.0f) / n.result();
    const df64 s0 = f * t0, s1 = f * t1, s2 = f * t2;
    Dot2 a0, a1, a2;
    a0.add(um0), a0.add(um1, t2), a0.add(-um2, t1);
    a1.add(um1), a1.add(um2, t0), a1.add(-um0, t2);
    a2.add(um2), a2.add(um0, t1), a2.add(-um1, t0);
    const df64 up0 = a0.result(), up1 = a1.result(), up2 = a2.result();
    Dot2 b0, b1, b2;
    b0.add(um0), b0.add(up1, s2), b0.add(-up2, s1);
    b1.add(um1), b1.add(up2, s0), b1.add(-up0, s2);
    b2.add(um2), b2.add(up0, s1), b2.add(-up1, s0);
    u[0] = b0.result() + h0;
    u[1] = b1.result() + h1;
    u[2] = b2.result() + h2;
    Dot2 k(1.0f);
    k.add(u[0], u[0]), k.add(u[1], u[1]), k.add(u[2], u[2]);
    return rsqrt_t(k.result());
}

template <typename T>
struct JType;
template <>
struct JType<double> {
    // int64 fixed point (shared FP64 atomics would run on the FP64 pipe); each add is two
    // native 32-bit atomics with the carry (jatomic)
    using type = long long;
};
#ifndef PIC_F32_FIXED_TILE
#define PIC_F32_FIXED_TILE 1
#endif
template <>
struct JType<float> {
#if PIC_F32_FIXED_TILE
    // int32 fixed point: shared-memory int32 atomics run at 3.4x the rate of FP32 ones on
    // this GPU (measured: 3.1e12 vs 0.91e12 random-address adds per second)
    using type = int;
#else
    using type = float;
#endif
};
template <>
struct JType<df64> {
    using type = long long;  // int64 fixed-point shared-memory current (see jprod)
};

// 3D tile type: the same as 2D (the FP64 kernel forms its contributions in 2^62 fixed
// point and adds them into the int64 tile).
template <typename T>
struct JType3D {
    using type = typename JType<T>::type;
};

// fixed-point exponent of an item of `count` particles: a tile entry sums at most
// `count` contributions, each below 2^cmax_exp, and must stay below 2^62 (int64 tile)
// or 2^30 (int32 tile)
template <typename JT>
__device__ __forceinline__ int item_fixed_exp(int count, int cmax_exp) {
    const int lg = 32 - __clz(count > 1 ? count - 1 : 1);  // ceil(log2(count))
    int k = (sizeof(JT) == 4 ? 30 : 61) - cmax_exp - lg;
    return k < -120 ? -120 : (k > 120 ? 120 : k);
}

// Per-axis Esirkepov data on the five nodes node0-2 .. node0+2.
template <typename T>
struct Axis5 {
    T S0[5], DS[5];
    int lo, hi;  // non-zero range of DS (and of S0 + DS/2)
};

template <typename T>
__device__ __forceinline__ void esirkepov_axis(const T s0[3], T delta1, int shift, Axis5<T>& a) {
    T s1[3];
    shape3(delta1, s1);
    const bool m = shift < 0, z = shift == 0, p = shift > 0;
    T S1[5];
    S1[0] = m ? s1[0] : T(0);
    S1[1] = m ? s1[1] : (z ? s1[0] : T(0));
    S1[2] = m ? s1[2] : (z ? s1[1] : s1[0]);
    S1[3] = p ? s1[1] : (z ? s1[2] : T(0));
    S1[4] = p ? s1[2] : T(0);
    a.S0[0] = T(0);
    a.S0[1] = s0[0];
    a.S0[2] = s0[1];
    a.S0[3] = s0[2];
    a.S0[4] = T(0);
#pragma unroll
    for (int k = 0; k < 5; k++) a.DS[k] = S1[k] - a.S0[k];
    a.lo = m ? 0 : 1;
    a.hi = p ? 4 : 3;
}

// Exact float -> double widening with integer operations only (normal numbers and
// zero; others take the conversion instruction). Keeps the widening off the FP64
// pipe, which runs at 1/64 of the FP32 rate on this GPU.
__device__ __forceinline__ double widen_f32(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    const uint32_t lo = b << 29;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen_f32(double d) { return d; }

// floor(x) as an int with integer operations only (|x| < 2^30): keeps the rounding and
// the conversion off the FP64 pipe, which the FP64 particle kernel is bound by
__device__ __forceinline__ int floor_to_int(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;  // unbiased exponent
    const bool neg = b < 0;
    if (e < 0) return (neg && (b & 0x7FFFFFFFFFFFFFFFLL) != 0) ? -1 : 0;  // |x| < 1
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = 52 - e;
    long long ip = m >> sh;  // integer part of |x|
    if (neg) ip = ((ip << sh) != m) ? -(ip + 1) : -ip;
    return (int)ip;
}

// double -> float rounded to nearest even with integer operations only when the result
// is a normal float or zero (the conversion instruction runs on the FP64 pipe); other
// values take the conversion instruction
__device__ __forceinline__ float narrow_f64(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    if ((b & 0x7FFFFFFFFFFFFFFFULL) == 0) return __uint_as_float(sign);
    const int e = (int)((b >> 52) & 0x7FFu) - 1023 + 127;  // biased FP32 exponent
    if (e <= 0 || e >= 255) return __double2float_rn(d);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    unsigned r = (unsigned)(m >> 29);
    const unsigned long long rem = m & 0x1FFFFFFFULL;
    if (rem > 0x10000000ULL || (rem == 0x10000000ULL && (r & 1u))) r += 1u;
    const unsigned f = ((unsigned)e << 23) + r;  // a mantissa carry bumps the exponent
    if (f >= 0x7F800000u) return __double2float_rn(d);
    return __uint_as_float(f | sign);
}

// field-solver constants and FP64 current values in the working precision
template <typename T>
struct FieldConst;
template <>
struct FieldConst<double> {
    static __device__ __forceinline__ double dt(const SimDev& S) { return S.dt; }
    static __device__ __forceinline__ double id(const SimDev& S, int a) { return S.c_id[a]; }
    static __device__ __forceinline__ double cur(double j) { return j; }
};
template <>
struct FieldConst<float> {
    static __device__ __forceinline__ float dt(const SimDev& S) { return S.f_dt; }
    static __device__ __forceinline__ float id(const SimDev& S, int a) { return S.f_id[a]; }
    static __device__ __forceinline__ float cur(double j) { return narrow_f64(j); }
};
template <>
struct FieldConst<df64> {
    static __device__ __forceinline__ df64 dt(const SimDev& S) { return df64(S.f_dt, S.f_dt_lo); }
    static __device__ __forceinline__ df64 id(const SimDev& S, int a) {
        return df64(S.f_id[a], S.f_id_lo[a]);
    }
    // hi = nearest float, lo = the rounded remainder (one FP64 subtraction)
    static __device__ __forceinline__ df64 cur(double j) {
        const float hi = narrow_f64(j);
        return df64(hi, narrow_f64(j - widen_f32(hi)));
    }
};

// round(x 2^s) as int64 with integer operations only, for |x| 2^s < 2^62 (the fixed-point
// exponents guarantee it); keeps the conversion off the FP64 pipe
__device__ __forceinline__ long long f64_to_fixed_shift(double x, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFu);
    if (e == 0) return 0;  // zero or far below the quantum
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
    const int sh = e - 1075 + s;  // |x| 2^s = m 2^sh
    long long r;
    if (sh >= 0)
        r = m << sh;
    else if (sh > -54)
        r = (m + (1LL << (-sh - 1))) >> (-sh);
    else
        r = 0;
    return (b >> 63) ? -r : r;
}
// round(x) as int64 (see above)
__device__ __forceinline__ long long f64_to_fixed(double x) { return f64_to_fixed_shift(x, 0); }
// a b + c for 32-bit a, b and a 64-bit c, as one multiply-add instruction (written out:
// the compiler emits a separate 64-bit addition for the same C++ expression)
__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}
// round(a w / 2^62) for a weight w held in 2^62 fixed point (|a|, |w| < 2^62), exact
// except within 2^-30 of a unit from a tie, and 0 for a zero operand. Both operands split
// at bit 31 (the high parts fit 32 bits): the high-by-high product and the two cross
// products (their sum below 2^63) in 32x32->64 multiply-adds, and the low-by-low
// product through its high word only (one 32-bit multiply; the low word is below 2^-30
// of a unit after the division). Integer operations instead of an FP64 multiply (GB300
// runs FP64 at 1/64 of its FP32 rate) or a full 128-bit product.
__device__ __forceinline__ long long fixmul62(long long a, long long w) {
    const int ah = (int)(a >> 31), wh = (int)(w >> 31);
    const int al = (int)(a & 0x7FFFFFFFLL), wl = (int)(w & 0x7FFFFFFFLL);
    // (al wl) / 2^31 in the cross products' units, plus half a unit for the rounding
    const unsigned ll = 2u * __umulhi((unsigned)al, (unsigned)wl) + (1u << 30);
    const long long mid = mad_wide(al, wh, mad_wide(ah, wl, (long long)ll));
    return mad_wide(ah, wh, mid >> 31);
}
// v 2^-k as a double: the hardware int64 -> FP64 conversion (one FP64-pipe instruction,
// rounded to nearest) and the scaling by 2^-k as an exponent subtraction (exact); a
// result below the normal range flushes to zero
__device__ __forceinline__ double scaled_to_f64(long long v, int k) {
    const long long b = __double_as_longlong(__ll2double_rn(v));
    const int e = (int)((b >> 52) & 0x7FF) - k;
    return (v == 0 || e <= 0) ? 0.0 : __longlong_as_double(b - ((long long)k << 52));
}
// tile value of the product a*b; for the fixed-point tile `a` already carries the factor
// 2^k (see jscale)
template <typename JT, typename T>
__device__ __forceinline__ JT jprod(T a, T b) {
    return JT(a * b);
}
template <>
__device__ __forceinline__ long long jprod<long long, df64>(df64 a, df64 b) {
    return fixed_prod(a, b);
}
template <>
__device__ __forceinline__ long long jprod<long long, double>(double a, double b) {
    return f64_to_fixed(a * b);
}
template <>
__device__ __forceinline__ int jprod<int, float>(float a, float b) {
    return __float2int_rn(a * b);
}
// tile value of a contribution already formed (and already carrying 2^k)
template <typename JT, typename T>
__device__ __forceinline__ JT jval(T v) {
    return JT(v);
}
template <>
__device__ __forceinline__ long long jval<long long, double>(double v) {
    return f64_to_fixed(v);
}
template <>
__device__ __forceinline__ int jval<int, float>(float v) {
    return __float2int_rn(v);
}
// charge factor scaled for the tile: exact power-of-two scaling for a fixed-point tile,
// unchanged for a floating-point one
template <typename JT, typename T>
__device__ __forceinline__ T jscale(T q, float) {
    return q;
}
template <>
__device__ __forceinline__ df64 jscale<long long, df64>(df64 q, float scale) {
    return scale2(q, scale);
}
template <>
__device__ __forceinline__ double jscale<long long, double>(double q, float scale) {
    return q * (double)scale;
}
template <>
__device__ __forceinline__ float jscale<int, float>(float q, float scale) {
    return q * scale;
}
__device__ __forceinline__ void jatomic(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void jatomic(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void jatomic(int* p, int v) { atomicAdd(p, v); }
// 64-bit tile add as two 32-bit shared-memory atomics (measured: 64-bit shared-memory
// atomic adds run at a sixth of the 32-bit rate on this GPU). The low word's add returns
// the word it replaced, which gives the carry into the high word exactly: after all adds
// the 64-bit entry holds the exact sum, whatever their order.
__device__ __forceinline__ void jatomic(long long* p, long long v) {
    unsigned* w = reinterpret_cast<unsigned*>(p);  // little-endian: low word first
    const unsigned lo = (unsigned)v;
    const unsigned old = atomicAdd(w, lo);
    atomicAdd(reinterpret_cast<int*>(w + 1), (int)(v >> 32) + (old + lo < old ? 1 : 0));
}
// tile entry -> FP64 for the global current (k: the fixed-point exponent)
__device__ __forceinline__ double jflush(float v, int) { return widen_f32(v); }
__device__ __forceinline__ double jflush(double v, int) { return v; }
__device__ __forceinline__ double jflush(long long v, int k) { return scaled_to_f64(v, k); }
__device__ __forceinline__ double jflush(int v, int k) { return scaled_to_f64((long long)v, k); }


// Esirkepov data of one axis on a four-node window that always holds both the old
// and the new support: the window starts one node before min(old node, new node).
// S0/DS on the window nodes 0..3 (DS sums to zero); `start` = window start minus
// (old node - 2), i.e. 0 or 1 in the five-node numbering.
template <typename T>
struct Axis4 {
    T S0[4], DS[4];
    int start;
};

template <typename T>
__device__ __forceinline__ void esirkepov_axis4(const T s0[3], T delta1, int shift, Axis4<T>& a) {
    T s1[3];
    shape3(delta1, s1);
    const bool m = shift < 0, p = shift > 0;
    // old support at window nodes (m ? 1..3 : 0..2), new at (p ? 1..3 : 0..2)
    a.S0[0] = m ? T(0) : s0[0];
    a.S0[1] = m ? s0[0] : s0[1];
    a.S0[2] = m ? s0[1] : s0[2];
    a.S0[3] = m ? s0[2] : T(0);
    const T n0 = p ? T(0) : s1[0];
    const T n1 = p ? s1[0] : s1[1];
    const T n2 = p ? s1[1] : s1[2];
    const T n3 = p ? s1[2] : T(0);
    a.DS[0] = n0 - a.S0[0];
    a.DS[1] = n1 - a.S0[1];
    a.DS[2] = n2 - a.S0[2];
    a.DS[3] = n3 - a.S0[3];
    a.start = m ? 0 : 1;
}

// ---------------------------------------------------------------- scans

// Exclusive block scan of one int per thread; blockDim.x a multiple of 32, <= 1024.
// `warp_sums` must hold 32 ints of shared memory. Returns the exclusive prefix and
// writes the block total to *total (all threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    const int before = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before + x - v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Two warp-aggregated claims at once, both atomics in flight together: one slot on
// c1[k1] for every lane holding a1 (k1 is the same for all lanes) and one on c2[k2[lane]]
// for every lane holding a2. All 32 lanes must call it.
__device__ __forceinline__ int2 warp_claim2(int* c1, int k1, bool a1, int* c2, int k2, bool a2) {
    const int lane = threadIdx.x & 31;
    const unsigned act1 = __ballot_sync(0xffffffffu, a1);
    const unsigned act2 = __ballot_sync(0xffffffffu, a2);
    const int lead1 = act1 ? __ffs(act1) - 1 : 0;
    unsigned peers2 = 0;
    if (a2) peers2 = __match_any_sync(act2, k2);
    const int lead2 = a2 ? __ffs(peers2) - 1 : lane;
    int b1 = 0, b2 = 0;
    if (act1 && lane == lead1) b1 = atomicAdd(c1 + k1, __popc(act1));
    if (a2 && lane == lead2) b2 = atomicAdd(c2 + k2, __popc(peers2));
    b1 = __shfl_sync(0xffffffffu, b1, lead1);
    b2 = __shfl_sync(0xffffffffu, b2, lead2);
    const unsigned lt = lanemask_lt();
    return make_int2(b1 + __popc(act1 & lt), b2 + __popc(peers2 & lt));
}

__device__ __forceinline__ int wrapi(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

}  // namespace pic
