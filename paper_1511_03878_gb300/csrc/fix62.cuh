// 2^62 fixed-point arithmetic for the FP64 particle kernels.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, while its integer units run at half the
// FP32 rate, so an FP64 particle kernel is bound by the FP64 pipe. Every quantity of the
// order-2 PIC cycle that is not itself a result of the FP64 push -- a particle's in-cell
// offset, its quadratic B-spline weights, the field gather (from a fixed-point copy of
// the staged field tile), the Esirkepov shape differences, path-averaged weights and
// running sums, and the products that form a current contribution -- is computed here
// exactly or to a few units of 2^-62 (2^-60 of the tile's largest field for the gather)
// in int64 arithmetic built from 32x32->64-bit products. That is finer than FP64
// rounding for values in [-1, 1] (2^-53 relative, 2^-54 absolute near 1), so the FP64
// results built from them (fields at the particle, current) agree with an all-FP64
// evaluation to rounding. The FP64 pipe keeps the Boris push, the move and the charge
// factors.
#pragma once
#include <stdint.h>

#include "pic_device.cuh"

namespace pic {

constexpr long long kOne62 = 1LL << 62;
constexpr long long kHalf62 = 1LL << 61;
// round(2^62 / 3): the 1/3 of the path-averaged weight of Esirkepov's transverse current
constexpr long long kThird62 = 1537228672809129301LL;

// floor(x) and the fractional part x - floor(x) in 2^62 fixed point ([0, 2^62)), from the
// bit pattern of x with integer operations only. Exact for |x| < 2^30 (a fraction below
// 2^-62 is truncated). Non-finite or larger |x| give i = -2^30, f = 0 (outside any grid).
__device__ __forceinline__ void split62(double x, int& i, long long& f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7FFu);
    const int e = eb - 1023;  // unbiased exponent
    if (eb == 0) {            // zero or subnormal: below the 2^-62 resolution
        i = 0;
        f = 0;
        return;
    }
    if (e >= 30) {
        i = -(1 << 30);
        f = 0;
        return;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);  // x = m 2^(e-52)
    unsigned long long ip, fr;
    if (e < -10) {
        ip = 0;
        const int s = -(e + 10);
        fr = s < 64 ? (m >> s) : 0;
    } else if (e < 0) {
        ip = 0;
        fr = m << (e + 10);  // below 2^62
    } else {
        ip = m >> (52 - e);
        fr = (m << (e + 10)) & (unsigned long long)(kOne62 - 1);
    }
    if (b >> 63) {  // negative: floor is -(ip + 1) unless x is an integer
        if (fr == 0) {
            i = -(int)ip;
            f = 0;
        } else {
            i = -(int)ip - 1;
            f = kOne62 - (long long)fr;
        }
    } else {
        i = (int)ip;
        f = (long long)fr;
    }
}

// Quadratic B-spline weights of nodes (i-1, i, i+1) for delta = D 2^-62 in [-1/2, 1/2]
// (S[k] in 2^62 fixed point): S0 = (1/2 - delta)^2 / 2, S1 = 3/4 - delta^2,
// S2 = (1/2 + delta)^2 / 2, written as q -/+ delta/2 with q = delta^2/2 + 1/8.
__device__ __forceinline__ void shape62(long long D, long long S[3]) {
    // delta^2 2^62 (<= 2^60) from |D| = ah 2^31 + al: ah^2 + 2 ah al 2^-31, the al^2 term
    // (below one unit) left out; within two units below the exact square
    const long long a = D < 0 ? -D : D;  // <= 2^61
    const int ah = (int)(a >> 31), al = (int)(a & 0x7FFFFFFFLL);
    const long long d2 = mad_wide(ah, ah, mad_wide(ah, al, 0LL) >> 30);
    const long long h = D >> 1;                                 // delta/2
    const long long q = (d2 >> 1) + (1LL << 59);                // delta^2/2 + 1/8
    S[0] = q - h;
    S[1] = 3LL * (1LL << 60) - d2;
    S[2] = q + h;
}

// ---- Field gather in fixed point. The FP64 kernel converts its staged field tile once per
// load: each component gets the exponent s that puts the tile's largest magnitude just
// below 2^60, and each entry F becomes round(F 2^s) = h 2^31 + l (0 <= l < 2^31, |h| <
// 2^29), stored as the 32-bit pair (l, h) in the 8 bytes of the double it replaces.

// exponent s of a component whose largest biased FP64 exponent field is emax:
// |F| < 2^(emax - 1022), so |F| 2^s < 2^60
__device__ __forceinline__ int fix_field_exp(int emax) { return 1082 - emax; }

// In-place conversion of the staged FP64 field tile (6 components of `pl` entries) to
// split fixed point; s_emax[6] (zeroed by the caller before the barrier that precedes
// this call) receives each component's largest exponent field (0x7FF: a non-finite
// entry). Every thread of the CTA calls it; it ends before the caller's next barrier
// only for the calling thread, so the caller synchronises before the tile is read.
__device__ __forceinline__ void fix_field_tile(double* F, int pl, int* s_emax) {
    for (int c = 0; c < 6; c++) {
        int m = 0;
        for (int i = threadIdx.x; i < pl; i += blockDim.x) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(F[c * pl + i]);
            m = max(m, (int)((b >> 52) & 0x7FFu));
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_emax[c], m);
    }
    __syncthreads();  // exponents complete; every entry read before any is overwritten
    for (int e = threadIdx.x; e < 6 * pl; e += blockDim.x) {
        const int c = e / pl;
        const int s = fix_field_exp(s_emax[c]);
        // round(F 2^s): the scaling as an exponent addition (exact), then the hardware
        // FP64 -> int64 conversion; magnitudes below 1/2 after scaling round to 0
        const long long b = __double_as_longlong(F[e]);
        const int eb = (int)((b >> 52) & 0x7FFu);
        const long long u = (eb == 0 || eb + s < 1022)
                                ? 0LL
                                : __double2ll_rn(__longlong_as_double(b + ((long long)s << 52)));
        reinterpret_cast<int2*>(F)[e] = make_int2((int)(u & 0x7FFFFFFFLL), (int)(u >> 31));
    }
}

// v 2^-k as a double with integer operations only (the mantissa truncated to 53 bits; 0
// below the normal range), for |v| < 2^62: the gathered fields' return to FP64 off the
// FP64 pipe
__device__ __forceinline__ double fix_to_f64_int(long long v, int k) {
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ULL;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll((long long)a);  // 64 for a = 0
    const unsigned long long m = a << (lz & 63);  // leading bit at 63
    const int e = 1086 - lz - k;                  // biased exponent of a 2^-k
    const unsigned long long bits = sgn | ((((unsigned long long)(e - 1)) << 52) + (m >> 11));
    return (a == 0 || e <= 0) ? 0.0 : __longlong_as_double((long long)bits);
}

// round(c w) for doubles c (a charge constant) and w (a weight) whose product's magnitude
// is below 2^61, with integer operations only: the 53-bit mantissas multiplied in 32-bit
// halves, the product's high 64 bits shifted into place and rounded to nearest
__device__ __forceinline__ long long mul_to_fixed(double c, double w) {
    const unsigned long long bc = (unsigned long long)__double_as_longlong(c);
    const unsigned long long bw = (unsigned long long)__double_as_longlong(w);
    const int ec = (int)((bc >> 52) & 0x7FF), ew = (int)((bw >> 52) & 0x7FF);
    if (ec == 0 || ew == 0) return 0;  // zero (or below the fixed point's quantum)
    const unsigned long long mc = (bc & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    const unsigned long long mw = (bw & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    const unsigned ch = (unsigned)(mc >> 32), cl = (unsigned)mc;
    const unsigned wh = (unsigned)(mw >> 32), wl = (unsigned)mw;
    // T = floor(mc mw / 2^42): high-by-high (below 2^42) times 2^22, the cross products
    // shifted by 10, the low-by-low product's high word shifted by 10 (its low word
    // is below 2^-10 of a unit of T)
    const unsigned long long hh = (unsigned long long)ch * wh;
    const unsigned long long cross = (unsigned long long)ch * wl + (unsigned long long)cl * wh +
                                     (unsigned long long)__umulhi(cl, wl);
    const unsigned long long T = (hh << 22) + (cross >> 10);
    // c w = mc mw 2^(ec + ew - 2150) = T 2^(ec + ew - 2108); |c w| < 2^61 keeps the
    // shift at 3 or more; a shift above 64 leaves less than half a unit. The shift by
    // one bit less comes first, then the rounding bit: T is up to 2^64, so adding half
    // a unit before the shift could overflow.
    const int sh = max(2108 - ec - ew, 1);
    if (sh > 64) return 0;
    const long long q = (long long)(((T >> (sh - 1)) + 1ULL) >> 1);
    return ((bc ^ bw) >> 63) ? -q : q;
}

// A 2^62 weight split as S = h 2^31 + l (0 <= l < 2^31; S >= 0, so h >= 0)
struct W31 {
    int h, l;
};
__device__ __forceinline__ W31 w31(long long S) {
    return W31{(int)(S >> 31), (int)(S & 0x7FFFFFFFLL)};
}

// Order-2 gather of one staggered component from the split fixed-point tile (f: first
// tap, BX: row stride): sum_b Sy_b sum_a Sx_a F(a, b) in the component's units 2^-s, to
// within 8 units below. Weights of an axis are non-negative and sum to at most 2^62, so
// each row's products accumulate in one int64 before a single shift: h-by-h products
// below 2^60, the cross products below 2^63 together, the l-by-l ones (under a unit
// each after the shift) left out. Integer multiply-adds only.
__device__ __forceinline__ long long gather9_fix(const int2* __restrict__ f, int BX,
                                                 const W31 sx[3], const W31 sy[3]) {
    long long hh = 0, mid = 0;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const int2* row = f + b * BX;
        long long rh = 0, rm = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int2 v = row[a];  // (l, h)
            rh = mad_wide(sx[a].h, v.y, rh);
            rm = mad_wide(sx[a].l, v.y, mad_wide(sx[a].h, v.x, rm));
        }
        const long long r = rh + (rm >> 31);  // |r| < 2^60: split like a tile entry
        const int rhi = (int)(r >> 31), rlo = (int)(r & 0x7FFFFFFFLL);
        hh = mad_wide(sy[b].h, rhi, hh);
        mid = mad_wide(sy[b].l, rhi, mad_wide(sy[b].h, rlo, mid));
    }
    return hh + (mid >> 31);
}

// Order-2 gather of one staggered component in 3D: three planes gathered as above
// (|plane| < 2^60, split like a tile entry), combined with the z weights the same way; to
// within 12 units below.
__device__ __forceinline__ long long gather27_fix(const int2* __restrict__ f, int BX, int BXY,
                                                  const W31 sx[3], const W31 sy[3],
                                                  const W31 sz[3]) {
    long long hh = 0, mid = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const long long p = gather9_fix(f + c * BXY, BX, sx, sy);
        const int phi = (int)(p >> 31), plo = (int)(p & 0x7FFFFFFFLL);
        hh = mad_wide(sz[c].h, phi, hh);
        mid = mad_wide(sz[c].l, phi, mad_wide(sz[c].h, plo, mid));
    }
    return hh + (mid >> 31);
}

// 2D Esirkepov deposition in fixed point when the particle keeps its nearest nodes on
// both axes: DS lives on stencil nodes 1..3, the running sums have two non-zero
// entries (their sum over the three nodes is zero), 6 + 6 + 9 tile atomics, the three
// rows in a rolled loop (a smaller body: fewer instruction-fetch stalls). Q* are the
// charge factors (tile scale 2^k included) as integers; S0*, S1* old and new shapes.
__device__ __forceinline__ void deposit2d_fast_fix(long long* jx, long long* jy, long long* jz,
                                                   int JX, const long long S0x[3],
                                                   const long long S0y[3], const long long S1x[3],
                                                   const long long S1y[3], long long QX,
                                                   long long QY, long long QZ) {
    long long A[3], B[3], WY[3], WX[3], WZ[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        A[k] = S1x[k] - S0x[k];
        B[k] = S1y[k] - S0y[k];
        WY[k] = S0y[k] + (B[k] >> 1);                     // S0y + DSy/2
        WX[k] = S0x[k] + (A[k] >> 1);                     // S0x + DSx/2
        WZ[k] = (S0y[k] >> 1) + fixmul62(B[k], kThird62);  // S0y/2 + DSy/3
    }
    const long long CX1 = fixmul62(QX, A[0]), CX2 = fixmul62(QX, A[0] + A[1]);
    const long long CY1 = fixmul62(QY, B[0]), CY2 = fixmul62(QY, B[0] + B[1]);
    // rows l = 0..2 (their weights rotating through registers):
    // Wz = S0x (S0y + DSy/2) + DSx (S0y/2 + DSy/3)
    long long wy0 = WY[0], wy1 = WY[1], wy2 = WY[2], wz0 = WZ[0], wz1 = WZ[1], wz2 = WZ[2];
#pragma unroll 1
    for (int l = 0; l < 3; l++) {
        jatomic(jx + l * JX + 0, fixmul62(CX1, wy0));
        jatomic(jx + l * JX + 1, fixmul62(CX2, wy0));
        const long long QWY = fixmul62(QZ, wy0), QWZ = fixmul62(QZ, wz0);
#pragma unroll
        for (int k = 0; k < 3; k++)
            jatomic(jz + l * JX + k, fixmul62(QWY, S0x[k]) + fixmul62(QWZ, A[k]));
        wy0 = wy1, wy1 = wy2, wz0 = wz1, wz1 = wz2;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        jatomic(jy + 0 * JX + k, fixmul62(CY1, WX[k]));
        jatomic(jy + 1 * JX + k, fixmul62(CY2, WX[k]));
    }
}

// Esirkepov data of one axis on a four-node window that always holds both the old and
// the new support (the window starts one node before min(old node, new node)), in 2^62
// fixed point; `start` = window start minus (old node - 2): 0 or 1.
__device__ __forceinline__ void esirkepov_axis4_fix(const long long s0[3], const long long s1[3],
                                                    int shift, Axis4<long long>& a) {
    const bool m = shift < 0, p = shift > 0;
    a.S0[0] = m ? 0 : s0[0];
    a.S0[1] = m ? s0[0] : s0[1];
    a.S0[2] = m ? s0[1] : s0[2];
    a.S0[3] = m ? s0[2] : 0;
    a.DS[0] = (p ? 0 : s1[0]) - a.S0[0];
    a.DS[1] = (p ? s1[0] : s1[1]) - a.S0[1];
    a.DS[2] = (p ? s1[1] : s1[2]) - a.S0[2];
    a.DS[3] = (p ? s1[2] : 0) - a.S0[3];
    a.start = m ? 0 : 1;
}

// General 2D Esirkepov deposition in fixed point (any shift in {-1, 0, 1} per axis) on a
// fixed four-node window per axis: running sums of three entries along each axis (the
// fourth is zero), 12 + 16 + 12 tile atomics, no per-node predicates, and rolled row
// and column loops whose weights rotate through registers (a compact body: the
// cell-crossing path is taken by many warps once a wake forms, and an unrolled body
// stalls them on instruction fetch). `jx/jy/jz` point at stencil node (0, 0) of the
// five-node numbering (old node - 2 on both axes).
__device__ __forceinline__ void deposit2d_general_fix(long long* jx, long long* jy, long long* jz,
                                                      int JX, const long long S0x[3],
                                                      const long long S0y[3],
                                                      const long long S1x[3],
                                                      const long long S1y[3], int sx, int sy,
                                                      long long QX, long long QY, long long QZ) {
    Axis4<long long> ax, ay;
    esirkepov_axis4_fix(S0x, S1x, sx, ax);
    esirkepov_axis4_fix(S0y, S1y, sy, ay);
    const int o = ay.start * JX + ax.start;
    const long long cx1 = fixmul62(QX, ax.DS[0]), cx2 = fixmul62(QX, ax.DS[0] + ax.DS[1]),
                    cx3 = fixmul62(QX, ax.DS[0] + ax.DS[1] + ax.DS[2]);
    const long long cy1 = fixmul62(QY, ay.DS[0]), cy2 = fixmul62(QY, ay.DS[0] + ay.DS[1]),
                    cy3 = fixmul62(QY, ay.DS[0] + ay.DS[1] + ay.DS[2]);
    // per-row weights S0y + DSy/2 and S0y/2 + DSy/3, rotating through registers
    long long wy0 = ay.S0[0] + (ay.DS[0] >> 1), wy1 = ay.S0[1] + (ay.DS[1] >> 1),
              wy2 = ay.S0[2] + (ay.DS[2] >> 1), wy3 = ay.S0[3] + (ay.DS[3] >> 1);
    long long wz0 = ay.S0[0] >> 1, wz1 = ay.S0[1] >> 1, wz2 = ay.S0[2] >> 1, wz3 = ay.S0[3] >> 1;
#pragma unroll 1
    for (int l = 0; l < 4; l++) {
        const long long wz = wz0 + fixmul62(ay.DS[0], kThird62);
        long long* rx = jx + o + l * JX;
        jatomic(rx + 0, fixmul62(cx1, wy0));
        jatomic(rx + 1, fixmul62(cx2, wy0));
        jatomic(rx + 2, fixmul62(cx3, wy0));
        const long long qwy = fixmul62(QZ, wy0), qwz = fixmul62(QZ, wz);
        long long* rz = jz + o + l * JX;
#pragma unroll
        for (int k = 0; k < 4; k++)
            jatomic(rz + k, fixmul62(qwy, ax.S0[k]) + fixmul62(qwz, ax.DS[k]));
        wy0 = wy1, wy1 = wy2, wy2 = wy3;
        wz0 = wz1, wz1 = wz2, wz2 = wz3;
        ay.DS[0] = ay.DS[1], ay.DS[1] = ay.DS[2], ay.DS[2] = ay.DS[3];
    }
    long long wx0 = ax.S0[0] + (ax.DS[0] >> 1), wx1 = ax.S0[1] + (ax.DS[1] >> 1),
              wx2 = ax.S0[2] + (ax.DS[2] >> 1), wx3 = ax.S0[3] + (ax.DS[3] >> 1);
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
        long long* cy = jy + o + k;
        jatomic(cy + 0 * JX, fixmul62(cy1, wx0));
        jatomic(cy + 1 * JX, fixmul62(cy2, wx0));
        jatomic(cy + 2 * JX, fixmul62(cy3, wx0));
        wx0 = wx1, wx1 = wx2, wx2 = wx3;
    }
}

// 3D Esirkepov weights of a node, W_a = DS_a (wa_b S0_c + wb_b DS_c) with
// wa = S0 + DS/2 and wb = S0/2 + DS/3, in 2^62 fixed point per axis
__device__ __forceinline__ void esirkepov_w3(long long S0, long long DS, long long& wa,
                                             long long& wb) {
    wa = S0 + (DS >> 1);
    wb = (S0 >> 1) + fixmul62(DS, kThird62);
}

// 3D deposition in fixed point when no axis changes its nearest node: S0 and DS on
// stencil nodes 1..3 of every axis, two non-zero running-sum entries per line, 54 tile
// adds. jt[a]: stencil node (1, 1, 1) of component a; Q[a]: the charge factors (tile
// scale included) as integers.
__device__ __forceinline__ void deposit3d_fast_fix(long long* const jt[3], int JX, int JXY,
                                                   const long long S0[3][3],
                                                   const long long S1[3][3],
                                                   const long long Q[3]) {
    long long DS[3][3], wa[3][3], wb[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            DS[a][k] = S1[a][k] - S0[a][k];
            esirkepov_w3(S0[a][k], DS[a][k], wa[a][k], wb[a][k]);
        }
    const int st[3] = {1, JX, JXY};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const long long c1 = fixmul62(Q[a], DS[a][0]), c2 = fixmul62(Q[a], DS[a][0] + DS[a][1]);
        // rolled over the c-axis nodes, their weights rotating through registers
        long long s0 = S0[c][0], s1 = S0[c][1], s2 = S0[c][2];
        long long d0 = DS[c][0], d1 = DS[c][1], d2 = DS[c][2];
#pragma unroll 1
        for (int kc = 0; kc < 3; kc++) {
#pragma unroll
            for (int kb = 0; kb < 3; kb++) {
                const long long A = fixmul62(wa[b][kb], s0) + fixmul62(wb[b][kb], d0);
                long long* p = jt[a] + kb * st[b] + kc * st[c];
                jatomic(p, fixmul62(c1, A));
                jatomic(p + st[a], fixmul62(c2, A));
            }
            s0 = s1, s1 = s2, d0 = d1, d1 = d2;
        }
    }
}

// General 3D deposition in fixed point (any shift in {-1, 0, 1} per axis) on a fixed
// four-node window per axis: 3 x 16 x 3 tile adds. j0: stencil node (0, 0, 0) of
// component 0 (old nodes - 2), jvol: the tile volume of one component.
__device__ __forceinline__ void deposit3d_general_fix(long long* j0, int jvol, int JX, int JXY,
                                                      const long long S0[3][3],
                                                      const long long S1[3][3],
                                                      const int sh[3], const long long Q[3]) {
    Axis4<long long> ax[3];
#pragma unroll
    for (int a = 0; a < 3; a++) esirkepov_axis4_fix(S0[a], S1[a], sh[a], ax[a]);
    long long wa[3][4], wb[3][4];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int q = 0; q < 4; q++) esirkepov_w3(ax[a].S0[q], ax[a].DS[q], wa[a][q], wb[a][q]);
    const int st[3] = {1, JX, JXY};
    const int o = ax[2].start * JXY + ax[1].start * JX + ax[0].start;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const long long c1 = fixmul62(Q[a], ax[a].DS[0]);
        const long long c2 = fixmul62(Q[a], ax[a].DS[0] + ax[a].DS[1]);
        const long long c3 = fixmul62(Q[a], ax[a].DS[0] + ax[a].DS[1] + ax[a].DS[2]);
        long long* jt = j0 + a * jvol + o;
        long long s0 = ax[c].S0[0], s1 = ax[c].S0[1], s2 = ax[c].S0[2], s3 = ax[c].S0[3];
        long long d0 = ax[c].DS[0], d1 = ax[c].DS[1], d2 = ax[c].DS[2], d3 = ax[c].DS[3];
#pragma unroll 1
        for (int kc = 0; kc < 4; kc++) {
#pragma unroll
            for (int kb = 0; kb < 4; kb++) {
                const long long A = fixmul62(wa[b][kb], s0) + fixmul62(wb[b][kb], d0);
                long long* p = jt + kb * st[b] + kc * st[c];
                jatomic(p, fixmul62(c1, A));
                jatomic(p + st[a], fixmul62(c2, A));
                jatomic(p + 2 * st[a], fixmul62(c3, A));
            }
            s0 = s1, s1 = s2, s2 = s3, d0 = d1, d1 = d2, d2 = d3;
        }
    }
}

}  // namespace pic
