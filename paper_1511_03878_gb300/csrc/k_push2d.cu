// 2D3V particle kernel: per patch chunk, order-2 interpolation of E and B^n from a
// TMA-staged field tile, relativistic Boris push, Esirkepov deposition into a
// shared-memory current tile, flush of the tile to the global FP64 current with
// atomics, and hand-off of particles that left the patch to the neighbour's
// exchange buffer. Work items come from a device queue (largest first) pulled by
// persistent CTAs, so no CTA idles while dense patches are pushed.
#include <cuda_runtime.h>

#include "fix62.cuh"
#include "pic_device.cuh"
#include "pic_internal.h"

namespace pic {

// Row stride of the 2D current tile, whose rows hold P0 + 5 nodes. The 4-byte (FP32) tile
// is padded to the field tile's stride P0 + 4 modulo the 32 shared-memory banks: a
// particle's scalar field taps (Ez, Bz) and current taps then sit in the same bank
// classes, so the bank interleaving of the particle order spreads the loads and the
// atomics of a warp alike (the float2 pairs put class c on banks 2c and 2c + 1).
template <typename T>
__host__ __device__ constexpr int jrow2d(int P0) {
    return sizeof(typename JType<T>::type) == 4 ? P0 + 4 + 32 : P0 + 5;
}

// Gather of one staggered component: Sx/Sy are the three weights, (tx, ty) the tile
// index of the first tap.
template <typename T>
__device__ __forceinline__ T gather9(const T* __restrict__ f, int BX, const T Sx[3],
                                     const T Sy[3]) {
    T r = T(0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const T* row = f + b * BX;
        r += Sy[b] * (Sx[0] * row[0] + Sx[1] * row[1] + Sx[2] * row[2]);
    }
    return r;
}

// FP32: the same gather for two components that share a stagger, interleaved in the
// tile as float2 (Ex with By, Ey with Bx): one 64-bit shared load per tap serves both.
__device__ __forceinline__ float2 gather9x2(const float2* __restrict__ f, int BX,
                                            const float Sx[3], const float Sy[3]) {
    float rx = 0.0f, ry = 0.0f;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const float2* row = f + b * BX;
        const float2 a0 = row[0], a1 = row[1], a2 = row[2];
        rx += Sy[b] * (Sx[0] * a0.x + Sx[1] * a1.x + Sx[2] * a2.x);
        ry += Sy[b] * (Sx[0] * a0.y + Sx[1] * a1.y + Sx[2] * a2.y);
    }
    return make_float2(rx, ry);
}

// Esirkepov deposition, 2D, when the particle stays on its nearest nodes along both
// axes (the common case): S0 and DS live on the stencil nodes 1..3 only, the running
// sums have two non-zero entries, 6 + 6 + 9 shared-memory atomics.
template <typename T, typename JT>
__device__ __forceinline__ void deposit2d_fast(JT* jx, JT* jy, JT* jz, int JX, const T S0x[3],
                                               const T S0y[3], T dx1, T dy1, T qx, T qy, T qz) {
    T S1x[3], S1y[3], a[3], b[3], wy[3], wz[3], wx[3];
    shape3(dx1, S1x);
    shape3(dy1, S1y);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        a[k] = S1x[k] - S0x[k];
        b[k] = S1y[k] - S0y[k];
        wy[k] = S0y[k] + T(0.5) * b[k];
        wz[k] = T(0.5) * S0y[k] + b[k] * T(1.0 / 3.0);
        wx[k] = S0x[k] + T(0.5) * a[k];
    }
    const T ax1 = qx * a[0], ax2 = qx * (a[0] + a[1]);
    const T by1 = qy * b[0], by2 = qy * (b[0] + b[1]);
    // stencil nodes 1..3 start one tile cell in: pointers already at (1, 1)
    if constexpr (std::is_same<T, df64>::value) {
        // double-word: rolled loops (the unrolled body overflows the instruction
        // cache); per-row weights rotate through registers instead of being indexed
        T wy0 = wy[0], wy1 = wy[1], wy2 = wy[2], wz0 = wz[0], wz1 = wz[1], wz2 = wz[2];
#pragma unroll 1
        for (int l = 0; l < 3; l++) {
            JT* r = jx + l * JX;
            jatomic(r + 0, jprod<JT>(ax1, wy0));
            jatomic(r + 1, jprod<JT>(ax2, wy0));
            JT* rz = jz + l * JX;
#pragma unroll
            for (int k = 0; k < 3; k++)
                jatomic(rz + k, jprod<JT>(qz, S0x[k] * wy0 + a[k] * wz0));
            wy0 = wy1, wy1 = wy2, wz0 = wz1, wz1 = wz2;
        }
        T wx0 = wx[0], wx1 = wx[1], wx2 = wx[2];
#pragma unroll 1
        for (int k = 0; k < 3; k++) {
            jatomic(jy + k, jprod<JT>(by1, wx0));
            jatomic(jy + JX + k, jprod<JT>(by2, wx0));
            wx0 = wx1, wx1 = wx2;
        }
    } else {
#pragma unroll
        for (int l = 0; l < 3; l++) {
            jatomic(jx + l * JX + 0, jprod<JT>(ax1, wy[l]));
            jatomic(jx + l * JX + 1, jprod<JT>(ax2, wy[l]));
            // qz folded into the row weights: one multiply and one FMA per node
            const T qwy = qz * wy[l], qwz = qz * wz[l];
#pragma unroll
            for (int k = 0; k < 3; k++)
                jatomic(jz + l * JX + k, jval<JT>(S0x[k] * qwy + a[k] * qwz));
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            jatomic(jy + 0 * JX + k, jprod<JT>(by1, wx[k]));
            jatomic(jy + 1 * JX + k, jprod<JT>(by2, wx[k]));
        }
    }
}

// General 2D Esirkepov deposition on the five-node stencil with per-node predicates
// (used for FP32, where it needs fewer registers than the four-node window).
template <typename T, typename JT>
__device__ __forceinline__ void deposit2d_general5(JT* jx, JT* jy, JT* jz, int JX, const T S0x[3],
                                                   const T S0y[3], T dx1, T dy1, int sx, int sy,
                                                   T qx, T qy, T qz) {
    Axis5<T> ax, ay;
    esirkepov_axis(S0x, dx1, sx, ax);
    esirkepov_axis(S0y, dy1, sy, ay);
#pragma unroll
    for (int l = 0; l < 5; l++) {
        if (l >= ay.lo && l <= ay.hi) {
            const T wy = ay.S0[l] + T(0.5) * ay.DS[l];
            const T wz = T(0.5) * ay.S0[l] + ay.DS[l] * T(1.0 / 3.0);
            T acc = T(0);
            const int r = l * JX;
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                if (kk >= ax.lo && kk < ax.hi) {
                    acc += ax.DS[kk] * wy;
                    jatomic(jx + r + kk, jprod<JT>(qx, acc));
                }
            }
#pragma unroll
            for (int kk = 0; kk < 5; kk++) {
                if (kk >= ax.lo && kk <= ax.hi) {
                    const T wzk = ax.S0[kk] * wy + ax.DS[kk] * wz;
                    jatomic(jz + r + kk, jprod<JT>(qz, wzk));
                }
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < 5; kk++) {
        if (kk >= ax.lo && kk <= ax.hi) {
            const T wx = ax.S0[kk] + T(0.5) * ax.DS[kk];
            T acc = T(0);
#pragma unroll
            for (int l = 0; l < 4; l++) {
                if (l >= ay.lo && l < ay.hi) {
                    acc += ay.DS[l] * wx;
                    jatomic(jy + l * JX + kk, jprod<JT>(qy, acc));
                }
            }
        }
    }
}

// General 2D Esirkepov deposition (any shift in {-1, 0, 1}) on a fixed four-node
// window per axis: running sums of three entries along each axis, 12 + 12 + 16
// atomics, no per-node predicates. `jx/jy/jz` point at stencil node (0, 0) of the
// five-node numbering (old node - 2 on both axes).
template <typename T, typename JT>
__device__ __forceinline__ void deposit2d_general(JT* jx, JT* jy, JT* jz, int JX, const T S0x[3],
                                                  const T S0y[3], T dx1, T dy1, int sx, int sy,
                                                  T qx, T qy, T qz) {
    Axis4<T> ax, ay;
    esirkepov_axis4(S0x, dx1, sx, ax);
    esirkepov_axis4(S0y, dy1, sy, ay);
    const int o = ay.start * JX + ax.start;
    T wy[4], wz[4], wx[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        wy[k] = ay.S0[k] + T(0.5) * ay.DS[k];
        wz[k] = T(0.5) * ay.S0[k] + ay.DS[k] * T(1.0 / 3.0);
        wx[k] = ax.S0[k] + T(0.5) * ax.DS[k];
    }
    const T cx1 = qx * ax.DS[0], cx2 = qx * (ax.DS[0] + ax.DS[1]),
            cx3 = qx * (ax.DS[0] + ax.DS[1] + ax.DS[2]);
    const T cy1 = qy * ay.DS[0], cy2 = qy * (ay.DS[0] + ay.DS[1]),
            cy3 = qy * (ay.DS[0] + ay.DS[1] + ay.DS[2]);
    // rolled loops, the per-row (per-column) weights rotating through registers
    T wy0 = wy[0], wy1 = wy[1], wy2 = wy[2], wy3 = wy[3];
    T wz0 = wz[0], wz1 = wz[1], wz2 = wz[2], wz3 = wz[3];
#pragma unroll 1
    for (int l = 0; l < 4; l++) {
        JT* rx = jx + o + l * JX;
        jatomic(rx + 0, jprod<JT>(cx1, wy0));
        jatomic(rx + 1, jprod<JT>(cx2, wy0));
        jatomic(rx + 2, jprod<JT>(cx3, wy0));
        JT* rz = jz + o + l * JX;
#pragma unroll
        for (int k = 0; k < 4; k++)
            jatomic(rz + k, jprod<JT>(qz, ax.S0[k] * wy0 + ax.DS[k] * wz0));
        wy0 = wy1, wy1 = wy2, wy2 = wy3, wz0 = wz1, wz1 = wz2, wz2 = wz3;
    }
    T wx0 = wx[0], wx1 = wx[1], wx2 = wx[2], wx3 = wx[3];
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
        JT* cy = jy + o + k;
        jatomic(cy + 0 * JX, jprod<JT>(cy1, wx0));
        jatomic(cy + 1 * JX, jprod<JT>(cy2, wx0));
        jatomic(cy + 2 * JX, jprod<JT>(cy3, wx0));
        wx0 = wx1, wx1 = wx2, wx2 = wx3;
    }
}

// double-word gather: compensated dot products (rows along x, then along y)
__device__ __forceinline__ df64 gather9(const df64* __restrict__ f, int BX, const df64 Sx[3],
                                       const df64 Sy[3]) {
    Dot2 outer;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const df64* row = f + b * BX;
        Dot2 inner;
        inner.add(Sx[0], row[0]);
        inner.add(Sx[1], row[1]);
        inner.add(Sx[2], row[2]);
        outer.add(Sy[b], inner.result());
    }
    return outer.result();
}

// CTA shape of the particle kernel per precision: threads per CTA and the CTAs per SM
// the register budget is sized for
#ifndef PIC_DF64_THREADS
#define PIC_DF64_THREADS 256
#endif
#ifndef PIC_DF64_MINB
#define PIC_DF64_MINB 2
#endif
#ifndef PIC_F64_THREADS
#define PIC_F64_THREADS 256
#endif
#ifndef PIC_F64_MINB
#define PIC_F64_MINB 2
#endif
#ifndef PIC_F32_MINB
#define PIC_F32_MINB 3
#endif
template <typename T>
struct Push2DShape {
    static constexpr int threads = PIC_F64_THREADS, min_blocks = PIC_F64_MINB;
};
template <>
struct Push2DShape<float> {
    static constexpr int threads = kThreads, min_blocks = PIC_F32_MINB;
};
template <>
struct Push2DShape<df64> {
    static constexpr int threads = PIC_DF64_THREADS, min_blocks = PIC_DF64_MINB;
};

// copy of a leaving particle's state (already stored in its slot) to arrival slot m
template <typename T>
__device__ __forceinline__ void handoff_copy(const SimDev& S, int slot, int m, int pid) {
    if constexpr (uses_cell<T>()) S.mcell[m] = S.cell[slot];
#pragma unroll
    for (int a = 0; a < 2; a++)
        reinterpret_cast<T*>(S.mxi[a])[m] = reinterpret_cast<const T*>(S.xi[a])[slot];
#pragma unroll
    for (int a = 0; a < 3; a++)
        reinterpret_cast<T*>(S.mu[a])[m] = reinterpret_cast<const T*>(S.u[a])[slot];
    reinterpret_cast<T*>(S.mw)[m] = reinterpret_cast<const T*>(S.w)[slot];
    S.mid[m] = pid;
}

template <typename T>
__global__ void __launch_bounds__(Push2DShape<T>::threads, Push2DShape<T>::min_blocks)
    push2d_kernel(const BatchDev* __restrict__ bd, int static_map) {
    using JT = typename JType<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int s_item;
    // particles of the current item that leave its patch: their slot and destination
    // (-1: deleted), handed off after the item so that the particle loop makes no
    // global round trip for them
    __shared__ int s_lv_n;
    __shared__ int s_lv_slot[kLeaveList];
    __shared__ int s_lv_dest[kLeaveList];
    // FP64: largest exponent field of each component of the staged field tile, which
    // holds the fields in split fixed point (see fix_field_tile)
    __shared__ int s_femax[6];

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&mbar, 1);
        fence_mbar_init();
        s_lv_n = 0;
    }
    __syncthreads();

    uint32_t phase = 0;
    int loaded_sim = -1, loaded_patch = -1, loaded_gen = -1;
    int next_static = blockIdx.x;

    for (;;) {
        __syncthreads();  // the previous item's tiles are no longer read
        if (tid == 0) s_item = static_map ? next_static : atomicAdd(bd->head, 1);
        next_static += gridDim.x;
        __syncthreads();
        const int it = s_item;
        if (it >= *bd->nitems || it >= bd->max_items) break;
        const int4 item = bd->items[it];
        const SimDev& S = bd->sims[item.x];
        const int patch = item.y;

        const int P0 = S.P[0], P1 = S.P[1];
        const int BX = S.BX, BY = S.BY;
        const int JX = jrow2d<T>(P0), JY = P1 + 5, JW = P0 + 5;  // stride, rows, row width
        const int nx = S.n[0], ny = S.n[1];
        const int NX = S.NX;
        const int px0 = (patch % S.np[0]) * P0;
        const int py0 = (patch / S.np[0]) * P1;
        const int gen = S.st->gen;
        const int shift = S.st->shift;
        const int window = S.window;

        T* Ft = reinterpret_cast<T*>(smem);
        const int fbytes = 6 * BX * BY * (int)sizeof(T);
        JT* Jt = reinterpret_cast<JT*>(smem + ((fbytes + 127) & ~127));
        const int jplane = JX * JY;

        // FP32 stages the six planes in the current tile's space, which is zeroed after
        // they are interleaved into the field tile
        constexpr bool kPaired = std::is_same<T, float>::value;
        auto zero_j = [&] {
            for (int e = tid; e < 3 * JY * JW; e += blockDim.x) {
                const int r = e / JW;  // component * JY + row
                Jt[r * JX + (e - r * JW)] = JT(0);
            }
        };
        if constexpr (!kPaired) zero_j();

        if (item.x != loaded_sim || patch != loaded_patch || gen != loaded_gen) {
            if constexpr (std::is_same<T, double>::value) {
                if (tid < 6) s_femax[tid] = 0;
            }
            if constexpr (kPaired) {
                // the previous item's atomics into the staging space come before the copy
                fence_proxy_async_smem();
                __syncthreads();
            }
            if (tid == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar, (uint32_t)fbytes);
                // box origin: interior index (px0 - 1, py0 - 1) = padded (px0, py0)
                tma_load_3d(kPaired ? reinterpret_cast<void*>(Jt) : reinterpret_cast<void*>(Ft),
                            S.tmap + gen, &mbar, px0 - 1 + kGuard, py0 - 1 + kGuard, 0);
            }
            const bool ok = mbar_wait_bounded(&mbar, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(S.status, ST_TIMEOUT);
                return;
            }
            if constexpr (std::is_same<T, double>::value)
                fix_field_tile(reinterpret_cast<double*>(Ft), BX * BY, s_femax);
            if constexpr (kPaired) {
                // planes Ex Ey Ez Bx By Bz -> (Ex, By) pairs, (Ey, Bx) pairs, Ez, Bz
                const int pl = BX * BY;
                const float* St = reinterpret_cast<const float*>(Jt);
                float2* FA = reinterpret_cast<float2*>(Ft);
                for (int i = tid; i < pl; i += blockDim.x) {
                    FA[i] = make_float2(St[i], St[4 * pl + i]);
                    FA[pl + i] = make_float2(St[pl + i], St[3 * pl + i]);
                    Ft[4 * pl + i] = St[2 * pl + i];
                    Ft[5 * pl + i] = St[5 * pl + i];
                }
                __syncthreads();
            }
            loaded_sim = item.x;
            loaded_patch = patch;
            loaded_gen = gen;
        }
        if constexpr (kPaired) zero_j();
        __syncthreads();  // J tile zeroed (FP64: field tile converted)

        // per-sim constants in the working precision (precomputed on the host)
        T dtdx, dtdy, eps, cjx, cjy, cjz;
        if constexpr (is_f64<T>::value) {
            dtdx = S.c_dtd[0], dtdy = S.c_dtd[1], eps = S.c_eps;
            cjx = S.c_j[0], cjy = S.c_j[1], cjz = S.c_j[2];
        } else if constexpr (std::is_same<T, float>::value) {
            dtdx = S.f_dtd[0], dtdy = S.f_dtd[1], eps = S.f_eps;
            cjx = S.f_j[0], cjy = S.f_j[1], cjz = S.f_j[2];
        } else {
            dtdx = T(S.c_dtd[0]), dtdy = T(S.c_dtd[1]), eps = T(S.c_eps);
            cjx = T(S.c_j[0]), cjy = T(S.c_j[1]), cjz = T(S.c_j[2]);
        }

        const int pb = S.pbase[patch];
        const int base = pb + item.z;
        const int cnt = item.w;
        // fixed-point exponent of the double-word current tile for this item
        const int jk = item_fixed_exp<JT>(cnt, S.cmax_exp);
        const float jsc = pow2f(jk);
        // charge factors carrying the tile's power-of-two scale (exact: the same values as
        // scaling each particle's product)
        const T cjxs = jscale<JT>(cjx, jsc), cjys = jscale<JT>(cjy, jsc),
                cjzs = jscale<JT>(cjz, jsc);
        const T* W = reinterpret_cast<const T*>(S.w);
        T* U0 = reinterpret_cast<T*>(S.u[0]);
        T* U1 = reinterpret_cast<T*>(S.u[1]);
        T* U2 = reinterpret_cast<T*>(S.u[2]);

        // raw particle state of the next iteration, loaded one iteration ahead so the
        // global-memory latency overlaps the current particle's arithmetic
        double nx0 = 0.0, ny0 = 0.0;  // FP64 positions
        int nc = 0;                   // FP32 packed cell
        T nfx = T(0), nfy = T(0), nu0 = T(0), nu1 = T(0), nu2 = T(0), nw = T(0);
        auto fetch = [&](int kk) {
            const int sl = base + kk;
            if constexpr (is_f64<T>::value) {
                nx0 = reinterpret_cast<const double*>(S.xi[0])[sl];
                ny0 = reinterpret_cast<const double*>(S.xi[1])[sl];
            } else {
                nc = S.cell[sl];
                nfx = reinterpret_cast<const T*>(S.xi[0])[sl];
                nfy = reinterpret_cast<const T*>(S.xi[1])[sl];
            }
            nu0 = U0[sl];
            nu1 = U1[sl];
            nu2 = U2[sl];
            nw = W[sl];
        };
        if (tid < cnt) fetch(tid);

        for (int k0 = 0; k0 < cnt; k0 += blockDim.x) {
            const int k = k0 + tid;
            const bool valid = k < cnt;
            const int slot = base + (valid ? k : 0);

            bool ok = false, leave = false;
            int dest = patch;
            if constexpr (std::is_same<T, double>::value) {
                // ---- FP64: in-cell offsets, shapes, the field gather, the charge factors and
                // every deposit weight, running sum and tap product in 2^62 fixed point
                // (integer units, 32 times the FP64 rate on this GPU); Boris and the move in
                // FP64. A field tile holding a non-finite value cannot be converted: its
                // particles are reported and dropped like non-finite particles.
                const bool ftile_ok = s_femax[0] < 0x7FF && s_femax[1] < 0x7FF &&
                                      s_femax[2] < 0x7FF && s_femax[3] < 0x7FF &&
                                      s_femax[4] < 0x7FF && s_femax[5] < 0x7FF;
                const double xi0 = nx0, eta0 = ny0;
                double u[3] = {nu0, nu1, nu2};
                const double w = nw;
                int ix = 0, iy = 0;
                long long FX = 0, FY = 0;
                if (valid) {
                    split62(xi0, ix, FX);
                    split62(eta0, iy, FY);
                }
                // primal node = ix + (f >= 1/2), dual node = ix
                const bool hx = FX >= kHalf62, hy = FY >= kHalf62;
                const int nxp = ix + (hx ? 1 : 0), nyp = iy + (hy ? 1 : 0);
                const int txp = nxp - px0, txd = ix - px0;
                const int typ = nyp - py0, tyd = iy - py0;
                ok = valid && ftile_ok && (unsigned)txp <= (unsigned)P0 &&
                     (unsigned)typ <= (unsigned)P1 && (unsigned)txd < (unsigned)P0 &&
                     (unsigned)tyd < (unsigned)P1;
                long long SXP[3], SYP[3], S1X[3], S1Y[3];
                int sx = 0, sy = 0, ix1 = 0, iy1 = 0;
                double xi1 = 0.0, eta1 = 0.0, vz = 0.0;
                if (ok) {
                    long long SXD[3], SYD[3];
                    shape62(hx ? FX - kOne62 : FX, SXP);
                    shape62(hy ? FY - kOne62 : FY, SYP);
                    shape62(FX - kHalf62, SXD);
                    shape62(FY - kHalf62, SYD);
                    const int pl = BX * BY;
                    // the gather on the integer units, from the fixed-point field tile
                    const int2* Fi = reinterpret_cast<const int2*>(Ft);
                    double E[3], B[3];
                    W31 Sxp[3], Syp[3], Sxd[3], Syd[3];
#pragma unroll
                    for (int k2 = 0; k2 < 3; k2++) {
                        Sxp[k2] = w31(SXP[k2]);
                        Syp[k2] = w31(SYP[k2]);
                        Sxd[k2] = w31(SXD[k2]);
                        Syd[k2] = w31(SYD[k2]);
                    }
                    {
                        // one rolled loop over Ex Ey Ez Bx By Bz: x primal for Ey Ez Bx, y
                        // primal for Ex Ez By; results rotate through six registers
                        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0, r5 = 0.0;
#pragma unroll 1
                        for (int c = 0; c < 6; c++) {
                            const bool xp = c >= 1 && c <= 3, yp = (c & 1) == 0;
                            W31 gx[3], gy[3];
#pragma unroll
                            for (int k2 = 0; k2 < 3; k2++) {
                                gx[k2] = xp ? Sxp[k2] : Sxd[k2];
                                gy[k2] = yp ? Syp[k2] : Syd[k2];
                            }
                            const long long v = gather9_fix(
                                Fi + c * pl + (yp ? typ : tyd) * BX + (xp ? txp : txd), BX, gx, gy);
                            r0 = r1, r1 = r2, r2 = r3, r3 = r4, r4 = r5;
                            r5 = fix_to_f64_int(v, fix_field_exp(s_femax[c]));
                        }
                        E[0] = r0, E[1] = r1, E[2] = r2, B[0] = r3, B[1] = r4, B[2] = r5;
                    }
                    const double ig = boris(eps, E, B, u);
                    vz = u[2] * ig;
                    xi1 = xi0 + dtdx * (u[0] * ig);
                    eta1 = eta0 + dtdy * (u[1] * ig);
                    long long FX1, FY1;
                    split62(xi1, ix1, FX1);
                    split62(eta1, iy1, FY1);
                    const bool h1x = FX1 >= kHalf62, h1y = FY1 >= kHalf62;
                    shape62(h1x ? FX1 - kOne62 : FX1, S1X);
                    shape62(h1y ? FY1 - kOne62 : FY1, S1Y);
                    sx = ix1 + (h1x ? 1 : 0) - nxp;
                    sy = iy1 + (h1y ? 1 : 0) - nyp;
                    ok = (sx >= -1 && sx <= 1 && sy >= -1 && sy <= 1);
                }
                long long QX = 0, QY = 0, QZ = 0;
                if (ok) {
                    // charge factors (carrying the tile's 2^k) as integers, formed on the
                    // integer units: q w d_a/dt for Jx, Jy and q w v_z for Jz
                    QX = mul_to_fixed(cjxs, w);
                    QY = mul_to_fixed(cjys, w);
                    QZ = fixmul62(mul_to_fixed(cjzs, w), f64_to_fixed_shift(vz, 62));
                    // ---- boundaries, destination patch (decisions on the integer floors) and
                    // the new state, stored before the deposit so that only the shapes and
                    // charge factors stay live through it
                    bool del = false;
                    double xs = xi1;
                    if (window) {
                        del = ix1 < 0 || ix1 >= nx || ix1 - shift < 0;
                        if (shift) xs = xi1 - 1.0;
                        ix1 -= shift;
                    } else {
                        if (ix1 < 0) {
                            xs = xi1 + (double)nx;
                            ix1 += nx;
                        } else if (ix1 >= nx) {
                            xs = xi1 - (double)nx;
                            ix1 -= nx;
                        }
                    }
                    if (iy1 < 0) {
                        eta1 += (double)ny;
                        iy1 += ny;
                    } else if (iy1 >= ny) {
                        eta1 -= (double)ny;
                        iy1 -= ny;
                    }
                    if (!del) {
                        // a wrap or shift by whole cells keeps the floor: recheck it on the
                        // stored double (a position just below a wrap can round onto it)
                        ix1 = floor_to_int(xs);
                        iy1 = floor_to_int(eta1);
                        if (!window && ix1 >= nx) { xs -= (double)nx; ix1 -= nx; }
                        if (iy1 >= ny) { eta1 -= (double)ny; iy1 -= ny; }
                        dest = ix1 / P0 + S.np[0] * (iy1 / P1);
                        leave = dest != patch;
                        reinterpret_cast<double*>(S.xi[0])[slot] = xs;
                        reinterpret_cast<double*>(S.xi[1])[slot] = eta1;
                        U0[slot] = u[0];
                        U1[slot] = u[1];
                        U2[slot] = u[2];
                    } else {
                        dest = -1;
                        leave = true;
                    }
                }
                // the next particle's state loads while this one deposits
                if (k + (int)blockDim.x < cnt) fetch(k + blockDim.x);
                const bool fast = __all_sync(0xffffffffu, !ok || (sx == 0 && sy == 0));
                if (ok) {
                    const int t0 = typ * JX + txp;  // stencil node 0 of both axes
                    if (fast) {
                        const int t1 = t0 + JX + 1;  // stencil nodes (1, 1)
                        deposit2d_fast_fix(Jt + t1, Jt + jplane + t1, Jt + 2 * jplane + t1, JX,
                                           SXP, SYP, S1X, S1Y, QX, QY, QZ);
                    } else {
                        deposit2d_general_fix(Jt + t0, Jt + jplane + t0, Jt + 2 * jplane + t0, JX,
                                              SXP, SYP, S1X, S1Y, sx, sy, QX, QY, QZ);
                    }
                }
            } else {
                // ---- FP32 and double-word: cell index + offset in [0, 1)
                // ---- A. take the prefetched state, start loading the next one
                int ix = 0, iy = 0;
                T fx = T(0), fy = T(0);
                T u[3] = {nu0, nu1, nu2};
                T w = nw;
                if (valid) {
                    ix = nc & 0xFFFF;
                    iy = (nc >> 16) & 0xFFFF;
                    fx = nfx;
                    fy = nfy;
                }
                if (k + (int)blockDim.x < cnt) fetch(k + blockDim.x);
                // nodes and deltas: primal node = ix + (f >= 1/2), dual node = ix
                const bool hx = fx >= T(0.5), hy = fy >= T(0.5);
                const int nxp = ix + (hx ? 1 : 0), nyp = iy + (hy ? 1 : 0);
                const T dxp = hx ? fx - T(1) : fx, dyp = hy ? fy - T(1) : fy;
                const T dxd = fx - T(0.5), dyd = fy - T(0.5);
                // tile-local first-tap indices (field tile origin at px0 - 1, py0 - 1)
                const int txp = nxp - px0, txd = ix - px0;
                const int typ = nyp - py0, tyd = iy - py0;
                ok = valid && (unsigned)txp <= (unsigned)P0 && (unsigned)typ <= (unsigned)P1 &&
                     (unsigned)txd < (unsigned)P0 && (unsigned)tyd < (unsigned)P1;

                // ---- B. interpolate, push, move
                T Sxp[3], Syp[3];
                T dxp1 = T(0), dyp1 = T(0), fx1 = T(0), fy1 = T(0), vz = T(0);
                int sx = 0, sy = 0, ix1 = 0, iy1 = 0;
                if (ok) {
                    T Sxd[3], Syd[3];
                    shape3(dxp, Sxp);
                    shape3(dxd, Sxd);
                    shape3(dyp, Syp);
                    shape3(dyd, Syd);
                    const int pl = BX * BY;
                    T E[3], B[3];
                    if constexpr (std::is_same<T, df64>::value) {
                        // one rolled loop over Ex Ey Ez Bx By Bz: x primal for Ey Ez Bx,
                        // y primal for Ex Ez By; results rotate through six registers
                        T r0(0.0f), r1(0.0f), r2(0.0f), r3(0.0f), r4(0.0f), r5(0.0f);
#pragma unroll 1
                        for (int c = 0; c < 6; c++) {
                            const bool xp = c >= 1 && c <= 3, yp = (c & 1) == 0;
                            T sx[3], sy[3];
#pragma unroll
                            for (int k = 0; k < 3; k++) {
                                sx[k] = xp ? Sxp[k] : Sxd[k];
                                sy[k] = yp ? Syp[k] : Syd[k];
                            }
                            const T g = gather9(Ft + c * pl + (yp ? typ : tyd) * BX + (xp ? txp : txd),
                                                BX, sx, sy);
                            r0 = r1, r1 = r2, r2 = r3, r3 = r4, r4 = r5, r5 = g;
                        }
                        E[0] = r0, E[1] = r1, E[2] = r2, B[0] = r3, B[1] = r4, B[2] = r5;
                    } else {
                        const float2* FA = reinterpret_cast<const float2*>(Ft);
                        const float2 exby = gather9x2(FA + typ * BX + txd, BX, Sxd, Syp);
                        const float2 eybx = gather9x2(FA + pl + tyd * BX + txp, BX, Sxp, Syd);
                        E[0] = exby.x, B[1] = exby.y, E[1] = eybx.x, B[0] = eybx.y;
                        E[2] = gather9(Ft + 4 * pl + typ * BX + txp, BX, Sxp, Syp);
                        B[2] = gather9(Ft + 5 * pl + tyd * BX + txd, BX, Sxd, Syd);
                    }

                    const T ig = boris(eps, E, B, u);
                    const T vx = u[0] * ig, vy = u[1] * ig;
                    vz = u[2] * ig;
                    int nxp1, nyp1;
                    {
                        fx1 = fx + dtdx * vx;
                        fy1 = fy + dtdy * vy;
                        ix1 = ix;
                        iy1 = iy;
                        if (fx1 < T(0)) {
                            fx1 += T(1);
                            ix1 -= 1;
                            if (fx1 >= T(1)) { fx1 = T(0); ix1 += 1; }
                        } else if (fx1 >= T(1)) {
                            fx1 -= T(1);
                            ix1 += 1;
                        }
                        if (fy1 < T(0)) {
                            fy1 += T(1);
                            iy1 -= 1;
                            if (fy1 >= T(1)) { fy1 = T(0); iy1 += 1; }
                        } else if (fy1 >= T(1)) {
                            fy1 -= T(1);
                            iy1 += 1;
                        }
                        const bool h1x = fx1 >= T(0.5), h1y = fy1 >= T(0.5);
                        nxp1 = ix1 + (h1x ? 1 : 0);
                        nyp1 = iy1 + (h1y ? 1 : 0);
                        dxp1 = h1x ? fx1 - T(1) : fx1;
                        dyp1 = h1y ? fy1 - T(1) : fy1;
                    }
                    sx = nxp1 - nxp;
                    sy = nyp1 - nyp;
                    ok = (sx >= -1 && sx <= 1 && sy >= -1 && sy <= 1);
                }

                // ---- C. Esirkepov deposition into the shared tile (origin px0-2, py0-2);
                // warp-uniform choice of the no-crossing fast path
                const bool fast = __all_sync(0xffffffffu, !ok || (sx == 0 && sy == 0));
                if (ok) {
                    const T qx = cjxs * w, qy = cjys * w, qz = cjzs * w * vz;
                    const int t0 = typ * JX + txp;  // stencil node 0 of both axes
                    if (fast) {
                        const int t1 = t0 + JX + 1;  // stencil nodes (1, 1)
                        deposit2d_fast<T, JT>(Jt + t1, Jt + jplane + t1, Jt + 2 * jplane + t1, JX, Sxp,
                                              Syp, dxp1, dyp1, qx, qy, qz);
                    } else {
                        if constexpr (std::is_same<T, df64>::value)
                            deposit2d_general<T, JT>(Jt + t0, Jt + jplane + t0, Jt + 2 * jplane + t0,
                                                     JX, Sxp, Syp, dxp1, dyp1, sx, sy, qx, qy, qz);
                        else
                            deposit2d_general5<T, JT>(Jt + t0, Jt + jplane + t0, Jt + 2 * jplane + t0,
                                                      JX, Sxp, Syp, dxp1, dyp1, sx, sy, qx, qy, qz);
                    }

                    // ---- D. boundaries and destination patch
                    bool del = false;
                    if (window) {
                        del = ix1 < 0 || ix1 >= nx;
                        ix1 -= shift;
                        del = del || ix1 < 0;
                    } else {
                        ix1 = wrapi(ix1, nx);
                    }
                    iy1 = wrapi(iy1, ny);
                    if (!del) {
                        dest = ix1 / P0 + S.np[0] * (iy1 / P1);
                        leave = dest != patch;
                        // the new state goes to the particle's own slot, also when it leaves:
                        // the hand-off after the item copies it from there
                        S.cell[slot] = ix1 | (iy1 << 16);
                        reinterpret_cast<T*>(S.xi[0])[slot] = fx1;
                        reinterpret_cast<T*>(S.xi[1])[slot] = fy1;
                        U0[slot] = u[0];
                        U1[slot] = u[1];
                        U2[slot] = u[2];
                    } else {
                        dest = -1;
                        leave = true;
                    }
                }
            }
            if (valid && !ok) {
                // corrupted or non-finite particle: report and drop it
                atomicOr(S.status, ST_NUMERIC);
                leave = true;
                dest = -1;
            }

            // ---- E. exchange hand-off. A leaver is listed in shared memory; only when the
            // list is full does it claim its slots here (warp-aggregated global counters)
            const bool lv = valid && leave;
            bool over = false;
            if (lv) {
                const int li = atomicAdd(&s_lv_n, 1);
                if (li < kLeaveList) {
                    s_lv_slot[li] = slot;
                    s_lv_dest[li] = dest;
                } else {
                    over = true;
                }
            }
            if (__any_sync(0xffffffffu, over)) {
                const bool send = over && dest >= 0;
                int pid = 0, mcap = 0, mb = 0;
                if (over) pid = S.id[slot];
                if (send) {
                    mcap = S.mcap[dest];
                    mb = S.mbase[dest];
                }
                const int2 cl = warp_claim2(S.hcount, patch, over, S.mcount, send ? dest : 0, send);
                if (over) {
                    S.holes[pb + cl.x] = slot;
                    S.id[slot] = -1;
                    if (send) {
                        if (cl.y < mcap)
                            handoff_copy<T>(S, slot, mb + cl.y, pid);
                        else
                            atomicOr(S.status, ST_MAILBOX);
                    }
                }
            }
        }
        __syncthreads();

        // ---- hand-off of the listed leavers: their holes and arrival slots are claimed
        // a warp at a time, and each is copied from its slot to its destination's buffer
        {
            const int nl = s_lv_n < kLeaveList ? s_lv_n : kLeaveList;
            for (int b0 = 0; b0 < nl; b0 += blockDim.x) {  // same trip count in every warp
                const int t = b0 + tid;
                const bool lv = t < nl;
                int slot = 0, dest = -1;
                if (lv) {
                    slot = s_lv_slot[t];
                    dest = s_lv_dest[t];
                }
                const bool send = lv && dest >= 0;
                int pid = 0, mcap = 0, mb = 0;
                if (lv) pid = S.id[slot];
                if (send) {
                    mcap = S.mcap[dest];
                    mb = S.mbase[dest];
                }
                const int2 cl = warp_claim2(S.hcount, patch, lv, S.mcount, send ? dest : 0, send);
                if (lv) {
                    S.holes[pb + cl.x] = slot;
                    if (send) {
                        if (cl.y < mcap)
                            handoff_copy<T>(S, slot, mb + cl.y, pid);
                        else
                            atomicOr(S.status, ST_MAILBOX);
                    }
                    S.id[slot] = -1;
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_lv_n = 0;  // every thread has read it; the next item's appends
                                   // come after its own barriers

        // ---- flush the current tile (origin px0-2, py0-2) into the global FP64 J
        double* Jg = S.J[gen];
        const long long fs = S.fstride;
        for (int e = tid; e < 3 * JY * JW; e += blockDim.x) {
            const int rr = e / JW, tx = e - rr * JW;  // rr = component * JY + row
            const int comp = rr / JY, ty = rr - comp * JY;
            const JT v = Jt[rr * JX + tx];
            if (v == JT(0)) continue;
            int gi = px0 - 2 + tx, gj = py0 - 2 + ty;
            if (window) {
                if (gi < 0 || gi >= nx) continue;
            } else {
                gi = wrapi(gi, nx);
            }
            gj = wrapi(gj, ny);
            atomicAdd(Jg + comp * fs + (long long)(gj + kGuard) * NX + (gi + kGuard), jflush(v, jk));
        }
    }
}

template <typename T>
static int smem_bytes_2d(int P0, int P1) {
    const int BX = ((P0 + 3) + 3) & ~3, BY = P1 + 3;
    const int fb = 6 * BX * BY * (int)sizeof(T);
    int jb = 3 * jrow2d<T>(P0) * (P1 + 5) * (int)sizeof(typename JType<T>::type);
    if (std::is_same<T, float>::value && jb < fb) jb = fb;  // FP32 stages the field tile there
    return ((fb + 127) & ~127) + jb;
}

template <typename T>
static int occupancy_2d(int P0, int P1, int* smem_bytes) {
    const int sb = smem_bytes_2d<T>(P0, P1);
    *smem_bytes = sb;
    int blocks = 0;
    if (cudaFuncSetAttribute(push2d_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb) !=
        cudaSuccess)
        return 0;
    cudaFuncSetAttribute(push2d_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, push2d_kernel<T>,
                                                      Push2DShape<T>::threads, sb) !=
        cudaSuccess)
        return 0;
    return blocks;
}

int push2d_smem(int prec, int P0, int P1) {
    int sb = 0;
    PIC_DISPATCH(prec, (sb = smem_bytes_2d<T>(P0, P1)));
    return sb;
}

int push_occupancy(int dims, int prec, int P0, int P1, int P2, int* smem_bytes) {
    if (dims == 3) return push3d_occupancy(prec, P0, P1, P2, smem_bytes);
    if (dims != 2) return 0;
    int blocks = 0;
    PIC_DISPATCH(prec, (blocks = occupancy_2d<T>(P0, P1, smem_bytes)));
    return blocks;
}

cudaError_t launch_push(const BatchDev* bd_dev, int dims, int prec, int mapping, int P0,
                        int P1, int P2, int grid, cudaStream_t s) {
    if (dims == 3) return launch_push3d(bd_dev, prec, mapping, P0, P1, P2, grid, s);
    if (dims != 2) return cudaErrorInvalidValue;
    const int static_map = mapping == 1;
    PIC_DISPATCH(prec, (push2d_kernel<T><<<grid, Push2DShape<T>::threads, smem_bytes_2d<T>(P0, P1), s>>>(
                            bd_dev, static_map)));
    return cudaGetLastError();
}

}  // namespace pic
