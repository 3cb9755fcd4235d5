// 3D3V particle kernel: the 2D kernel's structure with a 4D TMA box (x, y, z,
// component), 27-tap order-2 interpolation and the 3D Esirkepov weights
//   W_a = DS_a ((S0_b + DS_b/2) S0_c + (S0_b/2 + DS_b/3) DS_c),
// J_a the running sum of -(q w/dV)(d_a/dt) W_a along +a. y and z are periodic; x is
// periodic or a moving window (particles leaving [0, nx) are absorbed, the shift is
// applied in the particle store, contributions outside the window are dropped).
// FP32 cells pack (ix | iy << 11 | iz << 22). The FP64 kernel runs everything but the Boris
// push and the move in 2^62 fixed point on the integer units, as the 2D one does
// (fix62.cuh): offsets, shapes, the 27-tap gather from a fixed-point copy of the field
// tile, the charge factors, the Esirkepov weights and products.
#include <cuda_runtime.h>

#include "fix62.cuh"
#include "pic_device.cuh"
#include "pic_internal.h"

namespace pic {

// 3D kernels exist in FP64 and FP32; the double-word precision is 2D only (in 3D it
// measured no faster than FP64: 6.19e8 against 6.51e8 pushes/s on the 3D LWFA window,
// at 255 registers and one CTA per SM). Other codes run nothing.
#define PIC_DISPATCH_3D(prec, body) \
    do {                            \
        if ((prec) == 0) {          \
            using T = double;       \
            body;                   \
        } else if ((prec) == 1) {   \
            using T = float;        \
            body;                   \
        }                           \
    } while (0)


template <typename T>
__device__ __forceinline__ T gather27(const T* __restrict__ f, int BX, int BXY, const T Sx[3],
                                      const T Sy[3], const T Sz[3]) {
    T r = T(0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        T plane = T(0);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const T* row = f + c * BXY + b * BX;
            plane += Sy[b] * (Sx[0] * row[0] + Sx[1] * row[1] + Sx[2] * row[2]);
        }
        r += Sz[c] * plane;
    }
    return r;
}

// FP32 particle state: the packed cell and the offsets in it (the FP64 kernel reads its
// positions directly)
template <typename T>
__device__ __forceinline__ void split_pos(const SimDev& S, int slot, int i[3], T f[3]) {
    const int c = S.cell[slot];
    i[0] = c & 0x7FF;
    i[1] = (c >> 11) & 0x7FF;
    i[2] = (c >> 22) & 0x3FF;
#pragma unroll
    for (int a = 0; a < 3; a++) f[a] = reinterpret_cast<const T*>(S.xi[a])[slot];
}

// 3D deposition when no axis changes its nearest node: S0 and DS live on stencil
// nodes 1..3 of every axis, each running sum has two non-zero entries (54 atomics).
// `jt[a]` point at stencil node (1, 1, 1) of component a.
template <typename T, typename JT>
__device__ __forceinline__ void deposit3d_fast(JT* const jt[3], int JX, int JXY, const T S0[3][3],
                                               const T d1[3], const T q[3]) {
    T DS[3][3], wa[3][3], wb[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T S1[3];
        shape3(d1[a], S1);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            DS[a][k] = S1[k] - S0[a][k];
            wa[a][k] = S0[a][k] + T(0.5) * DS[a][k];
            wb[a][k] = T(0.5) * S0[a][k] + DS[a][k] * T(1.0 / 3.0);
        }
    }
    const int st[3] = {1, JX, JXY};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const T c1 = q[a] * DS[a][0], c2 = q[a] * (DS[a][0] + DS[a][1]);
#pragma unroll
        for (int kc = 0; kc < 3; kc++)
#pragma unroll
            for (int kb = 0; kb < 3; kb++) {
                const T A = wa[b][kb] * S0[c][kc] + wb[b][kb] * DS[c][kc];
                JT* p = jt[a] + kb * st[b] + kc * st[c];
                jatomic(p, jprod<JT>(c1, A));
                jatomic(p + st[a], jprod<JT>(c2, A));
            }
    }
}

// copy of a leaving particle's state (already stored in its slot) to arrival slot m
template <typename T>
__device__ __forceinline__ void handoff_copy3d(const SimDev& S, int slot, int m, int pid) {
    if constexpr (uses_cell<T>()) S.mcell[m] = S.cell[slot];
#pragma unroll
    for (int a = 0; a < 3; a++)
        reinterpret_cast<T*>(S.mxi[a])[m] = reinterpret_cast<const T*>(S.xi[a])[slot];
#pragma unroll
    for (int a = 0; a < 3; a++)
        reinterpret_cast<T*>(S.mu[a])[m] = reinterpret_cast<const T*>(S.u[a])[slot];
    reinterpret_cast<T*>(S.mw)[m] = reinterpret_cast<const T*>(S.w)[slot];
    S.mid[m] = pid;
}

// CTA shape per precision: threads per CTA and the CTAs per SM the register budget is
// sized for. FP64 tiles of an 8x8x8 patch take about 122 KB of shared memory, so one CTA
// per SM; 512 threads (128 registers) measured 2-4 % faster than 256 (255 registers) and
// level with 384 on the 3D stress case, 4 % faster than both on the 3D LWFA window.
#ifndef PIC_F64_3D_THREADS
#define PIC_F64_3D_THREADS 512
#endif
template <typename T>
struct Push3DShape {
    static constexpr int threads = PIC_F64_3D_THREADS, min_blocks = 1;
};
template <>
struct Push3DShape<float> {
    static constexpr int threads = kThreads, min_blocks = 2;
};

template <typename T>
__global__ void __launch_bounds__(Push3DShape<T>::threads, Push3DShape<T>::min_blocks)
    push3d_kernel(const BatchDev* __restrict__ bd, int static_map) {
    using JT = typename JType3D<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int s_item;
    // leavers of the current item (slot, destination or -1), handed off after the item
    __shared__ int s_lv_n;
    __shared__ int s_lv_slot[kLeaveList];
    __shared__ int s_lv_dest[kLeaveList];
    // FP64: largest exponent field of each component of the staged field tile, which then
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
        __syncthreads();
        if (tid == 0) s_item = static_map ? next_static : atomicAdd(bd->head, 1);
        next_static += gridDim.x;
        __syncthreads();
        const int it = s_item;
        if (it >= *bd->nitems || it >= bd->max_items) break;
        const int4 item = bd->items[it];
        const SimDev& S = bd->sims[item.x];
        const int patch = item.y;

        const int P[3] = {S.P[0], S.P[1], S.P[2]};
        const int BX = S.BX, BY = S.BY, BZ = S.BZ;
        const int BXY = BX * BY;
        const int JX = P[0] + 5, JY = P[1] + 5, JZ = P[2] + 5;
        const int JXY = JX * JY;
        const int n[3] = {S.n[0], S.n[1], S.n[2]};
        const int p0[3] = {(patch % S.np[0]) * P[0], ((patch / S.np[0]) % S.np[1]) * P[1],
                           (patch / (S.np[0] * S.np[1])) * P[2]};
        const int gen = S.st->gen;
        const int shift = S.st->shift;
        const bool window = S.window != 0;

        T* Ft = reinterpret_cast<T*>(smem);
        const int fbytes = 6 * BXY * BZ * (int)sizeof(T);
        JT* Jt = reinterpret_cast<JT*>(smem + ((fbytes + 127) & ~127));
        const int jvol = JXY * JZ;

        for (int e = tid; e < 3 * jvol; e += blockDim.x) Jt[e] = JT(0);

        if (item.x != loaded_sim || patch != loaded_patch || gen != loaded_gen) {
            if constexpr (is_f64<T>::value) {
                if (tid < 6) s_femax[tid] = 0;
            }
            if (tid == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar, (uint32_t)fbytes);
                tma_load_4d(Ft, S.tmap + gen, &mbar, p0[0] - 1 + kGuard, p0[1] - 1 + kGuard,
                            p0[2] - 1 + kGuard, 0);
            }
            const bool ok = mbar_wait_bounded(&mbar, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(S.status, ST_TIMEOUT);
                return;
            }
            if constexpr (is_f64<T>::value)
                fix_field_tile(reinterpret_cast<double*>(Ft), BXY * BZ, s_femax);
            loaded_sim = item.x;
            loaded_patch = patch;
            loaded_gen = gen;
        }
        __syncthreads();  // J tile zeroed (FP64: field tile converted)

        T dtd[3], cj[3], eps;
        if constexpr (is_f64<T>::value) {
            for (int a = 0; a < 3; a++) dtd[a] = S.c_dtd[a], cj[a] = S.c_j[a];
            eps = S.c_eps;
        } else if constexpr (std::is_same<T, float>::value) {
            for (int a = 0; a < 3; a++) dtd[a] = S.f_dtd[a], cj[a] = S.f_j[a];
            eps = S.f_eps;
        } else {
            for (int a = 0; a < 3; a++) dtd[a] = T(S.c_dtd[a]), cj[a] = T(S.c_j[a]);
            eps = T(S.c_eps);
        }
        const int pb = S.pbase[patch];
        const int base = pb + item.z;
        const int cnt = item.w;
        const int jk = item_fixed_exp<JT>(cnt, S.cmax_exp);
        const float jsc = pow2f(jk);
        // charge factors carrying the tile's power-of-two scale (exact: the same values as
        // scaling each particle's product)
        T cjs[3];
#pragma unroll
        for (int a = 0; a < 3; a++) cjs[a] = jscale<JT>(cj[a], jsc);
        T* U0 = reinterpret_cast<T*>(S.u[0]);
        T* U1 = reinterpret_cast<T*>(S.u[1]);
        T* U2 = reinterpret_cast<T*>(S.u[2]);
        const T* W = reinterpret_cast<const T*>(S.w);

        // next iteration's raw state, loaded one iteration ahead
        int nic[3] = {0, 0, 0};
        T nf[3] = {T(0), T(0), T(0)};
        double nxi[3] = {0.0, 0.0, 0.0};
        T nu[3] = {T(0), T(0), T(0)};
        T nw = T(0);
        auto fetch = [&](int kk) {
            const int sl = base + kk;
            if constexpr (is_f64<T>::value) {
#pragma unroll
                for (int a = 0; a < 3; a++) nxi[a] = reinterpret_cast<const double*>(S.xi[a])[sl];
            } else {
                split_pos<T>(S, sl, nic, nf);
            }
            nu[0] = U0[sl];
            nu[1] = U1[sl];
            nu[2] = U2[sl];
            nw = W[sl];
        };
        if (tid < cnt) fetch(tid);

        for (int k0 = 0; k0 < cnt; k0 += blockDim.x) {
            const int k = k0 + tid;
            const bool valid = k < cnt;
            const int slot = base + (valid ? k : 0);
            bool ok = valid;
            bool leave = false;
            int dest = patch;
            if constexpr (is_f64<T>::value) {
                // ---- FP64: offsets, shapes, gather, charge factors, deposit weights and
                // products in 2^62 fixed point on the integer units; Boris and the move in
                // FP64. A field tile holding a non-finite value cannot be converted: its
                // particles are reported and dropped like non-finite particles.
                const bool ftile_ok = s_femax[0] < 0x7FF && s_femax[1] < 0x7FF &&
                                      s_femax[2] < 0x7FF && s_femax[3] < 0x7FF &&
                                      s_femax[4] < 0x7FF && s_femax[5] < 0x7FF;
                const double xi0[3] = {nxi[0], nxi[1], nxi[2]};
                double u[3] = {nu[0], nu[1], nu[2]};
                const double w = nw;
                int ic[3] = {0, 0, 0}, np_[3], tp[3], td[3];
                long long F[3] = {0, 0, 0};
                bool hp[3];
                ok = ok && ftile_ok;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (valid) split62(xi0[a], ic[a], F[a]);
                    hp[a] = F[a] >= kHalf62;  // primal node = ic + (f >= 1/2), dual = ic
                    np_[a] = ic[a] + (hp[a] ? 1 : 0);
                    tp[a] = np_[a] - p0[a];
                    td[a] = ic[a] - p0[a];
                    ok = ok && (unsigned)tp[a] <= (unsigned)P[a] && (unsigned)td[a] < (unsigned)P[a];
                }
                long long S0[3][3], S1[3][3], Q[3] = {0, 0, 0};
                int sh[3] = {0, 0, 0};
                if (ok) {
                    W31 Wp[3][3], Wd[3][3];
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        long long SD[3];
                        shape62(hp[a] ? F[a] - kOne62 : F[a], S0[a]);
                        shape62(F[a] - kHalf62, SD);
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            Wp[a][q] = w31(S0[a][q]);
                            Wd[a][q] = w31(SD[q]);
                        }
                    }
                    // one rolled loop over Ex (d,p,p) Ey (p,d,p) Ez (p,p,d) Bx (p,d,d)
                    // By (d,p,d) Bz (d,d,p); results rotate through six registers
                    const int2* Fi = reinterpret_cast<const int2*>(Ft);
                    const int vol = BXY * BZ;
                    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0, r5 = 0.0;
#pragma unroll 1
                    for (int c = 0; c < 6; c++) {
                        const bool xp = c >= 1 && c <= 3, yp = c == 0 || c == 2 || c == 4,
                                   zp = c == 0 || c == 1 || c == 5;
                        W31 gx[3], gy[3], gz[3];
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            gx[q] = xp ? Wp[0][q] : Wd[0][q];
                            gy[q] = yp ? Wp[1][q] : Wd[1][q];
                            gz[q] = zp ? Wp[2][q] : Wd[2][q];
                        }
                        const int off = (zp ? tp[2] : td[2]) * BXY + (yp ? tp[1] : td[1]) * BX +
                                        (xp ? tp[0] : td[0]);
                        const long long v = gather27_fix(Fi + c * vol + off, BX, BXY, gx, gy, gz);
                        r0 = r1, r1 = r2, r2 = r3, r3 = r4, r4 = r5;
                        r5 = fix_to_f64_int(v, fix_field_exp(s_femax[c]));
                    }
                    const double E[3] = {r0, r1, r2}, B[3] = {r3, r4, r5};
                    const double ig = boris(eps, E, B, u);
                    double xin[3];
                    int icn[3];
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        xin[a] = xi0[a] + dtd[a] * (u[a] * ig);
                        long long F1;
                        split62(xin[a], icn[a], F1);
                        const bool h1 = F1 >= kHalf62;
                        sh[a] = icn[a] + (h1 ? 1 : 0) - np_[a];
                        ok = ok && sh[a] >= -1 && sh[a] <= 1;
                        shape62(h1 ? F1 - kOne62 : F1, S1[a]);
                        Q[a] = mul_to_fixed(cjs[a], w);  // charge factor, tile scale included
                    }
                    // ---- boundaries, destination patch and the new state, stored before
                    // the deposit: periodic, except a moving-window x axis (this step's
                    // shift applied, particles leaving [0, nx) absorbed)
                    if (ok) {
                        bool del = false;
                        if (window) {
                            del = xin[0] < 0.0 || xin[0] >= (double)n[0];
                            xin[0] -= (double)shift;
                            del = del || xin[0] < 0.0;
                        }
                        int dp_[3];
#pragma unroll
                        for (int a = 0; a < 3; a++) {
                            if (!(window && a == 0)) {
                                if (xin[a] < 0.0) xin[a] += (double)n[a];
                                if (xin[a] >= (double)n[a]) xin[a] -= (double)n[a];
                            }
                            icn[a] = floor_to_int(xin[a]);
                            dp_[a] = icn[a] / P[a];
                        }
                        dest = del ? -1 : dp_[0] + S.np[0] * (dp_[1] + S.np[1] * dp_[2]);
                        leave = del || dest != patch;
                        if (!del) {  // also a leaver: the hand-off copies its state from here
                            for (int a = 0; a < 3; a++)
                                reinterpret_cast<double*>(S.xi[a])[slot] = xin[a];
                            U0[slot] = u[0];
                            U1[slot] = u[1];
                            U2[slot] = u[2];
                        }
                    }
                }
                // the next particle's state loads while this one deposits
                if (k + (int)blockDim.x < cnt) fetch(k + blockDim.x);
                const bool fast =
                    __all_sync(0xffffffffu, !ok || (sh[0] == 0 && sh[1] == 0 && sh[2] == 0));
                if (ok) {
                    const int t000 = tp[2] * JXY + tp[1] * JX + tp[0];
                    if (fast) {
                        long long* jt3[3];
                        const int t111 = t000 + JXY + JX + 1;
                        for (int a = 0; a < 3; a++) jt3[a] = Jt + a * jvol + t111;
                        deposit3d_fast_fix(jt3, JX, JXY, S0, S1, Q);
                    } else {
                        deposit3d_general_fix(Jt + t000, jvol, JX, JXY, S0, S1, sh, Q);
                    }
                }
            } else {
            int ic[3] = {nic[0], nic[1], nic[2]};
            T f[3] = {nf[0], nf[1], nf[2]};
            T u[3] = {nu[0], nu[1], nu[2]};
            T w = nw;
            if (k + (int)blockDim.x < cnt) fetch(k + blockDim.x);
            int np_[3], tp[3], td[3];
            T dp[3], dd[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const bool h = f[a] >= T(0.5);
                np_[a] = ic[a] + (h ? 1 : 0);
                dp[a] = h ? f[a] - T(1) : f[a];
                dd[a] = f[a] - T(0.5);
                tp[a] = np_[a] - p0[a];
                td[a] = ic[a] - p0[a];
                ok = ok && (unsigned)tp[a] <= (unsigned)P[a] && (unsigned)td[a] < (unsigned)P[a];
            }
            int icn[3] = {0, 0, 0};
            T fn[3] = {T(0), T(0), T(0)};
            T S0keep[3][3] = {}, d1keep[3] = {T(0), T(0), T(0)};
            int shkeep[3] = {0, 0, 0};
            if (ok) {
                T Sp[3][3], Sd[3][3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    shape3(dp[a], Sp[a]);
                    shape3(dd[a], Sd[a]);
                }
                T E[3], B[3];
                // Ex (d,p,p) Ey (p,d,p) Ez (p,p,d) Bx (p,d,d) By (d,p,d) Bz (d,d,p)
                E[0] = gather27(Ft + 0 * BXY * BZ + tp[2] * BXY + tp[1] * BX + td[0], BX, BXY, Sd[0], Sp[1], Sp[2]);
                E[1] = gather27(Ft + 1 * BXY * BZ + tp[2] * BXY + td[1] * BX + tp[0], BX, BXY, Sp[0], Sd[1], Sp[2]);
                E[2] = gather27(Ft + 2 * BXY * BZ + td[2] * BXY + tp[1] * BX + tp[0], BX, BXY, Sp[0], Sp[1], Sd[2]);
                B[0] = gather27(Ft + 3 * BXY * BZ + td[2] * BXY + td[1] * BX + tp[0], BX, BXY, Sp[0], Sd[1], Sd[2]);
                B[1] = gather27(Ft + 4 * BXY * BZ + td[2] * BXY + tp[1] * BX + td[0], BX, BXY, Sd[0], Sp[1], Sd[2]);
                B[2] = gather27(Ft + 5 * BXY * BZ + tp[2] * BXY + td[1] * BX + td[0], BX, BXY, Sd[0], Sd[1], Sp[2]);
                const T ig = boris(eps, E, B, u);
                const T v[3] = {u[0] * ig, u[1] * ig, u[2] * ig};
                int np1[3], sh[3];
                T dp1[3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    T g = f[a] + dtd[a] * v[a];
                    int i1 = ic[a];
                    if (g < T(0)) {
                        g += T(1);
                        i1 -= 1;
                        if (g >= T(1)) { g = T(0); i1 += 1; }
                    } else if (g >= T(1)) {
                        g -= T(1);
                        i1 += 1;
                    }
                    const bool h1 = g >= T(0.5);
                    np1[a] = i1 + (h1 ? 1 : 0);
                    dp1[a] = h1 ? g - T(1) : g;
                    icn[a] = i1;
                    fn[a] = g;
                    sh[a] = np1[a] - np_[a];
                    ok = ok && sh[a] >= -1 && sh[a] <= 1;
                }
                for (int a = 0; a < 3; a++) {
                    for (int q = 0; q < 3; q++) S0keep[a][q] = Sp[a][q];
                    d1keep[a] = dp1[a];
                    shkeep[a] = sh[a];
                }
            }
            // warp-uniform choice of the no-crossing deposition
            const bool fast = __all_sync(0xffffffffu, !ok || (shkeep[0] == 0 && shkeep[1] == 0 &&
                                                              shkeep[2] == 0));
            if (ok) {
                {
                    const T* dp1 = d1keep;
                    const int* sh = shkeep;
                    T Sp[3][3];
                    for (int a = 0; a < 3; a++)
                        for (int q = 0; q < 3; q++) Sp[a][q] = S0keep[a][q];
                    if (fast) {
                        JT* jt3[3];
                        const T q3[3] = {cjs[0] * w, cjs[1] * w, cjs[2] * w};
                        const int t111 = (tp[2] + 1) * JXY + (tp[1] + 1) * JX + (tp[0] + 1);
                        for (int a = 0; a < 3; a++) jt3[a] = Jt + a * jvol + t111;
                        deposit3d_fast<T, JT>(jt3, JX, JXY, Sp, dp1, q3);
                    } else {
                    // four-node window per axis (any shift): 3 x 16 x 3 atomics
                    Axis4<T> ax[3];
#pragma unroll
                    for (int a = 0; a < 3; a++) esirkepov_axis4(Sp[a], dp1[a], sh[a], ax[a]);
                    T wa[3][4], wb[3][4];
#pragma unroll
                    for (int a = 0; a < 3; a++)
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            wa[a][q] = ax[a].S0[q] + T(0.5) * ax[a].DS[q];
                            wb[a][q] = T(0.5) * ax[a].S0[q] + ax[a].DS[q] * T(1.0 / 3.0);
                        }
                    const int st3[3] = {1, JX, JXY};
                    const int o3 = (tp[2] + ax[2].start) * JXY + (tp[1] + ax[1].start) * JX +
                                   (tp[0] + ax[0].start);
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        const int b = (a + 1) % 3, c = (a + 2) % 3;
                        const T qa = cjs[a] * w;
                        const T c1 = qa * ax[a].DS[0], c2 = qa * (ax[a].DS[0] + ax[a].DS[1]),
                                c3 = qa * (ax[a].DS[0] + ax[a].DS[1] + ax[a].DS[2]);
                        JT* jt = Jt + a * jvol + o3;
#pragma unroll
                        for (int kc = 0; kc < 4; kc++)
#pragma unroll
                            for (int kb = 0; kb < 4; kb++) {
                                const T A = wa[b][kb] * ax[c].S0[kc] + wb[b][kb] * ax[c].DS[kc];
                                JT* p = jt + kb * st3[b] + kc * st3[c];
                                jatomic(p, jprod<JT>(c1, A));
                                jatomic(p + st3[a], jprod<JT>(c2, A));
                                jatomic(p + 2 * st3[a], jprod<JT>(c3, A));
                            }
                    }
                    }
                }
                    // boundaries and destination patch: periodic, except a moving-window x
                    // axis (this step's shift applied, particles leaving [0, nx) absorbed)
                    bool del = false;
                    if (window) {
                        del = icn[0] < 0 || icn[0] >= n[0];
                        icn[0] -= shift;
                        del = del || icn[0] < 0;
                    }
                    int dp_[3];
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        if (!(window && a == 0)) icn[a] = wrapi(icn[a], n[a]);
                        dp_[a] = icn[a] / P[a];
                    }
                    dest = del ? -1 : dp_[0] + S.np[0] * (dp_[1] + S.np[1] * dp_[2]);
                    leave = del || dest != patch;
                    if (!del) {  // also a leaver: the hand-off copies its state from here
                        S.cell[slot] = icn[0] | (icn[1] << 11) | (icn[2] << 22);
                        for (int a = 0; a < 3; a++)
                            reinterpret_cast<T*>(S.xi[a])[slot] = fn[a];
                        U0[slot] = u[0];
                        U1[slot] = u[1];
                        U2[slot] = u[2];
                    }
            }
            }
            if (valid && !ok) {
                atomicOr(S.status, ST_NUMERIC);
                leave = true;
                dest = -1;
            }
            // exchange hand-off: a leaver is listed in shared memory; only when the list
            // is full does it claim its slots here (warp-aggregated global counters)
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
                            handoff_copy3d<T>(S, slot, mb + cl.y, pid);
                        else
                            atomicOr(S.status, ST_MAILBOX);
                    }
                }
            }
        }
        __syncthreads();

        // hand-off of the listed leavers, a warp-aggregated claim at a time
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
                            handoff_copy3d<T>(S, slot, mb + cl.y, pid);
                        else
                            atomicOr(S.status, ST_MAILBOX);
                    }
                    S.id[slot] = -1;
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_lv_n = 0;  // read by every thread before the barrier above
        __syncthreads();

        // flush the current tile (origin p0 - 2) into the global FP64 J (periodic)
        double* Jg = S.J[gen];
        const long long fs = S.fstride;
        for (int e = tid; e < 3 * jvol; e += blockDim.x) {
            const JT v = Jt[e];
            if (v == JT(0)) continue;
            const int comp = e / jvol;
            const int r = e - comp * jvol;
            const int tz = r / JXY;
            const int r2 = r - tz * JXY;
            const int ty = r2 / JX, tx = r2 - ty * JX;
            int gi = p0[0] - 2 + tx;
            if (window) {
                if (gi < 0 || gi >= n[0]) continue;  // outside the window: dropped
            } else {
                gi = wrapi(gi, n[0]);
            }
            const int gj = wrapi(p0[1] - 2 + ty, n[1]);
            const int gk = wrapi(p0[2] - 2 + tz, n[2]);
            atomicAdd(Jg + comp * fs + ((long long)(gk + kGuard) * S.NY + (gj + kGuard)) * S.NX +
                          (gi + kGuard),
                      jflush(v, jk));
        }
    }
}

template <typename T>
int smem_bytes_3d(int P0, int P1, int P2) {
    const int BX = P0 + 4, BY = P1 + 3, BZ = P2 + 3;
    const int fb = 6 * BX * BY * BZ * (int)sizeof(T);
    const int jb = 3 * (P0 + 5) * (P1 + 5) * (P2 + 5) * (int)sizeof(typename JType3D<T>::type);
    return ((fb + 127) & ~127) + jb;
}

int push3d_smem(int prec, int P0, int P1, int P2) {
    int sb = 0;
    PIC_DISPATCH_3D(prec, (sb = smem_bytes_3d<T>(P0, P1, P2)));
    return sb;
}

template <typename T>
static int occupancy_3d(int sb) {
    int blocks = 0;
    if (cudaFuncSetAttribute(push3d_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb) !=
        cudaSuccess)
        return 0;
    cudaFuncSetAttribute(push3d_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, push3d_kernel<T>,
                                                      Push3DShape<T>::threads, sb) !=
        cudaSuccess)
        return 0;
    return blocks;
}

int push3d_occupancy(int prec, int P0, int P1, int P2, int* smem_bytes) {
    const int sb = push3d_smem(prec, P0, P1, P2);
    *smem_bytes = sb;
    int blocks = 0;
    PIC_DISPATCH_3D(prec, (blocks = occupancy_3d<T>(sb)));
    return blocks;
}

cudaError_t launch_push3d(const BatchDev* bd_dev, int prec, int mapping, int P0, int P1, int P2,
                          int grid, cudaStream_t s) {
    const int sb = push3d_smem(prec, P0, P1, P2);
    const int static_map = mapping == 1;
    if (prec != 0 && prec != 1) return cudaErrorInvalidValue;
    PIC_DISPATCH_3D(prec, (push3d_kernel<T><<<grid, Push3DShape<T>::threads, sb, s>>>(
                              bd_dev, static_map)));
    return cudaGetLastError();
}

}  // namespace pic
