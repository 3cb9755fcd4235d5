// Sixth-order Maxwell solver: the higher-order field scheme of the paper's Photon-Plasma
// runs (Sec. 2.1), as leapfrog in time with sixth-order staggered space differences
//   D f(x) = sum_{l=1..3} c_l [f(x + (l - 1/2) h) - f(x - (l - 1/2) h)] / h,
//   c = (75/64, -25/384, 3/640)   (exact for polynomials up to degree 6),
// in place of Yee's two-point difference in both half-updates:
//   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2})
//   B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1},   B^{n+1} = (B^{n+1/2} + B^{n+3/2}) / 2.
// Staggering, buffers and the window are those of the two-point kernels: periodic axes
// wrap their indices; a moving-window x axis reads zero outside the window; the shift
// of this step is folded into the write index (outputs go to x = ox, inputs are read
// at x = ox + shift of the old frame).
//
// The wide stencil reaches one column further back than Yee's: the B update of the new
// frame's columns 0 and 1 reads E^{n+1} at old-frame x = 0, the column the shift drops.
// When the window shifts, the E kernel therefore also evaluates that column and leaves
// it in S.ecol, where the B kernel reads it.
//
// One thread per cell; the 6-point reads along x are coalesced, and the ones along y
// and z hit rows that neighbouring CTAs also read (L1/L2), so DRAM traffic stays close
// to the two-point kernels' per-cell bytes.
#include <cuda_runtime.h>

#include "fields.cuh"
#include "pic_device.cuh"
#include "pic_internal.h"

namespace pic {

namespace {

// ------------------------------------------------------------------------ 2D

// Read access to the old-frame B^{n+1/2} (component c at interior (i, j)); x outside the
// window is zero, periodic axes wrap.
template <typename T>
struct H2 {
    const T* h;
    long long fs;
    int NX, nx, ny;
    bool win;
    __device__ __forceinline__ T operator()(int c, int i, int j) const {
        if (win) {
            if (i < 0 || i >= nx) return T(0);
        } else {
            i = wrap_index(i, nx);
        }
        j = wrap_index(j, ny);
        return h[c * fs + (long long)(j + kGuard) * NX + (i + kGuard)];
    }
};

// E^{n+1} at old-frame x = m: new-frame column m - shift, or the dropped column
template <typename T>
struct E2 {
    const T* e;
    const T* col;  // [3][ny], valid when shift = 1
    long long fs;
    int NX, nx, ny, shift;
    bool win;
    __device__ __forceinline__ T operator()(int c, int m, int j) const {
        j = wrap_index(j, ny);
        if (win) {
            if (m < 0 || m >= nx) return T(0);
            if (m < shift) return col[(long long)c * ny + j];
            m -= shift;
        } else {
            m = wrap_index(m, nx);
        }
        return e[c * fs + (long long)(j + kGuard) * NX + (m + kGuard)];
    }
};

// E^{n+1} at old-frame (i, j): E^n + dt (curl B^{n+1/2} - J^{n+1/2})
template <typename T>
__device__ __forceinline__ void e_update_2d(const SimDev& S, const H2<T>& H, const T* Ein,
                                            const double* Jin, int i, int j, T e[3]) {
    using C = FieldConst<T>;
    using K = Stencil6<T>;
    const T dt = C::dt(S);
    T dxbz = T(0), dxby = T(0), dybz = T(0), dybx = T(0);
#pragma unroll
    for (int l = 0; l < 3; l++) {
        const T kx = K::k(S, 0, l), ky = K::k(S, 1, l);
        // backward-staggered pairs: (i + l, i - l - 1) in x, (j + l, j - l - 1) in y
        dxbz += kx * (H(2, i + l, j) - H(2, i - l - 1, j));
        dxby += kx * (H(1, i + l, j) - H(1, i - l - 1, j));
        dybz += ky * (H(2, i, j + l) - H(2, i, j - l - 1));
        dybx += ky * (H(0, i, j + l) - H(0, i, j - l - 1));
    }
    const long long p = (long long)(j + kGuard) * S.NX + (i + kGuard);
    const long long fs = S.fstride;
    e[0] = Ein[p] + dt * (dybz - C::cur(Jin[p]));
    e[1] = Ein[fs + p] + dt * (-dxbz - C::cur(Jin[fs + p]));
    e[2] = Ein[2 * fs + p] + dt * (dxby - dybx - C::cur(Jin[2 * fs + p]));
}

template <typename T>
__global__ void __launch_bounds__(256) maxwell6_e2d_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int nx = S.n[0], ny = S.n[1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nx * ny) return;
    const int ox = idx % nx, oy = idx / nx;
    const int g = S.st->gen, s = S.st->shift;
    const int NX = S.NX;
    const long long fs = S.fstride;
    const bool win = S.window != 0;
    const T* Ein = reinterpret_cast<const T*>(S.F[g]);
    T* Eout = reinterpret_cast<T*>(S.F[1 - g]);
    const H2<T> H{reinterpret_cast<const T*>(S.H[g]), fs, NX, nx, ny, win};
    const double* Jin = S.J[g];
    double* Jnext = S.J[1 - g];
    const long long po = (long long)(oy + kGuard) * NX + (ox + kGuard);
    Jnext[po] = 0.0;
    Jnext[fs + po] = 0.0;
    Jnext[2 * fs + po] = 0.0;
    const int i = ox + s;
    T e[3] = {T(0), T(0), T(0)};
    if (i < nx) e_update_2d(S, H, Ein, Jin, i, oy, e);
#pragma unroll
    for (int c = 0; c < 3; c++) put2d(Eout + c * fs, NX, ox, oy, nx, ny, !win, e[c]);
    if (win && s == 1 && ox == 0) {
        // the column this shift drops, for the B update of the first new columns
        T d[3];
        e_update_2d(S, H, Ein, Jin, 0, oy, d);
        T* col = reinterpret_cast<T*>(S.ecol);
#pragma unroll
        for (int c = 0; c < 3; c++) col[(long long)c * ny + oy] = d[c];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) maxwell6_b2d_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int nx = S.n[0], ny = S.n[1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nx * ny) return;
    const int ox = idx % nx, oy = idx / nx;
    const int g = S.st->gen, s = S.st->shift;
    const int NX = S.NX;
    const long long fs = S.fstride;
    const bool win = S.window != 0;
    const E2<T> E{reinterpret_cast<const T*>(S.F[1 - g]), reinterpret_cast<const T*>(S.ecol),
                  fs, NX, nx, ny, s, win};
    T* Bn = reinterpret_cast<T*>(S.F[1 - g]) + 3 * fs;
    const T* Hin = reinterpret_cast<const T*>(S.H[g]);
    T* Hout = reinterpret_cast<T*>(S.H[1 - g]);
    const int i = ox + s, j = oy;
    T h[3] = {T(0), T(0), T(0)}, nb[3] = {T(0), T(0), T(0)};
    if (i < nx) {
        using C = FieldConst<T>;
        using K = Stencil6<T>;
        const T dt = C::dt(S);
        T dxez = T(0), dxey = T(0), dyez = T(0), dyex = T(0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const T kx = K::k(S, 0, l), ky = K::k(S, 1, l);
            // forward-staggered pairs: (i + l + 1, i - l) in x, (j + l + 1, j - l) in y
            dxez += kx * (E(2, i + l + 1, j) - E(2, i - l, j));
            dxey += kx * (E(1, i + l + 1, j) - E(1, i - l, j));
            dyez += ky * (E(2, i, j + l + 1) - E(2, i, j - l));
            dyex += ky * (E(0, i, j + l + 1) - E(0, i, j - l));
        }
        const long long p = (long long)(j + kGuard) * NX + (i + kGuard);
        const T h0[3] = {Hin[p], Hin[fs + p], Hin[2 * fs + p]};
        h[0] = h0[0] - dt * dyez;
        h[1] = h0[1] + dt * dxez;
        h[2] = h0[2] - dt * (dxey - dyex);
#pragma unroll
        for (int c = 0; c < 3; c++) nb[c] = T(0.5) * (h0[c] + h[c]);
    }
    const long long po = (long long)(oy + kGuard) * NX + (ox + kGuard);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        Hout[c * fs + po] = h[c];
        put2d(Bn + c * fs, NX, ox, oy, nx, ny, !win, nb[c]);
    }
}

// ------------------------------------------------------------------------ 3D

template <typename T>
struct H3 {
    const SimDev* S;
    const T* h;
    __device__ __forceinline__ T operator()(int c, int i, int j, int k) const {
        if (S->window) {
            if (i < 0 || i >= S->n[0]) return T(0);
        } else {
            i = wrap_index(i, S->n[0]);
        }
        j = wrap_index(j, S->n[1]);
        k = wrap_index(k, S->n[2]);
        return h[c * S->fstride + pidx3(*S, i, j, k)];
    }
};

template <typename T>
struct E3 {
    const SimDev* S;
    const T* e;
    const T* col;  // [3][nz][ny]
    int shift;
    __device__ __forceinline__ T operator()(int c, int m, int j, int k) const {
        const int nx = S->n[0], ny = S->n[1], nz = S->n[2];
        j = wrap_index(j, ny);
        k = wrap_index(k, nz);
        if (S->window) {
            if (m < 0 || m >= nx) return T(0);
            if (m < shift) return col[((long long)c * nz + k) * ny + j];
            m -= shift;
        } else {
            m = wrap_index(m, nx);
        }
        return e[c * S->fstride + pidx3(*S, m, j, k)];
    }
};

template <typename T>
__device__ __forceinline__ void e_update_3d(const SimDev& S, const H3<T>& H, const T* Ein,
                                            const double* Jin, int i, int j, int k, T e[3]) {
    using C = FieldConst<T>;
    using K = Stencil6<T>;
    const T dt = C::dt(S);
    // d_a B_c for the six (axis, component) pairs of the curl
    T dybz = T(0), dzby = T(0), dzbx = T(0), dxbz = T(0), dxby = T(0), dybx = T(0);
#pragma unroll
    for (int l = 0; l < 3; l++) {
        const T kx = K::k(S, 0, l), ky = K::k(S, 1, l), kz = K::k(S, 2, l);
        dxbz += kx * (H(2, i + l, j, k) - H(2, i - l - 1, j, k));
        dxby += kx * (H(1, i + l, j, k) - H(1, i - l - 1, j, k));
        dybz += ky * (H(2, i, j + l, k) - H(2, i, j - l - 1, k));
        dybx += ky * (H(0, i, j + l, k) - H(0, i, j - l - 1, k));
        dzby += kz * (H(1, i, j, k + l) - H(1, i, j, k - l - 1));
        dzbx += kz * (H(0, i, j, k + l) - H(0, i, j, k - l - 1));
    }
    const long long p = pidx3(S, i, j, k);
    const long long fs = S.fstride;
    e[0] = Ein[p] + dt * (dybz - dzby - C::cur(Jin[p]));
    e[1] = Ein[fs + p] + dt * (dzbx - dxbz - C::cur(Jin[fs + p]));
    e[2] = Ein[2 * fs + p] + dt * (dxby - dybx - C::cur(Jin[2 * fs + p]));
}

template <typename T>
__global__ void __launch_bounds__(256) maxwell6_e3d_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int nx = S.n[0], ny = S.n[1];
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S.ncell) return;
    const int ox = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const int g = S.st->gen, s = S.st->shift;
    const long long fs = S.fstride;
    const T* Ein = reinterpret_cast<const T*>(S.F[g]);
    T* Eout = reinterpret_cast<T*>(S.F[1 - g]);
    const H3<T> H{&S, reinterpret_cast<const T*>(S.H[g])};
    const double* Jin = S.J[g];
    double* Jnext = S.J[1 - g];
    const long long po = pidx3(S, ox, j, k);
    Jnext[po] = 0.0;
    Jnext[fs + po] = 0.0;
    Jnext[2 * fs + po] = 0.0;
    const int i = ox + s;
    T e[3] = {T(0), T(0), T(0)};
    if (i < nx) e_update_3d(S, H, Ein, Jin, i, j, k, e);
#pragma unroll
    for (int q = 0; q < 3; q++) put3d(S, Eout + q * fs, ox, j, k, e[q]);
    if (S.window && s == 1 && ox == 0) {
        T d[3];
        e_update_3d(S, H, Ein, Jin, 0, j, k, d);
        T* col = reinterpret_cast<T*>(S.ecol);
        const int nz = S.n[2];
#pragma unroll
        for (int q = 0; q < 3; q++) col[((long long)q * nz + k) * ny + j] = d[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) maxwell6_b3d_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int nx = S.n[0], ny = S.n[1];
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S.ncell) return;
    const int ox = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const int g = S.st->gen, s = S.st->shift;
    const long long fs = S.fstride;
    const E3<T> E{&S, reinterpret_cast<const T*>(S.F[1 - g]),
                  reinterpret_cast<const T*>(S.ecol), s};
    T* Bn = reinterpret_cast<T*>(S.F[1 - g]) + 3 * fs;
    const T* Hin = reinterpret_cast<const T*>(S.H[g]);
    T* Hout = reinterpret_cast<T*>(S.H[1 - g]);
    const int i = ox + s;
    T h[3] = {T(0), T(0), T(0)}, nb[3] = {T(0), T(0), T(0)};
    if (i < nx) {
        using C = FieldConst<T>;
        using K = Stencil6<T>;
        const T dt = C::dt(S);
        T dyez = T(0), dzey = T(0), dzex = T(0), dxez = T(0), dxey = T(0), dyex = T(0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const T kx = K::k(S, 0, l), ky = K::k(S, 1, l), kz = K::k(S, 2, l);
            dxez += kx * (E(2, i + l + 1, j, k) - E(2, i - l, j, k));
            dxey += kx * (E(1, i + l + 1, j, k) - E(1, i - l, j, k));
            dyez += ky * (E(2, i, j + l + 1, k) - E(2, i, j - l, k));
            dyex += ky * (E(0, i, j + l + 1, k) - E(0, i, j - l, k));
            dzey += kz * (E(1, i, j, k + l + 1) - E(1, i, j, k - l));
            dzex += kz * (E(0, i, j, k + l + 1) - E(0, i, j, k - l));
        }
        const long long p = pidx3(S, i, j, k);
        const T h0[3] = {Hin[p], Hin[fs + p], Hin[2 * fs + p]};
        h[0] = h0[0] - dt * (dyez - dzey);
        h[1] = h0[1] - dt * (dzex - dxez);
        h[2] = h0[2] - dt * (dxey - dyex);
#pragma unroll
        for (int q = 0; q < 3; q++) nb[q] = T(0.5) * (h0[q] + h[q]);
    }
    const long long po = pidx3(S, ox, j, k);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        Hout[q * fs + po] = h[q];
        put3d(S, Bn + q * fs, ox, j, k, nb[q]);
    }
}

}  // namespace

cudaError_t launch_maxwell6(const BatchDev* bd, int nsims, long long max_ncell, int dims,
                           int prec, cudaStream_t s) {
    dim3 grid((unsigned)((max_ncell + 255) / 256), nsims);
    if (dims == 2) {
        PIC_DISPATCH(prec, (maxwell6_e2d_kernel<T><<<grid, 256, 0, s>>>(bd),
                            maxwell6_b2d_kernel<T><<<grid, 256, 0, s>>>(bd)));
    } else if (dims == 3) {
        PIC_DISPATCH(prec, (maxwell6_e3d_kernel<T><<<grid, 256, 0, s>>>(bd),
                            maxwell6_b3d_kernel<T><<<grid, 256, 0, s>>>(bd)));
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pic
