// Helpers shared by the field-solver kernels (two-point and sixth-order): writes of a
// cell value together with its periodic images in the guard cells, padded indexing,
// index wrapping and the sixth-order difference coefficients per precision.
#pragma once
#include "pic_device.cuh"
#include "pic_internal.h"

namespace pic {

// Writes v at interior (i, j) of a padded component and at its periodic images in
// the guard cells (x images only when x is periodic).
template <typename T>
__device__ __forceinline__ void put2d(T* a, int NX, int i, int j, int nx, int ny, bool px, T v) {
    int xs[2] = {i + kGuard, -1}, ys[2] = {j + kGuard, -1};
    if (px) {
        if (i == nx - 1) xs[1] = 0;
        else if (i == 0) xs[1] = nx + kGuard;
        else if (i == 1) xs[1] = nx + 1 + kGuard;
    }
    if (j == ny - 1) ys[1] = 0;
    else if (j == 0) ys[1] = ny + kGuard;
    else if (j == 1) ys[1] = ny + 1 + kGuard;
#pragma unroll
    for (int a2 = 0; a2 < 2; a2++)
#pragma unroll
        for (int b2 = 0; b2 < 2; b2++)
            if (xs[a2] >= 0 && ys[b2] >= 0) a[(long long)ys[b2] * NX + xs[a2]] = v;
}

__device__ __forceinline__ long long pidx3(const SimDev& S, int i, int j, int k) {
    return ((long long)(k + kGuard) * S.NY + (j + kGuard)) * S.NX + (i + kGuard);
}

// value at interior (i, j, k) and its periodic images in the guard cells (no x images
// along a moving-window x axis, whose guards stay zero)
template <typename T>
__device__ __forceinline__ void put3d(const SimDev& S, T* a, int i, int j, int k, T v) {
    int xs[2] = {i + kGuard, -1}, ys[2] = {j + kGuard, -1}, zs[2] = {k + kGuard, -1};
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    if (!S.window) {
        if (i == nx - 1) xs[1] = 0; else if (i == 0) xs[1] = nx + kGuard; else if (i == 1) xs[1] = nx + 1 + kGuard;
    }
    if (j == ny - 1) ys[1] = 0; else if (j == 0) ys[1] = ny + kGuard; else if (j == 1) ys[1] = ny + 1 + kGuard;
    if (k == nz - 1) zs[1] = 0; else if (k == 0) zs[1] = nz + kGuard; else if (k == 1) zs[1] = nz + 1 + kGuard;
#pragma unroll
    for (int c = 0; c < 2; c++)
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int a2 = 0; a2 < 2; a2++)
                if (xs[a2] >= 0 && ys[b] >= 0 && zs[c] >= 0)
                    a[((long long)zs[c] * S.NY + ys[b]) * S.NX + xs[a2]] = v;
}

// v + n or v - n for an index at most one period outside [0, n)
__device__ __forceinline__ int wrap_index(int v, int n) {
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// c_l / d[a] of the sixth-order staggered difference (l = 0, 1, 2 for c_1, c_2, c_3)
template <typename T>
struct Stencil6;
template <>
struct Stencil6<double> {
    static __device__ __forceinline__ double k(const SimDev& S, int a, int l) { return S.c_k[a][l]; }
};
template <>
struct Stencil6<float> {
    static __device__ __forceinline__ float k(const SimDev& S, int a, int l) { return S.f_k[a][l]; }
};
template <>
struct Stencil6<df64> {
    static __device__ __forceinline__ df64 k(const SimDev& S, int a, int l) {
        return df64(S.f_k[a][l], S.f_k_lo[a][l]);
    }
};

}  // namespace pic
