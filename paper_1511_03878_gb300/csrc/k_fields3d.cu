// 3D Yee FDTD half-updates (periodic on all axes) and the 3D diagnostics kernels.
//   E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2})
//   B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1},  B^{n+1} = (B^{n+1/2} + B^{n+3/2}) / 2
// Staggering: Ex (i+1/2,j,k) Ey (i,j+1/2,k) Ez (i,j,k+1/2) Bx (i,j+1/2,k+1/2)
// By (i+1/2,j,k+1/2) Bz (i+1/2,j+1/2,k).
#include <cuda_runtime.h>

#include "pic_device.cuh"
#include "pic_internal.h"
#include "fields.cuh"

namespace pic {

template <typename T>
__global__ void __launch_bounds__(256) yee_e3d_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S.ncell) return;
    // output cell (ox, j, k) of the new frame; input cell i = ox + shift of the old one
    const int ox = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const int g = S.st->gen;
    const int i = ox + S.st->shift;
    const bool win = S.window != 0;
    const long long fs = S.fstride;
    const T* Ein = reinterpret_cast<const T*>(S.F[g]);
    T* Eout = reinterpret_cast<T*>(S.F[1 - g]);
    const T* H = reinterpret_cast<const T*>(S.H[g]);
    const double* Jin = S.J[g];
    double* Jnext = S.J[1 - g];
    const long long po = pidx3(S, ox, j, k);
    Jnext[po] = 0.0;
    Jnext[fs + po] = 0.0;
    Jnext[2 * fs + po] = 0.0;
    T ex = T(0), ey = T(0), ez = T(0);
    if (i < nx) {
        const bool has_im = !(win && i == 0);
        const int im = i == 0 ? nx - 1 : i - 1, jm = j == 0 ? ny - 1 : j - 1,
                  km = k == 0 ? nz - 1 : k - 1;
        using C = FieldConst<T>;
        const T dt = C::dt(S), ix = C::id(S, 0), iy = C::id(S, 1), iz = C::id(S, 2);
        const long long p = pidx3(S, i, j, k);
        const T bx = H[p], by = H[fs + p], bz = H[2 * fs + p];
        const T bx_jm = H[pidx3(S, i, jm, k)], bx_km = H[pidx3(S, i, j, km)];
        const T by_im = has_im ? H[fs + pidx3(S, im, j, k)] : T(0);
        const T by_km = H[fs + pidx3(S, i, j, km)];
        const T bz_im = has_im ? H[2 * fs + pidx3(S, im, j, k)] : T(0);
        const T bz_jm = H[2 * fs + pidx3(S, i, jm, k)];
        ex = Ein[p] + dt * ((bz - bz_jm) * iy - (by - by_km) * iz - C::cur(Jin[p]));
        ey = Ein[fs + p] + dt * ((bx - bx_km) * iz - (bz - bz_im) * ix - C::cur(Jin[fs + p]));
        ez = Ein[2 * fs + p] +
             dt * ((by - by_im) * ix - (bx - bx_jm) * iy - C::cur(Jin[2 * fs + p]));
    }
    put3d(S, Eout, ox, j, k, ex);
    put3d(S, Eout + fs, ox, j, k, ey);
    put3d(S, Eout + 2 * fs, ox, j, k, ez);
}

template <typename T>
__global__ void __launch_bounds__(256) yee_b3d_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S.ncell) return;
    // output cell (ox, j, k): E^{n+1} is already in the new frame, B^{n+1/2} is read at
    // i = ox + shift of the old one
    const int ox = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const int g = S.st->gen;
    const int i = ox + S.st->shift;
    const bool win = S.window != 0;
    const long long fs = S.fstride;
    const T* E = reinterpret_cast<const T*>(S.F[1 - g]);
    T* Bn = reinterpret_cast<T*>(S.F[1 - g]) + 3 * fs;
    const T* H = reinterpret_cast<const T*>(S.H[g]);
    T* Hout = reinterpret_cast<T*>(S.H[1 - g]);
    const long long po = pidx3(S, ox, j, k);
    T hx = T(0), hy = T(0), hz = T(0), nbx = T(0), nby = T(0), nbz = T(0);
    if (i < nx) {
        const bool has_ip = !(win && ox + 1 >= nx);
        const int ip = ox == nx - 1 ? 0 : ox + 1, jp = j == ny - 1 ? 0 : j + 1,
                  kp = k == nz - 1 ? 0 : k + 1;
        using C = FieldConst<T>;
        const T dt = C::dt(S), ix = C::id(S, 0), iy = C::id(S, 1), iz = C::id(S, 2);
        const T ex = E[po], ey = E[fs + po], ez = E[2 * fs + po];
        const T ex_jp = E[pidx3(S, ox, jp, k)], ex_kp = E[pidx3(S, ox, j, kp)];
        const T ey_ip = has_ip ? E[fs + pidx3(S, ip, j, k)] : T(0);
        const T ey_kp = E[fs + pidx3(S, ox, j, kp)];
        const T ez_ip = has_ip ? E[2 * fs + pidx3(S, ip, j, k)] : T(0);
        const T ez_jp = E[2 * fs + pidx3(S, ox, jp, k)];
        const long long p = pidx3(S, i, j, k);
        const T h0x = H[p], h0y = H[fs + p], h0z = H[2 * fs + p];
        hx = h0x - dt * ((ez_jp - ez) * iy - (ey_kp - ey) * iz);
        hy = h0y - dt * ((ex_kp - ex) * iz - (ez_ip - ez) * ix);
        hz = h0z - dt * ((ey_ip - ey) * ix - (ex_jp - ex) * iy);
        nbx = T(0.5) * (h0x + hx);
        nby = T(0.5) * (h0y + hy);
        nbz = T(0.5) * (h0z + hz);
    }
    Hout[po] = hx;
    Hout[fs + po] = hy;
    Hout[2 * fs + po] = hz;
    put3d(S, Bn, ox, j, k, nbx);
    put3d(S, Bn + fs, ox, j, k, nby);
    put3d(S, Bn + 2 * fs, ox, j, k, nbz);
}

cudaError_t launch_yee3d(const BatchDev* bd, int nsims, long long max_ncell, int prec,
                         cudaStream_t s) {
    dim3 grid((unsigned)((max_ncell + 255) / 256), nsims);
    PIC_DISPATCH(prec, (yee_e3d_kernel<T><<<grid, 256, 0, s>>>(bd), yee_b3d_kernel<T><<<grid, 256, 0, s>>>(bd)));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- diagnostics (3D)

// Charge density on the nodes, one CTA per patch: the particles' order-2 weights add
// into a shared tile of the patch's nodes plus one below and two above each axis, which is
// then added to the global array once (27 shared atomics per particle, one global atomic
// per touched node). A tap that would fall outside the tile (a particle outside its
// patch) goes to the global array directly. tiled = 0: every tap goes there.
template <typename T>
__global__ void rho3d_kernel(const SimDev* __restrict__ sd, double* rho, double sign, int tiled) {
    extern __shared__ double tile[];
    const SimDev& S = *sd;
    const int p = blockIdx.x;
    if (p >= S.npatch) return;
    const int b0 = S.pbase[p], cnt = S.pcount[p];
    const int n[3] = {S.n[0], S.n[1], S.n[2]};
    const int TX = S.P[0] + 3, TY = S.P[1] + 3, TZ = S.P[2] + 3;
    const int o[3] = {(p % S.np[0]) * S.P[0] - 1, ((p / S.np[0]) % S.np[1]) * S.P[1] - 1,
                      (p / (S.np[0] * S.np[1])) * S.P[2] - 1};  // tile origin (node index)
    if (tiled) {
        for (int e = threadIdx.x; e < TX * TY * TZ; e += blockDim.x) tile[e] = 0.0;
        __syncthreads();
    }
    // global node of a tap: periodic wrap, or -1 outside a moving window's x range
    auto node = [&](int ii, int jj, int kk) -> long long {
        if (S.window) {
            if (ii < 0 || ii >= n[0]) return -1;
        } else {
            ii = wrapi(ii, n[0]);
        }
        return ((long long)wrapi(kk, n[2]) * n[1] + wrapi(jj, n[1])) * n[0] + ii;
    };
    const double qdv = sign * S.q / (S.d[0] * S.d[1] * S.d[2]);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int t = b0 + k;
        int ic[3];
        double f[3];
        if constexpr (is_f64<T>::value) {
            for (int a = 0; a < 3; a++) {
                const double xi = reinterpret_cast<const double*>(S.xi[a])[t];
                ic[a] = (int)floor(xi);
                f[a] = xi - ic[a];
            }
        } else {
            const int c = S.cell[t];
            ic[0] = c & 0x7FF;
            ic[1] = (c >> 11) & 0x7FF;
            ic[2] = (c >> 22) & 0x3FF;
            for (int a = 0; a < 3; a++) f[a] = (double)reinterpret_cast<const T*>(S.xi[a])[t];
        }
        double Sw[3][3];
        int nd[3];
        for (int a = 0; a < 3; a++) {
            const int h = f[a] >= 0.5;
            nd[a] = ic[a] + h;
            shape3(f[a] - h, Sw[a]);
        }
        const double qw = qdv * (double)reinterpret_cast<const T*>(S.w)[t];
        // first tap in tile coordinates; the 3x3x3 block fits when all are in [0, T - 3]
        const int tx = nd[0] - 1 - o[0], ty = nd[1] - 1 - o[1], tz = nd[2] - 1 - o[2];
        const bool in = tiled && (unsigned)tx <= (unsigned)(TX - 3) &&
                        (unsigned)ty <= (unsigned)(TY - 3) && (unsigned)tz <= (unsigned)(TZ - 3);
        for (int c3 = 0; c3 < 3; c3++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    const double v = qw * Sw[0][a] * Sw[1][b] * Sw[2][c3];
                    if (in) {
                        atomicAdd(&tile[((tz + c3) * TY + ty + b) * TX + tx + a], v);
                    } else {
                        const long long g = node(nd[0] + a - 1, nd[1] + b - 1, nd[2] + c3 - 1);
                        if (g >= 0) atomicAdd(rho + g, v);
                    }
                }
    }
    if (!tiled) return;
    __syncthreads();
    for (int e = threadIdx.x; e < TX * TY * TZ; e += blockDim.x) {
        const double v = tile[e];
        if (v == 0.0) continue;
        const int ex = e % TX, ey = (e / TX) % TY, ez = e / (TX * TY);
        const long long g = node(o[0] + ex, o[1] + ey, o[2] + ez);
        if (g >= 0) atomicAdd(rho + g, v);
    }
}

template <typename T>
__global__ void gauss3d_kernel(const SimDev* __restrict__ sd) {
    const SimDev& S = *sd;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S.ncell) return;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const T* E = reinterpret_cast<const T*>(S.F[S.st->step & 1]);  // current time level
    const long long fs = S.fstride;
    const int im = i == 0 ? nx - 1 : i - 1, jm = j == 0 ? ny - 1 : j - 1, km = k == 0 ? nz - 1 : k - 1;
    const double exm = (S.window && i == 0) ? 0.0 : (double)E[pidx3(S, im, j, k)];
    const double div = ((double)E[pidx3(S, i, j, k)] - exm) / S.d[0] +
                       ((double)E[fs + pidx3(S, i, j, k)] - (double)E[fs + pidx3(S, i, jm, k)]) / S.d[1] +
                       ((double)E[2 * fs + pidx3(S, i, j, k)] - (double)E[2 * fs + pidx3(S, i, j, km)]) / S.d[2];
    S.rho[c] = div - S.rho[c] - S.rho_bg[c];
}

cudaError_t launch_gauss3d(const SimDev* sd, const SimDev& hs, int prec, int mode, cudaStream_t s) {
    double* target = mode == 0 ? hs.rho_bg : hs.rho;
    cudaError_t e = cudaMemsetAsync(target, 0, hs.ncell * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const double sign = mode == 0 ? -1.0 : 1.0;
    // the node tile of one patch in shared memory when the device grants it
    const size_t tile = (size_t)(hs.P[0] + 3) * (hs.P[1] + 3) * (hs.P[2] + 3) * sizeof(double);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int tiled = tile <= (size_t)optin ? 1 : 0;
    const size_t smem = tiled ? tile : 0;
    PIC_DISPATCH(prec, (cudaFuncSetAttribute(rho3d_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem),
                        rho3d_kernel<T><<<hs.npatch, 256, smem, s>>>(sd, target, sign, tiled)));
    if (mode == 1) {
        const unsigned g2 = (unsigned)((hs.ncell + 255) / 256);
        PIC_DISPATCH(prec, (gauss3d_kernel<T><<<g2, 256, 0, s>>>(sd)));
    }
    return cudaGetLastError();
}

}  // namespace pic
