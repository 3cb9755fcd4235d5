// Load limiting by particle merging (Sec. 3.2: the SP count of overloaded regions is
// bounded by merging SP; the paper gives no algorithm). Inside every patch holding more
// than merge_above particles, each group of N >= 3 particles sharing a cell and a
// momentum bin (floor(u_a / merge_dp) per axis) is replaced by two particles that keep
// the group's total weight W, momentum P and energy E, following the published merge
// of Vranic et al., Comput. Phys. Commun. 191 (2015) 65:
//   w = W/2 each, gamma = E/W each, momenta symmetric about P at the half angle theta,
//   cos(theta) = |P| / (W |u|).
// Free choices, the same as the oracle states: members in increasing id, the two
// smallest ids (and their positions) survive, the momenta lie in the plane of P and the
// smallest-id member's momentum (a coordinate axis when those are parallel, that
// momentum or the x axis when P = 0).
//
// A patch is merged when it holds more than merge_above particles and more than 5/4 of its
// count after its previous merge pass (the oracle's rule), so that patches merging cannot
// bring below the threshold are not reprocessed every step.
// One CTA per overloaded patch (grid-stride over patches), at the end of the step after
// the exchange: counting sort of the patch's slots by cell in shared memory, one thread
// per cell sorts its slots by (momentum bin, id) and merges the groups, then the holes
// left below the new count are filled from the tail. The arithmetic is FP64 for every
// precision (merges are rare; the results are stored back in the working precision).
#include <cuda_runtime.h>

#include "pic_device.cuh"
#include "pic_internal.h"

namespace pic {

template <typename T>
__device__ __forceinline__ double to_f64(T v) {
    return (double)v;
}
template <>
__device__ __forceinline__ double to_f64<float>(float v) {
    return widen_f32(v);
}

template <typename T>
__device__ __forceinline__ T from_f64(double v) {
    return T(v);
}

template <typename T>
__device__ __forceinline__ int merge_local_cell(const SimDev& S, int slot, const int o[3]) {
    int i[3] = {0, 0, 0};
    if constexpr (is_f64<T>::value) {
        for (int a = 0; a < S.dims; a++)
            i[a] = (int)floor(reinterpret_cast<const double*>(S.xi[a])[slot]);
    } else {
        const int c = S.cell[slot];
        if (S.dims == 2) {
            i[0] = c & 0xFFFF;
            i[1] = (c >> 16) & 0xFFFF;
        } else {
            i[0] = c & 0x7FF;
            i[1] = (c >> 11) & 0x7FF;
            i[2] = (c >> 22) & 0x3FF;
        }
    }
    int l[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        l[a] = i[a] - o[a];
        l[a] = l[a] < 0 ? 0 : (l[a] >= S.P[a] ? S.P[a] - 1 : l[a]);
    }
    return (l[2] * S.P[1] + l[1]) * S.P[0] + l[0];
}

// (bin x, bin y, bin z, id) of slot s, compared lexicographically
__device__ __forceinline__ bool merge_less(const int* bx, const int* by, const int* bz,
                                           const int* id, int s, int t) {
    if (bx[s] != bx[t]) return bx[s] < bx[t];
    if (by[s] != by[t]) return by[s] < by[t];
    if (bz[s] != bz[t]) return bz[s] < bz[t];
    return id[s] < id[t];
}

// Replace the group ord[0..m) (slots sorted by id) by two particles; marks the others
// as holes (id = -1).
template <typename T>
__device__ void merge_one_group(const SimDev& S, const int* ord, int m) {
    T* U[3] = {reinterpret_cast<T*>(S.u[0]), reinterpret_cast<T*>(S.u[1]),
               reinterpret_cast<T*>(S.u[2])};
    T* Wt = reinterpret_cast<T*>(S.w);
    double W = 0.0, P[3] = {0.0, 0.0, 0.0}, E = 0.0;
    for (int k = 0; k < m; k++) {
        const int s = ord[k];
        const double w = to_f64(Wt[s]);
        const double ux = to_f64(U[0][s]), uy = to_f64(U[1][s]), uz = to_f64(U[2][s]);
        W += w;
        P[0] += w * ux;
        P[1] += w * uy;
        P[2] += w * uz;
        E += w * sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    }
    const double gn = E / W;
    const double un = sqrt(fmax(gn * gn - 1.0, 0.0));
    const double pm = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    const int s0 = ord[0];
    const double r[3] = {to_f64(U[0][s0]), to_f64(U[1][s0]), to_f64(U[2][s0])};
    const double rm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double e1[3];
    if (pm > 0.0) {
        for (int i = 0; i < 3; i++) e1[i] = P[i] / pm;
    } else if (rm > 0.0) {
        for (int i = 0; i < 3; i++) e1[i] = r[i] / rm;
    } else {
        e1[0] = 1.0, e1[1] = 0.0, e1[2] = 0.0;
    }
    double v[3] = {r[0], r[1], r[2]};
    double dot = v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2];
    double t[3] = {v[0] - dot * e1[0], v[1] - dot * e1[1], v[2] - dot * e1[2]};
    double tm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    if (!(tm > 1e-12 * (rm > 0.0 ? rm : 1.0))) {  // reference parallel to P
        int ax = 0;
        for (int i = 1; i < 3; i++)
            if (fabs(e1[i]) < fabs(e1[ax])) ax = i;
        for (int i = 0; i < 3; i++) t[i] = (i == ax ? 1.0 : 0.0) - e1[ax] * e1[i];
        tm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    }
    double ct = un > 0.0 ? pm / (W * un) : 0.0;
    ct = ct > 1.0 ? 1.0 : ct;
    const double st = sqrt(1.0 - ct * ct);
    for (int i = 0; i < 3; i++) {
        const double e2 = t[i] / tm;
        U[i][ord[0]] = from_f64<T>(un * (ct * e1[i] + st * e2));
        U[i][ord[1]] = from_f64<T>(un * (ct * e1[i] - st * e2));
    }
    Wt[ord[0]] = from_f64<T>(0.5 * W);
    Wt[ord[1]] = from_f64<T>(0.5 * W);
    for (int k = 2; k < m; k++) S.id[ord[k]] = -1;
}

template <typename T>
__global__ void __launch_bounds__(512) merge_kernel(const BatchDev* __restrict__ bd) {
    __shared__ int start[kMergeCells];
    __shared__ int cursor[kMergeCells];
    __shared__ int warp_sums[32];
    __shared__ int s_removed, s_nh, s_nl;
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    if (S.merge_above <= 0) return;
    const int cells = S.P[0] * S.P[1] * S.P[2];
    if (cells > kMergeCells) return;
    const int tid = threadIdx.x;
    int* bx = reinterpret_cast<int*>(S.au[0]);  // scratch: momentum bins per slot
    int* by = reinterpret_cast<int*>(S.au[1]);
    int* bz = reinterpret_cast<int*>(S.au[2]);
    int* ord = S.aid;                            // scratch: slots in cell order
    for (int p = blockIdx.x; p < S.npatch; p += gridDim.x) {
        __syncthreads();  // the previous patch's shared state is no longer read
        const int n = S.pcount[p];
        // above the threshold and grown by a quarter since the patch's last merge pass
        const int last = S.mlast[p];
        if (n <= S.merge_above || n <= last + last / 4) continue;  // uniform over the CTA
        const int base = S.pbase[p];
        const int o[3] = {(p % S.np[0]) * S.P[0], ((p / S.np[0]) % S.np[1]) * S.P[1],
                          (p / (S.np[0] * S.np[1])) * S.P[2]};
        for (int c = tid; c < cells; c += blockDim.x) start[c] = 0;
        if (tid == 0) s_removed = 0, s_nh = 0, s_nl = 0;
        __syncthreads();
        const double idp = 1.0 / S.merge_dp;
        for (int k = tid; k < n; k += blockDim.x) {
            const int s = base + k;
            atomicAdd(&start[merge_local_cell<T>(S, s, o)], 1);
            const double u[3] = {to_f64(reinterpret_cast<const T*>(S.u[0])[s]),
                                 to_f64(reinterpret_cast<const T*>(S.u[1])[s]),
                                 to_f64(reinterpret_cast<const T*>(S.u[2])[s])};
            int b[3];
            for (int a = 0; a < 3; a++) {
                const double f = floor(u[a] * idp);
                b[a] = f < -1e9 ? -1000000000 : (f > 1e9 ? 1000000000 : (int)f);
            }
            bx[s] = b[0], by[s] = b[1], bz[s] = b[2];
        }
        __syncthreads();
        // exclusive prefix of the cell counts: a contiguous run per thread, then a scan
        const int per = (cells + blockDim.x - 1) / blockDim.x;
        const int c0 = tid * per, c1 = min(c0 + per, cells);
        int run = 0;
        for (int c = c0; c < c1; c++) run += start[c];
        int tot;
        int acc = block_exclusive_scan(run, warp_sums, &tot);
        for (int c = c0; c < c1; c++) {
            const int h = start[c];
            start[c] = acc;
            cursor[c] = acc;
            acc += h;
        }
        __syncthreads();
        for (int k = tid; k < n; k += blockDim.x) {
            const int s = base + k;
            ord[base + atomicAdd(&cursor[merge_local_cell<T>(S, s, o)], 1)] = s;
        }
        __syncthreads();
        // one thread per cell: sort its slots by (bin, id), merge the groups of >= 3
        for (int c = tid; c < cells; c += blockDim.x) {
            const int m = cursor[c] - start[c];
            if (m < 3) continue;
            int* q = ord + base + start[c];
            for (int i = 1; i < m; i++) {
                const int x = q[i];
                int j = i - 1;
                while (j >= 0 && merge_less(bx, by, bz, S.id, x, q[j])) {
                    q[j + 1] = q[j];
                    j--;
                }
                q[j + 1] = x;
            }
            int removed = 0;
            for (int i = 0; i < m;) {
                int j = i + 1;
                while (j < m && bx[q[j]] == bx[q[i]] && by[q[j]] == by[q[i]] && bz[q[j]] == bz[q[i]])
                    j++;
                if (j - i >= 3) {
                    merge_one_group<T>(S, q + i, j - i);
                    removed += j - i - 2;
                }
                i = j;
            }
            if (removed) atomicAdd(&s_removed, removed);
        }
        __syncthreads();
        const int removed = s_removed;
        if (tid == 0) S.mlast[p] = n - removed;
        if (removed == 0) continue;  // uniform
        // fill the holes below the new count with the live particles above it
        const int nn = n - removed;
        int* H = S.holes + base;
        int* L = ord + base;
        for (int k = tid; k < n; k += blockDim.x) {
            const int s = base + k;
            const bool hole = S.id[s] < 0;
            if (k < nn && hole) H[atomicAdd(&s_nh, 1)] = s;
            if (k >= nn && !hole) L[atomicAdd(&s_nl, 1)] = s;
        }
        __syncthreads();
        const int nm = min(s_nh, s_nl);
        for (int i = tid; i < nm; i += blockDim.x) {
            const int dst = H[i], src = L[i];
            if constexpr (uses_cell<T>()) S.cell[dst] = S.cell[src];
            for (int a = 0; a < S.dims; a++)
                reinterpret_cast<T*>(S.xi[a])[dst] = reinterpret_cast<const T*>(S.xi[a])[src];
            for (int a = 0; a < 3; a++)
                reinterpret_cast<T*>(S.u[a])[dst] = reinterpret_cast<const T*>(S.u[a])[src];
            reinterpret_cast<T*>(S.w)[dst] = reinterpret_cast<const T*>(S.w)[src];
            S.id[dst] = S.id[src];
            S.id[src] = -1;
        }
        if (tid == 0) {
            S.pcount[p] = nn;
            atomicAdd(reinterpret_cast<unsigned long long*>(&S.st->nmerged),
                      (unsigned long long)removed);
        }
        __syncthreads();
    }
}

cudaError_t launch_merge(const BatchDev* bd, int nsims, int max_patches, int prec,
                         cudaStream_t s) {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    dim3 grid(max_patches < 2 * nsm ? max_patches : 2 * nsm, nsims);
    PIC_DISPATCH(prec, (merge_kernel<T><<<grid, 512, 0, s>>>(bd)));
    return cudaGetLastError();
}

}  // namespace pic
