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

// ---------------------------------------------------------------- splitting
//
// Load limiting in low-density cells (Sec. 3.2: SP are split where the SP density is
// low, merged where it is high). The oracle's rule: a cell holding n particles,
// 1 <= n < split_below, has its particles of weight >= 2 split_wmin, in increasing id,
// split until it holds split_below particles or each has been split once; a split keeps
// (x + delta, u, w/2) under the parent's id and adds (x - delta, u, w/2) with
// delta_a = min(f_a, 1 - f_a) d_a / 2, f_a the in-cell offset, so both halves stay in the
// cell. New ids are the next free id plus the split's rank in (patch, cell, parent id)
// order. Three passes: splits per patch (shared cell histograms), the id offsets (a scan
// over the patches, one CTA per sim), the splits themselves (counting sort of the slots
// by cell, one thread per cell sorting its few particles by id). All three return at
// once when a sim's split_below is 0.

template <typename T>
__device__ __forceinline__ bool split_eligible(const SimDev& S, int slot) {
    return to_f64(reinterpret_cast<const T*>(S.w)[slot]) >= 2.0 * S.split_wmin;
}

// splits of one cell from its particle and eligible counts
__device__ __forceinline__ int split_cell_count(int n, int e, int below) {
    return (n >= 1 && n < below) ? min(e, below - n) : 0;
}

template <typename T>
__global__ void __launch_bounds__(512) split_count_kernel(const BatchDev* __restrict__ bd) {
    __shared__ int cnt[kMergeCells];
    __shared__ int elig[kMergeCells];
    __shared__ int s_tot;
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int below = S.split_below;
    if (below <= 0) return;
    const int cells = S.P[0] * S.P[1] * S.P[2];
    if (cells > kMergeCells) return;
    const int tid = threadIdx.x;
    for (int p = blockIdx.x; p < S.npatch; p += gridDim.x) {
        __syncthreads();
        for (int c = tid; c < cells; c += blockDim.x) cnt[c] = 0, elig[c] = 0;
        if (tid == 0) s_tot = 0;
        __syncthreads();
        const int n = S.pcount[p], base = S.pbase[p];
        const int o[3] = {(p % S.np[0]) * S.P[0], ((p / S.np[0]) % S.np[1]) * S.P[1],
                          (p / (S.np[0] * S.np[1])) * S.P[2]};
        for (int k = tid; k < n; k += blockDim.x) {
            const int c = merge_local_cell<T>(S, base + k, o);
            atomicAdd(&cnt[c], 1);
            if (split_eligible<T>(S, base + k)) atomicAdd(&elig[c], 1);
        }
        __syncthreads();
        int m = 0;
        for (int c = tid; c < cells; c += blockDim.x) m += split_cell_count(cnt[c], elig[c], below);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
        if ((tid & 31) == 0 && m) atomicAdd(&s_tot, m);
        __syncthreads();
        if (tid == 0) S.soff[p] = s_tot;
    }
}

// soff[p] <- first free id + (splits of the patches before p); soff[npatch] <- the next
// free id. The column injected by this step's window shift already holds ids from
// next_id on (the end of the step advances next_id past them), so the first free id is
// past that column.
__global__ void __launch_bounds__(1024) split_scan_kernel(const BatchDev* __restrict__ bd) {
    __shared__ int warp_sums[32];
    const int sim = blockIdx.x;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    if (S.split_below <= 0) return;
    long long column = 0;
    if (S.st->shift) {
        column = (long long)S.n[1] * S.ippc[0] * S.ippc[1];
        if (S.dims == 3) column *= (long long)S.n[2] * S.ippc[2];
    }
    const long long first = S.st->next_id + column;
    long long carry = 0;
    for (int p0 = 0; p0 < S.npatch; p0 += blockDim.x) {
        const int p = p0 + threadIdx.x;
        const int v = p < S.npatch ? S.soff[p] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, warp_sums, &tot);
        if (p < S.npatch) S.soff[p] = (int)(first + carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        S.soff[S.npatch] = (int)(first + carry);
        S.st->next_id += carry;  // the end of the step adds the injected column
        S.st->nsplit += carry;
    }
}

// one split: the parent keeps its id at x + delta, the new particle (slot cs, id nid)
// goes to x - delta; both with half the weight and the parent's momentum
template <typename T>
__device__ void split_one(const SimDev& S, int s, int cs, int nid) {
    for (int a = 0; a < S.dims; a++) {
        T* X = reinterpret_cast<T*>(S.xi[a]);
        if constexpr (is_f64<T>::value) {
            const double xi = X[s];  // global cell-unit position
            const double fl = floor(xi);
            const double f = xi - fl;
            const double dl = 0.5 * fmin(f, 1.0 - f);
            double xp = xi + dl;
            if (floor(xp) != fl) xp = xi;  // rounding onto the next cell: keep the parent
            X[s] = xp;
            X[cs] = xi - dl;
        } else {
            const T f = X[s];  // in-cell offset in [0, 1)
            const T g = T(1.0f) - f;
            const T dl = T(0.5f) * (g < f ? g : f);
            T fp = f + dl;
            if (!(fp < T(1.0f))) fp = f;
            X[s] = fp;
            X[cs] = f - dl;
        }
    }
    if constexpr (uses_cell<T>()) S.cell[cs] = S.cell[s];
    for (int a = 0; a < 3; a++) {
        T* U = reinterpret_cast<T*>(S.u[a]);
        U[cs] = U[s];
    }
    T* W = reinterpret_cast<T*>(S.w);
    const T wh = W[s] * T(0.5f);
    W[s] = wh;
    W[cs] = wh;
    S.id[cs] = nid;
}

template <typename T>
__global__ void __launch_bounds__(512) split_apply_kernel(const BatchDev* __restrict__ bd) {
    extern __shared__ int sh[];  // start, cursor, new-particle offsets: kMergeCells each
    __shared__ int warp_sums[32];
    int* start = sh;
    int* cursor = sh + kMergeCells;
    int* coff = sh + 2 * kMergeCells;
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int below = S.split_below;
    if (below <= 0) return;
    const int cells = S.P[0] * S.P[1] * S.P[2];
    if (cells > kMergeCells) return;
    const int tid = threadIdx.x;
    int* ord = S.aid;  // scratch: slots in cell order
    for (int p = blockIdx.x; p < S.npatch; p += gridDim.x) {
        __syncthreads();
        const int total = S.soff[p + 1] - S.soff[p];
        if (total == 0) continue;  // uniform over the CTA
        const int n = S.pcount[p], base = S.pbase[p];
        if (n + total > S.pcap[p]) {  // no room for the new particles
            if (tid == 0) atomicOr(S.status, ST_CAPACITY);
            continue;
        }
        const int o[3] = {(p % S.np[0]) * S.P[0], ((p / S.np[0]) % S.np[1]) * S.P[1],
                          (p / (S.np[0] * S.np[1])) * S.P[2]};
        for (int c = tid; c < cells; c += blockDim.x) start[c] = 0, coff[c] = 0;
        __syncthreads();
        for (int k = tid; k < n; k += blockDim.x) {
            const int c = merge_local_cell<T>(S, base + k, o);
            atomicAdd(&start[c], 1);
            if (split_eligible<T>(S, base + k)) atomicAdd(&coff[c], 1);
        }
        __syncthreads();
        // per-cell splits, then exclusive prefixes of the counts (slot order) and of the
        // splits (new-particle order): a contiguous run of cells per thread, then a scan
        const int per = (cells + blockDim.x - 1) / blockDim.x;
        const int c0 = tid * per, c1 = min(c0 + per, cells);
        int run_n = 0, run_m = 0;
        for (int c = c0; c < c1; c++) {
            coff[c] = split_cell_count(start[c], coff[c], below);
            run_n += start[c];
            run_m += coff[c];
        }
        int tot_n, tot_m;
        int acc_n = block_exclusive_scan(run_n, warp_sums, &tot_n);
        int acc_m = block_exclusive_scan(run_m, warp_sums, &tot_m);
        for (int c = c0; c < c1; c++) {
            const int h = start[c], m = coff[c];
            start[c] = acc_n;
            cursor[c] = acc_n;
            coff[c] = acc_m;
            acc_n += h;
            acc_m += m;
        }
        __syncthreads();
        for (int k = tid; k < n; k += blockDim.x) {
            const int s = base + k;
            ord[base + atomicAdd(&cursor[merge_local_cell<T>(S, s, o)], 1)] = s;
        }
        __syncthreads();
        const int first_id = S.soff[p];
        for (int c = tid; c < cells; c += blockDim.x) {
            const int m = (c + 1 < cells ? coff[c + 1] : tot_m) - coff[c];
            if (m == 0) continue;
            const int nc = cursor[c] - start[c];  // < below <= 64
            int* q = ord + base + start[c];
            for (int i = 1; i < nc; i++) {  // by id
                const int x = q[i];
                int j = i - 1;
                while (j >= 0 && S.id[q[j]] > S.id[x]) {
                    q[j + 1] = q[j];
                    j--;
                }
                q[j + 1] = x;
            }
            int j = 0;
            for (int i = 0; i < nc && j < m; i++) {
                const int s = q[i];
                if (!split_eligible<T>(S, s)) continue;
                split_one<T>(S, s, base + n + coff[c] + j, first_id + coff[c] + j);
                j++;
            }
        }
        __syncthreads();
        if (tid == 0) S.pcount[p] = n + total;
    }
}

constexpr int kSplitDynSmem = 3 * kMergeCells * (int)sizeof(int);

cudaError_t split_setup() {
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < 3 && e == cudaSuccess; p++)
        PIC_DISPATCH(p, (e = cudaFuncSetAttribute(split_apply_kernel<T>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  kSplitDynSmem)));
    return e;
}

cudaError_t launch_split(const BatchDev* bd, int nsims, int max_patches, int prec,
                         cudaStream_t s) {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    dim3 grid(max_patches < 2 * nsm ? max_patches : 2 * nsm, nsims);
    PIC_DISPATCH(prec, (split_count_kernel<T><<<grid, 512, 0, s>>>(bd)));
    split_scan_kernel<<<nsims, 1024, 0, s>>>(bd);
    PIC_DISPATCH(prec, (split_apply_kernel<T><<<grid, 512, kSplitDynSmem, s>>>(bd)));
    return cudaGetLastError();
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
