// Support kernels of one PIC step:
//   queue_build  - per-step work queue: patch chunks of at most `chunk` particles,
//                  full chunks first then remainders in descending size (an
//                  approximate longest-processing-time order), so the persistent
//                  particle kernel starts the heaviest work first (the single-GPU
//                  form of the patch load balancing of Sec. 3.1).
//   exchange     - moves particles that changed patch (and injected ones) into their
//                  new patch, filling the holes they left; one CTA per patch.
//   inject       - moving window: cold lattice column on the uncovered edge.
//   yee_e/yee_b  - Yee FDTD half-updates with the window shift folded into the write
//                  index, periodic guard cells, and zeroing of the next current buffer.
//   end_step     - advances the device-side step state.
//   diagnostics  - energy sums, charge deposition for Gauss's law, field unpadding.
#include <cuda_runtime.h>

#include "pic_device.cuh"
#include "pic_internal.h"
#include "fields.cuh"

namespace pic {

// ================================================================ work queue

__global__ void __launch_bounds__(kQueueThreads) queue_build_kernel(const BatchDev* __restrict__ bd) {
    __shared__ int warp_sums[32];
    __shared__ int bucket_cnt[kBuckets];
    __shared__ int bucket_off[kBuckets];
    __shared__ int s_full_total;
    const int tid = threadIdx.x;
    const int nsims = bd->nsims;
    const int chunk = bd->chunk;
    const int total = bd->total_patches;
    const int static_map = bd->sims[0].mapping == 1;

    // begin-of-step state per sim: shift decision and buffer generation
    for (int s = tid; s < nsims; s += blockDim.x) {
        StepState* st = bd->sims[s].st;
        const SimDev& S = bd->sims[s];
        const long long n = st->step;
        int shift = 0;
        if (S.window) {
            const double a = floor((double)(n + 1) * S.dt / S.d[0]);
            const double b = floor((double)n * S.dt / S.d[0]);
            shift = a > b;
        }
        st->shift = shift;
        st->gen = (int)(n & 1);
    }
    for (int b = tid; b < kBuckets; b += blockDim.x) bucket_cnt[b] = 0;
    __syncthreads();
    // pass 1: full chunks (scan-ordered by global patch index) + remainder histogram
    int carry = 0;
    for (int g0 = 0; g0 < total; g0 += blockDim.x) {
        const int g = g0 + tid;
        int sim = 0, p = 0, cnt = 0;
        if (g < total) {
            while (sim + 1 < nsims && bd->patch_prefix[sim + 1] <= g) sim++;
            p = g - bd->patch_prefix[sim];
            cnt = bd->sims[sim].pcount[p];
        }
        int full = static_map ? 0 : cnt / chunk;
        int tot;
        const int ex = block_exclusive_scan(full, warp_sums, &tot);
        for (int c = 0; c < full; c++) {
            const int pos = carry + ex + c;
            if (pos < bd->max_items) bd->items[pos] = make_int4(sim, p, c * chunk, chunk);
        }
        if (!static_map) {
            const int rem = cnt - full * chunk;
            if (rem > 0) {
                const int b = kBuckets - 1 - (int)((long long)rem * kBuckets / (chunk + 1));
                atomicAdd(&bucket_cnt[b < 0 ? 0 : b], 1);
            }
        }
        carry += tot;
    }
    if (tid == 0) s_full_total = carry;
    __syncthreads();
    if (static_map) {
        // one item per non-empty patch, in patch order
        int c2 = 0;
        for (int g0 = 0; g0 < total; g0 += blockDim.x) {
            const int g = g0 + tid;
            int sim = 0, p = 0, cnt = 0;
            if (g < total) {
                while (sim + 1 < nsims && bd->patch_prefix[sim + 1] <= g) sim++;
                p = g - bd->patch_prefix[sim];
                cnt = bd->sims[sim].pcount[p];
            }
            int tot;
            const int ex = block_exclusive_scan(cnt > 0, warp_sums, &tot);
            if (cnt > 0 && c2 + ex < bd->max_items) bd->items[c2 + ex] = make_int4(sim, p, 0, cnt);
            c2 += tot;
        }
        if (tid == 0) {
            *bd->nitems = c2 < bd->max_items ? c2 : bd->max_items;
            if (c2 > bd->max_items) atomicOr(bd->sims[0].status, ST_QUEUE);
            *bd->head = 0;
        }
        return;
    }
    if (tid == 0) {
        int acc = s_full_total;
        for (int b = 0; b < kBuckets; b++) {
            bucket_off[b] = acc;
            acc += bucket_cnt[b];
        }
        *bd->nitems = acc < bd->max_items ? acc : bd->max_items;
        if (acc > bd->max_items) atomicOr(bd->sims[0].status, ST_QUEUE);
        *bd->head = 0;
    }
    __syncthreads();
    // pass 2: remainder chunks into their bucket (largest bucket first)
    for (int g = tid; g < total; g += blockDim.x) {
        int sim = 0;
        while (sim + 1 < nsims && bd->patch_prefix[sim + 1] <= g) sim++;
        const int p = g - bd->patch_prefix[sim];
        const int cnt = bd->sims[sim].pcount[p];
        const int full = cnt / chunk;
        const int rem = cnt - full * chunk;
        if (rem > 0) {
            int b = kBuckets - 1 - (int)((long long)rem * kBuckets / (chunk + 1));
            b = b < 0 ? 0 : b;
            const int pos = atomicAdd(&bucket_off[b], 1);
            if (pos < bd->max_items) bd->items[pos] = make_int4(sim, p, full * chunk, rem);
        }
    }
}

cudaError_t launch_queue_build(const BatchDev* bd, cudaStream_t s) {
    queue_build_kernel<<<1, kQueueThreads, 0, s>>>(bd);
    return cudaGetLastError();
}

// ================================================================ exchange

template <typename T>
__device__ __forceinline__ void copy_particle(const SimDev& S, int dims, int dst, int src,
                                              bool from_mailbox) {
    if (from_mailbox) {
        if constexpr (uses_cell<T>()) S.cell[dst] = S.mcell[src];
        for (int a = 0; a < dims; a++)
            reinterpret_cast<T*>(S.xi[a])[dst] = reinterpret_cast<const T*>(S.mxi[a])[src];
        for (int a = 0; a < 3; a++)
            reinterpret_cast<T*>(S.u[a])[dst] = reinterpret_cast<const T*>(S.mu[a])[src];
        reinterpret_cast<T*>(S.w)[dst] = reinterpret_cast<const T*>(S.mw)[src];
        S.id[dst] = S.mid[src];
    } else {
        if constexpr (uses_cell<T>()) S.cell[dst] = S.cell[src];
        for (int a = 0; a < dims; a++)
            reinterpret_cast<T*>(S.xi[a])[dst] = reinterpret_cast<const T*>(S.xi[a])[src];
        for (int a = 0; a < 3; a++)
            reinterpret_cast<T*>(S.u[a])[dst] = reinterpret_cast<const T*>(S.u[a])[src];
        reinterpret_cast<T*>(S.w)[dst] = reinterpret_cast<const T*>(S.w)[src];
        S.id[dst] = S.id[src];
    }
}

// One CTA per patch. Holes (slots of particles that left, id = -1) below the new
// count are filled first with arrivals from the mailbox, then with live particles
// moved down from the tail; extra arrivals are appended.
template <typename T>
__global__ void __launch_bounds__(256) exchange_kernel(const BatchDev* __restrict__ bd) {
    __shared__ int warp_sums[32];
    __shared__ int s_n, s_nh, s_nm, s_new;
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    const int p = blockIdx.x;
    if (p >= S.npatch) return;
    const int tid = threadIdx.x;
    const int base = S.pbase[p];
    if (tid == 0) {
        const int n = S.pcount[p];
        const int nh = S.hcount[p];
        int nm = S.mcount[p];
        const int mc = S.mcap[p];
        if (nm > mc) nm = mc;
        const int cap = S.pcap[p];
        // arrivals beyond the free room stay in the exchange buffer; the repack at the
        // end of this step enlarges the patch and places them
        const int room = cap - (n - nh);
        int pend = 0;
        if (nm > room) {
            pend = nm - room;
            nm = room;
        }
        S.mpend[p] = pend;
        S.mpoff[p] = nm;
        const int nn = n - nh + nm;
        // ask for a repack before a patch or its exchange buffer runs out
        if (pend > 0 || nn > cap - cap / 8 - 16 || S.mcount[p] > mc / 4) atomicOr(&S.st->repack, 1);
        s_n = n;
        s_nh = nh;
        s_nm = nm;
        s_new = nn;
        S.hcount[p] = 0;
        S.mcount[p] = 0;
        S.pcount[p] = nn;
    }
    __syncthreads();
    const int n = s_n, nh = s_nh, nm = s_nm, nn = s_new;
    if (nh == 0 && nm == 0) return;
    int* holes = S.holes + base;
    int* aux = S.aux + base;
    const int mb = S.mbase[p];

    // targets T1: holes below the new count, compacted into aux[0..t1)
    int t1 = 0;
    for (int k0 = 0; k0 < nh; k0 += blockDim.x) {
        const int k = k0 + tid;
        int h = -1;
        if (k < nh) h = holes[k];
        const bool keep = k < nh && (h - base) < nn;
        int tot;
        const int ex = block_exclusive_scan(keep, warp_sums, &tot);
        if (keep) aux[t1 + ex] = h;
        t1 += tot;
    }
    __syncthreads();
    // sources S2: live slots in [nn, n), compacted into holes[0..s2)
    int s2 = 0;
    for (int k0 = nn; k0 < n; k0 += blockDim.x) {
        const int k = k0 + tid;
        const bool live = k < n && S.id[base + k] >= 0;
        int tot;
        const int ex = block_exclusive_scan(live, warp_sums, &tot);
        if (live) holes[s2 + ex] = base + k;
        s2 += tot;
    }
    __syncthreads();
    const int ntarget = t1 + (nn > n ? nn - n : 0);
    for (int k = tid; k < ntarget; k += blockDim.x) {
        const int dst = k < t1 ? aux[k] : base + n + (k - t1);
        if (k < nm)
            copy_particle<T>(S, S.dims, dst, mb + k, true);
        else if (k - nm < s2)
            copy_particle<T>(S, S.dims, dst, holes[k - nm], false);
    }
}

cudaError_t launch_exchange(const BatchDev* bd, int nsims, int max_patches, int prec,
                            cudaStream_t s) {
    dim3 grid(max_patches, nsims);
    PIC_DISPATCH(prec, (exchange_kernel<T><<<grid, 256, 0, s>>>(bd)));
    return cudaGetLastError();
}

// ================================================================ moving-window injection

// Lattice point t of the uncovered column (2D: ny cells, 3D: ny x nz cells): row j
// varies fastest so that the lanes of a warp sit in different cells (no shared-memory
// atomic collisions in the next push). Lattice index (id offset) =
// (((k ny + j) pz + c) py + b) px + a, the oracle's order.
template <typename T>
__global__ void inject_kernel(const BatchDev* __restrict__ bd) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    if (!S.window || !S.st->shift) return;
    const bool d3 = S.dims == 3;
    const int nx = S.n[0], ny = S.n[1], nz = d3 ? S.n[2] : 1;
    const int px = S.ippc[0], py = S.ippc[1], pz = d3 ? S.ippc[2] : 1;
    const long long npts = (long long)ny * nz * px * py * pz;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= npts) return;
    const int j = (int)(t % ny);
    long long r = t / ny;
    const int k = (int)(r % nz);
    r /= nz;
    const int cz = (int)(r % pz);
    r /= pz;
    const int b = (int)(r % py);
    const int a = (int)(r / py);
    const double dx = S.d[0];
    const double xw = ((double)(nx - 1) + ((double)a + 0.5) / px) * dx;
    const double xl = xw + (double)(S.st->nshift + 1) * dx;
    double f = (xl - S.ramp_x0) / S.ramp_len;
    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
    const double dens = S.n0 * f;
    if (!(dens > 0.0)) return;
    const double dV = dx * S.d[1] * (d3 ? S.d[2] : 1.0);
    const double wgt = dens * dV / ((double)px * py * pz);
    const long long lat = ((((long long)k * ny + j) * pz + cz) * py + b) * px + a;
    const int dest = ((nx - 1) / S.P[0]) + S.np[0] * (j / S.P[1] + S.np[1] * (k / S.P[2]));
    // one claim per destination among the warp's remaining lanes (consecutive rows
    // share a patch), instead of one global atomic per particle
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, dest);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int first = 0;
    if (lane == leader) first = atomicAdd(S.mcount + dest, __popc(peers));
    first = __shfl_sync(peers, first, leader);
    const int slot = first + __popc(peers & ((1u << lane) - 1u));
    if (slot >= S.mcap[dest]) {
        atomicOr(S.status, ST_MAILBOX);
        return;
    }
    const int m = S.mbase[dest] + slot;
    const double ox = ((double)a + 0.5) / px, oy = ((double)b + 0.5) / py,
                 oz = ((double)cz + 0.5) / pz;
    if constexpr (is_f64<T>::value) {
        reinterpret_cast<double*>(S.mxi[0])[m] = (double)(nx - 1) + ox;
        reinterpret_cast<double*>(S.mxi[1])[m] = (double)j + oy;
        if (d3) reinterpret_cast<double*>(S.mxi[2])[m] = (double)k + oz;
    } else {
        S.mcell[m] = d3 ? ((nx - 1) | (j << 11) | (k << 22)) : ((nx - 1) | (j << 16));
        reinterpret_cast<T*>(S.mxi[0])[m] = T(ox);
        reinterpret_cast<T*>(S.mxi[1])[m] = T(oy);
        if (d3) reinterpret_cast<T*>(S.mxi[2])[m] = T(oz);
    }
    reinterpret_cast<T*>(S.mu[0])[m] = T(0);
    reinterpret_cast<T*>(S.mu[1])[m] = T(0);
    reinterpret_cast<T*>(S.mu[2])[m] = T(0);
    reinterpret_cast<T*>(S.mw)[m] = (T)wgt;
    S.mid[m] = (int)(S.st->next_id + lat);
}

cudaError_t launch_inject(const BatchDev* bd, int nsims, int max_column_pts, int prec,
                          cudaStream_t s) {
    if (max_column_pts <= 0) return cudaSuccess;
    dim3 grid((max_column_pts + 255) / 256, nsims);
    PIC_DISPATCH(prec, (inject_kernel<T><<<grid, 256, 0, s>>>(bd)));
    return cudaGetLastError();
}

// ================================================================ Yee (2D)

// E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2}); output written shifted by the
// window shift of this step; the next step's current buffer is zeroed.
template <typename T>
__global__ void __launch_bounds__(256) yee_e2d_kernel(const BatchDev* __restrict__ bd) {
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
    const T* Hin = reinterpret_cast<const T*>(S.H[g]);
    const double* Jin = S.J[g];
    double* Jnext = S.J[1 - g];
    const long long po = (long long)(oy + kGuard) * NX + (ox + kGuard);
    Jnext[po] = 0.0;
    Jnext[fs + po] = 0.0;
    Jnext[2 * fs + po] = 0.0;
    const int i = ox + s, j = oy;
    T ex = T(0), ey = T(0), ez = T(0);
    if (i < nx) {
        using C = FieldConst<T>;
        const T dt = C::dt(S), idx_ = C::id(S, 0), idy = C::id(S, 1);
        const int jm = j == 0 ? ny - 1 : j - 1;
        const bool has_im = !(win && i == 0);
        const int im = i == 0 ? nx - 1 : i - 1;
        auto at = [&](const T* a, int c, int ii, int jj) {
            return a[c * fs + (long long)(jj + kGuard) * NX + (ii + kGuard)];
        };
        const long long pi = (long long)(j + kGuard) * NX + (i + kGuard);
        const T bz = at(Hin, 2, i, j), bzjm = at(Hin, 2, i, jm);
        const T bzim = has_im ? at(Hin, 2, im, j) : T(0);
        const T by = at(Hin, 1, i, j), byim = has_im ? at(Hin, 1, im, j) : T(0);
        const T bx = at(Hin, 0, i, j), bxjm = at(Hin, 0, i, jm);
        ex = Ein[pi] + dt * ((bz - bzjm) * idy - C::cur(Jin[pi]));
        ey = Ein[fs + pi] + dt * (-(bz - bzim) * idx_ - C::cur(Jin[fs + pi]));
        ez = Ein[2 * fs + pi] +
             dt * ((by - byim) * idx_ - (bx - bxjm) * idy - C::cur(Jin[2 * fs + pi]));
    }
    put2d(Eout, NX, ox, oy, nx, ny, !win, ex);
    put2d(Eout + fs, NX, ox, oy, nx, ny, !win, ey);
    put2d(Eout + 2 * fs, NX, ox, oy, nx, ny, !win, ez);
}

// B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1};  B^{n+1} = (B^{n+1/2} + B^{n+3/2}) / 2.
template <typename T>
__global__ void __launch_bounds__(256) yee_b2d_kernel(const BatchDev* __restrict__ bd) {
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
    const T* E = reinterpret_cast<const T*>(S.F[1 - g]);  // E^{n+1}, output frame
    T* Bn = reinterpret_cast<T*>(S.F[1 - g]) + 3 * fs;
    const T* Hin = reinterpret_cast<const T*>(S.H[g]);
    T* Hout = reinterpret_cast<T*>(S.H[1 - g]);
    const int i = ox + s, j = oy;
    T hx = T(0), hy = T(0), hz = T(0), nbx = T(0), nby = T(0), nbz = T(0);
    if (i < nx) {
        using C = FieldConst<T>;
        const T dt = C::dt(S), idx_ = C::id(S, 0), idy = C::id(S, 1);
        auto at = [&](const T* a, int c, int ii, int jj) {
            return a[c * fs + (long long)(jj + kGuard) * NX + (ii + kGuard)];
        };
        const int jp = oy == ny - 1 ? 0 : oy + 1;
        const bool has_ip = !(win && ox + 1 >= nx);
        const int ip = ox + 1 >= nx ? 0 : ox + 1;
        const T ez = at(E, 2, ox, oy), ezjp = at(E, 2, ox, jp);
        const T ezip = has_ip ? at(E, 2, ip, oy) : T(0);
        const T ey = at(E, 1, ox, oy), eyip = has_ip ? at(E, 1, ip, oy) : T(0);
        const T ex = at(E, 0, ox, oy), exjp = at(E, 0, ox, jp);
        const T h0x = at(Hin, 0, i, j), h0y = at(Hin, 1, i, j), h0z = at(Hin, 2, i, j);
        hx = h0x - dt * ((ezjp - ez) * idy);
        hy = h0y + dt * ((ezip - ez) * idx_);
        hz = h0z - dt * ((eyip - ey) * idx_ - (exjp - ex) * idy);
        nbx = T(0.5) * (h0x + hx);
        nby = T(0.5) * (h0y + hy);
        nbz = T(0.5) * (h0z + hz);
    }
    const long long po = (long long)(oy + kGuard) * NX + (ox + kGuard);
    Hout[po] = hx;
    Hout[fs + po] = hy;
    Hout[2 * fs + po] = hz;
    put2d(Bn, NX, ox, oy, nx, ny, !win, nbx);
    put2d(Bn + fs, NX, ox, oy, nx, ny, !win, nby);
    put2d(Bn + 2 * fs, NX, ox, oy, nx, ny, !win, nbz);
}

cudaError_t launch_yee(const BatchDev* bd, int nsims, int max_ncell, int dims, int prec,
                       int order, cudaStream_t s) {
    if (order == 6) return launch_maxwell6(bd, nsims, max_ncell, dims, prec, s);
    if (dims == 3) return launch_yee3d(bd, nsims, max_ncell, prec, s);
    if (dims != 2) return cudaErrorInvalidValue;
    dim3 grid((max_ncell + 255) / 256, nsims);
    PIC_DISPATCH(prec, (yee_e2d_kernel<T><<<grid, 256, 0, s>>>(bd), yee_b2d_kernel<T><<<grid, 256, 0, s>>>(bd)));
    return cudaGetLastError();
}

// ================================================================ capacity repack

// New per-patch capacities from the current counts (free slots shared half by count,
// half evenly, each rounded up to kSlotAlign, as at load) and their prefix bases. One
// CTA per sim.
__global__ void __launch_bounds__(1024) repack_plan_kernel(const BatchDev* __restrict__ bd) {
    __shared__ int warp_sums[32];
    __shared__ long long s_total;
    const SimDev& S = bd->sims[blockIdx.x];
    if (blockIdx.x >= bd->nsims || !S.st->repack) return;
    const int tid = threadIdx.x;
    if (tid == 0) s_total = 0;
    __syncthreads();
    long long part = 0;
    for (int p = tid; p < S.npatch; p += blockDim.x) part += S.pcount[p] + S.mpend[p];
    atomicAdd((unsigned long long*)&s_total, (unsigned long long)part);
    __syncthreads();
    const long long N = s_total;
    if (N > S.ucap) {  // more particles (with pending arrivals) than the capacity
        if (tid == 0) {
            atomicOr(S.status, ST_CAPACITY);
            S.st->repack = 2;
        }
        return;
    }
    const double spare = (double)(S.ucap - N);
    int carry = 0, mcarry = 0;
    for (int p0 = 0; p0 < S.npatch; p0 += blockDim.x) {
        const int p = p0 + tid;
        int cap = 0, mc = 0;
        if (p < S.npatch) {
            const int c = S.pcount[p] + S.mpend[p];
            const double share = N > 0 ? 0.5 * (double)c / (double)N + 0.5 / S.npatch : 1.0 / S.npatch;
            cap = (int)align_slots(c + (long long)floor(spare * share));
            // exchange buffer: half the capacity, at least kMailboxMin, and at least four
            // times the arrivals of this step (placed + pending): a patch flooded from
            // denser neighbours gets room even while its own count is still small, and the
            // arrivals may grow fourfold before the next repack (triggered at a quarter)
            const int arr = S.mpoff[p] + S.mpend[p];
            mc = cap / kMailboxDiv > kMailboxMin ? cap / kMailboxDiv : kMailboxMin;
            mc = (int)align_slots(mc > 4 * arr ? mc : 4 * arr);
        }
        int tot, mtot;
        const int ex = block_exclusive_scan(cap, warp_sums, &tot);
        const int mex = block_exclusive_scan(mc, warp_sums, &mtot);
        if (p < S.npatch) {
            S.pcap_new[p] = cap;
            S.pbase_new[p] = carry + ex;
            S.mcap_new[p] = mc;
            S.mbase_new[p] = mcarry + mex;
        }
        carry += tot;
        mcarry += mtot;
    }
    if (tid == 0 && (carry > S.capacity || mcarry > S.mtotal)) {
        atomicOr(S.status, ST_CAPACITY);
        S.st->repack = 2;  // failed: keep the current layout, drop the pending arrivals
    }
}

// Live particles of patch p -> scratch buffer at the new base (move), then back to
// the primary arrays at the same new offsets (back).
template <typename T>
__global__ void __launch_bounds__(256) repack_copy_kernel(const BatchDev* __restrict__ bd, int back) {
    const int sim = blockIdx.y;
    if (sim >= bd->nsims) return;
    const SimDev& S = bd->sims[sim];
    if (S.st->repack != 1) return;  // the usual case: a small grid that exits at once
    for (int p = blockIdx.x; p < S.npatch; p += gridDim.x) {
    const int cnt = S.pcount[p];
    const int from = back ? S.pbase_new[p] : S.pbase[p];
    const int to = S.pbase_new[p];
    const int pend = S.mpend[p];
    if ((long long)to + cnt + pend > S.capacity || (long long)from + cnt > S.capacity) continue;
    if (back && pend > 0) {  // arrivals that did not fit before: append after the live ones
        const int m0 = S.mbase[p] + S.mpoff[p];
        for (int k = threadIdx.x; k < pend; k += blockDim.x)
            copy_particle<T>(S, S.dims, to + cnt + k, m0 + k, true);
    }
    const int dims = S.dims;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int a0 = from + k, b0 = to + k;
        if (back) {
            if constexpr (uses_cell<T>()) S.cell[b0] = S.acell[a0];
            for (int a = 0; a < dims; a++)
                reinterpret_cast<T*>(S.xi[a])[b0] = reinterpret_cast<const T*>(S.axi[a])[a0];
            for (int a = 0; a < 3; a++)
                reinterpret_cast<T*>(S.u[a])[b0] = reinterpret_cast<const T*>(S.au[a])[a0];
            reinterpret_cast<T*>(S.w)[b0] = reinterpret_cast<const T*>(S.aw)[a0];
            S.id[b0] = S.aid[a0];
        } else {
            if constexpr (uses_cell<T>()) S.acell[b0] = S.cell[a0];
            for (int a = 0; a < dims; a++)
                reinterpret_cast<T*>(S.axi[a])[b0] = reinterpret_cast<const T*>(S.xi[a])[a0];
            for (int a = 0; a < 3; a++)
                reinterpret_cast<T*>(S.au[a])[b0] = reinterpret_cast<const T*>(S.u[a])[a0];
            reinterpret_cast<T*>(S.aw)[b0] = reinterpret_cast<const T*>(S.w)[a0];
            S.aid[b0] = S.id[a0];
        }
    }
    }
}

cudaError_t launch_repack(const BatchDev* bd, int nsims, int max_patches, int prec,
                          cudaStream_t s) {
    repack_plan_kernel<<<nsims, 1024, 0, s>>>(bd);
    // CTAs loop over patches: eight per SM keep enough loads in flight to copy at full
    // bandwidth, and an idle step (no repack) launches only those
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    dim3 grid(max_patches < 8 * nsm ? max_patches : 8 * nsm, nsims);
    for (int back = 0; back < 2; back++) {
        PIC_DISPATCH(prec, (repack_copy_kernel<T><<<grid, 256, 0, s>>>(bd, back)));
    }
    return cudaGetLastError();
}

// ================================================================ failure-path self-test

// One CTA waits, through the kernels' bounded wait, on an mbarrier phase that no
// transfer and no thread completes, and latches ST_TIMEOUT when the wait gives up.
__global__ void bounded_wait_selftest_kernel(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

cudaError_t launch_bounded_wait_selftest(int* status, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

// ================================================================ particle load

// Offset of a particle in its cell, f in [0, 1), in a cell-based precision: rounding
// to float32 (or to the double-word's leading float) must not reach 1.
template <typename T>
__device__ __forceinline__ T offset_below_one(double f) {
    const T g(f);
    if constexpr (std::is_same<T, df64>::value) {
        if (g.hi >= 1.0f) return T(nextafterf(1.0f, 0.0f));
    } else {
        if (g >= 1.0f) return T(nextafterf(1.0f, 0.0f));
    }
    return g;
}

// ================================================================ particle load
// The caller's FP64 arrays are staged chunk by chunk in the repack scratch as they are
// (positions in axi, momenta in au, weights in aw, ids in aid); chunk index k holds the
// call's particle k0 + k. Three passes place them.

// Pass 1, per particle: validation (the first invalid particle of the call by index, with
// its reason: 1 a position outside the grid, 2 a non-finite momentum or weight, 3 a
// negative id), its patch, the shared-memory bank class of its cell in the patch's field
// tile (the tile address modulo 32), and its rank among the particles of the same patch
// and class (an atomic add on that pair's counter). Writes the key patch * 32 + class to
// holes[k0 + k] and the rank to aux[k0 + k]. The counters are npatch x 32 ints in the
// Gauss scratch rho (zeroed by the caller); red holds {first invalid (index << 2 |
// reason), largest id, largest |w| as its bits}, set to {~0, 0, 0} by the caller. None of
// these is live state between steps, so a rejected load leaves the sim as it was.
__global__ void __launch_bounds__(256) load_bin_kernel(const BatchDev* __restrict__ bd,
                                                       long long m, long long k0) {
    const SimDev& S = bd->sims[0];
    int* cnt = reinterpret_cast<int*>(S.rho);
    unsigned long long* red = reinterpret_cast<unsigned long long*>(S.red);
    int idmax = 0;
    unsigned long long wmax = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        const long long p = k0 + k;
        int ic[3] = {0, 0, 0};
        int code = 0;
        for (int a = 0; a < S.dims; a++) {
            const double v = reinterpret_cast<const double*>(S.axi[a])[k];
            if (!isfinite(v) || v < 0.0 || v >= S.n[a] * S.d[a]) {
                code = 1;
                break;
            }
            ic[a] = (int)floor(cell_coord(v, S.d[a], S.n[a]));
        }
        const double w = reinterpret_cast<const double*>(S.aw)[k];
        if (!code && (!isfinite(reinterpret_cast<const double*>(S.au[0])[k]) ||
                      !isfinite(reinterpret_cast<const double*>(S.au[1])[k]) ||
                      !isfinite(reinterpret_cast<const double*>(S.au[2])[k]) || !isfinite(w)))
            code = 2;
        const int id = S.aid[k];
        if (!code && id < 0) code = 3;
        if (code) {
            atomicMin(&red[0], ((unsigned long long)p << 2) | (unsigned long long)code);
            continue;
        }
        idmax = max(idmax, id);
        wmax = max(wmax, (unsigned long long)__double_as_longlong(fabs(w)));
        const int pc[3] = {ic[0] / S.P[0], ic[1] / S.P[1], ic[2] / S.P[2]};
        const int pp = pc[0] + S.np[0] * (pc[1] + S.np[1] * pc[2]);
        const int lx = ic[0] - pc[0] * S.P[0], ly = ic[1] - pc[1] * S.P[1];
        const int lz = ic[2] - pc[2] * S.P[2];
        const int key = pp * 32 + (((lz * S.BY + ly) * S.BX + lx) & 31);
        S.holes[p] = key;
        S.aux[p] = atomicAdd(&cnt[key], 1);
    }
    // largest id and |w| of the CTA, then one atomic each
    __shared__ int s_id[32];
    __shared__ unsigned long long s_w[32];
    idmax = __reduce_max_sync(0xffffffffu, idmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_down_sync(0xffffffffu, wmax, o);
        wmax = x > wmax ? x : wmax;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_id[wid] = idmax;
        s_w[wid] = wmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            idmax = max(idmax, s_id[i]);
            wmax = s_w[i] > wmax ? s_w[i] : wmax;
        }
        atomicMax(&red[1], (unsigned long long)idmax);
        atomicMax(&red[2], wmax);
    }
}

// Pass 2, per particle of the call: its slot, the patch's base plus its place in the run
// order (run r holds the r-th particle of every class present in the patch, classes in
// order), so that the lanes of a warp read and add into different banks. The rank is
// scrambled by a fixed bijection of [0, class count), r -> r * 1000003 mod count (the
// multiplier is prime, so coprime to any smaller count): particles of one cell, which
// tend to take consecutive ranks, land in different runs.
__global__ void __launch_bounds__(256) load_slot_kernel(const BatchDev* __restrict__ bd,
                                                        long long n) {
    const SimDev& S = bd->sims[0];
    const int* cnt = reinterpret_cast<const int*>(S.rho);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int key = S.holes[p];
        const int pp = key >> 5, q = key & 31;
        const int* nb = cnt + pp * 32;
        const int c = nb[q];
        int r = S.aux[p];
        if (c < 1000003) r = (int)(((long long)r * 1000003LL) % c);
        int off = 0;
#pragma unroll 8
        for (int t = 0; t < 32; t++) {
            const int x = nb[t];
            off += min(x, r) + ((t < q && x > r) ? 1 : 0);
        }
        S.holes[p] = S.pbase[pp] + off;
    }
}

// Pass 3, one chunk: each particle converted to the sim's representation (FP64: position
// in cell units; FP32 and double-word: the packed cell index plus the offset in the cell)
// and stored in its slot holes[k0 + k]. Free slots were cleared beforehand (id -1).
template <typename T>
__global__ void __launch_bounds__(256) load_scatter_kernel(const BatchDev* __restrict__ bd,
                                                           long long m, long long k0) {
    const SimDev& S = bd->sims[0];
    const int dims = S.dims;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        const long long dst = S.holes[k0 + k];
        int cellv = 0;
        for (int a = 0; a < dims; a++) {
            const double c =
                cell_coord(reinterpret_cast<const double*>(S.axi[a])[k], S.d[a], S.n[a]);
            if constexpr (uses_cell<T>()) {
                const int i = (int)floor(c);
                reinterpret_cast<T*>(S.xi[a])[dst] = offset_below_one<T>(c - (double)i);
                cellv |= i << (dims == 2 ? 16 * a : 11 * a);
            } else {
                reinterpret_cast<T*>(S.xi[a])[dst] = T(c);
            }
        }
        if constexpr (uses_cell<T>()) S.cell[dst] = cellv;
#pragma unroll
        for (int a = 0; a < 3; a++)
            reinterpret_cast<T*>(S.u[a])[dst] = T(reinterpret_cast<const double*>(S.au[a])[k]);
        reinterpret_cast<T*>(S.w)[dst] = T(reinterpret_cast<const double*>(S.aw)[k]);
        S.id[dst] = S.aid[k];
    }
}

static int elementwise_grid(long long n) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    const long long want = (n + 255) / 256;
    return (int)(want < 8LL * nsm ? want : 8LL * nsm);
}

cudaError_t launch_load_bin(const BatchDev* bd, long long m, long long k0, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    load_bin_kernel<<<elementwise_grid(m), 256, 0, s>>>(bd, m, k0);
    return cudaGetLastError();
}

cudaError_t launch_load_slot(const BatchDev* bd, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    load_slot_kernel<<<elementwise_grid(n), 256, 0, s>>>(bd, n);
    return cudaGetLastError();
}

cudaError_t launch_load_scatter(const BatchDev* bd, long long m, long long k0, int prec,
                                cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int grid = elementwise_grid(m);
    PIC_DISPATCH(prec, (load_scatter_kernel<T><<<grid, 256, 0, s>>>(bd, m, k0)));
    return cudaGetLastError();
}

// Field load: the caller's E (staged in J[0]) and B (in J[1]), three arrays of ncell
// values each with x fastest, to the padded arrays of generation 0 in the sim's
// precision: F holds E then B, H holds B. Guard cells take the periodic image (zero
// below and above x in a moving window); the last x column is zero.
template <typename T>
__global__ void __launch_bounds__(256) load_fields_kernel(const SimDev* __restrict__ sd) {
    const SimDev& S = *sd;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const long long fs = S.fstride, nc = S.ncell;
    const double* E = S.J[0];
    const double* B = S.J[1];
    T* F = reinterpret_cast<T*>(S.F[0]);
    T* H = reinterpret_cast<T*>(S.H[0]);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < fs;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ip = (int)(idx % S.NX) - kGuard;
        const long long r = idx / S.NX;
        const int jp = (int)(r % S.NY) - kGuard;
        const int kp = S.dims == 3 ? (int)(r / S.NY) - kGuard : 0;
        int i = -1;
        if (ip >= 0 && ip < nx) i = ip;
        else if (!S.window && ip < nx + 2) i = (ip + nx) % nx;
        const int j = (jp + ny) % ny;
        const int k = S.dims == 3 ? (kp + nz) % nz : 0;
        const long long src = ((long long)k * ny + j) * nx + i;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double e = i >= 0 ? E[a * nc + src] : 0.0;
            const double b = i >= 0 ? B[a * nc + src] : 0.0;
            F[a * fs + idx] = T(e);
            F[(3 + a) * fs + idx] = T(b);
            H[a * fs + idx] = T(b);
        }
    }
}

cudaError_t launch_load_fields(const SimDev* sd, long long fstride, int prec, cudaStream_t s) {
    const int grid = elementwise_grid(fstride);
    PIC_DISPATCH(prec, (load_fields_kernel<T><<<grid, 256, 0, s>>>(sd)));
    return cudaGetLastError();
}

// ================================================================ end of step

// End of step, one CTA per sim: install the layout of a repack done in this step
// (bases, capacities, counts including placed arrivals), then advance the state.
__global__ void end_step_kernel(const BatchDev* __restrict__ bd) {
    const int s = blockIdx.x;
    if (s >= bd->nsims) return;
    const SimDev& S = bd->sims[s];
    StepState* st = S.st;
    const int rp = st->repack;
    if (rp == 1) {
        for (int p = threadIdx.x; p < S.npatch; p += blockDim.x) {
            S.pbase[p] = S.pbase_new[p];
            S.pcap[p] = S.pcap_new[p];
            S.mbase[p] = S.mbase_new[p];
            S.mcap[p] = S.mcap_new[p];
            S.pcount[p] += S.mpend[p];
            S.mpend[p] = 0;
        }
    } else if (rp == 2) {  // failed repack (status latched): the pending arrivals are lost
        for (int p = threadIdx.x; p < S.npatch; p += blockDim.x) S.mpend[p] = 0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (rp) {
        st->repack = 0;
        st->nrepack += rp == 1;
    }
    st->step += 1;
    if (st->shift) {
        st->nshift += 1;
        long long pts = (long long)S.n[1] * S.ippc[0] * S.ippc[1];
        if (S.dims == 3) pts *= (long long)S.n[2] * S.ippc[2];
        st->next_id += pts;
    }
    st->shift = 0;
}

cudaError_t launch_end_step(const BatchDev* bd, int nsims, int max_patches, cudaStream_t s) {
    (void)max_patches;
    end_step_kernel<<<nsims, 256, 0, s>>>(bd);
    return cudaGetLastError();
}

// ================================================================ diagnostics

template <typename T>
__global__ void energy_kernel(const SimDev* __restrict__ sd, long long ncell, long long cap) {
    const SimDev& S = *sd;
    __shared__ double sh[3][256 / 32];
    const int g = (int)(S.st->step & 1);  // fields of the current time level
    const T* F = reinterpret_cast<const T*>(S.F[g]);
    double we = 0, wb = 0, wk = 0;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += stride) {
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        const long long pi = ((long long)(S.dims == 3 ? k + kGuard : 0) * S.NY + (j + kGuard)) * S.NX +
                             (i + kGuard);
        (void)nz;
        for (int a = 0; a < 3; a++) {
            const double e = (double)F[a * S.fstride + pi];
            const double b = (double)F[(3 + a) * S.fstride + pi];
            we += e * e;
            wb += b * b;
        }
    }
    // particles: live slots of each patch (grid-stride over patches, block over slots)
    const T* U0 = reinterpret_cast<const T*>(S.u[0]);
    const T* U1 = reinterpret_cast<const T*>(S.u[1]);
    const T* U2 = reinterpret_cast<const T*>(S.u[2]);
    const T* W = reinterpret_cast<const T*>(S.w);
    for (int p = blockIdx.x; p < S.npatch; p += gridDim.x) {
        const int b0 = S.pbase[p], cnt = S.pcount[p];
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int sidx = b0 + k;
            const double ux = (double)U0[sidx], uy = (double)U1[sidx], uz = (double)U2[sidx];
            wk += (double)W[sidx] * S.m * (sqrt(1.0 + ux * ux + uy * uy + uz * uz) - 1.0);
        }
    }
    (void)cap;
    for (int o = 16; o > 0; o >>= 1) {
        we += __shfl_down_sync(0xffffffffu, we, o);
        wb += __shfl_down_sync(0xffffffffu, wb, o);
        wk += __shfl_down_sync(0xffffffffu, wk, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = we;
        sh[1][threadIdx.x >> 5] = wb;
        sh[2][threadIdx.x >> 5] = wk;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); w2++) v += sh[threadIdx.x][w2];
        atomicAdd(S.red + threadIdx.x, v);
    }
}

cudaError_t launch_energy(const SimDev* sd, long long ncell, long long cap, int prec,
                          cudaStream_t s) {
    int grid = 152 * 4;
    PIC_DISPATCH(prec, (energy_kernel<T><<<grid, 256, 0, s>>>(sd, ncell, cap)));
    return cudaGetLastError();
}

// Order-2 charge density of every live particle, FP64 atomics into rho (unpadded).
template <typename T>
__global__ void rho2d_kernel(const SimDev* __restrict__ sd, double* rho, double sign) {
    const SimDev& S = *sd;
    const int p = blockIdx.x;
    if (p >= S.npatch) return;
    const int b0 = S.pbase[p], cnt = S.pcount[p];
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int t = b0 + k;
    const int nx = S.n[0], ny = S.n[1];
    int ix, iy;
    double fx, fy;
    if constexpr (is_f64<T>::value) {
        const double xi = reinterpret_cast<const double*>(S.xi[0])[t];
        const double eta = reinterpret_cast<const double*>(S.xi[1])[t];
        ix = (int)floor(xi);
        iy = (int)floor(eta);
        fx = xi - ix;
        fy = eta - iy;
    } else {
        const int c = S.cell[t];
        ix = c & 0xFFFF;
        iy = (c >> 16) & 0xFFFF;
        fx = (double)reinterpret_cast<const T*>(S.xi[0])[t];
        fy = (double)reinterpret_cast<const T*>(S.xi[1])[t];
    }
    const int hx = fx >= 0.5, hy = fy >= 0.5;
    double Sx[3], Sy[3];
    shape3(fx - hx, Sx);
    shape3(fy - hy, Sy);
    const double qw = sign * S.q * (double)reinterpret_cast<const T*>(S.w)[t] / (S.d[0] * S.d[1]);
    for (int b = 0; b < 3; b++) {
        const int j = wrapi(iy + hy + b - 1, ny);
        for (int a = 0; a < 3; a++) {
            int i = ix + hx + a - 1;
            if (S.window) {
                if (i < 0 || i >= nx) continue;
            } else {
                i = wrapi(i, nx);
            }
            atomicAdd(rho + (long long)j * nx + i, qw * Sx[a] * Sy[b]);
        }
    }
    }
}

// mode 0: rho_bg = -rho_e (into S.rho_bg);  mode 1: out = div E - rho_e - rho_bg (into S.rho)
template <typename T>
__global__ void gauss2d_kernel(const SimDev* __restrict__ sd) {
    const SimDev& S = *sd;
    const int nx = S.n[0], ny = S.n[1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nx * ny) return;
    const int i = idx % nx, j = idx / nx;
    const T* E = reinterpret_cast<const T*>(S.F[S.st->step & 1]);  // current time level
    const long long fs = S.fstride;
    auto at = [&](int c, int ii, int jj) -> double {
        if (S.window && (ii < 0 || ii >= nx)) return 0.0;
        ii = wrapi(ii, nx);
        jj = wrapi(jj, ny);
        return (double)E[c * fs + (long long)(jj + kGuard) * S.NX + (ii + kGuard)];
    };
    const double div = (at(0, i, j) - at(0, i - 1, j)) / S.d[0] + (at(1, i, j) - at(1, i, j - 1)) / S.d[1];
    S.rho[idx] = div - S.rho[idx] - S.rho_bg[idx];
}

cudaError_t launch_gauss(const SimDev* sd, const SimDev& hs, int prec, int mode, cudaStream_t s) {
    if (hs.dims == 3) return launch_gauss3d(sd, hs, prec, mode, s);
    const long long nc = hs.ncell;
    double* target = mode == 0 ? hs.rho_bg : hs.rho;
    cudaError_t e = cudaMemsetAsync(target, 0, nc * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int g1 = hs.npatch;
    const double sign = mode == 0 ? -1.0 : 1.0;
    if (hs.dims != 2) return cudaErrorInvalidValue;
    PIC_DISPATCH(prec, (rho2d_kernel<T><<<g1, 256, 0, s>>>(sd, target, sign)));
    if (mode == 1) {
        const int g2 = (int)((nc + 255) / 256);
        PIC_DISPATCH(prec, (gauss2d_kernel<T><<<g2, 256, 0, s>>>(sd)));
    }
    return cudaGetLastError();
}

}  // namespace pic
