// Internal device-visible data model of the patch-PIC library (host + device).
//
// Fields: every component is a padded array [NZ][NY][NX] with one guard cell
// below each axis (interior index i is stored at i + 1). The particle kernel
// stages a patch tile of E and B^n (6 components, contiguous) with one TMA box;
// periodic axes keep their guard cells filled with periodic images.
// Particles: patch-sorted SoA. Patch p owns slots [pbase[p], pbase[p] + pcap[p]),
// the first pcount[p] of them live. FP64 path: positions are float64 in cell units
// (xi = x / d). FP32 path: a global linear cell index plus float32 offsets in [0,1).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace pic {

// position along an axis in cell units, c = v / d, kept below the cell count n when v
// lies just under the domain's end; host and device compute it identically (IEEE
// division), so the host's binning and the device's conversion see the same cell
__host__ __device__ inline double cell_coord(double v, double d, int n) {
    double c = v / d;
    if (c >= (double)n) c = nextafter((double)n, 0.0);
    return c;
}

constexpr int kGuard = 1;        // guard cells below each axis in the padded field arrays
constexpr int kThreads = 256;    // threads per CTA of the particle kernel
constexpr int kQueueThreads = 1024;
constexpr int kBuckets = 64;     // remainder buckets of the approximate LPT order
constexpr int kMailboxMin = 1024; // exchange-buffer slots per patch at least (a step's arrivals)
constexpr int kMailboxDiv = 2;    // exchange-buffer slots per patch: capacity / kMailboxDiv
                                  // (a compressed 3D LWFA patch took in more than 1/4 of its
                                  // capacity in one step)
constexpr int kMergeCells = 4096;  // largest patch (in cells) the merge kernel sorts
constexpr int kSplitBelowMax = 64; // largest split_below (a cell's particles sorted by one
                                   // thread)
constexpr int kSlotAlign = 32;    // per-patch particle and exchange-buffer bases are multiples
                                  // of this, so that a warp's particle loads start a line
constexpr int kLeaveList = 512;   // leavers of one work item handed off after the item;
                                  // more than this are handed off on the spot
constexpr int kPush2DStatic = 2 * 4 * kLeaveList + 64;  // static shared bytes of the push
                                                        // kernels (2D and 3D)

__host__ __device__ inline long long align_slots(long long v) {
    return (v + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
}

// status bits latched by device code
enum : int {
    ST_CAPACITY = 1,   // patch overflow in the exchange
    ST_MAILBOX = 2,    // exchange buffer overflow
    ST_TIMEOUT = 4,    // bounded wait expired
    ST_NUMERIC = 8,    // non-finite or too-large move
    ST_QUEUE = 16,     // work queue overflow
};

struct StepState {
    long long step;     // steps completed
    long long nshift;   // window shifts completed
    long long next_id;  // next particle id handed to injected particles
    int shift;          // 1 if the current step ends with a window shift
    int gen;            // field buffer generation read by the current step (step & 1)
    int repack;         // set by the exchange when a patch nears or exceeds its capacity
    int nrepack;        // repacks done
    long long nmerged;  // particles removed by merging
    long long nsplit;   // particles added by splitting
};

struct SimDev {
    int dims, prec, window, mapping;
    int n[3];        // cells
    int P[3];        // cells per patch
    int np[3];       // patches per axis
    int npatch;
    int NX, NY, NZ;  // padded extents
    int BX, BY, BZ;  // TMA box extents
    long long fstride;  // elements per padded component
    double d[3], dt, q, m;
    double n0, ramp_x0, ramp_len;
    int ippc[3];
    int pad0;
    // per-step constants of the particle kernel, computed once on the host
    double c_dtd[3];   // dt / d[a]
    double c_eps;      // q dt / (2 m)
    double c_j[3];     // 2D: -q/dV d[a]/dt for Jx, Jy and q/dV for Jz (times v_z)
    float f_dtd[3], f_eps, f_j[3];
    // field-solver constants: dt and 1/d[a] in FP64, and as FP32 (hi) + FP32 (lo) pairs
    double c_id[3];
    float f_dt, f_dt_lo, f_id[3], f_id_lo[3];
    int order;         // field solver: 2 (Yee) or 6 (sixth-order staggered differences)
    // sixth order: c_l / d[a] for l = 1..3 in FP64 and as FP32 hi + lo pairs
    double c_k[3][3];
    float f_k[3][3], f_k_lo[3][3];
    int cmax_exp;      // one particle's current contribution stays below 2^cmax_exp
    int merge_above;   // load limiting: patches above this count are merged (0: off)
    double merge_dp;   // momentum-bin width of the merge
    int split_below;   // load limiting: cells below this count are split (0: off)
    double split_wmin; // weight floor of the split
    // fields
    void* F[2];      // [6][NZ][NY][NX]: Ex Ey Ez Bnx Bny Bnz (B^n for the push)
    void* H[2];      // [3][...]: B^{n+1/2}
    double* J[2];    // [3][...] (guards unused)
    const CUtensorMap* tmap;  // [2], in global memory
    // particles
    int* cell;       // FP32 only
    void* xi[3];     // FP64: double positions in cell units; FP32: float offsets
    void* u[3];
    void* w;
    int* id;
    int* pbase; int* pcap; int* pcount;
    int* hcount; int* holes; int* aux;
    // exchange mailboxes (same SoA layout)
    int* mbase; int* mcap; int* mcount;
    int* mcell;
    void* mxi[3];
    void* mu[3];
    void* mw;
    int* mid;
    long long capacity;  // particle slots in the arrays (ucap + alignment slack)
    long long mtotal;    // exchange-buffer slots
    long long ucap;      // particles the sim may hold (the configured capacity)
    // repack: scratch particle buffer (capacity slots) and the next layout
    int* acell;
    void* axi[3];
    void* au[3];
    void* aw;
    int* aid;
    int* pbase_new; int* pcap_new; int* mbase_new; int* mcap_new;
    int* mpend;      // arrivals left in the exchange buffer for want of room (repack places them)
    int* mpoff;      // offset of the first of them in the patch's exchange buffer
    int* mlast;      // per patch: count after its last merge pass (0 = none yet)
    int* soff;       // [npatch + 1] splitting: splits per patch, then the first new id of
                     // each patch (soff[npatch] = the next free id after the pass)
    void* ecol;      // sixth order with the window: [3][nz][ny] E^{n+1} of the column a
                     // shift drops (old-frame x = 0), read by the B update
    // state and scratch
    StepState* st;
    int* status;
    double* red;     // 8 reduction slots
    double* rho;     // [ncell] scratch for the Gauss diagnostic
    double* rho_bg;  // [ncell]
    long long ncell;
};

struct BatchDev {
    int nsims;
    int chunk;
    int max_items;
    int total_patches;
    int max_patches;     // largest npatch over sims
    int max_ncell;
    const SimDev* sims;  // device array [nsims]
    const int* patch_prefix;  // [nsims + 1]
    int4* items;         // {sim, patch, first, count}
    int* nitems;
    int* head;
};

// ---- launchers (each enqueues on the given stream) ----
cudaError_t launch_queue_build(const BatchDev* bd, cudaStream_t s);
// capacity repack (no-op unless a sim's exchange flagged it)
cudaError_t launch_repack(const BatchDev* bd, int nsims, int max_patches, int prec,
                          cudaStream_t s);
cudaError_t launch_push(const BatchDev* bd_dev, int dims, int prec, int mapping,
                        int P0, int P1, int P2, int grid, cudaStream_t s);
int push_occupancy(int dims, int prec, int P0, int P1, int P2, int* smem_bytes);
cudaError_t launch_inject(const BatchDev* bd, int nsims, int max_column_pts, int prec,
                          cudaStream_t s);
cudaError_t launch_exchange(const BatchDev* bd, int nsims, int max_patches, int prec,
                            cudaStream_t s);
cudaError_t launch_yee(const BatchDev* bd, int nsims, int max_ncell, int dims, int prec,
                       int order, cudaStream_t s);
cudaError_t launch_end_step(const BatchDev* bd, int nsims, int max_patches, cudaStream_t s);
// load limiting by merging (no-op for sims with merge_above = 0)
cudaError_t launch_merge(const BatchDev* bd, int nsims, int max_patches, int prec,
                         cudaStream_t s);
// load limiting by splitting (no-op for sims with split_below = 0): count, id offsets,
// apply
cudaError_t launch_split(const BatchDev* bd, int nsims, int max_patches, int prec,
                         cudaStream_t s);
// the split kernel's shared-memory opt-in (once, outside any stream capture)
cudaError_t split_setup();
// 3D variants
int push2d_smem(int prec, int P0, int P1);
int push3d_smem(int prec, int P0, int P1, int P2);
int push3d_occupancy(int prec, int P0, int P1, int P2, int* smem_bytes);
cudaError_t launch_push3d(const BatchDev* bd_dev, int prec, int mapping, int P0, int P1, int P2,
                          int grid, cudaStream_t s);
// failure-path self-test: a bounded wait on an mbarrier that nothing completes
cudaError_t launch_bounded_wait_selftest(int* status, cudaStream_t s);
// particle load, one chunk: m particles of the caller's FP64 arrays staged in the repack
// scratch (positions axi, momenta au, weights aw, ids aid; slots in holes), converted to
// the sim's representation and stored in their slots
cudaError_t launch_load_bin(const BatchDev* bd, long long m, long long k0, cudaStream_t s);
cudaError_t launch_load_slot(const BatchDev* bd, long long n, cudaStream_t s);
cudaError_t launch_load_scatter(const BatchDev* bd, long long m, long long k0, int prec,
                                cudaStream_t s);
// field load: E staged in J[0] and B in J[1] (three ncell arrays each, x fastest) to the
// padded F (E, B) and H (B) of generation 0 in the sim's precision
cudaError_t launch_load_fields(const SimDev* sd, long long fstride, int prec, cudaStream_t s);
cudaError_t launch_maxwell6(const BatchDev* bd, int nsims, long long max_ncell, int dims,
                           int prec, cudaStream_t s);
cudaError_t launch_yee3d(const BatchDev* bd, int nsims, long long max_ncell, int prec,
                         cudaStream_t s);
cudaError_t launch_gauss3d(const SimDev* sd, const SimDev& hs, int prec, int mode, cudaStream_t s);
// diagnostics on one sim
cudaError_t launch_energy(const SimDev* sd, long long ncell, long long cap, int prec,
                          cudaStream_t s);
cudaError_t launch_gauss(const SimDev* sd, const SimDev& hs, int prec, int mode,
                         cudaStream_t s);

}  // namespace pic
