/*
 * pic.h - C ABI of the GB300 (sm_103a) patch-based particle-in-cell hot path.
 *
 * What the library computes: the explicit electromagnetic PIC cycle of a patch-based
 * code (Sec. 3, "The importance of computational load-management"; Sec. 3.1,
 * "Dynamic load balancing": the simulation domain is cut into many small patches,
 * each holding the fields and the super-particles (SP) of a sub-domain, and the
 * load of a patch is its SP count). One step is
 *   order-2 interpolation of E, B from the Yee grid at each SP, relativistic Boris
 *   push, Esirkepov charge-conserving current deposition, exchange of SP between
 *   neighbouring patches, Yee FDTD update of E and B (the standard second-order
 *   scheme of Sec. 2.1), and for laser-wakefield runs a moving window with plasma
 *   injection (Sec. 2.2 setup: laser focused at the foot of a density ramp).
 * The paper's load-imbalance problem (Sec. 3: some regions hold about forty times
 * their initial SP count, Fig. 2) is handled on one GPU by a persistent kernel that
 * pulls patch chunks from a device work queue ordered by SP count.
 *
 * Units are normalised: c = eps0 = 1, dE/dt = curl B - J, dB/dt = -curl E.
 * Grid staggering (array index i of a component stands for position (i + s/2) d):
 *   Ex (1,0,0) Ey (0,1,0) Ez (0,0,1) Bx (0,1,1) By (1,0,1) Bz (1,1,0); J like E.
 * Host field arrays are plain row-major [nz][ny][nx] float64 (nz = 1 in 2D).
 *
 * Memory: the caller owns all device memory. pic_required_bytes() gives the size
 * of one device arena; pic_create() carves everything out of it and never calls
 * cudaMalloc. The arena must stay valid until pic_destroy(). Host buffers passed
 * to the library are read or written during the call only and never retained.
 *
 * Errors: no exception crosses the ABI. Every call returns a pic_status. Errors
 * raised on the device (capacity overflow, non-finite particles, an expired
 * bounded wait) latch in a device status word and are returned by the next call
 * that synchronises (pic_diag, pic_sync). A failed call leaves the sim destroyable.
 * pic_last_error() gives a one-line description.
 *
 * Threading: a sim is used by one host thread at a time; all its work is ordered
 * on the CUDA stream given at creation.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_sim pic_sim;
typedef struct pic_batch pic_batch;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_INVALID = -1,  /* bad argument or configuration */
    PIC_ERR_NOMEM = -2,    /* arena or output buffer too small, or a host allocation failed */
    PIC_ERR_CAPACITY = -3, /* a patch or exchange buffer overflowed on the device */
    PIC_ERR_CUDA = -4,     /* a CUDA runtime call failed */
    PIC_ERR_NUMERIC = -5,  /* non-finite particle state or a move of a cell or more */
    PIC_ERR_TIMEOUT = -6   /* a bounded device-side wait expired */
} pic_status;

/* Precision of particles and fields (the global current is FP64 in all three):
 *   PIC_FP64  IEEE binary64 throughout.
 *   PIC_FP32  binary32 particles (cell index + offset) and fields.
 *   PIC_DF64  double-word: every real held and computed as a pair of binary32 numbers
 *             (hi + lo, about 48 significant bits), particles as cell index + pair
 *             offset. FP64-class accuracy (relative errors of a few 2^-48) from FP32
 *             arithmetic, for GPUs whose FP64 units are a small fraction of FP32. 2D
 *             only (a 3D config with it is invalid). */
enum { PIC_FP64 = 0, PIC_FP32 = 1, PIC_DF64 = 2 };

/* Work distribution of the particle kernel. */
enum {
    PIC_MAP_QUEUE = 0, /* persistent CTAs pull chunks, largest first (default) */
    PIC_MAP_STATIC = 1 /* one CTA per patch, no chunking (baseline for comparison) */
};

typedef struct {
    int dims;           /* 2 (2D3V) or 3 (3D3V) */
    int n[3];           /* cells per axis; n[2] = 1 in 2D */
    double d[3];        /* cell sizes */
    double dt;          /* time step; below every d[a] and within the stability limit
                           of the field solver (maxwell_order) */
    int patch[3];       /* cells per patch per axis: a multiple of 4 in [4, 64], dividing
                           n[a]; the patch's field and current tiles must fit in the 227 KB
                           of shared memory of one CTA (pic_required_bytes returns 0 when
                           they do not) */
    int precision;      /* PIC_FP64, PIC_FP32 or PIC_DF64 (see above) */
    int window;         /* 0: all axes periodic.  1: x is a moving window at c
                           (fields zero outside, particles absorbed), y/z periodic */
    double n0;          /* window only: injected density n(x) = n0 *        */
    double ramp_x0;     /*   clamp((x_lab - ramp_x0)/ramp_len, 0, 1)          */
    double ramp_len;    /*                                                    */
    int inject_ppc[3];  /* window only: injected lattice per cell per axis */
    double q, m;        /* species charge and mass (electrons: -1, 1) */
    long long capacity; /* particles the sim may hold (>= the largest count held); the
                           arena adds 32 slots per patch so that per-patch bases stay
                           aligned */
    int chunk;          /* work-queue chunk size in particles (0 = 2048); the Python
                           autotuner measures patch and chunk candidates on a workload */
    int mapping;        /* PIC_MAP_QUEUE or PIC_MAP_STATIC */
    int merge_above;    /* load limiting (Sec. 3.2): at the end of every step, each patch
                           holding more than this many particles has every group of >= 3
                           particles sharing a cell and a momentum bin replaced by two
                           particles with the group's total weight, momentum and energy
                           (Vranic et al. 2015); 0 = off. Needs patches of at most 4096
                           cells. */
    double merge_dp;    /* momentum-bin width (units of m c) of the merge; > 0 when
                           merge_above > 0 */
    int maxwell_order;  /* field solver (Sec. 2.1): 0 or 2 = Yee's two-point staggered
                           differences; 6 = sixth-order staggered space differences
                           sum_{l=1..3} c_l [f(x + (l-1/2)h) - f(x - (l-1/2)h)] / h with
                           c = (75/64, -25/384, 3/640), leapfrog in time. The time step
                           must satisfy dt * kappa * sqrt(sum_a 1/d[a]^2) < 1 with kappa = 1
                           (order 2) or 149/120 (order 6), else the config is invalid.
                           Esirkepov's current conserves charge for the two-point
                           divergence, so with order 6 the GAUSS diagnostic is no longer
                           preserved to round-off. */
    int split_below;    /* load limiting (Sec. 3.2: SP are split in cells of low SP density):
                           at the end of every step (after merging), a cell holding n
                           particles with 1 <= n < split_below has its particles of weight
                           >= 2 split_wmin, in increasing id, split until it holds
                           split_below particles or each has been split once. A split
                           replaces (x, u, w) by (x + delta, u, w/2) and (x - delta, u, w/2)
                           with delta_a = min(f_a, 1 - f_a) d_a / 2 (f_a the in-cell offset),
                           so charge, momentum, energy and the charge centroid are kept and
                           both halves stay in the cell; the new particle's id is the next
                           free id in (patch, cell, parent id) order. 0 = off; at most 64;
                           needs patches of at most 4096 cells. A patch without room for its
                           new particles latches PIC_ERR_CAPACITY (size capacity for them). */
    double split_wmin;  /* weight floor of splitting (>= 0): a particle splits only while
                           its weight is at least 2 split_wmin */
} pic_config;

/* sizeof(pic_config) as this library was built: a binding compares it with its own
 * layout of the struct before passing one. The paper has no counterpart. */
size_t pic_config_bytes(void);

/* Device bytes one arena needs for this configuration (0 if the config is invalid):
 * the fields and the super-particles of every patch plus the exchange buffers (Sec.
 * 3.1: a patch holds the fields and SP of its sub-domain). Used to admit simulations
 * into a fixed device budget. */
size_t pic_required_bytes(const pic_config* cfg);

/* Create a sim in a caller-owned device arena (>= pic_required_bytes, 256-byte
 * aligned). The grid is cut into patches of cfg->patch cells, each owning its fields
 * and its SP (Sec. 3.1, "Dynamic load balancing": many small patches per process, so
 * that load can be traded patch by patch). cuda_stream: a cudaStream_t (NULL = legacy default stream) on which all
 * work of this sim is ordered. On success *out owns host-side state only. */
pic_status pic_create(const pic_config* cfg, void* dev_arena, size_t arena_bytes,
                      void* cuda_stream, pic_sim** out);

/* Load n particles from host SoA arrays (float64 physical positions, momenta
 * u = gamma v, weights; int32 ids, unique and >= 0). Each SP is binned into the patch
 * that holds it; the SP count per patch is the load measure (Sec. 3: the load of a
 * region is its number of SP) that orders the work queue. z may be NULL in 2D. Positions
 * must lie in [0, n[a] d[a]). The arrays are copied to the device as they are (in
 * chunks of the repack scratch); the device validates the particles, bins them by patch
 * and orders each patch's particles by shared-memory bank class, and the host reads back
 * only the per-patch counts to split the capacities: the free slots half by count, half
 * evenly. The arrays are not retained: every copy has completed when the call returns,
 * on success and on error. Returns
 * PIC_ERR_CAPACITY if n > capacity, PIC_ERR_INVALID for a position outside the grid or
 * a negative id, PIC_ERR_NUMERIC for a non-finite momentum or weight; a rejected load
 * leaves the sim as it was. Resets the step counter to 0. */
pic_status pic_load_particles(pic_sim* sim, long long n, const double* x, const double* y,
                              const double* z, const double* ux, const double* uy,
                              const double* uz, const double* w, const int* id);

/* Load fields from host arrays [nz][ny][nx] on the staggered Yee nodes of the
 * second-order scheme (Sec. 2.1): E at t = 0, B at t = +dt/2 (the first
 * push uses that B at integer time too). For laser-wakefield runs these hold the laser
 * pulse at the foot of the density ramp (Sec. 2.2). rho_bg: immobile background charge on
 * nodes for the Gauss diagnostic; NULL = minus the charge density of the particles
 * loaded now. Zeroes the current. The arrays are copied as they are and padded with
 * guard cells on the device; they are not retained. */
pic_status pic_load_fields(pic_sim* sim, const double* const E[3], const double* const B[3],
                           const double* rho_bg);

/* Enqueue nsteps steps on the sim's stream (asynchronous: returns before the GPU
 * finishes). Each step is one replay of a CUDA graph of the kernels above: one PIC
 * cycle (Sec. 3: the per-SP work of interpolation, push and deposition, then the field
 * update, Sec. 2.1), with the exchange of SP between neighbouring patches that
 * independent patches need (Sec. 3.1). */
pic_status pic_step(pic_sim* sim, int nsteps);

/* Wait for the sim's stream; returns any latched device error. The paper has no
 * counterpart. */
pic_status pic_sync(pic_sim* sim);

/* Diagnostics (synchronise first, then copy to the host buffer out of out_bytes;
 * *written = bytes written). PATCH_COUNTS is the SP count per patch, the load measure
 * whose spread across the domain the paper plots (Sec. 3, Fig. 2: SP per process in a
 * 3D run); ENERGY and EX_AXIS are the energy and wake-field diagnostics of a
 * laser-wakefield run (Sec. 2.2). Kinds: */
enum {
    PIC_DIAG_ENERGY = 0,        /* 3 float64: W_E, W_B (with B^n), W_kin          */
    PIC_DIAG_GAUSS = 1,         /* ncell float64: div E - rho - rho_bg on nodes    */
    PIC_DIAG_FIELDS = 2,        /* 12 * ncell float64: E^n, B^{n+1/2}, B^n, last J */
    PIC_DIAG_PARTICLES = 3,     /* n * 7 float64 (x,y,z,ux,uy,uz,w, each array of n)
                                   then n int32 ids; sorted by id; x in the window
                                   frame                                          */
    PIC_DIAG_NUM_PARTICLES = 4, /* 1 int64                                        */
    PIC_DIAG_PATCH_COUNTS = 5,  /* npatch int32 (x fastest)                        */
    PIC_DIAG_STEP = 6,          /* 3 int64: steps taken, window shifts, capacity
                                   repacks (per-patch capacities re-split on the
                                   device when a patch nears its capacity); a 4th,
                                   particles removed by merging, and a 5th,
                                   particles added by splitting, when out_bytes
                                   allows                                         */
    PIC_DIAG_EX_AXIS = 7,       /* nx float64: Ex on the row (and plane) ny/2      */
    PIC_DIAG_QUEUE = 8,         /* int32 m, then m x 4 int32 {sim, patch, first,
                                   count}: the work items of the last step's queue
                                   (built from the patch counts at the start of that
                                   step): full chunks of `chunk` particles in patch
                                   order, then each patch's remainder in 64 buckets of
                                   decreasing size (an approximate largest-first order;
                                   the order inside a bucket is not fixed); with the
                                   static mapping one item per non-empty patch in patch
                                   order. Sec. 3: load = SP count, so the largest loads
                                   are handed out first                          */
    PIC_DIAG_SLOTS = 9          /* n int32, sorted by id as PIC_DIAG_PARTICLES: each
                                   SP's slot within its patch's range (0 = the patch's
                                   first slot), the order in which work items take a
                                   patch's SP (Sec. 3.1: a patch owns its SP)   */
};
pic_status pic_diag(pic_sim* sim, int kind, void* out, size_t out_bytes, size_t* written);

/* The step record without a wait: enqueues, on the sim's stream after the work already
 * enqueued, a copy of the device step state and status word into a page-locked staging
 * slot the library owns (slot 0 or 1, created on first use), then an event, and returns
 * at once. pic_record_wait(sim, slot, ...) later waits for that event only. A caller
 * that enqueues step k + 1 before it waits for step k's record keeps the device busy
 * between steps. Enqueueing a slot again before its wait overwrites the record. The
 * paper has no counterpart (host plumbing). Errors: PIC_ERR_INVALID (null sim, slot not
 * 0 or 1); PIC_ERR_NOMEM (no page-locked memory or event); PIC_ERR_CUDA (the copy or
 * the event could not be enqueued). */
pic_status pic_step_record_async(pic_sim* sim, int slot);

/* Waits for the record pic_step_record_async enqueued in `slot` and writes it to out as
 * PIC_DIAG_STEP does (3 int64: steps taken, window shifts, capacity repacks; a 4th,
 * particles removed by merging, and a 5th, particles added by splitting, when out_bytes
 * allows; *written = bytes written). Returns the device status latched up to that
 * record as pic_sync does (PIC_ERR_TIMEOUT, PIC_ERR_CAPACITY, PIC_ERR_NUMERIC, ...),
 * and then writes nothing. Errors: PIC_ERR_INVALID (null sim or out, slot not 0 or 1,
 * or no record pending in the slot); PIC_ERR_NOMEM (out_bytes < 24); PIC_ERR_CUDA. The
 * paper has no counterpart. */
pic_status pic_record_wait(pic_sim* sim, int slot, void* out, size_t out_bytes,
                           size_t* written);

/* Instrumentation (per-kernel timing): runs nsteps steps with one plain launch per
 * kernel (no graph) and CUDA events around each kernel on the sim's stream, then
 * synchronises. ms[0..7] receive the summed times in milliseconds of: work-queue
 * build, particle push/deposit, window injection, particle exchange, capacity repack
 * (kernels that return at once unless a patch needs room), Yee E+B, end of step, and
 * the whole steps. n_ms must be >= 8. Same kernels and launch shapes as pic_step; the
 * state advances by nsteps. The paper has no counterpart (it reports wall times per
 * process, Fig. 4; this is the per-kernel breakdown on one GPU). */
pic_status pic_profile(pic_sim* sim, int nsteps, double* ms, int n_ms);

/* Destroy the host-side state (synchronises; does not free the arena). The paper has
 * no counterpart (resource management of this library). */
pic_status pic_destroy(pic_sim* sim);

/* One-line description of the last error on this sim (never NULL). The paper has no
 * counterpart. */
const char* pic_last_error(const pic_sim* sim);

/* ---- batching: many sims stepped together, one persistent particle launch ----
 * All sims of a batch share dims and precision; each keeps its own arena, state
 * and step counter. The batch needs a small arena of its own (work queue). The patches
 * of all sims share one work queue ordered by SP count, so uneven sims balance the way
 * uneven patches do (Sec. 3.1: work distributed by patch load), which serves the
 * parameter-scan campaigns of Sec. 2.2. */
size_t pic_batch_required_bytes(pic_sim* const* sims, int nsims);
pic_status pic_batch_create(pic_sim* const* sims, int nsims, void* dev_arena,
                            size_t arena_bytes, void* cuda_stream, pic_batch** out);
pic_status pic_batch_step(pic_batch* batch, int nsteps);
pic_status pic_batch_destroy(pic_batch* batch);

/* ---- allocation-free entry point (the paper has no counterpart) ----
 * Gauss's-law residual div E - rho_e - rho_bg on the nodes of a 2D grid, computed
 * from caller-owned device arrays, for callers that cannot allocate device memory:
 * code that runs inside another framework's memory pool or under a fixed device
 * budget, where a cudaMalloc would fail, fragment the pool, or implicitly
 * synchronise the device in the middle of asynchronous work. This call allocates
 * nothing: its charge-density accumulator is a file-scope static device array of
 * PIC_STATIC_MAX_CELLS float64 (8 MiB), which every GPU that loads the library
 * holds until the process exits.
 *   x, y, w : n particle positions (physical, in [0, nx dx) x [0, ny dy)) and
 *             weights, device float64; particles outside the grid are skipped. The
 *             cell coordinate is x / dx in IEEE division, kept below nx for a position
 *             just under the end (as pic_load_particles computes it).
 *   q       : species charge.
 *   Ex, Ey  : device float64 [ny][nx], Yee staggering (Ex at (i+1/2, j), Ey at
 *             (i, j+1/2)).
 *   rho_bg  : device float64 [ny][nx] background charge, or NULL for none.
 *   out     : device float64 [ny][nx], written completely.
 *   window  : 0 = x periodic; 1 = values outside [0, nx) along x are zero.
 * y is periodic. The work is enqueued on cuda_stream and returns before it runs.
 * Returns PIC_ERR_NOMEM if nx * ny > PIC_STATIC_MAX_CELLS (nothing is launched),
 * PIC_ERR_INVALID for bad arguments, PIC_ERR_CUDA if a lookup or launch fails.
 * Every call shares the scratch array, which keeps the last call's contents; each
 * call clears the part it uses before depositing. Calls that overlap on the GPU
 * (other streams, other host threads) race on that array: serialise them.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again when the
 * device's context has changed since (after a cudaDeviceReset, for instance); make
 * the first call on a device, and the first after a reset, before any stream
 * capture. */
#define PIC_STATIC_MAX_CELLS (1 << 20)
pic_status pic_gauss_residual_2d_static(long long n, const double* x, const double* y,
                                        const double* w, double q, const double* Ex,
                                        const double* Ey, const double* rho_bg, double* out,
                                        int nx, int ny, double dx, double dy, int window,
                                        void* cuda_stream);

/* ---- patch decomposition across ranks (host only; Sec. 3.1, Figs. 3-4) ----
 * The paper balances load between MPI processes by ordering the patches along a
 * Hilbert curve, giving each process a contiguous segment of that order whose total
 * load (SP count, Sec. 3) is balanced, and moving patches between processes when the
 * loads change. These two calls compute the order and the segments; moving the patches'
 * particles and fields is the caller's (paper_1511_03878_gb300/decomp.py does it over
 * torch.distributed). Neither touches a GPU.
 *
 * pic_hilbert_order: order[k] = the index (x fastest) of the k-th patch along the
 * Hilbert curve of the smallest 2^b x 2^b (x 2^b) box holding the np[0] x np[1]
 * (x np[2]) patches, restricted to the patches that exist (consecutive patches are
 * face neighbours when every np[a] is the same power of two). order holds
 * np[0] np[1] (np[2]) ints, caller-owned. PIC_ERR_INVALID for dims other than 2 or 3,
 * np[a] < 1 or more than 2^30 patches. */
pic_status pic_hilbert_order(int dims, const int np[3], int* order);

/* pic_partition: splits n loads (>= 0, in curve order) into nranks contiguous segments,
 * each of at least one patch, with the largest segment load as small as possible
 * (within 1e-12 relative): rank r owns positions first[r] .. first[r+1]-1; first holds
 * nranks + 1 ints (first[nranks] = n), caller-owned. *max_load (if not NULL) receives the
 * largest segment load. PIC_ERR_INVALID for nranks outside [1, n] or a negative or
 * non-finite load. */
pic_status pic_partition(int n, const double* load, int nranks, int* first, double* max_load);

/* Failure-path self-test of the bounded device waits (the paper has no counterpart). Every wait of the library's
 * kernels on an asynchronous transfer (the mbarrier of a TMA tile load) gives up after
 * about 2^31 SM clocks (about a second) and latches a status bit instead of hanging.
 * This call launches one CTA that waits, through that same bounded wait, on an
 * mbarrier phase that nothing completes, then synchronises cuda_stream and reads the
 * status back. Expected result: PIC_ERR_TIMEOUT after about a second, with the CUDA
 * context still usable. PIC_OK would mean the wait completed without its transfer;
 * PIC_ERR_CUDA reports a failed launch or copy. Allocates 4 bytes of device memory
 * for the status and frees them. */
pic_status pic_selftest_bounded_wait(void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
