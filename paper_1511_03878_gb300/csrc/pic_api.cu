// Host side of the C ABI declared in include/pic.h: arena carving, TMA tensor maps,
// host binning of particles into patches, CUDA-graph capture of one step, and
// diagnostics. Device memory is never allocated here: everything lives in the
// caller's arena.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <numeric>
#include <memory>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "df64.cuh"
#include "pic.h"
#include "pic_internal.h"

using namespace pic;

namespace {

// Everything carved out of one sim arena.
struct Layout {
    SimDev S{};          // host copy of the device descriptor
    SimDev* ds = nullptr;   // device copy
    BatchDev B{};        // single-sim batch descriptor (host copy)
    BatchDev* db = nullptr; // device copy
    int* prefix = nullptr;  // [2] patch prefix of the single-sim batch
    size_t bytes = 0;
};

struct Carver {
    char* base;
    bool dry;
    size_t off = 0;
    template <class T>
    T* take(long long count, size_t align = 256) {
        off = (off + align - 1) / align * align;
        T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
        off += (size_t)std::max(count, 0LL) * sizeof(T);
        return p;
    }
};

int default_chunk(const pic_config* c) {
    if (c->mapping == PIC_MAP_STATIC) return 1 << 30;
    return c->chunk > 0 ? c->chunk : 2048;
}

}  // namespace

struct pic_sim {
    pic_config cfg{};
    Layout L;
    char* arena = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap0 = nullptr, cap1 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int push_grid = 0;
    int column_pts = 0;
    // asynchronous step records: two page-locked slots (the device step state, then the
    // status word) and their events, created on first use
    unsigned char* rec_host = nullptr;
    cudaEvent_t rec_ev[2] = {nullptr, nullptr};
    bool rec_pending[2] = {false, false};
    std::string err;
};

struct pic_batch {
    std::vector<pic_sim*> sims;
    BatchDev hb{};
    BatchDev* db = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap0 = nullptr, cap1 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
};

namespace {

const char* validate(const pic_config* c) {
    if (!c) return "null config";
    if (c->dims != 2 && c->dims != 3) return "dims must be 2 or 3";
    if (c->precision != PIC_FP64 && c->precision != PIC_FP32 && c->precision != PIC_DF64)
        return "bad precision";
    if (c->window != 0 && c->window != 1) return "bad window flag";
    if (c->mapping != PIC_MAP_QUEUE && c->mapping != PIC_MAP_STATIC) return "bad mapping";
    for (int a = 0; a < c->dims; a++) {
        if (c->n[a] < 4) return "each axis needs at least 4 cells";
        if (!(c->d[a] > 0) || !std::isfinite(c->d[a])) return "cell sizes must be positive";
        if (c->patch[a] < 4 || c->patch[a] % 4 != 0 || c->patch[a] > 64)
            return "patch sides must be multiples of 4 in [4, 64]";
        if (c->n[a] % c->patch[a] != 0) return "patch sides must divide the grid";
        if (!(c->dt < c->d[a])) return "dt must be below every cell size";
    }
    if (c->dims == 2 && c->n[2] != 1) return "2D needs n[2] = 1";
    if (c->dims == 2 && (c->n[0] >= 65536 || c->n[1] >= 32768)) return "grid too large";
    if (c->dims == 2 &&
        push2d_smem(c->precision, c->patch[0], c->patch[1]) + kPush2DStatic > 227 * 1024)
        return "2D patch tile does not fit in shared memory";
    if (c->dims == 3) {
        if (c->precision == PIC_DF64) return "the double-word precision is 2D only";
        if (c->n[0] > 2048 || c->n[1] > 2048 || c->n[2] > 1024) return "3D grid too large";
        if (push3d_smem(c->precision, c->patch[0], c->patch[1], c->patch[2]) + kPush2DStatic >
            227 * 1024)
            return "3D patch tile does not fit in shared memory";
    }
    if (!(c->dt > 0) || !std::isfinite(c->dt)) return "dt must be positive";
    if (c->maxwell_order != 0 && c->maxwell_order != 2 && c->maxwell_order != 6)
        return "maxwell_order must be 0, 2 or 6";
    {
        // leapfrog is stable while (dt/2) max|K| < 1 over the grid's waves; the symbol of
        // the staggered difference peaks at the Nyquist wave at (2/d) sum_l |c_l|, i.e.
        // 2/d (Yee) and (2/d) 149/120 (sixth order)
        double s2 = 0.0;
        for (int a = 0; a < c->dims; a++) s2 += 1.0 / (c->d[a] * c->d[a]);
        const double kappa = c->maxwell_order == 6 ? 149.0 / 120.0 : 1.0;
        if (!(c->dt * kappa * std::sqrt(s2) < 1.0))
            return "dt above the stability limit of the field solver";
    }
    if (!(c->m > 0)) return "mass must be positive";
    if (c->capacity < 0 || c->capacity > (1LL << 31) - (1LL << 24)) return "bad capacity";
    if (c->chunk < 0) return "bad chunk";
    if (c->merge_above < 0) return "bad merge_above";
    if (c->merge_above > 0) {
        if (!(c->merge_dp > 0) || !std::isfinite(c->merge_dp)) return "merge_dp must be positive";
        long long cells = 1;
        for (int a = 0; a < c->dims; a++) cells *= c->patch[a];
        if (cells > kMergeCells) return "merging needs patches of at most 4096 cells";
    }
    if (c->split_below < 0 || c->split_below > kSplitBelowMax) return "split_below in [0, 64]";
    if (c->split_below > 0) {
        if (!(c->split_wmin >= 0) || !std::isfinite(c->split_wmin))
            return "split_wmin must be finite and >= 0";
        long long cells = 1;
        for (int a = 0; a < c->dims; a++) cells *= c->patch[a];
        if (cells > kMergeCells) return "splitting needs patches of at most 4096 cells";
    }
    if (c->window) {
        if (!(c->ramp_len > 0)) return "ramp_len must be positive";
        for (int a = 0; a < c->dims; a++)
            if (c->inject_ppc[a] < 1 || c->inject_ppc[a] > 16) return "inject_ppc in [1,16]";
    }
    return nullptr;
}

// Geometry + arena carve (base == nullptr: dry run for the byte count).
Layout plan(const pic_config* c, char* base) {
    Layout L;
    Carver cv{base, base == nullptr};
    SimDev& S = L.S;
    S.dims = c->dims;
    S.prec = c->precision;
    S.window = c->window;
    S.mapping = c->mapping;
    S.merge_above = c->merge_above;
    S.merge_dp = c->merge_dp;
    S.split_below = c->split_below;
    S.split_wmin = c->split_wmin;
    S.order = c->maxwell_order == 6 ? 6 : 2;
    for (int a = 0; a < 3; a++) {
        S.n[a] = a < c->dims ? c->n[a] : 1;
        S.P[a] = a < c->dims ? c->patch[a] : 1;
        S.np[a] = S.n[a] / S.P[a];
        S.d[a] = a < c->dims ? c->d[a] : 1.0;
        S.ippc[a] = a < c->dims ? std::max(1, c->inject_ppc[a]) : 1;
    }
    S.npatch = S.np[0] * S.np[1] * S.np[2];
    // TMA box: interior [p0-1, p0+P+3) in x (P + 4 columns, 16-byte rows), P + 3 rows
    S.BX = S.P[0] + 4;
    S.BY = S.P[1] + 3;
    S.BZ = c->dims == 3 ? S.P[2] + 3 : 1;
    S.NX = S.n[0] + 4;
    S.NY = S.n[1] + 3;
    S.NZ = c->dims == 3 ? S.n[2] + 3 : 1;
    S.fstride = (long long)S.NX * S.NY * S.NZ;
    S.dt = c->dt;
    S.q = c->q;
    S.m = c->m;
    S.n0 = c->n0;
    S.ramp_x0 = c->ramp_x0;
    S.ramp_len = c->ramp_len;
    S.ncell = (long long)S.n[0] * S.n[1] * S.n[2];
    {
        const double dV = S.d[0] * S.d[1] * (c->dims == 3 ? S.d[2] : 1.0);
        const double qdv = S.q / dV;
        for (int a = 0; a < 3; a++) {
            S.c_dtd[a] = S.dt / S.d[a];
            S.c_j[a] = -qdv * S.d[a] / S.dt;
        }
        if (c->dims == 2) S.c_j[2] = qdv;
        S.c_eps = S.q * S.dt / (2.0 * S.m);
        for (int a = 0; a < 3; a++) {
            S.f_dtd[a] = (float)S.c_dtd[a];
            S.f_j[a] = (float)S.c_j[a];
        }
        S.f_eps = (float)S.c_eps;
        S.f_dt = (float)S.dt;
        S.f_dt_lo = (float)(S.dt - (double)S.f_dt);
        for (int a = 0; a < 3; a++) {
            S.c_id[a] = 1.0 / S.d[a];
            S.f_id[a] = (float)S.c_id[a];
            S.f_id_lo[a] = (float)(S.c_id[a] - (double)S.f_id[a]);
        }
        // sixth-order staggered difference: the coefficients fixed by exactness up to
        // degree 6, pre-divided by the cell size
        const double c6[3] = {75.0 / 64.0, -25.0 / 384.0, 3.0 / 640.0};
        for (int a = 0; a < 3; a++)
            for (int l = 0; l < 3; l++) {
                S.c_k[a][l] = c6[l] / S.d[a];
                S.f_k[a][l] = (float)S.c_k[a][l];
                S.f_k_lo[a][l] = (float)(S.c_k[a][l] - (double)S.f_k[a][l]);
            }
    }
    const long long es = c->precision == PIC_FP32 ? 4 : 8;
    // slots: the configured capacity plus one alignment's slack per patch, so that every
    // per-patch base can be a multiple of kSlotAlign
    S.ucap = c->capacity;
    S.capacity = align_slots(c->capacity) + (long long)kSlotAlign * S.npatch;
    const long long cap = S.capacity;

    L.ds = cv.take<SimDev>(1);
    L.db = cv.take<BatchDev>(1);
    L.prefix = cv.take<int>(2);
    S.tmap = cv.take<CUtensorMap>(2, 128);
    S.st = cv.take<StepState>(1);
    S.status = cv.take<int>(1);
    S.red = cv.take<double>(8);
    for (int g = 0; g < 2; g++) S.F[g] = cv.take<char>(6 * S.fstride * es);
    for (int g = 0; g < 2; g++) S.H[g] = cv.take<char>(3 * S.fstride * es);
    for (int g = 0; g < 2; g++) S.J[g] = cv.take<double>(3 * S.fstride);
    S.rho = cv.take<double>(S.ncell);
    S.rho_bg = cv.take<double>(S.ncell);
    S.cell = c->precision != PIC_FP64 ? cv.take<int>(cap) : nullptr;
    for (int a = 0; a < 3; a++) S.xi[a] = a < c->dims ? cv.take<char>(cap * es) : nullptr;
    for (int a = 0; a < 3; a++) S.u[a] = cv.take<char>(cap * es);
    S.w = cv.take<char>(cap * es);
    S.id = cv.take<int>(cap);
    S.holes = cv.take<int>(cap);
    S.aux = cv.take<int>(cap);
    S.pbase = cv.take<int>(S.npatch);
    S.pcap = cv.take<int>(S.npatch);
    S.pcount = cv.take<int>(S.npatch);
    S.hcount = cv.take<int>(S.npatch);
    S.mbase = cv.take<int>(S.npatch);
    S.mcap = cv.take<int>(S.npatch);
    S.mcount = cv.take<int>(S.npatch);
    // exchange-buffer slots: room for the per-patch minimum, half of every capacity and
    // for the arrival-driven enlargements a repack may grant
    S.mtotal = cap + (long long)(kMailboxMin + kSlotAlign) * S.npatch;
    S.mcell = c->precision != PIC_FP64 ? cv.take<int>(S.mtotal) : nullptr;
    for (int a = 0; a < 3; a++) S.mxi[a] = a < c->dims ? cv.take<char>(S.mtotal * es) : nullptr;
    for (int a = 0; a < 3; a++) S.mu[a] = cv.take<char>(S.mtotal * es);
    S.mw = cv.take<char>(S.mtotal * es);
    S.mid = cv.take<int>(S.mtotal);
    S.acell = c->precision != PIC_FP64 ? cv.take<int>(cap) : nullptr;
    for (int a = 0; a < 3; a++) S.axi[a] = a < c->dims ? cv.take<char>(cap * es) : nullptr;
    for (int a = 0; a < 3; a++) S.au[a] = cv.take<char>(cap * es);
    S.aw = cv.take<char>(cap * es);
    S.aid = cv.take<int>(cap);
    S.pbase_new = cv.take<int>(S.npatch);
    S.pcap_new = cv.take<int>(S.npatch);
    S.mbase_new = cv.take<int>(S.npatch);
    S.mcap_new = cv.take<int>(S.npatch);
    S.mpend = cv.take<int>(S.npatch);
    S.mpoff = cv.take<int>(S.npatch);
    S.mlast = cv.take<int>(S.npatch);
    S.soff = cv.take<int>(S.npatch + 1);
    // sixth order in a moving window: E^{n+1} of the column the shift drops, which the
    // B update of the new frame's first columns still reads
    S.ecol = S.order == 6 && c->window ? cv.take<char>(3 * (long long)S.n[1] * S.n[2] * es)
                                       : nullptr;

    BatchDev& B = L.B;
    B.nsims = 1;
    B.chunk = default_chunk(c);
    B.max_items = (int)std::min<long long>(S.npatch + cap / std::max(1, B.chunk) + 64, 1LL << 30);
    B.total_patches = S.npatch;
    B.max_patches = S.npatch;
    B.max_ncell = (int)S.ncell;
    B.items = cv.take<int4>(B.max_items);
    B.nitems = cv.take<int>(1);
    B.head = cv.take<int>(1);
    B.sims = L.ds;
    B.patch_prefix = L.prefix;
    L.bytes = cv.off + 256;
    return L;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// One tensor map per field generation: the six components E, B^n of F[g] as a
// (x, y, component) tensor; the box is one patch tile plus guards.
bool encode_field_maps(const SimDev& S, CUtensorMap out[2]) {
    auto fn = encode_fn();
    if (!fn) return false;
    // 8-byte elements (FP64 or a double-word pair) move as FLOAT64; TMA copies bytes
    const cuuint64_t es = S.prec == PIC_FP32 ? 4 : 8;
    const CUtensorMapDataType dt =
        S.prec == PIC_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    for (int g = 0; g < 2; g++) {
        CUresult r;
        if (S.dims == 2) {
            cuuint64_t dims[3] = {(cuuint64_t)S.NX, (cuuint64_t)S.NY, 6};
            cuuint64_t strides[2] = {(cuuint64_t)S.NX * es, (cuuint64_t)S.NX * S.NY * es};
            cuuint32_t box[3] = {(cuuint32_t)S.BX, (cuuint32_t)S.BY, 6};
            cuuint32_t estr[3] = {1, 1, 1};
            r = fn(&out[g], dt, 3, S.F[g], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        } else {
            // (x, y, z, component) with a 4D box: one patch tile of all six components
            cuuint64_t dims[4] = {(cuuint64_t)S.NX, (cuuint64_t)S.NY, (cuuint64_t)S.NZ, 6};
            cuuint64_t strides[3] = {(cuuint64_t)S.NX * es, (cuuint64_t)S.NX * S.NY * es,
                                     (cuuint64_t)S.NX * S.NY * S.NZ * es};
            cuuint32_t box[4] = {(cuuint32_t)S.BX, (cuuint32_t)S.BY, (cuuint32_t)S.BZ, 6};
            cuuint32_t estr[4] = {1, 1, 1, 1};
            r = fn(&out[g], dt, 4, S.F[g], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

pic_status fail(std::string* err, pic_status st, const std::string& msg) {
    if (err) *err = msg;
    return st;
}

pic_status cuda_fail(std::string* err, cudaError_t e, const char* where) {
    return fail(err, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// No C++ exception crosses the C ABI. A failed host allocation or thread start inside an
// entry point becomes PIC_ERR_NOMEM; any other exception becomes PIC_ERR_INVALID. The
// message is kept when there is memory for it.
pic_status note(std::string* err, pic_status st, const char* msg) noexcept {
    try {
        if (err) *err = msg;
    } catch (...) {
    }
    return st;
}

template <typename F>
pic_status guarded(std::string* err, F&& body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return note(err, PIC_ERR_NOMEM, "host memory allocation failed");
    } catch (const std::system_error& e) {
        return note(err, PIC_ERR_NOMEM, e.what());
    } catch (const std::exception& e) {
        return note(err, PIC_ERR_INVALID, e.what());
    } catch (...) {
        return note(err, PIC_ERR_INVALID, "unexpected host exception");
    }
}

template <typename F>
size_t guarded_size(F&& body) noexcept {
    try {
        return body();
    } catch (...) {
        return 0;
    }
}

#define CK(call, where)                                                \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail(&s->err, e_, where);   \
    } while (0)

pic_status status_to_error(std::string* err, int st) {
    if (st == 0) return PIC_OK;
    if (st & ST_TIMEOUT) return fail(err, PIC_ERR_TIMEOUT, "a bounded device wait expired");
    if (st & ST_CAPACITY)
        return fail(err, PIC_ERR_CAPACITY, "more particles than the arena's capacity");
    if (st & ST_MAILBOX) return fail(err, PIC_ERR_CAPACITY, "an exchange buffer overflowed");
    if (st & ST_QUEUE) return fail(err, PIC_ERR_CAPACITY, "the work queue overflowed");
    if (st & ST_NUMERIC)
        return fail(err, PIC_ERR_NUMERIC, "non-finite particle state or a move of a cell or more");
    return fail(err, PIC_ERR_CUDA, "unknown device status");
}

struct GraphOwner {
    cudaStream_t* cap0;
    cudaStream_t* cap1;
    cudaEvent_t* ev_fork;
    cudaEvent_t* ev_join;
    cudaGraph_t* graph;
    cudaGraphExec_t* gexec;
};

// Captures one step into a graph: queue build -> particle kernel -> (Yee on a
// second branch) | (injection -> exchange) -> end of step.
cudaError_t capture_step(GraphOwner o, const BatchDev* db, int nsims, int max_patches,
                         int max_ncell, int max_column, int dims, int prec, int order,
                         int mapping, const int P[3], int grid, bool window, bool merge,
                         bool split) {
    cudaError_t e;
    if (!*o.cap0) {
        if ((e = cudaStreamCreateWithFlags(o.cap0, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(o.cap1, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(o.ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(o.ev_join, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaStreamBeginCapture(*o.cap0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
    cudaError_t le = launch_queue_build(db, *o.cap0);
    if (le == cudaSuccess) le = launch_push(db, dims, prec, mapping, P[0], P[1], P[2], grid, *o.cap0);
    if (le == cudaSuccess) le = cudaEventRecord(*o.ev_fork, *o.cap0);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(*o.cap1, *o.ev_fork, 0);
    if (le == cudaSuccess) le = launch_yee(db, nsims, max_ncell, dims, prec, order, *o.cap1);
    if (le == cudaSuccess) le = cudaEventRecord(*o.ev_join, *o.cap1);
    if (le == cudaSuccess && window) le = launch_inject(db, nsims, max_column, prec, *o.cap0);
    if (le == cudaSuccess) le = launch_exchange(db, nsims, max_patches, prec, *o.cap0);
    if (le == cudaSuccess && merge) le = launch_merge(db, nsims, max_patches, prec, *o.cap0);
    if (le == cudaSuccess && split) le = launch_split(db, nsims, max_patches, prec, *o.cap0);
    if (le == cudaSuccess) le = launch_repack(db, nsims, max_patches, prec, *o.cap0);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(*o.cap0, *o.ev_join, 0);
    if (le == cudaSuccess) le = launch_end_step(db, nsims, max_patches, *o.cap0);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(*o.cap0, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    if (*o.gexec) cudaGraphExecDestroy(*o.gexec);
    if (*o.graph) cudaGraphDestroy(*o.graph);
    *o.graph = g;
    *o.gexec = nullptr;
    return cudaGraphInstantiate(o.gexec, g, 0);
}

void destroy_graph_owner(GraphOwner o) {
    if (*o.gexec) cudaGraphExecDestroy(*o.gexec);
    if (*o.graph) cudaGraphDestroy(*o.graph);
    if (*o.ev_fork) cudaEventDestroy(*o.ev_fork);
    if (*o.ev_join) cudaEventDestroy(*o.ev_join);
    if (*o.cap0) cudaStreamDestroy(*o.cap0);
    if (*o.cap1) cudaStreamDestroy(*o.cap1);
}

// Grid of the particle kernel: one CTA per patch (static mapping) or the number of
// CTAs resident at once (persistent queue). Also sets the kernel's shared-memory
// attribute, which every launch needs.
int push_grid_size(int dims, int prec, const int P[3], bool static_map, int npatch) {
    int dev = 0, nsm = 0, smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per = push_occupancy(dims, prec, P[0], P[1], P[2], &smem);
    if (per < 1) per = 1;
    return static_map ? std::max(1, npatch) : nsm * per;
}

template <typename T>
void unpad_field(const SimDev& S, const T* src, double* dst) {
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const long long pi =
                    ((long long)(S.dims == 3 ? k + kGuard : 0) * S.NY + (j + kGuard)) * S.NX +
                    (i + kGuard);
                dst[((long long)k * ny + j) * nx + i] = (double)src[pi];
            }
}

size_t elem_size(int prec) { return prec == PIC_FP32 ? 4 : 8; }

double load_real(int prec, const void* a, long long i) {
    if (prec == PIC_FP64) return static_cast<const double*>(a)[i];
    if (prec == PIC_FP32) return (double)static_cast<const float*>(a)[i];
    return (double)static_cast<const df64*>(a)[i];
}

}  // namespace

// ===================================================================== C ABI

extern "C" size_t pic_config_bytes(void) { return sizeof(pic_config); }

static pic_status selftest_bounded_wait_body(void* cuda_stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return PIC_ERR_CUDA;
    int h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_bounded_wait_selftest(d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return PIC_ERR_CUDA;
    std::string err;
    return status_to_error(&err, h);
}

extern "C" pic_status pic_selftest_bounded_wait(void* cuda_stream) {
    return guarded(nullptr, [&] { return selftest_bounded_wait_body(cuda_stream); });
}

static size_t required_bytes_body(const pic_config* cfg) {
    if (validate(cfg)) return 0;
    return plan(cfg, nullptr).bytes;
}

extern "C" size_t pic_required_bytes(const pic_config* cfg) {
    return guarded_size([&] { return required_bytes_body(cfg); });
}

static pic_status create_body(const pic_config* cfg, void* dev_arena, size_t arena_bytes,
                              void* cuda_stream, pic_sim** out) {
    if (!out) return PIC_ERR_INVALID;
    *out = nullptr;
    if (validate(cfg)) return PIC_ERR_INVALID;
    if (!dev_arena || (reinterpret_cast<uintptr_t>(dev_arena) & 255)) return PIC_ERR_INVALID;
    if (arena_bytes < plan(cfg, nullptr).bytes) return PIC_ERR_NOMEM;
    pic_sim* s = new (std::nothrow) pic_sim();
    if (!s) return PIC_ERR_NOMEM;
    s->cfg = *cfg;
    s->arena = static_cast<char*>(dev_arena);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->L = plan(cfg, s->arena);
    const SimDev& S = s->L.S;
    s->column_pts = cfg->window ? S.n[1] * S.ippc[0] * S.ippc[1] *
                                      (S.dims == 3 ? S.n[2] * S.ippc[2] : 1)
                                : 0;
    auto bail = [&](pic_status st) {
        GraphOwner o{&s->cap0, &s->cap1, &s->ev_fork, &s->ev_join, &s->graph, &s->gexec};
        destroy_graph_owner(o);
        delete s;
        return st;
    };
    if (cudaMemsetAsync(s->arena, 0, s->L.bytes - 256, s->stream) != cudaSuccess)
        return bail(PIC_ERR_CUDA);
    CUtensorMap maps[2];
    if (!encode_field_maps(S, maps)) return bail(PIC_ERR_CUDA);
    int prefix[2] = {0, S.npatch};
    if (cudaMemcpyAsync((void*)S.tmap, maps, sizeof(maps), cudaMemcpyHostToDevice, s->stream) ||
        cudaMemcpyAsync(s->L.ds, &S, sizeof(SimDev), cudaMemcpyHostToDevice, s->stream) ||
        cudaMemcpyAsync(s->L.db, &s->L.B, sizeof(BatchDev), cudaMemcpyHostToDevice, s->stream) ||
        cudaMemcpyAsync(s->L.prefix, prefix, sizeof(prefix), cudaMemcpyHostToDevice, s->stream))
        return bail(PIC_ERR_CUDA);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return bail(PIC_ERR_CUDA);
    s->push_grid = push_grid_size(S.dims, S.prec, S.P, cfg->mapping == PIC_MAP_STATIC, S.npatch);
    if (S.split_below > 0 && split_setup() != cudaSuccess) return bail(PIC_ERR_CUDA);
    GraphOwner o{&s->cap0, &s->cap1, &s->ev_fork, &s->ev_join, &s->graph, &s->gexec};
    if (capture_step(o, s->L.db, 1, S.npatch, (int)S.ncell, s->column_pts, S.dims, S.prec,
                     S.order, S.mapping, S.P, s->push_grid, S.window != 0,
                     S.merge_above > 0, S.split_below > 0) != cudaSuccess)
        return bail(PIC_ERR_CUDA);
    *out = s;
    return PIC_OK;
}

extern "C" pic_status pic_create(const pic_config* cfg, void* dev_arena, size_t arena_bytes,
                                 void* cuda_stream, pic_sim** out) {
    return guarded(nullptr,
                   [&] { return create_body(cfg, dev_arena, arena_bytes, cuda_stream, out); });
}

static pic_status load_particles_body(pic_sim* s, long long n, const double* x,
                                      const double* y, const double* z, const double* ux,
                                      const double* uy, const double* uz, const double* w,
                                      const int* id) {
    if (!s) return PIC_ERR_INVALID;
    const SimDev& S = s->L.S;
    if (n < 0) return fail(&s->err, PIC_ERR_INVALID, "negative particle count");
    if (n > S.ucap) return fail(&s->err, PIC_ERR_CAPACITY, "more particles than capacity");
    if (n > 0 && (!x || !y || !ux || !uy || !uz || !w || !id || (S.dims == 3 && !z)))
        return fail(&s->err, PIC_ERR_INVALID, "null particle array");
    CK(cudaStreamSynchronize(s->stream), "sync before load");
    // every return waits for the stream, so no copy from the caller's arrays outlives
    // the call
    struct Drain {
        cudaStream_t st;
        ~Drain() { cudaStreamSynchronize(st); }
    } drain{s->stream};
    const int dims = S.dims;
    const double* pos[3] = {x, y, z};
    const double* mom[3] = {ux, uy, uz};
    // the caller's arrays go to the device as they are, in chunks that fit the repack
    // scratch (FP64 values, so a 4-byte precision takes half its slots per chunk)
    const size_t es = elem_size(S.prec);
    const long long cap = S.capacity;
    const long long chunk = cap * (long long)es / (long long)sizeof(double);
    auto copy_chunk = [&](long long k0, long long m) -> cudaError_t {
        const size_t db = m * sizeof(double);
        cudaError_t e = cudaSuccess;
        for (int a = 0; a < dims && e == cudaSuccess; a++)
            e = cudaMemcpyAsync(S.axi[a], pos[a] + k0, db, cudaMemcpyHostToDevice, s->stream);
        for (int a = 0; a < 3 && e == cudaSuccess; a++)
            e = cudaMemcpyAsync(S.au[a], mom[a] + k0, db, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S.aw, w + k0, db, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S.aid, id + k0, m * sizeof(int), cudaMemcpyHostToDevice, s->stream);
        return e;
    };
    // pass 1 on the device, chunk by chunk: validation, patch and bank class, rank within
    // (patch, class); only scratch is written (see load_bin_kernel)
    const size_t ccount_bytes = (size_t)S.npatch * 32 * sizeof(int);
    std::vector<int> ccount(S.npatch * 32, 0);
    unsigned long long red[3] = {~0ULL, 0ULL, 0ULL};
    if (n > 0) {
        CK(cudaMemsetAsync(S.rho, 0, ccount_bytes, s->stream), "zero counters");
        CK(cudaMemcpyAsync(S.red, red, sizeof(red), cudaMemcpyHostToDevice, s->stream),
           "init reductions");
        for (long long k0 = 0; k0 < n; k0 += chunk) {
            const long long m = std::min(chunk, n - k0);
            CK(copy_chunk(k0, m), "copy particles");
            CK(launch_load_bin(s->L.db, m, k0, s->stream), "bin particles");
        }
        CK(cudaMemcpyAsync(red, S.red, sizeof(red), cudaMemcpyDeviceToHost, s->stream),
           "read reductions");
        CK(cudaMemcpyAsync(ccount.data(), S.rho, ccount_bytes, cudaMemcpyDeviceToHost, s->stream),
           "read counters");
        CK(cudaStreamSynchronize(s->stream), "bin particles");
    }
    if (red[0] != ~0ULL) {  // the first invalid particle of the call
        const int code = (int)(red[0] & 3ULL);
        if (code == 1) return fail(&s->err, PIC_ERR_INVALID, "particle position outside the grid");
        if (code == 2) return fail(&s->err, PIC_ERR_NUMERIC, "non-finite particle momentum or weight");
        return fail(&s->err, PIC_ERR_INVALID, "negative particle id");
    }
    std::vector<int> counts(S.npatch, 0);
    for (int p = 0; p < S.npatch; p++)
        for (int q = 0; q < 32; q++) counts[p] += ccount[p * 32 + q];
    const int maxid = n > 0 ? (int)red[1] : -1;
    double wmax = 0.0;
    std::memcpy(&wmax, &red[2], sizeof(wmax));
    // per-patch capacity: the free slots are shared half by count, half evenly; every
    // capacity is rounded up to kSlotAlign so that all bases stay aligned
    const long long spare = S.ucap - n;
    std::vector<int> pcap(S.npatch), pbase(S.npatch), mcap(S.npatch), mbase(S.npatch);
    long long acc = 0, macc = 0;
    for (int p = 0; p < S.npatch; p++) {
        double share = n > 0 ? 0.5 * (double)counts[p] / (double)n + 0.5 / S.npatch : 1.0 / S.npatch;
        long long c = align_slots(counts[p] + (long long)std::floor((double)spare * share));
        pcap[p] = (int)c;
        pbase[p] = (int)acc;
        acc += c;
        mcap[p] = (int)align_slots(std::max(kMailboxMin, pcap[p] / kMailboxDiv));
        mbase[p] = (int)macc;
        macc += mcap[p];
    }
    if (acc > S.capacity || macc > S.mtotal)
        return fail(&s->err, PIC_ERR_CAPACITY, "capacity split failed");
    // the load is accepted: from here on the sim's state is replaced
    const size_t pb = S.npatch * sizeof(int);
    CK(cudaMemcpyAsync(S.pbase, pbase.data(), pb, cudaMemcpyHostToDevice, s->stream), "copy pbase");
    // pass 2: every particle's slot (patch base plus its place in the bank-class run order)
    CK(launch_load_slot(s->L.db, n, s->stream), "order particles");
    // pass 3: clear every slot (zero state, id -1), then per chunk the device converts and
    // places the particles; the last chunk of pass 1 is still staged, so it goes first
    for (int a = 0; a < dims; a++) CK(cudaMemsetAsync(S.xi[a], 0, cap * es, s->stream), "clear x");
    for (int a = 0; a < 3; a++) CK(cudaMemsetAsync(S.u[a], 0, cap * es, s->stream), "clear u");
    CK(cudaMemsetAsync(S.w, 0, cap * es, s->stream), "clear w");
    CK(cudaMemsetAsync(S.id, 0xFF, cap * sizeof(int), s->stream), "clear id");
    if (S.prec != PIC_FP64) CK(cudaMemsetAsync(S.cell, 0, cap * sizeof(int), s->stream), "clear cell");
    if (n > 0) {
        const long long last = ((n - 1) / chunk) * chunk;
        for (long long k0 = last; k0 >= 0; k0 -= chunk) {
            const long long m = std::min(chunk, n - k0);
            if (k0 != last) CK(copy_chunk(k0, m), "copy particles");
            CK(launch_load_scatter(s->L.db, m, k0, S.prec, s->stream), "place particles");
        }
    }
    CK(cudaMemcpyAsync(S.pcap, pcap.data(), pb, cudaMemcpyHostToDevice, s->stream), "copy pcap");
    CK(cudaMemcpyAsync(S.pcount, counts.data(), pb, cudaMemcpyHostToDevice, s->stream), "copy pcount");
    CK(cudaMemcpyAsync(S.mbase, mbase.data(), pb, cudaMemcpyHostToDevice, s->stream), "copy mbase");
    CK(cudaMemcpyAsync(S.mcap, mcap.data(), pb, cudaMemcpyHostToDevice, s->stream), "copy mcap");
    CK(cudaMemsetAsync(S.hcount, 0, pb, s->stream), "zero hcount");
    CK(cudaMemsetAsync(S.mcount, 0, pb, s->stream), "zero mcount");
    CK(cudaMemsetAsync(S.mlast, 0, pb, s->stream), "zero mlast");
    // bound of one particle's current contribution (|cumulative DS| <= 1, |v| < 1):
    // sets the double-word fixed-point current scale
    {
        if (S.window) {
            const double dV = S.d[0] * S.d[1] * (S.dims == 3 ? S.d[2] : 1.0);
            wmax = std::max(wmax, std::fabs(S.n0) * dV /
                                      ((double)S.ippc[0] * S.ippc[1] * (S.dims == 3 ? S.ippc[2] : 1)));
        }
        double cj = 0.0;
        for (int a = 0; a < 3; a++) cj = std::max(cj, std::fabs(S.c_j[a]));
        const double cmax = cj * wmax;
        int e = -100;
        if (cmax > 0) std::frexp(cmax, &e);  // cmax < 2^e
        s->L.S.cmax_exp = e;
        CK(cudaMemcpyAsync(s->L.ds, &s->L.S, sizeof(SimDev), cudaMemcpyHostToDevice, s->stream),
           "copy descriptor");
    }
    StepState st{};
    st.next_id = (long long)maxid + 1;
    CK(cudaMemcpyAsync(S.st, &st, sizeof(st), cudaMemcpyHostToDevice, s->stream), "copy state");
    CK(cudaMemsetAsync(S.status, 0, sizeof(int), s->stream), "zero status");
    CK(cudaStreamSynchronize(s->stream), "load particles");
    return PIC_OK;
}

extern "C" pic_status pic_load_particles(pic_sim* s, long long n, const double* x,
                                         const double* y, const double* z, const double* ux,
                                         const double* uy, const double* uz, const double* w,
                                         const int* id) {
    return guarded(s ? &s->err : nullptr,
                   [&] { return load_particles_body(s, n, x, y, z, ux, uy, uz, w, id); });
}

static pic_status load_fields_body(pic_sim* s, const double* const E[3],
                                   const double* const B[3], const double* rho_bg) {
    if (!s || !E || !B) return PIC_ERR_INVALID;
    for (int a = 0; a < 3; a++)
        if (!E[a] || !B[a]) return fail(&s->err, PIC_ERR_INVALID, "null field array");
    const SimDev& S = s->L.S;
    CK(cudaStreamSynchronize(s->stream), "sync before fields");
    const size_t es = elem_size(S.prec);
    const long long fs = S.fstride, nc = S.ncell;
    // the caller's arrays go as they are to the current buffers (3 fstride >= 3 ncell
    // values each), the device pads them into generation 0 in the sim's precision
    for (int a = 0; a < 3; a++) {
        CK(cudaMemcpyAsync(S.J[0] + a * nc, E[a], nc * sizeof(double), cudaMemcpyHostToDevice,
                           s->stream), "copy E");
        CK(cudaMemcpyAsync(S.J[1] + a * nc, B[a], nc * sizeof(double), cudaMemcpyHostToDevice,
                           s->stream), "copy B");
    }
    CK(launch_load_fields(s->L.ds, fs, S.prec, s->stream), "pad fields");
    CK(cudaMemsetAsync(S.F[1], 0, 6 * fs * es, s->stream), "zero F1");
    CK(cudaMemsetAsync(S.H[1], 0, 3 * fs * es, s->stream), "zero H1");
    CK(cudaMemsetAsync(S.J[0], 0, 3 * fs * sizeof(double), s->stream), "zero J0");
    CK(cudaMemsetAsync(S.J[1], 0, 3 * fs * sizeof(double), s->stream), "zero J1");
    // the fields belong to step 0
    StepState st{};
    CK(cudaMemcpyAsync(&st, S.st, sizeof(st), cudaMemcpyDeviceToHost, s->stream), "read state");
    CK(cudaStreamSynchronize(s->stream), "read state");
    st.step = 0;
    st.nshift = 0;
    st.gen = 0;
    st.shift = 0;
    CK(cudaMemcpyAsync(S.st, &st, sizeof(st), cudaMemcpyHostToDevice, s->stream), "write state");
    if (rho_bg) {
        CK(cudaMemcpyAsync(S.rho_bg, rho_bg, S.ncell * sizeof(double), cudaMemcpyHostToDevice,
                           s->stream),
           "copy rho_bg");
    } else {
        CK(launch_gauss(s->L.ds, S, S.prec, 0, s->stream), "rho_bg");
    }
    CK(cudaStreamSynchronize(s->stream), "load fields");
    return PIC_OK;
}

extern "C" pic_status pic_load_fields(pic_sim* s, const double* const E[3], const double* const B[3],
                                      const double* rho_bg) {
    return guarded(s ? &s->err : nullptr, [&] { return load_fields_body(s, E, B, rho_bg); });
}

extern "C" pic_status pic_step(pic_sim* s, int nsteps) {
    if (!s || nsteps < 0) return PIC_ERR_INVALID;
    for (int i = 0; i < nsteps; i++) CK(cudaGraphLaunch(s->gexec, s->stream), "graph launch");
    return PIC_OK;
}

extern "C" pic_status pic_sync(pic_sim* s) {
    if (!s) return PIC_ERR_INVALID;
    CK(cudaStreamSynchronize(s->stream), "sync");
    int st = 0;
    CK(cudaMemcpy(&st, s->L.S.status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    return status_to_error(&s->err, st);
}

static pic_status diag_body(pic_sim* s, int kind, void* out, size_t out_bytes, size_t* written) {
    if (!s) return PIC_ERR_INVALID;
    if (written) *written = 0;
    pic_status rc = pic_sync(s);
    if (rc != PIC_OK) return rc;
    const SimDev& S = s->L.S;
    const size_t es = elem_size(S.prec);
    auto need = [&](size_t b) { return out && out_bytes >= b; };
    StepState st{};
    CK(cudaMemcpy(&st, S.st, sizeof(st), cudaMemcpyDeviceToHost), "read state");
    const int g = (int)(st.step & 1);
    std::vector<int> counts(S.npatch);
    auto read_counts = [&]() -> cudaError_t {
        return cudaMemcpy(counts.data(), S.pcount, S.npatch * sizeof(int), cudaMemcpyDeviceToHost);
    };
    switch (kind) {
        case PIC_DIAG_ENERGY: {
            if (!need(3 * sizeof(double))) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            CK(cudaMemsetAsync(S.red, 0, 8 * sizeof(double), s->stream), "zero red");
            CK(launch_energy(s->L.ds, S.ncell, S.capacity, S.prec, s->stream), "energy");
            double r[3];
            CK(cudaMemcpyAsync(r, S.red, sizeof(r), cudaMemcpyDeviceToHost, s->stream), "read red");
            CK(cudaStreamSynchronize(s->stream), "energy");
            const double dV = S.d[0] * S.d[1] * (S.dims == 3 ? S.d[2] : 1.0);
            double* o = static_cast<double*>(out);
            o[0] = 0.5 * r[0] * dV;
            o[1] = 0.5 * r[1] * dV;
            o[2] = r[2];
            if (written) *written = 3 * sizeof(double);
            return PIC_OK;
        }
        case PIC_DIAG_GAUSS: {
            const size_t b = S.ncell * sizeof(double);
            if (!need(b)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            CK(launch_gauss(s->L.ds, S, S.prec, 1, s->stream), "gauss");
            CK(cudaMemcpyAsync(out, S.rho, b, cudaMemcpyDeviceToHost, s->stream), "read gauss");
            CK(cudaStreamSynchronize(s->stream), "gauss");
            if (written) *written = b;
            return PIC_OK;
        }
        case PIC_DIAG_EX_AXIS: {
            // the row (j, k) = (ny/2, nz/2) of Ex is contiguous in the padded array
            const int nx = S.n[0];
            const size_t b = nx * sizeof(double);
            if (!need(b)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            const long long row =
                ((long long)(S.dims == 3 ? S.n[2] / 2 + kGuard : 0) * S.NY + (S.n[1] / 2 + kGuard)) *
                    S.NX + kGuard;
            std::vector<char> h(nx * es);
            CK(cudaMemcpy(h.data(), static_cast<const char*>(S.F[g]) + row * es, h.size(),
                          cudaMemcpyDeviceToHost),
               "read Ex");
            double* o = static_cast<double*>(out);
            for (int i = 0; i < nx; i++) o[i] = load_real(S.prec, h.data(), i);
            if (written) *written = b;
            return PIC_OK;
        }
        case PIC_DIAG_FIELDS: {
            const long long nc = S.ncell, fs = S.fstride;
            const size_t b = 12 * nc * sizeof(double);
            if (!need(b)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            std::vector<char> hF(6 * fs * es), hH(3 * fs * es);
            std::vector<double> hJ(3 * fs);
            CK(cudaMemcpy(hF.data(), S.F[g], hF.size(), cudaMemcpyDeviceToHost), "read F");
            CK(cudaMemcpy(hH.data(), S.H[g], hH.size(), cudaMemcpyDeviceToHost), "read H");
            CK(cudaMemcpy(hJ.data(), S.J[1 - g], hJ.size() * sizeof(double), cudaMemcpyDeviceToHost),
               "read J");
            std::vector<double> all(12 * nc);
            auto unpad_all = [&](const auto* F, const auto* H) {
                for (int a = 0; a < 3; a++) {
                    unpad_field(S, F + a * fs, &all[(0 + a) * nc]);
                    unpad_field(S, H + a * fs, &all[(3 + a) * nc]);
                    unpad_field(S, F + (3 + a) * fs, &all[(6 + a) * nc]);
                }
            };
            if (S.prec == PIC_FP64)
                unpad_all(reinterpret_cast<double*>(hF.data()), reinterpret_cast<double*>(hH.data()));
            else if (S.prec == PIC_FP32)
                unpad_all(reinterpret_cast<float*>(hF.data()), reinterpret_cast<float*>(hH.data()));
            else
                unpad_all(reinterpret_cast<df64*>(hF.data()), reinterpret_cast<df64*>(hH.data()));
            for (int a = 0; a < 3; a++) unpad_field(S, hJ.data() + a * fs, &all[(9 + a) * nc]);
            memcpy(out, all.data(), b);
            if (written) *written = b;
            return PIC_OK;
        }
        case PIC_DIAG_NUM_PARTICLES: {
            if (!need(sizeof(long long))) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            CK(read_counts(), "read counts");
            long long n = 0;
            for (int c : counts) n += c;
            *static_cast<long long*>(out) = n;
            if (written) *written = sizeof(long long);
            return PIC_OK;
        }
        case PIC_DIAG_PATCH_COUNTS: {
            const size_t b = S.npatch * sizeof(int);
            if (!need(b)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            CK(read_counts(), "read counts");
            memcpy(out, counts.data(), b);
            if (written) *written = b;
            return PIC_OK;
        }
        case PIC_DIAG_STEP: {
            if (!need(3 * sizeof(long long))) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            long long* o = static_cast<long long*>(out);
            o[0] = st.step;
            o[1] = st.nshift;
            o[2] = st.nrepack;
            size_t wb = 3 * sizeof(long long);
            if (out_bytes >= 4 * sizeof(long long)) {
                o[3] = st.nmerged;
                wb = 4 * sizeof(long long);
            }
            if (out_bytes >= 5 * sizeof(long long)) {
                o[4] = st.nsplit;
                wb = 5 * sizeof(long long);
            }
            if (written) *written = wb;
            return PIC_OK;
        }
        case PIC_DIAG_PARTICLES: {
            CK(read_counts(), "read counts");
            long long n = 0;
            for (int c : counts) n += c;
            const size_t b = (size_t)n * (7 * sizeof(double) + sizeof(int));
            if (!need(b)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            const long long cap = S.capacity;
            std::vector<char> hx[3], hu[3], hw(cap * es);
            std::vector<int> hid(cap), hcell;
            for (int a = 0; a < S.dims; a++) {
                hx[a].resize(cap * es);
                CK(cudaMemcpy(hx[a].data(), S.xi[a], cap * es, cudaMemcpyDeviceToHost), "read x");
            }
            for (int a = 0; a < 3; a++) {
                hu[a].resize(cap * es);
                CK(cudaMemcpy(hu[a].data(), S.u[a], cap * es, cudaMemcpyDeviceToHost), "read u");
            }
            CK(cudaMemcpy(hw.data(), S.w, cap * es, cudaMemcpyDeviceToHost), "read w");
            CK(cudaMemcpy(hid.data(), S.id, cap * sizeof(int), cudaMemcpyDeviceToHost), "read id");
            if (S.prec != PIC_FP64) {
                hcell.resize(cap);
                CK(cudaMemcpy(hcell.data(), S.cell, cap * sizeof(int), cudaMemcpyDeviceToHost), "read cell");
            }
            std::vector<int> pbase(S.npatch);
            CK(cudaMemcpy(pbase.data(), S.pbase, S.npatch * sizeof(int), cudaMemcpyDeviceToHost),
               "read pbase");
            std::vector<std::pair<int, long long>> live;
            live.reserve(n);
            for (int p = 0; p < S.npatch; p++)
                for (int c = 0; c < counts[p]; c++) {
                    const long long sl = (long long)pbase[p] + c;
                    live.emplace_back(hid[sl], sl);
                }
            std::sort(live.begin(), live.end());
            double* o = static_cast<double*>(out);
            int* oid = reinterpret_cast<int*>(o + 7 * n);
            for (long long k = 0; k < n; k++) {
                const long long sl = live[k].second;
                double pos[3] = {0, 0, 0}, uu[3], ww;
                for (int a = 0; a < S.dims; a++) {
                    if (S.prec == PIC_FP64) {
                        pos[a] = reinterpret_cast<double*>(hx[a].data())[sl] * S.d[a];
                    } else {
                        const int sh = S.dims == 2 ? 16 * a : 11 * a;
                        const int mask = S.dims == 2 ? 0xFFFF : (a < 2 ? 0x7FF : 0x3FF);
                        const int i = (hcell[sl] >> sh) & mask;
                        pos[a] = ((double)i + load_real(S.prec, hx[a].data(), sl)) * S.d[a];
                    }
                }
                for (int a = 0; a < 3; a++) uu[a] = load_real(S.prec, hu[a].data(), sl);
                ww = load_real(S.prec, hw.data(), sl);
                o[0 * n + k] = pos[0];
                o[1 * n + k] = pos[1];
                o[2 * n + k] = pos[2];
                o[3 * n + k] = uu[0];
                o[4 * n + k] = uu[1];
                o[5 * n + k] = uu[2];
                o[6 * n + k] = ww;
                oid[k] = live[k].first;
            }
            if (written) *written = b;
            return PIC_OK;
        }
        case PIC_DIAG_SLOTS: {
            CK(read_counts(), "read counts");
            long long n = 0;
            for (int c : counts) n += c;
            if (!need((size_t)n * sizeof(int))) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            std::vector<int> hid(S.capacity), pbase(S.npatch);
            CK(cudaMemcpy(hid.data(), S.id, S.capacity * sizeof(int), cudaMemcpyDeviceToHost), "read id");
            CK(cudaMemcpy(pbase.data(), S.pbase, S.npatch * sizeof(int), cudaMemcpyDeviceToHost),
               "read pbase");
            std::vector<std::pair<int, int>> live;  // (id, slot within the patch)
            live.reserve(n);
            for (int p = 0; p < S.npatch; p++)
                for (int c = 0; c < counts[p]; c++) live.emplace_back(hid[(long long)pbase[p] + c], c);
            std::sort(live.begin(), live.end());
            int* o = static_cast<int*>(out);
            for (long long k = 0; k < n; k++) o[k] = live[k].second;
            if (written) *written = (size_t)n * sizeof(int);
            return PIC_OK;
        }
        case PIC_DIAG_QUEUE: {
            int nitems = 0;
            CK(cudaMemcpy(&nitems, s->L.B.nitems, sizeof(int), cudaMemcpyDeviceToHost),
               "read queue length");
            const size_t b = sizeof(int) + (size_t)nitems * sizeof(int4);
            if (!need(b)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
            static_cast<int*>(out)[0] = nitems;
            if (nitems > 0)
                CK(cudaMemcpy(static_cast<int*>(out) + 1, s->L.B.items, nitems * sizeof(int4),
                              cudaMemcpyDeviceToHost),
                   "read queue");
            if (written) *written = b;
            return PIC_OK;
        }
        default:
            return fail(&s->err, PIC_ERR_INVALID, "unknown diagnostic kind");
    }
}

extern "C" pic_status pic_diag(pic_sim* s, int kind, void* out, size_t out_bytes, size_t* written) {
    return guarded(s ? &s->err : nullptr,
                   [&] { return diag_body(s, kind, out, out_bytes, written); });
}

static pic_status profile_body(pic_sim* s, int nsteps, double* ms, int n_ms) {
    if (!s || nsteps < 0 || !ms || n_ms < 8) return PIC_ERR_INVALID;
    const SimDev& S = s->L.S;
    cudaEvent_t ev[8];
    for (int i = 0; i < 8; i++) CK(cudaEventCreate(&ev[i]), "event create");
    for (int i = 0; i < 8; i++) ms[i] = 0.0;
    pic_status rc = PIC_OK;
    for (int it = 0; it < nsteps && rc == PIC_OK; it++) {
        cudaError_t e = cudaEventRecord(ev[0], s->stream);
        if (e == cudaSuccess) e = launch_queue_build(s->L.db, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s->stream);
        if (e == cudaSuccess)
            e = launch_push(s->L.db, S.dims, S.prec, S.mapping, S.P[0], S.P[1], S.P[2], s->push_grid,
                            s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], s->stream);
        if (e == cudaSuccess && S.window) e = launch_inject(s->L.db, 1, s->column_pts, S.prec, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3], s->stream);
        if (e == cudaSuccess) e = launch_exchange(s->L.db, 1, S.npatch, S.prec, s->stream);
        if (e == cudaSuccess && S.merge_above > 0)
            e = launch_merge(s->L.db, 1, S.npatch, S.prec, s->stream);
        if (e == cudaSuccess && S.split_below > 0)
            e = launch_split(s->L.db, 1, S.npatch, S.prec, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[4], s->stream);
        if (e == cudaSuccess) e = launch_repack(s->L.db, 1, S.npatch, S.prec, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[5], s->stream);
        if (e == cudaSuccess)
            e = launch_yee(s->L.db, 1, (int)S.ncell, S.dims, S.prec, S.order, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[6], s->stream);
        if (e == cudaSuccess) e = launch_end_step(s->L.db, 1, S.npatch, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[7], s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[7]);
        if (e != cudaSuccess) {
            rc = cuda_fail(&s->err, e, "profile");
            break;
        }
        for (int k = 0; k < 7; k++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms[k] += t;
        }
        float tt = 0.f;
        cudaEventElapsedTime(&tt, ev[0], ev[7]);
        ms[7] += tt;
    }
    for (int i = 0; i < 8; i++) cudaEventDestroy(ev[i]);
    return rc;
}

extern "C" pic_status pic_profile(pic_sim* s, int nsteps, double* ms, int n_ms) {
    return guarded(s ? &s->err : nullptr, [&] { return profile_body(s, nsteps, ms, n_ms); });
}

extern "C" pic_status pic_destroy(pic_sim* s) {
    if (!s) return PIC_ERR_INVALID;
    cudaStreamSynchronize(s->stream);
    GraphOwner o{&s->cap0, &s->cap1, &s->ev_fork, &s->ev_join, &s->graph, &s->gexec};
    destroy_graph_owner(o);
    for (cudaEvent_t& e : s->rec_ev)
        if (e) cudaEventDestroy(e);
    if (s->rec_host) cudaFreeHost(s->rec_host);
    delete s;
    return PIC_OK;
}

namespace {
constexpr size_t kRecSlot = 64;  // StepState, then the status word
static_assert(sizeof(StepState) + sizeof(int) <= kRecSlot, "record slot too small");
}  // namespace

static pic_status step_record_async_body(pic_sim* s, int slot) {
    if (!s || (slot != 0 && slot != 1)) return PIC_ERR_INVALID;
    if (!s->rec_host) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, 2 * kRecSlot, cudaHostAllocDefault) != cudaSuccess)
            return fail(&s->err, PIC_ERR_NOMEM, "page-locked record slots");
        s->rec_host = static_cast<unsigned char*>(h);
    }
    if (!s->rec_ev[slot] &&
        cudaEventCreateWithFlags(&s->rec_ev[slot], cudaEventDisableTiming) != cudaSuccess) {
        s->rec_ev[slot] = nullptr;
        return fail(&s->err, PIC_ERR_NOMEM, "record event");
    }
    unsigned char* r = s->rec_host + slot * kRecSlot;
    const SimDev& S = s->L.S;
    CK(cudaMemcpyAsync(r, S.st, sizeof(StepState), cudaMemcpyDeviceToHost, s->stream),
       "record copy");
    CK(cudaMemcpyAsync(r + sizeof(StepState), S.status, sizeof(int), cudaMemcpyDeviceToHost,
                       s->stream),
       "record status copy");
    CK(cudaEventRecord(s->rec_ev[slot], s->stream), "record event");
    s->rec_pending[slot] = true;
    return PIC_OK;
}

extern "C" pic_status pic_step_record_async(pic_sim* s, int slot) {
    return guarded(s ? &s->err : nullptr, [&] { return step_record_async_body(s, slot); });
}

static pic_status record_wait_body(pic_sim* s, int slot, void* out, size_t out_bytes,
                                   size_t* written) {
    if (!s || !out || (slot != 0 && slot != 1)) return PIC_ERR_INVALID;
    if (written) *written = 0;
    if (!s->rec_pending[slot]) return fail(&s->err, PIC_ERR_INVALID, "no record pending");
    CK(cudaEventSynchronize(s->rec_ev[slot]), "record wait");
    s->rec_pending[slot] = false;
    const unsigned char* r = s->rec_host + slot * kRecSlot;
    StepState st;
    int status = 0;
    memcpy(&st, r, sizeof(st));
    memcpy(&status, r + sizeof(StepState), sizeof(int));
    pic_status rc = status_to_error(&s->err, status);
    if (rc != PIC_OK) return rc;
    if (out_bytes < 3 * sizeof(long long)) return fail(&s->err, PIC_ERR_NOMEM, "output too small");
    long long* o = static_cast<long long*>(out);
    o[0] = st.step;
    o[1] = st.nshift;
    o[2] = st.nrepack;
    size_t wb = 3 * sizeof(long long);
    if (out_bytes >= 4 * sizeof(long long)) {
        o[3] = st.nmerged;
        wb = 4 * sizeof(long long);
    }
    if (out_bytes >= 5 * sizeof(long long)) {
        o[4] = st.nsplit;
        wb = 5 * sizeof(long long);
    }
    if (written) *written = wb;
    return PIC_OK;
}

extern "C" pic_status pic_record_wait(pic_sim* s, int slot, void* out, size_t out_bytes,
                                      size_t* written) {
    return guarded(s ? &s->err : nullptr,
                   [&] { return record_wait_body(s, slot, out, out_bytes, written); });
}

extern "C" const char* pic_last_error(const pic_sim* s) {
    if (!s) return "null sim";
    return s->err.c_str();
}

// ===================================================================== batches

namespace {
struct BatchLayout {
    SimDev* sims;
    int* prefix;
    BatchDev* db;
    int4* items;
    int* nitems;
    int* head;
    int max_items;
    size_t bytes;
};

BatchLayout plan_batch(pic_sim* const* sims, int nsims, char* base) {
    Carver cv{base, base == nullptr};
    BatchLayout b{};
    b.sims = cv.take<SimDev>(nsims);
    b.prefix = cv.take<int>(nsims + 1);
    b.db = cv.take<BatchDev>(1);
    long long items = 64;
    for (int i = 0; i < nsims; i++) {
        const SimDev& S = sims[i]->L.S;
        items += S.npatch + S.capacity / std::max(1, default_chunk(&sims[0]->cfg));
    }
    b.max_items = (int)std::min<long long>(items, 1LL << 30);
    b.items = cv.take<int4>(b.max_items);
    b.nitems = cv.take<int>(1);
    b.head = cv.take<int>(1);
    b.bytes = cv.off + 256;
    return b;
}

const char* batch_check(pic_sim* const* sims, int nsims) {
    if (!sims || nsims < 1) return "empty batch";
    for (int i = 0; i < nsims; i++) {
        if (!sims[i]) return "null sim";
        if (sims[i]->L.S.dims != sims[0]->L.S.dims || sims[i]->L.S.prec != sims[0]->L.S.prec)
            return "sims of a batch must share dims and precision";
        if (sims[i]->L.S.P[0] != sims[0]->L.S.P[0] || sims[i]->L.S.P[1] != sims[0]->L.S.P[1] ||
            sims[i]->L.S.P[2] != sims[0]->L.S.P[2])
            return "sims of a batch must share the patch size";
        if (sims[i]->cfg.mapping != sims[0]->cfg.mapping) return "sims must share the mapping";
        if (sims[i]->L.S.order != sims[0]->L.S.order)
            return "sims of a batch must share the field solver order";
    }
    return nullptr;
}
}  // namespace

static size_t batch_required_bytes_body(pic_sim* const* sims, int nsims) {
    if (batch_check(sims, nsims)) return 0;
    return plan_batch(sims, nsims, nullptr).bytes;
}

extern "C" size_t pic_batch_required_bytes(pic_sim* const* sims, int nsims) {
    return guarded_size([&] { return batch_required_bytes_body(sims, nsims); });
}

static pic_status batch_create_body(pic_sim* const* sims, int nsims, void* dev_arena,
                                    size_t arena_bytes, void* cuda_stream, pic_batch** out) {
    if (!out) return PIC_ERR_INVALID;
    *out = nullptr;
    if (batch_check(sims, nsims)) return PIC_ERR_INVALID;
    if (!dev_arena || (reinterpret_cast<uintptr_t>(dev_arena) & 255)) return PIC_ERR_INVALID;
    BatchLayout bl = plan_batch(sims, nsims, nullptr);
    if (arena_bytes < bl.bytes) return PIC_ERR_NOMEM;
    bl = plan_batch(sims, nsims, static_cast<char*>(dev_arena));
    std::unique_ptr<pic_batch> owner(new (std::nothrow) pic_batch());
    if (!owner) return PIC_ERR_NOMEM;
    pic_batch* b = owner.get();
    b->sims.assign(sims, sims + nsims);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    std::vector<SimDev> hsims(nsims);
    std::vector<int> prefix(nsims + 1, 0);
    int max_patches = 0, max_ncell = 0, max_column = 0;
    bool any_window = false;
    for (int i = 0; i < nsims; i++) {
        hsims[i] = sims[i]->L.S;
        prefix[i + 1] = prefix[i] + hsims[i].npatch;
        max_patches = std::max(max_patches, hsims[i].npatch);
        max_ncell = std::max(max_ncell, (int)hsims[i].ncell);
        max_column = std::max(max_column, sims[i]->column_pts);
        any_window = any_window || hsims[i].window;
    }
    BatchDev& B = b->hb;
    B.nsims = nsims;
    B.chunk = default_chunk(&sims[0]->cfg);
    B.max_items = bl.max_items;
    B.total_patches = prefix[nsims];
    B.max_patches = max_patches;
    B.max_ncell = max_ncell;
    B.sims = bl.sims;
    B.patch_prefix = bl.prefix;
    B.items = bl.items;
    B.nitems = bl.nitems;
    B.head = bl.head;
    b->db = bl.db;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nsims && e == cudaSuccess; i++) e = cudaStreamSynchronize(sims[i]->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bl.sims, hsims.data(), nsims * sizeof(SimDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bl.prefix, prefix.data(), (nsims + 1) * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bl.db, &B, sizeof(B), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    const SimDev& S0 = hsims[0];
    const int grid = push_grid_size(S0.dims, S0.prec, S0.P, sims[0]->cfg.mapping == PIC_MAP_STATIC,
                                    prefix[nsims]);
    GraphOwner o{&b->cap0, &b->cap1, &b->ev_fork, &b->ev_join, &b->graph, &b->gexec};
    bool any_merge = false, any_split = false;
    for (int i = 0; i < nsims; i++) {
        any_merge = any_merge || hsims[i].merge_above > 0;
        any_split = any_split || hsims[i].split_below > 0;
    }
    if (e == cudaSuccess)
        e = capture_step(o, bl.db, nsims, max_patches, max_ncell, max_column, S0.dims, S0.prec,
                         S0.order, sims[0]->cfg.mapping, S0.P, grid, any_window, any_merge,
                         any_split);
    if (e != cudaSuccess) {
        destroy_graph_owner(o);
        return PIC_ERR_CUDA;
    }
    *out = owner.release();
    return PIC_OK;
}

extern "C" pic_status pic_batch_create(pic_sim* const* sims, int nsims, void* dev_arena,
                                       size_t arena_bytes, void* cuda_stream, pic_batch** out) {
    return guarded(nullptr, [&] {
        return batch_create_body(sims, nsims, dev_arena, arena_bytes, cuda_stream, out);
    });
}

extern "C" pic_status pic_batch_step(pic_batch* b, int nsteps) {
    if (!b || nsteps < 0) return PIC_ERR_INVALID;
    for (int i = 0; i < nsteps; i++)
        if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return PIC_ERR_CUDA;
    return PIC_OK;
}

extern "C" pic_status pic_batch_destroy(pic_batch* b) {
    if (!b) return PIC_ERR_INVALID;
    cudaStreamSynchronize(b->stream);
    GraphOwner o{&b->cap0, &b->cap1, &b->ev_fork, &b->ev_join, &b->graph, &b->gexec};
    destroy_graph_owner(o);
    delete b;
    return PIC_OK;
}
