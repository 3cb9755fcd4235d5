// Allocation-free Gauss's-law residual (div E - rho_e - rho_bg) for callers that
// cannot allocate device memory. The charge-density accumulator is a file-scope
// static device array; see pic_gauss_residual_2d_static in pic.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "pic.h"
#include "pic_device.cuh"

namespace {

constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device; held by each GPU that loads the library
// until the process exits. Host code must not pass `g_rho_scratch` itself to a
// kernel: on the host that name is a stand-in, not a device address.
__device__ __align__(256) double g_rho_scratch[PIC_STATIC_MAX_CELLS];

// Device address of the scratch per device, with the id of the CUDA context it was
// looked up in: a device reset (or any new primary context) gets a new context id,
// and the address is then looked up again instead of reusing a stale one.
struct ScratchAddr {
    unsigned long long ctx_id;
    double* ptr;
};
std::mutex g_mutex;
ScratchAddr g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// unique id of the current context (ids are never reused within a process); 0 if
// there is none yet or the driver cannot say
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    }
    if (!get_cur || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device, looked up with that
// device current (once per device and context).
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long id = current_ctx_id();
    ScratchAddr& c = g_scratch[dev];
    if (!c.ptr || id == 0 || c.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rho_scratch);  // creates the context if needed
        if (e != cudaSuccess) return e;
        c.ptr = static_cast<double*>(p);
        c.ctx_id = current_ctx_id();
    }
    *out = c.ptr;
    return cudaSuccess;
}

__global__ void zero_kernel(double* rho, long long ncell) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < ncell) rho[i] = 0.0;
}

// Order-2 B-spline charge of each particle on the nodes. The range test is taken on the
// physical position against L = n d, and the cell coordinate is the IEEE quotient x / d
// kept below n (pic::cell_coord), as the particle loader computes them: a particle just
// under the domain's end whose quotient rounds to n still deposits its charge. Particles
// outside the grid or with non-finite data are skipped (no out-of-range access).
__global__ void deposit_kernel(long long n, const double* __restrict__ x,
                               const double* __restrict__ y, const double* __restrict__ w,
                               double qdv, double* rho, int nx, int ny, double dx, double dy,
                               double Lx, double Ly, int window) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double xv = x[p], yv = y[p];
    if (!(xv >= 0.0 && xv < Lx && yv >= 0.0 && yv < Ly)) return;
    const double xi = pic::cell_coord(xv, dx, nx), eta = pic::cell_coord(yv, dy, ny);
    const double wq = qdv * w[p];
    if (!isfinite(wq)) return;
    const double fx = floor(xi + 0.5), fy = floor(eta + 0.5);
    double Sx[3], Sy[3];
    pic::shape3(xi - fx, Sx);
    pic::shape3(eta - fy, Sy);
    const int ix = (int)fx, iy = (int)fy;
    for (int b = 0; b < 3; b++) {
        int j = iy + b - 1;
        j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
        for (int a = 0; a < 3; a++) {
            int i = ix + a - 1;
            if (window) {
                if (i < 0 || i >= nx) continue;
            } else {
                i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
            }
            atomicAdd(rho + (long long)j * nx + i, wq * Sx[a] * Sy[b]);
        }
    }
}

__global__ void residual_kernel(const double* __restrict__ Ex, const double* __restrict__ Ey,
                                const double* __restrict__ rho, const double* __restrict__ rho_bg,
                                double* out, int nx, int ny, double dx, double dy, int window) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= (long long)nx * ny) return;
    const int i = (int)(c % nx), j = (int)(c / nx);
    const int jm = j == 0 ? ny - 1 : j - 1;
    double exm = 0.0;
    if (i > 0)
        exm = Ex[(long long)j * nx + i - 1];
    else if (!window)
        exm = Ex[(long long)j * nx + nx - 1];
    const double div = (Ex[c] - exm) / dx + (Ey[c] - Ey[(long long)jm * nx + i]) / dy;
    out[c] = div - rho[c] - (rho_bg ? rho_bg[c] : 0.0);
}

}  // namespace

extern "C" pic_status pic_gauss_residual_2d_static(long long n, const double* x, const double* y,
                                                   const double* w, double q, const double* Ex,
                                                   const double* Ey, const double* rho_bg,
                                                   double* out, int nx, int ny, double dx,
                                                   double dy, int window, void* cuda_stream) {
    if (n < 0 || nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0) || !Ex || !Ey || !out)
        return PIC_ERR_INVALID;
    if (n > 0 && (!x || !y || !w)) return PIC_ERR_INVALID;
    const long long ncell = (long long)nx * ny;
    if (ncell > PIC_STATIC_MAX_CELLS) return PIC_ERR_NOMEM;  // beyond the static scratch
    double* rho = nullptr;
    if (scratch_for_current_device(&rho) != cudaSuccess) return PIC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int T = 256;
    zero_kernel<<<(unsigned)((ncell + T - 1) / T), T, 0, s>>>(rho, ncell);
    if (n > 0)
        deposit_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(
            n, x, y, w, q / (dx * dy), rho, nx, ny, dx, dy, (double)nx * dx, (double)ny * dy,
            window);
    residual_kernel<<<(unsigned)((ncell + T - 1) / T), T, 0, s>>>(Ex, Ey, rho, rho_bg, out, nx, ny,
                                                                  dx, dy, window);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}
