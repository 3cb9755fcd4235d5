"""The 2^62 fixed-point helpers of the FP64 particle kernels (fix62.cuh, pic_device.cuh),
run on the GPU and checked against exact rational arithmetic at the bounds their
comments state:
  fixmul62(a, w)         round(a w / 2^62) within 2^-30 of a unit from a tie
  shape62(D)             quadratic B-spline weights, within two units of 2^-62
  split62(x)             floor and 2^62 fraction of a double, exact
  gather9_fix/27_fix     order-2 gathers from split fixed-point fields, 8 / 12 units below
  fix_to_f64_int(v, k)   v 2^-k to a double, truncated to 53 bits
  mul_to_fixed(c, w)     round(c w) for doubles, nearest
  jatomic(long long*)    64-bit adds as 32-bit atomic pairs: the exact sum
The kernels' own parity against the oracle is in the other GPU tests."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1511_03878_gb300", "csrc")
L = 1 << 62

PROGRAM = r"""
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>
#include "fix62.cuh"
using namespace pic;
// one record per input line; every kernel reads its inputs and writes int64 results
__global__ void k_mul(const long long* in, long long* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fixmul62(in[2 * i], in[2 * i + 1]);
}
__global__ void k_shape(const long long* in, long long* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) shape62(in[i], out + 3 * i);
}
__global__ void k_split(const double* in, long long* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int c;
        long long f;
        split62(in[i], c, f);
        out[2 * i] = c;
        out[2 * i + 1] = f;
    }
}
__global__ void k_tof64(const long long* in, double* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fix_to_f64_int(in[2 * i], (int)in[2 * i + 1]);
}
__global__ void k_mulfix(const double* in, long long* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = mul_to_fixed(in[2 * i], in[2 * i + 1]);
}
// gathers: 27 field values (split), 9 weights (3 per axis) per record
__global__ void k_gather(const long long* f, const long long* w, long long* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2 t[27];
    for (int k = 0; k < 27; k++) {
        const long long u = f[27 * i + k];
        t[k] = make_int2((int)(u & 0x7FFFFFFFLL), (int)(u >> 31));
    }
    W31 sx[3], sy[3], sz[3];
    for (int k = 0; k < 3; k++) {
        sx[k] = w31(w[9 * i + k]);
        sy[k] = w31(w[9 * i + 3 + k]);
        sz[k] = w31(w[9 * i + 6 + k]);
    }
    out[2 * i] = gather9_fix(t, 3, sx, sy);
    out[2 * i + 1] = gather27_fix(t, 3, 9, sx, sy, sz);
}
// all threads add their values into 8 shared 64-bit entries; entry sums written out
__global__ void k_atomic(const long long* v, long long* out, int n) {
    __shared__ long long acc[8];
    if (threadIdx.x < 8) acc[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) jatomic(&acc[i & 7], v[i]);
    __syncthreads();
    if (threadIdx.x < 8) out[threadIdx.x] = acc[threadIdx.x];
}
template <typename A, typename B>
static int run(void (*k)(const A*, B*, int), const A* h, size_t na, B* o, size_t no, int n) {
    A* d;
    B* e;
    if (cudaMalloc(&d, na * sizeof(A)) || cudaMalloc(&e, no * sizeof(B))) return 1;
    cudaMemcpy(d, h, na * sizeof(A), cudaMemcpyHostToDevice);
    k<<<(n + 255) / 256, 256>>>(d, e, n);
    if (cudaDeviceSynchronize() != cudaSuccess) return 2;
    cudaMemcpy(o, e, no * sizeof(B), cudaMemcpyDeviceToHost);
    cudaFree(d);
    cudaFree(e);
    return 0;
}
int main() {
    char what[16];
    int n;
    if (scanf("%15s %d", what, &n) != 2 || n <= 0 || n > (1 << 16)) return 3;
    const int per = !strcmp(what, "mul") || !strcmp(what, "tof64") || !strcmp(what, "mulfix") ? 2
                    : !strcmp(what, "gather") ? 36 : 1;
    long long* in = new long long[(size_t)n * per];
    for (long long i = 0; i < (long long)n * per; i++) {
        unsigned long long b;
        if (scanf("%llx", &b) != 1) return 3;
        memcpy(&in[i], &b, 8);
    }
    long long* out = new long long[(size_t)n * 3 + 8];
    int rc = 0;
    size_t nout = n;
    if (!strcmp(what, "mul")) rc = run(k_mul, in, 2 * n, out, nout = n, n);
    else if (!strcmp(what, "shape")) rc = run(k_shape, in, n, out, nout = 3 * n, n);
    else if (!strcmp(what, "split")) rc = run(k_split, (const double*)in, n, out, nout = 2 * n, n);
    else if (!strcmp(what, "tof64")) rc = run(k_tof64, in, 2 * n, (double*)out, nout = n, n);
    else if (!strcmp(what, "mulfix")) rc = run(k_mulfix, (const double*)in, 2 * n, out, nout = n, n);
    else if (!strcmp(what, "gather")) {
        long long *df, *dw, *dout;
        if (cudaMalloc(&df, 27 * n * 8) || cudaMalloc(&dw, 9 * n * 8) || cudaMalloc(&dout, 2 * n * 8)) return 1;
        long long* f = new long long[27 * n];
        long long* w = new long long[9 * n];
        for (int i = 0; i < n; i++) {
            memcpy(f + 27 * i, in + 36 * i, 27 * 8);
            memcpy(w + 9 * i, in + 36 * i + 27, 9 * 8);
        }
        cudaMemcpy(df, f, 27 * n * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(dw, w, 9 * n * 8, cudaMemcpyHostToDevice);
        k_gather<<<(n + 255) / 256, 256>>>(df, dw, dout, n);
        if (cudaDeviceSynchronize() != cudaSuccess) return 2;
        cudaMemcpy(out, dout, 2 * n * 8, cudaMemcpyDeviceToHost);
        nout = 2 * n;
    } else if (!strcmp(what, "atomic")) {  // one CTA: all adds into the same 8 entries
        long long *dv, *dout;
        if (cudaMalloc(&dv, (size_t)n * 8) || cudaMalloc(&dout, 8 * 8)) return 1;
        cudaMemcpy(dv, in, (size_t)n * 8, cudaMemcpyHostToDevice);
        k_atomic<<<1, 256>>>(dv, dout, n);
        if (cudaDeviceSynchronize() != cudaSuccess) return 2;
        cudaMemcpy(out, dout, 8 * 8, cudaMemcpyDeviceToHost);
        nout = 8;
    } else return 4;
    if (rc) return rc;
    for (size_t i = 0; i < nout; i++) printf("%llx\n", (unsigned long long)out[i]);
    return 0;
}
"""


def _u64(v):
    return v & 0xFFFFFFFFFFFFFFFF


def _s64(u):
    return u - (1 << 64) if u >> 63 else u


def _dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dval(u):
    return struct.unpack("<d", struct.pack("<Q", u))[0]


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    d = tmp_path_factory.mktemp("fixed")
    src = d / "fixed.cu"
    src.write_text(PROGRAM)
    out = d / "fixed"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-I", CSRC, "-o", str(out), str(src)])
    return str(out)


def _run(exe, what, words):
    n = len(words) // {"mul": 2, "tof64": 2, "mulfix": 2, "gather": 36}.get(what, 1)
    text = "%s %d\n" % (what, n) + "\n".join("%x" % _u64(w) for w in words)
    res = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    return [_s64(int(h, 16)) for h in res.split()]


@pytest.mark.gpu
def test_fixmul62_rounds_to_nearest(exe):
    rng = np.random.default_rng(7)
    a = [int(v) for v in rng.integers(-(1 << 61), 1 << 61, 4000)]
    w = [int(v) for v in rng.integers(-L + 1, L, 4000)]
    a += [0, 5, -(1 << 61) + 1, 1 << 40, -1]  # zero, tiny and extreme operands
    w += [123456789, 0, L - 1, -(L - 1), L // 3]
    a = [x >> int(s) for x, s in zip(a, rng.integers(0, 50, len(a)))]
    got = _run(exe, "mul", [v for pair in zip(a, w) for v in pair])
    for x, y, g in zip(a, w, got):
        err = abs(Fraction(g) - Fraction(x * y, L))
        assert err <= Fraction(1, 2) + Fraction(1, 1 << 29), (x, y, g)
        if x == 0 or y == 0:
            assert g == 0


@pytest.mark.gpu
def test_shape62_weights(exe):
    rng = np.random.default_rng(8)
    D = [int(v) for v in rng.integers(-(1 << 61), (1 << 61) + 1, 3000)] + [0, 1 << 61, -(1 << 61)]
    got = _run(exe, "shape", D)
    for k, d in enumerate(D):
        s = got[3 * k:3 * k + 3]
        delta = Fraction(d, L)
        exact = [(Fraction(1, 2) - delta) ** 2 / 2, Fraction(3, 4) - delta ** 2,
                 (Fraction(1, 2) + delta) ** 2 / 2]
        for g, e in zip(s, exact):
            assert abs(Fraction(g, L) - e) <= Fraction(2, L), (d, s)
        assert sum(s) <= L  # the weights never sum above one


@pytest.mark.gpu
def test_split62_exact(exe):
    rng = np.random.default_rng(9)
    xs = list(rng.uniform(0, 4096, 2000)) + list(rng.uniform(-3, 3, 500)) + \
        [0.0, 1.0, -1.0, 2.0 ** -70, 1023.9999999999999, -2.0 ** -40, 3.5]
    got = _run(exe, "split", [_dbits(float(x)) for x in xs])
    for k, x in enumerate(xs):
        c, f = got[2 * k], got[2 * k + 1]
        fx = Fraction(float(x))
        fl = fx.numerator // fx.denominator
        assert c == fl, x
        frac = (fx - fl) * L
        # exact when the fraction has at most 62 bits below the point, else truncated
        assert 0 <= frac - f < 1, x


@pytest.mark.gpu
def test_gathers_within_bound(exe):
    rng = np.random.default_rng(10)
    words = []
    cases = []
    for _ in range(1500):
        F = [int(v) for v in rng.integers(-(1 << 59), 1 << 59, 27)]
        W = []
        for _a in range(3):
            d = Fraction(int(rng.integers(-(1 << 61), 1 << 61)), L)
            W += [int(((Fraction(1, 2) - d) ** 2 / 2) * L), int((Fraction(3, 4) - d * d) * L),
                  int(((Fraction(1, 2) + d) ** 2 / 2) * L)]
        words += F + W
        cases.append((F, W))
    got = _run(exe, "gather", words)
    for k, (F, W) in enumerate(cases):
        g9, g27 = got[2 * k], got[2 * k + 1]
        e9 = sum(Fraction(W[3 + b] * W[a] * F[3 * b + a], L * L) for b in range(3) for a in range(3))
        e27 = sum(Fraction(W[6 + c] * W[3 + b] * W[a] * F[9 * c + 3 * b + a], L * L * L)
                  for c in range(3) for b in range(3) for a in range(3))
        assert -8 <= g9 - e9 <= 1, (g9, float(e9))
        assert -12 <= g27 - e27 <= 1, (g27, float(e27))


@pytest.mark.gpu
def test_conversions(exe):
    rng = np.random.default_rng(11)
    v = [int(x) for x in rng.integers(-(1 << 60), 1 << 60, 2000)] + [0, 1, -1]
    k = [int(x) for x in rng.integers(-100, 1000, len(v))]
    got = _run(exe, "tof64", [t for pair in zip(v, k) for t in pair])
    for x, s, g in zip(v, k, got):
        d = _dval(_u64(g))
        exact = Fraction(x) / Fraction(2) ** s if s >= 0 else Fraction(x) * 2 ** (-s)
        if x == 0 or abs(exact) < Fraction(1, 2) ** 1022:  # zero, or below the normal range
            assert d == 0.0
            continue
        assert abs(Fraction(d) - exact) < abs(exact) * Fraction(1, 1 << 52), (x, s)
    c = list(rng.uniform(-1, 1, 2000) * 2.0 ** rng.integers(0, 40, 2000))
    w = list(rng.uniform(0, 1, 2000) * 2.0 ** rng.integers(-30, 10, 2000))
    pairs = [(a, b) for a, b in zip(c, w) if 1 <= abs(a * b) < 2.0 ** 60]
    got = _run(exe, "mulfix", [_dbits(float(t)) for p in pairs for t in p])
    for (a, b), g in zip(pairs, got):
        assert abs(Fraction(g) - Fraction(float(a)) * Fraction(float(b))) <= Fraction(1, 2) + \
            Fraction(1, 1 << 8), (a, b, g)


@pytest.mark.gpu
def test_tile_adds_exact(exe):
    rng = np.random.default_rng(12)
    v = [int(x) for x in rng.integers(-(1 << 50), 1 << 50, 8192)]
    got = _run(exe, "atomic", v)
    for e in range(8):
        assert got[e] == sum(v[e::8])
