// Patch decomposition across ranks (Sec. 3.1, "Dynamic load balancing", Figs. 3-4): the
// patches are ordered along a Hilbert curve, each rank owns one contiguous segment of
// that order, and the segments are chosen from the patch loads (SP counts, Sec. 3) so
// that the most loaded rank carries as little as possible; when loads change, patches
// whose segment changed move between ranks. Host code only: it runs on the CPU of every
// rank, and the data movement it plans is done by the caller (see decomp.py).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "pic.h"

namespace {

// Hilbert index of the point X (n axes, b bits each) by Skilling's transposition
// ("Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): undo the excess work of
// the curve's reflections and exchanges level by level, Gray-encode, then interleave the
// bits of the transposed form, most significant level first.
uint64_t hilbert_index(unsigned X[3], int n, int b) {
    if (b == 0) return 0;
    const unsigned M = 1u << (b - 1);
    for (unsigned Q = M; Q > 1; Q >>= 1) {
        const unsigned P = Q - 1;
        for (int i = 0; i < n; i++) {
            if (X[i] & Q) {
                X[0] ^= P;  // invert the low bits of axis 0
            } else {
                const unsigned t = (X[0] ^ X[i]) & P;  // exchange low bits of axes 0 and i
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < n; i++) X[i] ^= X[i - 1];
    unsigned t = 0;
    for (unsigned Q = M; Q > 1; Q >>= 1)
        if (X[n - 1] & Q) t ^= Q - 1;
    for (int i = 0; i < n; i++) X[i] ^= t;
    uint64_t h = 0;
    for (int bit = b - 1; bit >= 0; bit--)
        for (int i = 0; i < n; i++) h = (h << 1) | ((X[i] >> bit) & 1u);
    return h;
}

// greedy: the fewest contiguous segments with load <= cap (count of segments needed)
long long segments_needed(const double* load, int n, double cap) {
    long long seg = 1;
    double acc = 0.0;
    for (int k = 0; k < n; k++) {
        if (acc + load[k] > cap && acc > 0.0) {
            seg++;
            acc = 0.0;
        }
        acc += load[k];
    }
    return seg;
}

}  // namespace

extern "C" pic_status pic_hilbert_order(int dims, const int np[3], int* order) {
    if ((dims != 2 && dims != 3) || !np || !order) return PIC_ERR_INVALID;
    long long total = 1;
    int m = 1;
    for (int a = 0; a < dims; a++) {
        if (np[a] < 1 || np[a] > (1 << 20)) return PIC_ERR_INVALID;
        total *= np[a];
        m = std::max(m, np[a]);
    }
    if (total > (1LL << 30)) return PIC_ERR_INVALID;
    int b = 0;
    while ((1 << b) < m) b++;
    std::vector<std::pair<uint64_t, int>> key((size_t)total);
    for (long long p = 0; p < total; p++) {
        unsigned X[3] = {0, 0, 0};
        X[0] = (unsigned)(p % np[0]);
        X[1] = (unsigned)((p / np[0]) % np[1]);
        if (dims == 3) X[2] = (unsigned)(p / ((long long)np[0] * np[1]));
        key[(size_t)p] = {hilbert_index(X, dims, b), (int)p};
    }
    std::sort(key.begin(), key.end());
    for (long long k = 0; k < total; k++) order[k] = key[(size_t)k].second;
    return PIC_OK;
}

extern "C" pic_status pic_partition(int n, const double* load, int nranks, int* first,
                                    double* max_load) {
    if (n < 1 || !load || nranks < 1 || nranks > n || !first) return PIC_ERR_INVALID;
    double sum = 0.0, big = 0.0;
    for (int k = 0; k < n; k++) {
        if (!(load[k] >= 0.0) || !std::isfinite(load[k])) return PIC_ERR_INVALID;
        sum += load[k];
        big = std::max(big, load[k]);
    }
    // smallest cap for which the greedy needs at most nranks segments (bisection on the
    // cap; the greedy count is monotone in it)
    double lo = std::max(big, sum / nranks), hi = std::max(sum, lo);
    if (segments_needed(load, n, lo) <= nranks) hi = lo;
    for (int it = 0; it < 200 && hi - lo > 1e-12 * std::max(1.0, hi); it++) {
        const double mid = 0.5 * (lo + hi);
        if (segments_needed(load, n, mid) <= nranks)
            hi = mid;
        else
            lo = mid;
    }
    // cut greedily at that cap, and also whenever the patches left equal the ranks left,
    // so that every rank owns at least one patch
    int r = 0;
    double acc = 0.0, worst = 0.0;
    first[0] = 0;
    for (int k = 0; k < n; k++) {
        const int ranks_left = nranks - r - 1;
        const bool over = acc > 0.0 && acc + load[k] > hi;
        const bool forced = ranks_left > 0 && n - k == ranks_left;
        if ((over || forced) && r + 1 < nranks && k > first[r]) {
            worst = std::max(worst, acc);
            first[++r] = k;
            acc = 0.0;
        }
        acc += load[k];
    }
    worst = std::max(worst, acc);
    while (r + 1 < nranks) first[++r] = n;  // unreachable with nranks <= n
    first[nranks] = n;
    if (max_load) *max_load = worst;
    return PIC_OK;
}
