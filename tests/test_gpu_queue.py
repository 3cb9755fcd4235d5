"""The work queue's contents (PIC_DIAG_QUEUE) against a host restatement of its rule
(Sec. 3: the load of a patch is its SP count; the largest loads go first): full chunks
of `chunk` particles in patch order, then each patch's remainder in one of 64 buckets
of decreasing size, bucket b = 63 - floor(64 rem / (chunk + 1)). The order inside a
bucket is not fixed (atomic claims), so each bucket is compared as a set; everything
else exactly. The static mapping gives one item per non-empty patch in patch order."""
import numpy as np
import pytest

from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding as b, build

    build.build()
    return b


def uneven_workload(seed=5):
    """A thermal plasma with very uneven patch loads: particles thinned per patch by a
    log-normal factor, one patch left very heavy."""
    w = inputs.thermal2d(nx=128, ny=64, d=0.1, ppc_side=4, uth=0.05, seed=seed, patch=(16, 16))
    p = w["particles"]
    rng = np.random.default_rng(seed)
    px = (p["x"] / 0.1 // 16).astype(int)
    py = (p["y"] / 0.1 // 16).astype(int)
    patch = px + 8 * py
    keep_frac = np.clip(rng.lognormal(-1.0, 1.0, 32), 0.01, 1.0)
    keep_frac[13] = 1.0
    keep = rng.uniform(0, 1, len(patch)) < keep_frac[patch]
    w["particles"] = {k: v[keep] for k, v in p.items()}
    return w


def expected_items(counts, chunk):
    full = [(0, p, c * chunk, chunk) for p, n in enumerate(counts) for c in range(n // chunk)]
    buckets = [[] for _ in range(64)]
    for p, n in enumerate(counts):
        rem = n - (n // chunk) * chunk
        if rem > 0:
            b = max(0, 63 - (rem * 64) // (chunk + 1))
            buckets[b].append((0, p, (n // chunk) * chunk, rem))
    return full, buckets


@pytest.mark.parametrize("chunk", [97, 300, 2048])
def test_queue_matches_host_restatement(binding, chunk):
    w = uneven_workload()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n, chunk=chunk)
    sim.load(w)
    counts = sim.patch_counts()
    assert counts.max() > 2.5 * counts.mean() and counts.max() > 10 * counts.min()  # uneven
    sim.step(1)
    items = [tuple(int(v) for v in r) for r in sim.queue()]
    full, buckets = expected_items(counts, chunk)
    assert len(items) == len(full) + sum(len(b) for b in buckets)
    assert items[:len(full)] == full
    pos = len(full)
    for b in buckets:
        assert sorted(items[pos:pos + len(b)]) == sorted(b)
        pos += len(b)
    # every particle of every patch is covered exactly once
    cover = np.zeros(len(counts), dtype=np.int64)
    for _, p, first, cnt in items:
        cover[p] += cnt
    assert np.array_equal(cover, counts)
    sim.close()


def test_static_mapping_queue(binding):
    w = uneven_workload(seed=6)
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n,
                      mapping=binding.PIC_MAP_STATIC)
    sim.load(w)
    counts = sim.patch_counts()
    sim.step(1)
    items = [tuple(int(v) for v in r) for r in sim.queue()]
    assert items == [(0, p, 0, int(c)) for p, c in enumerate(counts) if c > 0]
    sim.close()
