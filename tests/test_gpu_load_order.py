"""The device loader's layout (pic_load_particles): every particle lands in its patch's
slot range, and within a patch the slots follow the bank-class run order, run r holding
the r-th particle of every class present, classes ascending. The class of a particle is
the shared-memory bank (modulo 32) of its cell in the patch's staged field tile. Checked
against a host restatement from the loaded positions, in 2D and 3D, FP64 and FP32,
with a chunked load."""
import numpy as np
import pytest

from paper_1511_03878_gb300 import inputs


@pytest.fixture(scope="module")
def binding():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding as b, build

    build.build()
    return b


def host_layout(params, pos):
    """Patch index and bank class of each particle from its physical position."""
    dims = params["dims"]
    n = params["n"][:dims]
    d = params["d"][:dims]
    P = params["patch"][:dims]
    npch = [a // b for a, b in zip(n, P)]
    ic = []
    for a in range(dims):
        c = pos[a] / d[a]
        c = np.where(c >= n[a], np.nextafter(float(n[a]), 0.0), c)
        ic.append(np.floor(c).astype(np.int64))
    pc = [ic[a] // P[a] for a in range(dims)]
    loc = [ic[a] - pc[a] * P[a] for a in range(dims)]
    BX, BY = P[0] + 4, P[1] + 3
    lz = loc[2] if dims == 3 else 0
    cls = ((lz * BY + loc[1]) * BX + loc[0]) & 31
    patch = pc[0] + npch[0] * pc[1]
    if dims == 3:
        patch = patch + npch[0] * npch[1] * pc[2]
    return patch, cls


def run_order(classes_in_patch):
    """The class sequence the run order gives for these class counts."""
    nb = np.bincount(classes_in_patch, minlength=32)
    seq = []
    for r in range(int(nb.max()) if len(nb) else 0):
        seq.extend(q for q in range(32) if nb[q] > r)
    return np.array(seq, dtype=np.int64)


def check(binding, w, prec, capacity):
    sim = binding.Sim(w["params"], precision=prec, capacity=capacity)
    sim.load(w)
    q = sim.particles()
    slot = sim.slots()
    counts = sim.patch_counts()
    sim.close()
    dims = w["params"]["dims"]
    pos = [q["x"], q["y"], q["z"]][:dims]
    patch, cls = host_layout(w["params"], pos)
    assert np.array_equal(np.bincount(patch, minlength=len(counts)), counts)
    checked = 0
    for p in np.flatnonzero(counts):
        m = patch == p
        s = slot[m]
        assert np.array_equal(np.sort(s), np.arange(counts[p]))  # a permutation of the range
        seq = cls[m][np.argsort(s)]
        assert np.array_equal(seq, run_order(cls[m])), p
        checked += 1
    assert checked == int((counts > 0).sum())


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_load_order_2d(binding, prec):
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=3, patch=(16, 16))
    n = len(w["particles"]["x"])
    check(binding, w, prec, 2 * n)


@pytest.mark.gpu
def test_load_order_chunked_fp32(binding):
    """Capacity equal to the count: the FP32 load stages the FP64 arrays in two chunks."""
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=4, patch=(16, 16))
    n = len(w["particles"]["x"])
    check(binding, w, 1, n)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_load_order_3d(binding, prec):
    w = inputs.stress3d(n=(32, 32, 32), patch=(8, 8, 8), total=200000, seed=5)
    n = len(w["particles"]["x"])
    check(binding, w, prec, 2 * n)
