"""Host logic of the autotuner that needs no GPU: the candidate filter follows the
library's own validation (divisibility, shared-memory fit of the patch tiles)."""
import pytest

from paper_1511_03878_gb300 import autotune, binding, build, inputs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def lwfa_params():
    return inputs.lwfa2d(nx=2048, ny=512, ppc=(1, 1), ramp_x0=1e9)["params"]


def test_lwfa_candidates_fit_and_divide(lib):
    p = lwfa_params()
    for prec in (binding.PIC_FP64, binding.PIC_FP32, binding.PIC_DF64):
        c = autotune.patch_candidates(p, prec)
        assert (32, 32) in c and (16, 16) in c
        for q in c:
            assert 2048 % q[0] == 0 and 512 % q[1] == 0
            assert max(q) <= 2 * min(q)
    # a 64x64 FP64 tile (6 field + 3 current planes of 68x67 / 69x69 doubles) is 333 KB,
    # beyond the 227 KB of shared memory of one CTA; in FP32 it is 166 KB
    assert (64, 64) not in autotune.patch_candidates(p, binding.PIC_FP64)
    assert (64, 64) in autotune.patch_candidates(p, binding.PIC_FP32)
    cfg = binding.make_config(dict(p, patch=(64, 64)), binding.PIC_FP64, capacity=10)
    assert binding.pic_required_bytes(cfg) == 0


def test_stress3d_candidates(lib):
    p = inputs.stress3d(n=(32, 32, 32), d=0.1, patch=(16, 16, 16), total=1000, sigma=1.5,
                        seed=3)["params"]
    p = dict(p, n=(256, 128, 128))
    c32 = autotune.patch_candidates(p, binding.PIC_FP32)
    c64 = autotune.patch_candidates(p, binding.PIC_FP64)
    assert (8, 8, 8) in c32 and (8, 8, 8) in c64
    assert (16, 16, 16) not in c32  # 16^3 tiles need 284 KB in FP32
    assert set(c64) <= set(c32)
    for q in c32:
        assert all(n % s == 0 for n, s in zip((256, 128, 128), q))


def test_thermal_candidates_include_small_patches(lib):
    p = inputs.thermal2d(seed=1511)["params"]  # 128x128 cells
    c = autotune.patch_candidates(p, binding.PIC_FP64)
    assert (8, 8) in c and (16, 16) in c and (32, 32) in c
    assert all(128 % q[0] == 0 and 128 % q[1] == 0 for q in c)
