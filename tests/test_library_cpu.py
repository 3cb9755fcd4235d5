"""Host-side checks of the C-ABI library that need no GPU: every symbol the header
declares is exported, and configuration validation / arena sizing behave."""
import re

import pytest

from paper_1511_03878_gb300 import binding, build, inputs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def test_header_symbols_exported(lib):
    hdr = open(build.INCLUDE + "/pic.h").read()
    declared = set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", hdr))
    assert declared == set(binding.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_required_bytes_and_validation(lib):
    p = inputs.thermal2d(nx=64, ny=64, patch=(16, 16))["params"]
    cfg = binding.make_config(p, capacity=100000)
    nb = binding.pic_required_bytes(cfg)
    assert nb > 100000 * (16 + 24 + 8 + 4)
    # FP32 arena is smaller
    cfg32 = binding.make_config(p, precision=binding.PIC_FP32, capacity=100000)
    assert 0 < binding.pic_required_bytes(cfg32) < nb
    # invalid: patch does not divide the grid, dt above a cell, bad dims
    bad = dict(p, patch=(24, 16))
    assert binding.pic_required_bytes(binding.make_config(bad, capacity=10)) == 0
    bad = dict(p, dt=0.2)
    assert binding.pic_required_bytes(binding.make_config(bad, capacity=10)) == 0
    bad = dict(p, dims=4)
    assert binding.pic_required_bytes(binding.make_config(bad, capacity=10)) == 0


def test_create_rejects_bad_arguments(lib):
    import ctypes
    p = inputs.thermal2d(nx=64, ny=64, patch=(16, 16))["params"]
    cfg = binding.make_config(p, capacity=1000)
    h = ctypes.c_void_p()
    # null arena and misaligned arena are rejected before any CUDA call
    assert lib.pic_create(ctypes.byref(cfg), None, 1 << 30, None, ctypes.byref(h)) == binding.PIC_ERR_INVALID
    assert lib.pic_create(ctypes.byref(cfg), ctypes.c_void_p(4096 + 8), 1 << 30, None,
                          ctypes.byref(h)) == binding.PIC_ERR_INVALID
    # too small an arena
    assert lib.pic_create(ctypes.byref(cfg), ctypes.c_void_p(4096), 16, None,
                          ctypes.byref(h)) == binding.PIC_ERR_NOMEM


def test_config_layout_matches_the_library(lib):
    import ctypes
    assert binding.pic_config_bytes() == ctypes.sizeof(binding.PicConfig)


def test_field_solver_order_and_stability_limit(lib):
    import math
    p = inputs.thermal2d(nx=64, ny=64, patch=(16, 16))["params"]
    lim2 = 1 / math.sqrt(sum(1 / x ** 2 for x in p["d"][:2]))
    lim6 = lim2 * 120 / 149
    ok = lambda **kw: binding.pic_required_bytes(binding.make_config(dict(p, **kw), capacity=10)) > 0
    assert ok(maxwell_order=2, dt=0.99 * lim2) and not ok(maxwell_order=2, dt=1.01 * lim2)
    assert ok(maxwell_order=6, dt=0.99 * lim6) and not ok(maxwell_order=6, dt=1.01 * lim6)
    assert not ok(maxwell_order=6, dt=0.9 * lim2)  # stable for Yee, not for order 6
    assert not ok(maxwell_order=4, dt=0.5 * lim6)
    # the moving window with order 6 keeps one extra column of E (3 x ny values)
    w = inputs.lwfa2d(nx=128, ny=64, patch=(16, 16), cfl=0.76)["params"]
    b2 = binding.pic_required_bytes(binding.make_config(w, capacity=1000))
    b6 = binding.pic_required_bytes(binding.make_config(dict(w, maxwell_order=6), capacity=1000))
    assert 3 * 64 * 8 <= b6 - b2 <= 3 * 64 * 8 + 512


def test_null_handles_are_rejected_without_a_gpu(lib):
    """Every entry point checks its handle before any CUDA call: a null sim or batch
    gives PIC_ERR_INVALID (0 bytes for the size queries), never a crash."""
    import ctypes
    nul = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)()
    ip = ctypes.POINTER(ctypes.c_int)()
    inv = binding.PIC_ERR_INVALID
    assert lib.pic_load_particles(nul, 0, dp, dp, dp, dp, dp, dp, dp, ip) == inv
    three = (ctypes.POINTER(ctypes.c_double) * 3)()
    assert lib.pic_load_fields(nul, three, three, dp) == inv
    assert lib.pic_step(nul, 1) == inv
    assert lib.pic_sync(nul) == inv
    written = ctypes.c_size_t(7)
    buf = ctypes.create_string_buffer(64)
    assert lib.pic_diag(nul, 0, buf, 64, ctypes.byref(written)) == inv
    ms = (ctypes.c_double * 8)()
    assert lib.pic_profile(nul, 1, ms, 8) == inv
    assert lib.pic_destroy(nul) == inv
    assert lib.pic_last_error(nul) == b"null sim"
    assert lib.pic_batch_required_bytes(None, 0) == 0
    out = ctypes.c_void_p()
    assert lib.pic_batch_create(None, 0, ctypes.c_void_p(4096), 1 << 20, None,
                                ctypes.byref(out)) == inv
    assert lib.pic_batch_step(nul, 1) == inv
    assert lib.pic_batch_destroy(nul) == inv


def test_workload_sizes_checked_before_the_library_reads_them():
    """Sim.load checks array sizes first (the library reads n particles and ncell field
    values from the host pointers): every generator's workload passes, a short field or
    particle array is refused."""
    import numpy as np

    cases = [inputs.thermal2d(nx=32, ny=16, patch=(16, 16)),
             inputs.lwfa2d(nx=128, ny=64, patch=(32, 32)),
             inputs.stress3d(n=(16, 8, 8), patch=(8, 8, 8), total=2000),
             inputs.lwfa3d(nx=32, ny=8, nz=8, patch=(16, 8, 8))]
    for w in cases:
        n = w["params"]["n"]
        ncell = n[0] * n[1] * (n[2] if w["params"]["dims"] == 3 else 1)
        binding.check_workload(w, ncell)
        binding.check_workload(w, ncell, np.zeros(ncell))
        with pytest.raises(ValueError):
            binding.check_workload(dict(w, E=[w["E"][0][:-1], w["E"][1], w["E"][2]]), ncell)
        with pytest.raises(ValueError):
            binding.check_workload(w, ncell, np.zeros(ncell - 1))
        short = dict(w["particles"], ux=w["particles"]["ux"][:-1])
        with pytest.raises(ValueError):
            binding.check_workload(dict(w, particles=short), ncell)


def test_module_level_loads_check_sizes_before_the_library_reads_them():
    """The same-name wrappers pic_load_particles / pic_load_fields refuse short arrays
    themselves (n from x; the grid's cell count remembered from pic_create, else the
    first array's), so no path into the C ABI hands the library a short host array."""
    import ctypes

    import numpy as np

    w = inputs.thermal2d(nx=32, ny=16, patch=(16, 16))
    h = ctypes.c_void_p(0)  # never reached: the checks raise first
    short = dict(w["particles"], w=w["particles"]["w"][:-1])
    with pytest.raises(ValueError):
        binding.pic_load_particles(h, short)
    noid = {k: v for k, v in w["particles"].items() if k != "id"}
    with pytest.raises(ValueError):
        binding.pic_load_particles(h, noid)
    E, B = w["E"], w["B"]
    with pytest.raises(ValueError):
        binding.pic_load_fields(h, [E[0], E[1], E[2][:, :-1]], B)
    with pytest.raises(ValueError):
        binding.pic_load_fields(h, E, B[:2])
    with pytest.raises(ValueError):
        binding.pic_load_fields(h, E, B, np.zeros(E[0].size - 1))
    # a handle made by pic_create is checked against its own grid
    binding._ncell[12345] = E[0].size + 1
    try:
        with pytest.raises(ValueError):
            binding.pic_load_fields(ctypes.c_void_p(12345), E, B)
    finally:
        binding._ncell.pop(12345, None)


def test_split_configuration_is_validated():
    """split_below in [0, 64] and a finite split_wmin >= 0 (pure host-side validation:
    pic_required_bytes returns 0 for an invalid config)."""
    w = inputs.thermal2d(nx=64, ny=64, patch=(16, 16))
    ok = binding.make_config(w["params"], capacity=1000, split_below=4, split_wmin=0.1)
    assert binding.pic_required_bytes(ok) > 0
    for kw in (dict(split_below=65, split_wmin=0.1), dict(split_below=-1),
               dict(split_below=4, split_wmin=-1.0), dict(split_below=4, split_wmin=float("nan"))):
        bad = binding.make_config(w["params"], capacity=1000, **kw)
        assert binding.pic_required_bytes(bad) == 0, kw


def test_double_word_precision_is_2d_only():
    """A 3D config with the double-word precision is invalid (in 3D it measured no faster
    than FP64, so only FP64 and FP32 kernels are built for 3D); 2D accepts it."""
    w3 = inputs.stress3d(n=(16, 8, 8), patch=(8, 8, 8), total=2000)
    w2 = inputs.thermal2d(nx=32, ny=16, patch=(16, 16))
    assert binding.pic_required_bytes(binding.make_config(w3["params"], binding.PIC_DF64, 4000)) == 0
    assert binding.pic_required_bytes(binding.make_config(w3["params"], binding.PIC_FP64, 4000)) > 0
    assert binding.pic_required_bytes(binding.make_config(w2["params"], binding.PIC_DF64, 4000)) > 0
