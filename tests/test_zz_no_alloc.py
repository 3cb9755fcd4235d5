"""The allocation-free Gauss-residual entry point (pic_gauss_residual_2d_static).

It serves callers that cannot allocate device memory (code inside another
framework's memory pool or under a fixed device budget, where cudaMalloc would fail
or synchronise the device). It keeps its charge-density scratch in a static device
array instead. This file is collected last, so that a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_gauss_residual_matches_diag():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding, build, inputs

    build.build()
    nx = ny = 64
    w = inputs.thermal2d(nx=nx, ny=ny, d=0.1, uth=0.1, seed=21, patch=(16, 16))
    p = w["params"]
    n = len(w["particles"]["x"])
    sim = binding.Sim(p, precision=binding.PIC_FP64, capacity=2 * n)
    binding.pic_load_particles(sim.h, w["particles"])
    # no background: the residual is div E - rho_e, an O(1) field worth comparing
    binding.pic_load_fields(sim.h, w["E"], w["B"], np.zeros((ny, nx)))
    sim.step(7)
    ref = sim.gauss()           # the existing entry point (pic_diag, PIC_DIAG_GAUSS)
    assert np.abs(ref).max() > 0.1
    q = sim.particles()
    f = sim.fields()
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, y, wt = dev(q["x"]), dev(q["y"]), dev(q["w"])
    ex, ey = dev(f["Ex"]), dev(f["Ey"])
    out = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row: the shared scratch is cleared each time
        out.fill_(float("nan"))
        rc = binding.pic_gauss_residual_2d_static(
            n, x.data_ptr(), y.data_ptr(), wt.data_ptr(), p["q"], ex.data_ptr(), ey.data_ptr(),
            0, out.data_ptr(), nx, ny, p["d"][0], p["d"][1], 0, stream.cuda_stream)
        assert rc == binding.PIC_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-12, (call, err)
    # sizes beyond the static scratch are rejected before any launch
    rc = binding.pic_gauss_residual_2d_static(
        n, x.data_ptr(), y.data_ptr(), wt.data_ptr(), p["q"], ex.data_ptr(), ey.data_ptr(), 0,
        out.data_ptr(), 2048, 1024, p["d"][0], p["d"][1], 0, stream.cuda_stream)
    assert rc == binding.PIC_ERR_NOMEM
    sim.close()
