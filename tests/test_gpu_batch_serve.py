"""Batching (one persistent particle launch over several simulations) and the
continuous-batching server: results are the same alone and in the mix, admission
respects the HBM budget, and late arrivals join while others run."""
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


def normwise(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _workloads():
    a = inputs.thermal2d(nx=64, ny=64, d=0.1, uth=0.1, seed=31, patch=(16, 16))
    b = inputs.thermal2d(nx=32, ny=64, d=0.1, ppc_side=3, uth=0.2, seed=32, patch=(16, 16))
    c = inputs.lwfa2d(nx=128, ny=64, dx=0.125, dy=0.5, ppc=(2, 2), n0=0.01, ramp_cells=16,
                      a0=3.0, w0=8.0, tau=4.0, laser_back=6.0, ramp_x0=4.0, patch=(16, 16))
    return [a, b, c]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_single(binding, prec):
    import torch

    P = binding.PIC_FP64 if prec == "fp64" else binding.PIC_FP32
    ws = _workloads()
    caps = [4 * len(w["particles"]["x"]) + 10000 for w in ws]
    single = []
    for w, cap in zip(ws, caps):
        s = binding.Sim(w["params"], precision=P, capacity=cap, chunk=300)
        s.load(w)
        s.step(8)
        single.append((s.fields(), s.particles()))
        s.close()
    sims = []
    for w, cap in zip(ws, caps):
        s = binding.Sim(w["params"], precision=P, capacity=cap, chunk=300)
        s.load(w)
        sims.append(s)
    handles = [s.h for s in sims]
    nb = binding.pic_batch_required_bytes(handles)
    arena = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    b = binding.pic_batch_create(handles, (arena.data_ptr() + 255) // 256 * 256, nb,
                                 stream.cuda_stream)
    binding.pic_batch_step(b, 3)
    binding.pic_batch_step(b, 5)
    stream.synchronize()
    binding.pic_batch_destroy(b)
    tol = 1e-11 if prec == "fp64" else 2e-4
    for s, (f1, q1) in zip(sims, single):
        assert s.step_info()[0] == 8
        f2, q2 = s.fields(), s.particles()
        assert np.array_equal(q1["id"], q2["id"])
        for k in ("Ex", "Ey", "Bz", "Jx", "Jz"):
            assert normwise(f2[k], f1[k]) < tol, (k, normwise(f2[k], f1[k]))
        for k in ("ux", "uy"):
            assert normwise(q2[k], q1[k]) < tol
        s.close()


def test_serve_same_alone_and_in_mix(binding):
    from paper_1511_03878_gb300 import serve

    reqs = [serve.Request(rid=i, nx=nx, ny=ny, a0=a0, n0=n0, ppc=ppc, steps=st, arrival=t)
            for i, (nx, ny, a0, n0, ppc, st, t) in enumerate([
                # all arrive together and run far longer than a preparation takes, so
                # they are resident together whatever the GPU's speed
                (256, 128, 3.0, 0.01, 4, 300, 0.0),
                (512, 256, 5.0, 0.005, 2, 400, 0.0),
                (256, 128, 2.0, 0.02, 8, 250, 0.0),
                (512, 256, 4.0, 0.015, 1, 350, 0.0)])]
    srv = serve.Server(budget_bytes=40 << 30, quantum=20)
    res = srv.run(reqs)
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert srv.max_resident >= 2  # their work overlapped on the device
    for r, q in zip(res, reqs):
        e, ax, n = serve.run_alone(q)
        assert r.particles == n
        de = abs(r.energy.sum() - e.sum()) / e.sum()
        err = np.linalg.norm(r.ex_axis - ax) / max(np.linalg.norm(ax), 1e-30)
        print(f"serve alone-vs-mix rid={q.rid} energy_rel={de:.3e} ex_axis_l2={err:.3e}")
        # The same FP32 kernels on the same inputs: alone and in the mix differ only in
        # the order of the FP64 global current atomics, measured on a GB300 at up to
        # 2.9e-8 (energy) and 5.7e-6 (Ex on axis) after 250-400 steps. The gates sit
        # about ten times above that, so a batching error of even 1e-4 fails.
        assert de < 3e-7, (q.rid, r.energy, e)
        assert err < 6e-5, (q.rid, err)


def test_serve_admission_respects_budget(binding):
    from paper_1511_03878_gb300 import serve

    reqs = [serve.Request(rid=i, nx=256, ny=128, a0=3.0, n0=0.01, ppc=4, steps=40 + 10 * i,
                          arrival=0.005 * i) for i in range(6)]
    srv = serve.Server(budget_bytes=1, quantum=10)
    one = srv._bytes(reqs[0])
    srv = serve.Server(budget_bytes=int(2.5 * one), quantum=10)
    res = srv.run(reqs)
    assert len(res) == 6
    assert srv.max_resident <= 2
    # continuous batching: some request starts while another is still running
    events = sorted(srv.timeline)
    starts = {rid: t for t, ev, rid in events if ev == "start"}
    dones = {rid: t for t, ev, rid in events if ev == "done"}
    assert any(starts[a] < dones[b] and starts[a] > starts[b] for a in starts for b in dones
               if a != b)
    summary = serve.summarize(res)
    assert summary["p99_s"] >= summary["p50_s"] > 0
