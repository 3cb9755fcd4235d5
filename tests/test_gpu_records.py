"""The asynchronous step record (pic_step_record_async / pic_record_wait): pipelined
reads, one step ahead, give the same records as pic_diag(PIC_DIAG_STEP) after each step,
on a moving window that shifts, and the calls refuse a bad slot or a slot with nothing
pending."""
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


def window():
    args = dict(nx=256, ny=64, dx=0.125, dy=0.5, ppc=(2, 2), n0=0.01, ramp_cells=16,
                a0=2.0, w0=10.0, tau=8.0, laser_back=12.0, patch=(32, 32))
    w = inputs.lwfa2d(**args)
    return inputs.lwfa2d(**args, ramp_x0=w["params"]["xc"] - 8.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pipelined_records_match_synchronous_ones(binding, prec):
    P = {"fp64": binding.PIC_FP64, "fp32": binding.PIC_FP32}[prec]
    w = window()
    n = len(w["particles"]["x"])
    K = 12
    a = binding.Sim(w["params"], precision=P, capacity=4 * n + 100000)
    a.load(w)
    sync = []
    for _ in range(K):
        a.step(1)
        sync.append(a.step_info())
    ea = a.energy()
    a.close()
    b = binding.Sim(w["params"], precision=P, capacity=4 * n + 100000)
    b.load(w)
    piped = []
    for k in range(K):
        b.step(1)
        b.step_record_async(k & 1)
        if k:
            piped.append(b.record_wait((k - 1) & 1))
    piped.append(b.record_wait((K - 1) & 1))
    eb = b.energy()
    b.close()
    assert piped == sync
    assert [s for s, _ in piped] == list(range(1, K + 1))
    assert piped[-1][1] > 0  # the window shifted
    # the reads do not change the run (up to the order of the FP64 current atomics)
    assert np.allclose(ea, eb, rtol=1e-12 if prec == "fp64" else 1e-6, atol=0)


def test_record_calls_refuse_bad_slots(binding):
    w = inputs.thermal2d(nx=32, ny=32, d=0.1, seed=1, patch=(16, 16))
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n)
    sim.load(w)
    with pytest.raises(binding.PicError):
        sim.step_record_async(2)
    with pytest.raises(binding.PicError):
        sim.record_wait(0)  # nothing pending
    sim.step(1)
    sim.step_record_async(0)
    assert sim.record_wait(0) == (1, 0)
    with pytest.raises(binding.PicError):
        sim.record_wait(0)  # already taken
    sim.close()
