"""Failure paths on the GPU without a fault: a bounded device wait that runs out.

The kernels' waits on asynchronous transfers (the mbarrier of each TMA tile load) give
up after about 2^31 SM clocks and latch a status bit. The self-test entry point waits,
through the same bounded wait, on an mbarrier phase that nothing completes; the host
must read PIC_ERR_TIMEOUT after about a second, and the CUDA context must stay usable.
"""
import time

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


def test_bounded_wait_expires_and_context_survives(binding):
    import torch

    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    rc = binding.pic_selftest_bounded_wait(stream.cuda_stream)
    elapsed = time.perf_counter() - t0
    assert rc == binding.PIC_ERR_TIMEOUT, rc
    assert 0.2 < elapsed < 20.0, elapsed
    # the context still runs the library's kernels
    w = inputs.thermal2d(nx=64, ny=64, patch=(16, 16))
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n)
    sim.load(w)
    sim.step(3)
    sim.sync()
    assert sim.num_particles() == n
    assert np.isfinite(sim.energy()).all()
    sim.close()
