"""Host logic of the scan server that needs no GPU: the request stream has the stated
statistics (Poisson arrivals at the mean rate, grids, a0, density, particles per cell
and step ranges). Each request's workload fits its capacity for the whole window, and
the summary's percentiles and aggregate follow their definitions."""
import math

import numpy as np

from paper_1511_03878_gb300 import serve


def test_scan_requests_statistics():
    reqs = serve.scan_requests()
    assert len(reqs) == 256 and [r.rid for r in reqs] == list(range(256))
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # exponential gaps of mean 1/4 s: mean within 4 standard errors, cv near 1
    assert abs(gaps.mean() - 0.25) < 4 * 0.25 / math.sqrt(256)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.2
    grids = {(r.nx, r.ny) for r in reqs}
    assert grids == {(256, 128), (512, 256), (1024, 256), (2048, 512)}
    assert all(2 <= r.a0 <= 6 and 0.003 <= r.n0 <= 0.02 for r in reqs)
    assert {r.ppc for r in reqs} == {1, 2, 4, 8}
    assert all(500 <= r.steps <= 2000 for r in reqs)
    # seeded: the same stream every time
    assert [(r.arrival, r.a0) for r in serve.scan_requests()] == [(r.arrival, r.a0) for r in reqs]


def test_request_workload_fits_its_capacity():
    for ppc in (1, 2, 4, 8):
        r = serve.Request(rid=3, nx=256, ny=128, a0=3.0, n0=0.01, ppc=ppc, steps=600)
        w = serve.request_workload(r)
        n = len(w["particles"]["x"])
        assert 0 < n <= serve.request_capacity(r)
        # the window full of plasma (what injection reaches) also fits
        assert r.nx * r.ny * ppc <= serve.request_capacity(r)
        lat = serve.PPC_LATTICE[ppc]
        assert lat[0] * lat[1] == ppc


def test_summary_definitions():
    res = [serve.Result(rid=i, arrival=float(i), admitted=float(i), started=float(i),
                        completed=float(i) + 1.0 + i, steps=10, pushes=100.0,
                        energy=np.zeros(3), ex_axis=np.zeros(4), particles=10, arena_bytes=1)
           for i in range(5)]
    s = serve.summarize(res)
    lat = np.array([1.0 + i for i in range(5)])
    assert s["p50_s"] == np.percentile(lat, 50) == 3.0
    assert s["p99_s"] == np.percentile(lat, 99)
    assert s["wall_s"] == (4.0 + 5.0) - 0.0
    assert s["aggregate_pushes_per_s"] == 500.0 / 9.0
