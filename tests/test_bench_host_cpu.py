"""Host logic of bench.py that needs no GPU: launch counts and the CPU timing samples."""
import types

import bench


def test_kernels_per_step_counts_injection_and_merge():
    assert bench.kernels_per_step(False) == 9
    assert bench.kernels_per_step(True) == 10
    assert bench.kernels_per_step(False, True) == 10
    assert bench.kernels_per_step(True, True) == 11
    assert bench.kernels_per_step(True, True, True) == 14


def _args(**kw):
    a = dict(nx=2048, ny=512, workload="lwfa", total=64 * 2 ** 20, maxwell_order=2)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_oracle_sample_cuts_rows_of_the_window():
    w, what = bench.oracle_sample(_args(nx=64, ny=256), 0.25)
    assert list(w["params"]["n"][:2]) == [64, 64]
    assert "64x64 rows" in what


def test_oracle_sample_thins_particles_on_the_same_grid():
    full, _ = bench.oracle_sample(_args(workload="thermal"), 1.0)
    w, what = bench.oracle_sample(_args(workload="thermal"), 0.25)
    assert list(w["params"]["n"]) == list(full["params"]["n"])
    assert len(w["particles"]["x"]) == len(full["particles"]["x"]) // 4
    assert "one particle in 4" in what


def test_oracle_sim_has_room_for_the_injected_columns():
    import oracle as orc

    orc.build()
    from paper_1511_03878_gb300 import inputs

    w = inputs.lwfa2d(nx=64, ny=32, ramp_x0=-8.0, patch=(16, 16))
    o = bench.oracle_sim(w, 12)
    n0 = o.num_particles()
    o.step(12)  # the window shifts about 11 times, dropping and injecting a column each time
    assert o.shifts >= 10
    assert abs(o.num_particles() - n0) <= 32 * 4


def test_algorithmic_bytes_per_push():
    """LWFA window at 4 particles per cell: the push's bytes (state read and written,
    weight read, E and B read and FP64 J written per cell) and the whole step's (plus
    the field update per cell)."""
    from paper_1511_03878_gb300 import inputs

    w = inputs.lwfa2d(nx=256, ny=64, ramp_x0=-8.0, patch=(32, 32))
    assert bench.bytes_per_push("fp64", w) == 2 * (16 + 24) + 8 + (48 + 24) / 4
    assert bench.bytes_per_push("fp32", w) == 2 * (12 + 12) + 4 + (24 + 24) / 4
    assert bench.step_bytes_per_push("fp32", w) == 88.0
    assert bench.step_bytes_per_push("fp64", w) == 142.0


def test_lwfa_line_is_timed_on_the_developed_run():
    """The default LWFA line starts from the configured initial condition (plasma from
    the pulse centre) and develops it 1800 steps before timing; its capacity covers the
    window full of plasma; the workload name says where the timing starts."""
    from paper_1511_03878_gb300 import inputs

    a = _args(lwfa_start="ramp", develop=-1, gpus=1)
    assert bench.develop_steps(a) == 1800
    assert bench.develop_steps(_args(lwfa_start="full", develop=-1)) == 0
    assert bench.develop_steps(_args(workload="stress3d", lwfa_start="ramp", develop=-1)) == 0
    assert bench.develop_steps(_args(lwfa_start="ramp", develop=5)) == 5
    assert bench.config_dict(a, "fp64")["workload"] == "lwfa2d-2048x512-ppc4-from-step1800"
    w = bench.workload(2048, 32, "lwfa", start="ramp")
    full = 2048 * 32 * 4
    assert len(w["particles"]["x"]) < full / 2  # plasma from the pulse centre only
    assert bench.capacity_for(w) == 3 * full
    wf = bench.workload(2048, 32, "lwfa", start="full")
    assert len(wf["particles"]["x"]) == full
    assert w["params"]["ramp_x0"] == inputs.lwfa2d(nx=2048, ny=32)["params"]["ramp_x0"]


def test_code_digest_ignores_comments_not_code():
    a = 'int f(int x) {  // twice\n    return 2 * x; /* doubled */\n}\nconst char* s = "a // b";\n'
    b = '/* header */\nint f(int x) {\n\n    return 2 * x;\n}   \nconst char* s = "a // b";'
    c = 'int f(int x) {\n    return 3 * x;\n}\nconst char* s = "a // b";\n'
    d = 'int f(int x) {\n    return 2 * x;\n}\nconst char* s = "a //  b";\n'
    e = '#define K 1\nint f(int x) { return K * x; }\n'
    f = '#define K 1 int f(int x) { return K * x; }\n'
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)   # code changed
    assert bench.code_only(a) != bench.code_only(d)   # a string literal changed
    assert bench.code_only(e) != bench.code_only(f)   # a line break that ends a macro


def test_traffic_table_covers_the_current_kernels():
    """The committed ncu traffic rows of the default bench line's kernels were taken on
    the current kernel code: a code change without a new capture fails here."""
    assert bench.measured_traffic("push2d_kernel<double>", "lwfa2d-2048x512-ppc4-from-step1800",
                                  (32, 32), 4096, 2) is not None
    assert bench.measured_traffic("push2d_kernel<float>", "lwfa2d-2048x512-ppc4-from-step1800",
                                  (32, 32), 4096, 2) is not None
    assert bench.measured_traffic("push3d_kernel<float>",
                                  "stress3d-256x128x128-lognormal1.5-n67108864",
                                  (8, 8, 8), 8192, 3) is not None


class _FakeSim:
    """Records the calls the end-to-end loop makes, with a device that runs in order."""

    def __init__(self):
        self.log = []
        self.enqueued = 0
        self.slots = {}

    def step(self, n):
        self.enqueued += n
        self.log.append(("step", self.enqueued))

    def step_record_async(self, slot):
        assert slot not in self.slots  # a slot is reused only after its wait
        self.slots[slot] = self.enqueued
        self.log.append(("record", slot))

    def record_wait(self, slot):
        steps = self.slots.pop(slot)
        self.log.append(("wait", slot))
        return steps, 0


def test_e2e_loop_waits_one_step_behind():
    sim = _FakeSim()
    recs = bench.pipelined_steps(sim, 5)
    assert [r[0] for r in recs] == [1, 2, 3, 4, 5]
    # steps enqueued when each wait starts: the wait for step k comes after step k + 1
    # was enqueued (the last one after the last step)
    steps_before = [max([a for w, a in sim.log[:i] if w == "step"], default=0)
                    for i, (w, _) in enumerate(sim.log) if w == "wait"]
    assert steps_before == [2, 3, 4, 5, 5]
    assert bench.pipelined_steps(_FakeSim(), 0) == []
