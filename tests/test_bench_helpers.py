"""The benchmark's measurement arithmetic on the host: per-stage roofline rows
from algorithmic bytes and CUDA-event times, the dominant single-kernel stage,
the whole-job rate over replicas, the clock record parsed from nvidia-smi
samples, and the schedule that times the last frames of the trajectory."""
import bench


def test_kernel_table_rows_and_the_dominant_kernel():
    st = {"occupied_voxels": 1000, "steppable_voxels": 600, "bricks_allocated": 10}
    peaks = {"hbm_gbs": 5000.0, "sm_max_mhz": 2000.0}
    stages = {"ccl_cross": (0.5, 10), "moments": (0.2, 10), "clusters": (0.9, 10), "eigen": (0.1, 10),
              "integrate": (0.9, 10), "pack": (0.0, 0)}
    t = bench.kernel_table(stages, st, peaks, n_points_segment=4000, frame_points=3000, frame_voxels=700)
    ccl = 600 * (24 + 4 * 2)  # per vertex: mean and normal read, label written and read once more
    assert t["ccl_cross"]["algorithmic"] == ccl
    assert abs(t["ccl_cross"]["achieved"] - round(ccl / 0.05e-3 / 1e9, 1)) < 1e-9
    assert abs(t["ccl_cross"]["frac"] - round(ccl / 0.05e-3 / 1e9 / 5000.0, 4)) < 1e-12
    assert t["moments"]["algorithmic"] == 1000 * 13 and t["moments"]["staged_bytes"] > 1000 * 13
    assert t["integrate"]["algorithmic"] == 3000 * 16 + 700 * 28 and t["integrate"]["kernels"] == 2
    alu = bench.SM_COUNT * bench.FP32_LANES * 2000e6 / 1e12
    assert t["eigen"]["bound"] == "alu" and t["eigen"]["peak"] == round(alu, 1)
    assert "bound" not in t["clusters"] and "pack" not in t  # several kernels; no calls
    r = bench.roofline(t, traffic={"ccl_cross": 9600.9})
    # the longest stage that is a single modelled kernel: not the longer multi-kernel ones
    assert r["kernel"] == "ccl_cross" and r["traffic"] == 9600 and r["avg_launch_ms"] == 0.05
    assert r["traffic_ratio"] == round(9600.9 / ccl, 3)
    assert bench.roofline(t)["traffic"] is None


def test_whole_job_rate_and_schedule():
    assert bench.whole_job_rate(100, 1, 50.0) == 2000.0
    assert bench.whole_job_rate(100, 4, 50.0) == 8000.0  # replicas: frames of every rank
    first, sched = bench.frame_schedule(100, 3)
    assert first == bench.N_FRAMES - 103 and sched[-1] == bench.N_FRAMES - 1 and len(sched) == 103
    first, sched = bench.frame_schedule(bench.N_FRAMES + 5, 3)  # longer than a trajectory: wraps
    assert first == 0 and len(sched) == bench.N_FRAMES + 8 and sched[bench.N_FRAMES] == 0


def test_clock_record_from_samples():
    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler(0)
    c.proc = Done()
    c.lines = ["2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
               "1965, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
               "2032, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    rec = c.stop()
    assert rec == {"sm_mhz": 2032.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c2 = bench.ClockSampler(0)
    assert c2.stop() is None  # never started: no record


def test_clock_record_keeps_the_samples_after_the_mark():
    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler(0)
    c.proc = Done()
    c.lines = ["1200, 2070, 300.0, Not Active, Not Active, Not Active, Not Active",
               "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
               "2040, 2070, 950.0, Not Active, Not Active, Not Active, Active"]
    c.times = [1.0, 2.0, 3.0]
    c.t_mark = 1.5  # the idle set-up sample is left out
    assert c.stop() == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    c.t_mark = 9.0  # nothing after the mark: the last sample stands in
    assert c.stop()["samples"] == 1
