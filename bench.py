"""Benchmark: 0.01 m integrate + segment, frames/s (and p50/p99 ms per frame).

Workload (default): the paper-scale trajectory -- a 4 x 4 x 2 m map at 0.01 m
(sparse 8^3 bricks), a 640 x 480 depth camera (87 x 58 deg, 0.3-4 m,
sigma = 1 mm + 0.2 % of range) walking 300 frames over an 8-step open-tread
stair, a desk with a 0.4 m overhang, a 15 deg ramp, floor and 20 boxes.
One step = integrate one frame (307,200 points) + segment the accumulated map
(normals, classification, clustering, RANSAC with I = 100, refit, hulls).
The timed steps are the LAST K frames of the trajectory (the largest maps);
earlier frames are integrated untimed first.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Multi-GPU (torchrun): every rank runs its own replica
of the workload on its own GPU (no collective on the data path); value is the
frames of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FRAMES = 300
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel, from one ncu capture of the kernel as it stands, divided by the
# stat its work scales with: {stage: (bytes per unit, stat)}.  Remove a
# kernel's entry when the kernel changes.
TRAFFIC_PER_UNIT = {
    # 60-frame trajectory case (1,498 bricks; profiles/segment_kernels_60frames.md): the halo is staged
    # per brick, so the traffic scales with the allocated bricks
    "ccl_local": (14557952.0 / 1498, "bricks_allocated"),
    "ccl_cross": ((15073792.0 + 1536.0) / 1498, "bricks_allocated"),
    "moments": ((9291776.0 + 0.0) / 1498, "bricks_allocated"),
    "eigen": ((4150016.0 + 77568.0) / 1498, "bricks_allocated"),
}
METRIC = "0.01 m integrate+segment: frames/s, p50/p99 ms, batched/served vs plain GPU"
WORKLOAD = ("paper-scale trajectory: 4x4x2 m map at 0.01 m (sparse 8^3 bricks), 640x480 depth camera "
            "(87x58 deg, 0.3-4 m, sigma 1 mm + 0.2% range) over an 8-step open-tread stair, overhanging desk, "
            "15 deg ramp, floor, 20 boxes; 300 frames; step = integrate 307,200 points + segment (I=100)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--ref-budget-s", type=float, default=150.0)
    ap.add_argument("--stages", action="store_true", help="print the per-stage breakdown to stderr")
    ap.add_argument("--no-clock-sampler", action="store_true",
                    help="for profiler runs: no nvidia-smi clock sampling (the line then carries no clocks)")
    ap.add_argument("--profile-case", type=int, default=0, metavar="F",
                    help="profiling driver: integrate frames 1..F, segment --profile-segments times, no timing")
    ap.add_argument("--profile-segments", type=int, default=3)
    ap.add_argument("--profile-tuning", default="auto", metavar="TILE,R,CTAS,cta|warp",
                    help="fit schedule of the profiling drivers: 'auto' runs the autotuner first "
                         "(--profile-case; --profile-fit keeps its default schedule)")
    ap.add_argument("--no-batching", action="store_true", help="skip the batched-fit and cluster-parallel variants")
    ap.add_argument("--no-serving", action="store_true", help="skip the 16-stream serving variant")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="Poisson-arrival serving run length")
    ap.add_argument("--no-stress", action="store_true", help="skip the LiDAR stress variant")
    ap.add_argument("--no-eval", action="store_true", help="skip the time sweeps and the plane IoU")
    ap.add_argument("--stress-seconds", type=float, default=10.0, help="stress variant arrival run length")
    ap.add_argument("--profile-fit", type=int, default=0, metavar="K",
                    help="profiling driver: K config-3 clusters (sizes log-uniform in [50, 200000]), "
                         "3 fits with the default schedule, no timing")
    return ap.parse_args()


def profile_case(frames, segments, tuning="auto"):
    """A small, fixed invocation of the path for profiler captures: frames
    1..F of the paper-scale trajectory integrated, one segment call, the fit
    schedule (the autotuner as the bench runs it, or a given one), then
    `segments` segment calls."""
    import torch
    from paper_2510_01592_gb300 import vm
    import synth
    spec = synth.config2_spec()
    scene = synth.config2_scene()
    m = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size)
    for f in range(1, frames + 1):
        p, pose = synth.config2_frame(f, scene, device="cuda")
        m.integrate(p, pose)
    m.segment(seg_params(vm))
    if tuning == "auto":
        tuning = m.autotune(seg_params(vm), reps=2)[0]  # the schedule the bench times with
    else:
        t, r, c, sched = tuning.split(",")
        tuning = dict(tile=int(t), hyp_per_thread=int(r), ctas_per_sm=int(c), schedule=sched)
        m.set_fit_tuning(tuning)
    for _ in range(segments):
        r = m.segment(seg_params(vm))
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": frames, "segments": segments, "planes": int(len(r["planes"])),
                      "fit_tuning": tuning, "stats": {k: v for k, v in m.stats().items() if isinstance(v, int)}}))


def profile_fit(k, tuning="default"):
    """A small, fixed batched fit for profiler captures: the first k clusters of
    the config-3 recipe, H = 256, three runs of one plan (the default schedule,
    or a given one: TILE,R,CTAS,cta|warp)."""
    import torch
    from paper_2510_01592_gb300 import vm
    import synth
    xyz, off, _ = synth.config3_clusters_device(n_clusters=k, device="cuda")
    plan = vm.FitPlan(k, xyz.shape[0], vm.segment_params(n_hyp=256, seed=7))
    if tuning not in ("default", "auto"):
        t, r, c, sched = tuning.split(",")
        plan.set_tuning(int(t), int(r), int(c), sched)
    for _ in range(3):
        r = plan.run(xyz, off)
    torch.cuda.synchronize()
    print(json.dumps({"profile_fit": k, "points": int(xyz.shape[0]), "planes": int((r["planes"]["best_h"] >= 0).sum()),
                      "tuning": plan.tuning}))


def batching_variant(dev, stream, alu_peak):
    """Config 3: one batch of 2,000 caller-formed clusters (sizes log-uniform in
    [50, 200,000], 47.7 M points, H = 256) fitted per frame.  Plain: vm_fit_planes
    (default schedule, kernels launched one by one, one host round trip for the
    point count).  Batched: a FitPlan with the autotuned schedule, the whole fit
    replayed as one CUDA graph.  Both read the same device-resident batch."""
    import torch
    from paper_2510_01592_gb300 import vm
    import synth
    xyz, off, _ = synth.config3_clusters_device(device=dev)
    k, n = off.numel() - 1, int(xyz.shape[0])
    H = 256
    p = vm.segment_params(n_hyp=H, seed=7)
    reps = 5

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    plain_ms = timed(lambda: vm.fit_planes(xyz, off, p, stream=stream))
    plan = vm.FitPlan(k, n, p, stream=stream)
    t0 = time.perf_counter()
    best, tune_ms, n_tried = plan.autotune(xyz, off, reps=1)
    tune_s = time.perf_counter() - t0
    res = plan.run(xyz, off)
    batched_ms = timed(lambda: plan.run(xyz, off))
    plan.close()
    pt = vm.FitPlan(k, n, p, stream=stream, stage_timing=True)
    pt.set_tuning(best["tile"], best["hyp_per_thread"], best["ctas_per_sm"], best["schedule"])
    pt.run(xyz, off)
    pt.stage_times()
    pt.run(xyz, off)
    st = pt.stage_times()
    pt.close()
    score_ms = st["ransac_score"][0]
    instr = 5.0 * H * n  # 3 FFMA + FSETP(|.|) + IADD per point-hypothesis test
    ach = instr / (score_ms / 1e3) / 1e12
    del xyz, off
    torch.cuda.empty_cache()
    return {
        "workload": "2,000 clusters, sizes log-uniform in [50, 200,000] (47.7 M points), tilts U[0, 35 deg], "
                    "5% outliers, H = 256, seed 7",
        "points": n, "planes": int((res["planes"]["best_h"] >= 0).sum()),
        "plain_fits_per_s": round(1e3 / plain_ms, 2), "plain_ms": round(plain_ms, 3),
        "batched_fits_per_s": round(1e3 / batched_ms, 2), "batched_ms": round(batched_ms, 3),
        "speedup": round(plain_ms / batched_ms, 3),
        "tuning": best, "autotune": {"candidates": n_tried, "seconds": round(tune_s, 2)},
        "stages_ms": {kk: round(v[0], 4) for kk, v in st.items()},
        "ransac_score_roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 2),
                                  "unit": "T instr/s", "frac": round(ach / alu_peak, 4),
                                  "point_tests_per_s": round(H * n / (score_ms / 1e3), 1)},
    }


def e5_variant(stream, runs=1000):
    """The paper's cluster-parallel ablation: m in {1, 2, 4, 8, 16} clusters of
    M ~ U[10k, 30k] points, H = 100.  Cluster-parallel: one plan over all m
    clusters.  One at a time: m plans of one cluster each, launched back to back
    on the same stream (no host round trip between them).  Graph replays."""
    import numpy as np
    import torch
    from paper_2510_01592_gb300 import vm
    import synth
    p = vm.segment_params(n_hyp=100, seed=0)
    out = {}
    for m in (1, 2, 4, 8, 16):
        xyz_np, off_np = synth.e5_clusters(m, seed=m)
        M = int(off_np[1])
        xyz = torch.from_numpy(xyz_np).to("cuda")
        off = torch.from_numpy(off_np.astype(np.int32)).to("cuda")
        singles = [(xyz[c * M:(c + 1) * M], torch.tensor([0, M], dtype=torch.int32, device="cuda"))
                   for c in range(m)]  # int32 offsets: the uint32 bits of values below 2^31
        labels = [torch.tensor([c], dtype=torch.int32, device="cuda") for c in range(m)]
        allp = vm.FitPlan(m, m * M, p, stream=stream)
        ones = [vm.FitPlan(1, M, p, stream=stream) for _ in range(m)]

        def par():
            allp.launch(xyz, off)
            allp.wait()

        def seq():
            for c in range(m):
                ones[c].launch(singles[c][0], singles[c][1], labels[c])
            for c in range(m):
                ones[c].wait()

        res = {}
        for name, fn in (("parallel", par), ("one_at_a_time", seq)):
            for _ in range(5):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(runs):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / runs
        out[str(m)] = {"M": M, "parallel_ms": round(res["parallel"], 4),
                       "one_at_a_time_ms": round(res["one_at_a_time"], 4),
                       "speedup": round(res["one_at_a_time"] / res["parallel"], 3)}
        allp.close()
        for o in ones:
            o.close()
    return {"runs": runs, "n_hyp": 100, "by_clusters": out}


def serving_variant(dev, seconds, frames_per_stream=32, backlog=96):
    """Config 4: 16 streams (extents U[2, 6] m x 2 m, resolutions from {0.01,
    0.02, 0.05} m), 307,200-point frames from the config-2 camera over each
    stream's own stair/desk/ramp scene, maps resident on the device.
    saturation: every stream given `backlog` frames at once; frames/s of the
    batched server, the per-stream-graph server, and the plain per-frame
    pipeline (one map at a time, one synchronous integrate + segment call per
    frame), each measured over a first and a second pass of `backlog` frames
    per stream (the second on maps already grown).  poisson: arrivals at 30 Hz
    per stream for `seconds` s, latency =
    arrival to result on the host (server clock)."""
    import threading

    import numpy as np
    import torch
    from paper_2510_01592_gb300 import serve, vm
    import synth
    sts = synth.config4_streams(16)
    data = []
    for st in sts:
        sc = synth.config4_scene(st)
        fr = [synth.config4_frame(st, sc, f, device=dev) for f in range(frames_per_stream)]
        nb = 1
        for d in st.spec.dims:
            nb *= (d + 7) // 8
        data.append((st, fr, min(nb, 16384)))
    torch.cuda.synchronize()
    params = vm.segment_params(n_hyp=100, seed=0)
    out = {"streams": len(sts), "resolutions_m": sorted({st.spec.voxel_size for st in sts}),
           "frames_pregenerated_per_stream": frames_per_stream}

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None

    def saturate(mode):
        """Two timed passes of `backlog` frames per stream after a 2-frame warm-up;
        the second pass runs on maps already grown by the first."""
        srv = serve.Server(params, mode=mode, max_batch=16, max_inflight=2, device=dev.index or 0)
        ids = [srv.open(st.spec.dims, st.spec.origin, st.spec.voxel_size, cap) for st, _, cap in data]
        for j in range(2):  # warm-up: maps allocate and graphs are captured
            for (st, fr, _), sid in zip(data, ids):
                srv.submit(sid, fr[j][0], fr[j][1])
        srv.drain()
        srv.poll(256, with_planes=False)
        passes = []
        for p_ in range(2):
            s0 = srv.stats()
            n = 0
            t0 = srv.now()
            for j in range(2 + p_ * backlog, 2 + (p_ + 1) * backlog):
                for (st, fr, _), sid in zip(data, ids):
                    srv.submit(sid, fr[j % len(fr)][0], fr[j % len(fr)][1], t_arrival=t0)
                    n += 1
            srv.drain()
            t1 = srv.now()
            res = []
            while len(res) < n:
                res += srv.poll(256, timeout_ms=1000, with_planes=False)
            assert all(r["status"] == vm.VM_OK for r in res)
            s1 = srv.stats()
            passes.append({"frames_per_s": round(n / (t1 - t0), 2), "frames": n, "wall_s": round(t1 - t0, 4),
                           "mean_requests_per_step": round((s1["requests_done"] - s0["requests_done"]) /
                                                           max(1, s1["steps"] - s0["steps"]), 2),
                           "scheduler_launch_s": round(s1["launch_seconds"] - s0["launch_seconds"], 4),
                           "scheduler_complete_s": round(s1["complete_seconds"] - s0["complete_seconds"], 4),
                           "graph_captures": s1["graph_captures"] - s0["graph_captures"],
                           "allocations": s1["allocations"] - s0["allocations"],
                           "fallbacks": s1["fallbacks"] - s0["fallbacks"]})
        st = srv.stats()
        srv.close()
        return {"first_pass": passes[0], "second_pass": passes[1],
                "frames_per_s": passes[1]["frames_per_s"], "hbm_committed_gb": round(st["hbm_committed"] / 1e9, 2)}

    out["saturation_batched"] = saturate("batched")
    out["saturation_streams"] = saturate("streams")
    # the plain per-frame pipeline: one map at a time, a synchronous call per frame
    maps = [vm.VoxelMap(st.spec.dims, st.spec.origin, st.spec.voxel_size, brick_capacity=cap)
            for st, _, cap in data]
    for j in range(2):
        for m, (st, fr, _) in zip(maps, data):
            m.integrate(fr[j][0], fr[j][1])
            m.segment(params)
    torch.cuda.synchronize()
    plain = []
    for p_ in range(2):
        t0 = time.perf_counter()
        n = 0
        for j in range(2 + p_ * backlog, 2 + (p_ + 1) * backlog):
            for m, (st, fr, _) in zip(maps, data):
                m.integrate(fr[j % len(fr)][0], fr[j % len(fr)][1])
                m.segment(params)
                n += 1
        plain.append(n / (time.perf_counter() - t0))
    for m in maps:
        m.close()
    out["saturation_plain_per_frame"] = {"first_pass_frames_per_s": round(plain[0], 2),
                                         "frames_per_s": round(plain[1], 2), "frames": n}
    out["served_vs_plain"] = round(out["saturation_batched"]["frames_per_s"] / plain[1], 3)
    # Poisson arrivals at 30 Hz per stream
    srv = serve.Server(params, mode="batched", max_batch=16, max_inflight=2, device=dev.index or 0)
    ids = [srv.open(st.spec.dims, st.spec.origin, st.spec.voxel_size, cap) for st, _, cap in data]
    for (st, fr, _), sid in zip(data, ids):
        srv.submit(sid, fr[0][0], fr[0][1])
    srv.drain()
    srv.poll(256, with_planes=False)
    sched = []
    for k, (st, fr, _) in enumerate(data):
        for j, t in enumerate(synth.poisson_arrivals(st.rate_hz, seconds, st.arrival_seed)):
            sched.append((float(t), k, 1 + j))
    sched.sort()
    results = []
    stop = threading.Event()

    def poller():
        while not stop.is_set():
            results.extend(srv.poll(256, timeout_ms=50, with_planes=False))

    th = threading.Thread(target=poller)
    th.start()
    t0 = srv.now() + 0.05
    for t, k, j in sched:
        ta = t0 + t
        while True:
            dt = ta - srv.now()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.002) if dt > 0.0003 else 0)
        st, fr, _ = data[k]
        srv.submit(ids[k], fr[j % len(fr)][0], fr[j % len(fr)][1], t_arrival=ta)
    srv.drain()
    t_end = srv.now()
    stop.set()
    th.join()
    results.extend(srv.poll(256, with_planes=False))
    lat = [1e3 * (r["t_done"] - r["t_arrival"]) for r in results]
    per_stream = {}
    for r in results:
        per_stream.setdefault(r["stream"], []).append(1e3 * (r["t_done"] - r["t_arrival"]))
    st = srv.stats()
    srv.close()
    out["poisson_30hz"] = {
        "seconds": seconds, "frames": len(results), "offered_frames_per_s": round(len(sched) / seconds, 1),
        "achieved_frames_per_s": round(len(results) / (t_end - t0), 1),
        "latency_ms": {"p50": round(pct(lat, 0.5), 3), "p99": round(pct(lat, 0.99), 3), "max": round(max(lat), 3)},
        "worst_stream_p99_ms": round(max(pct(v, 0.99) for v in per_stream.values()), 3),
        "mean_requests_per_step": round(st["mean_step_requests"], 2),
        "ok": all(r["status"] == vm.VM_OK for r in results),
    }
    del data
    torch.cuda.empty_cache()
    return out


def stress_variant(dev, seconds, lidar_frames=40, cam_frames=32):
    """Config 5: one 8 x 8 x 3 m map at 0.01 m fed by a 128-beam spinning LiDAR
    (1,300,480 rays a frame, 20 Hz) over multi-level floors and 500 boxes and
    slabs, served alongside 8 paper-scale camera streams (4 x 4 x 2 m at 0.01 m,
    30 Hz, the trajectory's frames at different phases) by one batched server.
    saturation: 200 LiDAR frames and 8 x 300 camera frames queued at once;
    arrivals: LiDAR every 50 ms and Poisson camera arrivals at 30 Hz for
    `seconds` s, latency = arrival to result on the host.  The first
    `lidar_frames` / `cam_frames` frames are generated and cycled."""
    import threading

    import numpy as np
    import torch
    from paper_2510_01592_gb300 import serve, vm
    import synth
    spec5, spec2 = synth.config5_spec(), synth.config2_spec()
    sc5, sc2 = synth.config5_scene(), synth.config2_scene()
    lid = [synth.config5_frame(f, sc5, device=dev) for f in range(lidar_frames)]
    cam = [synth.config2_frame(f, sc2, device=dev) for f in range(1, cam_frames + 1)]
    torch.cuda.synchronize()
    params = vm.segment_params(n_hyp=100, seed=0)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None

    def setup():
        srv = serve.Server(params, mode="batched", max_batch=16, max_inflight=2, device=dev.index or 0)
        s5 = srv.open(spec5.dims, spec5.origin, spec5.voxel_size, 131072)
        s2 = [srv.open(spec2.dims, spec2.origin, spec2.voxel_size, 4096) for _ in range(8)]
        for f in range(2):  # warm-up
            srv.submit(s5, lid[f][0], lid[f][1])
            for j, sid in enumerate(s2):
                srv.submit(sid, cam[(f + 4 * j) % cam_frames][0], cam[(f + 4 * j) % cam_frames][1])
        srv.drain()
        srv.poll(256, with_planes=False)
        return srv, s5, s2

    out = {"lidar_rays_per_frame": int(lid[0][0].shape[0]),
           "lidar_returns_per_frame": int(torch.isfinite(lid[0][0]).all(1).sum()),
           "camera_streams": 8}
    srv, s5, s2 = setup()
    t0 = srv.now()
    n5 = n2 = 0
    for f in range(2, 202):
        srv.submit(s5, lid[f % lidar_frames][0], lid[f % lidar_frames][1], t_arrival=t0)
        n5 += 1
    for f in range(2, 302):
        for j, sid in enumerate(s2):
            k = (f + 4 * j) % cam_frames
            srv.submit(sid, cam[k][0], cam[k][1], t_arrival=t0)
            n2 += 1
    srv.drain()
    t1 = srv.now()
    res = []
    while len(res) < n5 + n2:
        res += srv.poll(512, timeout_ms=1000, with_planes=False)
    lid_done = max(r["t_done"] for r in res if r["stream"] == s5)
    out["saturation"] = {"frames": n5 + n2, "seconds": round(t1 - t0, 3),
                         "frames_per_s": round((n5 + n2) / (t1 - t0), 1),
                         "lidar_frames_per_s": round(n5 / (lid_done - t0), 2),
                         "ok": all(r["status"] == vm.VM_OK for r in res)}
    st = srv.stats()
    out["map_bricks_committed_gb"] = round(st["hbm_committed"] / 1e9, 2)
    srv.close()
    srv, s5, s2 = setup()
    sched = [(k * 0.05, -1, 2 + k) for k in range(int(seconds * 20))]
    for j in range(8):
        sched += [(float(t), j, 2 + i) for i, t in enumerate(synth.poisson_arrivals(30.0, seconds, 9000 + j))]
    sched.sort()
    results, stop = [], threading.Event()

    def poller():
        while not stop.is_set():
            results.extend(srv.poll(256, timeout_ms=50, with_planes=False))

    th = threading.Thread(target=poller)
    th.start()
    t0 = srv.now() + 0.05
    for t, j, f in sched:
        ta = t0 + t
        while True:
            dt = ta - srv.now()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.002) if dt > 0.0003 else 0)
        if j < 0:
            srv.submit(s5, lid[f % lidar_frames][0], lid[f % lidar_frames][1], t_arrival=ta)
        else:
            k = (f + 4 * j) % cam_frames
            srv.submit(s2[j], cam[k][0], cam[k][1], t_arrival=ta)
    srv.drain()
    stop.set()
    th.join()
    results.extend(srv.poll(512, with_planes=False))
    srv.close()
    l5 = [1e3 * (r["t_done"] - r["t_arrival"]) for r in results if r["stream"] == s5]
    l2 = [1e3 * (r["t_done"] - r["t_arrival"]) for r in results if r["stream"] != s5]
    out["arrivals"] = {"seconds": seconds, "lidar_frames": len(l5), "camera_frames": len(l2),
                       "lidar_latency_ms": {"p50": round(pct(l5, 0.5), 3), "p99": round(pct(l5, 0.99), 3)},
                       "camera_latency_ms": {"p50": round(pct(l2, 0.5), 3), "p99": round(pct(l2, 0.99), 3)},
                       "ok": all(r["status"] == vm.VM_OK for r in results)}
    del lid, cam
    torch.cuda.empty_cache()
    return out


def polygon_area(P):
    """Signed area of a polygon (shoelace), positive counter-clockwise."""
    import numpy as np
    P = np.asarray(P, float)
    x, y = P[:, 0], P[:, 1]
    return 0.5 * float(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def convex_iou(A, B):
    """Intersection over union of two convex polygons (Sutherland-Hodgman
    clipping of A by each edge of B, both counter-clockwise)."""
    import numpy as np
    A = [tuple(p) for p in np.asarray(A, float)]
    B = [tuple(p) for p in np.asarray(B, float)]
    if polygon_area(A) < 0:
        A = A[::-1]
    if polygon_area(B) < 0:
        B = B[::-1]
    out = A
    for i in range(len(B)):
        if not out:
            break
        c0, c1 = B[i], B[(i + 1) % len(B)]

        def side(p):
            return (c1[0] - c0[0]) * (p[1] - c0[1]) - (c1[1] - c0[1]) * (p[0] - c0[0])

        inp, out = out, []
        for j in range(len(inp)):
            p, q = inp[j], inp[(j + 1) % len(inp)]
            sp, sq = side(p), side(q)
            if sp >= 0:
                out.append(p)
            if (sp >= 0) != (sq >= 0):
                t = sp / (sp - sq)
                out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    inter = polygon_area(out) if len(out) >= 3 else 0.0
    union = polygon_area(A) + polygon_area(B) - inter
    return inter / union if union > 0 else 0.0


def evaluation_variant(dev, stream):
    """The paper's evaluation shapes on synthetic scenes.  Mapping time against
    points per frame (a LiDAR frame's first n rays into the 8 x 8 x 3 m map);
    segmentation time against accumulated occupied voxels along the
    paper-scale trajectory; the stage top's plane IoU against its exact
    region after a 48-frame orbit of the single-stage scene."""
    import numpy as np
    import torch
    from paper_2510_01592_gb300 import vm
    import synth
    out = {}
    params = vm.segment_params(n_hyp=100, seed=0)

    def ev_ms(fn, reps):
        """Median device time of reps calls (after one untimed call)."""
        fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        ev[0].record(stream)
        for i in range(reps):
            fn()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return statistics.median(ev[i].elapsed_time(ev[i + 1]) for i in range(reps))

    # mapping time against points per frame
    spec5, sc5 = synth.config5_spec(), synth.config5_scene()
    lp, lpose = synth.config5_frame(0, sc5, device=dev)
    m5 = vm.VoxelMap(spec5.dims, spec5.origin, spec5.voxel_size, brick_capacity=131072, stream=stream)
    m5.integrate(lp, lpose)
    sweep = []
    for n in (19200, 76800, 307200, 650240, 1300480):
        sub = lp[:n].contiguous()
        ms = ev_ms(lambda: m5.integrate(sub, lpose), 10)
        msc = ev_ms(lambda: m5.integrate(sub, lpose, clear=True), 5)
        sweep.append({"points": n, "integrate_ms": round(ms, 4), "clear_and_integrate_ms": round(msc, 4)})
    m5.close()
    out["mapping_vs_points"] = sweep
    # segmentation time against accumulated occupied voxels
    spec2, sc2 = synth.config2_spec(), synth.config2_scene()
    m2 = vm.VoxelMap(spec2.dims, spec2.origin, spec2.voxel_size, stream=stream)
    marks = {10, 30, 60, 100, 150, 200, 250, 300}
    curve = []
    for f in range(1, N_FRAMES + 1):
        p, pose = synth.config2_frame(f, sc2, device=dev)
        m2.integrate(p, pose)
        if f in marks:
            ms = ev_ms(lambda: m2.segment(params), 15)
            st = m2.stats()
            curve.append({"frame": f, "occupied_voxels": st["occupied_voxels"], "clusters": st["clusters"],
                          "segment_ms": round(ms, 4)})
    m2.close()
    out["segmentation_vs_voxels"] = curve
    # plane IoU of the stage top
    spec = synth.config2_spec()
    sc = synth.stage_scene()
    ms_ = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size, stream=stream)
    for k in range(48):
        p, pose = synth.stage_orbit_frame(k, 48, sc, device=dev)
        ms_.integrate(p, pose)
    r = ms_.segment(params)
    ms_.close()
    (x0, y0), (x1, y1), h = synth.STAGE
    gt = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    best = None
    for i, pl in enumerate(r["planes"]):
        if pl["best_h"] < 0 or abs(float(pl["normal"][2])) < 0.99 or abs(-float(pl["offset"]) - h) > 0.02:
            continue
        o, c = int(pl["hull_offset"]), int(pl["hull_count"])
        poly = r["hull_xyz"][o:o + c, :2]
        iou = convex_iou(poly, gt)
        if best is None or iou > best["iou"]:
            best = {"iou": round(iou, 4), "inliers": int(pl["inlier_count"]), "hull_vertices": c,
                    "height_m": round(-float(pl["offset"]), 5)}
    out["stage_top_iou"] = best
    out["planes_found"] = int(len(r["planes"]))
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, device):
    """The elementwise maximum of values over every rank (the slowest rank's
    times); needs the process group when WORLD_SIZE > 1."""
    ws, _, _ = dist_env()
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(steps, ws, slowest_ms):
    """Frames of every rank (replicas of the same steps) over the slowest rank's time."""
    return steps * ws / (slowest_ms / 1e3)


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.times = []
        self.t_mark = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.times.append(time.perf_counter())

    def mark(self):
        """Samples before this call are left out of the record (set-up work)."""
        self.t_mark = time.perf_counter()

    def wait_first(self, timeout_s=10.0):
        """Blocks until the sampler has printed its first line: nvidia-smi's own
        start-up (driver and NVML initialisation) then lies before the timed
        region instead of inside it."""
        t_end = time.perf_counter() + timeout_s
        while self.proc and not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.t_mark is not None and len(self.times) == len(self.lines):
            lines = [ln for ln, t in zip(self.lines, self.times) if t >= self.t_mark] or self.lines[-1:]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_frames(device):
    """All 300 frames on the device (float32 [300, 307200, 3]) and their poses."""
    import torch
    import synth
    scene = synth.config2_scene()
    pts = torch.empty((N_FRAMES, 640 * 480, 3), dtype=torch.float32, device=device)
    poses = []
    for f in range(1, N_FRAMES + 1):
        p, pose = synth.config2_frame(f, scene, device=device)
        pts[f - 1].copy_(p)
        poses.append(pose)
    return pts, poses


def frame_schedule(steps, warmup):
    """Frame index (0-based) of every warm-up and timed step; the timed steps end
    at the last frame.  Steps beyond one trajectory restart it on a reset map."""
    total = steps + warmup
    first = max(0, N_FRAMES - total)
    sched = [(first + i) % N_FRAMES for i in range(total)]
    return first, sched


def seg_params(vm):
    return vm.segment_params(n_hyp=100, seed=0)


def bench_config(steps, warmup, ws=1):
    """The workload description both arms print (the GPU arm and the oracle's
    reference arm time the same frames of the same trajectory)."""
    first, _ = frame_schedule(steps, warmup)
    return {"workload": WORKLOAD,
            "frames_timed": f"{first + warmup + 1}..{first + warmup + steps}"
            if first + warmup + steps <= N_FRAMES else "wrapping trajectory",
            "voxel_m": 0.01, "map_m": [4, 4, 2], "points_per_frame": 307200, "ransac_hypotheses": 100,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": "inputs larger than L2: a distinct 3.7 MB frame per step from a 1.1 GB resident "
                  "trajectory; the map state (pool + segmentation arrays, about 105 MB touched a step at "
                  "frame 300, near the 129 MB L2) is the pipeline's own state carried from step to step"}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2510_01592_gb300 import vm
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # the clock sampler starts here, its own start-up overlapping the set-up
    # work; its record keeps only the samples taken from the first timed pass on
    sampler = ClockSampler(local)
    if not args.no_clock_sampler:
        sampler.start()
    spec = synth.config2_spec()
    pts, poses = make_frames(dev)
    first, sched = frame_schedule(args.steps, args.warmup)
    params = seg_params(vm)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)  # the maps' stream is torch's current one: no cross-stream waits per frame

    tuning = None

    def fresh_map(timing=False):
        m = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size, stream=stream, stage_timing=timing)
        if tuning:
            m.set_fit_tuning(tuning)
        for f in range(first):
            m.integrate(pts[f], poses[f])
        return m

    # ---------------- device-resident inputs: the metric
    m = fresh_map()
    for i in range(args.warmup):
        f = sched[i]
        if f == 0 and i:
            m.reset()
        m.integrate(pts[f], poses[f])
        m.segment(params)
    # the fit schedule chosen by the autotuner on the warmed-up map (results do not depend on it)
    tuning, tune_ms, tune_n = m.autotune(params, reps=3)
    # one more segmentation of the same map (it does not change the map): the
    # scratch the chosen schedule needs is sized, and its graph captured, here
    m.segment(params)
    sampler.wait_first()
    # no cyclic garbage collection inside the timed passes (a full collection
    # over torch's objects takes milliseconds of host time between two steps)
    gc.collect()
    gc.disable()
    # one untimed pass of the warm-up and timed steps on a throwaway map: in a
    # fresh process the first such pass runs some 6% slower than every later
    # one (segmenting an unchanged map again does not take that away); the
    # timed map is not touched by it
    mw = fresh_map()
    for j, f in enumerate(sched[:args.warmup + min(args.steps, 100)]):
        if f == 0 and j:
            mw.reset()
        mw.integrate(pts[f], poses[f])
        mw.segment(params)
    mw.close()
    # then the timed map's own graph, segmenting the unchanged map for a tenth of a second
    t_warm = time.perf_counter()
    while time.perf_counter() - t_warm < 0.1:
        m.segment(params)
    torch.cuda.synchronize()
    sampler.mark()
    if ws > 1:
        torch.distributed.barrier()
    # throughput: the K steps bracketed by two events only (an event recorded
    # between two steps would stand between one step's last kernel and the
    # next step's first, as in the plain arm below, which records none)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0, captures0 = vm.launch_count(), vm.capture_count()
    torch.cuda.synchronize()
    e0.record(stream)
    n_planes = []
    for i in range(args.steps):
        f = sched[args.warmup + i]
        if f == 0 and (args.warmup + i):
            m.reset()
        m.integrate(pts[f], poses[f])
        r = m.segment(params)
        n_planes.append(len(r["planes"]))
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = vm.launch_count() - launches0
    graph = dict(m.graph_shape(), captures_in_timed_steps=int(vm.capture_count() - captures0))
    total_ms = e0.elapsed_time(e1)
    st = m.stats()
    m.close()
    # ---------------- per-step latency: the same steps on a fresh map, an event around each step
    ml = fresh_map()
    for i in range(args.warmup):
        f = sched[i]
        if f == 0 and i:
            ml.reset()
        ml.integrate(pts[f], poses[f])
        ml.segment(params)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]  # where each step's GPU work begins
    ev[0].record(stream)
    for i in range(args.steps):
        f = sched[args.warmup + i]
        if f == 0 and (args.warmup + i):
            ml.reset()
        evs[i].record(stream)
        ml.integrate(pts[f], poses[f])
        ml.segment(params)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    ml.close()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    # the GPU's idle time between steps: the host reads a step's result and
    # enqueues the next step (a synchronous segment call per frame)
    host_gap_ms = statistics.median(ev[i].elapsed_time(evs[i]) for i in range(1, args.steps)) if args.steps > 1 else 0.0
    # ---------------- plain per-frame launches (kernel by kernel, no graph), same frames
    mp = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size, stream=stream, eager=True)
    mp.set_fit_tuning(tuning)
    for f in range(first):
        mp.integrate(pts[f], poses[f])
    for i in range(args.warmup):
        f = sched[i]
        mp.integrate(pts[f], poses[f])
        mp.segment(params)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        f = sched[args.warmup + i]
        if f == 0 and (args.warmup + i):
            mp.reset()
        mp.integrate(pts[f], poses[f])
        mp.segment(params)
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    mp.close()
    # ---------------- stage breakdown over the same frames (separate instrumented pass)
    mt = fresh_map(timing=True)
    for i in range(args.warmup):
        f = sched[i]
        mt.integrate(pts[f], poses[f])
        mt.segment(params)
    mt.stage_times()
    for i in range(args.steps):
        f = sched[args.warmup + i]
        if f == 0 and (args.warmup + i):
            mt.reset()
        mt.integrate(pts[f], poses[f])
        mt.segment(params)
    stages = mt.stage_times()
    mt.close()
    # ---------------- end to end: host (pinned) inputs, host results
    host_pts = [pts[f].cpu().pin_memory() for f in sorted(set(sched))]
    host_of = {f: host_pts[j] for j, f in enumerate(sorted(set(sched)))}
    # three passes over the same steps, each on a fresh map; the median pass is
    # the figure (a wall-clock pass on the shared host sees its jitter)
    e2e_passes = []
    for _ in range(3):
        me = fresh_map()
        for i in range(args.warmup):
            f = sched[i]
            me.integrate(host_of[f].numpy(), poses[f])
            me.segment(params)
        torch.cuda.synchronize()
        d2h = 0
        t0 = time.perf_counter()
        for i in range(args.steps):
            f = sched[args.warmup + i]
            if f == 0 and (args.warmup + i):
                me.reset()
            me.integrate(host_of[f].numpy(), poses[f])
            r = me.segment(params)
            d2h += r["planes"].nbytes + r["hull_xy"].nbytes + r["hull_xyz"].nbytes
        torch.cuda.synchronize()
        e2e_passes.append(time.perf_counter() - t0)
        me.close()
    e2e_s = sorted(e2e_passes)[1]

    # ---------------- the same steps with ray-cast clearing (Eq. 2) before each frame's update
    mc = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size, stream=stream)
    mc.set_fit_tuning(tuning)
    for f in range(first):
        mc.integrate(pts[f], poses[f], clear=True)
    for i in range(args.warmup):
        f = sched[i]
        mc.integrate(pts[f], poses[f], clear=True)
        mc.segment(params)
    torch.cuda.synchronize()
    c0 = mc.stats()["voxels_cleared"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        f = sched[args.warmup + i]
        if f == 0 and (args.warmup + i):
            mc.reset()
        mc.integrate(pts[f], poses[f], clear=True)
        mc.segment(params)
    e1.record(stream)
    torch.cuda.synchronize()
    clear_ms = e0.elapsed_time(e1)
    cleared = mc.stats()["voxels_cleared"] - c0
    mc.close()
    mct = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size, stream=stream, stage_timing=True)
    for f in range(first):
        mct.integrate(pts[f], poses[f], clear=True)
    mct.stage_times()
    for i in range(args.steps):
        f = sched[args.warmup + i]
        mct.integrate(pts[f], poses[f], clear=True)
    clear_stage = mct.stage_times().get("clear", (0.0, 0))
    mct.close()

    # ---------------- sequential multi-plane extraction: the same steps with up to 3 planes per cluster
    def steps_pass(prm):
        mm = fresh_map()
        for i in range(args.warmup):
            f = sched[i]
            mm.integrate(pts[f], poses[f])
            mm.segment(prm)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        planes, extra = [], []
        a.record(stream)
        for i in range(args.steps):
            f = sched[args.warmup + i]
            if f == 0 and (args.warmup + i):
                mm.reset()
            mm.integrate(pts[f], poses[f])
            p = mm.segment(prm)["planes"]
            planes.append(len(p))
            extra.append(int((((p["flags"] >> 8) & 0xFF) > 0).sum()))
        b.record(stream)
        torch.cuda.synchronize()
        mm.close()
        return {"frames_per_s": round(args.steps / (a.elapsed_time(b) / 1e3), 2),
                "planes_per_frame": round(float(np.mean(planes)), 2),
                "later_round_planes_per_frame": round(float(np.mean(extra)), 2)}

    multiplane = {"steppable_p3": steps_pass(vm.segment_params(n_hyp=100, seed=0, planes_per_cluster=3)),
                  "all_occupied_p1": steps_pass(vm.segment_params(n_hyp=100, seed=0, classify=0)),
                  "all_occupied_p3": steps_pass(vm.segment_params(n_hyp=100, seed=0, classify=0,
                                                                  planes_per_cluster=3)),
                  "note": "the same timed steps with up to 3 planes per cluster (round r + 1 on round r's "
                          "non-inliers); steppable: the paper's clustering, all_occupied: every occupied voxel "
                          "clustered, where clusters join walls and ledges; graph replay"}

    # ---------------- config 1: the single frame (20,000 points, 50 x 50 x 25 map at 0.02 m, 64 hypotheses)
    spec1, pts1_np, _ = synth.config1()
    pts1 = torch.from_numpy(pts1_np).to(dev)
    eye = np.eye(3, 4, dtype=np.float32).reshape(12)
    p1 = vm.segment_params(n_hyp=64, seed=0)
    m1 = vm.VoxelMap(spec1.dims, spec1.origin, spec1.voxel_size, stream=stream)
    for _ in range(5):
        m1.reset()
        m1.integrate(pts1, eye)
        m1.segment(p1)
    torch.cuda.synchronize()
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(51)]
    ev1[0].record(stream)
    for i in range(50):
        m1.reset()
        m1.integrate(pts1, eye)
        n1 = len(m1.segment(p1)["planes"])
        ev1[i + 1].record(stream)
    torch.cuda.synchronize()
    c1 = sorted(ev1[i].elapsed_time(ev1[i + 1]) for i in range(50))
    config1 = {"frames_per_s": round(50 / (ev1[0].elapsed_time(ev1[-1]) / 1e3), 2), "p50_ms": round(c1[25], 4),
               "p99_ms": round(c1[49], 4), "planes": n1,
               "note": "reset + integrate the 20,000-point frame + segment (64 hypotheses) per step, graph replay"}
    m1.close()

    # ---------------- robot-centric map: a 5 m cube at 0.01 m (the paper's mapping volume) centred on the
    # camera before every frame, the same timed steps
    def cam_of(f):
        return np.float32([poses[f][3], poses[f][7], poses[f][11]])

    mr = vm.VoxelMap((500, 500, 500), (-2.5, -2.5, -2.5), 0.01, stream=stream)
    mr.set_fit_tuning(tuning)
    for f in range(first):
        mr.scroll_to(cam_of(f))
        mr.integrate(pts[f], poses[f])
    for i in range(args.warmup):
        f = sched[i]
        mr.scroll_to(cam_of(f))
        mr.integrate(pts[f], poses[f])
        mr.segment(params)
    torch.cuda.synchronize()
    ev0, w0 = mr.stats()["voxels_evicted"], mr.window()["offset"].copy()
    n_scroll, rc_planes = 0, []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(args.steps):
        f = sched[args.warmup + i]
        if f == 0 and (args.warmup + i):
            mr.reset()
        n_scroll += int(mr.scroll_to(cam_of(f)).any())
        mr.integrate(pts[f], poses[f])
        rc_planes.append(len(mr.segment(params)["planes"]))
    b.record(stream)
    torch.cuda.synchronize()
    rst = mr.stats()
    robot_centric = {"frames_per_s": round(args.steps / (a.elapsed_time(b) / 1e3), 2),
                     "scrolls": n_scroll, "window_moved_voxels": (mr.window()["offset"] - w0).tolist(),
                     "voxels_evicted_per_frame": round((rst["voxels_evicted"] - ev0) / args.steps, 1),
                     "planes_per_frame": round(float(np.mean(rc_planes)), 2), "bricks": rst["bricks_allocated"],
                     "note": "a 5 x 5 x 5 m window at 0.01 m (500^3 voxels) re-centred on the camera in whole "
                             "bricks before every frame (vm_scroll_to: eviction, pool compaction, re-anchoring), "
                             "then integrate + segment; graph replay"}
    mr.close()
    clocks = sampler.stop()
    gc.enable()

    total_ms, e2e_s = max_over_ranks([total_ms, e2e_s], dev)
    frames = args.steps * ws
    value = whole_job_rate(args.steps, ws, total_ms)
    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic (ray-cast scenes)",
        "config": bench_config(args.steps, args.warmup, ws),
        "fit_tuning": dict(tuning, autotune_candidates=tune_n, autotune_ms=round(tune_ms, 4)),
        "host_gap_ms": round(host_gap_ms, 4),
        "segment_graph": graph,
        "latency_pass": "p50_ms, p99_ms and host_gap_ms: the same steps again on a fresh map, an event pair around "
                        "each step; value and ms_per_step: the steps bracketed by two events",
        "p50_ms": round(statistics.median(per_step), 4),
        "p99_ms": round(sorted(per_step)[min(len(per_step) - 1, int(math.ceil(0.99 * len(per_step))) - 1)], 4),
        "gpu_launches": int(launches),
        "e2e": {"value": round(frames / e2e_s, 2), "unit": "frames/s", "h2d_bytes_per_step": 640 * 480 * 12,
                "d2h_bytes_per_step": int(d2h / max(1, args.steps)),
                "passes_frames_per_s": [round(args.steps / t, 2) for t in e2e_passes],
                "note": "the median of three wall-clock passes over the same steps, each on a fresh map"},
        "planes_per_frame": round(float(np.mean(n_planes)), 2),
        "variants": {"clearing": {"frames_per_s": round(args.steps / (clear_ms / 1e3), 2),
                                  "clear_ms_per_frame": round(clear_stage[0] / max(1, clear_stage[1]), 4),
                                  "voxels_cleared_per_frame": round(cleared / args.steps, 1),
                                  "note": "the same timed steps with ray-cast clearing (Eq. 2) of every frame's "
                                          "rays before its update; graph replay"},
                     "config1_single_frame": config1,
                     "multiplane": multiplane,
                     "robot_centric": robot_centric,
                     "graph_frames_per_s": round(value, 2),
                     "plain_eager_frames_per_s": round(args.steps / (eager_ms / 1e3), 2),
                     "note": "graph: each segment call replays one captured CUDA graph of the whole device-driven "
                             "pipeline; plain: the same kernels launched one by one"},
        "map": {"occupied_voxels": st["occupied_voxels"], "steppable_voxels": st["steppable_voxels"],
                "clustered_points": st["clustered_points"], "clusters": st["clusters"],
                "bricks": st["bricks_allocated"], "device_bytes": st["device_bytes"]},
    }
    if clocks:
        res["clocks"] = clocks
    if not args.no_batching and rank == 0:
        peaks = load_peaks() or {}
        alu_peak = SM_COUNT * FP32_LANES * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        res["variants"]["batching_config3"] = batching_variant(dev, stream, alu_peak)
        res["variants"]["cluster_parallel_e5"] = e5_variant(stream)
    if not args.no_serving and rank == 0:
        res["variants"]["serving_config4"] = serving_variant(dev, args.serve_seconds)
    if not args.no_stress and rank == 0:
        res["variants"]["stress_config5"] = stress_variant(dev, args.stress_seconds)
    if not args.no_eval and rank == 0:
        res["variants"]["evaluation"] = evaluation_variant(dev, stream)
    res["stages_ms_per_step"] = {k: round(v[0] / max(1, args.steps), 4) for k, v in stages.items() if v[1]}
    timed = [sched[args.warmup + i] for i in range(args.steps)]
    fv = sum(frame_voxels(pts[f], poses[f], spec) for f in timed) / max(1, len(timed))
    table = kernel_table(stages, st, load_peaks(), st["clustered_points"], frame_points=640 * 480,
                         frame_voxels=fv)
    res["kernels"] = table
    res["roofline"] = roofline(table, {k: v * st[unit] for k, (v, unit) in TRAFFIC_PER_UNIT.items()})
    return res, rank


# FP32 lanes x clock: one instruction per lane per cycle on 152 SMs x 128 lanes
SM_COUNT, FP32_LANES = 152, 128


def kernel_table(stages, st, peaks, n_points_segment, frame_points=0, frame_voxels=0, n_hyp=100):
    """Per-stage average launch time and, for the stages the method's own
    units price, the achieved rate against the measured peak: algorithmic
    bytes (or instructions) of one launch / its average CUDA-event time.

    Algorithmic units (what the method must move, whatever the kernel
    stages): integrate 12 B read per frame point + 4 B brick-table probe per
    point + 28 B read-modify-write per distinct voxel the frame touches;
    finalize 28 B sums and count read + 12 B mean written + 4 B id per
    occupied voxel; moments 12 B mean read + 1 B neighbour count written per
    occupied voxel; eigen ~520 FP32 instructions per occupied voxel; CCL 24 B
    (mean, normal) + 4 B label x (1 + 1 pass) per vertex (steppable voxel):
    the in-brick pass is priced at 24 B + 4 B (its reads and its labels), the
    cross-brick pass, which completes the labels, at the whole 32 B;
    RANSAC scoring 5 instructions per point-hypothesis test.  staged_bytes:
    what the kernel as written reads and writes for the same launch, where
    it differs (per-slot staging of allocated bricks: slots = bricks x 512).
    kernels: launches in the stage; only single-kernel stages are roofline
    candidates."""
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    clk = (peaks or {}).get("sm_max_mhz", 2070.0) * 1e6
    alu_peak = SM_COUNT * FP32_LANES * clk / 1e12  # T instructions/s
    occ = st["occupied_voxels"]
    vert = st["steppable_voxels"]
    slots = st["bricks_allocated"] * 512
    model = {  # name: (bound, algorithmic amount, staged bytes or None, kernels in the stage)
        "integrate": ("hbm", frame_points * (12 + 4) + frame_voxels * 28,
                      frame_points * (12 * 2 + 4) + frame_voxels * 28, 2),
        "finalize": ("hbm", occ * (28 + 12 + 4), slots * (4 + 1 + 12) + occ * 24, 1),
        "moments": ("hbm", occ * (12 + 1), slots * (12 + 16 + 8) + occ * (4 + 24 + 1), 1),
        "eigen": ("alu", occ * 520, None, 1),
        "ccl_local": ("hbm", vert * (24 + 4), None, 1),
        "ccl_cross": ("hbm", vert * (24 + 4 * 2), None, 1),
        "ransac_score": ("alu", n_points_segment * n_hyp * 5, None, 1),
    }
    out = {}
    for name, (ms_tot, calls) in stages.items():
        if not calls:
            continue
        ms = ms_tot / calls
        row = {"avg_launch_ms": round(ms, 4)}
        if name in model:
            bound, amount, staged, nk = model[name]
            if bound == "hbm":
                ach = amount / (ms / 1e3) / 1e9
                row.update(bound="hbm", achieved=round(ach, 1), peak=hbm, unit="GB/s", frac=round(ach / hbm, 4),
                           algorithmic=int(amount))
            else:
                ach = amount / (ms / 1e3) / 1e12
                row.update(bound="alu", achieved=round(ach, 3), peak=round(alu_peak, 1), unit="T instr/s",
                           frac=round(ach / alu_peak, 4), algorithmic=int(amount))
            if staged is not None:
                row["staged_bytes"] = int(staged)
            row["kernels"] = nk
        out[name] = row
    return out


def roofline(table, traffic=None):
    """The dominant single-kernel stage's row; traffic: DRAM bytes per launch
    from an ncu capture of that kernel, and its ratio to the algorithmic
    bytes."""
    single = {k: v for k, v in table.items() if "bound" in v and v.get("kernels", 1) == 1}
    if not single:
        return None
    dom = max(single, key=lambda k: single[k]["avg_launch_ms"])
    r = dict(single[dom])
    r["kernel"] = dom
    t = (traffic or {}).get(dom)
    r["traffic"] = None if t is None else int(t)
    if t is not None and r["bound"] == "hbm" and r["algorithmic"]:
        r["traffic_ratio"] = round(t / r["algorithmic"], 3)
    r["peak_source"] = "MEASURED_PEAKS.json" if load_peaks() else "fallback"
    return r


def frame_voxels(pts, pose, spec):
    """Distinct voxels a frame's points fall in (the integrate stage's
    algorithmic unit), counted with torch on the frame's device."""
    import torch
    R = torch.tensor(pose, dtype=torch.float32, device=pts.device).reshape(3, 4)
    w = pts @ R[:, :3].T + R[:, 3]
    o = torch.tensor(spec.origin, dtype=torch.float32, device=pts.device)
    k = torch.floor((w - o) * (1.0 / spec.voxel_size)).to(torch.int64)
    d = torch.tensor(spec.dims, dtype=torch.int64, device=pts.device)
    ok = ((k >= 0) & (k < d)).all(dim=1)
    k = k[ok]
    return int(torch.unique((k[:, 2] * d[1] + k[:, 1]) * d[0] + k[:, 0]).numel())


def headline(res):
    """The batched / served figures against the plain per-frame pipeline,
    gathered from the variants into flat keys."""
    v = res.get("variants", {})
    h = {"graph_frames_per_s": v.get("graph_frames_per_s"),
         "plain_eager_frames_per_s": v.get("plain_eager_frames_per_s")}
    sv = v.get("serving_config4")
    if sv:
        h.update(served_fps=sv["saturation_batched"]["frames_per_s"],
                 served_streams_fps=sv["saturation_streams"]["frames_per_s"],
                 plain_fps=sv["saturation_plain_per_frame"]["frames_per_s"],
                 served_p50_ms=sv["poisson_30hz"]["latency_ms"]["p50"],
                 served_p99_ms=sv["poisson_30hz"]["latency_ms"]["p99"],
                 served_worst_stream_p99_ms=sv["poisson_30hz"]["worst_stream_p99_ms"],
                 served_streams=sv["streams"], served_rate_hz=30)
    bt = v.get("batching_config3")
    if bt:
        h.update(batch_ms=bt["batched_ms"], plain_batch_ms=bt["plain_ms"], batch_speedup=bt["speedup"])
    return {k: x for k, x in h.items() if x is not None}


def cpu_baseline(budget_s, all_cores=True, steps=30, warmup=0):
    """The oracle as it stands, single-threaded on the host, over a bounded
    sample of the frames the GPU arm times: the frames before them
    integrated untimed (the warm-up frames integrated and segmented), then
    integrate + segment per frame until the frames or the budget run out.
    all_cores adds the same sample with the oracle's independent stages
    (integration over point ranges, normals over voxels, fits over clusters)
    on every host core; its results are identical."""
    import torch

    import oracle
    import synth
    spec = synth.config2_spec()
    scene = synth.config2_scene()
    prm = oracle.make_params(n_hyp=100, seed=0)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    first, _ = frame_schedule(steps, warmup)
    start = first + warmup if first + warmup + steps <= N_FRAMES else N_FRAMES - min(steps, N_FRAMES)
    frames = [synth.config2_frame(f, scene, device=dev) for f in range(1, N_FRAMES + 1)]
    frames = [(p.cpu().numpy(), pose) for p, pose in frames]

    def timed(threads):
        oracle.set_threads(threads)
        try:
            om = oracle.OracleMap(spec.dims, spec.origin, spec.voxel_size)
            for f in range(start):
                om.integrate(*frames[f])
                if f >= start - warmup:
                    om.segment(prm)
            done, t_used = 0, 0.0
            while t_used < budget_s and done < steps and start + done < N_FRAMES:
                host, pose = frames[start + done]
                t0 = time.perf_counter()
                om.integrate(host, pose)
                om.segment(prm)
                t_used += time.perf_counter() - t0
                done += 1
            om.close()
            return done, t_used
        finally:
            oracle.set_threads(1)

    done, t_used = timed(1)
    out = {"value": round(done / t_used, 4), "unit": "frames/s", "cores": 1, "kind": "oracle",
           "sample": f"frames {start + 1}..{start + done} of the 300-frame trajectory (frames 1..{start} "
                     f"integrated untimed first), integrate + segment each, single-threaded C oracle"}
    if all_cores:
        n = os.cpu_count() or 1
        d2, t2 = timed(n)
        out["all_cores"] = {"value": round(d2 / t2, 4), "unit": "frames/s", "cores": n,
                            "sample": f"the same frames {start + 1}..{start + d2}, the oracle's integration, "
                                      f"normals and per-cluster fits split over {n} threads (CCL and "
                                      f"cluster formation stay sequential)"}
    return out


def cpu_baseline_configs(config3_sample_every=20):
    """The oracle on the other configurations' single units, on the host:
    config 1 (one frame of 20,000 points into the 50 x 50 x 25 map at 0.02 m,
    integrate + segment with 64 hypotheses), 1 core and all cores; config 3
    (the 2,000-cluster batch, H = 256), all cores on the whole batch and 1 core
    on every config3_sample_every-th cluster, scaled by point-hypothesis tests
    to the whole batch."""
    import numpy as np
    import torch

    import oracle
    import synth
    out = {}
    spec, pts, _ = synth.config1()
    prm1 = oracle.make_params(n_hyp=64, seed=0)
    n = os.cpu_count() or 1
    for th in (1, n):
        oracle.set_threads(th)
        try:
            ts = []
            for _ in range(5):
                om = oracle.OracleMap(spec.dims, spec.origin, spec.voxel_size)
                t0 = time.perf_counter()
                om.integrate(pts)
                om.segment(prm1)
                ts.append(time.perf_counter() - t0)
                om.close()
        finally:
            oracle.set_threads(1)
        out.setdefault("config1", {})["ms_1core" if th == 1 else "ms_all_cores"] = round(1e3 * min(ts), 3)
    out["config1"]["cores"] = n
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    xyz, off, _ = synth.config3_clusters_device(device=dev)
    xyz, off = xyz.cpu().numpy(), off.cpu().numpy().astype(np.uint32)
    prm3 = oracle.make_params(n_hyp=256, seed=7)
    oracle.set_threads(n)
    try:
        t0 = time.perf_counter()
        oracle.fit_planes(xyz, off, prm3)
        t_all = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    sel = np.arange(0, off.shape[0] - 1, config3_sample_every)
    sizes = (off[1:] - off[:-1]).astype(np.int64)
    sub_off = np.concatenate([[0], np.cumsum(sizes[sel])]).astype(np.uint32)
    sub = np.concatenate([xyz[off[c]:off[c + 1]] for c in sel])
    t0 = time.perf_counter()
    oracle.fit_planes(sub, sub_off, prm3, labels=sel.astype(np.uint32))
    t_one = time.perf_counter() - t0
    out["config3"] = {"ms_all_cores": round(1e3 * t_all, 1), "cores": n,
                      "ms_1core_scaled": round(1e3 * t_one * float(sizes.sum()) / float(sizes[sel].sum()), 1),
                      "sample_1core": f"every {config3_sample_every}th cluster ({len(sel)} clusters, "
                                      f"{int(sizes[sel].sum())} points) timed on 1 core, scaled by points"}
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None, rank
    cb = cpu_baseline(args.ref_budget_s, all_cores=False, steps=args.steps, warmup=args.warmup)
    res = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "frames/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic (ray-cast scenes)",
           "config": bench_config(args.steps, args.warmup),
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return res, rank


def main():
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case, args.profile_segments, args.profile_tuning)
        return
    if args.profile_fit:
        profile_fit(args.profile_fit, args.profile_tuning)
        return
    if args.impl == "reference":
        res, rank = run_reference(args)
        if res is not None and rank == 0:
            print(json.dumps(res))
        return
    res, rank = run_gpu(args)
    ws, _, _ = dist_env()
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(args.cpu_budget_s, steps=args.steps, warmup=args.warmup)
            res["cpu_baseline"]["other_configs"] = cpu_baseline_configs()
        if args.stages:
            print(json.dumps(res["stages_ms_per_step"], indent=1), file=sys.stderr)
        # flat headline keys near the front of the line, and the same object
        # again as the line's last key (where a truncated tail still shows it)
        h = headline(res)
        front = {k: res[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step")}
        front.update(h)
        res = dict(front, **{k: x for k, x in res.items() if k not in front})
        res["headline"] = h
        print(json.dumps(res))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
