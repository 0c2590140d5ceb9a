"""GPU: the multi-stream server.  Each stream's result is the same served in a
mix (continuous batching, one batched fit over several maps per step, or one
graph per map on its own stream) as its frames run alone through a plain
VoxelMap; admission waits for device memory and resumes when a stream
closes; a served result also matches the oracle."""
import numpy as np
import pytest

import synth
from parity import compare_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_01592_gb300 import vm
    vm.load()
    return vm


def _streams(n, frames):
    """n small config-4 streams (mixed resolutions) and their frames on the GPU."""
    out = []
    for st in synth.config4_streams(n_streams=n, seed=23):
        dims = tuple(min(d, int(round(2.4 / st.spec.voxel_size))) if a < 2 else d
                     for a, d in enumerate(st.spec.dims))
        st.spec = synth.MapSpec(dims, st.spec.origin, st.spec.voxel_size)
        sc = synth.config4_scene(st)
        fr = [synth.config4_frame(st, sc, f, device="cuda") for f in range(frames)]
        out.append((st, fr))
    return out


def _alone(vm, st, frames, params):
    m = vm.VoxelMap(st.spec.dims, st.spec.origin, st.spec.voxel_size)
    res = []
    for pts, pose in frames:
        m.integrate(pts, pose)
        res.append(m.segment(params))
    m.close()
    return res


def _collect(srv, n, timeout_s=120.0):
    """At least n results, or fail after timeout_s."""
    import time
    out, t_end = [], time.monotonic() + timeout_s
    while len(out) < n:
        assert time.monotonic() < t_end, f"{len(out)} of {n} results after {timeout_s} s"
        out += srv.poll(64, timeout_ms=500)
    return out


def _same(a, b):
    for key in ("planes", "hull_xy", "hull_xyz"):
        assert a[key].shape == b[key].shape, key
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("mode", ["batched", "streams"])
def test_each_result_is_the_same_alone_and_in_the_mix(vmmod, mode):
    from paper_2510_01592_gb300 import serve
    params = vmmod.segment_params(n_hyp=100, seed=3)
    data = _streams(5, 6)
    ref = {st.stream_id: _alone(vmmod, st, fr, params) for st, fr in data}
    srv = serve.Server(params, mode=mode, max_batch=4, max_inflight=2)
    sids = {st.stream_id: srv.open(st.spec.dims, st.spec.origin, st.spec.voxel_size) for st, _ in data}
    tickets = {}
    for f in range(6):  # interleaved, all queued at once: steps mix streams and frames
        for st, fr in data:
            tickets[srv.submit(sids[st.stream_id], fr[f][0], fr[f][1])] = (st.stream_id, f)
    srv.drain(120000)
    got = {}
    for r in _collect(srv, len(tickets)):
        assert r["status"] == vmmod.VM_OK, r
        got[r["ticket"]] = r
    for t, (sid, f) in tickets.items():
        _same(got[t], ref[sid][f])
    s = srv.stats()
    assert s["requests_done"] == len(tickets) and s["streams_admitted"] == len(data)
    if mode == "batched":
        assert s["mean_step_requests"] > 1.0  # several maps per batched fit
    srv.close()


def test_served_result_matches_the_oracle(orc, vmmod):
    from paper_2510_01592_gb300 import serve
    (st, fr), = _streams(1, 3)
    params = vmmod.segment_params(n_hyp=64, seed=9)
    srv = serve.Server(params, max_batch=2)
    sid = srv.open(st.spec.dims, st.spec.origin, st.spec.voxel_size)
    om = orc.OracleMap(st.spec.dims, st.spec.origin, st.spec.voxel_size)
    for pts, pose in fr:
        srv.submit(sid, pts, pose)
        om.integrate(pts.cpu().numpy(), pose)
    srv.drain(60000)
    res = _collect(srv, 3)
    last = max(res, key=lambda r: r["ticket"])
    compare_planes(last, om.segment(orc.make_params(n_hyp=64, seed=9)))
    srv.close()


def test_admission_waits_for_memory_and_resumes_on_close(vmmod):
    from paper_2510_01592_gb300 import serve
    params = vmmod.segment_params(n_hyp=32, seed=1)
    data = _streams(3, 2)
    fps = [serve.footprint(st.spec.dims, st.spec.origin, st.spec.voxel_size, params=params) for st, _ in data]
    budget = fps[0] + fps[1] + fps[2] // 2  # room for the first two streams, not all three
    assert fps[2] <= budget
    srv = serve.Server(params, hbm_budget=budget)
    ids = [srv.open(st.spec.dims, st.spec.origin, st.spec.voxel_size) for st, _ in data]
    for (st, fr), sid in zip(data, ids):
        for pts, pose in fr:
            srv.submit(sid, pts, pose)
    done = _collect(srv, 4)  # the two admitted streams finish
    assert {r["stream"] for r in done} == {ids[0], ids[1]}
    s = srv.stats()
    assert s["streams_waiting"] == 1 and s["hbm_committed"] <= budget
    assert srv.poll(16, timeout_ms=300) == []  # the third stream has not run
    srv.close_stream(ids[0])
    srv.close_stream(ids[1])
    rest = _collect(srv, 2)
    assert {r["stream"] for r in rest} == {ids[2]}
    assert all(r["status"] == vmmod.VM_OK for r in done + rest)
    srv.close()


def test_server_rejects_bad_requests(vmmod):
    from paper_2510_01592_gb300 import serve
    params = vmmod.segment_params()
    srv = serve.Server(params, hbm_budget=1 << 30)
    with pytest.raises(vmmod.VmError) as ei:
        srv.open((0, 10, 10), (0, 0, 0), 0.05)
    assert ei.value.status == vmmod.VM_ERR_INVALID_ARG
    with pytest.raises(vmmod.VmError) as ei:  # a 16 x 16 x 2 m map at 0.01 m cannot fit in 1 GiB
        srv.open((1600, 1600, 200), (0, 0, 0), 0.01)
    assert ei.value.status == vmmod.VM_ERR_OUT_OF_MEMORY
    with pytest.raises(vmmod.VmError):
        srv.submit(12345, np.zeros((4, 3), np.float32), np.eye(3, 4))
    srv.close()
