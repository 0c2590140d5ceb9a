"""vm_ransac_static: the RANSAC entry point that allocates nothing.

Some callers cannot allocate device memory while running (a control loop with
a deadline, or a program whose device memory is owned by another allocator);
vm_ransac_static serves them from scratch compiled into the library.  This
test calls it through the C ABI, twice in a row on different batches, and
checks each result against vm_fit_planes and against the CPU oracle on the
same clusters: selected hypothesis, plane and inlier count must be equal bit
for bit (the tolerance the parity tests use for RANSAC).  A first call with
no clusters does the per-device set-up.  The file sorts last so a stop-at-first-
failure run has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _static_fn(L):
    f = L.vm_ransac_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p]
    return f


def _batch(seed, n_clusters, hi):
    xyz, off, _ = synth.config3_clusters(n_clusters=n_clusters, seed=seed, size_hi=hi)
    return xyz, off


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2510_01592_gb300 import vm
    return vm, vm.load()


def test_static_ransac_matches_fit_planes_twice(lib, orc):
    import torch
    vm, L = lib
    fn = _static_fn(L)
    # the set-up call: k == 0 loads the array and looks up its address
    prm0 = vm.segment_params(n_hyp=16)
    assert fn(None, None, None, 0, C.addressof(prm0), None, None, None, None) == vm.VM_OK
    for call, (seed, k, hi, H, key) in enumerate([(21, 300, 30000, 256, 7), (22, 57, 5000, 100, 99)]):
        xyz, off = _batch(seed, k, hi)
        labels = (np.arange(k, dtype=np.uint32) * 3 + call).astype(np.uint32)
        d_xyz = torch.from_numpy(xyz).cuda()
        d_off = torch.from_numpy(off).cuda()
        d_lab = torch.from_numpy(labels).cuda()
        prm = vm.segment_params(n_hyp=H, seed=key)
        ref = vm.fit_planes(d_xyz, d_off, prm, labels=d_lab)["planes"]
        planes = torch.empty((k, 4), dtype=torch.float32, device="cuda")
        best = torch.empty(k, dtype=torch.int32, device="cuda")
        inl = torch.empty(k, dtype=torch.uint32, device="cuda")
        st = fn(d_xyz.data_ptr(), d_off.data_ptr(), d_lab.data_ptr(), k, C.addressof(prm), None,
                planes.data_ptr(), best.data_ptr(), inl.data_ptr())
        assert st == vm.VM_OK, L.vm_last_error()
        torch.cuda.synchronize()
        planes, best, inl = planes.cpu().numpy(), best.cpu().numpy(), inl.cpu().numpy()
        assert np.array_equal(best, ref["best_h"])
        ok = best >= 0
        assert ok.sum() == k
        assert np.array_equal(planes[ok, :3].view(np.uint32), ref["ransac_normal"][ok].view(np.uint32))
        assert np.array_equal(planes[ok, 3].view(np.uint32), ref["ransac_offset"][ok].view(np.uint32))
        assert np.array_equal(inl[ok], ref["inlier_count"][ok])
        # and directly against the oracle's stages a-c on the same clusters
        o = orc.fit_planes(xyz, off, orc.make_params(n_hyp=H, seed=key), labels=labels)["planes"]
        assert np.array_equal(best, o["best_h"])
        assert np.array_equal(planes[ok, :3].view(np.uint32), o["ransac_n"][ok].view(np.uint32))
        assert np.array_equal(planes[ok, 3].view(np.uint32), o["ransac_d"][ok].view(np.uint32))
        assert np.array_equal(inl[ok], o["inlier_count"][ok])


def test_static_ransac_rejects_oversize_requests(lib):
    vm, L = lib
    fn = _static_fn(L)
    prm = vm.segment_params(n_hyp=1024)
    dummy = C.c_void_p(1)  # never dereferenced: the size check comes first
    st = fn(dummy, dummy, None, 1000, C.addressof(prm), None, dummy, dummy, dummy)
    assert st == vm.VM_ERR_CAPACITY
    assert b"static scratch" in L.vm_last_error()
    st = fn(dummy, dummy, None, 5000, C.addressof(vm.segment_params(n_hyp=16)), None, dummy, dummy, dummy)
    assert st == vm.VM_ERR_CAPACITY
