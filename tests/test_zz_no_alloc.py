"""The allocation-free tree ordering (hpfmm_tree_order_noalloc).

Some callers cannot let a library allocate device memory: host runtimes
that own every device allocation themselves, or processes that must not
grow their device memory use after start-up.  For them the library offers
one entry point whose temporaries live in a static device array instead of
memory from cudaMalloc.  This test calls it through the C ABI and checks, on
two calls in a row (the array keeps the previous call's contents), that it
returns exactly the ordering of the allocating path (hpfmm_create +
hpfmm_get_order), including leaves far larger than the shared-memory sort,
and that the calls leave the device's free memory unchanged.  It sits in a
file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402


def _noalloc(xd, yd, levels, keys=None, perm=None):
    n = xd.numel()
    if keys is None:
        keys = torch.empty(n, dtype=torch.int64, device=xd.device)
        perm = torch.empty(n, dtype=torch.int64, device=xd.device)
    st = torch.cuda.current_stream(xd.device).cuda_stream
    rc = hp.lib().hpfmm_tree_order_noalloc(
        ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), n, levels,
        ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
        ctypes.c_void_p(st))
    return rc, keys, perm


def test_noalloc_order_matches_allocating_path_twice():
    dev = torch.device("cuda:0")
    # levels 6 and 3: leaves of ~16 and ~64 points (warp sorts); levels 1 on
    # 65536 points: four leaves of ~16k points (the in-place global sort)
    cases = [(workloads.uniform(65536, seed=31), 6), (workloads.uniform(4097, seed=32), 3),
             (workloads.uniform(65536, seed=34), 1)]
    for (x, y, _), levels in cases:
        xd = torch.tensor(x, device=dev)
        yd = torch.tensor(y, device=dev)
        plan = hp.hpfmm_create(xd, yd, kappa=1.0, p=4, leaf_size=32)
        keys_ref, perm_ref = hp.hpfmm_get_order(plan)
        for _ in range(2):  # the second call sees the first call's leftovers
            rc, keys, perm = _noalloc(xd, yd, levels)
            assert rc == hp.HPFMM_OK, hp.lib().hpfmm_last_error()
            assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_ref)
            assert np.array_equal(perm.cpu().numpy(), perm_ref)


def test_noalloc_leaves_device_memory_unchanged():
    dev = torch.device("cuda:0")
    x, y, _ = workloads.uniform(65536, seed=35)
    xd = torch.tensor(x, device=dev)
    yd = torch.tensor(y, device=dev)
    keys = torch.empty(65536, dtype=torch.int64, device=dev)
    perm = torch.empty(65536, dtype=torch.int64, device=dev)
    rc, _, _ = _noalloc(xd, yd, 5, keys, perm)  # first call: module and symbol set-up
    assert rc == hp.HPFMM_OK, hp.lib().hpfmm_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for levels in (5, 1):
        rc, _, _ = _noalloc(xd, yd, levels, keys, perm)
        assert rc == hp.HPFMM_OK, hp.lib().hpfmm_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_maximum():
    dev = torch.device("cuda:0")
    x, y, _ = workloads.uniform(65537, seed=33)
    rc, _, _ = _noalloc(torch.tensor(x, device=dev), torch.tensor(y, device=dev), 4)
    assert rc == hp.HPFMM_EINVAL
    assert b"65536" in hp.lib().hpfmm_last_error()
