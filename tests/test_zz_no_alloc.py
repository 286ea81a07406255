"""The allocation-free full scan against the allocating entry point.

Callers that cannot allocate device memory while running (allocation
forbidden after start-up, or device memory held by another allocator) use
mc_capforest_full_noalloc, whose scratch is a static device array.  Its
results must equal those of mc_step_capforest_full, which runs the same
kernel on scratch it allocated: labels and counts are integers, so the
comparison is exact, and it is repeated on two calls in a row because the
static array keeps the previous call's contents.
"""
import ctypes

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu


def _device_inputs(torch, G):
    rp, col, w = G.export()
    adj = np.stack([col, w], axis=1).reshape(-1).astype(np.int32)
    return torch.from_numpy(rp).cuda(), torch.from_numpy(adj).cuda()


@pytest.mark.parametrize("which", ["tiny", "planted", "rhg", "weighted"])
def test_noalloc_matches_allocating_scan_twice(which):
    import torch
    import paper_1808_05458_gb300 as mc
    from paper_1808_05458_gb300 import mincut

    torch.cuda.set_device(0)
    mc.load_library()
    if which == "tiny":
        g = graphgen.random_connected(9, 14, seed=3, wmax=5)
    elif which == "planted":
        g = graphgen.planted(2)
    elif which == "rhg":
        g = graphgen.rhg(4, 1 << 13, 20.0)
    else:
        g = graphgen.random_connected(3000, 20000, seed=8, wmax=100)
    with mc.Graph(*g) as G:
        d_rp, d_adj = _device_inputs(torch, G)
        lam = int(G.degrees().min())
        n = G.n
        for start in (0, n // 2):
            ref_lab, ref_lam, ref_un = G.capforest_full(lam, start)
            labels = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            before = torch.cuda.memory_allocated()
            # the library's next device allocation would fail: the calls
            # below must not make one
            mc.test_fail_alloc_after(0)
            try:
                got = [mincut.capforest_full_noalloc(d_rp, d_adj, lam, start, labels)
                       + (labels.cpu().numpy(),) for _ in range(2)]
            finally:
                mc.test_fail_alloc_after(-1)
            assert torch.cuda.memory_allocated() == before
            for lo, un, lab in got:
                assert lo == ref_lam and un == ref_un
                assert (lab == ref_lab).all()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    from paper_1808_05458_gb300 import mincut

    lib = mincut.load_library()
    rp = torch.zeros(8, dtype=torch.int32, device="cuda")
    adj = torch.zeros(2, dtype=torch.int32, device="cuda")
    lab = torch.zeros(8, dtype=torch.int32, device="cuda")
    lo, un = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.mc_capforest_full_noalloc(mincut.NOALLOC_MAX_N + 1, 1, ctypes.c_void_p(rp.data_ptr()),
                                       ctypes.c_void_p(adj.data_ptr()), 1, 0,
                                       ctypes.c_void_p(lab.data_ptr()), ctypes.byref(lo),
                                       ctypes.byref(un), None)
    assert rc == mincut.MC_EINVAL
    rc = lib.mc_capforest_full_noalloc(4, mincut.NOALLOC_MAX_ARCS + 1, ctypes.c_void_p(rp.data_ptr()),
                                       ctypes.c_void_p(adj.data_ptr()), 1, 0,
                                       ctypes.c_void_p(lab.data_ptr()), ctypes.byref(lo),
                                       ctypes.byref(un), None)
    assert rc == mincut.MC_EINVAL


def test_noalloc_rejects_malformed_arrays():
    # bad offsets or arcs are caught on the device before the scan indexes
    # anything with them, and the next good call still works
    import torch
    from paper_1808_05458_gb300 import mincut

    g = graphgen.cycle(12, 3)
    rp = torch.from_numpy(g[0]).cuda()
    adj = torch.from_numpy(np.stack([g[1], g[2]], axis=1).reshape(-1).astype(np.int32)).cuda()
    lab = torch.zeros(12, dtype=torch.int32, device="cuda")
    bad_cases = []
    a = adj.clone(); a[6] = 12            # neighbour out of range
    bad_cases.append((rp, a))
    a = adj.clone(); a[6] = -1            # negative neighbour
    bad_cases.append((rp, a))
    a = adj.clone(); a[7] = 0             # weight below 1
    bad_cases.append((rp, a))
    a = adj.clone(); a[0] = 0             # self-loop in row 0
    bad_cases.append((rp, a))
    r = rp.clone(); r[5] = 30             # offsets not monotone
    bad_cases.append((r, adj))
    r = rp.clone(); r[0] = 1              # row_ptr[0] != 0
    bad_cases.append((r, adj))
    for d_rp, d_adj in bad_cases:
        with pytest.raises(mincut.MinCutError) as ei:
            mincut.capforest_full_noalloc(d_rp, d_adj, 6, 0, lab)
        assert ei.value.code == mincut.MC_EINVAL
    lo, un = mincut.capforest_full_noalloc(rp, adj, 6, 0, lab)
    assert lo == 6 and un >= 1
