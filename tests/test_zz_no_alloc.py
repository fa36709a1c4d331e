"""The allocation-free aggregation entry point gives what the regular one gives.

saamg_mis2_aggregate_noalloc serves callers that cannot allocate device memory during
the call (a fixed memory pool, a callback that must not re-enter the allocator): it works
in a static scratch array owned by the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sps

pytestmark = pytest.mark.gpu

MAX_NODES = 1 << 18


@pytest.fixture(scope="module")
def S():
    import torch
    from paper_0907_4863_gb300 import build
    build.build()
    from paper_0907_4863_gb300 import saamg
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return saamg


def _graph(n, deg, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, n, n * deg // 2)
    cols = rng.integers(0, n, n * deg // 2)
    A = sps.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n)).tocsr()
    A = (A + A.T + sps.eye(n)).tocsr()
    A.sort_indices()
    ids = rng.permutation(4 * n)[:n].astype(np.uint32)
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), ids


def _run(S, fn, rp, cc, ids, seed):
    import torch
    n = len(rp) - 1
    rp_d = torch.from_numpy(rp).cuda()
    cc_d = torch.from_numpy(cc).cuda()
    ids_d = torch.from_numpy(ids.view(np.int32)).cuda()
    root = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    agg = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    nagg = C.c_int(-1)
    st = fn(n, C.c_void_p(rp_d.data_ptr()), C.c_void_p(cc_d.data_ptr()), C.c_void_p(ids_d.data_ptr()),
            seed, C.c_void_p(root.data_ptr()), C.c_void_p(agg.data_ptr()), C.byref(nagg),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == S.OK, S.last_error()
    return nagg.value, root.cpu().numpy(), agg.cpu().numpy()


def test_noalloc_matches_regular_on_two_calls_in_a_row(S):
    L = S.lib()
    # a larger graph first, then a smaller one: the second call must not see leftovers
    for n, deg, seed in ((200_000, 7, 1), (37_000, 12, 2)):
        rp, cc, ids = _graph(n, deg, seed)
        want = _run(S, L.saamg_mis2_aggregate, rp, cc, ids, 0x1234567 + seed)
        got = _run(S, L.saamg_mis2_aggregate_noalloc, rp, cc, ids, 0x1234567 + seed)
        assert got[0] == want[0] and got[0] > 0
        assert np.array_equal(got[1], want[1])
        assert np.array_equal(got[2], want[2])


def test_noalloc_rejects_graphs_over_the_limit(S):
    import torch
    L = S.lib()
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    nagg = C.c_int(-1)
    p = C.c_void_p(small.data_ptr())
    st = L.saamg_mis2_aggregate_noalloc(MAX_NODES + 1, p, p, None, 0, p, p, C.byref(nagg), None)
    assert st == S.EINVAL and nagg.value == 0
    assert "262144" in S.last_error()


def test_noalloc_calls_no_allocator(S):
    """The point of the entry point: with an allocator hook that refuses every request and
    counts the requests, the allocation-free call still succeeds and the hook is never
    called, while the regular entry point asks the hook and fails with ENOMEM."""
    L = S.lib()
    rp, cc, ids = _graph(60_000, 8, 3)
    # warm-up call: loads the library's device code and the scratch on this device
    want = _run(S, L.saamg_mis2_aggregate_noalloc, rp, cc, ids, 0x51)
    counts = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        counts["alloc"] += 1
        return None

    def _free(ptr, stream, ctx):
        counts["free"] += 1

    hooks = (S.ALLOC_FN(_alloc), S.FREE_FN(_free))
    saved = S._hooks
    assert L.saamg_set_allocator(hooks[0], hooks[1], None) == S.OK
    try:
        got = _run(S, L.saamg_mis2_aggregate_noalloc, rp, cc, ids, 0x51)
        assert counts == {"alloc": 0, "free": 0}
        assert got[0] == want[0] and np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])
        # control: the regular entry point does allocate, so the refusing hook makes it fail
        import torch
        n = len(rp) - 1
        rp_d, cc_d = torch.from_numpy(rp).cuda(), torch.from_numpy(cc).cuda()
        root = torch.zeros(n, dtype=torch.uint8, device="cuda")
        agg = torch.zeros(n, dtype=torch.int32, device="cuda")
        nagg = C.c_int(-1)
        st = L.saamg_mis2_aggregate(n, C.c_void_p(rp_d.data_ptr()), C.c_void_p(cc_d.data_ptr()),
                                    None, 0x51, C.c_void_p(root.data_ptr()),
                                    C.c_void_p(agg.data_ptr()), C.byref(nagg),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == S.ENOMEM and counts["alloc"] > 0
        torch.cuda.synchronize()
    finally:
        if saved is not None:
            L.saamg_set_allocator(saved[0], saved[1], None)
        else:
            L.saamg_set_allocator(S.ALLOC_FN(), S.FREE_FN(), None)
