"""Allocator failures during build, setup and solve.

The library takes device memory only from the installed allocator hook.  A hook that runs
dry at its k-th request (and refuses everything after) must make the call in progress fail
with ENOMEM and a message, for every k across a whole build + setup + solve, without a crash
and without keeping a block: once the handles that were created are freed and the library's
block cache is handed back, every block the hook gave out has been returned.  A single
refused request is absorbed: the library returns its cached blocks to the hook and asks once
more, so the call succeeds with the same result.
"""
import ctypes as C

import pytest

from paper_0907_4863_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    from paper_0907_4863_gb300 import build
    build.build()
    from paper_0907_4863_gb300 import saamg
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return saamg


class FailingHook:
    """Counts requests; refuses request number `fail_at` (1-based) and, if `dry`, every later
    one.  Blocks come from torch's caching allocator; live blocks are tracked."""

    def __init__(self, S, fail_at, dry=True):
        import torch
        self.calls = 0
        self.fail_at = fail_at
        self.dry = dry
        self.live = {}
        self.refused = 0

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at or (self.dry and self.calls > self.fail_at > 0):
                self.refused += 1
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                   stream or 0)
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, stream, ctx):
            assert ptr in self.live, "freed a block the hook never gave out"
            del self.live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

        self.fns = (S.ALLOC_FN(_alloc), S.FREE_FN(_free))
        S._all_hooks.append(self.fns)  # callbacks stay referenced for the life of the process

    def install(self, S):
        S._hooks = None
        assert S.lib().saamg_set_allocator(self.fns[0], self.fns[1], None) == S.OK


def _run(S, w, rho):
    """build + setup + solve; returns (status, the solution or None, handles to free)."""
    import torch
    handles = []
    try:
        op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
        handles.append(op)
        h = S.setup(op, S.params_default(max_coarse=60))
        handles.append(h)
        phi = torch.zeros_like(rho)
        S.solve(h, rho, phi)
        torch.cuda.synchronize()
        return S.OK, phi, handles
    except S.SaamgError as e:
        torch.cuda.synchronize()
        return e.status, None, handles


def _release(S, hook, handles):
    for hd in reversed(handles):
        hd.free()
    # hand the block cache back (to the hook each block came from)
    assert S.lib().saamg_set_allocator(S.ALLOC_FN(), S.FREE_FN(), None) == S.OK
    assert hook.live == {}, f"{len(hook.live)} blocks never returned"


def test_every_allocation_failure_is_reported_and_nothing_leaks(S):
    import torch
    w = I.pipe_workload(24, I.LINEAR)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 3)).cuda()
    counter = FailingHook(S, fail_at=0)
    counter.install(S)
    st, ref, handles = _run(S, w, rho)
    assert st == S.OK
    _release(S, counter, handles)
    total = counter.calls
    assert total > 10
    for k in range(1, total + 1):
        hook = FailingHook(S, fail_at=k, dry=True)
        hook.install(S)
        st, phi, handles = _run(S, w, rho)
        assert st == S.ENOMEM, (k, st)
        assert S.last_error() != ""
        assert hook.refused >= 1
        _release(S, hook, handles)
    S.use_torch_allocator()


def test_single_refusal_is_absorbed(S):
    """One refused request anywhere: the library hands its cached blocks back, asks again and
    completes the call; the solution is the same bits as without the refusal."""
    import torch
    w = I.pipe_workload(24, I.LINEAR)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 3)).cuda()
    counter = FailingHook(S, fail_at=0)
    counter.install(S)
    st, ref, handles = _run(S, w, rho)
    _release(S, counter, handles)
    for k in range(1, counter.calls + 1, 3):
        hook = FailingHook(S, fail_at=k, dry=False)
        hook.install(S)
        st, phi, handles = _run(S, w, rho)
        assert st == S.OK, (k, st, S.last_error())
        assert torch.equal(phi, ref)
        _release(S, hook, handles)
    S.use_torch_allocator()
