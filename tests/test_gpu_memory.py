"""Device memory through the allocator hook and the library's block cache: results do not
depend on which allocator served a hierarchy, the cache survives switching allocators, and
repeated setups do not grow the memory held."""
import numpy as np
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
    saamg.use_torch_allocator()
    return saamg


def _solve(S, w, rho):
    import torch
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    h = S.setup(op, S.params_default(max_coarse=200))
    phi = torch.zeros_like(rho)
    info = S.solve(h, rho, phi, rtol=1e-10)
    h.free()
    op.free()
    return phi, info


def test_results_do_not_depend_on_the_allocator(S):
    import torch
    w = I.pipe_workload(48, I.LINEAR)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 3)).cuda()
    ref, iref = _solve(S, w, rho)
    try:
        S.use_cuda_malloc()
        a, ia = _solve(S, w, rho)
        b, ib = _solve(S, w, rho)
    finally:
        S.use_torch_allocator()
    c, ic = _solve(S, w, rho)
    assert iref["converged"] == 1
    for x, i in ((a, ia), (b, ib), (c, ic)):
        assert i["iters"] == iref["iters"] and torch.equal(x, ref)


def test_repeated_setups_do_not_grow_memory(S):
    import torch
    w = I.pipe_workload(64, I.QUADRATIC)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 4)).cuda()
    _solve(S, w, rho)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    phis = [_solve(S, w, rho)[0] for _ in range(12)]
    torch.cuda.synchronize()
    after = torch.cuda.memory_allocated()
    # the phis themselves plus at most the cache bound (1 GB) of blocks kept for reuse
    held = sum(p.numel() * 8 for p in phis)
    assert after - before <= held + (1 << 30)
    assert all(torch.equal(p, phis[0]) for p in phis)
