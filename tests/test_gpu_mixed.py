"""Mixed-precision V-cycle (FP32, FP32 with BF16 coarse operators) with FP64 outer CG.

The FP64 CG residual, dot products, search direction and coarsest solve keep the final
relative residual at rtol; the error against the (tightly solved) discrete solution of the
FP64 oracle is reported and bounded, and the V-cycle is compared with the oracle's FP64
V-cycle within the rounding of the working precision.
"""
import numpy as np
import pytest

from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import oracle_hierarchy, oracle_operator

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


CASES = [(I.pipe_workload(48, I.QUADRATIC), dict(max_coarse=300)),
         (I.pipe_workload(40, I.LINEAR), dict(max_coarse=200)),
         (I.taper_workload(36, 31, 52, I.QUADRATIC), dict(max_coarse=150)),
         (I.cylinder_workload(32, I.CONSTANT), dict(max_coarse=1000, max_levels=3))]


@pytest.mark.parametrize("prec", [1, 2], ids=["fp32", "bf16"])
@pytest.mark.parametrize("w,prm", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_mixed_solve_reaches_fp64_accuracy(S, w, prm, prec):
    import torch
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, **prm)
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=4)
    exact, _ = oh.solve(rho, rtol=1e-13)
    ref, oinfo = oh.solve(rho, rtol=1e-8, beta_rule=1)
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    h = S.setup(op, S.params_default(precision=prec, beta_rule=1, **prm))
    phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
    info = S.solve(h, torch.from_numpy(rho).cuda(), phi, rtol=1e-8)
    got = phi.cpu().numpy()
    assert info["converged"] == 1 and info["relres"] <= 1e-8
    # the FP64 outer recursion keeps the recomputed residual at the target
    assert info["relres_true"] <= 1.5e-8, info
    # a few more iterations than the FP64 preconditioner at most
    assert info["iters"] <= oinfo["iters"] + (2 if prec == 1 else 4), (info, oinfo)
    scale = np.max(np.abs(exact))
    err = np.max(np.abs(got - exact)) / scale
    err_ref = np.max(np.abs(ref - exact)) / scale
    assert err <= max(10 * err_ref, 1e-7), (err, err_ref)


@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (2, 5e-2)], ids=["fp32", "bf16"])
def test_mixed_vcycle_close_to_fp64(S, prec, tol):
    import torch
    w = I.pipe_workload(40, I.QUADRATIC)
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, max_coarse=150)
    h = S.setup(S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode),
                S.params_default(precision=prec, max_coarse=150))
    r = np.random.default_rng(3).standard_normal(o.n)
    z = torch.empty(o.n, dtype=torch.float64, device="cuda")
    S.vcycle(h, torch.from_numpy(r).cuda(), z)
    ref = oh.vcycle(r)
    rel = np.max(np.abs(z.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert rel < tol, rel
    if prec == 1:
        assert rel > 1e-12  # really computed in FP32
