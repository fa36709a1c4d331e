"""Gauss-Seidel coarse solver (Sec. 3.2, "Coarse level solver") on the GPU against the oracle:
V-cycle and solve parity with MIS-2 and cube hierarchies, a coarse level spanning many warps,
the device-loop graph, mixed precision."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import oracle_hierarchy, oracle_operator

pytestmark = pytest.mark.gpu

GS = O.Hierarchy.COARSE_GS


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


def gpu_op(S, w):
    return S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)


CASES = [(I.pipe_workload(40, I.LINEAR), dict(max_coarse=300)),
         (I.taper_workload(30, 26, 44, I.QUADRATIC), dict(max_coarse=200, aggregation=1)),
         # two levels: a coarse level of several thousand rows, many rows per colour and warp
         (I.pipe_workload(56, I.LINEAR), dict(max_coarse=4096, max_levels=2)),
         (I.cylinder_workload(32, I.CONSTANT), dict(max_coarse=1000, max_levels=3, coarse_sweeps=1))]


@pytest.mark.parametrize("w,prm", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_gs_vcycle_and_solve_match_oracle(S, w, prm):
    import torch
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, coarse_solver=GS, **prm)
    assert oh.colours() is not None
    rule = 1 if w.mode == I.QUADRATIC else 0
    h = S.setup(gpu_op(S, w), S.params_default(coarse_solver=1, beta_rule=rule, **prm))
    assert h.info()["n"] == [oh.n(l) for l in range(oh.levels)]
    r = np.random.default_rng(8).standard_normal(o.n)
    z = torch.empty(o.n, dtype=torch.float64, device="cuda")
    S.vcycle(h, torch.from_numpy(r).cuda(), z)
    ref = oh.vcycle(r)
    assert np.max(np.abs(z.cpu().numpy() - ref)) <= 1e-11 * np.max(np.abs(ref))
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, 9)
    phi_ref, oinfo = oh.solve(rho, rtol=1e-8, beta_rule=rule)
    phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
    info = S.solve(h, torch.from_numpy(rho).cuda(), phi, rtol=1e-8)
    assert info["converged"] == 1 and abs(info["iters"] - oinfo["iters"]) <= 1
    assert np.max(np.abs(phi.cpu().numpy() - phi_ref)) <= 1e-10 * np.max(np.abs(phi_ref))


def test_gs_device_loop_equals_host_loop_and_mixed_precision(S):
    import torch
    w = I.pipe_workload(40, I.LINEAR)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 2)).cuda()
    for prec in (0, 1):
        h = S.setup(gpu_op(S, w), S.params_default(coarse_solver=1, max_coarse=300, precision=prec,
                                                    beta_rule=1 if prec else 0))
        a = torch.zeros_like(rho)
        ia = S.solve(h, rho, a, rtol=1e-9)
        b = torch.zeros_like(rho)
        S.solve_async(h, rho, b, rtol=1e-9)
        ib = S.solve_wait(h)
        assert ia["iters"] == ib["iters"] and torch.equal(a, b)
        assert ia["converged"] == 1 and ia["relres_true"] <= 1.5e-9


def test_gs_bad_parameters_are_rejected(S):
    w = I.pipe_workload(16, I.LINEAR)
    for bad in (dict(coarse_solver=5), dict(coarse_solver=1, coarse_sweeps=0)):
        with pytest.raises(S.SaamgError):
            S.setup(gpu_op(S, w), S.params_default(**bad))
