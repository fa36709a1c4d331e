"""Continuous-batching server: each result is the same alone and in the mix."""
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


def _small_world():
    geoms = I.serving_geometries(6, seed=11, sizes=(16, 20, 24, 32, 40))
    reqs = I.serving_requests(90, mean_gap_s=0.0003, ngeom=6, seed=5)
    return geoms, reqs


def _alone(S, w, req, params):
    import torch
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    h = S.setup(op, params)
    c = (w.centre[0], w.centre[1], w.centre[2] + 0.005 * req.step)
    rho = I.gaussian_bunch_torch(w.grid, c, w.sigma, req.seed)
    phi = torch.zeros_like(rho)
    info = S.solve(h, rho, phi)
    return phi, info


@pytest.mark.parametrize("tight", [False, True], ids=["roomy", "tight_budget_evicts"])
def test_served_results_equal_solo_results(S, tight):
    import torch
    from paper_0907_4863_gb300 import serve
    geoms, reqs = _small_world()
    params = S.params_default(max_coarse=64, precision=S.PREC_FP32, beta_rule=1)
    hints = None
    budget = 4 << 30
    if tight:
        # measure every hierarchy once, then leave room for about one of the largest
        probe = serve.Server(geoms, slots=8, params=params)
        probe.run(reqs)
        probe.close()
        hints = dict(probe.sizes)
        big = max(w.grid.nbox for w in geoms)
        budget = int(1.3 * max(hints.values())) + 8 * 2 * big * 8
    srv = serve.Server(geoms, budget_bytes=budget, slots=8, params=params, keep_results=True,
                       size_hints=hints)
    records, stats = srv.run(reqs)
    assert stats["requests"] == len(reqs) and stats["rejected"] == 0 and stats["all_converged"]
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["peak_bytes"] <= budget
    if tight:
        assert stats["evictions"] > 0
    torch.cuda.synchronize()
    for r in reqs[::7]:
        phi_alone, info = _alone(S, geoms[r.geometry], r, params)
        assert info["converged"] == 1
        assert torch.equal(srv.results[r.rid], phi_alone), r
    srv.close()


def test_warm_start_reduces_iterations(S):
    from paper_0907_4863_gb300 import serve
    geoms, reqs = _small_world()
    params = S.params_default(max_coarse=64, precision=S.PREC_FP32, beta_rule=1)
    cold = serve.Server(geoms, slots=8, params=params)
    rc, _ = cold.run(reqs)
    warm = serve.Server(geoms, slots=8, params=params, warm_start=True)
    rw, _ = warm.run(reqs)
    assert np.mean([r["iters"] for r in rw]) < np.mean([r["iters"] for r in rc])
    cold.close()
    warm.close()


def test_requests_that_cannot_fit_are_rejected(S):
    from paper_0907_4863_gb300 import serve
    geoms, reqs = _small_world()
    params = S.params_default(max_coarse=64, precision=S.PREC_FP32, beta_rule=1)
    srv = serve.Server(geoms, budget_bytes=64 << 10, slots=4, params=params)
    records, stats = srv.run(reqs[:10])
    assert stats["rejected"] == 10 and stats["requests"] == 0
    srv.close()
