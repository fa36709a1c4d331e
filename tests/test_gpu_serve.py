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
    for rec in records:
        assert rec["queue"] >= 0 and rec["service"] > 0
        assert abs(rec["queue"] + rec["service"] - rec["latency"]) < 1e-9
    if tight:
        assert stats["evictions"] > 0
    else:
        assert stats["work_sets"] > 0 and stats["max_inflight_same_geometry"] > 1
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


def test_work_sets_solve_concurrently_and_equal_the_hierarchy(S):
    """Work sets share the hierarchy's levels and own their vectors: solves of different
    right-hand sides on the hierarchy and two work sets (one made from the other), in flight
    at the same time on three streams, each equal a solve on a fresh hierarchy bit for bit;
    the work sets keep working after the hierarchy itself is freed."""
    import torch
    w = I.pipe_workload(40, I.LINEAR)
    for prec in (S.PREC_FP64, S.PREC_FP32):
        params = S.params_default(max_coarse=200, precision=prec, beta_rule=1 if prec else 0)
        op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
        h = S.setup(op, params)
        w1 = S.hierarchy_work_set(h)
        w2 = S.hierarchy_work_set(w1)
        assert w1.info()["device_bytes"] < h.info()["device_bytes"]
        rhos = [I.gaussian_bunch_torch(w.grid, (w.centre[0], w.centre[1], w.centre[2] + 0.01 * k),
                                       w.sigma, 50 + k) for k in range(3)]
        solo = []
        ref_h = S.setup(op, params)
        for rho in rhos:
            phi = torch.zeros_like(rho)
            assert S.solve(ref_h, rho, phi)["converged"] == 1
            solo.append(phi)
        ref_h.free()
        streams = [torch.cuda.Stream() for _ in range(3)]
        phis = [torch.zeros_like(r) for r in rhos]
        torch.cuda.synchronize()
        for hd, rho, phi, st in zip((h, w1, w2), rhos, phis, streams):
            S.solve_async(hd, rho, phi, 1e-8, stream=st.cuda_stream)
        for hd in (h, w1, w2):
            assert S.solve_wait(hd)["converged"] == 1
        for a, b in zip(phis, solo):
            assert torch.equal(a, b)
        # the shared levels outlive the hierarchy's own handle
        h.free()
        torch.cuda.empty_cache()
        for hd in (w2, w1):
            phi = torch.zeros_like(rhos[0])
            S.solve(hd, rhos[0], phi)
            assert torch.equal(phi, solo[0])
        # batched solves across the work sets (merged and per-solve forms)
        for _ in range(2):
            outs = [torch.zeros_like(r) for r in rhos[:2]]
            S.solve_batched([w1, w2], rhos[:2], outs, 1e-8)
            for a, b in zip(outs, solo[:2]):
                assert torch.equal(a, b)
        S.release_batch_cache()
        w1.free()
        w2.free()
        op.free()


def test_work_set_degree_is_its_own(S):
    """saamg_set_cheb_degree on a work set leaves its hierarchy's smoother as it was."""
    import torch
    w = I.cylinder_workload(32, I.LINEAR)
    params = S.params_default(max_coarse=100)
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    h = S.setup(op, params)
    ws = S.hierarchy_work_set(h)
    rho = I.gaussian_bunch_torch(w.grid, w.centre, w.sigma, 3)
    a = torch.zeros_like(rho)
    ia = S.solve(h, rho, a)
    S.set_cheb_degree(ws, 4)
    b = torch.zeros_like(rho)
    S.solve(h, rho, b)
    assert torch.equal(a, b)
    c = torch.zeros_like(rho)
    ic = S.solve(ws, rho, c)
    assert ia["converged"] == 1 and ic["converged"] == 1 and not torch.equal(a, c)
    ws.free()
    h.free()
    op.free()
