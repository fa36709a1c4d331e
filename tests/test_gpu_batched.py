"""Device-loop (graph) solves, batched solves and the Chebyshev-degree autotuner."""
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


def _setup(S, w, **prm):
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    return S.setup(op, S.params_default(**prm))


def _rho(w, seed):
    import torch
    return torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, seed)).cuda()


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("w", [I.pipe_workload(40, I.LINEAR), I.taper_workload(30, 27, 45, I.QUADRATIC)],
                         ids=lambda w: w.name)
def test_device_loop_equals_host_loop(S, w, prec):
    import torch
    # the synchronous call on the host-driven loop, the asynchronous one on the device loop
    prm = dict(max_coarse=100, precision=prec, beta_rule=1 if prec else 0, device_loop=0)
    h = _setup(S, w, **prm)
    rho = _rho(w, 1)
    a = torch.zeros_like(rho)
    ia = S.solve(h, rho, a)
    b = torch.full_like(rho, 0.0)
    S.solve_async(h, rho, b)
    ib = S.solve_wait(h)
    assert ib["status"] == 0 and ib["iters"] == ia["iters"]
    assert ib["relres"] == pytest.approx(ia["relres"], rel=0, abs=0)
    assert ib["relres_true"] == pytest.approx(ia["relres_true"], rel=1e-12)
    assert torch.equal(a, b)
    # again, the captured graph is reused
    c = torch.zeros_like(rho)
    S.solve_async(h, rho, c)
    while not S.solve_test(h):
        pass
    assert S.solve_wait(h)["iters"] == ia["iters"] and torch.equal(a, c)


def test_device_loop_edge_cases(S):
    import torch
    w = I.pipe_workload(24, I.LINEAR)
    h = _setup(S, w, max_coarse=100)
    phi = torch.full((w.grid.nbox,), 2.0, dtype=torch.float64, device="cuda")
    S.solve_async(h, torch.zeros_like(phi), phi)
    info = S.solve_wait(h)
    assert info["status"] == 0 and info["iters"] == 0 and torch.all(phi == 0)
    rho = _rho(w, 0)
    bad = rho.clone()
    m = w.grid.n[0] // 2
    bad[m + w.grid.n[0] * (m + w.grid.n[1] * m)] = float("nan")
    S.solve_async(h, bad, torch.zeros_like(rho))
    with pytest.raises(S.SaamgError) as e:
        S.solve_wait(h)
    assert e.value.status == S.NUMERICAL
    h2 = _setup(S, w, max_coarse=100, maxit=3)
    S.solve_async(h2, rho, torch.zeros_like(rho))
    info = S.solve_wait(h2)
    assert info["status"] == S.NOT_CONVERGED and info["iters"] == 3
    # warm start through the device loop
    x = torch.zeros_like(rho)
    S.solve_async(h, rho, x)
    cold = S.solve_wait(h)["iters"]
    S.solve_async(h, rho, x)
    assert S.solve_wait(h)["iters"] == 0


def test_batched_results_equal_solo_results(S):
    """Uneven instances (sizes, geometries, modes, precisions) and several rhs per instance:
    every result in the batch equals the same solve run alone, bit for bit."""
    import torch
    ws = [(I.pipe_workload(36, I.LINEAR), dict(max_coarse=150)),
          (I.Workload("cyl48x40x64", I.cell_centred_grid(48, 40, 64), I.Domain(0.45, 0.45), I.CONSTANT),
           dict(max_coarse=200, precision=1, beta_rule=1)),
          (I.taper_workload(28, 33, 52, I.QUADRATIC), dict(max_coarse=100, precision=2, beta_rule=1)),
          (I.pipe_workload(20, I.QUADRATIC), dict(max_coarse=50))]
    hs, rhos, phis, solo = [], [], [], []
    for w, prm in ws:
        h = _setup(S, w, **prm)
        for seed in range(3):
            rho = _rho(w, seed)
            phi = torch.zeros_like(rho)
            S.solve(h, rho, phi)
            solo.append(phi)
            hs.append(h)
            rhos.append(rho)
            phis.append(torch.full_like(rho, 7.0) * 0.0)
    infos = S.solve_batched(hs, rhos, phis, rtol=1e-8)
    assert all(i["converged"] == 1 for i in infos)
    for a, b in zip(solo, phis):
        assert torch.equal(a, b)


def test_batched_graph_is_reused_and_rebuilt(S):
    """A repeated batch (same hierarchies, arrays and tolerance) is one launch of the cached
    graph and must see the arrays' new contents; a hierarchy changed since (a new Chebyshev
    degree) or another tolerance gets a new graph.  Every result equals the solo solve."""
    import torch
    wa, wb = I.pipe_workload(32, I.LINEAR), I.taper_workload(26, 24, 40, I.QUADRATIC)
    ha = _setup(S, wa, max_coarse=100)
    hb = _setup(S, wb, max_coarse=100, precision=1, beta_rule=1)
    hs = [ha, hb, ha]
    rhos = [_rho(wa, 1), _rho(wb, 2), _rho(wa, 3)]
    phis = [torch.zeros_like(r) for r in rhos]

    def check(rtol):
        for x in phis:
            x.zero_()
        infos = S.solve_batched(hs, rhos, phis, rtol=rtol)
        for h, r, x, info in zip(hs, rhos, phis, infos):
            ref = torch.zeros_like(r)
            solo = S.solve(h, r, ref, rtol=rtol)
            assert info["converged"] == 1 and info["iters"] == solo["iters"]
            assert torch.equal(x, ref)
        return infos

    first = check(1e-8)
    for r in rhos:
        r.mul_(-0.5).add_(1e-3)  # same arrays, new contents
    check(1e-8)
    S.set_cheb_degree(ha, 3)
    check(1e-8)
    loose = check(1e-4)
    assert all(a["iters"] < b["iters"] for a, b in zip(loose, first))


def test_batched_with_a_domain_without_unknowns(S):
    """A pipe thinner than the lattice spacing has no unknowns: its solve in a batch is
    phi = 0 at once, the other solves are untouched."""
    import torch
    w0 = I.Workload("empty", I.cell_centred_grid(16), I.Domain(1e-3, 1e-3), I.LINEAR)
    w1 = I.pipe_workload(24, I.LINEAR)
    h0 = _setup(S, w0, max_coarse=100)
    assert h0.info()["n"][0] == 0
    h1 = _setup(S, w1, max_coarse=100)
    r0, r1 = _rho(w0, 0), _rho(w1, 0)
    x0 = torch.full_like(r0, 5.0)
    x1 = torch.zeros_like(r1)
    infos = S.solve_batched([h0, h1], [r0, r1], [x0, x1])
    assert infos[0]["converged"] == 1 and infos[0]["iters"] == 0 and torch.all(x0 == 0)
    ref = torch.zeros_like(r1)
    assert infos[1]["iters"] == S.solve(h1, r1, ref)["iters"] and torch.equal(x1, ref)


def test_autotune_picks_a_degree_and_keeps_accuracy(S):
    import torch
    w = I.pipe_workload(48, I.LINEAR)
    h = _setup(S, w, max_coarse=200, precision=1, beta_rule=1)
    rho = _rho(w, 2)
    best, ms = S.autotune_cheb_degree(h, rho, 2, 4)
    assert 2 <= best <= 4 and ms > 0
    phi = torch.zeros_like(rho)
    info = S.solve(h, rho, phi)
    assert info["converged"] == 1 and info["relres_true"] <= 1.5e-8
    S.set_cheb_degree(h, 3)
    info3 = S.solve(h, rho, torch.zeros_like(rho))
    assert info3["converged"] == 1
    with pytest.raises(S.SaamgError):
        S.set_cheb_degree(h, 0)


def test_batched_engine_mixed_batch_equals_solo(S):
    """One launch per operation across the whole batch: hierarchies of different depth,
    Chebyshev degree (2, 3, 4), precision (FP64, FP32, BF16 storage), aggregation (MIS-2,
    cubes), extrapolation and beta rule, several right-hand sides per hierarchy (solved side
    by side with their own work vectors), one hierarchy of a single level.  Every result, its
    iteration count and its residuals equal the solo solve's; a second run reuses the graph."""
    import torch
    c4 = sorted(I.batched_instances(), key=lambda w: w.grid.nbox)
    specs = [(c4[0], dict(max_coarse=300, precision=1, beta_rule=1), 2),
             (c4[1], dict(max_coarse=300, precision=1, beta_rule=1), 4),
             (c4[2], dict(max_coarse=300, precision=2, beta_rule=1), 3),
             (I.taper_workload(30, 27, 45, I.QUADRATIC), dict(max_coarse=100, precision=1, beta_rule=0), 2),
             (I.pipe_workload(36, I.LINEAR), dict(max_coarse=150), 2),
             (I.pipe_workload(28, I.QUADRATIC), dict(max_coarse=100, beta_rule=1), 3),
             (I.cylinder_workload(30, I.CONSTANT), dict(max_coarse=200, aggregation=1, precision=1, beta_rule=1), 2),
             (I.pipe_workload(12, I.LINEAR), dict(max_coarse=5000), 2)]
    hs, rhos, solo, solo_info = [], [], [], []
    for k, (w, prm, deg) in enumerate(specs):
        h = _setup(S, w, **prm)
        if deg != 2:
            S.set_cheb_degree(h, deg)
        for seed in range(2 if k % 2 else 3):
            rho = _rho(w, 10 * k + seed)
            phi = torch.zeros_like(rho)
            solo_info.append(S.solve(h, rho, phi))
            solo.append(phi)
            hs.append(h)
            rhos.append(rho)
    assert hs[-1].info()["levels"] == 1
    phis = [torch.zeros_like(r) for r in rhos]
    forms = []
    for rep in range(3):  # merged form, per-solve form, then the faster one
        for x in phis:
            x.zero_()
        infos = S.solve_batched(hs, rhos, phis, rtol=1e-8)
        forms.append(S.batch_last())
        for a, b, ia, ib in zip(solo, phis, solo_info, infos):
            assert ib["converged"] == 1 and ib["iters"] == ia["iters"]
            assert ib["relres"] == ia["relres"] and ib["relres_true"] == ia["relres_true"]
            assert torch.equal(a, b)
    assert [f["form"] for f in forms[:2]] == ["merged", "per-solve"]
    faster = "merged" if forms[1]["ms_merged"] <= forms[1]["ms_per_solve"] else "per-solve"
    assert forms[2]["form"] == faster


def test_batched_engine_warm_start_and_limits(S):
    """Warm starts (phi holds the initial guess), a zero right-hand side, and an iteration
    limit reached by one solve of the batch while the others converge."""
    import torch
    w = I.pipe_workload(32, I.LINEAR)
    h = _setup(S, w, max_coarse=100, precision=1, beta_rule=1)
    h3 = _setup(S, w, max_coarse=100, maxit=3)
    rho = _rho(w, 4)
    x0 = torch.zeros_like(rho)
    S.solve(h, rho, x0, rtol=1e-4)  # a warm start
    cases = [(h, rho, x0.clone()), (h, torch.zeros_like(rho), torch.full_like(rho, 2.0)),
             (h3, rho, torch.zeros_like(rho)), (h, _rho(w, 5), torch.zeros_like(rho))]
    solo = []
    for hh, r, x in cases:
        y = x.clone()
        try:
            info = S.solve(hh, r, y)
        except S.SaamgError:
            raise
        solo.append((y, info))
    phis = [x.clone() for _, _, x in cases]
    infos = S.solve_batched([c[0] for c in cases], [c[1] for c in cases], phis)
    for (y, si), x, bi in zip(solo, phis, infos):
        assert torch.equal(x, y)
        assert bi["iters"] == si["iters"] and bi["converged"] == si["converged"]
    assert infos[1]["iters"] == 0 and torch.all(phis[1] == 0)
    assert infos[2]["converged"] == 0 and infos[2]["iters"] == 3
