"""Batched solves, served requests and reused hierarchies against the FP64 oracle.

The batched call, the serving loop and the setup that reuses an aggregation hierarchy are
also checked elsewhere as bit-for-bit copies of the GPU's own one-at-a-time solve; here each
of their results is put beside the oracle directly: FP64 V-cycles within relative 1e-10 of
the oracle's solution with CG iterations within +-1, FP32 / BF16 V-cycles at the FP64
accuracy (recomputed residual <= 1.5e-8, error against the tightly solved discrete solution at
most ten times the FP64 path's own error).
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


def _check_against_oracle(oh, rho, got, info, prec, degree_note=""):
    """FP64: within 1e-10 of the oracle's rtol-1e-8 solution, iterations +-1.  Mixed: the
    recomputed residual at the target and the error against the oracle's tight solution at
    most 10x that of the oracle's own rtol-1e-8 solution (Polak-Ribiere, as the mixed path)."""
    assert info["converged"] == 1, (info, degree_note)
    if prec == 0:
        ref, oinfo = oh.solve(rho, rtol=1e-8)
        assert abs(info["iters"] - oinfo["iters"]) <= 1, (info, oinfo, degree_note)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 1e-10, (err, degree_note)
        return err
    exact, _ = oh.solve(rho, rtol=1e-13)
    ref, oinfo = oh.solve(rho, rtol=1e-8, beta_rule=1)
    assert info["relres_true"] <= 1.5e-8, (info, degree_note)
    assert info["iters"] <= oinfo["iters"] + (2 if prec == 1 else 4), (info, oinfo, degree_note)
    scale = np.max(np.abs(exact))
    err = np.max(np.abs(got - exact)) / scale
    err_ref = np.max(np.abs(ref - exact)) / scale
    assert err <= max(10 * err_ref, 1e-7), (err, err_ref, degree_note)
    return err


def test_batched_instances_against_oracle(S):
    """Instances of the 64-instance batch (non-cubic grids, cylinder / elliptic pipe / taper)
    plus quadratic-mode instances, FP64, FP32 and BF16 V-cycles, the Chebyshev degree of the
    FP32 hierarchies picked by the autotuner: one batched call, every result against the
    oracle hierarchy with the same degree."""
    import torch
    c4 = sorted(I.batched_instances(), key=lambda w: w.grid.nbox)
    picks = [c4[0], c4[1], next(w for w in c4 if w.domain.taper != 1.0)]
    extra = [I.Workload("ell52x44x60_quad", I.cell_centred_grid(52, 44, 60), I.Domain(0.45, 0.30),
                        I.QUADRATIC, centre=(0.05, -0.03, 0.08)),
             I.taper_workload(48, 50, 64, I.QUADRATIC)]
    cases = []
    for k, w in enumerate(picks + extra):
        for prec in ((0, 1) if k < 3 else (1, 2) if k == 3 else (0, 2)):
            cases.append((w, prec))
    hs, rhos, phis, meta = [], [], [], []
    for w, prec in cases:
        op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
        h = S.setup(op, S.params_default(max_coarse=400, precision=prec, beta_rule=1 if prec else 0))
        rho0 = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 40)).cuda()
        degree = 2
        if prec == 1:
            degree, _ = S.autotune_cheb_degree(h, rho0, 2, 4)
        for seed in (41, 42):
            rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed)
            hs.append(h)
            rhos.append(torch.from_numpy(rho).cuda())
            phis.append(torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda"))
            meta.append((w, prec, degree, rho))
    infos = S.solve_batched(hs, rhos, phis, rtol=1e-8)
    oracle_cache = {}
    for (w, prec, degree, rho), phi, info in zip(meta, phis, infos):
        key = (w.name, degree)
        if key not in oracle_cache:
            oracle_cache[key] = oracle_hierarchy(oracle_operator(w), max_coarse=400,
                                                 cheb_degree=degree)
        _check_against_oracle(oracle_cache[key], rho, phi.cpu().numpy(), info, prec,
                              f"{w.name} prec {prec} degree {degree}")


def test_served_requests_against_oracle(S):
    """A short stretch of the Poisson-arrival stream over three geometries (time steps with the
    bunch drifting in z, hierarchies kept across steps, several requests in flight): each
    served result against the oracle's solve of that request's right-hand side."""
    import torch
    from paper_0907_4863_gb300 import serve
    geoms = [I.cylinder_workload(40, I.LINEAR), I.pipe_workload(36, I.LINEAR),
             I.taper_workload(32, 32, 44, I.LINEAR)]
    reqs = [r for r in I.serving_requests(60, mean_gap_s=0.0005, ngeom=3)][:18]
    for prec in (1, 0):
        params = S.params_default(max_coarse=300, precision=prec, beta_rule=1 if prec else 0)
        srv = serve.Server(geoms, budget_bytes=8 << 30, slots=4, params=params, keep_results=True)
        records, st = srv.run(reqs)
        srv.close()
        torch.cuda.synchronize()
        assert st["requests"] == len(reqs) and st["all_converged"]
        ohs = {}
        for rec in records:
            w = geoms[rec["geometry"]]
            req = next(r for r in reqs if r.rid == rec["rid"])
            c = (w.centre[0], w.centre[1], w.centre[2] + 0.005 * req.step)
            rho = I.gaussian_bunch_torch(w.grid, c, w.sigma, req.seed).cpu().numpy()
            if rec["geometry"] not in ohs:
                ohs[rec["geometry"]] = oracle_hierarchy(oracle_operator(w), max_coarse=300)
            info = {"converged": rec["converged"], "iters": rec["iters"],
                    "relres_true": rec["relres_true"]}
            _check_against_oracle(ohs[rec["geometry"]], rho, srv.results[rec["rid"]].cpu().numpy(),
                                  info, prec, f"request {rec['rid']} prec {prec}")


def _stretched(w, hz_factor):
    """The same lattice of unknowns with another z spacing: the pipe's cross-section does not
    depend on z, so only the z couplings and the Robin rows change (a grid that follows the
    bunch along the beam axis)."""
    g = w.grid
    hz = g.h[2] * hz_factor
    grid = I.Grid(g.n, (g.h[0], g.h[1], hz), (g.origin[0], g.origin[1], -0.5 * (g.n[2] - 1) * hz))
    return I.Workload(w.name + f"_hz{hz_factor}", grid, w.domain, w.mode, centre=w.centre)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_reuse_after_the_operator_changes_against_oracle(S, prec):
    """Sec. 5.2, reusing the aggregation hierarchy: time step 1 sets up on one operator, time
    step 2 has a new operator (other z spacing, same unknowns) and keeps step 1's aggregates.
    The reused hierarchy is compared level by level with the oracle's fresh hierarchy of the
    new operator (aggregation depends on the pattern only, so the two must agree), and its
    solve with the oracle's."""
    import torch
    w1 = I.pipe_workload(44, I.LINEAR)
    w2 = _stretched(w1, 1.15)
    prm = dict(max_coarse=250, precision=prec, beta_rule=1 if prec else 0)
    op1 = S.build_operator(S.make_domain(w1.domain), S.make_grid(w1.grid), w1.mode)
    h1 = S.setup(op1, S.params_default(**prm))
    op2 = S.build_operator(S.make_domain(w2.domain), S.make_grid(w2.grid), w2.mode)
    h2 = S.setup_reuse(op2, h1, S.params_default(**prm))
    o2 = oracle_operator(w2)
    assert op2.size() == (o2.n, o2.nnz)
    oh2 = oracle_hierarchy(o2, max_coarse=250)
    info = h2.info()
    assert info["n"] == [oh2.n(l) for l in range(oh2.levels)]
    for l in range(oh2.levels):
        lv = S.hierarchy_copy_level(h2, l)
        if l < oh2.levels - 1:
            agg, root = oh2.agg(l)
            assert np.array_equal(lv["agg"], agg) and np.array_equal(lv["root"], root)
            P = oh2.P(l)
            assert np.array_equal(lv["p_rowptr"], P[0]) and np.array_equal(lv["p_col"], P[1])
            assert np.max(np.abs(lv["p_val"] - P[2])) <= 1e-12 * np.max(np.abs(P[2]))
        A = oh2.A(l)
        assert np.array_equal(lv["rowptr"], A[0]) and np.array_equal(lv["col"], A[1])
        assert np.max(np.abs(lv["val"] - A[2])) <= 1e-12 * np.max(np.abs(A[2]))
        if l < oh2.levels - 1:
            assert info["lam"][l] == pytest.approx(oh2.lam(l), rel=1e-12)
    # the new operator really differs from the old one
    assert not np.allclose(S.hierarchy_copy_level(h1, 1)["val"], S.hierarchy_copy_level(h2, 1)["val"])
    rho = I.gaussian_bunch(w2.grid, w2.centre, w2.sigma, 8)
    phi = torch.zeros(w2.grid.nbox, dtype=torch.float64, device="cuda")
    si = S.solve(h2, torch.from_numpy(rho).cuda(), phi, rtol=1e-8)
    _check_against_oracle(oh2, rho, phi.cpu().numpy(), si, prec, "reused hierarchy")
