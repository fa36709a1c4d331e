"""Cube aggregation (the paper's 3^3 "decoupled" aggregates, Sec. 3.2) on the GPU against the
oracle: aggregates and roots bit-exact on every level, A_l / P_l / R_l patterns exact and
values to rounding, V-cycle and solve parity, reuse of a cube hierarchy."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import oracle_hierarchy, oracle_operator

pytestmark = pytest.mark.gpu

CUBES = O.Hierarchy.AGG_CUBES


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


def _csr_close(rp, cc, vv, rp2, cc2, vv2, rtol):
    assert np.array_equal(rp, rp2) and np.array_equal(cc, cc2)
    if len(vv):
        assert np.max(np.abs(vv - vv2)) / np.max(np.abs(vv2)) < rtol


CASES = [(I.pipe_workload(40, I.LINEAR), dict(max_coarse=60)),
         (I.taper_workload(30, 26, 44, I.QUADRATIC), dict(max_coarse=50)),
         (I.cylinder_workload(32, I.CONSTANT), dict(max_coarse=1000, max_levels=3)),
         (I.Workload("box27", I.cell_centred_grid(27), I.Domain(5.0, 5.0), I.LINEAR),
          dict(max_coarse=30))]


@pytest.mark.parametrize("w,prm", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_cube_hierarchy_matches_oracle(S, w, prm):
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, aggregation=CUBES, **prm)
    h = S.setup(gpu_op(S, w), S.params_default(aggregation=1, **prm))
    info = h.info()
    assert info["levels"] == oh.levels >= 2
    assert info["n"] == [oh.n(l) for l in range(oh.levels)]
    for l in range(oh.levels):
        c = S.hierarchy_copy_level(h, l)
        _csr_close(c["rowptr"], c["col"], c["val"], *oh.A(l), 1e-12)
        if l + 1 < oh.levels:
            agg, root = oh.agg(l)
            assert np.array_equal(c["agg"], agg)
            assert np.array_equal(c["root"], root)
            assert info["lam"][l] == pytest.approx(oh.lam(l), rel=1e-12)
            _csr_close(c["p_rowptr"], c["p_col"], c["p_val"], *oh.P(l), 1e-12)
            _csr_close(c["r_rowptr"], c["r_col"], c["r_val"], *oh.R(l), 1e-12)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("w,prm", CASES[:2], ids=lambda v: getattr(v, "name", str(v)))
def test_cube_vcycle_and_solve(S, w, prm, prec):
    import torch
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, aggregation=CUBES, **prm)
    rule = 1 if (w.mode == I.QUADRATIC or prec) else 0
    h = S.setup(gpu_op(S, w), S.params_default(aggregation=1, precision=prec, beta_rule=rule,
                                                **prm))
    r = np.random.default_rng(2).standard_normal(o.n)
    z = torch.empty(o.n, dtype=torch.float64, device="cuda")
    S.vcycle(h, torch.from_numpy(r).cuda(), z)
    ref = oh.vcycle(r)
    err = np.max(np.abs(z.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < (1e-11 if prec == 0 else 2e-5), err
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, 6)
    phi_ref, oinfo = oh.solve(rho, rtol=1e-8, beta_rule=rule)
    phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
    info = S.solve(h, torch.from_numpy(rho).cuda(), phi, rtol=1e-8)
    assert info["converged"] == 1 and info["relres_true"] <= 1.5e-8
    if prec == 0:
        assert abs(info["iters"] - oinfo["iters"]) <= 1
        got = phi.cpu().numpy()
        assert np.max(np.abs(got - phi_ref)) <= 1e-10 * np.max(np.abs(phi_ref))
    else:
        assert info["iters"] <= oinfo["iters"] + 2


def test_cube_hierarchy_reuse_equals_fresh_setup(S):
    import torch
    w = I.pipe_workload(36, I.LINEAR)
    prm = S.params_default(aggregation=1, max_coarse=60)
    g1 = gpu_op(S, w)
    h1 = S.setup(g1, prm)
    g2 = gpu_op(S, w)
    h2 = S.setup_reuse(g2, h1, prm)
    h3 = S.setup(g2, prm)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 1)).cuda()
    outs = []
    for h in (h2, h3):
        phi = torch.zeros_like(rho)
        S.solve(h, rho, phi, rtol=1e-10)
        outs.append(phi.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_bad_aggregation_kind_is_rejected(S):
    w = I.pipe_workload(16, I.LINEAR)
    with pytest.raises(S.SaamgError):
        S.setup(gpu_op(S, w), S.params_default(aggregation=7))
