"""Reusing the aggregation hierarchy for a new operator with the same pattern (Sec. 5.2, Table 6)."""
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


def _op(S, w):
    return S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)


def _stretched(w, fz):
    g = w.grid
    n, h, o = g.n, list(g.h), list(g.origin)
    h[2] = g.h[2] * fz
    o[2] = -0.5 * (n[2] - 1) * h[2]
    return I.Workload(w.name + f"_z{fz}", I.Grid(n, tuple(h), tuple(o)), w.domain, w.mode)


@pytest.mark.parametrize("case", ["mode_change", "z_stretch"])
def test_reuse_equals_fresh_setup(S, case):
    import torch
    base = I.pipe_workload(40, I.LINEAR) if case == "mode_change" else I.cylinder_workload(36, I.LINEAR)
    new = I.pipe_workload(40, I.QUADRATIC) if case == "mode_change" else _stretched(base, 1.35)
    prm = S.params_default(max_coarse=60)
    h_old = S.setup(_op(S, base), prm)
    op_new = _op(S, new)
    h_reuse = S.setup_reuse(op_new, h_old)
    h_fresh = S.setup(op_new, prm)
    a, b = h_reuse.info(), h_fresh.info()
    assert a["n"] == b["n"] and a["nnz"] == b["nnz"] and a["levels"] >= 3
    assert a["lam"] == b["lam"]
    for l in range(a["levels"]):
        x = S.hierarchy_copy_level(h_reuse, l)
        y = S.hierarchy_copy_level(h_fresh, l)
        for k in x:
            assert np.array_equal(x[k], y[k]), (l, k)
    rho = torch.from_numpy(I.gaussian_bunch(new.grid, new.centre, new.sigma, 3)).cuda()
    p1, p2 = torch.zeros_like(rho), torch.zeros_like(rho)
    i1 = S.solve(h_reuse, rho, p1)
    i2 = S.solve(h_fresh, rho, p2)
    assert i1["converged"] == 1 and i1["iters"] == i2["iters"] and torch.equal(p1, p2)
    # the old hierarchy is untouched and still solves its own problem
    p0 = torch.zeros(base.grid.nbox, dtype=torch.float64, device="cuda")
    assert S.solve(h_old, torch.from_numpy(I.gaussian_bunch(base.grid, base.centre, base.sigma, 1)).cuda(),
                   p0)["converged"] == 1


def test_reuse_rejects_a_different_pattern(S):
    w1 = I.pipe_workload(32, I.LINEAR)
    w2 = I.Workload("other", w1.grid, I.Domain(0.40, 0.30), I.LINEAR)
    h = S.setup(_op(S, w1), S.params_default(max_coarse=60))
    with pytest.raises(S.SaamgError) as e:
        S.setup_reuse(_op(S, w2), h)
    assert e.value.status == S.EINVAL
