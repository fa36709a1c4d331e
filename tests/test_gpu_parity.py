"""GPU path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sps

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import oracle_hierarchy, oracle_operator, small_workloads

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


def gpu_op(S, w):
    return S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)


def aniso_workloads():
    return [I.Workload("aniso48x40x64_lin", I.cell_centred_grid(48, 40, 64), I.Domain(0.45, 0.30), I.LINEAR),
            I.Workload("aniso37x53x29_quad_taper", I.cell_centred_grid(37, 53, 29),
                       I.Domain(0.45, 0.45, taper=0.30 / 0.45), I.QUADRATIC),
            I.Workload("raw_robin_lin", I.cell_centred_grid(20), I.Domain(0.45, 0.30, symmetrize=0), I.LINEAR)]


PARITY = small_workloads() + aniso_workloads()


@pytest.mark.parametrize("w", PARITY, ids=lambda w: w.name)
def test_operator_bitwise(S, w):
    """Unknowns, boundary treatment and scaling are the same IEEE operations on both sides."""
    o = oracle_operator(w)
    g = gpu_op(S, w)
    c = S.operator_copy(g)
    assert g.size() == (o.n, o.nnz)
    assert np.array_equal(c["node_of_row"], o.node_of_row)
    assert np.array_equal(c["scale"], o.scale)
    assert np.array_equal(c["rowptr"], o.rowptr)
    assert np.array_equal(c["col"], o.col)
    assert np.array_equal(c["val"], o.ahat)
    # the regular rows really are interior rows with the constant coefficients
    reg = c["is_regular"].astype(bool)
    lens = np.diff(o.rowptr)
    assert np.all(lens[reg] == 7)


@pytest.mark.parametrize("w", PARITY, ids=lambda w: w.name)
def test_stencil_apply(S, w):
    import torch
    o = oracle_operator(w)
    g = gpu_op(S, w)
    x = np.random.default_rng(7).standard_normal(o.n)
    y = torch.empty(o.n, dtype=torch.float64, device="cuda")
    S.operator_apply(g, torch.from_numpy(x).cuda(), y)
    A = o.scipy()
    ref = A @ x
    scale = abs(A) @ np.abs(x)
    assert np.max(np.abs(y.cpu().numpy() - ref) / scale) < 4e-16 * 8


def _csr_close(rp, cc, vv, rp2, cc2, vv2, rtol):
    assert np.array_equal(rp, rp2) and np.array_equal(cc, cc2)
    if len(vv):
        err = np.max(np.abs(vv - vv2)) / np.max(np.abs(vv2))
        assert err < rtol, err


# the 64^3 pipe coarsened to 40 rows: level 2 has rows of more than 64 entries (five of 170),
# which take the general path of the coarse-level A T lists
HIER = [(I.cylinder_workload(32, I.CONSTANT), 1000, 3), (I.pipe_workload(40, I.LINEAR), 60, 10),
        (I.pipe_workload(28, I.QUADRATIC), 40, 10), (I.taper_workload(30, 26, 44, I.LINEAR), 50, 10),
        (aniso_workloads()[0], 80, 10), (I.pipe_workload(64, I.LINEAR), 40, 10)]


@pytest.mark.parametrize("w,max_coarse,max_levels", HIER, ids=lambda v: getattr(v, "name", str(v)))
def test_hierarchy(S, w, max_coarse, max_levels):
    """Aggregates bit-exact; A_l, P_l, R_l patterns exact and values to rounding; lambda."""
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, max_coarse=max_coarse, max_levels=max_levels)
    g = gpu_op(S, w)
    h = S.setup(g, S.params_default(max_coarse=max_coarse, max_levels=max_levels))
    info = h.info()
    assert info["levels"] == oh.levels
    assert info["n"] == [oh.n(l) for l in range(oh.levels)]
    for l in range(oh.levels):
        c = S.hierarchy_copy_level(h, l)
        rp, cc, vv = oh.A(l)
        _csr_close(c["rowptr"], c["col"], c["val"], rp, cc, vv, 1e-12)
        if l + 1 < oh.levels:
            agg, root = oh.agg(l)
            assert np.array_equal(c["root"], root)
            assert np.array_equal(c["agg"], agg)
            assert info["lam"][l] == pytest.approx(oh.lam(l), rel=1e-12)
            _csr_close(c["p_rowptr"], c["p_col"], c["p_val"], *oh.P(l), 1e-12)
            _csr_close(c["r_rowptr"], c["r_col"], c["r_val"], *oh.R(l), 1e-12)


@pytest.mark.parametrize("w,max_coarse,max_levels", HIER[:3], ids=lambda v: getattr(v, "name", str(v)))
def test_vcycle(S, w, max_coarse, max_levels):
    import torch
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, max_coarse=max_coarse, max_levels=max_levels)
    g = gpu_op(S, w)
    h = S.setup(g, S.params_default(max_coarse=max_coarse, max_levels=max_levels))
    r = np.random.default_rng(11).standard_normal(o.n)
    z = torch.empty(o.n, dtype=torch.float64, device="cuda")
    S.vcycle(h, torch.from_numpy(r).cuda(), z)
    ref = oh.vcycle(r)
    assert np.max(np.abs(z.cpu().numpy() - ref)) < 1e-11 * np.max(np.abs(ref))


SOLVES = [(I.cylinder_workload(32, I.CONSTANT), dict(max_coarse=1000, max_levels=3)),
          (I.pipe_workload(48, I.LINEAR), dict(max_coarse=4096)),
          (I.pipe_workload(40, I.QUADRATIC), dict(max_coarse=200)),
          (I.taper_workload(33, 30, 47, I.QUADRATIC), dict(max_coarse=100)),
          (I.Workload("dirichlet_vertex", I.vertex_grid(36), I.Domain(0.5, 0.5, zbc=I.Z_DIRICHLET), I.LINEAR),
           dict(max_coarse=300)),
          (aniso_workloads()[0], dict(max_coarse=150))]


@pytest.mark.parametrize("w,prm", SOLVES, ids=lambda v: getattr(v, "name", str(v)))
def test_solve(S, w, prm):
    """FP64 solution within relative 1e-10 of the oracle, CG iterations within +-1."""
    import torch
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, **prm)
    for seed in (0, 3):
        rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed)
        ref, oinfo = oh.solve(rho, rtol=1e-8)
        g = gpu_op(S, w)
        h = S.setup(g, S.params_default(**prm))
        phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
        info = S.solve(h, torch.from_numpy(rho).cuda(), phi, rtol=1e-8)
        got = phi.cpu().numpy()
        assert info["status"] == 0 and info["converged"] == 1
        assert abs(info["iters"] - oinfo["iters"]) <= 1, (info, oinfo)
        assert info["relres"] <= 1e-8 and info["relres_true"] <= 1.01e-8
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
        outside = np.ones(w.grid.nbox, bool)
        outside[o.node_of_row] = False
        assert np.all(got[outside] == 0.0)


def test_solve_tight_tolerance_matches_oracle(S):
    """At rtol 1e-12 both sides approach the exact discrete solution."""
    import torch
    w = I.pipe_workload(36, I.LINEAR)
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, max_coarse=100)
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, 5)
    ref, oinfo = oh.solve(rho, rtol=1e-12)
    h = S.setup(gpu_op(S, w), S.params_default(max_coarse=100))
    phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
    info = S.solve(h, torch.from_numpy(rho).cuda(), phi, rtol=1e-12)
    assert abs(info["iters"] - oinfo["iters"]) <= 1
    assert np.max(np.abs(phi.cpu().numpy() - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_solve_edge_cases(S):
    import torch
    w = I.pipe_workload(24, I.LINEAR)
    g = gpu_op(S, w)
    h = S.setup(g, S.params_default(max_coarse=100))
    nbox = w.grid.nbox
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 0)).cuda()
    # zero right-hand side
    phi = torch.full((nbox,), 3.0, dtype=torch.float64, device="cuda")
    info = S.solve(h, torch.zeros(nbox, dtype=torch.float64, device="cuda"), phi)
    assert info["iters"] == 0 and info["converged"] == 1 and torch.all(phi == 0)
    # iteration limit
    h2 = S.setup(g, S.params_default(max_coarse=100, maxit=2))
    phi = torch.zeros(nbox, dtype=torch.float64, device="cuda")
    info = S.solve(h2, rho, phi)
    assert info["status"] == S.NOT_CONVERGED and info["iters"] == 2
    # converged solve, then an exact warm start needs no iteration
    phi = torch.zeros(nbox, dtype=torch.float64, device="cuda")
    info = S.solve(h, rho, phi)
    assert info["converged"] == 1
    info2 = S.solve(h, rho, phi.clone())
    assert info2["iters"] == 0
    # warm start from the previous time step needs fewer iterations
    rho2 = torch.from_numpy(I.gaussian_bunch(w.grid, (0.08, 0.04, 0.105), w.sigma, 0)).cuda()
    info3 = S.solve(h, rho2, phi.clone())
    assert info3["converged"] == 1 and info3["iters"] < info["iters"]
    # NaN in the right-hand side
    bad = rho.clone()
    m = w.grid.n[0] // 2
    bad[m + w.grid.n[0] * (m + w.grid.n[1] * m)] = float("nan")  # the box centre is an unknown
    with pytest.raises(S.SaamgError) as e:
        S.solve(h, bad, torch.zeros_like(phi))
    assert e.value.status == S.NUMERICAL
    # host arrays through the same call
    rh = rho.cpu().numpy()
    ph = np.zeros(nbox)
    infoh = S.solve_host(h, rh, ph)
    assert infoh["iters"] == info["iters"]
    assert np.array_equal(ph, phi.cpu().numpy())
    # pinned host arrays (read and written in place by the gather and scatter kernels); the
    # box corner lies outside the pipe: its initial value is ignored and 0 comes back
    rp = torch.from_numpy(rh).pin_memory()
    pp = torch.zeros(nbox, dtype=torch.float64).pin_memory()
    pp[0] = 7.0
    infop = S.solve_host(h, rp.numpy(), pp.numpy())
    assert infop["iters"] == info["iters"]
    assert torch.equal(pp, phi.cpu())
    # single level: the V-cycle is the exact inverse
    w1 = I.cylinder_workload(10, I.QUADRATIC)
    h1 = S.setup(gpu_op(S, w1), S.params_default(max_coarse=10 ** 6))
    assert h1.info()["levels"] == 1
    phi1 = torch.zeros(w1.grid.nbox, dtype=torch.float64, device="cuda")
    info1 = S.solve(h1, torch.from_numpy(I.gaussian_bunch(w1.grid, w1.centre, w1.sigma, 0)).cuda(), phi1)
    assert info1["iters"] == 1
    # invalid arguments
    with pytest.raises(S.SaamgError):
        S.solve(h, rho, phi, rtol=-1.0)
    with pytest.raises(S.SaamgError):
        S.setup(g, S.params_default(cheb_degree=0))


@pytest.mark.parametrize("n", [10, 13, 16, 18])
def test_dense_coarse_inverse_sizes(S, n):
    """A single level of 600 .. 3744 unknowns: the coarse inverse takes a panel of
    5, 4, 5 and 3 pivot steps per launch, the own columns staged in shared memory for the
    two smaller sizes and read from the matrix for the two larger.  The V-cycle is then the
    exact inverse: PCG stops after one iteration with the true residual at rounding level."""
    import torch
    w = I.cylinder_workload(n, I.LINEAR)
    h = S.setup(gpu_op(S, w), S.params_default(max_coarse=10 ** 6))
    assert h.info()["levels"] == 1
    phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 0)).cuda()
    info = S.solve(h, rho, phi, rtol=1e-10)
    assert info["iters"] == 1
    assert info["relres_true"] < 1e-11


def test_determinism(S):
    import torch
    w = I.pipe_workload(32, I.QUADRATIC)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 2)).cuda()
    outs = []
    for _ in range(2):
        h = S.setup(gpu_op(S, w), S.params_default(max_coarse=100))
        phi = torch.zeros(w.grid.nbox, dtype=torch.float64, device="cuda")
        S.solve(h, rho, phi)
        outs.append(phi.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def _sym_graph(n, p, rng, loops):
    m = rng.random((n, n)) < p
    m = np.triu(m, 1)
    m = m | m.T
    if loops:
        m |= np.eye(n, dtype=bool)
    A = sps.csr_matrix(m.astype(float))
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32)


@pytest.mark.parametrize("trial", range(6))
def test_mis2_aggregate_standalone(S, trial):
    import torch
    rng = np.random.default_rng(100 + trial)
    n = int(rng.integers(50, 3000))
    rp, cc = _sym_graph(n, 6.0 / n, rng, loops=trial % 2 == 0)
    ids = rng.permutation(10 * n)[:n].astype(np.uint32)  # distinct, in no particular order
    seed = int(rng.integers(0, 2 ** 32))
    # oracle with explicit self loops (closed neighbourhoods)
    A = sps.csr_matrix((np.ones(len(cc)), cc, rp), shape=(n, n)) + sps.eye(n)
    A = A.tocsr()
    A.sort_indices()
    root_ref = O.mis2(A.indptr, A.indices, ids, seed)
    agg_ref, nagg_ref = O.aggregate(A.indptr, A.indices, ids, seed, root_ref)
    root = torch.empty(n, dtype=torch.uint8, device="cuda")
    agg = torch.empty(n, dtype=torch.int32, device="cuda")
    nagg = S.mis2_aggregate(torch.from_numpy(rp).cuda(), torch.from_numpy(cc).cuda(),
                            torch.from_numpy(ids.view(np.int32)).cuda(), seed, root, agg)
    assert nagg == nagg_ref
    assert np.array_equal(root.cpu().numpy(), root_ref)
    assert np.array_equal(agg.cpu().numpy(), agg_ref)


@pytest.mark.parametrize("deg,loops", [(7.0, True), (30.0, False)], ids=["deg7", "deg30"])
def test_mis2_aggregate_large_graph(S, deg, loops):
    """300k nodes: the late rounds run on the list of undecided rows (large levels only); the
    set and the aggregates still equal the sequential greedy oracle's."""
    import torch
    rng = np.random.default_rng(7 + int(deg))
    n = 300_000
    m = int(n * deg / 2)
    r, c = rng.integers(0, n, m), rng.integers(0, n, m)
    keep = r != c
    G = sps.coo_matrix((np.ones(int(keep.sum())), (r[keep], c[keep])), shape=(n, n)).tocsr()
    G = ((G + G.T) > 0).astype(float).tocsr()
    if loops:
        G = (G + sps.eye(n)).tocsr()
    G.sort_indices()
    rp, cc = G.indptr.astype(np.int32), G.indices.astype(np.int32)
    ids = rng.permutation(4 * n)[:n].astype(np.uint32)
    seed = int(rng.integers(0, 2 ** 32))
    A = sps.csr_matrix((np.ones(len(cc)), cc, rp), shape=(n, n)) + sps.eye(n)
    A = A.tocsr()
    A.sort_indices()
    root_ref = O.mis2(A.indptr, A.indices, ids, seed)
    agg_ref, nagg_ref = O.aggregate(A.indptr, A.indices, ids, seed, root_ref)
    root = torch.empty(n, dtype=torch.uint8, device="cuda")
    agg = torch.empty(n, dtype=torch.int32, device="cuda")
    nagg = S.mis2_aggregate(torch.from_numpy(rp).cuda(), torch.from_numpy(cc).cuda(),
                            torch.from_numpy(ids.view(np.int32)).cuda(), seed, root, agg)
    assert nagg == nagg_ref
    assert np.array_equal(root.cpu().numpy(), root_ref)
    assert np.array_equal(agg.cpu().numpy(), agg_ref)
