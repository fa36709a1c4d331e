"""The PIC-step transfers around the solve on the GPU against the oracle: cloud-in-cell
deposition (fixed-point, deterministic), E = -grad phi (bitwise), CIC gather (bitwise), and
the chain deposit -> solve -> gradient -> gather."""
import numpy as np
import pytest

from oracle import oracle as O
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def particles(g, n, seed):
    x, y, z, q = I.bunch_particles(g, n, (0.04, -0.03, 0.05), (0.1, 0.1, 0.2), seed=seed)
    # a few particles whose cells reach past the box, and unequal charges
    lo = np.array(g.origin)
    x[:3], y[:3], z[:3] = lo[0] - 0.3 * g.h[0], lo[1] + 0.2 * g.h[1], 0.0
    q = q * (1.0 + (np.arange(n) % 5))
    return x, y, z, q


@pytest.mark.parametrize("grid", [I.cell_centred_grid(64), I.cell_centred_grid(48, 40, 72)],
                         ids=["64^3", "48x40x72"])
def test_deposit_matches_oracle_and_is_deterministic(S, grid):
    import torch
    x, y, z, q = particles(grid, 200_000, 5)
    ref = O.deposit_cic(grid, x, y, z, q)
    G = S.make_grid(grid)
    rho = torch.empty(grid.nbox, dtype=torch.float64, device="cuda")
    S.deposit_cic(G, dev(x), dev(y), dev(z), dev(q), rho)
    got = rho.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    rho2 = torch.empty_like(rho)
    S.deposit_cic(G, dev(x), dev(y), dev(z), dev(q), rho2)
    assert torch.equal(rho, rho2)


def test_deposit_edge_cases(S):
    import torch
    g = I.cell_centred_grid(16)
    G = S.make_grid(g)
    rho = torch.full((g.nbox,), 7.0, dtype=torch.float64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    S.deposit_cic(G, e, e, e, e, rho)  # no particles: zero density
    assert torch.count_nonzero(rho) == 0
    q = np.array([1.0, np.nan])
    S.deposit_cic(G, dev([0.0, 0.1]), dev([0.0, 0.0]), dev([0.0, 0.0]), dev(q), rho)
    assert torch.all(torch.isnan(rho))


@pytest.mark.parametrize("w", [I.pipe_workload(40, I.LINEAR),
                               I.taper_workload(30, 26, 44, I.QUADRATIC),
                               I.Workload("dirichlet_vertex", I.vertex_grid(30),
                                          I.Domain(0.5, 0.5, zbc=I.Z_DIRICHLET), I.LINEAR)],
                         ids=lambda w: w.name)
def test_gradient_and_gather_bitwise(S, w):
    import torch
    o = oracle_operator(w)
    phi = np.random.default_rng(3).standard_normal(w.grid.nbox)
    ref = O.field_gradient(o, phi)
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    e = [torch.empty(w.grid.nbox, dtype=torch.float64, device="cuda") for _ in range(3)]
    S.field_gradient(op, dev(phi), *e)
    for a, b in zip(e, ref):
        assert np.array_equal(a.cpu().numpy(), b)
    x, y, z, _ = particles(w.grid, 50_000, 8)
    ep_ref = O.gather_cic(w.grid, ref, x, y, z)
    ep = [torch.empty(len(x), dtype=torch.float64, device="cuda") for _ in range(3)]
    S.gather_cic(S.make_grid(w.grid), *e, dev(x), dev(y), dev(z), *ep)
    for a, b in zip(ep, ep_ref):
        assert np.array_equal(a.cpu().numpy(), b)


def test_pic_step_chain_matches_oracle(S):
    """deposit -> solve -> E -> gather, each stage against the oracle's chain."""
    import torch
    w = I.pipe_workload(48, I.LINEAR)
    x, y, z, q = particles(w.grid, 300_000, 12)
    o = oracle_operator(w)
    oh = oracle_hierarchy(o, max_coarse=4096)
    rho_ref = O.deposit_cic(w.grid, x, y, z, q)
    phi_ref, _ = oh.solve(rho_ref, rtol=1e-10)
    e_ref = O.field_gradient(o, phi_ref)
    ep_ref = O.gather_cic(w.grid, e_ref, x, y, z)
    G = S.make_grid(w.grid)
    op = S.build_operator(S.make_domain(w.domain), G, w.mode)
    h = S.setup(op, S.params_default(max_coarse=4096))
    rho = torch.empty(w.grid.nbox, dtype=torch.float64, device="cuda")
    S.deposit_cic(G, dev(x), dev(y), dev(z), dev(q), rho)
    phi = torch.zeros_like(rho)
    info = S.solve(h, rho, phi, rtol=1e-10)
    assert info["converged"] == 1
    e = [torch.empty_like(rho) for _ in range(3)]
    S.field_gradient(op, phi, *e)
    ep = [torch.empty(len(x), dtype=torch.float64, device="cuda") for _ in range(3)]
    S.gather_cic(G, *e, dev(x), dev(y), dev(z), *ep)
    scale = np.max(np.abs(phi_ref))
    assert np.max(np.abs(phi.cpu().numpy() - phi_ref)) <= 1e-9 * scale
    for a, b in zip(ep, ep_ref):
        assert np.max(np.abs(a.cpu().numpy() - b)) <= 1e-8 * np.max(np.abs(b))
