"""Oracle pins for the steps around the solve in a PIC time step (Sec. 1, Sec. 4.1): cloud-in-
cell deposition, E = -grad phi, and the field gathered back to the particles."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import box_coords, oracle_operator


def test_deposition_conserves_charge_and_first_moments():
    g = I.cell_centred_grid(20, 18, 24)
    x, y, z, q = I.bunch_particles(g, 5000, (0.03, -0.02, 0.05), (0.1, 0.1, 0.2), seed=3)
    q = q * (1.0 + np.arange(len(q)) % 7)  # unequal charges
    rho = O.deposit_cic(g, x, y, z, q)
    vol = g.h[0] * g.h[1] * g.h[2]
    X, Y, Z = box_coords(g)
    assert rho.sum() * vol == pytest.approx(q.sum(), rel=1e-13)
    # CIC reproduces linear functions: sum_node w x_node = x_p, so the dipole moments agree
    for node, part in ((X, x), (Y, y), (Z, z)):
        assert (rho * node).sum() * vol == pytest.approx((q * part).sum(), rel=1e-12, abs=1e-14)


def test_particle_on_a_node_deposits_there_only():
    g = I.cell_centred_grid(8)
    X, Y, Z = box_coords(g)
    v = 3 + 8 * (4 + 8 * 5)
    rho = O.deposit_cic(g, [X[v]], [Y[v]], [Z[v]], [2.0])
    vol = g.h[0] * g.h[1] * g.h[2]
    assert rho[v] == pytest.approx(2.0 / vol, rel=1e-14)
    assert np.count_nonzero(np.abs(rho) > 1e-12 * rho[v]) == 1
    # particles whose cell leaves the box drop the outside nodes
    rho = O.deposit_cic(g, [g.origin[0] - 0.5 * g.h[0]], [0.0], [0.0], [1.0])
    assert rho.sum() * vol == pytest.approx(0.5, rel=1e-14)


@pytest.mark.parametrize("mode", [I.CONSTANT, I.LINEAR, I.QUADRATIC])
def test_gradient_exact_for_a_quadratic_vanishing_on_the_wall(mode):
    """phi = C (1 - ((x-cx)/a)^2 - ((y-cy)/b)^2) is zero on the pipe wall and quadratic, so the
    three-point formula through the wall point is exact at every unknown: E_x, E_y exact also
    next to the wall, E_z = 0 away from the Robin planes; zero outside the unknowns."""
    d = I.Domain(0.45, 0.30, cx=0.013, cy=-0.021)
    w = I.Workload("ell", I.cell_centred_grid(26, 22, 12), d, mode)
    op = oracle_operator(w)
    X, Y, Z = box_coords(w.grid)
    C = 2.5
    phi = C * (1 - ((X - d.cx) / d.a) ** 2 - ((Y - d.cy) / d.b) ** 2)
    inside = np.zeros(w.grid.nbox, bool)
    inside[op.node_of_row] = True
    phi[~inside] = 0.0
    ex, ey, ez = O.field_gradient(op, phi)
    r = op.node_of_row
    assert np.allclose(ex[r], 2 * C * (X[r] - d.cx) / d.a ** 2, rtol=0, atol=1e-9 * C)
    assert np.allclose(ey[r], 2 * C * (Y[r] - d.cy) / d.b ** 2, rtol=0, atol=1e-9 * C)
    nz = w.grid.n[2]
    k = r // (w.grid.n[0] * w.grid.n[1])
    mid = (k > 0) & (k < nz - 1)
    assert np.all(np.abs(ez[r[mid]]) <= 1e-12 * C)
    # on the Robin end planes the z-derivative is the one the Robin condition gives
    dist = 0.5 * (nz - 1) * w.grid.h[2]
    bot, top = r[k == 0], r[k == nz - 1]
    assert np.allclose(ez[bot], -phi[bot] / dist, rtol=1e-14, atol=0)
    assert np.allclose(ez[top], phi[top] / dist, rtol=1e-14, atol=0)
    assert np.all(ex[~inside] == 0) and np.all(ey[~inside] == 0) and np.all(ez[~inside] == 0)


def test_gradient_is_central_difference_in_the_interior():
    w = I.pipe_workload(16, I.LINEAR)
    op = oracle_operator(w)
    phi = np.random.default_rng(1).standard_normal(w.grid.nbox)
    ex, _, _ = O.field_gradient(op, phi)
    nx = w.grid.n[0]
    r = op.node_of_row
    inside = np.zeros(w.grid.nbox, bool)
    inside[r] = True
    both = r[inside[r - 1] & inside[(r + 1) % w.grid.nbox] & (r % nx > 0) & (r % nx < nx - 1)]
    assert np.allclose(ex[both], -(phi[both + 1] - phi[both - 1]) / (2 * w.grid.h[0]),
                       rtol=1e-14, atol=1e-14)


def test_gather_exact_for_linear_fields_and_adjoint_to_deposition():
    g = I.cell_centred_grid(14, 15, 16)
    x, y, z, q = I.bunch_particles(g, 3000, (0.0, 0.0, 0.0), (0.15, 0.15, 0.2), seed=9)
    X, Y, Z = box_coords(g)
    e = [1.5 + 2 * X - Y, -0.5 + 3 * Z, 0.25 * X + Y + Z]
    ep = O.gather_cic(g, e, x, y, z)
    assert np.allclose(ep[0], 1.5 + 2 * x - y, rtol=0, atol=1e-13)
    assert np.allclose(ep[1], -0.5 + 3 * z, rtol=0, atol=1e-13)
    assert np.allclose(ep[2], 0.25 * x + y + z, rtol=0, atol=1e-13)
    # sum_p q_p E(x_p) = sum_node rho_node E_node V for any nodal field (same weights)
    f = np.random.default_rng(2).standard_normal(g.nbox)
    fp = O.gather_cic(g, [f, f, f], x, y, z)[0]
    rho = O.deposit_cic(g, x, y, z, q)
    vol = g.h[0] * g.h[1] * g.h[2]
    assert (q * fp).sum() == pytest.approx((rho * f).sum() * vol, rel=1e-12)
