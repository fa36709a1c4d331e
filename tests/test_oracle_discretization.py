"""Pins of the oracle's discretisation (Sec. 2) against the paper and mathematics.

None of these tests re-types the oracle's coefficient formulas: the rows are
re-derived symbolically from the paper's extrapolation rules, checked for exactness
on a manufactured quadratic solution, against the paper's Tables 3-5, and against
the matrix properties Sec. 2 states.
"""
import json
import os

import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import box_coords, oracle_hierarchy, oracle_operator, small_workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------
def test_lattice_count_matches_integer_brute_force():
    """Circle radius 0.45 in a 40^3 cell-centred box: x_i = (2i+1-n)/(2n), so
    x^2 + y^2 < R^2  <=>  (2i+1-n)^2 + (2j+1-n)^2 < (2nR)^2 = 36^2, exactly in integers
    (no lattice point lies on the circle: odd^2 + odd^2 = 2 mod 8, 1296 = 0 mod 8)."""
    n = 40
    w = I.Workload("c40", I.cell_centred_grid(n), I.Domain(0.45, 0.45), I.LINEAR)
    op = oracle_operator(w)
    a = 2 * np.arange(n) + 1 - n
    per_plane = int(np.sum((a[:, None] ** 2 + a[None, :] ** 2) < 36 ** 2))
    assert op.n == per_plane * n  # Robin ends: every z-plane holds unknowns
    # Dirichlet ends drop the first and last plane
    w2 = I.Workload("c40d", I.cell_centred_grid(n), I.Domain(0.45, 0.45, zbc=I.Z_DIRICHLET), I.LINEAR)
    assert oracle_operator(w2).n == per_plane * (n - 2)


@pytest.mark.parametrize("w", small_workloads(), ids=lambda w: w.name)
def test_boundary_fractions_locate_the_wall(w):
    """Sec. 2, Fig. 2: x* = x -/+ s h e_i is the wall point nearest x on the segment to the
    outside neighbour.  Checked with an independent evaluation of the wall function."""
    op = oracle_operator(w)
    g, d = w.grid, w.domain
    X, Y, Z = box_coords(g)
    fr = op.fractions()
    z0, z1 = g.origin[2], g.origin[2] + (g.n[2] - 1) * g.h[2]

    def F(x, y, z):
        sg = 1.0 + (d.taper - 1.0) * (z - z0) / (z1 - z0)
        return ((x - d.cx) / (d.a * sg)) ** 2 + ((y - d.cy) / (d.b * sg)) ** 2 - 1.0

    checked = 0
    for r in range(op.n):
        q = op.node_of_row[r]
        for dirn in range(6):
            s = fr[r, dirn]
            if s < 0:
                continue
            ax, sgn = dirn // 2, (-1.0 if dirn % 2 == 0 else 1.0)
            p = np.array([X[q], Y[q], Z[q]])
            assert 0.0 < s <= 1.0
            star = p.copy()
            star[ax] += sgn * s * g.h[ax]
            if s < 1.0:
                assert abs(F(*star)) < 1e-9, (r, dirn, s)
                checked += 1
            else:
                nb = p.copy()
                nb[ax] += sgn * g.h[ax]
                # the wall is at least one step away: the neighbour is a box face,
                # a Dirichlet end plane, or beyond the wall
                on_plane = ax == 2 and (nb[2] <= z0 + 1e-12 or nb[2] >= z1 - 1e-12)
                off_box = not (-0.5 < nb[ax] < 0.5)
                assert on_plane or off_box or F(*nb) >= -1e-12
    assert checked > 0


# ---------------------------------------------------------------------------
# Rows: substitution of the extrapolation rules into the difference star
# ---------------------------------------------------------------------------
def _symbolic_rows():
    """Coefficients of u(x) and of the inside neighbours after substituting Eqs. (7)-(11)
    into the star Eq. (6) (g = 0), derived by sympy from the paper's formulas."""
    u, um, up, s, t, c, h, dd = sp.symbols("u um up s t c h d", positive=True)
    star = c * (-um + 2 * u - up)
    rules = {
        0: {"one": 0, "two": (0, 0)},
        1: {"one": (1 - 1 / s) * u, "two": ((1 - 1 / s) * u, (1 - 1 / t) * u)},
        2: {"one": 2 * (s - 1) / s * u - (s - 1) / (s + 1) * up,
            "two": ((s - 1) * (t + 1) / (s * t) * u, (s + 1) * (t - 1) / (s * t) * u)},
    }
    out = {}
    for mode, rr in rules.items():
        e1 = sp.expand(star.subs(um, rr["one"]))  # minus side outside with fraction s
        e2 = sp.expand(star.subs({um: rr["two"][0], up: rr["two"][1]}))
        out[(mode, "one")] = (sp.lambdify((s, c), e1.coeff(u)), sp.lambdify((s, c), e1.coeff(up)))
        out[(mode, "two")] = sp.lambdify((s, t, c), e2.coeff(u))
    # Robin end plane, Eq. (11): virtual point um := up - (2h/d) u
    er = sp.expand(star.subs(um, up - 2 * h / dd * u))
    out["robin"] = (sp.lambdify((h, dd, c), er.coeff(u)), sp.lambdify((h, dd, c), er.coeff(up)))
    # corner reading: inner neighbour outside, replaced by its one-sided rule
    for mode in (0, 1, 2):
        inner = 0 if mode == 0 else (1 - 1 / t) * u
        ec = sp.expand(star.subs(um, up - 2 * h / dd * u).subs(up, inner))
        out[("corner", mode)] = sp.lambdify((t, h, dd, c), ec.coeff(u))
    return out


SYM = _symbolic_rows()


@pytest.mark.parametrize("w", small_workloads(), ids=lambda w: w.name)
def test_rows_equal_substituted_star(w):
    op = oracle_operator(w)
    g, d = w.grid, w.domain
    nx, ny, nz = g.n
    fr = op.fractions()
    row_of = -np.ones(g.nbox, np.int64)
    row_of[op.node_of_row] = np.arange(op.n)
    dist = 0.5 * (nz - 1) * g.h[2]
    robin = d.zbc == I.Z_ROBIN
    for r in range(op.n):
        q = int(op.node_of_row[r])
        i, j, k = q % nx, (q // nx) % ny, q // (nx * ny)
        diag = 0.0
        off = {}
        for ax in range(3):
            c = 1.0 / g.h[ax] ** 2
            step = [1, nx, nx * ny][ax]
            coord = [i, j, k][ax]
            lim = g.n[ax]
            nm = q - step if coord - 1 >= 0 else None
            npl = q + step if coord + 1 < lim else None
            in_m = nm is not None and row_of[nm] >= 0
            in_p = npl is not None and row_of[npl] >= 0
            if ax == 2 and robin and k in (0, nz - 1):
                inner, in_inner = (npl, in_p) if k == 0 else (nm, in_m)
                if in_inner:
                    diag += SYM["robin"][0](g.h[2], dist, c)
                    off[inner] = off.get(inner, 0.0) + SYM["robin"][1](g.h[2], dist, c)
                else:
                    tt = fr[r, 5 if k == 0 else 4]
                    diag += SYM[("corner", w.mode)](tt, g.h[2], dist, c)
                continue
            if in_m and in_p:
                diag += 2 * c
                off[nm] = -c
                off[npl] = -c
            elif not in_m and not in_p:
                diag += SYM[(w.mode, "two")](fr[r, 2 * ax], fr[r, 2 * ax + 1], c)
            else:
                f = fr[r, 2 * ax] if not in_m else fr[r, 2 * ax + 1]
                cu, cn = SYM[(w.mode, "one")]
                diag += cu(f, c)
                off[npl if in_p else nm] = cn(f, c)
        if robin and d.symmetrize and k in (0, nz - 1):
            diag *= 0.5
            off = {kk: 0.5 * v for kk, v in off.items()}
            assert op.bfac[r] == 0.5
        else:
            assert op.bfac[r] == 1.0
        lo, hi = op.rowptr[r], op.rowptr[r + 1]
        got = dict(zip(op.col[lo:hi].tolist(), op.aval[lo:hi].tolist()))
        want = {int(row_of[kk]): v for kk, v in off.items()}
        want[r] = diag
        assert set(got) == set(want), r
        for cidx, v in want.items():
            assert got[cidx] == pytest.approx(v, rel=1e-13, abs=1e-13 * abs(diag))


# ---------------------------------------------------------------------------
# Exactness on a manufactured quadratic solution (quadratic extrapolation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,a,b,cx,cy", [(16, 0.45, 0.45, 0.0, 0.0), (20, 0.45, 0.30, 0.02, -0.03),
                                         (24, 0.40, 0.33, -0.011, 0.017)])
def test_quadratic_mode_exact_for_manufactured_quadratic(n, a, b, cx, cy):
    """u = (1 - X^2 - Y^2)(1 - z^2/(3 d^2)) vanishes on the wall, satisfies the Robin
    condition du/dn + u/d = 0 on z = +-d and is quadratic along every grid line, so the
    star, Shortley-Weller and the central Robin difference reproduce it exactly."""
    w = I.Workload("mms", I.cell_centred_grid(n), I.Domain(a, b, cx=cx, cy=cy), I.QUADRATIC)
    op = oracle_operator(w)
    g = w.grid
    X, Y, Z = box_coords(g)
    dist = 0.5 * (g.n[2] - 1) * g.h[2]
    zc = Z - (g.origin[2] + dist)
    G = 1 - ((X - cx) / a) ** 2 - ((Y - cy) / b) ** 2
    Zf = 1 - zc ** 2 / (3 * dist ** 2)
    u = G * Zf
    f = (2 / a ** 2 + 2 / b ** 2) * Zf + G * 2 / (3 * dist ** 2)
    A = op.scipy(scaled=False)
    rows = op.node_of_row
    res = A @ u[rows] - op.bfac * f[rows]
    assert np.max(np.abs(res)) <= 1e-9 * np.max(np.abs(op.bfac * f[rows])) * n ** 2
    # and the full solver recovers it
    h = oracle_hierarchy(op)
    phi, info = h.solve(f, rtol=1e-12, beta_rule=0)
    assert info["rc"] == 0
    assert np.max(np.abs(phi[rows] - u[rows])) < 1e-9


def test_linear_mode_not_exact_but_consistent():
    """Linear extrapolation is not exact for the quadratic manufactured solution: a plausible
    swap of the linear and quadratic rules would make this residual vanish."""
    n, a, b = 16, 0.45, 0.45
    w = I.Workload("mms_lin", I.cell_centred_grid(n), I.Domain(a, b), I.LINEAR)
    op = oracle_operator(w)
    g = w.grid
    X, Y, Z = box_coords(g)
    dist = 0.5 * (g.n[2] - 1) * g.h[2]
    G = 1 - (X / a) ** 2 - (Y / b) ** 2
    Zf = 1 - Z ** 2 / (3 * dist ** 2)
    f = (2 / a ** 2 + 2 / b ** 2) * Zf + G * 2 / (3 * dist ** 2)
    res = op.scipy(scaled=False) @ (G * Zf)[op.node_of_row] - op.bfac * f[op.node_of_row]
    assert np.max(np.abs(res)) > 1e-3


# ---------------------------------------------------------------------------
# Tables 3-5: analytic cylinder with homogeneous Dirichlet data
# ---------------------------------------------------------------------------
def _analytic_errors(mode, m):
    g = I.vertex_grid(m)
    w = I.Workload("analytic", g, I.Domain(0.5, 0.5, zbc=I.Z_DIRICHLET), mode)
    op = oracle_operator(w)
    X, Y, Z = box_coords(g)
    r2 = X ** 2 + Y ** 2
    rho = -(np.pi ** 2 * r2 - np.pi ** 2 / 4 - 4) * np.sin(np.pi * (Z - 0.5))
    exact = (0.25 - r2) * np.sin(np.pi * (Z - 0.5))
    h = oracle_hierarchy(op)
    phi, info = h.solve(rho, rtol=1e-12)
    assert info["rc"] == 0
    e = phi[op.node_of_row] - exact[op.node_of_row]
    hh = 1.0 / m
    return np.sqrt(hh ** 3 * np.sum(e ** 2)), np.max(np.abs(e))


@pytest.mark.slow
@pytest.mark.parametrize("mode,name", [(0, "constant"), (1, "linear"), (2, "quadratic")])
def test_tables_3_to_5(mode, name):
    ref = json.load(open(os.path.join(GOLDEN, "paper_tables_3_5.json")))[name]
    got = {m: _analytic_errors(mode, m) for m in (64, 128)}
    for m in (64, 128):
        e2, einf = got[m]
        # The paper does not print its grid offset or solver tolerance; the discrete
        # errors must agree to within 25 %.
        assert 0.8 < e2 / ref[str(m)]["e2"] < 1.25, (m, e2)
        assert 0.8 < einf / ref[str(m)]["einf"] < 1.25, (m, einf)
    rate2 = np.log2(got[64][0] / got[128][0])
    rinf = np.log2(got[64][1] / got[128][1])
    # max-norm rates depend on where the wall cuts the lattice (the paper's own range
    # from 0.88 to 2.07); both rates must match the printed ones to within 0.3
    assert abs(rate2 - ref["rate_e2"]) < 0.3
    assert abs(rinf - ref["rate_einf"]) < 0.3


# ---------------------------------------------------------------------------
# Matrix properties stated in Sec. 2
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w", small_workloads(), ids=lambda w: w.name)
def test_m_matrix_and_symmetry(w):
    op = oracle_operator(w)
    A = op.scipy(scaled=False).tocoo()
    offd = A.row != A.col
    assert np.all(A.data[offd] < 0) and np.all(A.data[~offd] > 0)
    # weak diagonal dominance of every row (M-matrix)
    Ad = op.scipy(scaled=False)
    diag = Ad.diagonal()
    rowsum_off = np.asarray(abs(Ad).sum(axis=1)).ravel() - diag
    assert np.all(diag >= rowsum_off * (1 - 1e-14))
    Ah = op.scipy(scaled=True)
    asym = abs(Ah - Ah.T).max()
    if w.mode in (I.CONSTANT, I.LINEAR):
        assert asym == 0.0  # bitwise: ahat_ij = a_ij (s_i s_j)
    else:
        assert asym > 0.0
    # scaled diagonal is one up to rounding
    assert np.allclose(Ah.diagonal(), 1.0, rtol=0, atol=4e-16)


def test_unsymmetrised_robin_rows_are_nonsymmetric():
    w = I.Workload("c12_raw", I.cell_centred_grid(12), I.Domain(0.45, 0.45, symmetrize=0), I.LINEAR)
    A = oracle_operator(w).scipy(scaled=False)
    assert abs(A - A.T).max() > 0


@pytest.mark.parametrize("n", [8, 11])
def test_quadratic_mode_positive_definite(n):
    """Sec. 2: quadratic extrapolation gives a nonsymmetric but positive definite matrix."""
    w = I.Workload("q", I.cell_centred_grid(n), I.Domain(0.45, 0.30, taper=0.8), I.QUADRATIC)
    A = oracle_operator(w).scipy(scaled=False).toarray()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
