"""Small helpers shared by the oracle tests and the parity tests (test code only)."""
import numpy as np

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I


def oracle_operator(w: I.Workload):
    g, d = w.grid, w.domain
    return O.Operator(g.n, g.h, g.origin, d.a, d.b, d.taper, d.cx, d.cy, d.zbc, d.symmetrize,
                      w.mode)


def oracle_hierarchy(op, **params):
    p = dict(cheb_degree=2, cheb_ratio=30.0, cheb_safety=1.1, max_coarse=1000, max_levels=10,
             power_iters=10)
    p.update(params)
    return O.Hierarchy(op, **p)


def box_coords(grid: I.Grid):
    x, y, z = grid.axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def small_workloads():
    """Workloads that span every branch of the discretisation at oracle-friendly sizes."""
    out = []
    for mode in (I.CONSTANT, I.LINEAR, I.QUADRATIC):
        out.append(I.Workload(f"cyl12_m{mode}", I.cell_centred_grid(12), I.Domain(0.45, 0.45), mode))
        out.append(I.Workload(f"ell14x11x9_m{mode}", I.cell_centred_grid(14, 11, 9),
                              I.Domain(0.45, 0.30, cx=0.013, cy=-0.021), mode))
        out.append(I.Workload(f"taper13x12x16_m{mode}", I.cell_centred_grid(13, 12, 16),
                              I.Domain(0.45, 0.45, taper=0.30 / 0.45), mode))
        out.append(I.Workload(f"dir_cyl10_m{mode}", I.vertex_grid(10),
                              I.Domain(0.5, 0.5, zbc=I.Z_DIRICHLET), mode))
    return out
