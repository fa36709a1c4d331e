"""Launch shapes of the level-0 stencil passes: every shape gives the same bits; the
autotuner picks one of them and the solve stays the same."""
import pytest

from paper_0907_4863_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [dict(chunks_per_step=k, packed=p, block=b, blocks_per_sm=g)
          for k, p, b, g in [(1, 0, 128, 8), (1, 1, 256, 16), (2, 0, 256, 16), (2, 1, 128, 32),
                             (4, 0, 256, 32), (4, 1, 128, 8)]]


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


def _solve(S, op, w, prec, rho):
    import torch
    params = S.params_default(max_coarse=200, precision=prec, beta_rule=1 if prec else 0)
    h = S.setup(op, params)
    phi = torch.zeros_like(rho)
    info = S.solve(h, rho, phi)
    h.free()
    return phi, info


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("wl", ["pipe", "taper"])
def test_every_shape_gives_the_same_bits(S, prec, wl):
    import torch
    w = I.pipe_workload(52, I.QUADRATIC) if wl == "pipe" else I.taper_workload(40, 36, 58, I.LINEAR)
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    rho = I.gaussian_bunch_torch(w.grid, w.centre, w.sigma, 11)
    ref, info = _solve(S, op, w, prec, rho)
    assert info["converged"] == 1
    sp = 0 if prec == 0 else 1
    for shape in SHAPES:
        S.set_stencil_config(op, sp, shape)
        assert S.stencil_config(op, sp) == shape
        phi, info2 = _solve(S, op, w, prec, rho)
        assert info2["iters"] == info["iters"]
        assert torch.equal(phi, ref), shape
    S.set_stencil_config(op, sp, None)
    op.free()


def test_autotuner_sets_a_valid_shape_and_keeps_the_bits(S):
    import torch
    w = I.pipe_workload(64, I.LINEAR)
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    rho = I.gaussian_bunch_torch(w.grid, w.centre, w.sigma, 3)
    for prec, sp in ((0, 0), (1, 1)):
        ref, _ = _solve(S, op, w, prec, rho)
        best, us = S.autotune_stencil(op, sp)
        assert us > 0
        assert best["chunks_per_step"] in (1, 2, 4) and best["packed"] in (0, 1)
        assert best["block"] in (128, 256) and best["blocks_per_sm"] in (8, 16, 32)
        assert S.stencil_config(op, sp) == best
        phi, _ = _solve(S, op, w, prec, rho)
        assert torch.equal(phi, ref)
    op.free()


def test_shape_outside_the_sets_is_rejected(S):
    w = I.cylinder_workload(24, I.LINEAR)
    op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
    before = S.stencil_config(op, 1)
    for bad in (dict(chunks_per_step=3, packed=0, block=256, blocks_per_sm=16),
                dict(chunks_per_step=2, packed=0, block=512, blocks_per_sm=16),
                dict(chunks_per_step=2, packed=2, block=256, blocks_per_sm=16),
                dict(chunks_per_step=2, packed=0, block=256, blocks_per_sm=12)):
        with pytest.raises(S.SaamgError):
            S.set_stencil_config(op, 1, bad)
    with pytest.raises(S.SaamgError):
        S.stencil_config(op, 2)
    assert S.stencil_config(op, 1) == before
    op.free()


def test_grid_too_long_in_x_is_rejected(S):
    """Chunk records hold lane offsets within a line in 16 bits: more than 30000 nodes along x
    is refused before any device work."""
    w = I.cylinder_workload(24, I.LINEAR)
    g = I.Grid((30001, 4, 4), (1.0 / 30001, 0.25, 0.25), (-0.5, -0.375, -0.375))
    with pytest.raises(S.SaamgError) as e:
        S.build_operator(S.make_domain(w.domain), S.make_grid(g), w.mode)
    assert e.value.status == S.EINVAL
