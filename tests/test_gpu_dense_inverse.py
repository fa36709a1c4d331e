"""The coarsest-level direct solver on its own (Sec. 3.2, "Coarse level solver"): the GPU's
Gauss-Jordan inverse against the oracle's dense LU with partial pivoting, on matrices that
pivot at every step, at sizes that reach every launch form of the elimination."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_0907_4863_gb300 import build
    build.build()
    from paper_0907_4863_gb300 import saamg
    return saamg


def permuted_dominant(n, seed):
    """Rows of a diagonally dominant matrix in a random order: column k's largest entry
    sits in row perm(k), so partial pivoting exchanges rows at almost every step, and the
    matrix stays well conditioned at any size."""
    rng = np.random.default_rng(seed)
    m = rng.uniform(-1.0, 1.0, (n, n)) / max(n, 1)
    m[np.arange(n), np.arange(n)] = 2.0 + rng.uniform(0.0, 1.0, n)
    return np.ascontiguousarray(m[rng.permutation(n)])


def gpu_inverse(S, a):
    import torch
    ad = torch.from_numpy(a).cuda()
    inv = torch.empty_like(ad)
    S.dense_inverse(ad, inv)
    return inv.cpu().numpy()


# 600, 1417: panels of 5 and 4 steps with the own columns in shared memory; 7: fewer columns
# than one panel
@pytest.mark.parametrize("n", [1, 2, 7, 64, 600, 1417])
def test_inverse_matches_oracle_lu(S, n):
    a = permuted_dominant(n, 11 + n)
    inv = gpu_inverse(S, a)
    rng = np.random.default_rng(n)
    b = rng.standard_normal((n, 3))
    for c in range(3):
        x_oracle = O.dense_lu_solve(a, b[:, c])
        x_gpu = inv @ b[:, c]
        assert np.linalg.norm(x_gpu - x_oracle) <= 1e-12 * np.linalg.norm(x_oracle)


def test_general_nonsymmetric_matrix_with_zero_diagonal(S):
    rng = np.random.default_rng(5)
    n = 300
    a = rng.standard_normal((n, n))
    a[np.arange(n), np.arange(n)] = 0.0  # no step can keep its diagonal pivot
    inv = gpu_inverse(S, a)
    b = rng.standard_normal(n)
    x_oracle = O.dense_lu_solve(a, b)
    assert np.linalg.norm(inv @ b - x_oracle) <= 1e-10 * np.linalg.norm(x_oracle)


@pytest.mark.parametrize("n", [2624, 3744, 6800])
def test_large_sizes_by_residual(S, n):
    """2624, 3744: panels of 5 and 3 steps reading the own columns from the matrix; 6800 is
    past the narrowest panel that fits shared memory: one launch per pivot step."""
    a = permuted_dominant(n, n)
    inv = gpu_inverse(S, a)
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n)
    x = inv @ b
    assert np.linalg.norm(a @ x - b) <= 1e-13 * np.linalg.norm(b) * np.sqrt(n)
    # the exact inverse of a permuted matrix: inv(P M) = M^-1 P^T, so inv @ a is I
    k = rng.integers(0, n, 8)
    assert np.allclose((inv[k] @ a), np.eye(n)[k], atol=1e-13 * np.sqrt(n))


def test_singular_and_bad_arguments(S):
    import torch
    z = torch.zeros((5, 5), dtype=torch.float64, device="cuda")
    out = torch.empty_like(z)
    with pytest.raises(S.SaamgError) as e:
        S.dense_inverse(z, out)
    assert e.value.status == S.NUMERICAL
    nan_col = torch.eye(4, dtype=torch.float64, device="cuda")
    nan_col[:, 2] = float("nan")
    with pytest.raises(S.SaamgError) as e:
        S.dense_inverse(nan_col, torch.empty_like(nan_col))
    assert e.value.status == S.NUMERICAL
    # n = 0 is a no-op
    e0 = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    S.dense_inverse(e0, torch.empty_like(e0))
    # the library rejects sizes and overlaps before touching memory
    a = torch.eye(3, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    import ctypes as C
    L = S.lib()
    assert L.saamg_dense_inverse(20000, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()),
                                 C.c_void_p(st)) == S.EINVAL
    assert L.saamg_dense_inverse(3, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()),
                                 C.c_void_p(st)) == S.EINVAL
    assert L.saamg_dense_inverse(-1, None, None, C.c_void_p(st)) == S.EINVAL
    with pytest.raises(ValueError):
        S.dense_inverse(a.float(), a.float())
