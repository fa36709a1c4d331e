"""Pins of the oracle's SA-AMG setup and solve (Sec. 3) against mathematics.

MIS-2 is checked against brute force and against a different algorithm (synchronous
rounds) that provably returns the same set; P and the Galerkin operator against dense
linear algebra; the Chebyshev smoother against its closed-form error polynomial; the
coarse LU against a library solve; the V-cycle against symmetry and the exact inverse;
PCG against a sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from oracle import oracle as O
from paper_0907_4863_gb300 import inputs as I
from tests.oracle_cases import oracle_hierarchy, oracle_operator, small_workloads

SEED0 = 0x9E3779B9


def _key(ids, seed):
    h = np.array([O.fmix32(int(v) ^ seed) for v in ids], dtype=np.uint64)
    return (h << np.uint64(32)) | ids.astype(np.uint64)


def _random_graph(n, p, rng):
    """Symmetric random graph in CSR with the diagonal included."""
    m = rng.random((n, n)) < p
    m = np.triu(m, 1)
    m = m | m.T | np.eye(n, dtype=bool)
    A = sps.csr_matrix(m.astype(float))
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), m


def _dist(m):
    """All-pairs graph distance by BFS on a dense adjacency (brute force)."""
    n = len(m)
    D = np.full((n, n), 99, int)
    for s in range(n):
        D[s, s] = 0
        front = [s]
        while front:
            nxt = []
            for v in front:
                for u in np.nonzero(m[v])[0]:
                    if D[s, u] > D[s, v] + 1:
                        D[s, u] = D[s, v] + 1
                        nxt.append(u)
            front = nxt
    return D


def _rounds_mis2(indptr, idx, key):
    """Synchronous rounds: an undecided node joins when its key is the largest among the
    undecided nodes within distance 2; nodes within distance 2 of a joined node leave."""
    n = len(indptr) - 1
    state = np.zeros(n, int)  # 0 undecided, 1 in, 2 out
    nb = [idx[indptr[i]:indptr[i + 1]] for i in range(n)]
    while np.any(state == 0):
        m1 = np.array([max([key[u] for u in nb[j] if state[u] == 0], default=0) for j in range(n)],
                      dtype=np.uint64)
        m2 = np.array([max([m1[j] for j in nb[i]], default=0) for i in range(n)], dtype=np.uint64)
        join = (state == 0) & (m2 == key)
        state[join] = 1
        o1 = np.array([any(state[u] == 1 for u in nb[j]) for j in range(n)])
        o2 = np.array([any(o1[j] for j in nb[i]) for i in range(n)])
        state[(state == 0) & o2] = 2
    return (state == 1).astype(np.uint8)


def test_fmix32_is_a_bijection_sample():
    assert O.fmix32(0) == 0
    vals = {O.fmix32(v) for v in range(1 << 14)}
    assert len(vals) == 1 << 14


def _murmur3_x86_32(data, seed):
    """MurmurHash3_x86_32 (Appleby) written from its description: 4-byte little-endian
    blocks mixed into h (k *= c1, rotl 15, k *= c2; h ^= k, rotl 13, h = 5 h + 0xe6546b64),
    the tail bytes mixed the same way without the h rotation, h ^= length, and the finaliser
    taken from the oracle."""
    m = 0xFFFFFFFF
    rotl = lambda x, r: ((x << r) | (x >> (32 - r))) & m  # noqa: E731
    c1, c2 = 0xCC9E2D51, 0x1B873593
    h = seed
    nb = len(data) // 4
    for i in range(nb):
        k = int.from_bytes(data[4 * i:4 * i + 4], "little")
        k = rotl((k * c1) & m, 15)
        h ^= (k * c2) & m
        h = (rotl(h, 13) * 5 + 0xE6546B64) & m
    tail = data[4 * nb:]
    if tail:
        k = int.from_bytes(tail, "little")
        k = rotl((k * c1) & m, 15)
        h ^= (k * c2) & m
    return O.fmix32(h ^ len(data))


# Published known answers of MurmurHash3_x86_32 (the reference implementation's widely
# quoted test values).  For the empty key the hash is fmix32(seed), so the first three pin
# the finaliser directly; the others reach it through the block and tail mixing.
_MURMUR3_KNOWN = [
    (b"", 0x00000000, 0x00000000),
    (b"", 0x00000001, 0x514E28B7),
    (b"", 0xFFFFFFFF, 0x81F16F39),
    (b"\x00\x00\x00\x00", 0x00000000, 0x2362F9DE),
    (b"\xff\xff\xff\xff", 0x00000000, 0x76293B50),
    (b"!Ce\x87", 0x00000000, 0xF55B516B),
    (b"abc", 0x00000000, 0xB3DD93FA),
    (b"aaaa", 0x9747B28C, 0x5A97808A),
    (b"Hello, world!", 0x9747B28C, 0x24884CBA),
    (b"The quick brown fox jumps over the lazy dog", 0x9747B28C, 0x2FA826CD),
]


@pytest.mark.parametrize("data,seed,want", _MURMUR3_KNOWN)
def test_fmix32_known_answers(data, seed, want):
    """The priority hash is the MurmurHash3 finaliser: a mistyped shift or multiplier would be
    a bijection all the same, but it would miss these published values."""
    assert _murmur3_x86_32(data, seed) == want


@pytest.mark.parametrize("trial", range(12))
def test_mis2_bruteforce_and_rounds(trial):
    rng = np.random.default_rng(trial)
    n = int(rng.integers(5, 40))
    indptr, idx, m = _random_graph(n, float(rng.uniform(0.03, 0.25)), rng)
    ids = rng.permutation(1000)[:n].astype(np.uint32)
    seed = int(rng.integers(0, 2 ** 32))
    root = O.mis2(indptr, idx, ids, seed)
    D = _dist(m)
    R = np.nonzero(root)[0]
    # independence at distance >= 3
    for a in R:
        for b in R:
            if a != b:
                assert D[a, b] >= 3
    # maximality: every node within distance 2 of some root
    assert np.all(D[:, R].min(axis=1) <= 2)
    # greedy by decreasing key: a node is out only if a higher-key root is within distance 2
    key = _key(ids, seed)
    for v in range(n):
        if not root[v]:
            assert any(D[v, r] <= 2 and key[r] > key[v] for r in R)
    # the synchronous-round algorithm gives the identical set
    assert np.array_equal(_rounds_mis2(indptr, idx, key), root)


@pytest.mark.parametrize("w", small_workloads()[:4], ids=lambda w: w.name)
def test_aggregates_partition_and_structure(w):
    op = oracle_operator(w)
    ids = op.node_of_row.astype(np.uint32)
    root = O.mis2(op.rowptr, op.col, ids, SEED0)
    agg, nagg = O.aggregate(op.rowptr, op.col, ids, SEED0, root)
    assert nagg == int(root.sum()) and nagg > 0
    assert agg.min() == 0 and agg.max() == nagg - 1
    # numbering by ascending root row
    roots = np.nonzero(root)[0]
    assert np.array_equal(agg[roots], np.arange(nagg))
    A = op.scipy()
    # every neighbour of a root belongs to the root's aggregate (phase 1)
    for r in roots:
        nbrs = A.indices[A.indptr[r]:A.indptr[r + 1]]
        assert np.all(agg[nbrs] == agg[r])
    # every aggregate is connected in G
    for J in range(nagg):
        members = set(np.nonzero(agg == J)[0].tolist())
        seen = {int(roots[J])}
        front = [int(roots[J])]
        while front:
            v = front.pop()
            for u in A.indices[A.indptr[v]:A.indptr[v + 1]]:
                if int(u) in members and int(u) not in seen:
                    seen.add(int(u))
                    front.append(int(u))
        assert seen == members


def test_aggregates_identical_across_boundary_modes():
    """G_0 is the structural graph of A, the same for all three extrapolations."""
    aggs = []
    for mode in (I.CONSTANT, I.LINEAR, I.QUADRATIC):
        w = I.pipe_workload(20, mode)
        op = oracle_operator(w)
        h = oracle_hierarchy(op, max_coarse=50)
        aggs.append([h.agg(l)[0] for l in range(h.levels - 1)])
    for l in range(len(aggs[0])):
        assert np.array_equal(aggs[0][l], aggs[1][l]) and np.array_equal(aggs[0][l], aggs[2][l])


def test_power_lambda_bounds_spectrum():
    w = I.cylinder_workload(12, I.LINEAR)
    op = oracle_operator(w)
    A = op.scipy().toarray()
    Dinv = 1.0 / np.diag(A)
    lam_max = np.linalg.eigvalsh(0.5 * (A + A.T) * np.sqrt(Dinv)[:, None] * np.sqrt(Dinv)[None, :]).max()
    ids = op.node_of_row.astype(np.uint32)
    lam10 = O.power_lambda(op.rowptr, op.col, op.ahat, ids, 10)
    lam400 = O.power_lambda(op.rowptr, op.col, op.ahat, ids, 400)
    assert lam10 <= lam_max * (1 + 1e-12)
    assert lam10 > 0.8 * lam_max
    assert abs(lam400 - lam_max) < 2e-3 * lam_max


@pytest.mark.parametrize("n,iters", [(10, 10), (13, 10), (10, 3), (16, 25)])
def test_power_lambda_closed_form_path_graph(n, iters):
    """The estimate after exactly `iters` steps, in closed form.  For the path-graph Laplacian
    tridiag(-1, 2, -1), D^-1 A has eigenvalues mu_k = 1 - cos(k pi / (n + 1)) with the sine
    eigenvectors e_k(j) = sqrt(2 / (n + 1)) sin(j k pi / (n + 1)).  Steps that normalise
    v <- M v / ||M v|| and end with ||M v|| give ||M^(K+1) v0|| / ||M^K v0|| for K = iters, i.e.
    sqrt(sum mu^(2K+2) c^2 / sum mu^(2K) c^2) with c_k = e_k . v0; one step more or fewer
    changes the value by about 1e-2 here."""
    ids = np.arange(n, dtype=np.uint32)
    rowptr, col, val = [0], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                col.append(j)
                val.append(v)
        rowptr.append(len(col))
    rowptr, col, val = (np.array(rowptr, np.int32), np.array(col, np.int32), np.array(val))
    v0 = np.array([0.5 + O.fmix32(int(i) ^ 0xA5A5A5A5) / 2.0 ** 32 for i in ids])
    k = np.arange(1, n + 1)
    j = np.arange(1, n + 1)
    mu = 1.0 - np.cos(k * np.pi / (n + 1))
    E = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(k, j) * np.pi / (n + 1))
    c2 = (E @ v0) ** 2

    def closed(K):
        return np.sqrt(np.sum(mu ** (2 * K + 2) * c2) / np.sum(mu ** (2 * K) * c2))

    lam = O.power_lambda(rowptr, col, val, ids, iters)
    assert abs(lam - closed(iters)) <= 1e-13 * closed(iters)
    for other in (iters - 1, iters + 1):
        assert abs(lam - closed(other)) > 1e-6 * closed(iters)


def _dense(rowptr, col, val, n, m):
    return sps.csr_matrix((val, col, rowptr), shape=(n, m)).toarray()


@pytest.mark.parametrize("mode", [I.CONSTANT, I.LINEAR, I.QUADRATIC])
def test_prolongator_and_galerkin_dense(mode):
    """P = T - omega D^-1 A T and A_{l+1} = P^T A_l P by dense matrix products (<= 8^3)."""
    w = I.Workload("e8", I.cell_centred_grid(8), I.Domain(0.45, 0.35, taper=0.9), mode)
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=4)
    assert h.levels >= 3
    for l in range(h.levels - 1):
        n, nc = h.n(l), h.n(l + 1)
        A = _dense(*h.A(l), n, n)
        agg, _ = h.agg(l)
        T = np.zeros((n, nc))
        T[np.arange(n), agg] = 1.0
        omega = h.omega(l)
        assert omega == pytest.approx(4.0 / (3.0 * h.lam(l)), rel=1e-15)
        P_ref = T - omega * (A @ T) / np.diag(A)[:, None]
        P = _dense(*h.P(l), n, nc)
        assert np.allclose(P, P_ref, rtol=1e-13, atol=1e-13)
        Rm = _dense(*h.R(l), nc, n)
        assert np.array_equal(Rm, P.T)
        Ac = _dense(*h.A(l + 1), nc, nc)
        Ac_ref = P.T @ A @ P
        assert np.allclose(Ac, Ac_ref, rtol=1e-12, atol=1e-12 * abs(Ac_ref).max())
        # structural pattern: contains every nonzero of the dense product
        rp, cc, _ = h.A(l + 1)
        pat = np.zeros((nc, nc), bool)
        for i in range(nc):
            pat[i, cc[rp[i]:rp[i + 1]]] = True
        assert np.all(pat[np.abs(Ac_ref) > 1e-14 * abs(Ac_ref).max()])


def test_chebyshev_error_polynomial():
    """Saad Alg. 12.1: after k steps from x0 = 0 the error is T_k((theta - lam)/delta) /
    T_k(theta/delta) applied to each eigencomponent of D^-1 A."""
    w = I.cylinder_workload(8, I.LINEAR)
    op = oracle_operator(w)
    A = op.scipy(scaled=False).toarray()  # unscaled: D != I, exercises D^-1
    n = A.shape[0]
    rp = op.rowptr
    invd = 1.0 / np.diag(A)
    rng = np.random.default_rng(3)
    xs = rng.standard_normal(n)
    b = A @ xs
    lam_hat = 1.7 * np.max(np.abs(np.linalg.eigvals(invd[:, None] * A)).real) / 1.1 / 1.5
    for k in (1, 2, 3, 4):
        x = O.cheb_smooth(rp, op.col, op.aval, invd, lam_hat, b, degree=k, ratio=30.0, safety=1.1)
        hi = 1.1 * lam_hat
        lo = hi / 30.0
        th, de = (hi + lo) / 2, (hi - lo) / 2
        # D^-1 A = D^-1/2 (D^-1/2 A D^-1/2) D^1/2 with a symmetric middle factor
        Sd = np.sqrt(invd)
        lam, V = np.linalg.eigh(Sd[:, None] * A * Sd[None, :])
        Tk = np.polynomial.chebyshev.chebval((th - lam) / de, [0] * k + [1])
        Tk0 = np.polynomial.chebyshev.chebval(th / de, [0] * k + [1])
        E = (V * (Tk / Tk0)) @ V.T
        err_ref = (E @ (xs / Sd)) * Sd
        assert np.allclose(xs - x, err_ref, rtol=1e-9, atol=1e-9 * np.abs(xs).max())


def test_dense_lu_against_library_and_pivoting():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 40):
        a = rng.standard_normal((n, n))
        b = rng.standard_normal(n)
        assert np.allclose(O.dense_lu_solve(a, b), np.linalg.solve(a, b), rtol=1e-10, atol=1e-12)
    a = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])  # needs pivoting
    b = np.array([1.0, 2.0, 3.0])
    assert np.allclose(O.dense_lu_solve(a, b), np.linalg.solve(a, b), rtol=1e-14)
    with pytest.raises(ZeroDivisionError):
        O.dense_lu_solve(np.zeros((3, 3)), b)


@pytest.mark.parametrize("mode", [I.CONSTANT, I.LINEAR])
def test_vcycle_symmetric_positive(mode):
    """Sec. 3.2: same pre- and post-smoother and R = P^T give a symmetric preconditioner."""
    w = I.cylinder_workload(14, mode)
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=30)
    assert h.levels >= 3
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(op.n), rng.standard_normal(op.n)
    Mx, My = h.vcycle(x), h.vcycle(y)
    assert abs(Mx @ y - x @ My) <= 1e-12 * abs(Mx @ y)
    assert Mx @ x > 0 and My @ y > 0


def test_vcycle_single_level_is_exact_inverse():
    w = I.cylinder_workload(8, I.QUADRATIC)
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=10 ** 6)
    assert h.levels == 1
    r = np.random.default_rng(2).standard_normal(op.n)
    z = h.vcycle(r)
    assert np.allclose(z, np.linalg.solve(op.scipy().toarray(), r), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("w", [I.cylinder_workload(12, I.CONSTANT), I.pipe_workload(12, I.LINEAR),
                               I.pipe_workload(12, I.QUADRATIC),
                               I.taper_workload(10, 9, 14, I.QUADRATIC)], ids=lambda w: w.name)
def test_pcg_matches_direct_solve(w):
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=40)
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=1)
    phi, info = h.solve(rho, rtol=1e-12)
    assert info["rc"] == 0
    b = op.bfac * rho[op.node_of_row]
    x_ref = spla.spsolve(op.scipy(scaled=False).tocsc(), b)
    x = phi[op.node_of_row]
    assert np.max(np.abs(x - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
    outside = np.ones(w.grid.nbox, bool)
    outside[op.node_of_row] = False
    assert np.all(phi[outside] == 0.0)


def test_pcg_edge_cases_and_warm_start():
    w = I.pipe_workload(16, I.LINEAR)
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=100)
    zero = np.zeros(w.grid.nbox)
    phi, info = h.solve(zero, rtol=1e-8)
    assert info["rc"] == 0 and info["iters"] == 0 and np.all(phi == 0)
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=0)
    phi, info = h.solve(rho, rtol=1e-8, maxit=2)
    assert info["rc"] == 1 and info["iters"] == 2
    phi, info = h.solve(rho, rtol=1e-8)
    assert info["rc"] == 0
    cold = info["iters"]
    # exact warm start needs no iteration
    _, info2 = h.solve(rho, phi0_box=phi, rtol=1e-8)
    assert info2["iters"] == 0
    # a drifted bunch (next time step) started from the previous solution needs fewer
    # iterations (Sec. 5.2 reports about 30 % fewer)
    rho2 = I.gaussian_bunch(w.grid, (w.centre[0], w.centre[1], w.centre[2] + 0.005), w.sigma, seed=0)
    _, info3 = h.solve(rho2, phi0_box=phi, rtol=1e-8)
    assert info3["rc"] == 0 and info3["iters"] < cold


def test_iterations_roughly_grid_independent():
    its = []
    for n in (16, 32, 48):
        w = I.pipe_workload(n, I.LINEAR)
        op = oracle_operator(w)
        h = oracle_hierarchy(op, max_coarse=200)
        _, info = h.solve(I.gaussian_bunch(w.grid, w.centre, w.sigma, 0), rtol=1e-8)
        assert info["rc"] == 0
        its.append(info["iters"])
    assert max(its) <= 1.6 * min(its) and max(its) <= 30, its


def test_polak_ribiere_matches_fletcher_reeves_for_fixed_preconditioner():
    w = I.pipe_workload(16, I.LINEAR)
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=100)
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, 0)
    p0, i0 = h.solve(rho, rtol=1e-10, beta_rule=0)
    p1, i1 = h.solve(rho, rtol=1e-10, beta_rule=1)
    assert abs(i0["iters"] - i1["iters"]) <= 1
    assert np.max(np.abs(p0 - p1)) <= 1e-8 * np.max(np.abs(p0))


@pytest.mark.parametrize("mode", [I.LINEAR, I.QUADRATIC])
def test_two_level_vcycle_closed_form(mode):
    """Algorithm 1 with two levels: the error propagator of one V-cycle is
    E (I - P A_c^-1 P^T A) E with E = p(D^-1 A) the Chebyshev error polynomial, so
    z = M r = (I - E (I - P A_c^-1 P^T A) E) A^-1 r."""
    w = I.Workload("e9", I.cell_centred_grid(9), I.Domain(0.45, 0.35), mode)
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_levels=2, max_coarse=1)
    assert h.levels == 2
    n, nc = h.n(0), h.n(1)
    A = _dense(*h.A(0), n, n)
    P = _dense(*h.P(0), n, nc)
    Ac = _dense(*h.A(1), nc, nc)
    invd = 1.0 / np.diag(A)
    hi = 1.1 * h.lam(0)
    lo = hi / 30.0
    th, de = (hi + lo) / 2, (hi - lo) / 2
    lam, V = np.linalg.eig(invd[:, None] * A)
    pk = (np.polynomial.chebyshev.chebval((th - lam) / de, [0, 0, 1])
          / np.polynomial.chebyshev.chebval(th / de, [0, 0, 1]))
    E = np.real((V * pk) @ np.linalg.inv(V))
    K = np.eye(n) - P @ np.linalg.solve(Ac, P.T @ A)
    r = np.random.default_rng(5).standard_normal(n)
    z_ref = np.linalg.solve(A, r) - E @ K @ E @ np.linalg.solve(A, r)
    assert np.allclose(h.vcycle(r), z_ref, rtol=1e-9, atol=1e-10 * np.abs(z_ref).max())


def test_phase2_nodes_join_highest_key_root():
    w = I.pipe_workload(14, I.LINEAR)
    op = oracle_operator(w)
    ids = op.node_of_row.astype(np.uint32)
    root = O.mis2(op.rowptr, op.col, ids, SEED0)
    agg, nagg = O.aggregate(op.rowptr, op.col, ids, SEED0, root)
    key = _key(ids, SEED0)
    roots = np.nonzero(root)[0]
    phase1 = -np.ones(op.n, int)
    for r in roots:
        phase1[op.col[op.rowptr[r]:op.rowptr[r + 1]]] = r
    for i in np.nonzero(phase1 < 0)[0]:
        cand = {phase1[u] for u in op.col[op.rowptr[i]:op.rowptr[i + 1]] if phase1[u] >= 0}
        assert cand, i
        best = max(cand, key=lambda r: key[r])
        assert agg[i] == agg[best]


# --- cube aggregation (Sec. 3.2, the paper's "decoupled" 3^d cubes) -------------------------

def _lattice(ids, dims):
    ids = np.asarray(ids, np.int64)
    return ids % dims[0], (ids // dims[0]) % dims[1], ids // (dims[0] * dims[1])


@pytest.mark.parametrize("w", [I.pipe_workload(20, I.LINEAR), I.taper_workload(13, 12, 16),
                               I.cylinder_workload(17, I.CONSTANT)], ids=lambda w: w.name)
def test_cube_aggregates_are_the_lattice_blocks(w):
    """Every aggregate is the set of unknowns of one 3x3x3 block of the lattice: two rows share
    an aggregate exactly when their block coordinates agree; aggregates are numbered by
    ascending block index; the coarse ids decode to the block coordinates."""
    op = oracle_operator(w)
    dims = w.grid.n
    agg, root, nxt, nd = O.cube_aggregate(op.node_of_row, dims)
    i, j, k = _lattice(op.node_of_row, dims)
    blk = np.stack([i // 3, j // 3, k // 3], 1)
    assert nd == tuple((d + 2) // 3 for d in dims)
    nagg = agg.max() + 1
    assert len(nxt) == nagg and np.all(np.diff(nxt.astype(np.int64)) > 0)
    for a in range(nagg):
        members = np.flatnonzero(agg == a)
        b = blk[members]
        assert np.all(b == b[0]) and 1 <= len(members) <= 27
        ci, cj, ck = _lattice([nxt[a]], nd)
        assert (ci[0], cj[0], ck[0]) == tuple(b[0])
        assert root[members].sum() == 1 and root[members[0]] == 1  # smallest row
    # rows of one block never split across aggregates
    key = blk[:, 0] + 1000 * (blk[:, 1] + 1000 * blk[:, 2])
    for kv in np.unique(key):
        assert len(np.unique(agg[key == kv])) == 1
    # interior blocks are complete cubes: 27 members
    counts = np.bincount(agg)
    assert counts.max() == 27


def test_cube_aggregation_of_a_full_box_is_regular():
    """Semi-axes larger than the box: every lattice node is an unknown, so with sides that
    are multiples of 3 each level has exactly (n/3)^3 aggregates of 27 rows and T has 27 ones
    per column."""
    w = I.Workload("box18", I.cell_centred_grid(18), I.Domain(5.0, 5.0), I.LINEAR)
    op = oracle_operator(w)
    assert op.n == 18 ** 3
    h = oracle_hierarchy(op, max_coarse=10, aggregation=O.Hierarchy.AGG_CUBES)
    assert [h.n(l) for l in range(h.levels)] == [18 ** 3, 6 ** 3, 2 ** 3]
    for l in range(h.levels - 1):
        agg, root = h.agg(l)
        assert np.all(np.bincount(agg) == 27) and root.sum() == h.n(l + 1)


@pytest.mark.parametrize("w", [I.pipe_workload(18, I.LINEAR), I.pipe_workload(15, I.QUADRATIC),
                               I.taper_workload(13, 12, 16, I.CONSTANT)], ids=lambda w: w.name)
def test_cube_hierarchy_solves_like_a_direct_solver(w):
    op = oracle_operator(w)
    h = oracle_hierarchy(op, max_coarse=40, aggregation=O.Hierarchy.AGG_CUBES)
    assert h.status == 0 and h.levels >= 2
    # the coarse levels are the cube lattices: level l+1 has at most ceil(n_l-lattice / 27)
    agg0, _ = h.agg(0)
    assert h.n(1) == agg0.max() + 1
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=3)
    phi, info = h.solve(rho, rtol=1e-12, beta_rule=1 if w.mode == I.QUADRATIC else 0)
    assert info["rc"] == 0
    b = op.bfac * rho[op.node_of_row]
    x_ref = spla.spsolve(op.scipy(scaled=False).tocsc(), b)
    assert np.max(np.abs(phi[op.node_of_row] - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
    # Galerkin coarse operator of the cube hierarchy is P^T A P
    rp, ci, va = h.A(0)
    A0 = sps.csr_matrix((va, ci, rp), shape=(h.n(0), h.n(0)))
    P0 = sps.csr_matrix((h.P(0)[2], h.P(0)[1], h.P(0)[0]), shape=(h.n(0), h.n(1)))
    A1 = sps.csr_matrix((h.A(1)[2], h.A(1)[1], h.A(1)[0]), shape=(h.n(1), h.n(1)))
    ref = (P0.T @ A0 @ P0).toarray()
    assert np.max(np.abs(A1.toarray() - ref)) <= 1e-12 * np.max(np.abs(ref))


# --- Gauss-Seidel coarse solver (Sec. 3.2, "Coarse level solver") ---------------------------

def _key(ids, seed=0x2545F491):
    return np.array([(O.fmix32(int(v) ^ seed) << 32) | int(v) for v in ids], dtype=object)


def _random_spd(n, seed, density=0.15):
    rng = np.random.default_rng(seed)
    M = sps.random(n, n, density=density, random_state=rng, format="csr")
    A = (M + M.T).tocsr()
    A.data = -np.abs(A.data)
    A = A + sps.diags(np.asarray(abs(A).sum(1)).ravel() + 0.5)
    A = A.tocsr()
    A.sort_indices()
    return A


@pytest.mark.parametrize("seed", range(4))
def test_colouring_is_the_rounds_of_local_key_maxima(seed):
    """colour(i) = c exactly when i beats every neighbour still uncoloured at round c, and in
    every earlier round some uncoloured neighbour beat it (the synchronous-round rule)."""
    A = _random_spd(60 + 20 * seed, seed)
    ids = np.arange(A.shape[0], dtype=np.uint32) * 7 + 3
    col, k = O.colour(A.indptr, A.indices, ids)
    key = _key(ids)
    assert col.min() == 0 and col.max() == k - 1
    for i in range(A.shape[0]):
        nb = [j for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i]
        assert all(col[j] != col[i] for j in nb)  # a proper colouring
        assert all(key[i] > key[j] for j in nb if col[j] >= col[i])
        for r in range(col[i]):
            assert any(key[j] > key[i] for j in nb if col[j] >= r)


def test_symmetric_gauss_seidel_step_closed_form():
    """One step from zero equals (D+U)^-1 (b - L (D+L)^-1 b) in the colour-sorted ordering
    (L, U: strictly lower / upper parts), computed with dense triangular solves."""
    import scipy.linalg as sla
    A = _random_spd(70, 11)
    n = A.shape[0]
    ids = np.arange(n, dtype=np.uint32)
    col, k = O.colour(A.indptr, A.indices, ids)
    b = np.random.default_rng(5).standard_normal(n)
    perm = np.lexsort((np.arange(n), col))  # by colour, then row
    Ap = A.toarray()[np.ix_(perm, perm)]
    bp = b[perm]
    Lw = np.tril(Ap)  # D + L
    Up = np.triu(Ap)  # D + U
    xh = sla.solve_triangular(Lw, bp, lower=True)
    x1 = sla.solve_triangular(Up, bp - np.tril(Ap, -1) @ xh, lower=False)
    got = O.sgs(A.indptr, A.indices, A.data, col, k, 1, b)
    ref = np.empty(n)
    ref[perm] = x1
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # many steps converge to the solution of A x = b
    x = O.sgs(A.indptr, A.indices, A.data, col, k, 200, b)
    assert np.max(np.abs(A @ x - b)) <= 1e-10 * np.max(np.abs(b))


@pytest.mark.parametrize("w", [I.pipe_workload(20, I.LINEAR), I.cylinder_workload(16, I.CONSTANT)],
                         ids=lambda w: w.name)
def test_gauss_seidel_coarse_solver_in_the_hierarchy(w):
    op = oracle_operator(w)
    hl = oracle_hierarchy(op, max_coarse=200)
    hg = oracle_hierarchy(op, max_coarse=200, coarse_solver=O.Hierarchy.COARSE_GS, coarse_sweeps=3)
    assert hg.status == 0 and hg.colours() is not None and hl.colours() is None
    c, k = hg.colours()
    A = hg.A(hg.levels - 1)
    for i in range(len(c)):
        nb = A[1][A[0][i]:A[0][i + 1]]
        assert all(c[j] != c[i] for j in nb if j != i)
    # the V-cycle stays symmetric: u'M v = v'M u
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(op.n), rng.standard_normal(op.n)
    mu, mv = hg.vcycle(u), hg.vcycle(v)
    assert abs(v @ mu - u @ mv) <= 1e-11 * abs(v @ mu)
    # three steps give about the quality of the exact coarse solve (the paper's finding)
    rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=2)
    _, il = hl.solve(rho, rtol=1e-8)
    phi, ig = hg.solve(rho, rtol=1e-8)
    assert ig["rc"] == 0 and ig["iters"] <= il["iters"] + 3
    b = op.bfac * rho[op.node_of_row]
    x_ref = spla.spsolve(op.scipy(scaled=False).tocsc(), b)
    assert np.max(np.abs(phi[op.node_of_row] - x_ref)) <= 1e-6 * np.max(np.abs(x_ref))
