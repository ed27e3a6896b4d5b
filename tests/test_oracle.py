"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a brute-force computation on a tiny input, a textbook routine on the
same matrix, or a value the paper prints (tests/golden/).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy import stats

from oracle import hss_oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ tree
@pytest.mark.parametrize("n,leaf,nleaves,sizes", [
    (2000, 128, 16, {125}),
    (20000, 256, 128, {156, 157}),
    (60000, 512, 128, {468, 469}),
    (1000, 1000, 1, {1000}),
])
def test_tree_bisection_sizes(n, leaf, nleaves, sizes):
    nodes = O.bisection_tree(n, leaf)
    leaves = [nd for nd in nodes if nd.is_leaf]
    assert len(leaves) == nleaves
    assert {nd.size for nd in leaves} == sizes
    # leaves tile [0, n) in order; children partition the parent (Section 2.1)
    assert sorted((nd.lo, nd.hi) for nd in leaves)[0][0] == 0
    cover = np.zeros(n, int)
    for nd in leaves:
        cover[nd.lo:nd.hi] += 1
    assert (cover == 1).all()
    for nd in nodes:
        if nd.children:
            a, b = (nodes[c] for c in nd.children)
            assert a.lo == nd.lo and a.hi == b.lo and b.hi == nd.hi
            assert a.size == nd.size // 2


# ------------------------------------------------------------ random R
def test_bf16_rounding_closed_form():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7 + 2.0 ** -9,
                  -3.0 - 2.0 ** -7, 0.0, 255.5, 1.0 + 2.0 ** -8 + 2.0 ** -30])
    want = np.array([1.0, 1.0, 1.0 + 2 * 2.0 ** -7, 1.0 + 2.0 ** -7,
                     -3.0, 0.0, 256.0, 1.0 + 2.0 ** -7])
    # ties go to the even 8-bit significand; 255.5 -> 256 (8 bits of 255.5 = 255.5 -> tie -> 256)
    np.testing.assert_array_equal(O.round_to_bf16(x), want)


def test_splitmix64_known_answers():
    # the first five outputs of SplitMix64 (Steele, Lea, Flood 2014) seeded
    # with 1234567, the known-answer values that accompany reference
    # implementations of the generator
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    got = O.splitmix64(1234567, np.arange(1, 6, dtype=np.uint64))
    assert [int(x) for x in got] == want


def test_random_matrix_is_gaussian_bf16():
    R = O.gaussian_bf16(1234, 4000, 0, 64)
    # every value is exactly representable in bfloat16 (8 significant bits)
    f, _ = np.frexp(R)
    assert np.all(f * 256 == np.round(f * 256))
    # standard normal: mean 0, variance 1, KS test against N(0,1)
    assert abs(R.mean()) < 0.01
    assert abs(R.var() - 1.0) < 0.01
    assert stats.kstest(R.ravel()[:200000], "norm").pvalue > 1e-4
    # columns are independent: sample correlation is O(1/sqrt(n))
    C = np.corrcoef(R.T)
    assert np.abs(C - np.eye(64)).max() < 5.0 / math.sqrt(4000)


def test_random_matrix_columns_extend_in_place():
    # adaptive sampling appends columns: column j never depends on d
    a = O.gaussian_bf16(7, 300, 0, 48)
    b = O.gaussian_bf16(7, 300, 16, 48)
    np.testing.assert_array_equal(a[:, 16:], b)
    assert not np.array_equal(O.gaussian_bf16(8, 300, 0, 48), a)


# ---------------------------------------------------------------- the ID
def _greedy_pivots(Y, kmax):
    """Brute-force greedy column selection: pick the column with the largest
    residual after least-squares projection on the columns already picked."""
    chosen, res = [], []
    m = Y.shape[1]
    for _ in range(kmax):
        best, bestn = -1, -1.0
        for j in range(m):
            if j in chosen:
                continue
            if chosen:
                c, *_ = np.linalg.lstsq(Y[:, chosen], Y[:, j], rcond=None)
                r = Y[:, j] - Y[:, chosen] @ c
            else:
                r = Y[:, j]
            nr = np.linalg.norm(r)
            if nr > bestn + 1e-12 * max(1.0, bestn):
                best, bestn = j, nr
        chosen.append(best)
        res.append(bestn)
    return chosen, np.array(res)


# ------------------------------------------------------- leaf local samples
@pytest.mark.parametrize("n_extra", [0, 4])
def test_leaf_local_samples_match_block_diagonal_removal(n_extra):
    """Algorithm 1's leaf samples S^r(I,:) - D R(I,:) and S^c(I,:) - D^T R(I,:)
    for every leaf equal (A - blockdiag(D)) R and (A - blockdiag(D))^T R with
    the block diagonal assembled independently (scipy.linalg.block_diag of
    the leaf blocks).  A is unsymmetric, so a D / D^T or row / column slip
    shows; n = 8 leaf + 4 puts leaves at two depths with uneven sizes."""
    leaf = 24
    n = 8 * leaf + n_extra
    rng = np.random.default_rng(11 + n_extra)
    A = rng.standard_normal((n, n)) + np.triu(rng.standard_normal((n, n)), 1) * 3.0
    R = rng.standard_normal((n, 7))
    nodes = O.bisection_tree(n, leaf)
    leaves = sorted((nd for nd in nodes if nd.is_leaf), key=lambda x: x.lo)
    assert (len({nd.size for nd in leaves}) > 1) == (n_extra > 0)
    assert (len({nd.depth for nd in leaves}) > 1) == (n_extra > 0)
    Dblk = sla.block_diag(*[A[nd.lo:nd.hi, nd.lo:nd.hi] for nd in leaves])
    assert Dblk.shape == (n, n)
    Sr, Sc = O.leaf_local_samples(A, R, nodes)
    np.testing.assert_allclose(Sr, (A - Dblk) @ R, rtol=0, atol=1e-12 * np.abs(A).sum())
    np.testing.assert_allclose(Sc, (A - Dblk).T @ R, rtol=0, atol=1e-12 * np.abs(A).sum())
    # and entry by entry from the definition, on a few rows
    for i in (0, n // 3, n - 1):
        lf = next(nd for nd in leaves if nd.lo <= i < nd.hi)
        outside = np.r_[0:lf.lo, lf.hi:n]
        np.testing.assert_allclose(Sr[i], A[i, outside] @ R[outside], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Sc[i], A[outside, i] @ R[outside], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_id_pivots_match_bruteforce_greedy(seed):
    rng = np.random.default_rng(seed)
    d, m = 7, 6
    Y = rng.standard_normal((d, m)) * np.array([1.0, 5.0, 0.3, 2.0, 0.01, 1.5])
    ref, res = _greedy_pivots(Y, m)
    idd = O.interpolative_decomposition(Y, 1e-14)
    assert idd.k == m
    assert list(idd.perm) == ref
    # |R_ii| is the residual norm of the i-th pivot column
    np.testing.assert_allclose(idd.rdiag, res, rtol=1e-10)


@pytest.mark.parametrize("r", [0, 1, 3, 9])
def test_id_exact_rank_and_reconstruction(r):
    rng = np.random.default_rng(r)
    d, m = 30, 20
    Y = rng.standard_normal((d, r)) @ rng.standard_normal((r, m))
    idd = O.interpolative_decomposition(Y, 1e-12)
    assert idd.k == r
    X = idd.basis().T                      # k x m,  Y ~= Y(:, J) X
    np.testing.assert_allclose(Y[:, idd.J] @ X, Y, atol=1e-11 * max(1.0, np.abs(Y).max()))
    # X restricted to J is the identity (the "I" block of U = Pi [I; E])
    np.testing.assert_array_equal(X[:, idd.J], np.eye(r))


def test_id_truncation_rule():
    # singular values 1, 1e-3, 1e-6, 1e-9: rank at rtol is the number above it
    rng = np.random.default_rng(5)
    Q1, _ = np.linalg.qr(rng.standard_normal((40, 4)))
    Q2, _ = np.linalg.qr(rng.standard_normal((25, 4)))
    Y = Q1 @ np.diag([1.0, 1e-3, 1e-6, 1e-9]) @ Q2.T
    for rtol, k in [(1e-2, 1), (1e-4, 2), (1e-7, 3), (1e-11, 4)]:
        idd = O.interpolative_decomposition(Y, rtol)
        assert idd.k == k
        assert idd.rdiag[k - 1] > rtol * idd.rdiag[0]
        if k < idd.rdiag.size:
            assert idd.rdiag[k] <= rtol * idd.rdiag[0]
    # absolute floor
    assert O.interpolative_decomposition(Y, 1e-11, atol=1e-4).k == 2
    assert O.interpolative_decomposition(np.zeros((5, 4)), 1e-6).k == 0


# ------------------------------------------------------------ compression
@pytest.mark.parametrize("n,leaf,rank", [(512, 64, 6), (700, 50, 4), (1024, 64, 12)])
def test_compress_recovers_known_ranks_exactly(n, leaf, rank):
    A, true_ranks = W.random_hss(n, leaf, rank, seed=n + rank, diag_shift=10.0)
    h = O.compress(A, 1e-14, leaf_size=leaf, d0=rank + 12, d_step=8, seed=11)
    for nd in h.nodes:
        if nd.id == 0:
            continue
        kr, kc = h.data[nd.id].idr.k, h.data[nd.id].idc.k
        assert (kr, kc) == (true_ranks[(nd.lo, nd.hi)],) * 2
    H = O.to_dense(h)
    assert np.linalg.norm(A - H) / np.linalg.norm(A) <= 1e-12


def test_compress_adaptive_restart_reaches_exact_ranks():
    A, true_ranks = W.random_hss(1024, 64, 20, seed=4, diag_shift=20.0)
    h = O.compress(A, 1e-13, leaf_size=64, d0=16, d_step=8, oversample_p=10, seed=7)
    assert h.passes > 1                      # started with too few samples
    assert h.d >= 20 + 10                    # k <= d - p at every compressed node
    assert set(h.ranks().values()) == {(20, 20)}
    assert all(dd.state == O.COMPRESSED for dd in h.data)
    assert np.linalg.norm(A - O.to_dense(h)) / np.linalg.norm(A) <= 1e-12


def test_simple_toeplitz_rank_two_matches_paper_table():
    # Table 3: SimpleToeplitz (a_ii = n^2, a_ij = i - j) has max HSS rank 2 at
    # eps = 1e-8 and 1e-6; its off-diagonal blocks (entries i - j) have rank 2.
    golden = {}
    with open(os.path.join(GOLDEN, "simple_toeplitz_table3.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                eps, r = line.split()
                golden[float(eps)] = int(r)
    A = W.simple_toeplitz(1200).numpy()
    for eps, r in golden.items():
        h = O.compress(A, eps, leaf_size=64, d0=16, d_step=8, seed=3)
        assert h.max_rank() == r
        assert np.linalg.norm(A - O.to_dense(h)) / np.linalg.norm(A) <= 1e-12


def test_hankel_blocks_against_dense_svd():
    # Every Hankel block A(I_t, I_0 \ I_t) is reproduced by H to O(rtol), and
    # the ID rank is not below the SVD rank at a tolerance well above rtol.
    n, leaf, rtol = 384, 48, 1e-8
    A = W.toeplitz_inv_distance(n).numpy()
    h = O.compress(A, rtol, leaf_size=leaf, d0=40, d_step=16, seed=2)
    H = O.to_dense(h)
    nA = np.linalg.norm(A, 2)
    for nd in h.nodes:
        if nd.id == 0:
            continue
        rest = np.r_[0:nd.lo, nd.hi:n]
        blk = A[nd.lo:nd.hi][:, rest]
        s = np.linalg.svd(blk, compute_uv=False)
        assert np.linalg.norm(blk - H[nd.lo:nd.hi][:, rest], 2) <= 100 * rtol * nA
        kr, kc = h.data[nd.id].idr.k, h.data[nd.id].idc.k
        assert kr >= int((s > 1e3 * rtol * s[0]).sum())
        assert kr <= int((s > 1e-4 * rtol * s[0]).sum()) + 2
        sc = np.linalg.svd(A[rest][:, nd.lo:nd.hi], compute_uv=False)
        assert kc >= int((sc > 1e3 * rtol * sc[0]).sum())


def test_compress_config1_toeplitz_accuracy():
    A = W.toeplitz_inv_distance(2000).numpy()
    h = O.compress(A, 1e-6, leaf_size=128, d0=64, d_step=32, seed=1001)
    assert np.linalg.norm(A - O.to_dense(h)) / np.linalg.norm(A) <= 2e-6


def test_single_node_tree_and_zero_rank():
    A = np.random.default_rng(1).standard_normal((50, 50)) + 10 * np.eye(50)
    h = O.compress(A, 1e-6, leaf_size=64)
    np.testing.assert_array_equal(O.to_dense(h), A)
    x = np.ones(50)
    np.testing.assert_allclose(O.matvec(h, x), A @ x, rtol=1e-13)
    O.ulv_factor(h)
    np.testing.assert_allclose(O.ulv_solve(h, x), np.linalg.solve(A, x), rtol=1e-10)
    # block-diagonal matrix: every off-diagonal block is zero -> rank 0 everywhere
    B = sla.block_diag(*[np.eye(32) * (i + 2) for i in range(8)])
    hb = O.compress(B, 1e-6, leaf_size=32, d0=16, d_step=8)
    assert set(hb.ranks().values()) == {(0, 0)}
    np.testing.assert_allclose(O.to_dense(hb), B, atol=0)
    O.ulv_factor(hb)
    b = np.arange(256.0)
    np.testing.assert_allclose(O.ulv_solve(hb, b), np.linalg.solve(B, b), rtol=1e-12)


def test_full_rank_leaves_when_samples_cover_them():
    # random dense matrix: no low-rank structure; with d >= m no node fails and
    # the ID keeps every row (k = m, E empty) -- still an exact representation
    A = np.random.default_rng(3).standard_normal((128, 128)) + 20 * np.eye(128)
    h = O.compress(A, 1e-12, leaf_size=16, d0=80, d_step=16, seed=1)
    leaves = [nd for nd in h.nodes if nd.is_leaf]
    assert all(h.data[nd.id].idr.k == 16 for nd in leaves)
    assert np.linalg.norm(A - O.to_dense(h)) / np.linalg.norm(A) <= 1e-12
    O.ulv_factor(h)
    b = np.random.default_rng(4).standard_normal((128, 2))
    np.testing.assert_allclose(O.ulv_solve(h, b), np.linalg.solve(A, b), rtol=1e-8, atol=1e-10)


def test_rank_cap_raises():
    A = np.random.default_rng(3).standard_normal((256, 256))
    with pytest.raises(O.RankCapError):
        O.compress(A, 1e-12, leaf_size=64, d0=16, d_step=16, d_max=32)


# ---------------------------------------------------- product and solve
@pytest.fixture(scope="module")
def hss_toeplitz():
    A = W.toeplitz_inv_distance(640).numpy() + np.triu(np.ones((640, 640))) * 0.01
    h = O.compress(A, 1e-9, leaf_size=40, d0=32, d_step=16, seed=5)
    return A, h


def test_matvec_equals_dense_product(hss_toeplitz):
    A, h = hss_toeplitz
    H = O.to_dense(h)
    X = np.random.default_rng(0).standard_normal((640, 5))
    np.testing.assert_allclose(O.matvec(h, X), H @ X, rtol=0, atol=1e-12 * np.abs(H @ X).max())
    # and H approximates the (unsymmetric) input
    assert np.linalg.norm(O.matvec(h, X) - A @ X) / np.linalg.norm(A @ X) < 1e-7


def test_ulv_solve_matches_dense_lu(hss_toeplitz):
    A, h = hss_toeplitz
    H = O.to_dense(h)
    O.ulv_factor(h)
    B = np.random.default_rng(1).standard_normal((640, 3))
    X = O.ulv_solve(h, B)
    Xd = sla.lu_solve(sla.lu_factor(H), B)
    np.testing.assert_allclose(X, Xd, rtol=0, atol=1e-10 * np.abs(Xd).max())
    # Omega U = [0; I] at every non-root node (Section 2.4)
    for nd in h.nodes:
        if nd.id == 0:
            continue
        idr = h.data[nd.id].idr
        OU = O._omega(idr) @ idr.basis()
        m, k = idr.perm.size, idr.k
        np.testing.assert_allclose(OU, np.vstack([np.zeros((m - k, k)), np.eye(k)]), atol=1e-13)


def test_ulv_two_level_by_hand():
    # one-level tree (root + 2 leaves): the solve is Section 2.5's five steps;
    # compare against the dense solve of the assembled 2x2 block HSS matrix.
    A, _ = W.random_hss(96, 48, 5, seed=9, diag_shift=8.0)
    h = O.compress(A, 1e-13, leaf_size=48, d0=24, d_step=8, seed=1)
    assert len(h.nodes) == 3
    O.ulv_factor(h)
    b = np.random.default_rng(2).standard_normal(96)
    np.testing.assert_allclose(A @ O.ulv_solve(h, b), b, atol=1e-9)


# --------------------------------------------- Schur complement input family
@pytest.mark.parametrize("k", [2, 3, 5, 6])
def test_laplacian_schur_closed_form_matches_sparse_elimination(k):
    """The closed form equals A22 - A21 A11^{-1} A12 of the explicit 7-point
    Laplacian on a k x k x (2k+1) grid (Dirichlet), middle plane last."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nz = 2 * k + 1

    def lap1(m):
        return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])

    I = sp.identity(k)
    Lxy = sp.kron(lap1(k), I) + sp.kron(I, lap1(k))
    L = sp.kron(lap1(nz), sp.identity(k * k)) + sp.kron(sp.identity(nz), Lxy)
    L = L.tocsc()
    mid = np.arange(k * k) + k * k * k          # plane z = k
    rest = np.setdiff1d(np.arange(nz * k * k), mid)
    A11 = L[rest][:, rest]
    A12 = L[rest][:, mid].toarray()
    S = L[mid][:, mid].toarray() - L[mid][:, rest] @ spla.spsolve(A11, A12)
    Sc = W.laplacian_schur(k, dtype=np.float64).numpy()
    np.testing.assert_allclose(Sc, S, atol=1e-12)
    # closed-form eigenvalues and solve
    ev = np.sort(W.laplacian_schur_eigs(k).ravel())
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(S)), ev, atol=1e-12)


# ------------------------------------------------------------- comb trees
def _oracle_nodes(n, splits):
    return [O.Node(i, lo, hi, dep, par, ch)
            for i, (lo, hi, dep, par, ch) in enumerate(W.split_intervals(n, splits))]


def test_split_list_of_bisection_reproduces_the_bisection_tree():
    """The breadth-first split list format (hss_opts.tree) describes the
    bisection tree of Section 2.1 exactly when its splits are the midpoints."""
    n, leaf = 1000, 60
    ref = O.bisection_tree(n, leaf)
    splits = [nd.lo + nd.size // 2 if not nd.is_leaf else -1 for nd in ref]
    got = _oracle_nodes(n, splits)
    assert [(a.lo, a.hi, a.depth, a.parent, a.children) for a in got] == \
        [(b.lo, b.hi, b.depth, b.parent, tuple(b.children)) for b in ref]


def test_comb_tree_compression_invariants():
    """A comb tree (Section 4's unbalanced tree): every non-leaf splits off a
    leaf.  The compressed form still satisfies the invariants that pin the
    bisection case: matvec equals the dense H, H approximates A at the
    tolerance, and the ULV solve equals a dense LU solve of H."""
    n, leaf = 600, 50
    A = W.toeplitz_inv_distance(n).numpy() + np.triu(np.ones((n, n))) * 0.01
    splits = W.comb_tree_splits(n, leaf)
    nodes = _oracle_nodes(n, splits)
    assert max(nd.depth for nd in nodes) == n // leaf - 1
    h = O.compress(A, 1e-9, d0=32, d_step=16, seed=5, tree=nodes)
    H = O.to_dense(h)
    assert np.linalg.norm(A - H) / np.linalg.norm(A) < 1e-7
    X = np.random.default_rng(0).standard_normal((n, 3))
    np.testing.assert_allclose(O.matvec(h, X), H @ X, rtol=0, atol=1e-12 * np.abs(H @ X).max())
    O.ulv_factor(h)
    Xs = O.ulv_solve(h, X)
    np.testing.assert_allclose(Xs, sla.lu_solve(sla.lu_factor(H), X), rtol=0,
                               atol=1e-10 * np.abs(Xs).max())
    # every off-diagonal block A(I_t, rest) of a comb tree has the rank the ID
    # found, to the tolerance (checked against its singular values)
    for nd in nodes[1:]:
        rest = np.r_[0:nd.lo, nd.hi:n]
        sv = np.linalg.svd(A[nd.lo:nd.hi][:, rest], compute_uv=False)
        kr = h.data[nd.id].idr.k
        assert kr >= int(np.sum(sv > 1e-7 * sv[0]))


def test_symmetric_compression_repeats_the_row_side():
    """symmetric=True on a symmetric matrix (Gaussian kernel, with adaptive
    restarts): the column side is the row side (same ID, V = U, I^c = I^r),
    so the reconstruction is symmetric to rounding; the ranks, passes and
    error match the general compression of the same matrix, whose column
    samples A^T R equal A R in exact arithmetic (Section 2.2 with one R)."""
    n, leaf, rtol = 800, 50, 1e-6
    pts = W.points_unit_cube(n, 7)
    pts = pts[W.rcb_order(pts, leaf)]
    A = W.gaussian_kernel(pts, 0.2, 1.0, dtype=np.float64).numpy()
    assert np.array_equal(A, A.T)
    g = O.compress(A, rtol, leaf_size=leaf, d0=16, d_step=16, seed=3)
    sy = O.compress(A, rtol, leaf_size=leaf, d0=16, d_step=16, seed=3, symmetric=True)
    assert sy.passes > 1 and abs(sy.passes - g.passes) <= 1
    for nd in sy.nodes[1:]:
        me = sy.data[nd.id]
        assert me.idc is me.idr and np.array_equal(me.Ic, me.Ir)
        kr, kc = g.ranks()[nd.id]
        assert abs(me.idr.k - kr) <= 1 and abs(me.idr.k - kc) <= 1
    H = O.to_dense(sy)
    assert np.linalg.norm(H - H.T) <= 1e-13 * np.linalg.norm(H)
    e_gen = np.linalg.norm(O.to_dense(g) - A) / np.linalg.norm(A)
    e_sym = np.linalg.norm(H - A) / np.linalg.norm(A)
    assert e_sym <= 2 * max(rtol, e_gen)


def test_symmetric_flag_on_an_unsymmetric_matrix_misses_it():
    """The flag is a promise, not a check: on a matrix whose off-diagonal
    blocks have column spaces unlike their row spaces (T + X Y^T, X and Y
    independent), the symmetric path's V = U cannot hold the row spaces and
    the compression misses A, while the general path meets its tolerance."""
    n, leaf = 400, 50
    rng = np.random.default_rng(8)
    i = np.arange(n)
    A = 1.0 / (1.0 + np.abs(i[:, None] - i[None, :]))
    K = rng.standard_normal((n, 6)) @ rng.standard_normal((6, n))
    A = A + K / np.linalg.norm(K) * np.linalg.norm(A)
    sy = O.compress(A, 1e-8, leaf_size=leaf, d0=32, d_step=16, seed=2, symmetric=True)
    g = O.compress(A, 1e-8, leaf_size=leaf, d0=32, d_step=16, seed=2)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(O.to_dense(g) - A) <= 1e-6 * nA
    assert np.linalg.norm(O.to_dense(sy) - A) >= 0.1 * nA
