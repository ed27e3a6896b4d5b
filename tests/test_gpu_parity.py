"""GPU path vs the CPU oracle, element by element where the result is unique.

Tolerances (from the arithmetic):
* R: bit-exact except where the FP64 Box-Muller value sits on a bfloat16
  rounding boundary (at most one bfloat16 ulp, at most 1e-6 of the entries).
* sampling: FP64 |dS| <= 1e-12 (|A||R|); FP32 |dS| <= 4 n eps32 (|A||R|).
* ID: same rank (+-1 only on a tie within 1e-12 of the threshold), same pivots,
  E to 1e-9 relative.
* compression (not unique: pivots and ranks may move near eps): ranks within
  +-2 of the oracle, ||A - H||_F / ||A||_F <= 2 max(rtol, e_oracle) where
  e_oracle is the oracle's own error at the same eps (the paper's stopping
  test is local and relative, so the global error of the method itself can
  exceed rtol), matvec vs the oracle's H x within 4 rtol, solve residual
  <= 10x the oracle's.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hss_oracle as O  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1503_05464_gb300 as pkg
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    return pkg


DEV = "cuda:0"


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# -------------------------------------------------------------------- R
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_random_matrix_matches_oracle(P, dtype):
    n, c0, c1 = 3001, 5, 77
    R = torch.zeros((n, 80), dtype=dtype, device=DEV)
    P.hss_random_gaussian(1234, n, c0, c1, R)
    got = R.cpu().numpy().astype(np.float64)
    want = O.gaussian_bf16(1234, n, c0, c1)
    assert np.all(got[:, :c0] == 0) and np.all(got[:, c1:] == 0)
    diff = got[:, c0:c1] != want
    assert diff.sum() <= max(1, int(1e-6 * want.size))
    if diff.any():   # a boundary flip is one bfloat16 ulp
        ulp = np.ldexp(1.0, np.frexp(want[diff])[1] - 8)
        assert np.all(np.abs(got[:, c0:c1][diff] - want[diff]) <= ulp)


def test_random_matrix_large_sample_matches_oracle(P):
    # a full-size block of R (2.56M entries): the FP32 evaluation with its
    # FP64 fallback near bfloat16 rounding midpoints gives the FP64 values
    n, c = 20000, 128
    R = torch.zeros((n, c), dtype=torch.float32, device=DEV)
    P.hss_random_gaussian(1003, n, 0, c, R)
    got = R.cpu().numpy().astype(np.float64)
    want = O.gaussian_bf16(1003, n, 0, c)
    assert int((got != want).sum()) <= max(1, int(1e-6 * want.size))


# ------------------------------------------------------------- sampling
@pytest.mark.parametrize("n,leaf,dtype,c0,c1", [
    (777, 50, torch.float64, 0, 70),
    (1000, 125, torch.float32, 0, 64),
    (1283, 100, torch.float32, 33, 161),     # ragged n, ragged chunk, column offset
    (300, 1000, torch.float64, 0, 20),       # single leaf: everything masked
])
def test_fused_sampling_matches_oracle(P, n, leaf, dtype, c0, c1):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 5 * np.eye(n)
    A[: n // 3] *= 3.0                        # unsymmetric, S^c != S^r
    At = torch.tensor(A, dtype=dtype, device=DEV)
    A64 = At.cpu().numpy().astype(np.float64)
    R = torch.zeros((n, c1), dtype=dtype, device=DEV)
    P.hss_random_gaussian(99, n, 0, c1, R)
    Sr = torch.full((n, c1), 7.0, dtype=dtype, device=DEV)
    Sc = torch.full((n, c1), 7.0, dtype=dtype, device=DEV)
    nodes = O.bisection_tree(n, leaf)
    starts = sorted(nd.lo for nd in nodes if nd.is_leaf) + [n]
    P.hss_sample(At, R, c0, c1, Sr, Sc, leaf_starts=starts)
    torch.cuda.synchronize()
    R64 = R.cpu().numpy().astype(np.float64)
    wr, wc = O.leaf_local_samples(A64, R64[:, c0:c1], nodes)
    mask = np.ones((n, n))
    for nd in nodes:
        if nd.is_leaf:
            mask[nd.lo:nd.hi, nd.lo:nd.hi] = 0
    br = (np.abs(A64) * mask) @ np.abs(R64[:, c0:c1])
    bc = (np.abs(A64) * mask).T @ np.abs(R64[:, c0:c1])
    tol = 1e-12 if dtype == torch.float64 else 4 * n * 2.0 ** -24
    gr = Sr.cpu().numpy().astype(np.float64)
    gc = Sc.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gr[:, c0:c1] - wr) <= tol * br + 1e-300)
    assert np.all(np.abs(gc[:, c0:c1] - wc) <= tol * bc + 1e-300)
    assert np.all(gr[:, :c0] == 7.0) and np.all(gc[:, :c0] == 7.0)


# representation error of A in each sampling mode (R is bfloat16-exact)
MODE_REL = {"tf32": 2.0 ** -11, "bf16x2": 2.0 ** -16, "bf16x3": 2.0 ** -23}


@pytest.mark.parametrize("mode", ["tf32", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("n,leaf,c0,c1,pad", [
    (1000, 125, 0, 64, 0), (1283, 100, 33, 161, 0), (517, 64, 0, 128, 0),
    # rows 16-byte aligned: the split modes run on tcgen05 (several column
    # tiles and panels with ragged tails, several sweeps of <= 128 columns,
    # panels split between CTAs, tiny and strided inputs)
    (1284, 100, 33, 161, 0), (516, 64, 0, 128, 0), (2052, 200, 0, 200, 0), (12, 4, 0, 16, 0),
    (300, 40, 5, 37, 0), (4100, 300, 0, 96, 0), (777, 90, 0, 80, 5)])
def test_tensor_core_sampling_matches_oracle(P, mode, n, leaf, c0, c1, pad):
    rng = np.random.default_rng(n + len(mode))
    A = rng.standard_normal((n, n)) * np.exp(rng.standard_normal((n, n)))   # wide magnitudes
    A[: n // 3] *= 3.0
    if pad:    # a view with a leading dimension n + pad rounded up to a multiple of 4
        ld = (n + pad + 3) // 4 * 4
        big = torch.zeros((n, ld), dtype=torch.float32, device=DEV)
        big[:, :n] = torch.tensor(A, dtype=torch.float32, device=DEV)
        At = big[:, :n]
    else:
        At = torch.tensor(A, dtype=torch.float32, device=DEV)
    A64 = At.cpu().numpy().astype(np.float64)
    R = torch.zeros((n, c1), dtype=torch.float32, device=DEV)
    P.hss_random_gaussian(5, n, 0, c1, R)
    Sr = torch.full((n, c1), 7.0, device=DEV)
    Sc = torch.full((n, c1), 7.0, device=DEV)
    nodes = O.bisection_tree(n, leaf)
    starts = sorted(nd.lo for nd in nodes if nd.is_leaf) + [n]
    P.hss_sample(At, R, c0, c1, Sr, Sc, leaf_starts=starts, mode=mode)
    torch.cuda.synchronize()
    R64 = R.cpu().numpy().astype(np.float64)
    wr, wc = O.leaf_local_samples(A64, R64[:, c0:c1], nodes)
    mask = np.ones((n, n))
    for nd in nodes:
        if nd.is_leaf:
            mask[nd.lo:nd.hi, nd.lo:nd.hi] = 0
    br = (np.abs(A64) * mask) @ np.abs(R64[:, c0:c1])
    bc = (np.abs(A64) * mask).T @ np.abs(R64[:, c0:c1])
    tol = MODE_REL[mode] + 4 * n * 2.0 ** -24
    gr = Sr.cpu().numpy().astype(np.float64)
    gc = Sc.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gr[:, c0:c1] - wr) <= tol * br)
    assert np.all(np.abs(gc[:, c0:c1] - wc) <= tol * bc)
    assert np.all(gr[:, :c0] == 7.0) and np.all(gc[:, :c0] == 7.0)
    # the split modes must actually be more accurate than one bfloat16 term
    if mode == "bf16x3":
        assert np.abs(gr[:, c0:c1] - wr).max() <= 1e-5 * np.abs(wr).max()


def test_tensor_core_sampling_accuracy_on_schur_complement(P):
    """bf16x3 samples of the Schur complement of the 7-point Laplacian
    (n = 10000, leaf 256, 128 columns) against the oracle's FP64 leaf
    samples: relative Frobenius error <= 6e-7 in both products.  The
    tensor core's FP32 accumulation runs over at most 24 MMAs in either
    product; with the row product accumulated over 16-tile groups its error
    was 1.65e-6 here (plain FP32 SIMT sampling: 1.1e-7 / 2.0e-7), enough to
    raise the ranks at rtol 1e-6 from 691 to 886."""
    At = W.laplacian_schur(100, dtype=np.float32, device=DEV)
    n, c = At.shape[0], 128
    nodes = O.bisection_tree(n, 256)
    starts = sorted(nd.lo for nd in nodes if nd.is_leaf) + [n]
    R = torch.zeros((n, c), dtype=torch.float32, device=DEV)
    P.hss_random_gaussian(11, n, 0, c, R)
    Sr = torch.empty((n, c), device=DEV)
    Sc = torch.empty((n, c), device=DEV)
    P.hss_sample(At, R, 0, c, Sr, Sc, leaf_starts=starts, mode="bf16x3")
    torch.cuda.synchronize()
    wr, wc = O.leaf_local_samples(At.cpu().numpy(), R.cpu().numpy(), nodes)
    er = _rel(Sr.cpu().numpy().astype(np.float64), wr)
    ec = _rel(Sc.cpu().numpy().astype(np.float64), wc)
    assert er <= 6e-7 and ec <= 6e-7, (er, ec)


@pytest.mark.parametrize("mode", ["tf32", "bf16x2", "bf16x3"])
def test_tensor_core_sampling_repeats_identically(P, mode):
    # many CTAs, a ragged tail and a masked leaf diagonal: every repeat must
    # give the same bits (a hand-off race in the staging pipeline shows up as
    # an occasional wrong 16-byte chunk of one tile in both products)
    n, c = 4100, 96
    rng = np.random.default_rng(11)
    At = torch.tensor(rng.standard_normal((n, n)), dtype=torch.float32, device=DEV)
    R = torch.zeros((n, c), device=DEV)
    P.hss_random_gaussian(5, n, 0, c, R)
    starts = list(range(0, n, 300)) + [n]
    ref = None
    for _ in range(16):
        Sr = torch.empty((n, c), device=DEV)
        Sc = torch.empty((n, c), device=DEV)
        P.hss_sample(At, R, 0, c, Sr, Sc, leaf_starts=starts, mode=mode)
        if ref is None:
            ref = (Sr, Sc)
        else:
            assert torch.equal(Sr, ref[0]) and torch.equal(Sc, ref[1])


@pytest.mark.parametrize("mode", ["native", "tf32", "bf16x2", "bf16x3"])
def test_row_samples_alone_equal_the_row_part(P, mode):
    # Sc = None forms S^r only (the symmetric path; the tensor-core kernel
    # skips the column product): the same bits as the row part of a full call
    n, c = 4100, 96
    rng = np.random.default_rng(12)
    At = torch.tensor(rng.standard_normal((n, n)), dtype=torch.float32, device=DEV)
    R = torch.zeros((n, c), device=DEV)
    P.hss_random_gaussian(6, n, 0, c, R)
    starts = list(range(0, n, 300)) + [n]
    Sr = torch.empty((n, c), device=DEV)
    Sc = torch.empty((n, c), device=DEV)
    P.hss_sample(At, R, 0, c, Sr, Sc, leaf_starts=starts, mode=mode)
    Sr1 = torch.full((n, c), 5.0, device=DEV)
    P.hss_sample(At, R, 0, c, Sr1, None, leaf_starts=starts, mode=mode)
    torch.cuda.synchronize()
    assert torch.equal(Sr, Sr1)


@pytest.mark.parametrize("mode", ["native", "bf16x3"])
def test_sampling_is_deterministic(P, mode):
    n = 900
    A = torch.randn(n, n, device=DEV)
    R = torch.zeros((n, 64), device=DEV)
    P.hss_random_gaussian(3, n, 0, 64, R)
    outs = []
    for _ in range(2):
        Sr = torch.empty((n, 64), device=DEV)
        Sc = torch.empty((n, 64), device=DEV)
        P.hss_sample(A, R, 0, 64, Sr, Sc, leaf_starts=[0, 300, 600, 900], mode=mode)
        outs.append((Sr.clone(), Sc.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


# ------------------------------------------------------------------- ID
def _decaying(rng, d, m, rate):
    U, _ = np.linalg.qr(rng.standard_normal((d, min(d, m))))
    V, _ = np.linalg.qr(rng.standard_normal((m, min(d, m))))
    s = rate ** np.arange(min(d, m))
    return U @ np.diag(s) @ V.T


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_id_matches_oracle(P, dtype):
    rng = np.random.default_rng(1)
    shapes = [(40, 30, 0.5), (64, 100, 0.7), (100, 64, 0.8), (7, 5, 0.9), (33, 1, 0.5),
              (1, 9, 0.5), (128, 156, 0.85)]
    Ys, ref = [], []
    rtol = 1e-6
    for d, m, rate in shapes:
        Y = _decaying(rng, d, m, rate)
        Yt = torch.tensor(Y.T.copy(), dtype=dtype, device=DEV)    # m rows of d values
        Ys.append(Yt)
        ref.append(O.interpolative_decomposition(Yt.cpu().numpy().astype(np.float64).T, rtol))
    outs = P.hss_id_batched(Ys, rtol)
    for (d, m, _), (k, perm, E), r, Yt in zip(shapes, outs, ref, Ys):
        Y = Yt.cpu().numpy().astype(np.float64).T
        assert abs(k - r.k) <= 1
        perm = perm.cpu().numpy()
        assert sorted(perm.tolist()) == list(range(m))
        if k == r.k:
            assert list(perm[:k]) == list(r.perm[:k])
            # E rows follow the order of perm[k:]; compare the generators
            G = np.zeros((m, k))
            G[perm[:k]] = np.eye(k)
            G[perm[k:]] = E.cpu().numpy()
            np.testing.assert_allclose(G, r.basis(), rtol=1e-7, atol=1e-9)
        # reconstruction Y ~= Y(:, J) X within the truncation level
        G = np.zeros((m, k))
        G[perm[:k]] = np.eye(k)
        G[perm[k:]] = E.cpu().numpy()
        err = np.linalg.norm(Y - Y[:, perm[:k]] @ G.T, 2)
        assert err <= 10 * math.sqrt(m) * rtol * np.linalg.norm(Y, 2) + 1e-12


def test_large_id_over_cta_groups_matches_oracle(P):
    """A node side too large for one cluster (m = 2048 columns, d = 1024
    samples): batches of 1, 2 and 3 items spread it over 152, 76 and 50 CTAs
    meeting at barriers in global memory.  Same pivots and generators as the
    oracle's CPQR (the smallest relative gap between the two largest residual
    norms along its 503 steps is 4.6e-6, far above rounding), and the same
    bits whatever the number of CTAs."""
    rng = np.random.default_rng(7)
    d, m, rtol = 1024, 2048, 1e-6
    Y = _decaying(rng, d, m, 0.97)
    r = O.interpolative_decomposition(Y, rtol)
    Yt = torch.tensor(Y.T.copy(), dtype=torch.float64, device=DEV)
    others = [torch.tensor(_decaying(rng, d, 1500, 0.9).T.copy(), dtype=torch.float64, device=DEV)
              for _ in range(2)]
    runs = [P.hss_id_batched([Yt] + others[:c], rtol)[0] for c in range(3)]
    k, perm, E = runs[0]
    assert k == r.k == 503
    perm = perm.cpu().numpy()
    assert list(perm[:k]) == list(r.perm[:k])
    assert sorted(perm.tolist()) == list(range(m))
    G = np.zeros((m, k))
    G[perm[:k]] = np.eye(k)
    G[perm[k:]] = E.cpu().numpy()
    np.testing.assert_allclose(G, r.basis(), rtol=1e-7, atol=1e-9)
    for k2, perm2, E2 in runs[1:]:
        assert k2 == k
        assert np.array_equal(perm2.cpu().numpy(), perm)
        assert torch.equal(E2, runs[0][2])


def test_batched_id_exact_rank(P):
    rng = np.random.default_rng(2)
    Ys = []
    for r in (0, 1, 5, 17):
        Y = rng.standard_normal((60, r)) @ rng.standard_normal((r, 45))
        Ys.append(torch.tensor(Y.T.copy(), dtype=torch.float64, device=DEV))
    outs = P.hss_id_batched(Ys, 1e-12)
    assert [o[0] for o in outs] == [0, 1, 5, 17]


# ----------------------------------------------------------- compression
def _ranks_close(P, h, ho, slack=2):
    ranks = P.hss_node_ranks(h)
    ro = ho.ranks()
    for i, (lo, hi, kr, kc) in enumerate(ranks):
        if i == 0:
            continue
        assert (lo, hi) == (ho.nodes[i].lo, ho.nodes[i].hi)
        assert abs(kr - ro[i][0]) <= slack and abs(kc - ro[i][1]) <= slack, (i, kr, kc, ro[i])
    return ranks


def _ranks_close_fp32(P, h, ho, frac=0.9):
    """FP32-class samples at a tolerance near the FP32 sample error: ranks
    within +-2 of the oracle's on at least `frac` of the nodes and within
    max(3, 5%) on all (the samples' rounding moves singular values across a
    flat stretch of the spectrum at the threshold)."""
    ranks = P.hss_node_ranks(h)
    ro = ho.ranks()
    diffs = []
    for i, (lo, hi, kr, kc) in enumerate(ranks[1:], start=1):
        assert (lo, hi) == (ho.nodes[i].lo, ho.nodes[i].hi)
        for a, b in ((kr, ro[i][0]), (kc, ro[i][1])):
            assert abs(a - b) <= max(3, 0.05 * b), (i, kr, kc, ro[i])
        diffs.append(max(abs(kr - ro[i][0]), abs(kc - ro[i][1])))
    assert sum(x <= 2 for x in diffs) >= frac * len(diffs), diffs


def _err_bound(A, ho, rtol):
    e_or = _rel(O.to_dense(ho), A)
    return 2 * max(rtol, e_or)


def _dense_from_gpu(P, h, n, dtype):
    eye = torch.eye(n, dtype=dtype, device=DEV)
    return P.hss_matvec(h, eye).cpu().numpy().astype(np.float64)


def test_compress_known_ranks_exact(P):
    A, true_ranks = W.random_hss(1024, 64, 10, seed=5, diag_shift=10.0)
    At = torch.tensor(A, device=DEV)
    h = P.hss_compress(At, leaf_size=64, rtol=1e-12, d0=24, d_step=16, seed=3)
    for i, (lo, hi, kr, kc) in enumerate(P.hss_node_ranks(h)):
        if i:
            assert (kr, kc) == (true_ranks[(lo, hi)],) * 2
    H = _dense_from_gpu(P, h, 1024, torch.float64)
    assert _rel(H, A) <= 1e-10


def test_compress_config1_toeplitz_fp64(P):
    """Toeplitz n=2000 FP64, leaf 128, d0 64, step 32, rtol 1e-6."""
    n, rtol = 2000, 1e-6
    At = W.toeplitz_inv_distance(n, dtype=np.float64, device=DEV)
    A = At.cpu().numpy()
    kw = dict(leaf_size=128, rtol=rtol, d0=64, d_step=32, seed=1001)
    h = P.hss_compress(At, **kw)
    ho = O.compress(A, rtol, leaf_size=128, d0=64, d_step=32, seed=1001)
    _ranks_close(P, h, ho)
    info = P.hss_info(h)
    assert info["passes"] == ho.passes and info["d_final"] == ho.d
    H = _dense_from_gpu(P, h, n, torch.float64)
    assert _rel(H, A) <= 2 * rtol and _rel(H, A) <= _err_bound(A, ho, rtol)
    x = np.random.default_rng(0).standard_normal((n, 1))
    b = P.hss_matvec(h, torch.tensor(x, device=DEV)).cpu().numpy()
    assert _rel(b, O.matvec(ho, x)) <= 4 * rtol
    assert _rel(b, A @ x) <= 2 * rtol
    P.hss_factor(h)
    xs = P.hss_solve(h, torch.tensor(x, device=DEV)).cpu().numpy()
    O.ulv_factor(ho)
    xo = O.ulv_solve(ho, x)
    res_gpu = _rel(A @ xs, x)
    res_ora = _rel(A @ xo, x)
    assert res_gpu <= 10 * max(res_ora, 1e-15)
    # the GPU solve inverts its own H to working precision
    assert _rel(H @ xs, x) <= 1e-10


def test_compress_adaptive_restarts_match_oracle(P):
    A, _ = W.random_hss(1024, 64, 20, seed=4, diag_shift=20.0)
    At = torch.tensor(A, device=DEV)
    h = P.hss_compress(At, leaf_size=64, rtol=1e-13, d0=16, d_step=8, seed=7)
    ho = O.compress(A, 1e-13, leaf_size=64, d0=16, d_step=8, seed=7)
    info = P.hss_info(h)
    assert info["passes"] == ho.passes > 1
    assert info["d_final"] == ho.d
    _ranks_close(P, h, ho, slack=0)
    assert _rel(_dense_from_gpu(P, h, 1024, torch.float64), A) <= 1e-10


def test_compress_unsymmetric_fp32(P):
    n, rtol = 1500, 1e-4
    A = W.toeplitz_inv_distance(n).numpy() + 0.05 * np.triu(np.ones((n, n)), 1)
    At = torch.tensor(A, dtype=torch.float32, device=DEV)
    A32 = At.cpu().numpy().astype(np.float64)
    h = P.hss_compress(At, leaf_size=96, rtol=rtol, d0=48, d_step=24, seed=11)
    ho = O.compress(A32, rtol, leaf_size=96, d0=48, d_step=24, seed=11)
    _ranks_close(P, h, ho)
    H = _dense_from_gpu(P, h, n, torch.float32)
    assert _rel(H, A32) <= _err_bound(A32, ho, rtol)
    P.hss_factor(h)
    b = np.random.default_rng(3).standard_normal((n, 3))
    xs = P.hss_solve(h, torch.tensor(b, dtype=torch.float32, device=DEV)).cpu().numpy()
    O.ulv_factor(ho)
    xo = O.ulv_solve(ho, b)
    assert _rel(A32 @ xs, b) <= 10 * max(_rel(A32 @ xo, b), 1e-6)


@pytest.mark.parametrize("mode", ["native", "bf16x3"])
def test_compress_gaussian_kernel_fp32_reduced(P, mode):
    """Config-2 family at n=4000 (points in the unit cube, RCB order)."""
    n, leaf, rtol = 4000, 256, 1e-4
    pts = W.points_unit_cube(n, 1002)
    pts = pts[W.rcb_order(pts, leaf)]
    At = W.gaussian_kernel(pts, 0.2, 1.0, dtype=np.float32, device=DEV)
    A32 = At.cpu().numpy().astype(np.float64)
    h = P.hss_compress(At, leaf_size=leaf, rtol=rtol, d0=128, d_step=64, seed=1003,
                       sample_mode=mode)
    ho = O.compress(A32, rtol, leaf_size=leaf, d0=128, d_step=64, seed=1003)
    _ranks_close(P, h, ho)
    H = _dense_from_gpu(P, h, n, torch.float32)
    assert _rel(H, A32) <= _err_bound(A32, ho, rtol)
    P.hss_factor(h)
    b = np.random.default_rng(4).standard_normal((n, 8))
    xs = P.hss_solve(h, torch.tensor(b, dtype=torch.float32, device=DEV)).cpu().numpy()
    O.ulv_factor(ho)
    xo = O.ulv_solve(ho, b)
    assert _rel(A32 @ xs, b) <= 10 * max(_rel(A32 @ xo, b), 1e-6)


def test_compress_gaussian_kernel_tf32(P):
    """TF32 sampling (A rounded to TF32, 2^-11, on kind::tf32) at rtol 1e-4,
    the tolerance class where it converges: the samples' rounding adds
    rank, never removes it (every node's rank at least the oracle's - 2,
    the largest within twice the oracle's), the reconstruction stays within
    the oracle's bound plus one TF32 rounding unit, and the ULV solve
    within 10x the oracle's residual."""
    n, leaf, rtol = 4000, 256, 1e-4
    pts = W.points_unit_cube(n, 1002)
    pts = pts[W.rcb_order(pts, leaf)]
    At = W.gaussian_kernel(pts, 0.2, 1.0, dtype=np.float32, device=DEV)
    A32 = At.cpu().numpy().astype(np.float64)
    h = P.hss_compress(At, leaf_size=leaf, rtol=rtol, d0=128, d_step=64, seed=1003,
                       sample_mode="tf32")
    ho = O.compress(A32, rtol, leaf_size=leaf, d0=128, d_step=64, seed=1003)
    ranks = P.hss_node_ranks(h)
    ro = ho.ranks()
    for i, (lo, hi, kr, kc) in enumerate(ranks[1:], start=1):
        assert (lo, hi) == (ho.nodes[i].lo, ho.nodes[i].hi)
        assert kr >= ro[i][0] - 2 and kc >= ro[i][1] - 2, (i, kr, kc, ro[i])
    mx = max(max(kr, kc) for (_, _, kr, kc) in ranks[1:])
    mo = max(max(a, b) for (a, b) in ro.values())
    assert mx <= 2 * mo, (mx, mo)
    H = _dense_from_gpu(P, h, n, torch.float32)
    assert _rel(H, A32) <= _err_bound(A32, ho, rtol) + 2.0 ** -11
    P.hss_factor(h)
    b = np.random.default_rng(4).standard_normal((n, 8))
    xs = P.hss_solve(h, torch.tensor(b, dtype=torch.float32, device=DEV)).cpu().numpy()
    O.ulv_factor(ho)
    xo = O.ulv_solve(ho, b)
    assert _rel(A32 @ xs, b) <= 10 * max(_rel(A32 @ xo, b), 1e-6)


@pytest.mark.parametrize("dtype,mode", [(torch.float64, "native"), (torch.float32, "bf16x3")])
def test_compress_symmetric_matches_oracle(P, dtype, mode):
    """symmetric=True on a symmetric matrix (Gaussian kernel, adaptive
    restarts): one ID per node and V = U, as the oracle's symmetric
    compression (Section 2.2 with one R: S^c = S^r).  Ranks match the
    oracle's (FP64: +-2; BF16x3: the FP32-class check) with k^c = k^r, the
    reconstruction is symmetric to rounding and within the oracle's bound,
    the ID work is half the general compression's, and the ULV solve is
    within 10x the oracle's residual."""
    n, leaf, rtol = 3000, 128, 1e-6
    f64 = dtype == torch.float64
    pts = W.points_unit_cube(n, 1012)
    pts = pts[W.rcb_order(pts, leaf)]
    At = W.gaussian_kernel(pts, 0.2, 1.0, dtype=np.float64 if f64 else np.float32, device=DEV)
    A = At.cpu().numpy().astype(np.float64)
    kw = dict(leaf_size=leaf, rtol=rtol, d0=64, d_step=32, seed=1013, sample_mode=mode)
    h = P.hss_compress(At, symmetric=True, **kw)
    hg = P.hss_compress(At, **kw)
    ho = O.compress(A, rtol, leaf_size=leaf, d0=64, d_step=32, seed=1013, symmetric=True)
    ranks = P.hss_node_ranks(h)
    assert all(kr == kc for (_, _, kr, kc) in ranks[1:])
    if f64:
        _ranks_close(P, h, ho)
    else:
        _ranks_close_fp32(P, h, ho)
    assert P.hss_info(h)["passes"] == ho.passes or not f64
    fs, fg = P.hss_info(h)["flops_id"], P.hss_info(hg)["flops_id"]
    assert 0.3 * fg <= fs <= 0.6 * fg, (fs, fg)
    H = _dense_from_gpu(P, h, n, dtype)
    assert np.linalg.norm(H - H.T) <= (1e-12 if f64 else 1e-5) * np.linalg.norm(H)
    assert _rel(H, A) <= _err_bound(A, ho, rtol)
    P.hss_factor(h)
    b = np.random.default_rng(5).standard_normal((n, 4))
    xs = P.hss_solve(h, torch.tensor(b, dtype=dtype, device=DEV)).cpu().numpy()
    O.ulv_factor(ho)
    xo = O.ulv_solve(ho, b)
    assert _rel(A @ xs, b) <= 10 * max(_rel(A @ xo, b), 1e-6 if not f64 else 1e-13)


@pytest.mark.parametrize("mode", ["bf16x2", "bf16x3"])
def test_compress_uneven_tree_split_modes(P, mode):
    """n = 8 * leaf + 4: leaves sit at two depths, so the breadth-first leaf
    numbering does not increase with the index; the leaf mask of the
    tensor-core sampling must follow index ranges, not id order."""
    n, leaf, rtol = 8 * 128 + 4, 128, 1e-4
    nodes = O.bisection_tree(n, leaf)
    depths = {nd.depth for nd in nodes if nd.is_leaf}
    assert len(depths) == 2
    pts = W.points_unit_cube(n, 77)
    pts = pts[W.rcb_order(pts, leaf)]
    At = W.gaussian_kernel(pts, 0.15, 1.0, dtype=np.float32, device=DEV)
    A32 = At.cpu().numpy().astype(np.float64)
    h = P.hss_compress(At, leaf_size=leaf, rtol=rtol, d0=64, d_step=32, seed=12,
                       sample_mode=mode)
    ho = O.compress(A32, rtol, leaf_size=leaf, d0=64, d_step=32, seed=12)
    H = _dense_from_gpu(P, h, n, torch.float32)
    assert _rel(H, A32) <= _err_bound(A32, ho, rtol)
    ranks = P.hss_node_ranks(h)
    ro = ho.ranks()
    for i in range(1, len(ranks)):
        assert abs(ranks[i][2] - ro[i][0]) <= 2 + (2 if mode == "bf16x2" else 0), (i, ranks[i], ro[i])


# ------------------------------------------------------------ Algorithm 2 widths
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_matvec_column_counts(P, dtype):
    """Algorithm 2 at 1 to 70 right-hand sides.  Up to 32 columns the level
    products run on the narrow kernel, wider ones on 64 x 64 tiles; in both a
    column's sums do not depend on the other columns, so a column of a wide
    call equals the call on that column alone (on the same kernel), and every
    width matches the dense product."""
    A = torch.tensor(W.random_hss(2000, 128, 12, seed=5, diag_shift=10.0)[0], device=DEV).to(dtype)
    f64 = dtype == torch.float64
    h = P.hss_compress(A, leaf_size=128, rtol=1e-10 if f64 else 1e-5, d0=64, d_step=32, seed=3)
    g = torch.Generator(device=DEV).manual_seed(12)
    X = torch.randn(2000, 70, dtype=torch.float64, device=DEV, generator=g).to(dtype)
    tol = 1e-9 if f64 else 1e-4
    outs = {}
    for k in (1, 2, 3, 5, 8, 17, 32, 33, 40, 70):
        Y = P.hss_matvec(h, X[:, :k].contiguous())
        ref = A.double() @ X[:, :k].double()
        assert float(torch.linalg.norm(Y.double() - ref) / torch.linalg.norm(ref)) <= tol, k
        outs[k] = Y
    for k in (2, 3, 5, 8, 17, 32):        # narrow kernel
        assert torch.equal(outs[k][:, :1], outs[1]), k
        assert torch.equal(outs[32][:, :k], outs[k]), k
    for k in (33, 40):                    # tile kernel
        assert torch.equal(outs[70][:, :k], outs[k]), k


# ------------------------------------------------------------ edge cases
def test_single_node_tree(P):
    n = 100
    A = np.random.default_rng(0).standard_normal((n, n)) + 10 * np.eye(n)
    At = torch.tensor(A, device=DEV)
    h = P.hss_compress(At, leaf_size=128)
    x = torch.randn(n, 2, dtype=torch.float64, device=DEV)
    xn = x.cpu().numpy()
    # H = D exactly; the product differs from numpy's only by the order of its
    # sums: the FP64 dot-product bound |err| <= n u |A| |x| per entry
    bound = n * np.finfo(np.float64).eps * (np.abs(A) @ np.abs(xn))
    assert np.all(np.abs(P.hss_matvec(h, x).cpu().numpy() - A @ xn) <= bound)
    P.hss_factor(h)
    xs = P.hss_solve(h, x).cpu().numpy()
    np.testing.assert_allclose(A @ xs, x.cpu().numpy(), atol=1e-10)


def test_block_diagonal_rank_zero(P):
    import scipy.linalg as sla
    B = sla.block_diag(*[np.eye(32) * (i + 2) for i in range(8)])
    h = P.hss_compress(torch.tensor(B, device=DEV), leaf_size=32, d0=16, d_step=8)
    assert all(r[2] == 0 and r[3] == 0 for r in P.hss_node_ranks(h)[1:])
    b = torch.arange(256.0, dtype=torch.float64, device=DEV)
    np.testing.assert_allclose(P.hss_matvec(h, b).cpu().numpy(), B @ b.cpu().numpy())
    P.hss_factor(h)
    np.testing.assert_allclose(P.hss_solve(h, b).cpu().numpy(), np.linalg.solve(B, b.cpu().numpy()),
                               rtol=1e-12)


def test_errors_are_status_codes(P):
    A = torch.randn(64, 64, device=DEV)
    with pytest.raises(P.HssError) as e:
        P.hss_compress(A, leaf_size=0)
    assert e.value.status == P.hss.HSS_ERR_INVALID
    h = P.hss_compress(A + 20 * torch.eye(64, device=DEV), leaf_size=16, rtol=1e-3, d0=8, d_step=8)
    with pytest.raises(P.HssError) as e:
        P.hss_solve(h, torch.ones(64, device=DEV))
    assert e.value.status == P.hss.HSS_ERR_STATE
    with pytest.raises(P.HssError) as e:     # d_max too small for a random matrix
        P.hss_compress(torch.randn(256, 256, device=DEV), leaf_size=64, rtol=1e-12, d0=16,
                       d_step=16, d_max=32)
    assert e.value.status == P.hss.HSS_ERR_RANK_CAP


# ------------------------------------------------- caller's tree (hss_opts.tree)
def _oracle_nodes(n, splits):
    return [O.Node(i, lo, hi, dep, par, ch)
            for i, (lo, hi, dep, par, ch) in enumerate(W.split_intervals(n, splits))]


@pytest.mark.parametrize("dtype,mode", [(torch.float64, "native"), (torch.float32, "bf16x3")])
def test_compress_comb_tree_matches_oracle(P, dtype, mode):
    """A comb tree (Section 4's unbalanced tree: each non-leaf splits off one
    leaf) passed through hss_opts.tree: ranks within +-2 of the oracle on the
    same tree (FP64: equal), the product against the oracle's and the solve
    residual within 10x the oracle's.  FP32 storage at rtol 1e-5: at 1e-6 the
    slowly decaying spectrum of the 1400-index node puts several singular
    values within the FP32 sample error of the threshold."""
    n, leaf = 1500, 100
    rtol = 1e-6 if dtype == torch.float64 else 1e-5
    A = W.toeplitz_inv_distance(n).numpy() + np.triu(np.ones((n, n))) * 0.01
    At = torch.tensor(A, dtype=dtype, device=DEV)
    A64 = At.cpu().numpy().astype(np.float64)
    splits = W.comb_tree_splits(n, leaf)
    h = P.hss_compress(At, tree=splits, rtol=rtol, d0=48, d_step=16, seed=21, sample_mode=mode)
    ho = O.compress(A64, rtol, d0=48, d_step=16, seed=21, tree=_oracle_nodes(n, splits))
    ranks = P.hss_node_ranks(h)
    assert len(ranks) == len(splits)
    assert [(lo, hi) for lo, hi, _, _ in ranks] == [(nd.lo, nd.hi) for nd in ho.nodes]
    _ranks_close(P, h, ho, slack=0 if dtype == torch.float64 else 2)
    x = np.random.default_rng(3).standard_normal((n, 2))
    b = P.hss_matvec(h, torch.tensor(x, dtype=dtype, device=DEV)).cpu().numpy().astype(np.float64)
    assert _rel(b, O.matvec(ho, x)) <= (1e-12 if dtype == torch.float64 else 4 * rtol + 1e-5)
    P.hss_factor(h)
    xs = P.hss_solve(h, torch.tensor(x, dtype=dtype, device=DEV)).cpu().numpy().astype(np.float64)
    O.ulv_factor(ho)
    xo = O.ulv_solve(ho, x)
    assert _rel(A64 @ xs, x) <= 10 * max(_rel(A64 @ xo, x), 1e-12 if dtype == torch.float64 else 1e-6)


def test_explicit_bisection_tree_gives_the_default_bits(P):
    """The default tree passed explicitly as a split list reproduces the
    default compression bit for bit (ranks and product)."""
    n, leaf = 2000, 128
    A = W.toeplitz_inv_distance(n, dtype=np.float64, device=DEV)
    nodes = O.bisection_tree(n, leaf)
    splits = [nd.lo + nd.size // 2 if not nd.is_leaf else -1 for nd in nodes]
    kw = dict(rtol=1e-6, d0=64, d_step=32, seed=1002)
    h0 = P.hss_compress(A, leaf_size=leaf, **kw)
    h1 = P.hss_compress(A, leaf_size=1, tree=splits, **kw)
    assert P.hss_node_ranks(h0) == P.hss_node_ranks(h1)
    x = torch.randn(n, 3, dtype=torch.float64, device=DEV)
    assert torch.equal(P.hss_matvec(h0, x), P.hss_matvec(h1, x))


def test_bad_tree_is_rejected(P):
    A = torch.eye(300, dtype=torch.float64, device=DEV)
    for splits in ([150, -1], [0, -1, -1], [150, -1, -1, -1], [400, -1, -1]):
        with pytest.raises(P.HssError) as e:
            P.hss_compress(A, tree=splits)
        assert e.value.status == P.hss.HSS_ERR_INVALID


# ------------------------------ acceptance at 2 rtol with the ID threshold scaled
@pytest.mark.parametrize("mode", ["native", "bf16x3"])
def test_compress_meets_two_rtol_under_eps_scaling(P, mode):
    """||A - H||_F / ||A||_F <= 2 rtol.  The paper's stopping test is local:
    at eps = rtol the oracle's own error on this Gaussian kernel is 8.2e-4 for
    rtol = 1e-4, above 2 rtol.  With the same scaling eps = rtol / 10 on both
    sides the oracle meets 2 rtol (1.4e-4), and so must the GPU."""
    n, leaf, rtol = 4000, 256, 1e-4
    eps = rtol / 10
    pts = W.points_unit_cube(n, 1002)
    pts = pts[W.rcb_order(pts, leaf)]
    At = W.gaussian_kernel(pts, 0.2, 1.0, dtype=np.float32, device=DEV)
    A32 = At.cpu().numpy().astype(np.float64)
    h = P.hss_compress(At, leaf_size=leaf, rtol=eps, d0=128, d_step=64, seed=1003,
                       sample_mode=mode)
    ho = O.compress(A32, eps, leaf_size=leaf, d0=128, d_step=64, seed=1003)
    e_or = _rel(O.to_dense(ho), A32)
    assert e_or <= 2 * rtol
    if mode == "native":
        _ranks_close(P, h, ho)
    else:
        # at eps = 1e-5 the split-BF16 samples (FP32 accumulation) move a
        # few adaptive decisions: the error bound is what is asserted here,
        # with the largest rank within 10% of the oracle's
        inf = P.hss_info(h)
        assert abs(max(inf["max_rank_r"], inf["max_rank_c"]) - ho.max_rank()) <= 0.1 * ho.max_rank()
    assert _rel(_dense_from_gpu(P, h, n, torch.float32), A32) <= 2 * rtol


# ------------------------------------------------- full size (bench workload)
def _gauss20k():
    import bench
    wl = bench.WORKLOADS["gauss20k"]
    A = bench.make_matrix(wl, DEV).contiguous()
    kw = dict(leaf_size=wl["leaf"], rtol=wl["rtol"], d0=wl["d0"], d_step=wl["step"],
              seed=wl["seed"] + 1)
    return wl, A, kw


def _probe_error(P, h, A, nprobe=32, seed=0):
    """||(A - H) G||_F / ||A G||_F with Gaussian probes G (any size)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    G = torch.randn(A.shape[0], nprobe, generator=g, dtype=torch.float64).to(DEV)
    AG = A.double() @ G
    HG = P.hss_matvec(h, G.to(A.dtype)).double()
    return float(torch.linalg.norm(AG - HG) / torch.linalg.norm(AG))


def test_full_size_gauss20k_matches_oracle(P):
    """n=20000 Gaussian kernel, the benchmark's workload and launch configuration.

    FP64 path (A upcast): ranks within +-2 of the oracle's (observed: equal)
    and the same pass count.  BF16x3 sampling (checked on accuracy): the probe
    error within 2x the oracle's own; ranks within +-2 on 95% of the nodes and
    +-5% on all, leaving out nodes within 2 of the adaptive boundary d - p of
    their pass (they may take another pass) and those nodes' ancestors.
    """
    wl, A, kw = _gauss20k()
    ho = O.compress(A.cpu().numpy().astype(np.float64), wl["rtol"], leaf_size=wl["leaf"],
                    d0=wl["d0"], d_step=wl["step"], seed=wl["seed"] + 1)
    ro = ho.ranks()
    h64 = P.hss_compress(A.double(), **kw)
    r64 = P.hss_node_ranks(h64)
    assert P.hss_info(h64)["passes"] == ho.passes
    assert max(max(abs(r64[i][2] - ro[i][0]), abs(r64[i][3] - ro[i][1]))
               for i in range(1, len(r64))) <= 2
    e64 = _probe_error(P, h64, A.double())
    # the oracle's own error with the same probes (its product, Algorithm 2)
    g = torch.Generator(device="cpu").manual_seed(0)
    G = torch.randn(A.shape[0], 32, generator=g, dtype=torch.float64)
    AG = (A.double() @ G.to(DEV)).cpu().numpy()
    e_or = np.linalg.norm(AG - O.matvec(ho, G.numpy())) / np.linalg.norm(AG)
    assert e64 <= 2 * max(wl["rtol"], e_or)
    h3 = P.hss_compress(A, sample_mode="bf16x3", **kw)
    r3 = P.hss_node_ranks(h3)
    # nodes whose oracle rank is within 2 of the adaptive boundary d - p of
    # the pass that compressed them may take another pass; skip them and
    # their ancestors (whose inputs then differ)
    skip = set()
    for nd in ho.nodes:
        if nd.id and max(ro[nd.id]) >= ho.data[nd.id].d_compressed - 10 - 2:
            q = nd.id
            while q >= 0:
                skip.add(q)
                q = ho.nodes[q].parent
    assert len(skip) < len(ho.nodes) // 4
    diffs = [max(abs(r3[i][2] - ro[i][0]), abs(r3[i][3] - ro[i][1]))
             for i in range(1, len(r3)) if i not in skip]
    # FP32-class sampling: ranks close (+-2 for 95% of the nodes, +-5% for all)
    assert sum(x <= 2 for x in diffs) >= 0.95 * len(diffs)
    for i in range(1, len(r3)):
        if i not in skip:
            assert abs(r3[i][2] - ro[i][0]) <= max(2, 0.05 * ro[i][0]), (i, r3[i], ro[i])
    assert _probe_error(P, h3, A) <= 2 * max(e_or, wl["rtol"])


def test_full_size_bem60k_matches_oracle_golden(P):
    """n = 60000 BEM-like matrix at rtol 1e-6 (leaf 512, d0/step 256/128), the
    benchmark's workload and launch configuration, against the FP64 oracle's
    run stored in tests/golden/bem60k_oracle.json (written by
    tests/golden/make_bem60k_golden.py from oracle/ and workloads/ only).

    * The matrix: the same FP32 bits as the oracle's (exact fingerprint).
    * FP64 GPU path (A upcast exactly, FP64 sampling): the oracle's pass
      count and final sample count, every node's ranks within +-2.
    * BF16x3 sampling (the benchmark's mode): the oracle's pass count and
      sample count, probe error within 2 max(rtol, e_oracle) with the
      oracle's own 64 probes.  Ranks: measured distribution of |k_gpu -
      k_oracle| over the 254 nodes 0:104, 1:90, 2:34, 3:18, 4:6, 9:1, 55:1,
      the same as the plain FP32 GPU method's (0:109, 1:93, 2:34, 3:12, 4:3,
      8:1, 9:1, 51:1): FP32 sample rounding, not the tensor-core split,
      moves ranks at this tolerance.  Required: +-2 on 85% of the nodes and
      within 2% on all nodes that are not on the adaptive boundary (oracle
      rank >= d - p - 2 at the pass that compressed them: they may compress
      a pass later with a larger rank) and not above one.
    """
    import json
    import os
    import bench
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bem60k_oracle.json")))
    wl = bench.WORKLOADS["bem60k"]
    A = bench.make_matrix(wl, DEV).contiguous()
    assert W.fingerprint(A) == gold["fingerprint_fp32"]
    n = A.shape[0]
    kw = dict(leaf_size=wl["leaf"], rtol=wl["rtol"], d0=wl["d0"], d_step=wl["step"],
              seed=wl["seed"] + 1)
    nodes = gold["nodes"]
    G = torch.tensor(np.random.default_rng(gold["spec"]["probe_seed"]).standard_normal(
        (n, gold["spec"]["probes"])), device=DEV)
    AG = torch.cat([A[r:r + 4096].double() @ G for r in range(0, n, 4096)])

    def check(h, strict):
        info = P.hss_info(h)
        assert info["passes"] == gold["passes"] and info["d_final"] == gold["d_final"]
        ranks = P.hss_node_ranks(h)
        assert len(ranks) == len(nodes)
        diffs = []
        for i, (lo, hi, kr, kc) in enumerate(ranks[1:], start=1):
            nd = nodes[i]
            assert (lo, hi) == (nd["lo"], nd["hi"])
            diffs.append((i, max(abs(kr - nd["kr"]), abs(kc - nd["kc"])), kr, kc))
        if strict:
            assert max(x[1] for x in diffs) <= 2, sorted(diffs, key=lambda x: -x[1])[:5]
        else:
            assert sum(x[1] <= 2 for x in diffs) >= 0.85 * len(diffs)
            skip = set()
            for nd in nodes[1:]:
                if max(nd["kr"], nd["kc"]) >= nd["d_compressed"] - 10 - 2:
                    q = nd["id"]
                    while q >= 0:
                        skip.add(q)
                        q = nodes[q]["parent"]
            assert len(skip) < len(nodes) // 4
            for i, dk, kr, kc in diffs:
                if i not in skip:
                    assert dk <= max(2, 0.02 * max(nodes[i]["kr"], nodes[i]["kc"])), (i, kr, kc)
        HG = P.hss_matvec(h, G.to(h.dtype)).double()
        return float(torch.linalg.norm(AG - HG) / torch.linalg.norm(AG))

    e_or = gold["probe_rel_err"]
    h3 = P.hss_compress(A, sample_mode="bf16x3", **kw)
    assert check(h3, strict=False) <= 2 * max(wl["rtol"], e_or)
    h3.close()
    A64 = A.double()
    del A
    torch.cuda.empty_cache()
    h64 = P.hss_compress(A64, **kw)
    assert check(h64, strict=True) <= 2 * max(wl["rtol"], e_or)


# ------------------------------------------------ ULV of large nodes (blocked path)
def test_full_size_simple_toeplitz_matches_paper_table3(P):
    """Table 3 (SimpleToeplitz, a_ii = n^2, a_ij = i - j, n = 80,000, double
    precision): max HSS rank 2 at eps = 1e-8 and 1e-6 (the stored values,
    tests/golden/simple_toeplitz_table3.txt); the ULV solve of this
    diagonally dominant system to a relative residual of 1e-12."""
    n = 80000
    rows = []
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "simple_toeplitz_table3.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#") and not line.startswith("eps"):
                eps, rank = line.split()
                rows.append((float(eps), int(rank)))
    assert rows
    A = W.simple_toeplitz(n, dtype=np.float64, device=DEV)
    b = torch.randn(n, 1, dtype=torch.float64, device=DEV,
                    generator=torch.Generator(device=DEV).manual_seed(3))
    for eps, want in rows:
        h = P.hss_compress(A, leaf_size=128, rtol=eps, d0=64, d_step=32, seed=1007)
        info = P.hss_info(h)
        assert max(info["max_rank_r"], info["max_rank_c"]) == want, (eps, info["max_rank_r"])
        P.hss_factor(h)
        x = P.hss_solve(h, b)
        assert float(torch.linalg.norm(A @ x - b) / torch.linalg.norm(b)) <= 1e-12
        h.close()
    del A
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ulv_large_nodes_match_dense_solve(P, dtype):
    """Leaves of 512 and ranks of 200 put every node (and the root LU) on the
    blocked multi-kernel path; the solution must match a dense solve and the
    oracle's ULV solution."""
    n, leaf, rank = 2048, 512, 200
    A, _ = W.random_hss(n, leaf, rank, seed=31, diag_shift=40.0)
    At = torch.tensor(A, dtype=dtype, device=DEV)
    A64 = At.cpu().numpy().astype(np.float64)
    rtol = 1e-12 if dtype == torch.float64 else 1e-6
    h = P.hss_compress(At, leaf_size=leaf, rtol=rtol, d0=256, d_step=128, seed=8,
                       sample_mode="native" if dtype == torch.float64 else "bf16x3")
    ranks = P.hss_node_ranks(h)
    assert max(max(kr, kc) for _, _, kr, kc in ranks[1:]) >= 160   # large nodes present
    P.hss_factor(h)
    b = np.random.default_rng(5).standard_normal((n, 3))
    xs = P.hss_solve(h, torch.tensor(b, dtype=dtype, device=DEV)).cpu().numpy().astype(np.float64)
    xd = np.linalg.solve(A64, b)
    if dtype == torch.float64:
        np.testing.assert_allclose(xs, xd, rtol=0, atol=1e-8 * np.abs(xd).max())
        # up to 64 right-hand sides the large nodes' triangular solves take one
        # launch (a column per warp); more take the blocked solve.  Both end at
        # the compression error (1e-12) times this matrix's conditioning: the
        # blocked solve's 70 columns were measured 1.4e-8 of max |x| from the
        # dense solve
        b70 = np.random.default_rng(6).standard_normal((n, 70))
        x70 = P.hss_solve(h, torch.tensor(b70, device=DEV)).cpu().numpy()
        xd70 = np.linalg.solve(A64, b70)
        np.testing.assert_allclose(x70, xd70, rtol=0, atol=1e-7 * np.abs(xd70).max())
        assert _rel(A64 @ x70, b70) <= 100 * _rel(A64 @ xs, b) + 1e-12
    else:
        ho = O.compress(A64, rtol, leaf_size=leaf, d0=256, d_step=128, seed=8)
        O.ulv_factor(ho)
        xo = O.ulv_solve(ho, b)
        assert _rel(A64 @ xs, b) <= 10 * max(_rel(A64 @ xo, b), 1e-6)
