"""Batched and incremental compression: every matrix must come out exactly as
it does alone (same ranks, bitwise-identical products), whatever else shares
its launches, and whenever it joined the batch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hss_oracle as O  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1503_05464_gb300 as pkg
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    return pkg


def _mats_f64():
    out = []
    for n in (700, 1500, 2000, 1024):
        A = W.toeplitz_inv_distance(n, dtype=np.float64, device=DEV)
        if n == 1024:
            A = torch.tensor(W.random_hss(1024, 64, 12, seed=2, diag_shift=10.0)[0], device=DEV)
        out.append(A.contiguous())
    return out


def _mats_f32():
    out = []
    for i, n in enumerate((1800, 3000, 2500)):
        pts = W.points_unit_cube(n, 50 + i)
        pts = pts[W.rcb_order(pts, 128)]
        out.append(W.gaussian_kernel(pts, 0.1 + 0.1 * i, 1.0, dtype=np.float32, device=DEV))
    out.append(W.toeplitz_inv_distance(2200, dtype=np.float32, device=DEV).contiguous())
    return out


def _same(P, h1, h2, n, dtype):
    assert P.hss_node_ranks(h1) == P.hss_node_ranks(h2)
    assert P.hss_info(h1)["passes"] == P.hss_info(h2)["passes"]
    x = torch.randn(n, 3, dtype=torch.float64, device=DEV, generator=torch.Generator(device=DEV).manual_seed(n)).to(dtype)
    assert torch.equal(P.hss_matvec(h1, x), P.hss_matvec(h2, x))


@pytest.mark.parametrize("mode", ["native", "bf16x3"])
def test_batched_equals_alone(P, mode):
    mats = _mats_f32()
    kw = dict(leaf_size=128, rtol=1e-5, d0=64, d_step=32, seed=9, sample_mode=mode)
    hs, sts = P.hss_compress_batched(mats, **kw)
    assert sts == [0] * len(mats)
    for A, h in zip(mats, hs):
        alone = P.hss_compress(A, **kw)
        _same(P, h, alone, A.shape[0], A.dtype)


def test_batched_symmetric_and_general_mixed_equal_alone(P):
    # symmetric matrices, every other one compressed with symmetric=True:
    # each handle comes out as it does alone, whatever shares its launches
    mats = _mats_f32()
    opts = [P.hss_default_opts(leaf_size=128, rtol=1e-5, d0=64, d_step=32, seed=9,
                               sample_mode="bf16x3", symmetric=(i % 2 == 0))
            for i in range(len(mats))]
    hs, sts = P.hss_compress_batched(mats, opts)
    assert sts == [0] * len(mats)
    for A, h, o in zip(mats, hs, opts):
        alone = P.hss_compress(A, o)
        _same(P, h, alone, A.shape[0], A.dtype)
        if o.symmetric:
            assert all(kr == kc for (_, _, kr, kc) in P.hss_node_ranks(h)[1:])


def test_batched_fp64_matches_oracle(P):
    mats = _mats_f64()
    kw = dict(leaf_size=64, rtol=1e-8, d0=48, d_step=16, seed=4)
    hs, sts = P.hss_compress_batched(mats, **kw)
    assert sts == [0] * len(mats)
    for A, h in zip(mats, hs):
        ho = O.compress(A.cpu().numpy(), 1e-8, leaf_size=64, d0=48, d_step=16, seed=4)
        ro = ho.ranks()
        for i, (lo, hi, kr, kc) in enumerate(P.hss_node_ranks(h)):
            if i:
                assert (kr, kc) == ro[i]
        x = np.random.default_rng(1).standard_normal((A.shape[0], 2))
        b = P.hss_matvec(h, torch.tensor(x, device=DEV)).cpu().numpy()
        np.testing.assert_allclose(b, O.matvec(ho, x), rtol=0, atol=1e-9 * np.abs(b).max())


def test_incremental_batch_admits_jobs_mid_flight(P):
    mats = _mats_f32()
    kw = dict(leaf_size=128, rtol=1e-5, d0=64, d_step=32, seed=9, sample_mode="bf16x3")
    opts = P.hss_default_opts(**kw)
    b = P.HssBatch(torch.float32)
    t0 = b.submit(mats[0], opts)
    t1 = b.submit(mats[1], opts)
    b.step()
    b.step()
    t2 = b.submit(mats[2], opts)          # joins while the first two are mid-tree
    b.step()
    t3 = b.submit(mats[3], opts)
    rounds = 3
    while b.step() > 0:
        rounds += 1
        assert rounds < 500
    for t, A in zip((t0, t1, t2, t3), mats):
        h, st = b.take(t)
        assert st == 0 and h is not None
        _same(P, h, P.hss_compress(A, opts), A.shape[0], A.dtype)
    h, st = b.take(t0)                      # already taken
    assert st == P.hss.HSS_ERR_INVALID
    b.close()


def test_batch_reports_per_job_failures(P):
    good = W.toeplitz_inv_distance(600, dtype=np.float32, device=DEV).contiguous()
    bad = torch.randn(512, 512, device=DEV)
    kw = dict(leaf_size=64, rtol=1e-7, d0=16, d_step=16, d_max=32, seed=1)
    hs, sts = P.hss_compress_batched([good, bad], **kw)
    assert sts[0] == 0 or sts[0] == P.hss.HSS_ERR_RANK_CAP
    assert sts[1] == P.hss.HSS_ERR_RANK_CAP    # random matrix: no low rank at d_max = 32
    assert hs[1] is not None                    # a rank-capped handle is still returned


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_factor_and_solve_equal_alone(P, dtype):
    """hss_factor_batched / hss_solve_batched (one launch per level round
    across all handles, Algorithms 3 and 4) give bitwise the solutions of one
    hss_factor / hss_solve per handle; trees of different depths, a
    single-node tree and a handle solved twice in one batch included."""
    # two matrices whose nodes (leaves of 512, ranks near 200) and roots take
    # the blocked large-node path, batched across handles
    big = [torch.tensor(W.random_hss(2048, 512, 200, seed=31 + i, diag_shift=40.0)[0], device=DEV)
           for i in range(2)]
    if dtype == "f32":
        mats = _mats_f32() + [W.toeplitz_inv_distance(90, dtype=np.float32, device=DEV)] + \
            [b.float() for b in big]
        kw = dict(leaf_size=128, rtol=1e-5, d0=64, d_step=32, seed=9, sample_mode="bf16x3")
    else:
        mats = _mats_f64() + [W.toeplitz_inv_distance(90, dtype=np.float64, device=DEV)] + big
        kw = dict(leaf_size=128, rtol=1e-8, d0=64, d_step=32, seed=9)
    kws = [dict(kw, leaf_size=512, d0=256, d_step=128) if A.shape[0] == 2048 else kw for A in mats]
    hs_b = [P.hss_compress(A, **k) for A, k in zip(mats, kws)]
    hs_a = [P.hss_compress(A, **k) for A, k in zip(mats, kws)]
    assert max(max(r[2], r[3]) for h in hs_b[-2:] for r in P.hss_node_ranks(h)) >= 160
    assert P.hss_factor_batched(hs_b) == [0] * len(mats)
    for h in hs_a:
        P.hss_factor(h)
    g = torch.Generator(device=DEV).manual_seed(4)
    Bs = [torch.randn(A.shape[0], 1 + 3 * i, device=DEV, generator=g).to(A.dtype)
          for i, A in enumerate(mats)]
    hs_q = hs_b + [hs_b[0]]
    Bs_q = Bs + [Bs[0][:, :2].contiguous()]
    Xs, sts = P.hss_solve_batched(hs_q, Bs_q)
    assert sts == [0] * len(hs_q)
    for h, B, X in zip(hs_a + [hs_a[0]], Bs_q, Xs):
        assert torch.equal(P.hss_solve(h, B), X)
    # residuals of the well-conditioned families (the random HSS inputs with
    # rank-200 generators at every level are not: they test the path only)
    for A, B, X in list(zip(mats, Bs, Xs))[:-2]:
        r = torch.linalg.norm(A.double() @ X.double() - B.double()) / torch.linalg.norm(B.double())
        assert float(r) < (1e-2 if dtype == "f32" else 1e-6)


def test_batched_factor_reports_each_handle(P):
    A = W.toeplitz_inv_distance(600, dtype=np.float64, device=DEV)
    h1 = P.hss_compress(A, leaf_size=64, rtol=1e-8, d0=32, d_step=16)
    h2 = P.hss_compress(A, leaf_size=64, rtol=1e-8, d0=32, d_step=16)
    P.hss_factor_batched([h1])
    X, sts = P.hss_solve_batched([h1, h2], [torch.ones(600, dtype=torch.float64, device=DEV)] * 2)
    assert sts[0] == 0 and sts[1] == P.hss.HSS_ERR_STATE
