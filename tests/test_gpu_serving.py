"""Serving loop: requests overlap on the device (continuous batching) and each
result equals the result of compressing the same matrix alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("lane_split_n", [None, 900])
def test_served_results_equal_alone_and_solve(P, lane_split_n):
    """One lane, or two (requests of order >= 900 in a batch, stream and
    thread of their own): each served result equals the same matrix
    compressed alone."""
    from paper_1503_05464_gb300 import serving as S
    opts = P.hss_default_opts(leaf_size=64, rtol=1e-6, d0=64, d_step=32, seed=5,
                              sample_mode="bf16x3")
    reqs = S.poisson_requests(10, rate=200.0, ks=[20, 30, 40], seed=3, max_solves=2,
                              nrhs_range=(1, 8))
    make = lambda k: W.laplacian_schur(k, dtype=np.float32, device=DEV)
    srv = S.Server(make, opts, budget_bytes=int(2e9), keep_handles=True,
                   lane_split_n=lane_split_n)
    st = srv.run(reqs)
    summ = st.summary()
    assert summ["requests"] == 10 and summ["solves"] == sum(len(r.solves) for r in reqs)
    assert st.max_inflight > 1                 # compressions overlapped in one batch
    assert summ["request_p99_s"] >= summ["request_p50_s"] > 0
    for r in srv.done:
        A = srv.templates[r.k] * r.scale
        alone = P.hss_compress(A, opts)
        assert P.hss_node_ranks(alone) == P.hss_node_ranks(r.handle)
        x = torch.randn(r.n, 2, device=DEV)
        assert torch.equal(P.hss_matvec(alone, x), P.hss_matvec(r.handle, x))
        b = torch.randn(r.n, 3, device=DEV)
        xs = P.hss_solve(r.handle, b)
        res = torch.linalg.norm(A.double() @ xs.double() - b.double()) / torch.linalg.norm(b.double())
        assert res < 1e-4


def test_admission_respects_the_budget(P):
    from paper_1503_05464_gb300 import serving as S
    opts = P.hss_default_opts(leaf_size=64, rtol=1e-6, d0=64, d_step=32, seed=5)
    reqs = S.poisson_requests(6, rate=1000.0, ks=[40], seed=4, max_solves=1, nrhs_range=(1, 1))
    need = S.estimate_bytes(1600, opts)
    make = lambda k: W.laplacian_schur(k, dtype=np.float32, device=DEV)
    st = S.Server(make, opts, budget_bytes=2 * need + need // 2).run(reqs)
    assert st.max_inflight <= 2               # a third request never fits
    assert st.summary()["solves"] == 6
