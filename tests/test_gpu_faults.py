"""Failure handling through the C ABI, without faulting the GPU.

* A bounded device wait that gives up: the ID's spread-out (group) mode meets
  at a barrier in global memory; with the wait limit forced down to a few
  cycles a CTA gives up, raises the launch's abort flag, every CTA returns at
  its next barrier and the call reports HSS_ERR_TIMEOUT.  The wait only polls
  a counter (no asynchronous copy is in flight), so giving up is safe; the
  same process then runs the same decomposition and a full compression.
* An allocation failure, injected on the host at the N-th device allocation:
  the call returns HSS_ERR_OOM, the library's memory pool returns to the
  bytes in use before the call (nothing leaks), and the next call succeeds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1503_05464_gb300 as pkg
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    yield pkg
    pkg.hss.hss_set_fault(pkg.hss.HSS_FAULT_NONE)


def _decaying(rng, d, m, rate):
    U = np.linalg.qr(rng.standard_normal((d, d)))[0]
    V = np.linalg.qr(rng.standard_normal((m, d)))[0]
    return (U * rate ** np.arange(d)) @ V.T


def test_group_barrier_timeout_is_reported_and_the_context_recovers(P):
    H = P.hss
    rng = np.random.default_rng(7)
    Y = torch.tensor(_decaying(rng, 1024, 2048, 0.97).T.copy(), dtype=torch.float64, device=DEV)
    ref = P.hss_id_batched([Y], 1e-6)[0]      # one large item: spread over every SM
    H.hss_set_fault(H.HSS_FAULT_WAIT_LIMIT, 16)
    try:
        with pytest.raises(P.HssError) as e:
            P.hss_id_batched([Y], 1e-6)
        assert e.value.status == H.HSS_ERR_TIMEOUT
    finally:
        H.hss_set_fault(H.HSS_FAULT_NONE)
    again = P.hss_id_batched([Y], 1e-6)[0]
    assert again[0] == ref[0]
    assert torch.equal(again[1], ref[1]) and torch.equal(again[2], ref[2])
    import workloads as W
    A = W.toeplitz_inv_distance(1000, dtype=np.float64, device=DEV)
    h = P.hss_compress(A, leaf_size=64, rtol=1e-8, d0=32, d_step=16)
    x = torch.randn(1000, 2, dtype=torch.float64, device=DEV)
    assert torch.allclose(P.hss_matvec(h, x), A @ x, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("mode", ["native", "bf16x3"])
def test_injected_oom_fails_cleanly_and_leaks_nothing(P, mode):
    H = P.hss
    import workloads as W
    n = 3000
    A = W.toeplitz_inv_distance(n, dtype=np.float32, device=DEV)
    kw = dict(leaf_size=128, rtol=1e-6, d0=64, d_step=32, seed=3, sample_mode=mode)
    ref = P.hss_node_ranks(P.hss_compress(A, **kw))
    torch.cuda.synchronize()
    used0, _ = H.hss_pool_bytes()
    seen_oom = 0
    for after in (1, 2, 3, 5, 8, 13, 21, 34, 55):
        H.hss_set_fault(H.HSS_FAULT_OOM, after)
        try:
            h = P.hss_compress(A, **kw)
        except P.HssError as e:
            assert e.status == H.HSS_ERR_OOM, str(e)
            seen_oom += 1
        else:
            assert P.hss_node_ranks(h) == ref       # fewer allocations than `after`
            h.close()
        finally:
            H.hss_set_fault(H.HSS_FAULT_NONE)
        torch.cuda.synchronize()
        assert H.hss_pool_bytes()[0] == used0, after
    assert seen_oom >= 5
    h = P.hss_compress(A, **kw)
    assert P.hss_node_ranks(h) == ref
    P.hss_factor(h)
    b = torch.ones(n, dtype=torch.float32, device=DEV)
    x = P.hss_solve(h, b)
    assert float(torch.linalg.norm(A @ x - b) / torch.linalg.norm(b)) < 1e-4
