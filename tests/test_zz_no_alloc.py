"""hss_sample_noalloc against hss_sample, through the C ABI.

The no-allocation variant is for callers that may not allocate device memory:
a host application whose own memory manager owns the whole GPU, or a serving
loop that allows no allocator call once it runs (cudaMalloc and cudaFree can
block or synchronize the device).  It keeps its scratch in fixed device
arrays of the library instead, so its results must equal those of the
allocating entry point, in every sampling mode, and the library's memory pool
must not move while it runs.  Two calls in a row check that the shared
scratch carries nothing from one call to the next.  This file sorts last so
that a failure here cannot hide another test's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# (n, leaf, c0, c1): a ragged order with a column offset, then the largest
# accepted order; n = 1500 and 1983 with 64 columns are the largest scratch
# needs of the tensor-core kernel
CASES = [(1500, 100, 3, 67), (2048, 256, 0, 64), (1983, 128, 0, 64)]


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1503_05464_gb300 as pkg
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    return pkg


def _inputs(P, call, n, c1, dtype):
    g = torch.Generator(device="cpu").manual_seed(call)
    A = torch.randn(n, n, generator=g, dtype=torch.float64) + 3 * torch.eye(n, dtype=torch.float64)
    A[: n // 4] *= 2.0
    A = A.to(dtype).to(DEV)
    R = torch.zeros((n, c1), dtype=dtype, device=DEV)
    P.hss_random_gaussian(17 + call, n, 0, c1, R)
    return A, R


@pytest.mark.parametrize("dtype,mode", [(torch.float64, "native"), (torch.float32, "native"),
                                        (torch.float32, "tf32"), (torch.float32, "bf16x2"),
                                        (torch.float32, "bf16x3")])
def test_noalloc_sampling_matches_allocating_entry_point(P, dtype, mode):
    # the tolerance of the sampling parity tests: a length-n dot product's
    # rounding bound (FP32) against sum |A||R|, for both entry points
    tol = 1e-12 if dtype == torch.float64 else 4 * 2048 * 2.0 ** -24
    if mode == "tf32":
        tol = 4 * 2.0 ** -11
    for call, (n, leaf, c0, c1) in enumerate(CASES):
        A, R = _inputs(P, call, n, c1, dtype)
        starts = list(range(0, n, leaf)) + [n]
        outs = [torch.full((n, c1), -1.0, dtype=dtype, device=DEV) for _ in range(4)]
        Sr0, Sc0, Sr1, Sc1 = outs
        P.hss_sample(A, R, c0, c1, Sr0, Sc0, leaf_starts=starts, mode=mode)
        torch.cuda.synchronize()
        used0, reserved0 = P.hss.hss_pool_bytes()
        P.hss_sample_noalloc(A, R, c0, c1, Sr1, Sc1, leaf_starts=starts, mode=mode)
        torch.cuda.synchronize()
        assert P.hss.hss_pool_bytes() == (used0, reserved0)
        An = A.double().cpu().numpy()
        Rn = R.double().cpu().numpy()[:, c0:c1]
        mask = np.ones((n, n))
        for lo in range(0, n, leaf):
            mask[lo:lo + leaf, lo:lo + leaf] = 0
        br = (np.abs(An) * mask) @ np.abs(Rn)
        bc = (np.abs(An) * mask).T @ np.abs(Rn)
        for got, ref, bound in [(Sr1, Sr0, br), (Sc1, Sc0, bc)]:
            g_ = got.double().cpu().numpy()
            r_ = ref.double().cpu().numpy()
            assert np.all(g_[:, :c0] == -1.0)
            assert np.all(np.abs(g_[:, c0:c1] - r_[:, c0:c1]) <= tol * bound + 1e-30)


def test_noalloc_rejects_problems_beyond_its_scratch(P):
    A = torch.zeros((2049, 2049), device=DEV)
    R = torch.zeros((2049, 8), device=DEV)
    S = torch.zeros((2049, 8), device=DEV)
    with pytest.raises(P.HssError) as e:
        P.hss_sample_noalloc(A, R, 0, 8, S, S.clone())
    assert e.value.status == P.hss.HSS_ERR_INVALID
    assert "2048" in str(e.value)
    A = torch.zeros((512, 512), device=DEV)
    R = torch.zeros((512, 65), device=DEV)
    S = torch.zeros((512, 65), device=DEV)
    with pytest.raises(P.HssError) as e:
        P.hss_sample_noalloc(A, R, 0, 65, S, S.clone(), mode="bf16x3")
    assert e.value.status == P.hss.HSS_ERR_INVALID
