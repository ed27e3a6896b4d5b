"""Input generators that tests and the benchmark share (no method arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402


@pytest.mark.parametrize("which", ["simple", "qchem"])
def test_toeplitz_operator_matches_the_stored_matrix(which):
    # the matrix-free Toeplitz operator (FFT products, entries by formula)
    # against the stored matrix of the same family: products to rounding,
    # entries exactly
    n = 300
    if which == "simple":
        T, A = W.ToeplitzOperator(n, W.simple_toeplitz_symbol(n), "cpu"), W.simple_toeplitz(n)
    else:
        T, A = W.ToeplitzOperator(n, W.qchem_toeplitz_symbol(1.0), "cpu"), W.qchem_toeplitz(n)
    A = A.numpy()
    X = torch.tensor(np.random.default_rng(3).standard_normal((n, 5)))
    Sr, Sc = torch.empty(n, 5, dtype=torch.float64), torch.empty(n, 5, dtype=torch.float64)
    T.sample(X, Sr, Sc)
    scale = np.abs(A @ X.numpy()).max()
    assert np.abs(Sr.numpy() - A @ X.numpy()).max() <= 1e-13 * scale
    assert np.abs(Sc.numpy() - A.T @ X.numpy()).max() <= 1e-13 * scale
    assert np.array_equal(T.matmul(X).numpy(), Sr.numpy())
    rows = torch.tensor([0, 5, 299, 17], dtype=torch.int32)
    cols = torch.tensor([0, 7, 3, 299, 17], dtype=torch.int32)
    out = torch.empty(4, 5, dtype=torch.float64)
    T.extract(rows, cols, out)
    assert np.array_equal(out.numpy(), A[np.ix_(rows.numpy(), cols.numpy())])


def test_qchem_toeplitz_is_symmetric_with_its_printed_entries():
    # Section 4.1: a_ii = pi^2/6, a_ij = (-1)^(i-j) / ((i-j)^2 h^2), h = 1
    A = W.qchem_toeplitz(6).numpy()
    assert np.array_equal(A, A.T)
    assert A[0, 0] == np.pi ** 2 / 6 and A[0, 1] == -1.0 and A[0, 2] == 0.25
    assert A[3, 0] == -1.0 / 9.0
