"""Seeded synthetic inputs for HSS compression.

This module only builds input matrices, point clouds and orderings; it holds
none of the compression, product, factorization or solve arithmetic.  The CPU
oracle and the GPU path both take their inputs from here, and nothing here
imports either of them.

Matrix families (stand-ins for the paper's application matrices, Section 4.1):

* ``toeplitz_inv_distance``  a_ij = 1/(1+|i-j|), a_ii = 10.
* ``simple_toeplitz``        the paper's SimpleToeplitz: a_ii = n^2, a_ij = i-j.
* ``qchem_toeplitz``         the paper's QChemToeplitz kinetic-energy matrix:
                             a_ii = pi^2/6, a_ij = (-1)^(i-j) / ((i-j)^2 h^2).
* ``ToeplitzOperator``       either Toeplitz matrix without storage: FFT
                             products and entries by formula (matrix-free).
* ``gaussian_kernel``        K_ij = exp(-|x_i-x_j|^2/(2h^2)) + lambda*delta_ij on
                             points uniform in the unit cube.
* ``bem_like``               a_ij = 1/(4*pi*|x_i-x_j|), a_ii = sqrt(n) on points
                             uniform on the unit sphere.
* ``random_hss``             a dense matrix assembled from random HSS generators
                             with prescribed ranks (known-rank test input).
* ``laplacian_schur``        the dense Schur complement, onto the middle plane,
                             of the 7-point Laplacian on a k x k x (2k+1) grid
                             with Dirichlet boundaries (n = k^2).

Point clouds are put in recursive-coordinate-bisection order whose splits match
the cluster tree's bisection (left part = floor(s/2) points), so that the
off-diagonal blocks of the tree are the far-field blocks.
"""
from __future__ import annotations

import math
import numpy as np

try:  # torch is only needed for the chunked on-device generators
    import torch
except ImportError:  # pragma: no cover
    torch = None


# ---------------------------------------------------------------- point clouds
def points_unit_cube(n: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1]^3 (float64, shape n x 3)."""
    return np.random.default_rng(seed).random((n, 3))


def points_unit_sphere(n: int, seed: int) -> np.ndarray:
    """n points uniform on the unit sphere (float64, shape n x 3).

    Points uniform in the ball (rejection from the cube [-1, 1]^3, keeping
    1e-4 <= |u|^2 <= 1) projected onto the sphere.  Only correctly rounded
    operations are used (2u - 1, products, sums in a fixed order, sqrt,
    division), so the points are bitwise the same on every platform.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3))
    filled = 0
    while filled < n:
        u = rng.random((2 * (n - filled) + 64, 3)) * 2.0 - 1.0
        r2 = u[:, 0] * u[:, 0]
        r2 = r2 + u[:, 1] * u[:, 1]
        r2 = r2 + u[:, 2] * u[:, 2]
        keep = np.nonzero((r2 <= 1.0) & (r2 >= 1e-4))[0][: n - filled]
        r = np.sqrt(r2[keep])
        out[filled:filled + keep.size] = u[keep] / r[:, None]
        filled += keep.size
    return out


def rcb_order(points: np.ndarray, leaf_size: int) -> np.ndarray:
    """Recursive coordinate bisection permutation.

    A range of s > leaf_size points is sorted (stably) along the longest axis
    of its bounding box and split into floor(s/2) and s - floor(s/2) points,
    the same split the cluster tree uses, down to ranges of <= leaf_size.
    """
    n = points.shape[0]
    perm = np.arange(n)
    stack = [(0, n)]
    while stack:
        lo, hi = stack.pop()
        s = hi - lo
        if s <= leaf_size:
            continue
        sub = points[perm[lo:hi]]
        axis = int(np.argmax(sub.max(axis=0) - sub.min(axis=0)))
        order = np.argsort(sub[:, axis], kind="stable")
        perm[lo:hi] = perm[lo:hi][order]
        mid = lo + s // 2
        stack.append((lo, mid))
        stack.append((mid, hi))
    return perm


# ------------------------------------------------------------ dense matrices
def _dev(device):
    if torch is None:
        raise RuntimeError("torch is required for the chunked generators")
    return torch.device(device)


def toeplitz_inv_distance(n: int, dtype=np.float64, device="cpu"):
    """a_ij = 1/(1+|i-j|) off the diagonal, a_ii = 10 (row-major n x n)."""
    dev = _dev(device)
    i = torch.arange(n, device=dev, dtype=torch.float64)
    a = 1.0 / (1.0 + (i[:, None] - i[None, :]).abs())
    a.diagonal().fill_(10.0)
    return a.to(_tdtype(dtype))


def simple_toeplitz(n: int, dtype=np.float64, device="cpu"):
    """The paper's SimpleToeplitz matrix: a_ii = n^2, a_ij = i - j."""
    dev = _dev(device)
    i = torch.arange(n, device=dev, dtype=torch.float64)
    a = i[:, None] - i[None, :]
    a.diagonal().fill_(float(n) * n)
    return a.to(_tdtype(dtype))


def qchem_toeplitz(n: int, spacing: float = 1.0, dtype=np.float64, device="cpu", chunk=2048):
    """The paper's QChemToeplitz matrix (Section 4.1, a kinetic-energy matrix
    from quantum chemistry): a_ii = pi^2/6, a_ij = (-1)^(i-j) / ((i-j)^2 h^2)
    with grid spacing h (row blocks of `chunk`; every operation exact or
    correctly rounded, so the bits are the same on the CPU and the GPU)."""
    dev = _dev(device)
    out = torch.empty((n, n), dtype=_tdtype(dtype), device=dev)
    j = torch.arange(n, device=dev, dtype=torch.float64)
    h2 = float(spacing) * float(spacing)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        k = torch.arange(r0, r1, device=dev, dtype=torch.float64)[:, None] - j[None, :]
        sgn = 1.0 - 2.0 * torch.remainder(k, 2.0)
        blk = sgn / ((k * k) * h2)
        idx = torch.arange(r0, r1, device=dev)
        blk[idx - r0, idx] = math.pi ** 2 / 6.0
        out[r0:r1] = blk.to(out.dtype)
    return out


def simple_toeplitz_symbol(n: int):
    """t(k) of SimpleToeplitz (a_ij = t(i - j)): n^2 at k = 0, else k."""
    return lambda k: torch.where(k == 0, torch.full_like(k, float(n) * n), k)


def qchem_toeplitz_symbol(spacing: float = 1.0):
    """t(k) of QChemToeplitz: pi^2/6 at k = 0, else (-1)^k / (k^2 h^2)."""
    h2 = float(spacing) * float(spacing)

    def t(k):
        sgn = 1.0 - 2.0 * torch.remainder(k, 2.0)
        return torch.where(k == 0, torch.full_like(k, math.pi ** 2 / 6.0),
                           sgn / (torch.where(k == 0, torch.ones_like(k), k * k) * h2))
    return t


class ToeplitzOperator:
    """An n x n Toeplitz matrix a_ij = t(i - j) that is never stored (FP64,
    on the device): products with A and A^T through a circulant embedding
    of length 2n (FFT), entries from t.  `sample` and `extract` have the
    form of the matrix-free callbacks of hss_compress_matfree."""

    def __init__(self, n, t, device="cuda"):
        self.n, self.t, self.dev = n, t, _dev(device)
        k = torch.arange(n, dtype=torch.float64, device=self.dev)
        col, row = t(k), t(-k)               # first column t(i), first row t(-j)
        c = torch.cat([col, col.new_zeros(1), row[1:].flip(0)])
        ct = torch.cat([row, row.new_zeros(1), col[1:].flip(0)])
        self.fc, self.fct = torch.fft.rfft(c), torch.fft.rfft(ct)

    def _mul(self, f, X):
        n = self.n
        Xp = torch.zeros((2 * n, X.shape[1]), dtype=torch.float64, device=self.dev)
        Xp[:n] = X
        return torch.fft.irfft(f[:, None] * torch.fft.rfft(Xp, dim=0), n=2 * n, dim=0)[:n]

    def matmul(self, X):
        """A X for an n x k FP64 device block (row-major result)."""
        return self._mul(self.fc, X).contiguous()

    def sample(self, R, Sr, Sc):
        Sr.copy_(self._mul(self.fc, R))
        if Sc is not None:
            Sc.copy_(self._mul(self.fct, R))

    def extract(self, rows, cols, out):
        k = rows.double()[:, None] - cols.double()[None, :]
        out.copy_(self.t(k))


def _tdtype(dtype):
    if dtype in (np.float32, "float32", "f32") or dtype == torch.float32:
        return torch.float32
    return torch.float64


def _chunked_kernel(points: np.ndarray, fn, dtype, device, chunk=2048):
    """Dense kernel matrix, row blocks of `chunk`: fn(d2, r0, r1) maps the FP64
    squared distances of rows [r0, r1) to the block's values.  d2 is summed
    coordinate by coordinate in a fixed order with one rounding per operation,
    so it is bitwise the same on the CPU and on the GPU."""
    dev = _dev(device)
    x = torch.as_tensor(points, dtype=torch.float64, device=dev)
    n = x.shape[0]
    out = torch.empty((n, n), dtype=_tdtype(dtype), device=dev)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        d2 = None
        for a in range(x.shape[1]):
            t = x[r0:r1, a, None] - x[None, :, a]
            t = t * t
            d2 = t if d2 is None else d2 + t
        blk = fn(d2, r0, r1)
        out[r0:r1] = blk.to(out.dtype)
    return out


def gaussian_kernel(points: np.ndarray, h: float, lam: float, dtype=np.float32, device="cpu"):
    """K_ij = exp(-|x_i-x_j|^2 / (2 h^2)) + lam * delta_ij (computed in FP64)."""
    def fn(d2, r0, r1):
        k = torch.exp(-d2 / (2.0 * h * h))
        idx = torch.arange(r0, r1, device=k.device)
        k[idx - r0, idx] += lam
        return k
    return _chunked_kernel(points, fn, dtype, device)


def bem_like(points: np.ndarray, dtype=np.float32, device="cpu"):
    """a_ij = 1/(4 pi |x_i-x_j|) for i != j, a_ii = sqrt(n) (computed in FP64
    with correctly rounded operations only: the same bits on CPU and GPU)."""
    n = points.shape[0]
    diag = math.sqrt(n)
    four_pi = 4.0 * math.pi

    def fn(d2, r0, r1):
        idx = torch.arange(r0, r1, device=d2.device)
        d2[idx - r0, idx] = 1.0
        k = torch.reciprocal(torch.sqrt(d2) * four_pi)
        k[idx - r0, idx] = diag
        return k
    return _chunked_kernel(points, fn, dtype, device)


def fingerprint(A) -> str:
    """Exact integer fingerprint of a matrix's stored bytes (any device):
    with w_i the row sums of the entries' bit patterns read as signed
    integers, returns hex(sum_i w_i) + ":" + hex(sum_i (i + 1) w_i)."""
    if torch is None:
        raise RuntimeError("torch is required")
    t = torch.as_tensor(A)
    ity = {4: torch.int32, 8: torch.int64, 2: torch.int16}[t.element_size()]
    s1 = s2 = 0
    for r0 in range(0, t.shape[0], 1024):
        blk = t[r0:r0 + 1024].contiguous().view(ity)
        if ity == torch.int64:   # split into two 32-bit halves to keep the sums exact
            lo = (blk & 0xFFFFFFFF).sum(dim=1)
            hi = (blk >> 32).sum(dim=1)
            w = [int(a) + (int(b) << 32) for a, b in zip(lo.tolist(), hi.tolist())]
        else:
            w = [int(v) for v in blk.to(torch.int64).sum(dim=1).tolist()]
        for i, v in enumerate(w):
            s1 += v
            s2 += (r0 + i + 1) * v
    return f"{s1:x}:{s2:x}"


# ---------------------------------------------------------------- cluster trees
def comb_tree_splits(n: int, leaf_size: int) -> list:
    """Split list (one entry per node, breadth-first, -1 = leaf) of a "comb"
    tree: every non-leaf splits off a leaf of leaf_size indices on its left
    and recurses on the rest, until the rest fits in a leaf (the unbalanced
    tree of the paper's Section 4 tree comparison).  Breadth-first, each
    depth holds the left leaf and then the remainder node, so the list is
    [split, -1, split, -1, ..., -1, -1]."""
    out = []
    lo = 0
    while n - lo > leaf_size:
        out.append(lo + leaf_size)   # node [lo, n): left leaf, right remainder
        out.append(-1)               # the left leaf of the next depth
        lo += leaf_size
    out.append(-1)                   # the last remainder
    return out


def split_intervals(n: int, splits) -> list:
    """(lo, hi, depth, parent, children) of every node of a split list, in
    breadth-first order (the input-side description of a caller's tree)."""
    nodes = [[0, n, 0, -1, ()]]
    q = 0
    while q < len(nodes):
        lo, hi, dep, _, _ = nodes[q]
        mid = splits[q]
        if mid != -1:
            if not lo < mid < hi:
                raise ValueError("split outside its node")
            a = len(nodes)
            nodes.append([lo, mid, dep + 1, q, ()])
            nodes.append([mid, hi, dep + 1, q, ()])
            nodes[q][4] = (a, a + 1)
        q += 1
    if len(nodes) != len(splits):
        raise ValueError("split list length does not match the tree")
    return [tuple(x) for x in nodes]


# ------------------------------------------------ known-rank random HSS input
def bisection_intervals(n: int, leaf_size: int):
    """Cluster tree by bisection, as nested tuples (lo, hi, left, right).

    Input-side copy of the tree rule (left child gets floor(s/2) indices, a
    range of <= leaf_size indices is a leaf); used only to lay out the random
    generators of ``random_hss``.
    """
    def rec(lo, hi):
        s = hi - lo
        if s <= leaf_size:
            return (lo, hi, None, None)
        mid = lo + s // 2
        return (lo, hi, rec(lo, mid), rec(mid, hi))
    return rec(0, n)


def random_hss(n: int, leaf_size: int, rank: int, seed: int, diag_shift: float = 0.0):
    """Dense n x n matrix whose every off-diagonal Hankel block has rank `rank`.

    Random Gaussian generators are drawn at every node: D at the leaves, U and
    V (size m x rank, m = leaf size or 2*rank) at every non-root node, B12 and
    B21 (rank x rank) at every non-leaf.  The dense matrix is assembled from
    the nested bases U^big = diag(U^big_1, U^big_2) U.  Returns (A, info) where
    info maps (lo, hi) of every non-root node to its row/column rank.
    """
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    ranks = {}

    def rec(node, is_root):
        lo, hi, left, right = node
        if left is None:
            m = hi - lo
            A[lo:hi, lo:hi] = rng.standard_normal((m, m)) + diag_shift * np.eye(m)
            k = min(rank, m)
            ub = rng.standard_normal((m, k))
            vb = rng.standard_normal((m, k))
        else:
            u1, v1 = rec(left, False)
            u2, v2 = rec(right, False)
            l0, l1 = left[0], left[1]
            r0, r1 = right[0], right[1]
            b12 = rng.standard_normal((u1.shape[1], v2.shape[1]))
            b21 = rng.standard_normal((u2.shape[1], v1.shape[1]))
            A[l0:l1, r0:r1] = u1 @ b12 @ v2.T
            A[r0:r1, l0:l1] = u2 @ b21 @ v1.T
            if is_root:
                return None, None
            m = u1.shape[1] + u2.shape[1]
            k = min(rank, m)
            ut = rng.standard_normal((m, k))
            vt = rng.standard_normal((m, k))
            ub = np.vstack([u1 @ ut[: u1.shape[1]], u2 @ ut[u1.shape[1]:]])
            vb = np.vstack([v1 @ vt[: v1.shape[1]], v2 @ vt[v1.shape[1]:]])
        ranks[(lo, hi)] = ub.shape[1]
        return ub, vb

    root = bisection_intervals(n, leaf_size)
    if root[2] is None:
        A[:, :] = rng.standard_normal((n, n)) + diag_shift * np.eye(n)
    else:
        rec(root, True)
    return A, ranks


# ------------------------------------------- Schur complement of a 3D Laplacian
def dst_basis(k: int) -> np.ndarray:
    """Orthonormal DST-I basis: phi[i, p] = sqrt(2/(k+1)) sin((i+1)(p+1) pi/(k+1))."""
    i = np.arange(1, k + 1)
    return np.sqrt(2.0 / (k + 1)) * np.sin(np.outer(i, i) * np.pi / (k + 1))


def laplacian_schur_eigs(k: int) -> np.ndarray:
    """Eigenvalues s[p, q] of the middle-plane Schur complement.

    With the 2D sine transform of the k x k plane, the 7-point operator splits
    into independent chains along z (diagonal 2 + mu_p + mu_q, off-diagonal
    -1, mu_p = 2 - 2 cos(p pi/(k+1))).  Eliminating the k-node chain on each
    side of the middle node leaves s = a - 2 c_k, with a = 2 + mu_p + mu_q,
    c_1 = 1/a, c_j = 1/(a - c_{j-1}) (the last diagonal entry of the inverse
    of a k-node chain).
    """
    p = np.arange(1, k + 1)
    mu = 2.0 - 2.0 * np.cos(p * np.pi / (k + 1))
    a = 2.0 + mu[:, None] + mu[None, :]
    c = 1.0 / a
    for _ in range(k - 1):
        c = 1.0 / (a - c)
    return a - 2.0 * c


def laplacian_schur(k: int, dtype=np.float32, device="cpu"):
    """Dense n x n (n = k^2) Schur complement S = A22 - A21 A11^{-1} A12 of the
    7-point Laplacian on a k x k x (2k+1) grid split at the middle plane, from
    its closed form S = (phi x phi) diag(s) (phi x phi)^T, computed in FP64."""
    dev = _dev(device)
    phi = torch.as_tensor(dst_basis(k), dtype=torch.float64, device=dev)
    sv = torch.as_tensor(laplacian_schur_eigs(k), dtype=torch.float64, device=dev)
    # M[p, i2, j2] = sum_q s[p,q] phi[i2,q] phi[j2,q]
    M = torch.einsum("pq,iq,jq->pij", sv, phi, phi).reshape(k, k * k)
    # S[(i1, j1), (i2, j2)] = sum_p phi[i1,p] phi[j1,p] M[p, (i2, j2)]
    PP = (phi[:, None, :] * phi[None, :, :]).reshape(k * k, k)
    S = (PP @ M).reshape(k, k, k, k).permute(0, 2, 1, 3).reshape(k * k, k * k)
    return S.to(_tdtype(dtype)).contiguous()


# --------------------------------------------------- mixed batch of matrices
def mixed_batch_specs(count: int, seed: int, n_range=(1000, 8000)):
    """Specs of `count` independent matrices for batched compression: n uniform
    in n_range, half Toeplitz a_ij = 1/(1+|i-j|) (a_ii = 10), half Gaussian
    kernel (h uniform in [0.1, 0.4], lambda = 1, points uniform in the unit
    cube in RCB order).  Per-family settings: Toeplitz rtol 1e-6, d0/step
    64/32; Gaussian rtol 1e-4, 128/64; leaf 128 below n = 4000, else 256."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        leaf = 128 if n < 4000 else 256
        if rng.random() < 0.5:
            out.append(dict(family="toeplitz_inv_distance", n=n, leaf=leaf, rtol=1e-6,
                            d0=64, step=32))
        else:
            out.append(dict(family="gaussian_kernel", n=n, leaf=leaf, rtol=1e-4, d0=128,
                            step=64, h=float(rng.uniform(0.1, 0.4)), lam=1.0,
                            seed=int(rng.integers(1 << 31))))
    return out


def build_matrix(spec: dict, dtype=np.float32, device="cpu"):
    """Dense matrix of one spec from mixed_batch_specs (or of the same keys)."""
    fam = spec["family"]
    if fam == "toeplitz_inv_distance":
        return toeplitz_inv_distance(spec["n"], dtype=dtype, device=device).contiguous()
    if fam == "gaussian_kernel":
        pts = points_unit_cube(spec["n"], spec["seed"])
        pts = pts[rcb_order(pts, spec["leaf"])]
        return gaussian_kernel(pts, spec["h"], spec["lam"], dtype=dtype, device=device)
    if fam == "laplacian_schur":
        return laplacian_schur(spec["k"], dtype=dtype, device=device)
    raise ValueError(fam)
