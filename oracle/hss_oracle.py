"""Plain FP64 CPU oracle for randomized HSS compression, product and ULV solve.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference that the GPU path is checked against.  Only the test-suite, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
library itself never calls it and shares no code with it.

What it follows (Rouet, Li, Ghysels, Napov, "A distributed-memory package for
dense HSS matrix computations using randomization", arXiv:1503.05464):

* cluster tree by bisection                      -- Section 2.1, Fig. 1
* random test matrix R and samples S^r = A R,
  S^c = A^T R                                     -- Section 2.2
* interpolative decomposition by truncated
  column-pivoted QR, stop at |R_ii| <= eps |R_11| -- Section 2.2, Section 3.1
* compression                                     -- Algorithm 1
* adaptive sampling, "late notification" form     -- Section 3.2, Algorithm 5
* HSS matrix-vector product                       -- Algorithm 2
* ULV-like factorization                          -- Algorithm 3
* solution with the ULV factors                   -- Algorithm 4, Appendix A

Readings taken where the paper is silent:

* One random matrix R serves both samples (S^r = A R, S^c = A^T R).
* R[i, j] is a standard Gaussian made from the splitmix64 sequence with
  Box-Muller, then rounded to the nearest bfloat16 value.
* ID threshold: stop at the first i with |R_ii| <= max(rtol |R_11|, atol);
  rank = number of columns eliminated before it, else min(rows, cols).
* A node fails (adaptive sampling) iff d < m and k > d - p on either side,
  where m is the number of rows of its local sample and p the oversampling.
* Level-synchronous schedule: each pass visits the tree by depth, deepest
  first; a COMPRESSED node only extends its samples with the new columns,
  every other node whose children are all COMPRESSED recomputes its local
  samples with all d columns and retries the ID.
* Root: no ID; B12/B21 are gathered and the ULV root is LU with partial
  pivoting.
* Symmetric matrices (optional): with A = A^T and one R for both samples,
  S^c = A^T R = A R = S^r, so every column-side quantity repeats the row
  side: the column ID is the row ID (V = U, I^c = I^r) and R^c_tau = R^r_tau.

Pins for every function here live in tests/test_oracle.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

UNTOUCHED, PARTIALLY, COMPRESSED = 0, 1, 2

# ---------------------------------------------------------------- cluster tree


@dataclass
class Node:
    """One cluster-tree node: index interval [lo, hi) (Section 2.1)."""
    id: int
    lo: int
    hi: int
    depth: int
    parent: int = -1
    children: tuple = ()

    @property
    def size(self):
        return self.hi - self.lo

    @property
    def is_leaf(self):
        return not self.children


def bisection_tree(n: int, leaf_size: int) -> list[Node]:
    """Cluster tree of [0, n) by bisection (Section 2.1, Fig. 1).

    A node with s > leaf_size indices gets children [lo, lo + floor(s/2)) and
    [lo + floor(s/2), hi).  Nodes are numbered breadth-first, root = 0.
    """
    if n <= 0 or leaf_size <= 0:
        raise ValueError("n and leaf_size must be positive")
    nodes = [Node(0, 0, n, 0)]
    q = 0
    while q < len(nodes):
        nd = nodes[q]
        q += 1
        if nd.size > leaf_size:
            mid = nd.lo + nd.size // 2
            a = Node(len(nodes), nd.lo, mid, nd.depth + 1, nd.id)
            nodes.append(a)
            b = Node(len(nodes), mid, nd.hi, nd.depth + 1, nd.id)
            nodes.append(b)
            nd.children = (a.id, b.id)
    return nodes


# ------------------------------------------------------ random test matrix R
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def _splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """counter-th output of the splitmix64 generator started at `seed`.

    splitmix64 advances its state by the golden-ratio constant and outputs the
    mix of the state, so output number c (c >= 1) is mix(seed + c * gamma).
    """
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + c * np.uint64(_GAMMA)
        return _splitmix64_mix(z)


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 value (ties to even).

    bfloat16 keeps 8 significant bits: write x = f * 2^e with f in [0.5, 1),
    round f * 256 to the nearest integer (half to even), scale back.
    """
    f, e = np.frexp(x)
    return np.ldexp(np.round(f * 256.0) / 256.0, e)


def gaussian_bf16(seed: int, rows: int, c0: int, c1: int) -> np.ndarray:
    """Columns [c0, c1) of the n x d random matrix R (Section 2.2, Alg. 1 data).

    Entry (i, j) uses splitmix64 outputs 2q+1 and 2q+2 with q = i * 2^32 + j:
    u1 = (top 53 bits + 1) / 2^53 in (0, 1], u2 = top 53 bits / 2^53 in [0, 1),
    g = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller), then rounded to bfloat16.
    """
    i = np.arange(rows, dtype=np.uint64)[:, None]
    j = np.arange(c0, c1, dtype=np.uint64)[None, :]
    q = (i << np.uint64(32)) | j
    a = splitmix64(0 if seed is None else seed, np.uint64(2) * q + np.uint64(1))
    b = splitmix64(0 if seed is None else seed, np.uint64(2) * q + np.uint64(2))
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (b >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return round_to_bf16(g)


# ------------------------------------------------ interpolative decomposition


@dataclass
class ID:
    """[X, J] = ID(Y, eps) with X = [I  T] P^T, T = R1^{-1} R2 (Section 2.2).

    perm[:k] = J are the selected columns of Y, perm[k:] the rest; E = T^T, so
    that the generator X^T = Pi [I; E] has the paper's U = Pi [I; E] form.
    """
    k: int
    perm: np.ndarray
    E: np.ndarray          # (m - k) x k
    rdiag: np.ndarray      # |R_ii| of the pivoted QR, for tests

    @property
    def J(self):
        return self.perm[: self.k]

    def basis(self) -> np.ndarray:
        """Dense m x k generator Pi [I; E]."""
        m = self.perm.size
        G = np.zeros((m, self.k))
        G[self.perm[: self.k], :] = np.eye(self.k)
        G[self.perm[self.k:], :] = self.E
        return G


def interpolative_decomposition(Y: np.ndarray, rtol: float, atol: float = 0.0) -> ID:
    """Truncated CPQR interpolative decomposition of Y (d x m) (Section 2.2, 3.1).

    Y P = Q [R1 R2]; the factorization stops at the first i with
    |R_ii| <= max(rtol |R_11|, atol); k = i.  If R_11 = 0, k = 0.
    The full LAPACK pivoted QR is taken and truncated: its first k pivots are
    exactly those of the truncated one.
    """
    d, m = Y.shape
    if m == 0:
        return ID(0, np.zeros(0, dtype=np.int64), np.zeros((0, 0)), np.zeros(0))
    if d == 0:
        return ID(0, np.arange(m), np.zeros((m, 0)), np.zeros(0))
    _, R, P = sla.qr(Y, mode="economic", pivoting=True)
    rd = np.abs(np.diag(R))
    k = rd.size
    if rd[0] == 0.0:
        k = 0
    else:
        thr = max(rtol * rd[0], atol)
        small = np.nonzero(rd <= thr)[0]
        if small.size:
            k = int(small[0])
    T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False) if k else np.zeros((0, m))
    return ID(k, P.astype(np.int64), np.ascontiguousarray(T.T), rd)


# ------------------------------------------------------------- compression


@dataclass
class NodeData:
    state: int = UNTOUCHED
    ncols: int = 0                       # sample columns incorporated so far
    d_compressed: int = 0                # sample count when the ID succeeded
    idr: ID | None = None                # row ID  -> U = Pi^r [I; E^r]
    idc: ID | None = None                # column ID -> V = Pi^c [I; E^c]
    Sr: np.ndarray | None = None         # S^r_tau  (k^r x d)
    Sc: np.ndarray | None = None         # S^c_tau  (k^c x d)
    Rr: np.ndarray | None = None         # R^r_tau = V^T R_in  (k^c x d)
    Rc: np.ndarray | None = None         # R^c_tau = U^T R_in  (k^r x d)
    Ir: np.ndarray | None = None         # global row skeleton I^r_tau
    Ic: np.ndarray | None = None         # global column skeleton I^c_tau
    D: np.ndarray | None = None          # leaves
    B12: np.ndarray | None = None        # non-leaves
    B21: np.ndarray | None = None

    @property
    def U(self):
        return self.idr.basis()

    @property
    def V(self):
        return self.idc.basis()


@dataclass
class HSS:
    n: int
    nodes: list
    data: list
    d: int
    passes: int
    rtol: float
    ulv: dict = field(default_factory=dict)

    def ranks(self):
        """{node id: (k^r, k^c)} for every non-root node."""
        return {nd.id: (self.data[nd.id].idr.k, self.data[nd.id].idc.k)
                for nd in self.nodes if nd.id != 0}

    def max_rank(self):
        r = self.ranks()
        return max((max(a, b) for a, b in r.values()), default=0)


class RankCapError(RuntimeError):
    pass


def compress(A, rtol, atol=0.0, leaf_size=128, d0=64, d_step=32, d_max=None,
             oversample_p=10, seed=0, tree=None, symmetric=False) -> HSS:
    """Randomized HSS compression, Algorithm 1 with Algorithm 5's adaptivity.

    A is upcast to FP64 as given (the stored values are the matrix).
    symmetric=True takes A = A^T (not checked): S^c is S^r (Section 2.2's
    samples with one R), the column side of every node is its row side
    (idc is idr, Sc/Rc/Ic are Sr/Rr/Ir); B12 and B21 are still read from A.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("A must be square")
    nodes = tree if tree is not None else bisection_tree(n, leaf_size)
    data = [NodeData() for _ in nodes]
    if d_max is None:
        d_max = n
    d = min(d0, d_max)
    R = gaussian_bf16(seed, n, 0, d)
    Sr = A @ R
    Sc = Sr if symmetric else A.T @ R
    maxdepth = max(nd.depth for nd in nodes)
    passes = 0
    for nd in nodes:
        if nd.is_leaf:
            data[nd.id].D = A[nd.lo:nd.hi, nd.lo:nd.hi].copy()
    while True:
        passes += 1
        for depth in range(maxdepth, 0, -1):
            for nd in nodes:
                if nd.depth == depth:
                    _process_node(A, R, Sr, Sc, nodes, data, nd, d, rtol, atol, oversample_p,
                                  symmetric)
        root = nodes[0]
        if root.is_leaf or all(data[c].state == COMPRESSED for c in root.children):
            if not root.is_leaf:
                c1, c2 = (data[c] for c in root.children)
                data[0].B12 = A[np.ix_(c1.Ir, c2.Ic)]
                data[0].B21 = A[np.ix_(c2.Ir, c1.Ic)]
            data[0].state = COMPRESSED
            break
        if d >= d_max:
            raise RankCapError(f"sample count reached d_max={d_max} without convergence")
        dn = min(d + d_step, d_max)
        Rn = gaussian_bf16(seed, n, d, dn)
        R = np.hstack([R, Rn])
        Sr = np.hstack([Sr, A @ Rn])
        Sc = Sr if symmetric else np.hstack([Sc, A.T @ Rn])
        d = dn
    return HSS(n, nodes, data, d, passes, rtol)


def _local_samples(A, R, Sr, Sc, nodes, data, nd, cols):
    """S^r_loc, S^c_loc and the stacked R inputs for columns `cols` (Alg. 1)."""
    if nd.is_leaf:
        I = slice(nd.lo, nd.hi)
        D = data[nd.id].D
        Rin = R[I, cols]
        srl = Sr[I, cols] - D @ Rin
        scl = Sc[I, cols] - D.T @ Rin
        return srl, scl, Rin, Rin
    c1, c2 = (data[c] for c in nd.children)
    me = data[nd.id]
    srl = np.vstack([c1.Sr[:, cols] - me.B12 @ c2.Rr[:, cols],
                     c2.Sr[:, cols] - me.B21 @ c1.Rr[:, cols]])
    scl = np.vstack([c1.Sc[:, cols] - me.B21.T @ c2.Rc[:, cols],
                     c2.Sc[:, cols] - me.B12.T @ c1.Rc[:, cols]])
    rin_r = np.vstack([c1.Rr[:, cols], c2.Rr[:, cols]])   # feeds R^r_tau = V^T [.]
    rin_c = np.vstack([c1.Rc[:, cols], c2.Rc[:, cols]])   # feeds R^c_tau = U^T [.]
    return srl, scl, rin_r, rin_c


def _fails(k, d, m, p):
    """Adaptive failure test: the rank is too close to the sample count."""
    return d < m and k > d - p


def _process_node(A, R, Sr, Sc, nodes, data, nd, d, rtol, atol, p, symmetric=False):
    """Process one node in one pass (Algorithm 5 in level-synchronous form).
    symmetric: the column side is the row side (see compress)."""
    me = data[nd.id]
    if not nd.is_leaf and any(data[c].state != COMPRESSED for c in nd.children):
        me.state = UNTOUCHED
        return
    if not nd.is_leaf and me.state != COMPRESSED:
        c1, c2 = (data[c] for c in nd.children)
        me.B12 = A[np.ix_(c1.Ir, c2.Ic)]
        me.B21 = A[np.ix_(c2.Ir, c1.Ic)]
    if me.state == COMPRESSED:
        if me.ncols == d:
            return
        cols = slice(me.ncols, d)
        srl, scl, rin_r, rin_c = _local_samples(A, R, Sr, Sc, nodes, data, nd, cols)
        me.Sr = np.hstack([me.Sr, srl[me.idr.J]])
        me.Rr = np.hstack([me.Rr, me.V.T @ rin_r])
        if symmetric:
            me.Sc, me.Rc = me.Sr, me.Rr
        else:
            me.Sc = np.hstack([me.Sc, scl[me.idc.J]])
            me.Rc = np.hstack([me.Rc, me.U.T @ rin_c])
        me.ncols = d
        return
    cols = slice(0, d)
    srl, scl, rin_r, rin_c = _local_samples(A, R, Sr, Sc, nodes, data, nd, cols)
    m = srl.shape[0]
    idr = interpolative_decomposition(srl.T, rtol, atol)
    if _fails(idr.k, d, m, p):
        me.state = PARTIALLY
        return
    if symmetric:
        idc = idr
    else:
        idc = interpolative_decomposition(scl.T, rtol, atol)
        if _fails(idc.k, d, scl.shape[0], p):
            me.state = PARTIALLY
            return
    me.idr, me.idc = idr, idc
    me.Sr = srl[idr.J]
    me.Rr = me.V.T @ rin_r
    if nd.is_leaf:
        idx = np.arange(nd.lo, nd.hi)
        me.Ir = idx[idr.J]
    else:
        c1, c2 = (data[c] for c in nd.children)
        me.Ir = np.concatenate([c1.Ir, c2.Ir])[idr.J]
    if symmetric:
        me.Sc, me.Rc, me.Ic = me.Sr, me.Rr, me.Ir
    else:
        me.Sc = scl[idc.J]
        me.Rc = me.U.T @ rin_c
        if nd.is_leaf:
            me.Ic = np.arange(nd.lo, nd.hi)[idc.J]
        else:
            me.Ic = np.concatenate([c1.Ic, c2.Ic])[idc.J]
    me.ncols = d
    me.d_compressed = d
    me.state = COMPRESSED


def leaf_local_samples(A, R, nodes):
    """Algorithm 1's leaf samples for every leaf, stacked in index order:
    S^r_loc(I_t,:) = S^r(I_t,:) - D_t R(I_t,:) and S^c_loc = S^c(I_t,:) - D_t^T R(I_t,:)
    with S^r = A R, S^c = A^T R (Section 2.2)."""
    A = np.asarray(A, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    Sr = A @ R
    Sc = A.T @ R
    for nd in nodes:
        if nd.is_leaf:
            I = slice(nd.lo, nd.hi)
            D = A[I, I]
            Sr[I] -= D @ R[I]
            Sc[I] -= D.T @ R[I]
    return Sr, Sc


# ------------------------------------------------------ dense reconstruction


def to_dense(h: HSS) -> np.ndarray:
    """Dense H from the generators by the nested-basis definition (Section 2.1).

    H(I_t, I_t) = D_t at leaves; H(I_1, I_2) = U^big_1 B12 (V^big_2)^T with
    U^big = diag(U^big_c1, U^big_c2) U at non-leaves.
    """
    H = np.zeros((h.n, h.n))
    big = {}
    for nd in sorted(h.nodes, key=lambda x: -x.depth):
        me = h.data[nd.id]
        if nd.is_leaf:
            H[nd.lo:nd.hi, nd.lo:nd.hi] = me.D
            if nd.id != 0:
                big[nd.id] = (me.U, me.V)
            continue
        a, b = nd.children
        na, nb = h.nodes[a], h.nodes[b]
        ua, va = big[a]
        ub, vb = big[b]
        H[na.lo:na.hi, nb.lo:nb.hi] = ua @ me.B12 @ vb.T
        H[nb.lo:nb.hi, na.lo:na.hi] = ub @ me.B21 @ va.T
        if nd.id != 0:
            U = me.U
            V = me.V
            ka, kb = ua.shape[1], ub.shape[1]
            la, lb = va.shape[1], vb.shape[1]
            big[nd.id] = (np.vstack([ua @ U[:ka], ub @ U[ka:ka + kb]]),
                          np.vstack([va @ V[:la], vb @ V[la:la + lb]]))
    return H


# ------------------------------------------------------------- Algorithm 2


def matvec(h: HSS, X: np.ndarray) -> np.ndarray:
    """b = H x by the two tree traversals of Algorithm 2."""
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    nodes = h.nodes
    if nodes[0].is_leaf:
        out = h.data[0].D @ X
        return out[:, 0] if vec else out
    y = {}
    for nd in sorted(nodes, key=lambda x: -x.depth):
        if nd.id == 0:
            continue
        me = h.data[nd.id]
        if nd.is_leaf:
            y[nd.id] = me.V.T @ X[nd.lo:nd.hi]
        else:
            a, b = nd.children
            y[nd.id] = me.V.T @ np.vstack([y[a], y[b]])
    z = {0: None}
    out = np.zeros((h.n, X.shape[1]))
    for nd in sorted(nodes, key=lambda x: x.depth):
        me = h.data[nd.id]
        if nd.is_leaf:
            out[nd.lo:nd.hi] = me.U @ z[nd.id] + me.D @ X[nd.lo:nd.hi]
            continue
        a, b = nd.children
        za = me.B12 @ y[b]
        zb = me.B21 @ y[a]
        if nd.id != 0:
            uz = me.U @ z[nd.id]
            ka = h.data[a].idr.k
            za = za + uz[:ka]
            zb = zb + uz[ka:]
        z[a], z[b] = za, zb
    return out[:, 0] if vec else out


# ------------------------------------------------------------- Algorithm 3


def _omega(idr: ID) -> np.ndarray:
    """Omega = [-E I; I 0] Pi^T, so that Omega U = [0; I] (Section 2.4)."""
    m, k = idr.perm.size, idr.k
    Om = np.zeros((m, m))
    P = np.zeros((m, m))                 # Pi: column j of Pi is e_{perm[j]}
    P[idr.perm, np.arange(m)] = 1.0
    T = np.zeros((m, m))
    T[: m - k, :k] = -idr.E
    T[: m - k, k:] = np.eye(m - k)
    T[m - k:, :k] = np.eye(k)
    Om = T @ P.T
    return Om


def ulv_factor(h: HSS) -> None:
    """ULV-like factorization, Algorithm 3; stores factors in h.ulv."""
    F = {}
    nodes = h.nodes
    for nd in sorted(nodes, key=lambda x: -x.depth):
        me = h.data[nd.id]
        f = {}
        if nd.is_leaf:
            Dt = me.D
            if nd.id != 0:
                Vhat = me.V
        else:
            a, b = nd.children
            fa, fb = F[a], F[b]
            Dt = np.block([[fa["Dtil"], me.B12 @ fb["Vtb"].T],
                           [me.B21 @ fa["Vtb"].T, fb["Dtil"]]])
            if nd.id != 0:
                Vhat = sla.block_diag(fa["Vtb"], fb["Vtb"]) @ me.V
        if nd.id == 0:
            f["lu"] = sla.lu_factor(Dt)
            f["m"] = Dt.shape[0]
            F[0] = f
            break
        k = me.idr.k
        m = Dt.shape[0]
        Om = _omega(me.idr)
        W = Om @ Dt
        Wt, Wb = W[: m - k], W[m - k:]
        if m - k > 0:
            Qf, Rf = sla.qr(Wt.T, mode="full")        # Wt^T = Qf Rf -> Wt = [L 0] Q
            L = Rf[: m - k, :].T
            Q = Qf.T
        else:
            L = np.zeros((0, 0))
            Q = np.eye(m)
        Qt, Qb = Q[: m - k], Q[m - k:]
        Vt = Q @ Vhat
        f.update(Om=Om, Wb=Wb, L=L, Q=Q, Qt=Qt, Qb=Qb,
                 Vtt=Vt[: m - k], Vtb=Vt[m - k:], Dtil=Wb @ Qb.T, k=k, m=m)
        F[nd.id] = f
    h.ulv = F


# ------------------------------------------------------------- Algorithm 4


def ulv_solve(h: HSS, B: np.ndarray) -> np.ndarray:
    """Solve H x = b with the ULV factors (Algorithm 4, Appendix A)."""
    if not h.ulv:
        raise RuntimeError("ulv_factor must run before ulv_solve")
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    if vec:
        B = B[:, None]
    F = h.ulv
    nodes = h.nodes
    if nodes[0].is_leaf:
        x = sla.lu_solve(F[0]["lu"], B)
        return x[:, 0] if vec else x
    bt, y, z, xs = {}, {}, {}, {}
    for nd in sorted(nodes, key=lambda x: -x.depth):
        me = h.data[nd.id]
        if nd.is_leaf:
            b = B[nd.lo:nd.hi]
        else:
            a, c = nd.children
            fa, fc = F[a], F[c]
            ta = bt[a][fa["m"] - fa["k"]:] - fa["Wb"] @ fa["Qt"].T @ y[a] - me.B12 @ z[c]
            tc = bt[c][fc["m"] - fc["k"]:] - me.B21 @ z[a] - fc["Wb"] @ fc["Qt"].T @ y[c]
            b = np.vstack([ta, tc])
        if nd.id == 0:
            xs[0] = sla.lu_solve(F[0]["lu"], b)
            break
        f = F[nd.id]
        bt[nd.id] = f["Om"] @ b
        nt = f["m"] - f["k"]
        y[nd.id] = sla.solve_triangular(f["L"], bt[nd.id][:nt], lower=True) if nt else np.zeros((0, B.shape[1]))
        zz = f["Vtt"].T @ y[nd.id]
        if not nd.is_leaf:
            a, c = nd.children
            zz = zz + me.V.T @ np.vstack([z[a], z[c]])
        z[nd.id] = zz
    X = np.zeros((h.n, B.shape[1]))
    for nd in sorted(nodes, key=lambda x: x.depth):
        if nd.is_leaf:
            X[nd.lo:nd.hi] = xs[nd.id]
            continue
        a, c = nd.children
        ka = h.data[a].idr.k
        xt, xb = xs[nd.id][:ka], xs[nd.id][ka:]
        xs[a] = F[a]["Q"].T @ np.vstack([y[a], xt])
        xs[c] = F[c]["Q"].T @ np.vstack([y[c], xb])
    return X[:, 0] if vec else X
