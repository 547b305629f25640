"""Zoom-SVD oracle in plain FP64 numpy — test infrastructure, not product code.

Follows the paper step by step:
  * Section 2.1  SVD, low-rank truncation, Eckart-Young error, Eq. 1 (xi rule)
  * Section 2.2 / Eq. 2-3  incremental SVD row append
  * Algorithm 1 (Section 3.2)  storage phase, Def. 1 blocks, Def. 2 sets
  * Algorithm 3 / Def. 3 / Eq. 5-6 (Section 3.3.1)  Partial-SVD
  * Algorithm 2 / Def. 4 / Eq. 7-9 (Section 3.3.2)  Stitched-SVD and the lift
  * Section 5.4  normalised reconstruction error
The one library primitive is ``numpy.linalg.svd`` (LAPACK gesdd), used as
the "SVD" step wherever the paper says "perform SVD".

Readings taken where the paper is silent or inconsistent (each is also a
test case):
  R1  rows are 0-based and a range [t_s, t_e] is inclusive (Problem 1 gives
      t_e - t_s + 1 rows): S = t_s // b, E = t_e // b, r_S = t_s % b,
      b_S = b - r_S, b_E = t_e % b + 1 (Algorithm 3's b_E = t_e % b is the
      half-open count).
  R2  S == E: one Partial-SVD keeps rows [t_s % b, t_e % b] of that block.
  R3  the last block may hold fewer than b rows (Def. 1 "current block");
      it is compressed as it stands, with rank min(k, rows, n).
  R4  Partial-SVD keeps every column it produces (rank <= min(b_S, k)); the
      stitched result is truncated to k_q = min(k_out, n, R) and padded with
      zero columns to the caller's width k_out.
  R5  singular values <= RANK_TOL * sigma_1 count as zero: their columns are
      output as zeros and rank_out excludes them.
  R6  sign: each pair (u_j, v_j) is flipped so that the entry of v_j with
      the largest magnitude (lowest index on ties) is positive.
  R7  V is n x k (Section 2.1); the store keeps V_i^T (k x n).
  R8  storage truncates once, when a block closes (Algorithm 1 without
      per-row truncation is an exact SVD of the block; Eckart-Young then
      gives the stored rank-k factors).

Parity pins (tests/test_oracle_pins.py): direct SVD of the range of the
reconstructed store (exact identity Eq. 7-9), lossless k = min(b, n) against
the raw range, Eckart-Young error per block, orthonormality, closed forms
(P D Q^T with known D; a single row), Eq. 2-3 incremental equivalence, tiny
exhaustive brute force over every range, and planted-mistake checks.  The xi
rule (Eq. 1) is pinned by hand-computed energies.  No function here is
parity-unpinned.
"""
from __future__ import annotations

import dataclasses

import numpy as np

RANK_TOL = 1e-13


# --------------------------------------------------------------------------
# Section 2.1: SVD, truncation, Eq. 1
# --------------------------------------------------------------------------
def svd(M: np.ndarray):
    """Thin SVD M = U diag(s) Vt, s descending (Section 2.1). LAPACK step."""
    U, s, Vt = np.linalg.svd(np.asarray(M, dtype=np.float64), full_matrices=False)
    return U, s, Vt


def truncate(U, s, Vt, k: int):
    """Top-k low-rank approximation U_k Sigma_k V_k^T (Section 2.1)."""
    k = max(0, min(k, s.shape[0]))
    return U[:, :k], s[:k], Vt[:k, :]


def rank_xi(s: np.ndarray, xi: float) -> int:
    """Eq. 1: smallest k with sum_{i<=k} sigma_i^2 / sum sigma_i^2 >= xi."""
    e = np.asarray(s, dtype=np.float64) ** 2
    tot = e.sum()
    if tot == 0.0:
        return 0
    cum = np.cumsum(e) / tot
    return int(np.searchsorted(cum, xi - 1e-15) + 1)


def canonical_signs(U, s, V):
    """Reading R6: make the largest-|.| entry of each v_j positive."""
    U = U.copy()
    V = V.copy()
    for j in range(V.shape[1]):
        if s[j] == 0.0:
            continue
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0.0:
            V[:, j] = -V[:, j]
            U[:, j] = -U[:, j]
    return U, s, V


def _pad(U, s, V, k_out: int):
    """Output width is always k_out: columns past the computed ones are zero."""
    extra = k_out - s.shape[0]
    if extra <= 0:
        return U, s, V
    return (np.hstack([U, np.zeros((U.shape[0], extra))]), np.concatenate([s, np.zeros(extra)]),
            np.hstack([V, np.zeros((V.shape[0], extra))]))


def _zero_small(U, s, V, ref: float):
    """Reading R5: sigma <= RANK_TOL * ref is zero; its columns are zeroed."""
    s = s.copy()
    U = U.copy()
    V = V.copy()
    dead = s <= RANK_TOL * ref
    s[dead] = 0.0
    U[:, dead] = 0.0
    V[:, dead] = 0.0
    return U, s, V, int((~dead).sum())


# --------------------------------------------------------------------------
# Section 2.2, Eq. 2-3: incremental SVD (row append)
# --------------------------------------------------------------------------
def incremental_svd(U, s, Vt, a):
    """Append row ``a`` to the block whose SVD is U diag(s) Vt (Eq. 2-3).

    [A; a] = blockdiag(U, 1) [diag(s) Vt; a];  SVD of the small stacked
    matrix gives U~ S~ V~^T; the new left factor is blockdiag(U, 1) U~.
    No truncation: the result is an exact SVD of the grown block.
    """
    a = np.asarray(a, dtype=np.float64).reshape(1, -1)
    K = np.vstack([s[:, None] * Vt, a])                 # (k+1) x n
    Ut, st, Vtt = svd(K)
    r, k = U.shape
    B = np.zeros((r + 1, k + 1))
    B[:r, :k] = U
    B[r, k] = 1.0
    return B @ Ut, st, Vtt


# --------------------------------------------------------------------------
# Algorithm 1 / Def. 1-2: storage phase
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Store:
    """The sets U, S, V of Def. 2 (V kept transposed, reading R7)."""
    b: int
    n: int
    k: int
    T: int
    U: list          # U_i  (rows_i x k_i)
    s: list          # sigma_i (k_i,)
    Vt: list         # V_i^T  (k_i x n)

    @property
    def nblocks(self) -> int:
        return len(self.U)

    def rows_of(self, i: int) -> int:
        return self.U[i].shape[0]

    def nbytes(self, itemsize: int = 8) -> int:
        return itemsize * sum(u.size + sv.size + v.size
                              for u, sv, v in zip(self.U, self.s, self.Vt))


def block_bounds(T: int, b: int):
    """Def. 1: block i holds rows [b*i, min(b*i + b, T)) (0-based, R1/R3)."""
    return [(lo, min(lo + b, T)) for lo in range(0, T, b)]


def compress_block(Ab: np.ndarray, k: int):
    """Stored factors of one block: its SVD truncated to k (R8)."""
    U, s, Vt = svd(Ab)
    U, s, Vt = truncate(U, s, Vt, k)
    return U, s, Vt


def compress_block_incremental(Ab: np.ndarray, k: int):
    """Algorithm 1 for one block, row by row via Eq. 2-3, truncating at close."""
    Ab = np.asarray(Ab, dtype=np.float64)
    U, s, Vt = svd(Ab[:1])                       # SVD of the first row
    for t in range(1, Ab.shape[0]):
        U, s, Vt = incremental_svd(U, s, Vt, Ab[t])
    return truncate(U, s, Vt, k)


def compress_block_rowwise(Ab: np.ndarray, k: int, discarded: list | None = None):
    """Algorithm 1 as printed, for one block: every arriving row updates the
    block's rank-k SVD by Eq. 2-3 (SVD of [diag(s) Vt; a] and U <- blockdiag(U,
    1) U~) and the result is truncated back to rank k after every row, so the
    state never holds more than k triplets (the cost of Theorem 1).  Unlike
    compress_block_incremental this is not the block's exact SVD once the
    block's rank exceeds k.  ``discarded`` (if a list) receives the singular
    value dropped at each row (0 while nothing is dropped)."""
    Ab = np.asarray(Ab, dtype=np.float64)
    U, s, Vt = truncate(*svd(Ab[:1]), k)
    for t in range(1, Ab.shape[0]):
        U, s, Vt = incremental_svd(U, s, Vt, Ab[t])
        if discarded is not None:
            discarded.append(float(s[k]) if s.size > k else 0.0)
        U, s, Vt = truncate(U, s, Vt, k)
    return U, s, Vt


def compress_block_xi(Ab: np.ndarray, k: int, xi: float):
    """Stored factors of one block under the energy rule (Eq. 1): rank
    k_i = min(k, smallest rank holding a fraction >= xi of the block's
    energy), kept in arrays of width k with columns k_i.. zero."""
    U, s, Vt = compress_block(Ab, k)
    ki = min(U.shape[1], rank_xi(svd(Ab)[1], xi))
    U, s, Vt = U.copy(), s.copy(), Vt.copy()
    U[:, ki:] = 0.0
    s[ki:] = 0.0
    Vt[ki:, :] = 0.0
    return U, s, Vt


def compress(A: np.ndarray, b: int, k: int, incremental: bool = False, xi: float | None = None,
             rowwise: bool = False) -> Store:
    """Storage phase (Algorithm 1): compress every block of A (T x n); with
    xi, each block keeps the rank Eq. 1 gives it (at most k); with rowwise,
    every block is built row by row with truncation to rank k after each row
    (compress_block_rowwise)."""
    A = np.asarray(A, dtype=np.float64)
    T, n = A.shape
    st = Store(b=b, n=n, k=k, T=T, U=[], s=[], Vt=[])
    if xi is not None:
        def f(Ab, kk):
            return compress_block_xi(Ab, kk, xi)
    elif rowwise:
        f = compress_block_rowwise
    else:
        f = compress_block_incremental if incremental else compress_block
    for lo, hi in block_bounds(T, b):
        U, s, Vt = f(A[lo:hi], k)
        st.U.append(U)
        st.s.append(s)
        st.Vt.append(Vt)
    return st


# --------------------------------------------------------------------------
# Algorithm 3 / Def. 3 / Eq. 5-6: Partial-SVD
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Plan:
    S: int
    E: int
    r_S: int      # rows of block S before t_s (eliminated by X_s)
    b_S: int      # rows of block S kept
    b_E: int      # rows of block E kept
    rows: int     # t_e - t_s + 1


def plan(t_s: int, t_e: int, b: int, T: int) -> Plan:
    """Algorithm 3, first two steps, under reading R1."""
    if not (0 <= t_s <= t_e < T):
        raise ValueError("range out of bounds")
    S, E = t_s // b, t_e // b
    r_S = t_s % b
    return Plan(S=S, E=E, r_S=r_S, b_S=b - r_S, b_E=t_e % b + 1, rows=t_e - t_s + 1)


def elimination_matrix(lo: int, hi: int, rows: int) -> np.ndarray:
    """Def. 3 (Eq. 4): X selecting rows [lo, hi) of a rows-row block."""
    X = np.zeros((hi - lo, rows))
    X[np.arange(hi - lo), np.arange(lo, hi)] = 1.0
    return X


def partial_svd(U, s, Vt, lo: int, hi: int):
    """Algorithm 3 for one boundary block: rows [lo, hi) of U_i Sigma_i V_i^T.

    SVD of X U Sigma -> U~ S~ V~^T, then U' = U~, Sigma' = S~,
    V'^T = V~^T V^T (Eq. 5-6).  Every column is kept (reading R4).
    """
    X = elimination_matrix(lo, hi, U.shape[0])
    Ut, st, Vtt = svd(X @ U @ np.diag(s))
    return Ut, st, Vtt @ Vt


# --------------------------------------------------------------------------
# Algorithm 2 / Def. 4 / Eq. 7-9: Stitched-SVD and the lift
# --------------------------------------------------------------------------
@dataclasses.dataclass
class QueryResult:
    U: np.ndarray      # (t_e - t_s + 1) x k_q
    s: np.ndarray      # k_q, descending
    V: np.ndarray      # n x k_q
    rank: int


def query(st: Store, t_s: int, t_e: int, k_out: int | None = None) -> QueryResult:
    """Query phase (Algorithm 2) for the inclusive range [t_s, t_e]."""
    p = plan(t_s, t_e, st.b, st.T)
    k_out = st.k if k_out is None else k_out
    # Partial-SVD of the boundary blocks (Algorithm 2 first step), R2 for S==E
    lefts, slabs = [], []
    if p.S == p.E:
        Ub, sb, Vtb = partial_svd(st.U[p.S], st.s[p.S], st.Vt[p.S], p.r_S, p.r_S + p.rows)
        lefts.append(Ub)
        slabs.append(sb[:, None] * Vtb)
    else:
        Us, ss, Vts = partial_svd(st.U[p.S], st.s[p.S], st.Vt[p.S], p.r_S, st.rows_of(p.S))
        lefts.append(Us)
        slabs.append(ss[:, None] * Vts)
        for i in range(p.S + 1, p.E):
            lefts.append(st.U[i])
            slabs.append(st.s[i][:, None] * st.Vt[i])
        Ue, se, Vte = partial_svd(st.U[p.E], st.s[p.E], st.Vt[p.E], 0, p.b_E)
        lefts.append(Ue)
        slabs.append(se[:, None] * Vte)
    # Stack Sigma V^T (Algorithm 2, second step)
    M = np.vstack(slabs)
    # Low-rank SVD of the stack (third and fourth steps)
    Ur, sr, Vtr = svd(M)
    kq = min(k_out, st.n, M.shape[0])
    Ur, sr, Vtr = truncate(Ur, sr, Vtr, kq)
    # Lift: U_{S:E} = diag(S:E) U_r, one block at a time (Eq. 9, fifth step)
    parts, off = [], 0
    for Ul, sl in zip(lefts, slabs):
        h = sl.shape[0]
        parts.append(Ul @ Ur[off:off + h])
        off += h
    U = np.vstack(parts)
    V = Vtr.T
    ref = sr[0] if sr.size else 0.0
    U, sr, V, rank = _zero_small(U, sr, V, ref)
    U, sr, V = _pad(U, sr, V, k_out)
    U, sr, V = canonical_signs(U, sr, V)
    return QueryResult(U=U, s=sr, V=V, rank=rank)


def block_diag_left(st: Store, t_s: int, t_e: int):
    """diag(S:E) of Def. 4 materialised (for the identity tests only)."""
    p = plan(t_s, t_e, st.b, st.T)
    mats, slabs = [], []
    rng = [(p.S, p.r_S, p.r_S + p.rows)] if p.S == p.E else (
        [(p.S, p.r_S, st.rows_of(p.S))] + [(i, 0, st.rows_of(i)) for i in range(p.S + 1, p.E)]
        + [(p.E, 0, p.b_E)])
    for i, lo, hi in rng:
        if (i in (p.S, p.E)):
            Ul, sl, Vtl = partial_svd(st.U[i], st.s[i], st.Vt[i], lo, hi)
        else:
            Ul, sl, Vtl = st.U[i], st.s[i], st.Vt[i]
        mats.append(Ul)
        slabs.append(sl[:, None] * Vtl)
    rows = sum(m.shape[0] for m in mats)
    cols = sum(m.shape[1] for m in mats)
    D = np.zeros((rows, cols))
    r = c = 0
    for m in mats:
        D[r:r + m.shape[0], c:c + m.shape[1]] = m
        r += m.shape[0]
        c += m.shape[1]
    return D, np.vstack(slabs)


# --------------------------------------------------------------------------
# Brute force and measures
# --------------------------------------------------------------------------
def reconstruct(st: Store, t_s: int, t_e: int) -> np.ndarray:
    """Rows [t_s, t_e] of A-hat, block by block from the stored factors."""
    out = []
    for i in range(t_s // st.b, t_e // st.b + 1):
        lo = i * st.b
        Ai = (st.U[i] * st.s[i][None, :]) @ st.Vt[i]
        a, z = max(t_s, lo), min(t_e + 1, lo + st.rows_of(i))
        out.append(Ai[a - lo:z - lo])
    return np.vstack(out)


def direct_svd(X: np.ndarray, k_out: int) -> QueryResult:
    """The naive baseline: SVD of the materialised range, truncated to k_q."""
    U, s, Vt = svd(X)
    kq = min(k_out, X.shape[1], X.shape[0])
    U, s, Vt = truncate(U, s, Vt, kq)
    ref = s[0] if s.size else 0.0
    U, s, V, rank = _zero_small(U, s, Vt.T, ref)
    U, s, V = _pad(U, s, V, k_out)
    U, s, V = canonical_signs(U, s, V)
    return QueryResult(U=U, s=s, V=V, rank=rank)


def reconstruction_error(X, res: QueryResult) -> float:
    """Section 5.4: ||X - U Sigma V^T||_F^2 / ||X||_F^2."""
    Xh = (res.U * res.s[None, :]) @ res.V.T
    return float(np.sum((X - Xh) ** 2) / np.sum(np.asarray(X) ** 2))


def similar_ranges(st: Store, base: tuple, stride: int, k_out: int = 1):
    """Case study (Section 6): slide a window of the base range's length
    back over the past with the given stride; score each window by the
    cosine of its first left singular vector with the base's."""
    t_s, t_e = base
    L = t_e - t_s + 1
    u1 = query(st, t_s, t_e, k_out).U[:, 0]
    out = []
    start = t_s - stride
    while start >= 0:
        u = query(st, start, start + L - 1, k_out).U[:, 0]
        c = float(u1 @ u / (np.linalg.norm(u1) * np.linalg.norm(u)))
        out.append((start, c))
        start -= stride
    return out
