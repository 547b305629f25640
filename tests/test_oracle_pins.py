"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check is a closed form,
an exact identity of the method (Eq. 2-3, Eq. 7-9), the Eckart-Young error
(Section 2.1), orthonormality (Section 3.3.2), a brute-force SVD of the
materialised range, or a planted mistake that one of these must catch.
"""
import itertools

import numpy as np
import pytest

import oracle
import synthetic


def _rand_orth(g, m, r):
    Q, _ = np.linalg.qr(g.standard_normal((m, r)))
    return Q


def _lowrank_noise(g, T, n, r, noise=0.05):
    return g.standard_normal((T, r)) @ g.standard_normal((r, n)) + noise * g.standard_normal((T, n))


def _subspace_sin(V1, V2):
    """sin of the largest principal angle between two column spaces."""
    if V1.shape[1] == 0:
        return 0.0
    Q1, _ = np.linalg.qr(V1)
    Q2, _ = np.linalg.qr(V2)
    return float(np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2))


def _same_result(r1, r2, s_tol, vec_tol, gap=1e-6):
    """sigma elementwise; vectors pairwise where the gap allows (R6)."""
    assert r1.s.shape == r2.s.shape
    s1 = max(r2.s[0], 1e-300) if r2.s.size else 1.0
    np.testing.assert_allclose(r1.s, r2.s, rtol=0, atol=s_tol * s1)
    assert r1.rank == r2.rank
    for j in range(r1.rank):
        lo = abs(r2.s[j] - r2.s[j - 1]) if j > 0 else np.inf
        hi = abs(r2.s[j] - r2.s[j + 1]) if j + 1 < r2.s.size else np.inf
        if min(lo, hi) / s1 < gap:
            continue
        c = np.sign(r1.V[:, j] @ r2.V[:, j]) or 1.0
        np.testing.assert_allclose(c * r1.V[:, j], r2.V[:, j], atol=vec_tol)
        np.testing.assert_allclose(c * r1.U[:, j], r2.U[:, j], atol=vec_tol)


# ----------------------------------------------------------------------------
# Section 2.1: the SVD step and Eq. 1
# ----------------------------------------------------------------------------
def test_svd_closed_form_pdq():
    g = np.random.default_rng(1)
    P, Q = _rand_orth(g, 40, 6), _rand_orth(g, 9, 6)
    D = np.array([9.0, 7.5, 3.0, 2.0, 0.5, 0.25])
    U, s, Vt = oracle.svd(P @ np.diag(D) @ Q.T)
    np.testing.assert_allclose(s[:6], D, rtol=1e-13)
    assert np.all(s[6:] < 1e-13)
    np.testing.assert_allclose(np.abs(np.sum(U[:, :6] * P, axis=0)), 1.0, atol=1e-12)


def test_svd_diagonal_and_descending():
    d = np.array([0.5, 4.0, 2.0])
    U, s, Vt = oracle.svd(np.diag(d))
    np.testing.assert_array_equal(s, [4.0, 2.0, 0.5])


def test_rank_xi_hand_values():
    s = np.array([3.0, 2.0, 1.0])            # energies 9, 4, 1 of 14
    assert oracle.rank_xi(s, 0.5) == 1        # 9/14 = 0.643
    assert oracle.rank_xi(s, 0.9) == 2        # 13/14 = 0.929
    assert oracle.rank_xi(s, 13 / 14) == 2    # ties meet the threshold
    assert oracle.rank_xi(s, 0.95) == 3
    assert oracle.rank_xi(s, 1.0) == 3
    assert oracle.rank_xi(np.zeros(3), 0.98) == 0


def test_canonical_signs_hand_example():
    U = np.array([[1.0, 2.0], [3.0, 4.0]])
    V = np.array([[0.2, -0.9], [-0.7, 0.1]])
    s = np.array([2.0, 1.0])
    U2, _, V2 = oracle.canonical_signs(U, s, V)
    # column 0: largest |.| is -0.7 -> flip; column 1: largest is -0.9 -> flip
    np.testing.assert_array_equal(V2, [[-0.2, 0.9], [0.7, -0.1]])
    np.testing.assert_array_equal(U2, [[-1.0, -2.0], [-3.0, -4.0]])
    # tie on |.|: the lowest index decides
    Vt = np.array([[-0.5], [0.5]])
    _, _, Vt2 = oracle.canonical_signs(np.ones((1, 1)), np.ones(1), Vt)
    np.testing.assert_array_equal(Vt2, [[0.5], [-0.5]])


# ----------------------------------------------------------------------------
# Section 2.2 / Eq. 2-3 and Algorithm 1
# ----------------------------------------------------------------------------
def test_incremental_row_append_is_exact():
    g = np.random.default_rng(2)
    A = _lowrank_noise(g, 30, 7, 3)
    U, s, Vt = oracle.svd(A[:12])
    U2, s2, Vt2 = oracle.incremental_svd(U, s, Vt, A[12])
    np.testing.assert_allclose((U2 * s2) @ Vt2, A[:13], atol=1e-12)
    np.testing.assert_allclose(U2.T @ U2, np.eye(U2.shape[1]), atol=1e-12)
    _, sd, _ = np.linalg.svd(A[:13])
    np.testing.assert_allclose(s2, sd[:s2.size], rtol=1e-12)


@pytest.mark.parametrize("rows,n,k", [(25, 6, 3), (9, 12, 4), (16, 5, 5)])
def test_algorithm1_incremental_equals_truncated_block_svd(rows, n, k):
    g = np.random.default_rng(rows * 31 + n)
    A = _lowrank_noise(g, rows, n, 3, 0.2)
    Ui, si, Vti = oracle.compress_block_incremental(A, k)
    Ud, sd, Vtd = oracle.compress_block(A, k)
    np.testing.assert_allclose(si, sd, rtol=1e-11)
    np.testing.assert_allclose((Ui * si) @ Vti, (Ud * sd) @ Vtd, atol=1e-10)


# Algorithm 1 as printed: truncation to rank k after every row
def test_rowwise_algorithm1_exact_when_block_rank_at_most_k():
    """Data of rank <= k: no row ever loses energy, so the row-by-row result
    is the block's exact truncated SVD (up to sign)."""
    g = np.random.default_rng(41)
    for rows, n, r, k in [(40, 9, 3, 3), (25, 12, 4, 6), (18, 5, 2, 4)]:
        A = g.standard_normal((rows, r)) @ g.standard_normal((r, n))
        dis = []
        Uw, sw, Vtw = oracle.compress_block_rowwise(A, k, dis)
        Ud, sd, Vtd = oracle.compress_block(A, k)
        np.testing.assert_allclose(sw, sd, rtol=1e-11, atol=1e-12 * sd[0])
        np.testing.assert_allclose((Uw * sw) @ Vtw, A, atol=1e-11 * np.abs(A).max())
        np.testing.assert_allclose(Uw.T @ Uw, np.eye(Uw.shape[1]), atol=1e-12)
        assert max(dis) <= 1e-11 * sd[0]


def test_rowwise_algorithm1_no_truncation_when_k_covers_the_rank():
    """k >= min(rows, n): nothing is ever discarded and the result is the
    block's exact SVD, like Algorithm 1 without per-row truncation."""
    g = np.random.default_rng(42)
    A = _lowrank_noise(g, 14, 6, 3, 0.3)
    Uw, sw, Vtw = oracle.compress_block_rowwise(A, 6)
    _, sd, _ = np.linalg.svd(A)
    np.testing.assert_allclose(sw, sd, rtol=1e-11)
    np.testing.assert_allclose((Uw * sw) @ Vtw, A, atol=1e-11)


def test_rowwise_algorithm1_energy_bookkeeping_and_bounds():
    """Each row's truncation drops exactly one singular value of the (k+1) x n
    stacked matrix, and blockdiag(U, 1) is orthonormal, so the energy kept
    falls by the dropped values' squares:
        ||A||_F^2 - ||A_hat||_F^2 = sum_t d_t^2.
    The error is at least the Eckart-Young optimum and at most the sum of
    the dropped values (triangle inequality over the rows)."""
    g = np.random.default_rng(43)
    A = _lowrank_noise(g, 60, 10, 4, 0.3)
    dis = []
    Uw, sw, Vtw = oracle.compress_block_rowwise(A, 4, dis)
    Ah = (Uw * sw) @ Vtw
    d = np.array(dis)
    np.testing.assert_allclose(np.sum(A ** 2) - np.sum(sw ** 2), np.sum(d ** 2), rtol=1e-10)
    err = np.linalg.norm(A - Ah)
    _, sd, _ = np.linalg.svd(A)
    assert err >= np.sqrt(np.sum(sd[4:] ** 2)) * (1 - 1e-12)
    assert err <= np.sum(d) * (1 + 1e-12)
    np.testing.assert_allclose(Uw.T @ Uw, np.eye(4), atol=1e-12)


def test_rowwise_catches_a_planted_left_update_mistake(monkeypatch):
    """The pins above must catch U <- [U; 0] U~ in place of blockdiag(U, 1) U~."""
    def bad(U, s, Vt, a):
        a = np.asarray(a, dtype=np.float64).reshape(1, -1)
        Ut, st, Vtt = oracle.svd(np.vstack([s[:, None] * Vt, a]))
        r, k = U.shape
        B = np.zeros((r + 1, k + 1))
        B[:r, :k] = U                       # the new row's "1" is missing
        return B @ Ut, st, Vtt
    monkeypatch.setattr(oracle.zoomsvd, "incremental_svd", bad)
    g = np.random.default_rng(41)
    A = g.standard_normal((40, 3)) @ g.standard_normal((3, 9))
    Uw, sw, Vtw = oracle.compress_block_rowwise(A, 3)
    assert not np.allclose((Uw * sw) @ Vtw, A, atol=1e-6 * np.abs(A).max())


def test_store_lossless_reconstructs_exactly():
    g = np.random.default_rng(3)
    A = _lowrank_noise(g, 103, 8, 4)
    st = oracle.compress(A, b=20, k=8)
    assert st.nblocks == 6 and st.rows_of(5) == 3          # ragged last block (R3)
    np.testing.assert_allclose(oracle.reconstruct(st, 0, 102), A, atol=1e-12)


def test_store_truncation_error_is_tail_energy():
    """Eckart-Young (Section 2.1): ||A - A_hat||_F^2 = sum_{j>k} sigma_j^2."""
    g = np.random.default_rng(4)
    A = _lowrank_noise(g, 120, 10, 3, 0.3)
    k = 4
    st = oracle.compress(A, b=40, k=k)
    for i, (lo, hi) in enumerate(oracle.block_bounds(120, 40)):
        sd = np.linalg.svd(A[lo:hi], compute_uv=False)
        err = np.sum((A[lo:hi] - (st.U[i] * st.s[i]) @ st.Vt[i]) ** 2)
        assert err == pytest.approx(np.sum(sd[k:] ** 2), rel=1e-10)
        np.testing.assert_allclose(st.s[i], sd[:k], rtol=1e-12)


def test_space_theorem3_count():
    st = oracle.compress(np.ones((1000, 32)) + np.arange(32), b=100, k=5)
    # Thm. 3: sum_i k_i (b + 1 + c) elements; the constant matrix has rank 1
    assert sum(u.shape[1] for u in st.U) == 50
    assert st.nbytes(8) == 8 * 10 * 5 * (100 + 1 + 32)


# ----------------------------------------------------------------------------
# Algorithm 3 planning under reading R1
# ----------------------------------------------------------------------------
def test_plan_paper_sized_example():
    p = oracle.plan(1_234, 15_678, 500, 20_000)
    assert (p.S, p.E, p.r_S, p.b_S, p.b_E) == (2, 31, 234, 266, 179)
    assert p.rows == 14_445          # half-open reading would give 14,444
    assert p.b_S + (p.E - p.S - 1) * 500 + p.b_E == p.rows


def test_plan_rejects_bad_ranges():
    for ts, te in [(-1, 3), (5, 4), (0, 100)]:
        with pytest.raises(ValueError):
            oracle.plan(ts, te, 10, 100)


# ----------------------------------------------------------------------------
# Algorithms 2-3 / Eq. 7-9: the query phase
# ----------------------------------------------------------------------------
def test_block_diag_identity_and_orthonormality():
    """Eq. 7: A_hat[ts..te] = diag(S:E) Sigma V^T; diag has orthonormal columns."""
    g = np.random.default_rng(5)
    A = _lowrank_noise(g, 300, 9, 4)
    st = oracle.compress(A, b=50, k=3)
    for ts, te in [(7, 211), (50, 99), (12, 40), (260, 299), (0, 299)]:
        D, M = oracle.block_diag_left(st, ts, te)
        np.testing.assert_allclose(D @ M, oracle.reconstruct(st, ts, te), atol=1e-11)
        np.testing.assert_allclose(D.T @ D, np.eye(D.shape[1]), atol=1e-12)


@pytest.mark.parametrize("k", [3, 9])
def test_query_equals_direct_svd_of_reconstruction(k):
    """The exact identity: Zoom-SVD returns the SVD of A_hat on the range."""
    g = np.random.default_rng(6)
    A = _lowrank_noise(g, 500, 9, 5, 0.1)
    st = oracle.compress(A, b=60, k=k)
    for ts, te in [(0, 499), (13, 377), (61, 118), (120, 179), (481, 499), (200, 200)]:
        r = oracle.query(st, ts, te)
        d = oracle.direct_svd(oracle.reconstruct(st, ts, te), st.k)
        _same_result(r, d, 1e-10, 1e-8)
        if r.U.shape[1]:
            np.testing.assert_allclose(r.U.T @ r.U, np.diag((r.s > 0).astype(float)), atol=1e-12)
            np.testing.assert_allclose(r.V.T @ r.V, np.diag((r.s > 0).astype(float)), atol=1e-12)


def test_query_lossless_matches_raw_range_plain_workload():
    """k = min(b, n): sigma equals the direct SVD of the raw range to 1e-10."""
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series, 0, 6_000)
    st = oracle.compress(A, b=w.b, k=32)
    r = oracle.query(st, 1_234, 5_678, k_out=32)
    d = oracle.direct_svd(A[1_234:5_679], 32)
    _same_result(r, d, 1e-10, 1e-8)
    assert r.U.shape == (4_445, 32)


def test_query_truncated_weyl_bound():
    """Against the raw range, |sigma_j(A_r) - sigma_j(A_hat_r)| <= ||A_r - A_hat_r||_2."""
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series, 0, 4_000)
    st = oracle.compress(A, b=w.b, k=w.k)
    ts, te = 321, 3_210
    r = oracle.query(st, ts, te)
    Ar = A[ts:te + 1]
    bound = np.linalg.norm(Ar - oracle.reconstruct(st, ts, te), 2)
    sd = np.linalg.svd(Ar, compute_uv=False)[: r.s.size]
    assert np.all(np.abs(sd - r.s) <= bound * (1 + 1e-12))
    assert oracle.reconstruction_error(Ar, r) < 1e-2


def test_closed_form_full_range():
    """A = P D Q^T: the full-range query returns D (special case ii)."""
    g = np.random.default_rng(7)
    P, Q = _rand_orth(g, 240, 5), _rand_orth(g, 7, 5)
    D = np.array([50.0, 20.0, 10.0, 3.0, 1.0])
    st = oracle.compress(P @ np.diag(D) @ Q.T, b=48, k=7)
    r = oracle.query(st, 0, 239, k_out=7)
    np.testing.assert_allclose(r.s[:5], D, rtol=1e-12)
    assert r.rank == 5 and np.all(r.s[5:] == 0.0)


def test_single_row_closed_form():
    g = np.random.default_rng(8)
    A = _lowrank_noise(g, 90, 6, 2)
    st = oracle.compress(A, b=30, k=6)
    r = oracle.query(st, 47, 47, k_out=3)
    row = A[47]
    assert r.rank == 1 and r.s[0] == pytest.approx(np.linalg.norm(row), rel=1e-12)
    np.testing.assert_allclose(np.abs(r.V[:, 0]), np.abs(row) / np.linalg.norm(row), atol=1e-12)
    np.testing.assert_allclose(np.abs(r.U), [[1.0, 0.0, 0.0]], atol=1e-12)


def test_whole_block_returns_stored_factors():
    g = np.random.default_rng(9)
    A = _lowrank_noise(g, 200, 8, 4, 0.2)
    st = oracle.compress(A, b=50, k=4)
    r = oracle.query(st, 100, 149)
    np.testing.assert_allclose(r.s, st.s[2], rtol=1e-12)
    for j in range(4):
        c = np.sign(r.V[:, j] @ st.Vt[2][j])
        np.testing.assert_allclose(c * r.V[:, j], st.Vt[2][j], atol=1e-10)
        np.testing.assert_allclose(c * r.U[:, j], st.U[2][:, j], atol=1e-10)


@pytest.mark.parametrize("b", [3, 5, 7])
def test_tiny_bruteforce_every_range(b):
    g = np.random.default_rng(10 + b)
    T, n = 23, 4
    A = g.standard_normal((T, n))
    lossless = oracle.compress(A, b=b, k=min(b, n))
    trunc = oracle.compress(A, b=b, k=2)
    for ts, te in itertools.combinations_with_replacement(range(T), 2):
        r = oracle.query(lossless, ts, te, k_out=n)
        _same_result(r, oracle.direct_svd(A[ts:te + 1], n), 1e-10, 1e-7)
        r2 = oracle.query(trunc, ts, te, k_out=2)
        _same_result(r2, oracle.direct_svd(oracle.reconstruct(trunc, ts, te), 2), 1e-10, 1e-7)


def _xi_rule_holds(xi, b=64, k=4):
    """Eq. 1 per block, checked against the data: the kept rank k_i holds at
    least xi of ||X_i||_F^2 (unless capped at k), one rank less does not, and
    the stored block's residual is the Eckart-Young tail."""
    g = np.random.default_rng(5)
    A = g.standard_normal((300, 6)) @ np.diag([5.0, 3.0, 2.0, 1.0, 0.5, 0.1])
    st = oracle.compress(A, b, k, xi=xi)
    for i, (lo, hi) in enumerate(oracle.block_bounds(300, b)):
        X = A[lo:hi]
        E = float(np.sum(X ** 2))
        s = st.s[i]
        ki = int(np.count_nonzero(s))
        kept = float(np.sum(s[:ki] ** 2))
        if ki > k or (ki < k and kept < xi * E * (1 - 1e-12)):
            return False
        if ki >= 1 and float(np.sum(s[:ki - 1] ** 2)) >= xi * E:
            return False
        R = X - st.U[i] @ np.diag(s) @ st.Vt[i]
        if abs(float(np.sum(R ** 2)) - (E - kept)) > 1e-9 * E:
            return False
    return True


@pytest.mark.parametrize("xi", [0.5, 0.9, 0.99])
def test_xi_compress_energy_rule(xi):
    assert _xi_rule_holds(xi)


def test_xi_one_is_fixed_rank():
    g = np.random.default_rng(6)
    A = g.standard_normal((200, 5))
    a, z = oracle.compress(A, 50, 3), oracle.compress(A, 50, 3, xi=1.0)
    for i in range(len(a.s)):
        np.testing.assert_array_equal(a.s[i], z.s[i])
        np.testing.assert_array_equal(a.U[i], z.U[i])


def test_similar_range_search_periodic():
    """Section 6: a window shifted by whole periods of a periodic signal matches."""
    t = np.arange(1200)
    A = np.outer(np.sin(2 * np.pi * t / 100.0), [1.0, 2.0, -1.0]) + np.outer(
        np.cos(2 * np.pi * t / 50.0), [0.5, -1.0, 1.0])
    st = oracle.compress(A, b=64, k=3)
    hits = oracle.similar_ranges(st, (900, 1099), stride=100)
    assert len(hits) == 9
    for start, c in hits:
        assert c == pytest.approx(1.0, abs=1e-9)


# ----------------------------------------------------------------------------
# Planted mistakes: each must make one of the pins above fail.
# ----------------------------------------------------------------------------
def _bruteforce_ok(T=17, n=3, b=5):
    g = np.random.default_rng(99)
    A = g.standard_normal((T, n))
    st = oracle.compress(A, b=b, k=n)
    try:
        for ts, te in itertools.combinations_with_replacement(range(T), 2):
            r = oracle.query(st, ts, te, k_out=n)
            _same_result(r, oracle.direct_svd(A[ts:te + 1], n), 1e-10, 1e-7)
    except (AssertionError, ValueError, IndexError):
        return False
    return True


def test_pins_catch_half_open_end(monkeypatch):
    real = oracle.zoomsvd.plan

    def bad(t_s, t_e, b, T):
        p = real(t_s, t_e, b, T)
        return oracle.zoomsvd.Plan(p.S, p.E, p.r_S, p.b_S, t_e % b, p.rows)
    monkeypatch.setattr(oracle.zoomsvd, "plan", bad)
    assert not _bruteforce_ok()


def test_pins_catch_partial_svd_without_sigma(monkeypatch):
    def bad(U, s, Vt, lo, hi):
        X = oracle.elimination_matrix(lo, hi, U.shape[0])
        Ut, st, Vtt = oracle.svd(X @ U)
        return Ut, st, Vtt @ Vt
    monkeypatch.setattr(oracle.zoomsvd, "partial_svd", bad)
    assert not _bruteforce_ok()


def test_pins_catch_lift_offset(monkeypatch):
    real_svd = oracle.zoomsvd.svd
    calls = {"n": 0}

    def shifted(M):
        U, s, Vt = real_svd(M)
        calls["n"] += 1
        if M.shape[0] > 3 and calls["n"] % 3 == 0:   # the stacked matrix
            U = np.roll(U, 1, axis=0)
        return U, s, Vt
    monkeypatch.setattr(oracle.zoomsvd, "svd", shifted)
    assert not _bruteforce_ok()


def test_pins_catch_wrong_truncation(monkeypatch):
    def bad(U, s, Vt, k):
        k = max(0, min(k, s.shape[0]))
        return U[:, -k:], s[-k:], Vt[-k:, :]
    monkeypatch.setattr(oracle.zoomsvd, "truncate", bad)
    g = np.random.default_rng(4)
    A = _lowrank_noise(g, 120, 10, 3, 0.3)
    st = oracle.compress(A, b=40, k=4)
    sd = np.linalg.svd(A[:40], compute_uv=False)
    err = np.sum((A[:40] - (st.U[0] * st.s[0]) @ st.Vt[0]) ** 2)
    assert err != pytest.approx(np.sum(sd[4:] ** 2), rel=1e-10)


def test_pins_catch_transposed_v(monkeypatch):
    def bad(U, s, Vt, a):
        a = np.asarray(a, dtype=np.float64).reshape(1, -1)
        K = np.vstack([s[:, None] * Vt, a])
        Ut, st, Vtt = oracle.svd(K)
        r, k = U.shape
        B = np.zeros((r + 1, k + 1))
        B[:r, :k] = U
        B[r, k] = 1.0
        return B @ Ut, st, Vtt[::-1]
    monkeypatch.setattr(oracle.zoomsvd, "incremental_svd", bad)
    g = np.random.default_rng(2)
    A = _lowrank_noise(g, 12, 5, 3)
    Ui, si, Vti = oracle.compress_block_incremental(A, 5)
    assert not np.allclose((Ui * si) @ Vti, A, atol=1e-8)


@pytest.mark.parametrize("shift", [-1, 1])
def test_pins_catch_xi_rank_off_by_one(monkeypatch, shift):
    true_rank = oracle.zoomsvd.rank_xi

    def bad(sv, xi):
        return max(0, true_rank(sv, xi) + shift)

    monkeypatch.setattr(oracle.zoomsvd, "rank_xi", bad)
    assert not all(_xi_rule_holds(xi) for xi in (0.5, 0.9))
