"""GPU parity of the energy rule (Eq. 1, zs_store_set_xi): per-block ranks,
stored factors and queries against the oracle's compress(..., xi=...).

The xi values are chosen so that every block's decision sits at least 1e-4
(FP64) or 2e-3 (FP32) away from the threshold in the oracle's energy ratios,
far above each path's error in sigma, and so that the ranks differ between
blocks."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._parity import F32, F64, compare_query, device_rows, _to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _xi_store(A64, b, k, dtype, xi):
    from paper_1805_00754_gb300 import Store
    rows, exact = device_rows(A64, dtype)
    st = Store(n=A64.shape[1], b=b, k=k, dtype=dtype, capacity_rows=A64.shape[0], xi=xi)
    st.append(rows)
    torch.cuda.synchronize()
    return st, exact


def _check_blocks(st, ost, rtol):
    ranks = []
    for i in range(len(ost.s)):
        U, s, Vt, ki = st.export_block(i)
        s = _to_np(s)
        ref = np.zeros_like(s)
        ref[:ost.s[i].shape[0]] = ost.s[i]
        r_gpu, r_ref = int(np.count_nonzero(s)), int(np.count_nonzero(ref))
        assert r_gpu == r_ref, f"block {i}: rank {r_gpu} != {r_ref}"
        np.testing.assert_allclose(s[:r_ref], ref[:r_ref], rtol=rtol)
        assert np.all(_to_np(U)[:, r_ref:] == 0) and np.all(_to_np(Vt)[r_ref:] == 0)
        ranks.append(r_ref)
    return ranks


def test_xi_f64_plain_workload():
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series)
    st, exact = _xi_store(A, w.b, w.k, "f64", 0.9)
    ost = oracle.compress(exact, w.b, w.k, xi=0.9)
    ranks = _check_blocks(st, ost, 1e-10)
    assert len(set(ranks)) > 1 and max(ranks) < w.k
    for a, z in [(1_234, 15_678), (0, 19_999), (499, 500), (7_000, 7_400)]:
        # the range's rank r can be below k here (a range inside one block has
        # that block's k_i); its r pairs meet the oracle, and the directions
        # past r, exactly zero in the oracle, come back through the Gram route
        # at most ~sqrt(eps) sigma_1
        full = oracle.query(ost, a, z, k_out=w.k)
        r = int(np.count_nonzero(full.s))
        out = st.query(a, z, k_out=r)
        torch.cuda.synchronize()
        compare_query(out, oracle.query(ost, a, z, k_out=r), **F64, label=f"xi f64 [{a},{z}]", ost=ost, ts=a, te=z)
        res = st.query(a, z, k_out=w.k)
        torch.cuda.synchronize()
        tail = _to_np(res.S)
        assert np.all(tail[r:] <= 1e-6 * tail[0]), f"[{a},{z}] tail {tail[r:]}"


def test_xi_f32_tensor_path_ragged():
    w = synthetic.WORKLOADS["ragged_batch_f32"]
    A = synthetic.rows(w.series, 0, 8 * w.b + 304)
    st, exact = _xi_store(A, w.b, w.k, "f32", 0.8)
    ost = oracle.compress(exact, w.b, w.k, xi=0.8)
    ranks = _check_blocks(st, ost, 1e-4)
    assert len(set(ranks)) > 1
    T = A.shape[0]
    for a, z in [(0, T - 1), (1_999, 2_000), (3_333, 12_345), (15_000, T - 1)]:
        out = st.query(a, z)
        torch.cuda.synchronize()
        compare_query(out, oracle.query(ost, a, z), **F32, label=f"xi f32 [{a},{z}]", ost=ost, ts=a, te=z)
    assert st.fault() == 0


def _check_stats(st, ost, exact, b, rtol):
    """zs_store_block_stats against the oracle's compress(..., xi): per-block
    ranks k_i (Eq. 1; they fix the paper's space sum k_i (b + n + 1),
    Theorem 3), kept energy, the block energy ||X_i||_F^2 and the stored
    blocks' relative reconstruction error (Section 5.4), which Eckart-Young
    fixes."""
    ranks, kept, en = st.block_stats()
    nb = len(ost.s)
    assert ranks.shape == (nb,)
    T, n = exact.shape
    want_r = np.array([np.count_nonzero(ost.s[i]) for i in range(nb)])
    np.testing.assert_array_equal(ranks, want_r)
    want_e = np.array([np.sum(exact[i * b:min((i + 1) * b, T)] ** 2) for i in range(nb)])
    np.testing.assert_allclose(en, want_e, rtol=1e-12)
    # sigma to rtol: the kept energy (a sum of squares) to 2 rtol
    np.testing.assert_allclose(kept, [np.sum(ost.s[i] ** 2) for i in range(nb)], rtol=2 * rtol)
    err_gpu = 1.0 - np.sum(kept) / np.sum(en)
    err_ref = sum(np.sum((exact[i * b:min((i + 1) * b, T)] - (ost.U[i] * ost.s[i]) @ ost.Vt[i]) ** 2)
                  for i in range(nb)) / np.sum(want_e)
    assert abs(err_gpu - err_ref) <= max(1e-9, 50 * rtol * err_ref), (err_gpu, err_ref)
    return ranks


def test_xi_block_stats_and_reconstruction_error():
    """Per-block ranks, energies, space and reconstruction error of xi stores
    (FP64 plain workload, FP32 ragged tensor path) against the oracle."""
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series)
    st, exact = _xi_store(A, w.b, w.k, "f64", 0.9)
    _check_stats(st, oracle.compress(exact, w.b, w.k, xi=0.9), exact, w.b, 1e-10)
    w = synthetic.WORKLOADS["ragged_batch_f32"]
    A = synthetic.rows(w.series, 0, 8 * w.b + 304)
    st, exact = _xi_store(A, w.b, w.k, "f32", 0.8)
    r = _check_stats(st, oracle.compress(exact, w.b, w.k, xi=0.8), exact, w.b, 1e-4)
    assert len(set(r.tolist())) > 1
    # fixed rank: k_i = min(k, rows_i, n), energies not measured
    st2, _ = _xi_store(A, w.b, w.k, "f32", None)
    r2, kept2, en2 = st2.block_stats()
    assert np.all(r2 == w.k) and np.all(en2 == -1.0) and np.all(kept2 > 0)


def test_xi_errors_and_reset_to_fixed():
    from paper_1805_00754_gb300 import Store, ZsError
    st = Store(n=16, b=64, k=4, dtype="f32", capacity_rows=256)
    with pytest.raises(ZsError) as e:
        st.set_xi(1.5)
    assert e.value.status == 1
    st.set_xi(0.0)                       # fixed rank again


def test_ragged_stack_full_ranks_reproduce_the_plain_stack():
    """With xi = 1 every block keeps k_i = k, so the ragged stack (row map,
    compact U_r spread back to the slab layout) holds the same rows in the
    same order as the fixed-rank stack.  The same store is queried through
    both (set_xi(0) turns the ragged stack off without touching the stored
    factors); on the ragged workload's shape (k = 20: both take the same
    projection kernel) the batch results must be identical, bit for bit."""
    from paper_1805_00754_gb300 import Store
    w = synthetic.WORKLOADS["ragged_batch_f32"]
    A = synthetic.rows(w.series, 0, 9 * w.b + 304).astype(np.float32)
    T = A.shape[0]
    ts, te = synthetic.queries(T, 48, 500, 15_000, seed=synthetic.SEED_BASE + 41)
    st = Store(n=w.series.n, b=w.b, k=w.k, dtype="f32", capacity_rows=T, xi=1.0)
    st.append(torch.from_numpy(A).cuda())
    ranks, _, _ = st.block_stats()
    assert np.all(ranks == w.k)
    outs = []
    for xi in (1.0, 0.0):
        st.set_xi(xi)
        res = st.query_batch(ts, te)
        torch.cuda.synchronize()
        outs.append([(r.U.cpu().numpy(), r.S.cpu().numpy(), r.V.cpu().numpy()) for r in res])
    assert st.status() == (0, 0) and st.fault() == 0
    st.close()
    for q, (a, z) in enumerate(zip(*outs)):
        for x, y in zip(a, z):
            np.testing.assert_array_equal(x, y, err_msg=f"query {q}")


def _varied_rank_rows(nblk, b, n, dims, seed):
    """Blocks whose rows span dims[i % len(dims)] directions (Gaussian
    coefficients on a seeded basis, decaying weights) plus N(0, 1e-4) noise:
    the energy rule gives them very different ranks."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(nblk):
        d = dims[i % len(dims)]
        Q, _ = np.linalg.qr(g.standard_normal((n, d)))
        wts = 1.0 / np.arange(1, d + 1)
        out.append((g.standard_normal((b, d)) * wts) @ Q.T + 1e-4 * g.standard_normal((b, n)))
    return np.vstack(out)


def test_ragged_stack_varied_ranks_against_oracle():
    """Blocks of 2 to 14 signal directions (n = 128, b = 512, k = 16,
    xi = 0.999): each interior slab stacks only its k_i rows.  Queries over
    many blocks meet the oracle's queries of its xi store, and in the factored
    form every coefficient row past a block's k_i is zero (the stack dropped
    it)."""
    b, n, k, xi = 512, 128, 16, 0.999
    A = _varied_rank_rows(24, b, n, (2, 5, 9, 14, 3, 12), synthetic.SEED_BASE + 43)
    st, exact = _xi_store(A, b, k, "f32", xi)
    ost = oracle.compress(exact, b, k, xi=xi)
    ranks = _check_blocks(st, ost, 1e-4)
    assert min(ranks) <= 3 and max(ranks) >= 12
    T = A.shape[0]
    ranges = [(0, T - 1), (100, 9_000), (b - 1, 5 * b), (3 * b + 17, 20 * b - 5), (7 * b, 7 * b + 300)]
    for a, z in ranges:
        out = st.query(a, z)
        torch.cuda.synchronize()
        compare_query(out, oracle.query(ost, a, z), **F32, label=f"ragged xi [{a},{z}]", ost=ost, ts=a, te=z)
    fac = st.query_batch_factored(np.array([r[0] for r in ranges]), np.array([r[1] for r in ranges]))
    torch.cuda.synchronize()
    for q, (a, z) in enumerate(ranges):
        S, E = a // b, z // b
        o = int(fac.offsets[q])
        C = fac.coef[o:o + (E - S + 1) * k].cpu().numpy()      # k rows per covered block
        for t in range(1, E - S):                  # interior slabs
            assert np.all(C[t * k + ranks[S + t]:(t + 1) * k] == 0), (q, t)
    assert st.status() == (0, 0) and st.fault() == 0
