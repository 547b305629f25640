"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Inputs are the seeded synthetic workloads (see ``synthetic``); sizes here are
ones the oracle finishes in seconds while still spanning many blocks, ragged
tails, partial boundary blocks and single-block ranges.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._parity import F32, F64, compare_query, gpu_store, sigma_rel_err, _to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _edge_ranges(T, b):
    last = T - 1
    out = [(0, last), (0, 0), (last, last), (b - 1, b), (b, 2 * b - 1), (3, b - 2), (b + 7, b + 7),
           (b - 3, 3 * b + 2), (last - b + 1, last), ((T // b - 1) * b - 5, last), (1, last - 1),
           (2 * b - 1, 2 * b), (5 * b // 2, 7 * b // 2)]
    return [(a, z) for a, z in out if 0 <= a <= z < T]


# ----------------------------------------------------------------------------
# FP64 plain method: 20,000 x 32, b = 500, k = 8, query (1234, 15678)
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def plain():
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series)
    st, exact = gpu_store(A, w.b, w.k, "f64")
    ost = oracle.compress(exact, w.b, w.k)
    return w, A, st, ost


def test_plain_store_factors(plain):
    w, A, st, ost = plain
    T, nb, _ = st.info()
    assert (T, nb) == (20_000, 40)
    for i in [0, 1, 17, 39]:
        U, s, Vt, ki = st.export_block(i)
        U, s, Vt = _to_np(U), _to_np(s), _to_np(Vt)
        assert ki == w.k
        np.testing.assert_allclose(s, ost.s[i], rtol=1e-10)
        for j in range(w.k):
            c = np.sign(Vt[j] @ ost.Vt[i][j])
            np.testing.assert_allclose(c * Vt[j], ost.Vt[i][j], atol=1e-8)
            np.testing.assert_allclose(c * U[:, j], ost.U[i][:, j], atol=1e-8)


def test_plain_query_paper_range(plain):
    w, A, st, ost = plain
    ts, te = w.single_query
    out = st.query(ts, te)
    torch.cuda.synchronize()
    ref = oracle.query(ost, ts, te)
    assert out.U.shape == (14_445, 8)
    compare_query(out, ref, **F64, label="plain", ost=ost, ts=ts, te=te, min_pairs=8)


def test_plain_edge_ranges(plain):
    w, A, st, ost = plain
    for ts, te in _edge_ranges(20_000, w.b):
        for kout in (1, w.k, 12):
            out = st.query(ts, te, kout)
            torch.cuda.synchronize()
            compare_query(out, oracle.query(ost, ts, te, kout), **F64, label=f"[{ts},{te}] k{kout}",
                          ost=ost, ts=ts, te=te)


def test_lossless_matches_raw_range():
    """k = min(b, n): the answer is the SVD of the raw rows (to 1e-10)."""
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series, 0, 5_000)
    st, exact = gpu_store(A, 500, 32, "f64")
    for ts, te in [(1_234, 4_321), (0, 4_999), (250, 740), (777, 777), (4_500, 4_999)]:
        out = st.query(ts, te, 32)
        torch.cuda.synchronize()
        compare_query(out, oracle.direct_svd(exact[ts:te + 1], 32), **F64, label=f"lossless [{ts},{te}]",
                      X=exact[ts:te + 1])


def test_ragged_tail_and_piecewise_append():
    """Appending in odd pieces (host and device) equals one append; the open
    block is queryable (Def. 1's current block)."""
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series, 0, 3_333)
    one, exact = gpu_store(A, 500, 8, "f64")
    from paper_1805_00754_gb300 import Store
    pieces = Store(n=32, b=500, k=8, dtype="f64", capacity_rows=4_000)
    cuts = [0, 1, 2, 499, 500, 1_000, 1_777, 2_999, 3_333]
    for a, z in zip(cuts[:-1], cuts[1:]):
        if (a // 7) % 2:
            pieces.append(A[a:z])                        # host rows
        else:
            pieces.append(torch.from_numpy(A[a:z]).cuda())
    torch.cuda.synchronize()
    assert pieces.info()[:2] == (3_333, 7)
    ost = oracle.compress(exact, 500, 8)
    for ts, te in [(0, 3_332), (3_100, 3_332), (2_999, 3_001), (1_500, 3_300)]:
        o1 = one.query(ts, te)
        o2 = pieces.query(ts, te)
        torch.cuda.synchronize()
        assert torch.equal(o1.S, o2.S) and torch.equal(o1.U, o2.U) and torch.equal(o1.V, o2.V)
        compare_query(o1, oracle.query(ost, ts, te), **F64, label=f"tail [{ts},{te}]", ost=ost, ts=ts, te=te)


def test_pipelined_small_appends_with_interleaved_queries():
    """Appends of 1-3 whole blocks go through the append pipeline (several
    streams); queries issued in between see every appended row, and the final
    store equals the one built by a single append."""
    w, A = _reduced("ragged_batch_f32", 9, 0)
    one, exact = gpu_store(A, w.b, w.k, "f32")
    from paper_1805_00754_gb300 import Store
    st = Store(n=128, b=w.b, k=w.k, dtype="f32", capacity_rows=A.shape[0])
    dev = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    ost = oracle.compress(exact, w.b, w.k)
    row = 0
    for nb in [1, 2, 1, 3, 2]:
        st.append(dev[row:row + nb * w.b])
        row += nb * w.b
        out = st.query(max(0, row - 3 * w.b // 2), row - 1)     # touches the newest blocks
        torch.cuda.synchronize()
        a, z = max(0, row - 3 * w.b // 2), row - 1
        compare_query(out, oracle.query(ost, a, z), **F32, label=f"pipe {row}", ost=ost, ts=a, te=z)
    assert st.info()[:2] == (A.shape[0], 9)
    for a, z in [(0, A.shape[0] - 1), (2_500, 13_333)]:
        o1, o2 = one.query(a, z), st.query(a, z)
        torch.cuda.synchronize()
        assert torch.equal(o1.S, o2.S) and torch.equal(o1.U, o2.U) and torch.equal(o1.V, o2.V)


def test_batch_equals_single(plain):
    w, A, st, ost = plain
    ts, te = synthetic.queries(20_000, 64, 10, 19_000, seed=5)
    outs = st.query_batch(ts, te)
    torch.cuda.synchronize()
    for q in range(len(ts)):
        one = st.query(int(ts[q]), int(te[q]))
        torch.cuda.synchronize()
        assert torch.equal(one.S, outs[q].S) and torch.equal(one.U, outs[q].U) and torch.equal(one.V, outs[q].V)
    for q in range(0, 64, 8):
        compare_query(outs[q], oracle.query(ost, int(ts[q]), int(te[q])), **F64, label=f"batch {q}",
                      ost=ost, ts=int(ts[q]), te=int(te[q]))


def test_graph_replay_equals_eager():
    """Query batches replayed from the captured CUDA graph equal eager launches."""
    from paper_1805_00754_gb300 import zoomsvd
    w, A = _reduced("ragged_batch_f32", 12, 304)
    st, exact = gpu_store(A, w.b, w.k, "f32")
    T = A.shape[0]
    ts, te = synthetic.queries(T, 24, 500, 20_000, seed=21)
    zoomsvd.profile(True)                 # profiler on: eager launches
    eager = st.query_batch(ts, te)
    torch.cuda.synchronize()
    zoomsvd.profile(False)
    st.query_batch(ts, te)                # warm (eager) batch of this shape
    graph1 = st.query_batch(ts, te)       # captured
    graph2 = st.query_batch(ts[::-1].copy(), te[::-1].copy())   # replayed, new plans
    sub = [3, 0, 17, 9, 11]                                       # replayed, fewer queries
    graph3 = st.query_batch(ts[sub], te[sub])
    torch.cuda.synchronize()
    for q in range(len(ts)):
        for a, b_ in [(eager[q], graph1[q]), (eager[q], graph2[len(ts) - 1 - q])]:
            assert torch.equal(a.S, b_.S) and torch.equal(a.U, b_.U) and torch.equal(a.V, b_.V)
    for i, q in enumerate(sub):
        a, b_ = eager[q], graph3[i]
        assert torch.equal(a.S, b_.S) and torch.equal(a.U, b_.U) and torch.equal(a.V, b_.V)


def test_autotune_keeps_results(tmp_path, monkeypatch):
    monkeypatch.setenv("ZS_TUNE_CACHE", str(tmp_path / "tune.txt"))
    w, A = _reduced("ragged_batch_f32", 10, 304)
    st, _ = gpu_store(A, w.b, w.k, "f32")
    ts, te = synthetic.queries(A.shape[0], 16, 500, 15_000, seed=31)
    before = st.query_batch(ts, te)
    torch.cuda.synchronize()
    st.autotune(32)
    after = st.query_batch(ts, te)
    torch.cuda.synchronize()
    for a, b_ in zip(before, after):
        assert torch.equal(a.S, b_.S) and torch.equal(a.U, b_.U) and torch.equal(a.V, b_.V)
    assert (tmp_path / "tune.txt").read_text().startswith("n=128,b=2000,k=20")


def test_errors(plain):
    from paper_1805_00754_gb300 import ZsError
    w, A, st, ost = plain
    for ts, te in [(-1, 5), (10, 9), (0, 20_000)]:
        with pytest.raises(ZsError) as e:
            st.query(max(ts, 0), max(te, 0)) if ts >= 0 and te < 20_000 and ts <= te else \
                st.query_batch([ts], [te])
        assert e.value.status == 2
    with pytest.raises(ZsError) as e:
        st.append(np.zeros((1, 32)))       # capacity is full
    assert e.value.status == 3


# ----------------------------------------------------------------------------
# FP32 and BF16 paths on reduced copies of the bench workloads
# ----------------------------------------------------------------------------
def _reduced(name, nblk, extra):
    w = synthetic.WORKLOADS[name]
    T = nblk * w.b + extra
    return w, synthetic.rows(w.series, 0, T)


@pytest.mark.parametrize("refine", [False, True])
def test_f32_compress_workload(refine):
    w, A = _reduced("compress_f32", 12, 333)
    st, exact = gpu_store(A, w.b, w.k, "f32", refine=refine)
    ost = oracle.compress(exact, w.b, w.k)
    for i in [0, 5, 12]:
        U, s, Vt, ki = st.export_block(i)
        np.testing.assert_allclose(_to_np(s)[:ki], ost.s[i][:ki], rtol=1e-4)
    T = A.shape[0]
    ts, te = synthetic.queries(T, 6, 1_000, T, seed=7)
    for a, z in list(zip(ts, te)) + _edge_ranges(T, w.b)[:6]:
        out = st.query(int(a), int(z))
        torch.cuda.synchronize()
        compare_query(out, oracle.query(ost, int(a), int(z)), **F32, label=f"f32 [{a},{z}]", ost=ost, ts=int(a),
                      te=int(z))
    assert st.fault() == 0          # no bounded wait of the tensor-core kernels gave up


def test_exact_gram_path_matches_oracle_and_tensor_path():
    """The FP32 CUDA-core Gram (ZS_FLAG_EXACT_GRAM) and the default tensor-core
    path both meet the oracle; they agree with each other to the same bar."""
    w, A = _reduced("ragged_batch_f32", 8, 304)
    st_tc, exact = gpu_store(A, w.b, w.k, "f32")
    st_ex, _ = gpu_store(A, w.b, w.k, "f32", exact_gram=True)
    ost = oracle.compress(exact, w.b, w.k)
    T = A.shape[0]
    for a, z in [(0, T - 1), (1_999, 2_000), (3_333, 12_345), (16_000, T - 1)]:
        o1, o2 = st_tc.query(a, z), st_ex.query(a, z)
        torch.cuda.synchronize()
        ref = oracle.query(ost, a, z)
        compare_query(o1, ref, **F32, label=f"tensor [{a},{z}]", ost=ost, ts=a, te=z)
        compare_query(o2, ref, **F32, label=f"exact [{a},{z}]", ost=ost, ts=a, te=z)


def test_bf16_precision_workload():
    w, A = _reduced("precision_bf16", 5, 100)
    st, exact = gpu_store(A, w.b, w.k, "bf16", refine=True)
    ost = oracle.compress(exact, w.b, w.k)
    T = A.shape[0]
    for a, z in [(0, T - 1), (1_000, 7_000), (2_047, 2_048), (4_000, 9_999)]:
        out = st.query(a, z)
        torch.cuda.synchronize()
        compare_query(out, oracle.query(ost, a, z), **F32, label=f"bf16 [{a},{z}]", ost=ost, ts=a, te=z)


def test_ragged_batch_f32():
    w, A = _reduced("ragged_batch_f32", 30, 304)
    st, exact = gpu_store(A, w.b, w.k, "f32")
    ost = oracle.compress(exact, w.b, w.k)
    T = A.shape[0]
    ts, te = synthetic.queries(T, 48, 1_000, 40_000, seed=11)
    outs = st.query_batch(ts, te)
    torch.cuda.synchronize()
    worst = 0.0
    for q in range(len(ts)):
        ref = oracle.query(ost, int(ts[q]), int(te[q]))
        compare_query(outs[q], ref, **F32, label=f"ragged {q}", ost=ost, ts=int(ts[q]), te=int(te[q]))
        worst = max(worst, sigma_rel_err(outs[q], ref))
    assert worst <= 1e-4
    assert st.fault() == 0


def test_serving_results_equal_alone():
    """Continuous batching: each served result equals the one computed alone."""
    from paper_1805_00754_gb300 import Server
    w, A = _reduced("serving_f32", 6, 1_000)
    st, exact = gpu_store(A, w.b, w.k, "f32")
    T = A.shape[0]
    ts, te = synthetic.queries(T, 96, 100, 20_000, seed=13)
    sv = Server(st, max_batch=16, max_inflight=3, memory_budget=64 << 20)
    tickets = [sv.submit(int(a), int(z)) for a, z in zip(ts, te)]
    for t, _ in tickets:
        assert sv.wait(t) == 0
    stats = sv.stop()
    assert stats["completed"] == 96 and stats["batches"] >= 6
    for (t, out), a, z in zip(tickets, ts, te):
        alone = st.query(int(a), int(z))
        torch.cuda.synchronize()
        assert torch.equal(alone.S, out.S) and torch.equal(alone.U, out.U) and torch.equal(alone.V, out.V)


def test_factored_batch_matches_materialised():
    """zs_query_batch_factored: S, V and rank equal the materialised batch's
    bit for bit, and the stored U_i rows times each block's coefficients
    (Eq. 9, composed here in FP64) give its U to FP32 rounding."""
    w, A = _reduced("ragged_batch_f32", 10, 304)
    st, exact = gpu_store(A, w.b, w.k, "f32")
    T = A.shape[0]
    ts, te = synthetic.queries(T, 20, 500, 15_000, seed=41)
    mat = st.query_batch(ts, te)
    fac = st.query_batch_factored(ts, te)
    torch.cuda.synchronize()
    blocks = {}
    for q in range(len(ts)):
        assert torch.equal(mat[q].S, fac.S[q]) and torch.equal(mat[q].V, fac.V[q])
        assert torch.equal(mat[q].rank[0], fac.rank[q])
        a, z = int(ts[q]), int(te[q])
        parts = []
        for t, i in enumerate(range(a // w.b, z // w.b + 1)):
            if i not in blocks:
                blocks[i] = _to_np(st.export_block(i)[0])
            lo, hi = max(a, i * w.b), min(z, (i + 1) * w.b - 1)
            C = _to_np(fac.coef[fac.offsets[q] + t * w.k: fac.offsets[q] + (t + 1) * w.k])
            parts.append(blocks[i][lo - i * w.b: hi - i * w.b + 1] @ C)
        U = np.vstack(parts)
        Um = _to_np(mat[q].U)
        assert U.shape == Um.shape
        assert np.max(np.abs(U - Um)) <= 1e-5 * max(1.0, np.max(np.abs(Um))), f"query {q}"
    from paper_1805_00754_gb300 import ZsError
    with pytest.raises(ZsError) as e:
        from paper_1805_00754_gb300.zoomsvd import FactoredBatch
        small = FactoredBatch(st, ts, te, w.k)
        small.coef = small.coef[:w.k]             # too few rows
        st.query_batch_factored(ts, te, out=small)
    assert e.value.status == 1
