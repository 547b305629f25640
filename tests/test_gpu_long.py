"""GPU parity at the query lengths the bench answers (Fig. 1's range lengths,
1e5..3.2e5 rows): the tall stitched matrices (hundreds of slabs) and the
many-slab lift through zs_query_batch, element by element against the
oracle's query of the same store.

Two shapes: the compression workload's (n = 256, b = 1024, k = 16, f32, with
the slow drift) over 320 blocks, and the ragged batch workload's (n = 128,
b = 2000, k = 20, f32) over 200 blocks plus a 304-row last block.  Sixteen
queries each, lengths log-uniform over [1e5, 3.2e5]."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._parity import F32, compare_query, gpu_store

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,nblk,extra", [("compress_f32", 320, 0), ("ragged_batch_f32", 200, 304)])
def test_long_ranges_against_oracle(name, nblk, extra):
    w = synthetic.WORKLOADS[name]
    T = nblk * w.b + extra
    A = synthetic.rows(w.series, 0, T)
    st, exact = gpu_store(A, w.b, w.k, "f32")
    ost = oracle.compress(exact, w.b, w.k)
    ts, te = synthetic.queries(T, 16, 100_000, 320_000, seed=synthetic.SEED_BASE + 7)
    # the longest range is kept as long as the shape allows
    assert np.max(te - ts + 1) >= min(300_000, T // 2)
    outs = st.query_batch(ts, te)
    torch.cuda.synchronize()
    pairs = 0
    for q in range(len(ts)):
        a, z = int(ts[q]), int(te[q])
        ref = oracle.query(ost, a, z)
        p, _ = compare_query(outs[q], ref, **F32, label=f"{name} [{a},{z}]", ost=ost, ts=a, te=z, min_pairs=1)
        pairs += p
    assert pairs >= 4 * len(ts)
    assert st.status() == (0, 0) and st.fault() == 0
