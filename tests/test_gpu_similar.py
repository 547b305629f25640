"""GPU parity of the similar-range search (Section 6 case study) through the
C ABI (zs_similar_ranges) against the oracle's similar_ranges."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._parity import gpu_store

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _compare(got, ref, tol):
    assert [s for s, _ in got] == [s for s, _ in ref]
    g = np.array([c for _, c in got])
    r = np.array([c for _, c in ref])
    np.testing.assert_allclose(g, r, rtol=0, atol=tol)


def test_similar_ranges_f64_plain_workload():
    w = synthetic.WORKLOADS["plain_f64"]
    A = synthetic.rows(w.series)
    st, exact = gpu_store(A, w.b, w.k, "f64")
    ost = oracle.compress(exact, w.b, w.k)
    base = (12_000, 13_999)
    got = st.similar_ranges(base, stride=500)
    assert len(got) == 24 and got[0][0] == 11_500 and got[-1][0] == 0
    _compare(got, oracle.similar_ranges(ost, base, stride=500), 1e-8)
    # a cap on the number of windows keeps the first ones
    assert st.similar_ranges(base, stride=500, max_windows=5) == got[:5]
    assert st.similar_ranges(base, stride=500, max_windows=0) == []


def test_similar_ranges_f32_periodic_windows_match():
    """Windows shifted by whole periods of a periodic signal score ~1 on the
    tensor-core path (n = 64), and every score meets the oracle."""
    T, n, P = 60_000, 64, 400
    g = np.random.default_rng(20260)
    t = np.arange(T)[:, None]
    w1, w2 = g.standard_normal((1, n)), g.standard_normal((1, n))
    A = 3.0 * np.sin(2 * np.pi * t / P) * w1 + np.sin(2 * np.pi * t / (P / 2) + 0.3) * w2
    A += 1e-3 * g.standard_normal((T, n))
    st, exact = gpu_store(A, 1_000, 4, "f32")
    ost = oracle.compress(exact, 1_000, 4)
    base = (50_000, 53_999)
    got = st.similar_ranges(base, stride=P)
    assert len(got) == 125
    assert min(c for _, c in got) > 0.999
    _compare(got, oracle.similar_ranges(ost, base, stride=P), 2e-3)
    assert st.fault() == 0


def test_similar_ranges_errors():
    from paper_1805_00754_gb300 import ZsError
    w = synthetic.WORKLOADS["plain_f64"]
    st, _ = gpu_store(synthetic.rows(w.series, 0, 2_000), w.b, w.k, "f64")
    with pytest.raises(ZsError) as e:
        st.similar_ranges((100, 5_000), stride=10)       # past the rows appended
    assert e.value.status == 2
    with pytest.raises(ZsError) as e:
        st.similar_ranges((500, 600), stride=0)
    assert e.value.status == 1
    assert st.similar_ranges((50, 99), stride=100) == []
