"""Host-side checks that need no GPU: the C-ABI library builds for sm_103a,
loads, and exports every entry point include/zoomsvd.h declares; the ctypes
binding declares exactly those; the input generators are deterministic."""
import ctypes
import os
import re

import numpy as np

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "zoomsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_00754_gb300 import zoomsvd
    lib = ctypes.CDLL(zoomsvd.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert sorted(zoomsvd.SIGNATURES) == names


def test_status_strings_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_00754_gb300 import zoomsvd
    lib = zoomsvd.load_library()
    assert lib.zs_status_str(2) == b"range out of bounds"
    assert lib.zs_launch_count() == 0


def test_store_create_rejects_bad_config_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_00754_gb300 import zoomsvd
    lib = zoomsvd.load_library()
    h = ctypes.c_void_p()
    cfg = zoomsvd.StoreConfig(32, 500, 99, 0, 1000, 0, 0)       # k > n
    assert lib.zs_store_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg = zoomsvd.StoreConfig(32, 500, 8, 7, 1000, 0, 0)        # bad dtype
    assert lib.zs_store_create(ctypes.byref(cfg), ctypes.byref(h)) == 6


def test_new_entry_points_reject_bad_arguments_without_gpu():
    """zs_similar_ranges and zs_store_set_xi check their arguments before any
    device call."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_00754_gb300 import zoomsvd
    lib = zoomsvd.load_library()
    starts = (ctypes.c_int64 * 4)()
    cos = (ctypes.c_double * 4)()
    nw = ctypes.c_int32()
    assert lib.zs_similar_ranges(None, 10, 20, 5, 4, starts, cos, ctypes.byref(nw), None) == 1
    assert lib.zs_store_set_xi(None, 0.9) == 1
    assert b"null" in lib.zs_last_error()


def test_generators_deterministic_and_chunk_independent():
    spec = synthetic.SeriesSpec(20_000, 8, 3, 0.05, 1e-3, 7)
    full = synthetic.rows(spec)
    part = synthetic.rows(spec, 9_000, 17_500)
    np.testing.assert_array_equal(full[9_000:17_500], part)
    ts, te = synthetic.queries(20_000, 100, 10, 5_000, seed=3)
    assert np.all(ts >= 0) and np.all(te < 20_000) and np.all(te >= ts)
    L = te - ts + 1
    assert L.min() >= 10 and L.max() <= 5_000


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5], dtype=np.float32)
    back = synthetic.bf16_bits_to_f64(synthetic.to_bf16_bits(x))
    np.testing.assert_array_equal(back, [1.0, 1.0, 1.0 + 2 ** -7, -2.5])
