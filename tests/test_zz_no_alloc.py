"""The allocation-free compression entry point (zs_compress_noalloc).

It exists for callers that cannot allocate device memory themselves or let
a library do it: code running while a CUDA graph is captured, plug-ins whose
host program owns every device allocation, loops that must never enter the
allocator.  Its scratch is a fixed array inside the library, so this test
checks that its factors match the store path (zs_store_append, which
allocates its own scratch) within the tolerances the other GPU tests use, on
two calls in a row with different inputs (the second call must not see the
first call's leftovers in the shared array).  Kept in its own file, collected
last, and independent of the other tests' state.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def _store_factors(rows_dev, n, b, k, dtype, refine=False):
    from paper_1805_00754_gb300 import Store
    st = Store(n=n, b=b, k=k, dtype=dtype, capacity_rows=rows_dev.shape[0], fp64_refine=refine)
    st.append(rows_dev)
    nb = st.info()[1]
    out = [st.export_block(i) for i in range(nb)]
    torch.cuda.synchronize()
    res = [(U.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64),
            Vt.cpu().numpy().astype(np.float64), ki) for U, s, Vt, ki in out]
    st.close()
    return res


def _noalloc(rows_dev, n, b, k, dtype_code, fdtype, flags=0):
    from paper_1805_00754_gb300 import zoomsvd
    nrows = rows_dev.shape[0]
    nb = (nrows + b - 1) // b
    U = torch.full((nb, b, k), float("nan"), dtype=fdtype, device=rows_dev.device)
    s = torch.full((nb, k), float("nan"), dtype=fdtype, device=rows_dev.device)
    Vt = torch.full((nb, k, n), float("nan"), dtype=fdtype, device=rows_dev.device)
    torch.cuda.synchronize()
    st = zoomsvd.lib().zs_compress_noalloc(rows_dev.data_ptr(), nrows, rows_dev.stride(0), dtype_code, n, b, k,
                                           flags, U.data_ptr(), s.data_ptr(), Vt.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert st == 0, zoomsvd.lib().zs_last_error().decode()
    torch.cuda.synchronize()
    # the call's status words (in the same fixed array): no bounded wait gave
    # up and every block passed the accuracy test
    assert zoomsvd.noalloc_status() == (0, 0)
    return U.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64), \
        Vt.cpu().numpy().astype(np.float64)


def _compare(ref, got, b, rtol_s, atol_v):
    U, s, Vt = got
    for i, (Ur, sr, Vtr, ki) in enumerate(ref):
        rows = Ur.shape[0]
        np.testing.assert_allclose(s[i][:ki], sr[:ki], rtol=rtol_s)
        assert np.all(s[i][ki:] == 0)
        for j in range(ki):
            c = 1.0 if Vt[i][j] @ Vtr[j] >= 0 else -1.0
            np.testing.assert_allclose(c * Vt[i][j], Vtr[j], atol=atol_v)
            np.testing.assert_allclose(c * U[i][:rows, j], Ur[:, j], atol=atol_v)
        assert np.all(U[i][rows:] == 0)


@pytest.mark.parametrize("case", ["f32", "f64"])
def test_noalloc_matches_store_two_calls(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    if case == "f32":
        w = synthetic.WORKLOADS["compress_f32"]
        n, b, k, code, fdt, rtol, atol = 256, w.b, w.k, 1, torch.float32, 1e-4, 2e-3
        inputs = [synthetic.rows(w.series, 0, 5 * b + 100).astype(np.float32),
                  synthetic.rows(w.series, 40 * b, 43 * b + 7).astype(np.float32)]
    else:
        w = synthetic.WORKLOADS["plain_f64"]
        n, b, k, code, fdt, rtol, atol = 32, w.b, w.k, 0, torch.float64, 1e-10, 1e-8
        inputs = [synthetic.rows(w.series, 0, 4_321), synthetic.rows(w.series, 9_000, 12_000)]
    for A in inputs:                       # two calls in a row, different inputs
        dev = torch.from_numpy(A).cuda()
        ref = _store_factors(dev, n, b, k, case)
        got = _noalloc(dev, n, b, k, code, fdt)
        _compare(ref, got, b, rtol, atol)


def test_noalloc_rejects_oversized_and_bad_args():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_00754_gb300 import zoomsvd
    lib = zoomsvd.lib()
    x = torch.zeros((4, 8), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # k > n
    assert lib.zs_compress_noalloc(x.data_ptr(), 4, 8, 1, 8, 2, 9, 0, x.data_ptr(), x.data_ptr(),
                                   x.data_ptr(), stream) == 1
    # bad dtype
    assert lib.zs_compress_noalloc(x.data_ptr(), 4, 8, 5, 8, 2, 2, 0, x.data_ptr(), x.data_ptr(),
                                   x.data_ptr(), stream) == 6


@pytest.mark.parametrize("case", ["f32_chunks", "f64_chunks", "bf16"])
def test_noalloc_several_chunks_and_bf16(case):
    """Inputs that take several passes through the fixed array (the chunk
    loop offsets the rows and the three outputs and reuses the scratch within
    one call), and bf16 input rows (FP64 refinement flag, as the precision
    workload uses it)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    flags = 0
    if case == "f32_chunks":
        # n = 128, b = 32768: about 5 MB of scratch per block, so 6 blocks per chunk
        spec = synthetic.SeriesSpec(13 * 32768 + 777, 128, 24, 0.05, 0.0, synthetic.SEED_BASE + 31)
        n, b, k, code, fdt, rtol, atol, dt = 128, 32768, 16, 1, torch.float32, 1e-4, 2e-3, "f32"
        dev = torch.from_numpy(synthetic.rows(spec).astype(np.float32)).cuda()
    elif case == "f64_chunks":
        # n = 512: a 2 MB Gram matrix per block, about 15 blocks per chunk
        spec = synthetic.SeriesSpec(40 * 500 + 123, 512, 12, 0.05, 0.0, synthetic.SEED_BASE + 32)
        n, b, k, code, fdt, rtol, atol, dt = 512, 500, 8, 0, torch.float64, 1e-10, 1e-8, "f64"
        dev = torch.from_numpy(synthetic.rows(spec)).cuda()
    else:
        w = synthetic.WORKLOADS["precision_bf16"]
        spec = dataclasses_replace(w.series, 3 * w.b + 100)
        n, b, k, code, fdt, rtol, atol, dt = 512, w.b, w.k, 2, torch.float32, 1e-4, 2e-3, "bf16"
        flags = 1
        bits = synthetic.to_bf16_bits(synthetic.rows(spec))
        dev = torch.from_numpy(bits.view(np.int16)).cuda()
    ref = _store_factors(dev, n, b, k, dt, refine=bool(flags))
    got = _noalloc(dev, n, b, k, code, fdt, flags)
    _compare(ref, got, b, rtol, atol)


def dataclasses_replace(spec, T):
    import dataclasses
    return dataclasses.replace(spec, T=T)


def test_noalloc_rejects_sizes_past_its_array():
    """n = 256, k = 16 with b = 2^20 rows per block needs ~180 MB of
    projections and Rayleigh-Ritz data per block, past the 32 MiB array."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_00754_gb300 import zoomsvd
    lib = zoomsvd.lib()
    x = torch.zeros((4, 256), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.zs_compress_noalloc(x.data_ptr(), 4, 256, 1, 256, 1 << 20, 16, 0, x.data_ptr(), x.data_ptr(),
                                   x.data_ptr(), stream) == 1
    assert b"scratch bytes per block" in lib.zs_last_error()
