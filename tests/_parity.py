"""Helpers shared by the GPU parity tests: build a device store from seeded rows
and compare a device result with the FP64 oracle's, element by element where
the result is unique (singular values; vectors of well-separated pairs, up to
the sign the method leaves free) and by invariants elsewhere."""
import numpy as np
import torch

import synthetic


def device_rows(A64: np.ndarray, dtype: str):
    """Rows as the library reads them, and the exact values the oracle gets."""
    if dtype == "f64":
        return torch.from_numpy(np.ascontiguousarray(A64)).cuda(), A64
    if dtype == "f32":
        A32 = np.ascontiguousarray(A64, dtype=np.float32)
        return torch.from_numpy(A32).cuda(), A32.astype(np.float64)
    bits = synthetic.to_bf16_bits(A64)
    return torch.from_numpy(bits.view(np.int16)).cuda(), synthetic.bf16_bits_to_f64(bits)


def gpu_store(A64, b, k, dtype, refine=False, capacity=None, exact_gram=False):
    from paper_1805_00754_gb300 import Store
    rows, exact = device_rows(A64, dtype)
    st = Store(n=A64.shape[1], b=b, k=k, dtype=dtype, capacity_rows=capacity or A64.shape[0],
               fp64_refine=refine, exact_gram=exact_gram)
    st.append(rows)
    torch.cuda.synchronize()
    return st, exact


def _to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def check_canonical(V, s):
    """Reading R6 on the device output: largest-|.| entry of each live v_j > 0."""
    for j in range(V.shape[1]):
        if s[j] == 0:
            assert np.all(V[:, j] == 0)
            continue
        i = int(np.argmax(np.abs(V[:, j])))
        # allow a near-tie decided differently by rounding
        top = np.sort(np.abs(V[:, j]))[::-1]
        if top.size > 1 and top[0] - top[1] <= 1e-6 * top[0]:
            continue
        assert V[i, j] > 0, f"column {j} not canonically signed"


def compare_query(out, ref, s_tol, vec_tol, gap=1e-4, orth_tol=None, label=""):
    """Compare a device QueryOut with an oracle QueryResult.

    s_tol: |sigma_gpu - sigma_ref| <= s_tol * sigma_ref_j for live pairs and
    <= s_tol * sigma_1 for the rest.  Vectors: per column after sign alignment,
    only where the relative gap to the neighbours is >= gap; clusters as
    subspaces (sin of the largest principal angle <= vec_tol / gap).
    """
    U, s, V = _to_np(out.U), _to_np(out.S), _to_np(out.V)
    rank = int(out.rank.cpu().item())
    rs = ref.s
    s1 = rs[0] if rs.size and rs[0] > 0 else 1.0
    assert s.shape == rs.shape, label
    err = np.abs(s - rs)
    lim = np.where(rs > 0, s_tol * np.maximum(rs, 1e-300), s_tol * s1)
    assert np.all(err <= np.maximum(lim, s_tol * s1 * 1e-3)), \
        f"{label} sigma mismatch: max rel {np.max(err / np.maximum(rs, 1e-300 + 0 * rs))}"
    assert rank == ref.rank, f"{label} rank {rank} != {ref.rank}"
    check_canonical(V, s)
    worst = 0.0
    for j in range(rank):
        lo = abs(rs[j] - rs[j - 1]) if j > 0 else np.inf
        hi = abs(rs[j] - rs[j + 1]) if j + 1 < rs.size and rs[j + 1] > 0 else np.inf
        if min(lo, hi) / s1 < gap:
            continue
        c = 1.0 if V[:, j] @ ref.V[:, j] >= 0 else -1.0
        dv = np.max(np.abs(c * V[:, j] - ref.V[:, j]))
        du = np.max(np.abs(c * U[:, j] - ref.U[:, j]))
        worst = max(worst, dv, du)
        assert dv <= vec_tol and du <= vec_tol, f"{label} vector {j}: dV {dv:.3g} dU {du:.3g}"
    # whole live subspaces
    if rank:
        Q1, Q2 = V[:, :rank], ref.V[:, :rank]
        sin = np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2)
        assert sin <= max(vec_tol / gap, 1e-12) * 10, f"{label} V subspace sin {sin}"
    if orth_tol is not None and rank:
        # Gram-route accuracy model: U columns built as M V Sigma^-1 carry an
        # orthonormality error ~ eps (sigma_1 / sigma_j)^2.  Well-conditioned
        # columns (sigma_j >= 1e-2 sigma_1 in FP64, >= 5e-2 sigma_1 in FP32)
        # must meet orth_tol; all live columns must meet that model with a
        # factor-100 margin.
        eps = 2.2e-16 if out.U.dtype == torch.float64 else 1.2e-7
        good = int(np.sum(s[:rank] >= (1e-2 if eps < 1e-10 else 5e-2) * s[0]))
        Ug, Vl = U[:, :good], V[:, :rank]
        eu = np.max(np.abs(Ug.T @ Ug - np.eye(good))) if good else 0.0
        ev = np.max(np.abs(Vl.T @ Vl - np.eye(rank)))
        assert eu <= orth_tol, f"{label} U not orthonormal: {eu:.3g}"
        assert ev <= orth_tol, f"{label} V not orthonormal: {ev:.3g}"
        Ul = U[:, :rank]
        ea = np.max(np.abs(Ul.T @ Ul - np.eye(rank)))
        model = max(orth_tol, 100 * eps * (s[0] / s[rank - 1]) ** 2)
        assert ea <= model, f"{label} U orthonormality {ea:.3g} above the Gram-route bound {model:.3g}"
    return worst


def sigma_rel_err(out, ref):
    s = _to_np(out.S)
    m = ref.s > 0
    return float(np.max(np.abs(s[m] - ref.s[m]) / ref.s[m])) if m.any() else 0.0
