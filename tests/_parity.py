"""Helpers shared by the GPU parity tests: build a device store from seeded rows
and compare a device result with the FP64 oracle's.

What is compared (reading R5/R6 of the oracle: the result is unique up to the
sign of each pair and rotations inside clusters of equal singular values):

* singular values, element by element, to ``s_tol`` relative;
* the rank and the canonical signs (R6) of the device output;
* residuals of the device pairs against the exact matrix of the range (the
  oracle store's reconstruction, Eq. 7, or the raw rows), computed here in
  FP64: r_j = |A^T u_j - s_j v_j| and |A v_j - s_j u_j|.  Each must stay below
  ``resid_tol * s_j + resid_abs * s_1`` (the accuracy the path promises);
* every pair whose singular value is separated from the others by at least
  ``gap * s_1``: the device vectors against the oracle's, within the
  Davis-Kahan bound sin(angle) <= sqrt(r_u^2 + r_v^2) / delta_j that the
  pair's own residuals imply (delta_j = distance from s_j to the other exact
  singular values), times a safety factor C = 2.  At least ``min_pairs``
  pairs must be compared;
* the whole block of live pairs as a subspace, within the Wedin bound
  sqrt(2) |R|_F / delta (delta = gap between the block and the next exact
  singular value), where that gap is >= gap * s_1;
* orthonormality of U and V.
"""
import numpy as np
import torch

import oracle
import synthetic

C_DK = 2.0
# FP64 store: results to ~1e-13; compare where pairs are 1e-6 s_1 apart
F64 = dict(s_tol=1e-10, gap=1e-6, resid_tol=1e-9, resid_abs=1e-11, orth_tol=1e-10)
# float stores: sigma to 1e-4 (the path's accuracy test passes at 1e-5), the
# residual its quadratic bound allows (sqrt(1e-5) s_j, factor 2), FP32 output
# rounding (1e-5 s_1), vectors where pairs are 1e-3 s_1 apart
F32 = dict(s_tol=1e-4, gap=1e-3, resid_tol=6.4e-3, resid_abs=1e-5, orth_tol=5e-4)


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


def store_products(ost, ts, te, U, V):
    """A^T U and A V for A = rows [ts, te] of the oracle store's reconstruction
    (Eq. 7), block by block without forming A."""
    AtU = np.zeros((ost.n, U.shape[1]))
    AV = np.zeros((te - ts + 1, V.shape[1]))
    for i, (lo, hi) in enumerate(oracle.block_bounds(ost.T, ost.b)):
        a, z = max(lo, ts), min(hi, te + 1)
        if a >= z:
            continue
        Ai = (ost.U[i][a - lo: z - lo] * ost.s[i][None, :]) @ ost.Vt[i]
        AtU += Ai.T @ U[a - ts: z - ts]
        AV[a - ts: z - ts] = Ai @ V
    return AtU, AV


def store_spectrum(ost, ts, te):
    """All singular values of rows [ts, te] of the oracle store's
    reconstruction (Eq. 7), from the eigenvalues of its n x n Gram matrix
    accumulated block by block (FP64)."""
    G = np.zeros((ost.n, ost.n))
    for i, (lo, hi) in enumerate(oracle.block_bounds(ost.T, ost.b)):
        a, z = max(lo, ts), min(hi, te + 1)
        if a < z:
            Ai = (ost.U[i][a - lo: z - lo] * ost.s[i][None, :]) @ ost.Vt[i]
            G += Ai.T @ Ai
    ev = np.linalg.eigvalsh(G)[::-1]
    return np.sqrt(np.maximum(ev, 0.0))


def compare_query(out, ref, s_tol, gap, resid_tol, resid_abs, orth_tol=None, label="",
                  ost=None, ts=None, te=None, X=None, ref_s=None, min_pairs=0):
    """Compare a device QueryOut with an oracle QueryResult (see the module
    docstring).  The exact range matrix comes from ``ost`` (oracle store) with
    ``ts``, ``te``, or from ``X`` (raw rows).  ``ref_s``: the range's full
    exact spectrum (else computed here).  Returns (pairs compared, worst
    sin(angle) over them)."""
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
    if rank == 0:
        return 0, 0.0
    if X is not None:
        AtU, AV = X.T @ U[:, :rank], X @ V[:, :rank]
        full = np.linalg.svd(X, compute_uv=False) if ref_s is None else ref_s
    else:
        AtU, AV = store_products(ost, ts, te, U[:, :rank], V[:, :rank])
        full = store_spectrum(ost, ts, te) if ref_s is None else ref_s
    rv = np.linalg.norm(AtU - V[:, :rank] * s[None, :rank], axis=0)
    ru = np.linalg.norm(AV - U[:, :rank] * s[None, :rank], axis=0)
    lim_r = resid_tol * s[:rank] + resid_abs * s1
    bad = np.nonzero(np.maximum(ru, rv) > lim_r)[0]
    assert bad.size == 0, (f"{label} residual of pair {bad[0]}: {max(ru[bad[0]], rv[bad[0]]) / s[bad[0]]:.3g} "
                           f"sigma_j > {lim_r[bad[0]] / s[bad[0]]:.3g}")
    floor = 1e-12 if out.U.dtype == torch.float64 else 1e-6
    pairs, worst = 0, 0.0
    for j in range(rank):
        others = np.delete(full, j) if j < full.size else full
        delta = np.min(np.abs(others - s[j])) if others.size else np.inf
        if delta < gap * s1:
            continue
        bound = C_DK * np.sqrt(2.0 * (ru[j] ** 2 + rv[j] ** 2)) / delta + floor
        c = 1.0 if V[:, j] @ ref.V[:, j] >= 0 else -1.0
        dv = np.linalg.norm(c * V[:, j] - ref.V[:, j])
        du = np.linalg.norm(c * U[:, j] - ref.U[:, j])
        assert dv <= bound and du <= bound, f"{label} vector {j}: dV {dv:.3g} dU {du:.3g} > bound {bound:.3g}"
        pairs += 1
        worst = max(worst, dv / np.sqrt(2.0), du / np.sqrt(2.0))
    assert pairs >= min_pairs, f"{label}: {pairs} pairs compared, fewer than {min_pairs}"
    # the live block as a subspace (Wedin)
    nxt = full[rank] if full.size > rank else 0.0
    dblk = s[rank - 1] - nxt
    if dblk >= gap * s1:
        Q1, Q2 = V[:, :rank], ref.V[:, :rank]
        sin = np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2)
        bound = C_DK * np.sqrt(2.0) * np.sqrt(np.sum(ru ** 2 + rv ** 2)) / dblk + floor
        assert sin <= bound, f"{label} V subspace sin {sin:.3g} > Wedin bound {bound:.3g}"
    if orth_tol is not None:
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
    return pairs, worst


def compare_block(U, s, Vt, ki, Aexact, k, s_tol, gap, resid_tol, resid_abs, label=""):
    """A stored block (device factors) against the exact SVD of its rows:
    sigma to s_tol, residuals, and Davis-Kahan vector bounds as in
    compare_query.  Returns the number of pairs compared."""
    U, s, Vt = _to_np(U), _to_np(s), _to_np(Vt)
    Ue, se, Vte = np.linalg.svd(Aexact, full_matrices=False)
    kk = min(k, se.size)
    assert ki == min(k, Aexact.shape[0], Aexact.shape[1]), label
    s1 = se[0]
    np.testing.assert_allclose(s[:kk], se[:kk], rtol=s_tol, atol=s_tol * 1e-3 * s1, err_msg=label)
    V = Vt[:kk].T
    ru = np.linalg.norm(Aexact @ V - U[:, :kk] * s[None, :kk], axis=0)
    rv = np.linalg.norm(Aexact.T @ U[:, :kk] - V * s[None, :kk], axis=0)
    lim_r = resid_tol * s[:kk] + resid_abs * s1
    assert np.all(np.maximum(ru, rv) <= lim_r), f"{label} residual {np.max(np.maximum(ru, rv) / s[:kk]):.3g}"
    pairs = 0
    for j in range(kk):
        delta = np.min(np.abs(np.delete(se, j) - s[j]))
        if delta < gap * s1:
            continue
        bound = C_DK * np.sqrt(2.0 * (ru[j] ** 2 + rv[j] ** 2)) / delta + 1e-6
        c = 1.0 if V[:, j] @ Vte[j] >= 0 else -1.0
        dv = np.linalg.norm(c * V[:, j] - Vte[j])
        du = np.linalg.norm(c * U[:, j] - Ue[:, j])
        assert dv <= bound and du <= bound, f"{label} vector {j}: dV {dv:.3g} dU {du:.3g} > {bound:.3g}"
        pairs += 1
    return pairs


def sigma_rel_err(out, ref):
    s = _to_np(out.S)
    m = ref.s > 0
    return float(np.max(np.abs(s[m] - ref.s[m]) / ref.s[m])) if m.any() else 0.0
