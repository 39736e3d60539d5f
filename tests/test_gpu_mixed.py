"""Mixed-precision form (tensor-core TF32 sweeps with FP32 accumulation, FP64
QR and Gram solves) against the FP64 oracle, through the C ABI (needs a GB300).

The oracle runs with the same reduced-precision Gaussian stream evaluated in
FP64, so the bases differ only by the TF32 rounding of the sweeps.
Tolerances, from the arithmetic: the split-TF32 products keep about 21 bits
(error <= 2^-20 relative to |x||y| per product) with FP32 accumulation; the
sketch of a well-separated signal moves the top-R subspace by about that
times the gap factor sigma_1 / (sigma_R - sigma_{l+1}) <= 100 on these
inputs, far inside the 1e-2 allowed on principal angles; compression
residuals agree to 1e-3 relative; "equal fit" is the final relative error
within 1e-3 of the FP64 oracle's (relative).
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import tensor

pytestmark = pytest.mark.gpu


def _mixed(w, seed=0, tol=None, max_iters=None, q=None):
    from paper_1703_09074_gb300 import Plan
    q = w.power_iters if q is None else q
    X = torch.from_numpy(np.ascontiguousarray(w.kolda)).cuda()
    with Plan(w.dims, w.rank, w.oversample, q, w.tol if tol is None else tol,
              w.max_iters if max_iters is None else max_iters, seed=seed,
              in_dtype=torch.float32, precision="mixed") as p:
        Qs = []
        for n in range(1, len(w.dims) + 1):
            Qs.append(p.sketch(X, n, return_basis=True).cpu().numpy())
            p.compress(X, n)
        B = p.core().cpu().numpy().T
        p.als(sync=False)
        A, lam = p.project()
        res = p.result()
        return dict(Q=Qs, B=B, A=[a.cpu().numpy() for a in A], lam=lam.cpu().numpy(), res=res)


def _sin_angle(U, Q):
    """sin of the largest principal angle between span(U) (orthonormal) and span(Q)."""
    return np.linalg.norm(U - Q @ (Q.T @ U), 2)


@pytest.mark.parametrize("dims,R,p,q", [((400, 60, 50), 8, 10, 0), ((400, 60, 50), 8, 10, 2),
                                        ((128, 40, 36, 20), 6, 8, 1), ((256, 90, 70), 12, 20, 1),
                                        ((200, 33, 31), 30, 18, 1)])
def test_mixed_bases_match_oracle_with_same_stream(dims, R, p, q):
    w = synth.cp_tensor(dims, R, seed=2, snr_db=15.0, dtype="f32", p=p, q=q)
    g = _mixed(w, seed=5, tol=0.0, max_iters=20)
    o = oracle.rcp.rcp_als(w.X, R, p, q, 0.0, 20, 5, omega="f32")
    assert g["res"]["device_status"] == 0
    T = np.asarray(w.X, dtype=np.float64)
    for n, (Qg, Qo) in enumerate(zip(g["Q"], o["Q"]), start=1):
        assert Qg.shape == Qo.shape
        assert np.abs(Qg.T @ Qg - np.eye(Qg.shape[1])).max() < 1e-12   # FP64 CholeskyQR2
        U = np.linalg.svd(tensor.unfold(T, n), full_matrices=False)[0][:, :R]
        assert _sin_angle(U, Qg) < _sin_angle(U, Qo) + 1e-2, n
        T = tensor.ttm(T, Qo.T, n)
    # compression quality |X - X x_n Q_n Q_n^T| equal within 1e-3 relative
    assert oracle.rcp.projection_residual(w.X, g["Q"]) == pytest.approx(
        oracle.rcp.projection_residual(w.X, o["Q"]), rel=1e-3)


def test_mixed_equal_fit_after_als_converges():
    w = synth.cp_tensor((400, 60, 52), 5, seed=4, snr_db=20.0, dtype="f32", p=10, q=2)
    g = _mixed(w, seed=0, tol=1e-12, max_iters=500)   # seed 0: ALS converges in ~10 sweeps
    o = oracle.rcp.rcp_als(w.X, 5, 10, 2, 1e-12, 500, 0, omega="f32")
    assert g["res"]["device_status"] == 0
    assert g["res"]["rel_err"] == pytest.approx(o["rel_err_identity"], rel=1e-3)


def test_mixed_mode1_sketch_is_the_tf32_product():
    # q = 0: Q_1 = qr+(X_(1) Omega_1) with the same stream; elementwise to TF32 accuracy
    w = synth.cp_tensor((512, 70, 66), 10, seed=3, snr_db=5.0, dtype="f32", p=22, q=0)
    g = _mixed(w, seed=9, tol=0.0, max_iters=2)
    X1 = tensor.unfold(np.asarray(w.X, dtype=np.float64), 1)
    Om = oracle.rcp.gaussian_test_matrix(9, 1, X1.shape[1], 32, "f32")
    Qo, _ = oracle.rcp.qr_pos(X1 @ Om)
    assert np.abs(g["Q"][0] - Qo).max() < 1e-5


def test_mixed_c2_equal_fit_with_fp64_oracle():
    w = synth.config("c2_400cubed_f32")
    g = _mixed(w, seed=0)
    o = oracle.rcp.rcp_als(w.X, w.rank, w.oversample, w.power_iters, w.tol, w.max_iters, 0)
    assert g["res"]["device_status"] == 0
    assert g["res"]["rel_err"] == pytest.approx(o["rel_err_identity"], rel=1e-3)
    # signal subspace of every mode within the TF32 bound of the FP64 oracle's
    for n, (Qg, Qo) in enumerate(zip(g["Q"], o["Q"]), start=1):
        F = w.factors[n - 1]
        U, _ = np.linalg.qr(F)
        if n == 1:
            assert _sin_angle(U, Qg) < _sin_angle(U, Qo) + 1e-2


def test_mixed_rejects_fp64_input():
    from paper_1703_09074_gb300 import Plan, RcpError
    with pytest.raises(RcpError):
        Plan((40, 30, 20), 3, 4, 1, in_dtype=torch.float64, precision="mixed")
