"""The compression options of the remarks after Algorithm 1 on the CUDA path
against the oracle, through the C ABI (needs a GB300): the pivoted-LU
normalisation of the power iterations (steps 8-9 as printed), per-mode
oversampling, and modes left uncompressed.

FP64 path: bases, compressed factors and lambda to 1e-8, the fit to 1e-10, as
for the default path; the LU factor is the same permuted unit lower-trapezoidal
matrix on both sides (partial pivoting with the same rule), so the final QR of
step 12 gives the same Q_n.
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _run(w, R, p, q, iters, seed, precision="f64", **opts):
    from paper_1703_09074_gb300 import Plan
    dt = torch.float64 if w.dtype == "f64" else torch.float32
    X = torch.from_numpy(np.ascontiguousarray(w.kolda)).cuda()
    with Plan(w.dims, R, p, q, 0.0, iters, seed=seed, in_dtype=dt, precision=precision,
              **opts) as pl:
        Qs = []
        for n in range(1, len(w.dims) + 1):
            Qs.append(pl.sketch(X, n, return_basis=True).cpu().numpy())
            pl.compress(X, n)
        pl.als(sync=False)
        At, lam_t = pl.compressed_factors()
        A, lam = pl.project()
        res = pl.result()
        return dict(Q=Qs, At=[a.cpu().numpy() for a in At], lam_t=lam_t.cpu().numpy(),
                    A=[a.cpu().numpy() for a in A], lam=lam.cpu().numpy(), res=res)


def _check(g, o):
    assert g["res"]["device_status"] == 0, g["res"]
    for Qg, Qo in zip(g["Q"], o["Q"]):
        assert Qg.shape == Qo.shape
        assert np.abs(Qg - Qo).max() < TOL
    assert abs(g["res"]["fit"] - o["fit"]) < 1e-10
    for Ag, Ao in zip(g["At"], o["A_tilde"]):
        assert np.abs(Ag - Ao).max() < TOL
    assert np.allclose(g["lam_t"], o["lam_tilde"], rtol=TOL, atol=0)
    for Ag, Ao in zip(g["A"], o["A"]):
        assert np.abs(Ag - Ao).max() < TOL
    assert g["res"]["norm_x2"] == pytest.approx(o["normX2"], rel=1e-12)


@pytest.mark.parametrize("dims,R,p,q", [((60, 45, 40), 4, 6, 1), ((50, 40, 30, 20), 3, 5, 2)])
def test_lu_normalised_power_iterations_match_oracle(dims, R, p, q):
    w = synth.cp_tensor(dims, R, seed=3, snr_db=20.0, dtype="f64", p=p, q=q)
    g = _run(w, R, p, q, 10, 5, lu_norm=True)
    o = oracle.rcp.rcp_als(w.X, R, p, q, 0.0, 10, 5, normalize="lu")
    _check(g, o)


def test_per_mode_oversampling_and_skipped_mode_match_oracle():
    w = synth.cp_tensor((70, 24, 50), 4, seed=4, snr_db=20.0, dtype="f64", p=6, q=1)
    g = _run(w, 4, 6, 1, 10, 2, mode_oversample=(3, 0, 8), skip_modes=(2,))
    o = oracle.rcp.rcp_als(w.X, 4, 6, 1, 0.0, 10, 2, p_modes=(3, 0, 8), skip=(2,))
    assert [q.shape[1] for q in g["Q"]] == [7, 24, 12]
    assert np.array_equal(g["Q"][1], np.eye(24))
    _check(g, o)


def test_skipped_first_mode_fp32_input_and_mixed_form():
    # mode 1 uncompressed: |X|^2 from its own pass, T_2 = X moved (and widened to
    # FP64 on the plain path)
    w = synth.cp_tensor((20, 60, 50), 3, seed=5, snr_db=25.0, dtype="f32", p=5, q=1)
    g = _run(w, 3, 5, 1, 10, 1, skip_modes=(1,))
    o = oracle.rcp.rcp_als(w.X, 3, 5, 1, 0.0, 10, 1, skip=(1,))
    _check(g, o)
    gm = _run(w, 3, 5, 1, 30, 1, precision="mixed", skip_modes=(1,))
    om = oracle.rcp.rcp_als(w.X, 3, 5, 1, 0.0, 30, 1, skip=(1,), omega="f32")
    assert gm["res"]["device_status"] == 0
    assert gm["res"]["norm_x2"] == pytest.approx(om["normX2"], rel=1e-6)
    assert gm["res"]["rel_err"] == pytest.approx(om["rel_err_identity"], rel=1e-3)


def test_invalid_options_are_rejected():
    from paper_1703_09074_gb300 import Plan, RcpError
    with pytest.raises(RcpError):   # an uncompressed mode wider than RCP_MAX_L
        Plan((100, 30, 20), 3, 4, 1, skip_modes=(1,), in_dtype=torch.float64)
    with pytest.raises(RcpError):   # the LU variant is a plain-path option
        Plan((100, 30, 20), 3, 4, 1, lu_norm=True, in_dtype=torch.float32, precision="mixed")


# ---------------------------------------------------------------- independent sketches

@pytest.mark.parametrize("dims,R,p,q", [((60, 45, 40), 4, 6, 1), ((30, 24, 20, 16), 3, 5, 2)])
def test_independent_sketches_match_oracle(dims, R, p, q):
    # Theorem 1's setting: every Q_n from X_(n) itself; B by the same chain
    w = synth.cp_tensor(dims, R, seed=7, snr_db=20.0, dtype="f64", p=p, q=q)
    g = _run(w, R, p, q, 10, 4, independent=True)
    o = oracle.rcp.rcp_als(w.X, R, p, q, 0.0, 10, 4, independent=True)
    _check(g, o)


def test_independent_with_lu_skip_and_mode_oversampling():
    w = synth.cp_tensor((40, 24, 36), 3, seed=8, snr_db=15.0, dtype="f32", p=4, q=1)
    g = _run(w, 3, 4, 1, 10, 6, independent=True, lu_norm=True, skip_modes=(2,),
             mode_oversample=(2, 0, 6))
    o = oracle.rcp.rcp_als(w.X, 3, 4, 1, 0.0, 10, 6, independent=True, normalize="lu",
                           skip=(2,), p_modes=(2, 0, 6))
    assert [q.shape[1] for q in g["Q"]] == [5, 24, 9]
    _check(g, o)


def test_independent_sketches_mixed_form():
    # mode 1 on the tensor cores, modes 2-3 by the FP32 sweeps over X itself
    w = synth.cp_tensor((64, 48, 40), 4, seed=9, snr_db=25.0, dtype="f32", p=6, q=1)
    g = _run(w, 4, 6, 1, 30, 2, precision="mixed", independent=True)
    o = oracle.rcp.rcp_als(w.X, 4, 6, 1, 0.0, 30, 2, independent=True, omega="f32")
    assert g["res"]["device_status"] == 0
    for Qg, Qo in zip(g["Q"], o["Q"]):
        # top-R principal angles between the GPU and oracle bases
        s = np.linalg.svd(Qo.T @ Qg, compute_uv=False)
        assert s[:4].min() > 1 - 1e-6
    assert g["res"]["norm_x2"] == pytest.approx(o["normX2"], rel=1e-6)
    assert g["res"]["rel_err"] == pytest.approx(o["rel_err_identity"], rel=1e-3)


def test_independent_plan_needs_x_for_every_mode():
    from paper_1703_09074_gb300 import Plan, _lib
    w = synth.cp_tensor((20, 16, 12), 2, seed=1, snr_db=20.0, dtype="f64", p=2, q=0)
    X = torch.from_numpy(np.ascontiguousarray(w.kolda)).cuda()
    with Plan(w.dims, 2, 2, 0, in_dtype=torch.float64, independent=True) as pl:
        pl.sketch(X, 1)
        pl.compress(X, 1)
        assert pl.lib.rcp_sketch(pl.h, None, 2, None) == _lib.RCP_EINVAL
