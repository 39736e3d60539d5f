"""Eigenvector initialisation (Algorithm 2 / 3 step 2) on the CUDA path against
the oracle, through the C ABI (needs a GB300).

FP64 path: the initial factors are the leading eigenvectors of B_(n) B_(n)^T
from the FP64 Jacobi method; LAPACK's and the GPU's eigenvectors of a
well-separated spectrum agree to about u |G| / gap (< 1e-12 here), so after a
fixed number of ALS sweeps bases, factors and lambda agree to 1e-8 and the fit
to 1e-10, as for the seeded initialisation.  A sign convention that differed
(largest-magnitude entry positive) would flip whole columns and fail by O(1).
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _run(w, R, p, q, tol, iters, seed, init, precision="f64", solver="als"):
    from paper_1703_09074_gb300 import Plan
    dt = torch.float64 if w.dtype == "f64" else torch.float32
    X = torch.from_numpy(np.ascontiguousarray(w.kolda)).cuda()
    with Plan(w.dims, R, p, q, tol, iters, seed=seed, in_dtype=dt, precision=precision,
              init=init, solver=solver) as pl:
        A, lam = pl.decompose(X)
        At, lam_t = pl.compressed_factors()
        res = pl.result()
        return dict(A=[a.cpu().numpy() for a in A], lam=lam.cpu().numpy(),
                    At=[a.cpu().numpy() for a in At], lam_t=lam_t.cpu().numpy(), res=res)


@pytest.mark.parametrize("dims,R,p,q", [((40, 33, 27), 4, 5, 1), ((30, 26, 22, 18), 3, 4, 1),
                                        ((120, 90, 70), 12, 10, 2)])
def test_eig_init_fp64_matches_oracle(dims, R, p, q):
    w = synth.cp_tensor(dims, R, seed=5, snr_db=25.0, dtype="f64", p=p, q=q)
    g = _run(w, R, p, q, 0.0, 12, 3, "eig")
    o = oracle.rcp.rcp_als(w.X, R, p, q, 0.0, 12, 3, init="eig")
    assert g["res"]["device_status"] == 0
    assert abs(g["res"]["fit"] - o["fit"]) < 1e-10
    for Ag, Ao in zip(g["At"], o["A_tilde"]):
        assert np.abs(Ag - Ao).max() < TOL
    assert np.allclose(g["lam_t"], o["lam_tilde"], rtol=TOL, atol=0)
    for Ag, Ao in zip(g["A"], o["A"]):
        assert np.abs(Ag - Ao).max() < TOL
    assert np.allclose(g["lam"], o["lam"], rtol=TOL, atol=0)


def test_eig_init_mixed_form_equal_fit():
    # precision form: the eigenvectors of the FP64 copy of the FP32 core; equal
    # fit with the oracle on the same reduced-precision Gaussian stream
    w = synth.cp_tensor((150, 120, 90), 8, seed=6, congruence=0.3, snr_db=20.0, dtype="f32",
                        p=8, q=1)
    g = _run(w, 8, 8, 1, 0.0, 30, 2, "eig", precision="mixed")
    o = oracle.rcp.rcp_als(w.X, 8, 8, 1, 0.0, 30, 2, init="eig", omega="f32")
    assert g["res"]["device_status"] == 0
    assert g["res"]["rel_err"] == pytest.approx(o["rel_err_identity"], rel=1e-3)


# ---------------------------------------------------------------- rCP-BCD (Algorithm 3)

def _check_fp64(g, o, R, iters=None):
    assert g["res"]["device_status"] == 0, g["res"]
    if iters is not None:
        assert g["res"]["iters"] == iters
    assert abs(g["res"]["fit"] - o["fit"]) < 1e-10
    for Ag, Ao in zip(g["At"], o["A_tilde"]):
        assert np.abs(Ag - Ao).max() < TOL
    assert np.allclose(g["lam_t"], o["lam_tilde"], rtol=TOL, atol=0)
    for Ag, Ao in zip(g["A"], o["A"]):
        assert np.abs(Ag - Ao).max() < TOL
    assert np.allclose(g["lam"], o["lam"], rtol=TOL, atol=0)


@pytest.mark.parametrize("init", ["eig", "randn"])
@pytest.mark.parametrize("dims,R,p,q", [((40, 33, 27), 4, 5, 1), ((24, 20, 18, 16), 3, 4, 1),
                                        ((60, 50), 3, 4, 1)])
def test_bcd_fp64_matches_oracle_fixed_sweeps(dims, R, p, q, init):
    # tol = 0: every component runs exactly max_iters sweeps on both sides
    w = synth.cp_tensor(dims, R, seed=7, snr_db=25.0, dtype="f64", p=p, q=q)
    g = _run(w, R, p, q, 0.0, 8, 2, init, solver="bcd")
    o = oracle.rcp.rcp_als(w.X, R, p, q, 0.0, 8, 2, init=init, solver="bcd")
    assert o["iters"] == 8 * R
    _check_fp64(g, o, R, iters=8 * R)


def test_bcd_fp64_stop_rule_matches_oracle():
    # a well-separated rank-3 tensor: each component's fit settles far from tol's edge
    w = synth.cp_tensor((50, 40, 30), 3, seed=8, snr_db=30.0, dtype="f64", p=5, q=1)
    g = _run(w, 3, 5, 1, 1e-9, 200, 2, "eig", solver="bcd")
    o = oracle.rcp.rcp_als(w.X, 3, 5, 1, 1e-9, 200, 2, init="eig", solver="bcd")
    _check_fp64(g, o, 3, iters=o["iters"])


def test_bcd_mixed_form_equal_fit():
    w = synth.cp_tensor((200, 150, 120), 6, seed=9, snr_db=20.0, dtype="f32", p=8, q=1)
    g = _run(w, 6, 8, 1, 1e-10, 100, 4, "eig", precision="mixed", solver="bcd")
    o = oracle.rcp.rcp_als(w.X, 6, 8, 1, 1e-10, 100, 4, init="eig", omega="f32", solver="bcd")
    assert g["res"]["device_status"] == 0
    assert g["res"]["rel_err"] == pytest.approx(o["rel_err_identity"], rel=1e-3)


def test_learned_start_on_the_single_tensor_path():
    # the untrained network (zero last layer) gives the eigenvector start, so a
    # plan with init="learned" must report the learned start and reach the fit
    # of init="eig" (FP32 versus FP64 eigenvectors of the same core)
    from paper_1703_09074_gb300 import Plan, WarmStartNet
    w = synth.cp_tensor((120, 100, 80), 8, seed=10, congruence=0.3, snr_db=20.0, dtype="f32",
                        p=10, q=1)
    X = torch.from_numpy(np.ascontiguousarray(w.kolda)).cuda()
    net = WarmStartNet(batch=128, seed=1)
    out = {}
    for init in ("learned", "eig"):
        with Plan(w.dims, 8, 10, 1, 0.0, 30, seed=2, in_dtype=torch.float32,
                  precision="mixed", init=init) as pl:
            if init == "learned":
                pl.set_warm_start(net)
            pl.decompose(X)
            out[init] = pl.result()
    net.close()
    assert out["learned"]["device_status"] == 0
    assert out["learned"]["info"] & 4
    assert out["learned"]["rel_err"] == pytest.approx(out["eig"]["rel_err"], rel=1e-3)
