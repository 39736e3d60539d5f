"""Failure handling, with the failures made on the host (needs a GB300).

No test here faults, traps or hangs the GPU.  Each one provokes a device-side
error condition through an argument the host controls, checks that the
library reports it in its status word, and then checks that a fresh plan on the
same GPU still matches the oracle -- the context stayed usable:

* a wait budget of one clock cycle makes the grid barriers of the persistent
  ALS kernel give up, which must be reported as RCP_ETIMEOUT (every wait in the
  library is bounded; this is the path that bound takes);
* RCP_FLAG_NO_SHIFT turns off the shifted-CholeskyQR3 fallback, so the sketch
  of a noiseless rank-3 tensor with l = 8 columns (rank-deficient Gram) must
  be reported as RCP_ESINGULAR instead of being repaired.
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

RCP_ESINGULAR, RCP_ETIMEOUT = 4, 6


def _fresh_plan_matches_oracle():
    w = synth.cp_tensor((40, 33, 27), 4, seed=11, snr_db=20.0, dtype="f64", p=5, q=1)
    X = torch.from_numpy(w.kolda).cuda()
    from paper_1703_09074_gb300 import Plan
    with Plan(w.dims, 4, 5, 1, 0.0, 12, seed=3, in_dtype=torch.float64) as p:
        A, lam = p.decompose(X)
        res = p.result()
        A = [a.cpu().numpy() for a in A]
    ref = oracle.rcp.rcp_als(w.X, 4, 5, 1, 0.0, 12, 3)
    assert res["device_status"] == 0
    assert abs(res["fit"] - ref["fit"]) < 1e-10
    for a, b in zip(A, ref["A"]):
        assert np.abs(a - b).max() < 1e-8


def test_grid_barrier_wait_budget_runs_out_and_reports_timeout():
    from paper_1703_09074_gb300 import Plan
    # l = 30 rows per factor: the persistent ALS kernel runs on 60 CTAs with grid
    # barriers between its phases; a one-cycle budget cannot outlast them
    w = synth.cp_tensor((60, 50, 40), 20, seed=12, snr_db=20.0, dtype="f64", p=10, q=0)
    X = torch.from_numpy(w.kolda).cuda()
    with Plan(w.dims, 20, 10, 0, 0.0, 50, seed=1, in_dtype=torch.float64,
              wait_budget=1) as p:
        p.decompose(X)
        res = p.result(raise_on_status=False)
    assert res["device_status"] == RCP_ETIMEOUT, res
    _fresh_plan_matches_oracle()


def test_no_shift_flag_reports_a_singular_sketch():
    from paper_1703_09074_gb300 import Plan
    w = synth.cp_tensor((30, 25, 20), 3, seed=1, snr_db=None, dtype="f64", p=5, q=1)
    X = torch.from_numpy(w.kolda).cuda()
    with Plan(w.dims, 3, 5, 1, 0.0, 20, seed=2, in_dtype=torch.float64, no_shift=True) as p:
        p.decompose(X)
        res = p.result(raise_on_status=False)
    assert res["device_status"] == RCP_ESINGULAR, res
    assert not (res["info"] & 1)   # the shifted fallback did not run
    # the same plan without the flag repairs the sketch with the shift
    with Plan(w.dims, 3, 5, 1, 0.0, 20, seed=2, in_dtype=torch.float64) as p:
        p.decompose(X)
        res = p.result()
    assert res["device_status"] == 0 and res["info"] & 1
    _fresh_plan_matches_oracle()
