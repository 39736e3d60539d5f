"""The allocation-free mode-1 range finder against the plan-based one (needs a GB300).

Collected last on purpose: it exercises the library's file-scope scratch array,
so a failure here leaves every other test already run.
"""

import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _static_sketch(lib, X, dtype_code, dims, rank, p, seed):
    I = dims[0]
    J = int(np.prod(dims[1:]))
    l = min(rank + p, I, J)
    Q = torch.full((l, I), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    d = (ctypes.c_int64 * len(dims))(*dims)
    code = lib.rcp_sketch_mode1_static(ctypes.c_void_p(X.data_ptr()), dtype_code, len(dims), d,
                                       rank, p, seed, ctypes.c_void_p(Q.data_ptr()),
                                       ctypes.c_void_p(status.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, Q.t().cpu().numpy(), int(status.item())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_static_sketch_matches_plan_sketch_on_two_calls(dtype):
    from paper_1703_09074_gb300 import Plan, _lib
    lib = _lib.load()
    code_dt = _lib.RCP_DTYPE_F32 if dtype == "f32" else _lib.RCP_DTYPE_F64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    cases = [((400, 60, 50), 20, 10, 5), ((37, 29, 23), 3, 4, 6)]
    for call in range(2):
        for dims, R, p, seed in cases:
            w = synth.cp_tensor(dims, R, seed=seed, snr_db=15.0, dtype=dtype, p=p, q=0)
            X = torch.from_numpy(w.kolda).cuda()
            with Plan(dims, R, p, 0, tol=0.0, max_iters=1, seed=seed, in_dtype=tdt) as plan:
                Qref = plan.sketch(X, 1, return_basis=True).cpu().numpy()
            code, Q, status = _static_sketch(lib, X, code_dt, dims, R, p, seed)
            assert code == _lib.RCP_OK and status == 0, (call, dims, code, status)
            assert Q.shape == Qref.shape
            assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-12
            assert np.abs(Q - Qref).max() < 1e-8, (call, dims)


def test_static_sketch_rejects_sizes_beyond_its_scratch():
    from paper_1703_09074_gb300 import _lib
    lib = _lib.load()
    X = torch.zeros(8, dtype=torch.float32, device="cuda")
    Q = torch.zeros(8, dtype=torch.float64, device="cuda")
    dims = (ctypes.c_int64 * 3)(9000, 100, 100)      # I_1 * l = 9000 * 40 > 259052
    code = lib.rcp_sketch_mode1_static(ctypes.c_void_p(X.data_ptr()), _lib.RCP_DTYPE_F32, 3, dims,
                                       30, 10, 0, ctypes.c_void_p(Q.data_ptr()), None, None)
    assert code == _lib.RCP_EINVAL
