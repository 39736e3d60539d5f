"""Full-size checks of the precision form on the 4-way and flow-like workloads.

The oracle cannot decompose these tensors (0.5 and 1.7 GB) in seconds, so the
checks are properties that hold at any size, evaluated in FP64 on the host
from the tensor and the GPU's own outputs, in the launch configuration the
benchmark times (rcp_decompose after a plan of the same shape):

* every Q_n has orthonormal columns (FP64 CholeskyQR2: 1e-12);
* the compressed tensor B equals X x_1 Q_1^T ... x_N Q_N^T formed on the host
  from the GPU's bases (split-TF32 products with FP32 accumulation and FP32
  storage of the intermediate tensors: 1e-5 relative);
* the reported relative error (the identity |X|^2 - rho |B|^2) equals
  |X - Xhat| / |X| formed explicitly from the returned factors.  The identity
  takes |B|^2 from the GPU's B, whose split-TF32 error eps_B (measured above)
  moves |X|^2 - |B|^2 by up to 2 eps_B |B|^2; relative to rel_err^2 that is
  amplified by |B|^2 / (|X|^2 rel_err^2), so the bound is
  |d rel_err| <= 1.5 (2 eps_B |B|^2 / |X|^2 + 1e-7) / (2 rel_err);
* the bases capture the signal: the projection residual of X stays within 10%
  above the noise level the SNR fixes (Theorem 1's bound is far looser).
"""

import numpy as np
import pytest
import torch

import synth
from oracle import tensor

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _ttm_chain(X, Qs):
    T = np.asarray(X, dtype=np.float64)
    for n, Q in enumerate(Qs, start=1):
        T = tensor.ttm(T, Q.T, n)
    return T


@pytest.mark.parametrize("name", ["c3_128cubed_x64_f32", "c4_flow_512x1024x800_f32"])
def test_fullsize_mixed_properties(name):
    from paper_1703_09074_gb300 import Plan
    w = synth.config(name)
    X = torch.from_numpy(w.kolda).cuda()
    with Plan(w.dims, w.rank, w.oversample, w.power_iters, w.tol, w.max_iters, seed=0,
              in_dtype=torch.float32, precision="mixed") as p:
        A, lam = p.decompose(X)
        res = p.result()
        Qs = []
        B = p.core().cpu().numpy().T
        A = [a.cpu().numpy() for a in A]
        lam = lam.cpu().numpy()
        # the bases of the same decomposition, mode by mode (same seed, same path)
        for n in range(1, len(w.dims) + 1):
            Qs.append(p.sketch(X, n, return_basis=True).cpu().numpy())
            p.compress(X, n)
        B2 = p.core().cpu().numpy().T
    assert res["device_status"] == 0
    assert np.array_equal(B, B2)  # the mode-by-mode calls reproduce rcp_decompose bit for bit
    for Q in Qs:
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-12
    Bh = _ttm_chain(w.X, Qs)
    eps_b = np.linalg.norm(B - Bh) / np.linalg.norm(Bh)
    assert eps_b <= 1e-5
    Xhat = tensor.kruskal(lam, A)
    nx = np.linalg.norm(np.asarray(w.X, dtype=np.float64))
    rel = np.linalg.norm(np.asarray(w.X, dtype=np.float64) - Xhat) / nx
    nb2 = np.linalg.norm(B) ** 2
    bound = 1.5 * (2.0 * eps_b * nb2 / nx ** 2 + 1e-7) / (2.0 * rel)
    assert abs(res["rel_err"] - rel) <= bound, (res["rel_err"], rel, bound)
    noise = np.sqrt(w.noise_norm2 / (w.signal_norm2 + w.noise_norm2))
    resid = np.sqrt(max(nx ** 2 - np.linalg.norm(B) ** 2, 0.0)) / nx
    assert resid <= 1.1 * noise
