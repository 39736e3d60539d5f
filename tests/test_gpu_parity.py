"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (FP64 path): projectors and bases 1e-8, compressed tensor 1e-8
relative, ALS factors 1e-8 and lambda 1e-8 relative under the identical seeded
initialisation, fit 1e-10 absolute.  Philox words are compared bit for bit.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import philox, tensor

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _plan(w, **kw):
    from paper_1703_09074_gb300 import Plan
    dt = torch.float64 if w.dtype == "f64" else torch.float32
    args = dict(oversample=w.oversample, power_iters=w.power_iters, tol=w.tol,
                max_iters=w.max_iters, seed=kw.pop("seed", 0), in_dtype=dt)
    args.update(kw)
    return Plan(w.dims, w.rank, **args)


def _x(w):
    return torch.from_numpy(np.ascontiguousarray(w.kolda)).cuda()


def _proj_dist(Qa, Qb):
    return np.linalg.norm(Qa @ Qa.T - Qb @ Qb.T) / np.sqrt(Qa.shape[1])


def _run_both(w, seed=0, tol=None, max_iters=None):
    tol = w.tol if tol is None else tol
    max_iters = w.max_iters if max_iters is None else max_iters
    X = _x(w)
    out = {}
    with _plan(w, seed=seed, tol=tol, max_iters=max_iters) as p:
        Qs = []
        for n in range(1, len(w.dims) + 1):
            Qs.append(p.sketch(X, n, return_basis=True).cpu().numpy())
            p.compress(X, n)
        B = p.core().cpu().numpy()
        lam_t, fit, iters = p.als()
        At, lam_t2 = p.compressed_factors()
        A, lam = p.project()
        res = p.result()
        out = dict(Q=Qs, B=B.T, lam_t=lam_t.numpy(), fit=fit, iters=iters,
                   At=[a.cpu().numpy() for a in At], A=[a.cpu().numpy() for a in A],
                   lam=lam.cpu().numpy(), res=res)
    ref = oracle.rcp.rcp_als(w.X, w.rank, w.oversample, w.power_iters, tol, max_iters, seed)
    return out, ref


def _compare(g, o, tol=TOL, fit_tol=1e-10, check_iters=True):
    assert g["res"]["device_status"] == 0
    for Qg, Qo in zip(g["Q"], o["Q"]):
        assert Qg.shape == Qo.shape
        assert np.abs(Qg.T @ Qg - np.eye(Qg.shape[1])).max() < 1e-12
        assert _proj_dist(Qg, Qo) < tol
        assert np.abs(Qg - Qo).max() < tol
    nb = np.linalg.norm(o["B"])
    assert np.linalg.norm(g["B"] - o["B"]) / nb < tol
    if check_iters:
        assert g["iters"] == o["iters"]
    assert abs(g["fit"] - o["fit"]) < fit_tol
    for Ag, Ao in zip(g["At"], o["A_tilde"]):
        assert np.abs(Ag - Ao).max() < tol
    assert np.allclose(g["lam_t"], o["lam_tilde"], rtol=tol, atol=0)
    for Ag, Ao in zip(g["A"], o["A"]):
        assert np.abs(Ag - Ao).max() < tol
    assert np.allclose(g["lam"], o["lam"], rtol=tol, atol=0)
    assert g["res"]["norm_x2"] == pytest.approx(o["normX2"], rel=1e-12)
    assert g["res"]["norm_b2"] == pytest.approx(o["normB2"], rel=1e-10)


# --------------------------------------------------------------- random streams

def test_philox_words_bit_exact_and_normals():
    from paper_1703_09074_gb300 import test_normals
    seed, stream, purpose = 0xDEADBEEF12345678, 3, philox.PURPOSE_SKETCH
    first, count = 1_000_001, 200_000
    z, words, f = test_normals(seed, stream, purpose, first, count)
    e = np.arange(first, first + count, dtype=np.uint64)
    ref_words = np.stack(philox._words(seed, stream, purpose, e >> np.uint64(1)), axis=1)
    assert np.array_equal(words.cpu().numpy().view(np.uint32).reshape(-1, 4),
                          ref_words.astype(np.uint32))
    ref = philox.normals_f64(seed, stream, purpose, first + count)[first:]
    assert np.abs(z.cpu().numpy() - ref).max() < 1e-13
    ref32 = philox.normals_f32_stream(seed, stream, purpose, first + count)[first:]
    assert np.abs(f.cpu().numpy().astype(np.float64) - ref32).max() < 5e-6


# --------------------------------------------------------------- whole method, small shapes

SMALL = [
    dict(dims=(13, 11, 9), R=3, p=2, q=1, snr=20.0, dtype="f64"),
    dict(dims=(40, 37, 35), R=4, p=5, q=2, snr=15.0, dtype="f64"),
    dict(dims=(40, 37, 35), R=4, p=5, q=2, snr=15.0, dtype="f32"),
    dict(dims=(12, 10, 9, 7), R=3, p=3, q=1, snr=20.0, dtype="f64"),
    dict(dims=(50, 40), R=3, p=4, q=2, snr=20.0, dtype="f64"),
    dict(dims=(6, 30, 25), R=3, p=5, q=1, snr=20.0, dtype="f64"),     # l_1 = I_1
    dict(dims=(300, 20, 17), R=3, p=3, q=1, snr=20.0, dtype="f32"),   # two row blocks
    dict(dims=(33, 65, 31), R=7, p=9, q=0, snr=10.0, dtype="f64"),    # q = 0, l = 16
    dict(dims=(70, 45, 60), R=20, p=12, q=1, snr=20.0, dtype="f64"),  # l = 32
    dict(dims=(64, 64, 60), R=30, p=18, q=1, snr=25.0, dtype="f64"),  # l = 48
]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: "x".join(map(str, c["dims"])) + f"_{c['dtype']}_q{c['q']}")
def test_small_parity_fixed_iterations(case):
    w = synth.cp_tensor(case["dims"], case["R"], seed=3, snr_db=case["snr"], dtype=case["dtype"],
                        p=case["p"], q=case["q"])
    g, o = _run_both(w, seed=11, tol=0.0, max_iters=12)
    _compare(g, o)


def test_c1_parity_with_stop_rule_and_fixed_iterations():
    w = synth.config("c1_100cubed_f64")
    g, o = _run_both(w, seed=0)                     # 50 iterations or fit change < 1e-10
    _compare(g, o)
    g, o = _run_both(w, seed=0, tol=0.0, max_iters=20)
    _compare(g, o)
    # rel. error through the identity vs the direct residual of the oracle's factors
    direct = oracle.rcp.rel_error(w.X, o["lam"], o["A"])
    assert g["res"]["rel_err"] == pytest.approx(direct, rel=1e-6)


def test_c2_full_size_fp64_parity():
    w = synth.config("c2_400cubed_f32")
    g, o = _run_both(w, seed=0, tol=0.0, max_iters=10)
    _compare(g, o)


# --------------------------------------------------------------- degenerate cases

def test_rank_deficient_noiseless_uses_shifted_qr():
    # noiseless rank 3 with l = 8: every sketch is rank-deficient, so CholeskyQR2
    # breaks down and the shifted CholeskyQR3 fallback must run
    w = synth.cp_tensor((30, 25, 20), 3, seed=1, snr_db=None, dtype="f64", p=5, q=1)
    X = _x(w)
    with _plan(w, seed=2, tol=0.0, max_iters=200) as p:
        Qs = []
        for n in (1, 2, 3):
            Qs.append(p.sketch(X, n, return_basis=True).cpu().numpy())
            p.compress(X, n)
        p.als(sync=False)
        A, lam = p.project()
        res = p.result()
        A = [a.cpu().numpy() for a in A]
        lam = lam.cpu().numpy()
    assert res["device_status"] == 0
    assert res["info"] & 1
    for n, Qg in enumerate(Qs, start=1):
        assert np.abs(Qg.T @ Qg - np.eye(Qg.shape[1])).max() < 1e-12
        U = np.linalg.svd(tensor.unfold(w.X, n), full_matrices=False)[0][:, :3]
        assert np.linalg.norm(U - Qg @ (Qg.T @ U)) < 1e-10   # top-R subspace captured
    assert oracle.rcp.projection_residual(w.X, Qs) < 1e-12
    assert oracle.rcp.rel_error(w.X, lam, A) < 1e-9


def test_nan_input_is_reported():
    from paper_1703_09074_gb300 import RcpError
    w = synth.cp_tensor((20, 18, 16), 3, seed=1, snr_db=20.0, dtype="f64", p=2, q=1)
    k = w.kolda.copy()
    k[3, 4, 5] = np.nan
    X = torch.from_numpy(k).cuda()
    with _plan(w) as p:
        p.decompose(X)
        with pytest.raises(RcpError) as ei:
            p.result()
        assert ei.value.code == 5


def test_order_of_calls_is_enforced():
    from paper_1703_09074_gb300 import RcpError
    w = synth.cp_tensor((20, 18, 16), 3, seed=1, snr_db=20.0, dtype="f64", p=2, q=1)
    X = _x(w)
    with _plan(w) as p:
        with pytest.raises(RcpError) as ei:
            p.compress(X, 1)
        assert ei.value.code == 7
        p.sketch(X, 1)
        with pytest.raises(RcpError):
            p.sketch(None, 2)
        with pytest.raises(RcpError):
            p.als()
        p.compress(X, 1)
        p.sketch(None, 2)
        p.compress(None, 2)
        with pytest.raises(RcpError):
            p.project()


def test_user_init_matches_oracle_user_init():
    w = synth.cp_tensor((25, 22, 19), 4, seed=4, snr_db=15.0, dtype="f64", p=3, q=1)
    X = _x(w)
    rng = np.random.default_rng(0)
    init = [None] + [rng.standard_normal((7, 4)) for _ in range(2)]
    with _plan(w, tol=0.0, max_iters=8) as p:
        for n in (1, 2, 3):
            p.sketch(X, n)
            p.compress(X, n)
        p.als_init([None] + [torch.from_numpy(a).cuda() for a in init[1:]])
        lam_t, fit, it = p.als()
    ref = oracle.rcp.rcp_als(w.X, 4, 3, 1, 0.0, 8, 0, init=init)
    assert abs(fit - ref["fit"]) < 1e-10
    assert np.allclose(lam_t.numpy(), ref["lam_tilde"], rtol=1e-8)


def test_host_entry_point_matches_device_entry_point():
    from paper_1703_09074_gb300 import Plan
    w = synth.cp_tensor((45, 40, 35), 4, seed=6, snr_db=20.0, dtype="f32", p=6, q=2)
    X = _x(w)
    with _plan(w, host_staging=True, tol=0.0, max_iters=10) as p:
        A, lam = p.decompose(X)
        A = [a.cpu().numpy() for a in A]
        lam = lam.cpu().numpy()
        Xh = torch.from_numpy(w.kolda).pin_memory()
        Ah, lamh, res = p.decompose_host(Xh)
    for a, b in zip(A, Ah):
        assert np.array_equal(a, b.numpy())
    assert np.array_equal(lam, lamh.numpy())
    assert res["device_status"] == 0
