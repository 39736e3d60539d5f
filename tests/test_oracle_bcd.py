"""Pins of the oracle's eigenvector initialisation (Algorithm 2 / 3 step 2) and
of rCP-BCD (Algorithm 3, Section 3.2.2) against closed forms, brute force and
the invariants of block coordinate descent.  CPU only (``-m "not gpu"``)."""

import numpy as np
import pytest

from oracle import rcp, tensor


def _orthodecomposable(dims, lam, seed):
    """B = sum_r lam_r u_1r o ... o u_Nr with orthonormal columns per mode."""
    rng = np.random.default_rng(seed)
    R = len(lam)
    U = [np.linalg.qr(rng.standard_normal((d, R)))[0] for d in dims]
    return tensor.kruskal(np.asarray(lam, dtype=np.float64), U), U


def test_eig_init_closed_form_on_orthogonally_decomposable_core():
    # B_(n) = U_n diag(lam) (KR of the others)^T and that Khatri-Rao product has
    # orthonormal columns, so B_(n) B_(n)^T = U_n diag(lam^2) U_n^T: the
    # eigenvectors are the factor columns in the order of lam
    lam = [5.0, 4.0, 3.0, 2.0, 1.0]
    B, U = _orthodecomposable((9, 8, 7), lam, seed=1)
    E = rcp.eig_init(B, 3)
    assert E[0] is None
    for n in (2, 3):
        V = E[n - 1]
        assert V.shape == (B.shape[n - 1], 3)
        for r in range(3):
            # the same vector up to sign, and the sign rule: largest |entry| positive
            assert abs(abs(V[:, r] @ U[n - 1][:, r]) - 1.0) < 1e-12
            k = np.argmax(np.abs(V[:, r]))
            assert V[k, r] > 0


def test_eig_init_is_an_eigenbasis_in_descending_order():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((6, 7, 5, 4))
    E = rcp.eig_init(B, 4)
    for n in range(2, 5):
        G = tensor.unfold(B, n) @ tensor.unfold(B, n).T
        V = E[n - 1]
        mu = np.einsum("ir,ij,jr->r", V, G, V)
        assert np.all(np.diff(mu) <= 0)
        assert np.abs(G @ V - V * mu[None, :]).max() < 1e-10 * np.abs(G).max()
        assert np.abs(V.T @ V - np.eye(4)).max() < 1e-13
        # no eigenvalue outside the chosen ones is larger than the smallest chosen
        w = np.linalg.eigvalsh(G)
        assert mu[-1] >= w[-4] - 1e-10 * w[-1]


def test_bcd_mode_update_is_rank_one_least_squares():
    # Algorithm 3 step (6): a = Y_(1) (c (.) b) (c^T c b^T b)^+ is the least-squares
    # solution of Y_(1) ~ a (c (.) b)^T for unnormalised b, c
    rng = np.random.default_rng(3)
    B = rng.standard_normal((6, 5, 4))
    b, c = rng.standard_normal(5), rng.standard_normal(4)
    k = np.kron(c, b)   # column of c (.) b, the index of b fastest
    ls = np.linalg.lstsq(k[:, None], tensor.unfold(B, 1).T, rcond=None)[0][0]
    lam, F, rho, it, hist = rcp.cp_bcd(B, 1, tol=0.0, max_iters=1, seed=0,
                                       init=[None, b[:, None], c[:, None]])
    # after the full sweep mode 1 keeps the normalised least-squares solution
    assert np.allclose(F[0][:, 0], ls / np.linalg.norm(ls), atol=1e-12)
    assert it == 1 and len(hist) == 1


def test_bcd_rank_one_noiseless_one_sweep():
    rng = np.random.default_rng(4)
    a, b, c = rng.standard_normal(7), rng.standard_normal(6), rng.standard_normal(5)
    B = np.einsum("i,j,k->ijk", a, b, c)
    init = rcp.eig_init(B, 1)
    lam, F, rho, it, hist = rcp.cp_bcd(B, 1, tol=0.0, max_iters=1, seed=0, init=init)
    assert rho == pytest.approx(1.0, abs=1e-12)
    assert lam[0] == pytest.approx(np.linalg.norm(a) * np.linalg.norm(b) * np.linalg.norm(c),
                                   rel=1e-12)


def test_bcd_deflation_recovers_orthogonal_decomposition_like_als():
    # successive rank-one deflation is exact for an orthogonally decomposable
    # core: each component found is one of the terms, and the residual loses it
    lam_true = [6.0, 4.5, 3.0, 2.0]
    B, U = _orthodecomposable((8, 7, 6), lam_true, seed=5)
    init = rcp.eig_init(B, 4)
    lam, F, rho, it, hist = rcp.cp_bcd(B, 4, tol=1e-15, max_iters=100, seed=0, init=init)
    assert rho == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(lam, lam_true, rtol=1e-10)
    for n in range(3):
        for r in range(4):
            assert abs(abs(F[n][:, r] @ U[n][:, r]) - 1.0) < 1e-10
    # ALS on the same core reaches the same fit
    _l, _F, rho_als, _it, _h = rcp.cp_als(B, 4, tol=1e-15, max_iters=500, seed=0, init=init)
    assert rho_als == pytest.approx(rho, abs=1e-10)


def test_bcd_fit_history_is_monotone_and_counted():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((7, 6, 5)) + 3.0 * np.einsum(
        "i,j,k->ijk", rng.standard_normal(7), rng.standard_normal(6), rng.standard_normal(5))
    lam, F, rho, it, hist = rcp.cp_bcd(B, 3, tol=1e-9, max_iters=60, seed=2)
    # every step is an exact block minimisation of |Y - lambda a o b o c|, and a
    # new component starts from the previous fit (a = 0 is feasible)
    assert np.all(np.diff(hist) >= -1e-12)
    assert len(hist) == it
    direct = 1.0 - tensor.fro2(B - tensor.kruskal(lam, F)) / tensor.fro2(B)
    assert rho == pytest.approx(direct, abs=1e-12)
    for Fn in F:
        assert np.allclose(np.linalg.norm(Fn, axis=0), 1.0)


def test_residual_free_rank_one_mttkrp_identity():
    # the deflated MTTKRP Y_(n) (KR of a_m) without forming Y (Section 3.2.2):
    # B_(n) (KR a_m) - sum_s lam_s a_{n,s} prod_{m != n} (a_{m,s}^T a_m), by brute force
    rng = np.random.default_rng(7)
    B = rng.standard_normal((5, 4, 3))
    lam = rng.standard_normal(2)
    P = [rng.standard_normal((d, 2)) for d in B.shape]
    a = [rng.standard_normal(d) for d in B.shape]
    Y = B - tensor.kruskal(lam, P)
    for n in range(3):
        lhs = np.zeros(B.shape[n])
        for idx in np.ndindex(*B.shape):
            w = np.prod([a[m][idx[m]] for m in range(3) if m != n])
            lhs[idx[n]] += Y[idx] * w
        kr = tensor.kr_except([v[:, None] for v in a], n + 1)[:, 0]
        rhs = tensor.unfold(B, n + 1) @ kr
        for s in range(2):
            rhs = rhs - lam[s] * P[n][:, s] * np.prod([P[m][:, s] @ a[m] for m in range(3) if m != n])
        assert np.allclose(lhs, rhs, atol=1e-12)


def test_rcp_bcd_whole_method_error_identity():
    rng = np.random.default_rng(8)
    F = [rng.standard_normal((d, 3)) for d in (12, 10, 9)]
    X = tensor.kruskal(np.array([3.0, 2.0, 1.0]), F) + 0.01 * rng.standard_normal((12, 10, 9))
    out = rcp.rcp_als(X, 3, 3, 1, tol=1e-12, max_iters=200, seed=1, solver="bcd", init="eig")
    direct = rcp.rel_error(X, out["lam"], out["A"])
    assert out["rel_err_identity"] == pytest.approx(direct, rel=1e-6)
    for An in out["A"]:
        assert np.allclose(np.linalg.norm(An, axis=0), 1.0, atol=1e-14)
