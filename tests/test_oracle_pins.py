"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test ties one oracle function to something other than itself: published
known-answer values, brute-force loops over the definitions, an independent
library routine, closed forms (exact recovery, Theorem 1), or invariants of
ALS.  They run on the CPU (``-m "not gpu"``).
"""

import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox, tensor, rcp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox / Omega

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(*[np.array([w], dtype=np.uint64) for w in r[:4]], r[4], r[5])
        assert [int(x[0]) for x in out] == r[6:]


def test_normals_are_standard_gaussian():
    z = philox.normals_f64(12345, 3, philox.PURPOSE_SKETCH, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-3
    z32 = philox.normals_f32_stream(12345, 3, philox.PURPOSE_SKETCH, 200000)
    assert abs(z32.mean()) < 0.01 and abs(z32.var() - 1.0) < 0.02
    assert stats.kstest(z32, "norm").pvalue > 1e-3


def test_box_muller_from_words_by_hand():
    # element 0/1 of a stream = the pair made from counter (0, 0, stream, purpose)
    seed, stream, purpose = 0x1234_5678_9ABC_DEF0, 2, philox.PURPOSE_ALS_INIT
    x = [int(v[0]) for v in philox.philox4x32_10(
        *[np.array([w], dtype=np.uint64) for w in (0, 0, stream, purpose)],
        seed & 0xFFFFFFFF, seed >> 32)]
    ua = ((x[0] >> 5) * 2 ** 26 + (x[1] >> 6)) / 2.0 ** 53
    ub = ((x[2] >> 5) * 2 ** 26 + (x[3] >> 6)) / 2.0 ** 53
    r = np.sqrt(-2.0 * np.log(1.0 - ua))
    z = philox.normals_f64(seed, stream, purpose, 2)
    assert z[0] == pytest.approx(r * np.cos(2 * np.pi * ub), rel=1e-15)
    assert z[1] == pytest.approx(r * np.sin(2 * np.pi * ub), rel=1e-15)


def test_streams_are_distinct_and_row_major():
    a = philox.gaussian_matrix(7, 1, philox.PURPOSE_SKETCH, 6, 5)
    b = philox.gaussian_matrix(7, 2, philox.PURPOSE_SKETCH, 6, 5)
    c = philox.gaussian_matrix(7, 1, philox.PURPOSE_ALS_INIT, 6, 5)
    flat = philox.normals_f64(7, 1, philox.PURPOSE_SKETCH, 30)
    assert np.array_equal(a.ravel(), flat)
    assert not np.allclose(a, b) and not np.allclose(a, c)


# ---------------------------------------------------------------- tensor algebra

def _rand(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("shape", [(2, 3, 4), (3, 2, 4, 2), (5, 1, 3)])
def test_unfold_brute_force(shape):
    X = _rand(shape)
    N = len(shape)
    for n in range(1, N + 1):
        U = tensor.unfold(X, n)
        assert U.shape == (shape[n - 1], X.size // shape[n - 1])
        for idx in np.ndindex(*shape):
            # Kolda & Bader: j = sum_{k != n} i_k prod_{m < k, m != n} I_m
            j, stride = 0, 1
            for k in range(N):
                if k == n - 1:
                    continue
                j += idx[k] * stride
                stride *= shape[k]
            assert U[idx[n - 1], j] == X[idx]
        assert np.array_equal(tensor.fold(U, n, shape), X)


def test_ttm_brute_force_and_identities():
    X = _rand((3, 4, 5))
    U = _rand((2, 4), 1)
    Y = tensor.ttm(X, U, 2)
    ref = np.zeros((3, 2, 5))
    for i in range(3):
        for k in range(2):
            for m in range(5):
                ref[i, k, m] = sum(X[i, j, m] * U[k, j] for j in range(4))
    assert np.allclose(Y, ref, rtol=0, atol=1e-13)
    A, B = _rand((6, 3), 2), _rand((2, 5), 3)
    # modes commute; same-mode products compose
    assert np.allclose(tensor.ttm(tensor.ttm(X, A, 1), B, 3), tensor.ttm(tensor.ttm(X, B, 3), A, 1))
    C = _rand((3, 2), 4)
    assert np.allclose(tensor.ttm(tensor.ttm(X, U, 2), C, 2), tensor.ttm(X, C @ U, 2))
    # Frobenius norm is the same for the tensor and each unfolding
    for n in (1, 2, 3):
        assert tensor.fro2(tensor.unfold(X, n)) == pytest.approx(tensor.fro2(X), rel=1e-15)


def test_khatri_rao_brute_force_and_gram():
    A, B, C = _rand((3, 4), 0), _rand((5, 4), 1), _rand((2, 4), 2)
    K = tensor.khatri_rao([A, B])
    for i in range(3):
        for j in range(5):
            for r in range(4):
                assert K[j + 5 * i, r] == A[i, r] * B[j, r]
    K3 = tensor.khatri_rao([C, B, A])
    assert np.allclose(K3.T @ K3, (C.T @ C) * (B.T @ B) * (A.T @ A))
    # Definition of the Khatri-Rao pseudo-inverse (Section 3.2.1) vs an SVD pinv
    assert np.allclose(np.linalg.pinv((A.T @ A) * (B.T @ B)) @ K.T, np.linalg.pinv(K), atol=1e-12)


def test_kruskal_brute_force_and_matricised_forms():
    lam = np.array([2.0, -0.5, 1.5])
    A, B, C = _rand((4, 3), 0), _rand((3, 3), 1), _rand((5, 3), 2)
    X = tensor.kruskal(lam, [A, B, C])
    ref = np.zeros((4, 3, 5))
    for r in range(3):
        ref += lam[r] * np.einsum("i,j,k->ijk", A[:, r], B[:, r], C[:, r])
    assert np.allclose(X, ref, atol=1e-13)
    L = np.diag(lam)
    # X_(1) = A (C (.) B)^T, X_(2) = B (C (.) A)^T, X_(3) = C (B (.) A)^T (Section 3.2.1)
    assert np.allclose(tensor.unfold(X, 1), A @ L @ tensor.khatri_rao([C, B]).T)
    assert np.allclose(tensor.unfold(X, 2), B @ L @ tensor.khatri_rao([C, A]).T)
    assert np.allclose(tensor.unfold(X, 3), C @ L @ tensor.khatri_rao([B, A]).T)


# ---------------------------------------------------------------- QR, range finder

def _mgs2(Y):
    """Modified Gram-Schmidt, run twice (a QR independent of LAPACK)."""
    Q = np.array(Y, dtype=np.float64)
    R = np.zeros((Y.shape[1], Y.shape[1]))
    for _pass in range(2):
        Rp = np.zeros_like(R)
        for k in range(Q.shape[1]):
            for j in range(k):
                Rp[j, k] = Q[:, j] @ Q[:, k]
                Q[:, k] -= Rp[j, k] * Q[:, j]
            Rp[k, k] = np.linalg.norm(Q[:, k])
            Q[:, k] /= Rp[k, k]
        R = Rp @ R if _pass else Rp
    return Q, R


def test_qr_pos_unique_factor():
    Y = _rand((40, 7), 5)
    Q, R = rcp.qr_pos(Y)
    Qm, Rm = _mgs2(Y)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.allclose(Q @ R, Y, atol=1e-13)
    assert np.abs(Q.T @ Q - np.eye(7)).max() < 1e-14
    assert np.abs(Q - Qm).max() < 1e-12 and np.abs(R - Rm).max() < 1e-12


def test_sketch_width_rule():
    assert rcp.sketch_width(5, 10, (100, 100, 100), 1) == 15
    assert rcp.sketch_width(5, 10, (8, 100, 100), 1) == 8
    assert rcp.sketch_width(5, 10, (100, 2, 3), 1) == 6


def test_range_finder_span_equals_power_scheme():
    # span(Q_n) = span((T T^T)^q T Omega) (Eq. IMPsampleMatrix), on a well-conditioned case
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    V, _ = np.linalg.qr(rng.standard_normal((48, 30)))
    s = np.linspace(3.0, 1.0, 30)
    M = (U * s) @ V.T                       # 30 x 48 with singular values in [1, 3]
    X = M.reshape(30, 6, 8, order="F")
    l = 12
    for q in (0, 1, 2):
        Qn = rcp.range_finder(X, 1, l, q, seed=9)
        Om = philox.gaussian_matrix(9, 1, philox.PURPOSE_SKETCH, 48, l)
        Y = np.linalg.matrix_power(M @ M.T, q) @ M @ Om
        Qy, _ = np.linalg.qr(Y)
        assert np.abs(Qn @ Qn.T - Qy @ Qy.T).max() < 1e-11


def _lowrank(dims, R, seed, snr_db=None):
    rng = np.random.default_rng(seed)
    F = [rng.standard_normal((d, R)) for d in dims]
    X = tensor.kruskal(np.ones(R), F)
    if snr_db is not None:
        G = rng.standard_normal(X.shape)
        X = X + G * np.sqrt(tensor.fro2(X) / tensor.fro2(G)) * 10 ** (-snr_db / 20)
    return X, F


@pytest.mark.parametrize("dims", [(12, 10, 9), (7, 6, 5, 8)])
def test_exact_recovery_noiseless(dims):
    # Section 2.2: a sketch of an exact-rank matrix spans its column space, so a
    # noiseless rank-R tensor with R + p <= I_n is compressed without loss and
    # ALS on B recovers it.
    R = 3
    X, _ = _lowrank(dims, R, 11)
    B, Qs = rcp.compress(X, R, 2, 1, seed=4)
    for Qn in Qs:
        assert np.abs(Qn.T @ Qn - np.eye(Qn.shape[1])).max() < 1e-13
    assert rcp.projection_residual(X, Qs) < 1e-13
    out = rcp.rcp_als(X, R, 2, 1, tol=0.0, max_iters=200, seed=4)
    assert rcp.rel_error(X, out["lam"], out["A"]) < 1e-10


def test_theorem1_bound_stated_form():
    # Theorem 1 with q = 0, p = 2: E|X - X x_1 P_1 ... x_N P_N| <= sqrt(1 + k/(p-1)) sqrt(sum_n sum_{j>k} s_nj^2)
    rng = np.random.default_rng(0)
    k, p = 4, 2
    for dims in [(20, 20, 20), (12, 12, 12, 12)]:
        X, _ = _lowrank(dims, 8, 1)
        X = X + 0.05 * rng.standard_normal(dims) * np.sqrt(tensor.fro2(X) / X.size)
        tail = 0.0
        for n in range(1, len(dims) + 1):
            s = np.linalg.svd(tensor.unfold(X, n), compute_uv=False)
            tail += float(np.sum(s[k:] ** 2))
        bound = np.sqrt(1 + k / (p - 1)) * np.sqrt(tail)
        errs = []
        for seed in range(40):
            _B, Qs = rcp.compress(X, k, p, 0, seed=seed)
            errs.append(rcp.projection_residual(X, Qs) * np.sqrt(tensor.fro2(X)))
        assert np.mean(errs) <= bound
        # and the bound is not vacuous: the error is at least the best rank-k tail of one mode
        assert np.mean(errs) > 0.3 * np.sqrt(tail / len(dims))


def test_error_decreases_with_p_and_q():
    X, _ = _lowrank((40, 40, 40), 6, 2, snr_db=5.0)

    def mean_err(p, q):
        return np.mean([rcp.projection_residual(X, rcp.compress(X, 6, p, q, seed=s)[1])
                        for s in range(6)])
    e_p = [mean_err(p, 0) for p in (2, 5, 10)]
    e_q = [mean_err(2, q) for q in (0, 1, 2)]
    assert e_p[0] > e_p[1] > e_p[2]
    assert e_q[0] > e_q[1] > e_q[2]


# ---------------------------------------------------------------- ALS

def test_als_update_is_least_squares_solution():
    # Algorithm 2 step (4) equals the least-squares solution of B_(1) ~ A (C (.) B)^T
    rng = np.random.default_rng(6)
    B = rng.standard_normal((6, 5, 4))
    A2, A3 = rng.standard_normal((5, 3)), rng.standard_normal((4, 3))
    K = tensor.khatri_rao([A3, A2])
    ls = np.linalg.lstsq(K, tensor.unfold(B, 1).T, rcond=None)[0].T
    init = [None, A2, A3]
    lam, F, rho, it, hist = rcp.cp_als(B, 3, tol=0.0, max_iters=1, seed=0, init=init)
    nu = np.linalg.norm(ls, axis=0)
    assert np.allclose(F[0], ls / nu, atol=1e-12)


def test_als_fit_monotone_and_formula():
    X, _ = _lowrank((9, 8, 7), 4, 3, snr_db=10.0)
    B, _ = rcp.compress(X, 4, 3, 1, seed=0)
    lam, F, rho, it, hist = rcp.cp_als(B, 4, tol=0.0, max_iters=30, seed=0)
    assert np.all(np.diff(hist) >= -1e-13)
    direct = 1.0 - tensor.fro2(B - tensor.kruskal(lam, F)) / tensor.fro2(B)
    assert rho == pytest.approx(direct, abs=1e-12)
    for n, Fn in enumerate(F):
        assert np.allclose(np.linalg.norm(Fn, axis=0), 1.0)


def test_als_rank_one_noiseless_one_sweep():
    rng = np.random.default_rng(8)
    a, b, c = rng.standard_normal(7), rng.standard_normal(6), rng.standard_normal(5)
    B = np.einsum("i,j,k->ijk", a, b, c)
    lam, F, rho, it, hist = rcp.cp_als(B, 1, tol=0.0, max_iters=1, seed=3)
    assert rho == pytest.approx(1.0, abs=1e-12)
    assert lam[0] == pytest.approx(np.linalg.norm(a) * np.linalg.norm(b) * np.linalg.norm(c), rel=1e-12)


def test_stop_rule_counts_sweeps():
    X, _ = _lowrank((9, 8, 7), 2, 5)
    B, _ = rcp.compress(X, 2, 2, 1, seed=0)
    _l, _F, _r, it, hist = rcp.cp_als(B, 2, tol=1e-3, max_iters=50, seed=0)
    assert len(hist) == it
    assert it == 1 or abs(hist[-1] - hist[-2]) < 1e-3
    assert all(abs(hist[j] - (hist[j - 1] if j else 0.0)) >= 1e-3 for j in range(it - 1))


def test_back_projection_and_error_identity():
    X, _ = _lowrank((10, 9, 8), 3, 9, snr_db=15.0)
    out = rcp.rcp_als(X, 3, 3, 2, tol=1e-12, max_iters=100, seed=1)
    for An in out["A"]:
        assert np.allclose(np.linalg.norm(An, axis=0), 1.0, atol=1e-14)
    # renormalisation after recovery only corrects rounding: Q_n is orthonormal
    assert np.allclose(out["lam"], out["lam_tilde"], rtol=1e-13)
    direct = rcp.rel_error(X, out["lam"], out["A"])
    assert out["rel_err_identity"] == pytest.approx(direct, rel=1e-6)
    # |X - Xhat|^2 = |X|^2 - |B|^2 + |B - Bhat|^2
    Bhat = tensor.kruskal(out["lam_tilde"], out["A_tilde"])
    lhs = direct ** 2 * out["normX2"]
    rhs = out["normX2"] - out["normB2"] + tensor.fro2(out["B"] - Bhat)
    assert lhs == pytest.approx(rhs, rel=1e-9)


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """A plausible mistake in the oracle (wrong unfolding order) fails the pins."""
    X = _rand((2, 3, 4))
    good = tensor.unfold(X, 2)
    monkeypatch.setattr(tensor, "unfold",
                        lambda X, n: np.moveaxis(np.asarray(X), n - 1, 0).reshape(X.shape[n - 1], -1))
    bad = tensor.unfold(X, 2)
    assert not np.array_equal(good, bad)
    with pytest.raises(AssertionError):
        test_kruskal_brute_force_and_matricised_forms()
