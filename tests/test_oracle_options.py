"""Pins of the oracle's compression options (the remarks after Algorithm 1):
the pivoted-LU normalisation of the power iterations (steps 8-9), per-mode
oversampling and uncompressed modes.  CPU only (``-m "not gpu"``)."""

import numpy as np
import pytest

from oracle import rcp, tensor


def _lu_by_hand(Y):
    """Doolittle elimination with partial pivoting, rows swapped physically
    (the first largest |entry| of the column is the pivot), returning P L."""
    A = np.array(Y, dtype=np.float64)
    m, n = A.shape
    perm = list(range(m))
    L = np.zeros((m, n))
    for k in range(n):
        piv = k + int(np.argmax(np.abs(A[k:, k])))
        A[[k, piv]] = A[[piv, k]]
        L[[k, piv]] = L[[piv, k]]
        perm[k], perm[piv] = perm[piv], perm[k]
        L[k, k] = 1.0
        for i in range(k + 1, m):
            L[i, k] = A[i, k] / A[k, k]
            A[i, k:] -= L[i, k] * A[k, k:]
    PL = np.zeros((m, n))
    for pos, orig in enumerate(perm):
        PL[orig] = L[pos]
    return PL


def test_lu_factor_matches_elimination_by_hand():
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((13, 5))
    PL = rcp.lu_psych(Y)
    assert np.allclose(PL, _lu_by_hand(Y), atol=1e-13)
    # the rows at the pivot positions form a unit lower-triangular matrix, and the
    # other rows' multipliers are bounded by 1 (partial pivoting)
    assert np.abs(PL).max() <= 1.0 + 1e-15
    assert np.linalg.matrix_rank(PL) == 5


def test_lu_normalised_range_finder_spans_the_same_subspace():
    # every normalisation differs by an invertible right factor, so the final
    # basis spans span((T T^T)^q T Omega) either way
    rng = np.random.default_rng(2)
    T = rng.standard_normal((20, 9, 8))
    for q in (1, 2):
        Qa = rcp.range_finder(T, 1, 7, q, seed=3)
        Qb = rcp.range_finder(T, 1, 7, q, seed=3, normalize="lu")
        assert np.abs(Qb.T @ Qb - np.eye(7)).max() < 1e-13
        assert np.linalg.norm(Qa @ Qa.T - Qb @ Qb.T) < 1e-10


def test_skipped_modes_keep_their_dimension():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((12, 6, 10))
    B, Qs = rcp.compress(X, 2, 2, 1, seed=0, skip=(2,))
    assert B.shape == (4, 6, 4)
    assert np.array_equal(Qs[1], np.eye(6))
    Bn, Qn = rcp.compress(X, 2, 2, 1, seed=0, skip=(1, 2, 3))
    assert np.array_equal(Bn, X)


def test_per_mode_oversampling_sets_the_widths():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((15, 14, 13))
    B, Qs = rcp.compress(X, 3, 0, 1, seed=0, p_modes=(1, 4, 2))
    assert [Q.shape[1] for Q in Qs] == [4, 7, 5]
    assert B.shape == (4, 7, 5)
    # noiseless rank 3: every width >= R captures the tensor exactly
    F = [rng.standard_normal((d, 3)) for d in (15, 14, 13)]
    Xl = tensor.kruskal(np.ones(3), F)
    out = rcp.rcp_als(Xl, 3, 0, 1, 1e-14, 300, 0, p_modes=(1, 4, 2), skip=(3,))
    assert out["B"].shape == (4, 7, 13)
    assert rcp.projection_residual(Xl, out["Q"]) < 1e-12


# ---------------------------------------------------------------- independent sketches

def _cp(dims, R, seed):
    rng = np.random.default_rng(seed)
    F = [rng.standard_normal((d, R)) for d in dims]
    return tensor.kruskal(np.ones(R), F)


def test_independent_sketches_span_each_unfolding():
    # noiseless rank 3: every unfolding of X has rank 3, so each independent
    # sketch (q = 0) contains the column space of X_(n) -- the leading left
    # singular vectors from numpy's SVD lie in span(Q_n) -- and B keeps all of X
    X = _cp((11, 9, 13), 3, 5)
    B, Qs = rcp.compress(X, 3, 2, 0, seed=1, independent=True)
    assert B.shape == (5, 5, 5)
    for n, Qn in enumerate(Qs, start=1):
        U = np.linalg.svd(tensor.unfold(X, n), full_matrices=False)[0][:, :3]
        assert np.abs(U - Qn @ (Qn.T @ U)).max() < 1e-12
    assert rcp.projection_residual(X, Qs) < 1e-13
    assert abs(tensor.fro2(B) - tensor.fro2(X)) < 1e-10 * tensor.fro2(X)


def test_independent_bases_do_not_see_the_other_modes():
    # the sequential variant's mode-2 basis changes when mode 1 is left
    # uncompressed; the independent variant's does not (it never reads T_2)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((10, 12, 9))
    _, Qa = rcp.compress(X, 3, 2, 1, seed=2, independent=True)
    _, Qb = rcp.compress(X, 3, 2, 1, seed=2, independent=True, skip=(1,))
    assert np.array_equal(Qa[1], Qb[1]) and np.array_equal(Qa[2], Qb[2])
    _, Qc = rcp.compress(X, 3, 2, 1, seed=2)
    _, Qd = rcp.compress(X, 3, 2, 1, seed=2, skip=(1,))
    assert np.abs(Qc[1] @ Qc[1].T - Qd[1] @ Qd[1].T).max() > 1e-3
    # mode 1 sees X in both variants
    assert np.array_equal(Qa[0], Qc[0])


def test_independent_sketches_meet_theorem1():
    # Theorem 1 is stated for exactly this setting (q = 0, p >= 2): the mean
    # error over seeds stays below sqrt(1 + k/(p-1)) sqrt(sum_n sum_{j>k} s_nj^2)
    rng = np.random.default_rng(7)
    k, p = 4, 2
    for dims in [(18, 16, 14), (9, 10, 8, 7)]:
        X = _cp(dims, 7, 8)
        X = X + 0.05 * rng.standard_normal(dims) * np.sqrt(tensor.fro2(X) / X.size)
        tail = 0.0
        for n in range(1, len(dims) + 1):
            s = np.linalg.svd(tensor.unfold(X, n), compute_uv=False)
            tail += float(np.sum(s[k:] ** 2))
        bound = np.sqrt(1 + k / (p - 1)) * np.sqrt(tail)
        errs = [rcp.projection_residual(X, rcp.compress(X, k, p, 0, seed=sd, independent=True)[1])
                * np.sqrt(tensor.fro2(X)) for sd in range(30)]
        assert np.mean(errs) <= bound
        assert np.mean(errs) > 0.3 * np.sqrt(tail / len(dims))


def test_independent_error_identity_and_recovery():
    # |X - Xhat|^2 = |X|^2 - |B|^2 + |B - Bhat|^2 holds for any orthonormal
    # bases (checked against the explicit residual); with noiseless rank 3 the
    # compression is lossless and ALS from the eigenvector start recovers X
    X = _cp((10, 8, 9), 3, 9)
    out = rcp.rcp_als(X, 3, 2, 1, 0.0, 300, 3, init="eig", independent=True)
    assert rcp.projection_residual(X, out["Q"]) < 1e-13
    assert rcp.rel_error(X, out["lam"], out["A"]) < 1e-9
    rng = np.random.default_rng(10)
    Xn = X + 0.1 * rng.standard_normal(X.shape)
    o2 = rcp.rcp_als(Xn, 3, 2, 0, 0.0, 30, 3, independent=True)
    direct = rcp.rel_error(Xn, o2["lam"], o2["A"])
    assert abs(o2["rel_err_identity"] - direct) < 1e-10
