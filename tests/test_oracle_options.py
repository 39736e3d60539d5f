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
