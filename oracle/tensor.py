"""Tensor algebra for the oracle (FP64 numpy), following the paper's notation.

Tensors are numpy arrays indexed X[i_1, ..., i_N] (modes are 1-based in the
paper, 0-based axes here: mode n is axis n - 1).  Memory order is irrelevant
to this module; every operation is written on logical indices.

* mode-n unfolding X_(n) (Section 2.1, notation; Kolda & Bader convention that
  the paper follows through the MATLAB Tensor Toolbox, Section 3.3): an
  I_n x prod_{m != n} I_m matrix whose column index runs over the remaining
  modes in increasing order with the earliest mode fastest,
* the n-mode matrix product of Section 3.1 (Definition 1): M = X x_n U  <=>
  M_(n) = U X_(n),
* the Khatri-Rao product (Section 3.2.1): column r of A (.) B is the Kronecker
  product a_r (x) b_r (index of B fastest), so that for a 3-way tensor
  X_(1) = A (C (.) B)^T, X_(2) = B (C (.) A)^T, X_(3) = C (B (.) A)^T,
* the Kruskal tensor [[lambda; A_1, ..., A_N]] of Eq. (CPlamb2).
"""

import numpy as np


def unfold(X, n):
    """Mode-n unfolding X_(n) for 1-based mode n."""
    X = np.asarray(X)
    ax = n - 1
    return np.moveaxis(X, ax, 0).reshape(X.shape[ax], -1, order="F")


def fold(M, n, shape):
    """Inverse of unfold: rebuild the tensor of ``shape`` from its mode-n unfolding."""
    ax = n - 1
    rest = [shape[m] for m in range(len(shape)) if m != ax]
    T = np.asarray(M).reshape([shape[ax]] + rest, order="F")
    return np.moveaxis(T, 0, ax)


def ttm(X, U, n):
    """n-mode product X x_n U (Definition 1): (X x_n U)_(n) = U X_(n)."""
    shape = list(X.shape)
    shape[n - 1] = U.shape[0]
    return fold(U @ unfold(X, n), n, shape)


def khatri_rao(mats):
    """Khatri-Rao product mats[0] (.) mats[1] (.) ... ; the last factor's index runs fastest."""
    R = mats[0].shape[1]
    out = mats[0]
    for M in mats[1:]:
        assert M.shape[1] == R
        out = np.einsum("ir,jr->ijr", out, M).reshape(-1, R)
    return out


def kr_except(factors, n):
    """The Khatri-Rao product used for mode n: A_N (.) ... (.) A_{n+1} (.) A_{n-1} (.) ... (.) A_1."""
    N = len(factors)
    return khatri_rao([factors[m] for m in range(N - 1, -1, -1) if m != n - 1])


def kruskal(lam, factors):
    """Full tensor sum_r lam_r a_{1,r} o ... o a_{N,r} (Eq. CPlamb2), via X_(1) = A_1 diag(lam) KR^T."""
    shape = tuple(F.shape[0] for F in factors)
    X1 = (factors[0] * np.asarray(lam)[None, :]) @ kr_except(factors, 1).T
    return fold(X1, 1, shape)


def fro2(X):
    """Squared Frobenius norm."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.vdot(X, X))
