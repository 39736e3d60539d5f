"""Randomized CP decomposition (rCP-ALS), stated step by step in FP64.

Follows Algorithm 1 (randomized tensor compression, Section 3.1), Algorithm 2
(CP-ALS on the compressed tensor and recovery, Section 3.2.1) and the fit of
Section 3.3.  Readings where the paper is silent or inconsistent:

* Omega_n is Gaussian (Section 3.1 text), drawn from the counter-based
  stream of ``oracle.philox`` (stream = mode n, purpose = sketch).
* Every normalisation inside the power iterations (Algorithm 1 steps 8-9,
  which the paper does with pivoted LU, and which Section 3.1 calls
  re-orthonormalisation) and the final QR (step 12) use ``qr_pos``, the unique
  thin QR whose R has a positive diagonal.  All of these differ from LU only by
  a right factor, so the span of the final Q_n is the same in exact arithmetic.
* The number of columns is l_n = min(k + p, I_n, J_n), so Y_n always has full
  column rank for generic data.
* The sketch of mode n is taken of the current compressed tensor
  (Algorithm 1, "X <- B_n" after each mode); ``compress(independent=True)``
  takes every sketch of X itself, the setting of Theorem 1.
* ALS starts from seeded N(0,1) factors (stream = mode n, purpose = ALS init,
  row-major l_n x R) for modes 2..N; mode 1 is computed first and needs none.
* ``norm`` in Algorithm 2 is the column 2-norm, applied every sweep; lambda is
  the column norms of the last mode.  A zero column stays zero, lambda_r = 0.
* The fit is the paper's literal formula (Section 3.3), evaluated on the
  compressed tensor that ALS sees:
      rho = 1 - (|B|^2 + |Bhat|^2 - 2 <Bhat, B>) / |B|^2
  and ALS stops after the first sweep j with |rho_j - rho_{j-1}| < tol
  (rho_0 = 0) or when j reaches max_iters.
* Recovery (Algorithm 2 steps 12-13): A_n = Q_n Atilde_n, re-normalised
  columns, lambda_r multiplied by the product of the removed norms.
"""

import numpy as np

from . import philox
from .tensor import unfold, ttm, kr_except, kruskal, fro2


def qr_pos(Y):
    """Thin QR with a positive diagonal of R (Householder via LAPACK, then sign fix)."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def sketch_width(R, p, dims_current, n):
    """l_n = min(R + p, I_n, J_n) for the current tensor shape and 1-based mode n."""
    I_n = dims_current[n - 1]
    J_n = int(np.prod([d for m, d in enumerate(dims_current) if m != n - 1]))
    return min(R + p, I_n, J_n)


def gaussian_test_matrix(seed, n, J, l, omega="f64"):
    """Omega_n (J x l, element (j, c) = stream element j l + c).

    omega="f64" draws the FP64 stream; omega="f32" evaluates, in FP64, the
    values of the reduced-precision stream that the tensor-core sweeps use.
    """
    if omega == "f32":
        return philox.normals_f32_stream(seed, n, philox.PURPOSE_SKETCH, J * l).reshape(J, l)
    return philox.gaussian_matrix(seed, n, philox.PURPOSE_SKETCH, J, l)


def lu_psych(Y):
    """[L, ~] = lu(Y) of Algorithm 1 steps 8-9: the permuted unit lower-trapezoidal
    factor P L of the partial-pivoting LU Y = P L U (LAPACK getrf via scipy), whose
    columns span the same space as Y's."""
    from scipy.linalg import lu
    PL, _U = lu(np.asarray(Y, dtype=np.float64), permute_l=True)
    return PL


def range_finder(T, n, l, q, seed, omega="f64", normalize="qr"):
    """Basis Q_n for mode n of the current tensor T (Algorithm 1 steps 4-12).

    Y = T_(n) Omega; q times: Q = norm(Y), Z = norm(T_(n)^T Q), Y = T_(n) Z;
    then Q_n = qr+(Y).  norm is qr+ (the default reading) or, with
    normalize="lu", the pivoted-LU factor of steps 8-9 as the paper prints them.
    """
    Tn = unfold(T, n)
    J = Tn.shape[1]
    Omega = gaussian_test_matrix(seed, n, J, l, omega)
    Y = Tn @ Omega
    for _ in range(q):
        if normalize == "lu":
            Q = lu_psych(Y)
            Z = lu_psych(Tn.T @ Q)
        else:
            Q, _r = qr_pos(Y)
            Z, _r = qr_pos(Tn.T @ Q)
        Y = Tn @ Z
    Qn, _r = qr_pos(Y)
    return Qn


def compress(X, R, p, q, seed, omega="f64", normalize="qr", p_modes=None, skip=(),
             independent=False):
    """Algorithm 1: returns the compressed tensor B and the bases [Q_1, ..., Q_N].

    Options of the remark after Algorithm 1: p_modes[n - 1] replaces p for
    mode n, and modes listed in ``skip`` (1-based) are not compressed
    (Q_n = I, the tensor keeps I_n in that mode).

    independent=True is the setting of Theorem 1 (Section 3.1.1): every Q_n is
    the range finder of the unfolding X_(n) of the input itself (width
    l_n = min(k + p, I_n, J_n) with J_n the product of the other input
    dimensions), not of the partly compressed tensor; B = X x_1 Q_1^T ...
    x_N Q_N^T is then the same chain of mode products."""
    X = np.asarray(X, dtype=np.float64)
    T = X
    Qs = []
    for n in range(1, T.ndim + 1):
        if n in skip:
            Qs.append(np.eye(T.shape[n - 1]))
            continue
        pn = p if p_modes is None else p_modes[n - 1]
        src = X if independent else T
        l = sketch_width(R, pn, src.shape, n)
        Qn = range_finder(src, n, l, q, seed, omega, normalize)
        Qs.append(Qn)
        T = ttm(T, Qn.T, n)
    return T, Qs


def als_init(dims, R, seed):
    """Seeded N(0,1) initial factors for modes 2..N (mode 1 entry is None)."""
    out = [None]
    for n in range(2, len(dims) + 1):
        out.append(philox.gaussian_matrix(seed, n, philox.PURPOSE_ALS_INIT, dims[n - 1], R))
    return out


def _colnorm(A):
    return np.sqrt(np.sum(A * A, axis=0))


def _safe_div(A, nu):
    d = np.where(nu > 0, nu, 1.0)
    return np.where(nu[None, :] > 0, A / d[None, :], 0.0)


def fit(B, lam, factors):
    """Section 3.3: rho = 1 - (|B|^2 + |Bhat|^2 - 2<Bhat, B>) / |B|^2 with Bhat formed explicitly."""
    Bhat = kruskal(lam, factors)
    nB = fro2(B)
    return 1.0 - (nB + fro2(Bhat) - 2.0 * float(np.vdot(Bhat, B))) / nB


def cp_als(B, R, tol, max_iters, seed, init=None):
    """Algorithm 2 steps 3-11 on the compressed tensor B.

    Each sweep updates modes 1..N in order with
        A_n = B_(n) (KR of the other factors) (Hadamard product of their Grams)^dagger
    normalises columns (lambda from the last mode), then evaluates the fit.
    Returns (lam, factors, rho, iterations, rho_history).
    """
    B = np.asarray(B, dtype=np.float64)
    N = B.ndim
    A = list(init) if init is not None else als_init(B.shape, R, seed)
    A = [None if F is None else np.array(F, dtype=np.float64) for F in A]
    lam = np.ones(R)
    rho_prev = 0.0
    hist = []
    it = 0
    for it in range(1, max_iters + 1):
        for n in range(1, N + 1):
            V = np.ones((R, R))
            for m in range(1, N + 1):
                if m != n:
                    V = V * (A[m - 1].T @ A[m - 1])
            An = unfold(B, n) @ kr_except(A, n) @ np.linalg.pinv(V)
            nu = _colnorm(An)
            if n < N:
                A[n - 1] = _safe_div(An, nu)
            else:
                lam = nu
                A[n - 1] = _safe_div(An, nu)
        rho = fit(B, lam, A)
        hist.append(rho)
        if abs(rho - rho_prev) < tol:
            break
        rho_prev = rho
    return lam, A, rho, it, hist


def eig_init(B, R):
    """Algorithm 2 step 2 / Algorithm 3 step 2: initial factors of modes 2..N.

    For each mode n >= 2, the eigenvectors of B_(n) B_(n)^T belonging to its R
    largest eigenvalues (in descending order), each with its largest-magnitude
    entry positive (the first such entry on a tie).  Mode 1 is computed first
    and needs none (entry None).
    """
    B = np.asarray(B, dtype=np.float64)
    out = [None]
    for n in range(2, B.ndim + 1):
        Bn = unfold(B, n)
        w, V = np.linalg.eigh(Bn @ Bn.T)
        V = V[:, np.argsort(-w, kind="stable")[:R]]
        piv = np.argmax(np.abs(V), axis=0)
        s = np.sign(V[piv, np.arange(V.shape[1])])
        s[s == 0] = 1.0
        out.append(V * s[None, :])
    return out


def initial_factors(B, R, seed, init="randn"):
    """Initial factors of the stage-2 solvers: seeded N(0,1) or eigenvectors."""
    if init == "eig":
        return eig_init(B, R)
    return als_init(np.asarray(B).shape, R, seed)


def cp_bcd(B, R, tol, max_iters, seed, init=None):
    """Algorithm 3 steps 3-15: CP by successive rank-one deflation (block
    coordinate descent, Section 3.2.2) on the compressed tensor B.

    The residual starts as Y = B.  Component r = 1..R starts from column r of
    the initial factors (modes 2..N) and repeats, for n = 1..N,
        a_n = Y_(n) (KR of the other a_m) / prod_{m != n} a_m^T a_m
    (the rank-one case of Definition 2's pseudo-inverse), normalising a_n for
    n < N and taking lambda_r = |a_N| with a_N normalised at n = N.  After each
    such sweep the fit of the rank-r model, rho = 1 - |Y - lambda_r a_1 o ...
    o a_N|^2 / |B|^2, is compared with the previous sweep's (before the first
    sweep: the fit of the rank-(r-1) model, 1 - |Y|^2 / |B|^2); the component
    is done when the change is below tol or after max_iters sweeps.  Then
    Y = B - [[lambda_{1..r}; A_{:,1..r}, ...]] (step 14).
    Returns (lam, factors, rho, total sweeps over all components, rho history).
    """
    B = np.asarray(B, dtype=np.float64)
    N = B.ndim
    A0 = list(init) if init is not None else als_init(B.shape, R, seed)
    F = [np.zeros((B.shape[n], R)) for n in range(N)]
    lam = np.zeros(R)
    nB = fro2(B)
    Y = B.copy()
    total = 0
    hist = []
    rho = 1.0 - fro2(Y) / nB
    for r in range(R):
        a = [None] + [np.array(A0[n][:, r], dtype=np.float64) for n in range(1, N)]
        lam_r = 0.0
        rho_prev = 1.0 - fro2(Y) / nB
        for _ in range(max_iters):
            for n in range(1, N + 1):
                cols = [None if v is None else v[:, None] for v in a]
                kr = kr_except(cols, n)[:, 0]
                denom = float(np.prod([a[m - 1] @ a[m - 1] for m in range(1, N + 1) if m != n]))
                an = unfold(Y, n) @ kr / denom
                nu = float(np.sqrt(an @ an))
                a[n - 1] = an / nu if nu > 0 else np.zeros_like(an)
                if n == N:
                    lam_r = nu
            total += 1
            rho = 1.0 - fro2(Y - kruskal(np.array([lam_r]), [v[:, None] for v in a])) / nB
            hist.append(rho)
            if abs(rho - rho_prev) < tol:
                break
            rho_prev = rho
        for n in range(N):
            F[n][:, r] = a[n]
        lam[r] = lam_r
        Y = B - kruskal(lam[:r + 1], [Fn[:, :r + 1] for Fn in F])
    return lam, F, rho, total, hist


def back_project(Qs, lam, factors):
    """Algorithm 2 steps 12-13: A_n = Q_n Atilde_n, then re-normalise and update lambda."""
    lam = np.array(lam, dtype=np.float64)
    out = []
    for Qn, At in zip(Qs, factors):
        An = Qn @ At
        nu = _colnorm(An)
        out.append(_safe_div(An, nu))
        lam = lam * nu
    return lam, out


def rcp_als(X, R, p, q, tol, max_iters, seed, init=None, omega="f64", solver="als",
            **compress_options):
    """The whole method: compress, ALS (Algorithm 2) or BCD (Algorithm 3) on B,
    recover.  ``init`` is a list of initial factors, "randn" (the default) or
    "eig" (eigenvectors of B_(n) B_(n)^T); ``compress_options`` go to compress
    (normalize, p_modes, skip).  Returns a dict of every intermediate."""
    X = np.asarray(X, dtype=np.float64)
    B, Qs = compress(X, R, p, q, seed, omega, **compress_options)
    if isinstance(init, str):
        init = initial_factors(B, R, seed, init)
    stage2 = cp_bcd if solver == "bcd" else cp_als
    lam_t, At, rho, iters, hist = stage2(B, R, tol, max_iters, seed, init=init)
    lam, A = back_project(Qs, lam_t, At)
    nX2 = fro2(X)
    nB2 = fro2(B)
    # |X - Xhat|^2 = |X|^2 - |B|^2 + |B - Bhat|^2 (Xhat lies in the span of the Q_n)
    res2 = nX2 - nB2 + nB2 * (1.0 - rho)
    return dict(B=B, Q=Qs, lam_tilde=lam_t, A_tilde=At, fit=rho, iters=iters,
                fit_history=hist, lam=lam, A=A, normX2=nX2, normB2=nB2,
                rel_err_identity=float(np.sqrt(max(res2, 0.0) / nX2)))


def rel_error(X, lam, factors):
    """Section 4: |X - Xhat|_F / |X|_F with Xhat formed explicitly."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.sqrt(fro2(X - kruskal(lam, factors)) / fro2(X)))


def projection_residual(X, Qs):
    """|X - X x_1 Q_1 Q_1^T ... x_N Q_N Q_N^T|_F / |X|_F (Theorem 1's error, relative)."""
    T = np.asarray(X, dtype=np.float64)
    for n, Qn in enumerate(Qs, start=1):
        T = ttm(T, Qn @ Qn.T, n)
    return float(np.sqrt(fro2(X - T) / fro2(X)))
