"""Learned warm start for CP-ALS, restated plainly in FP64 (test infrastructure).

The paper starts ALS from eigenvectors or random factors (Section 3.2); the
warm-start network is an addition whose computation is fixed here, step by
step, so that the CUDA path can be checked against it:

* canonical input: U_n = eigenvectors of B_(n) B_(n)^T, eigenvalues
  descending, each vector's largest-magnitude entry (first on ties) positive;
  x = (B x_1 U_1^T x_2 U_2^T x_3 U_3^T) / |B|_F zero-padded to 24^3 with
  index i1 + 24 i2 + 576 i3 (the core of the higher-order SVD, De Lathauwer,
  De Moor & Vandewalle 2000);
* network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3 with
  BF16 rounding (round to nearest even) of the GEMM operands -- inputs,
  weights, h1, h2 and the backward signals dY, dZ2, dZ1 -- exactly where the
  CUDA path rounds them; ``rounding=False`` gives the exact network;
* output: F_n = E + Y_n on l_n rows and R columns (E: first R unit vectors),
  initial factors A_n = U_n F_n;
* loss: D[r, s] = sum_n (1 - (F_n[:, r] . T_n[:, s])^2 / |F_n[:, r]|^2) for unit
  target columns T_n[:, s]; the one-to-one matching of minimum total cost
  (scipy's linear_sum_assignment); loss = (1/R) sum_r D[r, match(r)];
* Adam (Kingma & Ba 2015) with bias correction.

Only tests, the smoke check and the benchmark's CPU baseline use this module.
"""

import numpy as np
from scipy.optimize import linear_sum_assignment

from .tensor import unfold

LPAD, RPAD = 24, 16
IN, HIDDEN, OUT = LPAD ** 3, 512, 3 * LPAD * RPAD


def bf16(a):
    """Round to the nearest BF16 value (ties to even) through FP32, returned as FP64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def layer_sizes(n_in=IN, n_hidden=HIDDEN, n_out=OUT):
    return (n_in, n_hidden, n_out)


def param_offsets(sizes=None):
    """Flat order W1 (H x In), b1, W2 (H x H), b2, W3 (Out x H), b3."""
    n_in, h, n_out = sizes or layer_sizes()
    off = [0]
    for n in (h * n_in, h, h * h, h, n_out * h, n_out):
        off.append(off[-1] + n)
    return off


def unpack(params, sizes=None):
    n_in, h, n_out = sizes or layer_sizes()
    o = param_offsets(sizes)
    p = np.asarray(params, dtype=np.float64)
    return (p[o[0]:o[1]].reshape(h, n_in), p[o[1]:o[2]], p[o[2]:o[3]].reshape(h, h), p[o[3]:o[4]],
            p[o[4]:o[5]].reshape(n_out, h), p[o[5]:o[6]])


def forward(params, x, rounding=True, sizes=None):
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for the rows of x; returns (y, cache)."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(params, sizes)
    X = r(x)
    h1 = np.maximum(X @ r(W1).T + b1, 0.0)
    H1 = r(h1)
    h2 = np.maximum(H1 @ r(W2).T + b2, 0.0)
    H2 = r(h2)
    y = H2 @ r(W3).T + b3
    return y, dict(X=X, H1=H1, H2=H2)


def backward(params, cache, dy, rounding=True, sizes=None):
    """Gradients of sum(dy * y) with respect to every parameter, in the flat order."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(params, sizes)
    X, H1, H2 = cache["X"], cache["H1"], cache["H2"]
    dy = np.asarray(dy, dtype=np.float64)
    dY = r(dy)
    g_b3 = dy.sum(axis=0)
    g_W3 = dY.T @ H2
    dz2 = (dY @ r(W3)) * (H2 > 0)
    dZ2 = r(dz2)
    g_b2 = dz2.sum(axis=0)
    g_W2 = dZ2.T @ H1
    dz1 = (dZ2 @ r(W2)) * (H1 > 0)
    dZ1 = r(dz1)
    g_b1 = dz1.sum(axis=0)
    g_W1 = dZ1.T @ X
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_W3.ravel(), g_b3])


def adam(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns (params, m, v)."""
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def canonical_basis(Bm):
    """[U_1, U_2, U_3] of a 3-way tensor (l_n x l_n each), sorted and sign-fixed."""
    out = []
    for n in range(1, 4):
        Bn = unfold(Bm, n)
        w, V = np.linalg.eigh(Bn @ Bn.T)
        V = V[:, np.argsort(-w, kind="stable")]
        piv = np.argmax(np.abs(V), axis=0)
        s = np.sign(V[piv, np.arange(V.shape[1])])
        s[s == 0] = 1.0
        out.append(V * s)
    return out


def canonicalize(Bpad, meta):
    """x rows (count x 24^3) and bases (count x 3 x 24 x 24) of padded compressed tensors."""
    C = len(meta)
    x = np.zeros((C, IN))
    U = np.zeros((C, 3, LPAD, LPAD))
    for b in range(C):
        l1, l2, l3, R = (int(v) for v in meta[b])
        if l1 == 0:
            continue
        cube = np.asarray(Bpad[b], np.float64).reshape(LPAD, LPAD, LPAD).transpose(2, 1, 0)
        Bm = cube[:l1, :l2, :l3]
        Us = canonical_basis(Bm)
        G = np.einsum("ijk,ia,jb,kc->abc", Bm, Us[0], Us[1], Us[2], optimize=True)
        nB = np.sqrt(np.sum(Bm * Bm))
        Gp = np.zeros((LPAD, LPAD, LPAD))
        if nB > 0:
            Gp[:l1, :l2, :l3] = G / nB
        x[b] = Gp.transpose(2, 1, 0).ravel()
        for n, (l, Un) in enumerate(zip((l1, l2, l3), Us)):
            U[b, n, :l, :l] = Un
    return x, U


def factors_from_output(y, meta_row):
    """F_n = E + Y_n on l_n rows and R columns (3 arrays)."""
    l1, l2, l3, R = (int(v) for v in meta_row)
    Y = np.asarray(y, np.float64).reshape(3, LPAD, RPAD)
    out = []
    for n, l in enumerate((l1, l2, l3)):
        F = Y[n, :l, :R].copy()
        F[np.arange(min(l, R)), np.arange(min(l, R))] += 1.0
        out.append(F)
    return out


def init_factors(y, U, meta_row):
    """Initial factors A_n = U_n F_n (l_n x R) for n = 1, 2, 3."""
    Fs = factors_from_output(y, meta_row)
    ls = [int(v) for v in meta_row[:3]]
    return [np.asarray(U[n][:l, :l], np.float64) @ F for n, (l, F) in enumerate(zip(ls, Fs))]


def targets(U, A, meta_row):
    """T_n = U_n^T A_n with unit columns, in the padded y-row layout."""
    l1, l2, l3, R = (int(v) for v in meta_row)
    T = np.zeros((3, LPAD, RPAD))
    for n, l in enumerate((l1, l2, l3)):
        Tn = np.asarray(U[n][:l, :l], np.float64).T @ np.asarray(A[n], np.float64)
        nrm = np.sqrt(np.sum(Tn * Tn, axis=0))
        T[n, :l, :R] = Tn / np.where(nrm > 0, nrm, 1.0)
    return T.ravel()


def cost_matrix(y, t, meta_row):
    """D[r, s] of one sample."""
    Fs = factors_from_output(y, meta_row)
    l1, l2, l3, R = (int(v) for v in meta_row)
    T = np.asarray(t, np.float64).reshape(3, LPAD, RPAD)
    D = np.zeros((R, R))
    for n, (l, F) in enumerate(zip((l1, l2, l3), Fs)):
        Tn = T[n, :l, :R]
        ff = np.maximum(np.sum(F * F, axis=0), 1e-12)
        D += 1.0 - (F.T @ Tn) ** 2 / ff[:, None]
    return D


def loss(y, t, meta, scale=1.0):
    """Per-sample losses and scale * dloss/dY (count x 1152)."""
    y = np.asarray(y, np.float64)
    C = len(meta)
    out = np.zeros(C)
    dy = np.zeros_like(y)
    for b in range(C):
        l1, l2, l3, R = (int(v) for v in meta[b])
        if R == 0:
            continue
        D = cost_matrix(y[b], t[b], meta[b])
        rows, cols = linear_sum_assignment(D)
        match = np.empty(R, dtype=int)
        match[rows] = cols
        out[b] = D[rows, cols].sum() / R
        Fs = factors_from_output(y[b], meta[b])
        T = np.asarray(t[b], np.float64).reshape(3, LPAD, RPAD)
        G = np.zeros((3, LPAD, RPAD))
        for n, (l, F) in enumerate(zip((l1, l2, l3), Fs)):
            Tm = T[n, :l, :R][:, match]          # matched target column for each r
            ff = np.maximum(np.sum(F * F, axis=0), 1e-12)
            c = np.sum(F * Tm, axis=0)
            G[n, :l, :R] = (scale / R) * (-2.0 * c * Tm / ff + 2.0 * c * c * F / ff ** 2)
        dy[b] = G.ravel()
    return out, dy
