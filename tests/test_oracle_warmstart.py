"""Pins of the warm-start oracle (oracle/warmstart.py) against mathematics it does not share.

* the network's backward pass against central finite differences of its
  forward pass (exact arithmetic, small layer sizes);
* the loss gradient against finite differences (the matching is locally
  constant);
* the matching against brute force over all permutations;
* the first Adam step against its closed form -lr g / (|g| + eps);
* BF16 rounding against torch's own float32 -> bfloat16 conversion;
* the canonical basis against the definition of the higher-order SVD: the
  U_n are orthogonal, diagonalise B_(n) B_(n)^T with descending eigenvalues,
  and the core's unfoldings have mutually orthogonal rows whose norms are the
  singular values (all-orthogonality and ordering, De Lathauwer et al. 2000);
* a zero network output reproduces the eigenvector initialisation of
  Section 3.2 (the leading R left singular vectors of each unfolding).
"""

import itertools

import numpy as np
import pytest

from oracle import warmstart as ws
from oracle.tensor import unfold


SMALL = (7, 5, 6)


def _params(rng, sizes):
    n = ws.param_offsets(sizes)[-1]
    return rng.standard_normal(n) * 0.5


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng, SMALL)
    x = rng.standard_normal((4, SMALL[0]))
    dy = rng.standard_normal((4, SMALL[2]))
    y, cache = ws.forward(p, x, rounding=False, sizes=SMALL)
    g = ws.backward(p, cache, dy, rounding=False, sizes=SMALL)
    h = 1e-6
    for k in rng.choice(len(p), size=40, replace=False):
        e = np.zeros_like(p)
        e[k] = h
        yp, _ = ws.forward(p + e, x, rounding=False, sizes=SMALL)
        ym, _ = ws.forward(p - e, x, rounding=False, sizes=SMALL)
        fd = np.sum(dy * (yp - ym)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * (1 + abs(fd)), (k, fd, g[k])


def test_forward_is_the_three_layer_formula():
    rng = np.random.default_rng(1)
    p = _params(rng, SMALL)
    x = rng.standard_normal((3, SMALL[0]))
    o = ws.param_offsets(SMALL)
    W1 = p[o[0]:o[1]].reshape(SMALL[1], SMALL[0])
    b1 = p[o[1]:o[2]]
    W2 = p[o[2]:o[3]].reshape(SMALL[1], SMALL[1])
    b2 = p[o[3]:o[4]]
    W3 = p[o[4]:o[5]].reshape(SMALL[2], SMALL[1])
    b3 = p[o[5]:o[6]]
    for i in range(3):
        h1 = [max(0.0, sum(W1[j, k] * x[i, k] for k in range(SMALL[0])) + b1[j]) for j in range(SMALL[1])]
        h2 = [max(0.0, sum(W2[j, k] * h1[k] for k in range(SMALL[1])) + b2[j]) for j in range(SMALL[1])]
        y = [sum(W3[j, k] * h2[k] for k in range(SMALL[1])) + b3[j] for j in range(SMALL[2])]
        got, _ = ws.forward(p, x[i:i + 1], rounding=False, sizes=SMALL)
        assert np.allclose(got[0], y, rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, -3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ws.bf16(a), ref)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    p1, m1, v1 = ws.adam(p, np.zeros(50), np.zeros(50), g, 1, lr, eps=eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_two_steps_by_hand():
    # one parameter p0 = 1, gradients 1/2 then -1/5, lr = 1/10, eps = 0 (Kingma & Ba,
    # Algorithm 1).  By hand: m1 = 1/20, v1 = 1/4000, bias-corrected 1/2 and 1/4,
    # p1 = 9/10; m2 = 1/40, v2 = 1159/4000000, bias-corrected by 1 - 0.9^2 and
    # 1 - 0.999^2 to 5/38 and 1159/7996, p2 = 9/10 - (1/10)(5/38)/sqrt(1159/7996).
    # A correction that used t = 1 again, or none, fails the second step.
    p1, m1, v1 = ws.adam(np.array([1.0]), np.zeros(1), np.zeros(1), np.array([0.5]), 1, 0.1,
                         eps=0.0)
    assert m1[0] == pytest.approx(1 / 20, abs=1e-16)
    assert v1[0] == pytest.approx(1 / 4000, abs=1e-18)
    assert p1[0] == pytest.approx(0.9, abs=1e-15)
    p2, m2, v2 = ws.adam(p1, m1, v1, np.array([-0.2]), 2, 0.1, eps=0.0)
    assert m2[0] == pytest.approx(1 / 40, abs=1e-16)
    assert v2[0] == pytest.approx(1159 / 4000000, abs=1e-18)
    assert p2[0] == pytest.approx(0.9 - 0.1 * (5 / 38) / np.sqrt(1159 / 7996), abs=1e-15)
    assert p2[0] == pytest.approx(0.8654394152087408, abs=1e-14)


def _sample(rng, l=(9, 8, 7), R=5):
    y = rng.standard_normal(ws.OUT) * 0.3
    t = np.zeros((3, ws.LPAD, ws.RPAD))
    for n, ln in enumerate(l):
        T = rng.standard_normal((ln, R))
        t[n, :ln, :R] = T / np.linalg.norm(T, axis=0)
    return y, t.ravel(), np.array([l[0], l[1], l[2], R])


def test_matching_is_the_minimum_over_permutations():
    rng = np.random.default_rng(4)
    for R in (1, 2, 3, 5, 6):
        y, t, meta = _sample(rng, R=R)
        D = ws.cost_matrix(y, t, meta)
        best = min(sum(D[r, p[r]] for r in range(R)) for p in itertools.permutations(range(R)))
        lo, _ = ws.loss(y[None], t[None], meta[None])
        assert abs(lo[0] * R - best) < 1e-12


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    y, t, meta = _sample(rng)
    _, g = ws.loss(y[None], t[None], meta[None], scale=1.0)
    h = 1e-6
    l1, l2, l3, R = meta
    idx = [n * ws.LPAD * ws.RPAD + i * ws.RPAD + r
           for n, ln in enumerate((l1, l2, l3)) for i in range(ln) for r in range(R)]
    for k in rng.choice(idx, size=30, replace=False):
        e = np.zeros_like(y)
        e[k] = h
        lp, _ = ws.loss((y + e)[None], t[None], meta[None])
        lm, _ = ws.loss((y - e)[None], t[None], meta[None])
        fd = (lp[0] - lm[0]) / (2 * h)
        assert abs(fd - g[0, k]) < 1e-6 * (1 + abs(fd))
    # entries outside l_n x R carry no gradient
    mask = np.zeros(ws.OUT, bool)
    mask[idx] = True
    assert np.all(g[0, ~mask] == 0)


def _padded(B):
    l1, l2, l3 = B.shape
    P = np.zeros((ws.LPAD,) * 3)
    P[:l1, :l2, :l3] = B
    return P.transpose(2, 1, 0).ravel()


def test_canonical_core_is_the_hosvd_core():
    rng = np.random.default_rng(6)
    l = (11, 9, 10)
    B = rng.standard_normal(l)
    x, U = ws.canonicalize(_padded(B)[None], np.array([[l[0], l[1], l[2], 4]]))
    G = x[0].reshape(ws.LPAD, ws.LPAD, ws.LPAD).transpose(2, 1, 0)[:l[0], :l[1], :l[2]]
    nB = np.linalg.norm(B)
    for n in range(3):
        Un = U[0, n, :l[n], :l[n]]
        assert np.allclose(Un.T @ Un, np.eye(l[n]), atol=1e-12)
        sv = np.linalg.svd(unfold(B, n + 1), compute_uv=False)
        Gn = unfold(G, n + 1) * nB
        # all-orthogonality: the rows of G_(n) are orthogonal with norms sigma_1 >= sigma_2 >= ...
        M = Gn @ Gn.T
        assert np.allclose(M, np.diag(sv ** 2), atol=1e-9 * sv[0] ** 2)
        piv = np.argmax(np.abs(Un), axis=0)
        assert np.all(Un[piv, np.arange(l[n])] > 0)
    # B is recovered from the core
    Bb = np.einsum("abc,ia,jb,kc->ijk", G * nB, U[0, 0, :l[0], :l[0]], U[0, 1, :l[1], :l[1]],
                   U[0, 2, :l[2], :l[2]])
    assert np.allclose(Bb, B, atol=1e-12)


def test_zero_output_is_the_eigenvector_init():
    rng = np.random.default_rng(7)
    l, R = (10, 9, 8), 4
    B = rng.standard_normal(l)
    x, U = ws.canonicalize(_padded(B)[None], np.array([[l[0], l[1], l[2], R]]))
    A = ws.init_factors(np.zeros(ws.OUT), U[0], [l[0], l[1], l[2], R])
    for n in range(3):
        Ul = np.linalg.svd(unfold(B, n + 1))[0][:, :R]
        # same leading singular subspace, column by column up to sign
        assert np.allclose(np.abs(np.sum(Ul * A[n], axis=0)), 1.0, atol=1e-10)


def test_targets_are_unit_columns_in_the_canonical_basis():
    rng = np.random.default_rng(8)
    l, R = (10, 9, 8), 4
    U = [np.linalg.qr(rng.standard_normal((ln, ln)))[0] for ln in l]
    A = [rng.standard_normal((ln, R)) for ln in l]
    T = ws.targets(U, A, [l[0], l[1], l[2], R]).reshape(3, ws.LPAD, ws.RPAD)
    for n in range(3):
        Tn = T[n, :l[n], :R]
        assert np.allclose(np.linalg.norm(Tn, axis=0), 1.0)
        back = U[n] @ Tn
        cos = np.sum(back * A[n], axis=0) / np.linalg.norm(A[n], axis=0)
        assert np.allclose(cos, 1.0)
