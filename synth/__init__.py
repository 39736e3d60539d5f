"""Seeded synthetic input tensors shaped like the paper's workloads.

This module holds none of the randomized-CP arithmetic: it only builds test
tensors X = sum_r lambda_r a_{1,r} o ... o a_{N,r} + noise (Eq. CPlamb2 as a
data model) and hands them, identically, to the CUDA path and to the oracle.
Every draw comes from numpy's PCG64 generator seeded from (seed, purpose).

Recipes (the paper's data are not available; these stand in for them):

* ``normal``: factor entries i.i.d. N(0, 1) (Section 4.1's random low-rank
  tensors).
* ``congruence`` c: factors G chol(C)^T with C = (1 - c) I + c 11^T, so that
  the columns have expected pairwise cosine c.
* ``weights``: lambda_r = decay^r, r = 1..R (else lambda_r = 1).
* ``flow``: a 3-way x-by-y-by-time field standing in for the cylinder-flow
  data of Section 4.3: x/y factors exp(-(i - mu)^2 / (2 w^2)) sin(2 pi kappa i / I + phi)
  with mu ~ U[0, I), w ~ U[20, 100], kappa ~ U{1..8}, phi ~ U[0, 2 pi);
  time factors sin(omega_r t + phi_r), omega_r ~ U[0.05, 0.5] rad/step.
* noise: N = sigma G with G i.i.d. N(0, 1) and sigma fixed from the realised
  norms so that 10 log10(|S|^2 / |N|^2) = SNR in dB.

Layout: ``kolda`` arrays are C-contiguous with shape (I_N, ..., I_1), i.e. the
linear index i_1 + I_1 (i_2 + I_2 (i_3 + ...)) with mode 1 fastest.  The
logical tensor X[i_1, ..., i_N] is ``kolda.T``.
"""

import dataclasses
import numpy as np

_PURPOSES = {"factors": 1, "noise": 2, "weights": 3, "shape": 4}


def _rng(seed, purpose, sub=0):
    return np.random.default_rng(np.random.SeedSequence([int(seed), _PURPOSES[purpose], int(sub)]))


@dataclasses.dataclass
class Workload:
    name: str
    dims: tuple          # (I_1, ..., I_N)
    rank: int            # R
    oversample: int      # p
    power_iters: int     # q
    tol: float
    max_iters: int
    dtype: str           # "f64" or "f32"
    seed: int
    kolda: np.ndarray    # C-contiguous (I_N, ..., I_1)
    lam: np.ndarray      # true weights
    factors: list        # true factors, I_n x R
    signal_norm2: float
    noise_norm2: float

    @property
    def X(self):
        """Logical view X[i_1, ..., i_N]."""
        return self.kolda.T

    @property
    def nbytes(self):
        return self.kolda.nbytes


def _congruent(rng, I, R, c):
    G = rng.standard_normal((I, R))
    if c == 0.0:
        return G
    C = (1.0 - c) * np.eye(R) + c * np.ones((R, R))
    return G @ np.linalg.cholesky(C).T


def _flow_factors(rng, dims, R):
    Ix, Iy, It = dims
    out = []
    for I in (Ix, Iy):
        i = np.arange(I, dtype=np.float64)[:, None]
        mu = rng.uniform(0.0, I, R)[None, :]
        w = rng.uniform(20.0, 100.0, R)[None, :]
        kap = rng.integers(1, 9, R)[None, :]
        phi = rng.uniform(0.0, 2.0 * np.pi, R)[None, :]
        out.append(np.exp(-(i - mu) ** 2 / (2.0 * w * w)) * np.sin(2.0 * np.pi * kap * i / I + phi))
    t = np.arange(It, dtype=np.float64)[:, None]
    om = rng.uniform(0.05, 0.5, R)[None, :]
    ph = rng.uniform(0.0, 2.0 * np.pi, R)[None, :]
    out.append(np.sin(om * t + ph))
    return out


def _signal_kolda(lam, factors, dtype, chunk_elems=1 << 26):
    """C-contiguous (I_N, ..., I_1) array of sum_r lam_r a_1r o ... o a_Nr, built slab by slab."""
    dims = [F.shape[0] for F in factors]
    N = len(dims)
    R = factors[0].shape[1]
    out = np.empty(tuple(reversed(dims)), dtype=dtype)
    # rows of the Khatri-Rao product of modes 2..N-1 (mode 2 fastest), slab over the last mode
    inner = np.ones((1, R))
    for F in factors[1:N - 1]:
        inner = np.einsum("ir,jr->ijr", F, inner).reshape(-1, R)
    A1 = factors[0] * lam[None, :]
    slab = inner.shape[0] * dims[0]
    step = max(1, chunk_elems // max(slab, 1))
    FN = factors[N - 1]
    for k0 in range(0, dims[N - 1], step):
        k1 = min(dims[N - 1], k0 + step)
        M = (FN[k0:k1, None, :] * inner[None, :, :]).reshape(-1, R)
        out.reshape(dims[N - 1], -1)[k0:k1] = (M @ A1.T).reshape(k1 - k0, -1).astype(dtype)
    return out


def _add_noise(Xk, snr_db, rng, chunk=1 << 25):
    if snr_db is None:
        return 0.0, float(np.vdot(Xk.ravel().astype(np.float64), Xk.ravel().astype(np.float64)))
    flat = Xk.reshape(-1)
    s2 = 0.0
    for a in range(0, flat.size, chunk):
        v = flat[a:a + chunk].astype(np.float64)
        s2 += float(v @ v)
    G = rng.standard_normal(flat.size, dtype=np.float32)
    g2 = 0.0
    for a in range(0, flat.size, chunk):
        v = G[a:a + chunk].astype(np.float64)
        g2 += float(v @ v)
    sigma = np.sqrt(s2 / g2) * 10.0 ** (-snr_db / 20.0)
    for a in range(0, flat.size, chunk):
        flat[a:a + chunk] += (sigma * G[a:a + chunk].astype(np.float64)).astype(flat.dtype)
    return sigma * sigma * g2, s2


def cp_tensor(dims, R, *, seed=0, kind="normal", congruence=0.0, decay=None,
              snr_db=None, dtype="f32", p=10, q=2, tol=1e-10, max_iters=50, name="custom"):
    """Seeded rank-R tensor plus noise, in Kolda layout."""
    dims = tuple(int(d) for d in dims)
    rng = _rng(seed, "factors")
    if kind == "flow":
        factors = _flow_factors(rng, dims, R)
    else:
        factors = [_congruent(rng, I, R, congruence) for I in dims]
    lam = np.ones(R) if decay is None else decay ** np.arange(1, R + 1, dtype=np.float64)
    npdt = np.float64 if dtype == "f64" else np.float32
    Xk = _signal_kolda(lam, factors, npdt)
    n2, s2 = _add_noise(Xk, snr_db, _rng(seed, "noise"))
    return Workload(name, dims, R, p, q, tol, max_iters, dtype, seed, Xk, lam, factors, s2, n2)


# The five named workloads (sizes and distributions of the paper's experiments).
CONFIGS = {
    "c1_100cubed_f64": dict(dims=(100, 100, 100), R=5, kind="normal", snr_db=20.0,
                            dtype="f64", p=10, q=2),
    "c2_400cubed_f32": dict(dims=(400, 400, 400), R=20, kind="normal", congruence=0.5,
                            snr_db=10.0, dtype="f32", p=10, q=2),
    "c3_128cubed_x64_f32": dict(dims=(128, 128, 128, 64), R=32, kind="normal", decay=0.9,
                                snr_db=15.0, dtype="f32", p=16, q=1),
    "c4_flow_512x1024x800_f32": dict(dims=(512, 1024, 800), R=10, kind="flow", snr_db=20.0,
                                     dtype="f32", p=10, q=2),
}


def config(name, seed=0, **over):
    kw = dict(CONFIGS[name])
    kw.update(over)
    dims = kw.pop("dims")
    R = kw.pop("R")
    return cp_tensor(dims, R, seed=seed, name=name, **kw)


def batch_shapes(count=256, seed=0, lo=32, hi=256, rlo=3, rhi=16):
    """Shapes of the batched workload: I_n ~ U{lo..hi}, R ~ U{rlo..rhi}, congruence ~ U[0, 0.6], SNR ~ U[10, 30] dB."""
    rng = _rng(seed, "shape")
    out = []
    for b in range(count):
        dims = tuple(int(x) for x in rng.integers(lo, hi + 1, 3))
        out.append(dict(dims=dims, R=int(rng.integers(rlo, rhi + 1)),
                        congruence=float(rng.uniform(0.0, 0.6)),
                        snr_db=float(rng.uniform(10.0, 30.0))))
    return out


def batch(count=256, seed=0, p=8, q=1):
    """The batched workload: ``count`` 3-way FP32 tensors of uneven sizes."""
    return [cp_tensor(s["dims"], s["R"], seed=seed * 100003 + b, congruence=s["congruence"],
                      snr_db=s["snr_db"], dtype="f32", p=p, q=q, name=f"batch{b}")
            for b, s in enumerate(batch_shapes(count, seed))]
