"""Python API over the C ABI: torch tensors in, torch tensors out.

PyTorch provides device memory and the CUDA stream; every step of the method
runs in the CUDA kernels of librcp.so.  Tensors are passed in the Kolda layout
of the paper's Tensor-Toolbox convention: a C-contiguous torch tensor of shape
(I_N, ..., I_1) holds X[i_1, ..., i_N] at i_1 + I_1 (i_2 + ...).
"""

import ctypes

import torch

from . import _lib
from ._lib import RcpConfig, RcpResult, check

_DT = {torch.float32: _lib.RCP_DTYPE_F32, torch.float64: _lib.RCP_DTYPE_F64}
_PREC = {"f64": _lib.RCP_PREC_F64, "mixed": _lib.RCP_PREC_MIXED}
_INIT = {"randn": _lib.RCP_INIT_RANDN, "eig": _lib.RCP_INIT_EIG, "learned": _lib.RCP_INIT_LEARNED}
_SOLVER = {"als": _lib.RCP_SOLVER_ALS, "bcd": _lib.RCP_SOLVER_BCD}


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for k, t in enumerate(tensors):
        arr[k] = None if t is None else t.data_ptr()
    return arr


class Plan:
    """One randomized-CP problem shape (Algorithm 2's inputs) bound to a CUDA stream."""

    def __init__(self, dims, rank, oversample=10, power_iters=2, tol=1e-10, max_iters=50,
                 seed=0, in_dtype=torch.float32, precision="f64", host_staging=False,
                 stream=None, init="randn", solver="als", wait_budget=0, no_shift=False,
                 skip_modes=(), mode_oversample=None, lu_norm=False, independent=False):
        self.lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.N = len(self.dims)
        self.R = int(rank)
        self.in_dtype = in_dtype
        cfg = RcpConfig()
        cfg.ndim = self.N
        for k, d in enumerate(self.dims):
            cfg.dims[k] = d
        cfg.in_dtype = _DT[in_dtype]
        cfg.rank = self.R
        cfg.oversample = int(oversample)
        cfg.power_iters = int(power_iters)
        cfg.tol = float(tol)
        cfg.max_iters = int(max_iters)
        cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        cfg.precision = _PREC[precision]
        cfg.flags = ((_lib.RCP_FLAG_HOST_STAGING if host_staging else 0) |
                     (_lib.RCP_FLAG_NO_SHIFT if no_shift else 0) |
                     (_lib.RCP_FLAG_LU_NORM if lu_norm else 0) |
                     (_lib.RCP_FLAG_INDEPENDENT if independent else 0) |
                     (_lib.RCP_FLAG_MODE_OVERSAMPLE if mode_oversample is not None else 0))
        for n in skip_modes:   # 1-based modes left uncompressed
            cfg.skip_modes |= 1 << (int(n) - 1)
        if mode_oversample is not None:
            for k, pn in enumerate(mode_oversample):
                cfg.mode_oversample[k] = int(pn)
        cfg.init = _INIT[init]
        cfg.solver = _SOLVER[solver]
        cfg.wait_budget = int(wait_budget)
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.rcp_plan(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), "rcp_plan")
        self.h = h
        self.widths = [self.lib.rcp_width(self.h, n) for n in range(1, self.N + 1)]

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.rcp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers
    def _check_x(self, X):
        if X is None:
            return None
        if not (X.is_cuda and X.dtype == self.in_dtype and X.is_contiguous()):
            raise ValueError("X must be a contiguous CUDA tensor of the plan's dtype")
        if tuple(reversed(X.shape)) != self.dims:
            raise ValueError(f"X must have shape {tuple(reversed(self.dims))} (Kolda layout)")
        return ctypes.c_void_p(X.data_ptr())

    def _f64(self, *shape):
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    # -- Algorithm 1
    def sketch(self, X, mode, return_basis=False):
        """Range finder of mode n (1-based); returns Q_n (I_n x l_n) when asked."""
        Q = None
        if return_basis:
            Q = self._f64(self.widths[mode - 1], self.dims[mode - 1])  # column-major I_n x l_n
        check(self.lib.rcp_sketch(self.h, self._check_x(X), mode,
                                  None if Q is None else ctypes.c_void_p(Q.data_ptr())),
              f"rcp_sketch({mode})")
        return None if Q is None else Q.t()

    def compress(self, X, mode):
        check(self.lib.rcp_compress(self.h, self._check_x(X), mode), f"rcp_compress({mode})")

    # -- Algorithm 2
    def als_init(self, factors):
        """Initial compressed factors for modes 2..N (each l_n x R); factors[0] is ignored."""
        mats = [None] + [f.to(torch.float64).t().contiguous() for f in factors[1:]]  # column-major
        self._init_keep = mats
        check(self.lib.rcp_als_init(self.h, _ptr_array(mats)), "rcp_als_init")

    def als(self, sync=True):
        if not sync:
            check(self.lib.rcp_als(self.h, None, None, None), "rcp_als")
            return None
        lam = (ctypes.c_double * self.R)()
        fit = ctypes.c_double()
        it = ctypes.c_int32()
        check(self.lib.rcp_als(self.h, lam, ctypes.byref(fit), ctypes.byref(it)), "rcp_als",
              ok=(_lib.RCP_OK, _lib.RCP_ENOTCONV))
        return torch.tensor(list(lam), dtype=torch.float64), fit.value, it.value

    def project(self):
        A = [self._f64(self.R, I) for I in self.dims]   # column-major I_n x R storage
        lam = self._f64(self.R)
        check(self.lib.rcp_project(self.h, _ptr_array(A), ctypes.c_void_p(lam.data_ptr())),
              "rcp_project")
        return [a.t() for a in A], lam

    def decompose(self, X):
        """Whole method, asynchronous on the plan's stream; returns (factors, lambda) on the device."""
        A = [self._f64(self.R, I) for I in self.dims]
        lam = self._f64(self.R)
        check(self.lib.rcp_decompose(self.h, self._check_x(X), _ptr_array(A),
                                     ctypes.c_void_p(lam.data_ptr())), "rcp_decompose")
        return [a.t() for a in A], lam

    def decompose_host(self, X_host, A_host=None, lam_host=None):
        """End to end on host buffers (copies inside the call); needs host_staging=True."""
        if A_host is None:
            A_host = [torch.empty((self.R, I), dtype=torch.float64, pin_memory=True)
                      for I in self.dims]
        if lam_host is None:
            lam_host = torch.empty(self.R, dtype=torch.float64, pin_memory=True)
        res = RcpResult()
        code = self.lib.rcp_decompose_host(
            self.h, ctypes.c_void_p(X_host.data_ptr()), _ptr_array(A_host),
            ctypes.cast(lam_host.data_ptr(), _lib.DP), ctypes.byref(res))
        check(code, "rcp_decompose_host")
        return [a.t() for a in A_host], lam_host, _result_dict(res, self.N)

    def result(self, raise_on_status=True):
        """Result record; a device error status raises unless raise_on_status is False."""
        res = RcpResult()
        code = self.lib.rcp_result_get(self.h, ctypes.byref(res))
        if raise_on_status or code in (_lib.RCP_EINVAL, _lib.RCP_ECUDA):
            check(code, "rcp_result_get")
        return _result_dict(res, self.N)

    def core(self):
        """The compressed tensor B, FP64, Kolda layout (shape (l_N, ..., l_1))."""
        B = self._f64(*reversed(self.widths))
        check(self.lib.rcp_get_core(self.h, ctypes.c_void_p(B.data_ptr())), "rcp_get_core")
        return B

    def compressed_factors(self):
        At = [self._f64(self.R, l) for l in self.widths]
        lam = self._f64(self.R)
        check(self.lib.rcp_get_compressed_factors(self.h, _ptr_array(At),
                                                  ctypes.c_void_p(lam.data_ptr())),
              "rcp_get_compressed_factors")
        return [a.t() for a in At], lam

    def set_warm_start(self, net):
        """Stage-2 start from the warm-start network (a plan made with init="learned")."""
        self._net = net
        check(self.lib.rcp_set_warm_start(self.h, None if net is None else net.h),
              "rcp_set_warm_start")

    def last_error(self):
        st = ctypes.c_int32()
        self.lib.rcp_last_error(self.h, ctypes.byref(st))
        return st.value


def _result_dict(res, N):
    return dict(fit=res.fit, iters=res.iters, info=res.info, norm_x2=res.norm_x2,
                norm_b2=res.norm_b2, rel_err=res.rel_err, device_status=res.device_status,
                widths=[res.widths[k] for k in range(N)])


def decompose(X, rank, oversample=10, power_iters=2, tol=1e-10, max_iters=50, seed=0,
              precision="f64"):
    """Randomized CP decomposition of a Kolda-layout CUDA tensor; returns a dict."""
    dims = tuple(reversed(X.shape))
    with Plan(dims, rank, oversample, power_iters, tol, max_iters, seed, X.dtype, precision) as p:
        A, lam = p.decompose(X)
        out = p.result()
    out.update(A=A, lam=lam)
    return out


def test_normals(seed, stream, purpose, first, count, device="cuda"):
    """The device's Gaussian test-matrix stream: (fp64 normals, Philox words, fp32-stream normals)."""
    lib = _lib.load()
    z = torch.empty(count, dtype=torch.float64, device=device)
    w = torch.empty(4 * count, dtype=torch.int32, device=device)
    f = torch.empty(count, dtype=torch.float32, device=device)
    s = torch.cuda.current_stream(device)
    check(lib.rcp_test_normals(seed, stream, purpose, first, count, ctypes.c_void_p(z.data_ptr()),
                               ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                               ctypes.c_void_p(s.cuda_stream)), "rcp_test_normals")
    return z, w, f


def measure_fma_rate(fp64=True, device="cuda"):
    """The device's FP64 (or FP32) FMA rate in TFLOP/s, from a timed FMA-chain kernel."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    with torch.cuda.device(device):
        s = torch.cuda.current_stream()
        check(lib.rcp_measure_fma_rate(1 if fp64 else 0, ctypes.byref(out),
                                       ctypes.c_void_p(s.cuda_stream)), "rcp_measure_fma_rate")
    return out.value


class BatchedPlan:
    """Many decompositions of uneven shapes run together (one CUDA graph per batch).

    ``problems``: list of dicts with keys dims, rank, oversample, power_iters,
    tol, max_iters, seed (FP32 inputs, mixed precision).
    """

    def __init__(self, problems, stream=None):
        self.lib = _lib.load()
        self.count = len(problems)
        arr = (RcpConfig * self.count)()
        self.dims = []
        self.ranks = []
        for b, pr in enumerate(problems):
            c = arr[b]
            dims = tuple(int(d) for d in pr["dims"])
            c.ndim = len(dims)
            for k, d in enumerate(dims):
                c.dims[k] = d
            c.in_dtype = _lib.RCP_DTYPE_F32
            c.rank = int(pr["rank"])
            c.oversample = int(pr.get("oversample", 8))
            c.power_iters = int(pr.get("power_iters", 1))
            c.tol = float(pr.get("tol", 1e-10))
            c.max_iters = int(pr.get("max_iters", 50))
            c.seed = int(pr.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
            c.precision = _lib.RCP_PREC_MIXED
            c.flags = 0
            self.dims.append(dims)
            self.ranks.append(c.rank)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        h = ctypes.c_void_p()
        check(self.lib.rcp_plan_batched(arr, self.count, ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h)), "rcp_plan_batched")
        self.h = h

    def _ptrs(self, Xs):
        if len(Xs) != self.count:
            raise ValueError("one tensor per problem")
        for X, d in zip(Xs, self.dims):
            if not (X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
                    and tuple(reversed(X.shape)) == d):
                raise ValueError(f"expected a contiguous FP32 CUDA tensor of shape {tuple(reversed(d))}")
        return _ptr_array(Xs)

    def run(self, Xs):
        self._keep = Xs
        check(self.lib.rcp_batched_run(self.h, self._ptrs(Xs)), "rcp_batched_run")

    def autotune(self, Xs):
        """Tune the batched sweeps' shapes on Xs; returns (row CTAs/SM, column CTAs/SM,
        row-sweep loads in flight, column blocks per item)."""
        ch = (ctypes.c_int32 * 4)()
        check(self.lib.rcp_batched_autotune(self.h, self._ptrs(Xs), ch), "rcp_batched_autotune")
        return tuple(ch)

    def result(self, b):
        A = [torch.empty((self.ranks[b], I), dtype=torch.float64, device=self.device)
             for I in self.dims[b]]
        lam = torch.empty(self.ranks[b], dtype=torch.float64, device=self.device)
        res = RcpResult()
        code = self.lib.rcp_batched_result(self.h, b, _ptr_array(A), ctypes.c_void_p(lam.data_ptr()),
                                           ctypes.byref(res))
        check(code, "rcp_batched_result")
        return [a.t() for a in A], lam, _result_dict(res, len(self.dims[b]))

    def intermediates(self, b):
        """Tensor b's bases Q_n (I_n x l_n), core B (Kolda layout, FP64) and ALS factors."""
        l = self.widths(b)
        dev = self.device
        Q = [torch.empty((ln, I), dtype=torch.float64, device=dev) for I, ln in zip(self.dims[b], l)]
        B = torch.empty(tuple(reversed(l)), dtype=torch.float64, device=dev)
        At = [torch.empty((self.ranks[b], ln), dtype=torch.float64, device=dev) for ln in l]
        lam_t = torch.empty(self.ranks[b], dtype=torch.float64, device=dev)
        check(self.lib.rcp_batched_intermediates(self.h, b, _ptr_array(Q), ctypes.c_void_p(B.data_ptr()),
                                                 _ptr_array(At), ctypes.c_void_p(lam_t.data_ptr())),
              "rcp_batched_intermediates")
        return [q.t() for q in Q], B, [a.t() for a in At], lam_t

    def widths(self, b):
        res = RcpResult()
        self.lib.rcp_batched_result(self.h, b, None, None, ctypes.byref(res))
        return [res.widths[k] for k in range(len(self.dims[b]))]

    def set_warm_start(self, net):
        """Start ALS from the network's factors in later runs (None: random init)."""
        self._net = net
        check(self.lib.rcp_batched_set_warm_start(self.h, None if net is None else net.h),
              "rcp_batched_set_warm_start")

    def export(self):
        """Training data of the last run: dict of device tensors B, meta, x, U, t."""
        C = self.count
        dev = self.device
        out = dict(B=torch.empty((C, _lib.MLP_IN), dtype=torch.float32, device=dev),
                   meta=torch.empty((C, 4), dtype=torch.int32, device=dev),
                   x=torch.empty((C, _lib.MLP_IN), dtype=torch.float32, device=dev),
                   U=torch.empty((C, 3, _lib.WS_LPAD, _lib.WS_LPAD), dtype=torch.float32, device=dev),
                   t=torch.empty((C, _lib.MLP_OUT), dtype=torch.float32, device=dev))
        check(self.lib.rcp_batched_export(self.h, out["B"].data_ptr(), out["meta"].data_ptr(),
                                          out["x"].data_ptr(), out["U"].data_ptr(),
                                          out["t"].data_ptr()), "rcp_batched_export")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.rcp_batched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class WarmStartNet:
    """The warm-start network (include/rcp.h, learned warm start) on one CUDA stream."""

    def __init__(self, batch=256, seed=0, stream=None):
        self.lib = _lib.load()
        self.batch = int(batch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        self.nparams = int(self.lib.rcp_mlp_param_count())
        h = ctypes.c_void_p()
        check(self.lib.rcp_mlp_create(self.batch, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
              "rcp_mlp_create")
        self.h = h

    def params(self):
        """(params, adam_m, adam_v, step) as host FP32 tensors (synchronises)."""
        w, m, v = (torch.empty(self.nparams, dtype=torch.float32) for _ in range(3))
        step = ctypes.c_int64()
        check(self.lib.rcp_mlp_get_params(self.h, w.data_ptr(), m.data_ptr(), v.data_ptr(),
                                          ctypes.byref(step)), "rcp_mlp_get_params")
        return w, m, v, step.value

    def set_params(self, w, m=None, v=None, step=0):
        w = w.detach().to("cpu", torch.float32).contiguous()
        m = None if m is None else m.detach().to("cpu", torch.float32).contiguous()
        v = None if v is None else v.detach().to("cpu", torch.float32).contiguous()
        check(self.lib.rcp_mlp_set_params(self.h, w.data_ptr(), None if m is None else m.data_ptr(),
                                          None if v is None else v.data_ptr(), int(step)),
              "rcp_mlp_set_params")

    def save(self, path):
        w, m, v, step = self.params()
        torch.save(dict(params=w, adam_m=m, adam_v=v, step=step), path)

    def load(self, path):
        d = torch.load(path, map_location="cpu")
        self.set_params(d["params"], d["adam_m"], d["adam_v"], d["step"])

    def forward(self, x, train=False):
        count = x.shape[0]
        y = torch.empty((count, _lib.MLP_OUT), dtype=torch.float32, device=self.device)
        check(self.lib.rcp_mlp_forward(self.h, x.data_ptr(), count, 1 if train else 0, y.data_ptr()),
              "rcp_mlp_forward")
        return y

    def backward(self, dy):
        g = torch.empty(self.nparams, dtype=torch.float32, device=self.device)
        check(self.lib.rcp_mlp_backward(self.h, dy.data_ptr(), g.data_ptr()), "rcp_mlp_backward")
        return g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        check(self.lib.rcp_mlp_adam(self.h, lr, beta1, beta2, eps), "rcp_mlp_adam")

    def train_step(self, x, t, meta, lr):
        count = x.shape[0]
        loss = torch.empty(count, dtype=torch.float32, device=self.device)
        check(self.lib.rcp_mlp_train_step(self.h, x.data_ptr(), t.data_ptr(), meta.data_ptr(), count,
                                          lr, loss.data_ptr()), "rcp_mlp_train_step")
        return loss

    def status(self):
        return self.lib.rcp_mlp_status(self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.rcp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ws_canonicalize(Bpad, meta, stream=None):
    """(x rows, canonical bases U) of padded compressed tensors (device tensors)."""
    lib = _lib.load()
    stream = stream if stream is not None else torch.cuda.current_stream()
    C = Bpad.shape[0]
    x = torch.empty((C, _lib.MLP_IN), dtype=torch.float32, device=Bpad.device)
    U = torch.empty((C, 3, _lib.WS_LPAD, _lib.WS_LPAD), dtype=torch.float32, device=Bpad.device)
    check(lib.rcp_ws_canonicalize(Bpad.data_ptr(), meta.data_ptr(), C, x.data_ptr(), U.data_ptr(),
                                  ctypes.c_void_p(stream.cuda_stream)), "rcp_ws_canonicalize")
    return x, U


def ws_loss(y, t, meta, scale=1.0, stream=None):
    """(per-sample loss, dLoss/dY * scale) of the matched-cosine warm-start loss."""
    lib = _lib.load()
    stream = stream if stream is not None else torch.cuda.current_stream()
    C = y.shape[0]
    loss = torch.empty(C, dtype=torch.float32, device=y.device)
    dy = torch.empty_like(y)
    check(lib.rcp_ws_loss(y.data_ptr(), t.data_ptr(), meta.data_ptr(), C, scale, dy.data_ptr(),
                          loss.data_ptr(), ctypes.c_void_p(stream.cuda_stream)), "rcp_ws_loss")
    return loss, dy


def synth_cp(factors, lam, sigma, seed, out=None, stream=None):
    """Device synthetic CP tensor (Kolda layout) from FP32 device factors (I_n x R each)."""
    lib = _lib.load()
    stream = stream if stream is not None else torch.cuda.current_stream()
    dims = [int(F.shape[0]) for F in factors]
    R = int(factors[0].shape[1])
    Fs = [F.t().contiguous() for F in factors]   # column-major I_n x R
    if out is None:
        out = torch.empty(tuple(reversed(dims)), dtype=torch.float32, device=factors[0].device)
    d = (ctypes.c_int64 * len(dims))(*dims)
    check(lib.rcp_synth_cp(len(dims), d, R, _ptr_array(Fs), lam.data_ptr(), float(sigma),
                           int(seed) & 0xFFFFFFFFFFFFFFFF, out.data_ptr(),
                           ctypes.c_void_p(stream.cuda_stream)), "rcp_synth_cp")
    out._keep = Fs
    return out
