"""Training and evaluation of the learned ALS warm start (the network of include/rcp.h).

Training data come from the method itself: synthetic CP tensors are generated
on the device (``synth_cp``), decomposed by the batched path from random ALS
initialisations, and exported as (canonical input x, converged factors in the
canonical basis t, meta) rows.  The network is trained by its own CUDA kernels
(forward, matched-cosine loss, backward, Adam); the epoch kept is the one whose
warm start reaches the highest mean fit within a fixed ALS sweep budget on a
held-out validation batch, run through the same batched path (epoch 0 is the
untrained network, whose zero last layer reproduces the eigenvector
initialisation).  A budget, not a count of sweeps to convergence, is the
yardstick because the mixed-precision ALS evaluates the fit from FP32
MTTKRP partial sums, whose rounding (about 1e-7 relative) sits above the
1e-10 fit-change tolerance: most of those runs stop at the sweep cap.  Random initialisation
stays available as the fallback and as the yardstick.

Tensor distribution (the batched workload): 3-way FP32, I_n ~ U{32..256},
R ~ U{3..16}, factor columns N(0, 1) mixed to pairwise congruence
c ~ U[0, 0.6], lambda_r = 1, Gaussian noise at SNR ~ U[10, 30] dB (noise
variance from the exact signal norm), p = 8, q = 1, ALS tolerance 1e-10,
at most 50 sweeps.
"""

import numpy as np
import torch

from .api import BatchedPlan, synth_cp


def draw_problems(count, seed, lo=32, hi=256, rlo=3, rhi=16):
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 77]))
    out = []
    for b in range(count):
        out.append(dict(dims=tuple(int(v) for v in rng.integers(lo, hi + 1, 3)),
                        rank=int(rng.integers(rlo, rhi + 1)),
                        congruence=float(rng.uniform(0.0, 0.6)),
                        snr_db=float(rng.uniform(10.0, 30.0)),
                        seed=int(seed) * 1000003 + b))
    return out


def make_tensors(problems, device):
    """Device tensors (Kolda layout, FP32) of the problems, generated on the GPU."""
    Xs = []
    for pr in problems:
        rng = np.random.default_rng(np.random.SeedSequence([pr["seed"], 78]))
        R, c = pr["rank"], pr["congruence"]
        C = (1.0 - c) * np.eye(R) + c * np.ones((R, R))
        Lc = np.linalg.cholesky(C)
        Fs = [rng.standard_normal((I, R)) @ Lc.T for I in pr["dims"]]
        # |S|^2 = sum_rs prod_n (A_n^T A_n)_rs for unit weights
        G = np.ones((R, R))
        for F in Fs:
            G = G * (F.T @ F)
        numel = int(np.prod(pr["dims"]))
        sigma = np.sqrt(G.sum() / numel * 10.0 ** (-pr["snr_db"] / 10.0))
        fac = [torch.from_numpy(F.astype(np.float32)).to(device) for F in Fs]
        lam = torch.ones(R, dtype=torch.float32, device=device)
        Xs.append(synth_cp(fac, lam, sigma, pr["seed"]))
    return Xs


def plan_configs(problems, p=8, q=1, tol=1e-10, max_iters=50):
    return [dict(dims=pr["dims"], rank=pr["rank"], oversample=p, power_iters=q, tol=tol,
                 max_iters=max_iters, seed=pr["seed"]) for pr in problems]


def generate(count, seed, device, chunk=256, target_sweeps=None):
    """Training rows (x, t, meta) of ``count`` method-generated tensors (eligible rows only).

    target_sweeps=None: the targets are the factors ALS converges to from random
    initial factors (at most 50 sweeps).  target_sweeps=k: the targets are the
    factors ALS reaches after exactly k sweeps from the eigenvector start (the
    untrained network), i.e. points further along the trajectory that the warm
    start itself begins; a network that predicts them lets ALS start k sweeps
    ahead on that trajectory.
    """
    from .api import WarmStartNet
    xs, ts, ms = [], [], []
    done = 0
    k = 0
    eig_net = None
    if target_sweeps is not None:
        eig_net = WarmStartNet(batch=((chunk + 127) // 128) * 128, seed=0,
                               stream=torch.cuda.current_stream(device))
    while done < count:
        n = min(chunk, count - done)
        probs = draw_problems(n, seed * 7919 + k)
        Xs = make_tensors(probs, device)
        if target_sweeps is None:
            cfgs = plan_configs(probs)
        else:
            cfgs = plan_configs(probs, tol=0.0, max_iters=int(target_sweeps))
        bp = BatchedPlan(cfgs, stream=torch.cuda.current_stream(device))
        if eig_net is not None:
            bp.set_warm_start(eig_net)
        bp.run(Xs)
        ex = bp.export()
        keep = ex["meta"][:, 3] > 0
        xs.append(ex["x"][keep].clone())
        ts.append(ex["t"][keep].clone())
        ms.append(ex["meta"][keep].clone())
        torch.cuda.synchronize(device)
        bp.close()
        del Xs, ex
        done += n
        k += 1
    if eig_net is not None:
        eig_net.close()
    return dict(x=torch.cat(xs), t=torch.cat(ts), meta=torch.cat(ms))


class Evaluator:
    """A held-out batch decomposed with random and with learned initial factors.

    One plan per ALS sweep budget (max_iters); ``run(net, budget)`` returns the
    per-tensor sweeps, fits and relative errors of that budget's plan.
    """

    def __init__(self, count, seed, device, budgets=(10,)):
        self.probs = draw_problems(count, seed)
        self.Xs = make_tensors(self.probs, device)
        st = torch.cuda.current_stream(device)
        self.plans = {int(k): BatchedPlan(plan_configs(self.probs, max_iters=int(k)), stream=st)
                      for k in budgets}
        self.budgets = tuple(int(k) for k in budgets)

    def run(self, net, budget=None):
        bp = self.plans[self.budgets[0] if budget is None else int(budget)]
        bp.set_warm_start(net)
        bp.run(self.Xs)
        res = [bp.result(b)[2] for b in range(len(self.probs))]
        return dict(iters=np.array([r["iters"] for r in res]),
                    fit=np.array([r["fit"] for r in res]),
                    rel_err=np.array([r["rel_err"] for r in res]),
                    learned=np.array([(r["info"] & 4) != 0 for r in res]))

    def close(self):
        for bp in self.plans.values():
            bp.close()


def train(net, data, epochs, lr, evaluator=None, seed=0, log=None):
    """Mini-batch training; keeps the epoch whose warm start gives the highest mean
    fit within the evaluator's first sweep budget (epoch 0: the untrained network)."""
    n = data["x"].shape[0]
    bs = net.batch
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    best = None
    if evaluator is not None:
        ev = evaluator.run(net)
        best = (float(ev["fit"].mean()), 0, net.params())
        hist.append(dict(epoch=0, val_fit=best[0]))
    for ep in range(1, epochs + 1):
        perm = torch.randperm(n, generator=gen).to(data["x"].device)
        tot, steps = 0.0, 0
        for k in range(0, n - bs + 1, bs):
            idx = perm[k:k + bs]
            loss = net.train_step(data["x"][idx].contiguous(), data["t"][idx].contiguous(),
                                  data["meta"][idx].contiguous(), lr)
            tot += float(loss.mean())
            steps += 1
        rec = dict(epoch=ep, train_loss=tot / max(steps, 1))
        if evaluator is not None:
            ev = evaluator.run(net)
            rec["val_fit"] = float(ev["fit"].mean())
            if rec["val_fit"] > best[0]:
                best = (rec["val_fit"], ep, net.params())
        hist.append(rec)
        if log:
            log(rec)
    if best is not None:
        w, m, v, step = best[2]
        net.set_params(w, m, v, step)
    return hist, (best[1] if best else epochs)
