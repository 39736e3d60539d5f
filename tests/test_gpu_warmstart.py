"""The learned warm start on the GPU against the FP64 oracle (oracle/warmstart.py).

Forward, backward and Adam of the network (BF16 operands, FP32 accumulation)
are compared with the oracle network that rounds the same operands to BF16;
the remaining differences are FP32 accumulation order and the rare BF16
rounding flips it causes, hence relative tolerances of a few 1e-3.  The
canonical basis, the matched loss and the synthetic generator follow FP32
arithmetic and are compared at 1e-4.  The gain test trains the network on
method-generated tensors and compares ALS started from it with ALS started
from random factors on a held-out batch.
"""

import numpy as np
import pytest
import torch

from oracle import warmstart as ows
from oracle import rcp as orcp

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _random_params(rng):
    o = ows.param_offsets()
    p = np.zeros(o[-1])
    p[o[0]:o[1]] = rng.standard_normal(o[1] - o[0]) / np.sqrt(ows.IN)
    p[o[1]:o[2]] = 0.05 * rng.standard_normal(o[2] - o[1])
    p[o[2]:o[3]] = rng.standard_normal(o[3] - o[2]) / np.sqrt(ows.HIDDEN)
    p[o[3]:o[4]] = 0.05 * rng.standard_normal(o[4] - o[3])
    p[o[4]:o[5]] = rng.standard_normal(o[5] - o[4]) / np.sqrt(ows.HIDDEN)
    p[o[5]:o[6]] = 0.05 * rng.standard_normal(o[6] - o[5])
    return p.astype(np.float32)


def test_forward_backward_adam_match_oracle(rcp_lib):
    from paper_1703_09074_gb300 import WarmStartNet
    rng = np.random.default_rng(11)
    net = WarmStartNet(batch=128, seed=1)
    p32 = _random_params(rng)
    net.set_params(torch.from_numpy(p32))
    count = 100
    x = (rng.standard_normal((count, ows.IN)) / np.sqrt(ows.IN) * 4.0).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda(), train=True).cpu().numpy()
    p = p32.astype(np.float64)
    yo, cache = ows.forward(p, x.astype(np.float64))
    assert _rel(y, yo) < 2e-3
    dy = np.zeros((128, ows.OUT), np.float32)
    dy[:count] = rng.standard_normal((count, ows.OUT)).astype(np.float32) / count
    g = net.backward(torch.from_numpy(dy).cuda()).cpu().numpy()
    go = ows.backward(p, cache, dy[:count].astype(np.float64))
    o = ows.param_offsets()
    for k, name in enumerate(["W1", "b1", "W2", "b2", "W3", "b3"]):
        assert _rel(g[o[k]:o[k + 1]], go[o[k]:o[k + 1]]) < 5e-3, name
    net.adam(1e-3)
    w1, m1, v1, step = net.params()
    assert step == 1
    wo, mo, vo = ows.adam(p, np.zeros_like(p), np.zeros_like(p), g.astype(np.float64), 1, 1e-3)
    assert np.max(np.abs(w1.numpy() - wo)) < 1e-6
    # the kernel forms 1 - beta in FP32: |fl(0.999) - 0.999| <= 3e-8 is up to 3e-5
    # of 1 - beta2 (3e-7 of 1 - beta1), the floor of these two comparisons
    assert _rel(m1.numpy(), mo) < 1e-6 and _rel(v1.numpy(), vo) < 5e-5
    assert net.status() == 0
    net.close()


def _cores(rng, count):
    meta = np.zeros((count, 4), np.int32)
    B = np.zeros((count, ows.IN), np.float32)
    for b in range(count):
        if b == 3:
            continue  # a row the network does not serve
        R = int(rng.integers(3, 17))
        l = [min(24, R + int(rng.integers(0, 9))) for _ in range(3)]
        cube = np.zeros((24, 24, 24))
        cube[:l[0], :l[1], :l[2]] = rng.standard_normal(l) * rng.uniform(0.1, 10)
        B[b] = cube.transpose(2, 1, 0).ravel()
        meta[b] = [l[0], l[1], l[2], R]
    return B, meta


def test_canonicalize_matches_oracle(rcp_lib):
    from paper_1703_09074_gb300 import ws_canonicalize
    rng = np.random.default_rng(12)
    B, meta = _cores(rng, 40)
    x, U = ws_canonicalize(torch.from_numpy(B).cuda(), torch.from_numpy(meta).cuda())
    x, U = x.cpu().numpy(), U.cpu().numpy()
    xo, Uo = ows.canonicalize(B.astype(np.float64), meta)
    assert np.max(np.abs(U - Uo)) < 1e-4
    assert np.max(np.abs(x - xo)) < 1e-4 * np.max(np.abs(xo))
    assert np.all(x[3] == 0)


def test_matched_loss_matches_oracle(rcp_lib):
    from paper_1703_09074_gb300 import ws_loss
    rng = np.random.default_rng(13)
    count = 48
    y = (0.3 * rng.standard_normal((count, ows.OUT))).astype(np.float32)
    t = np.zeros((count, ows.OUT), np.float32)
    meta = np.zeros((count, 4), np.int32)
    for b in range(count):
        R = int(rng.integers(1, 17))
        l = [min(24, R + int(rng.integers(0, 9))) for _ in range(3)]
        T = np.zeros((3, 24, 16))
        for n in range(3):
            M = rng.standard_normal((l[n], R))
            T[n, :l[n], :R] = M / np.linalg.norm(M, axis=0)
        t[b] = T.ravel()
        meta[b] = [l[0], l[1], l[2], R]
    lo, dyo = ows.loss(y.astype(np.float64), t.astype(np.float64), meta, scale=0.5)
    loss, dy = ws_loss(torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(),
                       torch.from_numpy(meta).cuda(), scale=0.5)
    assert np.max(np.abs(loss.cpu().numpy() - lo)) < 1e-5
    assert _rel(dy.cpu().numpy(), dyo) < 1e-4


def test_synth_cp_is_the_cp_formula(rcp_lib):
    from paper_1703_09074_gb300 import synth_cp
    rng = np.random.default_rng(14)
    dims, R = (7, 5, 3), 2
    F = [rng.standard_normal((I, R)).astype(np.float32) for I in dims]
    lam = np.array([1.5, -0.5], np.float32)
    X = synth_cp([torch.from_numpy(f).cuda() for f in F], torch.from_numpy(lam).cuda(), 0.0, 1)
    ref = np.einsum("r,ir,jr,kr->ijk", lam.astype(np.float64), *[f.astype(np.float64) for f in F])
    assert np.allclose(X.cpu().numpy().T, ref, rtol=1e-5, atol=1e-5)
    # noise: zero-mean, standard deviation sigma
    Z = synth_cp([torch.zeros((I, 1), device="cuda") for I in (100, 100, 100)],
                 torch.ones(1, device="cuda"), 2.0, 7).double()
    assert abs(Z.mean().item()) < 0.01 and abs(Z.std().item() / 2.0 - 1.0) < 0.005


def test_export_and_eigenvector_warm_start(rcp_lib):
    """Zero network output = eigenvector init; its ALS agrees with the oracle's ALS."""
    from paper_1703_09074_gb300 import WarmStartNet
    from paper_1703_09074_gb300 import warmstart as W
    dev = torch.device("cuda")
    probs = W.draw_problems(12, seed=5, lo=32, hi=64)
    Xs = W.make_tensors(probs, dev)
    from paper_1703_09074_gb300 import BatchedPlan
    bp = BatchedPlan(W.plan_configs(probs))
    bp.run(Xs)
    ex = bp.export()
    meta = ex["meta"].cpu().numpy()
    assert np.all(meta[:, 3] == [p["rank"] for p in probs])
    xo, Uo = ows.canonicalize(ex["B"].cpu().numpy().astype(np.float64), meta)
    assert np.max(np.abs(ex["x"].cpu().numpy() - xo)) < 1e-4 * np.max(np.abs(xo))
    T = ex["t"].cpu().numpy().reshape(-1, 3, 24, 16)
    for b, m in enumerate(meta):
        for n in range(3):
            nrm = np.linalg.norm(T[b, n, :m[n], :m[3]], axis=0)
            assert np.allclose(nrm, 1.0, atol=1e-5)
    net = WarmStartNet(batch=128, seed=2)   # untrained: zero last layer
    bp.set_warm_start(net)
    bp.run(Xs)
    for b, m in enumerate(meta):
        _, _, res = bp.result(b)
        assert res["info"] & 4
        l1, l2, l3, R = (int(v) for v in m)
        cube = ex["B"][b].cpu().numpy().astype(np.float64).reshape(24, 24, 24).transpose(2, 1, 0)
        Bm = cube[:l1, :l2, :l3]
        U = ex["U"][b].cpu().numpy().astype(np.float64)
        init = [None, U[1, :l2, :R], U[2, :l3, :R]]
        _, _, rho, it, _ = orcp.cp_als(Bm, R, 1e-10, 50, 0, init=init)
        if it < 50 and res["iters"] < 50:
            assert abs(res["fit"] - rho) < 1e-3, (b, res["fit"], rho)
    bp.set_warm_start(None)
    bp.run(Xs)
    assert all(not (bp.result(b)[2]["info"] & 4) for b in range(len(probs)))
    bp.close()
    net.close()


def test_training_lowers_the_loss(rcp_lib):
    from paper_1703_09074_gb300 import WarmStartNet
    from paper_1703_09074_gb300 import warmstart as W
    dev = torch.device("cuda")
    data = W.generate(512, seed=21, device=dev)
    net = WarmStartNet(batch=128, seed=3)
    hist, _ = W.train(net, data, epochs=6, lr=1e-3)
    assert hist[-1]["train_loss"] < hist[0]["train_loss"]
    assert net.status() == 0
    net.close()


@pytest.mark.slow
def test_learned_warm_start_gain(rcp_lib):
    """Held-out batch: fit within fixed ALS sweep budgets, trained network vs random init.

    The mixed-precision ALS cannot resolve the 1e-10 fit-change tolerance (its fit
    carries FP32 rounding of about 1e-7), so both arms run to the sweep cap; the
    gain is measured as the mean fit reached within 5, 10, 20 and 50 sweeps.
    """
    from paper_1703_09074_gb300 import WarmStartNet
    from paper_1703_09074_gb300 import warmstart as W
    dev = torch.device("cuda")
    data = W.generate(4096, seed=31, device=dev)
    net = WarmStartNet(batch=256, seed=4)
    val = W.Evaluator(256, seed=32, device=dev, budgets=(10,))
    hist, best_epoch = W.train(net, data, epochs=8, lr=3e-4, evaluator=val)
    val.close()
    budgets = (5, 10, 20, 50)
    test = W.Evaluator(256, seed=33, device=dev, budgets=budgets)
    lines = [f"warm-start gain (best epoch {best_epoch}):"]
    for k in budgets:
        rnd = test.run(None, k)
        lrn = test.run(net, k)
        lines.append(f"  {k:2d} sweeps: mean fit random {rnd['fit'].mean():.6f} learned "
                     f"{lrn['fit'].mean():.6f}; mean rel err random {rnd['rel_err'].mean():.5f} "
                     f"learned {lrn['rel_err'].mean():.5f}")
        assert lrn["learned"].mean() > 0.95 and not rnd["learned"].any()
        assert lrn["fit"].mean() >= rnd["fit"].mean() - 1e-4, k
    test.close()
    print("\n" + "\n".join(lines))
    net.close()


@pytest.mark.slow
def test_trained_network_against_its_untrained_start(rcp_lib):
    """Held-out batch: the trained network against the untrained one (epoch 0, whose
    zero last layer gives the eigenvector initialisation of Algorithm 2 step 2).

    Training targets are the factors ALS reaches after 10 sweeps from that very
    start.  What holds, and is asserted: model selection keeps an epoch whose
    validation fit within 5 sweeps is at least epoch 0's, and on a held-out batch
    the kept network stays within 3e-3 of the untrained start's mean fit within 5
    and within 10 sweeps.  Training has not been found to beat the untrained start
    on held-out data by more than noise (the measured gains are printed): once the
    matched loss leaves its initial plateau the validation fit falls, for every
    learning rate and target tried, so the kept epoch is an early one."""
    from paper_1703_09074_gb300 import WarmStartNet
    from paper_1703_09074_gb300 import warmstart as W
    dev = torch.device("cuda")
    data = W.generate(8192, seed=41, device=dev, target_sweeps=10)
    net = WarmStartNet(batch=256, seed=5)
    val = W.Evaluator(256, seed=42, device=dev, budgets=(5,))
    hist, best_epoch = W.train(net, data, epochs=4, lr=1e-4, evaluator=val)
    val.close()
    vals = [h["val_fit"] for h in hist]
    assert vals[best_epoch] >= vals[0]
    untrained = WarmStartNet(batch=256, seed=5)
    test = W.Evaluator(256, seed=43, device=dev, budgets=(5, 10))
    lines = [f"trained vs untrained network (best epoch {best_epoch}, "
             f"validation fit by epoch {[round(v, 6) for v in vals]}):"]
    for k in (5, 10):
        e0 = test.run(untrained, k)
        tr = test.run(net, k)
        gain = tr["fit"].mean() - e0["fit"].mean()
        lines.append(f"  {k:2d} sweeps: mean fit untrained {e0['fit'].mean():.6f} trained "
                     f"{tr['fit'].mean():.6f} (gain {gain:+.6f})")
        assert tr["learned"].mean() > 0.95 and e0["learned"].mean() > 0.95
        assert gain > -3e-3, (k, gain)
    test.close()
    print("\n" + "\n".join(lines))
    untrained.close()
    net.close()
