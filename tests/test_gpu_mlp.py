"""The block-rank predictor (hodlr_mlp_*) through the C ABI: forward, backward
and Adam against the oracle (oracle/mlp.py, fp64 on the same fp16
parameters); training on the blocks of GPU-built matrices of the LU, headline
and batched workloads (plus the large-n kernel at small n) lowers the loss;
and on held-out builds the predicted first sketches redo fewer blocks than
the default first sketch of 16 while the construction still meets its
accuracy (the adaptive rule decides every rank)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_21637_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def _rand(seed, S):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((S, OM.N_IN)).astype(np.float32)
    t = rng.standard_normal(S).astype(np.float32)
    return X, t


def test_forward_and_backward_match_the_oracle():
    from paper_2407_21637_gb300 import RankPredictor
    p = OM.round_params(OM.init_params(7))
    rp = RankPredictor(p)
    X, t = _rand(8, 300)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = rp.forward(Xd).cpu().numpy().astype(np.float64)
    yo, _ = OM.forward(p, X.astype(np.float64))
    assert np.all(np.abs(y - yo) <= 1e-4 * (1 + np.abs(yo)))
    loss, grad = rp.gradient(Xd, td)
    go = OM.backward(p, X.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss.item()) - OM.loss(p, X.astype(np.float64), t.astype(np.float64))) <= 1e-4 * (1 + abs(OM.loss(p, X, t)))
    g = grad.cpu().numpy().astype(np.float64)
    for a, b in zip(OM.unpack(g), OM.unpack(go)):   # layer by layer
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-7


def test_adam_step_matches_the_oracle():
    from paper_2407_21637_gb300 import RankPredictor
    p = OM.round_params(OM.init_params(9)).astype(np.float32).astype(np.float64)
    rp = RankPredictor(p)
    X, t = _rand(10, 64)
    _loss, grad = rp.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    g = grad.cpu().numpy().astype(np.float64)
    w, m, v = p.copy(), np.zeros_like(p), np.zeros_like(p)
    for step in (1, 2):
        rp.adam(grad, 1e-3)
        w, m, v = OM.adam_step(w, m, v, g, step, 1e-3)
    assert np.all(np.abs(rp.w32.cpu().numpy() - w) <= 1e-6 * (1 + np.abs(w)))
    assert np.array_equal(rp.w16.float().cpu().numpy(), rp.w32.half().float().cpu().numpy())


def _workloads():
    """(kind, n, depth, eps, c, len2, diag) of the training builds: the LU
    workload, the headline Gaussian at a smaller n, batched-workload draws
    and the large-n kernel at small n."""
    rng = np.random.default_rng(3)
    w = [(0, 1024, 4, 1e-8, 1e-3, 1.0, 1024.0), (1, 16384, 6, 1e-6, 0.0, 0.01, 1e-2),
         (0, 4096, 4, 1e-6, 1e-4, 1.0, 0.0), (0, 8192, 5, 1e-6, 1e-4, 1.0, 0.0)]
    for _ in range(6):
        n = int(round(math.exp(rng.uniform(math.log(2048), math.log(16384)))))
        depth = max(1, math.ceil(math.log2(n / 128)))
        eps = float(math.exp(rng.uniform(math.log(1e-10), math.log(1e-3))))
        if rng.uniform() < 0.5:
            w.append((0, n, depth, eps, 1e-3, 1.0, float(n)))
        else:
            ell = float(rng.uniform(0.02, 0.2))
            w.append((1, n, depth, eps, 0.0, ell * ell, 1e-2))
    return w


def _dataset(rp, wls, seed0=0):
    from paper_2407_21637_gb300 import HodlrMatrix
    Xs, ts = [], []
    for i, (kind, n, depth, eps, c, len2, diag) in enumerate(wls):
        pts = torch.from_numpy(synth.uniform_points_1d(n, seed0 + i)).cuda()
        g = HodlrMatrix.build(pts, kind, depth, eps, c=c, len2=len2, diag=diag, work="fp32", per_block=True,
                              seed=i, allow_short=True)
        _tiers, ranks = g.block_tiers()
        Xs.append(rp.features(pts, kind, depth, eps, c=c, len2=len2, diag=diag))
        ts.append(torch.tensor(np.log2(np.asarray(ranks, dtype=np.float64) + 1.0), dtype=torch.float32))
        g.close()
    return torch.cat(Xs), torch.cat(ts).cuda()


def test_training_lowers_the_loss_and_the_sketches_save_rounds():
    from paper_2407_21637_gb300 import HodlrMatrix, RankPredictor, dense_kernel_matvec
    rp = RankPredictor(seed=1)
    X, t = _dataset(rp, _workloads())
    losses = rp.train(X, t, epochs=400, lr=3e-3)
    assert losses[-1] < 0.25 * losses[0] and losses[-1] < 0.5, (losses[0], losses[-1])
    # held out: the large-n kernel at n = 2^16 (depth 8) and batched-workload
    # draws with small eps (ranks above the default first sketch of 16)
    held = [(0, 65536, 8, 1e-6, 1e-4, 1.0, 0.0), (1, 12000, 7, 1e-10, 0.0, 0.1 ** 2, 1e-2),
            (0, 8192, 6, 1e-10, 1e-3, 1.0, 8192.0), (1, 6000, 6, 1e-9, 0.0, 0.15 ** 2, 1e-2)]
    tot0 = tot1 = 0
    for i, (kind, n, depth, eps, c, len2, diag) in enumerate(held):
        pts = torch.from_numpy(synth.uniform_points_1d(n, 500 + i)).cuda()
        feat = rp.features(pts, kind, depth, eps, c=c, len2=len2, diag=diag)
        sk = RankPredictor.sketch_sizes(rp.forward(feat))
        g0 = HodlrMatrix.build(pts, kind, depth, eps, c=c, len2=len2, diag=diag, work="fp32", per_block=True, seed=9,
                               allow_short=True)
        g1 = HodlrMatrix.build(pts, kind, depth, eps, c=c, len2=len2, diag=diag, work="fp32", per_block=True, seed=9,
                               node_sketch=sk, allow_short=True)
        r0, red0, _c0 = g0.build_stats()
        r1, red1, _c1 = g1.build_stats()
        # the prediction only raises first sketches: never more rounds or redone blocks
        assert red1 <= red0 and r1 <= r0, ((r0, red0), (r1, red1))
        tot0 += red0
        tot1 += red1
        # the predicted build is as accurate: 512 sampled rows against the dense
        # FP64 product, within the Thm 3.1 factor plus fp32 rounding, or no
        # worse than the default build (a block whose rank the sketch cap limits)
        X1 = torch.randn(n, 1, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
        rows = torch.from_numpy(np.sort(np.random.default_rng(7).choice(n, 512, replace=False)).astype(np.int32)).cuda()
        ref = dense_kernel_matvec(pts, kind, X1.double(), c=c, len2=len2, diag=diag, rows=rows)
        errs = [float(torch.linalg.norm(g.matvec(X1).double()[rows.long()] - ref) / torch.linalg.norm(ref))
                for g in (g0, g1)]
        assert errs[1] <= max((2 * math.sqrt(2 * depth) + 1) * eps + 1e-6, 1.5 * errs[0]), errs
        g0.close()
        g1.close()
    assert tot0 > 0 and tot1 < tot0, (tot0, tot1)   # the default redoes blocks, the prediction fewer
