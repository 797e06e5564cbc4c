"""Learned dual warm start (GPU, through the C ABI): features and targets,
the tensor-core MLP forward and gradient against a plain PyTorch fp32
reference with the same BF16 operand rounding, training, and warm-started
solves that reach the cold-start optimum (Dykstra/Hildreth, Sec. II-B,
converges to the unique QP solution from any nonnegative dual start)."""
import numpy as np
import pytest

import oracle
from instances import chung_lu, planted_partition

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _solver(n, d, w, **kw):
    import paper_1901_10084_gb300 as cc
    kw.setdefault("interleave", False)
    return cc.Solver(n, d, w, **kw)


def _bf(t):
    torch = _torch()
    return t.to(torch.bfloat16).to(torch.float32)


def _reference_forward(params, feat):
    """Plain fp32 MLP with BF16-rounded weights, inputs and hidden
    activations (the operands the tensor cores see); biases stay fp32."""
    torch = _torch()
    from paper_1901_10084_gb300.warmstart import unpack
    W1, b1, W2, b2, W3, b3 = [torch.tensor(a) for a in unpack(params)]
    x = _bf(feat[:, :10])
    h1 = x @ _bf(W1) + b1
    h2 = _bf(torch.relu(h1)) @ _bf(W2) + b2
    o = _bf(torch.relu(h2)) @ _bf(W3) + b3
    return torch.nn.functional.softplus(o)


def _features_numpy(n, d):
    """Candidates and features in packed (a, b) order, c ascending, from d."""
    D = np.zeros((n, n))
    iu, ju = np.triu_indices(n, 1)
    D[iu, ju] = d
    D = D + D.T
    A = (D == 0.0) & ~np.eye(n, dtype=bool)
    deg = A.sum(1)
    mean = deg.sum() / n
    rows, trip = [], []
    for a, b in zip(iu, ju):
        for c in range(b + 1, n):
            if A[a, b] or A[a, c] or A[b, c]:
                cn = [int(np.sum(A[u] & A[v])) for u, v in ((a, b), (a, c), (b, c))]
                common = int(np.sum(A[a] & A[b] & A[c]))
                rows.append([D[a, b], D[a, c], D[b, c], np.log1p(deg[a] / mean), np.log1p(deg[b] / mean),
                             np.log1p(deg[c] / mean), *np.log1p(cn), np.log1p(common)])
                trip.append((a, b, c))
    return np.array(rows, dtype=np.float64).reshape(-1, 10), trip


@pytest.mark.parametrize("n,tile", [(60, 16), (75, 8)])
def test_features_and_targets_match_a_numpy_recount(n, tile):
    from paper_1901_10084_gb300 import warmstart
    d, w, _ = planted_partition(n, 4, 0.6, 0.1, seed=n)
    ref, trip = _features_numpy(n, d)
    with _solver(n, d, w, tile=tile) as s:
        s.sweep(9)
        feat, targ = warmstart.samples(s)
        yt, _ = s.get_duals()
    feat = feat.cpu().numpy()
    targ = targ.cpu().numpy()
    assert feat.shape[0] == len(trip)
    np.testing.assert_allclose(feat[:, :10], ref, rtol=1e-6, atol=1e-6)
    assert np.all(feat[:, 10:] == 0)
    idx = np.array([oracle.trank(n, a, b, c) for a, b, c in trip])
    expect = yt.reshape(-1, 3)[idx]
    np.testing.assert_allclose(targ, expect, rtol=1e-6, atol=1e-30)


def _sample_features(count, seed):
    rng = np.random.default_rng(seed)
    f = np.zeros((count, 12), dtype=np.float32)
    f[:, :3] = rng.integers(0, 2, (count, 3))
    f[:, 3:6] = rng.uniform(0.1, 2.5, (count, 3))
    f[:, 6:10] = rng.uniform(0.0, 3.0, (count, 4))
    return f


@pytest.mark.parametrize("count", [1, 15, 16, 1000, 4099])
def test_forward_matches_fp32_reference(count):
    torch = _torch()
    from paper_1901_10084_gb300 import warmstart
    params = warmstart.init_params(seed=count, out_bias=0.0)
    feat = torch.tensor(_sample_features(count, count))
    out = warmstart.forward(params, feat.cuda()).cpu()
    ref = _reference_forward(params, feat)
    torch.testing.assert_close(out, ref, rtol=2e-2, atol=2e-3)


def test_forward_of_empty_input():
    torch = _torch()
    from paper_1901_10084_gb300 import warmstart
    out = warmstart.forward(warmstart.init_params(0), torch.zeros((0, 12), device="cuda"))
    assert out.shape == (0, 3)


@pytest.mark.parametrize("count,pos_weight", [(16, 1.0), (333, 1.0), (2048, 1.0), (333, 4.0), (2048, 0.25)])
def test_gradient_matches_fp32_autograd(count, pos_weight):
    """The weighted loss: terms of positive targets (half of them here) count
    pos_weight times, the zero targets once."""
    torch = _torch()
    from paper_1901_10084_gb300 import warmstart
    params = warmstart.init_params(seed=7, out_bias=-0.5)
    feat = torch.tensor(_sample_features(count, 100 + count))
    rng = np.random.default_rng(count)
    t = rng.exponential(0.3, (count, 3)) * (rng.random((count, 3)) < 0.5)
    target = torch.tensor(t.astype(np.float32))
    g, loss = warmstart.grad(params, feat.cuda(), target.cuda(), pos_weight=pos_weight)
    p = torch.tensor(params, requires_grad=True)
    parts, o = [], 0
    for size in (10 * 64, 64, 64 * 64, 64, 64 * 3, 3):
        parts.append(p[o:o + size])
        o += size
    W1, b1, W2, b2, W3, b3 = (parts[0].view(10, 64), parts[1], parts[2].view(64, 64), parts[3],
                              parts[4].view(64, 3), parts[5])
    x = _bf(feat[:, :10])
    h1 = x @ W1 + b1
    h2 = torch.relu(h1) @ W2 + b2
    out = torch.nn.functional.softplus(torch.relu(h2) @ W3 + b3)
    v = torch.where(target > 0, torch.tensor(pos_weight), torch.tensor(1.0))
    ref_loss = (v * (out - target) ** 2).mean()
    ref_loss.backward()
    gref = p.grad.numpy()
    assert abs(loss - ref_loss.item()) <= 2e-2 * ref_loss.item()
    o = 0
    for size in (10 * 64, 64, 64 * 64, 64, 64 * 3, 3):
        a, b = g[o:o + size], gref[o:o + size]
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-7, (o, size)
        o += size


def test_training_lowers_the_loss_on_solver_duals():
    from paper_1901_10084_gb300 import warmstart
    inst = [chung_lu(150, 2.5, 8.0, seed=s)[:2] for s in (11, 12)]
    feat, targ, sweeps = warmstart.collect([(150, d, w) for d, w in inst], tol=1e-4)
    assert all(k > 0 for k in sweeps)
    p0 = warmstart.init_params(3)
    _, l0 = warmstart.grad(p0, feat, targ)
    params, losses = warmstart.train(feat, targ, steps=400, batch=2048, lr=3e-3, seed=3, params=p0)
    _, l1 = warmstart.grad(params, feat, targ)
    assert np.all(np.isfinite(losses))
    assert l1 < 0.5 * l0
    assert losses[-20:].mean() < losses[:20].mean()


def _trained(seed=5):
    from paper_1901_10084_gb300 import warmstart
    inst = [chung_lu(150, 2.5, 8.0, seed=s)[:2] for s in (21, 22)]
    feat, targ, _ = warmstart.collect([(150, d, w) for d, w in inst], tol=1e-4)
    params, _ = warmstart.train(feat, targ, steps=300, batch=2048, lr=3e-3, seed=seed)
    return params


@pytest.mark.parametrize("interleave", [False, True])
def test_warm_started_solve_reaches_the_cold_optimum(interleave):
    params = _trained()
    n = 200
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=40)
    res = {}
    for mode in ("cold", "warm"):
        with _solver(n, d, w, tile=16, interleave=interleave, check_every=5) as s:
            if mode == "warm":
                cand = s.warm_start(params, threshold=1e-3)
                assert cand > 0
                yt, yp = s.get_duals()
                assert yt.min() >= 0.0 and yp.min() >= 0.0   # pair duals from the pair passes
                x, f = s.get_x()
                from oracle.dense import invariant_residual
                assert invariant_residual(n, d, w, 0.2, x, f, yt, yp) <= 1e-12
            ok, k = s.solve(1e-7, 20000)
            assert ok
            res[mode] = (s.check(), s.get_x()[0])
    (c0, x0), (c1, x1) = res["cold"], res["warm"]
    assert abs(c1["lp_objective"] - c0["lp_objective"]) <= 1e-6 * abs(c0["lp_objective"])
    assert np.max(np.abs(x1 - x0)) <= 1e-4


def test_zero_prediction_is_the_cold_start_plus_pair_passes_bitwise():
    """Threshold above every output: all triangle duals 0, so the rebuilt
    state is x0 and the warm start ends with CC_WS_PAIR_PASSES pair passes
    from it; that state and the following sweeps match a fresh solver given
    the same pair passes, bit for bit."""
    from paper_1901_10084_gb300 import _native, warmstart
    n = 90
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=9, weights=(0.5, 2.0))
    params = warmstart.init_params(1)
    with _solver(n, d, w, tile=16) as a, _solver(n, d, w, tile=16) as b:
        a.sweep(4)
        a.warm_start(params, threshold=1e30)
        b.pair_passes(_native.CC_WS_PAIR_PASSES)
        for _ in range(2):
            xa, fa = a.get_x()
            xb, fb = b.get_x()
            assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
            for u, v in zip(a.get_duals(), b.get_duals()):
                assert np.array_equal(u, v)
            a.sweep(3)
            b.sweep(3)
        assert a.stats()["sweeps"] == 6


def test_fp32_bulk_warm_start_is_the_fp64_one_rounded():
    """In the FP32 bulk phase the warm start runs in FP64 and rounds its
    result: x and f are the FP64 warm start's values rounded to FP32, the
    duals within FP32 rounding; the solve then reaches the cold optimum."""
    params = _trained()
    n = 200
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=40)
    with _solver(n, d, w, tile=16) as a, _solver(n, d, w, tile=16, precision="fp32_refine", check_every=5) as b:
        b.sweep(3)                      # a bulk state to overwrite
        ca = a.warm_start(params, threshold=1e-3)
        cb = b.warm_start(params, threshold=1e-3)
        assert ca == cb > 0
        xa, fa = a.get_x()
        xb, fb = b.get_x()
        np.testing.assert_array_equal(xb, xa.astype(np.float32).astype(np.float64))
        np.testing.assert_array_equal(fb, fa.astype(np.float32).astype(np.float64))
        for u, v in zip(b.get_duals(), a.get_duals()):
            np.testing.assert_allclose(u, v, rtol=2e-7, atol=0)
        assert b.stats()["sweeps"] == 0
        ok, k = b.solve(1e-4, 20000)
        assert ok and 0 < b.stats()["fp32_sweeps"] <= k - 5     # the refinement ran in FP64
        # the FP64 warm-started state swept as many times: the FP32 bulk form
        # with its FP64 refinement gives the same objective (1e-6 relative)
        a.sweep(k)
        lp_b, lp_a = b.check()["lp_objective"], a.check()["lp_objective"]
        assert abs(lp_b - lp_a) <= 1e-6 * abs(lp_a)
        assert b.check()["max_violation"] <= 1e-4
        with _solver(n, d, w, tile=16, check_every=5) as c:
            assert c.solve(1e-7, 20000)[0]
            lp = c.check()["lp_objective"]
        assert abs(lp_b - lp) <= 1e-4 * abs(lp)


def test_warm_start_rejects_the_exact_form():
    import paper_1901_10084_gb300 as cc
    from paper_1901_10084_gb300 import warmstart
    n = 40
    d, w, _ = planted_partition(n, 2, 0.7, 0.1, seed=1)
    with _solver(n, d, w, tile=8, exact=True) as s:
        with pytest.raises(cc.CCError) as e:
            s.warm_start(warmstart.init_params(0))
        assert e.value.code == cc.CC_ERR_UNSUPPORTED
