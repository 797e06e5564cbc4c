"""Learned dual warm start (not in the paper): training data, training and
warm-started solves on top of the C ABI's cc_ws_samples / cc_mlp_train /
cc_warm_start_mlp.

The method being warm-started is Dykstra's (Hildreth's) projection method of
Sec. II-B (Algorithm 1): coordinate ascent on the dual of Eq. (qp), which
reaches the same optimum from any nonnegative dual start once the primal
iterate is rebuilt from the duals.  A network 10 -> 64 -> 64 -> 3 maps
features of a triplet with at least one edge to its three duals; its
forward and backward passes and the Adam steps run in the library's
tensor-core kernels.  Device buffers come from PyTorch (plumbing only).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native
from ._native import CC_WS_FEAT, CC_WS_NPARAM

N_IN, N_H, N_OUT = 10, 64, 3


def unpack(params):
    """Split a flat parameter vector into (W1, b1, W2, b2, W3, b3)."""
    p = np.asarray(params, dtype=np.float32)
    o, out = 0, []
    for shape in ((N_IN, N_H), (N_H,), (N_H, N_H), (N_H,), (N_H, N_OUT), (N_OUT,)):
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape))
        o += size
    assert o == CC_WS_NPARAM
    return out


def init_params(seed: int = 0, out_bias: float = -3.0) -> np.ndarray:
    """He-normal weights, zero hidden biases; the output bias starts negative
    so that initial predictions are small (most duals are zero)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / N_IN), (N_IN, N_H)), np.zeros(N_H),
             rng.normal(0, np.sqrt(2.0 / N_H), (N_H, N_H)), np.zeros(N_H),
             rng.normal(0, np.sqrt(1.0 / N_H), (N_H, N_OUT)), np.full(N_OUT, out_bias)]
    return np.concatenate([a.ravel() for a in parts]).astype(np.float32)


def dpattern_constant(feat: torch.Tensor, target: torch.Tensor):
    """Mean training dual of the rows a cold start violates first: the row
    whose hypotenuse is the only non-edge (d = 1) of a triplet whose other
    two pairs are edges (d = 0).  Returns (constant, number of such rows)."""
    dv = feat[:, :3]
    tot, cnt = 0.0, 0
    for r in range(3):
        legs = [q for q in range(3) if q != r]
        m = (dv[:, r] == 1) & (dv[:, legs[0]] == 0) & (dv[:, legs[1]] == 0)
        cnt += int(m.sum())
        tot += float(target[m, r].double().sum())
    return (tot / cnt if cnt else 0.0), cnt


def dpattern_params(c: float, off: float = -12.0) -> np.ndarray:
    """Network parameters that compute the trivial d-pattern predictor on the
    same inference path: hidden unit r = relu(d_r - d_a - d_b), which is 1
    exactly on the pattern of ``dpattern_constant`` for row r (d in {0, 1})
    and 0 otherwise, carried through layer 2 unchanged; output r =
    softplus(a h_r + off) with a chosen so that the pattern gives about c
    (BF16 rounding of a moves it by under 5 %) and the rest softplus(off),
    about 6e-6, which any threshold above it sets to 0."""
    W1, b1, W2, b2, W3, b3 = [np.zeros_like(a) for a in unpack(np.zeros(CC_WS_NPARAM, dtype=np.float32))]
    for r in range(3):
        W1[:, r] = 0.0
        W1[r, r] = 1.0
        for q in range(3):
            if q != r:
                W1[q, r] = -1.0
        W2[r, r] = 1.0
        W3[r, r] = (np.log(np.expm1(c)) - off) if c > 0 else 0.0
    b3[:] = off
    return np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float32)


def samples(solver, device=None):
    """(features, targets) of a solver's current state as device tensors of
    shape (m, CC_WS_FEAT) and (m, 3)."""
    dev = torch.device("cuda", solver_device(solver) if device is None else device)
    m = _native.cc_ws_samples(solver.h)
    feat = torch.empty((max(m, 1), CC_WS_FEAT), dtype=torch.float32, device=dev)
    targ = torch.empty((max(m, 1), 3), dtype=torch.float32, device=dev)
    if m > 0:
        _native.cc_ws_samples(solver.h, feat.data_ptr(), targ.data_ptr(), m)
    return feat[:m], targ[:m]


def solver_device(solver) -> int:
    opts = getattr(solver, "opts", None)
    return int(opts.device) if opts is not None else 0


def collect(instances, eps=0.2, tol=1e-4, max_sweeps=20000, tile=16, device=0):
    """Solve each (n, d, w) instance to `tol` (FP64, tiled schedule) and
    concatenate its training samples; returns (features, targets, sweeps)."""
    from . import Solver
    feats, targs, sweeps = [], [], []
    for n, d, w in instances:
        with Solver(n, d, w, eps=eps, schedule="tiled", tile=tile, device=device, check_every=10) as s:
            ok, k = s.solve(tol, max_sweeps)
            f, t = samples(s, device)
            feats.append(f)
            targs.append(t)
            sweeps.append(k if ok else -1)
    return torch.cat(feats), torch.cat(targs), sweeps


def forward(params, feat: torch.Tensor) -> torch.Tensor:
    """Network outputs (m, 3) for device features (m, CC_WS_FEAT)."""
    feat = feat.contiguous()
    out = torch.empty((feat.shape[0], 3), dtype=torch.float32, device=feat.device)
    if feat.shape[0] > 0:
        _native.cc_mlp_forward(params, feat.data_ptr(), out.data_ptr(), feat.shape[0],
                               torch.cuda.current_stream(feat.device).cuda_stream)
    return out


def grad(params, feat: torch.Tensor, target: torch.Tensor, pos_weight=1.0):
    """Full-batch (gradient, loss) of the mean squared error, the terms of
    positive targets weighted by ``pos_weight``."""
    feat, target = feat.contiguous(), target.contiguous()
    return _native.cc_mlp_grad(params, feat.data_ptr(), target.data_ptr(), feat.shape[0], pos_weight,
                               torch.cuda.current_stream(feat.device).cuda_stream)


def train(feat: torch.Tensor, target: torch.Tensor, steps=2000, batch=4096, lr=3e-3, seed=0, params=None,
          pos_weight=1.0):
    """Adam on minibatches of ``grad``'s loss; returns (params, per-step losses)."""
    feat, target = feat.contiguous(), target.contiguous()
    p0 = init_params(seed) if params is None else params
    return _native.cc_mlp_train(p0, feat.data_ptr(), target.data_ptr(), feat.shape[0], batch, steps, lr, seed,
                                pos_weight, torch.cuda.current_stream(feat.device).cuda_stream)


def collect_batch(instances, eps=0.2, tol=1e-4, max_sweeps=20000, tile=16, device=0, group=256):
    """As ``collect``, solving the instances ``group`` at a time as one
    batch (one launch per sweep for the whole group); returns
    (features, targets, sweeps per instance, -1 where not converged)."""
    from . import Batch
    feats, targs, sweeps = [], [], []
    for g0 in range(0, len(instances), group):
        part = instances[g0:g0 + group]
        with Batch(part, eps=eps, tile=tile, device=device, check_every=10) as b:
            _, _, per = b.solve(tol, max_sweeps)
            for i in range(len(part)):
                f, t = samples(b.instance(i), device)
                feats.append(f)
                targs.append(t)
            sweeps.extend(per)
    return torch.cat(feats), torch.cat(targs), sweeps
