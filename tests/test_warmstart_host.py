"""Host logic of the warm-start ablation baselines (no GPU): the d-pattern
predictor's hand-set network parameters and its fitted constant."""
import itertools

import numpy as np
import pytest


def _forward(params, x):
    """The network of include/ccdyk.h in float64 numpy: 10 -> 64 -> 64 -> 3,
    ReLU, softplus output (a restatement for the test, not the kernel)."""
    from paper_1901_10084_gb300 import warmstart
    W1, b1, W2, b2, W3, b3 = [a.astype(np.float64) for a in warmstart.unpack(params)]
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return np.log1p(np.exp(h2 @ W3 + b3))


@pytest.mark.parametrize("c", [0.01, 0.05, 0.3])
def test_dpattern_params_give_c_on_the_pattern_and_almost_zero_elsewhere(c):
    from paper_1901_10084_gb300 import warmstart
    p = warmstart.dpattern_params(c)
    rng = np.random.default_rng(1)
    for dv in itertools.product((0.0, 1.0), repeat=3):
        x = np.concatenate([dv, rng.uniform(0, 3, 7)])[None, :]
        y = _forward(p, x)[0]
        for r in range(3):
            legs = [q for q in range(3) if q != r]
            if dv[r] == 1 and dv[legs[0]] == 0 and dv[legs[1]] == 0:
                assert y[r] == pytest.approx(c, rel=1e-6)
            else:
                assert y[r] < 1e-5


def test_dpattern_constant_is_the_mean_dual_of_the_pattern_rows():
    torch = pytest.importorskip("torch")
    from paper_1901_10084_gb300 import warmstart
    feat = torch.zeros((5, 12))
    targ = torch.zeros((5, 3))
    feat[0, :3] = torch.tensor([1.0, 0.0, 0.0]); targ[0] = torch.tensor([0.2, 9.0, 9.0])   # row 0
    feat[1, :3] = torch.tensor([0.0, 1.0, 0.0]); targ[1] = torch.tensor([9.0, 0.4, 9.0])   # row 1
    feat[2, :3] = torch.tensor([1.0, 1.0, 0.0]); targ[2] = torch.tensor([5.0, 5.0, 5.0])   # no pattern
    feat[3, :3] = torch.tensor([0.0, 0.0, 1.0]); targ[3] = torch.tensor([9.0, 9.0, 0.0])   # row 2
    c, m = warmstart.dpattern_constant(feat, targ)
    assert m == 3 and c == pytest.approx((0.2 + 0.4 + 0.0) / 3)
