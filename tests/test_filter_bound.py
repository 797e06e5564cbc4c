"""The float pre-filter of the fused sweep must be sound: whenever it
declares a triplet inactive, every row delta evaluated the way the fused
update evaluates it ((x_h - x_a) - x_b, in double for FP64 state and in float
for FP32 state) is negative.  Checked here with IEEE float32/float64
arithmetic from numpy on adversarial inputs (near-tight triangles, mixed
magnitudes, subnormals); the GPU tests exercise the kernel itself."""
import numpy as np

TAU_REL = np.float32(2.0 ** -20)
TAU_ABS = np.float32(2.0 ** -100)


def _fma32(a, b, c):
    # a*b + c rounded once to float32 (exact in double for these operands)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def inactive_fast(a, b, c):
    s = (a + b) + c
    mx = np.maximum(np.maximum(a, b), c)
    dmax = _fma32(np.float32(2.0) * np.ones_like(mx), mx, -s)
    S = (np.abs(a) + np.abs(b)) + np.abs(c)
    return dmax <= -_fma32(S, TAU_REL * np.ones_like(S), TAU_ABS * np.ones_like(S))


def _cases(rng, m):
    base = rng.uniform(0, 1.5, (m, 3))
    xij = base[:, 1] + base[:, 2]                       # x_ij = x_ik + x_jk: a tight row
    eps = rng.choice([0.0, 1e-16, 1e-12, 1e-9, 1e-8, 1e-7, 3e-7, 1e-6, 1e-5, 1e-3], m)
    sign = rng.choice([-1.0, 1.0], m)
    x = np.stack([xij + sign * eps * rng.uniform(0.5, 2, m), base[:, 1], base[:, 2]], 1)
    perm = rng.permuted(np.tile([0, 1, 2], (m, 1)), axis=1)   # tight row in any position
    x = np.take_along_axis(x, perm, 1)
    scale = rng.choice([1e-30, 1e-6, 1.0, 1e3], (m, 1))
    return x * scale


def test_filter_is_sound_for_fp64_state():
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = _cases(rng, 200000)
        f = x.astype(np.float32)
        ok = inactive_fast(f[:, 0], f[:, 1], f[:, 2])
        d0 = (x[:, 0] - x[:, 1]) - x[:, 2]
        d1 = (x[:, 1] - x[:, 0]) - x[:, 2]
        d2 = (x[:, 2] - x[:, 0]) - x[:, 1]
        assert np.all(np.maximum(np.maximum(d0, d1), d2)[ok] < 0)
        assert ok.mean() > 0.05         # the near-tight cases are built to be hard


def test_filter_accepts_clearly_satisfied_triangles():
    rng = np.random.default_rng(2)
    x = rng.uniform(0.5, 1.0, (100000, 3))     # every row delta <= 1 - 0.5 - 0.5 = 0, mostly << 0
    x[:, 0] = np.minimum(x[:, 0], x[:, 1] + x[:, 2] - 1e-3)
    f = x.astype(np.float32)
    assert inactive_fast(f[:, 0], f[:, 1], f[:, 2]).all()


def test_filter_is_sound_for_fp32_state():
    rng = np.random.default_rng(1)
    for _ in range(20):
        f = _cases(rng, 200000).astype(np.float32)
        ok = inactive_fast(f[:, 0], f[:, 1], f[:, 2])
        d0 = (f[:, 0] - f[:, 1]) - f[:, 2]
        d1 = (f[:, 1] - f[:, 0]) - f[:, 2]
        d2 = (f[:, 2] - f[:, 0]) - f[:, 1]
        assert np.all(np.maximum(np.maximum(d0, d1), d2)[ok] < 0)
