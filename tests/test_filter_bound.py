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


def f32_trunc(x):
    """The kernels' integer double-to-float copy: sign, exponent and the
    leading 23 significand bits; +-0 below 2^-126."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = x.view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    sign = hi & np.uint32(0x80000000)
    e = ((hi >> np.uint32(20)) & np.uint32(0x7FF)).astype(np.int64)
    m = ((hi & np.uint32(0xFFFFF)) << np.uint32(3)) | (lo >> np.uint32(29))
    body = (np.clip(e - 896, 0, 255).astype(np.uint32) << np.uint32(23)) | m
    out = np.where(e < 897, sign, sign | body)
    out = np.where(e > 1150, sign | np.uint32(0x7F800000), out)
    return out.astype(np.uint32).view(np.float32)


def row_inactive(h, a, b):
    d = (h - a) - b
    S = (np.abs(h) + np.abs(a)) + np.abs(b)
    return d <= -_fma32(S, TAU_REL * np.ones_like(S), TAU_ABS * np.ones_like(S))


def test_truncated_copy_error_bound():
    rng = np.random.default_rng(5)
    x = rng.uniform(-2, 2, 400000) * rng.choice([1e-30, 1e-6, 1.0, 1e3, 1e30], 400000)
    f = f32_trunc(x).astype(np.float64)
    assert np.all(np.abs(f - x) < 2.0 ** -23 * np.abs(x))
    assert np.all(np.abs(f) <= np.abs(x)) and np.all(np.sign(f) == np.sign(x))
    tiny = np.array([1e-40, -1e-45, 2.0 ** -127, 0.0, -0.0])
    assert np.all(f32_trunc(tiny) == 0.0)
    exact = np.array([1.0, -0.75, 2.0 ** -126, 3.0 * 2.0 ** 100])     # 23-bit significands stay exact
    assert np.array_equal(f32_trunc(exact).astype(np.float64), exact)


def test_filter_is_sound_with_truncated_copies():
    rng = np.random.default_rng(6)
    for _ in range(20):
        x = _cases(rng, 200000)
        f = f32_trunc(x.ravel()).reshape(x.shape)
        ok = inactive_fast(f[:, 0], f[:, 1], f[:, 2])
        d0 = (x[:, 0] - x[:, 1]) - x[:, 2]
        d1 = (x[:, 1] - x[:, 0]) - x[:, 2]
        d2 = (x[:, 2] - x[:, 0]) - x[:, 1]
        assert np.all(np.maximum(np.maximum(d0, d1), d2)[ok] < 0)
        assert ok.mean() > 0.05


def test_row_filter_is_sound_and_the_skipped_row_is_a_no_op():
    """row_inactive on float copies (truncated or rounded) proves the double
    row delta negative; with a zero dual the fused row update then leaves
    z' = max(fma(delta, 1/3, 0), 0) = 0 and c = 0."""
    rng = np.random.default_rng(7)
    for copy in (f32_trunc, lambda v: v.astype(np.float32)):
        hits = 0
        for _ in range(10):
            x = _cases(rng, 200000)
            f = copy(x.ravel()).reshape(x.shape)
            for h, a, b in ((0, 1, 2), (1, 0, 2), (2, 0, 1)):
                ok = row_inactive(f[:, h], f[:, a], f[:, b])
                d = (x[:, h] - x[:, a]) - x[:, b]
                assert np.all(d[ok] < 0)
                zn = d[ok] * (1.0 / 3.0)        # fma(d, r, 0) = round(d * r): same sign as d
                assert np.all(np.maximum(zn, 0.0) == 0.0)
                hits += ok.sum()
        assert hits > 0


def _check_skips(f, m):
    """The convergence check's skip rule (k_maxviol_tiled): a triplet's rows
    are left out of the FP64 evaluation when RN(dmax_f + tau) <= m_f, with
    dmax_f = RN(2 max - sum) the float estimate of its largest row delta,
    tau = RN(S 2^-19 + 2^-100), m_f = m rounded down to float."""
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    mx = np.maximum(np.maximum(a, b), c)
    dmax = _fma32(np.float32(2.0) * np.ones_like(mx), mx, -((a + b) + c))
    S = (np.abs(a) + np.abs(b)) + np.abs(c)
    tau = _fma32(S, np.float32(2.0 ** -19) * np.ones_like(S), np.float32(2.0 ** -100) * np.ones_like(S))
    mf = m.astype(np.float32)
    mf = np.where(mf.astype(np.float64) > m, np.nextafter(mf, np.float32(-np.inf)), mf)   # round down
    return dmax + tau <= mf


def test_check_skip_rule_never_hides_a_row_above_the_running_maximum():
    """With truncated (or rounded) float copies of double x, a skipped
    triplet's exact double row deltas never exceed the running maximum m:
    the check's maximum equals a serial FP64 evaluation over all rows."""
    rng = np.random.default_rng(11)
    for copy in (f32_trunc, lambda v: v.astype(np.float32)):
        skipped = 0
        for _ in range(10):
            x = _cases(rng, 200000)
            d0 = (x[:, 0] - x[:, 1]) - x[:, 2]
            d1 = (x[:, 1] - x[:, 0]) - x[:, 2]
            d2 = (x[:, 2] - x[:, 0]) - x[:, 1]
            exact = np.maximum(np.maximum(d0, d1), d2)
            # running maxima just above, at and below each triplet's own
            # largest delta, and unrelated ones of other magnitudes
            for m in (exact * (1 + 1e-7), exact, exact * (1 - 1e-7), np.abs(exact) + 1e-9,
                      rng.choice([0.0, 1e-12, 1e-6, 1e-3, 1.0], exact.size)):
                m = np.maximum(m, 0.0)
                f = copy(x.ravel()).reshape(x.shape)
                skip = _check_skips(f, m)
                assert np.all(exact[skip] <= m[skip])
                skipped += int(skip.sum())
        assert skipped > 0
