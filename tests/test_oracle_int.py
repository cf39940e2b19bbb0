"""Pins for the oracle's integer path (the paper's own data type, Sec. 5: int32
re/im pairs) and for the compensated f of Sec. 3.2."""
from fractions import Fraction

import numpy as np

from paper_1503_00638_gb300 import synth

I32_MAX, I32_MIN = 2 ** 31 - 1, -2 ** 31


def exact_round_int(x, k):
    """Nearest multiple of 2^k to the integer x, ties to even; the lower
    multiple when the nearest one is above INT32_MAX (reading R17)."""
    if k <= 0:
        return x
    g = 2 ** k
    m = round(Fraction(x, g))                  # banker's rounding
    y = m * g
    if y > I32_MAX:
        y -= g
    return y


def test_round_int_exact(orc):
    rng = np.random.default_rng(0)
    xs = list(rng.integers(I32_MIN, I32_MAX, size=3000, endpoint=True))
    xs += [0, 1, -1, 2, -2, 3, -3, I32_MAX, I32_MIN, I32_MAX - 1, I32_MIN + 1, 2 ** 30, -2 ** 30]
    for x in xs:
        for k in (-3, 0, 1, 2, 3, 7, 16, 30, 31, 32, 40, 63, 70):
            assert orc.round_int(int(x), k) == exact_round_int(int(x), k), (x, k)


def test_round_int_ties_and_overflow(orc):
    assert [orc.round_int(v, 1) for v in (1, 3, 5, -1, -3, -5)] == [0, 4, 4, 0, -4, -4]
    assert orc.round_int(I32_MAX, 4) == I32_MAX - 15      # 2^31 is not an int32
    assert orc.round_int(I32_MIN, 4) == I32_MIN
    assert orc.round_int(I32_MIN, 31) == I32_MIN


def int_cube(cfg, scale):
    v = synth.visibilities(cfg)
    a = np.stack([np.rint(v.real * scale), np.rint(v.imag * scale)], axis=-1)
    return a.astype(np.int32)


def test_int_cube_bounds_and_unity_granularity(orc):
    cfg = synth.VisConfig(4, 8, 32, 2 ** 10, 0.01, seed=2)
    for scale in (1.0, 2 ** 10, 2 ** 16):
        a = int_cube(cfg, scale)
        r = orc.reduce_precision(a, cfg.n_samp, cfg.f)
        d = (r.astype(np.int64) - a.astype(np.int64))
        # autos imaginary parts untouched, nothing moves by more than half a granularity
        pii = [synth.auto_product_index(i, 8) for i in range(8)]
        assert np.array_equal(r[:, pii, :, 1], a[:, pii, :, 1])
        A = a[:, pii, :, 0].astype(np.float64)
        assert np.all(np.abs(d) <= np.max(A) * np.sqrt(12 * cfg.f / cfg.n_samp))
        if scale == 1.0:
            # granularity below unity everywhere: integers stay as they are (Sec. 5.1)
            assert np.array_equal(r, a)


def test_int_path_equals_float_path_on_exact_values(orc):
    """Integers below 2^24 are exact float32 values, and a multiple of 2^k for
    k <= 0: the integer and the float rounding must then agree exactly."""
    cfg = synth.VisConfig(3, 6, 32, 2 ** 12, 0.05, seed=4)
    a = int_cube(cfg, 2 ** 12)
    assert np.max(np.abs(a)) < 2 ** 24
    f32 = (a[..., 0].astype(np.float32) + 1j * a[..., 1].astype(np.float32)).astype(np.complex64)
    for comp in (False, True):
        ri = orc.reduce_precision(a, cfg.n_samp, cfg.f, comp)
        rf = orc.reduce_precision(f32, cfg.n_samp, cfg.f, comp)
        rf2 = np.stack([rf.real, rf.imag], axis=-1)
        assert np.array_equal(ri.astype(np.float32), rf2)


def test_compensation_closed_form(orc):
    """Two inputs, A_0 = 4, A_1 = 16, V_01 = 4 + 0j: |V_01|^2 / (A_0 A_1) = 1/4,
    so f is multiplied by 3/4 (Sec. 3.2)."""
    F, T = 1, 8
    v = np.zeros((F, 3, T), dtype=np.complex64)
    v[:, 0, :] = 4.0
    v[:, 2, :] = 16.0
    v[:, 1, :] = 4.0 + 0.0j
    rng = np.random.default_rng(1)
    for t in range(T):
        assert orc.compensation_min(v, 0, t) == np.float32(0.75)
    # data to round: keep the autos/cross levels, add fine structure to round
    w = v.copy()
    w[:, 1, :] += (rng.standard_normal(T) * 1e-3).astype(np.float32)
    w[:, 0, :] += (rng.standard_normal(T) * 1e-3).astype(np.float32)
    N = 64.0
    m = np.array([orc.compensation_min(w, 0, t) for t in range(T)])
    for f in (0.01, 0.1):
        on = orc.reduce_precision(w, N, f, compensate=True)
        for t in range(T):
            off = orc.reduce_precision(w[:, :, t:t + 1].copy(), N, f * float(m[t]))
            assert np.array_equal(on[:, :, t:t + 1].view(np.uint32), off.view(np.uint32))


def test_compensation_no_rounding_when_cross_exceeds_autos(orc):
    v = np.zeros((1, 3, 2), dtype=np.complex64)
    v[:, 0, :] = 4.0
    v[:, 2, :] = 4.0
    v[:, 1, 0] = 5.0 + 0.123j        # |V|^2 > A_0 A_1: nothing can be trusted
    v[:, 1, 1] = 1.0 + 0.123j
    assert orc.compensation_min(v, 0, 0) == 0.0
    r = orc.reduce_precision(v, 256.0, 0.5, compensate=True)
    ru, vu = r.view(np.uint32).reshape(1, 3, 2, 2), v.view(np.uint32).reshape(1, 3, 2, 2)
    assert np.array_equal(ru[:, :, 0], vu[:, :, 0])
    assert not np.array_equal(ru[:, :, 1], vu[:, :, 1])


def test_compensation_on_synthetic_sky(orc):
    """rho = 0.05 sky amplitude: |V_ij|^2 / (A_i A_j) ~ 0.0025 plus noise, so the
    factor sits just below one; without crosses it is exactly one."""
    cfg = synth.CONFIG_SMALL
    v = synth.visibilities(cfg)
    ms = np.array([orc.compensation_min(v, fr, t) for fr in range(0, 16, 5) for t in range(0, 64, 9)])
    assert np.all(ms < 1.0) and np.all(ms > 0.99)
    one = synth.visibilities(synth.VisConfig(2, 1, 4, 2 ** 10, 0.1, seed=1))
    assert orc.compensation_min(one, 0, 0) == 1.0
    # compensating never increases the rounding: every |error| shrinks or stays
    a = orc.reduce_precision(v, cfg.n_samp, cfg.f, False).view(np.float32).astype(np.float64)
    b = orc.reduce_precision(v, cfg.n_samp, cfg.f, True).view(np.float32).astype(np.float64)
    x = v.view(np.float32).astype(np.float64)
    assert np.mean(np.abs(b - x)) <= np.mean(np.abs(a - x))
