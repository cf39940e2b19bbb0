"""Pins for the oracle's precision reduction (Sec. 3.2, Sec. 5.1).

* the granularity exponent against an exact integer derivation of
  max{k : 4^k < q} from q's rational value (Eq. trunc_error, strict);
* rounding against Python's exact rational arithmetic with banker's rounding
  (ties to even, the footnote of Sec. 3.2);
* the error bounds, flatness, symmetry and variance bound of Sec. 5.1;
* the exact power-of-two scaling invariants behind the 4^5 remark of Sec. 5.1;
* the bits-kept figure of Sec. 5.2 (about 15 bits for CHIME at f = 1e-3).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1503_00638_gb300 import synth


def exact_k(q):
    """max{k : 4^k < q} for a positive float q, by integer bit lengths.
    q = num / 2^d exactly; with b = bit length of num:
      num a power of two (num = 2^(b-1)): log2 q = b-1-d exactly, 2k < b-1-d;
      otherwise log2 q lies strictly inside (b-1-d, b-d).                  """
    num, den = Fraction(float(q)).as_integer_ratio()
    d = den.bit_length() - 1
    assert den == 1 << d
    b = num.bit_length()
    L = b - 1 - d                          # floor(log2 q)
    if num == 1 << (b - 1):                # q = 2^L exactly: need 2k < L
        return (L - 1) // 2 if L % 2 else L // 2 - 1
    return L // 2                          # need 2k <= L (since log2 q > L)


def exact_round(x, k):
    """Nearest multiple of 2^k to float32 x, ties to even, as float32 (sign of
    zero kept, overflow to inf)."""
    x = np.float32(x)
    if not np.isfinite(x):
        return x
    m = round(Fraction(float(x)) / Fraction(2) ** k)          # round-half-even
    if m == 0:
        return np.float32(math.copysign(0.0, float(x)))
    v = Fraction(m) * Fraction(2) ** k
    if abs(v) > Fraction(float(np.finfo(np.float32).max)):
        return np.float32(math.copysign(math.inf, float(x)))
    fv = np.float32(float(v))
    assert Fraction(float(fv)) == v                          # representable
    return fv


def bits(x):
    return np.float32(x).view(np.uint32)


def test_granularity_exponent_exact(orc):
    rng = np.random.default_rng(3)
    qs = rng.integers(0x00800000, 0x7F800000, size=4000, dtype=np.uint32).view(np.float32)
    special = [4.0 ** m for m in range(-60, 60)]
    special += [np.nextafter(np.float32(s), np.float32(0)) for s in special]
    special += [np.nextafter(np.float32(s), np.float32(np.inf)) for s in special[:120]]
    for q in list(qs) + special:
        q = np.float32(q)
        if not (q >= np.finfo(np.float32).tiny and np.isfinite(q)):
            continue
        assert orc.granularity_exponent(q) == exact_k(q), q


def test_granularity_strict_inequality(orc):
    # Eq. trunc_error is strict: q exactly 4^m gives g = 2^(m-1)
    for m in range(-20, 20):
        assert orc.granularity_exponent(4.0 ** m) == m - 1
        assert orc.granularity_exponent(np.nextafter(np.float32(4.0 ** m), np.float32(np.inf))) == m


def test_granularity_unusable_q(orc):
    # reading R2: no rounding for q <= 0, NaN, inf or subnormal q
    for q in [0.0, -1.0, np.nan, np.inf, 1e-40]:
        assert orc.granularity_exponent(q) is None
        assert bits(orc.round_element(1.2345, q)) == bits(1.2345)


def test_round_pow2_exact(orc):
    rng = np.random.default_rng(4)
    xs = rng.integers(0, 2 ** 32, size=3000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    for x in xs:
        if not np.isfinite(x):
            r = orc.round_pow2(x, 0)      # (the scalar ctypes call may quiet a NaN)
            assert (np.isnan(r) and np.isnan(x)) or bits(r) == bits(x)
            continue
        e = int(np.frexp(np.float64(x))[1]) if x != 0 else -126
        for k in (e - 30, e - 24, e - 23, e - 10, e - 2, e - 1, e, e + 1, e + 3):
            if -400 < k < 400:
                assert bits(orc.round_pow2(x, k)) == bits(exact_round(x, k)), (x, k)


def test_round_ties_to_even(orc):
    for k in (-10, -4, 0, 3):
        for m in range(-40, 40):
            x = (m + 0.5) * 2.0 ** k
            r = orc.round_pow2(x, k)
            want = (m if m % 2 == 0 else m + 1) * 2.0 ** k
            assert float(r) == want and r / 2.0 ** k % 2 == 0
    # below and above the half-way point of a tiny value: sign of zero kept (R5)
    assert bits(orc.round_pow2(-0.3, 0)) == bits(-0.0)
    assert bits(orc.round_pow2(0.5, 0)) == bits(0.0)
    assert float(orc.round_pow2(1.5, 0)) == 2.0
    # rounding up past FLT_MAX gives inf (R7)
    big = np.finfo(np.float32).max
    assert np.isinf(orc.round_pow2(big, 105))   # (2^24-1) 2^104 -> tie -> 2^128


@pytest.fixture(scope="module")
def small_cube():
    return synth.visibilities(synth.CONFIG_SMALL)


def _split(orc, vis, N, f):
    out = orc.reduce_precision_c64(vis, N, f)
    kmap = orc.granularity_map_c64(vis, N, f)
    x = vis.view(np.float32).reshape(kmap.shape)
    xr = out.view(np.float32).reshape(kmap.shape)
    return x, xr, kmap


def _q_of(vis, N, f):
    """q per float from the fp64 radiometer equation (for bounds only)."""
    F, P, T = vis.shape
    n = int(round((np.sqrt(8 * P + 1) - 1) / 2))
    ii, jj = np.triu_indices(n)
    pii = np.array([synth.auto_product_index(i, n) for i in range(n)])
    A = vis.real[:, pii, :].astype(np.float64)                  # [F][n][T]
    Ai, Aj = A[:, ii, :], A[:, jj, :]
    s2 = np.where((ii == jj)[None, :, None], Ai * Ai / N, Ai * Aj / (2 * N))
    return 12 * f * s2


def test_error_bounds_on_cube(orc, small_cube):
    """S3 on every element: |x_r - x| <= 2^(k-1) < sqrt(q)/2, x_r a multiple of
    2^k, k maximal; Im of autos untouched."""
    cfg = synth.CONFIG_SMALL
    x, xr, k = _split(orc, small_cube, cfg.n_samp, cfg.f)
    q = _q_of(small_cube, cfg.n_samp, cfg.f)
    ok = k > -1000
    xd, xrd = x.astype(np.float64), xr.astype(np.float64)
    g = np.where(ok, np.ldexp(1.0, np.where(ok, k, 0)), 0.0)
    assert np.all(np.abs(xrd - xd)[ok] <= g[ok] / 2)
    assert np.all(np.mod(xrd[ok], g[ok]) == 0)
    qq = np.stack([q, q], axis=-1)
    assert np.all(g[ok] ** 2 < qq[ok] * (1 + 1e-6))
    assert np.all((2 * g[ok]) ** 2 >= qq[ok] * (1 - 1e-6))
    assert np.array_equal(xr[~ok].view(np.uint32), x[~ok].view(np.uint32))
    # cross g for A ~ 100 at N = 2^16, f = 0.01 is 2^-4
    assert np.median(k[..., 0][k[..., 0] > -1000]) == -4


def test_error_distribution(orc, small_cube):
    """S4 / Sec. 5.1: error / sqrt(q) lies in [-1/2, 1/2], is flat on
    [-1/4, 1/4], symmetric with zero mean, and adds variance below f s^2."""
    cfg = synth.CONFIG_SMALL
    vis = np.concatenate([small_cube] + [synth.visibilities(synth.VisConfig(
        16, 16, 64, 2 ** 16, 0.01, seed=s)) for s in (1, 2, 3)], axis=0)
    x, xr, k = _split(orc, vis, cfg.n_samp, cfg.f)
    q = np.stack([_q_of(vis, cfg.n_samp, cfg.f)] * 2, axis=-1)
    ok = k > -1000
    err = (xr.astype(np.float64) - x.astype(np.float64))[ok]
    u = err / np.sqrt(q[ok])
    assert np.all(np.abs(u) <= 0.5)
    inner = u[np.abs(u) < 0.25]
    hist, _ = np.histogram(inner, bins=10, range=(-0.25, 0.25))
    expect = inner.size / 10
    chi2 = np.sum((hist - expect) ** 2 / expect)
    assert chi2 < 40, hist                                   # 9 dof
    assert abs(u.mean()) < 5 * u.std() / np.sqrt(u.size)
    # symmetric about zero: the two halves hold equal mass
    pos, neg = np.sum(u > 0), np.sum(u < 0)
    assert abs(pos - neg) < 5 * np.sqrt(pos + neg)
    # added variance below f s^2 on average and element by element via g^2/12
    assert np.mean(err ** 2) < np.mean(q[ok]) / 12
    # no correlation of errors along time (lag-1 autocorrelation consistent with 0)
    e_t = (xr.astype(np.float64) - x.astype(np.float64))[..., 0][:, :, 1:]
    e_t = e_t[k[..., 0][:, :, 1:] > -1000].reshape(-1)
    e_all = (xr.astype(np.float64) - x.astype(np.float64))[..., 0]
    ok_t = (k[..., 0] > -1000)
    a = e_all[:, :, 1:][ok_t[:, :, 1:] & ok_t[:, :, :-1]]
    b = e_all[:, :, :-1][ok_t[:, :, 1:] & ok_t[:, :, :-1]]
    r = np.corrcoef(a, b)[0, 1]
    assert abs(r) < 5 / np.sqrt(a.size)


def test_power_of_two_scaling(orc, small_cube):
    """S5: x and autos scaled by 2^m round to 2^m x_r exactly; f -> 4^m f
    shifts every exponent by m (the scaling relation of Sec. 5.1)."""
    cfg = synth.CONFIG_SMALL
    base = orc.reduce_precision_c64(small_cube, cfg.n_samp, cfg.f)
    for m in (-3, 2, 5):
        # scale the float32 components (complex multiplication would flip signed zeros)
        scaled = (small_cube.view(np.float32) * np.float32(2.0 ** m)).view(np.complex64)
        got = orc.reduce_precision_c64(scaled, cfg.n_samp, cfg.f)
        want = base.view(np.float32) * np.float32(2.0 ** m)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    k0 = orc.granularity_map_c64(small_cube, cfg.n_samp, 1e-5)
    k5 = orc.granularity_map_c64(small_cube, cfg.n_samp, 1e-5 * 4 ** 5)
    ok = k0 > -1000
    assert np.array_equal(k5[ok], k0[ok] + 5)


def test_4_to_the_5_distributions_match(orc, small_cube):
    """Sec. 5.1: f values a factor 4^5 apart give the same distribution of
    error / sqrt(q) (compared by a two-sample KS statistic)."""
    cfg = synth.CONFIG_SMALL
    us = []
    for f in (1e-5, 1e-5 * 1024):
        x, xr, k = _split(orc, small_cube, cfg.n_samp, f)
        q = np.stack([_q_of(small_cube, cfg.n_samp, f)] * 2, axis=-1)
        ok = k > -1000
        us.append(np.sort((xr.astype(np.float64) - x)[ok] / np.sqrt(q[ok])))
    a, b = us
    grid = np.linspace(-0.5, 0.5, 201)
    d = np.max(np.abs(np.searchsorted(a, grid) / a.size - np.searchsorted(b, grid) / b.size))
    assert d < 1.95 * np.sqrt(2.0 / min(a.size, b.size)) * 1.5


def test_bits_kept_for_autos(orc, small_cube):
    """S6 / Sec. 5.2: an auto keeps about -log(12 f / N) / (2 log 2) bits; with
    g in [sqrt(q)/2, sqrt(q)) the kept precision log2(A/g) lies in
    (b, b+1] for b = log2(N / 12 f) / 2."""
    cfg = synth.CONFIG_SMALL
    x, xr, k = _split(orc, small_cube, cfg.n_samp, cfg.f)
    n = cfg.n_inputs
    pii = [synth.auto_product_index(i, n) for i in range(n)]
    A = x[:, pii, :, 0].astype(np.float64)
    kk = k[:, pii, :, 0]
    kept = np.log2(A) - kk
    b = -np.log(12 * cfg.f / cfg.n_samp) / (2 * np.log(2))
    assert np.all(kept > b - 1e-6) and np.all(kept <= b + 1 + 1e-6)


def test_paper_bits_figure(orc):
    """Sec. 5.2 prints ~15 bits for CHIME at f = 1e-3 (N = 0.39 MHz x 21.45 s)."""
    N = 400e6 / 1024 * 21.45
    f = 1e-3
    b = -np.log(12 * f / N) / (2 * np.log(2))
    assert 14.5 < b < 15.5
    A = np.float32(1000.0)
    k = orc.granularity_exponent(orc.q32(True, A, A, f, N))
    assert b < np.log2(A) - k <= b + 1
    # and five bits between f = 1e-5 and f = 1e-2 (Sec. 5.2: "a factor of sqrt(1000), or 5.0 bits")
    assert abs(0.5 * np.log2(1e-2 / 1e-5) - 5.0) < 0.02
