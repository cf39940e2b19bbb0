"""Pins for the oracle's noise model (Sec. 3.1) against brute force.

The radiometer variances and the rad_full covariances are checked against a
direct simulation of complex Gaussian voltages correlated over N samples; the
oracle's q = 12 f s^2 in float32 (reading R1) is checked against the same
quantity in fp64.
"""
import numpy as np
import pytest


def _simulate(R, N, M, seed):
    """M independent integrations of N samples of circular complex Gaussian
    voltages with covariance R; returns V[m, i, j] = <a_i a_j^*>."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = R.shape[0]
    L = np.linalg.cholesky(R)
    out = np.empty((M, n, n), dtype=np.complex128)
    step = 1000
    for m0 in range(0, M, step):
        m1 = min(M, m0 + step)
        z = (rng.standard_normal((m1 - m0, N, n)) + 1j * rng.standard_normal((m1 - m0, N, n))) / np.sqrt(2)
        a = z @ L.T                                   # a[k] = L z[k]
        out[m0:m1] = np.einsum("mki,mkj->mij", a, a.conj()) / N
    return out


def _comp(V, alpha, i, j):
    return V[:, i, j].real if alpha == 0 else V[:, i, j].imag


def test_rad_simple_closed_forms(orc):
    # Eq. 1-3 of Sec. 3.1 written out: Re V_ii: V_ii^2/N, Im V_ii: 0, V_ij: V_ii V_jj / 2N
    N, Vii, Vjj = 1234.0, 97.0, 61.0
    assert orc.rad_simple_var(3, 3, 0, Vii, Vii, N) == pytest.approx(Vii * Vii / N, rel=1e-15)
    assert orc.rad_simple_var(3, 3, 1, Vii, Vii, N) == 0.0
    for a in (0, 1):
        assert orc.rad_simple_var(1, 4, a, Vii, Vjj, N) == pytest.approx(Vii * Vjj / (2 * N), rel=1e-15)


@pytest.mark.parametrize("sky", [False, True])
def test_radiometer_brute_force(orc, sky):
    """Empirical (co)variances of simulated visibilities vs Eq. rad_full1-3,
    and vs Eq. rad_simple when the channels are uncorrelated (S1)."""
    n, N, M = 3, 256, 20000
    noise = np.diag([100.0, 70.0, 130.0]).astype(np.complex128)
    if sky:
        gains = np.array([1.0, 0.8 * np.exp(0.7j), 1.2 * np.exp(-1.9j)])
        R = noise + 60.0 * np.outer(gains, gains.conj())    # a bright point source
    else:
        R = noise
    V = _simulate(R, N, M, seed=11 + sky)
    comps = [(a, i, j) for i in range(n) for j in range(i, n) for a in (0, 1) if not (i == j and a == 1)]
    for (a, i, j) in comps:
        for (b, g, h) in comps:
            x, y = _comp(V, a, i, j), _comp(V, b, g, h)
            emp = np.mean((x - x.mean()) * (y - y.mean()))
            model = orc.rad_full_cov(R, a, i, j, b, g, h, N)
            se = np.sqrt((x.var() * y.var() + emp ** 2) / M)
            assert abs(emp - model) < 5 * se + 1e-12, (a, i, j, b, g, h, emp, model)
    if not sky:
        for (a, i, j) in comps + [(1, 0, 0)]:
            x = _comp(V, a, i, j)
            model = orc.rad_simple_var(i, j, a, R[i, i].real, R[j, j].real, N)
            assert abs(x.var() - model) <= 5 * np.sqrt(2.0 / M) * model + 1e-12


def test_rad_full_special_cases(orc):
    """The special cases printed after Eq. rad_full3 (Sec. 3.1)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    V = A @ A.conj().T
    N = 300.0
    i, j = 0, 2
    Vii, Vjj, Vij = V[i, i].real, V[j, j].real, V[i, j]
    assert orc.rad_full_cov(V, 0, i, i, 0, i, i, N) == pytest.approx(Vii ** 2 / N, rel=1e-12)
    assert orc.rad_full_cov(V, 1, i, i, 1, i, i, N) == pytest.approx(0.0, abs=1e-12)
    assert orc.rad_full_cov(V, 0, i, i, 0, i, j, N) == pytest.approx(Vii * Vij.real / N, rel=1e-12)
    assert orc.rad_full_cov(V, 0, i, j, 0, i, j, N) == pytest.approx(
        (Vii * Vjj + Vij.real ** 2 - Vij.imag ** 2) / (2 * N), rel=1e-12)
    assert orc.rad_full_cov(V, 1, i, j, 1, i, j, N) == pytest.approx(
        (Vii * Vjj - Vij.real ** 2 + Vij.imag ** 2) / (2 * N), rel=1e-12)
    assert orc.rad_full_cov(V, 0, i, j, 1, i, j, N) == pytest.approx(Vij.real * Vij.imag / N, rel=1e-12)


def test_rad_full_reduces_to_rad_simple(orc):
    """With V diagonal, Eq. rad_full1-3 collapse to Eq. rad_simple."""
    V = np.diag([80.0, 120.0, 95.0]).astype(np.complex128)
    N = 4096.0
    for i in range(3):
        for j in range(i, 3):
            for a in (0, 1):
                full = orc.rad_full_cov(V, a, i, j, a, i, j, N)
                simple = orc.rad_simple_var(i, j, a, V[i, i].real, V[j, j].real, N)
                assert full == pytest.approx(simple, rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("f", [1e-5, 1e-3, 0.01, 0.1])
def test_q32_matches_12fs2(orc, f):
    """Reading R1: the float32 q agrees with 12 f s^2 (fp64) to float32 rounding."""
    rng = np.random.default_rng(1)
    for N in (2.0 ** 16, 2.0 ** 17, 8.4e6):
        for _ in range(200):
            Ai, Aj = rng.uniform(1, 1e4, 2).astype(np.float32)
            for auto in (False, True):
                Aj_ = Ai if auto else Aj
                s2 = orc.rad_simple_var(0, 0 if auto else 1, 0, float(Ai), float(Aj_), N)
                q = orc.q32(auto, float(Ai), float(Aj_), f, N)
                assert abs(float(q) - 12 * f * s2) <= 4 * np.finfo(np.float32).eps * 12 * f * s2
