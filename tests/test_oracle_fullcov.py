"""Pins for the oracle's full-covariance noise (Sec. 3.1, Eq. rad_full1-3 and
Eq. noise): closed forms, an independent inverse, brute-force simulation of
the conditional variance, and the paper's point-source example."""
import numpy as np
import pytest

from paper_1503_00638_gb300 import synth


def test_component_index_is_a_bijection(orc):
    for n in (1, 2, 5, 16):
        idx = [orc.full_index(n, i, j, a) for i in range(n) for j in range(i, n) for a in (0, 1)
               if not (a == 1 and i == j)]
        assert sorted(idx) == list(range(n * n))


def test_uncorrelated_inputs_give_the_radiometer_variances(orc):
    # no cross correlation: C is diagonal and s^2 is Eq. rad_simple's
    n, N = 4, 1000.0
    A = np.array([50.0, 80.0, 120.0, 99.0])
    V = np.diag(A).astype(np.complex128)
    C = orc.full_cov_matrix(V, N)
    assert np.count_nonzero(C - np.diag(np.diag(C))) == 0
    rc, s2 = orc.full_noise_var(V, N)
    assert rc == 0
    for i in range(n):
        for j in range(i, n):
            want = A[i] * A[j] / (2 * N) * (2.0 if i == j else 1.0)
            assert s2[orc.full_index(n, i, j, 0)] == pytest.approx(want, rel=1e-14)
            if i != j:
                assert s2[orc.full_index(n, i, j, 1)] == pytest.approx(want, rel=1e-14)


def test_inverse_against_numpy(orc):
    rng = np.random.default_rng(0)
    for M in (1, 3, 16, 49):
        X = rng.standard_normal((M, M + 5))
        A = X @ X.T / M + 0.1 * np.eye(M)
        rc, Ai = orc.invert_spd(A)
        assert rc == 0
        assert np.allclose(Ai, np.linalg.inv(A), rtol=1e-10, atol=1e-12)
    rc, _ = orc.invert_spd(np.array([[1.0, 2.0], [2.0, 1.0]]))   # indefinite
    assert rc == -1


def fisher_s2(V, N):
    """s^2 = 1/(C^-1)_kk from W = V^-1 alone: C is the covariance of the real
    components of a circular complex Gaussian correlation matrix, whose
    inverse is the Fisher information N tr(E_a W E_b W) of those components
    (E_a: the Hermitian matrix with a one in component a).  Its diagonal is
    N W_ii^2 for Re V_ii and 2 N (W_ii W_jj +- Re(W_ij^2)) for Re / Im V_ij."""
    n = V.shape[0]
    W = np.linalg.inv(V)
    P = n * (n + 1) // 2
    out = np.empty(n * n)
    p = 0
    for i in range(n):
        for j in range(i, n):
            if i == j:
                out[p] = 1.0 / (N * W[i, i].real ** 2)
            else:
                ww, r2 = W[i, i].real * W[j, j].real, (W[i, j] ** 2).real
                out[p] = 1.0 / (2 * N * (ww + r2))
                out[P + p - i - 1] = 1.0 / (2 * N * (ww - r2))
            p += 1
    return out


def wishart(n, rng, scale=1.0):
    z = rng.standard_normal((n, 3 * n)) + 1j * rng.standard_normal((n, 3 * n))
    return scale * (z @ z.conj().T) / (3 * n)


def test_inverse_diagonal_matches_the_fisher_closed_form(orc):
    # the oracle inverts the n^2 x n^2 matrix of Eq. rad_full1-3; the Fisher
    # information gives the same diagonal from the n x n inverse of V
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 5, 8):
        V = wishart(n, rng, 50.0) + np.diag(rng.uniform(1, 5, n))
        rc, s2 = orc.full_noise_var(V, 1000.0)
        assert rc == 0
        assert np.allclose(s2, fisher_s2(V, 1000.0), rtol=1e-10, atol=0), n


def test_definiteness_of_c_follows_v(orc):
    # C is quadratic in V: -V gives the same C (positive definite), an
    # indefinite V an indefinite C
    rng = np.random.default_rng(12)
    V = wishart(4, rng, 10.0) + np.eye(4)
    rc, s2 = orc.full_noise_var(V, 500.0)
    rcn, s2n = orc.full_noise_var(-V, 500.0)
    assert rc == 0 and rcn == 0 and np.allclose(s2, s2n, rtol=1e-12)
    U = V.copy()
    U[2, :] = 0
    U[:, 2] = 0
    U[2, 2] = -3.0      # one negative eigenvalue
    rcu, s2u = orc.full_noise_var(U, 500.0)
    assert rcu == -1 and np.all(s2u == 0)


def simulate_components(R, N, trials, rng):
    """Visibility components of `trials` integrations of N samples of
    complex Gaussian voltages with covariance R, in the oracle's order."""
    n = R.shape[0]
    L = np.linalg.cholesky(R)
    out = np.empty((trials, n * n))
    iu = [(i, j) for i in range(n) for j in range(i, n)]
    P = len(iu)
    for t in range(trials):
        z = (rng.standard_normal((n, N)) + 1j * rng.standard_normal((n, N))) / np.sqrt(2)
        a = L @ z
        V = a @ a.conj().T / N
        out[t, :P] = [V[i, j].real for i, j in iu]
        out[t, P:] = [V[i, j].imag for i, j in iu if i < j]
    return out


def test_conditional_variance_by_simulation(orc):
    # a sky-dominated 3-input array: strongly correlated components, where
    # s^2 = 1/(C^-1)_kk is well below the marginal variance C_kk
    rng = np.random.default_rng(7)
    n, N, trials = 3, 64, 30000
    g = np.array([1.0, 0.8 + 0.3j, 0.6 - 0.5j])
    R = np.outer(g, g.conj()) * 3.0 + np.diag([1.0, 1.3, 0.7])
    x = simulate_components(R, N, trials, rng)
    emp = np.cov(x, rowvar=False)
    cond_emp = 1.0 / np.diag(np.linalg.inv(emp))
    rc, s2 = orc.full_noise_var(R, N)
    C = orc.full_cov_matrix(R, N)
    assert rc == 0
    # sampling error of a variance estimate: ~sqrt(2/trials) relative
    assert np.allclose(s2, cond_emp, rtol=0.05)
    assert np.allclose(np.diag(C), np.diag(emp), rtol=0.05)
    assert np.all(s2 < np.diag(C))


def test_point_source_self_noise(orc):
    # the paper's example: one bright source at zenith, calibrated inputs:
    # all visibilities share Re = S; the marginal noise is large, but
    # differences of visibilities are quiet, so the unmarginalized noise of
    # each cross product is far below its marginal variance
    n, N, S, Tsys = 4, 1000.0, 100.0, 1.0
    V = np.full((n, n), S, dtype=np.complex128) + np.diag(np.full(n, Tsys))
    C = orc.full_cov_matrix(V, N)
    rc, s2 = orc.full_noise_var(V, N)
    assert rc == 0
    for i in range(n):
        for j in range(i + 1, n):
            k = orc.full_index(n, i, j, 0)
            assert s2[k] < C[k, k] / 20


def test_full_rounding_matches_plain_when_uncorrelated(orc):
    # with rho = 0 the crosses carry only thermal scatter and the full
    # covariance is close to diagonal: granularities agree with Eq.
    # rad_simple's except where the two noise estimates straddle a power of 4
    cfg = synth.VisConfig(2, 4, 8, 2 ** 14, 0.05, seed=3, rho=0.0)
    v = synth.visibilities(cfg)
    full = orc.reduce_precision_full(v, cfg.n_samp, cfg.f)
    plain = orc.reduce_precision_c64(v, cfg.n_samp, cfg.f)
    same = np.mean(full.view(np.uint32) == plain.view(np.uint32))
    assert same > 0.9
    # and the rounding error respects each granularity's bound
    err = np.abs(full.view(np.float32).astype(np.float64) - v.view(np.float32))
    assert np.all(err <= np.abs(v.view(np.float32)) + 1e-30)


def test_full_rounding_is_finer_with_a_bright_sky(orc):
    # a physical cube (positive definite samples) dominated by a source
    cfg = synth.VisConfig(2, 4, 8, 2 ** 12, 0.1, seed=4, rho=0.9)
    v = synth.visibilities_physical(cfg)
    x = v.view(np.float32).astype(np.float64)
    full = orc.reduce_precision_full(v, cfg.n_samp, cfg.f).view(np.float32)
    plain = orc.reduce_precision_c64(v, cfg.n_samp, cfg.f).view(np.float32)
    assert np.any(full != x)          # the full-covariance path did round
    assert np.abs(full - x).sum() < np.abs(plain - x).sum()
