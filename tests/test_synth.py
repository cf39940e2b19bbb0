"""The synthetic visibilities carry the thermal scatter of Sec. 3.1 (S2)."""
import numpy as np
import pytest

from paper_1503_00638_gb300 import synth


def test_cross_and_auto_scatter_match_radiometer(orc):
    cfg = synth.VisConfig(2, 4, 8192, 2 ** 12, 0.01, seed=3, rho=0.0)
    v = synth.visibilities(cfg)
    n, N, T = cfg.n_inputs, cfg.n_samp, cfg.n_time
    pii = [synth.auto_product_index(i, n) for i in range(n)]
    p = 0
    for i in range(n):
        for j in range(i, n):
            for fr in range(cfg.n_freq):
                Ai, Aj = v[fr, pii[i]].real.mean(), v[fr, pii[j]].real.mean()
                for a, comp in ((0, v[fr, p].real), (1, v[fr, p].imag)):
                    model = orc.rad_simple_var(i, j, a, Ai, Aj, N)
                    if model == 0:
                        assert np.all(comp == 0)
                        continue
                    assert abs(comp.var() - model) < 5 * np.sqrt(2.0 / T) * model
            p += 1


def test_shapes_and_slices():
    cfg = synth.CONFIG_SMALL
    v = synth.visibilities(cfg)
    assert v.shape == (16, 136, 64) and v.dtype == np.complex64 and v.nbytes == 1114112
    assert np.array_equal(synth.visibilities(cfg, 5, 9), v[5:9])
    n = cfg.n_inputs
    for i in range(n):
        p = synth.auto_product_index(i, n)
        assert np.all(v[:, p].imag == 0) and np.all(v[:, p].real > 30)
    assert synth.CONFIG_CHIME.nbytes == 1024 * 8256 * 16 * 8


def test_random_walk_steps():
    for dt in (np.uint8, np.uint16, np.int32, np.float64):
        w = synth.random_walk(10000, dt, seed=1)
        assert w.dtype == dt
        d = np.diff(w.astype(np.int64) if dt != np.float64 else w)
        if dt in (np.uint8, np.uint16):
            d = (d + 2 ** (8 * w.itemsize - 1)) % 2 ** (8 * w.itemsize) - 2 ** (8 * w.itemsize - 1)
        a = np.abs(d)
        assert set(np.unique(a).astype(int).tolist()) <= {1, 2, 4, 8, 16, 32, 64}


def test_visibilities_int_is_the_scaled_cube():
    cfg = synth.VisConfig(2, 3, 4, 2 ** 10, 0.1, seed=5)
    v = synth.visibilities(cfg)
    a = synth.visibilities_int(cfg, 1000.0)
    assert a.dtype == np.int32 and a.shape == v.shape + (2,)
    assert np.array_equal(a[..., 0], np.rint(v.real.astype(np.float64) * 1000.0))
    assert np.array_equal(a[..., 1], np.rint(v.imag.astype(np.float64) * 1000.0))
    big = synth.visibilities_int(cfg, 1e9)  # autos ~100 * 1e9: clipped to int32
    assert big.max() == np.iinfo(np.int32).max


def test_torch_generators_follow_the_recipe():
    torch = pytest.importorskip("torch")
    # rho = 0: crosses are pure thermal scatter of variance A_i A_j / (2N)
    cfg = synth.VisConfig(4, 6, 4096, 2 ** 10, 0.1, seed=3, rho=0.0)
    v = synth.visibilities_torch(cfg, device="cpu").numpy()
    n = cfg.n_inputs
    ii, jj = np.triu_indices(n)
    A = v[:, [synth.auto_product_index(i, n) for i in range(n)], :].real.mean(axis=2)
    for p in range(ii.size):
        i, j = ii[p], jj[p]
        if i == j:
            assert np.all(v[:, p].imag == 0)
            rel = v[:, p].real / A[:, i][:, None] - 1.0
            assert abs(rel.var() * cfg.n_samp - 1.0) < 0.1       # Var = A^2 / N
        else:
            want = A[:, i] * A[:, j] / (2 * cfg.n_samp)
            got = (v[:, p].real ** 2).mean(axis=1)
            assert np.all(np.abs(got / want - 1.0) < 0.1)
    w = synth.random_walk_torch(10000, 4, seed=1, device="cpu").view(torch.int32).numpy()
    d = np.diff(w.astype(np.int64))
    assert set(np.abs(d).tolist()) <= {1, 2, 4, 8, 16, 32, 64}


def test_physical_visibilities_are_sample_covariances():
    # the mean over many (freq, time) draws of the same R approaches R, and
    # every sample matrix is positive definite
    cfg = synth.VisConfig(1, 3, 4000, 64, 0.1, seed=1, rho=0.6, t_sky=1e12)  # no drift
    v = synth.visibilities_physical(cfg)
    n = 3
    ii, jj = np.triu_indices(n)
    mats = np.zeros((cfg.n_time, n, n), dtype=np.complex128)
    mats[:, ii, jj] = v[0].T
    mats[:, jj, ii] = np.conj(v[0].T)
    assert np.all(np.linalg.eigvalsh(mats).min(axis=1) > 0)
    mean = mats.mean(axis=0)
    A = np.real(np.diag(mean))
    # |R_ij| = rho sqrt(A_i A_j) off the diagonal
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert abs(abs(mean[i, j]) / np.sqrt(A[i] * A[j]) - 0.6) < 0.02
