"""GPU parity of the full-covariance noise (Sec. 3.1, Eq. rad_full1-3 and Eq.
noise) and its rounding.  s^2 comes from fp64 inverses along different
routes (the GPU: the n x n inverse of V and the closed form of (C^-1)_kk;
the oracle: Gauss-Jordan on the n^2 x n^2 C), so s^2 is compared to a
relative 1e-9; the rounding is
bit-exact wherever both sides' q = fl32(12 f s^2) agree, and elsewhere the
GPU value must be the exact rounding for its own q (q straddles a float32
step there, and both results are correct)."""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu
    return bsgpu


def sample_matrix(v, n, fr, t):
    """Complex n x n V at (fr, t) of a [F][P][T] (complex64) or [F][P][T][2]
    (int32) cube, as the stored values in fp64."""
    if v.dtype == np.int32:
        x = v[fr, :, t, 0].astype(np.float32).astype(np.float64) + \
            1j * v[fr, :, t, 1].astype(np.float32).astype(np.float64)
    else:
        x = v[fr, :, t].astype(np.complex128)
    V = np.zeros((n, n), dtype=np.complex128)
    ii, jj = np.triu_indices(n)
    V[ii, jj] = x
    V[jj, ii] = np.conj(x)
    return V


CASES = [
    ("n1", synth.VisConfig(2, 1, 3, 2 ** 10, 0.05, seed=1), 0),
    ("n2-bright", synth.VisConfig(2, 2, 4, 2 ** 10, 0.1, seed=2, rho=0.9), 0),
    ("n4", synth.VisConfig(3, 4, 8, 2 ** 12, 0.05, seed=3, rho=0.5), 0),
    ("n9", synth.VisConfig(2, 9, 3, 2 ** 14, 0.02, seed=4, rho=0.3), 0),
    ("n16", synth.VisConfig(2, 16, 16, 2 ** 16, 0.01, seed=5), 0),
    ("n16-int", synth.VisConfig(1, 16, 8, 2 ** 16, 0.01, seed=6, rho=0.5), 4096.0),
    ("n5-int", synth.VisConfig(2, 5, 3, 2 ** 12, 0.1, seed=7, rho=0.9), 2.0 ** 18),
]


def cube(cfg, scale):
    """A physical cube (every sample matrix positive definite), scaled to
    int32 when scale is given."""
    v = synth.visibilities_physical(cfg)
    if not scale:
        return v
    a = np.stack([v.real, v.imag], axis=-1).astype(np.float64) * scale
    return np.clip(np.rint(a), -2 ** 31, 2 ** 31 - 1).astype(np.int32)


@pytest.mark.parametrize("name,cfg,scale", CASES, ids=[c[0] for c in CASES])
def test_noise_variances(bs, orc, name, cfg, scale):
    v = cube(cfg, scale)
    s2 = bs.full_noise_var(torch.from_numpy(v.copy()).cuda(), cfg.n_samp).cpu().numpy()
    n = cfg.n_inputs
    for fr in range(cfg.n_freq):
        for t in range(cfg.n_time):
            rc, want = orc.full_noise_var(sample_matrix(v, n, fr, t), cfg.n_samp)
            assert rc == 0
            assert np.allclose(s2[fr, t], want, rtol=1e-9, atol=0), (fr, t)


def check_rounding(orc, v, got, s2_gpu, cfg):
    want = orc.reduce_precision_full(v, cfg.n_samp, cfg.f)
    n, P = cfg.n_inputs, synth.n_products(cfg.n_inputs)
    ii, jj = np.triu_indices(n)
    is_int = v.dtype == np.int32
    flat = (lambda a: a.reshape(-1)) if is_int else (lambda a: a.view(np.float32).reshape(-1))
    g, w, xs = flat(got), flat(want), flat(v)
    diff = np.nonzero(g.view(np.uint32) != w.view(np.uint32))[0]
    assert diff.size <= max(2, g.size // 1000)
    for e in diff:
        c, part = divmod(int(e), 2)
        fp, t = divmod(c, cfg.n_time)
        fr, p = divmod(fp, P)
        k = orc.full_index(n, int(ii[p]), int(jj[p]), part)
        q = np.float32(12.0 * cfg.f * s2_gpu[fr, t, k])
        _, s2o = orc.full_noise_var(sample_matrix(v, n, fr, t), cfg.n_samp)
        assert np.float32(12.0 * cfg.f * s2o[k]) != q     # only where the q differ
        if is_int:
            kk = orc.granularity_exponent(q)
            assert g[e] == (orc.round_int(int(xs[e]), kk) if kk is not None else xs[e])
        else:
            assert g[e].view(np.uint32) == orc.round_element(float(xs[e]), float(q)).view(np.uint32)


@pytest.mark.parametrize("name,cfg,scale", CASES, ids=[c[0] for c in CASES])
def test_rounding(bs, orc, name, cfg, scale):
    v = cube(cfg, scale)
    d = torch.from_numpy(v.copy()).cuda()
    got = bs.reduce_precision(d, cfg.n_samp, cfg.f, full_cov=True).cpu().numpy()
    s2 = bs.full_noise_var(d, cfg.n_samp).cpu().numpy()
    check_rounding(orc, v, got, s2, cfg)


@pytest.mark.parametrize("es,B,tslow,scale", [(4, 2048, False, 0), (8, 1024, True, 0),
                                              (4, 96, False, 0), (4, 2048, False, 2.0 ** 16),
                                              (4, 1024, True, 2.0 ** 12), (8, 1024, False, 0)])
def test_compression(bs, orc, es, B, tslow, scale):
    # full blocks of 4-byte components take the fast kernel's per-component
    # q rows (float and int32, in order and time-slowest), 8-byte samples its
    # per-sample path, B = 96 the general kernel
    cfg = synth.VisConfig(2, 8, 16, 2 ** 14, 0.02, seed=9, rho=0.4)
    v = cube(cfg, scale)
    d = torch.from_numpy(v.copy()).cuda()
    rounded = bs.reduce_precision(d, cfg.n_samp, cfg.f, full_cov=True).cpu().numpy()
    src = torch.from_numpy(np.ascontiguousarray(np.moveaxis(v, 2, 0))).cuda() if tslow else d
    c = bs.compress_vis_ex(src, cfg.n_samp, cfg.f, False, es, B, time_slowest=tslow, full_cov=True)
    assert bs.status(c.ws) == 0
    flat = np.ascontiguousarray(rounded).view(np.uint32 if es == 4 else np.uint64).reshape(-1)
    rc, back = orc.decompress(c.buf[:c.nbytes].cpu().numpy().tobytes(), flat.size, flat.dtype, B)
    assert rc == 0 and np.array_equal(back, flat)


def test_singular_samples_stay_unrounded(bs, orc):
    cfg = synth.VisConfig(1, 3, 4, 2 ** 10, 0.5, seed=10)
    v = synth.visibilities_physical(cfg)
    # input 0 dead at t = 1: its auto and crosses are zero, C is singular there
    for p, (i, j) in enumerate(zip(*np.triu_indices(3))):
        if i == 0:
            v[0, p, 1] = 0
    want = orc.reduce_precision_full(v, cfg.n_samp, cfg.f)
    got = bs.reduce_precision(torch.from_numpy(v.copy()).cuda(), cfg.n_samp, cfg.f,
                              full_cov=True).cpu().numpy()
    col = lambda a: np.ascontiguousarray(a[:, :, 1]).view(np.uint32)  # noqa: E731
    assert np.array_equal(col(got), col(v)) and np.array_equal(col(want), col(v))
    assert not np.array_equal(np.ascontiguousarray(got[:, :, 0]).view(np.uint32),
                              np.ascontiguousarray(v[:, :, 0]).view(np.uint32))
    s2 = bs.full_noise_var(torch.from_numpy(v.copy()).cuda(), cfg.n_samp).cpu().numpy()
    assert np.all(s2[0, 1] == 0) and np.all(s2[0, 0] > 0)


def test_definiteness_like_the_oracle(bs, orc):
    # t = 0: V negated (negative definite: C is still positive definite and
    # s^2 the same); t = 1: one input's auto negative and its crosses zero
    # (indefinite: C indefinite, unrounded); t = 2: as generated
    cfg = synth.VisConfig(1, 5, 3, 2 ** 12, 0.3, seed=13, rho=0.6)
    v = synth.visibilities_physical(cfg)
    ii, jj = np.triu_indices(5)
    v[0, :, 0] = -v[0, :, 0]
    for p, (i, j) in enumerate(zip(ii, jj)):
        if i == 3 or j == 3:
            v[0, p, 1] = -1.0 if i == j else 0.0
    s2 = bs.full_noise_var(torch.from_numpy(v.copy()).cuda(), cfg.n_samp).cpu().numpy()
    for t in range(3):
        rc, want = orc.full_noise_var(sample_matrix(v, 5, 0, t), cfg.n_samp)
        assert rc == (-1 if t == 1 else 0), t
        assert np.allclose(s2[0, t], want, rtol=1e-9, atol=0), t
    got = bs.reduce_precision(torch.from_numpy(v.copy()).cuda(), cfg.n_samp, cfg.f,
                              full_cov=True).cpu().numpy()
    want = orc.reduce_precision_full(v, cfg.n_samp, cfg.f)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_argument_errors(bs):
    z = torch.zeros((1, 153, 2), dtype=torch.complex64, device="cuda")   # 17 inputs
    with pytest.raises(bs.BsgpuError):
        bs.reduce_precision(z, 1000.0, 0.1, full_cov=True)
    z = torch.zeros((1, 10, 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(bs.BsgpuError):
        bs.reduce_precision(z, 1000.0, 0.1, compensate=True, full_cov=True)
