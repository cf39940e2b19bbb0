"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *makes* data; it holds none of the compression arithmetic.
The same bytes feed the CUDA path and the CPU oracle.

Visibility cubes stand in for the CHIME Pathfinder data of Sec. 5 (shape
[freq][product][time], time fastest, products in upper-triangle row-major
order, complex64).  Each (freq, time) sample is made like a correlator output:

* autos V_ii: a per-input, per-frequency system power A_i(f), plus its own
  thermal scatter of variance A_i^2 / N_samp; the imaginary part is +0.0;
* crosses V_ij: a sky term rho * sqrt(A_i A_j) * exp(i(2 pi t (j - i) / (n T_s) + phi_ij))
  (rho = 0.05: the sky adds well under 40 % of the power, as Sec. 3.1 says of
  CHIME) plus thermal scatter of variance A_i A_j / (2 N_samp) per component.

The thermal scatter levels are the physics of a synthetic instrument that
integrates N_samp samples; ``tests/test_synth.py`` checks them against a
brute-force simulation of voltages.  Random walks (Sec. 5's "highly
correlated along time" regime, without rounding) feed the codec-only cases.
"""
from __future__ import annotations

import numpy as np

__all__ = ["VisConfig", "CONFIG_SMALL", "CONFIG_CHIME", "visibilities", "visibilities_physical",
           "random_walk", "random_walk_device", "batch_specs",
           "n_products", "auto_product_index"]


class VisConfig:
    def __init__(self, n_freq, n_inputs, n_time, n_samp, f, seed=0, drift=False,
                 rho=0.05, t_sky=64.0):
        self.n_freq, self.n_inputs, self.n_time = n_freq, n_inputs, n_time
        self.n_samp, self.f, self.seed, self.drift = float(n_samp), f, seed, drift
        self.rho, self.t_sky = rho, t_sky

    @property
    def n_prod(self):
        return n_products(self.n_inputs)

    @property
    def shape(self):
        return (self.n_freq, self.n_prod, self.n_time)

    @property
    def nbytes(self):
        return self.n_freq * self.n_prod * self.n_time * 8

    def describe(self):
        return (f"{self.n_freq} freq x {self.n_prod} products ({self.n_inputs} inputs) x "
                f"{self.n_time} time, complex64, N=2^{int(np.log2(self.n_samp))}, f={self.f}, "
                f"seed {self.seed}")


# 16 freq x 136 products (16 inputs) x 64 time, N = 2^16, f = 0.01
CONFIG_SMALL = VisConfig(16, 16, 64, 2 ** 16, 0.01, seed=0)
# CHIME-Pathfinder-shaped: 1024 freq x 8256 products (128 inputs) x 16 time, N = 2^17
CONFIG_CHIME = VisConfig(1024, 128, 16, 2 ** 17, 0.01, seed=0, drift=True)


def n_products(n_inputs: int) -> int:
    return n_inputs * (n_inputs + 1) // 2


def auto_product_index(i: int, n_inputs: int) -> int:
    """Index of product (i, i) in upper-triangle row-major order."""
    return i * n_inputs - i * (i - 1) // 2


def _pairs(n):
    ii, jj = np.triu_indices(n)
    return ii, jj


def visibilities(cfg: VisConfig, freq_lo: int = 0, freq_hi: int | None = None) -> np.ndarray:
    """The [freq][prod][time] complex64 cube of ``cfg`` (frequencies
    [freq_lo, freq_hi) only, identical to slicing the full cube)."""
    F, n, T = cfg.n_freq, cfg.n_inputs, cfg.n_time
    freq_hi = F if freq_hi is None else freq_hi
    ii, jj = _pairs(n)
    P = ii.size
    g0 = np.random.Generator(np.random.PCG64(cfg.seed))
    base = g0.uniform(50.0, 150.0, size=(n, F))          # A_i(f) before drift
    phase_in = g0.uniform(0.0, 2 * np.pi, size=n)
    phi = g0.uniform(0.0, 2 * np.pi, size=P)              # sky phase per product
    fr = np.arange(F)
    if cfg.drift:
        # smooth bandpass drift with frequency, one phase per input
        A = base[:, :1] * (1.0 + 0.2 * np.sin(2 * np.pi * 3.0 * fr[None, :] / F
                                              + phase_in[:, None]))
    else:
        A = base
    t = np.arange(T)
    out = np.empty((freq_hi - freq_lo, P, T), dtype=np.complex64)
    cross = ii != jj
    for k, fi in enumerate(range(freq_lo, freq_hi)):
        g = np.random.Generator(np.random.PCG64([cfg.seed, 1 + fi]))
        Af = A[:, fi]
        z = g.standard_normal(size=(P, T, 2))
        # autos: power plus thermal scatter of variance A^2 / N_samp
        auto_re = Af[ii][:, None] * (1.0 + z[..., 0] / np.sqrt(cfg.n_samp))
        # crosses: sky term plus thermal scatter of variance A_i A_j / (2 N_samp)
        amp = np.sqrt(Af[ii] * Af[jj])
        ang = (2 * np.pi * t[None, :] * (jj - ii)[:, None] / (n * cfg.t_sky)
               + phi[:, None])
        sig = amp[:, None] / np.sqrt(2.0 * cfg.n_samp)
        re = cfg.rho * amp[:, None] * np.cos(ang) + sig * z[..., 0]
        im = cfg.rho * amp[:, None] * np.sin(ang) + sig * z[..., 1]
        v = np.where(cross[:, None], re, auto_re)
        w = np.where(cross[:, None], im, 0.0)
        out[k].real = v
        out[k].imag = w
    return out


def visibilities_physical(cfg: VisConfig) -> np.ndarray:
    """A [freq][prod][time] complex64 cube whose every (freq, time) matrix is
    a sample covariance of Gaussian voltages (so positive definite, as a
    correlator's output is): true covariance R_ij = sqrt(A_i A_j) (rho
    e^{i(th_i - th_j)} + (1 - rho) delta_ij), a point source of fraction
    rho of the power drifting through the phases th_i(t) = 2 pi t i / (n T_s)
    + th_i0, then V = L W L^H / N with L L^H = R and W a complex Wishart
    matrix with N degrees of freedom (drawn by its Bartlett decomposition:
    W = B B^H, B lower triangular, |B_ii|^2 ~ Gamma(N - i, 1), B_ij ~ CN(0, 1)
    below the diagonal)."""
    F, n, T = cfg.n_freq, cfg.n_inputs, cfg.n_time
    N = int(cfg.n_samp)
    g = np.random.Generator(np.random.PCG64([cfg.seed, 11]))
    A = g.uniform(50.0, 150.0, size=(F, n))
    th0 = g.uniform(0.0, 2 * np.pi, size=n)
    ii, jj = np.triu_indices(n)
    out = np.empty((F, ii.size, T), dtype=np.complex64)
    for fr in range(F):
        sa = np.sqrt(A[fr])
        for t in range(T):
            u = np.exp(1j * (2 * np.pi * t * np.arange(n) / (n * cfg.t_sky) + th0))
            R = np.outer(sa * u, np.conj(sa * u)) * cfg.rho + np.diag(A[fr]) * (1 - cfg.rho)
            L = np.linalg.cholesky(R)
            B = np.zeros((n, n), dtype=np.complex128)
            B[np.diag_indices(n)] = np.sqrt(g.gamma(N - np.arange(n), 1.0))
            lo = np.tril_indices(n, -1)
            B[lo] = (g.standard_normal(lo[0].size) + 1j * g.standard_normal(lo[0].size)) / np.sqrt(2)
            LB = L @ B
            V = LB @ LB.conj().T / N
            out[fr, :, t] = V[ii, jj]
    return out


def visibilities_int(cfg: VisConfig, scale: float, freq_lo: int = 0,
                     freq_hi: int | None = None) -> np.ndarray:
    """The cube of ``cfg`` as a correlator's integers: an int32 array of shape
    [freq][prod][time][2] holding (re, im) of ``visibilities(cfg) * scale``
    rounded to the nearest integer and clipped to the int32 range."""
    v = visibilities(cfg, freq_lo, freq_hi)
    a = np.stack([v.real, v.imag], axis=-1).astype(np.float64) * scale
    lim = np.iinfo(np.int32)
    return np.clip(np.rint(a), lim.min, lim.max).astype(np.int32)


def random_walk(n: int, dtype, seed: int = 0) -> np.ndarray:
    """x_{t+1} = x_t +- 2^k with k ~ U{0..6} and a fair sign; integers wrap."""
    dtype = np.dtype(dtype)
    g = np.random.Generator(np.random.PCG64([seed, 7]))
    k = g.integers(0, 7, size=n, dtype=np.int64)
    s = g.integers(0, 2, size=n, dtype=np.int64) * 2 - 1
    steps = s << k
    if dtype.kind in "ui":
        walk = np.cumsum(steps, dtype=np.int64)
        if dtype.itemsize < 8:
            walk = walk & ((1 << (8 * dtype.itemsize)) - 1)
        return walk.astype(np.dtype(f"u{dtype.itemsize}")).view(dtype)
    return np.cumsum(steps.astype(np.float64)).astype(dtype)


# -- the same recipes built on the GPU, for workloads too large for the host --
# (same distributions as visibilities() / random_walk(), not the same numbers:
# torch's generator replaces numpy's)

def visibilities_torch(cfg: VisConfig, device="cuda"):
    """A complex64 [freq][prod][time] cube following the recipe of
    visibilities(cfg), generated on `device` with torch's generator."""
    import torch
    F, n, T = cfg.n_freq, cfg.n_inputs, cfg.n_time
    g = torch.Generator(device=device)
    g.manual_seed(int(cfg.seed))
    ii, jj = torch.triu_indices(n, n, device=device)
    A = 50.0 + 100.0 * torch.rand((F, n), generator=g, device=device, dtype=torch.float64)
    if cfg.drift:
        ph = 2 * np.pi * torch.rand(n, generator=g, device=device, dtype=torch.float64)
        fr = torch.arange(F, device=device, dtype=torch.float64)[:, None]
        A = A[:1] * (1.0 + 0.2 * torch.sin(2 * np.pi * 3.0 * fr / F + ph[None, :]))
    phi = 2 * np.pi * torch.rand(ii.numel(), generator=g, device=device, dtype=torch.float64)
    t = torch.arange(T, device=device, dtype=torch.float64)
    z = torch.randn((F, ii.numel(), T, 2), generator=g, device=device, dtype=torch.float64)
    Ai, Aj = A[:, ii][..., None], A[:, jj][..., None]
    auto_re = Ai * (1.0 + z[..., 0] / np.sqrt(cfg.n_samp))
    amp = torch.sqrt(Ai * Aj)
    ang = 2 * np.pi * t * (jj - ii).to(torch.float64)[:, None] / (n * cfg.t_sky) + phi[:, None]
    sig = amp / np.sqrt(2.0 * cfg.n_samp)
    cross = (ii != jj)[:, None]
    re = torch.where(cross, cfg.rho * amp * torch.cos(ang) + sig * z[..., 0], auto_re)
    im = torch.where(cross, cfg.rho * amp * torch.sin(ang) + sig * z[..., 1],
                     torch.zeros((), device=device, dtype=torch.float64))
    return torch.complex(re.float(), im.float())


def random_walk_torch(n: int, elem_size: int, seed: int = 0, device="cuda"):
    """The random walk of random_walk() as the bytes of n integers of
    elem_size bytes (wrapping), generated on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    k = torch.randint(0, 7, (n,), generator=g, device=device)
    s = torch.randint(0, 2, (n,), generator=g, device=device) * 2 - 1
    w = torch.cumsum(s << k, 0)
    if elem_size == 1:
        return (w & 0xff).to(torch.uint8)
    if elem_size == 2:
        return (w & 0xffff).to(torch.int32).to(torch.int16).view(torch.uint8)
    if elem_size == 4:
        return w.to(torch.int32).view(torch.uint8)
    return w.view(torch.uint8)


def random_walk_device(n: int, elem_size: int, seed: int = 0, floating: bool = False,
                       device="cuda", chunk: int = 1 << 26):
    """The random walk of random_walk() made on `device` in pieces of `chunk`
    steps (so that multi-GB arrays need no multi-GB temporaries), as the bytes
    of n elements of elem_size bytes: wrapping integers, or float64 values
    (floating=True, elem_size 8) as random_walk() makes them for float64."""
    import torch
    if floating and elem_size != 8:
        raise ValueError("floating walks are float64")
    out = torch.empty(n * elem_size, dtype=torch.uint8, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    carry_i = torch.zeros((), dtype=torch.int64, device=device)
    carry_f = torch.zeros((), dtype=torch.float64, device=device)
    for a in range(0, n, chunk):
        m = min(chunk, n - a)
        k = torch.randint(0, 7, (m,), generator=g, device=device, dtype=torch.int32)
        sgn = torch.randint(0, 2, (m,), generator=g, device=device, dtype=torch.int32) * 2 - 1
        step = (sgn << k).to(torch.int64)
        dst = out[a * elem_size:(a + m) * elem_size]
        if floating:
            w = torch.cumsum(step.to(torch.float64), 0) + carry_f
            carry_f = w[-1].clone()
            dst.copy_(w.view(torch.uint8))
        else:
            w = torch.cumsum(step, 0) + carry_i
            carry_i = w[-1].clone()
            if elem_size == 8:
                dst.copy_(w.view(torch.uint8))
            else:
                low = (w & ((1 << (8 * elem_size)) - 1)).to(torch.int32)
                if elem_size == 4:
                    dst.copy_(low.view(torch.uint8))
                elif elem_size == 2:
                    dst.copy_(low.to(torch.int16).view(torch.uint8))
                else:
                    dst.copy_(low.to(torch.uint8))
        del k, sgn, step, w
    return out


def batch_specs(n_chunks: int, seed: int):
    """The shapes of a batch of uneven chunks: (bytes, element size, kind) per
    chunk, sizes log-uniform on [64 KiB, 64 MiB], element size uniform on
    {2, 4, 8}, kind "vis" (a visibility cube to be rounded) or "walk" (a
    random walk) with equal odds."""
    rng = np.random.default_rng([seed, 4])
    sizes = np.exp(rng.uniform(np.log(64 << 10), np.log(64 << 20), n_chunks)).astype(np.int64)
    es = rng.choice([2, 4, 8], n_chunks)
    kind = rng.random(n_chunks) < 0.5
    return [(int(b) // int(e) * int(e), int(e), "vis" if k else "walk")
            for b, e, k in zip(sizes, es, kind)]
