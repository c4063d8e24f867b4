"""Seeded synthetic density fields: the inputs both the CUDA path and the oracle read.

This module holds no arithmetic of the column-density method.  It only draws
densities with the statistics of the paper's workloads (log-normal,
multi-decade, turbulent-like, refined by density thresholds as an AMR code
would, §4.2 and §5) so that the library and the tests can be fed without the
paper's simulation outputs, which are not available.

Recipes (numpy PCG64, seed s):
  * ``lognormal_iid``: z ~ N(0,1) i.i.d. per cell, n = exp(mu + sigma z) with
    mu = ln(mean) - sigma^2/2, rescaled so that the sample mean is exactly
    ``mean``.
  * ``lognormal_grf``: g = irfft(FFT(white noise) x k^(-11/6)) with the k = 0
    mode removed, so that P(k) ~ k^(-11/3); g is normalised to zero mean and
    unit variance and exponentiated as above.
  * ``amr_leaves``: refine a uniform base grid by thresholds on the block mean
    of a finer field (level base+l cells whose mean exceeds thr[l] are split),
    the way the paper's runs refine on density.
  * ``sphere``: the uniform spherical cloud of §4.1 (n_in inside radius R,
    n_out elsewhere) sampled at cell centres.
  * ``mlp_init`` / ``mlp_inputs``: seeded initial weights of the learned
    correction's network (uniform in +-1/sqrt(fan_in), packed W1 b1 W2 b2 W3
    b3) and seeded stand-in input rows, so that both sides start from the same
    numbers.
Arrays are float32 and indexed [z, y, x] (x fastest).
"""
from __future__ import annotations

import numpy as np

PC_CM = 3.0857e18


def _rescale_lognormal(g: np.ndarray, mean: float, sigma_ln: float) -> np.ndarray:
    mu = np.log(mean) - 0.5 * sigma_ln * sigma_ln
    n = np.exp(mu + sigma_ln * g)
    n *= mean / n.mean(dtype=np.float64)
    return n.astype(np.float32)


def lognormal_iid(n: int, mean: float, sigma_ln: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((n, n, n))
    return _rescale_lognormal(z, mean, sigma_ln)


def gaussian_random_field(n: int, seed: int, slope: float = -11.0 / 3.0) -> np.ndarray:
    """Zero-mean, unit-variance field with power spectrum P(k) ~ k^slope."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n)).astype(np.float32)
    wk = np.fft.rfftn(w)
    kz = np.fft.fftfreq(n) * n
    ky = np.fft.fftfreq(n) * n
    kx = np.fft.rfftfreq(n) * n
    k2 = (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)          # |k|^(slope/2)
    amp[0, 0, 0] = 0.0
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_grf(n: int, mean: float, sigma_ln: float, seed: int) -> np.ndarray:
    return _rescale_lognormal(gaussian_random_field(n, seed), mean, sigma_ln)


def sphere(n: int, box_cm: float, radius_cm: float, n_in: float = 1000.0,
           n_out: float = 10.0, centre_cm=None) -> np.ndarray:
    c = np.full(3, 0.5 * box_cm) if centre_cm is None else np.asarray(centre_cm, float)
    h = box_cm / n
    x = (np.arange(n) + 0.5) * h
    r2 = ((x[None, None, :] - c[0]) ** 2 + (x[None, :, None] - c[1]) ** 2
          + (x[:, None, None] - c[2]) ** 2)
    return np.where(r2 <= radius_cm * radius_cm, n_in, n_out).astype(np.float32)


def _block_mean(f: np.ndarray, b: int) -> np.ndarray:
    n = f.shape[0] // b
    return f.reshape(n, b, n, b, n, b).mean(axis=(1, 3, 5), dtype=np.float64)


def amr_leaves(fine: np.ndarray, base_level: int, thresholds) -> dict:
    """Leaves of an octree refined on density.

    ``fine`` is the field at the finest level lmax = base_level + len(thresholds).
    A cell at level base_level + l (l = 0, 1, ...) is split when the mean of
    ``fine`` over it exceeds thresholds[l]; a leaf carries that mean.
    Returns dict(level int8 [n], ijk int32 [n,3] (x, y, z), rho float32 [n],
    base, lmax)."""
    nf = fine.shape[0]
    lmax = int(round(np.log2(nf)))
    assert (1 << lmax) == nf and lmax == base_level + len(thresholds)
    levels, ijks, rhos = [], [], []
    refined = None  # boolean mask of refined cells at the current level
    for l in range(base_level, lmax + 1):
        m = _block_mean(fine, 1 << (lmax - l))
        n = 1 << l
        if refined is None:
            exists = np.ones((n, n, n), dtype=bool)
        else:
            exists = np.repeat(np.repeat(np.repeat(refined, 2, 0), 2, 1), 2, 2)
        if l < lmax:
            split = exists & (m > thresholds[l - base_level])
        else:
            split = np.zeros_like(exists)
        leaf = exists & ~split
        z, y, x = np.nonzero(leaf)
        levels.append(np.full(z.shape[0], l, dtype=np.int8))
        ijks.append(np.stack([x, y, z], axis=1).astype(np.int32))
        rhos.append(m[leaf].astype(np.float32))
        refined = split
    return dict(level=np.concatenate(levels), ijk=np.concatenate(ijks),
                rho=np.concatenate(rhos), base=base_level, lmax=lmax)


def _grf_torch(n: int, seed: int, device):
    """The field g of ``gaussian_random_field`` drawn from a seeded
    torch.Generator on ``device`` (zero mean, unit variance)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    w = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float32)
    wk = torch.fft.rfftn(w)
    del w
    kz = torch.fft.fftfreq(n, device=device) * n
    kx = torch.fft.rfftfreq(n, device=device) * n
    for i in range(n):          # one z plane at a time keeps the amplitude array small
        k2 = kz[i] ** 2 + kz[:, None] ** 2 + kx[None, :] ** 2
        amp = k2.clamp_min(1e-30) ** (-11.0 / 12.0)
        if i == 0:
            amp[0, 0] = 0.0
        wk[i] *= amp
    f = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    f -= f.mean()
    f /= f.std()
    return f


def _lognormal_torch(f, mean: float, sigma_ln: float):
    import torch
    mu = float(np.log(mean) - 0.5 * sigma_ln * sigma_ln)
    f = torch.exp(mu + sigma_ln * f)
    f *= mean / float(f.double().mean())
    return f


def lognormal_grf_torch(n: int, mean: float, sigma_ln: float, seed: int, device="cuda"):
    """The recipe of ``lognormal_grf`` with torch on a GPU, for sizes numpy
    handles slowly (512^3).  Returns a float32 torch tensor [z, y, x] on
    ``device``.  Deterministic for a given device type."""
    return _lognormal_torch(_grf_torch(n, seed, device), mean, sigma_ln)


def amr_leaves_grf_torch(lmax: int, base_level: int, thresholds, mean: float, sigma_ln: float, seed: int,
                         device="cuda") -> dict:
    """The recipe of ``lognormal_grf`` + ``amr_leaves`` at sizes numpy cannot
    hold comfortably (a 1024^3 finest field), generated with torch on a GPU
    from a seeded torch.Generator.  Deterministic for a given device type."""
    import torch
    f = lognormal_grf_torch(1 << lmax, mean, sigma_ln, seed, device)
    levels, ijks, rhos = [], [], []
    refined = None  # boolean mask of refined cells at the current level
    for l in range(base_level, lmax + 1):
        m = _block_mean(fine, 1 << (lmax - l))
        n = 1 << l
        if refined is None:
            exists = np.ones((n, n, n), dtype=bool)
        else:
            exists = np.repeat(np.repeat(np.repeat(refined, 2, 0), 2, 1), 2, 2)
        if l < lmax:
            split = exists & (m > thresholds[l - base_level])
        else:
            split = np.zeros_like(exists)
        leaf = exists & ~split
        z, y, x = np.nonzero(leaf)
        levels.append(np.full(z.shape[0], l, dtype=np.int8))
        ijks.append(np.stack([x, y, z], axis=1).astype(np.int32))
        rhos.append(m[leaf].astype(np.float32))
        refined = split
    return dict(level=np.concatenate(levels), ijk=np.concatenate(ijks),
                rho=np.concatenate(rhos), base=base_level, lmax=lmax)


def amr_leaves_grf_torch(lmax: int, base_level: int, thresholds, mean: float, sigma_ln: float, seed: int,
                         device="cuda") -> dict:
    """The recipe of ``lognormal_grf`` + ``amr_leaves`` at sizes numpy cannot
    hold comfortably (a 1024^3 finest field), generated with torch on a GPU
    from a seeded torch.Generator.  Deterministic for a given device type."""
    import torch
    n = 1 << lmax
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    w = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float32)
    wk = torch.fft.rfftn(w)
    del w
    kz = torch.fft.fftfreq(n, device=device) * n
    kx = torch.fft.rfftfreq(n, device=device) * n
    for i in range(n):          # one z plane at a time keeps the amplitude array small
        k2 = kz[i] ** 2 + kz[:, None] ** 2 + kx[None, :] ** 2
        amp = k2.clamp_min(1e-30) ** (-11.0 / 12.0)
        if i == 0:
            amp[0, 0] = 0.0
        wk[i] *= amp
    f = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    f -= f.mean()
    f /= f.std()
    mu = float(np.log(mean) - 0.5 * sigma_ln * sigma_ln)
    f = torch.exp(mu + sigma_ln * f)
    f *= mean / float(f.double().mean())
    levels, ijks, rhos = [], [], []
    refined = None
    x = f[None, None]
    for l in range(base_level, lmax + 1):
        b = 1 << (lmax - l)
        m = torch.nn.functional.avg_pool3d(x, b)[0, 0] if b > 1 else f
        if refined is None:
            exists = torch.ones_like(m, dtype=torch.bool)
        else:
            exists = refined.repeat_interleave(2, 0).repeat_interleave(2, 1).repeat_interleave(2, 2)
        split = exists & (m > thresholds[l - base_level]) if l < lmax else torch.zeros_like(exists)
        leaf = exists & ~split
        idx = torch.nonzero(leaf)
        levels.append(np.full(idx.shape[0], l, dtype=np.int8))
        ijks.append(idx.flip(1).to(torch.int32).cpu().numpy())
        rhos.append(m[leaf].float().cpu().numpy())
        refined = split
    return dict(level=np.concatenate(levels), ijk=np.concatenate(ijks), rho=np.concatenate(rhos),
                base=base_level, lmax=lmax)


def mlp_init(n_dir: int, hidden: int, seed: int, out_scale: float = 1.0, slots: int = 8) -> np.ndarray:
    """Seeded initial parameters of the learned correction's network, packed
    W1 [hidden, slots*n_dir+1], b1, W2 [hidden, hidden], b2, W3 [n_dir, hidden],
    b3; every entry U(-1/sqrt(fan_in), 1/sqrt(fan_in)), the last layer scaled
    by out_scale.  float32."""
    rng = np.random.default_rng(seed)
    n_in = slots * n_dir + 1
    parts = []
    for rows, fan_in, scale in ((hidden, n_in, 1.0), (hidden, hidden, 1.0), (n_dir, hidden, out_scale)):
        b = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-b, b, size=rows * fan_in) * scale)
        parts.append(rng.uniform(-b, b, size=rows) * scale)
    return np.concatenate(parts).astype(np.float32)


def mlp_inputs(n: int, n_in: int, seed: int, centre: float = 42.0, spread: float = 3.0) -> np.ndarray:
    """Seeded stand-in input rows [n, n_in] (float32) with the scale of log
    column densities in cm^-2: N(centre, spread^2) per entry."""
    rng = np.random.default_rng(seed)
    return (centre + spread * rng.standard_normal((n, n_in))).astype(np.float32)
