"""Seeded synthetic inputs for the five workloads.

This module only draws data; it holds none of the codec's arithmetic, so the
CUDA path and the CPU oracle can both consume what it makes.  Small parameter
draws (frequencies, amplitudes, phases, message sizes) come from numpy's PCG64
and are identical on every machine; bulk noise comes from a seeded torch
generator on the requested device.

Stand-ins (the paper's RTM volumes and image-stacking inputs are not
available): workload 1 is a smooth 1-D signal, workload 2 a 3-D Gaussian random
field with a k^-3 power spectrum like a seismic volume, workload 3 the
image-stacking Allreduce of Sec. 4.5 (a shared image plus per-rank noise),
workload 4 gradient-bucket-like messages of uneven size and mixed precision.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _tgen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


# ---- workload 1: sum of 8 sinusoids + Gaussian noise ----------------------

def sinusoids_1d(n: int = 1 << 20, seed: int = 1000, noise: float = 1e-3,
                 device="cpu") -> torch.Tensor:
    """x_i = sum_k a_k sin(2 pi f_k i / n + phi_k) + N(0, noise^2), f_k in
    [1, 64] cycles, a_k in [0.1, 1], phi_k in [0, 2 pi)."""
    r = _rng(seed)
    f = r.uniform(1.0, 64.0, 8)
    a = r.uniform(0.1, 1.0, 8)
    ph = r.uniform(0.0, 2 * math.pi, 8)
    i = torch.arange(n, dtype=torch.float64, device=device)
    x = torch.zeros(n, dtype=torch.float64, device=device)
    for k in range(8):
        x += a[k] * torch.sin(2 * math.pi * f[k] * i / n + ph[k])
    x += noise * torch.randn(n, generator=_tgen(device, seed), dtype=torch.float64,
                             device=device)
    return x.to(torch.float32)


# ---- workload 2: 3-D Gaussian random field, P(k) ~ k^-3 -----------------

def grf_3d(side: int = 512, seed: int = 2000, device="cpu") -> torch.Tensor:
    """White noise shaped in Fourier space by amplitude k^-3/2 (power k^-3),
    k = 0 removed, min-max scaled to [-1, 1]; returned flat in C order."""
    g = _tgen(device, seed)
    w = torch.randn((side, side, side), generator=g, dtype=torch.float32, device=device)
    W = torch.fft.rfftn(w)
    del w
    kx = torch.fft.fftfreq(side, device=device).to(torch.float32)
    kz = torch.fft.rfftfreq(side, device=device).to(torch.float32)
    k2 = (kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    k2[0, 0, 0] = 1.0
    amp = k2.pow(-0.75)  # |k|^-3/2
    amp[0, 0, 0] = 0.0
    W *= amp
    del amp, k2
    x = torch.fft.irfftn(W, s=(side, side, side))
    del W
    lo, hi = x.min(), x.max()
    x = (x - lo) * (2.0 / (hi - lo)) - 1.0
    return x.reshape(-1).contiguous().to(torch.float32)


# ---- workload 3: image stacking, shared base + per-rank Poisson noise ----

def _base_params(seed: int):
    r = _rng(seed)
    return (r.uniform(1.0, 64.0, 8), r.uniform(1.0, 64.0, 8), r.uniform(0.1, 1.0, 8),
            r.uniform(0.0, 2 * math.pi, 8))


def stacking_base(side: int = 8192, seed: int = 3000, device="cpu") -> torch.Tensor:
    """2-D analog of workload 1: sum of 8 plane waves in (u, v)."""
    fu, fv, a, ph = _base_params(seed)
    u = torch.arange(side, dtype=torch.float64, device=device) / side
    img = torch.zeros((side, side), dtype=torch.float64, device=device)
    for k in range(8):
        img += a[k] * torch.sin(2 * math.pi * (fu[k] * u[None, :] + fv[k] * u[:, None]) + ph[k])
    return img.reshape(-1).to(torch.float32)


def stacking_rank(base: torch.Tensor, rank: int, seed: int = 3000, lam: float = 50.0,
                  scale: float = 1e-2) -> torch.Tensor:
    """Rank image = base + scale * (K - lam) / sqrt(lam), K ~ Poisson(lam)."""
    g = _tgen(base.device, seed * 1000 + 1 + rank)
    rate = torch.full_like(base, lam)
    K = torch.poisson(rate, generator=g)
    return (base + scale * (K - lam) / math.sqrt(lam)).to(torch.float32)


# ---- workload 4: uneven mixed-precision messages ------------------------

def message_specs(m: int = 1000, lo_bytes: int = 4096, hi_bytes: int = 64 << 20,
                  seed: int = 4000):
    """Sizes log-uniform in [lo, hi] bytes, half FP32 / half BF16 in random
    order, sigma log-uniform in [1e-4, 1e-1]; eb = 1e-3 sigma."""
    r = _rng(seed)
    nbytes = np.exp(r.uniform(math.log(lo_bytes), math.log(hi_bytes), m))
    kinds = np.array([0] * (m // 2) + [1] * (m - m // 2))
    r.shuffle(kinds)
    sigma = np.exp(r.uniform(math.log(1e-4), math.log(1e-1), m))
    specs = []
    for i in range(m):
        es = 4 if kinds[i] == 0 else 2
        n = max(1, int(nbytes[i]) // es)
        specs.append(dict(n=n, dtype="f32" if kinds[i] == 0 else "bf16",
                          sigma=float(sigma[i]), eb=float(1e-3 * sigma[i]), seed=seed + 1 + i))
    return specs


def uniform(n: int, seed: int, device="cpu") -> torch.Tensor:
    """U[0, 1) FP32: the uniformly distributed synthetic data of the paper's
    compressor characterization over message sizes (Sec. 3.2.2)."""
    return torch.rand(n, generator=_tgen(device, seed), dtype=torch.float32, device=device)


def student_t3(n: int, sigma: float, seed: int, device="cpu",
               dtype=torch.float32) -> torch.Tensor:
    """sigma * T with T ~ Student-t(3) = Z / sqrt(chi2_3 / 3)."""
    g = _tgen(device, seed)
    z = torch.randn(4, n, generator=g, dtype=torch.float32, device=device)
    chi2 = (z[1:] ** 2).sum(0)
    t = z[0] / torch.sqrt(chi2 / 3.0)
    return (sigma * t).to(dtype)


def message(spec: dict, device="cpu") -> torch.Tensor:
    dt = torch.float32 if spec["dtype"] == "f32" else torch.bfloat16
    return student_t3(spec["n"], spec["sigma"], spec["seed"], device=device, dtype=dt)


def bf16_bits(t: torch.Tensor) -> np.ndarray:
    """BF16 tensor -> numpy uint16 bit patterns (how the oracle takes BF16)."""
    return t.detach().cpu().contiguous().view(torch.int16).numpy().view(np.uint16)
