"""The seeded input generators follow their stated recipes (CPU only, small
sizes): reproducible per seed, and with the shapes, ranges and distributions
the workloads are defined by."""
import math

import numpy as np
import pytest
import torch

from paper_2308_05199_gb300 import workloads as W


def test_every_generator_is_reproducible_and_seed_dependent():
    cases = [
        lambda s: W.sinusoids_1d(n=4096, seed=s),
        lambda s: W.grf_3d(side=16, seed=s),
        lambda s: W.stacking_rank(W.stacking_base(side=64, seed=s), 3, seed=s),
        lambda s: W.uniform(5000, s),
        lambda s: W.student_t3(5000, 0.1, s),
    ]
    for make in cases:
        a, b, c = make(7), make(7), make(8)
        assert a.dtype == torch.float32
        assert torch.equal(a, b)
        assert not torch.equal(a, c)


def test_sinusoids_are_the_eight_waves_plus_small_noise():
    n = 1 << 14
    x = W.sinusoids_1d(n=n, seed=1000, noise=0.0).double()
    y = W.sinusoids_1d(n=n, seed=1000).double()
    resid = (y - x).numpy()
    assert abs(resid.mean()) < 1e-4 and resid.std() == pytest.approx(1e-3, rel=0.05)
    # eight waves of amplitude at most 1; smooth: neighbouring samples differ
    # by at most 2 pi * sum(a_k f_k) / n <= 2 pi * 8 * 64 / n
    assert float(x.abs().max()) <= 8.0
    assert float((x[1:] - x[:-1]).abs().max()) <= 2 * math.pi * 8 * 64 / n


def test_grf_is_scaled_to_minus_one_one_with_a_k_minus_3_spectrum():
    side = 32
    x = W.grf_3d(side=side, seed=2000)
    assert x.numel() == side ** 3
    assert float(x.min()) == pytest.approx(-1.0, abs=1e-6)
    assert float(x.max()) == pytest.approx(1.0, abs=1e-6)
    f = np.fft.fftn(x.double().numpy().reshape(side, side, side))
    p = np.abs(f) ** 2
    k = np.fft.fftfreq(side)
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    # radially averaged power between |k| = 2/side and 12/side, slope in log-log
    bins = np.arange(2, 13) / side
    centres, power = [], []
    for lo, hi in zip(bins[:-1], bins[1:]):
        m = (kk >= lo) & (kk < hi)
        centres.append(math.log((lo + hi) / 2))
        power.append(math.log(p[m].mean()))
    slope = np.polyfit(centres, power, 1)[0]
    assert -3.5 < slope < -2.5


def test_stacking_ranks_share_the_base_and_differ_by_standardised_poisson_noise():
    base = W.stacking_base(side=128, seed=3000)
    r0 = W.stacking_rank(base, 0)
    r1 = W.stacking_rank(base, 1)
    d0 = (r0.double() - base.double()).numpy()
    assert abs(d0.mean()) < 2e-4
    assert d0.std() == pytest.approx(1e-2, rel=0.03)
    # the noise takes values 1e-2 (K - 50) / sqrt(50) for integer K
    k = d0 / 1e-2 * math.sqrt(50) + 50
    assert np.abs(k - np.round(k)).max() < 1e-3
    assert not torch.equal(r0, r1)


def test_message_specs_follow_the_recipe():
    specs = W.message_specs()
    assert len(specs) == 1000
    assert sum(s["dtype"] == "f32" for s in specs) == 500
    nbytes = np.array([s["n"] * (4 if s["dtype"] == "f32" else 2) for s in specs])
    assert nbytes.min() >= 4096 - 4 and nbytes.max() <= 64 << 20
    # log-uniform: the median is near the geometric mean of the limits (512 KiB)
    assert 2 ** 17 < np.median(nbytes) < 2 ** 21
    sig = np.array([s["sigma"] for s in specs])
    assert sig.min() >= 1e-4 and sig.max() <= 1e-1
    assert all(s["eb"] == pytest.approx(1e-3 * s["sigma"]) for s in specs)
    assert len({s["seed"] for s in specs}) == 1000


def test_student_t3_has_the_t3_median_and_heavy_tails():
    x = W.student_t3(400000, 2.0, 11).double().numpy() / 2.0
    # median |T| of Student-t with 3 degrees of freedom: 0.7649
    assert np.median(np.abs(x)) == pytest.approx(0.7649, abs=0.01)
    # P(|T| > 5.841) = 0.01 for 3 degrees of freedom
    assert np.mean(np.abs(x) > 5.841) == pytest.approx(0.01, abs=0.002)
    b = W.student_t3(1000, 2.0, 11, dtype=torch.bfloat16)
    assert b.dtype == torch.bfloat16
    assert W.bf16_bits(b).dtype == np.uint16


def test_uniform_is_in_the_unit_interval():
    u = W.uniform(100000, 5).numpy()
    assert u.min() >= 0.0 and u.max() < 1.0
    assert u.mean() == pytest.approx(0.5, abs=0.01)
