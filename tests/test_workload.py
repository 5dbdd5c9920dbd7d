"""The seeded input generators (no solver arithmetic), on the CPU.

The device field generator pads its FFT grid to twice the size rounded up to
a multiple of `pad`; padding that changes nothing gives the same field, and
any padding keeps the target variance and correlation of the covariance.
"""
import numpy as np
import pytest

from paper_2001_05798_gb300 import workload as wl

torch = pytest.importorskip("torch")


def test_padding_to_twice_the_size_is_the_default_recipe():
    a = wl.lnk_field_device(16, 16, 16, 2.0, 4.0, 7, device="cpu")
    b = wl.lnk_field_device(16, 16, 16, 2.0, 4.0, 7, device="cpu", pad=32)  # 2 * 16 = 32 already
    assert torch.equal(a, b)


@pytest.mark.parametrize("pad", [1, 32, 48])
def test_padded_fields_keep_variance_and_correlation(pad):
    var, corr, n = 1.5, 2.0, 40
    vals, lag1 = [], []
    for seed in range(6):
        f = wl.lnk_field_device(n, n, n, var, corr, 100 + seed, device="cpu", pad=pad).numpy().reshape(n, n, n)
        vals.append(f.var())
        lag1.append(np.mean(f[:, :, 1:] * f[:, :, :-1]) - f.mean() ** 2)
    assert np.mean(vals) == pytest.approx(var, rel=0.15)
    # exponential covariance at one cell: var * exp(-1 / corr)
    assert np.mean(lag1) == pytest.approx(var * np.exp(-1.0 / corr), rel=0.2)


def test_serving_requests_are_reproducible():
    a = wl.serving_requests(count=50, seed=4)
    b = wl.serving_requests(count=50, seed=4)
    assert a == b
    sides = [r["side"] for r in a]
    assert min(sides) >= 32 and max(sides) <= 160
