"""Pins of the generator oracle (oracle/noise.py): the counter-based generator
against its published known-answer vectors, the uniform and normal deviates
against their distributions, and the periodic field against closed forms for
single Fourier modes (Sec. 2.1: delta(k) = A(|k|) mu(k))."""

import os

import numpy as np
import pytest

from oracle.noise import amplitude, gaussian_field, kmag, philox4x32_10, uniform53, white_noise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            rows.append([int(w, 16) for w in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat_rows(), ids=lambda r: "%08x" % r[0])
def test_philox_known_answers(row):
    ctr = np.array(row[0:4], dtype=np.uint32).reshape(4, 1)
    key = np.array(row[4:6], dtype=np.uint32).reshape(2, 1)
    out = philox4x32_10(ctr, key)[:, 0]
    assert [int(v) for v in out] == row[6:10]


def test_philox_vectorised_equals_one_at_a_time():
    rng = np.random.Generator(np.random.PCG64(3))
    ctr = rng.integers(0, 2 ** 32, size=(4, 17), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(2, 17), dtype=np.uint64).astype(np.uint32)
    all_at_once = philox4x32_10(ctr, key)
    for i in range(17):
        one = philox4x32_10(ctr[:, i:i + 1], key[:, i:i + 1])[:, 0]
        assert np.array_equal(one, all_at_once[:, i])


def test_uniforms_open_interval_and_extremes():
    # the extreme words give the smallest and largest representable values, never 0 or 1
    assert uniform53(0, 0) == 0.5 / 2 ** 53
    assert uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 0.5 / 2 ** 53
    u = uniform53(np.arange(0, 2 ** 32, 2 ** 20, dtype=np.uint64), 12345)
    assert np.all(np.diff(u) > 0)


def test_normal_deviates_have_the_standard_normal_distribution():
    stats = pytest.importorskip("scipy.stats")
    n = 1 << 20
    z = white_noise(7, n)
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair, and neighbouring pairs, are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5.0 / np.sqrt(n / 2)
    assert abs(np.corrcoef(z[0:-2:2], z[2::2])[0, 1]) < 5.0 / np.sqrt(n / 2)
    # the radius r = sqrt(z0^2 + z1^2) of a pair is Rayleigh: r^2 / 2 ~ Exp(1)
    r2 = z[0::2] ** 2 + z[1::2] ** 2
    assert stats.kstest(r2 / 2.0, "expon").pvalue > 1e-3


def test_noise_is_counter_based_and_keyed():
    a = white_noise(11, 1001)
    assert np.array_equal(white_noise(11, 20), a[:20])        # a prefix of the same stream
    b = white_noise(12, 1001)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15                  # another seed, another stream
    big = white_noise(2 ** 40 + 5, 64)                          # 64-bit seeds use both key words
    assert not np.array_equal(big, white_noise(5, 64))


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 10, 14), (9, 8, 7)])
def test_single_mode_passes_with_its_amplitude(shape):
    h = 0.37
    x = [np.arange(n) for n in shape]
    i, j, k = np.meshgrid(*x, indexing="ij")
    m = (1, 2, 3)
    phase = 2 * np.pi * (m[0] * i / shape[0] + m[1] * j / shape[1] + m[2] * k / shape[2])
    noise = np.cos(phase)
    k0 = 2 * np.pi * np.sqrt(sum((m[a] / (shape[a] * h)) ** 2 for a in range(3)))
    dk = 0.05
    table = 2.5 + 0.3 * np.arange(400) * dk        # A(|k|) = 2.5 + 0.3 |k|, linear: exact
    out = gaussian_field(noise, h, table, dk)
    np.testing.assert_allclose(out, (2.5 + 0.3 * k0) * noise, atol=1e-12)


def test_field_zero_mode_and_beyond_table():
    noise = np.ones((8, 8, 8)) * 3.0
    assert np.abs(gaussian_field(noise, 1.0, np.ones(100), 0.1)).max() < 1e-13   # k = 0 removed
    z = white_noise(3, 512).reshape(8, 8, 8)
    # a table that ends below the grid's smallest |k| kills every mode
    kmin = 2 * np.pi / 8.0
    assert np.abs(gaussian_field(z, 1.0, np.ones(10), kmin / 20.0)).max() < 1e-13


def test_white_noise_field_has_the_table_spectrum():
    shape, h, dk = (32, 32, 32), 1.0, 0.01
    table = np.exp(-np.arange(2000) * dk)          # A(|k|) = exp(-|k|)
    z = white_noise(21, np.prod(shape)).reshape(shape)
    d = gaussian_field(z, h, table, dk)
    a = amplitude(kmag(shape, h), table, dk)
    a.flat[0] = 0.0
    # E|delta_k|^2 = N A^2 for unit white noise; the ratio averages to 1
    sel = a > 0
    ratio = np.abs(np.fft.fftn(d))[sel] ** 2 / (np.prod(shape) * a[sel] ** 2)
    assert abs(ratio.mean() - 1.0) < 0.02
