"""GPU density generator (Sec. 2.1: delta = IFFT[A(|k|) FFT[mu]]) against the oracle
(oracle/noise.py): the white noise element by element (the Philox words decide
every value, so any integer mismatch would show as an O(1) difference; the
remaining difference is the rounding of log, sqrt and the angle), and the
periodic field on cubic, ragged and odd grids with a BBKS amplitude table."""

import numpy as np
import pytest

from oracle.noise import gaussian_field, white_noise
from synthetic.spectra import BBKSPower, PowerLaw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    from paper_1103_6031_gb300 import mg
    pkg.mg = mg
    return pkg


def bbks_table(h, shape, nt=4096):
    kmax = 2 * np.pi / h * np.sqrt(3) * 0.5 * 1.01
    dk = kmax / (nt - 1)
    k = np.arange(nt) * dk
    p = BBKSPower()(np.maximum(k, 1e-12))
    amp = np.sqrt(p / h ** 3)
    amp[0] = 0.0
    return amp, dk


@pytest.mark.parametrize("seed,n", [(1, 1000001), (2 ** 40 + 17, 4096), (0, 1), (7, 2)])
def test_white_noise_matches_oracle(lib, seed, n):
    z = lib.white_noise(seed, n).cpu().numpy()
    ref = white_noise(seed, n)
    assert z.shape == ref.shape
    assert np.abs(z - ref).max() < 1e-12


@pytest.mark.parametrize("shape", [(64, 64, 64), (48, 40, 36), (35, 33, 31), (128, 128, 128)])
def test_field_matches_oracle(lib, shape):
    import torch
    h = 100.0 / 128
    amp, dk = bbks_table(h, shape)
    noise = white_noise(5, int(np.prod(shape))).reshape(shape)
    ref = gaussian_field(noise, h, amp, dk)
    f = lib.Field(shape, h, amp, dk)
    out = f.convolve(torch.from_numpy(noise).cuda()).cpu().numpy()
    f.close()
    err = np.sqrt(np.sum((out - ref) ** 2) / np.sum(ref ** 2))
    assert err < 1e-12, err


def test_generate_equals_convolved_noise(lib):
    import torch
    shape, h = (40, 48, 64), 0.5
    k = np.arange(2000) * 0.01
    amp = np.sqrt(PowerLaw(-2.0)(np.maximum(k, 1e-12)))
    amp[0] = 0.0
    f = lib.Field(shape, h, amp, 0.01)
    a = f.generate(123)
    b = f.convolve(lib.white_noise(123, int(np.prod(shape))).reshape(shape))
    assert torch.equal(a, b)
    ref = gaussian_field(white_noise(123, int(np.prod(shape))).reshape(shape), h, amp, 0.01)
    out = a.cpu().numpy()
    assert np.sqrt(np.sum((out - ref) ** 2) / np.sum(ref ** 2)) < 1e-12
    f.close()


def test_generator_rejects_bad_arguments(lib):
    from paper_1103_6031_gb300.mg import MGError
    with pytest.raises(MGError):
        lib.Field((1, 8, 8), 1.0, np.ones(4), 0.1)
    with pytest.raises(MGError):
        lib.Field((8, 8, 8), 1.0, np.ones(1), 0.1)
    with pytest.raises(MGError):
        lib.Field((8, 8, 8), -1.0, np.ones(4), 0.1)


MULTI = [
    ("L2_cube", lambda: __import__("synthetic").Geometry(
        (32, 32, 32), 64.0, 6, (__import__("synthetic").NestSpec((32, 32, 32), (8, 8, 8)),))),
    ("L3_o4", lambda: __import__("synthetic").small_zoom(24, ((20, 7), (16, 6)), order=4, box=50.0)),
    ("aniso", lambda: __import__("synthetic").Geometry(
        (24, 32, 40), 24.0, 6, (__import__("synthetic").NestSpec((14, 20, 18), (7, 6, 9)),))),
]


@pytest.mark.parametrize("name,make", MULTI, ids=[m[0] for m in MULTI])
def test_multiscale_density_matches_oracle(lib, name, make):
    from oracle.density import multiscale
    geom = make()
    dk = 0.01
    k = np.arange(6000) * dk
    table = np.sqrt(BBKSPower()(np.maximum(k, 1e-12)))
    table[0] = 0.0
    cfg = lib.config_from_geometry(geom)
    got = lib.mg.density_multiscale(cfg, 2 ** 33 + 7, table, dk)
    want = multiscale(geom, 2 ** 33 + 7, table, dk)
    for g, w in zip(got, want):
        g = g.cpu().numpy()
        err = np.sqrt(np.sum((g - w) ** 2) / np.sum(w * w))
        assert err < 1e-11, (name, err)
