"""Planted mistakes in the generator, hybrid-correction and local-Lagrangian oracles
must fail at least one of their pins (on the CPU, for the duration of one test):
a wrong Philox multiplier, a missing key bump, a uniform without its half-unit
offset, a Box-Muller pair built from one trigonometric function, a sign error in
the finite-difference gradient symbol of the hybrid correction, a dropped factor i
of the exact gradient, density determinants with the sign of the Hessian or the
mixed derivatives wrong, and in the multi-scale density a non-conservative or
mirrored tricubic interpolation, Hoffman-Ribak without its 1/sqrt(8), a convolution
without the cell-volume factor and a nest without the parent's long waves.
"""

import numpy as np
import pytest

import oracle.hybrid as hyb
import oracle.lpt as lpt
import oracle.noise as noise
from tests import test_oracle_hybrid as t_hyb
from tests import test_oracle_lla as t_lla
from tests import test_oracle_noise as t_noise


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_wrong_philox_multiplier_is_caught(monkeypatch):
    monkeypatch.setattr(noise, "_M0", np.uint64(0xD2511F55))
    for row in t_noise._kat_rows():
        _fails(t_noise.test_philox_known_answers, row)


def test_missing_key_bump_is_caught(monkeypatch):
    monkeypatch.setattr(noise, "_W1", np.uint32(0))
    for row in t_noise._kat_rows():
        _fails(t_noise.test_philox_known_answers, row)


def test_uniform_without_half_offset_is_caught(monkeypatch):
    def no_offset(a, b):
        hi = (np.asarray(a, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
        lo = (np.asarray(b, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
        return (hi * 67108864.0 + lo) / 9007199254740992.0

    monkeypatch.setattr(t_noise, "uniform53", no_offset)
    _fails(t_noise.test_uniforms_open_interval_and_extremes)


def test_box_muller_with_one_function_is_caught(monkeypatch):
    pytest.importorskip("scipy.stats")
    good = noise.white_noise

    def cos_only(seed, n, stream=0):
        z = good(seed, n + (n & 1), stream)
        r = np.hypot(z[0::2], z[1::2])
        ang = np.arctan2(z[1::2], z[0::2])
        out = np.empty_like(z)
        out[0::2] = r * np.cos(ang)
        out[1::2] = r * np.cos(ang)     # should be the sine
        return out[:n]

    monkeypatch.setattr(t_noise, "white_noise", cos_only)
    _fails(t_noise.test_normal_deviates_have_the_standard_normal_distribution)


def test_hybrid_gradient_symbol_sign_is_caught(monkeypatch):
    good = hyb.gradient_symbol_1d
    monkeypatch.setattr(hyb, "gradient_symbol_1d", lambda order, t: -good(order, t))
    _fails(t_hyb.test_periodic_level_becomes_exact, 4, (16, 16, 16))


def test_hybrid_without_factor_i_is_caught(monkeypatch):
    def real_multiplier(f, h, order, pad=True):
        # the exact gradient taken as k_j / k^2 instead of i k_j / k^2
        f = np.asarray(f, dtype=np.float64)
        n = f.shape
        shape = tuple(2 * m for m in n) if pad else n
        grid = np.zeros(shape)
        grid[:n[0], :n[1], :n[2]] = f
        fk = np.fft.fftn(grid)
        t = np.meshgrid(*[2.0 * np.pi * np.fft.fftfreq(m) for m in shape], indexing="ij")
        k = [ta / h for ta in t]
        ksq = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
        lt = sum(hyb.laplacian_symbol_1d(order, ta) for ta in t) / (h * h)
        zero = ksq == 0.0
        ksq[zero] = 1.0
        lt[zero] = 1.0
        out = []
        for j in range(3):
            mult = k[j] / ksq + 1j * hyb.gradient_symbol_1d(order, t[j]) / h / lt
            mult[zero] = 0.0
            out.append(np.fft.ifftn(mult * fk).real[:n[0], :n[1], :n[2]].copy())
        return out

    monkeypatch.setattr(t_hyb, "hybrid_correction", real_multiplier)
    _fails(t_hyb.test_periodic_level_becomes_exact, 2, (12, 10, 14))


def test_lla_with_the_hessian_sign_flipped_is_caught(monkeypatch):
    good = lpt.second_derivatives

    def flipped(lev):
        diag, mixed = good(lev)
        return [-d for d in diag], {k: -v for k, v in mixed.items()}

    monkeypatch.setattr(lpt, "second_derivatives", flipped)
    _fails(t_lla.test_plane_wave, 4)


def test_lla_without_mixed_derivatives_is_caught(monkeypatch):
    good = lpt.second_derivatives

    def no_mixed(lev):
        diag, mixed = good(lev)
        return diag, {k: np.zeros_like(v) for k, v in mixed.items()}

    monkeypatch.setattr(lpt, "second_derivatives", no_mixed)
    _fails(t_lla.test_diagonal_mode, 6)


# ---- multi-scale density (Sec. 2.3) ----

import oracle.density as dens  # noqa: E402
from tests import test_oracle_density as t_dens  # noqa: E402


def test_tricubic_without_conservation_is_caught(monkeypatch):
    # no shift restoring each parent's mean: the plain tricubic values
    monkeypatch.setattr(dens, "inject", lambda c: np.zeros(tuple(2 * m for m in c.shape)))
    _fails(t_dens.test_tricubic_conservative_interpolation)


def test_tricubic_with_swapped_parities_is_caught(monkeypatch):
    good = dens.cubic_weights

    def swapped(t):
        return good(1.0 - t)

    monkeypatch.setattr(dens, "cubic_weights", swapped)
    _fails(t_dens.test_tricubic_conservative_interpolation)


def test_hoffman_ribak_without_rescaling_is_caught(monkeypatch):
    def unscaled(geom, seed):
        mu = [noise.white_noise(seed, int(np.prod(geom.base_n)), 0).reshape(tuple(geom.base_n))]
        for lvl, nest in enumerate(geom.nests, start=1):
            own = noise.white_noise(seed, int(np.prod(nest.n)), lvl).reshape(tuple(nest.n))
            mu.append(own - dens.inject(dens.children_mean(own))
                      + dens.inject(mu[-1][dens._region(nest)]))     # missing 1/sqrt(8)
        return mu

    monkeypatch.setattr(t_dens, "level_noise", unscaled)
    _fails(t_dens.test_hoffman_ribak_constraint_and_variance)


def test_convolution_without_cell_volume_factor_is_caught(monkeypatch):
    good = dens.convolve_periodic

    def no_volume(noise_, h, sqrt_p, dk):
        return good(noise_, h, sqrt_p, dk) * h ** 1.5

    monkeypatch.setattr(dens, "convolve_periodic", no_volume)
    _fails(t_dens.test_single_level_is_the_periodic_field)


def test_nest_without_the_parent_contribution_is_caught(monkeypatch):
    good = dens.tricubic_conservative
    monkeypatch.setattr(dens, "tricubic_conservative",
                        lambda parent, off, n: np.zeros_like(good(parent, off, n)))
    _fails(t_dens.test_nest_carries_the_parent_large_scales)
