"""Power spectra for the synthetic source fields.

P(k) = alpha k^{n_s} T^2(k) (Sec. 2.1, P(k) equation).  The paper takes T(k)
from a Boltzmann solver or a fitting formula; the stand-in workloads use the
BBKS fitting formula (Bardeen, Bond, Kaiser & Szalay 1986, their eq. G3) with
the shape parameter of Sugiyama (1995), normalised to sigma_8 with a top-hat
window of radius 8 Mpc/h and scaled to the target redshift with the linear
growth factor of a flat LCDM cosmology.  Units: k in h/Mpc, lengths in Mpc/h.
"""

from dataclasses import dataclass

import numpy as np
from scipy import integrate


@dataclass(frozen=True)
class Cosmology:
    omega_m: float = 0.276
    omega_b: float = 0.045
    h: float = 0.70
    n_s: float = 0.96
    sigma_8: float = 0.81
    z: float = 50.0


def _bbks_transfer(k, cosmo):
    """BBKS transfer function T(q), q = k / Gamma with Sugiyama's Gamma."""
    gamma = cosmo.omega_m * cosmo.h * np.exp(
        -cosmo.omega_b * (1.0 + np.sqrt(2.0 * cosmo.h) / cosmo.omega_m))
    q = np.asarray(k, dtype=np.float64) / gamma
    q = np.maximum(q, 1e-30)
    poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
    return np.log1p(2.34 * q) / (2.34 * q) * poly ** -0.25


def _tophat(x):
    x = np.asarray(x, dtype=np.float64)
    small = x < 1e-4
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(small, 1.0 - x * x / 10.0, w)


def growth_factor(a, omega_m):
    """Linear growing mode of flat LCDM, D(a) ∝ H(a) ∫_0^a da' / (a' H(a'))^3."""
    omega_l = 1.0 - omega_m

    def hubble(x):
        return np.sqrt(omega_m / x ** 3 + omega_l)

    integral, _ = integrate.quad(lambda x: 1.0 / (x * hubble(x)) ** 3, 0.0, a,
                                 epsabs=0.0, epsrel=1e-12, limit=200)
    return 2.5 * omega_m * hubble(a) * integral


class BBKSPower:
    """P(k) = A k^{n_s} T_BBKS^2(k) normalised to sigma_8 at z=0, scaled by D(z)^2."""

    def __init__(self, cosmo: Cosmology = Cosmology()):
        self.cosmo = cosmo
        unnorm = self._sigma2(8.0, 1.0)
        a = 1.0 / (1.0 + cosmo.z)
        growth = growth_factor(a, cosmo.omega_m) / growth_factor(1.0, cosmo.omega_m)
        self.amplitude = cosmo.sigma_8 ** 2 / unnorm * growth ** 2

    def _shape(self, k):
        k = np.asarray(k, dtype=np.float64)
        return k ** self.cosmo.n_s * _bbks_transfer(k, self.cosmo) ** 2

    def _sigma2(self, radius, amplitude):
        lnk = np.linspace(np.log(1e-5), np.log(1e3), 20001)
        k = np.exp(lnk)
        integrand = amplitude * self._shape(k) * _tophat(k * radius) ** 2 * k ** 3
        return np.trapezoid(integrand, lnk) / (2.0 * np.pi ** 2)

    def sigma(self, radius):
        return np.sqrt(self._sigma2(radius, self.amplitude))

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        out = self.amplitude * self._shape(np.where(k > 0, k, 1.0))
        return np.where(k > 0, out, 0.0)


class PowerLaw:
    """P(k) ∝ k^index with P(0) = 0 (the unit amplitude is rescaled afterwards)."""

    def __init__(self, index: float = -2.0):
        self.index = index

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        return np.where(k > 0, np.where(k > 0, k, 1.0) ** self.index, 0.0)
