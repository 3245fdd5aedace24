"""Closed-form results the paper uses to validate the scheme (Sec. 3).

TEST INFRASTRUCTURE (see the package docstring).  Plain numpy.

* Eq. 43-45: Miller-Scriven viscous correction to Lamb's n-th mode
  frequency of an oscillating drop.
* Laplace's law for a spherical drop: p_in - p_out = 2 sigma / R.
* Eq. 42: the equilibrium density profile across a flat/large interface.
* Rayleigh-Plateau criterion for a perturbed thread: unstable iff k < 1 (Sec. 3.3).
"""
from __future__ import annotations

import math


def lamb_frequency(n, Re, rho_l, rho_g, sigma):
    """Eq. 44: omega_n^* = sqrt(n(n-1)(n+1)(n+2) sigma / (Re^3 [n rho_g + (n+1) rho_l]))."""
    return math.sqrt(n * (n - 1) * (n + 1) * (n + 2) * sigma /
                     (Re ** 3 * (n * rho_g + (n + 1) * rho_l)))


def miller_scriven_alpha(n, Re, rho_l, rho_g, nu_l, nu_g):
    """Eq. 45."""
    num = (2 * n + 1) ** 2 * rho_l * rho_g * math.sqrt(nu_l * nu_g)
    den = (math.sqrt(2.0) * Re * (n * rho_g + (n + 1) * rho_l) *
           (rho_l * math.sqrt(nu_l) + rho_g * math.sqrt(nu_g)))
    return num / den


def miller_scriven_frequency(n, Re, rho_l, rho_g, nu_l, nu_g, sigma):
    """Eq. 43: omega_n = omega* - 0.5 alpha sqrt(omega*) + 0.25 alpha^2."""
    w = lamb_frequency(n, Re, rho_l, rho_g, sigma)
    a = miller_scriven_alpha(n, Re, rho_l, rho_g, nu_l, nu_g)
    return w - 0.5 * a * math.sqrt(w) + 0.25 * a * a


def equilibrium_radius(Rz, Rr):
    """Sec. 3.2: R_e = (R_r^2 R_z)^(1/3) from volume conservation."""
    return (Rr * Rr * Rz) ** (1.0 / 3.0)


def laplace_jump(sigma, R):
    """Young-Laplace pressure jump of a sphere (two equal principal curvatures)."""
    return 2.0 * sigma / R


def density_profile(d, R, W, rho_l, rho_g):
    """Eq. 42 as a function of the distance d from the drop centre."""
    return 0.5 * (rho_l + rho_g) + 0.5 * (rho_l - rho_g) * math.tanh(2.0 * (R - d) / W)


def rayleigh_unstable(R, wavelength):
    """Sec. 3.3: a thread of radius R is unstable iff k = 2 pi R / lambda < 1."""
    return 2.0 * math.pi * R / wavelength < 1.0
