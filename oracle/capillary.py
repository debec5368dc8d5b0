"""Closed-form interface position of the small-amplitude capillary wave between
two fluids of equal kinematic viscosity (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU legs may load it;
the product library never does.

Sec. "Capillary wave in 2D", Eq. cap-wave-analytical: the scaled deviation
h~(t) = (h_eq - h_0(t)) / A_p of the interface from its equilibrium, with
t' = omega_0 t, omega_0^2 = sigma k^3 / (rho_L + rho_G), eps = nu k^2 /
omega_0, beta = rho_L rho_G / (rho_L + rho_G)^2, is

  h~ = 4 (1 - 4 beta) eps^2 / (8 (1 - 4 beta) eps^2 + 1) erfc(sqrt(eps t'))
       + sum_i z_i omega_0^2 / (Z_i (z_i^2 - eps omega_0))
               exp((z_i^2 - eps omega_0) t) erfc(z_i sqrt(t)),

z_i the four roots of the quartic printed with it and Z_i the products of
their differences.  The product exp(z^2 t) erfc(z sqrt t) is evaluated as
the Faddeeva function w(i z sqrt t), which stays finite where its two
factors would overflow.
"""
from __future__ import annotations

import math

import numpy as np


def roots(omega0: float, eps: float, beta: float) -> np.ndarray:
    """The four roots of z^4 - 4 beta sqrt(eps w) z^3 + 2 (1 - 6 beta) eps w z^2
    + 4 (1 - 3 beta) (eps w)^(3/2) z + (1 - 4 beta) (eps w)^2 + w^2 = 0, w = omega_0."""
    a = eps * omega0
    coef = [1.0, -4.0 * beta * math.sqrt(a), 2.0 * (1.0 - 6.0 * beta) * a,
            4.0 * (1.0 - 3.0 * beta) * a ** 1.5, (1.0 - 4.0 * beta) * a * a + omega0 * omega0]
    return np.roots(coef).astype(complex)


def h_tilde(t, sigma: float, rho_l: float, rho_g: float, nu: float, k: float):
    """h~ at the times t (array), in the units of sigma, rho, nu and k."""
    from scipy.special import erfc, wofz
    t = np.asarray(t, dtype=float)
    omega0 = math.sqrt(sigma * k ** 3 / (rho_l + rho_g))
    eps = nu * k * k / omega0
    beta = rho_l * rho_g / (rho_l + rho_g) ** 2
    z = roots(omega0, eps, beta)
    Z = np.array([np.prod([z[j] - z[i] for j in range(4) if j != i]) for i in range(4)])
    a = eps * omega0
    first = 4.0 * (1.0 - 4.0 * beta) * eps ** 2 / (8.0 * (1.0 - 4.0 * beta) * eps ** 2 + 1.0) * erfc(np.sqrt(a * t))
    s = np.zeros(t.shape, dtype=complex)
    for i in range(4):
        c = z[i] * omega0 ** 2 / (Z[i] * (z[i] ** 2 - a))
        s += c * np.exp(-a * t) * wofz(1j * z[i] * np.sqrt(t))
    return first + s.real


def omega0_of(sigma: float, rho_l: float, rho_g: float, k: float) -> float:
    return math.sqrt(sigma * k ** 3 / (rho_l + rho_g))
