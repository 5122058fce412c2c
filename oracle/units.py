"""Plasma-accelerator scalings in Gaussian units -- TEST INFRASTRUCTURE ONLY.

The introduction of the paper states the linear-theory lengths: the plasma
wavelength lambda_p = sqrt(pi c^2 m / (e^2 n_e)) and the depletion length
L_d = lambda_p^3 / (2 lambda0^2); its first section quotes the laser group
velocity gamma_g of the 100 MeV stage.  These helpers restate those formulas;
the critical density n_c = pi m c^2 / (e^2 lambda0^2) is the density at which
the plasma wavelength equals lambda0, and gamma_g = omega0/omega_p =
sqrt(n_c / n_e) is the linear group-velocity Lorentz factor.
"""
import math

C_CM_S = 2.99792458e10          # speed of light, cm/s
E_ESU = 4.803204712570263e-10   # elementary charge, statcoulomb
M_G = 9.1093837015e-28          # electron mass, g


def plasma_wavelength_cm(n_e_cm3: float) -> float:
    """lambda_p = sqrt(pi c^2 m / (e^2 n_e)) (introduction)."""
    return math.sqrt(math.pi * C_CM_S ** 2 * M_G / (E_ESU ** 2 * n_e_cm3))


def critical_density_cm3(lambda0_cm: float) -> float:
    """n_c: the density whose plasma wavelength is lambda0."""
    return math.pi * M_G * C_CM_S ** 2 / (E_ESU ** 2 * lambda0_cm ** 2)


def depletion_length_cm(n_e_cm3: float, lambda0_cm: float) -> float:
    """L_d = lambda_p^3 / (2 lambda0^2) (introduction)."""
    lp = plasma_wavelength_cm(n_e_cm3)
    return lp ** 3 / (2.0 * lambda0_cm ** 2)


def depletion_time_s(n_e_cm3: float, lambda0_cm: float) -> float:
    """T_d = L_d / c (section on the numerical instability)."""
    return depletion_length_cm(n_e_cm3, lambda0_cm) / C_CM_S


def gamma_group(n_e_cm3: float, lambda0_cm: float) -> float:
    """Linear laser group-velocity factor sqrt(n_c / n_e)."""
    return math.sqrt(critical_density_cm3(lambda0_cm) / n_e_cm3)


def wake_amplitude_linear(a0: float, sigma: float, n_over_nc: float) -> float:
    """Peak on-axis wake E_z (units m c omega0 / e) of a Gaussian pulse whose field
    envelope is a0 exp(-xi^2/sigma^2) (sigma in lambda0), from 1D linear quasi-static
    theory: (d^2/dxi^2 + k_p^2) phi = k_p^2 <a^2>/2 with <a^2> = (a0^2/2) exp(-2 xi^2/sigma^2)
    gives E_z,max / E_0 = (a0^2/4) k_p sigma sqrt(pi/2) exp(-k_p^2 sigma^2 / 8),
    E_0 = m c omega_p / e = sqrt(n/n_c) in these units."""
    kp = 2.0 * math.pi * math.sqrt(n_over_nc)
    e0 = math.sqrt(n_over_nc)
    return e0 * (a0 ** 2 / 4.0) * kp * sigma * math.sqrt(math.pi / 2.0) * math.exp(-(kp * sigma) ** 2 / 8.0)
