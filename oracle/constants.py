"""CODATA 2018 constants and the unit conversions of the oracle (the paper states none).

Units: eV, Angstrom, amu, ps.  Frequencies f in THz, angular frequencies w = 2 pi f in
rad/ps.
"""
import math

HBAR_EV_PS = 6.582119569e-4          # hbar in eV*ps
KB_EV_K = 8.617333262e-5             # Boltzmann constant in eV/K
EV_J = 1.602176634e-19               # J per eV
AMU_KG = 1.66053906660e-27           # kg per amu

# eV / (A^2 amu) expressed in ps^-2:  (EV_J / (1e-20 * AMU_KG)) s^-2 * 1e-24 ps^2/s^2
EV_A2_AMU_TO_PS2 = EV_J / (1e-20 * AMU_KG) * 1e-24
# eV / (ps * A * K) expressed in W / (m K)
EV_PS_A_K_TO_W_MK = EV_J / 1e-12 / 1e-10

TWO_PI = 2.0 * math.pi
