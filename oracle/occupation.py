"""Bose-Einstein occupation and modal heat capacity (paper Sec. "Phonon Populations and
Heat Capacity", Eqs. (bose) and (heatcap)); classical forms under is_classic.

Modes with f <= 0 get n = c = 0 (they are excluded from every sum downstream).
"""
import numpy as np

from .constants import HBAR_EV_PS, KB_EV_K, TWO_PI


def bose(freq_thz, temperature, is_classic=False):
    f = np.asarray(freq_thz, dtype=np.float64)
    w = f * TWO_PI
    out = np.zeros_like(f)
    pos = f > 0
    x = HBAR_EV_PS * w[pos] / (KB_EV_K * temperature)
    out[pos] = 1.0 / x if is_classic else 1.0 / np.expm1(x)
    return out


def heat_capacity(freq_thz, temperature, is_classic=False):
    """c in eV/K: k_B x^2 e^x / (e^x - 1)^2, x = hbar w / (k_B T); k_B classically."""
    f = np.asarray(freq_thz, dtype=np.float64)
    out = np.zeros_like(f)
    pos = f > 0
    if is_classic:
        out[pos] = KB_EV_K
        return out
    x = HBAR_EV_PS * f[pos] * TWO_PI / (KB_EV_K * temperature)
    em = np.expm1(x)
    out[pos] = KB_EV_K * x * x * np.exp(x) / (em * em)
    return out
