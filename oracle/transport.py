"""RTA thermal conductivity (paper Sec. "Boltzmann Transport Equation", Eq. (rta)):

    kappa_ab = 1/(N_q V) sum_mu c_mu v_mu,a v_mu,b / Gamma0_mu

over the full mesh, skipping modes with f < f_min (Sec. "Computational Implementation",
selective calculation).  V is the unit-cell volume, N_q the number of mesh points.
Result in W/(m K).
"""
import numpy as np

from .constants import EV_PS_A_K_TO_W_MK
from . import occupation as _occ


def kappa_rta(freq, vel, gamma_full, temperature, volume, f_min=0.01, is_classic=False):
    nq = freq.shape[0]
    c = _occ.heat_capacity(freq, temperature, is_classic)
    ok = (freq >= f_min) & (gamma_full > 0)
    tau = np.where(ok, 1.0 / np.where(ok, gamma_full, 1.0), 0.0)
    k = np.einsum("qn,qna,qnb->ab", c * tau, vel, vel)
    return k / (nq * volume) * EV_PS_A_K_TO_W_MK


def unfold(gamma_irr, full_to_irr):
    """Map irreducible linewidths onto the full mesh (band index preserved)."""
    return np.asarray(gamma_irr)[np.asarray(full_to_irr)]


def kappa_rta_vv(freq, vv, gamma_full, temperature, volume, f_min=0.01, is_classic=False):
    """Eq. (rta) with the basis-invariant velocity products vv [nq, n, 3, 3]."""
    nq = freq.shape[0]
    c = _occ.heat_capacity(freq, temperature, is_classic)
    ok = (freq >= f_min) & (gamma_full > 0)
    tau = np.where(ok, 1.0 / np.where(ok, gamma_full, 1.0), 0.0)
    k = np.einsum("qn,qnab->ab", c * tau, vv)
    return k / (nq * volume) * EV_PS_A_K_TO_W_MK
