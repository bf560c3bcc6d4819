"""Gamma-only linewidths of a large cell, mode by mode, with a sparse Phi3 (paper Sec.
"Three-Phonon Scattering": Eq. (phi3_proj) at q = q' = q'' = 0, where the eigenvectors of the
real symmetric dynamical matrix, Eq. (eigenvalue), are real; Eq. (gamma) with N_q = 1; the
broadening of Eq. (broadening), Lorentzian or Gaussian, with the 2 sigma window).

For one mode lam the projection is taken in the order the equation nests its sums:

    W_lam[j, k]       = sum_i  Phi3[i, j, k] / sqrt(m_i m_j m_k) * e[i, lam]      (sparse COO)
    Phi[lam, mu', mu''] = sum_jk e[j, mu'] W_lam[j, k] e[k, mu'']  = (E^T W_lam E)[mu', mu'']

and gamma_lam is the sum over all ordered (mu', mu'') of |Phi|^2 times the pair weights of
anharmonic.pair_weights.  Images of one (i, j, k) triple are summed (all phases are 1).

TEST INFRASTRUCTURE ONLY (see the package header).
"""
import numpy as np

from . import anharmonic as _anh
from . import occupation as _occ


def mass_scaled(ifc3_idx, ifc3_val, masses):
    """(i, j, k, w) with w = Phi3 / sqrt(m_i m_j m_k); image translations dropped."""
    idx = np.asarray(ifc3_idx, dtype=np.int64)
    m = np.repeat(np.asarray(masses, dtype=np.float64), 3)
    i, j, k = idx[:, 0], idx[:, 1], idx[:, 2]
    w = np.asarray(ifc3_val, dtype=np.float64) / np.sqrt(m[i] * m[j] * m[k])
    return i, j, k, w


def projected_slice(coo, n, evec, lam):
    """Phi[lam, :, :] (n x n): Eq. (phi3_proj) with the first eigenvector fixed to mode lam."""
    i, j, k, w = coo
    W = np.bincount(j * n + k, weights=w * evec[i, lam], minlength=n * n).reshape(n, n)
    return evec.T @ W @ evec


def gamma_modes(ifc3_idx, ifc3_val, masses, freq, evec, modes, temperature, shape="lorentz",
                sigma=0.1, f_min=0.01, window=2.0):
    """gamma (1/ps) of the listed Gamma-point modes; freq [n] THz, evec [n, n] real (columns)."""
    freq = np.asarray(freq, dtype=np.float64)
    evec = np.asarray(evec, dtype=np.float64)
    n = freq.shape[0]
    coo = mass_scaled(ifc3_idx, ifc3_val, masses)
    nocc = _occ.bose(freq, temperature)
    pref = _anh.prefactor(1)
    out = np.zeros(len(modes))
    for s, lam in enumerate(modes):
        if freq[lam] < f_min:
            continue
        P = projected_slice(coo, n, evec, lam)
        Wt = _anh.pair_weights(freq[lam:lam + 1], freq, freq, nocc, nocc, shape, sigma, f_min, window)[0]
        out[s] = pref * np.sum(P * P * Wt)
    return out


def dynmat(ifc2_idx, ifc2_val, masses):
    """Real Gamma-point dynamical matrix (images summed), eV/(A^2 amu)."""
    idx = np.asarray(ifc2_idx, dtype=np.int64)
    na = masses.shape[0]
    acc = np.zeros((na, na, 3, 3))
    scale = 1.0 / np.sqrt(masses[idx[:, 0]] * masses[idx[:, 1]])
    flat = idx[:, 0] * na + idx[:, 1]
    vals = np.asarray(ifc2_val).reshape(-1, 9) * scale[:, None]
    acc = np.stack([np.bincount(flat, weights=vals[:, t], minlength=na * na) for t in range(9)], axis=1)
    D = acc.reshape(na, na, 3, 3).transpose(0, 2, 1, 3).reshape(3 * na, 3 * na)
    return 0.5 * (D + D.T)
