"""Gamma-only brute force on a supercell: Eq. (phi3_proj) evaluated literally, with real
eigenvectors of the Gamma-point dynamical matrix (Eqs. (dynmat), (eigenvalue)), and the
linewidth of Eq. (gamma) with N_q = 1.

A q-mesh n1 x n2 x n3 on a cell is the same physical problem as the Gamma point of the
n1 x n2 x n3 supercell with periodic (image-summed) IFCs; since a Bloch mode normalised
on the supercell carries 1/sqrt(N_q), |Phi_supercell|^2 = |Phi_cell|^2 / N_q and the mesh
linewidths averaged over each set of equal frequency equal the supercell ones.  This
module builds the supercell side from the supercell's own IFC list, independently of the
mesh code path.
"""
import numpy as np

from .constants import EV_A2_AMU_TO_PS2, TWO_PI
from . import anharmonic as _anh
from . import occupation as _occ


def gamma_point_dynmat(ifc2_idx, ifc2_val, masses):
    n = 3 * masses.shape[0]
    D = np.zeros((n, n))
    for (i, j, _r1, _r2, _r3), blk in zip(ifc2_idx, ifc2_val):
        D[3 * i:3 * i + 3, 3 * j:3 * j + 3] += blk / np.sqrt(masses[i] * masses[j])
    return 0.5 * (D + D.T)


def folded_phi3(ifc3_idx, ifc3_val, masses):
    """Periodic supercell Phi3[a,b,c] / sqrt(m_a m_b m_c): all images summed."""
    m = np.repeat(np.asarray(masses, dtype=np.float64), 3)
    n = m.shape[0]
    idx = np.asarray(ifc3_idx, dtype=np.int64)
    F = np.zeros((n, n, n))
    w = np.asarray(ifc3_val) / np.sqrt(m[idx[:, 0]] * m[idx[:, 1]] * m[idx[:, 2]])
    np.add.at(F, (idx[:, 0], idx[:, 1], idx[:, 2]), w)
    return F


def gamma_only(ifc2_idx, ifc2_val, ifc3_idx, ifc3_val, masses, temperature, shape="gauss",
               sigma=0.1, f_min=0.01, window=2.0):
    """Frequencies (THz) and linewidths (1/ps) of every Gamma-point mode of the supercell."""
    D = gamma_point_dynmat(ifc2_idx, ifc2_val, masses)
    lam, eta = np.linalg.eigh(D)
    freq = np.sign(lam) * np.sqrt(np.abs(lam) * EV_A2_AMU_TO_PS2) / TWO_PI
    F = folded_phi3(ifc3_idx, ifc3_val, masses)
    # Eq. (phi3_proj): Phi[mu, mu', mu''] = sum_abc F[a,b,c] eta[a,mu] eta[b,mu'] eta[c,mu'']
    P = np.einsum("abc,ai,bj,ck->ijk", F, eta, eta, eta, optimize=True)
    nocc = _occ.bose(freq, temperature)
    W = _anh.pair_weights(freq, freq, freq, nocc, nocc, shape, sigma, f_min, window)
    g = _anh.prefactor(1) * np.einsum("ijk,ijk->i", P * P, W)
    g = np.where(freq >= f_min, g, 0.0)
    return freq, g
