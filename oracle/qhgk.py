"""Quasi-harmonic Green-Kubo conductivity (paper Sec. "Quasi-Harmonic Green-Kubo (QHGK)",
Eq. (qhgk) for a Gamma-only cell and Eq. (qhgk_crystal) for a q-mesh):

    kappa_ab = 1/V sum_{mu mu'} c_{mu mu'} Re(v^a_{mu mu'} v^b_{mu' mu}) tau_{mu mu'}

Readings of the parts the section leaves garbled or open (the same in the mesh form):
  * c_{mu mu'} = (hbar w w' / T) (n - n') / (w' - w) (the printed k_B/T prefactor is read as
    hbar/T: it is the only one with the units of a heat capacity and whose w' -> w limit is
    c_mu of Eq. (heatcap)); pairs closer than 1e-5 f_max take (c_mu + c_mu') / 2.
  * v^a_{mu mu'} = <e_mu| dD/dq_a |e_mu'> / (2 sqrt(w w')): the derivative of the dynamical
    matrix at q = 0 in the atom-position gauge, dD/dq_a = -i G^a with
    G^a_{ij} = sum_R (x_j + R - x_i)_a Phi2(0i, Rj) / sqrt(m_i m_j); the second velocity of
    the product carries swapped indices (as in Eq. (qhgk_crystal)), so for the Hermitian
    velocity matrices the product is real.  The diagonal is the group velocity (Eq. groupvel).
  * tau_{mu mu'} = g / (2 ((w - w')^2 + g^2)) with the half-width g = (gamma_mu + gamma_mu')/4
    (gamma = 1/tau of Eq. (gamma)), so that tau_{mu mu} = 1/gamma_mu as in Eq. (rta).
  * modes below f_min and modes with gamma = 0 are left out.
Result in W/(m K).

TEST INFRASTRUCTURE ONLY (see the package header).
"""
import numpy as np

from .constants import EV_A2_AMU_TO_PS2, EV_PS_A_K_TO_W_MK, HBAR_EV_PS, TWO_PI
from . import harmonic as _harm
from . import occupation as _occ


def bond_derivative(ifc2_idx, ifc2_val, masses, positions, lattice):
    """G[a] (3, n, n) real: sum_R (x_j + R.L - x_i)_a Phi2_block / sqrt(m_i m_j), eV/(A amu)."""
    idx = np.asarray(ifc2_idx, dtype=np.int64)
    val = np.asarray(ifc2_val, dtype=np.float64).reshape(-1, 3, 3)
    na = masses.shape[0]
    G = np.zeros((3, 3 * na, 3 * na))
    for (i, j, r1, r2, r3), blk in zip(idx, val):
        r = positions[j] + np.array([r1, r2, r3], dtype=np.float64) @ lattice - positions[i]
        for a in range(3):
            G[a, 3 * i:3 * i + 3, 3 * j:3 * j + 3] += r[a] * blk / np.sqrt(masses[i] * masses[j])
    return G


def heat_capacity_matrix(freq, temperature, f_min=0.01, rel_tol=1e-5):
    """c_{mu mu'} in eV/K."""
    f = np.asarray(freq, dtype=np.float64)
    w = TWO_PI * f
    nocc = _occ.bose(f, temperature)
    cm = _occ.heat_capacity(f, temperature)
    dw = w[None, :] - w[:, None]                                                       # w' - w
    close = np.abs(f[None, :] - f[:, None]) < rel_tol * max(np.abs(f).max(), 1e-30)
    with np.errstate(divide="ignore", invalid="ignore"):
        c = HBAR_EV_PS * w[:, None] * w[None, :] * (nocc[:, None] - nocc[None, :]) / (temperature * dw)
    c = np.where(close, 0.5 * (cm[:, None] + cm[None, :]), c)
    ok = f >= f_min
    return np.where(ok[:, None] & ok[None, :], c, 0.0)


def lifetime_matrix(freq, gamma):
    """tau_{mu mu'} in ps (Lorentzian form with half-width (gamma + gamma')/4)."""
    w = TWO_PI * np.asarray(freq, dtype=np.float64)
    g = 0.25 * (np.asarray(gamma)[:, None] + np.asarray(gamma)[None, :])
    dw = w[:, None] - w[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        t = g / (2.0 * (dw * dw + g * g))
    return np.where(g > 0, t, 0.0)


def velocity_matrix(dD, freq, evec, f_min=0.01):
    """v[a] (3, n, n) complex in A/ps from dD/dq (3, n, n) in eV/(A amu) and eigenvectors."""
    w = TWO_PI * np.asarray(freq, dtype=np.float64)
    M = np.einsum("im,aij,jn->amn", evec.conj(), dD, evec) * EV_A2_AMU_TO_PS2
    ok = np.asarray(freq) >= f_min
    with np.errstate(divide="ignore", invalid="ignore"):
        d = 2.0 * np.sqrt(np.outer(np.where(ok, w, 1.0), np.where(ok, w, 1.0)))
    return np.where((ok[:, None] & ok[None, :])[None], M / d[None], 0.0)


def kappa_pairs(c, v, tau, volume):
    """kappa_ab = 1/V sum c Re(v^a_{mu mu'} v^b_{mu' mu}) tau in W/(m K)."""
    k = np.real(np.einsum("mn,amn,bnm->ab", c * tau, v, v))
    return k / volume * EV_PS_A_K_TO_W_MK


def kappa_gamma_cell(ifc2_idx, ifc2_val, masses, positions, lattice, freq, evec, gamma, temperature, f_min=0.01):
    """Eq. (qhgk) for a Gamma-only cell: freq [n] THz, evec [n, n] (real), gamma [n] 1/ps."""
    G = bond_derivative(ifc2_idx, ifc2_val, masses, positions, lattice)
    dD = -1j * G
    v = velocity_matrix(dD, freq, np.asarray(evec, dtype=np.complex128), f_min)
    c = heat_capacity_matrix(freq, temperature, f_min)
    ok = (np.asarray(freq) >= f_min) & (np.asarray(gamma) > 0)
    tau = lifetime_matrix(freq, np.where(ok, gamma, 0.0))
    tau = np.where(ok[:, None] & ok[None, :], tau, 0.0)
    volume = abs(np.linalg.det(lattice))
    return kappa_pairs(c, v, tau, volume)


def kappa_mesh(ifc2_idx, ifc2_val, masses, lattice, q_red, freq, evec, gamma_full, temperature, f_min=0.01,
               pairs="all"):
    """Eq. (qhgk_crystal) with the mesh dD/dq (cell-origin gauge, equal to the atom-position
    gauge for a one-atom cell).  pairs = "all": RTA plus the interband pairs (s != s') at each
    q; "degenerate": only pairs inside a degenerate set (|df| < 1e-5 f_max), i.e. Eq. (rta)
    with the basis-invariant velocity products."""
    nq = q_red.shape[0]
    volume = abs(np.linalg.det(lattice))
    k = np.zeros((3, 3))
    for iq in range(nq):
        dD = _harm.dynamical_matrix_derivative(ifc2_idx, ifc2_val, masses, lattice, q_red[iq])
        v = velocity_matrix(dD, freq[iq], evec[iq], f_min)
        c = heat_capacity_matrix(freq[iq], temperature, f_min)
        ok = (freq[iq] >= f_min) & (gamma_full[iq] > 0)
        tau = lifetime_matrix(freq[iq], np.where(ok, gamma_full[iq], 0.0))
        tau = np.where(ok[:, None] & ok[None, :], tau, 0.0)
        if pairs == "degenerate":
            f = freq[iq]
            same = np.abs(f[:, None] - f[None, :]) < 1e-5 * max(np.abs(f).max(), 1e-30)
            tau = np.where(same, tau, 0.0)
        k += kappa_pairs(c, v, tau, volume)
    return k / nq
