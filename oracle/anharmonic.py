"""Three-phonon matrix elements and linewidths (paper Sec. "Three-Phonon Scattering",
Eqs. (phi3_proj), (gamma), (broadening), (lifetime), and Sec. "Computational
Implementation": selective calculation above min_frequency).

Projected potential, all-incoming convention (q + q' + q'' = G), with the same phase sign
and cell-origin gauge as the dynamical matrix:

    Phi(q nu, q' nu', q'' nu'') = sum_{a,b,c} sum_{l', l''} phi(0 a, l' b, l'' c)
        exp(-i q'.R_l') exp(-i q''.R_l'') e_q[a,nu] e_q'[b,nu'] e_q''[c,nu''] / sqrt(m_a m_b m_c)

(a, b, c run over atom x Cartesian; at q = q' = q'' = 0 this is Eq. (phi3_proj) literally).

Readings of the garbled/silent parts of Eqs. (gamma) and (lifetime):
  * The printed Delta^+ pairs (n'-n'') with delta(w - w' + w''), which is negative as
    written; it is read as the absorption term with its sign lost.  Summed over ordered
    (nu', nu'') pairs the rate holds a decay term (1 + n' + n'') delta(w - w' - w'') and an
    absorption term 2 (n' - n'') delta(w + w' - w''), both with the prefactor hbar pi / 8.
  * The reported linewidth gamma = 1/tau is the Gamma^0 of Eq. (rta) with this counting.
  * A 1/N_q goes with the unit-cell Fourier form of Phi (pinned by the supercell-folding
    test: |Phi_supercell|^2 = |Phi_cell|^2 / N_q).
  * sigma is in THz and is applied to f; delta(w) = g(f) / (2 pi).
  * Gaussian g = exp(-x^2/s^2)/(sqrt(pi) s); Lorentzian g = (s/2)/(pi (x^2 + (s/2)^2)).
  * Terms with |Delta f| >= window * sigma (window = 2) are dropped for both shapes.
  * Modes with f < f_min get gamma = 0; partners with f' or f'' < f_min are skipped.
  * The decay term uses the outgoing modes (-q', nu') and (q + q', nu''); their |Phi|^2
    equals that of the incoming element by time reversal, so one |Phi|^2 per
    (lambda, q', nu', nu'') serves both processes.
"""
import math

import numpy as np

from .constants import EV_A2_AMU_TO_PS2, HBAR_EV_PS, TWO_PI
from . import grid as _grid
from . import occupation as _occ


def broadening(df, shape, sigma, window=2.0):
    """g(df) in 1/THz (Eq. (broadening)), zero where |df| >= window * sigma."""
    df = np.asarray(df, dtype=np.float64)
    if shape == "gauss":
        g = np.exp(-(df / sigma) ** 2) / (math.sqrt(math.pi) * sigma)
    elif shape == "lorentz":
        h = 0.5 * sigma
        g = h / (math.pi * (df * df + h * h))
    else:
        raise ValueError(shape)
    return np.where(np.abs(df) < window * sigma, g, 0.0)


class FC3:
    """COO third-order IFCs with the mass factor applied (input of Eq. (phi3_proj))."""

    def __init__(self, idx, val, masses):
        idx = np.asarray(idx, dtype=np.int64)
        self.a = idx[:, 0]
        self.b = idx[:, 1]
        self.c = idx[:, 2]
        self.R1 = idx[:, 3:6].astype(np.float64)
        self.R2 = idx[:, 6:9].astype(np.float64)
        m = np.repeat(np.asarray(masses, dtype=np.float64), 3)
        self.w = np.asarray(val, dtype=np.float64) / np.sqrt(m[self.a] * m[self.b] * m[self.c])
        self.n = m.shape[0]


def phi_tensor(fc3, q1_red, q2_red):
    """F[a,b,c] = sum over entries of phi exp(-i q'.R') exp(-i q''.R'') / sqrt(mmm)."""
    ph = np.exp(-1j * TWO_PI * (fc3.R1 @ np.asarray(q1_red) + fc3.R2 @ np.asarray(q2_red)))
    F = np.zeros((fc3.n, fc3.n, fc3.n), dtype=np.complex128)
    np.add.at(F, (fc3.a, fc3.b, fc3.c), fc3.w * ph)
    return F


def v3(fc3, e0, q1_red, e1, q2_red, e2):
    """Phi[nu, nu', nu''] for modes e0 (at q), e1 (at q1), e2 (at q2), q + q1 + q2 = G.
    The first mode's q enters only through e0 (its atom sits in the home cell)."""
    F = phi_tensor(fc3, q1_red, q2_red)
    A = np.tensordot(e0, F, axes=([0], [0]))        # [nu, b, c]
    A = np.tensordot(A, e1, axes=([1], [0]))        # [nu, c, nu']
    return np.tensordot(A, e2, axes=([1], [0]))     # [nu, nu', nu'']


def pair_weights(f0, f1, f2, n1, n2, shape, sigma, f_min, window):
    """W[nu, nu', nu''] = [(1+n'+n'') g(f-f'-f'') + 2 (n'-n'') g(f+f'-f'')] / (2 pi w w' w''),
    in ps^4 (times |Phi|^2 and the prefactor gives 1/ps).  Zero outside the window and
    where any of the three frequencies is below f_min."""
    F0 = f0[:, None, None]
    F1 = f1[None, :, None]
    F2 = f2[None, None, :]
    N1 = n1[None, :, None]
    N2 = n2[None, None, :]
    decay = (1.0 + N1 + N2) * broadening(F0 - F1 - F2, shape, sigma, window)
    absorb = 2.0 * (N1 - N2) * broadening(F0 + F1 - F2, shape, sigma, window)
    ok = (F0 >= f_min) & (F1 >= f_min) & (F2 >= f_min)
    with np.errstate(divide="ignore", invalid="ignore"):
        www = (TWO_PI ** 3) * F0 * F1 * F2
        W = np.where(ok, (decay + absorb) / TWO_PI / www, 0.0)
    return W


def prefactor(nq):
    """pi hbar / (8 N_q) with the eV^3/(A^6 amu^3) -> ps^-6 conversion of |Phi|^2 / hbar^0."""
    return math.pi * HBAR_EV_PS * EV_A2_AMU_TO_PS2 ** 3 / (8.0 * nq)


def gamma(fc3, mesh, freq, evec, irr_q, temperature, shape="gauss", sigma=0.1,
          f_min=0.01, window=2.0, is_classic=False, want_wp2=False, keep_v2=False):
    """Linewidth gamma = 1/tau (1/ps) for every band of each q in irr_q.

    freq [nq, n] (THz) and evec [nq, n, n] cover the full mesh.  Returns gamma [n_irr, n]
    (and WP2 [n_irr, n] in ps^4 if want_wp2: the same sum with |Phi|^2 -> 1 and without the
    hbar pi / 8 factor, keeping 1/N_q; and the per-pair |Phi|^2 if keep_v2)."""
    mesh = tuple(int(x) for x in mesh)
    qred = _grid.mesh_qred(mesh)
    kint = _grid.mesh_int(mesh)
    nq = qred.shape[0]
    nocc = _occ.bose(freq, temperature, is_classic)
    pref = prefactor(nq)
    irr_q = np.asarray(irr_q, dtype=np.int64)
    n = freq.shape[1]
    g_out = np.zeros((irr_q.shape[0], n))
    wp2 = np.zeros((irr_q.shape[0], n))
    v2_store = {}
    for s, iq in enumerate(irr_q):
        for iqp in range(nq):
            iqpp = int(_grid.mesh_index(-(kint[iq] + kint[iqp]), mesh))
            q1 = qred[iqp]
            q2 = -(qred[iq] + qred[iqp])          # unfolded: exp(-i q''.R) is G-periodic
            V = v3(fc3, evec[iq], q1, evec[iqp], q2, evec[iqpp])
            V2 = np.abs(V) ** 2
            W = pair_weights(freq[iq], freq[iqp], freq[iqpp], nocc[iqp], nocc[iqpp],
                             shape, sigma, f_min, window)
            g_out[s] += pref * np.einsum("ijk,ijk->i", V2, W)
            if want_wp2:
                wp2[s] += W.sum(axis=(1, 2)) / nq
            if keep_v2:
                v2_store[(int(iq), iqp)] = V2
        g_out[s] = np.where(freq[iq] >= f_min, g_out[s], 0.0)
        wp2[s] = np.where(freq[iq] >= f_min, wp2[s], 0.0)
    out = [g_out]
    if want_wp2:
        out.append(wp2)
    if keep_v2:
        out.append(v2_store)
    return out[0] if len(out) == 1 else tuple(out)


def gamma_from_v2(v2_store, mesh, freq, irr_q, temperature, shape="gauss", sigma=0.1,
                  f_min=0.01, window=2.0):
    """Temperature-dependent half of the split of Sec. "Performance Optimization"
    (multi-temperature): gamma from cached |Phi|^2, re-weighted at a new temperature."""
    mesh = tuple(int(x) for x in mesh)
    kint = _grid.mesh_int(mesh)
    nq = kint.shape[0]
    nocc = _occ.bose(freq, temperature)
    pref = prefactor(nq)
    n = freq.shape[1]
    g_out = np.zeros((len(irr_q), n))
    for s, iq in enumerate(irr_q):
        for iqp in range(nq):
            iqpp = int(_grid.mesh_index(-(kint[iq] + kint[iqp]), mesh))
            W = pair_weights(freq[iq], freq[iqp], freq[iqpp], nocc[iqp], nocc[iqpp],
                             shape, sigma, f_min, window)
            g_out[s] += pref * np.einsum("ijk,ijk->i", v2_store[(int(iq), iqp)], W)
        g_out[s] = np.where(freq[iq] >= f_min, g_out[s], 0.0)
    return g_out


def degenerate_average(freq_row, values, rel_tol=1e-5):
    """Average values over sets of equal frequency (|df| < rel_tol * max f) in one q."""
    f = np.asarray(freq_row)
    v = np.asarray(values, dtype=np.float64).copy()
    tol = rel_tol * max(float(np.abs(f).max()), 1e-30)
    order = np.argsort(f)
    i = 0
    out = v.copy()
    while i < len(order):
        j = i + 1
        while j < len(order) and f[order[j]] - f[order[i]] < tol:
            j += 1
        idx = order[i:j]
        out[idx] = v[idx].mean()
        i = j
    return out
