"""Isotope / mass-variance scattering (paper Sec. "Isotopic Scattering", Eq. (isotope),
Tamura's perturbation theory).

    gamma_iso(q s) = pi / (2 N_q) * w^2 * sum_{q' s'} delta(w - w') * sum_i g_i |<e_i(q s) | e_i(q' s')>|^2

with <e_i|e'_i> = sum_alpha conj(e[3i+alpha]) e'[3i+alpha] the overlap of the displacement
pattern on atom i (reading: the printed equation places alpha in the outer sum; the sum is
taken inside the modulus as in Tamura's form, the only placement that is invariant under a
rotation of the Cartesian frame), delta(w) = g(f)/(2 pi) with the broadening and window of
anharmonic.broadening, and modes below f_min (and partners below f_min) skipped.

TEST INFRASTRUCTURE ONLY (see the package header).
"""
import numpy as np

from .constants import TWO_PI
from . import anharmonic as _anh
from . import grid as _grid


def g_factor(fractions, masses):
    """g = sum_s f_s (1 - m_s / mbar)^2 with mbar = sum_s f_s m_s (relative mass variance)."""
    f = np.asarray(fractions, dtype=np.float64)
    m = np.asarray(masses, dtype=np.float64)
    mbar = float((f * m).sum())
    return float((f * (1.0 - m / mbar) ** 2).sum())


def gamma_iso(freq, evec, irr_q, g_atom, shape="gauss", sigma=0.1, f_min=0.01, window=2.0):
    """gamma_iso [n_irr, n] in 1/ps; freq [nq, n] THz and evec [nq, n, n] over the full mesh."""
    freq = np.asarray(freq, dtype=np.float64)
    nq, n = freq.shape
    g_atom = np.asarray(g_atom, dtype=np.float64)
    na = g_atom.shape[0]
    out = np.zeros((len(irr_q), n))
    for s, iq in enumerate(irr_q):
        e = evec[iq].reshape(na, 3, n)
        w = TWO_PI * freq[iq]
        acc = np.zeros(n)
        for iqp in range(nq):
            ep = evec[iqp].reshape(na, 3, n)
            # overlap per atom: O[i, s, s'] = sum_alpha conj(e[i, alpha, s]) e'[i, alpha, s']
            O = np.einsum("ias,iat->ist", e.conj(), ep)
            A = np.einsum("i,ist->st", g_atom, np.abs(O) ** 2)
            df = freq[iq][:, None] - freq[iqp][None, :]
            delta = _anh.broadening(df, shape, sigma, window) / TWO_PI
            ok = (freq[iqp] >= f_min)[None, :]
            acc += np.sum(np.where(ok, A * delta, 0.0), axis=1)
        out[s] = np.where(freq[iq] >= f_min, np.pi / (2.0 * nq) * w * w * acc, 0.0)
    return out
