"""Iterative solution of the linearised BTE (paper Sec. "Boltzmann Transport Equation":
Eqs. (BTE), (gamma1), (invBTE), (kappa_general), (rta), (sc_iter), (inverse)).

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never imports it.

The unknown of Eq. (invBTE) is the mean free path lambda_mu (a 3-vector per mode):
    v_mu = Gamma0_mu lambda_mu + sum_mu' Gamma1[mu, mu'] lambda_mu'
and Eq. (sc_iter) iterates lambda^(k+1) = (v - Gamma1 lambda^(k)) / Gamma0 from the RTA
start lambda^(0) = v / Gamma0 (Eq. rta), stopping when Tr(kappa)/3 changes by less than tol
(relative) or after n_iter iterations.  Eq. (inverse) solves the same system directly.

Readings of the parts the paper leaves open:
  * Gamma0 is the linewidth gamma = 1/tau of Eq. (gamma) with the counting of
    oracle.anharmonic (decay (1+n'+n'') g(f-f'-f''), absorption 2 (n'-n'') g(f+f'-f'')).
  * Eq. (gamma1) prints Gamma1 as minus a sum of four rate terms without saying which
    partners are incoming or outgoing.  It is read as the linearised three-phonon collision
    operator of the iterative scheme the paper cites for Eq. (sc_iter) (Omini and
    Sparavigna; Broido et al.), acting on mean free paths:
        Delta_mu = sum_{absorption mu + mu' -> mu''} r (f''/f lambda_mu'' - f'/f lambda_mu')
                 + sum_{decay mu -> mu' + mu''}      r (f''/f lambda_mu'' + f'/f lambda_mu')
        (Gamma1 lambda)_mu = -Delta_mu
    where r is that process's term in the linewidth sum (so the r of mu sum to Gamma0_mu).
  * lambda is odd under time reversal, like v: lambda(-q, nu) = -lambda(q, nu).  In the
    all-incoming labelling of Eq. (phi3_proj) (q + q' + q'' = G) the outgoing partners of
    both processes are the time-reversal images of incoming ones, and every element
    (q', nu', nu'') of mu's linewidth sum, with weight w = its decay plus absorption term,
    gives
        Gamma1[mu, (q', nu')] += w f'/f        Gamma1[mu, (q'', nu'')] += w f''/f
    which is Eq. (gamma1)'s sum of rate terms with the printed overall minus absorbed by
    labelling the partners as incoming modes.
  * The unknowns live on a time-reversal-only irreducible set (each orbit {q, -q} keeps its
    smallest index): the column of mesh point p is added into its representative's with
    sign +1 (p listed) or -1 (-p listed); points with p = -p mod G carry lambda = 0.
  * kappa (Eq. kappa_general) sums the full mesh: a representative counts twice when
    -q != q (v lambda is even under time reversal), else once.
  * Modes with f < f_min or Gamma0 = 0 carry lambda = 0, as in Eq. (rta).
"""
import numpy as np

from .constants import EV_PS_A_K_TO_W_MK
from . import anharmonic as _anh
from . import grid as _grid
from . import occupation as _occ


def time_reversal_set(mesh):
    """Representatives of the orbits {q, -q} (smallest index) and, for every mesh point,
    (position of its representative, sign): +1 if the point is listed, -1 if its negative
    is, 0 where q = -q mod G."""
    mesh = tuple(int(x) for x in mesh)
    k = _grid.mesh_int(mesh)
    nq = k.shape[0]
    neg = _grid.mesh_index(-k, mesh)
    rep = np.minimum(np.arange(nq), neg)
    irr = np.unique(rep)
    pos = np.searchsorted(irr, rep)
    sign = np.where(neg == np.arange(nq), 0, np.where(rep == np.arange(nq), 1, -1))
    return irr, pos, sign


def scattering_rows(fc3, mesh, freq, evec, rows_q, temperature, shape="gauss", sigma=0.1,
                    f_min=0.01, window=2.0):
    """Gamma0 [len(rows_q), n] (1/ps) and Gamma1 rows [len(rows_q) * n, nq * n] (1/ps) with
    columns over the full mesh in the all-incoming labelling (reading above)."""
    mesh = tuple(int(x) for x in mesh)
    qred = _grid.mesh_qred(mesh)
    kint = _grid.mesh_int(mesh)
    nq, n = freq.shape
    nocc = _occ.bose(freq, temperature)
    pref = _anh.prefactor(nq)
    rows_q = np.asarray(rows_q, dtype=np.int64)
    g0 = np.zeros((rows_q.shape[0], n))
    g1 = np.zeros((rows_q.shape[0] * n, nq * n))
    for s, iq in enumerate(rows_q):
        f0 = freq[iq]
        inv0 = np.where(f0 >= f_min, 1.0 / np.where(f0 > 0, f0, 1.0), 0.0)
        for iqp in range(nq):
            iqpp = int(_grid.mesh_index(-(kint[iq] + kint[iqp]), mesh))
            V = _anh.v3(fc3, evec[iq], qred[iqp], evec[iqp], -(qred[iq] + qred[iqp]), evec[iqpp])
            W = _anh.pair_weights(f0, freq[iqp], freq[iqpp], nocc[iqp], nocc[iqpp],
                                  shape, sigma, f_min, window)
            w = pref * np.abs(V) ** 2 * W                       # [nu, nu', nu'']
            g0[s] += w.sum(axis=(1, 2))
            r = slice(s * n, (s + 1) * n)
            g1[r, iqp * n:(iqp + 1) * n] += w.sum(axis=2) * freq[iqp][None, :] * inv0[:, None]
            g1[r, iqpp * n:(iqpp + 1) * n] += w.sum(axis=1) * freq[iqpp][None, :] * inv0[:, None]
        g0[s] = np.where(f0 >= f_min, g0[s], 0.0)
    return g0, g1


def reduce_columns(g1_full, mesh, n):
    """Fold full-mesh columns onto the time-reversal representatives with their signs."""
    irr, pos, sign = time_reversal_set(mesh)
    out = np.zeros((g1_full.shape[0], irr.shape[0] * n))
    for p in range(pos.shape[0]):
        if sign[p] != 0:
            out[:, pos[p] * n:(pos[p] + 1) * n] += sign[p] * g1_full[:, p * n:(p + 1) * n]
    return out


def kappa_from_mfp(cv, vel, mfp, mult, volume, nq):
    """Eq. (kappa_general) over the representatives, each counted mult times (W/(m K))."""
    k = np.einsum("q,qn,qna,qnb->ab", mult.astype(np.float64), cv, vel, mfp)
    return k / (nq * volume) * EV_PS_A_K_TO_W_MK


def _system(mesh, freq, vel, gamma0, temperature, f_min):
    irr, _, sign = time_reversal_set(mesh)
    live = (gamma0 > 0) & (freq[irr] >= f_min) & (sign[irr] != 0)[:, None]
    mult = np.where(sign[irr] != 0, 2, 1)
    cv = _occ.heat_capacity(freq[irr], temperature)
    return irr, live, mult, cv, vel[irr]


def iterate(mesh, freq, vel, gamma0, gamma1, temperature, volume, n_iter=100, tol=1e-6, f_min=0.01):
    """Eq. (sc_iter) on the time-reversal representatives.

    gamma0 [n_irr, n] and gamma1 [n_irr * n, n_irr * n] come from scattering_rows (rows of
    the representatives) and reduce_columns.  Returns (kappa history [k+1, 3, 3] with the
    RTA iterate first, mean free paths [n_irr, n, 3] (A), converged flag)."""
    nq = freq.shape[0]
    irr, live, mult, cv, v = _system(mesh, freq, vel, gamma0, temperature, f_min)
    g0 = np.where(live, gamma0, 1.0)
    lam = np.where(live[..., None], v / g0[..., None], 0.0)
    hist = [kappa_from_mfp(cv, v, lam, mult, volume, nq)]
    converged = False
    for _ in range(n_iter):
        coupled = (gamma1 @ lam.reshape(-1, 3)).reshape(lam.shape)
        lam = np.where(live[..., None], (v - coupled) / g0[..., None], 0.0)
        hist.append(kappa_from_mfp(cv, v, lam, mult, volume, nq))
        k_old, k_new = np.trace(hist[-2]) / 3.0, np.trace(hist[-1]) / 3.0
        if abs(k_new - k_old) < tol * abs(k_old):
            converged = True
            break
    return np.array(hist), lam, converged


def kappa_inverse(mesh, freq, vel, gamma0, gamma1, temperature, volume, f_min=0.01):
    """Eq. (inverse): lambda = (diag(Gamma0) + Gamma1)^-1 v on the live modes, then
    Eq. (kappa_general).  Returns (kappa, mean free paths)."""
    nq = freq.shape[0]
    irr, live, mult, cv, v = _system(mesh, freq, vel, gamma0, temperature, f_min)
    idx = np.nonzero(live.ravel())[0]
    A = gamma1[np.ix_(idx, idx)] + np.diag(gamma0.ravel()[idx])
    lam = np.zeros((live.size, 3))
    lam[idx] = np.linalg.solve(A, v.reshape(-1, 3)[idx])
    lam = lam.reshape(v.shape)
    return kappa_from_mfp(cv, v, lam, mult, volume, nq), lam
