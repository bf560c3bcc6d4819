"""Harmonic phonons (paper Sec. "Interatomic Force Constants" and "Group Velocities").

Eq. (dynmat) with Eq. (dynmat_reciprocal):
    D_{i a, j b}(q) = sum_l Phi2(0 i a, l j b) exp(-i q.R_l) / sqrt(m_i m_j)
with R_l the cell-origin lattice vector (so D(q + G) = D(q)).
Eq. (eigenvalue_crystal): D(q) e = w^2 e, solved with a Hermitian eigensolver.
Eq. (groupvel): v_a = Re <e| dD/dq_a |e> / (2 w) with the analytic derivative
    dD/dq_a = sum_l (-i R_l,a) exp(-i q.R_l) Phi2(0i, lj) / sqrt(m_i m_j).
"""
import numpy as np

from .constants import EV_A2_AMU_TO_PS2, TWO_PI


def _blocks_sum(ifc2_idx, ifc2_val, masses, weights):
    """sum_b weights[b] * Phi2_b / sqrt(m_i m_j) placed at block (i, j); weights [nb] complex."""
    idx = np.asarray(ifc2_idx, dtype=np.int64)
    na = masses.shape[0]
    acc = np.zeros((na, na, 3, 3), dtype=np.complex128)
    scale = weights / np.sqrt(masses[idx[:, 0]] * masses[idx[:, 1]])
    np.add.at(acc, (idx[:, 0], idx[:, 1]), np.asarray(ifc2_val) * scale[:, None, None])
    return acc.transpose(0, 2, 1, 3).reshape(3 * na, 3 * na)


def dynamical_matrix(ifc2_idx, ifc2_val, masses, q_red):
    """D(q) in eV/(A^2 amu) for reduced q.  ifc2_idx rows (i, j, R1, R2, R3)."""
    R = np.asarray(ifc2_idx, dtype=np.float64)[:, 2:5]
    ph = np.exp(-1j * TWO_PI * (R @ np.asarray(q_red, dtype=np.float64)))
    return _blocks_sum(ifc2_idx, ifc2_val, masses, ph)


def dynamical_matrix_derivative(ifc2_idx, ifc2_val, masses, lattice, q_red):
    """dD/dq_alpha (alpha = x, y, z; q Cartesian in rad/A), shape (3, n, n), in eV A/(A^2 amu)."""
    R = np.asarray(ifc2_idx, dtype=np.float64)[:, 2:5]
    ph = np.exp(-1j * TWO_PI * (R @ np.asarray(q_red, dtype=np.float64)))
    Rc = R @ lattice
    return np.array([_blocks_sum(ifc2_idx, ifc2_val, masses, -1j * Rc[:, a] * ph) for a in range(3)])


def frequencies_from_eigenvalues(lam):
    """Signed frequency in THz: sign(lam) sqrt(|lam| * conv) / (2 pi)."""
    w = np.sqrt(np.abs(lam) * EV_A2_AMU_TO_PS2)
    return np.sign(lam) * w / TWO_PI


def solve(ifc2_idx, ifc2_val, masses, lattice, q_list):
    """Frequencies (THz, [nq, n]), eigenvectors ([nq, n, n], column nu), velocities (A/ps, [nq, n, 3])."""
    q_list = np.atleast_2d(q_list)
    nq = q_list.shape[0]
    n = 3 * masses.shape[0]
    freq = np.zeros((nq, n))
    evec = np.zeros((nq, n, n), dtype=np.complex128)
    vel = np.zeros((nq, n, 3))
    for k, q in enumerate(q_list):
        D = dynamical_matrix(ifc2_idx, ifc2_val, masses, q)
        D = 0.5 * (D + D.conj().T)
        lam, e = np.linalg.eigh(D)
        freq[k] = frequencies_from_eigenvalues(lam)
        evec[k] = e
        vel[k] = velocities(ifc2_idx, ifc2_val, masses, lattice, q, freq[k], e)
    return freq, evec, vel


def velocities(ifc2_idx, ifc2_val, masses, lattice, q_red, freq_thz, e):
    """Eq. (groupvel) per mode in the given eigenvector basis; 0 where f <= 0."""
    dD = dynamical_matrix_derivative(ifc2_idx, ifc2_val, masses, lattice, q_red)
    w = freq_thz * TWO_PI                                   # rad/ps
    n = e.shape[1]
    v = np.zeros((n, 3))
    for a in range(3):
        num = np.real(np.einsum("in,ij,jn->n", e.conj(), dD[a], e)) * EV_A2_AMU_TO_PS2
        with np.errstate(divide="ignore", invalid="ignore"):
            v[:, a] = np.where(w > 0, num / (2.0 * w), 0.0)
    return v


def degenerate_sets(freq_row, rel_tol=1e-5):
    """Groups of band indices whose frequencies differ by less than rel_tol * max|f|."""
    f = np.asarray(freq_row)
    tol = rel_tol * max(float(np.abs(f).max()), 1e-30)
    order = np.argsort(f, kind="stable")
    sets, i = [], 0
    while i < len(order):
        j = i + 1
        while j < len(order) and f[order[j]] - f[order[i]] < tol:
            j += 1
        sets.append(np.sort(order[i:j]))
        i = j
    return sets


def velocity_products(ifc2_idx, ifc2_val, masses, lattice, q_red, freq_thz, e, rel_tol=1e-5):
    """Basis-invariant v (x) v per mode, [n, 3, 3] in (A/ps)^2.

    Reading of Eq. (groupvel) for degenerate modes, where per-mode velocities depend on the
    eigenvector basis: within a degenerate set S every mode gets
        (1/|S|) sum_{mu, mu' in S} Re(V^a_{mu mu'} V^b_{mu' mu}) / (4 w^2),
    V^a_{mu mu'} = <e_mu| dD/dq_a |e_mu'>.  For a non-degenerate mode this is v_a v_b."""
    dD = dynamical_matrix_derivative(ifc2_idx, ifc2_val, masses, lattice, q_red)
    w = freq_thz * TWO_PI
    n = e.shape[1]
    out = np.zeros((n, 3, 3))
    Vm = np.einsum("im,aij,jn->amn", e.conj(), dD, e) * EV_A2_AMU_TO_PS2     # [3, n, n]
    for S in degenerate_sets(freq_thz, rel_tol):
        ws = w[S[0]]
        if ws <= 0:
            continue
        blk = Vm[:, S][:, :, S]                                          # [3, s, s]
        t = np.real(np.einsum("amn,bnm->ab", blk, blk)) / (4.0 * ws * ws) / len(S)
        out[S] = t
    return out
