"""Pins of the iterative-BTE oracle (oracle.bte, Eqs. (gamma1), (sc_iter), (inverse)).

The oracle assembles Gamma1 in the all-incoming labelling with the time-reversal
substitution.  These tests rebuild the collision operator from the processes themselves
(absorption mu + (q', nu') -> (q + q', nu''), decay mu -> (-q', nu') + (q + q', nu''), with
the outgoing partners at their own mesh points and no time-reversal assumption), and check:
the two operators agree on time-reversal-odd fields; the iteration on the full mesh with the
process operator gives the oracle's kappa history; the RTA start is Eq. (rta); the converged
iterate is the direct solution of Eq. (inverse); the s^2 scaling of Phi3; and detailed
balance of the collision operator on shell, with planted mistakes that it rejects.
"""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _tr_gauged(c, f2, mesh):
    """Harmonic solution on the mesh with the time-reversal gauge: at -q the conjugate
    eigenvectors, the same frequencies and the negated velocities."""
    q = O.grid.mesh_qred(mesh)
    freq, evec, vel = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    irr, pos, sign = O.bte.time_reversal_set(mesh)
    for p in range(q.shape[0]):
        if sign[p] == -1:
            r = irr[pos[p]]
            freq[p], evec[p], vel[p] = freq[r], evec[r].conj(), -vel[r]
    return freq, evec, vel


CASES = {
    # two-atom cell (one light, one heavy), odd mesh: only Gamma is its own negative
    "diatomic-333-gauss": dict(mult=(2, 1, 1), mesh=(3, 3, 3), T=50.0, shape="gauss", sigma=0.3),
    # even mesh: eight points with q = -q mod G (lambda = 0 there); Lorentzian
    "diatomic-422-lorentz": dict(mult=(2, 1, 1), mesh=(4, 2, 2), T=40.0, shape="lorentz", sigma=0.4),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    cfg = CASES[request.param]
    c = P.random_masses(P.fcc_primitive_multiple(5.26, cfg["mult"]), 39.95, 83.8, seed=1)
    pot = P.LennardJones()
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    mesh = cfg["mesh"]
    freq, evec, vel = _tr_gauged(c, f2, mesh)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    irr, pos, sign = O.bte.time_reversal_set(mesh)
    kw = dict(shape=cfg["shape"], sigma=cfg["sigma"])
    g0, g1f = O.bte.scattering_rows(fc3, mesh, freq, evec, irr, cfg["T"], **kw)
    n = freq.shape[1]
    return dict(c=c, f3=f3, fc3=fc3, mesh=mesh, freq=freq, evec=evec, vel=vel, T=cfg["T"], kw=kw,
                irr=irr, pos=pos, sign=sign, g0=g0, g1f=g1f, g1=O.bte.reduce_columns(g1f, mesh, n),
                vol=abs(np.linalg.det(c.lattice)))


def _process_operator(s):
    """Delta = B lambda over every mode of the full mesh, written process by process
    (the linearisation of Omini-Sparavigna / Broido et al. for mean free paths), plus the
    decay and absorption parts of the linewidth."""
    mesh, freq, evec = s["mesh"], s["freq"], s["evec"]
    kint, qred = O.grid.mesh_int(mesh), O.grid.mesh_qred(mesh)
    nq, n = freq.shape
    nocc = O.occupation.bose(freq, s["T"])
    pref = O.anharmonic.prefactor(nq)
    shape, sigma = s["kw"]["shape"], s["kw"]["sigma"]
    g = lambda x: O.anharmonic.broadening(x, shape, sigma, 2.0)
    fmin = 0.01
    B = np.zeros((nq * n, nq * n))
    gdec = np.zeros((nq, n))
    gabs = np.zeros((nq, n))
    for iq in range(nq):
        for iqp in range(nq):
            i_out = int(O.grid.mesh_index(kint[iq] + kint[iqp], mesh))     # q + q'
            i_neg = int(O.grid.mesh_index(-kint[iqp], mesh))               # -q'
            i_in = int(O.grid.mesh_index(-(kint[iq] + kint[iqp]), mesh))   # incoming third point
            V2 = np.abs(O.anharmonic.v3(s["fc3"], evec[iq], qred[iqp], evec[iqp],
                                        -(qred[iq] + qred[iqp]), evec[i_in])) ** 2
            f0 = freq[iq][:, None, None]
            f1 = freq[iqp][None, :, None]
            f2 = freq[i_out][None, None, :]
            n1 = nocc[iqp][None, :, None]
            n2 = nocc[i_out][None, None, :]
            ok = (f0 >= fmin) & (f1 >= fmin) & (f2 >= fmin)
            den = np.where(ok, (2 * np.pi) ** 4 * f0 * f1 * f2, 1.0)
            r_abs = np.where(ok, pref * V2 * 2.0 * (n1 - n2) * g(f0 + f1 - f2) / den, 0.0)
            r_dec = np.where(ok, pref * V2 * (1.0 + n1 + n2) * g(f0 - f1 - f2) / den, 0.0)
            gabs[iq] += r_abs.sum(axis=(1, 2))
            gdec[iq] += r_dec.sum(axis=(1, 2))
            inv0 = np.where(freq[iq] >= fmin, 1.0 / np.where(freq[iq] > 0, freq[iq], 1.0), 0.0)[:, None]
            rows = slice(iq * n, (iq + 1) * n)
            # absorption: + f''/f lambda(q+q', nu''), - f'/f lambda(q', nu')
            # decay:      + f''/f lambda(q+q', nu''), + f'/f lambda(-q', nu')
            B[rows, i_out * n:(i_out + 1) * n] += (r_abs + r_dec).sum(axis=1) * freq[i_out][None, :] * inv0
            B[rows, iqp * n:(iqp + 1) * n] -= r_abs.sum(axis=2) * freq[iqp][None, :] * inv0
            B[rows, i_neg * n:(i_neg + 1) * n] += r_dec.sum(axis=2) * freq[iqp][None, :] * inv0
    return B, gdec, gabs


@pytest.fixture(scope="module")
def proc(case):
    return _process_operator(case)


def test_linewidth_is_the_sum_of_process_rates(case, proc):
    B, gdec, gabs = proc
    g_ref = O.anharmonic.gamma(case["fc3"], case["mesh"], case["freq"], case["evec"], case["irr"], case["T"],
                               **case["kw"])
    assert g_ref.max() > 0
    assert np.abs(case["g0"] - g_ref).max() <= 1e-12 * g_ref.max()
    tot = (gdec + gabs)[case["irr"]]
    tot = np.where(case["freq"][case["irr"]] >= 0.01, tot, 0.0)
    assert np.abs(tot - g_ref).max() <= 1e-12 * g_ref.max()


def test_incoming_labelling_equals_process_operator_on_odd_fields(case, proc):
    """On fields with lambda(-q) = -lambda(q), the oracle's Gamma1 rows act as -Delta."""
    B, _, _ = proc
    nq, n = case["freq"].shape
    rng = np.random.default_rng(3)
    lam = rng.normal(size=(nq, n, 3))
    _, pos, sign = case["irr"], case["pos"], case["sign"]
    rep = case["irr"][pos]
    lam = lam[rep] * sign[:, None, None]             # odd under time reversal, 0 at q = -q
    delta = (B @ lam.reshape(-1, 3)).reshape(nq, n, 3)[case["irr"]]
    mine = -(case["g1f"] @ lam.reshape(-1, 3)).reshape(len(case["irr"]), n, 3)
    scale = np.abs(delta).max()
    assert scale > 0 and np.abs(case["g1f"]).max() > 0
    assert np.abs(mine - delta).max() <= 1e-12 * scale


def test_reduced_iteration_equals_full_mesh_process_iteration(case, proc):
    B, gdec, gabs = proc
    freq, vel = case["freq"], case["vel"]
    nq, n = freq.shape
    hist, lam, _ = O.bte.iterate(case["mesh"], freq, vel, case["g0"], case["g1"], case["T"], case["vol"],
                                 n_iter=6, tol=0.0)
    gam = gdec + gabs
    live = (freq >= 0.01) & (gam > 0)
    g = np.where(live, gam, 1.0)
    cv = O.occupation.heat_capacity(freq, case["T"])
    x = np.where(live[..., None], vel / g[..., None], 0.0)
    conv = O.constants.EV_PS_A_K_TO_W_MK / (nq * case["vol"])
    ref = [np.einsum("qn,qna,qnb->ab", cv, vel, x) * conv]
    for _ in range(6):
        x = np.where(live[..., None], (vel + (B @ x.reshape(-1, 3)).reshape(nq, n, 3)) / g[..., None], 0.0)
        ref.append(np.einsum("qn,qna,qnb->ab", cv, vel, x) * conv)
    ref = np.array(ref)
    assert hist.shape == ref.shape
    assert np.abs(hist - ref).max() <= 1e-10 * np.abs(ref).max()
    assert abs(np.trace(ref[-1]) / np.trace(ref[0]) - 1.0) > 1e-3     # the coupling does something


def test_start_is_rta(case):
    hist, _, _ = O.bte.iterate(case["mesh"], case["freq"], case["vel"], case["g0"], case["g1"], case["T"],
                               case["vol"], n_iter=0)
    gfull = O.transport.unfold(case["g0"], case["pos"])
    k = O.transport.kappa_rta(case["freq"], case["vel"], gfull, case["T"], case["vol"])
    assert np.abs(hist[0] - k).max() <= 1e-12 * np.abs(k).max()


def test_converged_iterate_solves_the_inverse_problem(case):
    g0, g1 = case["g0"], case["g1"]
    live = g0.ravel() > 0
    A = g1[np.ix_(live, live)] / g0.ravel()[live][:, None]
    rho = np.abs(np.linalg.eigvals(A)).max()
    assert rho < 1.0                                   # the case is one where Eq. (sc_iter) converges
    hist, lam, conv = O.bte.iterate(case["mesh"], case["freq"], case["vel"], g0, g1, case["T"], case["vol"],
                                    n_iter=2000, tol=1e-15)
    k_inv, lam_inv = O.bte.kappa_inverse(case["mesh"], case["freq"], case["vel"], g0, g1, case["T"], case["vol"])
    assert np.abs(hist[-1] - k_inv).max() <= 1e-10 * np.abs(k_inv).max()
    assert np.abs(lam - lam_inv).max() <= 1e-8 * np.abs(lam_inv).max()


def test_phi3_scaling(case):
    """Phi3 -> 2 Phi3: Gamma0 and Gamma1 grow 4x, every kappa iterate shrinks 4x."""
    s = case
    fc3b = O.anharmonic.FC3(s["f3"].idx, 2.0 * s["f3"].val, s["c"].masses)
    g0b, g1fb = O.bte.scattering_rows(fc3b, s["mesh"], s["freq"], s["evec"], s["irr"][:3], s["T"], **s["kw"])
    n = s["freq"].shape[1]
    assert np.abs(g0b - 4 * s["g0"][:3]).max() <= 1e-12 * g0b.max()
    assert np.abs(g1fb - 4 * s["g1f"][:3 * n]).max() <= 1e-12 * np.abs(g1fb).max()
    h1, _, _ = O.bte.iterate(s["mesh"], s["freq"], s["vel"], s["g0"], s["g1"], s["T"], s["vol"], n_iter=3, tol=0)
    h4, _, _ = O.bte.iterate(s["mesh"], s["freq"], s["vel"], 4 * s["g0"], 4 * s["g1"], s["T"], s["vol"], n_iter=3,
                             tol=0)
    assert np.abs(4 * h4 - h1).max() <= 1e-12 * np.abs(h1).max()


def _on_shell_rows(s, pair_weights=None, monkeypatch=None):
    """Folded Gamma1 rows of the representatives, with the case's eigenvectors but whole-number
    frequencies (1, 2 or 3 THz, equal at q and -q) and a window of 0.4 THz: every triplet that
    survives the window is exactly resonant (f = f' + f'' or f + f' = f'')."""
    mesh, n = s["mesh"], s["freq"].shape[1]
    rng = np.random.default_rng(5)
    freq = rng.integers(1, 4, size=(len(s["irr"]), n)).astype(np.float64)[s["pos"]]
    if pair_weights is not None:
        monkeypatch.setattr(O.anharmonic, "pair_weights", pair_weights)
    _, g1f = O.bte.scattering_rows(s["fc3"], mesh, freq, s["evec"], s["irr"], s["T"], shape=s["kw"]["shape"],
                                   sigma=0.2, window=2.0)
    return freq, O.bte.reduce_columns(g1f, mesh, n)


def _detailed_balance_asym(s, freq, g1):
    """max |D - D^T| / max |D| for D = diag(n(n+1) f) Gamma1 diag(1/f) over the representatives
    with -q != q (the others carry lambda = 0)."""
    n = freq.shape[1]
    f = freq[s["irr"]].ravel()
    nb = O.occupation.bose(freq[s["irr"]], s["T"]).ravel()
    live = np.repeat(s["sign"][s["irr"]] != 0, n)
    d = (nb * (nb + 1) * f)[:, None] * g1 / f[None, :]
    d = np.where(live[:, None] & live[None, :], d, 0.0)
    assert np.abs(d).max() > 0
    return float(np.abs(d - d.T).max() / np.abs(d).max())


def test_gamma1_detailed_balance_on_shell(case):
    """Detailed balance, a property of the linearised collision operator that the oracle's
    assembly does not use: a process couples its partners through one equilibrium rate P,
    which is n(n+1) times that process's linewidth term of every participant, so
    diag(n(n+1) f) (Gamma0 + Gamma1) diag(1/f) is symmetric on time-reversal-odd fields
    (the Boltzmann-equation symmetry behind the paper's variational and direct solvers).
    The rate identity n (1 + n' + n'') = n' n'' behind it holds on shell only, so the pin uses
    frequencies for which every triplet inside the window is exactly resonant.  With the
    broadened, off-shell occupations of real spectra the symmetry holds only to O(sigma)."""
    freq, g1 = _on_shell_rows(case)
    assert _detailed_balance_asym(case, freq, g1) < 1e-12


@pytest.mark.parametrize("mistake", ["absorption-sign", "decay-occupation"])
def test_gamma1_detailed_balance_catches_planted_mistakes(case, mistake, monkeypatch):
    """The on-shell pin rejects an oracle whose weights carry a plausible mistake."""
    good = O.anharmonic.pair_weights

    def planted(f0, f1, f2, n1, n2, shape, sigma, f_min, window):
        if mistake == "absorption-sign":            # (n'' - n') in place of (n' - n'')
            return _swap_abs(good, f0, f1, f2, n1, n2, shape, sigma, f_min, window)
        # (n' + n'') in place of (1 + n' + n'') in the decay term; absorption unchanged
        return good(f0, f1, f2, n1 - 0.5, n2 - 0.5, shape, sigma, f_min, window)

    freq, g1 = _on_shell_rows(case, planted, monkeypatch)
    assert _detailed_balance_asym(case, freq, g1) > 1e-3


def _swap_abs(good, f0, f1, f2, n1, n2, shape, sigma, f_min, window):
    """Weights with the absorption term's occupation difference negated."""
    dec = good(f0, f1, f2, n1, n2, shape, sigma, f_min, window)
    F0, F1, F2 = f0[:, None, None], f1[None, :, None], f2[None, None, :]
    N1, N2 = n1[None, :, None], n2[None, None, :]
    ok = (F0 >= f_min) & (F1 >= f_min) & (F2 >= f_min)
    www = np.where(ok, (2 * np.pi) ** 4 * F0 * F1 * F2, 1.0)
    absorb = 2.0 * (N1 - N2) * O.anharmonic.broadening(F0 + F1 - F2, shape, sigma, window)
    return dec - np.where(ok, 2.0 * absorb / www, 0.0)
