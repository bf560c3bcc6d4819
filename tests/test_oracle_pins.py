"""Pins of the FP64 oracle against what the paper and the mathematics fix, independently of
the oracle's own formulas: closed forms, invariants, special cases and brute force.

Each test names the kind of mistake it would catch.
"""
import math

import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------------------- fixtures

@pytest.fixture(scope="module")
def fcc1():
    w = P.fcc_monatomic_5()
    f2, f3 = w.ifc2(), w.ifc3()
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, vel = O.harmonic.solve(f2.idx, f2.val, w.crystal.masses, w.crystal.lattice, q)
    return dict(w=w, f2=f2, f3=f3, q=q, freq=freq, evec=evec, vel=vel,
                fc3=O.anharmonic.FC3(f3.idx, f3.val, w.crystal.masses))


def _chain(a=4.0, rc=6.0):
    c = P.linear_chain(a=a)
    pot = P.LennardJones(rc=rc)
    return c, pot, P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)


# ----------------------------------------------------------------------------- P1 closed forms

def test_p1_fcc_dynmat_closed_form(fcc1):
    """Monatomic Bravais lattice: D(q) = (1/m) sum_j H(r_j) (1 - cos q.r_j), H computed here
    from the LJ derivatives directly (catches a wrong phase sign, self term or mass factor)."""
    w = fcc1["w"]
    c = w.crystal
    pot = w.pot
    _, _, R, rv = P.neighbours(c, pot.rc)
    rho = np.linalg.norm(rv, axis=1)
    _, f1, f2, _ = pot.derivs(rho)
    nh = rv / rho[:, None]
    H = (f2 - f1 / rho)[:, None, None] * nh[:, :, None] * nh[:, None, :] + (f1 / rho)[:, None, None] * np.eye(3)
    B = 2 * np.pi * np.linalg.inv(c.lattice).T
    rng = np.random.default_rng(0)
    for q_red in rng.uniform(-0.5, 0.5, size=(5, 3)):
        qc = q_red @ B
        Dref = (H * (1.0 - np.cos(rv @ qc))[:, None, None]).sum(axis=0) / c.masses[0]
        D = O.harmonic.dynamical_matrix(fcc1["f2"].idx, fcc1["f2"].val, c.masses, q_red)
        assert np.abs(D - Dref).max() < 1e-12 * np.abs(Dref).max()


def test_p1_chain_dispersion_closed_form():
    """Nearest-neighbour chain: w_L = 2 sqrt(f''(a)/m)|sin(qa/2)|, w_T = 2 sqrt(f'(a)/(a m))|sin(qa/2)|."""
    a = 4.0
    c, pot, f2, _ = _chain(a)
    _, f1a, f2a, _ = pot.derivs(a)
    m = c.masses[0]
    qs = np.array([[k / 12.0, 0, 0] for k in range(12)])
    freq, _, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, qs)
    conv = 9648.533212      # eV/(A^2 amu) in ps^-2, CODATA
    for k, q in enumerate(qs):
        s = abs(math.sin(math.pi * q[0]))
        wl = 2 * math.sqrt(f2a / m * conv) * s / (2 * math.pi)
        wt = 2 * math.sqrt(f1a / (a * m) * conv) * s / (2 * math.pi)
        ref = np.sort([wt, wt, wl])
        assert np.allclose(np.sort(freq[k]), ref, rtol=1e-12, atol=1e-7)


# ----------------------------------------------------------------------------- P2 invariants

def test_p2_asr_hermitian_unitary(fcc1):
    w = fcc1["w"]
    f0 = fcc1["freq"][0]
    assert np.abs(f0).max() < 1e-6                     # acoustic sum rule at Gamma
    c32 = P.fcc_massdisorder_32()
    f2 = c32.ifc2()
    D0 = O.harmonic.dynamical_matrix(f2.idx, f2.val, c32.crystal.masses, np.zeros(3))
    lam = np.linalg.eigvalsh(0.5 * (D0 + D0.conj().T))
    assert np.abs(lam[:3]).max() < 1e-10 * np.abs(lam).max()
    for q in [np.array([0.1, 0.27, -0.33]), np.array([0.5, 0.5, 0.0])]:
        D = O.harmonic.dynamical_matrix(f2.idx, f2.val, c32.crystal.masses, q)
        assert np.abs(D - D.conj().T).max() < 1e-12 * np.abs(D).max()
    e = fcc1["evec"]
    eye = np.eye(3)
    for k in range(e.shape[0]):
        assert np.abs(e[k].conj().T @ e[k] - eye).max() < 1e-12


def test_p2_velocity_matches_finite_difference(fcc1):
    """v = d w / d q by central differences in Cartesian q (generic, non-degenerate q)."""
    w = fcc1["w"]
    c = w.crystal
    f2 = fcc1["f2"]
    A = c.lattice
    q_red = np.array([0.13, 0.29, 0.07])
    freq, e, v = O.harmonic.solve(f2.idx, f2.val, c.masses, A, q_red[None])
    h = 1e-5   # 1/A
    for al in range(3):
        dq = np.zeros(3)
        dq[al] = h
        dq_red = A @ dq / (2 * np.pi)      # q_red = A q_cart / (2 pi)
        fp, _, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, A, (q_red + dq_red)[None])
        fm, _, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, A, (q_red - dq_red)[None])
        dw = (fp[0] - fm[0]) * 2 * np.pi / (2 * h)        # rad/ps per (1/A) = A/ps
        assert np.allclose(v[0][:, al], dw, rtol=1e-6, atol=1e-6)


# ----------------------------------------------------------------------------- P3 fixture vs forces

def test_p3_ifcs_match_force_differences():
    """Folded supercell IFCs from the analytic tensors equal central differences of LJ forces
    (h = 1e-4 A); Phi3 fully symmetric and sums to zero over the last index."""
    # (a 2x2x2 fcc supercell has every folded Phi3 = 0 by inversion through each atom; 3x2x2 not)
    sc = P.fcc_primitive_multiple(5.26, (3, 2, 2))
    pot = P.LennardJones()
    f2 = P.ifc2_lj(sc, pot)
    f3 = P.ifc3_lj(sc, pot)
    n = 3 * sc.n_atoms
    ones = np.ones(sc.n_atoms)
    K2 = O.supercell.gamma_point_dynmat(f2.idx, f2.val, ones)
    K3 = O.supercell.folded_phi3(f3.idx, f3.val, ones)
    h = 1e-4
    x0 = sc.positions.copy()
    for ia in [0, 4]:
        for al in range(3):
            xp = x0.copy(); xp[ia, al] += h
            xm = x0.copy(); xm[ia, al] -= h
            Fp = P.lj_forces(xp, sc.lattice, pot).ravel()
            Fm = P.lj_forces(xm, sc.lattice, pot).ravel()
            Fd = -(Fp - Fm) / (2 * h)
            assert np.allclose(K2[3 * ia + al], Fd, rtol=1e-6, atol=1e-6 * np.abs(K2).max())
    # Phi3(i a, j b, :) = -d^2 F / dx_ia dx_jb
    for (ia, al, jb, be) in [(0, 0, 0, 0), (0, 1, 3, 2), (2, 2, 5, 0)]:
        def F(di, dj):
            x = x0.copy(); x[ia, al] += di; x[jb, be] += dj
            return P.lj_forces(x, sc.lattice, pot).ravel()
        hh = 1e-3
        d2 = -(F(hh, hh) - F(hh, -hh) - F(-hh, hh) + F(-hh, -hh)) / (4 * hh * hh)
        ref = K3[3 * ia + al, 3 * jb + be]
        assert np.allclose(ref, d2, rtol=1e-5, atol=2e-5 * np.abs(K3).max())
    for perm in [(1, 0, 2), (0, 2, 1), (2, 1, 0)]:
        assert np.abs(K3 - K3.transpose(perm)).max() < 1e-12 * np.abs(K3).max()
    assert np.abs(K3.sum(axis=2)).max() < 1e-12 * np.abs(K3).max()
    assert np.abs(K2.sum(axis=1)).max() < 1e-12 * np.abs(K2).max()


# ----------------------------------------------------------------------------- P4 V3 symmetry

def test_p4_v3_permutation_and_time_reversal():
    w = P.fcc_massdisorder_32(mesh=(2, 2, 2))
    c = P.random_masses(P.fcc_conventional(), 39.95, 83.8, seed=7)
    f2 = P.ifc2_lj(c, w.pot)
    f3 = P.ifc3_lj(c, w.pot)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    q = np.array([0.25, -0.125, 0.375])
    q1 = np.array([-0.5, 0.25, 0.125])
    q2 = -(q + q1)
    fr, e, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, np.array([q, q1, q2]))
    V = O.anharmonic.v3(fc3, e[0], q1, e[1], q2, e[2])
    V_swap = O.anharmonic.v3(fc3, e[1], q, e[0], q2, e[2])        # Phi(q' nu', q nu, q'' nu'')
    assert np.abs(V_swap.transpose(1, 0, 2) - V).max() < 1e-10 * np.abs(V).max()
    V_cyc = O.anharmonic.v3(fc3, e[2], q, e[0], q1, e[1])         # Phi(q'' nu'', q nu, q' nu')
    assert np.abs(V_cyc.transpose(1, 2, 0) - V).max() < 1e-10 * np.abs(V).max()
    # time reversal: e_{-k} = conj(e_k) gives Phi(-q,-q',-q'') = conj(Phi)
    Vtr = O.anharmonic.v3(fc3, e[0].conj(), -q1, e[1].conj(), -q2, e[2].conj())
    assert np.abs(Vtr - V.conj()).max() < 1e-10 * np.abs(V).max()
    # |Phi|^2 unchanged by per-mode phases
    rng = np.random.default_rng(1)
    ph = [np.exp(1j * rng.uniform(0, 2 * np.pi, e.shape[2])) for _ in range(3)]
    Vp = O.anharmonic.v3(fc3, e[0] * ph[0], q1, e[1] * ph[1], q2, e[2] * ph[2])
    assert np.abs(np.abs(Vp) - np.abs(V)).max() < 1e-10 * np.abs(V).max()


# ----------------------------------------------------------------------------- P5 chain element

def test_p5_chain_longitudinal_element_closed_form():
    """|Phi_LLL|^2 = f'''(a)^2 prod_j |2 sin(q_j a / 2)|^2 / m^3 for a NN chain."""
    a = 4.0
    c, pot, f2, f3 = _chain(a)
    _, _, _, f3a = pot.derivs(a)
    m = c.masses[0]
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    ex = np.zeros((3, 3), dtype=complex)
    ex[0, 0] = 1.0                                          # mode 0 = x polarised
    for (k0, k1) in [(1, 2), (3, 5), (7, 11), (0, 4)]:
        q = np.array([k0 / 12.0, 0, 0]); q1 = np.array([k1 / 12.0, 0, 0]); q2 = -(q + q1)
        V = O.anharmonic.v3(fc3, ex, q1, ex, q2, ex)[0, 0, 0]
        ref = f3a ** 2 * np.prod([(2 * math.sin(math.pi * x[0])) ** 2 for x in (q, q1, q2)]) / m ** 3
        assert abs(abs(V) ** 2 - ref) <= 1e-12 * max(ref, 1e-30) + 1e-18


# ----------------------------------------------------------------------------- P6 folding

@pytest.mark.parametrize("cell,mesh", [("fcc1", (3, 3, 3)), ("fcc1", (3, 2, 1)), ("fcc2", (1, 2, 3))])
def test_p6_supercell_folding(cell, mesh):
    """Mesh linewidths (degenerate-averaged over equal-frequency sets of the full mesh) equal
    the Gamma-only linewidths of the mesh-sized supercell built from its own IFC list."""
    pot = P.LennardJones()
    if cell == "fcc1":
        c = P.fcc_primitive()
    else:
        c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
        c = P.Crystal(c.lattice, c.positions, np.array([39.95, 83.8]), "fcc2")
    T, sig = 60.0, 0.3
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    q = O.grid.mesh_qred(mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    g = O.anharmonic.gamma(fc3, mesh, freq, evec, np.arange(q.shape[0]), T, "gauss", sig)
    sc = P.supercell(c, mesh)
    s2, s3 = P.ifc2_lj(sc, pot), P.ifc3_lj(sc, pot)
    fs, gs = O.supercell.gamma_only(s2.idx, s2.val, s3.idx, s3.val, sc.masses, T, "gauss", sig)
    fm = freq.ravel()
    gm = g.ravel()
    assert np.allclose(np.sort(fm), np.sort(fs), atol=1e-6)   # acoustic zeros are ~1e-8 noise
    tol = 1e-5 * np.abs(fs).max()
    used = 0
    for f in np.unique(np.round(fs, 6)):
        if f < 0.01:
            continue
        mm = np.abs(fm - f) < tol
        ms = np.abs(fs - f) < tol
        assert mm.sum() == ms.sum()
        assert abs(gm[mm].mean() - gs[ms].mean()) <= 1e-10 * max(gs.max(), 1e-30)
        used += 1
    assert used > 3 and gs.max() > 0


# ----------------------------------------------------------------------------- P7 invariants of gamma

def test_p7_gamma_invariants(fcc1):
    w = fcc1["w"]
    irr, f2i, _ = O.grid.irreducible(w.mesh, w.rotations)
    g = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], irr,
                           w.temperature, w.shape, w.sigma_thz)
    f_irr = fcc1["freq"][irr]
    assert np.all(g[f_irr > 2 * w.sigma_thz] >= 0)
    assert g.max() > 0
    # gamma scales as s^2 under Phi3 -> s Phi3
    fc3s = O.anharmonic.FC3(fcc1["f3"].idx, 3.0 * fcc1["f3"].val, w.crystal.masses)
    gs = O.anharmonic.gamma(fc3s, w.mesh, fcc1["freq"], fcc1["evec"], irr[:4], w.temperature,
                            w.shape, w.sigma_thz)
    assert np.allclose(gs, 9.0 * g[:4], rtol=1e-12)
    fc30 = O.anharmonic.FC3(fcc1["f3"].idx, 0.0 * fcc1["f3"].val, w.crystal.masses)
    g0 = O.anharmonic.gamma(fc30, w.mesh, fcc1["freq"], fcc1["evec"], irr[:2], w.temperature)
    assert np.all(g0 == 0)
    # star members: every q of the mesh gives the linewidth of its irreducible representative
    allq = np.arange(125)
    ga = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], allq, w.temperature,
                            w.shape, w.sigma_thz)
    for i in allq:
        a = O.anharmonic.degenerate_average(fcc1["freq"][i], ga[i])
        r = irr[f2i[i]]
        b = O.anharmonic.degenerate_average(fcc1["freq"][r], ga[r])
        assert np.allclose(a, b, rtol=1e-10, atol=1e-14)


# ----------------------------------------------------------------------------- P8 broadening

def test_p8_broadening_normalisation():
    sig = 0.1
    x = np.linspace(-60 * sig, 60 * sig, 2_400_001)
    dx = x[1] - x[0]
    for shape, outside in [("gauss", math.erfc(2.0)),
                           ("lorentz", 1.0 - 2.0 / math.pi * math.atan(4.0))]:
        g_inf = O.anharmonic.broadening(x, shape, sig, window=1e9)
        total = np.trapezoid(g_inf, dx=dx)
        if shape == "lorentz":   # add the analytic tails beyond the grid
            total += 1.0 - 2.0 / math.pi * math.atan(60 * sig / (0.5 * sig))
        assert abs(total - 1.0) < 1e-9
        g2 = O.anharmonic.broadening(x, shape, sig, window=2.0)
        inside = g2.sum() * dx
        assert abs(inside - (1.0 - outside)) < 1e-6


# ----------------------------------------------------------------------------- occupations

def test_occupations_closed_forms():
    f = np.array([0.3, 1.0, 2.5])
    T = 37.0
    # c = hbar w dn/dT (Eq. (heatcap), second form) by central differences in T
    h = 1e-4
    dn = (O.occupation.bose(f, T + h) - O.occupation.bose(f, T - h)) / (2 * h)
    c = O.occupation.heat_capacity(f, T)
    hw = O.constants.HBAR_EV_PS * 2 * np.pi * f
    assert np.allclose(c, hw * dn, rtol=1e-7)
    # high temperature: c -> k_B and n -> k_B T / (hbar w)
    ch = O.occupation.heat_capacity(f, 1e6)
    assert np.allclose(ch, O.constants.KB_EV_K, rtol=1e-8)
    nh = O.occupation.bose(f, 1e6)
    assert np.allclose(nh, O.constants.KB_EV_K * 1e6 / hw - 0.5, rtol=1e-6)
    assert np.allclose(O.occupation.heat_capacity(f, T, is_classic=True), O.constants.KB_EV_K)


# ----------------------------------------------------------------------------- P9 kappa

def test_p9_kappa_isotropy_and_constant_tau(fcc1):
    w = fcc1["w"]
    c = w.crystal
    f2 = fcc1["f2"]
    irr, f2i, _ = O.grid.irreducible(w.mesh, w.rotations)
    g = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], irr, w.temperature,
                           w.shape, w.sigma_thz)
    g = np.array([O.anharmonic.degenerate_average(fcc1["freq"][i], g[s]) for s, i in enumerate(irr)])
    gf = O.transport.unfold(g, f2i)
    vv = np.array([O.harmonic.velocity_products(f2.idx, f2.val, c.masses, c.lattice, fcc1["q"][k],
                                                fcc1["freq"][k], fcc1["evec"][k])
                   for k in range(125)])
    K = O.transport.kappa_rta_vv(fcc1["freq"], vv, gf, w.temperature, c.volume)
    d = np.diag(K)
    assert np.allclose(d, d.mean(), rtol=1e-10)
    assert np.abs(K - np.diag(d)).max() < 1e-10 * d.mean()
    assert d.mean() > 0
    # constant tau: kappa = tau/(N V) sum c v v
    tau = 7.5
    Kc = O.transport.kappa_rta_vv(fcc1["freq"], vv, np.full_like(gf, 1.0 / tau), w.temperature, c.volume)
    cc = O.occupation.heat_capacity(fcc1["freq"], w.temperature)
    ok = fcc1["freq"] >= 0.01
    ref = tau * np.einsum("qn,qnab->ab", np.where(ok, cc, 0), vv) / (125 * c.volume) * 1602.176634
    assert np.allclose(Kc, ref, rtol=1e-9)
    # for non-degenerate modes the invariant product is v v
    k = 7
    sets = O.harmonic.degenerate_sets(fcc1["freq"][k])
    for S in sets:
        if len(S) == 1 and fcc1["freq"][k][S[0]] > 0.01:
            v = fcc1["vel"][k][S[0]]
            assert np.allclose(vv[k][S[0]], np.outer(v, v), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------- P10 T split

def test_p10_temperature_split_exact(fcc1):
    w = fcc1["w"]
    irr = np.array([3, 17])
    g1, v2 = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], irr, 30.0,
                                keep_v2=True)
    g2 = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], irr, 75.0)
    g2s = O.anharmonic.gamma_from_v2(v2, w.mesh, fcc1["freq"], irr, 75.0)
    assert np.allclose(g2s, g2, rtol=1e-14, atol=0)
    assert not np.allclose(g1, g2)


# ----------------------------------------------------------------------------- grid

def _burnside(mesh, rots):
    """Orbit count of the group {R} U {-R} acting on the mesh, by Burnside's lemma."""
    k = O.grid.mesh_int(mesh)
    ops = [r for r in rots] + [-r for r in rots]
    # close the set under composition
    seen = {tuple(np.asarray(o).ravel()) for o in ops}
    ops = [np.array(t).reshape(3, 3) for t in seen]
    fixed = 0
    for r in ops:
        img = O.grid.mesh_index(k @ r.T, mesh)
        fixed += int((img == np.arange(k.shape[0])).sum())
    return fixed // len(ops)


@pytest.mark.parametrize("mesh,which", [((5, 5, 5), "oh1"), ((8, 8, 8), "tr"), ((4, 4, 4), "tr"),
                                        ((8, 8, 8), "oh4"), ((12, 12, 12), "tr")])
def test_grid_irreducible_counts(mesh, which):
    if which == "oh1":
        rots = P.cubic_rotations_reduced(P.fcc_primitive().lattice)
    elif which == "oh4":
        rots = P.cubic_rotations_reduced(P.fcc_conventional().lattice)
    else:
        rots = P.identity_rotation()
    irr, f2i, wts = O.grid.irreducible(mesh, rots)
    assert len(irr) == _burnside(mesh, rots)
    assert wts.sum() == np.prod(mesh)
    assert np.all(irr[f2i] <= np.arange(np.prod(mesh)))


def test_grid_third_index_momentum():
    mesh = (4, 3, 5)
    k = O.grid.mesh_int(mesh)
    for iq in [0, 7, 33]:
        for iqp in range(k.shape[0]):
            iqpp = O.grid.third_index(iq, iqp, mesh)
            s = k[iq] + k[iqp] + k[iqpp]
            assert np.all(np.mod(s, mesh) == 0)


# ----------------------------------------------------------------------------- constants, weights

def test_unit_conversions_literal():
    """The conversions against their CODATA-derived literal values."""
    assert abs(O.constants.EV_A2_AMU_TO_PS2 - 9648.533212) < 1e-5
    assert abs(O.constants.EV_PS_A_K_TO_W_MK - 1602.176634) < 1e-9
    assert O.constants.HBAR_EV_PS == 6.582119569e-4 and O.constants.KB_EV_K == 8.617333262e-5


def test_gamma_matches_self_energy_form(fcc1):
    """The ordered-pair counting with 2 (n' - n'') delta(w + w' - w'') equals the textbook
    imaginary self-energy form (n' - n'') [delta(w + w' - w'') - delta(w - w' + w'')], which
    needs no symmetrisation (catches a dropped factor 2 or a swapped delta argument)."""
    w = fcc1["w"]
    freq, evec, fc3 = fcc1["freq"], fcc1["evec"], fcc1["fc3"]
    k = O.grid.mesh_int(w.mesh)
    qred = O.grid.mesh_qred(w.mesh)
    nocc = O.occupation.bose(freq, w.temperature)
    sig = w.sigma_thz
    g = lambda x: np.where(np.abs(x) < 2 * sig, np.exp(-(x / sig) ** 2) / (np.sqrt(np.pi) * sig), 0.0)
    for iq in [6, 31]:
        acc = np.zeros(3)
        for iqp in range(125):
            iqpp = int(O.grid.mesh_index(-(k[iq] + k[iqp]), w.mesh))
            V = O.anharmonic.v3(fc3, evec[iq], qred[iqp], evec[iqp], -(qred[iq] + qred[iqp]), evec[iqpp])
            f0 = freq[iq][:, None, None]; f1 = freq[iqp][None, :, None]; f2 = freq[iqpp][None, None, :]
            n1 = nocc[iqp][None, :, None]; n2 = nocc[iqpp][None, None, :]
            br = (1 + n1 + n2) * g(f0 - f1 - f2) + (n1 - n2) * (g(f0 + f1 - f2) - g(f0 - f1 + f2))
            ok = (f1 >= 0.01) & (f2 >= 0.01)
            wt = np.where(ok, br / ((2 * np.pi) ** 3 * f0 * f1 * f2), 0.0) / (2 * np.pi)
            acc += (np.abs(V) ** 2 * wt).sum(axis=(1, 2))
        ref = np.pi * 6.582119569e-4 * 9648.533212 ** 3 / (8 * 125) * acc
        got = O.anharmonic.gamma(fc3, w.mesh, freq, evec, [iq], w.temperature, "gauss", sig)[0]
        assert np.allclose(got, ref, rtol=1e-6)


# ----------------------------------------------------------------------------- surrogate reference

def test_surrogate_reference_gradient_matches_finite_differences():
    """The FP64 reference network's backpropagated gradient against central differences."""
    rng = np.random.default_rng(4)
    n_in, width, depth = 4, 8, 3
    shapes = O.surrogate.layer_shapes(n_in, width, depth)
    n_par = sum(i * o + o for i, o in shapes)
    p = rng.normal(scale=0.4, size=n_par)
    norm = np.concatenate([rng.normal(size=n_in), rng.uniform(0.5, 2, n_in), [0.3, 1.7]])
    X = np.exp(rng.normal(size=(13, n_in)))
    y = np.exp(rng.normal(size=13))
    loss, g = O.surrogate.loss_and_grad(p, norm, X, y, n_in, width, depth)
    h = 1e-6
    for k in rng.choice(n_par, 25, replace=False):
        e = np.zeros(n_par); e[k] = h
        lp, _ = O.surrogate.loss_and_grad(p + e, norm, X, y, n_in, width, depth)
        lm, _ = O.surrogate.loss_and_grad(p - e, norm, X, y, n_in, width, depth)
        assert abs((lp - lm) / (2 * h) - g[k]) <= 1e-7 * max(1.0, abs(g[k]))
    # prediction is the de-standardised network output
    pr = O.surrogate.predict(p, norm, X, n_in, width, depth)
    assert pr.shape == (13,) and np.all(np.isfinite(pr))
