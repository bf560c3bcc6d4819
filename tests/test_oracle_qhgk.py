"""Pins of the QHGK oracle (Eqs. (qhgk), (qhgk_crystal)): the generalized heat capacity's
diagonal limit (closed form), the degenerate-pair limit equal to the RTA conductivity with
invariant velocity products, and supercell folding: Gamma-only QHGK of an n^3 supercell
(bond-vector velocity operator) equals the mesh QHGK with interband pairs."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_heat_capacity_matrix_limit_and_symmetry():
    T = 40.0
    f = np.array([0.7, 0.7 * (1 + 1e-4), 1.3, 2.0])
    c = O.qhgk.heat_capacity_matrix(f, T)
    cm = O.occupation.heat_capacity(f, T)
    assert np.allclose(c, c.T, rtol=1e-13)
    assert abs(c[0, 1] - cm[0]) < 2e-4 * cm[0]                  # formula tends to c_mu
    assert np.allclose(np.diag(c), cm, rtol=1e-14)
    # hbar w w' (n - n') / (T (w' - w)) written out for one pair
    w = 2 * np.pi * f
    n = O.occupation.bose(f, T)
    ref = O.constants.HBAR_EV_PS * w[0] * w[2] * (n[0] - n[2]) / (T * (w[2] - w[0]))
    assert abs(c[0, 2] - ref) < 1e-14 * abs(ref)


def _fcc1_mesh(mesh):
    c = P.fcc_primitive()
    f2 = P.ifc2_lj(c, P.LennardJones())
    q = O.grid.mesh_qred(mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    return c, f2, q, freq, evec


def test_degenerate_pairs_reduce_to_rta_with_invariant_velocities():
    c, f2, q, freq, evec = _fcc1_mesh((4, 4, 4))
    T = 40.0
    gam = 0.05 + 0.3 * freq ** 2
    k = O.qhgk.kappa_mesh(f2.idx, f2.val, c.masses, c.lattice, q, freq, evec, gam, T, pairs="degenerate")
    vv = np.array([O.harmonic.velocity_products(f2.idx, f2.val, c.masses, c.lattice, q[i], freq[i], evec[i])
                   for i in range(q.shape[0])])
    ref = O.transport.kappa_rta_vv(freq, vv, gam, T, c.volume)
    assert np.abs(k - ref).max() <= 1e-11 * np.abs(ref).max()


def test_supercell_gamma_qhgk_equals_mesh_qhgk():
    mesh = (3, 3, 3)
    c, f2, q, freq, evec = _fcc1_mesh(mesh)
    T = 60.0
    gfun = lambda f: 0.08 + 0.25 * f ** 2                       # a function of frequency alone
    k_mesh = O.qhgk.kappa_mesh(f2.idx, f2.val, c.masses, c.lattice, q, freq, evec, gfun(freq), T)
    sc = P.supercell(c, mesh)
    s2 = P.ifc2_lj(sc, P.LennardJones())
    D = O.gammapoint.dynmat(s2.idx, s2.val.reshape(-1, 9), sc.masses)
    lam, E = np.linalg.eigh(D)
    fs = O.harmonic.frequencies_from_eigenvalues(lam)
    k_sc = O.qhgk.kappa_gamma_cell(s2.idx, s2.val, sc.masses, sc.positions, sc.lattice, fs, E, gfun(fs), T)
    assert np.abs(k_mesh).max() > 0
    assert np.abs(k_sc - k_mesh).max() <= 1e-9 * np.abs(k_mesh).max()
    assert abs(k_sc[0, 0] - k_sc[1, 1]) <= 1e-9 * k_sc[0, 0] and abs(k_sc[0, 1]) <= 1e-9 * k_sc[0, 0]
